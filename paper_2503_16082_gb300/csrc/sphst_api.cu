// sphst_api.cu -- the C ABI declared in include/sphst.h: argument checks,
// case and batch records, cell-grid set-up and engine placement.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sphst_engine.cuh"

struct sphst_case_s {
    sphst::CaseRec r;
};

struct sphst_batch_s {
    int32_t precision = 32;
    cudaStream_t stream = nullptr;
    std::vector<sphst::CaseRec *> members;
    sphst::Engine *engine = nullptr;
    bool dirty = true;
};

namespace sphst {

static thread_local std::string g_error;

void set_error(const std::string &msg) { g_error = msg; }

int cuda_fail(cudaError_t e, const char *what) {
    g_error = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SPHST_ERR_OOM : SPHST_ERR_CUDA;
}

int map_status(int32_t s) {
    switch (s) {
    case DEV_OK: return SPHST_OK;
    case DEV_ERR_NONFINITE: return SPHST_ERR_NONFINITE;
    case DEV_ERR_DOMAIN: return SPHST_ERR_DOMAIN;
    case DEV_ERR_COINCIDENT: return SPHST_ERR_COINCIDENT;
    case DEV_ERR_STALLED: return SPHST_ERR_STALLED;
    case DEV_ERR_NBR_OVERFLOW: return SPHST_ERR_NEIGHBORS;
    }
    return SPHST_ERR_CUDA;
}

static const char *status_text(int s) {
    switch (s) {
    case SPHST_ERR_NONFINITE: return "non-finite velocity or time step";
    case SPHST_ERR_DOMAIN: return "a particle left the cell grid";
    case SPHST_ERR_COINCIDENT: return "two particles at the same position";
    case SPHST_ERR_STALLED: return "advection step exceeded max_substeps";
    case SPHST_ERR_NEIGHBORS: return "a particle has more neighbours than max_neighbors";
    }
    return "error";
}

static double cell_width(const CaseRec *c) {
    const double h = c->P.h_factor * c->P.dx;
    const double cs0 = 2.0 * h * (1.0 + 1.0 / 65536.0);
    double cs = cs0;
    for (int a = 0; a < c->P.dim; ++a)       // a periodic axis fixes the width: L / floor(L / cs0)
        if ((c->P.periodic >> a) & 1) {
            const double L = c->P.period_hi[a] - c->P.period_lo[a];
            cs = L / std::floor(L / cs0);
        }
    return cs;
}

// Grid over the initial bounding box with grid_pad spare cells per side; the
// arithmetic order matches the key definition used by the checks.
int make_grid(CaseRec *c) {
    const int dim = c->P.dim;
    const double cs = cell_width(c);
    const int pad = c->P.grid_pad;
    int maxn = 1;
    for (int a = 0; a < 3; ++a) { c->origin[a] = 0.0; c->ncell[a] = 1; }
    for (int a = 0; a < dim; ++a) {
        if ((c->P.periodic >> a) & 1) {      // the period itself, no spare cells
            const double L = c->P.period_hi[a] - c->P.period_lo[a];
            c->origin[a] = c->P.period_lo[a];
            c->ncell[a] = (int32_t)std::floor(L / (2.0 * c->P.h_factor * c->P.dx * (1.0 + 1.0 / 65536.0)));
            maxn = std::max(maxn, c->ncell[a]);
            continue;
        }
        double lo = c->n ? c->pos[a] : 0.0, hi = lo;
        for (int64_t i = 1; i < c->n; ++i) {
            const double x = c->pos[3 * i + a];
            if (x < lo) lo = x;
            if (x > hi) hi = x;
        }
        c->origin[a] = lo - (double)pad * cs;
        const double span = std::floor((hi - c->origin[a]) / cs);
        if (!(span < 60000.0)) {
            set_error("cell grid too large");
            return SPHST_ERR_UNSUPPORTED;
        }
        c->ncell[a] = (int32_t)span + 1 + pad;
        maxn = std::max(maxn, c->ncell[a]);
    }
    int bits = 0;
    while ((1 << bits) < maxn) ++bits;
    if ((dim == 3 && bits > 10) || (dim == 2 && bits > 15)) {
        set_error("cell grid too large: more than 1024 (3D) or 32768 (2D) cells per axis");
        return SPHST_ERR_UNSUPPORTED;
    }
    c->bits = bits;
    c->cs = cs;
    c->table_size = (int64_t)1 << (dim * bits);
    c->gridded = true;
    return SPHST_OK;
}

template <typename T> static CasePhys<T> phys_of(const CaseRec *c) {
    const sphst_case_params &P = c->P;
    const int dim = P.dim;
    const double h = P.h_factor * P.dx;
    const double pi = 3.14159265358979323846;
    const double alpha = dim == 2 ? 7.0 / (4.0 * pi * h * h) : 21.0 / (16.0 * pi * h * h * h);
    const double vol = dim == 2 ? P.dx * P.dx : P.dx * P.dx * P.dx;
    double xi = P.xi;
    if (xi < 0.0) {
        if (c->n_fluid_phases == 2) {
            const double hi = std::max(c->rho0[0], c->rho0[1]), lo = std::min(c->rho0[0], c->rho0[1]);
            xi = 1.3 * std::log10(hi / lo) + 0.6;
        } else {
            xi = 0.6;
        }
    }
    const double rsum = c->rho0[0] + c->rho0[1];
    CasePhys<T> p;
    p.h = (T)h;
    p.inv_h = (T)(1.0 / h);
    p.four_h2 = (T)((2.0 * h) * (2.0 * h));
    p.kcoef = (T)(-5.0 * alpha / h);
    p.cs = (T)cell_width(c);
    p.c0 = (T)P.c0;
    p.c0sq = (T)(P.c0 * P.c0);
    p.inv_c0 = (T)(1.0 / P.c0);
    p.gamma = (T)P.gamma;
    // limiter (Eq. 11): density reading min(max(3 dU / c0, 0), 1); beta = 1; beta = 0
    p.beta_k = (T)((P.limiter == SPHST_LIMITER_DENSITY || P.limiter == SPHST_LIMITER_PRINTED) ? 3.0 / P.c0 : 0.0);
    p.beta_lo = (T)(P.limiter == SPHST_LIMITER_NONE ? 1.0 : 0.0);
    p.beta_hi = (T)(P.limiter == SPHST_LIMITER_ZERO ? 0.0 : 1.0);
    p.xi = (T)xi;
    for (int k = 0; k < 2; ++k) {
        p.rho0[k] = (T)c->rho0[k];
        p.eta[k] = (T)c->eta[k];
        p.mass[k] = (T)(c->rho0[k] * vol);
        p.two_phi[k] = (T)(2.0 * c->rho0[k] / rsum);
    }
    p.four_phi_phi = (T)(4.0 * c->rho0[0] * c->rho0[1] / (rsum * rsum));
    p.vol_wall = (T)vol;
    p.nhat_eps = (T)1e-4;
    p.tvf_coef = (T)(-P.tvf_alpha * h * h);
    return p;
}

CaseDesc make_desc(const CaseRec *c) {
    CaseDesc d;
    std::memset(&d, 0, sizeof(d));
    d.dim = c->P.dim;
    d.limiter = c->P.limiter;
    d.grad_mode = c->P.grad_mode;
    d.penalty_form = c->P.penalty_form;
    d.penalty_scope = c->P.penalty_scope;
    d.wall_form = c->P.wall_form;
    d.stress_weights = c->P.stress_weights;
    d.surface_corr = c->P.surface_corr;
    d.n_fluid_phases = c->n_fluid_phases;
    d.bits = c->bits;
    for (int a = 0; a < 3; ++a) { d.ncell[a] = c->ncell[a]; d.origin[a] = c->origin[a]; }
    d.tvf_on = c->P.tvf_alpha > 0.0 ? 1 : 0;
    d.table_size = c->table_size;
    d.cs = c->cs;
    d.h = c->P.h_factor * c->P.dx;
    d.c0 = c->P.c0;
    d.gamma = c->P.gamma;
    for (int k = 0; k < 2; ++k) { d.rho0[k] = c->rho0[k]; d.eta[k] = c->eta[k]; }
    d.max_substeps = c->P.max_substeps > 0 ? c->P.max_substeps : 1000000;
    d.cfl_ad = c->P.cfl_ad;
    d.cfl_ac = c->P.cfl_ac;
    // Eq. 17's surface-tension bound sqrt(rho0 h^3 / (2 pi gamma)) depends on
    // the case only: formed once here, with the same IEEE operations in the
    // same order as the per-substep criterion used to
    for (int k = 0; k < 2; ++k)
        d.dt_surf[k] = d.gamma > 0.0
                           ? std::sqrt((c->rho0[k] * d.h * d.h * d.h) / (2.0 * 3.14159265358979323846 * d.gamma))
                           : 0.0;
    d.nbr_mode = c->P.nbr_mode;
    d.periodic = c->P.periodic;
    d.vstar_printed = c->P.vstar_form == SPHST_VSTAR_PRINTED;
    for (int a = 0; a < 3; ++a)
        d.period_len[a] = ((c->P.periodic >> a) & 1) ? c->P.period_hi[a] - c->P.period_lo[a] : 0.0;
    d.nbr_k = c->P.max_neighbors > 0 ? c->P.max_neighbors : (c->P.dim == 3 ? 128 : 48);
    d.pf = phys_of<float>(c);
    d.pd = phys_of<double>(c);
    return d;
}

int64_t footprint(const sphst_case_params *P, int64_t n) {
    const int64_t tsz = P->precision == 64 ? 8 : 4;
    const int64_t kmax = P->nbr_mode == SPHST_NBR_LIST
                             ? (P->max_neighbors > 0 ? P->max_neighbors : (P->dim == 3 ? 128 : 48)) : 0;
    // V4 arrays, scalars, ints, list (+ its pair geometry), band + band list
    const int64_t per = 9 * 4 * tsz + 2 * tsz + 6 * 4 + 4 * kmax + (SPHST_LIST_GEO ? 4 * tsz * kmax : 0) + 4 + 1 + 8 +
                        (P->surface_corr == 1 ? 2 * 4 * tsz : 0);   // own-fluid correction matrices
    // cell table: cells ~ n / 2.6^d per axis padded to a power of two
    const double side = std::pow((double)std::max<int64_t>(n, 1), 1.0 / P->dim) / 2.6 + 2.0 * P->grid_pad + 2.0;
    int bits = 0;
    while ((double)(1 << bits) < side) ++bits;
    const int64_t table = ((int64_t)1 << (P->dim * bits)) * 4 + 4;
    return per * n + table + 4096 + (int64_t)(DIAG_BLOCKS + 1) * DIAG_Q * 8;
}

// Move `cases` into one new engine (copying resident state), release
// engines nobody references any more.
static int relayout(const std::vector<CaseRec *> &cases, int precision, int block,
                    cudaStream_t stream, Engine **out) {
    Engine *e = precision == 64 ? new_engine_f64() : new_engine_f32();
    const int rc = e->setup(cases, block, stream);
    if (rc) {
        delete e;
        return rc;
    }
    for (size_t s = 0; s < cases.size(); ++s) {
        CaseRec *r = cases[s];
        Engine *old = r->engine;
        if (old) {
            for (auto &m : old->members)
                if (m == r) m = nullptr;
        }
        r->engine = e;
        r->slot = (int32_t)s;
        e->refs++;
        if (old && --old->refs == 0) delete old;
    }
    *out = e;
    return e->sync_state();
}

static void release(CaseRec *r) {
    Engine *e = r->engine;
    if (!e) return;
    for (auto &m : e->members)
        if (m == r) m = nullptr;
    r->engine = nullptr;
    if (--e->refs == 0) delete e;
}

static int live_members(const Engine *e) {
    int k = 0;
    for (auto *m : e->members)
        if (m && m->engine == e) ++k;
    return k;
}

}  // namespace sphst

using namespace sphst;

extern "C" {

void sphst_default_params(sphst_case_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->dim = 2;
    p->precision = 32;
    p->dx = 0.0;
    p->h_factor = 1.3;
    p->c0 = 10.0;
    p->gamma = 1.0;
    p->xi = -1.0;
    p->tvf_alpha = 0.2;
    p->limiter = SPHST_LIMITER_DENSITY;
    p->grad_mode = SPHST_GRAD_COMMON;
    p->penalty_form = SPHST_PENALTY_NN;
    p->loop_mode = SPHST_LOOP_GRAPH;
    p->grid_pad = 2;
    p->block = 128;
    p->lanes = 1;
    p->max_substeps = 1000000;
    p->cfl_ad = 0.1;
    p->cfl_ac = 0.6;
    p->nbr_mode = SPHST_NBR_LIST;
    p->max_neighbors = 0;
}

const char *sphst_last_error(void) { return g_error.c_str(); }

int sphst_create_case(const sphst_case_params *params, sphst_case *out) {
    if (!params || !out) { set_error("NULL argument"); return SPHST_ERR_INVALID_ARG; }
    const sphst_case_params &P = *params;
    if (P.dim != 2 && P.dim != 3) { set_error("dim must be 2 or 3"); return SPHST_ERR_UNSUPPORTED; }
    if (P.precision != 32 && P.precision != 64) { set_error("precision must be 32 or 64"); return SPHST_ERR_UNSUPPORTED; }
    if (!(P.dx > 0.0) || !(P.h_factor > 0.0) || !(P.c0 > 0.0) || !(P.gamma >= 0.0) ||
        !(P.tvf_alpha >= 0.0) || !std::isfinite(P.xi) || !(P.cfl_ad > 0.0) || !(P.cfl_ac > 0.0)) {
        set_error("dx, h_factor, c0, cfl_ad and cfl_ac must be > 0; gamma and tvf_alpha >= 0; xi finite");
        return SPHST_ERR_INVALID_ARG;
    }
    if (P.limiter < 0 || P.limiter > 3 || P.grad_mode < 0 || P.grad_mode > 1 ||
        P.penalty_form < 0 || P.penalty_form > 2 || P.loop_mode < 0 || P.loop_mode > 1 ||
        P.vstar_form < 0 || P.vstar_form > 1 || P.penalty_scope < 0 || P.penalty_scope > 1 ||
        P.wall_form < 0 || P.wall_form > 1 || P.work_lists < 0 || P.work_lists > 1 ||
        P.stress_weights < 0 || P.stress_weights > 1 || P.surface_corr < 0 || P.surface_corr > 1) {
        set_error("unknown reading, loop or work-list flag");
        return SPHST_ERR_INVALID_ARG;
    }
    if (P.nbr_mode < 0 || P.nbr_mode > 1 || P.max_neighbors < 0 || P.max_neighbors > 1024) {
        set_error("nbr_mode must be 0 or 1 and max_neighbors 0..1024");
        return SPHST_ERR_INVALID_ARG;
    }
    if (P.grid_pad < 1 || P.grid_pad > 64 || P.block < 32 || P.block > 256 || P.block % 32 ||
        (P.lanes != 1 && P.lanes != 2 && P.lanes != 4 && P.lanes != 8)) {
        set_error("grid_pad must be 1..64, block a multiple of 32 in 32..256 and lanes 1, 2, 4 or 8");
        return SPHST_ERR_INVALID_ARG;
    }
    if (P.periodic < 0 || P.periodic >= (1 << P.dim)) {
        set_error("periodic: a bit mask of the case's axes");
        return SPHST_ERR_INVALID_ARG;
    }
    double per_cs = 0.0;
    for (int a = 0; a < P.dim; ++a) {
        if (!((P.periodic >> a) & 1)) continue;
        const double L = P.period_hi[a] - P.period_lo[a];
        const double cs0 = 2.0 * P.h_factor * P.dx * (1.0 + 1.0 / 65536.0);
        if (!(L > 0.0) || !std::isfinite(L) || !(std::floor(L / cs0) >= 3.0)) {
            set_error("a periodic axis must span at least 3 cells of width 2h (1 + 2^-16)");
            return SPHST_ERR_INVALID_ARG;
        }
        const double cs = L / std::floor(L / cs0);
        if (per_cs > 0.0 && std::fabs(cs - per_cs) > 1e-12 * cs) {
            set_error("periodic axes give different cell widths: use commensurate periods");
            return SPHST_ERR_INVALID_ARG;
        }
        per_cs = cs;
    }
    sphst_case c = new (std::nothrow) sphst_case_s();
    if (!c) { set_error("host allocation failed"); return SPHST_ERR_OOM; }
    c->r.P = P;
    *out = c;
    return SPHST_OK;
}

int sphst_add_phase_particles(sphst_case c, const sphst_phase_props *props, int64_t n,
                              const double *pos, const double *vel, const double *rho,
                              int32_t *phase_id_out) {
    if (!c || !props) { set_error("NULL argument"); return SPHST_ERR_INVALID_ARG; }
    CaseRec &r = c->r;
    if (r.engine || r.gridded) { set_error("particles can only be added before the first step"); return SPHST_ERR_STATE; }
    if (n < 0 || (n > 0 && !pos)) { set_error("bad particle count or NULL positions"); return SPHST_ERR_INVALID_ARG; }
    if (r.n + n >= (int64_t)0x7fffffff) { set_error("too many particles in one case"); return SPHST_ERR_UNSUPPORTED; }
    const int dim = r.P.dim;
    PhaseRec ph;
    ph.props = *props;
    ph.first = r.n;
    ph.count = n;
    uint8_t kind;
    if (props->kind == SPHST_FLUID) {
        if (!(props->rho0 > 0.0) || !(props->eta > 0.0)) { set_error("fluid rho0 and eta must be > 0"); return SPHST_ERR_INVALID_ARG; }
        if (r.n_fluid_phases >= 2) { set_error("at most two fluid phases"); return SPHST_ERR_UNSUPPORTED; }
        ph.fluid_index = r.n_fluid_phases;
        kind = (uint8_t)r.n_fluid_phases;
    } else if (props->kind == SPHST_WALL) {
        kind = 2;
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(props->wall_vel[a])) { set_error("non-finite wall velocity"); return SPHST_ERR_INVALID_ARG; }
    } else {
        set_error("unknown particle kind");
        return SPHST_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < n * dim; ++i)
        if (!std::isfinite(pos[i]) || (vel && kind < 2 && !std::isfinite(vel[i]))) {
            set_error("non-finite position or velocity");
            return SPHST_ERR_INVALID_ARG;
        }
    if (rho && kind < 2)
        for (int64_t i = 0; i < n; ++i)
            if (!(rho[i] > 0.0) || !std::isfinite(rho[i])) { set_error("densities must be finite and > 0"); return SPHST_ERR_INVALID_ARG; }
    if (kind < 2) {
        r.rho0[kind] = props->rho0;
        r.eta[kind] = props->eta;
        r.n_fluid_phases++;
        r.n_fluid += n;
    }
    const size_t base = (size_t)r.n;
    r.pos.resize(3 * (base + n), 0.0);
    r.vel.resize(3 * (base + n), 0.0);
    r.rho.resize(base + n, 0.0);
    r.kind.resize(base + n, kind);
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < dim; ++a) {
            r.pos[3 * (base + i) + a] = pos[i * dim + a];
            r.vel[3 * (base + i) + a] = kind < 2 ? (vel ? vel[i * dim + a] : 0.0) : props->wall_vel[a];
        }
        r.rho[base + i] = kind < 2 ? (rho ? rho[i] : props->rho0) : 0.0;
    }
    r.n += n;
    r.phases.push_back(ph);
    if (phase_id_out) *phase_id_out = (int32_t)r.phases.size() - 1;
    return SPHST_OK;
}

static void fill_info(const CaseRec &r, sphst_step_info *info) {
    if (info) *info = r.info;
}

int sphst_step(sphst_case c, int64_t n_adv, sphst_step_info *info) {
    if (!c || n_adv < 0) { set_error("NULL case or negative step count"); return SPHST_ERR_INVALID_ARG; }
    CaseRec &r = c->r;
    if (r.batch) { set_error("case is a batch member; step the batch"); return SPHST_ERR_STATE; }
    if (r.info.status) { set_error(status_text(r.info.status)); fill_info(r, info); return r.info.status; }
    if (r.n_fluid == 0) { set_error("case has no fluid particles"); return SPHST_ERR_STATE; }
    if (!r.engine || live_members(r.engine) != 1) {
        Engine *e = nullptr;
        std::vector<CaseRec *> one{&r};
        const int rc = relayout(one, r.P.precision, r.P.block, r.user_stream, &e);
        if (rc) return rc;
    }
    const int rc = r.engine->step(n_adv);
    fill_info(r, info);
    if (rc) return rc;
    if (r.info.status) set_error(status_text(r.info.status));
    return r.info.status;
}

int sphst_set_stream(sphst_case c, void *cuda_stream) {
    if (!c) { set_error("NULL case"); return SPHST_ERR_INVALID_ARG; }
    if (c->r.engine) { set_error("the stream must be set before the first step"); return SPHST_ERR_STATE; }
    c->r.user_stream = (cudaStream_t)cuda_stream;
    return SPHST_OK;
}

int sphst_profile_step(sphst_case c, double *kernel_ms, int64_t *launches) {
    if (!c || !kernel_ms || !launches) { set_error("NULL argument"); return SPHST_ERR_INVALID_ARG; }
    CaseRec &r = c->r;
    if (r.batch) { set_error("case is a batch member; step the batch"); return SPHST_ERR_STATE; }
    if (r.info.status) { set_error(status_text(r.info.status)); return r.info.status; }
    if (r.n_fluid == 0) { set_error("case has no fluid particles"); return SPHST_ERR_STATE; }
    if (!r.engine || live_members(r.engine) != 1) {
        Engine *e = nullptr;
        std::vector<CaseRec *> one{&r};
        const int rc = relayout(one, r.P.precision, r.P.block, r.user_stream, &e);
        if (rc) return rc;
    }
    const int rc = r.engine->profile_step(kernel_ms, launches);
    if (rc) return rc;
    return r.info.status;
}

int sphst_case_info(sphst_case c, sphst_step_info *info) {
    if (!c || !info) { set_error("NULL argument"); return SPHST_ERR_INVALID_ARG; }
    *info = c->r.info;
    return SPHST_OK;
}

// q[] layout: see k_diag_partial (DIAG_Q quantities)
static void diag_from_q(const double *q, sphst_diagnostics *out) {
    for (int a = 0; a < 3; ++a) out->momentum[a] = q[a];
    out->kinetic = q[3];
    out->count[0] = (int64_t)q[4];
    out->count[1] = (int64_t)q[5];
    for (int a = 0; a < 3; ++a) out->first[a] = q[6 + a];
    for (int a = 0; a < 6; ++a) out->second[a] = q[9 + a];
    out->p_in = q[15];
    out->p_out = q[16];
    out->n_in = (int64_t)q[17];
    out->n_out = (int64_t)q[18];
    out->n_nonfinite = (int64_t)q[19];
}

int sphst_diagnose(sphst_case c, const double *center, double r_in, double r_out, sphst_diagnostics *out) {
    if (!c || !center || !out) { set_error("NULL argument"); return SPHST_ERR_INVALID_ARG; }
    if (!(r_in >= 0.0) || !(r_out >= 0.0)) { set_error("r_in and r_out must be >= 0"); return SPHST_ERR_INVALID_ARG; }
    const CaseRec &r = c->r;
    double q[DIAG_Q] = {0};
    if (r.engine) {
        const int rc = r.engine->diagnose(r.slot, center, r_in, r_out, q);
        if (rc) return rc;
        diag_from_q(q, out);
        return SPHST_OK;
    }
    // staged input, before the first step: the same sums on the host
    const int dim = r.P.dim;
    const double vol = dim == 2 ? r.P.dx * r.P.dx : r.P.dx * r.P.dx * r.P.dx;
    for (int64_t i = 0; i < r.n; ++i) {
        const int k = r.kind[i];
        if (k > 1) continue;
        const double *x = &r.pos[3 * i], *v = &r.vel[3 * i];
        const double m = r.rho0[k] * vol;
        bool finite = std::isfinite(r.rho[i]);
        for (int a = 0; a < 3; ++a) finite = finite && std::isfinite(x[a]) && std::isfinite(v[a]);
        if (!finite) { q[19] += 1.0; continue; }
        for (int a = 0; a < 3; ++a) q[a] += m * v[a];
        q[3] += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        q[4 + k] += 1.0;
        double r2 = 0.0;
        for (int a = 0; a < dim; ++a) r2 += (x[a] - center[a]) * (x[a] - center[a]);
        const double pr = r.P.c0 * r.P.c0 * (r.rho[i] - r.rho0[k]);
        if (k == 0) {
            for (int a = 0; a < 3; ++a) q[6 + a] += x[a];
            q[9] += x[0] * x[0]; q[10] += x[1] * x[1]; q[11] += x[2] * x[2];
            q[12] += x[0] * x[1]; q[13] += x[0] * x[2]; q[14] += x[1] * x[2];
            if (r2 < r_in * r_in) { q[15] += pr; q[17] += 1.0; }
        } else if (r2 > r_out * r_out) {
            q[16] += pr; q[18] += 1.0;
        }
    }
    diag_from_q(q, out);
    return SPHST_OK;
}

int sphst_num_particles(sphst_case c, int64_t *n_total, int64_t *n_fluid) {
    if (!c) { set_error("NULL case"); return SPHST_ERR_INVALID_ARG; }
    if (n_total) *n_total = c->r.n;
    if (n_fluid) *n_fluid = c->r.n_fluid;
    return SPHST_OK;
}

int sphst_read_fields(sphst_case c, int32_t field, double *dst, int64_t capacity) {
    if (!c || (!dst && c->r.n > 0)) { set_error("NULL argument"); return SPHST_ERR_INVALID_ARG; }
    const CaseRec &r = c->r;
    if (field < 0 || field > 6) { set_error("unknown field"); return SPHST_ERR_INVALID_ARG; }
    const int dim = r.P.dim;
    const int w = (field == SPHST_FIELD_POS || field == SPHST_FIELD_VEL || field == SPHST_FIELD_GRADC ||
                   field == SPHST_FIELD_ACC_VISC) ? dim : 1;
    if (capacity < r.n * w) { set_error("destination buffer too small"); return SPHST_ERR_CAPACITY; }
    if (field == SPHST_FIELD_PHASE) {
        for (size_t p = 0; p < r.phases.size(); ++p)
            for (int64_t i = 0; i < r.phases[p].count; ++i) dst[r.phases[p].first + i] = (double)p;
        return SPHST_OK;
    }
    if (!r.engine) {
        for (int64_t i = 0; i < r.n; ++i) {
            const int k = r.kind[i];
            switch (field) {
            case SPHST_FIELD_POS: for (int a = 0; a < dim; ++a) dst[i * dim + a] = r.pos[3 * i + a]; break;
            case SPHST_FIELD_VEL: for (int a = 0; a < dim; ++a) dst[i * dim + a] = r.vel[3 * i + a]; break;
            case SPHST_FIELD_RHO: dst[i] = k < 2 ? r.rho[i] : r.rho0[0]; break;
            case SPHST_FIELD_PRESSURE: dst[i] = k < 2 ? r.P.c0 * r.P.c0 * (r.rho[i] - r.rho0[k]) : 0.0; break;
            default: for (int a = 0; a < w; ++a) dst[i * w + a] = 0.0; break;
            }
        }
        return SPHST_OK;
    }
    return r.engine->read_field(r.slot, field, dst);
}

int sphst_destroy(sphst_case c) {
    if (!c) return SPHST_OK;
    if (c->r.batch) { set_error("remove the case from its batch first"); return SPHST_ERR_STATE; }
    release(&c->r);
    delete c;
    return SPHST_OK;
}

int sphst_debug_grid(sphst_case c, double *origin3, double *cell_size, int32_t *ncell3) {
    if (!c) { set_error("NULL case"); return SPHST_ERR_INVALID_ARG; }
    if (!c->r.gridded) { set_error("the grid is fixed at the first step"); return SPHST_ERR_STATE; }
    for (int a = 0; a < 3; ++a) {
        if (origin3) origin3[a] = c->r.origin[a];
        if (ncell3) ncell3[a] = c->r.ncell[a];
    }
    if (cell_size) *cell_size = c->r.cs;
    return SPHST_OK;
}

int sphst_debug_keys(sphst_case c, uint64_t *keys, int64_t *ids, int64_t capacity) {
    if (!c || !keys || !ids) { set_error("NULL argument"); return SPHST_ERR_INVALID_ARG; }
    if (!c->r.engine) { set_error("case not stepped yet"); return SPHST_ERR_STATE; }
    if (capacity < c->r.n) { set_error("destination buffer too small"); return SPHST_ERR_CAPACITY; }
    return c->r.engine->debug_keys(c->r.slot, keys, ids);
}

int sphst_debug_neighbor_counts(sphst_case c, int32_t *counts, int64_t capacity) {
    if (!c || !counts) { set_error("NULL argument"); return SPHST_ERR_INVALID_ARG; }
    if (!c->r.engine) { set_error("case not stepped yet"); return SPHST_ERR_STATE; }
    if (capacity < c->r.n) { set_error("destination buffer too small"); return SPHST_ERR_CAPACITY; }
    return c->r.engine->debug_counts(c->r.slot, counts);
}

int sphst_struct_sizes(int64_t *params_bytes, int64_t *phase_props_bytes, int64_t *step_info_bytes) {
    if (params_bytes) *params_bytes = (int64_t)sizeof(sphst_case_params);
    if (phase_props_bytes) *phase_props_bytes = (int64_t)sizeof(sphst_phase_props);
    if (step_info_bytes) *step_info_bytes = (int64_t)sizeof(sphst_step_info);
    return SPHST_OK;
}

int sphst_footprint_bytes(const sphst_case_params *params, int64_t n, int64_t *bytes_out) {
    if (!params || !bytes_out || n < 0 || (params->dim != 2 && params->dim != 3)) {
        set_error("bad argument");
        return SPHST_ERR_INVALID_ARG;
    }
    *bytes_out = footprint(params, n);
    return SPHST_OK;
}

// ------------------------------------------------------------------ batch
int sphst_batch_create(int32_t precision, sphst_batch *out) {
    if (!out) { set_error("NULL argument"); return SPHST_ERR_INVALID_ARG; }
    if (precision != 32 && precision != 64) { set_error("precision must be 32 or 64"); return SPHST_ERR_UNSUPPORTED; }
    sphst_batch b = new (std::nothrow) sphst_batch_s();
    if (!b) { set_error("host allocation failed"); return SPHST_ERR_OOM; }
    b->precision = precision;
    *out = b;
    return SPHST_OK;
}

int sphst_batch_add(sphst_batch b, sphst_case c) {
    if (!b || !c) { set_error("NULL argument"); return SPHST_ERR_INVALID_ARG; }
    if (c->r.batch) { set_error("case already belongs to a batch"); return SPHST_ERR_STATE; }
    if (c->r.P.precision != b->precision) { set_error("case precision differs from the batch's"); return SPHST_ERR_UNSUPPORTED; }
    if (c->r.n_fluid == 0) { set_error("case has no fluid particles"); return SPHST_ERR_STATE; }
    c->r.batch = b;
    b->members.push_back(&c->r);
    b->dirty = true;
    return SPHST_OK;
}

int sphst_batch_remove(sphst_batch b, sphst_case c) {
    if (!b || !c) { set_error("NULL argument"); return SPHST_ERR_INVALID_ARG; }
    auto it = std::find(b->members.begin(), b->members.end(), &c->r);
    if (it == b->members.end()) { set_error("case is not a member"); return SPHST_ERR_STATE; }
    b->members.erase(it);
    c->r.batch = nullptr;
    b->dirty = true;
    return SPHST_OK;
}

int sphst_batch_size(sphst_batch b, int64_t *n) {
    if (!b || !n) { set_error("NULL argument"); return SPHST_ERR_INVALID_ARG; }
    *n = (int64_t)b->members.size();
    return SPHST_OK;
}

int sphst_batch_step(sphst_batch b, int64_t n_adv, sphst_step_info *info) {
    if (!b || n_adv < 0) { set_error("NULL batch or negative step count"); return SPHST_ERR_INVALID_ARG; }
    sphst_step_info agg{};
    if (!b->members.empty()) {
        bool need = b->dirty || !b->engine || live_members(b->engine) != (int)b->members.size();
        for (auto *m : b->members) need = need || m->engine != b->engine;
        if (need) {
            const int rc = relayout(b->members, b->precision, b->members[0]->P.block, b->stream, &b->engine);
            if (rc) return rc;
            b->dirty = false;
        }
        const int rc = b->engine->step(n_adv);
        if (rc) return rc;
        for (auto *m : b->members) {
            agg.n_adv += m->info.n_adv;
            agg.n_sub += m->info.n_sub;
            agg.t = std::max(agg.t, m->info.t);
            if (m->info.status && !agg.status) agg.status = m->info.status;
        }
    }
    if (info) *info = agg;
    return SPHST_OK;
}

int sphst_batch_destroy(sphst_batch b) {
    if (!b) return SPHST_OK;
    for (auto *m : b->members) m->batch = nullptr;
    delete b;
    return SPHST_OK;
}

}  // extern "C"
