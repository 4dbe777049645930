/*
 * sph_oracle.c -- plain FP64 CPU oracle of the Riemann-based multiphase SPH
 * scheme with momentum-conserving surface stress and the zero-surface-energy
 * penalty force (Zhang, Lourenco & Hu, arXiv 2503.16082, Sections 2-4).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no source with
 * the CUDA library: no header, helper, table or constant generator.
 *
 * It is written to be checked against the paper by eye: every per-pair term
 * is evaluated from the printed formula (matrices stay matrices, the Riemann
 * star velocity stays a vector), neighbours are found by an O(N^2) search or
 * a plain uniform grid, sums run over neighbours in ascending index order,
 * and the time loop takes the steps in the order stated below.  OpenMP only
 * splits the loop over particles i; each i is summed by one thread.
 *
 * Readings taken where the paper is silent, garbled or inconsistent (each is
 * marked "reading:" where it is used):
 *   kernel      Wendland C2 with support 2h: W = a_d (1-q/2)^4 (1+2q), q=r/h.
 *   neighbours  j != i with 0 < r_ij < 2h, from positions frozen at the start
 *               of the advection step (Section 3.3).
 *   v*          the normal component of v* is -U* along e_ij (U = -v.e_ij in
 *               Eq. 10), the tangential part is that of the pair average.
 *   limiter     Eq. 11 with (P_L+P_R) replaced by (rho_L+rho_R), which makes
 *               beta dimensionless; flags give beta = 1 and beta = 0.
 *   n-hat       n = gradC/|gradC| when |gradC| h > 1e-4, else the particle
 *               is not on an interface: Pi = 0, T = I, N = 0.
 *   walls       fixed particles of volume dx^d carrying a prescribed
 *               velocity; pressure pairs use the mirror state (rho_i, p_i,
 *               2 U_w - U_L), whose P* the flag wall_form = 1 floors at zero
 *               (a wall then never pulls a particle in tension towards
 *               itself); continuity uses v* = v_w; viscous pairs use
 *               eta_i and v_i - v_w; walls take no part in the colour
 *               function or the surface force.
 *   surface     Eq. 33 divided by m_i, so the acceleration carries 1/rho_i.
 *   C-hat       Eq. 30 with A = gradCbar (x) r_ij, contracted as below.
 *   gradCbar    for a pair of different phases the colour of j is taken on
 *               the same side as i: gradCbar = (gradC_i - gradC_j)/2 (flag:
 *               the printed (gradC_i + gradC_j)/2).
 *   integrator  per acoustic substep: kick v with a(rho^n, v^n), continuity
 *               with the kicked v, drift r with the kicked v.
 *   viscosity   Eq. 13 already is an acceleration (it carries 1/rho_i).
 *   C-hat       (the contraction) A A^T/|A| = |gradCbar| r_ij nbar nbar^T with
 *               nbar = gradCbar/|gradCbar|; the flag penalty_form = 1 takes
 *               A^T A/|A| = |gradCbar| r_ij e e^T instead.  The flag
 *               penalty_scope = 1 drops the penalty from the same-phase line
 *               of Eq. 33 and keeps it on the cross-phase line (an ablation).
 *   correction  the same-phase line of Eq. 33 with grad_i W_ij as printed; the
 *               flag surface_corr = 1 takes (B^k_i + B^k_j)/2 grad_i W_ij, B^k
 *               the correction matrix of Eq. 15 summed over the particle's own
 *               fluid (once per advection step, frozen configuration).
 *   stresses    the cross-phase line of Eqs. 26 and 33 as printed,
 *               2 phi_j Pi_i + 2 phi_i Pi_j; the flag stress_weights = 1 takes
 *               2 phi_i Pi_i + 2 phi_j Pi_j (each stress with its own
 *               particle's weight; the same at density ratio 1).
 *   periodic    an axis flagged periodic (the shear drop of Section 5.2 is
 *               periodic in x) wraps positions into [box_lo, box_hi) and takes
 *               every pair vector as its minimum image; the key grid of a
 *               periodic axis has floor(L / cs0) cells of width L / that count
 *               (cs0 = 2h (1 + 2^-16)), starting at box_lo.
 *   TVF         Eq. 14 with the sign that moves a particle away from the side
 *               where its neighbours crowd: dr_i = -alpha h^2 sum_j (B_i + B_j)
 *               grad_i W_ij V_j.  With the stated grad W convention
 *               sum_j r_ij (x) grad_i W_ij V_j is close to -I, so B_i (Eq. 15)
 *               is close to +I and the printed sign would move particles
 *               towards crowds.  Walls lend their fluid partner's B_i; a
 *               particle whose moment matrix is near singular (|det| < 1e-3)
 *               takes B = I.  dr_i is computed from the frozen configuration
 *               with the viscous force and added to the positions once per
 *               advection step.
 *
 * Pinned by closed forms: every term of Eq. 33 for a single pair.  The
 * cross-phase line by an isolated pair of different fluids (the penalty) and,
 * through ora_surface_pair, by a pair whose normals lie at angles to e_ij
 * (the two stresses and their weights, for both readings); the same-phase
 * line, through ora_surface_pair (the routine the force loop calls), by
 * three configurations that reduce by hand: normals across the pair (no
 * penalty with the default contraction, a repulsion with A^T A / |A|),
 * normals along the pair (T-bar removes the penalty) and mirrored normals
 * (a closed form that separates the three contractions of Eq. 30).  The
 * integrator and the wall reading's mirror pressure and volume are pinned in
 * the linear regime by acoustic modes (a standing wave, and the lowest mode
 * between walls), v* = v_w at a wall by the water hammer (p = rho c0 U
 * behind the front), the wall's dissipative term (mirrored normal velocity,
 * limiter) by the closed form of a fluid particle beside one wall particle.
 * Integral observables (the Laplace jump, the oscillation period) are
 * checked against the paper's closed forms in runs of the whole scheme.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* parameters (mirrors the problem statement of Sections 2-3)                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t dim;          /* 2 or 3 */
    int32_t limiter;      /* 0: dimensionless reading of Eq. 11; 1: beta = 1; 2: beta = 0;
                             3: Eq. 11 as printed, (P_L + P_R) kept */
    int32_t grad_mode;    /* 0: common colour side for gradCbar; 1: as printed */
    int32_t nbr_mode;     /* 0: O(N^2) search; 1: uniform grid */
    int32_t n_threads;    /* <= 0: OpenMP default */
    int32_t penalty_form; /* 0: C-hat = C I - A A^T/|A|; 1: C I - A^T A/|A|;
                             2: the scalar C_ij - gradCbar.r_ij of Eq. 29 times I
                             (not momentum-conserving, an ablation) */
    double dx;            /* initial particle spacing dp */
    double h;             /* smoothing length (1.3 dp in Section 5) */
    double c0;            /* one sound speed for all phases (Section 2) */
    double gamma;         /* surface tension coefficient */
    double xi;            /* penalty coefficient; < 0: 1.3 n + 0.6 (Section 4.2) */
    double rho0[2];       /* reference densities of fluid 0 and fluid 1 */
    double eta[2];        /* dynamic viscosities */
    double nhat_eps;      /* |gradC| h threshold for an interface particle */
    int64_t max_substeps; /* guard against a stalled advection step */
    double tvf_alpha;     /* transport-velocity coefficient (0.2 in Section 3.2); 0: off */
    double cfl_ad;        /* advection factor of Eq. 16 (0.1 as printed) */
    double cfl_ac;        /* acoustic factor of Eq. 17 (0.6 as printed) */
    int32_t periodic;     /* bit d set: axis d is periodic on [box_lo[d], box_hi[d]) */
    int32_t pad2_;
    double box_lo[3], box_hi[3];
    int32_t vstar_form;   /* 0: normal component -U* (reading); 1: Eq. 8 as printed */
    int32_t penalty_scope; /* 0: the penalty on both lines of Eq. 33 (as printed);
                              1: on the cross-phase line only (an ablation) */
    int32_t wall_form;    /* 0: the wall pair's P* from the mirror state as it comes;
                             1: max(P*, 0), a wall pushes and never pulls */
    int32_t stress_weights; /* cross-phase line of Eq. 26/33: 0: 2 phi_j Pi_i + 2 phi_i Pi_j
                               as printed; 1: 2 phi_i Pi_i + 2 phi_j Pi_j (each stress
                               weighted by its own particle's phi) */
    int32_t surface_corr; /* same-phase line of Eq. 33: 0: grad_i W_ij as printed;
                             1: (B^k_i + B^k_j)/2 grad_i W_ij with B^k the correction
                             matrix of Eq. 15 summed over the particle's own fluid */
    int32_t pad4_;
} ora_params;

typedef struct {
    int64_t n_adv;        /* advection steps taken */
    int64_t n_sub;        /* acoustic substeps taken */
    double t;             /* physical time advanced */
    double last_dt_ad;
    double last_dt_ac;
    int32_t status;       /* 0 ok, 1 non-finite, 2 stalled, 3 coincident particles */
    int32_t pad_;
} ora_info;

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */
/* ------------------------------------------------------------------------ */
static int is_fluid(int32_t k) { return k == 0 || k == 1; }

static double dot3(const double *a, const double *b, int dim)
{
    double s = 0.0;
    for (int d = 0; d < dim; ++d) s += a[d] * b[d];
    return s;
}

static double norm3(const double *a, int dim) { return sqrt(dot3(a, a, dim)); }

static int is_periodic(const ora_params *P, int d) { return (P->periodic >> d) & 1; }

/* minimum image of a pair vector on the periodic axes */
static void min_image(const ora_params *P, double *rv)
{
    for (int d = 0; d < P->dim; ++d) {
        if (!is_periodic(P, d)) continue;
        double L = P->box_hi[d] - P->box_lo[d];
        if (rv[d] > 0.5 * L) rv[d] -= L;
        else if (rv[d] < -0.5 * L) rv[d] += L;
    }
}

/* a coordinate of a periodic axis brought back into [box_lo, box_hi) */
static double wrap_coord(const ora_params *P, int d, double x)
{
    if (!is_periodic(P, d)) return x;
    double L = P->box_hi[d] - P->box_lo[d];
    double y = x - L * floor((x - P->box_lo[d]) / L);
    return y >= P->box_hi[d] ? y - L : y;
}

static void set_threads(const ora_params *P)
{
#ifdef _OPENMP
    if (P->n_threads > 0) omp_set_num_threads(P->n_threads);
#else
    (void)P;
#endif
}

/* Section 4.2, after Eq. 33: xi = 1.3 n + 0.6 for a density ratio of 10^n. */
double ora_xi(const ora_params *P)
{
    if (P->xi >= 0.0) return P->xi;
    double hi = P->rho0[0] > P->rho0[1] ? P->rho0[0] : P->rho0[1];
    double lo = P->rho0[0] > P->rho0[1] ? P->rho0[1] : P->rho0[0];
    return 1.3 * log10(hi / lo) + 0.6;
}

/* particle mass: reference density times the lattice volume dp^d */
static double mass_of(const ora_params *P, int32_t k)
{
    double vol = P->dim == 2 ? P->dx * P->dx : P->dx * P->dx * P->dx;
    return P->rho0[k] * vol;
}

static double wall_volume(const ora_params *P)
{
    return P->dim == 2 ? P->dx * P->dx : P->dx * P->dx * P->dx;
}

/* ------------------------------------------------------------------------ */
/* kernel (Section 5: 5th-order Wendland, h = 1.3 dp, cut-off 2.6 dp)         */
/* ------------------------------------------------------------------------ */
static double wendland_alpha(int dim, double h)
{
    /* normalisation so that the kernel integrates to one over its support */
    return dim == 2 ? 7.0 / (4.0 * ORA_PI * h * h)
                    : 21.0 / (16.0 * ORA_PI * h * h * h);
}

double ora_kernel_W(int32_t dim, double h, double r)
{
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return wendland_alpha(dim, h) * t * t * t * t * (1.0 + 2.0 * q);
}

/* dW/dr, the radial derivative used by grad_i W_ij = dW/dr e_ij (Section 3.1) */
double ora_kernel_dW(int32_t dim, double h, double r)
{
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return -5.0 * wendland_alpha(dim, h) * q * t * t * t / h;
}

/* ------------------------------------------------------------------------ */
/* neighbour search                                                          */
/* ------------------------------------------------------------------------ */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* |x_i - x_j|^2 of the pair's minimum image */
static double pair_dist2(const ora_params *P, const double *xi, const double *xj)
{
    double rv[3] = {0, 0, 0};
    for (int d = 0; d < P->dim; ++d) rv[d] = xi[d] - xj[d];
    min_image(P, rv);
    double r2 = 0.0;
    for (int d = 0; d < P->dim; ++d) r2 += rv[d] * rv[d];
    return r2;
}

/* cell of a position in the search grid */
static void grid_cell(const ora_params *P, const double *x, const double *lo, const double *cwd,
                      const int64_t *nc, int64_t *ci)
{
    for (int d = 0; d < P->dim; ++d) {
        ci[d] = (int64_t)floor((wrap_coord(P, d, x[d]) - lo[d]) / cwd[d]);
        if (ci[d] >= nc[d]) ci[d] = nc[d] - 1;
        if (ci[d] < 0) ci[d] = 0;
    }
}

/* linear index of the neighbour cell ci + o (wrapped on periodic axes);
 * 0 when it lies outside a non-periodic axis */
static int grid_neighbour(const ora_params *P, const int64_t *ci, int64_t ox, int64_t oy, int64_t oz,
                          const int64_t *nc, int64_t *c_out)
{
    int64_t c3[3] = {ci[0] + ox, ci[1] + oy, ci[2] + oz};
    for (int d = 0; d < P->dim; ++d) {
        if (c3[d] >= 0 && c3[d] < nc[d]) continue;
        if (!is_periodic(P, d)) return 0;
        c3[d] = (c3[d] + nc[d]) % nc[d];
    }
    int64_t c = 0;
    for (int d = P->dim - 1; d >= 0; --d) c = c * nc[d] + c3[d];
    *c_out = c;
    return 1;
}

/* A neighbour of i is any j != i with 0 < r_ij < 2h.  Returns the total
 * number of pairs; fills counts[n] and, when idx != NULL and the total fits
 * in cap, the CSR column array (ascending j within each row).  Returns -1 on
 * a coincident pair (r_ij = 0, j != i). */
int64_t ora_neighbors(const ora_params *P, int64_t n, const double *pos,
                      int32_t *counts, int32_t *idx, int64_t cap)
{
    const int dim = P->dim;
    const double R2 = (2.0 * P->h) * (2.0 * P->h);
    int coincident = 0;
    int64_t *cell_of = NULL, *cell_start = NULL, *order = NULL;
    int64_t nc[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0};
    double cwd[3] = {2.0 * P->h, 2.0 * P->h, 2.0 * P->h};
    int brute = P->nbr_mode == 0 || n == 0;
    for (int d = 0; d < dim; ++d)      /* a periodic axis shorter than 3 cells: brute force */
        if (is_periodic(P, d) && floor((P->box_hi[d] - P->box_lo[d]) / (2.0 * P->h)) < 3.0) brute = 1;

    if (!brute) {
        /* plain uniform grid of cell width 2h over the bounding box; a
         * periodic axis is cut into floor(L / 2h) cells that wrap around */
        double hi[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) { lo[d] = pos[d]; hi[d] = pos[d]; }
        for (int64_t i = 0; i < n; ++i)
            for (int d = 0; d < dim; ++d) {
                if (pos[3 * i + d] < lo[d]) lo[d] = pos[3 * i + d];
                if (pos[3 * i + d] > hi[d]) hi[d] = pos[3 * i + d];
            }
        int64_t total = 1;
        for (int d = 0; d < dim; ++d) {
            if (is_periodic(P, d)) {
                double L = P->box_hi[d] - P->box_lo[d];
                lo[d] = P->box_lo[d];
                nc[d] = (int64_t)floor(L / (2.0 * P->h));
                cwd[d] = L / (double)nc[d];
            } else {
                nc[d] = (int64_t)floor((hi[d] - lo[d]) / cwd[d]) + 1;
            }
            total *= nc[d];
        }
        cell_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        cell_start = (int64_t *)calloc((size_t)total + 1, sizeof(int64_t));
        order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            int64_t c = 0;
            for (int d = dim - 1; d >= 0; --d) {
                int64_t k = (int64_t)floor((wrap_coord(P, d, pos[3 * i + d]) - lo[d]) / cwd[d]);
                if (k >= nc[d]) k = nc[d] - 1;
                if (k < 0) k = 0;
                c = c * nc[d] + k;
            }
            cell_of[i] = c;
            cell_start[c + 1]++;
        }
        for (int64_t c = 0; c < total; ++c) cell_start[c + 1] += cell_start[c];
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)total);
        memcpy(fill, cell_start, sizeof(int64_t) * (size_t)total);
        for (int64_t i = 0; i < n; ++i) order[fill[cell_of[i]]++] = i;
        free(fill);
    }

    int64_t total_pairs = 0;
    set_threads(P);
    /* pass 1: counts */
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : total_pairs) reduction(| : coincident)
    for (int64_t i = 0; i < n; ++i) {
        int32_t cnt = 0;
        const double *xi = pos + 3 * i;
        if (brute) {
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double r2 = pair_dist2(P, xi, pos + 3 * j);
                if (r2 == 0.0) coincident = 1;
                else if (r2 < R2) cnt++;
            }
        } else {
            int64_t ci[3] = {0, 0, 0};
            grid_cell(P, xi, lo, cwd, nc, ci);
            for (int64_t oz = (dim == 3 ? -1 : 0); oz <= (dim == 3 ? 1 : 0); ++oz)
                for (int64_t oy = -1; oy <= 1; ++oy)
                    for (int64_t ox = -1; ox <= 1; ++ox) {
                        int64_t c = 0;
                        if (!grid_neighbour(P, ci, ox, oy, oz, nc, &c)) continue;
                        for (int64_t s = cell_start[c]; s < cell_start[c + 1]; ++s) {
                            int64_t j = order[s];
                            if (j == i) continue;
                            double r2 = pair_dist2(P, xi, pos + 3 * j);
                            if (r2 == 0.0) coincident = 1;
                            else if (r2 < R2) cnt++;
                        }
                    }
        }
        counts[i] = cnt;
        total_pairs += cnt;
    }

    if (idx != NULL && total_pairs <= cap) {
        int64_t *row = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
        row[0] = 0;
        for (int64_t i = 0; i < n; ++i) row[i + 1] = row[i] + counts[i];
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            int64_t w = row[i];
            const double *xi = pos + 3 * i;
            if (brute) {
                for (int64_t j = 0; j < n; ++j) {
                    if (j == i) continue;
                    double r2 = pair_dist2(P, xi, pos + 3 * j);
                    if (r2 > 0.0 && r2 < R2) idx[w++] = (int32_t)j;
                }
            } else {
                int64_t ci[3] = {0, 0, 0};
                grid_cell(P, xi, lo, cwd, nc, ci);
                for (int64_t oz = (dim == 3 ? -1 : 0); oz <= (dim == 3 ? 1 : 0); ++oz)
                    for (int64_t oy = -1; oy <= 1; ++oy)
                        for (int64_t ox = -1; ox <= 1; ++ox) {
                            int64_t c = 0;
                            if (!grid_neighbour(P, ci, ox, oy, oz, nc, &c)) continue;
                            for (int64_t s = cell_start[c]; s < cell_start[c + 1]; ++s) {
                                int64_t j = order[s];
                                if (j == i) continue;
                                double r2 = pair_dist2(P, xi, pos + 3 * j);
                                if (r2 > 0.0 && r2 < R2) idx[w++] = (int32_t)j;
                            }
                        }
                qsort(idx + row[i], (size_t)counts[i], sizeof(int32_t), cmp_i32);
            }
        }
        free(row);
    }
    free(cell_of);
    free(cell_start);
    free(order);
    return coincident ? -1 : total_pairs;
}

/* ------------------------------------------------------------------------ */
/* cell keys (the library's Morton-ordered cell list, restated for checking) */
/* ------------------------------------------------------------------------ */
/* Cell width cs = 2h (1 + 2^-16); grid origin = bounding-box minimum minus
 * pad cells; cells per axis = floor((max - origin)/cs) + 1 + pad.  With a
 * periodic axis of length L: cs = L / floor(L / (2h (1 + 2^-16))) for every
 * axis, and that axis starts at box_lo with exactly L / cs cells.  Cell
 * coordinates interleave into a Morton code with axis 0 in the lowest bit.
 * The canonical particle order sorts by (Morton code, insertion index). */
void ora_grid(const ora_params *P, int64_t n, const double *pos, int32_t pad,
              double *origin3, double *cs_out, int32_t *ncell3)
{
    double cs = 2.0 * P->h * (1.0 + 1.0 / 65536.0);
    for (int d = 0; d < P->dim; ++d)   /* a periodic axis sets the width: L / floor(L / cs0) */
        if (is_periodic(P, d)) {
            double L = P->box_hi[d] - P->box_lo[d];
            cs = L / floor(L / (2.0 * P->h * (1.0 + 1.0 / 65536.0)));
        }
    for (int d = 0; d < 3; ++d) { origin3[d] = 0.0; ncell3[d] = 1; }
    for (int d = 0; d < P->dim; ++d) {
        if (is_periodic(P, d)) {
            double L = P->box_hi[d] - P->box_lo[d];
            origin3[d] = P->box_lo[d];
            ncell3[d] = (int32_t)floor(L / (2.0 * P->h * (1.0 + 1.0 / 65536.0)));
            continue;
        }
        double lo = pos[d], hi = pos[d];
        for (int64_t i = 1; i < n; ++i) {
            if (pos[3 * i + d] < lo) lo = pos[3 * i + d];
            if (pos[3 * i + d] > hi) hi = pos[3 * i + d];
        }
        origin3[d] = lo - (double)pad * cs;
        ncell3[d] = (int32_t)floor((hi - origin3[d]) / cs) + 1 + pad;
    }
    *cs_out = cs;
}

static uint64_t morton_code(const int64_t *c, int dim)
{
    uint64_t code = 0;
    int bits = dim == 2 ? 16 : 10;
    for (int b = 0; b < bits; ++b)
        for (int d = 0; d < dim; ++d)
            code |= (uint64_t)((c[d] >> b) & 1) << (b * dim + d);
    return code;
}

/* keys[i] = Morton code of i's cell, cells[3i..] = its cell coordinates;
 * order[k] = insertion index of the k-th particle in canonical order.
 * Returns the number of particles outside the grid (their key is ~0). */
int64_t ora_cell_keys(const ora_params *P, int64_t n, const double *pos,
                      const double *origin3, double cs, const int32_t *ncell3,
                      uint64_t *keys, int32_t *cells, int64_t *order)
{
    int64_t outside = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3] = {0, 0, 0};
        int bad = 0;
        for (int d = 0; d < P->dim; ++d) {
            if (is_periodic(P, d)) {
                /* position brought into the period, then its cell (the last
                 * cell also takes a position that rounds onto box_hi) */
                double L = P->box_hi[d] - P->box_lo[d];
                double rel = pos[3 * i + d] - origin3[d];
                rel = rel - L * floor(rel / L);
                c[d] = (int64_t)floor(rel / cs);
                if (c[d] >= ncell3[d]) c[d] = ncell3[d] - 1;
                continue;
            }
            c[d] = (int64_t)floor((pos[3 * i + d] - origin3[d]) / cs);
            if (c[d] < 0 || c[d] >= ncell3[d]) bad = 1;
        }
        for (int d = 0; d < 3; ++d) cells[3 * i + d] = (int32_t)c[d];
        keys[i] = bad ? ~(uint64_t)0 : morton_code(c, P->dim);
        outside += bad;
        order[i] = i;
    }
    /* insertion sort is too slow for large n; a plain merge sort on (key, i) */
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t a = lo, b = mid, w = lo;
            while (a < mid && b < hi) {
                int64_t x = order[a], y = order[b];
                int take_a = keys[x] < keys[y] || (keys[x] == keys[y] && x < y);
                tmp[w++] = take_a ? order[a++] : order[b++];
            }
            while (a < mid) tmp[w++] = order[a++];
            while (b < hi) tmp[w++] = order[b++];
        }
        memcpy(order, tmp, sizeof(int64_t) * (size_t)n);
    }
    free(tmp);
    return outside;
}

/* ------------------------------------------------------------------------ */
/* Riemann solver along a particle pair (Section 3.1, Eqs. 8-12)             */
/* ------------------------------------------------------------------------ */
typedef struct { double rho, U, p, c; } rstate;

/* Eq. 11, dissipation limiter. reading: (P_L + P_R) -> (rho_L + rho_R). */
static double limiter_beta(const ora_params *P, rstate L, rstate R)
{
    if (P->limiter == 1) return 1.0;
    if (P->limiter == 2) return 0.0;
    double num = P->limiter == 3 ? L.p + R.p : L.rho + R.rho;   /* 3: as printed */
    double x = num * (L.U - R.U) / (L.rho * L.c + R.rho * R.c);
    double b = 3.0 * (x > 0.0 ? x : 0.0);
    return b < 1.0 ? b : 1.0;
}

/* Eq. 12, third line: density-weighted pair pressure */
static double pair_pbar(double rho_i, double p_i, double rho_j, double p_j)
{
    return (rho_i * p_j + rho_j * p_i) / (rho_i + rho_j);
}

/* Eq. 8, second line */
static double riemann_Pstar(const ora_params *P, rstate L, rstate R, double pbar)
{
    double beta = limiter_beta(P, L, R);
    double zl = L.rho * L.c, zr = R.rho * R.c;
    return pbar + beta * zl * zr * (L.U - R.U) / (zl + zr);
}

/* Eq. 9 */
static double riemann_Ustar(rstate L, rstate R)
{
    double zl = L.rho * L.c, zr = R.rho * R.c;
    return (zl * L.U + zr * R.U + L.p - R.p) / (zl + zr);
}

/* Eq. 8, first line, with Eq. 12's pair averages.  reading: with
 * U = -v.e_ij (Eq. 10) the star velocity has normal component -U* along
 * e_ij and keeps the tangential part of the averaged velocity. */
static void riemann_vstar(const ora_params *P, rstate L, rstate R, double rho_i, const double *v_i,
                          double rho_j, const double *v_j, const double *e,
                          int dim, double *vstar)
{
    double Us = riemann_Ustar(L, R);
    double Ubar = (L.rho * L.U + R.rho * R.U) / (L.rho + R.rho);
    for (int d = 0; d < dim; ++d) {
        double vbar = (rho_i * v_i[d] + rho_j * v_j[d]) / (rho_i + rho_j);
        vstar[d] = P->vstar_form == 1 ? Us * e[d] + (vbar - Ubar * e[d])     /* as printed */
                                      : -Us * e[d] + (vbar + Ubar * e[d]);
    }
}

/* Exposed for the Riemann pins: given i and j states along e, return
 * out[0] = P*, out[1] = U*, out[2] = beta, out[3] = pbar, out[4..6] = v*. */
void ora_riemann_pair(const ora_params *P, double rho_i, double p_i,
                      const double *v_i, double rho_j, double p_j,
                      const double *v_j, const double *e, double *out)
{
    int dim = P->dim;
    rstate L = {rho_i, -dot3(v_i, e, dim), p_i, P->c0};   /* Eq. 10 */
    rstate R = {rho_j, -dot3(v_j, e, dim), p_j, P->c0};
    double pbar = pair_pbar(rho_i, p_i, rho_j, p_j);
    out[0] = riemann_Pstar(P, L, R, pbar);
    out[1] = riemann_Ustar(L, R);
    out[2] = limiter_beta(P, L, R);
    out[3] = pbar;
    double vs[3] = {0, 0, 0};
    riemann_vstar(P, L, R, rho_i, v_i, rho_j, v_j, e, dim, vs);
    for (int d = 0; d < 3; ++d) out[4 + d] = vs[d];
}

/* ------------------------------------------------------------------------ */
/* frozen pair geometry of one advection step                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    int64_t *row;     /* CSR row starts, n+1 */
    int32_t *col;     /* neighbour j */
    double *r;        /* r_ij */
    double *e;        /* e_ij = (r_i - r_j)/r_ij, 3 per pair */
    double *dW;       /* dW/dr at r_ij */
} pairs_t;

static void pairs_free(pairs_t *pp)
{
    free(pp->row); free(pp->col); free(pp->r); free(pp->e); free(pp->dW);
    memset(pp, 0, sizeof(*pp));
}

static int pairs_build(const ora_params *P, int64_t n, const double *snap, pairs_t *pp)
{
    memset(pp, 0, sizeof(*pp));
    pp->n = n;
    int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t tot = ora_neighbors(P, n, snap, cnt, NULL, 0);
    if (tot < 0) { free(cnt); return -1; }
    pp->row = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    pp->row[0] = 0;
    for (int64_t i = 0; i < n; ++i) pp->row[i + 1] = pp->row[i] + cnt[i];
    size_t m = (size_t)(tot > 0 ? tot : 1);
    pp->col = (int32_t *)malloc(sizeof(int32_t) * m);
    pp->r = (double *)malloc(sizeof(double) * m);
    pp->e = (double *)malloc(sizeof(double) * 3 * m);
    pp->dW = (double *)malloc(sizeof(double) * m);
    ora_neighbors(P, n, snap, cnt, pp->col, tot);
    free(cnt);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = pp->row[i]; k < pp->row[i + 1]; ++k) {
            int64_t j = pp->col[k];
            double rv[3] = {0, 0, 0};
            for (int d = 0; d < P->dim; ++d) rv[d] = snap[3 * i + d] - snap[3 * j + d];
            min_image(P, rv);
            double r = norm3(rv, P->dim);
            pp->r[k] = r;
            for (int d = 0; d < 3; ++d) pp->e[3 * k + d] = rv[d] / r;
            pp->dW[k] = ora_kernel_dW(P->dim, P->h, r);
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* state                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    double *pos, *vel, *rho;  /* 3, 3, 1 per particle (fluids; walls: vel = v_w) */
    const int32_t *kind;      /* 0/1 fluid phase, 2 wall */
} state_t;

/* particle volume V_j = m_j / rho_j (walls: dp^d) */
static double volume_of(const ora_params *P, const state_t *S, int64_t j)
{
    if (!is_fluid(S->kind[j])) return wall_volume(P);
    return mass_of(P, S->kind[j]) / S->rho[j];
}

/* Eq. 3: p = c0^2 (rho - rho0) */
static double pressure_of(const ora_params *P, const state_t *S, int64_t j)
{
    return P->c0 * P->c0 * (S->rho[j] - P->rho0[S->kind[j]]);
}

/* Eq. 23 */
static double phi_of(const ora_params *P, int32_t ki, int32_t kj)
{
    return P->rho0[ki] / (P->rho0[ki] + P->rho0[kj]);
}

/* Eq. 22: gradC_i = sum_j 2 phi_i C_ij grad_i W_ij V_j, C_ij = 1 for j in
 * the other fluid and 0 otherwise (walls carry no colour). */
static void color_gradient(const ora_params *P, const state_t *S, const pairs_t *pp,
                           double *gradC)
{
    const int dim = P->dim;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < S->n; ++i) {
        double g[3] = {0, 0, 0};
        if (is_fluid(S->kind[i])) {
            for (int64_t k = pp->row[i]; k < pp->row[i + 1]; ++k) {
                int64_t j = pp->col[k];
                if (!is_fluid(S->kind[j])) continue;
                double Cij = S->kind[j] == S->kind[i] ? 0.0 : 1.0;
                if (Cij == 0.0) continue;
                double phi_i = phi_of(P, S->kind[i], S->kind[j]);
                double Vj = volume_of(P, S, j);
                for (int d = 0; d < dim; ++d)
                    g[d] += 2.0 * phi_i * Cij * pp->dW[k] * pp->e[3 * k + d] * Vj;
            }
        }
        for (int d = 0; d < 3; ++d) gradC[3 * i + d] = g[d];
    }
}

/* Eqs. 21 and 24 plus the projections below Eq. 33 (3x3 row-major) */
typedef struct { double nhat[3]; double Pi[9], T[9], N[9]; } stress_t;

static void surface_stress(const ora_params *P, const double *g, stress_t *st)
{
    const int dim = P->dim;
    double gn = norm3(g, dim);
    memset(st, 0, sizeof(*st));
    int iface = gn * P->h > P->nhat_eps;
    for (int d = 0; d < dim; ++d) st->nhat[d] = iface ? g[d] / gn : 0.0;
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) {
            double I = a == b ? 1.0 : 0.0;
            double nn = st->nhat[a] * st->nhat[b];
            st->N[3 * a + b] = nn;
            st->T[3 * a + b] = I - nn;
            st->Pi[3 * a + b] = iface ? P->gamma * (I - nn) * gn : 0.0;
        }
}

/* Eq. 13: viscous acceleration.  reading: the printed F^v_i already carries
 * the 1/rho_i prefactor, so it is used as an acceleration as it stands.
 * Walls: eta_bar = eta_i and v_ij = v_i - v_w. */
static void viscous_acc(const ora_params *P, const state_t *S, const pairs_t *pp,
                        double *av)
{
    const int dim = P->dim;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < S->n; ++i) {
        double a[3] = {0, 0, 0};
        int32_t ki = S->kind[i];
        if (is_fluid(ki)) {
            for (int64_t k = pp->row[i]; k < pp->row[i + 1]; ++k) {
                int64_t j = pp->col[k];
                int32_t kj = S->kind[j];
                double eta_bar = is_fluid(kj)
                    ? 2.0 * P->eta[ki] * P->eta[kj] / (P->eta[ki] + P->eta[kj])
                    : P->eta[ki];
                double Vj = volume_of(P, S, j);
                for (int d = 0; d < dim; ++d) {
                    double vij = S->vel[3 * i + d] - S->vel[3 * j + d];
                    a[d] += eta_bar * (vij / pp->r[k]) * pp->dW[k] * Vj;
                }
            }
            for (int d = 0; d < dim; ++d) a[d] *= 2.0 / S->rho[i];
        }
        for (int d = 0; d < 3; ++d) av[3 * i + d] = a[d];
    }
}

/* The pair matrix S_ij of Eq. 33 (the bracket that multiplies grad_i W_ij V_j)
 * for fluids ki, kj with stresses si, sj (Eq. 24 and the projections below
 * Eq. 33), colour gradients gi, gj, unit vector e = e_ij and distance r:
 *   same phase:  Pi_i + Pi_j + xi gamma T-bar C-hat / r
 *   other phase: 2 phi_j Pi_i + 2 phi_i Pi_j - 4 phi_i phi_j xi gamma N-bar C-hat / r
 * with C-hat from Eq. 30 (the contraction of the flag penalty_form) and
 * grad C-bar from Eq. 28 (the colour side of the flag grad_mode). */
static void surface_pair_matrix(const ora_params *P, int32_t ki, int32_t kj, const stress_t *si,
                                const stress_t *sj, const double *gi, const double *gj,
                                const double *e, double r, double xi, double *S)
{
    const int dim = P->dim;
    int same = kj == ki;
    double Cij = same ? 0.0 : 1.0;
    double phi_i = phi_of(P, ki, kj), phi_j = phi_of(P, kj, ki);
    /* Eq. 28 average gradient; reading: common colour side */
    double gbar[3] = {0, 0, 0};
    double sgn = (same || P->grad_mode == 1) ? 1.0 : -1.0;
    for (int d = 0; d < dim; ++d)
        gbar[d] = 0.5 * (gi[d] + sgn * gj[d]);
    /* Eq. 30: C-hat = C_ij I - (A/|A|) A, A = gbar (x) r_ij, with the
     * matrix product taken as A A^T (penalty_form 0) or A^T A (1) */
    double rvec[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) rvec[d] = r * e[d];
    double A[9] = {0}, AtA[9] = {0}, normA = 0.0;
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) {
            A[3 * a + b] = gbar[a] * rvec[b];
            normA += A[3 * a + b] * A[3 * a + b];
        }
    normA = sqrt(normA);
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) {
            double s = 0.0;
            for (int c = 0; c < dim; ++c)
                s += P->penalty_form == 0 ? A[3 * a + c] * A[3 * b + c]
                                          : A[3 * c + a] * A[3 * c + b];
            AtA[3 * a + b] = s;
        }
    double Chat[9] = {0};
    double gr = dot3(gbar, rvec, dim);            /* Eq. 29: scalar C-hat */
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b)
            Chat[3 * a + b] = P->penalty_form == 2
                ? (a == b ? Cij - gr : 0.0)
                : (a == b ? Cij : 0.0) - (normA > 0.0 ? AtA[3 * a + b] / normA : 0.0);
    /* projection: T-bar (same phase) or N-bar (other phase) */
    double M[9] = {0};
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b)
            M[3 * a + b] = same ? 0.5 * (si->T[3 * a + b] + sj->T[3 * a + b])
                                : 0.5 * (si->N[3 * a + b] + sj->N[3 * a + b]);
    double MC[9] = {0};
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) {
            double s = 0.0;
            for (int c = 0; c < dim; ++c) s += M[3 * a + c] * Chat[3 * c + b];
            MC[3 * a + b] = s;
        }
    memset(S, 0, 9 * sizeof(double));
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) {
            double pen = xi * P->gamma * MC[3 * a + b] / r;
            S[3 * a + b] = same
                ? si->Pi[3 * a + b] + sj->Pi[3 * a + b] + (P->penalty_scope == 1 ? 0.0 : pen)
                : (P->stress_weights == 1
                       ? 2.0 * phi_i * si->Pi[3 * a + b] + 2.0 * phi_j * sj->Pi[3 * a + b]
                       : 2.0 * phi_j * si->Pi[3 * a + b] + 2.0 * phi_i * sj->Pi[3 * a + b])
                  - 4.0 * phi_i * phi_j * pen;
        }
}

/* One pair's surface term of Eq. 33 on its own: S_ij e_ij for fluids ki and
 * kj (0 or 1) with colour gradients gi, gj (3 entries), unit vector e (3
 * entries) and distance r; out (3 entries) receives S_ij e_ij, so that the
 * pair adds out W'_ij V_j / rho_i to a^s_i. */
void ora_surface_pair(const ora_params *P, int32_t ki, int32_t kj, const double *gi,
                      const double *gj, const double *e, double r, double *out)
{
    stress_t si, sj;
    surface_stress(P, gi, &si);
    surface_stress(P, gj, &sj);
    double S[9];
    surface_pair_matrix(P, ki, kj, &si, &sj, gi, gj, e, r, ora_xi(P), S);
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int b = 0; b < P->dim; ++b) s += S[3 * a + b] * e[b];
        out[a] = a < P->dim ? s : 0.0;
    }
}

/* The same pair matrix S_ij applied to any vector v (3 entries): out = S_ij v.
 * With the surface_corr reading the force loop applies the same-phase S_ij
 * to the corrected kernel gradient instead of e_ij. */
void ora_surface_pair_apply(const ora_params *P, int32_t ki, int32_t kj, const double *gi,
                            const double *gj, const double *e, double r, const double *v, double *out)
{
    stress_t si, sj;
    surface_stress(P, gi, &si);
    surface_stress(P, gj, &sj);
    double S[9];
    surface_pair_matrix(P, ki, kj, &si, &sj, gi, gj, e, r, ora_xi(P), S);
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int b = 0; b < P->dim; ++b) s += S[3 * a + b] * v[b];
        out[a] = a < P->dim ? s : 0.0;
    }
}

/* Eq. 7 (pressure) and Eq. 33 (surface tension with the projected penalty),
 * the latter divided by m_i.  ap and as receive the two accelerations. */
static void pressure_surface_acc(const ora_params *P, const state_t *S,
                                 const pairs_t *pp, const double *gradC, const double *Bk,
                                 double *ap, double *as)
{
    const int dim = P->dim;
    const double xi = ora_xi(P);
    const double c0 = P->c0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < S->n; ++i) {
        double a_p[3] = {0, 0, 0}, a_s[3] = {0, 0, 0};
        int32_t ki = S->kind[i];
        if (is_fluid(ki)) {
            const double *vi = S->vel + 3 * i;
            double rho_i = S->rho[i], p_i = pressure_of(P, S, i);
            stress_t si;
            surface_stress(P, gradC + 3 * i, &si);
            for (int64_t k = pp->row[i]; k < pp->row[i + 1]; ++k) {
                int64_t j = pp->col[k];
                int32_t kj = S->kind[j];
                const double *e = pp->e + 3 * k;
                double gradW[3] = {0, 0, 0};
                for (int d = 0; d < dim; ++d) gradW[d] = pp->dW[k] * e[d];
                double Vj = volume_of(P, S, j);
                const double *vj = S->vel + 3 * j;

                /* ---- pressure, Eqs. 7-12 ---- */
                rstate L = {rho_i, -dot3(vi, e, dim), p_i, c0};   /* Eq. 10 */
                rstate R;
                double pbar;
                if (is_fluid(kj)) {
                    double rho_j = S->rho[j], p_j = pressure_of(P, S, j);
                    R.rho = rho_j; R.U = -dot3(vj, e, dim); R.p = p_j; R.c = c0;
                    pbar = pair_pbar(rho_i, p_i, rho_j, p_j);
                } else {
                    /* reading: mirror state behind a wall moving with v_w */
                    double Uw = -dot3(vj, e, dim);
                    R.rho = rho_i; R.U = 2.0 * Uw - L.U; R.p = p_i; R.c = c0;
                    pbar = pair_pbar(rho_i, p_i, rho_i, p_i);
                }
                double Ps = riemann_Pstar(P, L, R, pbar);
                /* reading (walls): with wall_form 1 a wall pair never pulls */
                if (!is_fluid(kj) && P->wall_form == 1 && Ps < 0.0) Ps = 0.0;
                for (int d = 0; d < dim; ++d)
                    a_p[d] += -2.0 / rho_i * Ps * gradW[d] * Vj;

                /* ---- surface tension, Eq. 33 / m_i (walls excluded) ---- */
                if (!is_fluid(kj)) continue;
                stress_t sj;
                surface_stress(P, gradC + 3 * j, &sj);
                double Sij[9];
                surface_pair_matrix(P, ki, kj, &si, &sj, gradC + 3 * i, gradC + 3 * j, e, pp->r[k], xi, Sij);
                /* reading (surface_corr 1): the same-phase line takes the kernel
                 * gradient corrected by the mean of the two particles' own-fluid
                 * correction matrices (Eq. 15), so the divergence of the stress,
                 * summed over one fluid only, is first-order consistent up to the
                 * interface; the mean keeps the pair term antisymmetric */
                double gW[3] = {gradW[0], gradW[1], gradW[2]};
                if (Bk && kj == ki) {
                    for (int a = 0; a < dim; ++a) {
                        double t = 0.0;
                        for (int b = 0; b < dim; ++b)
                            t += 0.5 * (Bk[9 * i + 3 * a + b] + Bk[9 * j + 3 * a + b]) * gradW[b];
                        gW[a] = t;
                    }
                }
                for (int a = 0; a < dim; ++a) {
                    double s = 0.0;
                    for (int b = 0; b < dim; ++b) s += Sij[3 * a + b] * gW[b];
                    a_s[a] += s * Vj / rho_i;
                }
            }
        }
        for (int d = 0; d < 3; ++d) {
            ap[3 * i + d] = a_p[d];
            as[3 * i + d] = a_s[d];
        }
    }
}

/* Eq. 6: continuity with the Riemann star velocity (walls: v* = v_w) */
static void continuity_rate(const ora_params *P, const state_t *S, const pairs_t *pp,
                            double *drho)
{
    const int dim = P->dim;
    const double c0 = P->c0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < S->n; ++i) {
        double s = 0.0;
        int32_t ki = S->kind[i];
        if (is_fluid(ki)) {
            const double *vi = S->vel + 3 * i;
            double rho_i = S->rho[i], p_i = pressure_of(P, S, i);
            for (int64_t k = pp->row[i]; k < pp->row[i + 1]; ++k) {
                int64_t j = pp->col[k];
                const double *e = pp->e + 3 * k;
                const double *vj = S->vel + 3 * j;
                double vs[3] = {0, 0, 0};
                if (is_fluid(S->kind[j])) {
                    double rho_j = S->rho[j], p_j = pressure_of(P, S, j);
                    rstate L = {rho_i, -dot3(vi, e, dim), p_i, c0};
                    rstate R = {rho_j, -dot3(vj, e, dim), p_j, c0};
                    riemann_vstar(P, L, R, rho_i, vi, rho_j, vj, e, dim, vs);
                } else {
                    for (int d = 0; d < dim; ++d) vs[d] = vj[d];
                }
                double Vj = volume_of(P, S, j);
                for (int d = 0; d < dim; ++d)
                    s += (vi[d] - vs[d]) * pp->dW[k] * e[d] * Vj;
            }
            s *= 2.0 * rho_i;
        }
        drho[i] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* transport-velocity formulation (Section 3.2, Eqs. 14-15)                  */
/* ------------------------------------------------------------------------ */
/* Eq. 15: B_i = -(sum_j r_ij (x) grad_i W_ij V_j)^-1, a dim x dim matrix. */
static void correction_matrix(const ora_params *P, const state_t *S, const pairs_t *pp,
                              double *B, int own_fluid)
{
    const int dim = P->dim;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < S->n; ++i) {
        double M[9] = {0};
        for (int64_t k = pp->row[i]; k < pp->row[i + 1]; ++k) {
            int64_t j = pp->col[k];
            /* own_fluid: the sum of Eq. 15 over the neighbours of i's fluid only */
            if (own_fluid && S->kind[j] != S->kind[i]) continue;
            double Vj = volume_of(P, S, j);
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b)
                    M[3 * a + b] += (pp->r[k] * pp->e[3 * k + a])
                                    * (pp->dW[k] * pp->e[3 * k + b]) * Vj;
        }
        double inv[9] = {0};
        double det;
        if (dim == 2) {
            det = M[0] * M[4] - M[1] * M[3];
            inv[0] = M[4] / det; inv[1] = -M[1] / det;
            inv[3] = -M[3] / det; inv[4] = M[0] / det;
        } else {
            /* inverse by cofactors */
            det = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6])
                  + M[2] * (M[3] * M[7] - M[4] * M[6]);
            inv[0] = (M[4] * M[8] - M[5] * M[7]) / det;
            inv[1] = (M[2] * M[7] - M[1] * M[8]) / det;
            inv[2] = (M[1] * M[5] - M[2] * M[4]) / det;
            inv[3] = (M[5] * M[6] - M[3] * M[8]) / det;
            inv[4] = (M[0] * M[8] - M[2] * M[6]) / det;
            inv[5] = (M[2] * M[3] - M[0] * M[5]) / det;
            inv[6] = (M[3] * M[7] - M[4] * M[6]) / det;
            inv[7] = (M[1] * M[6] - M[0] * M[7]) / det;
            inv[8] = (M[0] * M[4] - M[1] * M[3]) / det;
        }
        int singular = !(fabs(det) >= 1e-3);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                B[9 * i + 3 * a + b] = singular ? (a == b && a < dim ? 1.0 : 0.0)
                                                : -inv[3 * a + b];
    }
}

/* Eq. 14 (sign reading in the header): position shift of fluid particles */
static void tvf_shift(const ora_params *P, const state_t *S, const pairs_t *pp,
                      const double *B, double *dr)
{
    const int dim = P->dim;
    const double coef = -P->tvf_alpha * P->h * P->h;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < S->n; ++i) {
        double s[3] = {0, 0, 0};
        if (is_fluid(S->kind[i])) {
            for (int64_t k = pp->row[i]; k < pp->row[i + 1]; ++k) {
                int64_t j = pp->col[k];
                const double *Bj = is_fluid(S->kind[j]) ? B + 9 * j : B + 9 * i;
                double Vj = volume_of(P, S, j);
                for (int a = 0; a < dim; ++a)
                    for (int b = 0; b < dim; ++b)
                        s[a] += (B[9 * i + 3 * a + b] + Bj[3 * a + b])
                                * pp->dW[k] * pp->e[3 * k + b] * Vj;
            }
        }
        for (int d = 0; d < 3; ++d) dr[3 * i + d] = d < dim ? coef * s[d] : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* time-step criteria (Section 3.3, Eqs. 16-18)                              */
/* ------------------------------------------------------------------------ */
static void vmax_per_phase(const state_t *S, int dim, double *vmax)
{
    vmax[0] = vmax[1] = 0.0;
    for (int64_t i = 0; i < S->n; ++i) {
        if (!is_fluid(S->kind[i])) continue;
        double v = norm3(S->vel + 3 * i, dim);
        if (v > vmax[S->kind[i]]) vmax[S->kind[i]] = v;
    }
}

static int phase_present(const state_t *S, int32_t k)
{
    for (int64_t i = 0; i < S->n; ++i) if (S->kind[i] == k) return 1;
    return 0;
}

/* Eq. 16 then Eq. 18 (terms with |v|max = 0 are infinite and dropped); the
 * factor 0.1 is the parameter cfl_ad */
double ora_dt_advection(const ora_params *P, const double *vmax, const int32_t *present)
{
    double dt = INFINITY;
    for (int k = 0; k < 2; ++k) {
        if (!present[k]) continue;
        double t = P->rho0[k] * P->h * P->h / P->eta[k];
        if (vmax[k] > 0.0 && P->h / vmax[k] < t) t = P->h / vmax[k];
        if (P->cfl_ad * t < dt) dt = P->cfl_ad * t;
    }
    return dt;
}

/* Eq. 17 then Eq. 18; the factor 0.6 is the parameter cfl_ac.  With the
 * kick-continuity-drift substep, a density-ratio-1000 interface whose step
 * is bound by the sound term is stable only below about 0.55 (2D) and 0.4
 * (3D), so such workloads pass a smaller factor. */
double ora_dt_acoustic(const ora_params *P, const double *vmax, const int32_t *present)
{
    double dt = INFINITY;
    for (int k = 0; k < 2; ++k) {
        if (!present[k]) continue;
        double t = P->h / (P->c0 + vmax[k]);
        if (P->gamma > 0.0) {
            double ts = sqrt(P->rho0[k] * P->h * P->h * P->h / (2.0 * ORA_PI * P->gamma));
            if (ts < t) t = ts;
        }
        if (P->cfl_ac * t < dt) dt = P->cfl_ac * t;
    }
    return dt;
}

/* ------------------------------------------------------------------------ */
/* exposed evaluation of all right-hand sides at one state (no integration)  */
/* ------------------------------------------------------------------------ */
int ora_forces(const ora_params *P, int64_t n, const double *pos, const double *vel,
               const double *rho, const int32_t *kind, double *gradC, double *ap,
               double *as, double *av, double *drho, double *dr)
{
    set_threads(P);
    state_t S = {n, (double *)pos, (double *)vel, (double *)rho, kind};
    pairs_t pp;
    if (pairs_build(P, n, pos, &pp) != 0) return 3;
    color_gradient(P, &S, &pp, gradC);
    double *Bk = 0;
    if (P->surface_corr == 1) {
        Bk = (double *)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
        correction_matrix(P, &S, &pp, Bk, 1);
    }
    pressure_surface_acc(P, &S, &pp, gradC, Bk, ap, as);
    free(Bk);
    viscous_acc(P, &S, &pp, av);
    continuity_rate(P, &S, &pp, drho);
    double *B = (double *)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
    correction_matrix(P, &S, &pp, B, 0);
    tvf_shift(P, &S, &pp, B, dr);
    free(B);
    pairs_free(&pp);
    return 0;
}

/* The correction matrix of Eq. 15 of every particle at one state, summed over
 * all neighbours (B, as the transport velocity uses it) and over the
 * neighbours of the particle's own fluid (Bk, the surface_corr reading); 9
 * entries each, row-major. */
int ora_correction_matrices(const ora_params *P, int64_t n, const double *pos, const double *vel,
                            const double *rho, const int32_t *kind, double *B, double *Bk)
{
    set_threads(P);
    state_t S = {n, (double *)pos, (double *)vel, (double *)rho, kind};
    pairs_t pp;
    if (pairs_build(P, n, pos, &pp) != 0) return 3;
    correction_matrix(P, &S, &pp, B, 0);
    correction_matrix(P, &S, &pp, Bk, 1);
    pairs_free(&pp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* the time loop (Section 3.3, dual-criteria time stepping)                  */
/* ------------------------------------------------------------------------ */
/* Advances n_adv advection steps in place.  Per advection step:
 *   1. dt_ad from Eq. 16/18;
 *   2. freeze the particle configuration (neighbours, r_ij, e_ij, dW/dr);
 *   3. the viscous acceleration (Eq. 13) from the velocities at this point,
 *      and the transport-velocity shift (Eqs. 14-15) added to the positions;
 *   4. acoustic substeps until the advection step is covered: dt = min(dt_ac,
 *      dt_ad - t_in); colour gradient (Eq. 22), pressure + surface + viscous
 *      acceleration, kick v, continuity (Eq. 6) with the kicked v, update rho,
 *      drift r with the kicked v.
 * gradC_out/av_out (optional) receive the last substep's colour gradient and
 * the last advection step's viscous acceleration. */
int ora_run(const ora_params *P, int64_t n, double *pos, double *vel, double *rho,
            const int32_t *kind, int64_t n_adv, ora_info *info,
            double *gradC_out, double *av_out)
{
    set_threads(P);
    const int dim = P->dim;
    state_t S = {n, pos, vel, rho, kind};
    size_t n3 = (size_t)(n > 0 ? n : 1) * 3;
    double *snap = (double *)malloc(sizeof(double) * n3);
    double *gradC = (double *)calloc(n3, sizeof(double));
    double *ap = (double *)calloc(n3, sizeof(double));
    double *as = (double *)calloc(n3, sizeof(double));
    double *av = (double *)calloc(n3, sizeof(double));
    double *drho = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *Bm = (double *)calloc(n3 * 3, sizeof(double));
    double *Bk = P->surface_corr == 1 ? (double *)calloc(n3 * 3, sizeof(double)) : 0;
    double *dr = (double *)calloc(n3, sizeof(double));
    int32_t present[2] = {phase_present(&S, 0), phase_present(&S, 1)};
    int64_t max_sub = P->max_substeps > 0 ? P->max_substeps : 1000000;
    int status = 0;
    memset(info, 0, sizeof(*info));

    for (int64_t step = 0; step < n_adv && status == 0; ++step) {
        double vmax[2];
        vmax_per_phase(&S, dim, vmax);
        double dt_ad = ora_dt_advection(P, vmax, present);
        if (!isfinite(dt_ad) || dt_ad <= 0.0) { status = 1; break; }
        info->last_dt_ad = dt_ad;

        memcpy(snap, pos, sizeof(double) * (size_t)n * 3);
        pairs_t pp;
        if (pairs_build(P, n, snap, &pp) != 0) { status = 3; break; }
        viscous_acc(P, &S, &pp, av);
        if (Bk) correction_matrix(P, &S, &pp, Bk, 1);
        if (P->tvf_alpha > 0.0) {
            correction_matrix(P, &S, &pp, Bm, 0);
            tvf_shift(P, &S, &pp, Bm, dr);
            for (int64_t i = 0; i < n; ++i)
                for (int d = 0; d < dim; ++d) pos[3 * i + d] = wrap_coord(P, d, pos[3 * i + d] + dr[3 * i + d]);
        }

        double t_in = 0.0;
        int64_t sub = 0;
        for (;;) {
            vmax_per_phase(&S, dim, vmax);
            double dt_ac = ora_dt_acoustic(P, vmax, present);
            if (!isfinite(dt_ac) || !(dt_ac > 0.0)) { status = 1; break; }
            info->last_dt_ac = dt_ac;
            double rem = dt_ad - t_in;
            int last = dt_ac >= rem;
            double dt = last ? rem : dt_ac;

            color_gradient(P, &S, &pp, gradC);
            pressure_surface_acc(P, &S, &pp, gradC, Bk, ap, as);
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) {
                if (!is_fluid(kind[i])) continue;
                for (int d = 0; d < dim; ++d)
                    vel[3 * i + d] += dt * (ap[3 * i + d] + as[3 * i + d] + av[3 * i + d]);
            }
            continuity_rate(P, &S, &pp, drho);
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) {
                if (!is_fluid(kind[i])) continue;
                rho[i] += dt * drho[i];
                for (int d = 0; d < dim; ++d) pos[3 * i + d] = wrap_coord(P, d, pos[3 * i + d] + dt * vel[3 * i + d]);
            }
            t_in += dt;
            ++sub;
            info->n_sub++;
            if (last) break;
            if (sub >= max_sub) { status = 2; break; }
        }
        pairs_free(&pp);
        for (int64_t i = 0; i < n && status == 0; ++i)
            if (is_fluid(kind[i]) && !isfinite(rho[i])) status = 1;
        if (status) break;
        info->t += dt_ad;
        info->n_adv++;
    }
    if (gradC_out) memcpy(gradC_out, gradC, sizeof(double) * (size_t)n * 3);
    if (av_out) memcpy(av_out, av, sizeof(double) * (size_t)n * 3);
    info->status = status;
    free(snap); free(gradC); free(ap); free(as); free(av); free(drho); free(Bm); free(Bk); free(dr);
    return status;
}

int32_t ora_max_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}
