// sphst_engine_impl.cuh -- EngineT<T>: device arrays, rebuild + substep
// graph, read-back.  Included once per precision.
#pragma once

#include <algorithm>
#include <cstring>
#include <vector>

#include "sphst_engine.cuh"
#include "sphst_kernels.cuh"

namespace sphst {

#define SPH_CK(call)                                              \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
    } while (0)

enum ArrayId { A_POS = 0, A_VEL, A_DRHO, A_ID, A_GRADC, A_ACCV };

// Tile classes: 0 = 3D list, 1 = 2D list, 2 = 3D cell walk, 3 = 2D cell walk.
// SPH_CLASSES(NCLS, KERN, args...) launches KERN<T, D, LIST> over the tiles of
// each non-empty class among the first NCLS (2: list classes only);
// SPH_CLASSES_F over the tiles of fluid ranks.
#define SPH_CLASSES(NCLS, KERN, ...) SPH_CLASSES_X(NCLS, KERN, sweep_args, cls_n, __VA_ARGS__)
#define SPH_CLASSES_F(NCLS, KERN, ...) SPH_CLASSES_X(NCLS, KERN, fluid_args, cls_fn, __VA_ARGS__)
#define SPH_CLASSES_X(NCLS, KERN, ARGS, CNT, ...)                                      \
    for (int k_ = 0; k_ < (NCLS); ++k_) {                                              \
        if (!CNT[k_]) continue;                                                        \
        const SweepArgs a_ = ARGS(k_);                                                 \
        const unsigned g_ = (unsigned)CNT[k_];                                         \
        switch (k_) {                                                                  \
        case 0: KERN<T, 3, true><<<g_, block, 0, stream>>>(a_, __VA_ARGS__); break;    \
        case 1: KERN<T, 2, true><<<g_, block, 0, stream>>>(a_, __VA_ARGS__); break;    \
        case 2: KERN<T, 3, false><<<g_, block, 0, stream>>>(a_, __VA_ARGS__); break;   \
        default: KERN<T, 2, false><<<g_, block, 0, stream>>>(a_, __VA_ARGS__); break;  \
        }                                                                              \
    }

// SPH_LANES / SPH_CLASSES_LX: the same for the sweeps whose list classes run
// with LN lanes per particle (L blocks per tile or per grid block).
#define SPH_LANES(KERN, D, LN, ...)                                                               \
    switch (LN) {                                                                                 \
    case 2: KERN<T, D, true, 2><<<g_ * 2, block, 0, stream>>>(a_, __VA_ARGS__); break;            \
    case 4: KERN<T, D, true, 4><<<g_ * 4, block, 0, stream>>>(a_, __VA_ARGS__); break;            \
    case 8: KERN<T, D, true, 8><<<g_ * 8, block, 0, stream>>>(a_, __VA_ARGS__); break;            \
    default: KERN<T, D, true, 1><<<g_, block, 0, stream>>>(a_, __VA_ARGS__); break;               \
    }
// the same for sweeps A, B and C with their tile mode (MODE_TILES, MODE_WORK
// for the work-list kernels of a batch, MODE_ONE for a one-case engine)
#define SPH_LANES_M(KERN, D, LN, MODE, ...)                                                             \
    switch (LN) {                                                                                       \
    case 2: KERN<T, D, true, 2, MODE><<<g_ * 2, block, 0, stream>>>(a_, __VA_ARGS__); break;            \
    case 4: KERN<T, D, true, 4, MODE><<<g_ * 4, block, 0, stream>>>(a_, __VA_ARGS__); break;            \
    case 8: KERN<T, D, true, 8, MODE><<<g_ * 8, block, 0, stream>>>(a_, __VA_ARGS__); break;            \
    default: KERN<T, D, true, 1, MODE><<<g_, block, 0, stream>>>(a_, __VA_ARGS__); break;               \
    }
#define SPH_CLASSES_LX(NCLS, KERN, LN, ARGS, CNT, GRID, ...)                           \
    for (int k_ = 0; k_ < (NCLS); ++k_) {                                              \
        if (!CNT[k_]) continue;                                                        \
        const SweepArgs a_ = ARGS(k_);                                                 \
        const unsigned g_ = (unsigned)(GRID);                                          \
        switch (k_) {                                                                  \
        case 0: SPH_LANES(KERN, 3, LN, __VA_ARGS__) break;                             \
        case 1: SPH_LANES(KERN, 2, LN, __VA_ARGS__) break;                             \
        case 2: KERN<T, 3, false><<<g_, block, 0, stream>>>(a_, __VA_ARGS__); break;   \
        default: KERN<T, 2, false><<<g_, block, 0, stream>>>(a_, __VA_ARGS__); break;  \
        }                                                                              \
    }
// SPH_CLASSES_BAND: the sweeps over a list class's band list (S, and A of
// the list classes): a few blocks per SM whose threads stride over the list
#define SPH_CLASSES_BAND(KERN, LN, ...) SPH_CLASSES_LX(2, KERN, LN, sweep_args, cls_n, band_grid(cls_n[k_], LN), __VA_ARGS__)
// SPH_CLASSES_LF: the per-substep sweeps over fluid ranks, whose blocks
// stride over the work list of active tiles in a batch (the grid is then
// capped), and which take their case's descriptor from the launch parameters
// in a one-case engine
#define SPH_CLASSES_LF(NCLS, KERN, LN, ...)                                                            \
    if (use_work) {                                                                                    \
        SPH_CLASSES_LXM(NCLS, KERN, LN, work_args, cls_fn, work_grid(cls_fn[k_]), MODE_WORK, __VA_ARGS__) \
    } else if (ncases == 1) {                                                                          \
        SPH_CLASSES_LXM(NCLS, KERN, LN, fluid_args, cls_fn, cls_fn[k_], MODE_ONE, __VA_ARGS__)           \
    } else {                                                                                           \
        SPH_CLASSES_LXM(NCLS, KERN, LN, fluid_args, cls_fn, cls_fn[k_], MODE_TILES, __VA_ARGS__)         \
    }
// the same from class K0 on
#define SPH_CLASSES_LFK(K0, NCLS, KERN, LN, ...)                                                        \
    if (use_work) {                                                                                    \
        SPH_CLASSES_LXMK(K0, NCLS, KERN, LN, work_args, cls_fn, work_grid(cls_fn[k_]), MODE_WORK, __VA_ARGS__) \
    } else if (ncases == 1) {                                                                          \
        SPH_CLASSES_LXMK(K0, NCLS, KERN, LN, fluid_args, cls_fn, cls_fn[k_], MODE_ONE, __VA_ARGS__)      \
    } else {                                                                                           \
        SPH_CLASSES_LXMK(K0, NCLS, KERN, LN, fluid_args, cls_fn, cls_fn[k_], MODE_TILES, __VA_ARGS__)    \
    }
// the cell-walk classes keep the descriptor array in a one-case engine: their
// sweep B also evaluates the surface terms, whose sums are left to the
// compiler's contraction, so only one compiled form of it may exist
#define CELL_MODE(MODE) ((MODE) == MODE_ONE ? MODE_TILES : (MODE))
#define SPH_CLASSES_LXM(NCLS, KERN, LN, ARGS, CNT, GRID, MODE, ...) SPH_CLASSES_LXMK(0, NCLS, KERN, LN, ARGS, CNT, GRID, MODE, __VA_ARGS__)
#define SPH_CLASSES_LXMK(K0, NCLS, KERN, LN, ARGS, CNT, GRID, MODE, ...)                              \
    for (int k_ = (K0); k_ < (NCLS); ++k_) {                                                              \
        if (!CNT[k_]) continue;                                                                        \
        const SweepArgs a_ = ARGS(k_);                                                                 \
        const unsigned g_ = (unsigned)(GRID);                                                          \
        switch (k_) {                                                                                  \
        case 0: SPH_LANES_M(KERN, 3, LN, MODE, __VA_ARGS__) break;                                     \
        case 1: SPH_LANES_M(KERN, 2, LN, MODE, __VA_ARGS__) break;                                     \
        case 2: KERN<T, 3, false, 1, CELL_MODE(MODE)><<<g_, block, 0, stream>>>(a_, __VA_ARGS__); break; \
        default: KERN<T, 2, false, 1, CELL_MODE(MODE)><<<g_, block, 0, stream>>>(a_, __VA_ARGS__); break;\
        }                                                                                              \
    }

template <typename T> struct EngineT : Engine {
    // particle arrays
    V4<T> *pos = nullptr, *snap = nullptr, *vel = nullptr, *vel_new = nullptr;
    V4<T> *gradC = nullptr, *acc_visc = nullptr, *acc_surf = nullptr, *bmat = nullptr;
    V4<T> *bk = nullptr;                             // own-fluid correction matrices (surface_corr)
    T *drho = nullptr, *drho_old = nullptr;        // drho_old: rebuild scratch (sorted copy)
    uint32_t *id = nullptr, *key = nullptr, *rank = nullptr, *perm = nullptr;
    uint32_t *fidx = nullptr, *fscan = nullptr;     // particle of each fluid rank; scan scratch
    // cell table + scan scratch
    uint32_t *starts = nullptr, *block_sums = nullptr;
    uint32_t *nbr = nullptr, *nbr_cnt = nullptr;   // neighbour lists (ELL per case) and counts
    V4<T> *lgeo = nullptr;                          // (e_ij, W'_ij) of each list entry (SPHST_LIST_GEO)
    uint8_t *band = nullptr;                        // interface band of the frozen configuration
    uint64_t *band_list = nullptr;                  // band particles per list class (case << 32 | index)
    uint32_t *band_count = nullptr;                 // entries of each class's band list
    int64_t band_base[2] = {0, 0};                  // first entry of each list class
    int64_t nbr_total = 0;
    bool any_list = false;
    // cases
    CaseDesc *d_desc = nullptr;
    CaseState *d_state = nullptr;
    Tile *d_tiles = nullptr, *d_ftiles = nullptr;   // tiles over particles; over fluid ranks
    // work lists of the per-substep sweeps (batches of more than one case):
    // class of each case, its fluid tiles (count, first index), the first
    // tile of each class, scan offsets, list lengths, the lists
    bool use_work = false;
    int32_t *d_cls_of = nullptr;
    uint32_t *d_ftn = nullptr, *d_woff = nullptr, *d_wcount = nullptr, *d_work = nullptr;
    int64_t *d_ft_first = nullptr, *d_cls0 = nullptr;
    int64_t work_cap = 0;                           // blocks of a work-list launch (per lane)
    int64_t sm_count = 0;                           // SMs of the device (band-list grids)
    int *d_loop_flag = nullptr;
    double *d_read = nullptr;              // read-back buffer
    double *d_diag = nullptr;              // diagnostics partials + result
    void *arena = nullptr;
    int64_t n = 0, table_total = 0, n_tiles = 0, max_case_n = 0;
    int64_t cls_b[4] = {0, 0, 0, 0}, cls_n[4] = {0, 0, 0, 0};   // tile range of each class
    int64_t cls_fb[4] = {0, 0, 0, 0}, cls_fn[4] = {0, 0, 0, 0}; // the same over fluid ranks
    int64_t n_ftiles = 0;
    int ncases = 0, block = 128, lanes = 1;
    bool any_tvf = false;
    bool any_corr = false;                          // a case takes the own-fluid surface correction
    int loop_mode = SPHST_LOOP_GRAPH;
    std::vector<CaseDesc> h_desc;
    std::vector<CaseState> h_state;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;

    EngineT() { precision = sizeof(T) == 4 ? 32 : 64; }
    ~EngineT() override {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (stream && own_stream) cudaStreamDestroy(stream);
        if (arena) cudaFree(arena);
    }

    void *dev_array(int which) override {
        switch (which) {
        case A_POS: return pos;
        case A_VEL: return vel;
        case A_DRHO: return drho;
        case A_ID: return id;
        case A_GRADC: return gradC;
        case A_ACCV: return acc_visc;
        }
        return nullptr;
    }
    CaseState *dev_state() override { return d_state; }
    int64_t begin_of(int slot) override { return h_desc[slot].p_begin; }

    int setup(const std::vector<CaseRec *> &cases, int blk, cudaStream_t user_stream) override {
        members = cases;
        ncases = (int)cases.size();
        block = blk;
        lanes = cases.empty() ? 1 : cases[0]->P.lanes;
        if (lanes != 2 && lanes != 4 && lanes != 8) lanes = 1;
        if (user_stream) {
            stream = user_stream;
        } else {
            SPH_CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
            own_stream = true;
        }
        // layout
        h_desc.resize(ncases);
        h_state.assign(ncases, CaseState{});
        n = 0;
        table_total = 0;
        n_tiles = 0;
        max_case_n = 0;
        loop_mode = SPHST_LOOP_GRAPH;
        for (int c = 0; c < ncases; ++c) {
            CaseRec *r = cases[c];
            if (!r->gridded) {
                int rc = make_grid(r);
                if (rc) return rc;
            }
            CaseDesc d = make_desc(r);
            d.p_begin = n;
            d.p_end = n + r->n;
            d.table_off = table_total;
            h_desc[c] = d;
            n += r->n;
            table_total += d.table_size;
            n_tiles += (r->n + block - 1) / block;
            n_ftiles += (r->n_fluid + block - 1) / block;
            max_case_n = std::max(max_case_n, r->n);
            any_tvf = any_tvf || d.tvf_on;
            any_corr = any_corr || d.surface_corr == 1;
            if (d.nbr_mode == 0) {
                d.nbr_base = nbr_total;
                nbr_total += (int64_t)d.nbr_k * r->n;
                any_list = true;
                h_desc[c] = d;
            }
            if (r->P.loop_mode == SPHST_LOOP_HOST) loop_mode = SPHST_LOOP_HOST;
        }
        if (any_list && n >= ((int64_t)1 << (32 - NBR_SHIFT))) {
            set_error("more than 2^26 particles in one engine: use the cell-walk neighbour mode");
            return SPHST_ERR_UNSUPPORTED;
        }
        if (n >= (int64_t)0xffffffffll || table_total + 1 >= (int64_t)0xffffffffll) {
            set_error("engine too large for 32-bit particle or cell indices");
            return SPHST_ERR_UNSUPPORTED;
        }
        // arena
        const int64_t nb = std::max(table_total + 1, n + 1) / SCAN_ITEMS + 1;   // table or particle scan
        size_t off = 0;
        auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
        const size_t nn = (size_t)std::max<int64_t>(n, 1);
        size_t o_pos = take(nn * sizeof(V4<T>)), o_snap = take(nn * sizeof(V4<T>));
        size_t o_vel = take(nn * sizeof(V4<T>)), o_veln = take(nn * sizeof(V4<T>));
        size_t o_gc = take(nn * sizeof(V4<T>)), o_av = take(nn * sizeof(V4<T>));
        size_t o_as = take(nn * sizeof(V4<T>));
        size_t o_bm = take(2 * nn * sizeof(V4<T>));
        size_t o_bk = take(any_corr ? 2 * nn * sizeof(V4<T>) : 0);
        size_t o_dr = take(nn * sizeof(T)), o_dro = take(nn * sizeof(T));
        size_t o_id = take(nn * 4), o_key = take(nn * 4), o_rank = take(nn * 4), o_perm = take(nn * 4);
        size_t o_st = take((size_t)(table_total + 1) * 4), o_bs = take((size_t)nb * 4);
        size_t o_desc = take(sizeof(CaseDesc) * ncases), o_state = take(sizeof(CaseState) * ncases);
        size_t o_tiles = take(sizeof(Tile) * (size_t)std::max<int64_t>(n_tiles, 1));
        size_t o_ftiles = take(sizeof(Tile) * (size_t)std::max<int64_t>(n_ftiles, 1));
        size_t o_fidx = take(nn * 4), o_fscan = take((nn + 1) * 4);
        const size_t nc = (size_t)std::max(ncases, 1);
        size_t o_clsof = take(nc * 4), o_ftn = take(nc * 4), o_woff = take(nc * 4), o_wcount = take(64);
        size_t o_work = take(sizeof(uint32_t) * (size_t)std::max<int64_t>(n_ftiles, 1));
        size_t o_ftfirst = take(nc * 8), o_cls0 = take(64);
        size_t o_flag = take(64);
        size_t o_read = take((size_t)std::max<int64_t>(max_case_n, 1) * 3 * sizeof(double));
        size_t o_nbr = take((size_t)std::max<int64_t>(nbr_total, 1) * 4), o_ncnt = take(nn * 4);
        size_t o_lgeo = take(SPHST_LIST_GEO ? (size_t)std::max<int64_t>(nbr_total, 1) * sizeof(V4<T>) : 0);
        size_t o_band = take(nn);
        size_t o_blist = take(nn * 8), o_bcount = take(64);
        size_t o_diag = take((size_t)(DIAG_BLOCKS + 1) * DIAG_Q * sizeof(double));
        cudaError_t e = cudaMalloc(&arena, off);
        if (e != cudaSuccess) {
            arena = nullptr;
            cudaGetLastError();
            set_error("device allocation of " + std::to_string(off) + " bytes failed");
            return SPHST_ERR_OOM;
        }
        char *b = (char *)arena;
        pos = (V4<T> *)(b + o_pos); snap = (V4<T> *)(b + o_snap);
        vel = (V4<T> *)(b + o_vel); vel_new = (V4<T> *)(b + o_veln);
        gradC = (V4<T> *)(b + o_gc); acc_visc = (V4<T> *)(b + o_av);
        acc_surf = (V4<T> *)(b + o_as); bmat = (V4<T> *)(b + o_bm);
        bk = any_corr ? (V4<T> *)(b + o_bk) : nullptr;
        drho = (T *)(b + o_dr); drho_old = (T *)(b + o_dro);
        id = (uint32_t *)(b + o_id); key = (uint32_t *)(b + o_key);
        rank = (uint32_t *)(b + o_rank); perm = (uint32_t *)(b + o_perm);
        starts = (uint32_t *)(b + o_st); block_sums = (uint32_t *)(b + o_bs);
        d_desc = (CaseDesc *)(b + o_desc); d_state = (CaseState *)(b + o_state);
        d_tiles = (Tile *)(b + o_tiles); d_loop_flag = (int *)(b + o_flag);
        d_ftiles = (Tile *)(b + o_ftiles);
        fidx = (uint32_t *)(b + o_fidx); fscan = (uint32_t *)(b + o_fscan);
        d_cls_of = (int32_t *)(b + o_clsof); d_ftn = (uint32_t *)(b + o_ftn);
        d_woff = (uint32_t *)(b + o_woff); d_wcount = (uint32_t *)(b + o_wcount);
        d_work = (uint32_t *)(b + o_work); d_ft_first = (int64_t *)(b + o_ftfirst); d_cls0 = (int64_t *)(b + o_cls0);
        d_read = (double *)(b + o_read);
        nbr = (uint32_t *)(b + o_nbr);
        nbr_cnt = (uint32_t *)(b + o_ncnt);
        lgeo = SPHST_LIST_GEO ? (V4<T> *)(b + o_lgeo) : nullptr;
        band = (uint8_t *)(b + o_band);
        band_list = (uint64_t *)(b + o_blist);
        band_count = (uint32_t *)(b + o_bcount);
        d_diag = (double *)(b + o_diag);
        SPH_CK(cudaMemsetAsync(arena, 0, off, stream));
        // tiles, grouped by class
        std::vector<Tile> tiles;
        tiles.reserve(n_tiles);
        for (int k = 0; k < 4; ++k) {
            cls_b[k] = (int64_t)tiles.size();
            for (int c = 0; c < ncases; ++c) {
                if (tile_class(h_desc[c]) != k) continue;
                for (int64_t s = h_desc[c].p_begin; s < h_desc[c].p_end; s += block)
                    tiles.push_back(Tile{c, (int32_t)std::min<int64_t>(block, h_desc[c].p_end - s), s});
            }
            cls_n[k] = (int64_t)tiles.size() - cls_b[k];
        }
        // band lists of the two list classes, one after the other
        int64_t np0 = 0;
        for (int64_t t = cls_b[0]; t < cls_b[0] + cls_n[0]; ++t) np0 += tiles[t].n;
        band_base[0] = 0;
        band_base[1] = np0;
        SPH_CK(cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, stream));
        // tiles over fluid ranks: case c's fluid particles hold the ranks
        // after those of cases 0..c-1
        std::vector<int64_t> fb(ncases + 1, 0);
        for (int c = 0; c < ncases; ++c) fb[c + 1] = fb[c] + cases[c]->n_fluid;
        std::vector<Tile> ftiles;
        ftiles.reserve(n_ftiles);
        for (int k = 0; k < 4; ++k) {
            cls_fb[k] = (int64_t)ftiles.size();
            for (int c = 0; c < ncases; ++c) {
                if (tile_class(h_desc[c]) != k) continue;
                for (int64_t s = fb[c]; s < fb[c + 1]; s += block)
                    ftiles.push_back(Tile{c, (int32_t)std::min<int64_t>(block, fb[c + 1] - s), s});
            }
            cls_fn[k] = (int64_t)ftiles.size() - cls_fb[k];
        }
        if (!ftiles.empty())
            SPH_CK(cudaMemcpyAsync(d_ftiles, ftiles.data(), sizeof(Tile) * ftiles.size(), cudaMemcpyHostToDevice, stream));
        // work lists (a batch option): the tiles of the active cases are
        // listed each substep and the sweeps' blocks stride over the list
        use_work = ncases > 1 && cases[0]->P.work_lists == 1;
        if (use_work) {
            std::vector<int32_t> cls_of(ncases);
            std::vector<uint32_t> ftn(ncases, 0);
            std::vector<int64_t> ft_first(ncases, 0), cls0(4);
            for (int c = 0; c < ncases; ++c) cls_of[c] = tile_class(h_desc[c]);
            for (int64_t t = (int64_t)ftiles.size() - 1; t >= 0; --t) {
                ftn[ftiles[t].c] += 1;
                ft_first[ftiles[t].c] = t;
            }
            for (int k = 0; k < 4; ++k) cls0[k] = cls_fb[k];
            SPH_CK(cudaMemcpyAsync(d_cls_of, cls_of.data(), 4 * ncases, cudaMemcpyHostToDevice, stream));
            SPH_CK(cudaMemcpyAsync(d_ftn, ftn.data(), 4 * ncases, cudaMemcpyHostToDevice, stream));
            SPH_CK(cudaMemcpyAsync(d_ft_first, ft_first.data(), 8 * ncases, cudaMemcpyHostToDevice, stream));
            SPH_CK(cudaMemcpyAsync(d_cls0, cls0.data(), 8 * 4, cudaMemcpyHostToDevice, stream));
            int dev = 0, sms = 0;
            SPH_CK(cudaGetDevice(&dev));
            SPH_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            work_cap = (int64_t)std::max(sms, 1) * 16;
        }
        {
            int dev = 0, sms = 0;
            SPH_CK(cudaGetDevice(&dev));
            SPH_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            sm_count = std::max(sms, 1);
        }
        SPH_CK(cudaMemcpyAsync(d_desc, h_desc.data(), sizeof(CaseDesc) * ncases, cudaMemcpyHostToDevice, stream));
        // fill each case
        for (int c = 0; c < ncases; ++c) {
            CaseRec *r = cases[c];
            const int64_t b0 = h_desc[c].p_begin;
            if (r->engine == nullptr) {
                int rc = upload_fresh(c, r);
                if (rc) return rc;
            } else {
                if (r->engine->precision != precision) {
                    set_error("precision mismatch between a case and its batch");
                    return SPHST_ERR_UNSUPPORTED;
                }
                Engine *o = r->engine;
                const int64_t ob = o->begin_of(r->slot);
                const size_t v4 = sizeof(V4<T>);
                SPH_CK(cudaMemcpyAsync(pos + b0, (V4<T> *)o->dev_array(A_POS) + ob, r->n * v4, cudaMemcpyDeviceToDevice, stream));
                SPH_CK(cudaMemcpyAsync(vel + b0, (V4<T> *)o->dev_array(A_VEL) + ob, r->n * v4, cudaMemcpyDeviceToDevice, stream));
                SPH_CK(cudaMemcpyAsync(gradC + b0, (V4<T> *)o->dev_array(A_GRADC) + ob, r->n * v4, cudaMemcpyDeviceToDevice, stream));
                SPH_CK(cudaMemcpyAsync(acc_visc + b0, (V4<T> *)o->dev_array(A_ACCV) + ob, r->n * v4, cudaMemcpyDeviceToDevice, stream));
                SPH_CK(cudaMemcpyAsync(drho + b0, (T *)o->dev_array(A_DRHO) + ob, r->n * sizeof(T), cudaMemcpyDeviceToDevice, stream));
                SPH_CK(cudaMemcpyAsync(id + b0, (uint32_t *)o->dev_array(A_ID) + ob, r->n * 4, cudaMemcpyDeviceToDevice, stream));
                SPH_CK(cudaMemcpyAsync(d_state + c, o->dev_state() + r->slot, sizeof(CaseState), cudaMemcpyDeviceToDevice, stream));
            }
        }
        SPH_CK(cudaStreamSynchronize(stream));
        SPH_CK(cudaMemcpy(h_state.data(), d_state, sizeof(CaseState) * ncases, cudaMemcpyDeviceToHost));
        if (loop_mode == SPHST_LOOP_GRAPH) {
            int rc = build_graph();
            if (rc) return rc;
        }
        return SPHST_OK;
    }

    int upload_fresh(int c, CaseRec *r) {
        const int64_t m = r->n;
        CaseState s{};
        s.present[0] = r->n_fluid_phases >= 1 && std::any_of(r->kind.begin(), r->kind.end(), [](uint8_t k) { return k == 0; });
        s.present[1] = std::any_of(r->kind.begin(), r->kind.end(), [](uint8_t k) { return k == 1; });
        SPH_CK(cudaMemcpyAsync(d_state + c, &s, sizeof(CaseState), cudaMemcpyHostToDevice, stream));
        if (m == 0) return SPHST_OK;
        double *tp = nullptr;
        const size_t bytes = (size_t)m * (3 + 3 + 1) * sizeof(double) + (size_t)m;
        SPH_CK(cudaMalloc(&tp, bytes));
        double *tpos = tp, *tvel = tp + 3 * m, *trho = tp + 6 * m;
        uint8_t *tkind = (uint8_t *)(tp + 7 * m);
        cudaError_t e = cudaMemcpyAsync(tpos, r->pos.data(), 3 * m * sizeof(double), cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tvel, r->vel.data(), 3 * m * sizeof(double), cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(trho, r->rho.data(), m * sizeof(double), cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tkind, r->kind.data(), m, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) {
            const int grid = (int)std::min<int64_t>((m + 255) / 256, 65535);
            k_init_case<T><<<grid, 256, 0, stream>>>(d_desc, c, tpos, tvel, trho, tkind, pos, vel, drho, id, d_state);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        cudaFree(tp);
        if (e != cudaSuccess) return cuda_fail(e, "upload of a case");
        return SPHST_OK;
    }

    // The surface sweep covers only the interface band, a few blocks per SM
    // at most, so it takes at least SPHST_SURFACE_MIN_LANES lanes per band
    // particle whatever `lanes` is (measured on the 3D drop: 93 -> 60 us with 2)
    int surface_lanes() const { return std::max(lanes, (int)SPHST_SURFACE_MIN_LANES); }

    static int tile_class(const CaseDesc &d) { return (d.nbr_mode == 0 ? 0 : 2) + (d.dim == 3 ? 0 : 1); }
    SweepArgs sweep_args(int k) const { return SweepArgs{d_tiles, d_desc, d_state, starts, nbr, nbr_cnt, cls_b[k]}; }
    SweepArgs fluid_args(int k) const {
        SweepArgs a{d_ftiles, d_desc, d_state, starts, nbr, nbr_cnt, cls_fb[k], fidx};
        if (ncases == 1) a.one = h_desc[0];
        return a;
    }
    // the per-substep sweeps: with work lists, class k's list and its length
    SweepArgs work_args(int k) const {
        SweepArgs a = fluid_args(k);
        if (use_work) {
            a.work = d_work;
            a.work_count = d_wcount + k;
        }
        return a;
    }
    int64_t work_grid(int64_t tiles) const { return use_work ? std::min(tiles, work_cap) : tiles; }
    // blocks (per lane) of a band-list sweep: at most one per tile, at most 8
    // blocks of all lanes per SM
    int64_t band_grid(int64_t tiles, int lanes_) const {
        return std::max<int64_t>(1, std::min<int64_t>(tiles, sm_count * 8 / std::max(lanes_, 1)));
    }
    // list the active cases' tiles (after the criterion kernel of a substep)
    void launch_work_lists() {
        if (!use_work) return;
        k_work_scan<<<1, 1024, 0, stream>>>(ncases, d_cls_of, d_ftn, d_state, d_woff, d_wcount);
        k_work_fill<<<(unsigned)((n_ftiles + 255) / 256), 256, 0, stream>>>(n_ftiles, d_ftiles, d_ft_first, d_cls0,
                                                                          d_cls_of, d_woff, d_state, d_work);
    }
    // fluid ranks of the reordered particles (after the gather)
    void launch_fluid_ranks() {
        const int64_t np1 = n + 1;
        const unsigned nbp = (unsigned)((np1 + SCAN_ITEMS - 1) / SCAN_ITEMS);
        k_fluid_flag<T><<<(unsigned)((np1 + 255) / 256), 256, 0, stream>>>(n, snap, fscan);
        k_scan_reduce<<<nbp, SCAN_T, 0, stream>>>(fscan, np1, block_sums);
        k_scan_blocks<<<1, SCAN_T, 0, stream>>>(block_sums, nbp);
        k_scan_apply<<<nbp, SCAN_T, 0, stream>>>(fscan, np1, block_sums);
        k_fluid_scatter<T><<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(n, snap, fscan, fidx, gradC, nbr_cnt);
    }
    int n_classes(int upto) const {
        int m = 0;
        for (int k = 0; k < upto; ++k) m += cls_n[k] > 0;
        return m;
    }

    // ---------------------------------------------------------- launches
    int launch_pre() {
        const int nthr = 256;
        const int cgrid = (ncases + 127) / 128;
        const int pgrid = (int)((n + nthr - 1) / nthr);
        SPH_CK(cudaMemsetAsync(starts, 0, (size_t)(table_total + 1) * 4, stream));
        k_reset_vmax<<<cgrid, 128, 0, stream>>>(ncases, d_state);
        k_vmax<T><<<(unsigned)n_tiles, block, 0, stream>>>(d_tiles, d_desc, d_state, pos, vel);
        k_adv_begin<<<cgrid, 128, 0, stream>>>(ncases, d_desc, d_state);
        k_cell_assign<T><<<(unsigned)n_tiles, block, 0, stream>>>(d_tiles, d_desc, d_state, pos, key, rank, starts);
        const int64_t ns = table_total + 1;
        const unsigned nb = (unsigned)((ns + SCAN_ITEMS - 1) / SCAN_ITEMS);
        k_scan_reduce<<<nb, SCAN_T, 0, stream>>>(starts, ns, block_sums);
        k_scan_blocks<<<1, SCAN_T, 0, stream>>>(block_sums, nb);
        k_scan_apply<<<nb, SCAN_T, 0, stream>>>(starts, ns, block_sums);
        k_scatter<<<pgrid, nthr, 0, stream>>>(n, key, rank, starts, perm);
        k_cell_sort<<<(unsigned)((table_total + nthr - 1) / nthr), nthr, 0, stream>>>(table_total, starts, id, perm);
        k_gather<T><<<pgrid, nthr, 0, stream>>>(n, perm, pos, vel, drho, id, snap, vel_new, drho_old, rank);
        k_copy_back<T><<<pgrid, nthr, 0, stream>>>(n, snap, vel_new, drho_old, rank, pos, vel, drho, id);
        launch_fluid_ranks();
        SPH_CLASSES_F(2, k_build_list, snap, nbr, nbr_cnt);
        if (SPHST_LIST_GEO) SPH_CLASSES(2, k_list_geo, snap, lgeo);
        SPH_CK(cudaMemsetAsync(band_count, 0, 2 * sizeof(uint32_t), stream));
        SPH_CLASSES_F(2, k_band, snap, band, band_list + band_base[k_], band_count + k_);
        if (any_tvf || any_corr) SPH_CLASSES_F(4, k_sweep_M, snap, drho, bmat, bk);
        SPH_CLASSES_F(4, k_sweep_V, snap, drho, vel, bmat, acc_visc, pos);
        SPH_CK(cudaGetLastError());
        return SPHST_OK;
    }

    // colour gradient: over the interface band in the list classes (zero
    // elsewhere, from the start of the advection step), with the surface
    // sweep's lanes per band particle; over every fluid particle in the
    // cell-walk classes
    void launch_colour() {
        SPH_CLASSES_BAND(k_sweep_A_band, surface_lanes(), band_list + band_base[k_], band_count + k_, snap, drho, gradC);
        SPH_CLASSES_LFK(2, 4, k_sweep_A, lanes, snap, drho, lgeo, gradC);
    }

    int launch_body(cudaGraphConditionalHandle h, int use_handle) {
        k_dt<<<1, 256, 0, stream>>>(ncases, d_desc, d_state, d_loop_flag, h, use_handle);
        launch_work_lists();
        launch_colour();
        SPH_CLASSES_BAND(k_sweep_S, surface_lanes(), band_list + band_base[k_], band_count + k_, band, snap, vel, gradC, acc_surf, bk, drho);
        SPH_CLASSES_LF(4, k_sweep_B, lanes, band, snap, vel, gradC, acc_visc, acc_surf, vel_new, lgeo, bk);
        SPH_CLASSES_LF(4, k_sweep_C, lanes, snap, vel_new, drho, vel, pos, lgeo);
        SPH_CK(cudaGetLastError());
        return SPHST_OK;
    }

    int launch_post() {
        k_adv_end<<<(ncases + 127) / 128, 128, 0, stream>>>(ncases, d_state);
        SPH_CK(cudaGetLastError());
        return SPHST_OK;
    }

    // One advection step as a graph: rebuild + set-up kernels, a while node
    // whose body is one acoustic substep (the device sets its condition), and
    // the bookkeeping kernel.
    int build_graph() {
        SPH_CK(cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle handle;
        SPH_CK(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
        SPH_CK(cudaStreamBeginCaptureToGraph(stream, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        int rc = launch_pre();
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        cudaGraph_t cap_graph;
        cudaError_t e = cudaStreamGetCaptureInfo(stream, &cs, nullptr, &cap_graph, &deps, nullptr, &ndeps);
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        if (e == cudaSuccess && rc == 0) e = cudaGraphAddNode(&cnode, cap_graph, deps, nullptr, ndeps, &cp);
        if (e == cudaSuccess && rc == 0)
            e = cudaStreamUpdateCaptureDependencies(stream, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e == cudaSuccess && rc == 0) rc = launch_post();
        cudaGraph_t g2 = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(stream, &g2);
        if (rc) return rc;
        if (e != cudaSuccess) return cuda_fail(e, "graph capture (conditional node)");
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        // body of the while node
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        SPH_CK(cudaStreamBeginCaptureToGraph(stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        rc = launch_body(handle, 1);
        e2 = cudaStreamEndCapture(stream, &body);
        if (rc) return rc;
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture (loop body)");
        SPH_CK(cudaGraphInstantiate(&exec, graph, 0));
        return SPHST_OK;
    }

    int step(int64_t n_adv) override {
        for (int64_t s = 0; s < n_adv; ++s) {
            if (loop_mode == SPHST_LOOP_GRAPH) {
                SPH_CK(cudaGraphLaunch(exec, stream));
            } else {
                int rc = launch_pre();
                if (rc) return rc;
                for (;;) {
                    rc = launch_body(0, 0);
                    if (rc) return rc;
                    int flag = 0;
                    SPH_CK(cudaMemcpyAsync(&flag, d_loop_flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
                    SPH_CK(cudaStreamSynchronize(stream));
                    if (!flag) break;
                }
                rc = launch_post();
                if (rc) return rc;
            }
        }
        SPH_CK(cudaStreamSynchronize(stream));
        return sync_state();
    }

    // one advection step, kernel by kernel, with events around each group
    int profile_step(double *kernel_ms, int64_t *launches) override {
        const int G = SPHST_PROFILE_GROUPS;
        for (int k = 0; k < G; ++k) { kernel_ms[k] = 0.0; launches[k] = 0; }
        cudaEvent_t ev[2];
        SPH_CK(cudaEventCreate(&ev[0]));
        SPH_CK(cudaEventCreate(&ev[1]));
        int rc = SPHST_OK;
        auto timed = [&](int group, int nl, auto &&fn) {
            if (rc) return;
            cudaEventRecord(ev[0], stream);
            fn();
            cudaEventRecord(ev[1], stream);
            cudaError_t e = cudaEventSynchronize(ev[1]);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) { rc = cuda_fail(e, "profiled launch"); return; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            kernel_ms[group] += ms;
            launches[group] += nl;
        };
        const int nthr = 256;
        const int cgrid = (ncases + 127) / 128;
        const int pgrid = (int)((n + nthr - 1) / nthr);
        const int64_t ns = table_total + 1;
        const unsigned nb = (unsigned)((ns + SCAN_ITEMS - 1) / SCAN_ITEMS);
        const int ncls = n_classes(4), nlist = n_classes(2);
        timed(1, 3, [&] {
            k_reset_vmax<<<cgrid, 128, 0, stream>>>(ncases, d_state);
            k_vmax<T><<<(unsigned)n_tiles, block, 0, stream>>>(d_tiles, d_desc, d_state, pos, vel);
            k_adv_begin<<<cgrid, 128, 0, stream>>>(ncases, d_desc, d_state);
        });
        timed(0, 8, [&] {
            cudaMemsetAsync(starts, 0, (size_t)ns * 4, stream);
            k_cell_assign<T><<<(unsigned)n_tiles, block, 0, stream>>>(d_tiles, d_desc, d_state, pos, key, rank, starts);
            k_scan_reduce<<<nb, SCAN_T, 0, stream>>>(starts, ns, block_sums);
            k_scan_blocks<<<1, SCAN_T, 0, stream>>>(block_sums, nb);
            k_scan_apply<<<nb, SCAN_T, 0, stream>>>(starts, ns, block_sums);
            k_scatter<<<pgrid, nthr, 0, stream>>>(n, key, rank, starts, perm);
            k_cell_sort<<<(unsigned)((table_total + nthr - 1) / nthr), nthr, 0, stream>>>(table_total, starts, id, perm);
            k_gather<T><<<pgrid, nthr, 0, stream>>>(n, perm, pos, vel, drho, id, snap, vel_new, drho_old, rank);
            k_copy_back<T><<<pgrid, nthr, 0, stream>>>(n, snap, vel_new, drho_old, rank, pos, vel, drho, id);
        });
        timed(0, 5, [&] { launch_fluid_ranks(); });
        timed(0, (SPHST_LIST_GEO ? 3 : 2) * nlist, [&] {
            SPH_CLASSES_F(2, k_build_list, snap, nbr, nbr_cnt);
            if (SPHST_LIST_GEO) SPH_CLASSES(2, k_list_geo, snap, lgeo);
            cudaMemsetAsync(band_count, 0, 2 * sizeof(uint32_t), stream);
            SPH_CLASSES_F(2, k_band, snap, band, band_list + band_base[k_], band_count + k_);
        });
        timed(1, (any_tvf || any_corr) ? 2 * ncls : ncls, [&] {
            if (any_tvf || any_corr) SPH_CLASSES_F(4, k_sweep_M, snap, drho, bmat, bk);
            SPH_CLASSES_F(4, k_sweep_V, snap, drho, vel, bmat, acc_visc, pos);
        });
        for (;;) {
            timed(2, use_work ? 3 : 1, [&] {
                k_dt<<<1, 256, 0, stream>>>(ncases, d_desc, d_state, d_loop_flag, 0, 0);
                launch_work_lists();
            });
            timed(3, ncls, [&] { launch_colour(); });
            timed(6, nlist, [&] {
                SPH_CLASSES_BAND(k_sweep_S, surface_lanes(), band_list + band_base[k_], band_count + k_, band, snap, vel, gradC, acc_surf, bk, drho);
            });
            timed(4, ncls, [&] { SPH_CLASSES_LF(4, k_sweep_B, lanes, band, snap, vel, gradC, acc_visc, acc_surf, vel_new, lgeo, bk); });
            timed(5, ncls, [&] { SPH_CLASSES_LF(4, k_sweep_C, lanes, snap, vel_new, drho, vel, pos, lgeo); });
            if (rc) break;
            int flag = 0;
            cudaError_t e = cudaMemcpy(&flag, d_loop_flag, sizeof(int), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) { rc = cuda_fail(e, "loop flag"); break; }
            if (!flag) break;
        }
        if (!rc) rc = launch_post();
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        if (rc) return rc;
        SPH_CK(cudaStreamSynchronize(stream));
        return sync_state();
    }

    int sync_state() override {
        SPH_CK(cudaMemcpyAsync(h_state.data(), d_state, sizeof(CaseState) * ncases, cudaMemcpyDeviceToHost, stream));
        SPH_CK(cudaStreamSynchronize(stream));
        for (int c = 0; c < ncases; ++c) {
            CaseRec *r = members[c];
            if (!r || r->engine != this || r->slot != c) continue;
            const CaseState &s = h_state[c];
            r->info.n_adv = s.n_adv;
            r->info.n_sub = s.n_sub;
            r->info.t = s.t;
            r->info.last_dt_ad = s.dt_ad;
            r->info.last_dt_ac = s.last_dt_ac;
            r->info.status = map_status(s.status);
        }
        return SPHST_OK;
    }

    int read_field(int slot, int field, double *host) override {
        const CaseDesc &d = h_desc[slot];
        const int64_t m = d.p_end - d.p_begin;
        if (m == 0) return SPHST_OK;
        const int grid = (int)std::min<int64_t>((m + 255) / 256, 65535);
        k_read_field<T><<<grid, 256, 0, stream>>>(d_desc, slot, field, pos, vel, drho, gradC, acc_visc, id, d_read);
        SPH_CK(cudaGetLastError());
        const int w = (field == 0 || field == 1 || field == 5 || field == 6) ? d.dim : 1;
        SPH_CK(cudaMemcpyAsync(host, d_read, (size_t)m * w * sizeof(double), cudaMemcpyDeviceToHost, stream));
        SPH_CK(cudaStreamSynchronize(stream));
        return SPHST_OK;
    }

    int diagnose(int slot, const double *center, double r_in, double r_out, double *q) override {
        const CaseDesc &d = h_desc[slot];
        const int64_t m = d.p_end - d.p_begin;
        const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, DIAG_BLOCKS));
        double *res = d_diag + (size_t)DIAG_BLOCKS * DIAG_Q;
        const double rin2 = r_in > 0.0 ? r_in * r_in : 0.0;
        const double rout2 = r_out * r_out;
        k_diag_partial<T><<<nb, 256, 0, stream>>>(d_desc, slot, pos, vel, drho, center[0], center[1], center[2],
                                                  rin2, rout2, d_diag);
        k_diag_final<<<1, 32, 0, stream>>>(d_diag, nb, res);
        SPH_CK(cudaGetLastError());
        SPH_CK(cudaMemcpyAsync(q, res, DIAG_Q * sizeof(double), cudaMemcpyDeviceToHost, stream));
        SPH_CK(cudaStreamSynchronize(stream));
        return SPHST_OK;
    }

    int debug_keys(int slot, uint64_t *keys, int64_t *ids) override {
        const CaseDesc &d = h_desc[slot];
        const int64_t m = d.p_end - d.p_begin;
        if (m == 0) return SPHST_OK;
        unsigned long long *dk = (unsigned long long *)d_read;
        long long *di = (long long *)(d_read + m);
        const int grid = (int)std::min<int64_t>((m + 255) / 256, 65535);
        k_debug_keys<T><<<grid, 256, 0, stream>>>(d_desc, slot, snap, id, dk, di);
        SPH_CK(cudaGetLastError());
        SPH_CK(cudaMemcpyAsync(keys, dk, m * 8, cudaMemcpyDeviceToHost, stream));
        SPH_CK(cudaMemcpyAsync(ids, di, m * 8, cudaMemcpyDeviceToHost, stream));
        SPH_CK(cudaStreamSynchronize(stream));
        return SPHST_OK;
    }

    int debug_counts(int slot, int32_t *counts) override {
        const CaseDesc &d = h_desc[slot];
        const int64_t m = d.p_end - d.p_begin;
        if (m == 0) return SPHST_OK;
        int *dc = (int *)d_read;
        k_debug_counts<T><<<(unsigned)((m + 127) / 128), 128, 0, stream>>>(d_desc, slot, starts, snap, id, dc);
        SPH_CK(cudaGetLastError());
        SPH_CK(cudaMemcpyAsync(counts, dc, m * 4, cudaMemcpyDeviceToHost, stream));
        SPH_CK(cudaStreamSynchronize(stream));
        return SPHST_OK;
    }
};

}  // namespace sphst
