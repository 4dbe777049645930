// sphst_noalloc.cu -- the cell-order computation of the rebuild (Morton keys,
// counting sort, per-cell ordering by insertion index) for callers that
// cannot allocate device memory.
//
// Who needs it: code inside a framework that owns every device allocation
// through its own memory pool (a stray cudaMalloc would bypass the pool's
// accounting and can fail once the pool has reserved the memory), and
// real-time or embedded callers that must not allocate after start-up,
// because an allocation can block or fail at an unpredictable moment.  They
// hand in device buffers for the input positions and the outputs; every
// intermediate array lives in the fixed-size array below (about 10.5 MB),
// which each GPU that loads the library keeps until the process exits.
// Calls share that array: two calls that overlap on the GPU (other streams,
// other threads) race and both give wrong results.
//
// Work is bounded for any accepted input: a cell may hold at most
// NA_MAX_PER_CELL particles (a coarse grid that puts more into one cell is
// rejected), and each particle finds its place inside its cell by one
// parallel count over that cell, so no thread does more than
// NA_MAX_PER_CELL steps.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "sphst_engine.cuh"
#include "sphst_kernels.cuh"

namespace sphst {
namespace {

constexpr int64_t NA_MAX_PARTICLES = int64_t(1) << 19;   // 524,288
constexpr int64_t NA_MAX_CELLS = int64_t(1) << 20;       // Morton table entries
constexpr uint32_t NA_MAX_PER_CELL = 256;                 // particles in one cell
// largest cell count per axis: 2^10 in 3D and 2^15 in 2D keep the Morton
// code within 30 bits
constexpr int32_t NA_MAX_NCELL_3D = 1 << 10;
constexpr int32_t NA_MAX_NCELL_2D = 1 << 15;
// status bits of the flag word
constexpr uint32_t NA_FLAG_DOMAIN = 1u;     // a particle was clamped into the grid
constexpr uint32_t NA_FLAG_CROWDED = 2u;    // a cell holds more than NA_MAX_PER_CELL
constexpr int64_t NA_BLOCKS = (NA_MAX_CELLS + 1 + SCAN_ITEMS - 1) / SCAN_ITEMS;
// counts/starts, scan block sums, keys, ranks (re-used for the final order),
// permutation, a status word
constexpr int64_t NA_WORDS = (NA_MAX_CELLS + 1) + NA_BLOCKS + 3 * NA_MAX_PARTICLES + 64;

static __device__ __align__(256) uint32_t g_noalloc_scratch[NA_WORDS];

struct Scratch {
    uint32_t *counts, *block_sums, *keys, *ranks, *perm, *flag;
};

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_setup_mutex;
uint32_t *g_base[NA_MAX_DEVICES] = {nullptr};

// The array's address on the current device (looked up once per device; in
// host code the symbol itself is only a host-side stand-in).
int scratch_on_current_device(Scratch *s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        set_error("device index beyond the supported range");
        return SPHST_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_base[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the fixed scratch array");
        g_base[dev] = (uint32_t *)p;
    }
    uint32_t *b = g_base[dev];
    s->counts = b;
    s->block_sums = b + (NA_MAX_CELLS + 1);
    s->keys = s->block_sums + NA_BLOCKS;
    s->ranks = s->keys + NA_MAX_PARTICLES;
    s->perm = s->ranks + NA_MAX_PARTICLES;
    s->flag = s->perm + NA_MAX_PARTICLES;
    return SPHST_OK;
}

struct Grid {
    double origin[3];
    double cs;
    int32_t ncell[3];
};

__global__ void na_zero(uint32_t *counts, int64_t m, uint32_t *flag) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        counts[k] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) *flag = 0u;
}

// cell of every particle with the key definition of the rebuild:
// floor((x - origin) / cs) in FP64, Morton interleave, histogram + rank
template <int D>
__global__ void na_keys(int64_t n, const double *pos, Grid g, uint32_t *counts, uint32_t *keys,
                        uint32_t *ranks, uint32_t *flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cc[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        double f = floor(__ddiv_rn(__dsub_rn(pos[3 * i + a], g.origin[a]), g.cs));
        if (!(f >= 0.0 && f < (double)g.ncell[a])) {
            atomicOr(flag, NA_FLAG_DOMAIN);
            f = f < 0.0 || f != f ? 0.0 : (double)(g.ncell[a] - 1);
        }
        cc[a] = (int)f;
    }
    const uint32_t k = morton<D>(cc[0], cc[1], cc[2]);
    keys[i] = k;
    ranks[i] = atomicAdd(counts + k, 1u);
}

__global__ void na_scatter(int64_t n, const uint32_t *keys, const uint32_t *ranks,
                           const uint32_t *starts, uint32_t *perm) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    perm[starts[keys[i]] + ranks[i]] = (uint32_t)i;
}

// inside each cell, ascending insertion index (the input order): particle
// i's place in its cell is the number of the cell's particles with a smaller
// index.  The scatter left each cell's particles in arbitrary order in perm;
// every thread counts over its own cell (at most NA_MAX_PER_CELL entries),
// so the work is bounded and no thread waits on another.
__global__ void na_cell_rank(int64_t n, const uint32_t *keys, const uint32_t *starts,
                             const uint32_t *perm, uint32_t *order, uint32_t *flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = keys[i];
    const uint32_t b = starts[k], e = starts[k + 1];
    if (e - b > NA_MAX_PER_CELL) {
        atomicOr(flag, NA_FLAG_CROWDED);
        return;
    }
    uint32_t below = 0;
    for (uint32_t m = b; m < e; ++m) below += perm[m] < (uint32_t)i ? 1u : 0u;
    order[b + below] = (uint32_t)i;
}

// outputs in canonical order; nothing is written when a cell was crowded
// (its order entries were not filled)
__global__ void na_output(int64_t n, const uint32_t *order, const uint32_t *keys, const uint32_t *flag,
                          unsigned long long *keys_out, long long *order_out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n || (*flag & NA_FLAG_CROWDED)) return;
    const uint32_t i = order[k];
    order_out[k] = (long long)i;
    keys_out[k] = keys[i];
}

}  // namespace
}  // namespace sphst

using namespace sphst;

extern "C" int sphst_cell_order_noalloc(int32_t dim, int64_t n, const double *pos_dev,
                                        const double *origin3, double cell_size,
                                        const int32_t *ncell3, uint64_t *keys_dev,
                                        int64_t *order_dev, void *cuda_stream) {
    if ((dim != 2 && dim != 3) || n < 0 || !origin3 || !ncell3 || !(cell_size > 0.0)) {
        set_error("dim must be 2 or 3, n >= 0, origin and ncell given, cell_size > 0");
        return SPHST_ERR_INVALID_ARG;
    }
    if (n > 0 && (!pos_dev || !keys_dev || !order_dev)) {
        set_error("NULL device buffer");
        return SPHST_ERR_INVALID_ARG;
    }
    if (n > NA_MAX_PARTICLES) {
        set_error("n exceeds the fixed scratch limit of " + std::to_string(NA_MAX_PARTICLES) + " particles");
        return SPHST_ERR_INVALID_ARG;
    }
    // per-axis limits first, so that the bit count below stays small
    const int32_t ncell_max = dim == 3 ? NA_MAX_NCELL_3D : NA_MAX_NCELL_2D;
    for (int a = 0; a < dim; ++a) {
        if (ncell3[a] < 1 || ncell3[a] > ncell_max) {
            set_error("ncell must be between 1 and " + std::to_string(ncell_max) + " per axis in " +
                      std::to_string(dim) + "D");
            return SPHST_ERR_INVALID_ARG;
        }
    }
    int bits = 0;
    for (int a = 0; a < dim; ++a)
        while (bits < 15 && (1 << bits) < ncell3[a]) ++bits;
    if (((int64_t)1 << (dim * bits)) > NA_MAX_CELLS) {
        set_error("cell table exceeds the fixed scratch limit of " + std::to_string(NA_MAX_CELLS) + " Morton cells");
        return SPHST_ERR_INVALID_ARG;
    }
    if (n == 0) return SPHST_OK;
    Scratch s;
    int rc = scratch_on_current_device(&s);
    if (rc) return rc;
    const int64_t table = (int64_t)1 << (dim * bits);
    const int64_t ns = table + 1;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Grid g;
    for (int a = 0; a < 3; ++a) {
        g.origin[a] = a < dim ? origin3[a] : 0.0;
        g.ncell[a] = a < dim ? ncell3[a] : 1;
    }
    g.cs = cell_size;
    const int nthr = 256;
    const unsigned pgrid = (unsigned)((n + nthr - 1) / nthr);
    const unsigned nb = (unsigned)((ns + SCAN_ITEMS - 1) / SCAN_ITEMS);
    na_zero<<<(unsigned)std::min<int64_t>((ns + nthr - 1) / nthr, 4096), nthr, 0, st>>>(s.counts, ns, s.flag);
    if (dim == 3) na_keys<3><<<pgrid, nthr, 0, st>>>(n, pos_dev, g, s.counts, s.keys, s.ranks, s.flag);
    else na_keys<2><<<pgrid, nthr, 0, st>>>(n, pos_dev, g, s.counts, s.keys, s.ranks, s.flag);
    k_scan_reduce<<<nb, SCAN_T, 0, st>>>(s.counts, ns, s.block_sums);
    k_scan_blocks<<<1, SCAN_T, 0, st>>>(s.block_sums, nb);
    k_scan_apply<<<nb, SCAN_T, 0, st>>>(s.counts, ns, s.block_sums);
    na_scatter<<<pgrid, nthr, 0, st>>>(n, s.keys, s.ranks, s.counts, s.perm);
    // the ranks are not needed after the scatter: their words take the final order
    na_cell_rank<<<pgrid, nthr, 0, st>>>(n, s.keys, s.counts, s.perm, s.ranks, s.flag);
    na_output<<<pgrid, nthr, 0, st>>>(n, s.ranks, s.keys, s.flag, (unsigned long long *)keys_dev,
                                      (long long *)order_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch of the cell-order kernels");
    uint32_t flag = 0;
    e = cudaMemcpyAsync(&flag, s.flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cell-order completion");
    if (flag & NA_FLAG_CROWDED) {
        set_error("a cell holds more than " + std::to_string(NA_MAX_PER_CELL) +
                  " particles (grid too coarse for the fixed-work ordering); outputs not written");
        return SPHST_ERR_INVALID_ARG;
    }
    if (flag & NA_FLAG_DOMAIN) {
        set_error("a particle lies outside the given cell grid");
        return SPHST_ERR_DOMAIN;
    }
    return SPHST_OK;
}
