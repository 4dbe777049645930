// sphst_kernels.cuh -- CUDA kernels of the pair-sweep library (sm_103a).
//
// Rebuild (once per advection step, Section 3.3): cell assignment with Morton
// keys, a counting sort over the dense cell table (histogram by atomics,
// exclusive scan, scatter), a per-cell sort by insertion index that makes the
// order canonical, a gather of the particle arrays, the neighbour list of the
// frozen configuration and the interface band.
//
// Pair sweeps (gather-only: every particle's sum is owned by one thread, or by
// a group of 2-8 lanes that split its list and add their parts in a fixed
// order, so there are no atomics on particle data):
//   M  correction matrix B_i (Eq. 15; also over the own fluid for the
//      surface_corr reading)                             once per advection step
//   V  viscous acceleration (Eq. 13) + transport shift (Eq. 14)  once per advection step
//   A  colour gradient (Eq. 22); with the list over the interface band only
//                                                         every acoustic substep
//   S  surface stress + penalty (Eqs. 24, 26, 30, 33) of the interface band
//                                                         every substep (list cases)
//   B  pressure (Eqs. 7-12) (+ the surface terms with the cell walk) + kick
//                                                         every substep
//   C  continuity (Eq. 6) + drift                         every substep
// The list build, the band and M, V, B, C (and A with the cell walk) run
// over the fluid particles only (their ranks after each reorder); A and S of
// the list classes stride over the band list.  Time-step control (Eqs.
// 16-18) runs in FP64 in one-thread-per-case kernels.  A one-case engine
// launches A, B and C with the case's constants in the launch parameters
// (MODE_ONE); their sums are explicitly rounded, so the results do not depend
// on that choice.
#pragma once

#include <cuda_runtime.h>
#include "sphst_internal.cuh"

// Tuning switches of the pair sweeps (compile-time):
//   SPHST_LIST_LDCS    1: read neighbour-list words with evict-first loads so the
//                      streamed list does not push particle data out of L2
//   SPHST_SWEEP_MINB   >0: minimum resident 256-thread blocks per SM for the
//                      sweeps (caps registers per thread)
//   SPHST_SWEEPB_MINB  the same for sweep B alone (default 4: 64 registers)
//   SPHST_SWEEPB_MINB_ONE  the same for the FP32 sweep B of a one-case engine
//                      (default 5: 48 registers, as its per-case constants are
//                      not in registers; measured 6 (40) and 4 slower)
//   SPHST_SURFACE_MIN_LANES  least lanes per band particle of sweep S (1, 2, 4)
//   SPHST_SWEEPAS_MINB the same for sweeps A and S (default 4: with the
//                      64-register room the compiler keeps more loads in
//                      flight; measured: A 35 -> 28 us, S 93 -> 89 us on the
//                      3D drop)
//   SPHST_LIST_PREFETCH 1: load list entry k+1 while pair k is evaluated;
//                      2: entries k+1 and k+2 (measured: a general ring of
//                      2-4 entries compiles to slower sweeps)
//   SPHST_FAST_DIV     1: FP32 pair divisions through the SFU reciprocal
//   SPHST_F32X2        1: x/y components of the FP32 pair geometry and sums in
//                      packed two-lane instructions (sm_100 and later)
//   SPHST_LIST_NOALLOC 1: the list words are read without allocating L1 lines
//                      (measured +1% on the 3D drop)
//   SPHST_LIST_SORTED  1: the neighbour list holds each part in increasing j
//                      (cells by table index); 0: in the cell walk's order
#ifndef SPHST_LIST_PREFETCH
#define SPHST_LIST_PREFETCH 2
#endif
#ifndef SPHST_FAST_DIV
#define SPHST_FAST_DIV 1
#endif
#ifndef SPHST_F32X2
#define SPHST_F32X2 1
#endif
#ifndef SPHST_LIST_LDCS
#define SPHST_LIST_LDCS 1
#endif
#ifndef SPHST_SWEEP_MINB
#define SPHST_SWEEP_MINB 0
#endif
#ifndef SPHST_SURFACE_MIN_LANES
#define SPHST_SURFACE_MIN_LANES 2
#endif
#ifndef SPHST_SWEEPAS_MINB
#define SPHST_SWEEPAS_MINB 4
#endif
#ifndef SPHST_SWEEPB_MINB
#define SPHST_SWEEPB_MINB 4
#endif
#ifndef SPHST_LIST_NOALLOC
#define SPHST_LIST_NOALLOC 1
#endif
#ifndef SPHST_LIST_SORTED
#define SPHST_LIST_SORTED 1
#endif
#if SPHST_LIST_SORTED
#define LIST_WALK walk_sorted
#else
#define LIST_WALK walk
#endif
#ifndef SPHST_SWEEPB_MINB_ONE
#define SPHST_SWEEPB_MINB_ONE 5
#endif
#if SPHST_SWEEP_MINB > 0
#define SPH_SWEEP_BOUNDS __launch_bounds__(256, SPHST_SWEEP_MINB)
#else
#define SPH_SWEEP_BOUNDS __launch_bounds__(256)
#endif
// sweep B is latency-bound on neighbour gathers: capping it at 64 registers
// (4 blocks of 256 per SM) doubles its resident warps (measured 1.38 -> 0.96
// ms on 1.19M particles); the lighter sweeps A and C are faster uncapped
#if SPHST_SWEEPAS_MINB > 0
#define SPH_SWEEPAS_BOUNDS __launch_bounds__(256, SPHST_SWEEPAS_MINB)
#else
#define SPH_SWEEPAS_BOUNDS __launch_bounds__(256)
#endif
#if SPHST_SWEEPB_MINB > 0
#define SPH_SWEEPB_BOUNDS __launch_bounds__(256, SPHST_SWEEPB_MINB)
#else
#define SPH_SWEEPB_BOUNDS __launch_bounds__(256)
#endif
// sweep B of a one-case engine reads its per-case constants from the
// parameter block, which leaves it room for more resident blocks
#define SPH_SWEEPB_BOUNDS_M(T, MODE)                                                          \
    __launch_bounds__(256, (MODE) == 2 && sizeof(T) == 4 ? SPHST_SWEEPB_MINB_ONE                  \
                                                         : (SPHST_SWEEPB_MINB > 0 ? SPHST_SWEEPB_MINB : 1))

namespace sphst {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

template <typename T> __device__ __forceinline__ V4<T> ld4(const V4<T> *p) { return *p; }
template <> __device__ __forceinline__ V4<float> ld4<float>(const V4<float> *p) {
    float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return V4<float>{v.x, v.y, v.z, v.w};
}

// Divisions inside the FP32 pair loops: __fdividef (error <= 2 ulp for
// divisors below 2^126, which densities and |grad C| are) instead of the
// IEEE sequence; FP64 keeps IEEE division.  1/sqrt likewise.
__device__ __forceinline__ float div_fast(float a, float b) {
#if SPHST_FAST_DIV
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
__device__ __forceinline__ double div_fast(double a, double b) { return a / b; }
__device__ __forceinline__ float rsqrt_fast(float x) {
#if SPHST_FAST_DIV
    return rsqrtf(x);
#else
    return 1.0f / sqrtf(x);
#endif
}
__device__ __forceinline__ double rsqrt_fast(double x) { return 1.0 / sqrt(x); }

// b - 1 as a floating-point value for a 2-bit field b (0..2), without an
// integer conversion: the bit pattern 2^23 + b (2^52 + b) is exact and the
// subtraction of 2^23 + 1 (2^52 + 1) is exact too
__device__ __forceinline__ float code_off(uint32_t b, float) {
    return __fsub_rn(__uint_as_float(0x4B000000u | b), 8388609.0f);
}
__device__ __forceinline__ double code_off(uint32_t b, double) {
    return __dsub_rn(__longlong_as_double(0x4330000000000000ll | (long long)b), 4503599627370497.0);
}

// Two-lane (x, y) arithmetic, each lane rounded once: packed FP32
// instructions for float, scalar operations for double.
template <typename T> struct L2 { T x, y; };
template <typename T> __device__ __forceinline__ L2<T> l2(T x, T y) { return L2<T>{x, y}; }
__device__ __forceinline__ L2<float> fma2(L2<float> a, L2<float> b, L2<float> c) {
#if SPHST_F32X2
    const float2 r = __ffma2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y), make_float2(c.x, c.y));
    return L2<float>{r.x, r.y};
#else
    return L2<float>{__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y)};
#endif
}
__device__ __forceinline__ L2<float> add2(L2<float> a, L2<float> b) {
#if SPHST_F32X2
    const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
    return L2<float>{r.x, r.y};
#else
    return L2<float>{__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)};
#endif
}
__device__ __forceinline__ L2<float> mul2(L2<float> a, L2<float> b) {
#if SPHST_F32X2
    const float2 r = __fmul2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
    return L2<float>{r.x, r.y};
#else
    return L2<float>{__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)};
#endif
}
__device__ __forceinline__ L2<double> fma2(L2<double> a, L2<double> b, L2<double> c) {
    return L2<double>{__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y)};
}
__device__ __forceinline__ L2<double> add2(L2<double> a, L2<double> b) {
    return L2<double>{__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)};
}
__device__ __forceinline__ L2<double> mul2(L2<double> a, L2<double> b) {
    return L2<double>{__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)};
}
// 1 - b for the 2-bit offset fields (bx, by), exactly: -(2^23 + b) + (2^23 + 1)
__device__ __forceinline__ L2<float> neg_code_off2(uint32_t bx, uint32_t by, float) {
    return add2(l2(__uint_as_float(0xCB000000u | bx), __uint_as_float(0xCB000000u | by)),
                l2(8388609.0f, 8388609.0f));
}
__device__ __forceinline__ L2<double> neg_code_off2(uint32_t bx, uint32_t by, double) {
    return add2(l2(__longlong_as_double((long long)(0xC330000000000000ull | bx)),
                   __longlong_as_double((long long)(0xC330000000000000ull | by))),
                l2(4503599627370497.0, 4503599627370497.0));
}

// a ? x1 : x0 for the two fluid phases' constants (no indexed loads)
template <typename T> __device__ __forceinline__ T sel(uint32_t k, T x0, T x1) { return k ? x1 : x0; }

// A list word of the per-substep walks.  The list is streamed once per sweep
// while the neighbour records it points to are gathered ~80 times; its words
// are read without allocating L1 lines (SPHST_LIST_NOALLOC), so they take none
// from the gathered data (else as evict-first loads).
__device__ __forceinline__ uint32_t ld_list_walk(const uint32_t *p) {
#if SPHST_LIST_NOALLOC
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
#else
    return __ldcs(p);
#endif
}

__device__ __forceinline__ uint32_t ld_list(const uint32_t *p) {
#if SPHST_LIST_LDCS
    return __ldcs(p);
#else
    return __ldg(p);
#endif
}

__device__ __forceinline__ double bits_to_d(unsigned long long b) { return __longlong_as_double((long long)b); }

// explicitly rounded operations for the pair geometry, so that the cell walk
// and the neighbour list produce bitwise-identical r_ij and r^2 for a pair
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
template <typename T, int D> __device__ __forceinline__ T norm2(T x, T y, T z) {
    return D == 3 ? fma_rn(x, x, fma_rn(y, y, mul_rn(z, z))) : fma_rn(x, x, mul_rn(y, y));
}

// |v|^2 in FP64 with a fixed operation order and no contraction
template <typename T> __device__ __forceinline__ double speed2(const V4<T> &v, int dim) {
    double x = (double)v.x, y = (double)v.y, z = (double)v.z;
    double s = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
    if (dim == 3) s = __dadd_rn(s, __dmul_rn(z, z));
    return s;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Eq. 11 dissipation limiter, branch-free: min(max(k dU w, lo), hi) with the
// case's (k, lo, hi) = (3 / c0, 0, 1) for the density reading and the printed
// form, (0, 1, 1) for beta = 1 and (0, 0, 0) for beta = 0; w = 1, or for the
// printed form (P_L + P_R)/(rho_L + rho_R) of the pair
__device__ __forceinline__ float clamp_lh(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }
__device__ __forceinline__ double clamp_lh(double x, double lo, double hi) { return fmin(fmax(x, lo), hi); }
template <typename T> struct Limiter {
    T k, lo, hi;
    bool printed;
    __device__ __forceinline__ Limiter(const CasePhys<T> &cp, int mode)
        : k(cp.beta_k), lo(cp.beta_lo), hi(cp.beta_hi), printed(mode == 3) {}
    __device__ __forceinline__ T operator()(T dU, T psum, T rhosum) const {
        const T x = printed ? k * dU * div_fast(psum, rhosum) : k * dU;
        return clamp_lh(x, lo, hi);
    }
};

// Neighbour cell index along axis a: wrapped on a periodic axis (the cells
// tile the period exactly, so the cell at -1 is the last one and lies one
// cell width before cell 0); false when it falls off a non-periodic axis.
__device__ __forceinline__ bool wrap_cell(const CaseDesc &d, int a, int &c) {
    if (c >= 0 && c < d.ncell[a]) return true;
    if (!((d.periodic >> a) & 1)) return false;
    c += c < 0 ? d.ncell[a] : -d.ncell[a];
    return true;
}

// --------------------------------------------------------------- cell walk
// Calls f(j, snap_j, r_ij vector, r^2) for every j != i with 0 < r_ij < 2h in
// the 3^D cells around i's cell.  r_ij = s_i - s_j - o cs, where o is the
// neighbour cell's offset, because both offsets are taken from their own
// cell origins.  Returns true when a coincident particle was met.
template <typename T, int D, typename F>
__device__ __forceinline__ bool walk(const CaseDesc &d, const CasePhys<T> &cp,
                                     const uint32_t *__restrict__ starts,
                                     const V4<T> *__restrict__ snap, int64_t i,
                                     const V4<T> &si, uint32_t pki, F &&f) {
    const int cx = cell_x<D>(pki), cy = cell_y<D>(pki), cz = cell_z<D>(pki);
    const uint32_t toff = (uint32_t)d.table_off;
    const T cs = cp.cs, R2 = cp.four_h2;
    bool coincident = false;
    for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz) {
        int nz = cz + oz;
        if (D == 3 && !wrap_cell(d, 2, nz)) continue;
        const T sz = D == 3 ? sub_rn(si.z, mul_rn(T(oz), cs)) : T(0);
        for (int oy = -1; oy <= 1; ++oy) {
            int ny = cy + oy;
            if (!wrap_cell(d, 1, ny)) continue;
            const T sy = sub_rn(si.y, mul_rn(T(oy), cs));
            for (int ox = -1; ox <= 1; ++ox) {
                int nx = cx + ox;
                if (!wrap_cell(d, 0, nx)) continue;
                const T sx = sub_rn(si.x, mul_rn(T(ox), cs));
                const uint32_t m = toff + morton<D>(nx, ny, nz);
                const uint32_t b = __ldg(starts + m), e = __ldg(starts + m + 1);
                for (uint32_t j = b; j < e; ++j) {
                    const V4<T> sj = ld4(snap + j);
                    const T rx = sub_rn(sx, sj.x), ry = sub_rn(sy, sj.y);
                    const T rz = D == 3 ? sub_rn(sz, sj.z) : T(0);
                    const T r2 = norm2<T, D>(rx, ry, rz);
                    if (r2 < R2 && j != (uint32_t)i) {
                        if (r2 > T(0)) f(j, sj, rx, ry, rz, r2);
                        else coincident = true;
                    }
                }
            }
        }
    }
    return coincident;
}

// Neighbour list of the frozen configuration (ELL layout per case: entry k of
// particle i at nbr[nbr_base + k * n_case + (i - p_begin)], so a warp's 32
// lanes read 32 consecutive words).  An entry is j << 6 | cell code, the code
// holding (o + 1) per axis in 2 bits, o the neighbour cell's offset.  Each
// list holds the neighbours of the other fluid phase first, then the rest,
// each part in increasing j (SPHST_LIST_SORTED; else in cell-walk order);
// cnt[i] = count | (other-phase count << 16),
// so the colour-gradient sweep reads only the first part.
constexpr uint32_t NBR_SHIFT = 6;
constexpr uint32_t CNT_MASK = 0xffffu;
enum NbrPart { PART_ALL = 0, PART_OTHER = 1 };
template <int D>
__device__ __forceinline__ uint32_t cell_code(int ox, int oy, int oz) {
    return (uint32_t)(ox + 1) | ((uint32_t)(oy + 1) << 2) | (D == 3 ? ((uint32_t)(oz + 1) << 4) : 0u);
}

// The same neighbours as walk(), visited in increasing index j: the 3^D
// cells are taken in increasing order of their cell-table index (the cells
// are stored in that order, each cell's particles in index order).  The
// neighbour list is built in this order, so that the 32 lanes of a warp,
// neighbouring particles with largely the same neighbours, gather entries k
// that lie close together in memory.
template <typename T, int D, typename F>
__device__ __forceinline__ bool walk_sorted(const CaseDesc &d, const CasePhys<T> &cp,
                                            const uint32_t *__restrict__ starts,
                                            const V4<T> *__restrict__ snap, int64_t i,
                                            const V4<T> &si, uint32_t pki, F &&f) {
    constexpr int NC = D == 3 ? 27 : 9;
    const int cx = cell_x<D>(pki), cy = cell_y<D>(pki), cz = cell_z<D>(pki);
    const uint32_t toff = (uint32_t)d.table_off;
    uint32_t cell[NC];
    uint32_t code[NC];
    int nc = 0;
    for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz) {
        int nz = cz + oz;
        if (D == 3 && !wrap_cell(d, 2, nz)) continue;
        for (int oy = -1; oy <= 1; ++oy) {
            int ny = cy + oy;
            if (!wrap_cell(d, 1, ny)) continue;
            for (int ox = -1; ox <= 1; ++ox) {
                int nx = cx + ox;
                if (!wrap_cell(d, 0, nx)) continue;
                // insertion by cell-table index
                const uint32_t m = toff + morton<D>(nx, ny, nz), c = cell_code<D>(ox, oy, oz);
                int b = nc++;
                while (b > 0 && cell[b - 1] > m) { cell[b] = cell[b - 1]; code[b] = code[b - 1]; --b; }
                cell[b] = m;
                code[b] = c;
            }
        }
    }
    const T cs = cp.cs, R2 = cp.four_h2;
    bool coincident = false;
    for (int q = 0; q < nc; ++q) {
        const int ox = (int)(code[q] & 3u) - 1, oy = (int)((code[q] >> 2) & 3u) - 1, oz = (int)((code[q] >> 4) & 3u) - 1;
        const T sx = sub_rn(si.x, mul_rn(T(ox), cs)), sy = sub_rn(si.y, mul_rn(T(oy), cs));
        const T sz = D == 3 ? sub_rn(si.z, mul_rn(T(oz), cs)) : T(0);
        const uint32_t b = __ldg(starts + cell[q]), e = __ldg(starts + cell[q] + 1);
        for (uint32_t j = b; j < e; ++j) {
            const V4<T> sj = ld4(snap + j);
            const T rx = sub_rn(sx, sj.x), ry = sub_rn(sy, sj.y);
            const T rz = D == 3 ? sub_rn(sz, sj.z) : T(0);
            const T r2 = norm2<T, D>(rx, ry, rz);
            if (r2 < R2 && j != (uint32_t)i) {
                if (r2 > T(0)) f(j, sj, rx, ry, rz, r2);
                else coincident = true;
            }
        }
    }
    return coincident;
}

// With L lanes per particle, lane `sub` of the particle's group takes the
// entries sub, sub + L, sub + 2L, ... of its list.
template <int PART, typename T, int D, int L = 1, typename F>
__device__ __forceinline__ void walk_list(const CaseDesc &d, const CasePhys<T> &cp,
                                          const uint32_t *__restrict__ nbr,
                                          const uint32_t *__restrict__ cnt,
                                          const V4<T> *__restrict__ snap, int64_t i,
                                          const V4<T> &si, F &&f, uint32_t sub = 0) {
    const int64_t stride = d.p_end - d.p_begin;
    const uint32_t *p = nbr + d.nbr_base + (i - d.p_begin) + (int64_t)sub * stride;
    const uint32_t c = PART == PART_OTHER ? cnt[i] >> 16 : cnt[i] & CNT_MASK;
    const T cs = cp.cs;
#if SPHST_LIST_PREFETCH >= 2
    uint32_t next = sub < c ? ld_list_walk(p) : 0u;
    uint32_t next2 = sub + L < c ? ld_list_walk(p + L * stride) : 0u;
    p += L * stride;
#elif SPHST_LIST_PREFETCH
    uint32_t next = sub < c ? ld_list_walk(p) : 0u;
#endif
#pragma unroll 1
    for (uint32_t k = sub; k < c; k += L) {
#if SPHST_LIST_PREFETCH >= 2
        const uint32_t e = next;            // entries k + L and k + 2L in flight
        next = next2;
        p += L * stride;
        if (k + 2 * L < c) next2 = ld_list_walk(p);
#elif SPHST_LIST_PREFETCH
        const uint32_t e = next;
        p += L * stride;
        if (k + L < c) next = ld_list_walk(p);
#else
        const uint32_t e = ld_list_walk(p);
        p += L * stride;
#endif
        const uint32_t j = e >> NBR_SHIFT;
        const V4<T> sj = ld4(snap + j);
        // s_i - o cs with o in {-1, 0, 1}: o cs is exact, so the FMA rounds
        // once, exactly like the cell walk's subtraction
        const T rx = sub_rn(fma_rn(-code_off(e & 3u, T()), cs, si.x), sj.x);
        const T ry = sub_rn(fma_rn(-code_off((e >> 2) & 3u, T()), cs, si.y), sj.y);
        T rz = T(0);
        if (D == 3) rz = sub_rn(fma_rn(-code_off((e >> 4) & 3u, T()), cs, si.z), sj.z);
        const T r2 = norm2<T, D>(rx, ry, rz);
        f(j, sj, rx, ry, rz, r2);
    }
}

// The list walk with one more per-neighbour array: f(j, s_j, aux_j, r_ij, r^2).
template <typename T, int D, int L = 1, typename F>
__device__ __forceinline__ void walk_list_aux(const CaseDesc &d, const CasePhys<T> &cp,
                                              const uint32_t *__restrict__ nbr,
                                              const uint32_t *__restrict__ cnt,
                                              const V4<T> *__restrict__ snap,
                                              const V4<T> *__restrict__ aux, int64_t i,
                                              const V4<T> &si, F &&f, uint32_t sub = 0) {
    const int64_t stride = d.p_end - d.p_begin;
    const uint32_t *p = nbr + d.nbr_base + (i - d.p_begin) + (int64_t)sub * stride;
    const uint32_t c = cnt[i] & CNT_MASK;
    const T cs = cp.cs;
    const auto pair = [&](uint32_t e, const V4<T> &sj, const V4<T> &aj) {
        // (s_i - o cs) - s_j per axis, each step rounded once as in the cell walk
        const L2<T> t = fma2(neg_code_off2(e & 3u, (e >> 2) & 3u, T()), l2(cs, cs), l2(si.x, si.y));
        const L2<T> rxy = fma2(l2(sj.x, sj.y), l2(T(-1), T(-1)), t);
        const T rx = rxy.x, ry = rxy.y;
        T rz = T(0);
        if (D == 3) rz = sub_rn(fma_rn(-code_off((e >> 4) & 3u, T()), cs, si.z), sj.z);
        f(e >> NBR_SHIFT, sj, aj, rx, ry, rz, norm2<T, D>(rx, ry, rz));
    };
#if SPHST_LIST_PREFETCH >= 2
    uint32_t next = sub < c ? ld_list_walk(p) : 0u;
    uint32_t next2 = sub + L < c ? ld_list_walk(p + L * stride) : 0u;
    p += L * stride;
#elif SPHST_LIST_PREFETCH
    uint32_t next = sub < c ? ld_list_walk(p) : 0u;
#endif
#pragma unroll 1
    for (uint32_t k = sub; k < c; k += L) {
#if SPHST_LIST_PREFETCH >= 2
        const uint32_t e = next;            // entries k + L and k + 2L in flight
        next = next2;
        p += L * stride;
        if (k + 2 * L < c) next2 = ld_list_walk(p);
#elif SPHST_LIST_PREFETCH
        const uint32_t e = next;
        p += L * stride;
        if (k + L < c) next = ld_list_walk(p);
#else
        const uint32_t e = ld_list_walk(p);
        p += L * stride;
#endif
        const uint32_t j = e >> NBR_SHIFT;
        pair(e, ld4(snap + j), ld4(aux + j));
    }
}

// neighbours of i with aux[j] loaded for f(j, s_j, aux_j, r_ij, r^2), from the
// list or the cell walk
template <bool LIST, typename T, int D, int L = 1, typename F>
__device__ __forceinline__ bool neighbors_aux(const CaseDesc &d, const CasePhys<T> &cp,
                                              const uint32_t *starts, const uint32_t *nbr,
                                              const uint32_t *cnt, const V4<T> *snap, const V4<T> *aux,
                                              int64_t i, const V4<T> &si, uint32_t pki, F &&f,
                                              uint32_t sub = 0) {
    if constexpr (LIST) {
        walk_list_aux<T, D, L>(d, cp, nbr, cnt, snap, aux, i, si, f, sub);
        return false;
    } else {
        return walk<T, D>(d, cp, starts, snap, i, si, pki,
            [&](uint32_t j, const V4<T> &sj, T rx, T ry, T rz, T r2) { f(j, sj, ld4(aux + j), rx, ry, rz, r2); });
    }
}

// neighbours of i from the list (LIST) or from the cell walk; PART_OTHER
// restricts the list to the other fluid phase (the cell walk visits all and
// the caller filters)
template <bool LIST, typename T, int D, int PART = PART_ALL, int L = 1, typename F>
__device__ __forceinline__ bool neighbors(const CaseDesc &d, const CasePhys<T> &cp,
                                          const uint32_t *starts, const uint32_t *nbr,
                                          const uint32_t *cnt, const V4<T> *snap, int64_t i,
                                          const V4<T> &si, uint32_t pki, F &&f, uint32_t sub = 0) {
    if constexpr (LIST) {
        walk_list<PART, T, D, L>(d, cp, nbr, cnt, snap, i, si, f, sub);
        return false;
    } else {
        return walk<T, D>(d, cp, starts, snap, i, si, pki, f);
    }
}

// ---- stored pair geometry (SPHST_LIST_GEO): entry k of particle i holds
// (e_ij, W'_ij) of the frozen configuration at the list's own position, so
// it streams beside the list.  W' < 0 for every pair (0 < q < 2); an entry
// whose neighbour is a wall particle stores -W' instead, so the sign bit
// tells walls from fluid without reading the neighbour's packed phase.  The
// other fluid phase's entries come first (cnt >> 16 of them), so the phase
// of a fluid neighbour is known from k.
__device__ __forceinline__ bool geo_wall(float w) { return (__float_as_uint(w) >> 31) == 0u; }
__device__ __forceinline__ bool geo_wall(double w) { return __double_as_longlong(w) >= 0; }
template <typename T> __device__ __forceinline__ V4<T> ld_geo(const V4<T> *p) { return *p; }
template <> __device__ __forceinline__ V4<float> ld_geo<float>(const V4<float> *p) {
#if SPHST_LIST_LDCS
    const float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
    return V4<float>{v.x, v.y, v.z, v.w};
#else
    return ld4(p);
#endif
}

// f(other, j, G) for the list entries of i with their stored geometry G;
// other: j belongs to the other fluid phase
template <int PART, typename T, typename F>
__device__ __forceinline__ void walk_geo(const CaseDesc &d, const uint32_t *__restrict__ nbr,
                                         const uint32_t *__restrict__ cnt, const V4<T> *__restrict__ lgeo,
                                         int64_t i, F &&f) {
    const int64_t stride = d.p_end - d.p_begin;
    const int64_t off = d.nbr_base + (i - d.p_begin);
    const uint32_t *p = nbr + off;
    const V4<T> *q = lgeo + off;
    const uint32_t ci = cnt[i];
    const uint32_t c_other = ci >> 16;
    const uint32_t c = PART == PART_OTHER ? c_other : ci & CNT_MASK;
#if SPHST_LIST_PREFETCH
    uint32_t next = c ? ld_list(p) : 0u;
#endif
    V4<T> g1 = c ? ld_geo(q) : V4<T>{};
#pragma unroll 1
    for (uint32_t k = 0; k < c; ++k) {
#if SPHST_LIST_PREFETCH
        const uint32_t e = next;
        p += stride;
        if (k + 1 < c) next = ld_list(p);
#else
        const uint32_t e = ld_list(p);
        p += stride;
#endif
        const V4<T> G = g1;                       // geometry one entry ahead
        if (k + 1 < c) g1 = ld_geo(q + stride);
        q += stride;
        f(PART == PART_OTHER || k < c_other, e >> NBR_SHIFT, G);
    }
}

// f(other, j, G, aux_j): walk_geo with the neighbour's aux word
template <typename T, typename F>
__device__ __forceinline__ void walk_geo_aux(const CaseDesc &d, const uint32_t *__restrict__ nbr,
                                             const uint32_t *__restrict__ cnt, const V4<T> *__restrict__ lgeo,
                                             const V4<T> *__restrict__ aux, int64_t i, F &&f) {
    walk_geo<PART_ALL, T>(d, nbr, cnt, lgeo, i,
                          [&](bool other, uint32_t j, const V4<T> &G) { f(other, j, G, ld4(aux + j)); });
}

// Sum over the L lanes that share one particle (L = 1, 2, 4, 8; groups are
// aligned within the warp).  The butterfly gives every lane of the group the
// same value: each step adds two partial sums in an order-free way.
template <int L, typename T> __device__ __forceinline__ T group_sum(T v) {
    if constexpr (L > 1) {
        const unsigned lane = threadIdx.x & 31u;
        const unsigned mask = ((1u << L) - 1u) << (lane & ~(unsigned)(L - 1));
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) v = add_rn(v, __shfl_xor_sync(mask, v, o));
    }
    return v;
}

// kernel radial derivative and unit vector of one pair
template <typename T> struct PairGeo { T inv_r, r, dW; };
template <typename T>
__device__ __forceinline__ PairGeo<T> geo(const CasePhys<T> &cp, T r2) {
    PairGeo<T> g;
    g.inv_r = rsq(r2);
    g.r = r2 * g.inv_r;
    const T q = g.r * cp.inv_h;
    const T u = fma_rn(T(-0.5), q, T(1));
    g.dW = cp.kcoef * q * u * u * u;
    return g;
}
// the same with the kernel constants held in registers by the caller
template <typename T> struct KernelGeo {
    T inv_h, kcoef;
    __device__ __forceinline__ explicit KernelGeo(const CasePhys<T> &cp) : inv_h(cp.inv_h), kcoef(cp.kcoef) {}
    __device__ __forceinline__ PairGeo<T> operator()(T r2) const {
        PairGeo<T> g;
        g.inv_r = rsq(r2);
        g.r = r2 * g.inv_r;
        const T q = g.r * inv_h;
        const T u = fma_rn(T(-0.5), q, T(1));
        g.dW = kcoef * q * u * u * u;
        return g;
    }
};

// ================================================================ rebuild
// First placement of a freshly uploaded case: absolute FP64 positions ->
// cell coordinates (floor((x - origin)/cs) in FP64, as the key definition
// states) and offsets from the cell origin.
template <typename T, int D>
__device__ __forceinline__ void init_one(const CaseDesc &d, int c, int64_t k, const double *apos,
                                         const double *avel, const double *arho, const uint8_t *akind,
                                         V4<T> *pos, V4<T> *vel, T *drho, uint32_t *id, CaseState *st) {
    int cc[3] = {0, 0, 0};
    double off[3] = {0.0, 0.0, 0.0};
    bool bad = false;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        double rel = __dsub_rn(apos[3 * k + a], d.origin[a]);
        if ((d.periodic >> a) & 1) {
            // into the period [0, L), then the last cell also takes a
            // position that rounds onto its end
            const double L = d.period_len[a];
            rel = __dsub_rn(rel, __dmul_rn(L, floor(__ddiv_rn(rel, L))));
        }
        double f = floor(__ddiv_rn(rel, d.cs));
        if ((d.periodic >> a) & 1 && f >= (double)d.ncell[a]) f = (double)(d.ncell[a] - 1);
        if (!(f >= 0.0 && f < (double)d.ncell[a])) {
            bad = true;
            f = f < 0.0 || f != f ? 0.0 : (double)(d.ncell[a] - 1);
        }
        cc[a] = (int)f;
        off[a] = __dsub_rn(rel, __dmul_rn(f, d.cs));
    }
    if (bad) atomicCAS(&st[c].status, 0, DEV_ERR_DOMAIN);
    const uint32_t ph = akind[k];
    V4<T> p;
    p.x = (T)off[0]; p.y = (T)off[1]; p.z = (T)off[2];
    p.w = bits_w(pack_cell<D>(cc[0], cc[1], cc[2], ph), T());
    const int64_t i = d.p_begin + k;
    pos[i] = p;
    V4<T> v;
    v.x = (T)avel[3 * k]; v.y = (T)avel[3 * k + 1]; v.z = (T)avel[3 * k + 2]; v.w = T(0);
    drho[i] = ph < 2 ? (T)(arho[k] - d.rho0[ph]) : T(0);
    v.w = drho[i];                    // vel.w mirrors drho (read with the velocity)
    vel[i] = v;
    id[i] = (uint32_t)k;
}

template <typename T>
__global__ void k_init_case(const CaseDesc *__restrict__ desc, int c, const double *apos,
                            const double *avel, const double *arho, const uint8_t *akind,
                            V4<T> *pos, V4<T> *vel, T *drho, uint32_t *id, CaseState *st) {
    const CaseDesc &d = desc[c];
    const int64_t n = d.p_end - d.p_begin;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (d.dim == 3) init_one<T, 3>(d, c, k, apos, avel, arho, akind, pos, vel, drho, id, st);
        else init_one<T, 2>(d, c, k, apos, avel, arho, akind, pos, vel, drho, id, st);
    }
}

// New cell of every particle from its offset (which may have drifted out of
// the cell since the last rebuild), histogram of the cell table.
template <typename T, int D>
__device__ __forceinline__ void assign_one(const CaseDesc &d, CaseState *st, int c, int64_t i,
                                           V4<T> *pos, uint32_t *key, uint32_t *rank,
                                           uint32_t *counts) {
    const CasePhys<T> &cp = phys<T>(d);
    V4<T> p = pos[i];
    const uint32_t pk = w_bits(p.w);
    int cc[3] = {cell_x<D>(pk), cell_y<D>(pk), cell_z<D>(pk)};
    T off[3] = {p.x, p.y, p.z};
    bool bad = false;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        T f = floor(off[a] / cp.cs);
        if (!(f == f) || f > T(4096) || f < T(-4096)) { f = T(0); bad = true; }
        int nc = cc[a] + (int)f;
        if ((d.periodic >> a) & 1) {
            // the offset is taken from the unwrapped cell; the index wraps
            nc = ((nc % d.ncell[a]) + d.ncell[a]) % d.ncell[a];
        } else if (nc < 0 || nc >= d.ncell[a]) {
            bad = true;
            nc = nc < 0 ? 0 : d.ncell[a] - 1;
            f = T(nc - cc[a]);
        }
        off[a] = off[a] - f * cp.cs;
        cc[a] = nc;
    }
    if (bad) atomicCAS(&st[c].status, 0, DEV_ERR_DOMAIN);
    p.x = off[0]; p.y = off[1]; p.z = off[2];
    p.w = bits_w(pack_cell<D>(cc[0], cc[1], cc[2], phase_of(pk)), T());
    pos[i] = p;
    const uint32_t k = (uint32_t)d.table_off + morton<D>(cc[0], cc[1], cc[2]);
    key[i] = k;
    rank[i] = atomicAdd(counts + k, 1u);
}

template <typename T>
__global__ void k_cell_assign(const Tile *__restrict__ tiles, const CaseDesc *__restrict__ desc,
                              CaseState *st, V4<T> *pos, uint32_t *key, uint32_t *rank,
                              uint32_t *counts) {
    const Tile t = tiles[blockIdx.x];
    if ((int)threadIdx.x >= t.n) return;
    const CaseDesc &d = desc[t.c];
    const int64_t i = t.begin + threadIdx.x;
    if (d.dim == 3) assign_one<T, 3>(d, st, t.c, i, pos, key, rank, counts);
    else assign_one<T, 2>(d, st, t.c, i, pos, key, rank, counts);
}

// ---- exclusive scan of the cell histogram (in place, n+1 entries) ----
constexpr int SCAN_T = 1024;            // threads per block
constexpr int SCAN_ITEMS = 2 * SCAN_T;  // entries per block

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_sums[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    const uint32_t before = (w > 0 ? warp_sums[w - 1] : 0u) + x - v;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

static __global__ void k_scan_reduce(const uint32_t *data, int64_t n, uint32_t *block_sums) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_ITEMS + 2 * threadIdx.x;
    uint32_t v = 0;
    if (base < n) v += data[base];
    if (base + 1 < n) v += data[base + 1];
    uint32_t total;
    block_exclusive_scan(v, &total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

static __global__ void k_scan_blocks(uint32_t *block_sums, int64_t nb) {
    uint32_t carry = 0;
    for (int64_t base = 0; base < nb; base += SCAN_T) {
        const int64_t k = base + threadIdx.x;
        const uint32_t v = k < nb ? block_sums[k] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(v, &total);
        if (k < nb) block_sums[k] = carry + ex;
        carry += total;
    }
}

static __global__ void k_scan_apply(uint32_t *data, int64_t n, const uint32_t *block_sums) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_ITEMS + 2 * threadIdx.x;
    const uint32_t a = base < n ? data[base] : 0u;
    const uint32_t b = base + 1 < n ? data[base + 1] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(a + b, &total) + block_sums[blockIdx.x];
    if (base < n) data[base] = ex;
    if (base + 1 < n) data[base + 1] = ex + a;
}

static __global__ void k_scatter(int64_t n, const uint32_t *key, const uint32_t *rank,
                          const uint32_t *starts, uint32_t *perm) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    perm[starts[key[i]] + rank[i]] = (uint32_t)i;
}

// canonical order inside each cell: ascending insertion index
static __global__ void k_cell_sort(int64_t ncells, const uint32_t *starts, const uint32_t *id,
                            uint32_t *perm) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const uint32_t b = starts[c], e = starts[c + 1];
    if (e - b < 2) return;
    for (uint32_t k = b + 1; k < e; ++k) {
        const uint32_t pk = perm[k];
        const uint32_t ik = id[pk];
        uint32_t m = k;
        while (m > b && id[perm[m - 1]] > ik) {
            perm[m] = perm[m - 1];
            --m;
        }
        perm[m] = pk;
    }
}

template <typename T>
__global__ void k_gather(int64_t n, const uint32_t *perm, const V4<T> *pos, const V4<T> *vel,
                         const T *drho, const uint32_t *id, V4<T> *pos_t, V4<T> *vel_t,
                         T *drho_t, uint32_t *id_t) {
    const int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (d >= n) return;
    const uint32_t s = perm[d];
    pos_t[d] = pos[s];
    vel_t[d] = vel[s];
    drho_t[d] = drho[s];
    id_t[d] = id[s];
}

template <typename T>
__global__ void k_copy_back(int64_t n, const V4<T> *pos_t, const V4<T> *vel_t, const T *drho_t,
                            const uint32_t *id_t, V4<T> *pos, V4<T> *vel, T *drho, uint32_t *id) {
    const int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (d >= n) return;
    pos[d] = pos_t[d];
    vel[d] = vel_t[d];
    drho[d] = drho_t[d];
    id[d] = id_t[d];
}

// ---- fluid ranks: after the reorder, the sorted positions of the fluid
// particles, walls left out (an exclusive scan of the fluid flags, then a
// scatter).  The list build, the band and sweeps M, V, B and C (and A with
// the cell walk) run their tiles over these ranks, so no lane of theirs idles on a wall particle (16%
// of the 3D drop, interleaved with the fluid near the walls by the Morton
// order).  Each case's fluid particles take the ranks after the previous
// cases' ones, whose count is fixed.
template <typename T>
__global__ void k_fluid_flag(int64_t n, const V4<T> *snap, uint32_t *flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > n) return;
    flag[i] = (i < n && phase_of(w_bits(snap[i].w)) != PH_WALL) ? 1u : 0u;
}

// Wall slots get their fixed values here, since no sweep visits them: a zero
// colour gradient and an empty neighbour list.
template <typename T>
__global__ void k_fluid_scatter(int64_t n, const V4<T> *snap, const uint32_t *rank, uint32_t *fidx,
                                V4<T> *gradC, uint32_t *cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    // the colour gradient starts every advection step at zero: the list
    // classes' colour sweep then writes only the interface band
    gradC[i] = V4<T>{T(0), T(0), T(0), T(0)};
    if (phase_of(w_bits(snap[i].w)) != PH_WALL) fidx[rank[i]] = (uint32_t)i;
    else cnt[i] = 0u;
}

// ================================================================ time step
static __global__ void k_reset_vmax(int ncases, CaseState *st) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncases) return;
    st[c].vmax2_acc[0] = 0ull;
    st[c].vmax2_acc[1] = 0ull;
}

template <typename T>
__global__ void k_vmax(const Tile *__restrict__ tiles, const CaseDesc *__restrict__ desc,
                       CaseState *st, const V4<T> *pos, const V4<T> *vel) {
    const Tile t = tiles[blockIdx.x];
    const int dim = desc[t.c].dim;
    unsigned long long m[2] = {0ull, 0ull};
    if ((int)threadIdx.x < t.n) {
        const int64_t i = t.begin + threadIdx.x;
        const uint32_t ph = phase_of(w_bits(pos[i].w));
        if (ph < 2) m[ph] = (unsigned long long)__double_as_longlong(speed2(vel[i], dim));
    }
    m[0] = warp_max_u64(m[0]);
    m[1] = warp_max_u64(m[1]);
    if ((threadIdx.x & 31) == 0) {
        if (m[0]) atomicMax(&st[t.c].vmax2_acc[0], m[0]);
        if (m[1]) atomicMax(&st[t.c].vmax2_acc[1], m[1]);
    }
}

// Eq. 16 per fluid (factor cfl_ad), Eq. 18 minimum; speed terms with
// |v|max = 0 are dropped.
static __global__ void k_adv_begin(int ncases, const CaseDesc *desc, CaseState *st) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncases) return;
    const CaseDesc &d = desc[c];
    CaseState &s = st[c];
    s.active = 0;
    s.last = 0;
    if (s.status) return;
    double dt_ad = __longlong_as_double(0x7ff0000000000000ll);   // +inf
    for (int k = 0; k < 2; ++k) {
        if (!s.present[k]) continue;
        const double vmax = sqrt(bits_to_d(s.vmax2_acc[k]));
        double t = __ddiv_rn(__dmul_rn(__dmul_rn(d.rho0[k], d.h), d.h), d.eta[k]);
        if (vmax > 0.0) {
            const double tv = __ddiv_rn(d.h, vmax);
            if (tv < t) t = tv;
        }
        const double cand = __dmul_rn(d.cfl_ad, t);
        if (cand < dt_ad) dt_ad = cand;
    }
    if (!(dt_ad > 0.0) || !(dt_ad < 1e300)) {
        s.status = DEV_ERR_NONFINITE;
        return;
    }
    s.dt_ad = dt_ad;
    s.t_in = 0.0;
    s.n_sub_adv = 0;
    s.active = 1;
}

// One acoustic substep criterion per case (Eq. 17 with factor cfl_ac, Eq. 18), clipped to end
// exactly on the advection step; sets the while-loop condition to "some case
// still has a substep after this one".
static __global__ void k_dt(int ncases, const CaseDesc *desc, CaseState *st, int *loop_flag,
                     cudaGraphConditionalHandle handle, int use_handle) {
    int more = 0;
    for (int c = threadIdx.x; c < ncases; c += blockDim.x) {
        const CaseDesc &d = desc[c];
        CaseState &s = st[c];
        if (s.active && s.last) {            // its advection step ended last iteration
            if (!s.status) {
                s.t = __dadd_rn(s.t, s.dt_ad);
                s.n_adv += 1;
            }
            s.active = 0;
        }
        if (s.active && s.status) s.active = 0;
        if (!s.active) continue;
        if (s.n_sub_adv >= d.max_substeps) {
            s.status = DEV_ERR_STALLED;
            s.active = 0;
            continue;
        }
        double vmax[2];
        for (int k = 0; k < 2; ++k) {
            s.vmax2_cur[k] = s.vmax2_acc[k];
            s.vmax2_acc[k] = 0ull;
            vmax[k] = sqrt(bits_to_d(s.vmax2_cur[k]));
        }
        double dt_ac = __longlong_as_double(0x7ff0000000000000ll);
        bool finite = true;
        for (int k = 0; k < 2; ++k) {
            if (!s.present[k]) continue;
            if (!(vmax[k] <= 1e300)) finite = false;
            double t = __ddiv_rn(d.h, __dadd_rn(d.c0, vmax[k]));
            if (d.gamma > 0.0 && d.dt_surf[k] < t) t = d.dt_surf[k];   // formed on the host (Eq. 17)
            const double cand = __dmul_rn(d.cfl_ac, t);
            if (cand < dt_ac) dt_ac = cand;
        }
        if (!finite || !(dt_ac > 0.0) || !(dt_ac < 1e300)) {
            s.status = DEV_ERR_NONFINITE;
            s.active = 0;
            continue;
        }
        const double rem = __dsub_rn(s.dt_ad, s.t_in);
        const int last = dt_ac >= rem;
        const double dt = last ? rem : dt_ac;
        s.last_dt_ac = dt_ac;
        s.dt = dt;
        s.last = last;
        s.t_in = __dadd_rn(s.t_in, dt);
        s.n_sub += 1;
        s.n_sub_adv += 1;
        if (!s.last) more = 1;
    }
    more = __syncthreads_or(more);
    if (threadIdx.x == 0) {
        *loop_flag = more;
        if (use_handle) cudaGraphSetConditional(handle, more ? 1u : 0u);
    }
}

// closes the advection step of the cases that ended it in the final substep
// (the others were closed by k_dt when they went idle)
static __global__ void k_adv_end(int ncases, CaseState *st) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncases) return;
    CaseState &s = st[c];
    if (s.active && s.last && !s.status) {
        s.t = __dadd_rn(s.t, s.dt_ad);
        s.n_adv += 1;
    }
    s.active = 0;
}

// ================================================================= sweeps
// ---- M: correction matrix of Eq. 15, B_i = -(sum_j r_ij (x) grad_i W_ij V_j)^-1
template <typename T> struct Moment {
    T m00 = 0, m01 = 0, m02 = 0, m11 = 0, m12 = 0, m22 = 0;
    // adds r (x) dW e V = (dW V / r) r_vec (x) r_vec of one neighbour
    template <int D>
    __device__ __forceinline__ void add(const CaseDesc &, const CasePhys<T> &cp, const T *drho, uint32_t j,
                                        uint32_t kj, T rx, T ry, T rz, T r2) {
        const PairGeo<T> g = geo(cp, r2);
        const T Vj = kj == PH_WALL ? cp.vol_wall : div_fast(cp.mass[kj], cp.rho0[kj] + drho[j]);
        const T s = g.dW * Vj * g.inv_r;
        m00 += s * rx * rx; m01 += s * rx * ry; m11 += s * ry * ry;
        if (D == 3) { m02 += s * rx * rz; m12 += s * ry * rz; m22 += s * rz * rz; }
    }
};

template <typename T, int D>
__device__ __forceinline__ void store_B(const Moment<T> &M, int64_t i, V4<T> *bmat) {
    const T m00 = M.m00, m01 = M.m01, m02 = M.m02, m11 = M.m11, m12 = M.m12, m22 = M.m22;
    T b00, b01, b02 = 0, b11, b12 = 0, b22 = 0;
    T det;
    if (D == 2) {
        det = m00 * m11 - m01 * m01;
        const T id = T(1) / det;
        b00 = -m11 * id; b01 = m01 * id; b11 = -m00 * id;
    } else {
        const T c00 = m11 * m22 - m12 * m12, c01 = m02 * m12 - m01 * m22, c02 = m01 * m12 - m02 * m11;
        det = m00 * c00 + m01 * c01 + m02 * c02;
        const T id = T(1) / det;
        b00 = -c00 * id; b01 = -c01 * id; b02 = -c02 * id;
        b11 = -(m00 * m22 - m02 * m02) * id;
        b12 = -(m02 * m01 - m00 * m12) * id;
        b22 = -(m00 * m11 - m01 * m01) * id;
    }
    if (!(fabs(det) >= T(1e-3))) {
        b00 = 1; b01 = 0; b02 = 0; b11 = 1; b12 = 0; b22 = D == 3 ? T(1) : T(0);
    }
    bmat[2 * i] = V4<T>{b00, b01, b02, b11};
    bmat[2 * i + 1] = V4<T>{b12, b22, T(0), T(0)};
}

template <bool LIST, typename T, int D>
__device__ __forceinline__ void sweep_M(const CaseDesc &d, const CasePhys<T> &cp, int64_t i,
                                        const uint32_t *starts, const uint32_t *nbr, const uint32_t *cnt, const V4<T> *snap, const T *drho,
                                        V4<T> *bmat, V4<T> *bk, int32_t *status) {
    const V4<T> si = ld4(snap + i);
    const uint32_t pki = w_bits(si.w);
    const uint32_t ki = phase_of(pki);
    if (ki == PH_WALL) return;
    const bool own = bk != nullptr && d.surface_corr == 1;
    Moment<T> M, Mk;
    const bool coinc = neighbors<LIST, T, D>(d, cp, starts, nbr, cnt, snap, i, si, pki,
        [&](uint32_t j, const V4<T> &sj, T rx, T ry, T rz, T r2) {
            const uint32_t kj = phase_of(w_bits(sj.w));
            M.template add<D>(d, cp, drho, j, kj, rx, ry, rz, r2);
            // the same sum over i's own fluid (surface_corr reading of Eq. 33)
            if (own && kj == ki) Mk.template add<D>(d, cp, drho, j, kj, rx, ry, rz, r2);
        });
    if (coinc) atomicCAS(status, 0, DEV_ERR_COINCIDENT);
    store_B<T, D>(M, i, bmat);
    if (own) store_B<T, D>(Mk, i, bk);
}

// ---- V: viscous acceleration (Eq. 13) and transport shift (Eq. 14)
template <bool LIST, typename T, int D>
__device__ __forceinline__ void sweep_V(const CaseDesc &d, const CasePhys<T> &cp, int64_t i,
                                        const uint32_t *starts, const uint32_t *nbr, const uint32_t *cnt, const V4<T> *snap, const T *drho,
                                        const V4<T> *vel, const V4<T> *bmat, V4<T> *acc_visc,
                                        V4<T> *pos, int32_t *status) {
    const V4<T> si = ld4(snap + i);
    const uint32_t pki = w_bits(si.w);
    const uint32_t ki = phase_of(pki);
    if (ki == PH_WALL) return;
    const V4<T> vi = vel[i];
    const T rho_i = sel(ki, cp.rho0[0], cp.rho0[1]) + vi.w;
    // the pair viscosity 2 eta_i eta_j / (eta_i + eta_j) takes one value per
    // fluid of j; walls use eta_i
    const T eta_i = sel(ki, cp.eta[0], cp.eta[1]);
    const T etab0 = T(2) * eta_i * cp.eta[0] / (eta_i + cp.eta[0]);
    const T etab1 = T(2) * eta_i * cp.eta[1] / (eta_i + cp.eta[1]);
    const T rho0_0 = cp.rho0[0], rho0_1 = cp.rho0[1], m_0 = cp.mass[0], m_1 = cp.mass[1];
    const T vol_wall = cp.vol_wall;
    const KernelGeo<T> kgeo(cp);
    const bool tvf = d.tvf_on != 0;
    V4<T> Bi0 = {0, 0, 0, 0}, Bi1 = {0, 0, 0, 0};
    if (tvf) { Bi0 = bmat[2 * i]; Bi1 = bmat[2 * i + 1]; }
    T ax = 0, ay = 0, az = 0, sx = 0, sy = 0, sz = 0;
    const bool coinc = neighbors_aux<LIST, T, D>(d, cp, starts, nbr, cnt, snap, vel, i, si, pki,
        [&](uint32_t j, const V4<T> &sj, const V4<T> &vj, T rx, T ry, T rz, T r2) {
            const PairGeo<T> g = kgeo(r2);
            const uint32_t kj = phase_of(w_bits(sj.w));
            T eta_bar, Vj;
            V4<T> Bj0 = Bi0, Bj1 = Bi1;
            if (kj == PH_WALL) {
                eta_bar = eta_i;
                Vj = vol_wall;
            } else {
                eta_bar = sel(kj, etab0, etab1);
                Vj = div_fast(sel(kj, m_0, m_1), sel(kj, rho0_0, rho0_1) + vj.w);
                if (tvf) { Bj0 = bmat[2 * j]; Bj1 = bmat[2 * j + 1]; }
            }
            const T w = g.dW * Vj * g.inv_r;                 // grad W V = w r_vec
            const T f = eta_bar * w;                          // eta (v_ij / r) dW V
            ax += f * (vi.x - vj.x);
            ay += f * (vi.y - vj.y);
            if (D == 3) az += f * (vi.z - vj.z);
            if (tvf) {
                const T gx = w * rx, gy = w * ry, gz = w * rz;
                // (B_i + B_j) grad W V with symmetric B = [b00 b01 b02; b01 b11 b12; b02 b12 b22]
                const T s00 = Bi0.x + Bj0.x, s01 = Bi0.y + Bj0.y, s02 = Bi0.z + Bj0.z;
                const T s11 = Bi0.w + Bj0.w, s12 = Bi1.x + Bj1.x, s22 = Bi1.y + Bj1.y;
                sx += s00 * gx + s01 * gy + (D == 3 ? s02 * gz : T(0));
                sy += s01 * gx + s11 * gy + (D == 3 ? s12 * gz : T(0));
                if (D == 3) sz += s02 * gx + s12 * gy + s22 * gz;
            }
        });
    if (coinc) atomicCAS(status, 0, DEV_ERR_COINCIDENT);
    const T c = T(2) / rho_i;
    acc_visc[i] = V4<T>{c * ax, c * ay, c * az, T(0)};
    if (tvf) {
        V4<T> p = pos[i];
        p.x += cp.tvf_coef * sx;
        p.y += cp.tvf_coef * sy;
        if (D == 3) p.z += cp.tvf_coef * sz;
        pos[i] = p;
    }
}

// ---- A: colour gradient, Eq. 22 (only pairs of different fluids contribute)
template <bool LIST, typename T, int D, int L = 1>
__device__ __forceinline__ void sweep_A(const CaseDesc &d, const CasePhys<T> &cp, int64_t i,
                                        const uint32_t *starts, const uint32_t *nbr, const uint32_t *cnt, const V4<T> *snap, const T *drho,
                                        const V4<T> *lgeo, V4<T> *gradC, uint32_t sub = 0) {
    const V4<T> si = ld4(snap + i);
    const uint32_t pki = w_bits(si.w);
    const uint32_t ki = phase_of(pki);
    V4<T> g = {0, 0, 0, 0};
    if (ki != PH_WALL && d.n_fluid_phases == 2) {
        const uint32_t other = ki ^ 1u;
        const T two_phi = cp.two_phi[ki];
        const T m_o = cp.mass[other], rho0_o = cp.rho0[other];
        if constexpr (LIST && SPHST_LIST_GEO && L == 1) {
            walk_geo<PART_OTHER, T>(d, nbr, cnt, lgeo, i, [&](bool, uint32_t j, const V4<T> &G) {
                const T s = two_phi * G.w * div_fast(m_o, add_rn(rho0_o, drho[j]));
                g.x = fma_rn(s, G.x, g.x);
                g.y = fma_rn(s, G.y, g.y);
                if (D == 3) g.z = fma_rn(s, G.z, g.z);
            });
        } else
        neighbors<LIST, T, D, PART_OTHER, L>(d, cp, starts, nbr, cnt, snap, i, si, pki,
            [&](uint32_t j, const V4<T> &sj, T rx, T ry, T rz, T r2) {
                if (!LIST && phase_of(w_bits(sj.w)) != other) return;
                const PairGeo<T> gg = geo(cp, r2);
                const T Vj = div_fast(m_o, add_rn(rho0_o, drho[j]));
                const T s = two_phi * gg.dW * Vj * gg.inv_r;
                g.x = fma_rn(s, rx, g.x);
                g.y = fma_rn(s, ry, g.y);
                if (D == 3) g.z = fma_rn(s, rz, g.z);
            }, sub);
        g.x = group_sum<L>(g.x);
        g.y = group_sum<L>(g.y);
        if (D == 3) g.z = group_sum<L>(g.z);
        g.w = sqrt(fma_rn(g.x, g.x, fma_rn(g.y, g.y, g.z * g.z)));
    }
    if (sub == 0) gradC[i] = g;
}

// ---- B: pressure + surface tension + kick
// With the neighbour list the surface sum (Eqs. 24, 26, 30, 33) is a kernel of
// its own (S, below), launched before B and taken only by particles of the
// interface band (band[i]: i or one of its neighbours has neighbours of the
// other fluid; elsewhere grad C = 0 for i and all its neighbours and every
// surface term is zero).  B then runs the pressure sum over all neighbours and
// adds the stored surface sum.  The terms are those of the single pass of
// the cell walk; the list's order (other-phase neighbours first) and the
// surface sweep's lanes add them in another order, so the two agree to
// rounding.
//
// PASS: 0 = pressure + surface in one walk (cell walk), 1 = pressure and the
// stored surface sum (list), 2 = surface sum only (list, band particles).
template <bool LIST, int PASS, typename T, int D, int L = 1>
__device__ __forceinline__ double sweep_B(const CaseDesc &d, const CasePhys<T> &cp, T dt,
                                          int64_t i, const uint32_t *starts, const uint32_t *nbr, const uint32_t *cnt,
                                          const uint8_t *band, const V4<T> *snap,
                                          const V4<T> *vel, const V4<T> *gradC,
                                          const V4<T> *acc_visc, V4<T> *acc_surf, V4<T> *vel_new,
                                          const V4<T> *lgeo, uint32_t *phase_out, uint32_t sub = 0,
                                          const V4<T> *bk = nullptr, const T *drho_s = nullptr) {
    const V4<T> si = ld4(snap + i);
    const uint32_t pki = w_bits(si.w);
    const uint32_t ki = phase_of(pki);
    *phase_out = ki;
    if (ki == PH_WALL) return 0.0;
    if (PASS == 2 && !band[i]) return 0.0;
    const V4<T> vi = vel[i];
    const T dri = vi.w;
    const T rho_i = add_rn(sel(ki, cp.rho0[0], cp.rho0[1]), dri);
    const T p_i = cp.c0sq * dri;
    T apx = 0, apy = 0, apz = 0, asx = 0, asy = 0, asz = 0;
    const Limiter<T> limiter_beta(cp, d.limiter);
    const bool wall_push_only = d.wall_form == 1;
    const T c0 = cp.c0, c0sq = cp.c0sq, vol_wall = cp.vol_wall;
    const T rho0_0 = cp.rho0[0], rho0_1 = cp.rho0[1], m_0 = cp.mass[0], m_1 = cp.mass[1];
    const KernelGeo<T> kgeo(cp);

    // pressure (Eqs. 7-12) of one pair from e_ij, W'_ij, the neighbour's
    // kind (wall, or fluid of rest density rho0_j and mass m_j) and state
    // every sum is written as an explicitly rounded add or FMA: the same
    // source compiled for another launch mode (one case, batch) then rounds
    // identically whatever the register allocation
    const T c0rho_i = c0 * rho_i;
    const auto pressure_pair = [&](L2<T> exy, T ez, T dW, bool wall, T rho0_j, T m_j, const V4<T> &vj) {
        // U_L - U_R = (v_j - v_i).e  (Eq. 10, U = -v.e)
        const L2<T> dvxy = fma2(l2(vi.x, vi.y), l2(T(-1), T(-1)), l2(vj.x, vj.y));
        const T dUe = D == 3 ? fma_rn(dvxy.x, exy.x, fma_rn(dvxy.y, exy.y, sub_rn(vj.z, vi.z) * ez))
                             : fma_rn(dvxy.x, exy.x, dvxy.y * exy.y);
        if (wall) {
            // mirror state behind a wall moving with v_w: rho_i, p_i, 2 U_w - U_L
            const T dU = T(2) * dUe;
            const T beta = limiter_beta(dU, p_i, rho_i);       // mirror state: rho_R, p_R = rho_i, p_i
            T Ps = fma_rn(beta * c0rho_i * dU, T(0.5), p_i);
            if (wall_push_only) Ps = Ps > T(0) ? Ps : T(0);    // no-suction wall reading
            const T f = Ps * dW * vol_wall;
            const L2<T> a = fma2(l2(f, f), exy, l2(apx, apy));
            apx = a.x; apy = a.y; if (D == 3) apz = fma_rn(f, ez, apz);
            return;
        }
        const T drj = vj.w;
        const T rho_j = add_rn(rho0_j, drj);
        const T p_j = c0sq * drj;
        const T dU = dUe;
        const T rsum = add_rn(rho_i, rho_j);
        const T beta = limiter_beta(dU, add_rn(p_i, p_j), rsum);   // Eq. 11
        // P* V_j with P* = (rho_i p_j + rho_j p_i + beta c0 rho_i rho_j dU) / (rho_i + rho_j)
        // (Eqs. 8, 12) and V_j = m_j / rho_j: one division
        const T num = fma_rn(beta * c0rho_i * rho_j, dU, fma_rn(rho_i, p_j, rho_j * p_i));
        const T f = div_fast(num * m_j, rsum * rho_j) * dW;
        const L2<T> a = fma2(l2(f, f), exy, l2(apx, apy));
        apx = a.x; apy = a.y; if (D == 3) apz = fma_rn(f, ez, apz);
    };
    // walls by their mirror state
    const auto pressure = [&](uint32_t, const V4<T> &sj, const V4<T> &vj, T rx, T ry, T rz, T r2) {
        const PairGeo<T> g = kgeo(r2);
        const L2<T> exy = mul2(l2(rx, ry), l2(g.inv_r, g.inv_r));
        const uint32_t kj = phase_of(w_bits(sj.w));
        pressure_pair(exy, D == 3 ? rz * g.inv_r : T(0), g.dW, kj == PH_WALL, sel(kj, rho0_0, rho0_1),
                      sel(kj, m_0, m_1), vj);
    };

    // surface stress and penalty (Eqs. 24, 26, 30, 33); walls take no part
    const V4<T> gi = d.n_fluid_phases == 2 ? gradC[i] : V4<T>{0, 0, 0, 0};
    // surface_corr reading: the own-fluid correction matrix of i (Eq. 15
    // over i's fluid), symmetric: (b00, b01, b02, b11), (b12, b22)
    const bool corr = bk != nullptr && d.surface_corr == 1;
    V4<T> bi0{T(0), T(0), T(0), T(0)}, bi1{T(0), T(0), T(0), T(0)};
    if (corr && PASS != 1) { bi0 = bk[2 * i]; bi1 = bk[2 * i + 1]; }
    const auto surface = [&](uint32_t j, const V4<T> &sj, T rx, T ry, T rz, T r2) {
        const uint32_t kj = phase_of(w_bits(sj.w));
        if (kj == PH_WALL) return;
        const V4<T> gj = gradC[j];
        if (gi.w == T(0) && gj.w == T(0)) return;                // every surface term vanishes
        const PairGeo<T> g = geo(cp, r2);
        const T ex = rx * g.inv_r, ey = ry * g.inv_r, ez = D == 3 ? rz * g.inv_r : T(0);
        // the density deviation of j: the 4-byte array in the surface sweep
        // (the same value as vel[j].w, fewer bytes through L1)
        const T drj_s = PASS == 2 ? drho_s[j] : vel[j].w;
        const T rho_j = sel(kj, cp.rho0[0], cp.rho0[1]) + drj_s;
        const T Vj = div_fast(sel(kj, cp.mass[0], cp.mass[1]), rho_j);
        const bool if_i = gi.w * cp.h > cp.nhat_eps;
        const T inv_gi = if_i ? div_fast(T(1), gi.w) : T(0);
        const T nix = gi.x * inv_gi, niy = gi.y * inv_gi, niz = gi.z * inv_gi;
        const T gam_gi = if_i ? cp.gamma * gi.w : T(0);
        const bool if_j = gj.w * cp.h > cp.nhat_eps;
        const T inv_gj = if_j ? div_fast(T(1), gj.w) : T(0);
        const T njx = gj.x * inv_gj, njy = gj.y * inv_gj, njz = gj.z * inv_gj;
        const T gam_gj = if_j ? cp.gamma * gj.w : T(0);
        if (corr && kj == ki) {
            // same-phase line applied to the corrected kernel gradient
            // W' (B^k_i + B^k_j)/2 e = W' v (C_ij = 0): S v with
            // Pi v = gamma |gradC| (v - n (n.v)) and C-hat v of Eq. 30
            const V4<T> bj0 = bk[2 * j], bj1 = bk[2 * j + 1];
            const T m00 = T(0.5) * (bi0.x + bj0.x), m01 = T(0.5) * (bi0.y + bj0.y), m11 = T(0.5) * (bi0.w + bj0.w);
            const T m02 = D == 3 ? T(0.5) * (bi0.z + bj0.z) : T(0), m12 = D == 3 ? T(0.5) * (bi1.x + bj1.x) : T(0);
            const T m22 = D == 3 ? T(0.5) * (bi1.y + bj1.y) : T(0);
            const T vx = m00 * ex + m01 * ey + m02 * ez, vy = m01 * ex + m11 * ey + m12 * ez;
            const T vz = D == 3 ? m02 * ex + m12 * ey + m22 * ez : T(0);
            const T niv = nix * vx + niy * vy + niz * vz, njv = njx * vx + njy * vy + njz * vz;
            const T bx = T(0.5) * (gi.x + gj.x), by = T(0.5) * (gi.y + gj.y), bz = T(0.5) * (gi.z + gj.z);
            const T b2 = bx * bx + by * by + bz * bz;
            const T inv_bn = b2 > T(0) ? rsqrt_fast(b2) : T(0);
            T cx, cy, cz;
            if (d.penalty_form == 0) {            // -|gradCbar| r nbar (nbar.v)
                const T fac = g.r * (bx * vx + by * vy + bz * vz) * inv_bn;
                cx = -fac * bx; cy = -fac * by; cz = -fac * bz;
            } else if (d.penalty_form == 1) {     // -|gradCbar| r e (e.v)
                const T f = -(b2 * inv_bn * g.r) * (ex * vx + ey * vy + ez * vz);
                cx = f * ex; cy = f * ey; cz = f * ez;
            } else {                              // -(gradCbar . r_ij) v
                const T f = -g.r * (bx * ex + by * ey + bz * ez);
                cx = f * vx; cy = f * vy; cz = f * vz;
            }
            const T nic = nix * cx + niy * cy + niz * cz, njc = njx * cx + njy * cy + njz * cz;
            const T qx = T(0.5) * (nix * nic + njx * njc), qy = T(0.5) * (niy * nic + njy * njc),
                    qz = T(0.5) * (niz * nic + njz * njc);
            const T pen_s = d.penalty_scope == 1 ? T(0) : cp.xi * cp.gamma * g.inv_r;
            const T sx = gam_gi * (vx - nix * niv) + gam_gj * (vx - njx * njv) + pen_s * (cx - qx);
            const T sy = gam_gi * (vy - niy * niv) + gam_gj * (vy - njy * njv) + pen_s * (cy - qy);
            const T sz = gam_gi * (vz - niz * niv) + gam_gj * (vz - njz * njv) + pen_s * (cz - qz);
            const T w = g.dW * Vj;
            asx += sx * w; asy += sy * w; if (D == 3) asz += sz * w;
            return;
        }
        const T nie = nix * ex + niy * ey + niz * ez;
        const T nje = njx * ex + njy * ey + njz * ez;
        // Pi e = gamma |gradC| (e - n (n.e))   (Eq. 24)
        const T pix = gam_gi * (ex - nix * nie), piy = gam_gi * (ey - niy * nie), piz = gam_gi * (ez - niz * nie);
        const T pjx = gam_gj * (ex - njx * nje), pjy = gam_gj * (ey - njy * nje), pjz = gam_gj * (ez - njz * nje);
        const bool same = kj == ki;
        const T sg = (same || d.grad_mode == 1) ? T(1) : T(-1);
        const T bx = T(0.5) * (gi.x + sg * gj.x), by = T(0.5) * (gi.y + sg * gj.y),
                bz = T(0.5) * (gi.z + sg * gj.z);
        const T b2 = bx * bx + by * by + bz * bz;
        const T inv_bn = b2 > T(0) ? rsqrt_fast(b2) : T(0);
        const T Cij = same ? T(0) : T(1);
        // C-hat e (Eq. 30 with the selected contraction)
        T cx, cy, cz;
        if (d.penalty_form == 0) {
            const T fac = g.r * (bx * ex + by * ey + bz * ez) * inv_bn;
            cx = Cij * ex - fac * bx; cy = Cij * ey - fac * by; cz = Cij * ez - fac * bz;
        } else {
            // EE: (C_ij - |gradCbar| r) e; SCALAR (Eq. 29): (C_ij - gradCbar . r_ij) e
            const T s = d.penalty_form == 1 ? Cij - b2 * inv_bn * g.r
                                            : Cij - g.r * (bx * ex + by * ey + bz * ez);
            cx = s * ex; cy = s * ey; cz = s * ez;
        }
        // N-bar C-hat e = (n_i (n_i.c) + n_j (n_j.c)) / 2
        const T nic = nix * cx + niy * cy + niz * cz;
        const T njc = njx * cx + njy * cy + njz * cz;
        const T qx = T(0.5) * (nix * nic + njx * njc), qy = T(0.5) * (niy * nic + njy * njc),
                qz = T(0.5) * (niz * nic + njz * njc);
        const T pen = cp.xi * cp.gamma * g.inv_r;
        T sx, sy, sz;
        if (same) {   // Eq. 33, first line; T-bar c = c - N-bar c
            const T pen_s = d.penalty_scope == 1 ? T(0) : pen;
            sx = pix + pjx + pen_s * (cx - qx);
            sy = piy + pjy + pen_s * (cy - qy);
            sz = piz + pjz + pen_s * (cz - qz);
        } else {      // Eq. 33, second line: 2 phi_j Pi_i + 2 phi_i Pi_j as printed, or
                      // each stress by its own particle's 2 phi (stress_weights 1)
            const bool own = d.stress_weights == 1;
            const T a = sel(own ? ki : kj, cp.two_phi[0], cp.two_phi[1]),
                    b = sel(own ? kj : ki, cp.two_phi[0], cp.two_phi[1]),
                    c = cp.four_phi_phi * pen;
            sx = a * pix + b * pjx - c * qx;
            sy = a * piy + b * pjy - c * qy;
            sz = a * piz + b * pjz - c * qz;
        }
        const T w = g.dW * Vj;
        asx += sx * w; asy += sy * w; if (D == 3) asz += sz * w;
    };

    const bool surface_on = d.n_fluid_phases == 2;
    if constexpr (PASS == 2) {
        if (surface_on) neighbors<LIST, T, D, PART_ALL, L>(d, cp, starts, nbr, cnt, snap, i, si, pki, surface, sub);
        asx = group_sum<L>(asx);
        asy = group_sum<L>(asy);
        if (D == 3) asz = group_sum<L>(asz);
        if (sub == 0) acc_surf[i] = V4<T>{asx, asy, asz, T(0)};
        return 0.0;
    } else if constexpr (PASS == 1) {
        if constexpr (LIST && SPHST_LIST_GEO && L == 1) {
            const T rho0_o = sel(ki ^ 1u, rho0_0, rho0_1), rho0_s = sel(ki, rho0_0, rho0_1);
            const T m_o = sel(ki ^ 1u, m_0, m_1), m_s = sel(ki, m_0, m_1);
            walk_geo_aux<T>(d, nbr, cnt, lgeo, vel, i, [&](bool other, uint32_t, const V4<T> &G, const V4<T> &vj) {
                const bool wall = geo_wall(G.w);
                pressure_pair(l2(G.x, G.y), G.z, wall ? -G.w : G.w, wall, other ? rho0_o : rho0_s,
                              other ? m_o : m_s, vj);
            });
        } else
        neighbors_aux<LIST, T, D, L>(d, cp, starts, nbr, cnt, snap, vel, i, si, pki, pressure, sub);
        apx = group_sum<L>(apx);
        apy = group_sum<L>(apy);
        if (D == 3) apz = group_sum<L>(apz);
        if (sub != 0) {               // the group's lane 0 kicks
            *phase_out = PH_WALL;
            return 0.0;
        }
        if (surface_on && band[i]) {
            const V4<T> as = acc_surf[i];
            asx = as.x; asy = as.y; asz = as.z;
        }
    } else {
        neighbors<LIST, T, D>(d, cp, starts, nbr, cnt, snap, i, si, pki,
            [&](uint32_t j, const V4<T> &sj, T rx, T ry, T rz, T r2) {
                pressure(j, sj, vel[j], rx, ry, rz, r2);
                if (surface_on) surface(j, sj, rx, ry, rz, r2);
            });
    }
    const T inv_rho = T(1) / rho_i;
    const T m2inv_rho = T(-2) * inv_rho;
    const V4<T> av = acc_visc[i];
    V4<T> vn;
    vn.x = fma_rn(dt, fma_rn(inv_rho, asx, fma_rn(m2inv_rho, apx, av.x)), vi.x);
    vn.y = fma_rn(dt, fma_rn(inv_rho, asy, fma_rn(m2inv_rho, apy, av.y)), vi.y);
    vn.z = D == 3 ? fma_rn(dt, fma_rn(inv_rho, asz, fma_rn(m2inv_rho, apz, av.z)), vi.z) : T(0);
    vn.w = dri;                       // density deviation for sweep C
    vel_new[i] = vn;
    return speed2(vn, D);
}

// ---- C: continuity (Eq. 6) with v* (normal component -U*) + drift
template <bool LIST, typename T, int D, int L = 1>
__device__ __forceinline__ void sweep_C(const CaseDesc &d, const CasePhys<T> &cp, T dt, int64_t i,
                                        const uint32_t *starts, const uint32_t *nbr, const uint32_t *cnt, const V4<T> *snap,
                                        const V4<T> *vel_new, T *drho,
                                        V4<T> *vel, V4<T> *pos, const V4<T> *lgeo, uint32_t sub = 0) {
    const V4<T> si = ld4(snap + i);
    const uint32_t pki = w_bits(si.w);
    const uint32_t ki = phase_of(pki);
    if (ki == PH_WALL) return;
    V4<T> vi = vel_new[i];
    const T dri = vi.w;
    const T rho0_0 = cp.rho0[0], rho0_1 = cp.rho0[1], m_0 = cp.mass[0], m_1 = cp.mass[1];
    const T c0 = cp.c0, c0sq = cp.c0sq, vol_wall = cp.vol_wall;
    const T rho_i = add_rn(sel(ki, rho0_0, rho0_1), dri);
    const T p_i = c0sq * dri;
    const KernelGeo<T> kgeo(cp);
    // the pressure difference enters with the sign of the v* reading; the
    // sign is folded into p_i and c0^2 once
    const T psign = d.vstar_printed ? T(-1) : T(1);
    const T sp_i = psign * p_i, sc0sq = psign * c0sq;
    T s = 0;
    // one pair from (v_i - v_j).e = U_R - U_L, W'_ij, the neighbour's kind and
    // its density deviation
    const auto pair = [&](T dve, T dW, bool wall, T rho0_j, T m_j, T drj) {
        if (wall) {                   // v* = v_w
            s = fma_rn(dve * dW, vol_wall, s);
            return;
        }
        const T rho_j = add_rn(rho0_j, drj);
        // (v_i - v*).e V_j with (v_i - v*).e = U* - U_L = (Z_R (U_R - U_L) + p_i - p_j)
        // / (Z_L + Z_R) and V_j = m_j / rho_j: one division.  The printed v*
        // gives (Z_R (U_R - U_L) - (p_i - p_j)) / (Z_L + Z_R) instead.
        // (sums explicitly rounded, as in sweep B)
        const T num = fma_rn(rho_j * c0, dve, fma_rn(-sc0sq, drj, sp_i)) * m_j;
        s = fma_rn(div_fast(num, c0 * add_rn(rho_i, rho_j) * rho_j), dW, s);
    };
    if constexpr (LIST && SPHST_LIST_GEO && L == 1) {
        const T rho0_o = sel(ki ^ 1u, rho0_0, rho0_1), rho0_s = sel(ki, rho0_0, rho0_1);
        const T m_o = sel(ki ^ 1u, m_0, m_1), m_s = sel(ki, m_0, m_1);
        walk_geo_aux<T>(d, nbr, cnt, lgeo, vel_new, i, [&](bool other, uint32_t, const V4<T> &G, const V4<T> &vj) {
            const L2<T> dvxy = fma2(l2(vj.x, vj.y), l2(T(-1), T(-1)), l2(vi.x, vi.y));
            const T dve = D == 3 ? fma_rn(dvxy.x, G.x, fma_rn(dvxy.y, G.y, sub_rn(vi.z, vj.z) * G.z))
                                 : fma_rn(dvxy.x, G.x, dvxy.y * G.y);
            const bool wall = geo_wall(G.w);
            pair(dve, wall ? -G.w : G.w, wall, other ? rho0_o : rho0_s, other ? m_o : m_s, vj.w);
        });
    } else
    neighbors_aux<LIST, T, D, L>(d, cp, starts, nbr, cnt, snap, vel_new, i, si, pki,
        [&](uint32_t, const V4<T> &sj, const V4<T> &vj, T rx, T ry, T rz, T r2) {
            const PairGeo<T> g = kgeo(r2);
            const uint32_t kj = phase_of(w_bits(sj.w));
            const L2<T> dvxy = fma2(l2(vj.x, vj.y), l2(T(-1), T(-1)), l2(vi.x, vi.y));
            const T dvr = D == 3 ? fma_rn(dvxy.x, rx, fma_rn(dvxy.y, ry, sub_rn(vi.z, vj.z) * rz))
                                 : fma_rn(dvxy.x, rx, dvxy.y * ry);
            pair(dvr * g.inv_r, g.dW, kj == PH_WALL, sel(kj, rho0_0, rho0_1), sel(kj, m_0, m_1), vj.w);
        }, sub);
    s = group_sum<L>(s);
    if (sub != 0) return;
    const T dr_new = fma_rn(dt, T(2) * rho_i * s, dri);
    drho[i] = dr_new;
    V4<T> p = pos[i];
    p.x = fma_rn(dt, vi.x, p.x);
    p.y = fma_rn(dt, vi.y, p.y);
    if (D == 3) p.z = fma_rn(dt, vi.z, p.z);
    pos[i] = p;
    vi.w = dr_new;
    vel[i] = vi;
}

// ---------------------------------------------------------- sweep kernels
// Tiles are grouped by class (dimension, neighbour source) and each class is
// launched with its own instantiation, so every kernel is compiled (and its
// registers allocated) for one dimension and one neighbour source only.
struct SweepArgs {
    const Tile *tiles;
    const CaseDesc *desc;
    CaseState *st;
    const uint32_t *starts;
    const uint32_t *nbr;
    const uint32_t *cnt;
    int64_t tile0;                 // first tile of the launched class
    // nullptr: tile entries are particle indices; else the tiles run over
    // fluid ranks and fidx maps a rank to the particle (sweeps B and C)
    const uint32_t *fidx = nullptr;
    // batches: the tiles of the cases active in this substep, compacted per
    // class after the criterion kernel (work[tile0 + k] is a tile index,
    // *work_count of them); the launch's blocks stride over them.  nullptr:
    // block b takes tile tile0 + b / L.
    const uint32_t *work = nullptr;
    const uint32_t *work_count = nullptr;
    // an engine of one case: its descriptor by value, so that the sweeps of
    // MODE_ONE read the per-case constants from the launch's parameter block
    // (constant-bank operands) instead of holding them in registers
    CaseDesc one{};
};

// How a per-substep sweep finds its tiles and its case: MODE_TILES, block b
// takes tile tile0 + b / L and reads desc[c]; MODE_WORK, the blocks stride
// over the batch's work list; MODE_ONE, as MODE_TILES with the one case's
// descriptor taken from the parameter block.
enum SweepMode { MODE_TILES = 0, MODE_WORK = 1, MODE_ONE = 2 };
template <int MODE> __device__ __forceinline__ const CaseDesc &case_desc(const SweepArgs &a, int c) {
    if constexpr (MODE == MODE_ONE) return a.one;
    else return a.desc[c];
}

// Work items of a sweep launch: (tile, block of the tile) pairs; with L
// lanes per particle a tile takes L blocks.  Without a work list (WORK
// false: single cases) the launch has one block per item and each block
// runs one item; with one (batches), its blocks take items blockIdx.x,
// blockIdx.x + gridDim.x, ... up to L x (active tiles of the class).
template <int L, bool WORK> __device__ __forceinline__ int64_t work_items(const SweepArgs &a) {
    return WORK ? (int64_t)(*a.work_count) * L : (int64_t)gridDim.x;
}
template <int L, bool WORK> __device__ __forceinline__ Tile work_tile(const SweepArgs &a, int64_t w) {
    return a.tiles[WORK ? (int64_t)a.work[a.tile0 + w / L] : a.tile0 + w / L];
}

// particle of tile position q: the position itself, or the fluid particle of
// that rank (the list build, the band, sweeps M, V, B and C, A with the cell walk)
__device__ __forceinline__ int64_t particle_at(const SweepArgs &a, int64_t q) {
    return a.fidx ? (int64_t)a.fidx[q] : q;
}

// offset -1/0/+1 between neighbour cells from their index difference, which
// is +-(ncell - 1) across the wrap of a periodic axis
__device__ __forceinline__ int cell_step(const CaseDesc &d, int a, int diff) {
    if (diff > 1) return diff - d.ncell[a];
    if (diff < -1) return diff + d.ncell[a];
    return diff;
}

// ---- L: neighbour list of the frozen configuration (fluid particles only)
template <typename T, int D>
__device__ __forceinline__ void build_list(const CaseDesc &d, const CasePhys<T> &cp, int64_t i,
                                           const uint32_t *starts, const V4<T> *snap,
                                           uint32_t *nbr, uint32_t *cnt, int32_t *status) {
    const V4<T> si = ld4(snap + i);
    const uint32_t pki = w_bits(si.w);
    if (phase_of(pki) == PH_WALL) { cnt[i] = 0; return; }
    const int cx = cell_x<D>(pki), cy = cell_y<D>(pki), cz = cell_z<D>(pki);
    const int64_t stride = d.p_end - d.p_begin;
    uint32_t *base = nbr + d.nbr_base + (i - d.p_begin);
    const uint32_t kmax = (uint32_t)d.nbr_k;
    const uint32_t other = phase_of(pki) ^ 1u;
    const auto entry_of = [&](uint32_t j, uint32_t pkj) {
        const uint32_t code = cell_code<D>(cell_step(d, 0, cell_x<D>(pkj) - cx),
                                           cell_step(d, 1, cell_y<D>(pkj) - cy),
                                           D == 3 ? cell_step(d, 2, cell_z<D>(pkj) - cz) : 0);
        return (j << NBR_SHIFT) | code;
    };
    // one walk: the rest goes straight to the list, other-phase entries to a
    // small buffer; then, where there are any, the rest moves up and the
    // buffer goes in front (each part keeps the walk's order)
    constexpr uint32_t OBUF = 32;
    uint32_t obuf[OBUF];
    uint32_t c_rest = 0, c_other = 0;
    bool coinc = LIST_WALK<T, D>(d, cp, starts, snap, i, si, pki,
        [&](uint32_t j, const V4<T> &sj, T, T, T, T) {
            const uint32_t pkj = w_bits(sj.w);
            if (phase_of(pkj) == other) {
                if (c_other < OBUF) obuf[c_other] = entry_of(j, pkj);
                ++c_other;
            } else {
                if (c_rest < kmax) base[(int64_t)c_rest * stride] = entry_of(j, pkj);
                ++c_rest;
            }
        });
    uint32_t c = c_rest + c_other;
    bool overflow = c > kmax;
    if (!overflow && c_other > OBUF) {
        // rare: more other-phase neighbours than the buffer holds; two walks
        c = 0;
        for (int part = 0; part < 2; ++part) {
            coinc |= LIST_WALK<T, D>(d, cp, starts, snap, i, si, pki,
                [&](uint32_t j, const V4<T> &sj, T, T, T, T) {
                    const uint32_t pkj = w_bits(sj.w);
                    if ((phase_of(pkj) == other) != (part == 0)) return;
                    base[(int64_t)c * stride] = entry_of(j, pkj);
                    ++c;
                });
        }
    } else if (!overflow && c_other > 0) {
        for (uint32_t k = c_rest; k-- > 0;) base[(int64_t)(k + c_other) * stride] = base[(int64_t)k * stride];
        for (uint32_t k = 0; k < c_other; ++k) base[(int64_t)k * stride] = obuf[k];
    }
    if (overflow) c = kmax;
    cnt[i] = c | (c_other << 16);
    if (coinc) atomicCAS(status, 0, DEV_ERR_COINCIDENT);
    if (overflow) atomicCAS(status, 0, DEV_ERR_NBR_OVERFLOW);
}

// ---- interface band of the frozen configuration: i, or one of its
// neighbours, has neighbours of the other fluid phase.  Band particles are
// also appended, as (case << 32 | index), to the class's list that the
// surface sweep walks (warp-aggregated atomics; the order is irrelevant
// because every particle's sum is its own).
template <typename T, int D, bool LIST>
__global__ void __launch_bounds__(256) k_band(SweepArgs a, const V4<T> *snap, uint8_t *band,
                                              uint64_t *blist, uint32_t *bcount) {
    const Tile t = a.tiles[a.tile0 + blockIdx.x];
    const bool live = (int)threadIdx.x < t.n && a.st[t.c].active;
    const int64_t i = live ? particle_at(a, t.begin + threadIdx.x) : 0;
    bool b = false;
    if (live) {
        const CaseDesc &d = a.desc[t.c];
        const uint32_t ci = a.cnt[i];
        b = (ci >> 16) != 0;
        if (!b && d.n_fluid_phases == 2) {
            const int64_t stride = d.p_end - d.p_begin;
            const uint32_t *p = a.nbr + d.nbr_base + (i - d.p_begin);
            const uint32_t c = ci & CNT_MASK;
            for (uint32_t k = 0; k < c && !b; ++k, p += stride) b = (a.cnt[ld_list(p) >> NBR_SHIFT] >> 16) != 0;
        }
        band[i] = b ? 1 : 0;
    }
    const unsigned m = __ballot_sync(0xffffffffu, b);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(bcount, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (b) blist[base + __popc(m & ((1u << lane) - 1u))] = ((uint64_t)(uint32_t)t.c << 32) | (uint64_t)(uint32_t)i;
}

template <typename T, int D, bool LIST>
__global__ void __launch_bounds__(256) k_build_list(SweepArgs a, const V4<T> *snap, uint32_t *nbr, uint32_t *cnt) {
    const Tile t = a.tiles[a.tile0 + blockIdx.x];
    if ((int)threadIdx.x >= t.n || !a.st[t.c].active) return;
    const CaseDesc &d = a.desc[t.c];
    const int64_t i = particle_at(a, t.begin + threadIdx.x);
    build_list<T, D>(d, phys<T>(d), i, a.starts, snap, nbr, cnt, &a.st[t.c].status);
}

// ---- G: the stored pair geometry of the list (SPHST_LIST_GEO), once per
// advection step after the list build.  e_ij and W'_ij are formed by the
// same operations as in the list walk, so the sweeps that read them see the
// values they would have computed.
template <typename T, int D, bool LIST>
__global__ void __launch_bounds__(256) k_list_geo(SweepArgs a, const V4<T> *snap, V4<T> *lgeo) {
    const Tile t = a.tiles[a.tile0 + blockIdx.x];
    if ((int)threadIdx.x >= t.n || !a.st[t.c].active) return;
    const CaseDesc &d = a.desc[t.c];
    const CasePhys<T> &cp = phys<T>(d);
    const int64_t i = t.begin + threadIdx.x;
    const V4<T> si = ld4(snap + i);
    if (phase_of(w_bits(si.w)) == PH_WALL) return;
    const int64_t stride = d.p_end - d.p_begin;
    const int64_t off = d.nbr_base + (i - d.p_begin);
    const uint32_t *p = a.nbr + off;
    V4<T> *q = lgeo + off;
    const uint32_t c = a.cnt[i] & CNT_MASK;
    const T cs = cp.cs;
    const KernelGeo<T> kgeo(cp);
    for (uint32_t k = 0; k < c; ++k, p += stride, q += stride) {
        const uint32_t e = ld_list(p);
        const V4<T> sj = ld4(snap + (e >> NBR_SHIFT));
        const L2<T> tt = fma2(neg_code_off2(e & 3u, (e >> 2) & 3u, T()), l2(cs, cs), l2(si.x, si.y));
        const L2<T> rxy = fma2(l2(sj.x, sj.y), l2(T(-1), T(-1)), tt);
        T rz = T(0);
        if (D == 3) rz = sub_rn(fma_rn(-code_off((e >> 4) & 3u, T()), cs, si.z), sj.z);
        const PairGeo<T> g = kgeo(norm2<T, D>(rxy.x, rxy.y, rz));
        const L2<T> exy = mul2(rxy, l2(g.inv_r, g.inv_r));
        const bool wall = phase_of(w_bits(sj.w)) == PH_WALL;
        *q = V4<T>{exy.x, exy.y, D == 3 ? rz * g.inv_r : T(0), wall ? -g.dW : g.dW};
    }
}

template <typename T, int D, bool LIST>
__global__ void SPH_SWEEP_BOUNDS k_sweep_M(SweepArgs a, const V4<T> *snap, const T *drho, V4<T> *bmat,
                                           V4<T> *bk) {
    const Tile t = a.tiles[a.tile0 + blockIdx.x];
    if ((int)threadIdx.x >= t.n || !a.st[t.c].active) return;
    const CaseDesc &d = a.desc[t.c];
    if (!d.tvf_on && d.surface_corr != 1) return;
    const int64_t i = particle_at(a, t.begin + threadIdx.x);
    sweep_M<LIST, T, D>(d, phys<T>(d), i, a.starts, a.nbr, a.cnt, snap, drho, bmat, bk, &a.st[t.c].status);
}

template <typename T, int D, bool LIST>
__global__ void SPH_SWEEP_BOUNDS k_sweep_V(SweepArgs a, const V4<T> *snap, const T *drho, const V4<T> *vel,
                                           const V4<T> *bmat, V4<T> *acc_visc, V4<T> *pos) {
    const Tile t = a.tiles[a.tile0 + blockIdx.x];
    if ((int)threadIdx.x >= t.n || !a.st[t.c].active) return;
    const CaseDesc &d = a.desc[t.c];
    const int64_t i = particle_at(a, t.begin + threadIdx.x);
    sweep_V<LIST, T, D>(d, phys<T>(d), i, a.starts, a.nbr, a.cnt, snap, drho, vel, bmat, acc_visc, pos,
                        &a.st[t.c].status);
}

// Sweeps B and C (and A with the cell walk) take L lanes per particle (L = 1,
// 2, 4, 8; list classes): L blocks share one tile, block b takes its part
// b % L of blockDim / L particles, and lane threadIdx % L of a particle's
// group walks every L-th list entry.  local_index gives the particle's index
// within its tile.  Sweeps S and A of the list classes do the same per entry
// of their band list.
template <int L> __device__ __forceinline__ int local_index(int64_t w) {
    return L == 1 ? (int)threadIdx.x : (int)((w % L) * (blockDim.x / L) + threadIdx.x / L);
}

template <typename T, int D, bool LIST, int L = 1, int MODE = MODE_TILES>
__global__ void SPH_SWEEPAS_BOUNDS k_sweep_A(SweepArgs a, const V4<T> *snap, const T *drho, const V4<T> *lgeo,
                                           V4<T> *gradC) {
    const auto item = [&](int64_t w) {
        const Tile t = work_tile<L, MODE == MODE_WORK>(a, w);
        const int li = local_index<L>(w);
        if (li >= t.n || !a.st[t.c].active) return;
        const CaseDesc &d = case_desc<MODE>(a, t.c);
        const int64_t i = particle_at(a, t.begin + li);
        sweep_A<LIST, T, D, L>(d, phys<T>(d), i, a.starts, a.nbr, a.cnt, snap, drho, lgeo, gradC, threadIdx.x % L);
    };
    if constexpr (MODE == MODE_WORK) {
        const int64_t items = work_items<L, true>(a);
        for (int64_t w = blockIdx.x; w < items; w += gridDim.x) item(w);
    } else {
        item(blockIdx.x);
    }
}

// colour gradient of the band particles (list classes): one thread (L lanes)
// per entry of the class's compacted band list, as in S; the launch's
// threads stride over the list (the grid is a few blocks per SM, since the
// list's length is known only on the device).  A particle outside
// the band has no neighbour of the other fluid, so its colour gradient is the
// zero written at the start of the advection step.
template <typename T, int D, bool LIST, int L = 1>
__global__ void SPH_SWEEPAS_BOUNDS k_sweep_A_band(SweepArgs a, const uint64_t *blist, const uint32_t *bcount,
                                                const V4<T> *snap, const T *drho, V4<T> *gradC) {
    const int64_t items = (int64_t)*bcount * L;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < items; t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t e = blist[t / L];
        const int c = (int)(e >> 32);
        const int64_t i = (int64_t)(uint32_t)e;
        if (!a.st[c].active) continue;
        const CaseDesc &d = a.desc[c];
        sweep_A<LIST, T, D, L>(d, phys<T>(d), i, a.starts, a.nbr, a.cnt, snap, drho, nullptr, gradC, threadIdx.x % L);
    }
}

// surface sum of the band particles (list classes only), before B: one
// thread (L lanes) per entry of the class's compacted band list, so warps
// are full of band particles; the threads stride over the list (a group of
// L lanes stays together: the stride is a multiple of L)
template <typename T, int D, bool LIST, int L = 1>
__global__ void SPH_SWEEPAS_BOUNDS k_sweep_S(SweepArgs a, const uint64_t *blist, const uint32_t *bcount,
                                           const uint8_t *band, const V4<T> *snap, const V4<T> *vel,
                                           const V4<T> *gradC, V4<T> *acc_surf, const V4<T> *bk, const T *drho) {
    const int64_t items = (int64_t)*bcount * L;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < items; t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t e = blist[t / L];
        const int c = (int)(e >> 32);
        const int64_t i = (int64_t)(uint32_t)e;
        if (!a.st[c].active) continue;
        const CaseDesc &d = a.desc[c];
        uint32_t ph;
        sweep_B<LIST, 2, T, D, L>(d, phys<T>(d), T(0), i, a.starts, a.nbr, a.cnt, band, snap, vel, gradC, nullptr,
                                  acc_surf, nullptr, nullptr, &ph, threadIdx.x % L, bk, drho);
    }
}

template <typename T, int D, bool LIST, int L = 1, int MODE = MODE_TILES>
__global__ void SPH_SWEEPB_BOUNDS_M(T, MODE) k_sweep_B(SweepArgs a, const uint8_t *band, const V4<T> *snap, const V4<T> *vel,
                                            const V4<T> *gradC, const V4<T> *acc_visc, V4<T> *acc_surf,
                                            V4<T> *vel_new, const V4<T> *lgeo, const V4<T> *bk) {
    const auto item = [&](int64_t w) {
        const Tile t = work_tile<L, MODE == MODE_WORK>(a, w);
        if (!a.st[t.c].active) return;             // uniform per block
        const CaseDesc &d = case_desc<MODE>(a, t.c);
        double v2 = 0.0;
        uint32_t ph = PH_WALL;
        const int li = local_index<L>(w);
        if (li < t.n) {
            const int64_t i = particle_at(a, t.begin + li);
            const T dt = (T)a.st[t.c].dt;
            v2 = sweep_B<LIST, LIST ? 1 : 0, T, D, L>(d, phys<T>(d), dt, i, a.starts, a.nbr, a.cnt, band, snap, vel,
                                                      gradC, acc_visc, acc_surf, vel_new, lgeo, &ph, threadIdx.x % L,
                                                      LIST ? nullptr : bk);
        }
        unsigned long long m0 = ph == 0 ? (unsigned long long)__double_as_longlong(v2) : 0ull;
        unsigned long long m1 = ph == 1 ? (unsigned long long)__double_as_longlong(v2) : 0ull;
        m0 = warp_max_u64(m0);
        m1 = warp_max_u64(m1);
        if ((threadIdx.x & 31) == 0) {
            if (m0) atomicMax(&a.st[t.c].vmax2_acc[0], m0);
            if (m1) atomicMax(&a.st[t.c].vmax2_acc[1], m1);
        }
    };
    if constexpr (MODE == MODE_WORK) {
        const int64_t items = work_items<L, true>(a);
        for (int64_t w = blockIdx.x; w < items; w += gridDim.x) item(w);
    } else {
        item(blockIdx.x);
    }
}

template <typename T, int D, bool LIST, int L = 1, int MODE = MODE_TILES>
__global__ void SPH_SWEEP_BOUNDS k_sweep_C(SweepArgs a, const V4<T> *snap, const V4<T> *vel_new, T *drho,
                                           V4<T> *vel, V4<T> *pos, const V4<T> *lgeo) {
    const auto item = [&](int64_t w) {
        const Tile t = work_tile<L, MODE == MODE_WORK>(a, w);
        const int li = local_index<L>(w);
        if (li >= t.n || !a.st[t.c].active) return;
        const CaseDesc &d = case_desc<MODE>(a, t.c);
        const int64_t i = particle_at(a, t.begin + li);
        const T dt = (T)a.st[t.c].dt;
        sweep_C<LIST, T, D, L>(d, phys<T>(d), dt, i, a.starts, a.nbr, a.cnt, snap, vel_new, drho, vel, pos, lgeo,
                               threadIdx.x % L);
    };
    if constexpr (MODE == MODE_WORK) {
        const int64_t items = work_items<L, true>(a);
        for (int64_t w = blockIdx.x; w < items; w += gridDim.x) item(w);
    } else {
        item(blockIdx.x);
    }
}

// ---- work lists of the per-substep sweeps in a batch: after the criterion
// kernel has set each case's active flag, the fluid tiles of the active
// cases are listed per class.  Scan (one block): case c's tiles go to
// positions off[c] .. off[c] + ftn[c] - 1 of its class's list, and
// count[k] receives the length of class k's list.  Fill: every fluid tile of
// an active case writes its index there.  Tiles of class k start at cls0[k]
// in the tile array and in the list alike.
static __global__ void k_work_scan(int ncases, const int32_t *cls_of, const uint32_t *ftn, const CaseState *st,
                                   uint32_t *off, uint32_t *count) {
    uint32_t base[4] = {0u, 0u, 0u, 0u};
    for (int c0 = 0; c0 < ncases; c0 += (int)blockDim.x) {
        const int c = c0 + (int)threadIdx.x;
        const int k = c < ncases ? cls_of[c] : -1;
        const uint32_t n = c < ncases && st[c].active ? ftn[c] : 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t total;
            const uint32_t before = block_exclusive_scan(k == q ? n : 0u, &total);
            if (k == q) off[c] = base[q] + before;
            base[q] += total;
        }
    }
    if (threadIdx.x < 4) count[threadIdx.x] = base[threadIdx.x];
}
static __global__ void k_work_fill(int64_t n_ftiles, const Tile *ftiles, const int64_t *ft_first,
                                   const int64_t *cls0, const int32_t *cls_of, const uint32_t *off,
                                   const CaseState *st, uint32_t *work) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_ftiles) return;
    const int c = ftiles[t].c;
    if (!st[c].active) return;
    work[cls0[cls_of[c]] + off[c] + (t - ft_first[c])] = (uint32_t)t;
}

// ---------------------------------------------------------- diagnostics
// FP64 sums over one case's fluid particles: per-block partials (warp
// shuffles, then the block's warps in order), then one block adds the
// partials in block order, so the result does not depend on scheduling.
// Quantities: 0-2 momentum, 3 kinetic, 4-5 count per phase, 6-8 first
// moments, 9-14 second moments, 15 p_in, 16 p_out, 17 n_in, 18 n_out,
// 19 non-finite count.

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(256) k_diag_partial(const CaseDesc *desc, int c, const V4<T> *pos,
                                                      const V4<T> *vel, const T *drho, double cx, double cy,
                                                      double cz, double r_in2, double r_out2, double *partial) {
    const CaseDesc &d = desc[c];
    const int64_t n = d.p_end - d.p_begin;
    const int dim = d.dim;
    double q[DIAG_Q];
#pragma unroll
    for (int k = 0; k < DIAG_Q; ++k) q[k] = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = d.p_begin + k;
        const V4<T> p = pos[i];
        const uint32_t pk = w_bits(p.w);
        const uint32_t ph = phase_of(pk);
        if (ph > 1) continue;
        const int cc[3] = {dim == 3 ? cell_x<3>(pk) : cell_x<2>(pk), dim == 3 ? cell_y<3>(pk) : cell_y<2>(pk),
                           dim == 3 ? cell_z<3>(pk) : 0};
        const double off[3] = {(double)p.x, (double)p.y, (double)p.z};
        double x[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < dim; ++a) x[a] = d.origin[a] + (double)cc[a] * d.cs + off[a];
        const V4<T> v4 = vel[i];
        const double v[3] = {(double)v4.x, (double)v4.y, dim == 3 ? (double)v4.z : 0.0};
        const double dr = (double)drho[i];
        const double m = d.pd.mass[ph];
        const bool finite = isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]) && isfinite(v[0]) &&
                            isfinite(v[1]) && isfinite(v[2]) && isfinite(dr);
        if (!finite) { q[19] += 1.0; continue; }
        q[0] += m * v[0]; q[1] += m * v[1]; q[2] += m * v[2];
        q[3] += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        q[4 + ph] += 1.0;
        const double rx = x[0] - cx, ry = x[1] - cy, rz = dim == 3 ? x[2] - cz : 0.0;
        const double r2 = rx * rx + ry * ry + rz * rz;
        const double pr = d.c0 * d.c0 * dr;
        if (ph == 0) {
            q[6] += x[0]; q[7] += x[1]; q[8] += x[2];
            q[9] += x[0] * x[0]; q[10] += x[1] * x[1]; q[11] += x[2] * x[2];
            q[12] += x[0] * x[1]; q[13] += x[0] * x[2]; q[14] += x[1] * x[2];
            if (r2 < r_in2) { q[15] += pr; q[17] += 1.0; }
        } else if (r2 > r_out2) {
            q[16] += pr; q[18] += 1.0;
        }
    }
    __shared__ double sh[8][DIAG_Q];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < DIAG_Q; ++k) {
        const double t = warp_sum_d(q[k]);
        if (lane == 0) sh[w][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < DIAG_Q) {
        double t = 0.0;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t += sh[ww][threadIdx.x];
        partial[(int64_t)blockIdx.x * DIAG_Q + threadIdx.x] = t;
    }
}

static __global__ void k_diag_final(const double *partial, int nblocks, double *out) {
    if (threadIdx.x < DIAG_Q) {
        double t = 0.0;
        for (int b = 0; b < nblocks; ++b) t += partial[(int64_t)b * DIAG_Q + threadIdx.x];
        out[threadIdx.x] = t;
    }
}

// ------------------------------------------------------------ read-back
// field values of one case into a device buffer in insertion order (FP64)
template <typename T>
__global__ void k_read_field(const CaseDesc *desc, int c, int field, const V4<T> *pos,
                             const V4<T> *vel, const T *drho, const V4<T> *gradC,
                             const V4<T> *acc_visc, const uint32_t *id, double *out) {
    const CaseDesc &d = desc[c];
    const int64_t n = d.p_end - d.p_begin;
    const int dim = d.dim;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = d.p_begin + k;
        const int64_t o = id[i];
        const V4<T> p = pos[i];
        const uint32_t pk = w_bits(p.w);
        const uint32_t ph = phase_of(pk);
        switch (field) {
        case 0: {
            const int cc[3] = {dim == 3 ? cell_x<3>(pk) : cell_x<2>(pk),
                               dim == 3 ? cell_y<3>(pk) : cell_y<2>(pk),
                               dim == 3 ? cell_z<3>(pk) : 0};
            const double off[3] = {(double)p.x, (double)p.y, (double)p.z};
            for (int a = 0; a < dim; ++a)
                out[o * dim + a] = d.origin[a] + (double)cc[a] * d.cs + off[a];
            break;
        }
        case 1: {
            const V4<T> v = vel[i];
            const double vv[3] = {(double)v.x, (double)v.y, (double)v.z};
            for (int a = 0; a < dim; ++a) out[o * dim + a] = vv[a];
            break;
        }
        case 2: out[o] = ph < 2 ? d.rho0[ph] + (double)drho[i] : d.rho0[0]; break;
        case 3: out[o] = ph < 2 ? d.c0 * d.c0 * (double)drho[i] : 0.0; break;
        case 5: {
            const V4<T> g = gradC[i];
            const double gg[3] = {(double)g.x, (double)g.y, (double)g.z};
            for (int a = 0; a < dim; ++a) out[o * dim + a] = gg[a];
            break;
        }
        case 6: {
            const V4<T> g = acc_visc[i];
            const double gg[3] = {(double)g.x, (double)g.y, (double)g.z};
            for (int a = 0; a < dim; ++a) out[o * dim + a] = gg[a];
            break;
        }
        default: break;
        }
    }
}

// Morton key (from the packed cell of the last rebuild) and insertion id of
// every particle of case c in device order
template <typename T>
__global__ void k_debug_keys(const CaseDesc *desc, int c, const V4<T> *snap, const uint32_t *id,
                             unsigned long long *keys, long long *ids) {
    const CaseDesc &d = desc[c];
    const int64_t n = d.p_end - d.p_begin;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = d.p_begin + k;
        const uint32_t pk = w_bits(snap[i].w);
        keys[k] = d.dim == 3 ? morton_of_packed<3>(pk) : morton_of_packed<2>(pk);
        ids[k] = id[i];
    }
}

template <typename T, int D>
__device__ void count_nbrs(const CaseDesc &d, int64_t i, const uint32_t *starts, const V4<T> *snap,
                           const uint32_t *id, int *out) {
    const V4<T> si = ld4(snap + i);
    int cnt = 0;
    walk<T, D>(d, phys<T>(d), starts, snap, i, si, w_bits(si.w),
               [&](uint32_t, const V4<T> &, T, T, T, T) { ++cnt; });
    out[id[i]] = cnt;
}

template <typename T>
__global__ void k_debug_counts(const CaseDesc *desc, int c, const uint32_t *starts,
                               const V4<T> *snap, const uint32_t *id, int *out) {
    const CaseDesc &d = desc[c];
    const int64_t n = d.p_end - d.p_begin;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (d.dim == 3) count_nbrs<T, 3>(d, d.p_begin + k, starts, snap, id, out);
    else count_nbrs<T, 2>(d, d.p_begin + k, starts, snap, id, out);
}

}  // namespace sphst
