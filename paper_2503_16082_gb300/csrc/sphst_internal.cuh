// sphst_internal.cuh -- device data model of the pair-sweep library.
//
// Particles of all cases that share an engine live in one set of SoA arrays
// (structure of arrays), each case in a contiguous range, ordered by
// (case, Morton cell code, insertion index) after every rebuild.  Positions
// are stored relative to the origin of the particle's cell at the last
// rebuild, so FP32 keeps ~1e-7 of the cell width instead of ~1e-7 of the
// domain size; the cell coordinates and the phase are packed into the fourth
// component of the position vector.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sphst {

// SPHST_LIST_GEO 1: with the neighbour list, the pair geometry of the frozen
// configuration (unit vector e_ij and kernel derivative W'_ij) is computed
// once per advection step and stored beside the list; the per-substep
// sweeps A, B and C stream it instead of recomputing it from positions.
// Measured on the 3D drop (1.19M particles): sweep B 0.36 -> 0.41-0.45 ms,
// sweep C 0.30 -> 0.38-0.43 ms, rebuild +0.5 ms.  The 20 bytes per pair come
// from HBM with its latency, the recomputation from positions that hit in
// L1; off.
#ifndef SPHST_LIST_GEO
#define SPHST_LIST_GEO 0
#endif

// ------------------------------------------------------------------ vectors
template <typename T> struct V4;
template <> struct __align__(16) V4<float> { float x, y, z, w; };
template <> struct __align__(16) V4<double> { double x, y, z, w; };

// packed cell coordinates + phase code in the w slot
// 3D: bits 0-9 x, 10-19 y, 20-29 z; 2D: bits 0-14 x, 15-29 y; bits 30-31 phase
// The dimension is a template parameter everywhere bits are packed or
// interleaved, so every mask and shift is a compile-time constant (a variant
// that chose the 2D or 3D pattern at run time was miscompiled for sm_103a).
constexpr uint32_t PH_FLUID0 = 0, PH_FLUID1 = 1, PH_WALL = 2;

template <int D> __host__ __device__ inline uint32_t pack_cell(int cx, int cy, int cz, uint32_t ph) {
    if (D == 3) return (uint32_t)cx | ((uint32_t)cy << 10) | ((uint32_t)cz << 20) | (ph << 30);
    (void)cz;
    return (uint32_t)cx | ((uint32_t)cy << 15) | (ph << 30);
}
template <int D> __host__ __device__ inline int cell_x(uint32_t p) { return D == 3 ? (int)(p & 0x3ffu) : (int)(p & 0x7fffu); }
template <int D> __host__ __device__ inline int cell_y(uint32_t p) { return D == 3 ? (int)((p >> 10) & 0x3ffu) : (int)((p >> 15) & 0x7fffu); }
template <int D> __host__ __device__ inline int cell_z(uint32_t p) { return D == 3 ? (int)((p >> 20) & 0x3ffu) : 0; }
__host__ __device__ inline uint32_t phase_of(uint32_t p) { return p >> 30; }

__device__ inline uint32_t w_bits(float w) { return __float_as_uint(w); }
__device__ inline uint32_t w_bits(double w) { return (uint32_t)__double_as_longlong(w); }
__device__ inline float bits_w(uint32_t b, float) { return __uint_as_float(b); }
__device__ inline double bits_w(uint32_t b, double) { return __longlong_as_double((long long)b); }

// Morton interleave by bit spreading (axis 0 in the lowest bit)
__host__ __device__ inline uint32_t spread_by_3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__host__ __device__ inline uint32_t spread_by_2(uint32_t v) {
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
template <int D> __host__ __device__ inline uint32_t morton(int cx, int cy, int cz) {
    if (D == 3)
        return spread_by_3((uint32_t)cx) | (spread_by_3((uint32_t)cy) << 1) | (spread_by_3((uint32_t)cz) << 2);
    (void)cz;
    return spread_by_2((uint32_t)cx) | (spread_by_2((uint32_t)cy) << 1);
}
template <int D> __host__ __device__ inline uint32_t morton_of_packed(uint32_t p) {
    return morton<D>(cell_x<D>(p), cell_y<D>(p), cell_z<D>(p));
}

// ------------------------------------------------------- per-case constants
// Problem statement of one case, in both precisions; read-only on device.
template <typename T> struct CasePhys {
    T h, inv_h, four_h2;       // smoothing length, 1/h, (2h)^2
    T kcoef;                   // dW/dr = kcoef * q (1 - q/2)^3, kcoef = -5 alpha_d / h
    T cs;                      // cell width
    T c0, c0sq, inv_c0, gamma, xi;
    T rho0[2], eta[2], mass[2];
    T two_phi[2];              // 2 phi_i of a cross-phase pair, i in fluid k (Eq. 23)
    T four_phi_phi;            // 4 phi_i phi_j of a cross-phase pair
    T vol_wall;                // dp^dim
    T nhat_eps;                // |gradC| h threshold of an interface particle
    T tvf_coef;                // -alpha h^2 (Eq. 14, sign reading)
    T beta_k, beta_lo, beta_hi; // Eq. 11 limiter as min(max(beta_k dU, lo), hi) per reading
};

struct CaseDesc {
    int32_t dim;
    int32_t limiter, grad_mode, penalty_form;
    int32_t penalty_scope;     // 1: the same-phase line of Eq. 33 carries no penalty
    int32_t wall_form;         // 1: wall pairs use max(P*, 0) (no suction)
    int32_t stress_weights;    // 1: cross-phase line 2 phi_i Pi_i + 2 phi_j Pi_j
    int32_t surface_corr;      // 1: same-phase line with the own-fluid corrected gradient
    int32_t n_fluid_phases;
    int32_t bits;              // Morton bits per axis of the cell table
    int32_t ncell[3];
    int32_t tvf_on;
    int64_t p_begin, p_end;    // particle range in the engine arrays
    int64_t table_off;         // first cell-table entry of this case
    int64_t table_size;        // 2^(dim*bits)
    int32_t periodic;          // bit a: axis a wraps (ncell[a] cells of width cs tile the period)
    int32_t vstar_printed;     // Eq. 8's v* as printed (else: normal component -U*)
    double period_len[3];      // period of each periodic axis
    double origin[3];
    double cs;
    double h, c0, gamma;
    double rho0[2], eta[2];
    int64_t max_substeps;
    double cfl_ad, cfl_ac;
    double dt_surf[2];         // the surface-tension bound of Eq. 17 per fluid (0: none)
    int32_t nbr_mode;          // 0: neighbour list built per advection step; 1: cell walk
    int32_t nbr_k;             // list capacity per particle
    int64_t nbr_base;          // first list word of this case
    CasePhys<float> pf;
    CasePhys<double> pd;
};

template <typename T> __device__ inline const CasePhys<T> &phys(const CaseDesc &d);
template <> __device__ inline const CasePhys<float> &phys<float>(const CaseDesc &d) { return d.pf; }
template <> __device__ inline const CasePhys<double> &phys<double>(const CaseDesc &d) { return d.pd; }

// mutable per-case time-stepping state (device)
struct CaseState {
    double dt_ad;              // current advection step length
    double t_in;               // time covered inside the advection step
    double dt;                 // current acoustic substep
    double t;                  // physical time
    double last_dt_ac;
    unsigned long long vmax2_acc[2];   // bits of max |v|^2 (FP64) accumulated by the kick
    unsigned long long vmax2_cur[2];   // value used by the current substep's criterion
    int32_t active;            // inside an advection step with substeps left
    int32_t last;              // the current substep ends the advection step
    int32_t status;            // 0 ok, else DEV_ERR_*
    int32_t present[2];        // fluid phase has particles
    int32_t pad_;
    int64_t n_sub, n_adv, n_sub_adv;
};

enum : int32_t { DEV_OK = 0, DEV_ERR_NONFINITE = 1, DEV_ERR_DOMAIN = 2, DEV_ERR_COINCIDENT = 3,
                 DEV_ERR_STALLED = 4, DEV_ERR_NBR_OVERFLOW = 5 };

struct Tile { int32_t c; int32_t n; int64_t begin; };   // one block: n particles of case c

// diagnostics: quantities per reduction and maximum partial blocks
constexpr int DIAG_Q = 20;
constexpr int DIAG_BLOCKS = 1024;

}  // namespace sphst
