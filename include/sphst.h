/*
 * sphst.h -- C ABI of the GB300 pair-sweep library for the Riemann-based
 * multiphase SPH scheme with momentum-conserving surface tension and the
 * zero-surface-energy penalty force (Zhang, Lourenco & Hu, arXiv 2503.16082).
 *
 * The problem statement follows Sections 2-3 of the paper: two immiscible
 * weakly compressible fluids, each with a reference density rho0 and a
 * dynamic viscosity eta, one surface tension coefficient gamma for their
 * interface, one artificial sound speed c0 for all phases (Eq. 3), the
 * Wendland C2 kernel with smoothing length h = 1.3 dp (Section 5) and no-slip
 * walls.  One call of sphst_step advances whole advection steps of the
 * dual-criteria time stepping (Section 3.3, Eqs. 16-18); each advection step
 * runs as many acoustic substeps as its length needs, all on the GPU.
 *
 * Conventions for every entry point:
 *   - the return value is a status code: SPHST_OK (0) or a negative error;
 *     sphst_last_error() then describes the failure (thread-local text);
 *   - pointers named pos/vel/rho/dst are HOST pointers; arrays of vectors are
 *     row-major with `dim` doubles per particle (x, y[, z]);
 *   - input arrays are copied; the caller keeps ownership of its buffers;
 *   - a case or batch handle is owned by the caller and released with the
 *     matching destroy call; destroy functions accept NULL;
 *   - calls on one handle must not run concurrently (one host thread per
 *     case or batch, or the caller serialises);
 *   - all device memory is allocated and freed by the library on the current
 *     CUDA device at the first step of a case (or of a batch).
 */
#ifndef SPHST_H
#define SPHST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define SPHST_OK               0
#define SPHST_ERR_INVALID_ARG (-1)   /* a NULL handle, bad size or bad value      */
#define SPHST_ERR_STATE       (-2)   /* call not allowed in the current state     */
#define SPHST_ERR_UNSUPPORTED (-3)   /* third fluid, dim not 2/3, grid too large  */
#define SPHST_ERR_OOM         (-4)   /* device allocation failed                  */
#define SPHST_ERR_CUDA        (-5)   /* a CUDA runtime call failed                */
#define SPHST_ERR_NONFINITE   (-6)   /* NaN/Inf velocity or time step in a case   */
#define SPHST_ERR_TIMEOUT     (-7)   /* reserved: a bounded device wait gave up   */
#define SPHST_ERR_OVER_BUDGET (-8)   /* batch admission beyond the memory budget  */
#define SPHST_ERR_DOMAIN      (-9)   /* a particle left the cell grid             */
#define SPHST_ERR_COINCIDENT (-10)   /* two particles at the same position        */
#define SPHST_ERR_STALLED    (-11)   /* advection step exceeded max_substeps      */
#define SPHST_ERR_CAPACITY   (-12)   /* destination buffer too small              */
#define SPHST_ERR_NEIGHBORS  (-13)   /* a particle has more neighbours than max_neighbors */

/* --------------------------------------------------------- particle kinds */
#define SPHST_FLUID 0
#define SPHST_WALL  1

/* ------------------------------------------------------------ readings    */
/* Eq. 11 dissipation limiter of the momentum Riemann solver.  DENSITY: the
 * printed (P_L + P_R) is read as (rho_L + rho_R), which makes beta
 * dimensionless; with one sound speed beta = min(3 max((U_L-U_R)/c0, 0), 1). */
#define SPHST_LIMITER_DENSITY 0
#define SPHST_LIMITER_NONE    1      /* beta = 1: full acoustic dissipation  */
#define SPHST_LIMITER_ZERO    2      /* beta = 0: P* is the pair average     */
#define SPHST_LIMITER_PRINTED 3      /* (P_L + P_R) kept as printed          */
/* Eq. 28 average colour gradient of a pair of different phases: COMMON takes
 * j's colour on i's side, (gradC_i - gradC_j)/2; PRINTED is (gradC_i + gradC_j)/2 */
#define SPHST_GRAD_COMMON  0
#define SPHST_GRAD_PRINTED 1
/* Eq. 30 with A = gradCbar (x) r_ij: NN contracts (A/|A|) A as A A^T/|A|
 * (= |gradCbar| r_ij nbar nbar^T); EE as A^T A/|A| (= |gradCbar| r_ij e e^T) */
#define SPHST_PENALTY_NN 0
#define SPHST_PENALTY_EE 1
/* the scalar C_ij - gradCbar . r_ij of Eq. 29 (the paper's first penalty,
 * which it notes does not conserve momentum), for ablation */
#define SPHST_PENALTY_SCALAR 2
/* which lines of Eq. 33 carry the penalty: BOTH as printed; CROSS_ONLY drops
 * it from the same-phase line and keeps it on the cross-phase line (an
 * ablation) */
#define SPHST_PENALTY_SCOPE_BOTH       0
#define SPHST_PENALTY_SCOPE_CROSS_ONLY 1
/* wall pairs of the pressure force (no wall model in the paper; Eqs. 8-11
 * with the mirror state rho_i, p_i, 2 U_w - U_L): MIRROR uses P* as it
 * comes, so a fluid particle in tension (p_i < 0) is pulled towards the
 * wall; NO_SUCTION takes max(P*, 0), so walls push and never pull */
#define SPHST_WALL_MIRROR     0
#define SPHST_WALL_NO_SUCTION 1
/* weights of the two surface stresses on the cross-phase line of Eqs. 26 and
 * 33 (i in fluid k, j in fluid l): PRINTED 2 phi_j Pi_i + 2 phi_i Pi_j as
 * printed; OWN 2 phi_i Pi_i + 2 phi_j Pi_j, each stress weighted by its own
 * particle's phi (Eq. 23); both conserve momentum and agree at density
 * ratio 1 */
#define SPHST_STRESS_PRINTED 0
#define SPHST_STRESS_OWN     1
/* kernel gradient of the same-phase line of Eq. 33: PRINTED grad_i W_ij;
 * OWN_FLUID (B^k_i + B^k_j)/2 grad_i W_ij with B^k the correction matrix of
 * Eq. 15 summed over the particle's own fluid (formed once per advection
 * step), so that each fluid's stress divergence stays first-order consistent
 * up to the interface */
#define SPHST_SURFACE_CORR_PRINTED   0
#define SPHST_SURFACE_CORR_OWN_FLUID 1
/* Eq. 8's star velocity: CORRECTED takes the normal component as -U* along
 * e_ij (U = -v.e_ij, Eq. 10) and the tangential part of the pair average;
 * PRINTED is U* e_ij + (vbar - Ubar e_ij) as printed */
#define SPHST_VSTAR_CORRECTED 0
#define SPHST_VSTAR_PRINTED   1
/* acoustic substep loop: GRAPH runs it as a device-driven while loop inside a
 * CUDA graph (no host round trip per substep); HOST polls a device flag after
 * every substep */
#define SPHST_LOOP_GRAPH 0
#define SPHST_LOOP_HOST  1
/* how the sweeps find neighbours: LIST builds a neighbour list of the frozen
 * configuration once per advection step (Section 3.3) and every substep's
 * sweeps read it; CELLS walks the 3^d cells around each particle every time.
 * Both find the same neighbours; the list holds those of the other fluid
 * first, each part in increasing particle index, so the sums are the same
 * terms in another order and agree to rounding. */
#define SPHST_NBR_LIST  0
#define SPHST_NBR_CELLS 1

/* ------------------------------------------------------------- fields     */
#define SPHST_FIELD_POS      0   /* n x dim positions                            */
#define SPHST_FIELD_VEL      1   /* n x dim velocities                           */
#define SPHST_FIELD_RHO      2   /* n densities (walls: their fluid partner's)   */
#define SPHST_FIELD_PRESSURE 3   /* n pressures c0^2 (rho - rho0), Eq. 3          */
#define SPHST_FIELD_PHASE    4   /* n phase ids as returned by add_phase_particles */
#define SPHST_FIELD_GRADC    5   /* n x dim colour gradient of the last substep  */
#define SPHST_FIELD_ACC_VISC 6   /* n x dim viscous acceleration of the last advection step */

typedef struct sphst_case_s *sphst_case;
typedef struct sphst_batch_s *sphst_batch;

typedef struct {
    int32_t dim;            /* 2 or 3                                          */
    int32_t precision;      /* 32: FP32 pair arithmetic, FP64 reductions; 64   */
    double  dx;             /* initial particle spacing dp (> 0)               */
    double  h_factor;       /* h = h_factor * dx; the paper uses 1.3           */
    double  c0;             /* artificial sound speed, one for all phases      */
    double  gamma;          /* surface tension coefficient (>= 0)              */
    double  xi;             /* penalty coefficient; < 0: 1.3 n + 0.6 for a
                               density ratio 10^n (Section 4.2)               */
    double  tvf_alpha;      /* transport-velocity coefficient (Section 3.2,
                               0.2); 0 switches the position shift off         */
    int32_t limiter;        /* SPHST_LIMITER_*                                 */
    int32_t grad_mode;      /* SPHST_GRAD_*                                    */
    int32_t penalty_form;   /* SPHST_PENALTY_*                                 */
    int32_t loop_mode;      /* SPHST_LOOP_*                                    */
    int32_t grid_pad;       /* spare cells around the initial bounding box (>= 1) */
    int32_t block;          /* threads per block of the pair sweeps: a multiple
                               of 32 in 32..256                                */
    int64_t max_substeps;   /* per advection step before SPHST_ERR_STALLED     */
    double  cfl_ad;         /* factor of the advection criterion, Eq. 16 (0.1) */
    double  cfl_ac;         /* factor of the acoustic criterion, Eq. 17 (0.6);
                               a density-ratio-1000 interface bound by the
                               sound term needs <= 0.5 (2D) / 0.4 (3D)        */
    int32_t nbr_mode;       /* SPHST_NBR_*                                     */
    int32_t max_neighbors;  /* list capacity per particle; 0: 128 (3D), 48 (2D) */
    int32_t periodic;       /* bit a set: axis a is periodic on [period_lo[a],
                               period_hi[a]) (the shear drop of Section 5.2 is
                               periodic in x).  Pairs use the minimum image and
                               particles leaving one end re-enter at the other.
                               A periodic axis of length L holds
                               m = floor(L / (2h (1 + 2^-16))) >= 3 cells of
                               width L / m; every periodic axis must give the
                               same width (else INVALID_ARG).  0: none         */
    int32_t vstar_form;     /* SPHST_VSTAR_* (continuity, Eq. 6)               */
    double  period_lo[3];
    double  period_hi[3];
    int32_t lanes;          /* lanes per particle in the per-substep sweeps
                               (colour gradient, pressure, continuity) with
                               the neighbour list: 1, 2, 4 or 8; the surface
                               sweep over the interface band takes at least 2.  With L > 1
                               the L lanes of a particle split its list and
                               add their partial sums (fixed order, so runs
                               repeat bit for bit; results differ from L = 1
                               by the rounding of the reordered sum).  More
                               lanes spread small cases over more of the GPU.
                               Speed only; a batch uses its first case's
                               value.                                        */
    int32_t penalty_scope;  /* SPHST_PENALTY_SCOPE_*                           */
    int32_t wall_form;      /* SPHST_WALL_* (pressure of wall pairs)           */
    int32_t work_lists;     /* batches only (the first case's value counts):
                               0 (default): every substep launches one block
                               (L blocks) per tile of every member, and the
                               tiles of members whose advection step has
                               ended return at once; 1: after each
                               substep's criterion the tiles of the active
                               members are listed per class and the sweeps'
                               blocks stride over that list.  Speed only:
                               both give the same bits.                      */
    int32_t stress_weights; /* SPHST_STRESS_* (cross-phase surface stress)     */
    int32_t surface_corr;   /* SPHST_SURFACE_CORR_* (same-phase surface line)  */
} sphst_case_params;

typedef struct {
    int32_t kind;           /* SPHST_FLUID or SPHST_WALL                       */
    int32_t pad_;
    double  rho0;           /* fluid: reference density (> 0)                  */
    double  eta;            /* fluid: dynamic viscosity (> 0)                  */
    double  wall_vel[3];    /* wall: prescribed velocity of its particles      */
} sphst_phase_props;

typedef struct {
    int64_t n_adv;          /* advection steps completed since creation        */
    int64_t n_sub;          /* acoustic substeps completed since creation      */
    double  t;              /* physical time reached                           */
    double  last_dt_ad;     /* length of the last advection step (Eq. 16/18)   */
    double  last_dt_ac;     /* last acoustic criterion (Eq. 17/18)             */
    int32_t status;         /* SPHST_OK or the case's sticky error code        */
    int32_t pad_;
} sphst_step_info;

/* Fill *p with the defaults: dim 2, precision 32, h_factor 1.3, c0 10,
 * gamma 1, xi -1 (derived), tvf_alpha 0.2, readings 0, graph loop,
 * grid_pad 2, block 128, lanes 1, max_substeps 1000000, cfl_ad 0.1, cfl_ac 0.6,
 * neighbour lists with the default capacity; dx must still be set. */
void sphst_default_params(sphst_case_params *p);

/* Create an empty case from the problem statement of Sections 2-3.
 * Errors: INVALID_ARG (dx <= 0, c0 <= 0, gamma < 0, bad flags),
 * UNSUPPORTED (dim not 2 or 3, precision not 32 or 64). */
int sphst_create_case(const sphst_case_params *params, sphst_case *out);

/* Add n particles of one phase.  pos: n x dim, copied.  vel: n x dim or
 * NULL for rest (ignored for walls, which move with wall_vel).  rho: n
 * initial densities or NULL for rho0 (fluids; used to resume a case).  Each
 * particle's mass is rho0 dp^dim and stays fixed.  *phase_id_out (optional)
 * receives 0, 1, 2... in call order.  Allowed only before the first step.
 * Errors: STATE after the first step, UNSUPPORTED for a third fluid phase,
 * INVALID_ARG for n < 0, NULL pos with n > 0, rho0/eta <= 0. */
int sphst_add_phase_particles(sphst_case c, const sphst_phase_props *props, int64_t n,
                              const double *pos, const double *vel, const double *rho,
                              int32_t *phase_id_out);

/* Advance n_adv advection steps (Section 3.3).  Per advection step, on the
 * device: the advection criterion from the FP64 maximum speed per fluid; the
 * cell list rebuild (Morton cell keys, counting sort, reorder) that freezes
 * the particle configuration; the viscous acceleration (Eq. 13) and the
 * transport-velocity shift (Eqs. 14-15); then acoustic substeps, each with
 * the acoustic criterion (Eq. 17), the colour gradient (Eq. 22), the
 * pressure (Eqs. 7-12), surface (Eqs. 24, 26, 33) and viscous accelerations
 * and a velocity kick, continuity (Eq. 6) and the position drift.  info
 * (optional) receives the case totals.  A case whose device status turns
 * non-zero stops where it failed and keeps returning that error; its fields
 * stay readable.  Errors: STATE (case is a batch member), NONFINITE, DOMAIN,
 * COINCIDENT, STALLED, NEIGHBORS, OOM, CUDA, UNSUPPORTED (cell grid too
 * large, or more than 2^26 particles in one engine with neighbour lists). */
int sphst_step(sphst_case c, int64_t n_adv, sphst_step_info *info);

/* Copy one field, in insertion order and FP64 whatever the internal
 * precision, into the caller's host buffer dst of capacity doubles (the
 * field needs n or n x dim doubles, n = all particles incl. walls).
 * Before the first step the staged input is returned.  Errors: INVALID_ARG
 * (unknown field), CAPACITY (buffer too small), CUDA. */
int sphst_read_fields(sphst_case c, int32_t field, double *dst, int64_t capacity);

/* Case totals (n_adv, n_sub, t, last criteria, status) without stepping. */
int sphst_case_info(sphst_case c, sphst_step_info *info);

/* Particle counts: all particles and fluid particles. */
int sphst_num_particles(sphst_case c, int64_t *n_total, int64_t *n_fluid);

/* Release a case and its device memory.  A batch member must be removed
 * from its batch first (else STATE).  NULL is accepted. */
int sphst_destroy(sphst_case c);

/* Text of the last error on the calling thread ("" if none). */
const char *sphst_last_error(void);

/* ------------------------------------------------------ inspection calls */
/* Cell grid of a stepped case: origin (3 doubles), cell width (2h(1+2^-16))
 * and cells per axis (3 ints, 1 for unused axes). */
int sphst_debug_grid(sphst_case c, double *origin3, double *cell_size, int32_t *ncell3);

/* Cell keys of the last rebuild in the device's particle order: keys[k] is
 * the Morton code of the k-th particle's cell and ids[k] its insertion index
 * (the order sorts by (key, insertion index)).  capacity counts entries. */
int sphst_debug_keys(sphst_case c, uint64_t *keys, int64_t *ids, int64_t capacity);

/* Number of neighbours (0 < r_ij < 2h) of each particle at the last rebuild,
 * in insertion order (walls included). */
int sphst_debug_neighbor_counts(sphst_case c, int32_t *counts, int64_t capacity);

/* Run the case's kernels on the caller's CUDA stream (a cudaStream_t passed
 * as void*, e.g. torch.cuda.current_stream().cuda_stream) instead of a
 * library-owned stream.  Must be called before the first step; NULL keeps
 * the library's own stream.  The caller keeps ownership of the stream. */
int sphst_set_stream(sphst_case c, void *cuda_stream);

/* Advance one advection step with every kernel launched on its own (no
 * graph) and bracketed by CUDA events on the case's stream.  kernel_ms[k]
 * receives the summed device time of kernel group k and launches[k] its
 * launch count, for k = 0 rebuild (keys, scan, sort, gather, neighbour
 * list, interface band), 1 set-up (speed reduction, criteria, correction
 * matrix, viscous + shift), 2 criterion per substep, 3 sweep A (colour
 * gradient), 4 sweep B (pressure + kick), 5 sweep C (continuity + drift),
 * 6 sweep S (surface sum of the interface band; neighbour-list cases only).
 * Both arrays hold SPHST_PROFILE_GROUPS entries.  The step is a normal step
 * of the case. */
#define SPHST_PROFILE_GROUPS 7
int sphst_profile_step(sphst_case c, double *kernel_ms, int64_t *launches);

/* Cell order without allocating (the paper has no counterpart: this serves
 * callers that may not allocate device memory -- a framework whose memory
 * pool owns every allocation, or a real-time caller that must not allocate
 * after start-up).  It computes what one rebuild computes for the particle
 * order: for n particles at pos_dev (DEVICE pointer, n x 3 doubles, the
 * unused coordinate of 2D ignored) on the grid (origin3, cell_size, ncell3;
 * origin3 and ncell3 are HOST arrays of 3 entries, the third ignored in 2D,
 * as returned by sphst_debug_grid), keys_dev[k] receives the Morton code of
 * the k-th particle in canonical order and order_dev[k] its index in pos_dev
 * (the order sorts by (Morton code, index)).  The grid is non-periodic: a
 * position outside it (also one on the far end of a periodic axis, which
 * the rebuild itself would wrap) is clamped into the nearest cell and
 * reported as DOMAIN.  keys_dev and order_dev are DEVICE buffers of n
 * entries owned by the caller; cuda_stream (a cudaStream_t as void*, NULL
 * for the default stream) runs the kernels, and the call ends by copying a
 * status word to the host and synchronising that stream.  All intermediate
 * data live in a fixed device
 * array of the library (about 10.5 MB per GPU, kept until exit): at most
 * 524,288 particles, at most 2^10 (3D) or 2^15 (2D) cells per axis, 2^20
 * Morton cells (2^(dim*bits) with 2^bits >= the largest ncell), and 256
 * particles in any one cell; larger inputs return INVALID_ARG (for a crowded
 * cell the outputs are left unwritten).  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress), so make the first
 * call on each device before any stream capture.  Calls that overlap on the
 * GPU share the array and race.  Errors: INVALID_ARG, DOMAIN (a
 * particle outside the grid; it is clamped to the nearest cell and the
 * outputs hold that clamped order), CUDA. */
int sphst_cell_order_noalloc(int32_t dim, int64_t n, const double *pos_dev,
                             const double *origin3, double cell_size, const int32_t *ncell3,
                             uint64_t *keys_dev, int64_t *order_dev, void *cuda_stream);

/* ------------------------------------------------------------- batches   */
/* A batch advances many independent cases together: their particles share
 * one set of device arrays, one segmented cell list (the case index selects
 * a segment of the cell table) and one captured CUDA graph per advection
 * step, in which every case keeps its own advection and acoustic time steps.
 * All members have the precision given here. */
int sphst_batch_create(int32_t precision, sphst_batch *out);

/* Make c a member.  c must have that precision and may already have been
 * stepped alone; it joins at the next sphst_batch_step.  Errors: STATE (c in
 * another batch), INVALID_ARG, UNSUPPORTED (precision mismatch). */
int sphst_batch_add(sphst_batch b, sphst_case c);

/* Remove c; it keeps its state and can be stepped alone or read. */
int sphst_batch_remove(sphst_batch b, sphst_case c);

/* Advance every member by n_adv of its own advection steps.  Members whose
 * status turns non-zero stop; the others continue.  info (optional) receives
 * n_adv/n_sub summed over members and the worst status. */
int sphst_batch_step(sphst_batch b, int64_t n_adv, sphst_step_info *info);

/* Number of members. */
int sphst_batch_size(sphst_batch b, int64_t *n_cases);

/* Release the batch (members stay valid and leave it). */
int sphst_batch_destroy(sphst_batch b);

/* ------------------------------------------------------------ diagnostics */
/* FP64 reductions over a case's fluid particles on the device, in a fixed
 * summation order (the same state gives the same bits).  Phase k has mass
 * m_k = rho0_k dp^dim per particle; p = c0^2 (rho - rho0) (Eq. 2).
 *   momentum      sum m v                          (conserved by Eqs. 8, 26, 33)
 *   kinetic       sum m |v|^2 / 2
 *   count[k]      particles of fluid phase k (k = 0: first fluid phase added)
 *   first         sum x over phase 0               (centroid = first / count[0])
 *   second        sum x_a x_b over phase 0: xx, yy, zz, xy, xz, yz
 *   p_in, n_in    sum and count of p over phase-0 particles with |x - center| < r_in
 *   p_out, n_out  sum and count of p over phase-1 particles with |x - center| > r_out
 *   n_nonfinite   particles with a non-finite position, velocity or density
 * These give the Laplace jump of Eq. 37 (p_in/n_in - p_out/n_out), the drop's
 * shape moments for the oscillation period (Eq. 35) and the momentum drift.
 * center: 3 doubles (unused axes ignored).  Before the first step the
 * staged input is reduced on the host.  Errors: INVALID_ARG, CUDA. */
typedef struct {
    double  momentum[3];
    double  kinetic;
    int64_t count[2];
    double  first[3];
    double  second[6];
    double  p_in, p_out;
    int64_t n_in, n_out;
    int64_t n_nonfinite;
} sphst_diagnostics;
int sphst_diagnose(sphst_case c, const double *center, double r_in, double r_out,
                   sphst_diagnostics *out);

/* Measured fused multiply-add throughput of the current GPU in TFLOP/s
 * (precision 32 or 64): independent FMA chains on every SM, the best of three
 * timed launches after a warm-up; kernel_ms (optional) receives that launch's
 * duration.  It is the arithmetic roof of the pair sweeps.  Errors:
 * INVALID_ARG, CUDA. */
int sphst_fma_peak(int32_t precision, double *tflops, double *kernel_ms);

/* Properties of the current GPU that the arithmetic and issue roofs of the
 * pair sweeps are derived from: the number of SMs, the peak SM clock in kHz
 * as the device reports it, and (optional) the compute capability.  No
 * device memory is touched.  Errors: INVALID_ARG, CUDA (no device). */
int sphst_device_info(int32_t *sm_count, int32_t *max_sm_clock_khz, int32_t *cc_major,
                      int32_t *cc_minor);

/* Device bytes one case of n particles needs (particle arrays, cell table,
 * scratch), for admission control.  Errors: INVALID_ARG. */
int sphst_footprint_bytes(const sphst_case_params *params, int64_t n_particles,
                          int64_t *bytes_out);

/* sizeof of the three structures of this header as the library was built,
 * so a binding can check its layout before the first call.  Any pointer may
 * be NULL.  Never fails. */
int sphst_struct_sizes(int64_t *params_bytes, int64_t *phase_props_bytes, int64_t *step_info_bytes);

#ifdef __cplusplus
}
#endif

#endif /* SPHST_H */
