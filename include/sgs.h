/*
 * sgs.h - C ABI of the GB300 (sm_103a) SGS-PFP solver for the steady Boltzmann equation
 *
 *     v . grad_x f = Q[f, f] / eps                                   (eq. (1))
 *
 * discretised by first-order upwind finite volumes in x (eqs. (7)-(11), slopes s = 0),
 * a periodic velocity grid with N^3 points on [-L, L]^3 and the Fourier spectral
 * collision operator in its steady-state-preserving form (eq. (16)), and solved by
 * symmetric Gauss-Seidel sweeps (eq. (29)) whose per-cell problem (eq. (20)) is solved by
 * the fixed-point iteration preconditioned with its small-eps limit (eqs. (24)-(26)),
 * optionally inside nonlinear multigrid V-cycles (eq. (30)).
 *
 * Conventions shared by every call
 *   - Velocity index i in [0, N): v = (i - N/2 + 1) * 2L/N; a cell's distribution is
 *     N^3 contiguous doubles [i1][i2][i3] (i3 fastest); v1 is the x-direction velocity.
 *   - A field (f, Q, P, rhs) holds all instances: instance q's cells start at the element
 *     offset given by sgs_layout(), cells contiguous, each N^3 doubles.
 *   - Every pointer named "device" is CUDA device memory owned by the caller, 16-byte
 *     aligned, never freed or retained by the library beyond the call (the workspace
 *     excepted: it stays bound until sgs_destroy). Storage is FP64 in every precision mode.
 *   - Every compute call is asynchronous on the given cudaStream_t (passed as void*, NULL =
 *     legacy default stream) and enqueues kernels only: no allocation, no host sync. Such
 *     calls may be captured in a CUDA graph.
 *   - Return value: SGS_OK (0) or a negative SGS_ERR_* detected on the host before anything
 *     is enqueued. Conditions found on the device (Newton failure, inner cap, non-finite
 *     values, wait timeout) set bits of a per-instance status word read by
 *     sgs_read_status(). No call traps or aborts.
 */
#ifndef SGS_H
#define SGS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SGS_OK 0
#define SGS_ERR_ARG (-1)         /* invalid argument or problem description */
#define SGS_ERR_UNSUPPORTED (-2) /* valid but not implemented (e.g. 2-D space) */
#define SGS_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define SGS_ERR_WORKSPACE (-4)   /* no or too small workspace bound */
#define SGS_ERR_NOMEM (-5)       /* host allocation failed */

/* Device status bits (per instance, OR-ed). */
#define SGS_ST_NEWTON_FAIL 1u       /* a discrete-Maxwellian Newton solve did not converge */
#define SGS_ST_INNER_CAP 2u         /* a cell solve stopped at inner_max */
#define SGS_ST_NONPOSITIVE 4u       /* density or temperature <= 0 met in a cell */
#define SGS_ST_NONFINITE 8u         /* NaN/Inf met */
#define SGS_ST_TIMEOUT 16u          /* a bounded device wait gave up */

enum sgs_collision { SGS_MAXWELL = 0, SGS_HARD_SPHERE = 1, SGS_BGK = 2 };
enum sgs_bc_kind { SGS_DIFFUSE = 0, SGS_INFLOW = 1 };
/* SGS_DF64 is an arithmetic for sgs_collide_prec and sgs_set_dc_precision only (not a problem
 * precision): double-float spectral sums, each value a pair of FP32 numbers (hi + lo), on the
 * FP32 pipes, about 2^-48 relative error per term; available on SGS_FP32 handles. */
enum sgs_precision { SGS_FP64 = 0, SGS_FP32 = 1, SGS_DF64 = 2 };
enum sgs_inner_method { SGS_PFP = 0, SGS_FP = 1, SGS_PFP_RELAX = 2 };

/* Boundary data of one side: a diffuse wall at temperature T moving with tangential
 * velocity u (eq. (31)), or an inflow Maxwellian (rho, u, T) for incoming velocities. */
typedef struct {
  int kind;
  double rho;
  double u[3];
  double T;
} sgs_bc;

/* One steady problem instance (1-D or 2-D space, 3-D velocity). In 2-D the cells form an
 * nx x ny grid stored row by row (cell (i, j) at j nx + i, i along x); one SGS iteration is
 * the four corner-to-corner orderings, and a handle holds one 2-D instance. */
typedef struct {
  int space_dim;      /* 1 or 2 */
  int nx;             /* cells along x, >= 1 */
  double x_lo, x_hi;  /* domain along x */
  int ny;             /* cells along y (2-D; ignored in 1-D) */
  double y_lo, y_hi;  /* domain along y (2-D) */
  int nv;             /* N: velocity points per dimension, one of 8, 12, 16, 20, 24, 28, 32 */
  double v_max;       /* L; the support radius is R = 2L / (3 sqrt 2 + 1) (Section 4.2) */
  int collision;      /* SGS_MAXWELL (B = b0), SGS_HARD_SPHERE (B = b0 |q|), SGS_BGK (P = 0) */
  double b0;          /* kernel constant; 1/(4 pi) gives nu = rho for Maxwell molecules */
  double eps;         /* Knudsen number, > 0 */
  sgs_bc bc[4];       /* x_lo, x_hi, y_lo, y_hi (the y sides in 2-D only); diffuse walls move
                         tangentially (u[0] = 0 on x walls, u[1] = 0 on y walls) */
  double total_mass;  /* C of eq. (32); <= 0 disables the rescale */
  int precision;      /* arithmetic of the collision sum: SGS_FP64 or SGS_FP32 */
  double inner_tol;   /* cell-equation residual tolerance (discrete L2 norm), e.g. 1e-8 */
  int inner_max;      /* cap on PFP/FP updates per cell visit, e.g. 200 */
  int inner_fixed;    /* > 0: exactly this many updates per visit (no tolerance test) */
  double newton_tol;  /* exponent-change tolerance of the Maxwellian Newton, e.g. 1e-10 */
  int newton_max;     /* e.g. 50 */
  int inner_method;   /* SGS_PFP (eqs. (24)-(25); the fixed-point step of eq. (22) where
                         eq. (26) fails), SGS_FP (eq. (22)), or SGS_PFP_RELAX (where eq. (26)
                         fails, the relaxed step 1 of the remark after it: target
                         (tau m_w + s)/(1 + tau), m_w the weighted moments of M[g], 1 + tau
                         doubling from 2 until eq. (26) holds) */
  int conserve_proj;  /* 0: the paper's Q (mass conserved to round-off, momentum and energy to
                         spectral accuracy); 1: Q projected in FP64 onto the zero-moment
                         subspace, Q_c = Q - C^T (C C^T)^-1 C Q with C = [w phi_i(v_k)],
                         phi = (1, v, |v|^2); 2: the Maxwellian-weighted projection
                         Q_c = Q - M (lambda . phi), (sum_k M phi phi^T) lambda = sum_k phi Q,
                         M the cell's discrete Maxwellian (the correction stays out of the
                         far velocity tails). Applied in FP64 in every collision step (all
                         levels and precisions) before P = Q_c - nu (M - f) is formed. Not in
                         the paper; equal in every instance of a handle; ignored for BGK. */
  int order;          /* spatial order: 1 (or 0): first order (s = 0); 2: linear reconstruction
                         with the slopes of eq. (slope) (central inside, one-sided in the end
                         cells, no limiter; in 2-D along x within each row and along y within
                         each column), explicit in the scans (taken from the state before each
                         scan or ordering, eq. (SGS_BGK)), zero ghost slopes, diffuse-wall
                         densities from the outgoing face value. Equal in every instance of a
                         handle. */
} sgs_problem;

/* Counters accumulated on the device since setup or the last sgs_reset_stats(). */
typedef struct {
  unsigned int status;          /* OR of every instance's status bits */
  unsigned long long visits;    /* cell visits (cell updates) */
  unsigned long long inner_iters;
  unsigned long long newton_iters;
  unsigned long long newton_solves;
  unsigned long long fallbacks; /* step 1 skipped (existence test, eq. (26), or Newton failure) */
} sgs_stats;

typedef struct sgs_handle sgs_handle;

/* Validates n_inst problems (all with the same nv and precision), builds the velocity
 * grid, the Fourier weights G (closed form of the radial integral) and the per-step weight
 * blocks on the host, and reports the device workspace size the caller must allocate and
 * bind. No device memory is allocated here. */
int sgs_setup(const sgs_problem* problems, int n_inst, sgs_handle** out, size_t* workspace_bytes);

/* Binds a caller-owned device buffer of at least workspace_bytes (256-byte aligned) and
 * uploads the tables (synchronous). Must precede every compute call. */
int sgs_bind_workspace(sgs_handle* h, void* device_ptr, size_t bytes);

/* Element offset of instance inst's first cell in every field, its cell count and N. */
int sgs_layout(const sgs_handle* h, int inst, size_t* f_offset, int* n_cells, int* nv);
/* Total elements of one field (all instances). */
size_t sgs_field_elems(const sgs_handle* h);

/* Collision step for every cell (eqs. (16), (28)):
 *   moments and discrete Maxwellian M (eqs. (13)-(14)), Q = Q^FSM[f,f] - Q^FSM[M,M]
 *   computed as the single symmetric bilinear sum Q_s(f - M, f + M), and
 *   P = Q - nu (M - f). With conserve_proj, Q is projected (FP64) before P is formed.
 *   f, Q (device, nullable), P (device, nullable). */
int sgs_collide(sgs_handle* h, const double* f, double* Q, double* P, void* stream);

/* One SGS scan (eq. (29)) over every instance, forward (x_lo -> x_hi) or backward, in a
 * single persistent launch (one thread-block cluster per instance, no host round trip).
 * f (device) is updated in place; P (device) from the preceding sgs_collide; rhs (device,
 * nullable) is the b of R(f) = b (multigrid / defect correction). Second order (order 2):
 * the slope terms of eq. (SGS_BGK) and the face-value wall densities are taken from f as it
 * is when the scan (in 2-D: the ordering) starts (explicit slopes). */
int sgs_sweep_forward(sgs_handle* h, double* f, const double* P, const double* rhs, void* stream);
int sgs_sweep_backward(sgs_handle* h, double* f, const double* P, const double* rhs, void* stream);
/* One scan in a given ordering. 1-D: 0 forward, 1 backward. 2-D (eq. (29) in each
 * direction): 0 SW->NE, 1 NE->SW, 2 NW->SE, 3 SE->NW; the cells of one anti-diagonal
 * wavefront are independent and visited concurrently (one cluster per cell), wavefront
 * after wavefront, which equals the row-by-row Gauss-Seidel order of that ordering.
 * sgs_sweep_forward / sgs_sweep_backward are orderings 0 / 1. */
int sgs_sweep_ordering(sgs_handle* h, double* f, const double* P, const double* rhs, int ordering, void* stream);

/* Uniform rescale of each instance to its total mass (eq. (32)); no-op where <= 0. */
int sgs_rescale(sgs_handle* h, double* f, void* stream);

/* Macroscopic quantities of every cell of f (device, the handle's field layout): density,
 * bulk velocity and temperature as defined with the moments (eq. (6) and the definitions
 * beside it, d = 3: rho T = (1/3) int |v - U|^2 f) and the heat flux of the lid-driven cavity
 * study (Section 4.2.2), q = 1/2 int (v - U)|v - U|^2 f dv, all by the velocity quadrature
 * (eq. (10)). out (device, caller-owned): 8 doubles per cell in the handle's cell order,
 * (rho, U1, U2, U3, T, q1, q2, q3). FP64 throughout; f is only read. Cells of zero density
 * give non-finite U, T, q. Needs a bound workspace (its cell tables); SGS_ERR_ARG for null
 * pointers. */
int sgs_macroscopic(const sgs_handle* h, const double* f, double* out, void* stream);

/* One source iteration (eq. (SI)), 1-D problems: the collision step of f (P = Q - nu (M - f),
 * eq. (28), written to P), then for every velocity node the upwind transport with
 * absorption (|v1|/dx + nu_j/eps) f_j = (|v1|/dx) f_upwind + P_j/eps + (nu_j/eps) M[f_j] + b_j,
 * marched from the node's inflow side with the diffuse-wall ghosts of the previous iterate,
 * then the mass rescale of eq. (32). The classical method the paper compares SGS with; it
 * slows down as eps -> 0 (Section 3.1). f (device) in place; P (device) receives the
 * penalty of the previous iterate; rhs (device, nullable) is b. SGS_ERR_UNSUPPORTED for
 * 2-D handles. */
int sgs_si_iteration(sgs_handle* h, double* f, double* P, const double* rhs, void* stream);

/* Outer residual R = T(f) - Q/eps - rhs (Section 4 stopping rule), res[q] (device,
 * n_inst doubles) = sqrt(dx sum_j sum_k w R^2) per instance. Q from sgs_collide(f). T is
 * the upwind transport of eq. (upwind) with the face values of the reconstruction (the
 * cell values at first order) and wall ghosts from the same f. */
int sgs_residual(sgs_handle* h, const double* f, const double* Q, const double* rhs, double* res, void* stream);

/* Outer residual of ONE instance that allocates nothing (no counterpart in the paper: it
 * is a service for callers). Callers that cannot allocate device memory - code inside a
 * host framework that owns every allocation, code under a hard memory budget, paths where
 * an allocation could synchronise the device - need neither a handle nor a workspace here:
 * p describes the instance (fields as for sgs_setup), f and Q (device, p->nx * nv^3
 * doubles, cells contiguous) and rhs (device, nullable) are the inputs, res (device, one
 * double) the output, as in sgs_residual. The per-cell partial sums live in a static
 * device array of the library (32 KiB + 64 B, kept by every GPU that loads the library
 * until the process exits), so at most 4096 cells are accepted; larger nx returns
 * SGS_ERR_ARG with a message naming the limit. The first call on a device looks up the
 * array's device address with that device current; make that first call before any
 * stream capture. All calls share the array: calls that overlap on the GPU race, so order
 * them on one stream. Every slot a call reads is written earlier in the same call.
 * The problem is validated as sgs_setup validates it (same return codes), then restricted to
 * one 1-D instance (SGS_ERR_ARG otherwise) at first order (SGS_ERR_UNSUPPORTED for order 2).
 * The looked-up address belongs to the device's context at the first call: after a
 * cudaDeviceReset() of that device the entry point must not be called again in the process. */
int sgs_residual_noalloc(const sgs_problem* p, const double* f, const double* Q, const double* rhs, double* res,
                         void* stream);

/* Collision step in a chosen arithmetic (SGS_FP32 and SGS_DF64 need a handle set up with
 * precision SGS_FP32, whose workspace then carries the FP64 and FP32 weight tables and the
 * FP32 remainder table). Same fields as sgs_collide. */
int sgs_collide_prec(sgs_handle* h, const double* f, double* Q, double* P, int precision, void* stream);

/* One full SGS iteration (eq. (29)): [collide], forward scan, collide, backward scan,
 * rescale; in 2-D: [collide], ordering 0, then collide + ordering 1, 2, 3, rescale (cell
 * measure dx dy). Q and P are caller-owned device fields.
 *   flags & SGS_IT_P_VALID: P already holds P[f] of the incoming f (skips the first collide).
 *   flags & SGS_IT_EVAL:    afterwards Q, P hold Q[f], P[f] of the new f and, when res
 *                           (device, n_inst doubles) is not NULL, res the outer residual.
 * With both flags set, consecutive calls cost two collision evaluations per iteration. */
#define SGS_IT_P_VALID 1
#define SGS_IT_EVAL 2
int sgs_iterate(sgs_handle* h, double* f, double* Q, double* P, const double* rhs, int flags, double* res,
                void* stream);

/* One step of FP64 defect correction for the mixed solver (handle set up with SGS_FP32):
 *   Q, P = high-precision collision of the current iterate f_k (double-float or FP64 sums,
 *   sgs_set_dc_precision); res = its FP64 residual (device, n_inst doubles, nullable); f_k
 *   becomes the reference state; then lo_iters SGS iterations in which every FP32
 *   collision is evaluated in increment form
 *     Q(f) = Q_hi(f_k) + [Q_s(a - a_k, b) + Q_s(a_k, b - b_k)]_FP32,  a = f - M, b = f + M,
 *   an exact identity of the symmetric bilinear form whose FP32 rounding error scales with
 *   f - f_k. Each step therefore moves f towards the FP64 solution R_FP64(f) = 0 without an
 *   FP32 noise floor. The reference stays in force for later FP32 collisions on this handle
 *   until sgs_dc_clear() or the next sgs_dc_step(). Q and P are caller-owned device fields. */
int sgs_dc_step(sgs_handle* h, double* f, double* Q, double* P, int lo_iters, double* res, void* stream);
int sgs_dc_clear(sgs_handle* h);
/* Arithmetic of the high-precision collision in sgs_dc_step: SGS_DF64 (default on SGS_FP32
 * handles: double-float sums on the FP32 pipes) or SGS_FP64 (FP64 sums). Moments, discrete
 * Maxwellians, transforms and the residual are FP64 in both. */
int sgs_set_dc_precision(sgs_handle* h, int precision);

/* One FAS V-cycle (eq. (30)) on every instance, on 2 <= levels <= sgs_max_levels(h) grids
 * with H = 2h: pre SGS-PFP iterations, restriction of f and of the residual field (mean of
 * the two children), coarse right-hand side b_H = R_H(I f) + I(b_h - R_h(f)), recursion
 * (coarse_iters SGS iterations on the coarsest grid), correction f += P(f_H - I f) by
 * piecewise-constant prolongation, post SGS iterations. The mass rescale acts on the finest
 * grid only. Coarse tables and fields live in the workspace. With an active defect-
 * correction reference (sgs_dc_step) the finest-grid FP32 collisions use the increment form. */
int sgs_vcycle(sgs_handle* h, double* f, int levels, int pre, int post, int coarse_iters, void* stream);
/* Number of grids available to sgs_vcycle: 1 + how often every instance's cell count halves. */
int sgs_max_levels(const sgs_handle* h);

/* Pipelined SGS iterations (on by default). A handle holding one 1-D instance of at least 64
 * cells (two lane groups of 32), first order, spectral collisions, runs the scans of
 * sgs_iterate, sgs_dc_step and the finest-level smoothing of sgs_vcycle in segments of 32
 * cells on a high-priority stream of its own and evaluates the collision step of each group
 * on the caller's stream as soon as the scan has left that group: the collision step for the
 * backward scan behind the forward scan and, with SGS_IT_EVAL, the one of the new iterate
 * behind the backward scan (the groups evaluated before the mass rescale of eq. (32) are then
 * scaled to the rescaled state: Q and P by lam^2, nu by lam; exact up to rounding). The order
 * of the method is unchanged: every cell sees the inputs of the sequential iteration. The two
 * streams are joined again before each call returns (events; also under stream capture).
 * sgs_dc_step then also evaluates the collision step after each of its iterations (Q and P
 * hold the last iterate's). sgs_get_overlap: 1 when the bound handle pipelines, else 0. */
int sgs_set_overlap(sgs_handle* h, int enable);
int sgs_get_overlap(const sgs_handle* h);

/* Kernel-time profiling. When enabled, every group of launches is bracketed by CUDA events
 * recorded on the launching stream; sgs_profile_read synchronises on them and returns, per
 * class, the summed milliseconds, the number of bracketed groups and (work, nullable) the
 * cells they processed: cells evaluated by the spectral sums, cells visited by the scans
 * (0 for the other classes), then clears them.
 * sgs_launch_count returns the number of kernels enqueued through the handle so far.
 * Launches enqueued while the stream is being captured into a CUDA graph are not timed. */
enum sgs_prof_class {
  SGS_PROF_MOMENTS = 0,     /* moments + discrete Maxwellian of every cell */
  SGS_PROF_DFT = 1,         /* forward DFT of f - M and f + M (3 kernels) */
  SGS_PROF_SUM = 2,         /* direct spectral sum, FP32 (mixed precision) */
  SGS_PROF_REDUCE_IDFT = 3, /* partial reduction + inverse DFT + P (4 kernels), or BGK */
  SGS_PROF_SWEEP = 4,       /* persistent SGS scan */
  SGS_PROF_RESIDUAL = 5,    /* outer residual */
  SGS_PROF_RESCALE = 6,     /* mass rescale, grid transfers and other vector updates */
  SGS_PROF_SUM_FP64 = 7,    /* direct spectral sum, FP64 */
  SGS_PROF_SUM_DF64 = 8,    /* direct spectral sum, double-float */
  SGS_PROF_FAST = 9,        /* fast spectral operator: tensor-core passes and the final transform */
  SGS_PROF_CLASSES = 10
};
int sgs_profile(sgs_handle* h, int enable);
int sgs_profile_read(sgs_handle* h, double* ms, unsigned long long* launches, double* work, int n_classes);
unsigned long long sgs_launch_count(const sgs_handle* h);

/* Batches: per-instance activity. Every instance starts active (at bind). An inactive
 * instance is converged: the scans (and the mass rescale) skip it, so its f stays as it
 * is; in a handle of several instances the collision steps skip its cells as well (their Q,
 * P and collision frequency from the last evaluation stay valid, f being unchanged), while
 * residuals still cover every cell.
 *   sgs_update_active: active[q] = !(res[q] < tol) for the device residuals res[n_inst]
 *     (as written by sgs_residual / sgs_dc_step); asynchronous, graph-capturable.
 *   sgs_activate_all: marks every instance active again; asynchronous.
 *   sgs_read_active: synchronises the stream and copies the n_inst flags to host memory. */
int sgs_update_active(sgs_handle* h, const double* res, double tol, void* stream);
int sgs_activate_all(sgs_handle* h, void* stream);
int sgs_read_active(sgs_handle* h, int* active, void* stream);

/* Launch shape of the persistent scan: nodes per thread (ept, a divisor of nv with a
 * compiled kernel: 2, 4, 8, 12, ..., 32), CTAs per cluster (a power of two <= 16; one
 * cluster walks one instance) and threads per CTA (a multiple of 32 in [160, 256]) with
 * ept * cluster * threads >= nv^3. sgs_set_sweep_shape returns SGS_ERR_ARG for an invalid
 * shape and SGS_ERR_UNSUPPORTED for one that cannot be resident on the device. */
int sgs_get_sweep_shape(const sgs_handle* h, int* ept, int* cluster, int* threads);
int sgs_set_sweep_shape(sgs_handle* h, int ept, int cluster, int threads);

typedef struct {
  int sweep_ept, sweep_cluster, sweep_threads; /* chosen scan shape */
  float sweep_ms;                              /* its forward + backward scan time, all instances */
  int candidates;                              /* shapes timed */
  int sum_warps, sum_units, sum_blocks;        /* chosen spectral-sum decomposition: warps (lane
                                                  groups of 32 cells) per block, work units, blocks */
  float sum_ms;                                /* its time per sum, all cells (handle's arithmetic) */
  int sum_candidates;                          /* decompositions timed */
} sgs_tuning;

/* Autotuner. Times every valid scan shape on the bound instances (reps forward + backward
 * scan pairs each, after one untimed pair, CUDA events on the stream), keeps the fastest
 * for all later scans and reports it. The timed scans are real SGS scans: f advances by
 * (reps + 1) symmetric sweeps with the given P per candidate. Then times the spectral sum
 * (the handle's arithmetic, all cells, two launches after one untimed one) for every
 * decomposition of 1, 2 or 4 lane groups per block and about 1500, 3000 or 6000 blocks, and
 * keeps the fastest for all later collision steps (the sums write only workspace buffers;
 * the reduction order of the partial sums follows the decomposition, so results may differ
 * in the last bits). Synchronises the stream; not graph-capturable (call it before
 * capturing). */
int sgs_autotune(sgs_handle* h, double* f, const double* P, int reps, sgs_tuning* out, void* stream);

/* Measurement probes (not part of the method; they supply the denominators of the
 * benchmark's rooflines and its latency model of the scan).
 *   sgs_peak_fma: FMA throughput of the CUDA-core pipes of the current device (SGS_FP32:
 *     FFMA, SGS_FP64: DFMA, SGS_FP32 | SGS_PEAK_PACKED: the packed FP32 pair FMA
 *     fma.rn.f32x2, two FMAs per instruction), independent FMA chains on every SM, iters
 *     instructions per chain; tflops = 2 flops per FMA over the CUDA-event time of the launch
 *     on stream; sms (nullable) the SM count used, ms (nullable) the time. Synchronises the
 *     stream; allocates nothing.
 *   sgs_probe_scan: latency of one building block of the persistent scan, in one cluster of
 *     `cluster` CTAs of `threads` threads on the nv^3 grid of [-v_max, v_max]^3, in the scan
 *     arithmetic of a handle of that precision (SGS_FP32: double-float, SGS_FP64: FP64):
 *     mode 0 a cluster reduction of seven values, mode 1 one Newton iteration of the
 *     discrete Maxwellian (evaluation, combination, factorisation), mode 2 the hardware
 *     cluster barrier alone (one step of the reduction). us_per_op = (time of reps
 *     operations - time of an empty launch) / reps in microseconds. Synchronises the stream. */
/*   sgs_tc_selftest: check of the tensor-core path of the fast spectral operator (no
 *     counterpart in the paper): D = A Bt^T for a 128 x K matrix A and an N x K matrix Bt of
 *     seeded values in [-1, 1), split into BF16 terms (terms 1: hi only; terms 3: hi hi + lo hi
 *     + hi lo), computed by tcgen05.mma with FP32 accumulation in TMEM and, from the same BF16
 *     terms, on the CUDA cores. K in {16, 32, 48, 64}, N a multiple of 16 up to 128; swap
 *     exchanges the two byte offsets of the operand descriptors. dev_scratch (device, at least
 *     4 (128 K + N K + 256 N) + 256 bytes) holds the operands. max_err = max |D - Dref| (-1 if
 *     the completion wait gave up), max_ref = max |Dref|. Synchronises the stream. */
int sgs_tc_selftest(int K, int N, int terms, int swap, void* dev_scratch, size_t bytes, double* max_err,
                    double* max_ref, void* stream);
#define SGS_PEAK_PACKED 256
int sgs_peak_fma(int precision, long long iters, double* tflops, int* sms, float* ms, void* stream);
int sgs_probe_scan(int nv, double v_max, int precision, int cluster, int threads, int mode, int reps,
                   float* us_per_op, void* stream);

/* The fast (Carleman-form) Fourier spectral operator for hard spheres (the fast methods the
 * paper cites for its binary-collision runs, Section 2.2): with both Carleman variables
 * truncated at T = 2R, the gain is a sum over the nodes e_p of a half-sphere rule (m_theta
 * Gauss-Legendre nodes in cos(theta) x m_phi azimuths) of products of the weighted spectra
 * phi(k.e_p) fhat and Psi(|k - (k.e_p) e_p|) fhat, phi(s) = 2 int_0^T r cos(pi r s / L) dr,
 * Psi(t) = 2 T L J1(pi T t / L) / t; the loss uses the same rule for beta(m, m). Each product
 * is formed on a zero-padded P^3 grid (P = 32 for N <= 16, else 48: no wrap-around) through
 * three separable DFT passes computed as tcgen05 matrix products (BF16 operands split from FP32,
 * FP32 accumulation in TMEM; terms 3: hi hi + lo hi + hi lo, about 1e-4 relative on Q; terms
 * 1: one BF16 product, about 2e-2); the intermediate operands between the passes are stored
 * as BF16 tiles in the tensor core's shared-memory layout and streamed by bulk copies; the
 * node sum is accumulated in FP32; the transforms of f, the final transform to the modes
 * |k_i| <= N/2 - 1 and the transform to the velocity grid run in FP32 (moments in FP64).
 *   sgs_fast_setup: for a hard-sphere handle (SGS_ERR_UNSUPPORTED otherwise); the nodes are
 *     processed `chunk` at a time (the workspace scales with chunk x cells); reports the
 *     workspace size of the operator (its own, besides the handle's).
 *   sgs_fast_bind: binds the caller's device buffer (256-byte aligned) and uploads the tables
 *     (synchronous).
 *   sgs_fast_collide: Q (device field of the handle) = the fast operator Q[f, f] of every cell
 *     of f; uses the handle's transform buffers (same stream as the handle's other calls).
 *     Asynchronous on the stream. */
typedef struct sgs_fast sgs_fast;
int sgs_fast_setup(const sgs_handle* h, int m_theta, int m_phi, int chunk, sgs_fast** out, size_t* workspace_bytes);
int sgs_fast_bind(sgs_fast* x, void* device_ptr, size_t bytes);
int sgs_fast_collide(sgs_fast* x, sgs_handle* h, const double* f, double* Q, int terms, void* stream);
void sgs_fast_destroy(sgs_fast* x);

/* Synchronises the stream and reads the accumulated status and counters. */
int sgs_read_status(sgs_handle* h, sgs_stats* out, void* stream);
int sgs_reset_stats(sgs_handle* h, void* stream);

void sgs_destroy(sgs_handle* h);
const char* sgs_strerror(int code);

/* Host-only helper (no GPU needed): the Fourier weight G(a, b) of the collision integral
 * for integer squared norms a2 = a^2, b2 = b^2, as tabulated by sgs_setup from its closed
 * form (Section 2.2, Fourier spectral method; weight conventions as in sgs_collide). */
double sgs_host_weight(int nv, double v_max, int collision, double b0, long long a2, long long b2);

#ifdef __cplusplus
}
#endif
#endif /* SGS_H */
