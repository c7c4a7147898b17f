/*
 * Plain FP64 CPU oracle for the SGS-PFP steady Boltzmann solver (Cai, Dong, Hu,
 * "Symmetric Gauss-Seidel Method with a Preconditioned Fixed-Point Iteration for
 * the Steady-State Boltzmann equation").
 *
 * TEST INFRASTRUCTURE ONLY. Only tests, the smoke check and the benchmark's CPU
 * baseline may load this library. The CUDA library never includes, links or calls it,
 * and this code includes nothing from the CUDA library.
 *
 * Conventions
 *   - Velocity grid: N points per dimension, v = j*dv, j in {-N/2+1, ..., N/2},
 *     dv = 2L/N, quadrature weight w = dv^3 (Section 2.2, periodic grid used for the
 *     Fourier spectral method).
 *   - A distribution of one cell is a contiguous array f[i1][i2][i3] (i3 fastest),
 *     i = j + N/2 - 1; x-direction velocity is v1.
 *   - Fourier modes k with |k_i| <= h = N/2 - 1 (Nyquist dropped), stored in a box
 *     [k1][k2][k3] of side n = 2h+1, index k_i + h, as interleaved (re, im) pairs.
 */
#ifndef SGS_ORACLE_H
#define SGS_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { OR_MAXWELL = 0, OR_HARD_SPHERE = 1, OR_BGK = 2 };
enum { OR_DIFFUSE = 0, OR_INFLOW = 1 };
enum { OR_PFP = 0, OR_FP = 1, OR_PFP_RELAX = 2 };

typedef struct {
  int N;            /* velocity points per dimension */
  double L;         /* velocity box [-L, L]^3 */
  int kernel;       /* OR_MAXWELL, OR_HARD_SPHERE, OR_BGK */
  double b0;        /* B = b0 (Maxwell) or b0*|q| (hard spheres) */
  int J;            /* cells */
  double x_lo, x_hi;
  double eps;       /* Knudsen number */
  int bc_kind[2];   /* left, right */
  double bc_rho[2], bc_u[2][3], bc_T[2];
  double total_mass;   /* C of the mass constraint; <= 0 disables the rescale */
  double inner_tol; int inner_max, inner_fixed;
  double newton_tol; int newton_max;
  int inner_method;    /* OR_PFP, OR_FP, or OR_PFP_RELAX (relaxed step 1 when eq. (26) fails) */
  int conserve_proj;   /* 1: project Q onto the zero-moment subspace (not in the paper);
                          2: the same with the correction weighted by the local Maxwellian */
  int order;           /* spatial order of the 1-D scheme: 1 (s = 0) or 2 (eq. (slope)); 0 means 1 */
} or_problem;

typedef struct {
  long inner_iters, visits, newton_iters, newton_solves, existence_fallbacks, newton_failures;
} or_stats;

/* Velocity nodes, one dimension: out[i] = (i - N/2 + 1) * 2L/N. */
void or_velocity_nodes(int N, double L, double* out);
/* Gauss-Legendre nodes and weights on [-1, 1]. */
void or_gauss_legendre(int n, double* x, double* w);
/* Spectral weight G(a, b) for integer squared norms a2 = a^2, b2 = b^2. */
double or_G(int N, double L, int kernel, double b0, long a2, long b2);
/* Separable 3-D DFT restricted to |k_i| <= h; out: n^3 complex. */
void or_dft(int N, const double* f, double* fhat);
/* Inverse: q(v) = Re sum_k qhat_k exp(i pi k.v / L). */
void or_idft(int N, const double* qhat, double* q);
/* Direct Fourier-Galerkin bilinear sum qhat_k = sum_m beta(k-m, m) ahat_{k-m} bhat_m. */
void or_qhat_direct(int N, double L, int kernel, double b0, const double* ahat, const double* bhat, double* qhat);
/* Q^FSM[f, f] on the velocity nodes. */
void or_qfsm(int N, double L, int kernel, double b0, const double* f, double* q);
/* Slopes of eq. (slope) for the second-order scheme (central inside, one-sided in the first
 * and the last cell, no limiter); all zero for the first-order scheme or a single cell.
 * f, s: J cells of N^3 values. */
void or_slopes(const or_problem* p, int J, const double* f, double* s);
/* Orthogonal projection of q (in place) onto {q : sum_k phi_i(v_k) q_k = 0, i = 0..4},
 * phi = (1, v1, v2, v3, |v|^2). Returns 0, or -1 if the 5x5 Gram matrix is singular. */
int or_conserve_project(int N, double L, double* q);
/* Maxwellian-weighted variant: q_c = q - M (lambda . phi) with (sum_k M phi phi^T) lambda =
 * sum_k phi q, the smallest change of q in the norm sum (.)^2 / M that zeroes the moments. */
int or_conserve_project_w(int N, double L, const double* M, double* q);
/* Moments (rho, rho*U, sum w|v|^2 f) with weights w. */
void or_moments(int N, double L, const double* f, double* m5);
/* rho, U1..3, T (eq. (6), d = 3) and the heat flux q1..3 of Section 4.2.2 of one cell */
void or_macroscopic(int N, double L, const double* f, double* out8);
/* Discrete Maxwellian exp(alpha + beta.v - gamma|v|^2) matching weighted moments.
 * wk: per-node weights (NULL -> w). theta in: initial guess (used if use_guess),
 * out: solution. Returns Newton iterations, or -1 on failure. */
int or_discrete_maxwellian(int N, double L, const double* wk, const double* target, double* theta,
                           int use_guess, double tol, int maxit);
void or_eval_maxwellian(int N, double L, const double* theta, double* M);
double or_collision_frequency(const or_problem* p, const double* f);
/* Q = Q^FSM[f,f] - Q^FSM[M,M] and P = Q - nu (M - f) for one cell (Q or P may be NULL). */
void or_collide_cell(const or_problem* p, const double* f, double* Q, double* P, double* nu, double* theta);
/* All cells of one level. */
void or_collide(const or_problem* p, int J, const double* f, double* Q, double* P, double* nu);
/* Cell equation (|v1|/dx) g + r = (nu/eps)(M[g] - g), solved by PFP or FP. */
int or_cell_solve(const or_problem* p, double dx, const double* r, double nu, double* g, or_stats* st);
/* The same with a per-node transport weight c (|v1|/dx in 1-D, |v1|/dx + |v2|/dy in 2-D). */
int or_cell_solve_c(const or_problem* p, const double* c, const double* r, double nu, double* g, or_stats* st);
/* Ghost density of a diffuse wall from the zero-mass-flux condition. */
double or_wall_density(const or_problem* p, int side, const double* f_adj);
void or_ghost(const or_problem* p, int side, const double* f_adj, double* ghost);
/* One sweep (dir = +1 forward, -1 backward) over J cells of spacing dx. */
void or_sweep(const or_problem* p, int J, double dx, int dir, double* f, const double* P, const double* nu,
              const double* b, or_stats* st);
void or_rescale(const or_problem* p, int J, double dx, double* f);
/* R = T(f) - Q/eps - b per node; returns sqrt(dx sum w R^2). Rout may be NULL. */
double or_residual(const or_problem* p, int J, double dx, const double* f, const double* Q, const double* b,
                   double* Rout);
/* One SGS iteration: collide, forward, collide, backward, rescale (if enabled and rescale != 0). */
void or_sgs_iteration(const or_problem* p, int J, double dx, double* f, const double* b, int rescale,
                      or_stats* st);
/* Source iteration (eq. (SI)), first order, the collision term split by the BGK penalty
 * (eq. (28)) with P, nu and M of the current iterate; one linear transport solve per
 * velocity node; diffuse-wall densities from the current iterate; then the mass rescale
 * when rescale != 0 and total_mass > 0. f in place. */
void or_si_iteration(const or_problem* p, int J, double dx, double* f, const double* b, int rescale);
/* One FAS V-cycle on the finest level (J cells). */
void or_vcycle(const or_problem* p, double* f, int levels, int pre, int post, int coarse_iters, or_stats* st);

/* ------------------------------------------------------------------------------------
 * 2-D space (sgs_oracle2d.c). The 1-D problem p describes the velocity grid, kernel, eps,
 * tolerances, the x extent (J = nx cells on [x_lo, x_hi]) and the x_lo / x_hi sides;
 * the y extent and the y_lo / y_hi sides are added here. Cell (i, j) at index j nx + i.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  or_problem p;
  int ny;
  double y_lo, y_hi;
  int bc_kind_y[2]; /* y_lo, y_hi */
  double bc_rho_y[2], bc_u_y[2][3], bc_T_y[2];
} or_problem2d;

double or_dx2d(const or_problem2d* q);
double or_dy2d(const or_problem2d* q);
/* Ghost of side s (0 x_lo, 1 x_hi, 2 y_lo, 3 y_hi) next to the cell f_adj. */
void or_ghost2d(const or_problem2d* q, int s, const double* f_adj, double* ghost);
/* One sweep in ordering o: 0 SW->NE, 1 NE->SW, 2 NW->SE, 3 SE->NW. */
void or_sweep2d(const or_problem2d* q, int o, double* f, const double* P, const double* nu, const double* b,
                or_stats* st);
void or_rescale2d(const or_problem2d* q, double* f);
double or_residual2d(const or_problem2d* q, const double* f, const double* Q, const double* b, double* Rout);
/* Four sweeps, each after a collision evaluation, then the rescale. */
void or_sgs_iteration2d(const or_problem2d* q, double* f, const double* b, int rescale, or_stats* st);
/* FAS V-cycle with 2 x 2 coarsening (nx, ny divisible by 2^(levels-1)). */
void or_vcycle2d(const or_problem2d* q, double* f, int levels, int pre, int post, int coarse_iters, or_stats* st);

#ifdef __cplusplus
}
#endif
#endif
