/*
 * Plain FP64 CPU oracle, 2-D space / 3-D velocity: the SGS-PFP iteration on an
 * nx x ny grid of square or rectangular cells (first order, s = 0), the four
 * corner-to-corner sweep orderings, diffuse walls on all four sides, the outer residual,
 * the mass rescale and the FAS V-cycle with 2 x 2 coarsening.
 *
 * TEST INFRASTRUCTURE ONLY (see sgs_oracle.h). Reuses the 1-D oracle's collision step
 * and cell solve, which are cell-local.
 *
 * Transport in 2-D (the 1-D scheme of eqs. (7)-(11) applied in each direction):
 *   v1 d/dx f + v2 d/dy f  ->  (v1^+ (f - f_W) + v1^- (f_E - f)) / dx
 *                            + (v2^+ (f - f_S) + v2^- (f_N - f)) / dy,
 * so the cell equation of eq. (20) has the transport weight c = |v1|/dx + |v2|/dy and
 *   r = (-v1^+ f_W + v1^- f_E) / dx + (-v2^+ f_S + v2^- f_N) / dy - P / eps - b.
 * Cells are stored row by row: cell (i, j) at index j nx + i, i along x.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "sgs_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static double weight2(int N, double L) {
  double dv = 2.0 * L / N;
  return dv * dv * dv;
}

/* Boundary data of side s: 0 x_lo, 1 x_hi (from the 1-D part), 2 y_lo, 3 y_hi. */
static void side_data(const or_problem2d* q, int s, int* kind, double* rho, const double** u, double* T) {
  if (s < 2) {
    *kind = q->p.bc_kind[s];
    *rho = q->p.bc_rho[s];
    *u = q->p.bc_u[s];
    *T = q->p.bc_T[s];
  } else {
    *kind = q->bc_kind_y[s - 2];
    *rho = q->bc_rho_y[s - 2];
    *u = q->bc_u_y[s - 2];
    *T = q->bc_T_y[s - 2];
  }
}

/* Normal velocity component of side s (v1 for x walls, v2 for y walls) and whether a node
 * enters the domain through it. */
static int side_dim(int s) { return s < 2 ? 0 : 1; }
static int incoming(int s, double vn) { return (s % 2 == 0) ? vn > 0.0 : vn < 0.0; }

/* Ghost distribution of side s next to the cell f_adj (eq. (31)): the incoming half is
 * rho^w times the unit wall Maxwellian, rho^w from the discrete zero normal mass flux
 * (diffuse) or given (inflow); the outgoing half of the ghost is not used and is zero. */
void or_ghost2d(const or_problem2d* q, int s, const double* f_adj, double* ghost) {
  int N = q->p.N;
  double L = q->p.L, w = weight2(N, L);
  int kind;
  double rho, T;
  const double* u;
  side_data(q, s, &kind, &rho, &u, &T);
  double* v = (double*)malloc(sizeof(double) * N);
  or_velocity_nodes(N, L, v);
  double c = 1.0 / pow(2.0 * M_PI * T, 1.5), out = 0.0, in = 0.0;
  int d = side_dim(s);
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int i3 = 0; i3 < N; i3++) {
        long i = ((long)i1 * N + i2) * N + i3;
        double d1 = v[i1] - u[0], d2 = v[i2] - u[1], d3 = v[i3] - u[2];
        double Mw = c * exp(-(d1 * d1 + d2 * d2 + d3 * d3) / (2.0 * T));
        double vn = d == 0 ? v[i1] : v[i2];
        if (incoming(s, vn)) {
          ghost[i] = Mw;
          in += w * vn * Mw;
        } else {
          ghost[i] = 0.0;
          if (vn != 0.0) out += w * vn * f_adj[i];
        }
      }
  double scale = kind == OR_INFLOW ? rho : -out / in;
  long K = (long)N * N * N;
  for (long i = 0; i < K; i++) ghost[i] *= scale;
  free(v);
}

/* Neighbour of cell (i, j) across side s, or its ghost (computed into buf). */
/* Second-order scheme in 2-D: the slopes of eq. (slope) in each direction, x along each row
 * and y along each column (central inside, one-sided in the end cells; zero for the
 * first-order scheme or a single cell in that direction). */
static void slopes2d(const or_problem2d* q, const double* f, double* sx, double* sy) {
  int nx = q->p.J, ny = q->ny, N = q->p.N;
  long K = (long)N * N * N;
  int o2 = q->p.order == 2;
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      long c = (long)j * nx + i;
      for (long k = 0; k < K; k++) {
        double a = 0.0, b = 0.0;
        if (o2 && nx >= 2) {
          if (i == 0)
            a = f[(c + 1) * K + k] - f[c * K + k];
          else if (i == nx - 1)
            a = f[c * K + k] - f[(c - 1) * K + k];
          else
            a = 0.5 * (f[(c + 1) * K + k] - f[(c - 1) * K + k]);
        }
        if (o2 && ny >= 2) {
          if (j == 0)
            b = f[(c + nx) * K + k] - f[c * K + k];
          else if (j == ny - 1)
            b = f[c * K + k] - f[(c - nx) * K + k];
          else
            b = 0.5 * (f[(c + nx) * K + k] - f[(c - nx) * K + k]);
        }
        sx[c * K + k] = a;
        sy[c * K + k] = b;
      }
    }
}

/* The neighbour across side s, or the wall ghost built from the outgoing face value of the
 * cell itself (f -/+ s/2 of the slope normal to that side; the cell value at first order). */
static const double* neighbour_face(const or_problem2d* q, const double* f, const double* sx, const double* sy,
                                    int i, int j, int s, double* buf, double* face) {
  int nx = q->p.J, ny = q->ny, N = q->p.N;
  long K = (long)N * N * N;
  int ii = i + (s == 1) - (s == 0), jj = j + (s == 3) - (s == 2);
  if (ii >= 0 && ii < nx && jj >= 0 && jj < ny) return f + ((long)jj * nx + ii) * K;
  long c = (long)j * nx + i;
  const double* sl = (s < 2 ? sx : sy) + c * K;
  double sign = (s == 0 || s == 2) ? -0.5 : 0.5;
  for (long k = 0; k < K; k++) face[k] = f[c * K + k] + sign * sl[k];
  or_ghost2d(q, s, face, buf);
  return buf;
}

double or_dx2d(const or_problem2d* q) { return (q->p.x_hi - q->p.x_lo) / q->p.J; }
double or_dy2d(const or_problem2d* q) { return (q->y_hi - q->y_lo) / q->ny; }

/* One sweep in ordering o: 0 = SW->NE (i and j ascending), 1 = NE->SW (both descending),
 * 2 = NW->SE (i ascending, j descending), 3 = SE->NW (i descending, j ascending). A cell
 * visit uses the latest values of its four neighbours and wall ghosts from its own value
 * stored before the visit. P, nu from the collision evaluation that preceded the sweep. */
void or_sweep2d(const or_problem2d* q, int o, double* f, const double* P, const double* nu, const double* b,
                or_stats* st) {
  /* Second order: the slopes are explicit, taken from the state before this ordering, and
   * enter r as -(v1^+ sx_W - v1 sx + v1^- sx_E)/(2 dx) - (v2^+ sy_S - v2 sy + v2^- sy_N)/(2 dy)
   * with zero slopes beyond the walls; wall ghosts from the outgoing face values. */
  int nx = q->p.J, ny = q->ny, N = q->p.N;
  long K = (long)N * N * N;
  double dx = or_dx2d(q), dy = or_dy2d(q), eps = q->p.eps;
  int dirx = (o == 0 || o == 2) ? 1 : -1;
  int diry = (o == 0 || o == 3) ? 1 : -1;
  int o2 = q->p.order == 2;
  double* v = (double*)malloc(sizeof(double) * N);
  double* c = (double*)malloc(sizeof(double) * K);
  double* r = (double*)malloc(sizeof(double) * K);
  double* face = (double*)malloc(sizeof(double) * K);
  double* sx = (double*)malloc(sizeof(double) * nx * ny * K);
  double* sy = (double*)malloc(sizeof(double) * nx * ny * K);
  double* gb[4];
  for (int s = 0; s < 4; s++) gb[s] = (double*)malloc(sizeof(double) * K);
  or_velocity_nodes(N, q->p.L, v);
  slopes2d(q, f, sx, sy);
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int i3 = 0; i3 < N; i3++) c[((long)i1 * N + i2) * N + i3] = fabs(v[i1]) / dx + fabs(v[i2]) / dy;
  for (int jj = 0; jj < ny; jj++) {
    int j = diry > 0 ? jj : ny - 1 - jj;
    for (int ii = 0; ii < nx; ii++) {
      int i = dirx > 0 ? ii : nx - 1 - ii;
      long cell = (long)j * nx + i;
      const double* nb[4];
      for (int s = 0; s < 4; s++) nb[s] = neighbour_face(q, f, sx, sy, i, j, s, gb[s], face);
      for (int i1 = 0; i1 < N; i1++) {
        double v1p = v[i1] > 0.0 ? v[i1] : 0.0, v1m = v[i1] < 0.0 ? v[i1] : 0.0;
        for (int i2 = 0; i2 < N; i2++) {
          double v2p = v[i2] > 0.0 ? v[i2] : 0.0, v2m = v[i2] < 0.0 ? v[i2] : 0.0;
          for (int i3 = 0; i3 < N; i3++) {
            long k = ((long)i1 * N + i2) * N + i3;
            r[k] = (-v1p * nb[0][k] + v1m * nb[1][k]) / dx + (-v2p * nb[2][k] + v2m * nb[3][k]) / dy -
                   P[cell * K + k] / eps - (b ? b[cell * K + k] : 0.0);
            if (o2) {
              double xw = i > 0 ? sx[(cell - 1) * K + k] : 0.0, xe = i < nx - 1 ? sx[(cell + 1) * K + k] : 0.0;
              double ys = j > 0 ? sy[(cell - nx) * K + k] : 0.0, yn = j < ny - 1 ? sy[(cell + nx) * K + k] : 0.0;
              r[k] -= (v1p * xw - v[i1] * sx[cell * K + k] + v1m * xe) / (2.0 * dx) +
                      (v2p * ys - v[i2] * sy[cell * K + k] + v2m * yn) / (2.0 * dy);
            }
          }
        }
      }
      or_cell_solve_c(&q->p, c, r, nu[cell], f + cell * K, st);
    }
  }
  for (int s = 0; s < 4; s++) free(gb[s]);
  free(v);
  free(c);
  free(r);
  free(face);
  free(sx);
  free(sy);
}

/* Mass rescale (eq. (32)) with the cell area dx dy. */
void or_rescale2d(const or_problem2d* q, double* f) {
  int N = q->p.N;
  long K = (long)N * N * N, C = (long)q->p.J * q->ny;
  double w = weight2(N, q->p.L), tot = 0.0, area = or_dx2d(q) * or_dy2d(q);
  for (long c = 0; c < C; c++) {
    double rho = 0.0;
    for (long i = 0; i < K; i++) rho += w * f[c * K + i];
    tot += area * rho;
  }
  double lam = q->p.total_mass / tot;
  for (long i = 0; i < C * K; i++) f[i] *= lam;
}

/* Outer residual R = T(f) - Q/eps - b with ghosts from the same f; returns
 * sqrt(dx dy sum_cells sum_k w R^2). Rout may be NULL. */
double or_residual2d(const or_problem2d* q, const double* f, const double* Q, const double* b, double* Rout) {
  /* The 2-D upwind residual with the face values of the reconstruction in each direction
   * (the cell values at first order) and wall ghosts from the outgoing face values. */
  int nx = q->p.J, ny = q->ny, N = q->p.N;
  long K = (long)N * N * N;
  double dx = or_dx2d(q), dy = or_dy2d(q), w = weight2(N, q->p.L), acc = 0.0;
  double* v = (double*)malloc(sizeof(double) * N);
  double* face = (double*)malloc(sizeof(double) * K);
  double* sx = (double*)malloc(sizeof(double) * nx * ny * K);
  double* sy = (double*)malloc(sizeof(double) * nx * ny * K);
  double* gb[4];
  for (int s = 0; s < 4; s++) gb[s] = (double*)malloc(sizeof(double) * K);
  or_velocity_nodes(N, q->p.L, v);
  slopes2d(q, f, sx, sy);
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      long cell = (long)j * nx + i;
      const double* fc = f + cell * K;
      const double* nb[4];
      for (int s = 0; s < 4; s++) nb[s] = neighbour_face(q, f, sx, sy, i, j, s, gb[s], face);
      /* slopes of the neighbours across each side (zero beyond a wall) */
      const double* sW = i > 0 ? sx + (cell - 1) * K : NULL;
      const double* sE = i < nx - 1 ? sx + (cell + 1) * K : NULL;
      const double* sS = j > 0 ? sy + (cell - nx) * K : NULL;
      const double* sN = j < ny - 1 ? sy + (cell + nx) * K : NULL;
      for (int i1 = 0; i1 < N; i1++) {
        double v1p = v[i1] > 0.0 ? v[i1] : 0.0, v1m = v[i1] < 0.0 ? v[i1] : 0.0;
        for (int i2 = 0; i2 < N; i2++) {
          double v2p = v[i2] > 0.0 ? v[i2] : 0.0, v2m = v[i2] < 0.0 ? v[i2] : 0.0;
          for (int i3 = 0; i3 < N; i3++) {
            long k = ((long)i1 * N + i2) * N + i3;
            double hx = 0.5 * sx[cell * K + k], hy = 0.5 * sy[cell * K + k];
            double xw = nb[0][k] + (sW ? 0.5 * sW[k] : 0.0), xe = nb[1][k] - (sE ? 0.5 * sE[k] : 0.0);
            double ys = nb[2][k] + (sS ? 0.5 * sS[k] : 0.0), yn = nb[3][k] - (sN ? 0.5 * sN[k] : 0.0);
            double R = (v1p * ((fc[k] + hx) - xw) + v1m * (xe - (fc[k] - hx))) / dx +
                       (v2p * ((fc[k] + hy) - ys) + v2m * (yn - (fc[k] - hy))) / dy - Q[cell * K + k] / q->p.eps -
                       (b ? b[cell * K + k] : 0.0);
            if (Rout) Rout[cell * K + k] = R;
            acc += w * R * R;
          }
        }
      }
    }
  for (int s = 0; s < 4; s++) free(gb[s]);
  free(v);
  free(face);
  free(sx);
  free(sy);
  return sqrt(dx * dy * acc);
}

/* One SGS iteration in 2-D: the four orderings, each preceded by a collision evaluation,
 * then the mass rescale (if enabled and rescale != 0). */
void or_sgs_iteration2d(const or_problem2d* q, double* f, const double* b, int rescale, or_stats* st) {
  long K = (long)q->p.N * q->p.N * q->p.N, C = (long)q->p.J * q->ny;
  double* P = (double*)malloc(sizeof(double) * C * K);
  double* nu = (double*)malloc(sizeof(double) * C);
  for (int o = 0; o < 4; o++) {
    or_collide(&q->p, (int)C, f, NULL, P, nu);
    or_sweep2d(q, o, f, P, nu, b, st);
  }
  if (rescale && q->p.total_mass > 0.0) or_rescale2d(q, f);
  free(P);
  free(nu);
}

/* ------------------------------------------------------------------------------------
 * FAS V-cycle (eq. (30)) with 2 x 2 coarsening: restriction = mean of the four children,
 * prolongation = piecewise-constant injection of f_H - I fbar_h, coarse right-hand side
 * b_H = R_H(I fbar_h) + I(b_h - R_h(fbar_h)); rescale on the finest level only.
 * ---------------------------------------------------------------------------------- */
static void restrict2d(int nx, int ny, long K, const double* fine, double* coarse) {
  int cx = nx / 2, cy = ny / 2;
  for (int j = 0; j < cy; j++)
    for (int i = 0; i < cx; i++) {
      double* dst = coarse + ((long)j * cx + i) * K;
      const double* a = fine + ((long)(2 * j) * nx + 2 * i) * K;
      const double* b = fine + ((long)(2 * j) * nx + 2 * i + 1) * K;
      const double* c = fine + ((long)(2 * j + 1) * nx + 2 * i) * K;
      const double* d = fine + ((long)(2 * j + 1) * nx + 2 * i + 1) * K;
      for (long k = 0; k < K; k++) dst[k] = 0.25 * (a[k] + b[k] + c[k] + d[k]);
    }
}

static void vcycle2d_level(const or_problem2d* q, double* f, const double* b, int levels, int pre, int post,
                           int coarse_iters, int finest, or_stats* st) {
  int nx = q->p.J, ny = q->ny;
  long K = (long)q->p.N * q->p.N * q->p.N, C = (long)nx * ny;
  if (levels <= 1) {
    for (int it = 0; it < coarse_iters; it++) or_sgs_iteration2d(q, f, b, finest, st);
    return;
  }
  for (int it = 0; it < pre; it++) or_sgs_iteration2d(q, f, b, finest, st);
  or_problem2d qc = *q;
  qc.p.J = nx / 2;
  qc.ny = ny / 2;
  long CC = (long)qc.p.J * qc.ny;
  double* Q = (double*)malloc(sizeof(double) * C * K);
  double* nu = (double*)malloc(sizeof(double) * C);
  double* R = (double*)malloc(sizeof(double) * C * K);
  or_collide(&q->p, (int)C, f, Q, NULL, nu);
  or_residual2d(q, f, Q, b, R);
  double* fH0 = (double*)malloc(sizeof(double) * CC * K);
  double* fH = (double*)malloc(sizeof(double) * CC * K);
  double* RH = (double*)malloc(sizeof(double) * CC * K);
  double* bH = (double*)malloc(sizeof(double) * CC * K);
  double* QH = (double*)malloc(sizeof(double) * CC * K);
  double* nuH = (double*)malloc(sizeof(double) * CC);
  restrict2d(nx, ny, K, f, fH0);
  restrict2d(nx, ny, K, R, RH);
  or_collide(&qc.p, (int)CC, fH0, QH, NULL, nuH);
  or_residual2d(&qc, fH0, QH, NULL, bH);  /* bH = R_H(I f) */
  for (long k = 0; k < CC * K; k++) bH[k] -= RH[k];
  memcpy(fH, fH0, sizeof(double) * CC * K);
  vcycle2d_level(&qc, fH, bH, levels - 1, pre, post, coarse_iters, 0, st);
  int cx = qc.p.J;
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      long cf = (long)j * nx + i, cc = (long)(j / 2) * cx + i / 2;
      for (long k = 0; k < K; k++) f[cf * K + k] += fH[cc * K + k] - fH0[cc * K + k];
    }
  for (int it = 0; it < post; it++) or_sgs_iteration2d(q, f, b, finest, st);
  free(Q);
  free(nu);
  free(R);
  free(fH0);
  free(fH);
  free(RH);
  free(bH);
  free(QH);
  free(nuH);
}

void or_vcycle2d(const or_problem2d* q, double* f, int levels, int pre, int post, int coarse_iters, or_stats* st) {
  vcycle2d_level(q, f, NULL, levels, pre, post, coarse_iters, 1, st);
}
