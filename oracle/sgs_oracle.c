/*
 * Plain FP64 CPU oracle for the SGS-PFP steady Boltzmann solver.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests, the smoke check and the CPU-baseline leg
 * of the benchmark; never by the CUDA library. It shares no code, header, table or
 * helper with the CUDA path. Everything is written for a reader checking it against
 * the paper by eye: no blocking, fusion or reordering beyond the separable DFT.
 *
 * Parity status: every function here is pinned by a CPU test against something other
 * than itself (closed forms, brute-force quadrature, invariants, library routines);
 * see the test files under tests/ whose names start with test_oracle_.
 */
#include "sgs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------------------
 * Velocity grid (Section 2.2): periodic grid v = (k1 dv, k2 dv, k3 dv) with
 * k_i in {-N/2+1, ..., N/2} and dv = 2L/N; all quadrature weights equal dv^3.
 * ---------------------------------------------------------------------------------- */
void or_velocity_nodes(int N, double L, double* out) {
  double dv = 2.0 * L / N;
  for (int i = 0; i < N; i++) out[i] = (double)(i - N / 2 + 1) * dv;
}

static double weight(int N, double L) {
  double dv = 2.0 * L / N;
  return dv * dv * dv;
}

/* ------------------------------------------------------------------------------------
 * Gauss-Legendre rule on [-1, 1]: roots of P_n by Newton from cos(pi (i + 3/4)/(n + 1/2)),
 * P_n from the three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},
 * weights 2 / ((1 - x^2) P_n'(x)^2).
 * ---------------------------------------------------------------------------------- */
void or_gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; i++) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; k++) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      /* p1 = P_n(z), p0 = P_{n-1}(z) */
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) {
        /* refresh the derivative at the converged root */
        p0 = 1.0; p1 = z;
        for (int k = 1; k < n; k++) {
          double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* ------------------------------------------------------------------------------------
 * Spectral weights of the Fourier-Galerkin collision operator (Section 2.2 and the
 * binary-collision setup of Section 4.2: compact support B(0, R), box [-L, L]^3,
 * L = (3 sqrt 2 + 1) R / 2).
 *
 * With f(v) = sum_k fhat_k exp(i xi k.v), xi = pi/L, and the relative velocity q = v - v_*
 * truncated to |q| <= 2R, the collision integral (eq. (2)) maps the pair (l, m) of
 * modes to mode l + m with weight
 *   gain: int_{|q|<=2R} int_{S^2} B e^{-i xi [(l+m).q + |q| (l-m).w]/2} dw dq
 *       = 16 pi^2 int_0^{2R} rho^2 B(rho) sinc(xi rho |l+m|/2) sinc(xi rho |l-m|/2) drho
 *       = G(|l+m|, |l-m|),
 *   loss (mode l on f(v_*), m on f(v)): int int B e^{-i xi l.q} dw dq = G(2|l|, 0),
 * using int_{S^2} exp(-i a.w) dw = 4 pi sinc|a| twice. G depends on its arguments only
 * through the integers a^2 and b^2. The oracle evaluates the radial integral by
 * adaptive Gauss-Legendre quadrature.
 * ---------------------------------------------------------------------------------- */
#define GL_N 20
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

static void gl_init(void) {
  if (!gl_ready) {
    or_gauss_legendre(GL_N, gl_x, gl_w);
    gl_ready = 1;
  }
}

static double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

typedef struct {
  int kernel;
  double b0, c, a, b;
} g_integrand;

static double g_f(const g_integrand* g, double rho) {
  double B = g->kernel == OR_HARD_SPHERE ? g->b0 * rho : g->b0;
  return 16.0 * M_PI * M_PI * rho * rho * B * sinc(g->c * g->a * rho) * sinc(g->c * g->b * rho);
}

static double gl_panel(const g_integrand* g, double lo, double hi) {
  double h = 0.5 * (hi - lo), mid = 0.5 * (hi + lo), s = 0.0;
  for (int i = 0; i < GL_N; i++) s += gl_w[i] * g_f(g, mid + h * gl_x[i]);
  return s * h;
}

static double gl_adapt(const g_integrand* g, double lo, double hi, double whole, double tol, int depth) {
  double mid = 0.5 * (lo + hi);
  double left = gl_panel(g, lo, mid), right = gl_panel(g, mid, hi);
  if (depth >= 30 || fabs(left + right - whole) <= tol) return left + right;
  return gl_adapt(g, lo, mid, left, tol, depth + 1) + gl_adapt(g, mid, hi, right, tol, depth + 1);
}

static double support_radius(double L) { return 2.0 * L / (3.0 * sqrt(2.0) + 1.0); }

double or_G(int N, double L, int kernel, double b0, long a2, long b2) {
  (void)N;
  gl_init();
  g_integrand g;
  g.kernel = kernel;
  g.b0 = b0;
  g.c = M_PI / (2.0 * L);
  g.a = sqrt((double)a2);
  g.b = sqrt((double)b2);
  double R2 = 2.0 * support_radius(L);
  /* scale of the integral: its value at a = b = 0 */
  double scale = kernel == OR_HARD_SPHERE ? 16.0 * M_PI * M_PI * b0 * pow(R2, 4) / 4.0
                                          : 16.0 * M_PI * M_PI * b0 * pow(R2, 3) / 3.0;
  double tol = 1e-17 * scale;
  const int panels = 16;
  double s = 0.0;
  for (int p = 0; p < panels; p++) {
    double lo = R2 * p / panels, hi = R2 * (p + 1) / panels;
    s += gl_adapt(&g, lo, hi, gl_panel(&g, lo, hi), tol, 0);
  }
  return s;
}

/* Tables for one (N, L, kernel, b0): gain G(a2, b2), a2 in [0, 3h^2], b2 in [0, 12h^2];
 * loss Lt(m2) = G(4 m2, 0), m2 in [0, 3h^2]. */
typedef struct {
  int N, kernel;
  double L, b0;
  long na, nb;
  double* gain;
  double* loss;
} g_tables;

static g_tables cache = {0, 0, 0.0, 0.0, 0, 0, NULL, NULL};

static const g_tables* tables(int N, double L, int kernel, double b0) {
  if (cache.gain && cache.N == N && cache.L == L && cache.kernel == kernel && cache.b0 == b0) return &cache;
  free(cache.gain);
  free(cache.loss);
  long h = N / 2 - 1;
  cache.N = N;
  cache.L = L;
  cache.kernel = kernel;
  cache.b0 = b0;
  cache.na = 3 * h * h + 1;
  cache.nb = 12 * h * h + 1;
  cache.gain = (double*)malloc(sizeof(double) * cache.na * cache.nb);
  cache.loss = (double*)malloc(sizeof(double) * cache.na);
  gl_init();
#pragma omp parallel for schedule(dynamic)
  for (long a2 = 0; a2 < cache.na; a2++) {
    for (long b2 = 0; b2 < cache.nb; b2++) cache.gain[a2 * cache.nb + b2] = or_G(N, L, kernel, b0, a2, b2);
    cache.loss[a2] = or_G(N, L, kernel, b0, 4 * a2, 0);
  }
  return &cache;
}

/* ------------------------------------------------------------------------------------
 * Discrete Fourier transform on the periodic grid (Section 2.2):
 *   fhat_k = N^-3 sum_v f(v) exp(-i pi k.v / L),  |k_i| <= h,
 * with pi k.v/L = 2 pi k j / N for v = j dv. Evaluated one dimension at a time.
 * ---------------------------------------------------------------------------------- */
static void twiddles(int N, int sign, double* c, double* s) {
  int h = N / 2 - 1, n = 2 * h + 1;
  for (int k = -h; k <= h; k++)
    for (int i = 0; i < N; i++) {
      int j = i - N / 2 + 1;
      long kj = ((long)k * j) % N;
      if (kj < 0) kj += N;
      double ang = 2.0 * M_PI * (double)kj / N;
      c[(k + h) * N + i] = cos(ang);
      s[(k + h) * N + i] = sign * sin(ang);
    }
  (void)n;
}

void or_dft(int N, const double* f, double* fhat) {
  int h = N / 2 - 1, n = 2 * h + 1;
  double* c = (double*)malloc(sizeof(double) * n * N);
  double* s = (double*)malloc(sizeof(double) * n * N);
  twiddles(N, -1, c, s);
  /* stage A: transform index 3: a[i1][i2][k3] */
  double* a = (double*)malloc(sizeof(double) * 2 * N * N * n);
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int k = 0; k < n; k++) {
        double re = 0, im = 0;
        for (int i3 = 0; i3 < N; i3++) {
          double v = f[((long)i1 * N + i2) * N + i3];
          re += v * c[k * N + i3];
          im += v * s[k * N + i3];
        }
        long o = (((long)i1 * N + i2) * n + k) * 2;
        a[o] = re;
        a[o + 1] = im;
      }
  /* stage B: index 2: b[i1][k2][k3] */
  double* b = (double*)malloc(sizeof(double) * 2 * N * n * n);
  for (int i1 = 0; i1 < N; i1++)
    for (int k2 = 0; k2 < n; k2++)
      for (int k3 = 0; k3 < n; k3++) {
        double re = 0, im = 0;
        for (int i2 = 0; i2 < N; i2++) {
          long o = (((long)i1 * N + i2) * n + k3) * 2;
          double cr = c[k2 * N + i2], ci = s[k2 * N + i2];
          re += a[o] * cr - a[o + 1] * ci;
          im += a[o] * ci + a[o + 1] * cr;
        }
        long o = (((long)i1 * n + k2) * n + k3) * 2;
        b[o] = re;
        b[o + 1] = im;
      }
  /* stage C: index 1 */
  double scale = 1.0 / ((double)N * N * N);
  for (int k1 = 0; k1 < n; k1++)
    for (int k2 = 0; k2 < n; k2++)
      for (int k3 = 0; k3 < n; k3++) {
        double re = 0, im = 0;
        for (int i1 = 0; i1 < N; i1++) {
          long o = (((long)i1 * n + k2) * n + k3) * 2;
          double cr = c[k1 * N + i1], ci = s[k1 * N + i1];
          re += b[o] * cr - b[o + 1] * ci;
          im += b[o] * ci + b[o + 1] * cr;
        }
        long o = (((long)k1 * n + k2) * n + k3) * 2;
        fhat[o] = re * scale;
        fhat[o + 1] = im * scale;
      }
  free(a);
  free(b);
  free(c);
  free(s);
}

void or_idft(int N, const double* qhat, double* q) {
  int h = N / 2 - 1, n = 2 * h + 1;
  double* c = (double*)malloc(sizeof(double) * n * N);
  double* s = (double*)malloc(sizeof(double) * n * N);
  twiddles(N, +1, c, s);
  /* stage A: index 1: a[i1][k2][k3] */
  double* a = (double*)malloc(sizeof(double) * 2 * N * n * n);
  for (int i1 = 0; i1 < N; i1++)
    for (int k2 = 0; k2 < n; k2++)
      for (int k3 = 0; k3 < n; k3++) {
        double re = 0, im = 0;
        for (int k1 = 0; k1 < n; k1++) {
          long o = (((long)k1 * n + k2) * n + k3) * 2;
          double cr = c[k1 * N + i1], ci = s[k1 * N + i1];
          re += qhat[o] * cr - qhat[o + 1] * ci;
          im += qhat[o] * ci + qhat[o + 1] * cr;
        }
        long o = (((long)i1 * n + k2) * n + k3) * 2;
        a[o] = re;
        a[o + 1] = im;
      }
  /* stage B: index 2: b[i1][i2][k3] */
  double* b = (double*)malloc(sizeof(double) * 2 * N * N * n);
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int k3 = 0; k3 < n; k3++) {
        double re = 0, im = 0;
        for (int k2 = 0; k2 < n; k2++) {
          long o = (((long)i1 * n + k2) * n + k3) * 2;
          double cr = c[k2 * N + i2], ci = s[k2 * N + i2];
          re += a[o] * cr - a[o + 1] * ci;
          im += a[o] * ci + a[o + 1] * cr;
        }
        long o = (((long)i1 * N + i2) * n + k3) * 2;
        b[o] = re;
        b[o + 1] = im;
      }
  /* stage C: index 3, real part */
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int i3 = 0; i3 < N; i3++) {
        double re = 0;
        for (int k3 = 0; k3 < n; k3++) {
          long o = (((long)i1 * N + i2) * n + k3) * 2;
          re += b[o] * c[k3 * N + i3] - b[o + 1] * s[k3 * N + i3];
        }
        q[((long)i1 * N + i2) * N + i3] = re;
      }
  free(a);
  free(b);
  free(c);
  free(s);
}

/* ------------------------------------------------------------------------------------
 * Fourier-Galerkin bilinear sum (Fourier spectral method, Section 2.2):
 *   qhat_k = sum_{m : |m_i| <= h, |k_i - m_i| <= h} beta(k - m, m) ahat_{k-m} bhat_m,
 *   beta(l, m) = G(|l+m|, |l-m|) - G(2|m|, 0),
 * no wrap-around (the aliasing-free truncation of the periodic method).
 * ---------------------------------------------------------------------------------- */
void or_qhat_direct(int N, double L, int kernel, double b0, const double* ahat, const double* bhat, double* qhat) {
  const g_tables* t = tables(N, L, kernel, b0);
  int h = N / 2 - 1, n = 2 * h + 1;
  for (int k1 = -h; k1 <= h; k1++)
    for (int k2 = -h; k2 <= h; k2++)
      for (int k3 = -h; k3 <= h; k3++) {
        long a2 = (long)k1 * k1 + (long)k2 * k2 + (long)k3 * k3;
        const double* grow = t->gain + a2 * t->nb;
        double re = 0.0, im = 0.0;
        for (int m1 = (k1 - h > -h ? k1 - h : -h); m1 <= (k1 + h < h ? k1 + h : h); m1++)
          for (int m2 = (k2 - h > -h ? k2 - h : -h); m2 <= (k2 + h < h ? k2 + h : h); m2++)
            for (int m3 = (k3 - h > -h ? k3 - h : -h); m3 <= (k3 + h < h ? k3 + h : h); m3++) {
              int l1 = k1 - m1, l2 = k2 - m2, l3 = k3 - m3;
              long d1 = l1 - m1, d2 = l2 - m2, d3 = l3 - m3;
              long b2 = d1 * d1 + d2 * d2 + d3 * d3;
              long mm = (long)m1 * m1 + (long)m2 * m2 + (long)m3 * m3;
              double beta = grow[b2] - t->loss[mm];
              long ol = (((long)(l1 + h) * n + (l2 + h)) * n + (l3 + h)) * 2;
              long om = (((long)(m1 + h) * n + (m2 + h)) * n + (m3 + h)) * 2;
              double ar = ahat[ol], ai = ahat[ol + 1], br = bhat[om], bi = bhat[om + 1];
              re += beta * (ar * br - ai * bi);
              im += beta * (ar * bi + ai * br);
            }
        long o = (((long)(k1 + h) * n + (k2 + h)) * n + (k3 + h)) * 2;
        qhat[o] = re;
        qhat[o + 1] = im;
      }
}

void or_qfsm(int N, double L, int kernel, double b0, const double* f, double* q) {
  int h = N / 2 - 1, n = 2 * h + 1;
  long nm = (long)n * n * n;
  double* fhat = (double*)malloc(sizeof(double) * 2 * nm);
  double* qhat = (double*)malloc(sizeof(double) * 2 * nm);
  or_dft(N, f, fhat);
  or_qhat_direct(N, L, kernel, b0, fhat, fhat, qhat);
  or_idft(N, qhat, q);
  free(fhat);
  free(qhat);
}

/* ------------------------------------------------------------------------------------
 * Moments (eq. (6)) by the velocity quadrature (eq. (10)): phi = (1, v1, v2, v3, |v|^2).
 * ---------------------------------------------------------------------------------- */
void or_moments(int N, double L, const double* f, double* m5) {
  double* v = (double*)malloc(sizeof(double) * N);
  or_velocity_nodes(N, L, v);
  double w = weight(N, L);
  for (int q = 0; q < 5; q++) m5[q] = 0.0;
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int i3 = 0; i3 < N; i3++) {
        double x = w * f[((long)i1 * N + i2) * N + i3];
        m5[0] += x;
        m5[1] += x * v[i1];
        m5[2] += x * v[i2];
        m5[3] += x * v[i3];
        m5[4] += x * (v[i1] * v[i1] + v[i2] * v[i2] + v[i3] * v[i3]);
      }
  free(v);
}

/* ------------------------------------------------------------------------------------
 * Macroscopic quantities of one cell by the velocity quadrature: rho, U and T as defined
 * with the moments (eq. (6) and the definitions beside it, d = 3), and the heat flux of the
 * lid-driven cavity study (Section 4.2.2), q = 1/2 int (v - U) |v - U|^2 f dv.
 * out = (rho, U1, U2, U3, T, q1, q2, q3). U first, then the central sums about it.
 * ---------------------------------------------------------------------------------- */
void or_macroscopic(int N, double L, const double* f, double* out) {
  double* v = (double*)malloc(sizeof(double) * N);
  or_velocity_nodes(N, L, v);
  double w = weight(N, L);
  double rho = 0.0, mom[3] = {0.0, 0.0, 0.0};
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int i3 = 0; i3 < N; i3++) {
        double x = w * f[((long)i1 * N + i2) * N + i3];
        rho += x;
        mom[0] += x * v[i1];
        mom[1] += x * v[i2];
        mom[2] += x * v[i3];
      }
  double U[3] = {mom[0] / rho, mom[1] / rho, mom[2] / rho};
  double e2 = 0.0, q[3] = {0.0, 0.0, 0.0};
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int i3 = 0; i3 < N; i3++) {
        double x = w * f[((long)i1 * N + i2) * N + i3];
        double c[3] = {v[i1] - U[0], v[i2] - U[1], v[i3] - U[2]};
        double c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        e2 += x * c2;
        for (int d = 0; d < 3; d++) q[d] += 0.5 * x * c[d] * c2;
      }
  out[0] = rho;
  for (int d = 0; d < 3; d++) out[1 + d] = U[d];
  out[4] = e2 / (3.0 * rho);
  for (int d = 0; d < 3; d++) out[5 + d] = q[d];
  free(v);
}

/* ------------------------------------------------------------------------------------
 * Discrete Maxwellian (eqs. (13)-(14)): M_k = exp(alpha + beta.v_k - gamma |v_k|^2)
 * whose weighted moments sum_k wk_k phi(v_k) M_k equal a target. Newton's method on
 * theta = (alpha, beta, gamma): F(theta) = sum wk phi M - target, Jacobian A D with
 * A = sum wk M phi phi^T (symmetric positive definite) and D = diag(1,1,1,1,-1).
 * The step is halved while the scaled residual grows; after the exponent change
 * |d alpha| + L sum|d beta| + L^2 |d gamma| drops below tol one more step is taken.
 * ---------------------------------------------------------------------------------- */
static void newton_eval(int N, const double* v, double w, const double* wk, const double* target,
                        const double* th, double* F, double* A) {
  double s[5] = {0, 0, 0, 0, 0}, a[15];
  for (int q = 0; q < 15; q++) a[q] = 0.0;
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int i3 = 0; i3 < N; i3++) {
        long idx = ((long)i1 * N + i2) * N + i3;
        double vv = v[i1] * v[i1] + v[i2] * v[i2] + v[i3] * v[i3];
        double M = exp(th[0] + th[1] * v[i1] + th[2] * v[i2] + th[3] * v[i3] - th[4] * vv);
        double x = (wk ? wk[idx] : w) * M;
        double phi[5] = {1.0, v[i1], v[i2], v[i3], vv};
        int t = 0;
        for (int i = 0; i < 5; i++) {
          s[i] += x * phi[i];
          for (int j = i; j < 5; j++) a[t++] += x * phi[i] * phi[j];
        }
      }
  for (int i = 0; i < 5; i++) F[i] = s[i] - target[i];
  int t = 0;
  for (int i = 0; i < 5; i++)
    for (int j = i; j < 5; j++) {
      A[i * 5 + j] = a[t];
      A[j * 5 + i] = a[t];
      t++;
    }
}

/* Solve A y = b for symmetric positive definite 5x5 A by Cholesky; returns 0 on success. */
static int chol5(const double* A, const double* b, double* y) {
  double Lm[25];
  memset(Lm, 0, sizeof(Lm));
  for (int i = 0; i < 5; i++)
    for (int j = 0; j <= i; j++) {
      double s = A[i * 5 + j];
      for (int k = 0; k < j; k++) s -= Lm[i * 5 + k] * Lm[j * 5 + k];
      if (i == j) {
        if (!(s > 0.0)) return -1;
        Lm[i * 5 + i] = sqrt(s);
      } else {
        Lm[i * 5 + j] = s / Lm[j * 5 + j];
      }
    }
  double z[5];
  for (int i = 0; i < 5; i++) {
    double s = b[i];
    for (int k = 0; k < i; k++) s -= Lm[i * 5 + k] * z[k];
    z[i] = s / Lm[i * 5 + i];
  }
  for (int i = 4; i >= 0; i--) {
    double s = z[i];
    for (int k = i + 1; k < 5; k++) s -= Lm[k * 5 + i] * y[k];
    y[i] = s / Lm[i * 5 + i];
  }
  return 0;
}

static double fnorm(const double* F, const double* target) {
  double m = 0.0;
  for (int i = 0; i < 5; i++)
    if (fabs(F[i]) > m) m = fabs(F[i]);
  return m / fabs(target[0]);
}

int or_discrete_maxwellian(int N, double L, const double* wk, const double* target, double* theta, int use_guess,
                           double tol, int maxit) {
  if (!(target[0] > 0.0)) return -1;
  double* v = (double*)malloc(sizeof(double) * N);
  or_velocity_nodes(N, L, v);
  double w = weight(N, L);
  if (!use_guess) {
    /* continuum Maxwellian with the same moments, eq. (5) */
    double rho = target[0];
    double U[3] = {target[1] / rho, target[2] / rho, target[3] / rho};
    double U2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
    double T = (target[4] / rho - U2) / 3.0;
    if (!(T > 0.0)) {
      free(v);
      return -1;
    }
    theta[4] = 1.0 / (2.0 * T);
    theta[1] = U[0] / T;
    theta[2] = U[1] / T;
    theta[3] = U[2] / T;
    theta[0] = log(rho / pow(2.0 * M_PI * T, 1.5)) - U2 / (2.0 * T);
  }
  double F[5], A[25], Ft[5], At[25], th[5];
  newton_eval(N, v, w, wk, target, theta, F, A);
  double fn = fnorm(F, target);
  int done = 0, it = 0, ok = 0;
  for (it = 0; it < maxit; it++) {
    double y[5], d[5];
    if (chol5(A, F, y) != 0) break;
    for (int i = 0; i < 5; i++) d[i] = -y[i];
    d[4] = -d[4]; /* delta = -D A^{-1} F */
    double lam = 1.0;
    for (int hv = 0; hv < 40; hv++) {
      for (int i = 0; i < 5; i++) th[i] = theta[i] + lam * d[i];
      newton_eval(N, v, w, wk, target, th, Ft, At);
      double fnt = fnorm(Ft, target);
      if (fnt == fnt && (fnt <= fn || fnt <= 1e-10)) {
        fn = fnt;
        break;
      }
      lam *= 0.5;
    }
    memcpy(theta, th, sizeof(th));
    memcpy(F, Ft, sizeof(Ft));
    memcpy(A, At, sizeof(At));
    double step = lam * (fabs(d[0]) + L * (fabs(d[1]) + fabs(d[2]) + fabs(d[3])) + L * L * fabs(d[4]));
    if (!(step == step)) break;
    if (done) {
      ok = 1;
      it++;
      break;
    }
    if (step <= tol) done = 1;
  }
  free(v);
  return ok ? it : -1;
}

void or_eval_maxwellian(int N, double L, const double* th, double* M) {
  double* v = (double*)malloc(sizeof(double) * N);
  or_velocity_nodes(N, L, v);
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int i3 = 0; i3 < N; i3++) {
        double vv = v[i1] * v[i1] + v[i2] * v[i2] + v[i3] * v[i3];
        M[((long)i1 * N + i2) * N + i3] = exp(th[0] + th[1] * v[i1] + th[2] * v[i2] + th[3] * v[i3] - th[4] * vv);
      }
  free(v);
}

/* ------------------------------------------------------------------------------------
 * Collision frequency nu of the BGK penalty (eq. (28)). Maxwell molecules: the loss
 * rate int int B dw f(v_*) dv_* = 4 pi b0 rho. Hard spheres (B = b0 |q|, truncated at
 * |q| <= 2R): the supremum of the loss rate, 4 pi b0 rho 2R, so that P keeps no stiff part
 * of the loss term (the loss rate grows with |v - U|; with its Maxwellian average the
 * explicitly treated remainder makes SGS diverge on a Mach-2 shock). nu only shapes the
 * iterates, not the converged solution. BGK mode uses the Maxwell value.
 * ---------------------------------------------------------------------------------- */
double or_collision_frequency(const or_problem* p, const double* f) {
  double m[5];
  or_moments(p->N, p->L, f, m);
  double rho = m[0];
  if (p->kernel == OR_HARD_SPHERE) {
    /* sup of the loss frequency of the truncated kernel b0 |q|, |q| <= 2R */
    double R = 2.0 * p->L / (3.0 * sqrt(2.0) + 1.0);
    return 4.0 * M_PI * p->b0 * rho * 2.0 * R;
  }
  return 4.0 * M_PI * p->b0 * rho;
}

/* ------------------------------------------------------------------------------------
 * Conservation projection (not in the paper, whose Fourier-spectral Q conserves mass to
 * round-off but momentum and energy only to spectral accuracy). With C = [w phi_i(v_k)]
 * (5 x K), the smallest Euclidean change of q that makes C q = 0 is
 *   q_c = q - C^T (C C^T)^{-1} C q;
 * the uniform weight w cancels, so lambda solves (sum_k phi phi^T) lambda = sum_k phi q
 * and q_c = q - sum_i lambda_i phi_i. Written out over the nodes in plain loops.
 * ---------------------------------------------------------------------------------- */
int or_conserve_project(int N, double L, double* q) {
  double* v = (double*)malloc(sizeof(double) * N);
  or_velocity_nodes(N, L, v);
  double A[25], s[5], lam[5];
  memset(A, 0, sizeof(A));
  memset(s, 0, sizeof(s));
  long t = 0;
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int i3 = 0; i3 < N; i3++, t++) {
        double phi[5] = {1.0, v[i1], v[i2], v[i3], v[i1] * v[i1] + v[i2] * v[i2] + v[i3] * v[i3]};
        for (int a = 0; a < 5; a++) {
          s[a] += phi[a] * q[t];
          for (int b = 0; b < 5; b++) A[a * 5 + b] += phi[a] * phi[b];
        }
      }
  int ok = chol5(A, s, lam);
  if (ok == 0) {
    t = 0;
    for (int i1 = 0; i1 < N; i1++)
      for (int i2 = 0; i2 < N; i2++)
        for (int i3 = 0; i3 < N; i3++, t++) {
          double phi[5] = {1.0, v[i1], v[i2], v[i3], v[i1] * v[i1] + v[i2] * v[i2] + v[i3] * v[i3]};
          for (int a = 0; a < 5; a++) q[t] -= lam[a] * phi[a];
        }
  }
  free(v);
  return ok;
}

/* Weighted variant: minimising sum_k (q_c - q)^2 / M_k under the same five constraints
 * gives q_c = q - M sum_i lambda_i phi_i with (sum_k M phi phi^T) lambda = sum_k phi q, so the
 * correction lives where the local Maxwellian M does and leaves the far tails untouched. */
int or_conserve_project_w(int N, double L, const double* M, double* q) {
  double* v = (double*)malloc(sizeof(double) * N);
  or_velocity_nodes(N, L, v);
  double A[25], s[5], lam[5];
  memset(A, 0, sizeof(A));
  memset(s, 0, sizeof(s));
  long t = 0;
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int i3 = 0; i3 < N; i3++, t++) {
        double phi[5] = {1.0, v[i1], v[i2], v[i3], v[i1] * v[i1] + v[i2] * v[i2] + v[i3] * v[i3]};
        for (int a = 0; a < 5; a++) {
          s[a] += phi[a] * q[t];
          for (int b = 0; b < 5; b++) A[a * 5 + b] += M[t] * phi[a] * phi[b];
        }
      }
  int ok = chol5(A, s, lam);
  if (ok == 0) {
    t = 0;
    for (int i1 = 0; i1 < N; i1++)
      for (int i2 = 0; i2 < N; i2++)
        for (int i3 = 0; i3 < N; i3++, t++) {
          double phi[5] = {1.0, v[i1], v[i2], v[i3], v[i1] * v[i1] + v[i2] * v[i2] + v[i3] * v[i3]};
          double c = 0.0;
          for (int a = 0; a < 5; a++) c += lam[a] * phi[a];
          q[t] -= M[t] * c;
        }
  }
  free(v);
  return ok;
}

/* ------------------------------------------------------------------------------------
 * Steady-state-preserving collision term (eq. (16)):
 *   Q = Q^FSM[f, f] - Q^FSM[M[f], M[f]]
 * and the BGK penalty split P = Q - nu (M - f) (eq. (28)). BGK mode: Q = nu (M - f),
 * P = 0 (eq. (12)). With conserve_proj, Q is projected (above) before P is formed.
 * ---------------------------------------------------------------------------------- */
void or_collide_cell(const or_problem* p, const double* f, double* Q, double* P, double* nu_out, double* theta_out) {
  int N = p->N;
  long K = (long)N * N * N;
  double m[5], th[5];
  or_moments(N, p->L, f, m);
  double* M = (double*)malloc(sizeof(double) * K);
  double* q = (double*)malloc(sizeof(double) * K);
  if (or_discrete_maxwellian(N, p->L, NULL, m, th, 0, p->newton_tol, p->newton_max) < 0) {
    /* keep the last iterate; the caller's status reflects the failure through NaN checks */
  }
  or_eval_maxwellian(N, p->L, th, M);
  double nu = or_collision_frequency(p, f);
  if (p->kernel == OR_BGK) {
    for (long i = 0; i < K; i++) q[i] = nu * (M[i] - f[i]);
  } else {
    double* qm = (double*)malloc(sizeof(double) * K);
    or_qfsm(N, p->L, p->kernel, p->b0, f, q);
    or_qfsm(N, p->L, p->kernel, p->b0, M, qm);
    for (long i = 0; i < K; i++) q[i] -= qm[i];
    free(qm);
    if (p->conserve_proj == 1) or_conserve_project(N, p->L, q);
    if (p->conserve_proj == 2) or_conserve_project_w(N, p->L, M, q);
  }
  if (Q) memcpy(Q, q, sizeof(double) * K);
  if (P) {
    if (p->kernel == OR_BGK)
      for (long i = 0; i < K; i++) P[i] = 0.0;
    else
      for (long i = 0; i < K; i++) P[i] = q[i] - nu * (M[i] - f[i]);
  }
  if (nu_out) *nu_out = nu;
  if (theta_out) memcpy(theta_out, th, sizeof(th));
  free(M);
  free(q);
}

void or_collide(const or_problem* p, int J, const double* f, double* Q, double* P, double* nu) {
  long K = (long)p->N * p->N * p->N;
  if (p->kernel != OR_BGK) (void)tables(p->N, p->L, p->kernel, p->b0); /* build before threads start */
#pragma omp parallel for schedule(dynamic)
  for (int j = 0; j < J; j++)
    or_collide_cell(p, f + j * K, Q ? Q + j * K : NULL, P ? P + j * K : NULL, nu ? nu + j : NULL, NULL);
}

/* ------------------------------------------------------------------------------------
 * Local problem of one cell visit (eq. (20)):
 *   (|v1|/dx) g + r = (nu/eps) (M[g] - g),
 * solved by the preconditioned fixed-point iteration (eqs. (24)-(25)):
 *   step 1: M+ = exp(alpha + beta.v - gamma|v|^2) with
 *           sum w phi (|v1|/dx) M+ = s := sum w phi ((|v1|/dx)(M[g] - g) - r),
 *           attempted only when s0 > 0 and s0 s4 > s1^2 + s2^2 + s3^2 (eq. (26));
 *           otherwise, or when its Newton solve fails, M+ = M[g] (plain FP, eq. (22));
 *   step 2: g = ((nu/eps) M+ - r) / (|v1|/dx + nu/eps).
 * Stops when the discrete L2 norm sqrt(sum w (.)^2) of the cell-equation residual falls
 * below inner_tol (Section 4), after inner_max updates, or after exactly inner_fixed
 * updates when inner_fixed > 0.
 * ---------------------------------------------------------------------------------- */
int or_cell_solve(const or_problem* p, double dx, const double* r, double nu, double* g, or_stats* st) {
  int N = p->N;
  long K = (long)N * N * N;
  double* v = (double*)malloc(sizeof(double) * N);
  double* c = (double*)malloc(sizeof(double) * K);
  or_velocity_nodes(N, p->L, v);
  for (int i1 = 0; i1 < N; i1++)
    for (long t = 0; t < (long)N * N; t++) c[(long)i1 * N * N + t] = fabs(v[i1]) / dx;
  int it = or_cell_solve_c(p, c, r, nu, g, st);
  free(v);
  free(c);
  return it;
}

/* The cell equation with a general transport weight c_k >= 0 per node (|v1|/dx in 1-D,
 * |v1|/dx + |v2|/dy in 2-D): c g + r = (nu/eps)(M[g] - g). Step 1 of PFP (eq. (24)) uses
 * the weights w c_k. */
int or_cell_solve_c(const or_problem* p, const double* c, const double* r, double nu, double* g, or_stats* st) {
  int N = p->N;
  long K = (long)N * N * N;
  double L = p->L, w = weight(N, L), eps = p->eps;
  double* v = (double*)malloc(sizeof(double) * N);
  double* wk = (double*)malloc(sizeof(double) * K);
  double* Mg = (double*)malloc(sizeof(double) * K);
  double* Mp = (double*)malloc(sizeof(double) * K);
  or_velocity_nodes(N, L, v);
  for (long i = 0; i < K; i++) wk[i] = w * c[i];
  double a = nu / eps;
  int it;
  for (it = 0;; it++) {
    double m[5], thg[5];
    or_moments(N, L, g, m);
    int ni = or_discrete_maxwellian(N, L, NULL, m, thg, 0, p->newton_tol, p->newton_max);
    if (st) {
      st->newton_solves++;
      if (ni > 0) st->newton_iters += ni;
      else st->newton_failures++;
    }
    or_eval_maxwellian(N, L, thg, Mg);
    if (p->inner_fixed > 0) {
      if (it == p->inner_fixed) break;
    } else {
      double res = 0.0;
      for (int i1 = 0; i1 < N; i1++)
        for (long t = 0; t < (long)N * N; t++) {
          long i = (long)i1 * N * N + t;
          double e = c[i] * g[i] + r[i] - a * (Mg[i] - g[i]);
          res += w * e * e;
        }
      if (sqrt(res) < p->inner_tol) break;
      if (it == p->inner_max) break;
    }
    const double* Mplus = Mg;
    if (p->inner_method == OR_PFP || p->inner_method == OR_PFP_RELAX) {
      /* s = sum w phi ((|v1|/dx)(M[g] - g) - r) */
      double s[5] = {0, 0, 0, 0, 0};
      for (int i1 = 0; i1 < N; i1++)
        for (int i2 = 0; i2 < N; i2++)
          for (int i3 = 0; i3 < N; i3++) {
            long i = ((long)i1 * N + i2) * N + i3;
            double e = w * (c[i] * (Mg[i] - g[i]) - r[i]);
            double vv = v[i1] * v[i1] + v[i2] * v[i2] + v[i3] * v[i3];
            s[0] += e;
            s[1] += e * v[i1];
            s[2] += e * v[i2];
            s[3] += e * v[i3];
            s[4] += e * vv;
          }
      int exists = s[0] > 0.0 && s[0] * s[4] > s[1] * s[1] + s[2] * s[2] + s[3] * s[3];
      if (!exists && p->inner_method == OR_PFP_RELAX) {
        /* Relaxed step 1 (the remark after eq. (26)): with a factor 1 + tau on the weighted
         * moments of the new and the current Maxwellian, the target becomes
         *   s_tau = (tau m_w + s) / (1 + tau),   m_w = sum w phi (|v1|/dx) M[g],
         * tau = 0 being step 1 and tau -> infinity the source iteration (M+ = M[g]).
         * 1 + tau = 2, 4, 8, ...: the first that passes eq. (26) is taken. */
        double mw[5] = {0, 0, 0, 0, 0};
        for (int i1 = 0; i1 < N; i1++)
          for (int i2 = 0; i2 < N; i2++)
            for (int i3 = 0; i3 < N; i3++) {
              long i = ((long)i1 * N + i2) * N + i3;
              double e = w * c[i] * Mg[i];
              double vv = v[i1] * v[i1] + v[i2] * v[i2] + v[i3] * v[i3];
              mw[0] += e;
              mw[1] += e * v[i1];
              mw[2] += e * v[i2];
              mw[3] += e * v[i3];
              mw[4] += e * vv;
            }
        for (double q = 2.0; q <= 1048576.0 && !exists; q *= 2.0) {
          double t[5];
          for (int k = 0; k < 5; k++) t[k] = ((q - 1.0) * mw[k] + s[k]) / q;
          if (t[0] > 0.0 && t[0] * t[4] > t[1] * t[1] + t[2] * t[2] + t[3] * t[3]) {
            exists = 1;
            for (int k = 0; k < 5; k++) s[k] = t[k];
          }
        }
      }
      if (exists) {
        double thp[5];
        memcpy(thp, thg, sizeof(thp));
        int np = or_discrete_maxwellian(N, L, wk, s, thp, 1, p->newton_tol, p->newton_max);
        if (st) {
          st->newton_solves++;
          if (np > 0) st->newton_iters += np;
        }
        if (np > 0) {
          or_eval_maxwellian(N, L, thp, Mp);
          Mplus = Mp;
        } else if (st) {
          st->newton_failures++;
          st->existence_fallbacks++;
        }
      } else if (st) {
        st->existence_fallbacks++;
      }
    }
    for (int i1 = 0; i1 < N; i1++)
      for (long t = 0; t < (long)N * N; t++) {
        long i = (long)i1 * N * N + t;
        g[i] = (a * Mplus[i] - r[i]) / (c[i] + a);
      }
  }
  if (st) {
    st->inner_iters += it;
    st->visits++;
  }
  free(v);
  free(wk);
  free(Mg);
  free(Mp);
  return it;
}

/* ------------------------------------------------------------------------------------
 * Diffuse wall (eq. (31)): incoming half [v - U^w].n < 0 carries
 * rho^w exp(-|v - U^w|^2 / (2 T^w)) / (2 pi T^w)^{3/2}; rho^w from the zero normal mass
 * flux condition written with the discrete quadrature, the outgoing half taken from the
 * adjacent cell's stored value. Side 0 is x_lo (outer normal -e1, incoming v1 > 0),
 * side 1 is x_hi (incoming v1 < 0). Inflow: the incoming half is the given Maxwellian.
 * ---------------------------------------------------------------------------------- */
static void unit_wall_maxwellian(int N, double L, const double* u, double T, double* Mw) {
  double* v = (double*)malloc(sizeof(double) * N);
  or_velocity_nodes(N, L, v);
  double c = 1.0 / pow(2.0 * M_PI * T, 1.5);
  for (int i1 = 0; i1 < N; i1++)
    for (int i2 = 0; i2 < N; i2++)
      for (int i3 = 0; i3 < N; i3++) {
        double d1 = v[i1] - u[0], d2 = v[i2] - u[1], d3 = v[i3] - u[2];
        Mw[((long)i1 * N + i2) * N + i3] = c * exp(-(d1 * d1 + d2 * d2 + d3 * d3) / (2.0 * T));
      }
  free(v);
}

double or_wall_density(const or_problem* p, int side, const double* f_adj) {
  int N = p->N;
  long K = (long)N * N * N;
  double* v = (double*)malloc(sizeof(double) * N);
  double* Mw = (double*)malloc(sizeof(double) * K);
  or_velocity_nodes(N, p->L, v);
  unit_wall_maxwellian(N, p->L, p->bc_u[side], p->bc_T[side], Mw);
  double out = 0.0, in = 0.0;
  double w = weight(N, p->L);
  for (int i1 = 0; i1 < N; i1++) {
    int outgoing = side == 0 ? v[i1] < 0.0 : v[i1] > 0.0;
    int incoming = side == 0 ? v[i1] > 0.0 : v[i1] < 0.0;
    for (long t = 0; t < (long)N * N; t++) {
      long i = (long)i1 * N * N + t;
      if (outgoing) out += w * v[i1] * f_adj[i];
      if (incoming) in += w * v[i1] * Mw[i];
    }
  }
  free(v);
  free(Mw);
  return -out / in;
}

void or_ghost(const or_problem* p, int side, const double* f_adj, double* ghost) {
  int N = p->N;
  long K = (long)N * N * N;
  double* v = (double*)malloc(sizeof(double) * N);
  or_velocity_nodes(N, p->L, v);
  double scale;
  if (p->bc_kind[side] == OR_INFLOW) {
    scale = p->bc_rho[side];
  } else {
    scale = or_wall_density(p, side, f_adj);
  }
  unit_wall_maxwellian(N, p->L, p->bc_u[side], p->bc_T[side], ghost);
  for (int i1 = 0; i1 < N; i1++) {
    int incoming = side == 0 ? v[i1] > 0.0 : v[i1] < 0.0;
    for (long t = 0; t < (long)N * N; t++) {
      long i = (long)i1 * N * N + t;
      ghost[i] = incoming ? scale * ghost[i] : 0.0;
    }
  }
  (void)K;
  free(v);
}

/* ------------------------------------------------------------------------------------
 * One scan of the symmetric Gauss-Seidel method for the quadratic collision operator
 * (eq. (29), first order: s_j = 0). Visiting cell j solves eq. (20) with
 *   r = (1/dx) (-v1^+ f_{j-1} + v1^- f_{j+1}) - P_j/eps - b_j,
 * where f_{j-1}, f_{j+1} hold the latest values (already updated on the upwind side of
 * the scan), and P_j, nu_j come from the collision evaluation that preceded the scan.
 * Wall ghosts use the adjacent cell's value stored before the visit.
 * ---------------------------------------------------------------------------------- */
/* ------------------------------------------------------------------------------------
 * Slopes of the linear reconstruction (eq. (reconstruction), eq. (slope)):
 *   s_0 = f_1 - f_0,  s_j = (f_{j+1} - f_{j-1})/2 inside,  s_{J-1} = f_{J-1} - f_{J-2};
 * face values f^-_{j+1/2} = f_j + s_j/2 and f^+_{j-1/2} = f_j - s_j/2. First order: s = 0.
 * ---------------------------------------------------------------------------------- */
void or_slopes(const or_problem* p, int J, const double* f, double* s) {
  long K = (long)p->N * p->N * p->N;
  if (p->order != 2 || J < 2) {
    memset(s, 0, sizeof(double) * J * K);
    return;
  }
  for (int j = 0; j < J; j++)
    for (long i = 0; i < K; i++) {
      double d;
      if (j == 0)
        d = f[K + i] - f[i];
      else if (j == J - 1)
        d = f[(long)j * K + i] - f[(long)(j - 1) * K + i];
      else
        d = 0.5 * (f[(long)(j + 1) * K + i] - f[(long)(j - 1) * K + i]);
      s[(long)j * K + i] = d;
    }
}

void or_sweep(const or_problem* p, int J, double dx, int dir, double* f, const double* P, const double* nu,
              const double* b, or_stats* st) {
  /* Second order: the slopes are explicit, taken from the state before this scan (eq.
   * (SGS_BGK): s^(n) in the forward and s^(n+1/2) in the backward scan), and enter r as
   *   -(v1^+ s_{j-1} - v1 s_j + v1^- s_{j+1}) / (2 dx),   with zero ghost slopes.
   * The wall ghosts take their density from the outgoing face value (f_0 - s_0/2 on the
   * left, f_{J-1} + s_{J-1}/2 on the right) of the stored state, like the first-order
   * ghosts from the stored cell value. */
  int N = p->N;
  long K = (long)N * N * N;
  double* v = (double*)malloc(sizeof(double) * N);
  double* r = (double*)malloc(sizeof(double) * K);
  double* gl = (double*)malloc(sizeof(double) * K);
  double* gr = (double*)malloc(sizeof(double) * K);
  double* face = (double*)malloc(sizeof(double) * K);
  double* sl = (double*)malloc(sizeof(double) * J * K);
  or_velocity_nodes(N, p->L, v);
  or_slopes(p, J, f, sl);
  for (int s = 0; s < J; s++) {
    int j = dir > 0 ? s : J - 1 - s;
    const double* left;
    const double* right;
    if (j == 0) {
      for (long i = 0; i < K; i++) face[i] = f[i] - 0.5 * sl[i];
      or_ghost(p, 0, face, gl);
      left = gl;
    } else {
      left = f + (long)(j - 1) * K;
    }
    if (j == J - 1) {
      for (long i = 0; i < K; i++) face[i] = f[(long)(J - 1) * K + i] + 0.5 * sl[(long)(J - 1) * K + i];
      or_ghost(p, 1, face, gr);
      right = gr;
    } else {
      right = f + (long)(j + 1) * K;
    }
    for (int i1 = 0; i1 < N; i1++) {
      double vp = v[i1] > 0.0 ? v[i1] : 0.0, vm = v[i1] < 0.0 ? v[i1] : 0.0;
      for (long t = 0; t < (long)N * N; t++) {
        long i = (long)i1 * N * N + t;
        r[i] = (-vp * left[i] + vm * right[i]) / dx - P[(long)j * K + i] / p->eps - (b ? b[(long)j * K + i] : 0.0);
        if (p->order == 2) {
          double sm = j > 0 ? sl[(long)(j - 1) * K + i] : 0.0;
          double sp = j < J - 1 ? sl[(long)(j + 1) * K + i] : 0.0;
          r[i] -= (vp * sm - v[i1] * sl[(long)j * K + i] + vm * sp) / (2.0 * dx);
        }
      }
    }
    or_cell_solve(p, dx, r, nu[j], f + (long)j * K, st);
  }
  free(v);
  free(r);
  free(gl);
  free(gr);
  free(face);
  free(sl);
}

/* Uniform scaling after each iteration to keep the total mass C (eq. (32)). */
void or_rescale(const or_problem* p, int J, double dx, double* f) {
  int N = p->N;
  long K = (long)N * N * N;
  double w = weight(N, p->L), tot = 0.0;
  for (int j = 0; j < J; j++) {
    double rho = 0.0;
    for (long i = 0; i < K; i++) rho += w * f[(long)j * K + i];
    tot += dx * rho;
  }
  double lam = p->total_mass / tot;
  for (long i = 0; i < (long)J * K; i++) f[i] *= lam;
}

/* Outer residual (Section 4 stopping rule) of the fully discrete equation (eq. (11)):
 * R = (v1^+ (f_j - f_{j-1}) + v1^- (f_{j+1} - f_j))/dx - Q_j/eps - b_j, ghosts from the
 * same f, norm sqrt(dx sum_j sum_k w R^2). */
double or_residual(const or_problem* p, int J, double dx, const double* f, const double* Q, const double* b,
                   double* Rout) {
  /* R_j = (v1^+ (f^-_{j+1/2} - f^-_{j-1/2}) + v1^- (f^+_{j+1/2} - f^+_{j-1/2}))/dx - Q_j/eps - b_j
   * (eq. (upwind)) with the face values of the reconstruction (first order: the cell
   * values) and wall ghosts from the same f. */
  int N = p->N;
  long K = (long)N * N * N;
  double w = weight(N, p->L);
  double* v = (double*)malloc(sizeof(double) * N);
  double* gl = (double*)malloc(sizeof(double) * K);
  double* gr = (double*)malloc(sizeof(double) * K);
  double* face = (double*)malloc(sizeof(double) * K);
  double* sl = (double*)malloc(sizeof(double) * J * K);
  or_velocity_nodes(N, p->L, v);
  or_slopes(p, J, f, sl);
  for (long i = 0; i < K; i++) face[i] = f[i] - 0.5 * sl[i];
  or_ghost(p, 0, face, gl);
  for (long i = 0; i < K; i++) face[i] = f[(long)(J - 1) * K + i] + 0.5 * sl[(long)(J - 1) * K + i];
  or_ghost(p, 1, face, gr);
  double acc = 0.0;
  for (int j = 0; j < J; j++) {
    const double* fj = f + (long)j * K;
    const double* sj = sl + (long)j * K;
    for (int i1 = 0; i1 < N; i1++) {
      double vp = v[i1] > 0.0 ? v[i1] : 0.0, vm = v[i1] < 0.0 ? v[i1] : 0.0;
      for (long t = 0; t < (long)N * N; t++) {
        long i = (long)i1 * N * N + t;
        double mr = fj[i] + 0.5 * sj[i];  /* f^-_{j+1/2} */
        double pl = fj[i] - 0.5 * sj[i];  /* f^+_{j-1/2} */
        double ml = j == 0 ? gl[i] : f[(long)(j - 1) * K + i] + 0.5 * sl[(long)(j - 1) * K + i];
        double pr = j == J - 1 ? gr[i] : f[(long)(j + 1) * K + i] - 0.5 * sl[(long)(j + 1) * K + i];
        double R = (vp * (mr - ml) + vm * (pr - pl)) / dx - Q[(long)j * K + i] / p->eps -
                   (b ? b[(long)j * K + i] : 0.0);
        if (Rout) Rout[(long)j * K + i] = R;
        acc += w * R * R;
      }
    }
  }
  free(v);
  free(gl);
  free(gr);
  free(face);
  free(sl);
  return sqrt(dx * acc);
}

void or_sgs_iteration(const or_problem* p, int J, double dx, double* f, const double* b, int rescale, or_stats* st) {
  long K = (long)p->N * p->N * p->N;
  double* P = (double*)malloc(sizeof(double) * J * K);
  double* nu = (double*)malloc(sizeof(double) * J);
  or_collide(p, J, f, NULL, P, nu);
  or_sweep(p, J, dx, +1, f, P, nu, b, st);
  or_collide(p, J, f, NULL, P, nu);
  or_sweep(p, J, dx, -1, f, P, nu, b, st);
  if (rescale && p->total_mass > 0.0) or_rescale(p, J, dx, f);
  free(P);
  free(nu);
}

/* ------------------------------------------------------------------------------------
 * Nonlinear multigrid V-cycle (eq. (30)) with H = 2h:
 *   smooth (pre) -> restrict fbar and the residual (mean of the two children) ->
 *   b_H = R_H(I fbar_h) + I(b_h - R_h(fbar_h)) -> solve on H (recursively, the
 *   coarsest level by coarse_iters SGS iterations) -> fhat_h = fbar_h + P(f_H - I fbar_h)
 *   with piecewise-constant prolongation -> smooth (post).
 * R_h(f) = T_h(f) - Q(f)/eps includes the nonlinear wall ghosts. The mass rescale acts
 * on the finest level only.
 * ---------------------------------------------------------------------------------- */
/* ------------------------------------------------------------------------------------
 * Source iteration (eq. (SI)) for the binary collision operator: with the penalty split
 * Q = P + nu (M - f) (eq. (28)), P[f^n], nu^n and M[f^n] are frozen and f^{n+1} solves, node
 * by node,
 *   v1^+ (f_j - f_{j-1})/dx + v1^- (f_{j+1} - f_j)/dx = P_j/eps + (nu_j/eps)(M_j - f_j) + b_j,
 * i.e. (|v1|/dx + nu_j/eps) f_j = (|v1|/dx) f_upwind + P_j/eps + (nu_j/eps) M_j + b_j,
 * marched from the node's inflow side; the wall ghosts are built from f^n (lagged like the
 * scans' ghosts). BGK mode: P = 0 and this is eq. (SI) itself.
 * ---------------------------------------------------------------------------------- */
void or_si_iteration(const or_problem* p, int J, double dx, double* f, const double* b, int rescale) {
  int N = p->N;
  long K = (long)N * N * N;
  double* v = (double*)malloc(sizeof(double) * N);
  double* P = (double*)malloc(sizeof(double) * J * K);
  double* M = (double*)malloc(sizeof(double) * J * K);
  double* nu = (double*)malloc(sizeof(double) * J);
  double* gl = (double*)malloc(sizeof(double) * K);
  double* gr = (double*)malloc(sizeof(double) * K);
  or_velocity_nodes(N, p->L, v);
  for (int j = 0; j < J; j++) {
    double th[5];
    or_collide_cell(p, f + (long)j * K, NULL, P + (long)j * K, nu + j, th);
    or_eval_maxwellian(N, p->L, th, M + (long)j * K);
  }
  or_ghost(p, 0, f, gl);
  or_ghost(p, 1, f + (long)(J - 1) * K, gr);
  for (int i1 = 0; i1 < N; i1++) {
    double c = fabs(v[i1]) / dx;
    for (long t = 0; t < (long)N * N; t++) {
      long i = (long)i1 * N * N + t;
      double up = v[i1] > 0.0 ? gl[i] : gr[i];
      for (int s = 0; s < J; s++) {
        int j = v[i1] < 0.0 ? J - 1 - s : s;
        long o = (long)j * K + i;
        double a = nu[j] / p->eps;
        double src = P[o] / p->eps + a * M[o] + (b ? b[o] : 0.0);
        f[o] = (c * up + src) / (c + a);
        up = f[o];
      }
    }
  }
  if (rescale && p->total_mass > 0.0) or_rescale(p, J, dx, f);
  free(v);
  free(P);
  free(M);
  free(nu);
  free(gl);
  free(gr);
}

static void vcycle_rec(const or_problem* p, int level, int levels, int J, double dx, double* f, const double* b,
                       int pre, int post, int coarse_iters, or_stats* st) {
  long K = (long)p->N * p->N * p->N;
  int finest = level == 0;
  if (level == levels - 1) {
    for (int it = 0; it < coarse_iters; it++) or_sgs_iteration(p, J, dx, f, b, finest, st);
    return;
  }
  for (int it = 0; it < pre; it++) or_sgs_iteration(p, J, dx, f, b, finest, st);
  int JH = J / 2;
  double dxH = 2.0 * dx;
  double* Q = (double*)malloc(sizeof(double) * J * K);
  double* R = (double*)malloc(sizeof(double) * J * K);
  or_collide(p, J, f, Q, NULL, NULL);
  or_residual(p, J, dx, f, Q, b, R); /* R = R_h(fbar) - b_h */
  double* fH0 = (double*)malloc(sizeof(double) * JH * K);
  double* fH = (double*)malloc(sizeof(double) * JH * K);
  double* bH = (double*)malloc(sizeof(double) * JH * K);
  double* QH = (double*)malloc(sizeof(double) * JH * K);
  for (int i = 0; i < JH; i++)
    for (long k = 0; k < K; k++) {
      fH0[(long)i * K + k] = 0.5 * (f[(long)(2 * i) * K + k] + f[(long)(2 * i + 1) * K + k]);
      bH[(long)i * K + k] = -0.5 * (R[(long)(2 * i) * K + k] + R[(long)(2 * i + 1) * K + k]);
    }
  or_collide(p, JH, fH0, QH, NULL, NULL);
  double* RH = (double*)malloc(sizeof(double) * JH * K);
  or_residual(p, JH, dxH, fH0, QH, NULL, RH); /* R_H(I fbar) */
  for (long i = 0; i < (long)JH * K; i++) bH[i] += RH[i];
  memcpy(fH, fH0, sizeof(double) * JH * K);
  vcycle_rec(p, level + 1, levels, JH, dxH, fH, bH, pre, post, coarse_iters, st);
  for (int i = 0; i < JH; i++)
    for (long k = 0; k < K; k++) {
      double c = fH[(long)i * K + k] - fH0[(long)i * K + k];
      f[(long)(2 * i) * K + k] += c;
      f[(long)(2 * i + 1) * K + k] += c;
    }
  for (int it = 0; it < post; it++) or_sgs_iteration(p, J, dx, f, b, finest, st);
  free(Q);
  free(R);
  free(fH0);
  free(fH);
  free(bH);
  free(QH);
  free(RH);
}

void or_vcycle(const or_problem* p, double* f, int levels, int pre, int post, int coarse_iters, or_stats* st) {
  double dx = (p->x_hi - p->x_lo) / p->J;
  vcycle_rec(p, 0, levels, p->J, dx, f, NULL, pre, post, coarse_iters, st);
}
