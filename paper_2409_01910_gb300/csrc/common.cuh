// Shared device-side definitions of the SGS-PFP CUDA library (sm_103a).
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sgs.h"

namespace sgs {

namespace cg = cooperative_groups;

constexpr int kMaxN = 32;          // velocity points per dimension supported
constexpr int kLanes = 32;         // cells per spectral group (one warp lane per cell)
constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------------------
// Per-instance description in device memory.
// ---------------------------------------------------------------------------------------
struct InstDev {
  long long f_off;       // element offset of cell 0 in every field
  int J;                 // cells
  int cell0;             // global index of cell 0 (collision-step cell list)
  int collision;         // sgs_collision
  int bc_kind[2];
  double dx, eps;
  double b0;
  double bc_rho[2];      // inflow density (unused for diffuse walls)
  double wall_denom[2];  // sum over incoming v of w v1 Mhat_wall (diffuse walls)
  double total_mass;
  double inner_tol;
  int inner_max, inner_fixed, inner_method, newton_max;
  double newton_tol;
  // Unit wall Maxwellian, separable: Mhat(v) = W[s][0][i1] W[s][1][i2] W[s][2][i3], with the
  // incoming half of v1 kept and the outgoing half zeroed in W[s][0].
  double wall[2][3][kMaxN];
};

struct Counters {
  unsigned int status;
  unsigned int pad;
  unsigned long long visits, inner_iters, newton_iters, newton_solves, fallbacks;
};

// ---------------------------------------------------------------------------------------
// Velocity grid helpers: v_i = (i - N/2 + 1) dv.
// ---------------------------------------------------------------------------------------
__host__ __device__ inline double node(int i, int N, double dv) { return (double)(i - N / 2 + 1) * dv; }

// ---------------------------------------------------------------------------------------
// Warp reductions (butterfly: every lane receives the total, in a fixed order).
// ---------------------------------------------------------------------------------------
template <int NV>
__device__ inline void warp_allsum(double (&x)[NV]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < NV; q++) x[q] += __shfl_xor_sync(0xffffffffu, x[q], o);
  }
}

// ---------------------------------------------------------------------------------------
// Discrete Maxwellian on the tensor grid (eqs. (13)-(14)).
//
// M_k = exp(alpha + beta.v_k - gamma |v_k|^2) factorises as
//   exp(alpha) * E_1(v_1) E_2(v_2) E_3(v_3),   E_d(v) = exp(beta_d v - gamma v^2),
// and so do the weights used here (w, or w |v1|/dx for step 1 of PFP, eq. (24)). Every
// weighted moment sum_k wk phi_i phi_j M_k with phi = (1, v1, v2, v3, |v|^2) is therefore a
// product of one-dimensional sums S_d^p = sum_i omega_d(v_i) E_d(v_i) v_i^p, p = 0..4, and a
// Newton iteration costs O(N) instead of O(N^3). The iteration itself (undamped Newton
// with step halving while the scaled residual grows; stop one step after the exponent
// change |da| + L sum|db| + L^2 |dg| falls below tol) follows the discrete conservation
// equations directly.
//
// Called by one full warp; lane i < N handles node i. All lanes return the same result.
// ---------------------------------------------------------------------------------------
struct NewtonOut {
  double th[5];
  int iters;   // > 0 on success, -1 on failure
};

struct MaxwEval {
  double F[5];
  double A[15];  // upper triangle of sum wk M phi phi^T, row-major (i <= j)
  double fn;     // max |F_i| / |target_0|
  double e[3];   // this lane's E_1 (with exp(alpha)), E_2, E_3
};

__device__ inline void maxw_eval(int N, double dv, double w, bool wv1, double inv_dx, const double* target,
                                 const double* th, MaxwEval& out) {
  int lane = threadIdx.x & 31;
  double s[15];
  double vi = node(lane < N ? lane : 0, N, dv);
  double v2 = vi * vi;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    double e = lane < N ? exp(th[1 + d] * vi - th[4] * v2) : 0.0;
    out.e[d] = e;
    double om = (d == 0 && wv1) ? fabs(vi) * inv_dx : 1.0;
    double x = om * e;
    s[5 * d + 0] = x;
    s[5 * d + 1] = x * vi;
    s[5 * d + 2] = x * v2;
    s[5 * d + 3] = x * v2 * vi;
    s[5 * d + 4] = x * v2 * v2;
  }
  warp_allsum<15>(s);
  double ea = exp(th[0]);
  out.e[0] *= ea;
  const double* S1 = s;
  const double* S2 = s + 5;
  const double* S3 = s + 10;
  double c = w * ea;
  // sums of phi_i phi_j M over the grid, from the 1-D sums
  double m00 = S1[0] * S2[0] * S3[0];
  double m1 = S1[1] * S2[0] * S3[0], m2 = S1[0] * S2[1] * S3[0], m3 = S1[0] * S2[0] * S3[1];
  double q11 = S1[2] * S2[0] * S3[0], q22 = S1[0] * S2[2] * S3[0], q33 = S1[0] * S2[0] * S3[2];
  double q12 = S1[1] * S2[1] * S3[0], q13 = S1[1] * S2[0] * S3[1], q23 = S1[0] * S2[1] * S3[1];
  double e2 = q11 + q22 + q33;  // sum |v|^2 M
  // sum v_d |v|^2 M
  double c1 = S1[3] * S2[0] * S3[0] + S1[1] * S2[2] * S3[0] + S1[1] * S2[0] * S3[2];
  double c2 = S1[2] * S2[1] * S3[0] + S1[0] * S2[3] * S3[0] + S1[0] * S2[1] * S3[2];
  double c3 = S1[2] * S2[0] * S3[1] + S1[0] * S2[2] * S3[1] + S1[0] * S2[0] * S3[3];
  // sum |v|^4 M
  double e4 = S1[4] * S2[0] * S3[0] + S1[0] * S2[4] * S3[0] + S1[0] * S2[0] * S3[4] +
              2.0 * (S1[2] * S2[2] * S3[0] + S1[2] * S2[0] * S3[2] + S1[0] * S2[2] * S3[2]);
  double mom[5] = {m00, m1, m2, m3, e2};
  double amax = 0.0;
#pragma unroll
  for (int i = 0; i < 5; i++) {
    out.F[i] = c * mom[i] - target[i];
    amax = fmax(amax, fabs(out.F[i]));
  }
  out.fn = amax / fabs(target[0]);
  double A[15] = {m00, m1, m2, m3, e2, q11, q12, q13, c1, q22, q23, c2, q33, c3, e4};
#pragma unroll
  for (int i = 0; i < 15; i++) out.A[i] = c * A[i];
}

// Solves A y = b for the symmetric positive definite 5x5 matrix given by its upper
// triangle (row-major). Returns false if A is not numerically positive definite.
__device__ inline bool chol5_solve(const double* Au, const double* b, double* y) {
  double a[5][5];
  int t = 0;
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = i; j < 5; j++) {
      a[i][j] = Au[t];
      a[j][i] = Au[t];
      t++;
    }
  double l[5][5];
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j < 5; j++) l[i][j] = 0.0;
#pragma unroll
  for (int j = 0; j < 5; j++) {
    double d = a[j][j];
#pragma unroll
    for (int k = 0; k < j; k++) d -= l[j][k] * l[j][k];
    if (!(d > 0.0)) return false;
    double ljj = sqrt(d);
    l[j][j] = ljj;
    double inv = 1.0 / ljj;
#pragma unroll
    for (int i = j + 1; i < 5; i++) {
      double s = a[i][j];
#pragma unroll
      for (int k = 0; k < j; k++) s -= l[i][k] * l[j][k];
      l[i][j] = s * inv;
    }
  }
  double z[5];
#pragma unroll
  for (int i = 0; i < 5; i++) {
    double s = b[i];
#pragma unroll
    for (int k = 0; k < i; k++) s -= l[i][k] * z[k];
    z[i] = s / l[i][i];
  }
#pragma unroll
  for (int i = 4; i >= 0; i--) {
    double s = z[i];
#pragma unroll
    for (int k = i + 1; k < 5; k++) s -= l[k][i] * y[k];
    y[i] = s / l[i][i];
  }
  return true;
}

// Continuum Maxwellian with the given moments (rho, rho U, sum |v|^2 f): initial guess.
__device__ inline bool continuum_guess(const double* m, double* th) {
  double rho = m[0];
  if (!(rho > 0.0)) return false;
  double U0 = m[1] / rho, U1 = m[2] / rho, U2 = m[3] / rho;
  double uu = U0 * U0 + U1 * U1 + U2 * U2;
  double T = (m[4] / rho - uu) / 3.0;
  if (!(T > 0.0)) return false;
  th[4] = 0.5 / T;
  th[1] = U0 / T;
  th[2] = U1 / T;
  th[3] = U2 / T;
  th[0] = log(rho / (2.0 * kPi * T * sqrt(2.0 * kPi * T))) - 0.5 * uu / T;
  return true;
}

// Newton for the weighted discrete Maxwellian. th holds the initial guess on entry.
// On return ev holds the evaluation at the returned theta (lane-local E factors included).
__device__ inline int maxwellian_newton(int N, double dv, double w, bool wv1, double inv_dx, const double* target,
                                        double* th, double tol, int maxit, MaxwEval& ev) {
  double L = node(N - 1, N, dv);
  maxw_eval(N, dv, w, wv1, inv_dx, target, th, ev);
  bool done = false;
  int it;
  for (it = 0; it < maxit; it++) {
    double y[5];
    if (!chol5_solve(ev.A, ev.F, y)) return -1;
    double d[5] = {-y[0], -y[1], -y[2], -y[3], y[4]};  // delta = -D A^{-1} F, D = diag(1,1,1,1,-1)
    double lam = 1.0;
    double fn = ev.fn;
    double tt[5];
    int hv;
    for (hv = 0; hv < 40; hv++) {
#pragma unroll
      for (int i = 0; i < 5; i++) tt[i] = th[i] + lam * d[i];
      maxw_eval(N, dv, w, wv1, inv_dx, target, tt, ev);
      if (ev.fn == ev.fn && (ev.fn <= fn || ev.fn <= 1e-10)) break;
      lam *= 0.5;
    }
#pragma unroll
    for (int i = 0; i < 5; i++) th[i] = tt[i];
    double step = lam * (fabs(d[0]) + L * (fabs(d[1]) + fabs(d[2]) + fabs(d[3])) + L * L * fabs(d[4]));
    if (!(step == step)) return -1;
    if (done) return it + 1;
    if (step <= tol) done = true;
  }
  return -1;
}

// ---------------------------------------------------------------------------------------
// PTX wrappers: mbarrier and bulk (TMA, non-tensor) global -> shared copies.
// ---------------------------------------------------------------------------------------
__device__ inline uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ inline void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ inline void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Bounded wait on the phase with the given parity; returns false after max_spins polls.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity, long long max_spins) {
  uint32_t addr = smem_addr(bar);
  for (long long i = 0; i < max_spins; i++) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// 1-D bulk copy global -> shared, completion signalled on bar (bytes % 16 == 0, both
// addresses 16-byte aligned).
__device__ inline void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace sgs
