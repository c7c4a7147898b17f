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
  int J;                 // cells (nx ny in 2-D)
  int nx, ny;            // grid (ny = 1 in 1-D)
  int space_dim;
  int cell0;             // global index of cell 0 (collision-step cell list)
  int collision;         // sgs_collision
  int bc_kind[4];        // x_lo, x_hi, y_lo, y_hi
  double dx, dy, eps;    // dy = 1 in 1-D (cell measure dx dy)
  double b0;
  double bc_rho[4];      // inflow density (unused for diffuse walls)
  double wall_denom[4];  // sum over incoming v of w (v.n) Mhat_wall (diffuse walls)
  double total_mass;
  double inner_tol;
  int inner_max, inner_fixed, inner_method, newton_max;
  double newton_tol;
  // Unit wall Maxwellian of side s, separable: Mhat(v) = W[s][0][i1] W[s][1][i2] W[s][2][i3],
  // with the incoming half of the normal component kept and the outgoing half zeroed (in
  // W[s][0] for the x sides, W[s][1] for the y sides).
  double wall[4][3][kMaxN];
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
// Double-float ("df64") arithmetic: a value is hi + lo with two FP32 numbers, |lo| <= ulp(hi)/2,
// carried through error-free transformations (Knuth's two-sum, Dekker's fast two-sum, and the
// FMA form of the exact product). Addition and multiplication keep about 48 significant bits
// relative to the operands, enough for the cancellations of the cell equation, and run on the
// FP32 pipes, which on this GPU have ~40x the FP64 throughput.
// ---------------------------------------------------------------------------------------
struct dfloat {
  float hi, lo;
};

__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  float s = a.hi + b.hi;
  float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  return df_fast_two_sum(s, e);
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }

// Exact split of a double into a double-float by bit manipulation (no FP64 instruction):
// hi keeps the leading 24 significand bits (truncated), lo the next bits rounded to 24.
// Magnitudes below 2^-100 (irrelevant next to the O(1) values they are summed with) map to 0.
__device__ __forceinline__ dfloat df_split(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  unsigned int sign = (unsigned int)(u >> 63) << 31;
  int e = (int)((u >> 52) & 0x7ff) - 1023;
  if (e < -100) return {0.0f, 0.0f};
  unsigned long long m = (u & 0xfffffffffffffULL) | 0x10000000000000ULL;  // 53-bit significand
  unsigned int mh = (unsigned int)(m >> 29);                               // top 24 bits
  float hi = __int_as_float((int)(sign | ((unsigned int)(e + 127) << 23) | (mh & 0x7fffff)));
  unsigned int ml = (unsigned int)(m & 0x1fffffffULL);                     // low 29 bits
  float lo = ldexpf((float)ml, e - 52);
  return {hi, sign ? -lo : lo};
}

// exp in double-float arithmetic (no FP64 instruction): Cody and Waite's additive argument
// reduction x = k ln2 + r with ln2 split into three floats (the first with trailing zero bits,
// so k * c1 is exact for |k| < 512), then exp(r), |r| <= ln2/2, from its Taylor series to
// degree 13 by Horner's rule, and exp(x) = 2^k exp(r).
__device__ inline dfloat df_exp(dfloat x) {
  const float c1 = 0.693145751953125f, c2 = 1.428606765330187e-06f, c3 = 5.497923148104107e-14f;
  const float inv_ln2 = 1.4426950408889634f;
  if (x.hi < -87.0f) return {0.0f, 0.0f};
  float kf = rintf(x.hi * inv_ln2);
  // x.hi - kf c1 is exact (kf c1 is exact and, by Sterbenz's lemma, so is the difference)
  dfloat r = dfloat{x.hi - kf * c1, 0.0f} + dfloat{x.lo, 0.0f};
  float p = kf * c2;
  dfloat kc2 = {p, fmaf(kf, c2, -p)};
  r = r - kc2;
  r = r - dfloat{kf * c3, 0.0f};
  const float ch[14] = {1.0f, 1.0f, 0.5f, 0.1666666716337204f, 0.0416666679084301f, 0.008333333767950535f,
                        0.0013888889225199819f, 0.00019841270113829523f, 2.4801587642286904e-05f,
                        2.7557318844628753e-06f, 2.755731998149713e-07f, 2.5052107943679403e-08f,
                        2.0876755879584152e-09f, 1.6059044372074283e-10f};
  const float cl[14] = {0.0f, 0.0f, 0.0f, -4.967053879312289e-09f, -1.2417634698280722e-09f,
                        -4.34617203337595e-10f, -3.3631094437103215e-11f, -2.725596874933456e-12f,
                        -3.40699609366682e-13f, 3.793571224297229e-14f, -7.575112209051195e-15f,
                        4.4176230446483665e-16f, 1.1082839147459852e-16f, -5.352526511562726e-18f};
  // Estrin's scheme: the same degree-13 polynomial with a dependency chain of four
  // multiply-add levels instead of thirteen
  dfloat c[14];
#pragma unroll
  for (int n = 0; n < 14; n++) c[n] = dfloat{ch[n], cl[n]};
  dfloat r2 = r * r;
  dfloat r4 = r2 * r2;
  dfloat r8 = r4 * r4;
  dfloat pr[7];
#pragma unroll
  for (int n = 0; n < 7; n++) pr[n] = c[2 * n] + c[2 * n + 1] * r;
  dfloat q0 = pr[0] + pr[1] * r2, q1 = pr[2] + pr[3] * r2, q2 = pr[4] + pr[5] * r2;
  dfloat s0 = q0 + q1 * r4, s1 = q2 + pr[6] * r4;
  dfloat acc = s0 + s1 * r8;
  int k = (int)kf;
  return {ldexpf(acc.hi, k), ldexpf(acc.lo, k)};
}

// Conversions used by code templated on the arithmetic type E.
template <typename E>
__device__ __forceinline__ E cvt(double x);
template <>
__device__ __forceinline__ double cvt<double>(double x) { return x; }
template <>
__device__ __forceinline__ float cvt<float>(double x) { return (float)x; }
template <>
__device__ __forceinline__ dfloat cvt<dfloat>(double x) {
  return df_split(x);
}
__device__ __forceinline__ double tod(double x) { return x; }
__device__ __forceinline__ double tod(float x) { return (double)x; }
__device__ __forceinline__ double tod(dfloat x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ float tof(double x) { return (float)x; }
__device__ __forceinline__ float tof(float x) { return x; }
__device__ __forceinline__ float tof(dfloat x) { return x.hi; }

// exp in the precision of E without leaving it
__device__ __forceinline__ double exp_in(double x) { return exp(x); }
__device__ __forceinline__ float exp_in(float x) { return expf(x); }
__device__ __forceinline__ dfloat exp_in(dfloat x) { return df_exp(x); }

// exp evaluated in FP64 for double and df64, in FP32 for float
template <typename E>
__device__ __forceinline__ E exp_e(double x) {
  return cvt<E>(exp(x));
}
template <>
__device__ __forceinline__ float exp_e<float>(double x) {
  return expf((float)x);
}

__device__ __forceinline__ double shfl_x(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shfl_x(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ dfloat shfl_x(dfloat v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// ---------------------------------------------------------------------------------------
// Warp reductions (butterfly: every lane receives the total, in a fixed order).
// ---------------------------------------------------------------------------------------
template <int NV, typename T>
__device__ inline void warp_allsum(T (&x)[NV]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < NV; q++) x[q] += shfl_x(x[q], o);
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
template <typename E>
struct MaxwEval {
  E F[5];        // weighted moments of M minus the target
  float A[15];   // upper triangle of sum wk M phi phi^T (row-major, i <= j): Newton direction only
  double fn;     // max |F_i| / |target_0|
  E e[3];        // this lane's E_1 (with exp(alpha)), E_2, E_3
};

template <typename E>
__device__ inline void maxw_eval(int N, double dv, double w, bool wv1, double inv_dx, const E* target,
                                 const double* th, MaxwEval<E>& out) {
  int lane = threadIdx.x & 31;
  E s[15];
  double vd = node(lane < N ? lane : 0, N, dv);
  E vi = cvt<E>(vd), v2 = cvt<E>(vd * vd);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    E e = lane < N ? exp_e<E>(th[1 + d] * vd - th[4] * vd * vd) : cvt<E>(0.0);
    out.e[d] = e;
    E x = (d == 0 && wv1) ? cvt<E>(fabs(vd) * inv_dx) * e : e;
    s[5 * d + 0] = x;
    s[5 * d + 1] = x * vi;
    s[5 * d + 2] = s[5 * d + 1] * vi;
    s[5 * d + 3] = s[5 * d + 2] * vi;
    s[5 * d + 4] = s[5 * d + 2] * v2;
  }
  warp_allsum<15, E>(s);
  E ea = exp_e<E>(th[0]);
  out.e[0] = out.e[0] * ea;
  const E* S1 = s;
  const E* S2 = s + 5;
  const E* S3 = s + 10;
  E c = cvt<E>(w) * ea;
  // sums of phi_i M over the grid, from the 1-D sums
  E s23 = S2[0] * S3[0];
  E m00 = S1[0] * s23;
  E m1 = S1[1] * s23, m2 = S1[0] * (S2[1] * S3[0]), m3 = S1[0] * (S2[0] * S3[1]);
  E e2 = S1[2] * s23 + S1[0] * (S2[2] * S3[0] + S2[0] * S3[2]);
  E mom[5] = {m00, m1, m2, m3, e2};
  double amax = 0.0;
#pragma unroll
  for (int i = 0; i < 5; i++) {
    out.F[i] = c * mom[i] - target[i];
    amax = fmax(amax, fabs(tod(out.F[i])));
  }
  out.fn = amax / fabs(tod(target[0]));
  // Jacobian entries in FP32: they only set the Newton direction
  float f1[5], f2[5], f3[5];
#pragma unroll
  for (int p = 0; p < 5; p++) {
    f1[p] = (float)tod(S1[p]);
    f2[p] = (float)tod(S2[p]);
    f3[p] = (float)tod(S3[p]);
  }
  float q11 = f1[2] * f2[0] * f3[0], q22 = f1[0] * f2[2] * f3[0], q33 = f1[0] * f2[0] * f3[2];
  float q12 = f1[1] * f2[1] * f3[0], q13 = f1[1] * f2[0] * f3[1], q23 = f1[0] * f2[1] * f3[1];
  float c1 = f1[3] * f2[0] * f3[0] + f1[1] * f2[2] * f3[0] + f1[1] * f2[0] * f3[2];
  float c2 = f1[2] * f2[1] * f3[0] + f1[0] * f2[3] * f3[0] + f1[0] * f2[1] * f3[2];
  float c3 = f1[2] * f2[0] * f3[1] + f1[0] * f2[2] * f3[1] + f1[0] * f2[0] * f3[3];
  float e4 = f1[4] * f2[0] * f3[0] + f1[0] * f2[4] * f3[0] + f1[0] * f2[0] * f3[4] +
             2.0f * (f1[2] * f2[2] * f3[0] + f1[2] * f2[0] * f3[2] + f1[0] * f2[2] * f3[2]);
  float cf = (float)tod(c);
  float A[15] = {f1[0] * f2[0] * f3[0], f1[1] * f2[0] * f3[0], f1[0] * f2[1] * f3[0], f1[0] * f2[0] * f3[1],
                 q11 + q22 + q33, q11, q12, q13, c1, q22, q23, c2, q33, c3, e4};
#pragma unroll
  for (int i = 0; i < 15; i++) out.A[i] = cf * A[i];
}

// Solves A y = b (FP32) for the symmetric positive definite 5x5 matrix given by its upper
// triangle (row-major). Returns false if A is not numerically positive definite. The
// solution only serves as a Newton direction; the residual F stays in the caller's precision.
__device__ inline bool chol5_solve(const float* Au, const float* b, float* y) {
  float a[5][5];
  int t = 0;
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = i; j < 5; j++) {
      a[i][j] = Au[t];
      a[j][i] = Au[t];
      t++;
    }
  // symmetric diagonal scaling keeps the FP32 factorisation well conditioned
  float sc[5];
#pragma unroll
  for (int i = 0; i < 5; i++) {
    if (!(a[i][i] > 0.0f)) return false;
    sc[i] = rsqrtf(a[i][i]);
  }
  float l[5][5], dinv[5];
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j < 5; j++) l[i][j] = 0.0f;
#pragma unroll
  for (int j = 0; j < 5; j++) {
    float d = a[j][j] * sc[j] * sc[j];
#pragma unroll
    for (int k = 0; k < j; k++) d -= l[j][k] * l[j][k];
    if (!(d > 0.0f)) return false;
    // approximate reciprocal square root: the result is only a Newton direction
    float inv = rsqrtf(d);
    l[j][j] = d * inv;
    dinv[j] = inv;
#pragma unroll
    for (int i = j + 1; i < 5; i++) {
      float s = a[i][j] * sc[i] * sc[j];
#pragma unroll
      for (int k = 0; k < j; k++) s -= l[i][k] * l[j][k];
      l[i][j] = s * inv;
    }
  }
  float z[5];
#pragma unroll
  for (int i = 0; i < 5; i++) {
    float s = b[i] * sc[i];
#pragma unroll
    for (int k = 0; k < i; k++) s -= l[i][k] * z[k];
    z[i] = s * dinv[i];
  }
#pragma unroll
  for (int i = 4; i >= 0; i--) {
    float s = z[i];
#pragma unroll
    for (int k = i + 1; k < 5; k++) s -= l[k][i] * y[k];
    y[i] = s * dinv[i];
  }
#pragma unroll
  for (int i = 0; i < 5; i++) y[i] *= sc[i];
  return true;
}

// Continuum Maxwellian with the given moments (rho, rho U, sum |v|^2 f): initial guess.
template <typename E>
__device__ inline bool continuum_guess(const E* m, double* th) {
  double rho = tod(m[0]);
  if (!(rho > 0.0)) return false;
  double U0 = tod(m[1]) / rho, U1 = tod(m[2]) / rho, U2 = tod(m[3]) / rho;
  double uu = U0 * U0 + U1 * U1 + U2 * U2;
  double T = (tod(m[4]) / rho - uu) / 3.0;
  if (!(T > 0.0)) return false;
  th[4] = 0.5 / T;
  th[1] = U0 / T;
  th[2] = U1 / T;
  th[3] = U2 / T;
  th[0] = log(rho / (2.0 * kPi * T * sqrt(2.0 * kPi * T))) - 0.5 * uu / T;
  return true;
}

// Newton for the weighted discrete Maxwellian from the guess in th. The residual F is
// evaluated in E (FP64 or FP32) and the direction from the FP32 factorisation (inexact
// Newton: the root is the one of F in E). The step is halved while the scaled residual
// grows; the iteration stops right after a step whose exponent change
// |da| + L sum|db| + L^2 |dg| is below tol. On return ev holds the evaluation at th.
template <typename E>
__device__ inline int maxwellian_newton(int N, double dv, double w, bool wv1, double inv_dx, const E* target,
                                        double* th, double tol, int maxit, MaxwEval<E>& ev) {
  double L = node(N - 1, N, dv);
  maxw_eval<E>(N, dv, w, wv1, inv_dx, target, th, ev);
  for (int it = 0; it < maxit; it++) {
    float y[5], Ff[5];
#pragma unroll
    for (int i = 0; i < 5; i++) Ff[i] = (float)tod(ev.F[i]);
    if (!chol5_solve(ev.A, Ff, y)) return -1;
    double d[5] = {-(double)y[0], -(double)y[1], -(double)y[2], -(double)y[3], (double)y[4]};  // -D A^{-1} F
    double lam = 1.0;
    double fn = ev.fn;
    double tt[5];
    for (int hv = 0; hv < 40; hv++) {
#pragma unroll
      for (int i = 0; i < 5; i++) tt[i] = th[i] + lam * d[i];
      maxw_eval<E>(N, dv, w, wv1, inv_dx, target, tt, ev);
      if (ev.fn == ev.fn && (ev.fn <= fn || ev.fn <= 1e-10)) break;
      lam *= 0.5;
    }
#pragma unroll
    for (int i = 0; i < 5; i++) th[i] = tt[i];
    double step = lam * (fabs(d[0]) + L * (fabs(d[1]) + fabs(d[2]) + fabs(d[3])) + L * L * fabs(d[4]));
    if (!(step == step)) return -1;
    if (step <= tol) return it + 1;
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
