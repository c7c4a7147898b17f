#include <algorithm>
// Collision step (eqs. (13)-(16), (28)) for every cell of every instance.
//
// Q = Q^FSM[f,f] - Q^FSM[M,M] is evaluated as the single symmetric bilinear sum
//   Q_s(a, b)_k = sum_{l+m=k} beta_s(l, m) ahat_l bhat_m,   a = f - M, b = f + M,
//   beta_s(l, m) = G(|l+m|, |l-m|) - (G(2|l|, 0) + G(2|m|, 0)) / 2,
// which equals the two-evaluation form exactly (Q_s is symmetric and Q_s(f,f) = Q^FSM[f,f])
// and carries no cancellation between two large terms at small eps.
//
// Data flow per launch sequence:
//   k_moments        f -> moments, discrete Maxwellian theta, nu            (FP64)
//   k_dft_i3/i2/i1   f -+ M -> ahat, bhat in the spectral layout [group][k1][k2][k3][lane]
//   k_sum            ahat, bhat, weight blocks -> partial qhat per work unit
//   k_sum_reduce     partials -> qhat (fixed order, FP64 accumulation), Hermitian mirror
//   k_idft_k1/k2/k3  qhat -> Q(v), P = Q - nu (M - f)
// A spectral group packs 32 cells, one per warp lane, so every weight is warp-uniform.
#include <cstdio>

#include "common.cuh"
#include "kernels.h"

namespace sgs {

// ---------------------------------------------------------------------------------------
// Moments and discrete Maxwellian of every cell.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_moments(const double* __restrict__ f, CellTables ct, int N, double dv,
                                                  double newton_tol, int newton_max, double* __restrict__ theta,
                                                  double* __restrict__ nu, Counters* cnt) {
  __shared__ double vv[kMaxN];
  __shared__ double part[8][5];
  int c = blockIdx.x;
  if (!cell_active(ct.active, ct.cell_inst, c)) return;
  int K = N * N * N;
  const double* fc = f + ct.cell_off[c];
  if (threadIdx.x < N) vv[threadIdx.x] = node(threadIdx.x, N, dv);
  __syncthreads();
  double s[5] = {0, 0, 0, 0, 0};
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    int i3 = e % N, i2 = (e / N) % N, i1 = e / (N * N);
    double x = fc[e];
    double a = vv[i1], b = vv[i2], d = vv[i3];
    s[0] += x;
    s[1] += x * a;
    s[2] += x * b;
    s[3] += x * d;
    s[4] += x * (a * a + b * b + d * d);
  }
  warp_allsum<5>(s);
  int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int q = 0; q < 5; q++) part[wid][q] = s[q];
  __syncthreads();
  if (wid != 0) return;
  double w = dv * dv * dv;
  double m[5];
  for (int q = 0; q < 5; q++) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += part[k][q];
    m[q] = w * t;
  }
  const InstDev& I = ct.inst[ct.cell_inst[c]];
  double th[5] = {0, 0, 0, 0, 0};
  MaxwEval<double> ev;
  int it = -1;
  if (continuum_guess<double>(m, th))
    it = maxwellian_newton<double>(N, dv, w, false, 0.0, m, th, newton_tol, newton_max, ev);
  double rho = m[0];
  double T = (m[4] / rho - (m[1] * m[1] + m[2] * m[2] + m[3] * m[3]) / (rho * rho)) / 3.0;
  // penalty frequency of eq. (28): the loss frequency 4 pi b0 rho for Maxwell molecules;
  // for hard spheres its supremum over the truncated kernel |q| <= 2R, 4 pi b0 rho 2R with
  // R = 2L / (3 sqrt 2 + 1) and 2L = N dv, so that no stiff part of the loss term is left
  // in P (a mean loss frequency lets the explicit remainder grow at large |v|)
  double nuv = 4.0 * kPi * I.b0 * rho;
  if (I.collision == SGS_HARD_SPHERE) nuv *= 2.0 * (N * dv) / (3.0 * sqrt(2.0) + 1.0);
  if (lane == 0) {
    for (int q = 0; q < 5; q++) theta[5 * c + q] = th[q];
    nu[c] = nuv;
    unsigned bits = 0;
    if (it < 0) bits |= SGS_ST_NEWTON_FAIL;
    if (!(rho > 0.0) || !(T > 0.0)) bits |= SGS_ST_NONPOSITIVE;
    if (!(rho == rho) || !(T == T)) bits |= SGS_ST_NONFINITE;
    if (bits) atomicOr(&cnt[ct.cell_inst[c]].status, bits);
  }
}

// Per-block factors E_d[i] of the discrete Maxwellian of cell c (E_1 carries exp(alpha)).
__device__ inline void maxwell_factors(const double* theta, int c, int N, double dv, double* E /*[3][kMaxN]*/);

// Separable factors of every cell's Maxwellian, once per collision step (one block per
// cell), for the transform passes to read instead of re-evaluating 3N exponentials per block.
__global__ void k_factors(const double* theta, int N, double dv, double* efac) {
  maxwell_factors(theta, blockIdx.x, N, dv, efac + (long long)blockIdx.x * 3 * kMaxN);
}

__device__ inline void maxwell_factors(const double* theta, int c, int N, double dv, double* E /*[3][kMaxN]*/) {
  if (threadIdx.x < 3 * N) {
    int d = threadIdx.x / N, i = threadIdx.x % N;
    const double* th = theta + 5 * c;
    double v = node(i, N, dv);
    double x = th[1 + d] * v - th[4] * v * v;
    if (d == 0) x += th[0];
    E[d * kMaxN + i] = exp(x);
  }
}

// ---------------------------------------------------------------------------------------
// Forward DFT, fhat_k = N^-3 sum_v f(v) exp(-i 2 pi k j / N), one index at a time.
// Pass 1 (index 3) forms a = f - M and b = f + M in FP64 and transforms them in T.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_dft_i3(const double* __restrict__ f, CellTables ct, const double* efac,
                                                 const double* efac_ref, SpecBufs<T> sb, int N, double dv,
                                                 DftMode md) {
  extern __shared__ __align__(16) unsigned char smraw[];
  int n = N - 1;
  T* cs = (T*)smraw;             // [N][n] cos, transposed: k3 fastest, so that the threads of
  T* sn = cs + n * N;            // [N][n] sin  a warp (consecutive k3) read consecutive banks
  T* sa = sn + n * N;            // [N][N] a slab (i2, i3)
  T* sbb = sa + N * N;           // [N][N] b slab
  // M = E1[i1] E2[i2] E3[i3]: E12[i2] = E1[i1] E2[i2] for this block's i1, then one product
  __shared__ double E12[kMaxN], E3[kMaxN], E12r[kMaxN], E3r[kMaxN];
  int c = blockIdx.x, i1 = blockIdx.y;
  if (!cell_active(ct.active, ct.cell_inst, c)) return;
  if (threadIdx.x < N) {
    const double* e = efac + (long long)c * 3 * kMaxN;
    E12[threadIdx.x] = e[i1] * e[kMaxN + threadIdx.x];
    E3[threadIdx.x] = e[2 * kMaxN + threadIdx.x];
    if (md.mode != 0) {
      const double* er = efac_ref + (long long)c * 3 * kMaxN;
      E12r[threadIdx.x] = er[i1] * er[kMaxN + threadIdx.x];
      E3r[threadIdx.x] = er[2 * kMaxN + threadIdx.x];
    }
  }
  for (int t = threadIdx.x; t < n * N; t += blockDim.x) {
    int k3 = t / N, i3 = t % N;
    cs[i3 * n + k3] = sb.twc[t];
    sn[i3 * n + k3] = sb.tws[t];
  }
  __syncthreads();
  const long long off = ct.cell_off[c] + (long long)i1 * N * N;
  const double* fc = f + off;
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    int i2 = t / N, i3 = t % N;
    double M = E12[i2] * E3[i3];
    double x = fc[t];
    if (md.mode == 0) {  // a = f - M, b = f + M
      sa[t] = (T)(x - M);
      sbb[t] = (T)(x + M);
    } else {  // increments against the reference state f_ref, M_ref (exact in FP64, then rounded)
      double Mr = E12r[i2] * E3r[i3];
      double xr = md.f_ref[off + t];
      if (md.mode == 1) {  // a = (f - M) - (f_ref - M_ref), b = f + M
        sa[t] = (T)((x - xr) - (M - Mr));
        sbb[t] = (T)(x + M);
      } else {  // a unused, b = (f + M) - (f_ref + M_ref)
        sa[t] = (T)0;
        sbb[t] = (T)((x - xr) + (M - Mr));
      }
    }
  }
  __syncthreads();
  typedef typename CplxOf<T>::type CT;
  CT* oa = sb.st1a + ((long long)c * N + i1) * N * n;
  CT* ob = sb.st1b + ((long long)c * N + i1) * N * n;
  for (int t = threadIdx.x; t < N * n; t += blockDim.x) {
    int i2 = t / n, k3 = t % n;
    T ar = 0, ai = 0, br = 0, bi = 0;
    for (int i3 = 0; i3 < N; i3++) {
      T co = cs[i3 * n + k3], si = sn[i3 * n + k3];
      T a = sa[i2 * N + i3], b = sbb[i2 * N + i3];
      ar += a * co;
      ai -= a * si;
      br += b * co;
      bi -= b * si;
    }
    oa[t] = make_cplx(ar, ai);
    ob[t] = make_cplx(br, bi);
  }
}

// Pass 2 (index 2): [c][i1][i2][k3] -> [c][i1][k2][k3].
template <typename T>
__global__ void __launch_bounds__(256) k_dft_i2(SpecBufs<T> sb, int N) {
  typedef typename CplxOf<T>::type CT;
  extern __shared__ __align__(16) unsigned char smraw[];
  int n = N - 1;
  T* cs = (T*)smraw;
  T* sn = cs + n * N;
  CT* xa = (CT*)(sn + n * N);  // [N][n]
  CT* xb = xa + N * n;
  int c = blockIdx.x, i1 = blockIdx.y;
  if (!cell_active(sb.active, sb.cell_inst, c)) return;
  for (int t = threadIdx.x; t < n * N; t += blockDim.x) {
    cs[t] = sb.twc[t];
    sn[t] = sb.tws[t];
  }
  const CT* ia = sb.st1a + ((long long)c * N + i1) * N * n;
  const CT* ib = sb.st1b + ((long long)c * N + i1) * N * n;
  for (int t = threadIdx.x; t < N * n; t += blockDim.x) {
    xa[t] = ia[t];
    xb[t] = ib[t];
  }
  __syncthreads();
  CT* oa = sb.st2a + ((long long)c * N + i1) * n * n;
  CT* ob = sb.st2b + ((long long)c * N + i1) * n * n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int k2 = t / n, k3 = t % n;
    T ar = 0, ai = 0, br = 0, bi = 0;
    for (int i2 = 0; i2 < N; i2++) {
      T co = cs[k2 * N + i2], si = -sn[k2 * N + i2];
      CT a = xa[i2 * n + k3], b = xb[i2 * n + k3];
      ar += a.x * co - a.y * si;
      ai += a.x * si + a.y * co;
      br += b.x * co - b.y * si;
      bi += b.x * si + b.y * co;
    }
    oa[t] = make_cplx(ar, ai);
    ob[t] = make_cplx(br, bi);
  }
}

// Pass 3 (index 1): [c][i1][k2][k3] -> spectral layout [g][k1][k2][k3][lane], times N^-3.
template <typename T>
__global__ void __launch_bounds__(256) k_dft_i1(SpecBufs<T> sb, int N) {
  typedef typename CplxOf<T>::type CT;
  extern __shared__ __align__(16) unsigned char smraw[];
  int n = N - 1;
  T* cs = (T*)smraw;
  T* sn = cs + n * N;
  CT* xa = (CT*)(sn + n * N);  // [N][n] (i1, k3)
  CT* xb = xa + N * n;
  int c = blockIdx.x, k2 = blockIdx.y;
  if (!cell_active(sb.active, sb.cell_inst, c)) return;
  for (int t = threadIdx.x; t < n * N; t += blockDim.x) {
    cs[t] = sb.twc[t];
    sn[t] = sb.tws[t];
  }
  for (int t = threadIdx.x; t < N * n; t += blockDim.x) {
    int i1 = t / n, k3 = t % n;
    long long src = (((long long)c * N + i1) * n + k2) * n + k3;
    xa[t] = sb.st2a[src];
    xb[t] = sb.st2b[src];
  }
  __syncthreads();
  T scale = (T)(1.0 / ((double)N * N * N));
  int g = c / kLanes, lane = c % kLanes;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int k1 = t / n, k3 = t % n;
    T ar = 0, ai = 0, br = 0, bi = 0;
    for (int i1 = 0; i1 < N; i1++) {
      T co = cs[k1 * N + i1], si = -sn[k1 * N + i1];
      CT a = xa[i1 * n + k3], b = xb[i1 * n + k3];
      ar += a.x * co - a.y * si;
      ai += a.x * si + a.y * co;
      br += b.x * co - b.y * si;
      bi += b.x * si + b.y * co;
    }
    long long o = ((((long long)g * n + k1) * n + k2) * n + k3) * kLanes + lane;
    sb.ahat[o] = make_cplx(ar * scale, ai * scale);
    sb.bhat[o] = make_cplx(br * scale, bi * scale);
  }
}

// ---------------------------------------------------------------------------------------
// Direct spectral sum. Work unit = one output row (k1, k2) of the Hermitian half and a
// range of m1; a step = one (m1, m2) with its weight block W[(m3, k3) valid pairs]
// precomputed at setup in exactly the loop order below. Each warp owns one group of 32
// cells (lane = cell) and accumulates the 2H+1 outputs k3 of the row in registers; the
// rows ahat[(k1-m1, k2-m2, .)] and bhat[(m1, m2, .)] and the weight block of the next
// step are brought in by bulk copies into shared memory while the current step computes.
// FP32 keeps both rows in registers (full unroll, weights read as warp-uniform shared
// loads); FP64 reads them from shared memory.
// ---------------------------------------------------------------------------------------
template <typename T, int H>
__global__ void __launch_bounds__(128) k_sum(SumArgs<T> a) {
  typedef typename CplxOf<T>::type CT;
  constexpr int n = 2 * H + 1;
  constexpr int NP = 3 * H * H + 3 * H + 1;
  constexpr int VEC = 16 / (int)sizeof(T);
  constexpr int PW = (NP + VEC - 1) / VEC * VEC;
  constexpr bool kRegs = sizeof(T) == 4;
  constexpr int kRowBufs = kRegs ? 1 : 2;
  typedef typename VecOf<T>::type VT;
  extern __shared__ __align__(128) unsigned char smraw[];
  T* Wb = (T*)smraw;                                   // [2][PW]
  CT* rows = (CT*)(smraw + 2 * PW * sizeof(T));        // [kRowBufs][NW][2][n][32]
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int s_err;

  const int NW = blockDim.x >> 5;
  const int4 ud = a.units[blockIdx.x];  // k1, k2, m1_lo, m1_hi
  const long long step0 = a.unit_step0[blockIdx.x];
  const int k1 = ud.x, k2 = ud.y, m1lo = ud.z, m1hi = ud.w;
  const int m2lo = max(-H, k2 - H), m2hi = min(H, k2 + H);
  const int nm2 = m2hi - m2lo + 1;
  const int S = (m1hi - m1lo + 1) * nm2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g0 = blockIdx.y * NW;
  const int ng = min(NW, a.G - g0);
  const uint32_t row_bytes = n * kLanes * sizeof(CT);
  const uint32_t stage_bytes = PW * sizeof(T) + ng * 2 * row_bytes;

  if (a.active) {
    // a block whose lane groups hold no cell of an active instance has nothing to compute
    __shared__ int s_any;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    const int c = (g0 + warp) * kLanes + lane;
    if (warp < ng && c < a.C && a.active[a.cell_inst[c]]) s_any = 1;
    __syncthreads();
    if (!s_any) return;
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_err = 0;
    fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](int s) {
    int m1 = m1lo + s / nm2, m2 = m2lo + s % nm2;
    int b = s & 1;
    mbar_arrive_expect_tx(&bar[b], stage_bytes);
    bulk_g2s(Wb + b * PW, a.W + (step0 + s) * PW, PW * sizeof(T), &bar[b]);
    int rb = kRegs ? 0 : b;
    for (int w = 0; w < ng; w++) {
      long long ga = (((long long)(g0 + w) * n + (k1 - m1 + H)) * n + (k2 - m2 + H)) * n * kLanes;
      long long gb = (((long long)(g0 + w) * n + (m1 + H)) * n + (m2 + H)) * n * kLanes;
      CT* dst = rows + ((rb * NW + w) * 2) * n * kLanes;
      bulk_g2s(dst, a.ahat + ga, row_bytes, &bar[b]);
      bulk_g2s(dst + n * kLanes, a.bhat + gb, row_bytes, &bar[b]);
    }
  };

  if (threadIdx.x == 0 && S > 0) issue(0);

  T accr[n], acci[n];
#pragma unroll
  for (int i = 0; i < n; i++) accr[i] = acci[i] = (T)0;

  const bool active = warp < ng;
  int fail_b = 0, fail_par = 0;
  for (int s = 0; s < S; s++) {
    const int b = s & 1;
    if (!mbar_wait(&bar[b], (s >> 1) & 1, a.spin_max)) {
      s_err = 1;
      fail_b = b;
      fail_par = (s >> 1) & 1;
    }
    const VT* W4 = (const VT*)(Wb + b * PW);
    if (kRegs) {
      CT Ar[n], Br[n];
      const CT* rw = rows + (warp * 2) * n * kLanes;
      if (active) {
#pragma unroll
        for (int i = 0; i < n; i++) {
          Ar[i] = rw[i * kLanes + lane];
          Br[i] = rw[(n + i) * kLanes + lane];
        }
      }
      __syncthreads();
      if (s_err) break;
      if (threadIdx.x == 0 && s + 1 < S) issue(s + 1);
      if (active) {
        VT wv;
        int p = 0;
#pragma unroll
        for (int m3 = -H; m3 <= H; m3++) {
          const CT bv = Br[m3 + H];
#pragma unroll
          for (int k3 = (m3 - H > -H ? m3 - H : -H); k3 <= (m3 + H < H ? m3 + H : H); k3++) {
            if (p % VEC == 0) wv = W4[p / VEC];
            const T w = vec_get(wv, p % VEC);
            p++;
            const CT av = Ar[k3 - m3 + H];
            const T br = w * bv.x, bi = w * bv.y;
            accr[k3 + H] = fma(av.x, br, accr[k3 + H]);
            accr[k3 + H] = fma(-av.y, bi, accr[k3 + H]);
            acci[k3 + H] = fma(av.x, bi, acci[k3 + H]);
            acci[k3 + H] = fma(av.y, br, acci[k3 + H]);
          }
        }
      }
    } else {
      __syncthreads();
      if (s_err) break;
      if (threadIdx.x == 0 && s + 1 < S) issue(s + 1);
      if (active) {
        const CT* rw = rows + ((b * NW + warp) * 2) * n * kLanes;
        VT wv;
        int p = 0;
#pragma unroll
        for (int m3 = -H; m3 <= H; m3++) {
          const CT bv = rw[(n + m3 + H) * kLanes + lane];
#pragma unroll
          for (int k3 = (m3 - H > -H ? m3 - H : -H); k3 <= (m3 + H < H ? m3 + H : H); k3++) {
            if (p % VEC == 0) wv = W4[p / VEC];
            const T w = vec_get(wv, p % VEC);
            p++;
            const CT av = rw[(k3 - m3 + H) * kLanes + lane];
            const T br = w * bv.x, bi = w * bv.y;
            accr[k3 + H] = fma(av.x, br, accr[k3 + H]);
            accr[k3 + H] = fma(-av.y, bi, accr[k3 + H]);
            acci[k3 + H] = fma(av.x, bi, acci[k3 + H]);
            acci[k3 + H] = fma(av.y, br, acci[k3 + H]);
          }
        }
      }
    }
  }
  if (s_err) {
    // A copy did not land within the spin limit: report, then wait (bounded) for that
    // phase so no copy is still writing this block's shared memory when it exits.
    if (threadIdx.x == 0) {
      atomicOr(&a.cnt[0].status, SGS_ST_TIMEOUT);
      mbar_wait(&bar[fail_b], fail_par, a.spin_max);
    }
    return;
  }
  if (active) {
    CT* out = a.partial + ((long long)blockIdx.x * a.Gs + (g0 + warp)) * n * kLanes;
#pragma unroll
    for (int i = 0; i < n; i++) out[i * kLanes + lane] = make_cplx(accr[i], acci[i]);
  }
}

// ---------------------------------------------------------------------------------------
// Direct spectral sum in double-float arithmetic on the FP32 pipes (the high-precision
// evaluation of the defect correction). Same units, steps and weight order as k_sum; the
// transformed rows arrive split into (hi, lo) float pairs (k_split_spec) and the weights as
// the FP32 table (hi) plus its FP32 remainder table (lo). Products are formed exactly in
// their leading part (FMA two-product) with first-order cross terms, and accumulated by
// error-free two-sums into (hi, lo) accumulators, so each term carries about 2^-48 relative
// error instead of FP32's 2^-24.
// One block of KW warps serves one group of 32 cells (lane = cell); warp w accumulates the
// outputs k3 = -H + w + KW j. Rows and weights are double-buffered in shared memory by
// bulk copies, as in k_sum.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void df_mul_acc(float xh, float xl, float yh, float yl, float& ah, float& al) {
  // (ah, al) += (xh + xl)(yh + yl), to first order in the low parts
  float q = xh * yh;
  float e = fmaf(xh, yh, -q);
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  float s = ah + q;
  float z = s - ah;
  float err = (ah - (s - z)) + (q - z);
  ah = s;
  al += err + e;
}

template <int H, int KW>
__global__ void __launch_bounds__(KW * 32, 2) k_sum_df(SumDfArgs a) {
  constexpr int n = 2 * H + 1;
  constexpr int NP = 3 * H * H + 3 * H + 1;
  constexpr int PW = (NP + 3) / 4 * 4;
  constexpr int NJ = (n + KW - 1) / KW;  // outputs per warp
  extern __shared__ __align__(128) unsigned char smraw[];
  float* Wb = (float*)smraw;                            // [2][2][PW]: buffer, (hi, lo)
  float4* rows = (float4*)(smraw + 4 * PW * sizeof(float));  // [2][2][n][32]: buffer, (a, b)
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int s_err;

  const int4 ud = a.units[blockIdx.x];
  const long long step0 = a.unit_step0[blockIdx.x];
  const int k1 = ud.x, k2 = ud.y, m1lo = ud.z, m1hi = ud.w;
  const int m2lo = max(-H, k2 - H), m2hi = min(H, k2 + H);
  const int nm2 = m2hi - m2lo + 1;
  const int S = (m1hi - m1lo + 1) * nm2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.y;
  const uint32_t row_bytes = n * kLanes * sizeof(float4);
  const uint32_t stage_bytes = 2 * PW * sizeof(float) + 2 * row_bytes;

  if (a.active) {
    // a group with no cell of an active instance has nothing to compute (every warp of the
    // block serves the same group: one warp's vote decides)
    const int c = g * kLanes + lane;
    const bool mine = c < a.C && a.active[a.cell_inst[c]];
    if (!__any_sync(0xffffffffu, mine)) return;
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_err = 0;
    fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](int s) {
    int m1 = m1lo + s / nm2, m2 = m2lo + s % nm2;
    int b = s & 1;
    mbar_arrive_expect_tx(&bar[b], stage_bytes);
    bulk_g2s(Wb + (2 * b) * PW, a.Whi + (step0 + s) * PW, PW * sizeof(float), &bar[b]);
    bulk_g2s(Wb + (2 * b + 1) * PW, a.Wlo + (step0 + s) * PW, PW * sizeof(float), &bar[b]);
    long long ga = (((long long)g * n + (k1 - m1 + H)) * n + (k2 - m2 + H)) * n * kLanes;
    long long gb = (((long long)g * n + (m1 + H)) * n + (m2 + H)) * n * kLanes;
    float4* dst = rows + (2 * b) * n * kLanes;
    bulk_g2s(dst, a.ahat + ga, row_bytes, &bar[b]);
    bulk_g2s(dst + n * kLanes, a.bhat + gb, row_bytes, &bar[b]);
  };

  if (threadIdx.x == 0 && S > 0) issue(0);

  float rh[NJ], rl[NJ], ih[NJ], il[NJ];
#pragma unroll
  for (int j = 0; j < NJ; j++) rh[j] = rl[j] = ih[j] = il[j] = 0.0f;

  int fail_b = 0, fail_par = 0;
  for (int s = 0; s < S; s++) {
    const int b = s & 1;
    if (!mbar_wait(&bar[b], (s >> 1) & 1, a.spin_max)) {
      s_err = 1;
      fail_b = b;
      fail_par = (s >> 1) & 1;
    }
    __syncthreads();
    if (s_err) break;
    // the other buffer was released by the barrier above: prefetch the next step into it
    if (threadIdx.x == 0 && s + 1 < S) issue(s + 1);
    const float* Wh = Wb + (2 * b) * PW;
    const float* Wl = Wh + PW;
    const float4* ra = rows + (2 * b) * n * kLanes;
    const float4* rb = ra + n * kLanes;
    int off = 0;  // first weight of the current m3 in the packed (m3, k3) order
    // m3 stays a loop (the body, unrolled over the warp's outputs, is long enough to
    // hide latency; unrolling m3 as well overflows the instruction cache)
#pragma unroll 1
    for (int m3 = -H; m3 <= H; m3++) {
      const int lo = m3 - H > -H ? m3 - H : -H, hi = m3 + H < H ? m3 + H : H;
      const float4 bv = rb[(m3 + H) * kLanes + lane];
#pragma unroll
      for (int j = 0; j < NJ; j++) {
        const int k3 = -H + warp + KW * j;
        if (k3 >= lo && k3 <= hi) {
          const int p = off + k3 - lo;
          const float wh = Wh[p], wl = Wl[p];
          const float4 av = ra[(k3 - m3 + H) * kLanes + lane];
          // w b = (w b_re, w b_im), leading parts exact
          float brh = wh * bv.x, brl = fmaf(wh, bv.x, -brh);
          brl = fmaf(wh, bv.y, brl);
          brl = fmaf(wl, bv.x, brl);
          float bih = wh * bv.z, bil = fmaf(wh, bv.z, -bih);
          bil = fmaf(wh, bv.w, bil);
          bil = fmaf(wl, bv.z, bil);
          // a (w b): re += a_re br - a_im bi, im += a_re bi + a_im br
          df_mul_acc(av.x, av.y, brh, brl, rh[j], rl[j]);
          df_mul_acc(-av.z, -av.w, bih, bil, rh[j], rl[j]);
          df_mul_acc(av.x, av.y, bih, bil, ih[j], il[j]);
          df_mul_acc(av.z, av.w, brh, brl, ih[j], il[j]);
        }
      }
      off += hi - lo + 1;
    }
  }
  if (s_err) {
    if (threadIdx.x == 0) {
      atomicOr(&a.cnt[0].status, SGS_ST_TIMEOUT);
      mbar_wait(&bar[fail_b], fail_par, a.spin_max);
    }
    return;
  }
  double2* out = a.partial + ((long long)blockIdx.x * a.Gs + g) * n * kLanes;
#pragma unroll
  for (int j = 0; j < NJ; j++) {
    const int k3 = -H + warp + KW * j;
    if (k3 <= H)
      out[(k3 + H) * kLanes + lane] = make_double2((double)rh[j] + (double)rl[j], (double)ih[j] + (double)il[j]);
  }
}

// In place: every complex FP64 value of the transformed rows becomes its (hi, lo) float pairs
// (re_hi, re_lo, im_hi, im_lo), the layout k_sum_df reads.
__global__ void k_split_spec(double2* x, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    double2 v = x[i];
    dfloat r = df_split(v.x), m = df_split(v.y);
    reinterpret_cast<float4*>(x)[i] = make_float4(r.hi, r.lo, m.hi, m.lo);
  }
}

// Fixed-order sum of a row's unit partials (FP64 accumulation), written to qhat at (k1, k2,
// k3) and conjugated at (-k1, -k2, -k3); row (0, 0) is computed in full and not mirrored.
template <typename T>
__global__ void k_sum_reduce(RedArgs<T> a) {
  typedef typename CplxOf<T>::type CT;
  int row = blockIdx.x, g = blockIdx.y;
  int n = a.n, H = (n - 1) / 2;
  int k1 = a.row_k[row].x, k2 = a.row_k[row].y;
  int u0 = a.row_start[row], u1 = a.row_start[row + 1];
  for (int t = threadIdx.x; t < n * kLanes; t += blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int q = u0; q < u1; q++) {
      int u = a.row_units[q];
      CT v = a.partial[((long long)u * a.Gs + g) * n * kLanes + t];
      sr += (double)v.x;
      si += (double)v.y;
    }
    if (a.partial2)
      for (int q = u0; q < u1; q++) {
        int u = a.row_units[q];
        CT v = a.partial2[((long long)u * a.Gs + g) * n * kLanes + t];
        sr += (double)v.x;
        si += (double)v.y;
      }
    int k3i = t / kLanes, lane = t % kLanes;
    long long o = ((((long long)g * n + (k1 + H)) * n + (k2 + H)) * n + k3i) * kLanes + lane;
    a.qhat[o] = make_cplx((T)sr, (T)si);
    if (k1 != 0 || k2 != 0) {
      long long om = ((((long long)g * n + (H - k1)) * n + (H - k2)) * n + (n - 1 - k3i)) * kLanes + lane;
      a.qhat[om] = make_cplx((T)sr, (T)(-si));
    }
  }
}

// ---------------------------------------------------------------------------------------
// Inverse DFT, q(v) = Re sum_k qhat_k exp(+i 2 pi k j / N).
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_idft_k1(SpecBufs<T> sb, int N) {
  typedef typename CplxOf<T>::type CT;
  extern __shared__ __align__(16) unsigned char smraw[];
  int n = N - 1;
  T* cs = (T*)smraw;
  T* sn = cs + n * N;
  CT* x = (CT*)(sn + n * N);  // [k1][k3]
  int c = blockIdx.x, k2 = blockIdx.y;
  if (!cell_active(sb.active, sb.cell_inst, c)) return;
  int g = c / kLanes, lane = c % kLanes;
  for (int t = threadIdx.x; t < n * N; t += blockDim.x) {
    cs[t] = sb.twc[t];
    sn[t] = sb.tws[t];
  }
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int k1 = t / n, k3 = t % n;
    x[t] = sb.qhat[((((long long)g * n + k1) * n + k2) * n + k3) * kLanes + lane];
  }
  __syncthreads();
  CT* o = sb.st2a + (long long)c * N * n * n;  // [i1][k2][k3]
  for (int t = threadIdx.x; t < N * n; t += blockDim.x) {
    int i1 = t / n, k3 = t % n;
    T re = 0, im = 0;
    for (int k1 = 0; k1 < n; k1++) {
      T co = cs[k1 * N + i1], si = sn[k1 * N + i1];
      CT q = x[k1 * n + k3];
      re += q.x * co - q.y * si;
      im += q.x * si + q.y * co;
    }
    o[((long long)i1 * n + k2) * n + k3] = make_cplx(re, im);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_idft_k2(SpecBufs<T> sb, int N) {
  typedef typename CplxOf<T>::type CT;
  extern __shared__ __align__(16) unsigned char smraw[];
  int n = N - 1;
  T* cs = (T*)smraw;
  T* sn = cs + n * N;
  CT* x = (CT*)(sn + n * N);  // [k2][k3]
  int c = blockIdx.x, i1 = blockIdx.y;
  if (!cell_active(sb.active, sb.cell_inst, c)) return;
  for (int t = threadIdx.x; t < n * N; t += blockDim.x) {
    cs[t] = sb.twc[t];
    sn[t] = sb.tws[t];
  }
  const CT* src = sb.st2a + ((long long)c * N + i1) * n * n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) x[t] = src[t];
  __syncthreads();
  CT* o = sb.st1a + ((long long)c * N + i1) * N * n;  // [i2][k3]
  for (int t = threadIdx.x; t < N * n; t += blockDim.x) {
    int i2 = t / n, k3 = t % n;
    T re = 0, im = 0;
    for (int k2 = 0; k2 < n; k2++) {
      T co = cs[k2 * N + i2], si = sn[k2 * N + i2];
      CT q = x[k2 * n + k3];
      re += q.x * co - q.y * si;
      im += q.x * si + q.y * co;
    }
    o[t] = make_cplx(re, im);
  }
}

// Last pass: real part along index 3, then Q and P = Q - nu (M - f) in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_idft_k3(SpecBufs<T> sb, const double* __restrict__ f, CellTables ct,
                                                  const double* efac, const double* nu, double* Q, double* P,
                                                  int N, double dv, const double* __restrict__ Qadd,
                                                  double* __restrict__ mom) {
  typedef typename CplxOf<T>::type CT;
  extern __shared__ __align__(16) unsigned char smraw[];
  int n = N - 1;
  T* cs = (T*)smraw;
  T* sn = cs + n * N;
  CT* x = (CT*)(sn + n * N);  // [i2][k3]
  __shared__ double E12[kMaxN], E3[kMaxN];
  int c = blockIdx.x, i1 = blockIdx.y;
  if (!cell_active(ct.active, ct.cell_inst, c)) return;
  if (threadIdx.x < N) {
    const double* e = efac + (long long)c * 3 * kMaxN;
    E12[threadIdx.x] = e[i1] * e[kMaxN + threadIdx.x];
    E3[threadIdx.x] = e[2 * kMaxN + threadIdx.x];
  }
  for (int t = threadIdx.x; t < n * N; t += blockDim.x) {
    cs[t] = sb.twc[t];
    sn[t] = sb.tws[t];
  }
  const CT* src = sb.st1a + ((long long)c * N + i1) * N * n;
  for (int t = threadIdx.x; t < N * n; t += blockDim.x) x[t] = src[t];
  __syncthreads();
  long long base = ct.cell_off[c] + (long long)i1 * N * N;
  double nuc = nu[c];
  // moments of this slab for the conservation projection: sum q, v2 q, v3 q, (v2^2 + v3^2) q
  double m0 = 0.0, m2 = 0.0, m3 = 0.0, m4 = 0.0;
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    int i2 = t / N, i3 = t % N;
    T re = 0;
    for (int k3 = 0; k3 < n; k3++) {
      CT q = x[i2 * n + k3];
      re += q.x * cs[k3 * N + i3] - q.y * sn[k3 * N + i3];
    }
    double q = (double)re;
    if (Qadd) q += Qadd[base + t];
    if (Q) Q[base + t] = q;
    if (P) {
      double M = E12[i2] * E3[i3];
      P[base + t] = q - nuc * (M - f[base + t]);
    }
    if (mom) {
      double v2 = (i2 - N / 2 + 1) * dv, v3 = (i3 - N / 2 + 1) * dv;
      m0 += q;
      m2 += v2 * q;
      m3 += v3 * q;
      m4 += (v2 * v2 + v3 * v3) * q;
    }
  }
  if (mom) {  // fixed-order block reduction (warp butterflies, then warps in order)
    __shared__ double red[4][8];
    for (int o = 16; o > 0; o >>= 1) {
      m0 += __shfl_xor_sync(0xffffffffu, m0, o);
      m2 += __shfl_xor_sync(0xffffffffu, m2, o);
      m3 += __shfl_xor_sync(0xffffffffu, m3, o);
      m4 += __shfl_xor_sync(0xffffffffu, m4, o);
    }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      red[0][w] = m0;
      red[1][w] = m2;
      red[2][w] = m3;
      red[3][w] = m4;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s[4] = {0.0, 0.0, 0.0, 0.0};
      for (int j = 0; j < 4; j++)
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) s[j] += red[j][k];
      double v1 = (i1 - N / 2 + 1) * dv;
      double* o = mom + ((long long)c * N + i1) * 5;
      o[0] = s[0];
      o[1] = v1 * s[0];
      o[2] = s[1];
      o[3] = s[2];
      o[4] = v1 * v1 * s[0] + s[3];
    }
  }
}

// Conservation projection (an option; not in the paper), applied to Q and to
// P = Q - nu (M - f) alike, with phi = (1, v1, v2, v3, |v|^2) and the moments sum_k phi Q from
// the slabs of k_idft_k3, summed here in i1 order (every block of a cell forms the same lambda):
//   mode 1: Q_c = Q - sum_i lambda_i phi_i,      (sum_k phi phi^T) lambda = sum_k phi Q,
//           with the inverse Gram matrix Ainv of the grid;
//   mode 2: Q_c = Q - M sum_i lambda_i phi_i,    (sum_k M phi phi^T) lambda = sum_k phi Q,
//           with the cell's Maxwellian M = E1(v1) E2(v2) E3(v3) (factors efac): its Gram
//           matrix is a sum of products of the 1-D sums S_d^p = sum_i E_d(v_i) v_i^p.
__device__ bool chol5_solve(double A[5][5], const double* b, double* x) {
  for (int i = 0; i < 5; i++)
    for (int j = 0; j <= i; j++) {
      double t = A[i][j];
      for (int k = 0; k < j; k++) t -= A[i][k] * A[j][k];
      if (i == j) {
        if (!(t > 0.0)) return false;
        A[i][i] = sqrt(t);
      } else {
        A[i][j] = t / A[j][j];
      }
    }
  double z[5];
  for (int i = 0; i < 5; i++) {
    double t = b[i];
    for (int k = 0; k < i; k++) t -= A[i][k] * z[k];
    z[i] = t / A[i][i];
  }
  for (int i = 4; i >= 0; i--) {
    double t = z[i];
    for (int k = i + 1; k < 5; k++) t -= A[k][i] * x[k];
    x[i] = t / A[i][i];
  }
  return true;
}

__global__ void __launch_bounds__(256) k_conserve_apply(const double* __restrict__ mom,
                                                        const double* __restrict__ Ainv,
                                                        const double* __restrict__ efac, int mode, CellTables ct,
                                                        double* Q, double* P, double* Qraw, int N, double dv) {
  __shared__ double sm[5], lam[5], S[3][5];
  int c = blockIdx.x, i1 = blockIdx.y;
  if (!cell_active(ct.active, ct.cell_inst, c)) return;
  const double* e = efac + (long long)c * 3 * kMaxN;
  if (threadIdx.x < 5) {
    double a = 0.0;
    const double* m = mom + (long long)c * N * 5 + threadIdx.x;
    for (int j = 0; j < N; j++) a += m[j * 5];
    sm[threadIdx.x] = a;
  } else if (mode == 2 && threadIdx.x < 20) {
    int d = (threadIdx.x - 5) / 5, p = (threadIdx.x - 5) % 5;
    double a = 0.0;
    for (int i = 0; i < N; i++) {
      double v = (i - N / 2 + 1) * dv, vp = 1.0;
      for (int k = 0; k < p; k++) vp *= v;
      a += e[d * kMaxN + i] * vp;
    }
    S[d][p] = a;
  }
  __syncthreads();
  if (mode == 1 && threadIdx.x < 5) {
    double a = 0.0;
    for (int k = 0; k < 5; k++) a += Ainv[threadIdx.x * 5 + k] * sm[k];
    lam[threadIdx.x] = a;
  } else if (mode == 2 && threadIdx.x == 0) {
    // phi as monomials v1^a v2^b v3^c: 1, v1, v2, v3 and |v|^2 = v1^2 + v2^2 + v3^2
    const int nm[5] = {1, 1, 1, 1, 3};
    const int mono[5][3][3] = {{{0, 0, 0}}, {{1, 0, 0}}, {{0, 1, 0}}, {{0, 0, 1}},
                               {{2, 0, 0}, {0, 2, 0}, {0, 0, 2}}};
    double A[5][5];
    for (int a = 0; a < 5; a++)
      for (int b = 0; b < 5; b++) {
        double t = 0.0;
        for (int x = 0; x < nm[a]; x++)
          for (int y = 0; y < nm[b]; y++)
            t += S[0][mono[a][x][0] + mono[b][y][0]] * S[1][mono[a][x][1] + mono[b][y][1]] *
                 S[2][mono[a][x][2] + mono[b][y][2]];
        A[a][b] = t;
      }
    double x[5];
    if (!chol5_solve(A, sm, x))
      for (int k = 0; k < 5; k++) x[k] = 0.0;
    for (int k = 0; k < 5; k++) lam[k] = x[k];
  }
  __syncthreads();
  double v1 = (i1 - N / 2 + 1) * dv;
  double c0 = lam[0] + lam[1] * v1 + lam[4] * v1 * v1;
  double e1 = mode == 2 ? e[i1] : 1.0;
  long long base = ct.cell_off[c] + (long long)i1 * N * N;
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    int i2 = t / N, i3 = t % N;
    double v2 = (i2 - N / 2 + 1) * dv, v3 = (i3 - N / 2 + 1) * dv;
    double corr = c0 + lam[2] * v2 + lam[3] * v3 + lam[4] * (v2 * v2 + v3 * v3);
    if (mode == 2) corr *= e1 * e[kMaxN + i2] * e[2 * kMaxN + i3];
    if (Qraw) Qraw[base + t] = Q[base + t];  // the unprojected operator (increment-form reference)
    if (Q) Q[base + t] -= corr;
    if (P) P[base + t] -= corr;
  }
}

// BGK mode (eq. (12)): Q = nu (M - f), P = 0.
__global__ void __launch_bounds__(256) k_collide_bgk(const double* __restrict__ f, CellTables ct,
                                                      const double* theta, const double* nu, double* Q, double* P,
                                                      int N, double dv) {
  __shared__ double E[3 * kMaxN];
  int c = blockIdx.x, i1 = blockIdx.y;
  if (!cell_active(ct.active, ct.cell_inst, c)) return;
  maxwell_factors(theta, c, N, dv, E);
  __syncthreads();
  long long base = ct.cell_off[c] + (long long)i1 * N * N;
  double nuc = nu[c];
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    int i2 = t / N, i3 = t % N;
    double M = E[i1] * E[kMaxN + i2] * E[2 * kMaxN + i3];
    if (Q) Q[base + t] = nuc * (M - f[base + t]);
    if (P) P[base + t] = 0.0;
  }
}

// ---------------------------------------------------------------------------------------
// Setup: weight blocks W[step][p] = beta_s for the (m3, k3) pairs of each (k1, k2, m1, m2)
// step, in the loop order of k_sum, from the tables G[a2][b2] and Lo[m2] = G(2|m|, 0).
// ---------------------------------------------------------------------------------------
template <typename T, bool LO>
__global__ void k_build_weights(const int4* units, const long long* unit_step0, int n_units, int H, int PW,
                                const double* G, long long nb, const double* Lo, T* W) {
  int u = blockIdx.x;
  if (u >= n_units) return;
  int4 ud = units[u];
  int k1 = ud.x, k2 = ud.y;
  int m2lo = max(-H, k2 - H), m2hi = min(H, k2 + H);
  int nm2 = m2hi - m2lo + 1;
  int S = (ud.w - ud.z + 1) * nm2;
  int np = 3 * H * H + 3 * H + 1;
  for (int s = blockIdx.y; s < S; s += gridDim.y) {
    int m1 = ud.z + s / nm2, m2 = m2lo + s % nm2;
    T* out = W + (unit_step0[u] + s) * PW;
    for (int p = threadIdx.x; p < PW; p += blockDim.x) {
      if (p >= np) {
        out[p] = (T)0;
        continue;
      }
      // invert p -> (m3, k3) in the k_sum loop order
      int q = p, m3 = -H, k3 = 0;
      for (m3 = -H; m3 <= H; m3++) {
        int lo = max(-H, m3 - H), hi = min(H, m3 + H);
        int cnt = hi - lo + 1;
        if (q < cnt) {
          k3 = lo + q;
          break;
        }
        q -= cnt;
      }
      long long a2 = (long long)k1 * k1 + (long long)k2 * k2 + (long long)k3 * k3;
      long long d1 = k1 - 2 * m1, d2 = k2 - 2 * m2, d3 = k3 - 2 * m3;
      long long b2 = d1 * d1 + d2 * d2 + d3 * d3;
      long long l1 = k1 - m1, l2 = k2 - m2, l3 = k3 - m3;
      long long ll = l1 * l1 + l2 * l2 + l3 * l3;
      long long mm = (long long)m1 * m1 + (long long)m2 * m2 + (long long)m3 * m3;
      double w = G[a2 * nb + b2] - 0.5 * (Lo[ll] + Lo[mm]);
      // LO: the FP32 remainder w - (float)w, the low half of a double-float weight whose high
      // half is the FP32 weight table
      out[p] = LO ? (T)(w - (double)(float)w) : (T)w;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Host-side launchers.
// ---------------------------------------------------------------------------------------
template <typename T>
static size_t dft_smem(int N, int extra_cplx, int extra_real) {
  typedef typename CplxOf<T>::type CT;
  int n = N - 1;
  return 2 * n * N * sizeof(T) + extra_cplx * sizeof(CT) + extra_real * sizeof(T);
}

template <typename T, int H>
static cudaError_t launch_sum_t(const SumArgs<T>& a, int NW, int n_units, cudaStream_t st) {
  typedef typename CplxOf<T>::type CT;
  constexpr int n = 2 * H + 1;
  constexpr int NP = 3 * H * H + 3 * H + 1;
  constexpr int VEC = 16 / (int)sizeof(T);
  constexpr int PW = (NP + VEC - 1) / VEC * VEC;
  constexpr int kRowBufs = sizeof(T) == 4 ? 1 : 2;
  size_t smem = 2 * PW * sizeof(T) + (size_t)kRowBufs * NW * 2 * n * kLanes * sizeof(CT);
  cudaError_t e = func_attr((const void*)k_sum<T, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(n_units, (a.G + NW - 1) / NW);
  k_sum<T, H><<<grid, NW * 32, smem, st>>>(a);
  return cudaGetLastError();
}

int sum_pad(int H, int elem_bytes) {
  int NP = 3 * H * H + 3 * H + 1, VEC = 16 / elem_bytes;
  return (NP + VEC - 1) / VEC * VEC;
}

template <typename T>
cudaError_t launch_sum(const SumArgs<T>& a, int H, int NW, int n_units, cudaStream_t st) {
  if (NW < 1 || NW > 4) return cudaErrorInvalidValue;
  switch (H) {
    case 3: return launch_sum_t<T, 3>(a, NW, n_units, st);
    case 5: return launch_sum_t<T, 5>(a, NW, n_units, st);
    case 7: return launch_sum_t<T, 7>(a, NW, n_units, st);
    case 9: return launch_sum_t<T, 9>(a, NW, n_units, st);
    case 11: return launch_sum_t<T, 11>(a, NW, n_units, st);
    case 13: return launch_sum_t<T, 13>(a, NW, n_units, st);
    case 15: return launch_sum_t<T, 15>(a, NW, n_units, st);
  }
  return cudaErrorInvalidValue;
}

template <int H>
static cudaError_t launch_sum_df_t(const SumDfArgs& a, int n_units, cudaStream_t st) {
  constexpr int n = 2 * H + 1;
  constexpr int NP = 3 * H * H + 3 * H + 1;
  constexpr int PW = (NP + 3) / 4 * 4;
  constexpr int KW = H >= 7 ? 8 : 4;
  size_t smem = 4 * PW * sizeof(float) + 4 * (size_t)n * kLanes * sizeof(float4);
  cudaError_t e = func_attr((const void*)k_sum_df<H, KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_sum_df<H, KW><<<dim3(n_units, a.G), KW * 32, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sum_df(const SumDfArgs& a, int H, int n_units, cudaStream_t st) {
  switch (H) {
    case 3: return launch_sum_df_t<3>(a, n_units, st);
    case 5: return launch_sum_df_t<5>(a, n_units, st);
    case 7: return launch_sum_df_t<7>(a, n_units, st);
    case 9: return launch_sum_df_t<9>(a, n_units, st);
    case 11: return launch_sum_df_t<11>(a, n_units, st);
    case 13: return launch_sum_df_t<13>(a, n_units, st);
    case 15: return launch_sum_df_t<15>(a, n_units, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_split_spec(double2* x, long long count, cudaStream_t st) {
  k_split_spec<<<(int)std::min<long long>((count + 255) / 256, 152 * 16), 256, 0, st>>>(x, count);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dft(const double* f, const CollideCtx<T>& x, const DftMode& md, cudaStream_t st) {
  int N = x.N, n = N - 1, C = x.C;
  cudaError_t e;
  k_factors<<<C, 3 * N, 0, st>>>(x.theta, N, x.dv, x.efac);
  if (md.mode != 0) k_factors<<<C, 3 * N, 0, st>>>(md.theta_ref, N, x.dv, x.efac_ref);
  size_t sm1 = dft_smem<T>(N, 0, 2 * N * N);
  e = func_attr((const void*)k_dft_i3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
  if (e != cudaSuccess) return e;
  k_dft_i3<T><<<dim3(C, N), 256, sm1, st>>>(f, x.ct, x.efac, x.efac_ref, x.sb, N, x.dv, md);
  size_t sm2 = dft_smem<T>(N, 2 * N * n, 0);
  e = func_attr((const void*)k_dft_i2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
  if (e != cudaSuccess) return e;
  k_dft_i2<T><<<dim3(C, N), 256, sm2, st>>>(x.sb, N);
  e = func_attr((const void*)k_dft_i1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
  if (e != cudaSuccess) return e;
  // groups beyond the last cell keep the zeros written at bind time
  k_dft_i1<T><<<dim3(C, n), 256, sm2, st>>>(x.sb, N);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spectral_sum(const CollideCtx<T>& x, typename CplxOf<T>::type* partial, cudaStream_t st) {
  SumArgs<T> a = x.sum;
  if (partial) a.partial = partial;
  return launch_sum<T>(a, x.H, x.NW, x.n_units, st);
}

template <typename T>
cudaError_t launch_reduce_idft(const double* f, double* Q, double* P, const CollideCtx<T>& x,
                               const typename CplxOf<T>::type* partial2, const double* Qadd, cudaStream_t st,
                               double* Qraw) {
  int N = x.N, n = N - 1, C = x.C;
  cudaError_t e;
  RedArgs<T> ra = x.red;
  ra.partial2 = partial2;
  // n_rows = 0: qhat is already complete (the fast operator writes it directly)
  if (x.red.n_rows > 0) k_sum_reduce<T><<<dim3(x.red.n_rows, x.red.G), 256, 0, st>>>(ra);
  size_t sm3 = dft_smem<T>(N, n * n, 0);
  e = func_attr((const void*)k_idft_k1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
  if (e != cudaSuccess) return e;
  k_idft_k1<T><<<dim3(C, n), 256, sm3, st>>>(x.sb, N);
  e = func_attr((const void*)k_idft_k2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
  if (e != cudaSuccess) return e;
  k_idft_k2<T><<<dim3(C, N), 256, sm3, st>>>(x.sb, N);
  size_t sm4 = dft_smem<T>(N, N * n, 0);
  e = func_attr((const void*)k_idft_k3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm4);
  if (e != cudaSuccess) return e;
  // the factors of this collision step were written by launch_dft
  k_idft_k3<T><<<dim3(C, N), 256, sm4, st>>>(x.sb, f, x.ct, x.efac, x.nu, Q, P, N, x.dv, Qadd, x.mom);
  e = cudaGetLastError();
  if (e != cudaSuccess || !x.mom) return e;
  if (Qraw && !Q) return cudaErrorInvalidValue;
  k_conserve_apply<<<dim3(C, N), 256, 0, st>>>(x.mom, x.cproj, x.efac, x.cproj_mode, x.ct, Q, P, Qraw, N, x.dv);
  return cudaGetLastError();
}

cudaError_t launch_factors(const double* theta, int C, int N, double dv, double* efac, cudaStream_t st) {
  k_factors<<<C, 3 * N, 0, st>>>(theta, N, dv, efac);
  return cudaGetLastError();
}

cudaError_t launch_moments(const double* f, const CellTables& ct, int C, int N, double dv, double tol, int maxit,
                           double* theta, double* nu, Counters* cnt, cudaStream_t st) {
  k_moments<<<C, 256, 0, st>>>(f, ct, N, dv, tol, maxit, theta, nu, cnt);
  return cudaGetLastError();
}

cudaError_t launch_collide_bgk(const double* f, const CellTables& ct, int C, int N, double dv, const double* theta,
                               const double* nu, double* Q, double* P, cudaStream_t st) {
  k_collide_bgk<<<dim3(C, N), 256, 0, st>>>(f, ct, theta, nu, Q, P, N, dv);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_build_weights(const int4* units, const long long* unit_step0, int n_units, int H, int PW,
                                 const double* G, long long nb, const double* Lo, T* W, cudaStream_t st) {
  k_build_weights<T, false><<<dim3(n_units, 8), 256, 0, st>>>(units, unit_step0, n_units, H, PW, G, nb, Lo, W);
  return cudaGetLastError();
}

cudaError_t launch_build_weights_lo(const int4* units, const long long* unit_step0, int n_units, int H, int PW,
                                    const double* G, long long nb, const double* Lo, float* W, cudaStream_t st) {
  k_build_weights<float, true><<<dim3(n_units, 8), 256, 0, st>>>(units, unit_step0, n_units, H, PW, G, nb, Lo, W);
  return cudaGetLastError();
}

template cudaError_t launch_dft<double>(const double*, const CollideCtx<double>&, const DftMode&, cudaStream_t);
template cudaError_t launch_dft<float>(const double*, const CollideCtx<float>&, const DftMode&, cudaStream_t);
template cudaError_t launch_spectral_sum<double>(const CollideCtx<double>&, double2*, cudaStream_t);
template cudaError_t launch_spectral_sum<float>(const CollideCtx<float>&, float2*, cudaStream_t);
template cudaError_t launch_reduce_idft<double>(const double*, double*, double*, const CollideCtx<double>&,
                                                const double2*, const double*, cudaStream_t, double*);
template cudaError_t launch_reduce_idft<float>(const double*, double*, double*, const CollideCtx<float>&,
                                               const float2*, const double*, cudaStream_t, double*);
template cudaError_t launch_build_weights<double>(const int4*, const long long*, int, int, int, const double*,
                                                  long long, const double*, double*, cudaStream_t);
template cudaError_t launch_build_weights<float>(const int4*, const long long*, int, int, int, const double*,
                                                 long long, const double*, float*, cudaStream_t);

}  // namespace sgs
