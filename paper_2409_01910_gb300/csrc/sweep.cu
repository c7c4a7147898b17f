// Persistent symmetric Gauss-Seidel scan (eq. (29), first order) with the preconditioned
// fixed-point cell solve (eqs. (20), (24)-(26)).
//
// One thread-block cluster per instance walks that instance's cells in scan order inside a
// single launch. Each thread owns EPT consecutive velocity nodes of one pencil (fixed i1, i2)
// in every cell, so a thread only ever reads and writes its own nodes: the upwind neighbour's
// new value is its own earlier write, and no two threads touch the same global element.
//
// The visit of a cell is a chain of short dependent steps (velocity sums, Newton solves of
// the discrete Maxwellian); the kernel is built to shorten that chain:
//   - a velocity sum: per-thread partials -> warp butterfly -> block -> one thread per
//     (value, CTA rank) reads the partial through distributed shared memory and a shuffle
//     tree forms the total, identical in every CTA of the cluster (identical branches);
//   - a Newton iteration: the Maxwellian is separable, so warps 0, 1, 2 (and one warp per
//     step-1 weight) evaluate the factors and 1-D sums of their velocity dimension
//     concurrently; after one barrier among those warps, each of them combines the sums,
//     factorises the Jacobian (FP32: inexact Newton) and takes the same decisions itself;
//   - after the first inner update, the residual and the step-1 target come from the
//     step-2 identity (|v1|/dx + A) g + r = A M+ and separable sums, without a pass over the
//     nodes or a cluster reduction.
//
// E is the arithmetic of the elementwise work, the sums and the Newton residuals: double for
// the FP64 solver, double-float (two FP32 numbers, FP64-class accuracy, no FP64 instruction
// on the critical path) for the mixed solver, float for experiments at FP32 resolution.
#include "common.cuh"
#include "kernels.h"

namespace sgs {

constexpr int kRedMax = 10;  // values per cluster reduction

template <typename E>
struct SweepSmem {
  E vv[kMaxN];         // nodes v_i
  E vq[kMaxN];         // v_i^2
  E c1e[kMaxN];        // |v_i| / dx (step-1 weights, x part)
  E c2e[kMaxN];        // |v_i| / dy (step-1 weights, y part; 2-D)
  E den[kMaxN];        // 1 / (|v_i|/dx + nu/eps) of the current cell
  E c1A[kMaxN];        // |v_i|/dx + nu/eps of the current cell
  E ef[3][kMaxN];      // factors of the last Newton evaluation (ef[0] carries exp(alpha))
  E Eg[3][kMaxN];      // factors of M[g]
  E Ep[3][kMaxN];      // factors of the step-1 Maxwellian
  E S[3][5];           // 1-D sums of the last evaluation (unweighted)
  E S1w[5];            // dimension-1 sums with the step-1 weights |v1|/dx, same evaluation
  E S2w[5];            // dimension-2 sums with the weights |v2|/dy (2-D), same evaluation
  E Sb[2][5][5];       // Newton evaluations, double-buffered: row r = sums of evaluating warp r
  E Gs[3][6];          // per-dimension sums for the norm of M+ - M[g] (derived residual)
  E svE[5];            // step-1 target s
  E W3[4][kMaxN];      // third factor of each wall's unit Maxwellian
  E red_warp[32][kRedMax];
  E red_tote[kRedMax];
  E thE[5];            // trial theta in E
  E scal[6];           // per-visit scalars: wall densities of the sides, nu/eps
  double red_part[2][kRedMax];
  double red_tot[kRedMax];
  double thg[5], thp[5], th_try[5], dir[5];
  float fn;
  float stepf;         // exponent change of the full Newton step
  int flag;
  int ctl;             // broadcast decisions of thread 0
  int wdims;           // space dimensions of the step-1 weights (1: |v1|/dx; 2: + |v2|/dy)
  int nret;            // Newton result, for the warps that do not evaluate
};

// ---------------------------------------------------------------------------------------
// Cluster-wide sum of NV values per thread; tot (double) and sm.red_tote (E) receive the
// totals, identical in every CTA.
// ---------------------------------------------------------------------------------------
template <int NV, typename E>
__device__ inline void cluster_reduce(E (&v)[NV], double (&tot)[NV], SweepSmem<E>& sm, int& buf,
                                      cg::cluster_group& cl, int CS) {
  warp_allsum<NV, E>(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; q++) sm.red_warp[wid][q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    E t = sm.red_warp[0][threadIdx.x];
    for (int k = 1; k < nw; k++) t += sm.red_warp[k][threadIdx.x];
    sm.red_part[buf][threadIdx.x] = tod(t);
  }
  cl.sync();
  // one thread per (value q, rank r): lanes of a warp hold segments of CS consecutive ranks
  if (CS == 1) {
    if (threadIdx.x < NV) sm.red_tot[threadIdx.x] = sm.red_part[buf][threadIdx.x];
  } else {
    const int per_warp = 32 / CS;  // values per warp
    const int nwarps = (NV + per_warp - 1) / per_warp;
    if (wid < nwarps) {
      int q = wid * per_warp + lane / CS, r = lane % CS;
      double x = 0.0;
      if (q < NV) x = cl.map_shared_rank(&sm.red_part[buf][0], r)[q];
      for (int o = CS >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (q < NV && r == 0) sm.red_tot[q] = x;
    }
  }
  __syncthreads();
  if (threadIdx.x < NV) sm.red_tote[threadIdx.x] = cvt<E>(sm.red_tot[threadIdx.x]);
#pragma unroll
  for (int q = 0; q < NV; q++) tot[q] = sm.red_tot[q];
  buf ^= 1;
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// Newton for the discrete Maxwellian, executed by the whole CTA with uniform control flow.
// ---------------------------------------------------------------------------------------
// Warps 0-2: factors and 1-D sums S_d^p of dimension d at the trial theta in sm.thE.
template <typename E>
__device__ __noinline__ void eval_cta(SweepSmem<E>& sm, int N) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (wid < 3 + sm.wdims) {
    // warps 0-2: dimension d; warp 3: dimension 1 again, weighted by |v1|/dx; warp 4 (2-D):
    // dimension 2 again, weighted by |v2|/dy (step 1, eq. (24))
    const int d = wid == 3 ? 0 : (wid == 4 ? 1 : wid);
    E e = cvt<E>(0.0);
    if (lane < N) {
      E x = sm.thE[1 + d] * sm.vv[lane] - sm.thE[4] * sm.vq[lane];
      if (d == 0) x += sm.thE[0];
      e = exp_in(x);
    }
    if (wid < 3) sm.ef[d][lane] = e;
    if (wid == 3) e = e * sm.c1e[lane];
    if (wid == 4) e = e * sm.c2e[lane];
    E s[5];
    s[0] = e;
    s[1] = e * sm.vv[lane];
    s[2] = e * sm.vq[lane];
    s[3] = s[2] * sm.vv[lane];
    s[4] = s[2] * sm.vq[lane];
    warp_allsum<5, E>(s);
    if (lane < 5) {
      E t = s[0];
#pragma unroll
      for (int q = 1; q < 5; q++)
        if (lane == q) t = s[q];
      if (wid < 3)
        sm.S[d][lane] = t;
      else if (wid == 3)
        sm.S1w[lane] = t;
      else
        sm.S2w[lane] = t;
    }
  }
  __syncthreads();
}

// Moments (E) and Jacobian (FP32) of the separable Maxwellian from its three 1-D sums.
template <typename E>
__device__ inline void moments_from_sums(const E* S1, const E* S2, const E* S3, E (&mom)[5], float (&Aa)[15]) {
  E s23 = S2[0] * S3[0];
  mom[0] = S1[0] * s23;
  mom[1] = S1[1] * s23;
  mom[2] = S1[0] * (S2[1] * S3[0]);
  mom[3] = S1[0] * (S2[0] * S3[1]);
  mom[4] = S1[2] * s23 + S1[0] * (S2[2] * S3[0] + S2[0] * S3[2]);
  float f1[5], f2[5], f3[5];
#pragma unroll
  for (int p = 0; p < 5; p++) {
    f1[p] = tof(S1[p]);
    f2[p] = tof(S2[p]);
    f3[p] = tof(S3[p]);
  }
  float q11 = f1[2] * f2[0] * f3[0], q22 = f1[0] * f2[2] * f3[0], q33 = f1[0] * f2[0] * f3[2];
  float q12 = f1[1] * f2[1] * f3[0], q13 = f1[1] * f2[0] * f3[1], q23 = f1[0] * f2[1] * f3[1];
  float c1 = f1[3] * f2[0] * f3[0] + f1[1] * f2[2] * f3[0] + f1[1] * f2[0] * f3[2];
  float c2 = f1[2] * f2[1] * f3[0] + f1[0] * f2[3] * f3[0] + f1[0] * f2[1] * f3[2];
  float c3 = f1[2] * f2[0] * f3[1] + f1[0] * f2[2] * f3[1] + f1[0] * f2[0] * f3[3];
  float e4 = f1[4] * f2[0] * f3[0] + f1[0] * f2[4] * f3[0] + f1[0] * f2[0] * f3[4] +
             2.0f * (f1[2] * f2[2] * f3[0] + f1[2] * f2[0] * f3[2] + f1[0] * f2[2] * f3[2]);
  float t[15] = {f1[0] * f2[0] * f3[0], f1[1] * f2[0] * f3[0], f1[0] * f2[1] * f3[0], f1[0] * f2[0] * f3[1],
                 q11 + q22 + q33, q11, q12, q13, c1, q22, q23, c2, q33, c3, e4};
#pragma unroll
  for (int i = 0; i < 15; i++) Aa[i] = t[i];
}

// Moment k of the separable Maxwellian from its three 1-D sums, the same expression as
// moments_from_sums gives for component k.
template <typename E>
__device__ inline E moment_k(const E* S1, const E* S2, const E* S3, int k) {
  const E s23 = S2[0] * S3[0];
  if (k == 0) return S1[0] * s23;
  if (k == 1) return S1[1] * s23;
  if (k == 2) return S1[0] * (S2[1] * S3[0]);
  if (k == 3) return S1[0] * (S2[0] * S3[1]);
  return S1[2] * s23 + S1[0] * (S2[2] * S3[0] + S2[0] * S3[2]);
}

// Component k of a five-element register array (static indices only).
template <typename E>
__device__ inline E pick5(const E (&v)[5], int k) {
  E r = v[0];
#pragma unroll
  for (int q = 1; q < 5; q++)
    if (k == q) r = v[q];
  return r;
}

// Warp 0: residual F (E), Jacobian (FP32) and the scaled residual norm from the 1-D sums.
// wmode 0: plain weights w; 1: w |v1|/dx; 2: w (|v1|/dx + |v2|/dy), a sum of two separable
// terms.
template <typename E>
__device__ inline void combine(const SweepSmem<E>& sm, E w, int wmode, const E* target, E (&F)[5], float (&A)[15],
                               float& fn) {
  E mom[5];
  float Aa[15];
  moments_from_sums<E>(wmode ? sm.S1w : sm.S[0], sm.S[1], sm.S[2], mom, Aa);
  if (wmode == 2) {
    E m2[5];
    float A2[15];
    moments_from_sums<E>(sm.S[0], sm.S2w, sm.S[2], m2, A2);
#pragma unroll
    for (int i = 0; i < 5; i++) mom[i] += m2[i];
#pragma unroll
    for (int i = 0; i < 15; i++) Aa[i] += A2[i];
  }
  float amax = 0.0f;
#pragma unroll
  for (int i = 0; i < 5; i++) {
    F[i] = w * mom[i] - target[i];
    amax = fmaxf(amax, fabsf(tof(F[i])));
  }
  fn = amax / fabsf(tof(target[0]));
  float cf = tof(w);
#pragma unroll
  for (int i = 0; i < 15; i++) A[i] = cf * Aa[i];
}

// One evaluation by evaluating warp wid (warps 0-2: dimension wid, unweighted; warp 3:
// dimension 1 weighted by |v1|/dx; warp 4: dimension 2 weighted by |v2|/dy) at the trial
// theta thE: factors of warps 0-2 to sm.ef, the five 1-D sums to row wid of sm.Sb[buf].
// The same arithmetic as eval_cta.
template <typename E>
__device__ inline void eval_warp(SweepSmem<E>& sm, int N, const E (&thE)[5], int wid, int buf) {
  const int lane = threadIdx.x & 31;
  const int d = wid == 3 ? 0 : (wid == 4 ? 1 : wid);
  E e = cvt<E>(0.0);
  if (lane < N) {
    E x = thE[1 + d] * sm.vv[lane] - thE[4] * sm.vq[lane];
    if (d == 0) x += thE[0];
    e = exp_in(x);
  }
  if (wid < 3) sm.ef[d][lane] = e;
  if (wid == 3) e = e * sm.c1e[lane];
  if (wid == 4) e = e * sm.c2e[lane];
  E s[5];
  s[0] = e;
  s[1] = e * sm.vv[lane];
  s[2] = e * sm.vq[lane];
  s[3] = s[2] * sm.vv[lane];
  s[4] = s[2] * sm.vq[lane];
  warp_allsum<5, E>(s);
  if (lane < 5) {
    E t = s[0];
#pragma unroll
    for (int q = 1; q < 5; q++)
      if (lane == q) t = s[q];
    sm.Sb[buf][wid][lane] = t;
  }
}

// combine on the sums of one buffer (rows as in eval_warp).
template <typename E>
__device__ inline void combine_rows(const E (*R)[5], E w, int wmode, const E* target, E (&F)[5], float (&A)[15],
                                    float& fn) {
  E mom[5];
  float Aa[15];
  moments_from_sums<E>(wmode ? R[3] : R[0], R[1], R[2], mom, Aa);
  if (wmode == 2) {
    E m2[5];
    float A2[15];
    moments_from_sums<E>(R[0], R[4], R[2], m2, A2);
#pragma unroll
    for (int i = 0; i < 5; i++) mom[i] += m2[i];
#pragma unroll
    for (int i = 0; i < 15; i++) Aa[i] += A2[i];
  }
  float amax = 0.0f;
#pragma unroll
  for (int i = 0; i < 5; i++) {
    F[i] = w * mom[i] - target[i];
    amax = fmaxf(amax, fabsf(tof(F[i])));
  }
  fn = amax / fabsf(tof(target[0]));
  float cf = tof(w);
#pragma unroll
  for (int i = 0; i < 15; i++) A[i] = cf * Aa[i];
}

// Barrier among the evaluating warps only (hardware barrier 1; __syncthreads uses 0).
__device__ __forceinline__ void eval_bar(int nwarps) {
  asm volatile("bar.sync 1, %0;" ::"r"(nwarps * 32) : "memory");
}

// Newton from the theta in th (shared memory). With have_eval the last evaluation (sm.S,
// sm.S1w, sm.S2w, sm.ef) is already at th and is reused. On success th holds the root, the
// last evaluation is at th, and the return value is the iteration count; -1 on failure.
//
// Only the evaluating warps (3 + wdims) take part, and each of them runs the whole iteration
// itself: it evaluates its dimension into a double-buffered row of sm.Sb, meets the others
// at one barrier, and then combines the rows, factorises the Jacobian (FP32: inexact Newton)
// and takes the line-search decisions in registers. All of them read the same rows and the
// same inputs through the same instructions, so their decisions agree and they pass every
// barrier the same number of times; one barrier per evaluation replaces the CTA barriers
// and thread-0 broadcasts of a split design. The FP64 trial theta is formed on lane 0 of
// each warp and shuffled to its lanes (FP64 is scarce on this GPU).
template <typename E>
__device__ __noinline__ int newton_cta(SweepSmem<E>& sm, int N, E w, int wmode, const E* target, double* th,
                                       double L, double tol, int maxit, bool have_eval) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nev = 3 + sm.wdims;
  // Converged as well once the scaled moment residual |F|/rho is at the arithmetic's
  // resolution (double-float and FP64 evaluate F to about 1e-14; 1e-13 bounds the relative
  // error of the Maxwellian near 1e-12 or below): with the residual already
  // there, a further step could only confirm it.
  constexpr float ftol = sizeof(E) == 4 ? 0.0f : 1e-13f;
  if (wid < nev) {
    double thc[5];
#pragma unroll
    for (int k = 0; k < 5; k++) thc[k] = th[k];
    E F[5];
    float A[15], fn = 0.0f;
    int buf = 0, last = -1;  // last: buffer of the latest evaluation (-1: the canonical sums)
    if (have_eval) {
      combine<E>(sm, w, wmode, target, F, A, fn);
    } else {
      E thE[5];
#pragma unroll
      for (int k = 0; k < 5; k++) thE[k] = cvt<E>(thc[k]);
      eval_warp<E>(sm, N, thE, wid, buf);
      eval_bar(nev);
      combine_rows<E>(sm.Sb[buf], w, wmode, target, F, A, fn);
      last = buf;
      buf ^= 1;
    }
    int ret = 0;
    if (!(fn <= ftol)) {
      ret = -1;
      float fn_cur = fn;
      for (int it = 0; it < maxit; it++) {
        float y[5], Ff[5];
#pragma unroll
        for (int i = 0; i < 5; i++) Ff[i] = tof(F[i]);
        if (!chol5_solve(A, Ff, y)) break;
        // exponent change of a full step, |d alpha| + L sum |d beta| + L^2 |d gamma|
        const float Lf = (float)L;
        const float stepf = fabsf(y[0]) + Lf * (fabsf(y[1]) + fabsf(y[2]) + fabsf(y[3])) + Lf * Lf * fabsf(y[4]);
        // -D A^{-1} F, D = diag(1,1,1,1,-1)
        const double dir[5] = {-(double)y[0], -(double)y[1], -(double)y[2], -(double)y[3], (double)y[4]};
        float lam = 1.0f;
        double tt[5];
        for (int hv = 0; hv < 40; hv++) {
          E thE[5];
#pragma unroll
          for (int k = 0; k < 5; k++) {
            double t = 0.0;
            if (lane == 0) t = thc[k] + (double)lam * dir[k];
            t = __shfl_sync(0xffffffffu, t, 0);
            tt[k] = t;
            thE[k] = cvt<E>(t);
          }
          eval_warp<E>(sm, N, thE, wid, buf);
          eval_bar(nev);
          combine_rows<E>(sm.Sb[buf], w, wmode, target, F, A, fn);
          last = buf;
          buf ^= 1;
          if (fn == fn && (fn <= fn_cur || fn <= 1e-10f)) {
            fn_cur = fn;
            break;
          }
          lam *= 0.5f;
        }
        const float step = lam * stepf;
#pragma unroll
        for (int k = 0; k < 5; k++) thc[k] = tt[k];
        if (!(step == step)) break;
        if (step <= (float)tol || fn_cur <= ftol) {
          ret = it + 1;
          break;
        }
      }
    }
    // publish the result: theta, and the latest evaluation's sums as the canonical ones (its
    // factors are in sm.ef already)
    if (wid == 0 && lane < 5) {
      th[lane] = thc[lane];
      sm.thE[lane] = cvt<E>(thc[lane]);
    }
    if (last >= 0 && lane < 5) {
      const E t = sm.Sb[last][wid][lane];
      if (wid < 3)
        sm.S[wid][lane] = t;
      else if (wid == 3)
        sm.S1w[lane] = t;
      else
        sm.S2w[lane] = t;
    }
    if (wid == 0 && lane == 0) sm.nret = ret;
  }
  __syncthreads();
  return sm.nret;
}

template <typename E>
__device__ inline void copy_factors(SweepSmem<E>& sm, E (*dst)[kMaxN]) {
  if (threadIdx.x < 3 * kMaxN) {
    int d = threadIdx.x / kMaxN, i = threadIdx.x % kMaxN;
    dst[d][i] = sm.ef[d][i];
  }
  __syncthreads();
}

// M[g] of the moments in mom: warm start from th0 (if any; have_eval: the last evaluation is
// at th0), then from the continuum Maxwellian; on failure keeps th0 (status reported).
// Result in sm.thg and sm.Eg; the last evaluation is at sm.thg afterwards.
template <typename E>
__device__ __noinline__ int solve_mg(SweepSmem<E>& sm, int N, E w, const E* mom, const double* th0, bool have_eval,
                                     double L, double tol, int maxit, unsigned& status) {
  const int tid = threadIdx.x;
  double keep[5];
  if (th0) {
#pragma unroll
    for (int k = 0; k < 5; k++) keep[k] = th0[k];
  }
  __syncthreads();
  int it = -1;
  if (th0) {
    if (tid < 5) sm.thg[tid] = keep[tid];
    __syncthreads();
    it = newton_cta<E>(sm, N, w, 0, mom, sm.thg, L, tol, maxit, have_eval);
  }
  if (it < 0) {
    if (tid == 0) {
      double tg[5];
      bool ok = continuum_guess<E>(mom, tg);
      sm.ctl = ok;
      if (ok)
        for (int k = 0; k < 5; k++) sm.thg[k] = tg[k];
    }
    __syncthreads();
    if (sm.ctl) {
      it = newton_cta<E>(sm, N, w, 0, mom, sm.thg, L, tol, maxit, false);
    } else {
      status |= SGS_ST_NONPOSITIVE;
    }
  }
  if (it < 0) {
    status |= SGS_ST_NEWTON_FAIL;
    if (th0 && tid < 5) sm.thg[tid] = keep[tid];
    // no warm start and no admissible guess (non-positive moments): a fixed theta (the unit
    // Maxwellian's), so that every CTA of the cluster continues from the same data and takes
    // the same decisions
    if (!th0 && !sm.ctl && tid < 5) sm.thg[tid] = tid == 0 ? -1.5 * log(2.0 * kPi) : (tid == 4 ? 0.5 : 0.0);
    __syncthreads();
    if (tid < 5) sm.thE[tid] = cvt<E>(sm.thg[tid]);
    __syncthreads();
    eval_cta<E>(sm, N);
  }
  copy_factors<E>(sm, sm.Eg);
  return it;
}

// Relaxed step 1 (the remark after eq. (26)), for thread 0 when eq. (26) fails for the
// target sd: with a factor 1 + tau on the weighted moments of the new and the current
// Maxwellian the target becomes (tau m_w + s)/(1 + tau), m_w = sum w phi c M[g] (c the
// step-1 weight; its moments come from the separable sums of the last evaluation, which is
// M[g]'s). 1 + tau = 2, 4, 8, ...: the first target that passes eq. (26) replaces sd and
// sm.svE. Returns whether one was found.
template <typename E>
__device__ inline bool relax_target(SweepSmem<E>& sm, E w, bool two_d, double (&sd)[5]) {
  E m1[5];
  float Aa[15];
  moments_from_sums<E>(sm.S1w, sm.S[1], sm.S[2], m1, Aa);
  double mw[5];
#pragma unroll
  for (int k = 0; k < 5; k++) mw[k] = tod(w * m1[k]);
  if (two_d) {
    E m2[5];
    moments_from_sums<E>(sm.S[0], sm.S2w, sm.S[2], m2, Aa);
#pragma unroll
    for (int k = 0; k < 5; k++) mw[k] += tod(w * m2[k]);
  }
  for (double q = 2.0; q <= 1048576.0; q *= 2.0) {
    double t[5];
#pragma unroll
    for (int k = 0; k < 5; k++) t[k] = ((q - 1.0) * mw[k] + sd[k]) / q;
    if (t[0] > 0.0 && t[0] * t[4] > t[1] * t[1] + t[2] * t[2] + t[3] * t[3]) {
#pragma unroll
      for (int k = 0; k < 5; k++) {
        sd[k] = t[k];
        sm.svE[k] = cvt<E>(t[k]);
      }
      return true;
    }
  }
  return false;
}

// After a step-2 update the cell equation holds up to the Maxwellians:
//   (|v1|/dx + A) g + r = A M+   =>   R(g) = A (M+ - M[g]),   A = nu/eps,
// where M+ is the Maxwellian step 2 used (step 1's, else M[g_old]). The norm of R then comes
// from per-dimension sums of the two factorisations P (M+, sm.Ep) and Q (M[g], sm.Eg): with
// d = Q - P per dimension, Q1Q2Q3 - P1P2P3 = d1 P2 P3 + Q1 d2 P3 + Q1 Q2 d3, whose squared
// norm is a sum of products of 1-D sums (no cancellation of large terms). Likewise the
// step-1 target s = sum w phi (c (M[g] - g) - r) (eq. (26)) with c g + r = A M+ - A g is
//   s = sum w phi c M[g] - A sum w phi M+ + A sum w phi g,
// from the separable sums of the last evaluation (M[g]'s), the moments of M+ and those of
// g. No pass over the nodes and no cluster reduction. Warps 0-2 form the sums; the caller's
// thread 0 takes the decisions. Returns the squared norm sum_k (M+ - M[g])^2 in thread 0.
template <typename E>
__device__ inline void derived_sums(SweepSmem<E>& sm) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (wid < 3) {
    const E p = sm.Ep[wid][lane], q = sm.Eg[wid][lane], dl = q - p;
    E x[6] = {p * p, p * dl, dl * dl, p * q, dl * q, q * q};
    warp_allsum<6, E>(x);
    if (lane < 6) {
      E t = x[0];
#pragma unroll
      for (int k = 1; k < 6; k++)
        if (lane == k) t = x[k];
      sm.Gs[wid][lane] = t;
    }
  }
  __syncthreads();
}

template <typename E>
__device__ inline E derived_norm2(const SweepSmem<E>& sm) {
  // columns of Gs: 0 PP, 1 Pd, 2 dd, 3 PQ, 4 dQ, 5 QQ
  const E* a = sm.Gs[0];
  const E* b = sm.Gs[1];
  const E* c = sm.Gs[2];
  E cross = a[4] * b[1] * c[0] + a[4] * b[3] * c[1] + a[5] * b[4] * c[1];
  return a[2] * b[0] * c[0] + a[5] * b[2] * c[0] + a[5] * b[5] * c[2] + cvt<E>(2.0) * cross;
}

template <typename E, int EPT>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int q = blockIdx.x / CS;
  if (q >= a.n_inst) return;  // whole cluster, uniformly
  if (a.active && !a.active[q]) return;
  const InstDev& I = a.inst[q];
  __shared__ SweepSmem<E> sm;
  const int N = a.N, K = N * N * N;
  const double dv = a.dv, wd = a.dv * a.dv * a.dv;
  const E w = cvt<E>(wd);
  const int J = I.J;
  const double inv_dx = 1.0 / I.dx;
  const double L = node(N - 1, N, dv);
  const int tid = threadIdx.x;
  const bool pfp = I.inner_method == SGS_PFP || I.inner_method == SGS_PFP_RELAX;
  const bool relax = I.inner_method == SGS_PFP_RELAX;
  const bool lowp = sizeof(E) == 4;  // plain FP32: tolerances at FP32 resolution
  const double ntol = lowp ? fmax(I.newton_tol, 1e-5) : I.newton_tol;
  const E inv_eps = cvt<E>(1.0 / I.eps);
  const E zero = cvt<E>(0.0);
  if (tid < kMaxN) {
    double v = tid < N ? node(tid, N, dv) : 0.0;
    sm.vv[tid] = cvt<E>(v);
    sm.vq[tid] = cvt<E>(v * v);
    sm.c1e[tid] = cvt<E>(fabs(v) * inv_dx);
    sm.c2e[tid] = zero;
    sm.W3[0][tid] = cvt<E>(tid < N ? I.wall[0][2][tid] : 0.0);
    sm.W3[1][tid] = cvt<E>(tid < N ? I.wall[1][2][tid] : 0.0);
  }
  if (tid == 0) sm.wdims = 1;
  __syncthreads();

  // this thread's nodes: pencil (i1, i2), i3 in [i30, i30 + EPT)
  const int tg = rank * blockDim.x + tid;
  const int e0 = tg * EPT;
  const bool own = e0 < K;
  const int pen = own ? e0 / N : 0, i30 = own ? e0 % N : 0;
  const int i1 = pen / N, i2 = pen % N;
  const double v1d = node(i1, N, dv);
  const E v1 = sm.vv[i1], v2 = sm.vv[i2];
  const E c1 = sm.c1e[i1];
  const E vpd = cvt<E>(fmax(v1d, 0.0) * inv_dx), vmd = cvt<E>(fmin(v1d, 0.0) * inv_dx);
  const E vq12 = sm.vq[i1] + sm.vq[i2];
  const E wl12 = cvt<E>(I.wall[0][0][i1] * I.wall[0][1][i2]);
  const E wr12 = cvt<E>(I.wall[1][0][i1] * I.wall[1][1][i2]);

  E g[EPT], r[EPT];
  int buf = 0;
  unsigned long long c_inner = 0, c_newton = 0, c_solves = 0, c_fallback = 0;
  unsigned int status = 0;

  const int s_end = min(a.s1, J);
  for (int s = a.s0; s < s_end; s++) {
    const int j = a.dir > 0 ? s : J - 1 - s;
    const long long cbase = I.f_off + (long long)j * K + e0;
    double* fj = a.f + cbase;
    const bool lw = j == 0, rw = j == J - 1;

    // ---- r = (-v1^+ f_{j-1} + v1^- f_{j+1}) / dx - P_j / eps - b_j (neighbours: latest values);
    //      a wall cell needs the wall density from reduction 1, every other cell forms r
    //      before it, so that its loads and conversions overlap the reduction
    auto form_r = [&](E rho_l, E rho_r) {
      const double* Pj = a.P + cbase;
      const double* bj = a.rhs ? a.rhs + cbase : nullptr;
#pragma unroll
      for (int t = 0; t < EPT; t++) {
        E left = lw ? rho_l * wl12 * sm.W3[0][i30 + t] : cvt<E>(fj[t - K]);
        E right = rw ? rho_r * wr12 * sm.W3[1][i30 + t] : cvt<E>(fj[t + K]);
        E rv = vmd * right - vpd * left - cvt<E>(Pj[t]) * inv_eps;
        if (bj) rv -= cvt<E>(bj[t]);
        r[t] = rv;
      }
    };
    const bool wall_cell = lw || rw;
    if (own && !wall_cell) form_r(zero, zero);
    // the cell's transport-plus-penalty coefficients (from its collision frequency), also
    // ahead of the reduction (read after its barriers)
    if (tid < N) {
      const double Ad = a.nu[I.cell0 + j] / I.eps;
      double c = fabs(node(tid, N, dv)) * inv_dx + Ad;
      sm.c1A[tid] = cvt<E>(c);
      sm.den[tid] = cvt<E>(1.0 / c);
      if (tid == 0) sm.scal[2] = cvt<E>(Ad);
    }

    // ---- reduction 1: moments of the stored value and the walls' outgoing fluxes
    E a0 = zero, a3 = zero, a4 = zero;
    if (own) {
#pragma unroll
      for (int t = 0; t < EPT; t++) {
        E x = cvt<E>(fj[t]);
        g[t] = x;
        a0 += x;
        a3 += x * sm.vv[i30 + t];
        a4 += x * sm.vq[i30 + t];
      }
    }
    E m7[7] = {a0, v1 * a0, v2 * a0, a3, vq12 * a0 + a4, (lw && v1d < 0.0) ? v1 * a0 : zero,
               (rw && v1d > 0.0) ? v1 * a0 : zero};
    double t7[7];
    cluster_reduce<7, E>(m7, t7, sm, buf, cl, CS);
    E mom[5];
#pragma unroll
    for (int k = 0; k < 5; k++) mom[k] = w * sm.red_tote[k];
    if (tid == 0) {
      sm.scal[0] = cvt<E>(I.bc_kind[0] == SGS_INFLOW ? I.bc_rho[0] : -(wd * t7[5]) / I.wall_denom[0]);
      sm.scal[1] = cvt<E>(I.bc_kind[1] == SGS_INFLOW ? I.bc_rho[1] : -(wd * t7[6]) / I.wall_denom[1]);
    }
    __syncthreads();
    const E rho_l = sm.scal[0], rho_r = sm.scal[1], Acoef = sm.scal[2];
    const E c1A = sm.c1A[i1], den = sm.den[i1];
    if (own && wall_cell) form_r(rho_l, rho_r);

    // ---- M[g] of the stored value, from the collision step's Maxwellian of the same f (the
    //      collision step that preceded this scan, or this group's, evaluated the stored
    //      value: the Newton solve only confirms it); a stale start costs iterations, not
    //      accuracy (the root is unique)
    {
      double th0[5];
#pragma unroll
      for (int k = 0; k < 5; k++) th0[k] = a.theta[5 * (long long)(I.cell0 + j) + k];
      int n0 = solve_mg<E>(sm, N, w, mom, th0, false, L, ntol, I.newton_max, status);
      if (n0 > 0) c_newton += n0;
      c_solves++;
    }

    int it = 0;
    // decisions from the step-2 identity (double-float and FP64 scans) after the first update
    bool derived = false;
    E momg[5];  // moments of the current iterate g
#pragma unroll
    for (int k = 0; k < 5; k++) momg[k] = mom[k];
    for (;;) {
      if (!derived) {
        // ---- pass B: cell-equation residual, its scale, and the step-1 target s (eq. (26))
        E e12 = sm.Eg[0][i1] * sm.Eg[1][i2];
        E rs = zero, sc = zero, b0 = zero, b3 = zero, b4 = zero;
        if (own) {
#pragma unroll
          for (int t = 0; t < EPT; t++) {
            E M = e12 * sm.Eg[2][i30 + t];
            // (|v1|/dx) g + r - (nu/eps)(M - g) = (|v1|/dx + nu/eps) g + r - (nu/eps) M
            E res = c1A * g[t] + r[t] - Acoef * M;
            rs += res * res;
            E mag = c1A * g[t];
            sc += mag * mag;
            E tt = c1 * (M - g[t]) - r[t];
            b0 += tt;
            b3 += tt * sm.vv[i30 + t];
            b4 += tt * sm.vq[i30 + t];
          }
        }
        E v7[7] = {rs, b0, v1 * b0, v2 * b0, b3, vq12 * b0 + b4, sc};
        double t6[7];
        cluster_reduce<7, E>(v7, t6, sm, buf, cl, CS);
        // thread 0 decides: stop, and whether step 1 is attempted (existence test, eq. (26))
        if (tid == 0) {
          const double res = sqrt(wd * t6[0]);
          double tol = I.inner_tol;
          if (lowp) tol = fmax(tol, 2e-6 * sqrt(wd * t6[6]));
          bool stop;
          if (I.inner_fixed > 0) {
            stop = it >= I.inner_fixed;
          } else {
            stop = res < tol || it >= I.inner_max;
            if (stop && !(res < tol)) status |= SGS_ST_INNER_CAP;
          }
          if (!(res == res)) {
            status |= SGS_ST_NONFINITE;
            stop = true;
          }
          double sd[5] = {wd * t6[1], wd * t6[2], wd * t6[3], wd * t6[4], wd * t6[5]};
#pragma unroll
          for (int k = 0; k < 5; k++) sm.svE[k] = w * sm.red_tote[1 + k];
          bool exists = pfp && sd[0] > 0.0 && sd[0] * sd[4] > sd[1] * sd[1] + sd[2] * sd[2] + sd[3] * sd[3];
          if (pfp && !exists && relax) exists = relax_target<E>(sm, w, false, sd);
          sm.ctl = (stop ? 1 : 0) | (exists ? 2 : 0);
        }
        __syncthreads();
      }
      const int ctl = sm.ctl;
      if (ctl & 1) break;

      // ---- step 1 (eq. (24)) from M[g]; else the plain fixed-point step (eq. (22))
      bool used = false;
      if (pfp) {
        if (ctl & 2) {
          E sv[5];
#pragma unroll
          for (int k = 0; k < 5; k++) sv[k] = sm.svE[k];
          if (tid < 5) sm.thp[tid] = sm.thg[tid];
          __syncthreads();
          // the last evaluation is M[g]'s: reused as the first one of step 1
          int n1 = newton_cta<E>(sm, N, w, 1, sv, sm.thp, L, ntol, I.newton_max, true);
          c_solves++;
          if (n1 >= 0) {
            c_newton += n1;
            used = true;
            copy_factors<E>(sm, sm.Ep);
          }
        }
        if (!used) c_fallback++;
      }
      const bool eval_at_start = used || !(ctl & 2);  // last evaluation at the warm start below
      E (*Eu)[kMaxN] = used ? sm.Ep : sm.Eg;
      // moments of M+: step 1's last evaluation is at M+; M[g] has the moments of g
      E momP[5];
      if (!lowp) {
        if (used) {
          float Aa[15];
          moments_from_sums<E>(sm.S[0], sm.S[1], sm.S[2], momP, Aa);
#pragma unroll
          for (int k = 0; k < 5; k++) momP[k] = w * momP[k];
        } else {
#pragma unroll
          for (int k = 0; k < 5; k++) momP[k] = momg[k];
        }
      }

      // ---- step 2 (eq. (25)) and the moments of the new iterate
      E ep = Eu[0][i1] * Eu[1][i2];
      E c0 = zero, c3 = zero, c4 = zero;
      if (own) {
#pragma unroll
        for (int t = 0; t < EPT; t++) {
          E x = (Acoef * (ep * Eu[2][i30 + t]) - r[t]) * den;
          g[t] = x;
          c0 += x;
          c3 += x * sm.vv[i30 + t];
          c4 += x * sm.vq[i30 + t];
        }
      }
      // keep the factors of M+ in sm.Ep (the reduction below orders this before solve_mg)
      if (!lowp && !used && tid < 3 * kMaxN) sm.Ep[tid / kMaxN][tid % kMaxN] = sm.Eg[tid / kMaxN][tid % kMaxN];
      E m5[5] = {c0, v1 * c0, v2 * c0, c3, vq12 * c0 + c4};
      double t5[5];
      cluster_reduce<5, E>(m5, t5, sm, buf, cl, CS);
      it++;
      E mm[5];
#pragma unroll
      for (int k = 0; k < 5; k++) mm[k] = w * sm.red_tote[k];
      // warm start: the step-1 Maxwellian approximates M of the updated iterate
      int n2 = solve_mg<E>(sm, N, w, mm, used ? sm.thp : sm.thg, eval_at_start, L, ntol, I.newton_max, status);
      if (n2 > 0) c_newton += n2;
      c_solves++;
      if (!lowp) {
        // ---- residual and step-1 target of the new iterate from the step-2 identity
        derived_sums<E>(sm);
        // warp 0 decides; its lanes form the five components of the step-1 target and the
        // residual norm concurrently (a serial chain of double-float operations otherwise)
        if (tid < 32) {
          const int lane = tid;
          E sk = zero;
          if (lane < 5) {
            const E mwk = moment_k<E>(sm.S1w, sm.S[1], sm.S[2], lane);  // sum phi (|v1|/dx) M[g]
            sk = w * mwk - Acoef * pick5<E>(momP, lane) + Acoef * pick5<E>(mm, lane);
            sm.svE[lane] = sk;
          }
          const double sdk = tod(sk);
          double nrm = lane == 5 ? tod(derived_norm2<E>(sm)) : 0.0;
          double sd[5];
#pragma unroll
          for (int k = 0; k < 5; k++) sd[k] = __shfl_sync(0xffffffffu, sdk, k);
          nrm = __shfl_sync(0xffffffffu, nrm, 5);
          __syncwarp();  // the lanes' sm.svE before lane 0 may replace them (relaxed step 1)
          if (lane == 0) {
            const double Ad = tod(Acoef);
            const double res = fabs(Ad) * sqrt(wd * nrm);
            bool stop;
            if (I.inner_fixed > 0) {
              stop = it >= I.inner_fixed;
            } else {
              stop = res < I.inner_tol || it >= I.inner_max;
              if (stop && !(res < I.inner_tol)) status |= SGS_ST_INNER_CAP;
            }
            if (!(res == res)) {
              status |= SGS_ST_NONFINITE;
              stop = true;
            }
            bool exists = pfp && sd[0] > 0.0 && sd[0] * sd[4] > sd[1] * sd[1] + sd[2] * sd[2] + sd[3] * sd[3];
            if (pfp && !exists && relax) exists = relax_target<E>(sm, w, false, sd);
            sm.ctl = (stop ? 1 : 0) | (exists ? 2 : 0);
          }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 5; k++) momg[k] = mm[k];
        derived = true;
      }
    }

    if (own) {
#pragma unroll
      for (int t = 0; t < EPT; t++) fj[t] = tod(g[t]);
    }
    c_inner += it;
    // the next visit's first reduction is a cluster barrier: every CTA has finished this
    // cell before any reads of the next one's neighbours (each thread reads only its own
    // nodes, so no cross-thread ordering is needed beyond program order)
  }
  // no CTA leaves while another may still read its shared memory (the last reduction's
  // distributed-shared-memory loads)
  cl.sync();

  if (rank == 0 && tid == 0) {
    Counters* c = a.cnt + q;
    atomicAdd(&c->visits, (unsigned long long)max(0, s_end - a.s0));
    atomicAdd(&c->inner_iters, c_inner);
    atomicAdd(&c->newton_iters, c_newton);
    atomicAdd(&c->newton_solves, c_solves);
    atomicAdd(&c->fallbacks, c_fallback);
  }
  if (tid == 0 && status) atomicOr(&a.cnt[q].status, status);
}

// ---------------------------------------------------------------------------------------
// 2-D space: one sweep ordering is a sequence of anti-diagonal wavefronts. Cells on one
// wavefront depend only on the previous wavefront (their upwind x and y neighbours) and on
// not-yet-visited cells (downwind), so the cells of a wavefront are visited concurrently,
// one thread-block cluster per cell, one launch per wavefront (the launch boundary orders
// the wavefronts). The visit is the 1-D visit with the transport weight
// c = |v1|/dx + |v2|/dy, four neighbours (or wall ghosts) and step-1 weights w c, whose
// Newton sums are two separable terms. The M[g] solve of the stored value starts from the
// Maxwellian of the collision step that preceded the sweep (same f, so it is converged).
// Ordering o: 0 SW->NE, 1 NE->SW, 2 NW->SE, 3 SE->NW; wavefront index wf counts from the
// ordering's starting corner.
// ---------------------------------------------------------------------------------------
template <typename E, int EPT>
__global__ void __launch_bounds__(256) k_sweep2d(SweepArgs a, int ordering, int wf) {
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const InstDev& I = a.inst[0];
  const int nx = I.nx, ny = I.ny;
  const int amin = max(0, wf - (ny - 1)), amax = min(nx - 1, wf);
  const int ak = amin + (int)(blockIdx.x / CS);
  if (ak > amax) return;  // whole cluster, uniformly
  if (a.active && !a.active[0]) return;
  const int dirx = (ordering == 0 || ordering == 2) ? 1 : -1;
  const int diry = (ordering == 0 || ordering == 3) ? 1 : -1;
  const int ci = dirx > 0 ? ak : nx - 1 - ak;
  const int bk = wf - ak;
  const int cj = diry > 0 ? bk : ny - 1 - bk;
  const int cell = cj * nx + ci;

  __shared__ SweepSmem<E> sm;
  const int N = a.N, K = N * N * N;
  const double dv = a.dv, wd = a.dv * a.dv * a.dv;
  const E w = cvt<E>(wd);
  const double inv_dx = 1.0 / I.dx, inv_dy = 1.0 / I.dy;
  const double L = node(N - 1, N, dv);
  const int tid = threadIdx.x;
  const bool pfp = I.inner_method == SGS_PFP || I.inner_method == SGS_PFP_RELAX;
  const bool relax = I.inner_method == SGS_PFP_RELAX;
  const bool lowp = sizeof(E) == 4;
  const double ntol = lowp ? fmax(I.newton_tol, 1e-5) : I.newton_tol;
  const E inv_eps = cvt<E>(1.0 / I.eps);
  const E zero = cvt<E>(0.0);
  if (tid < kMaxN) {
    double v = tid < N ? node(tid, N, dv) : 0.0;
    sm.vv[tid] = cvt<E>(v);
    sm.vq[tid] = cvt<E>(v * v);
    sm.c1e[tid] = cvt<E>(fabs(v) * inv_dx);
    sm.c2e[tid] = cvt<E>(fabs(v) * inv_dy);
#pragma unroll
    for (int sd = 0; sd < 4; sd++) sm.W3[sd][tid] = cvt<E>(tid < N ? I.wall[sd][2][tid] : 0.0);
  }
  if (tid == 0) sm.wdims = 2;
  __syncthreads();

  // this thread's nodes: pencil (i1, i2), i3 in [i30, i30 + EPT)
  const int tg = rank * blockDim.x + tid;
  const int e0 = tg * EPT;
  const bool own = e0 < K;
  const int pen = own ? e0 / N : 0, i30 = own ? e0 % N : 0;
  const int i1 = pen / N, i2 = pen % N;
  const double v1d = node(i1, N, dv), v2d = node(i2, N, dv);
  const E v1 = sm.vv[i1], v2 = sm.vv[i2];
  const E cw = sm.c1e[i1] + sm.c2e[i2];  // transport weight |v1|/dx + |v2|/dy
  const E v1p = cvt<E>(fmax(v1d, 0.0) * inv_dx), v1m = cvt<E>(fmin(v1d, 0.0) * inv_dx);
  const E v2p = cvt<E>(fmax(v2d, 0.0) * inv_dy), v2m = cvt<E>(fmin(v2d, 0.0) * inv_dy);
  const E vq12 = sm.vq[i1] + sm.vq[i2];
  E w12[4];
#pragma unroll
  for (int sd = 0; sd < 4; sd++) w12[sd] = cvt<E>(I.wall[sd][0][i1] * I.wall[sd][1][i2]);
  const bool bnd[4] = {ci == 0, ci == nx - 1, cj == 0, cj == ny - 1};

  E g[EPT], r[EPT];
  int buf = 0;
  unsigned long long c_newton = 0, c_solves = 0, c_fallback = 0;
  unsigned int status = 0;
  const long long cbase = I.f_off + (long long)cell * K + e0;
  double* fj = a.f + cbase;
  const int gcell = I.cell0 + cell;

  // ---- reduction 1: moments of the stored value and its outgoing fluxes through wall faces
  E a0 = zero, a3 = zero, a4 = zero;
  if (own) {
#pragma unroll
    for (int t = 0; t < EPT; t++) {
      E x = cvt<E>(fj[t]);
      g[t] = x;
      a0 += x;
      a3 += x * sm.vv[i30 + t];
      a4 += x * sm.vq[i30 + t];
    }
  }
  E m9[9] = {a0,
             v1 * a0,
             v2 * a0,
             a3,
             vq12 * a0 + a4,
             (bnd[0] && v1d < 0.0) ? v1 * a0 : zero,
             (bnd[1] && v1d > 0.0) ? v1 * a0 : zero,
             (bnd[2] && v2d < 0.0) ? v2 * a0 : zero,
             (bnd[3] && v2d > 0.0) ? v2 * a0 : zero};
  double t9[9];
  cluster_reduce<9, E>(m9, t9, sm, buf, cl, CS);
  E mom[5];
#pragma unroll
  for (int k = 0; k < 5; k++) mom[k] = w * sm.red_tote[k];
  const double Ad = a.nu[gcell] / I.eps;
  if (tid < 4) {
    const int sd = tid;
    sm.scal[sd] = cvt<E>(I.bc_kind[sd] == SGS_INFLOW ? I.bc_rho[sd] : -(wd * t9[5 + sd]) / I.wall_denom[sd]);
  }
  if (tid == 4) sm.scal[4] = cvt<E>(Ad);
  __syncthreads();
  const E Acoef = sm.scal[4];
  const double cAd = fabs(v1d) * inv_dx + fabs(v2d) * inv_dy + Ad;
  const E cA = cvt<E>(cAd), den = cvt<E>(1.0 / cAd);

  // ---- r = (-v1^+ f_W + v1^- f_E)/dx + (-v2^+ f_S + v2^- f_N)/dy - P/eps - b (latest values)
  if (own) {
    const double* Pj = a.P + cbase;
    const double* bj = a.rhs ? a.rhs + cbase : nullptr;
#pragma unroll
    for (int t = 0; t < EPT; t++) {
      const int i3 = i30 + t;
      E fw = bnd[0] ? sm.scal[0] * w12[0] * sm.W3[0][i3] : cvt<E>(fj[t - K]);
      E fe = bnd[1] ? sm.scal[1] * w12[1] * sm.W3[1][i3] : cvt<E>(fj[t + K]);
      E fs = bnd[2] ? sm.scal[2] * w12[2] * sm.W3[2][i3] : cvt<E>(fj[t - (long long)nx * K]);
      E fn = bnd[3] ? sm.scal[3] * w12[3] * sm.W3[3][i3] : cvt<E>(fj[t + (long long)nx * K]);
      E rv = v1m * fe - v1p * fw + v2m * fn - v2p * fs - cvt<E>(Pj[t]) * inv_eps;
      if (bj) rv -= cvt<E>(bj[t]);
      r[t] = rv;
    }
  }

  // ---- M[g] of the stored value, from the collision step's Maxwellian of the same f
  {
    double th0[5];
#pragma unroll
    for (int k = 0; k < 5; k++) th0[k] = a.theta[5 * (long long)gcell + k];
    int n0 = solve_mg<E>(sm, N, w, mom, th0, false, L, ntol, I.newton_max, status);
    if (n0 > 0) c_newton += n0;
    c_solves++;
  }

  int it = 0;
  // decisions from the step-2 identity (double-float and FP64 scans) after the first update
  bool derived = false;
  E momg[5];  // moments of the current iterate g
#pragma unroll
  for (int k = 0; k < 5; k++) momg[k] = mom[k];
  for (;;) {
    if (!derived) {
      // ---- pass B: cell-equation residual, its scale, and the step-1 target s (eq. (26))
      E e12 = sm.Eg[0][i1] * sm.Eg[1][i2];
      E rs = zero, sc = zero, b0 = zero, b3 = zero, b4 = zero;
      if (own) {
#pragma unroll
        for (int t = 0; t < EPT; t++) {
          E M = e12 * sm.Eg[2][i30 + t];
          E res = cA * g[t] + r[t] - Acoef * M;
          rs += res * res;
          E mag = cA * g[t];
          sc += mag * mag;
          E tt = cw * (M - g[t]) - r[t];
          b0 += tt;
          b3 += tt * sm.vv[i30 + t];
          b4 += tt * sm.vq[i30 + t];
        }
      }
      E v7[7] = {rs, b0, v1 * b0, v2 * b0, b3, vq12 * b0 + b4, sc};
      double t6[7];
      cluster_reduce<7, E>(v7, t6, sm, buf, cl, CS);
      if (tid == 0) {
        const double res = sqrt(wd * t6[0]);
        double tol = I.inner_tol;
        if (lowp) tol = fmax(tol, 2e-6 * sqrt(wd * t6[6]));
        bool stop;
        if (I.inner_fixed > 0) {
          stop = it >= I.inner_fixed;
        } else {
          stop = res < tol || it >= I.inner_max;
          if (stop && !(res < tol)) status |= SGS_ST_INNER_CAP;
        }
        if (!(res == res)) {
          status |= SGS_ST_NONFINITE;
          stop = true;
        }
        double sd[5] = {wd * t6[1], wd * t6[2], wd * t6[3], wd * t6[4], wd * t6[5]};
#pragma unroll
        for (int k = 0; k < 5; k++) sm.svE[k] = w * sm.red_tote[1 + k];
        bool exists = pfp && sd[0] > 0.0 && sd[0] * sd[4] > sd[1] * sd[1] + sd[2] * sd[2] + sd[3] * sd[3];
        if (pfp && !exists && relax) exists = relax_target<E>(sm, w, true, sd);
        sm.ctl = (stop ? 1 : 0) | (exists ? 2 : 0);
      }
      __syncthreads();
    }
    const int ctl = sm.ctl;
    if (ctl & 1) break;

    // ---- step 1 (eq. (24)) with the 2-D weights; else the plain fixed-point step (eq. (22))
    bool used = false;
    if (pfp) {
      if (ctl & 2) {
        E sv[5];
#pragma unroll
        for (int k = 0; k < 5; k++) sv[k] = sm.svE[k];
        if (tid < 5) sm.thp[tid] = sm.thg[tid];
        __syncthreads();
        int n1 = newton_cta<E>(sm, N, w, 2, sv, sm.thp, L, ntol, I.newton_max, true);
        c_solves++;
        if (n1 >= 0) {
          c_newton += n1;
          used = true;
          copy_factors<E>(sm, sm.Ep);
        }
      }
      if (!used) c_fallback++;
    }
    const bool eval_at_start = used || !(ctl & 2);
    E (*Eu)[kMaxN] = used ? sm.Ep : sm.Eg;
    // moments of M+: step 1's last evaluation is at M+; M[g] has the moments of g
    E momP[5];
    if (!lowp) {
      if (used) {
        float Aa[15];
        moments_from_sums<E>(sm.S[0], sm.S[1], sm.S[2], momP, Aa);
#pragma unroll
        for (int k = 0; k < 5; k++) momP[k] = w * momP[k];
      } else {
#pragma unroll
        for (int k = 0; k < 5; k++) momP[k] = momg[k];
      }
    }

    // ---- step 2 (eq. (25)) and the moments of the new iterate
    E ep = Eu[0][i1] * Eu[1][i2];
    E c0 = zero, c3 = zero, c4 = zero;
    if (own) {
#pragma unroll
      for (int t = 0; t < EPT; t++) {
        E x = (Acoef * (ep * Eu[2][i30 + t]) - r[t]) * den;
        g[t] = x;
        c0 += x;
        c3 += x * sm.vv[i30 + t];
        c4 += x * sm.vq[i30 + t];
      }
    }
    // keep the factors of M+ in sm.Ep (the reduction below orders this before solve_mg)
    if (!lowp && !used && tid < 3 * kMaxN) sm.Ep[tid / kMaxN][tid % kMaxN] = sm.Eg[tid / kMaxN][tid % kMaxN];
    E m5[5] = {c0, v1 * c0, v2 * c0, c3, vq12 * c0 + c4};
    double t5[5];
    cluster_reduce<5, E>(m5, t5, sm, buf, cl, CS);
    it++;
    E mm[5];
#pragma unroll
    for (int k = 0; k < 5; k++) mm[k] = w * sm.red_tote[k];
    int n2 = solve_mg<E>(sm, N, w, mm, used ? sm.thp : sm.thg, eval_at_start, L, ntol, I.newton_max, status);
    if (n2 > 0) c_newton += n2;
    c_solves++;
    if (!lowp) {
      // ---- residual and step-1 target of the new iterate from the step-2 identity (the
      //      step-1 weight |v1|/dx + |v2|/dy is a sum of two separable terms)
      derived_sums<E>(sm);
      if (tid == 0) {
        E mw[5], mw2[5];
        float Aa[15];
        moments_from_sums<E>(sm.S1w, sm.S[1], sm.S[2], mw, Aa);
        moments_from_sums<E>(sm.S[0], sm.S2w, sm.S[2], mw2, Aa);
        const double Ad = tod(Acoef);
        const double res = fabs(Ad) * sqrt(wd * tod(derived_norm2<E>(sm)));
        bool stop;
        if (I.inner_fixed > 0) {
          stop = it >= I.inner_fixed;
        } else {
          stop = res < I.inner_tol || it >= I.inner_max;
          if (stop && !(res < I.inner_tol)) status |= SGS_ST_INNER_CAP;
        }
        if (!(res == res)) {
          status |= SGS_ST_NONFINITE;
          stop = true;
        }
        double sd[5];
#pragma unroll
        for (int k = 0; k < 5; k++) {
          E sk = w * (mw[k] + mw2[k]) - Acoef * momP[k] + Acoef * mm[k];
          sm.svE[k] = sk;
          sd[k] = tod(sk);
        }
        bool exists = pfp && sd[0] > 0.0 && sd[0] * sd[4] > sd[1] * sd[1] + sd[2] * sd[2] + sd[3] * sd[3];
        if (pfp && !exists && relax) exists = relax_target<E>(sm, w, true, sd);
        sm.ctl = (stop ? 1 : 0) | (exists ? 2 : 0);
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 5; k++) momg[k] = mm[k];
      derived = true;
    }
  }

  if (own) {
#pragma unroll
    for (int t = 0; t < EPT; t++) fj[t] = tod(g[t]);
  }
  cl.sync();  // the last reduction's remote loads are done before any CTA leaves
  if (rank == 0 && tid == 0) {
    Counters* c = a.cnt;
    atomicAdd(&c->visits, 1ULL);
    atomicAdd(&c->inner_iters, (unsigned long long)it);
    atomicAdd(&c->newton_iters, c_newton);
    atomicAdd(&c->newton_solves, c_solves);
    atomicAdd(&c->fallbacks, c_fallback);
  }
  if (tid == 0 && status) atomicOr(&a.cnt[0].status, status);
}

// Default launch shape: nodes per thread (a divisor of N), cluster size (a power of two, at
// most 16) and threads per CTA (a multiple of 32 in [160, 256]; warps 0-4 serve the Newton
// evaluations).
SweepShape sweep_shape(int N, int arith) {
  SweepShape s;
  int K = N * N * N;
  s.ept = arith == kSweepF32 ? N : (N <= 8 ? 2 : (N % 8 == 0 ? 8 : 4));
  int threads = K / s.ept;
  s.cluster = 1;
  while (s.cluster < 16 && s.cluster * 256 < threads) s.cluster *= 2;
  s.tpb = ((threads + s.cluster - 1) / s.cluster + 31) / 32 * 32;
  if (s.tpb < 160) s.tpb = 160;
  return s;
}

// ---------------------------------------------------------------------------------------
// Latency probe of the scan's two serial building blocks in one cluster of a given launch
// shape: mode 0 runs `reps` cluster reductions of seven values (cluster_reduce, as in every
// cell visit); mode 1 runs `reps` dependent Newton iterations of the discrete Maxwellian by
// the evaluating warps (factors and 1-D sums of each velocity dimension, the barrier among
// those warps, the combination into moments and Jacobian, the 5x5 factorisation and solve).
// The results feed a runtime test that never passes (the sentinel), so nothing is stored
// and nothing allocated.
// ---------------------------------------------------------------------------------------
__device__ double g_probe_sink;

template <typename E>
__global__ void __launch_bounds__(256) k_probe_scan(int N, double dv, int mode, int reps, double sentinel) {
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  __shared__ SweepSmem<E> sm;
  const int tid = threadIdx.x;
  if (tid < kMaxN) {
    double v = tid < N ? node(tid, N, dv) : 0.0;
    sm.vv[tid] = cvt<E>(v);
    sm.vq[tid] = cvt<E>(v * v);
    sm.c1e[tid] = cvt<E>(fabs(v));
    sm.c2e[tid] = cvt<E>(0.0);
  }
  if (tid == 0) sm.wdims = 1;
  __syncthreads();
  double acc = 0.0;
  if (mode == 0) {
    // inputs formed once (FP64 is scarce: forming them per repetition would time FP64
    // conversions, not the reduction); each repetition reduces a fresh copy
    int buf = 0;
    E v0[7];
#pragma unroll
    for (int q = 0; q < 7; q++) v0[q] = cvt<E>(1e-3 * (double)(tid + q));
    E accE = cvt<E>(0.0);
    for (int r = 0; r < reps; r++) {
      E v[7];
#pragma unroll
      for (int q = 0; q < 7; q++) v[q] = v0[q];
      double t[7];
      cluster_reduce<7, E>(v, t, sm, buf, cl, CS);
      accE = accE + sm.red_tote[0];
    }
    acc = tod(accE);
  } else if (mode == 2) {
    // the hardware cluster barrier alone (one of the reduction's steps)
    for (int r = 0; r < reps; r++) {
      cl.sync();
      acc += (double)(tid + r);
    }
  } else {
    const int wid = tid >> 5;
    const int nev = 3 + sm.wdims;
    if (wid < nev) {
      // unit Maxwellian exponents and its continuum moments as the target
      E thE[5] = {cvt<E>(-1.5 * log(2.0 * kPi)), cvt<E>(0.0), cvt<E>(0.0), cvt<E>(0.0), cvt<E>(0.5)};
      const E target[5] = {cvt<E>(1.0), cvt<E>(0.0), cvt<E>(0.0), cvt<E>(0.0), cvt<E>(3.0)};
      const E w = cvt<E>(dv * dv * dv);
      int buf = 0;
      float accf = 0.0f;
      for (int r = 0; r < reps; r++) {
        eval_warp<E>(sm, N, thE, wid, buf);
        eval_bar(nev);
        E F[5];
        float A[15], fn;
        combine_rows<E>(sm.Sb[buf], w, 0, target, F, A, fn);
        buf ^= 1;
        float y[5], Ff[5];
#pragma unroll
        for (int i = 0; i < 5; i++) Ff[i] = tof(F[i]);
        chol5_solve(A, Ff, y);
        accf += y[0] + fn;  // FP32: the probe times the iteration, not FP64 adds
        thE[0] = thE[0] + cvt<E>(1e-9 * (double)y[0]);  // the next evaluation depends on this one
      }
      acc = (double)accf;
    }
    __syncthreads();
  }
  cl.sync();  // the last reduction's remote loads are done before any CTA leaves
  if (acc == sentinel) g_probe_sink = acc;
}

template <typename E>
static cudaError_t launch_probe_scan(int N, double dv, int cluster, int threads, int mode, int reps,
                                     cudaStream_t st) {
  cudaError_t e = func_attr((const void*)k_probe_scan<E>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster);
  cfg.blockDim = dim3(threads);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_probe_scan<E>, N, dv, mode, reps, -1.0e300);
}

cudaError_t probe_scan(int N, double dv, int arith, int cluster, int threads, int mode, int reps, cudaStream_t st) {
  if (cluster < 1 || cluster > 16 || (cluster & (cluster - 1)) || threads < 160 || threads > 256 || threads % 32 ||
      threads < 32 * ((kRedMax * cluster + 31) / 32) || N < 8 || N > kMaxN || reps < 0)
    return cudaErrorInvalidConfiguration;
  if (arith == kSweepDF64) return launch_probe_scan<dfloat>(N, dv, cluster, threads, mode, reps, st);
  if (arith == kSweepF32) return launch_probe_scan<float>(N, dv, cluster, threads, mode, reps, st);
  return launch_probe_scan<double>(N, dv, cluster, threads, mode, reps, st);
}

template <typename E, int EPT>
static cudaError_t launch_sweep_t(const SweepArgs& a, const SweepShape& sh, cudaStream_t st) {
  cudaError_t e = func_attr((const void*)k_sweep<E, EPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.n_inst * sh.cluster);
  cfg.blockDim = dim3(sh.tpb);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = sh.cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_sweep<E, EPT>, a);
}

template <typename E, int EPT>
static cudaError_t launch_sweep2d_t(const SweepArgs& a, const SweepShape& sh, int ordering, int wf, int ncells,
                                    cudaStream_t st) {
  cudaError_t e = func_attr((const void*)k_sweep2d<E, EPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ncells * sh.cluster);
  cfg.blockDim = dim3(sh.tpb);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = sh.cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_sweep2d<E, EPT>, a, ordering, wf);
}

template <typename E>
static cudaError_t launch_sweep2d_e(const SweepArgs& a, const SweepShape& sh, int ordering, int wf, int ncells,
                                    cudaStream_t st) {
  switch (sh.ept) {
    case 2: return launch_sweep2d_t<E, 2>(a, sh, ordering, wf, ncells, st);
    case 4: return launch_sweep2d_t<E, 4>(a, sh, ordering, wf, ncells, st);
    case 8: return launch_sweep2d_t<E, 8>(a, sh, ordering, wf, ncells, st);
    case 12: return launch_sweep2d_t<E, 12>(a, sh, ordering, wf, ncells, st);
    case 16: return launch_sweep2d_t<E, 16>(a, sh, ordering, wf, ncells, st);
    case 20: return launch_sweep2d_t<E, 20>(a, sh, ordering, wf, ncells, st);
    case 24: return launch_sweep2d_t<E, 24>(a, sh, ordering, wf, ncells, st);
    case 28: return launch_sweep2d_t<E, 28>(a, sh, ordering, wf, ncells, st);
    case 32: return launch_sweep2d_t<E, 32>(a, sh, ordering, wf, ncells, st);
  }
  return cudaErrorInvalidConfiguration;
}

cudaError_t launch_sweep2d(const SweepArgs& a, const SweepShape& sh, int arith, int ordering, int wf, int ncells,
                           cudaStream_t st) {
  if (arith == kSweepF64) return launch_sweep2d_e<double>(a, sh, ordering, wf, ncells, st);
  if (arith == kSweepDF64) return launch_sweep2d_e<dfloat>(a, sh, ordering, wf, ncells, st);
  return launch_sweep2d_e<float>(a, sh, ordering, wf, ncells, st);
}

template <typename E>
static cudaError_t launch_sweep_e(const SweepArgs& a, const SweepShape& sh, cudaStream_t st) {
  switch (sh.ept) {
    case 2: return launch_sweep_t<E, 2>(a, sh, st);
    case 4: return launch_sweep_t<E, 4>(a, sh, st);
    case 8: return launch_sweep_t<E, 8>(a, sh, st);
    case 12: return launch_sweep_t<E, 12>(a, sh, st);
    case 16: return launch_sweep_t<E, 16>(a, sh, st);
    case 20: return launch_sweep_t<E, 20>(a, sh, st);
    case 24: return launch_sweep_t<E, 24>(a, sh, st);
    case 28: return launch_sweep_t<E, 28>(a, sh, st);
    case 32: return launch_sweep_t<E, 32>(a, sh, st);
  }
  return cudaErrorInvalidConfiguration;
}

template <typename E, int EPT>
static cudaError_t max_clusters_t(const SweepShape& sh, int* n) {
  cudaError_t e = func_attr((const void*)k_sweep<E, EPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sh.cluster);
  cfg.blockDim = dim3(sh.tpb);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = sh.cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(n, k_sweep<E, EPT>, &cfg);
}

template <typename E>
static cudaError_t max_clusters_e(const SweepShape& sh, int* n) {
  switch (sh.ept) {
    case 2: return max_clusters_t<E, 2>(sh, n);
    case 4: return max_clusters_t<E, 4>(sh, n);
    case 8: return max_clusters_t<E, 8>(sh, n);
    case 12: return max_clusters_t<E, 12>(sh, n);
    case 16: return max_clusters_t<E, 16>(sh, n);
    case 20: return max_clusters_t<E, 20>(sh, n);
    case 24: return max_clusters_t<E, 24>(sh, n);
    case 28: return max_clusters_t<E, 28>(sh, n);
    case 32: return max_clusters_t<E, 32>(sh, n);
  }
  return cudaErrorInvalidConfiguration;
}

bool sweep_ept_compiled(int ept) {
  return ept == 2 || ept == 4 || ept == 8 || ept == 12 || ept == 16 || ept == 20 || ept == 24 || ept == 28 ||
         ept == 32;
}

cudaError_t sweep_max_clusters(const SweepShape& sh, int arith, int* n) {
  *n = 0;
  if (arith == kSweepF64) return max_clusters_e<double>(sh, n);
  if (arith == kSweepDF64) return max_clusters_e<dfloat>(sh, n);
  return max_clusters_e<float>(sh, n);
}

bool sweep_shape_valid(int N, const SweepShape& sh) {
  int K = N * N * N;
  if (sh.ept <= 0 || N % sh.ept != 0) return false;
  if (sh.cluster < 1 || sh.cluster > 16 || (sh.cluster & (sh.cluster - 1))) return false;
  if (sh.tpb < 160 || sh.tpb > 256 || sh.tpb % 32) return false;
  if (sh.tpb < 32 * ((kRedMax * sh.cluster + 31) / 32)) return false;  // warps for the cluster gather
  if ((long long)sh.cluster * sh.tpb * sh.ept < K) return false;
  int e[] = {2, 4, 8, 12, 16, 20, 24, 28, 32};
  for (int x : e)
    if (x == sh.ept) return true;
  return false;
}

cudaError_t launch_sweep(const SweepArgs& a, const SweepShape& sh, int arith, cudaStream_t st) {
  if (!sweep_shape_valid(a.N, sh)) return cudaErrorInvalidConfiguration;
  if (arith == kSweepDF64) return launch_sweep_e<dfloat>(a, sh, st);
  if (arith == kSweepF32) return launch_sweep_e<float>(a, sh, st);
  return launch_sweep_e<double>(a, sh, st);
}

}  // namespace sgs
