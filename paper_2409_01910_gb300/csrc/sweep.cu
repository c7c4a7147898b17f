// Persistent symmetric Gauss-Seidel scan (eq. (29), first order) with the preconditioned
// fixed-point cell solve (eqs. (20), (24)-(26)).
//
// One thread-block cluster per instance walks that instance's cells in scan order inside a
// single launch. Each thread owns EPT consecutive velocity nodes of one pencil (fixed i1, i2)
// in every cell, so a thread only ever reads and writes its own nodes: the upwind neighbour's
// new value is its own earlier write, and no two threads touch the same global element.
// Every velocity sum (moments, cell-equation residual, step-1 target) is a cluster-wide
// reduction: per-thread partials -> warp butterfly -> block -> each CTA reads every CTA's
// partial through distributed shared memory in rank order, so all CTAs hold bit-identical
// totals and take identical branches. The discrete-Maxwellian Newton solves need only O(N)
// work on the tensor grid (separable Maxwellian) and run redundantly in warp 0 of every CTA,
// warm-started from the previous solution of the visit.
//
// E is the arithmetic of the elementwise work, the reductions and the Newton residuals:
// double for the FP64 solver, float for the low-precision smoother of the mixed solver (whose
// FP64 accuracy comes from the FP64 collision and residual of the defect-correction loop).
#include "common.cuh"
#include "kernels.h"

namespace sgs {

template <typename E>
struct SweepSmem {
  E vv[kMaxN];   // nodes v_i
  E vq[kMaxN];   // v_i^2
  E E1[kMaxN];   // factors of the Maxwellian in use (E1 carries exp(alpha))
  E E2[kMaxN];
  E E3[kMaxN];
  E W3[2][kMaxN];  // third factor of each wall's unit Maxwellian
  E red_warp[32][8];
  double red_part[2][8];
  double red_tot[8];
  double thg[5];  // theta of M[g]
  double thp[5];  // theta of the step-1 Maxwellian
};

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
  if (threadIdx.x < NV) {
    double t = 0.0;
    for (int r = 0; r < CS; r++) {
      const double* p = cl.map_shared_rank(&sm.red_part[buf][0], r);
      t += p[threadIdx.x];
    }
    sm.red_tot[threadIdx.x] = t;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; q++) tot[q] = sm.red_tot[q];
  buf ^= 1;
}

// Newton for the (weighted) discrete Maxwellian run by warp 0: warm start from th0 when
// given, else (or on failure) from the continuum guess. Stores the factors and theta.
template <typename E>
__device__ inline int newton_store(SweepSmem<E>& sm, int N, double dv, double w, bool wv1, double inv_dx,
                                   const E* target,
                                   const double* th0, double* th_out, double tol, int maxit, unsigned& status,
                                   bool store_on_fail) {
  const int lane = threadIdx.x & 31;
  double th[5];
  MaxwEval<E> ev;
  int it = -1;
  if (th0) {
#pragma unroll
    for (int k = 0; k < 5; k++) th[k] = th0[k];
    it = maxwellian_newton<E>(N, dv, w, wv1, inv_dx, target, th, tol, maxit, ev);
  }
  if (it < 0 && !wv1) {
    if (continuum_guess<E>(target, th)) it = maxwellian_newton<E>(N, dv, w, wv1, inv_dx, target, th, tol, maxit, ev);
    else status |= SGS_ST_NONPOSITIVE;
  }
  if (it < 0 && !wv1) status |= SGS_ST_NEWTON_FAIL;
  if (it > 0 || store_on_fail) {
    if (it < 0) {
      // keep the last usable theta (warm start) so the sweep can continue and report
      if (th0) {
#pragma unroll
        for (int k = 0; k < 5; k++) th[k] = th0[k];
      }
      maxw_eval<E>(N, dv, w, wv1, inv_dx, target, th, ev);
    }
    __syncwarp();
    if (lane < N) {
      sm.E1[lane] = ev.e[0];
      sm.E2[lane] = ev.e[1];
      sm.E3[lane] = ev.e[2];
    }
    if (lane < 5) th_out[lane] = th[lane];
  }
  return it;
}

template <typename E, int EPT>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int q = blockIdx.x / CS;
  if (q >= a.n_inst) return;  // whole cluster, uniformly
  const InstDev& I = a.inst[q];
  __shared__ SweepSmem<E> sm;
  const int N = a.N, K = N * N * N;
  const double dv = a.dv, w = a.dv * a.dv * a.dv;
  const int J = I.J;
  const double inv_dx = 1.0 / I.dx;
  const E inv_eps = cvt<E>(1.0 / I.eps);
  const int tid = threadIdx.x, wid = tid >> 5;
  const bool pfp = I.inner_method == SGS_PFP;
  const bool lowp = sizeof(E) == 4;  // plain FP32 (not df64): tolerances at FP32 resolution
  const double ntol = lowp ? fmax(I.newton_tol, 1e-5) : I.newton_tol;
  const E zero = cvt<E>(0.0);
  if (tid < N) {
    double v = node(tid, N, dv);
    sm.vv[tid] = cvt<E>(v);
    sm.vq[tid] = cvt<E>(v * v);
    sm.W3[0][tid] = cvt<E>(I.wall[0][2][tid]);
    sm.W3[1][tid] = cvt<E>(I.wall[1][2][tid]);
  }
  __syncthreads();

  // this thread's nodes: pencil (i1, i2), i3 in [i30, i30 + EPT)
  const int tg = rank * blockDim.x + tid;
  const int e0 = tg * EPT;
  const bool own = e0 < K;
  const int pen = own ? e0 / N : 0, i30 = own ? e0 % N : 0;
  const int i1 = pen / N, i2 = pen % N;
  const double v1d = node(i1, N, dv), v2d = node(i2, N, dv);
  const E v1 = cvt<E>(v1d), v2 = cvt<E>(v2d);
  const E c1 = cvt<E>(fabs(v1d) * inv_dx);
  const E vpd = cvt<E>(fmax(v1d, 0.0) * inv_dx), vmd = cvt<E>(fmin(v1d, 0.0) * inv_dx);
  const E vq12 = cvt<E>(v1d * v1d + v2d * v2d);
  const E wl12 = cvt<E>(I.wall[0][0][i1] * I.wall[0][1][i2]);
  const E wr12 = cvt<E>(I.wall[1][0][i1] * I.wall[1][1][i2]);

  E g[EPT], r[EPT];
  int buf = 0;
  unsigned long long c_inner = 0, c_newton = 0, c_solves = 0, c_fallback = 0;
  unsigned int status = 0;
  bool have_th = false;

  for (int s = 0; s < J; s++) {
    const int j = a.dir > 0 ? s : J - 1 - s;
    const long long cbase = I.f_off + (long long)j * K + e0;
    double* fj = a.f + cbase;
    const bool lw = j == 0, rw = j == J - 1;

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
    for (int k = 0; k < 5; k++) mom[k] = cvt<E>(w * t7[k]);
    const E rho_l = cvt<E>(I.bc_kind[0] == SGS_INFLOW ? I.bc_rho[0] : -(w * t7[5]) / I.wall_denom[0]);
    const E rho_r = cvt<E>(I.bc_kind[1] == SGS_INFLOW ? I.bc_rho[1] : -(w * t7[6]) / I.wall_denom[1]);

    // ---- r = (-v1^+ f_{j-1} + v1^- f_{j+1}) / dx - P_j / eps - b_j (neighbours: latest values)
    const double nuj = a.nu[I.cell0 + j];
    const double Ad = nuj / I.eps;
    const E Acoef = cvt<E>(Ad);
    const E den = cvt<E>(1.0 / (fabs(v1d) * inv_dx + Ad));
    const E c1A = cvt<E>(fabs(v1d) * inv_dx + Ad);
    if (own) {
      const double* Pj = a.P + cbase;
      const double* bj = a.rhs ? a.rhs + cbase : nullptr;
#pragma unroll
      for (int t = 0; t < EPT; t++) {
        E left = lw ? rho_l * wl12 * sm.W3[0][i30 + t] : cvt<E>(fj[t - K]);
        E right = rw ? rho_r * wr12 * sm.W3[1][i30 + t] : cvt<E>(fj[t + K]);
        double pb = Pj[t] / I.eps + (bj ? bj[t] : 0.0);
        r[t] = vmd * right - vpd * left - cvt<E>(pb);
      }
    }

    // ---- M[g] of the stored value (warm start from the previous cell's M[g])
    if (wid == 0) {
      int n0 = newton_store<E>(sm, N, dv, w, false, 0.0, mom, have_th ? sm.thg : nullptr, sm.thg, ntol,
                               I.newton_max, status, true);
      if (n0 > 0) c_newton += n0;
      c_solves++;
    }
    have_th = true;
    __syncthreads();

    int it = 0;
    for (;;) {
      // ---- pass B: cell-equation residual, its scale, and the step-1 target s (eq. (26))
      E e12 = sm.E1[i1] * sm.E2[i2];
      E rs = zero, sc = zero, b0 = zero, b3 = zero, b4 = zero;
      if (own) {
#pragma unroll
        for (int t = 0; t < EPT; t++) {
          E M = e12 * sm.E3[i30 + t];
          E d = M - g[t];
          // (|v1|/dx) g + r - (nu/eps)(M - g) = (|v1|/dx + nu/eps) g + r - (nu/eps) M
          E res = c1A * g[t] + r[t] - Acoef * M;
          rs += res * res;
          E mag = c1A * g[t];
          sc += mag * mag;
          E tt = c1 * d - r[t];
          b0 += tt;
          b3 += tt * sm.vv[i30 + t];
          b4 += tt * sm.vq[i30 + t];
        }
      }
      E v7[7] = {rs, b0, v1 * b0, v2 * b0, b3, vq12 * b0 + b4, sc};
      double t6[7];
      cluster_reduce<7, E>(v7, t6, sm, buf, cl, CS);
      const double res = sqrt(w * t6[0]);
      double tol = I.inner_tol;
      if (lowp) tol = fmax(tol, 2e-6 * sqrt(w * t6[6]));
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
      if (stop) break;

      // ---- step 1 (eq. (24)) from M[g]; else the plain fixed-point step (eq. (22))
      bool used = false;  // meaningful in warp 0 only
      if (wid == 0) {
        double sd[5] = {w * t6[1], w * t6[2], w * t6[3], w * t6[4], w * t6[5]};
        if (pfp) {
          bool exists = sd[0] > 0.0 && sd[0] * sd[4] > sd[1] * sd[1] + sd[2] * sd[2] + sd[3] * sd[3];
          if (exists) {
            E sv[5] = {cvt<E>(sd[0]), cvt<E>(sd[1]), cvt<E>(sd[2]), cvt<E>(sd[3]), cvt<E>(sd[4])};
            int n1 = newton_store<E>(sm, N, dv, w, true, inv_dx, sv, sm.thg, sm.thp, ntol, I.newton_max, status,
                                     false);
            c_solves++;
            if (n1 > 0) {
              c_newton += n1;
              used = true;
            }
          }
          if (!used) c_fallback++;
        }
      }
      __syncthreads();

      // ---- step 2 (eq. (25)) and the moments of the new iterate
      E ep = sm.E1[i1] * sm.E2[i2];
      E c0 = zero, c3 = zero, c4 = zero;
      if (own) {
#pragma unroll
        for (int t = 0; t < EPT; t++) {
          E x = (Acoef * (ep * sm.E3[i30 + t]) - r[t]) * den;
          g[t] = x;
          c0 += x;
          c3 += x * sm.vv[i30 + t];
          c4 += x * sm.vq[i30 + t];
        }
      }
      E m5[5] = {c0, v1 * c0, v2 * c0, c3, vq12 * c0 + c4};
      double t5[5];
      cluster_reduce<5, E>(m5, t5, sm, buf, cl, CS);
      it++;
      if (wid == 0) {
        E mm[5] = {cvt<E>(w * t5[0]), cvt<E>(w * t5[1]), cvt<E>(w * t5[2]), cvt<E>(w * t5[3]), cvt<E>(w * t5[4])};
        // warm start: the step-1 Maxwellian approximates M of the updated iterate
        int n2 = newton_store<E>(sm, N, dv, w, false, 0.0, mm, used ? sm.thp : sm.thg, sm.thg, ntol,
                                 I.newton_max, status, true);
        if (n2 > 0) c_newton += n2;
        c_solves++;
      }
      __syncthreads();
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

  if (rank == 0 && tid == 0) {
    Counters* c = a.cnt + q;
    atomicAdd(&c->visits, (unsigned long long)J);
    atomicAdd(&c->inner_iters, c_inner);
    atomicAdd(&c->newton_iters, c_newton);
    atomicAdd(&c->newton_solves, c_solves);
    atomicAdd(&c->fallbacks, c_fallback);
  }
  if (tid == 0 && status) atomicOr(&a.cnt[q].status, status);
}

// Default launch shape: nodes per thread (a divisor of N), cluster size (a power of two, at
// most 16) and threads per CTA (a multiple of 32, at most 256).
SweepShape sweep_shape(int N, int arith) {
  SweepShape s;
  int K = N * N * N;
  s.ept = arith == kSweepF32 ? N : (N <= 8 ? 2 : (N % 8 == 0 ? 8 : 4));
  int threads = K / s.ept;
  s.cluster = 1;
  while (s.cluster < 16 && s.cluster * 256 < threads) s.cluster *= 2;
  s.tpb = ((threads + s.cluster - 1) / s.cluster + 31) / 32 * 32;
  return s;
}

template <typename E, int EPT>
static cudaError_t launch_sweep_t(const SweepArgs& a, const SweepShape& sh, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_sweep<E, EPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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

bool sweep_shape_valid(int N, const SweepShape& sh) {
  int K = N * N * N;
  if (sh.ept <= 0 || N % sh.ept != 0) return false;
  if (sh.cluster < 1 || sh.cluster > 16 || sh.tpb < 32 || sh.tpb > 256 || sh.tpb % 32) return false;
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
