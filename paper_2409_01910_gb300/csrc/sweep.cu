// Persistent symmetric Gauss-Seidel scan (eq. (29), first order) with the preconditioned
// fixed-point cell solve (eqs. (20), (24)-(26)).
//
// One thread-block cluster per instance walks that instance's cells in scan order inside a
// single launch. A thread owns the same velocity nodes in every cell, so the upwind
// neighbour's new value (just computed) stays in registers; only the downwind neighbour's
// old value, P_j and rhs_j are read from global memory. Every velocity sum (moments,
// cell-equation residual, step-1 target) is a cluster-wide reduction: per-thread FP64
// partials -> warp butterfly -> block -> each CTA reads every CTA's partial through
// distributed shared memory in rank order, so all CTAs hold bit-identical totals and take
// identical branches. The discrete-Maxwellian Newton solves need only O(N) work on the
// tensor grid (separable Maxwellian) and run redundantly in warp 0 of every CTA.
#include "common.cuh"
#include "kernels.h"

namespace sgs {

struct SweepSmem {
  double vv[kMaxN];   // nodes v_i
  double vq[kMaxN];   // v_i^2
  double c1[kMaxN];   // |v_i| / dx
  double vpd[kMaxN];  // max(v_i, 0) / dx
  double vmd[kMaxN];  // min(v_i, 0) / dx
  double den[kMaxN];  // 1 / (|v_i|/dx + nu/eps)
  double E[3][kMaxN]; // factors of the Maxwellian in use (E[0] carries exp(alpha))
  double red_warp[32][8];
  double red_part[2][8];
  double red_tot[8];
  double thg[5];
};

template <int NV>
__device__ inline void cluster_reduce(double (&v)[NV], SweepSmem& sm, int& buf, cg::cluster_group& cl, int CS) {
  warp_allsum<NV>(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; q++) sm.red_warp[wid][q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double t = 0.0;
    for (int k = 0; k < nw; k++) t += sm.red_warp[k][threadIdx.x];
    sm.red_part[buf][threadIdx.x] = t;
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
  for (int q = 0; q < NV; q++) v[q] = sm.red_tot[q];
  buf ^= 1;
}

// Warp 0 writes the Maxwellian factors of its last Newton evaluation to shared memory.
__device__ inline void store_factors(SweepSmem& sm, const MaxwEval& ev, int N) {
  int lane = threadIdx.x & 31;
  if (lane < N) {
    sm.E[0][lane] = ev.e[0];
    sm.E[1][lane] = ev.e[1];
    sm.E[2][lane] = ev.e[2];
  }
}

template <int EPT>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int q = blockIdx.x / CS;
  if (q >= a.n_inst) return;  // whole cluster, uniformly
  const InstDev& I = a.inst[q];
  __shared__ SweepSmem sm;
  const int N = a.N, K = N * N * N;
  const double dv = a.dv, w = dv * dv * dv;
  const int J = I.J;
  const double inv_dx = 1.0 / I.dx, inv_eps = 1.0 / I.eps;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int stride = CS * blockDim.x, e0 = rank * blockDim.x + tid;
  const bool pfp = I.inner_method == SGS_PFP;
  if (tid < N) {
    double v = node(tid, N, dv);
    sm.vv[tid] = v;
    sm.vq[tid] = v * v;
    sm.c1[tid] = fabs(v) * inv_dx;
    sm.vpd[tid] = fmax(v, 0.0) * inv_dx;
    sm.vmd[tid] = fmin(v, 0.0) * inv_dx;
  }
  __syncthreads();

  int idx[EPT];
#pragma unroll
  for (int t = 0; t < EPT; t++) {
    int e = e0 + t * stride;
    idx[t] = e < K ? (((e / (N * N)) << 16) | (((e / N) % N) << 8) | (e % N)) : -1;
  }
  double g[EPT], r[EPT], gp[EPT];
#pragma unroll
  for (int t = 0; t < EPT; t++) gp[t] = 0.0;

  int buf = 0;
  unsigned long long c_inner = 0, c_newton = 0, c_solves = 0, c_fallback = 0;
  unsigned int status = 0;

  for (int s = 0; s < J; s++) {
    const int j = a.dir > 0 ? s : J - 1 - s;
    const long long cbase = I.f_off + (long long)j * K;
    double* fj = a.f + cbase;
    const double* Pj = a.P + cbase;
    const double* bj = a.rhs ? a.rhs + cbase : nullptr;
    const bool lw = j == 0, rw = j == J - 1;

    // ---- reduction 1: moments of the stored value and the walls' outgoing fluxes
    double m7[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int t = 0; t < EPT; t++) {
      if (idx[t] < 0) {
        g[t] = 0.0;
        continue;
      }
      int e = e0 + t * stride;
      int i1 = idx[t] >> 16, i2 = (idx[t] >> 8) & 0xff, i3 = idx[t] & 0xff;
      double x = fj[e];
      g[t] = x;
      double v1 = sm.vv[i1];
      m7[0] += x;
      m7[1] += x * v1;
      m7[2] += x * sm.vv[i2];
      m7[3] += x * sm.vv[i3];
      m7[4] += x * (sm.vq[i1] + sm.vq[i2] + sm.vq[i3]);
      if (lw && v1 < 0.0) m7[5] += v1 * x;
      if (rw && v1 > 0.0) m7[6] += v1 * x;
    }
    cluster_reduce<7>(m7, sm, buf, cl, CS);
    double mom[5];
#pragma unroll
    for (int k = 0; k < 5; k++) mom[k] = w * m7[k];
    const double rho_l = I.bc_kind[0] == SGS_INFLOW ? I.bc_rho[0] : -(w * m7[5]) / I.wall_denom[0];
    const double rho_r = I.bc_kind[1] == SGS_INFLOW ? I.bc_rho[1] : -(w * m7[6]) / I.wall_denom[1];

    // ---- r = (-v1^+ f_{j-1} + v1^- f_{j+1}) / dx - P_j / eps - b_j
    const double nuj = a.nu[I.cell0 + j];
    const double Acoef = nuj * inv_eps;
    const double* fdn = nullptr;  // downwind neighbour (old value) if interior
    if (a.dir > 0 && !rw) fdn = fj + K;
    if (a.dir < 0 && !lw) fdn = fj - K;
#pragma unroll
    for (int t = 0; t < EPT; t++) {
      if (idx[t] < 0) {
        r[t] = 0.0;
        continue;
      }
      int e = e0 + t * stride;
      int i1 = idx[t] >> 16, i2 = (idx[t] >> 8) & 0xff, i3 = idx[t] & 0xff;
      double left, right;
      if (lw)
        left = rho_l * I.wall[0][0][i1] * I.wall[0][1][i2] * I.wall[0][2][i3];
      else
        left = a.dir > 0 ? gp[t] : fdn[e];
      if (rw)
        right = rho_r * I.wall[1][0][i1] * I.wall[1][1][i2] * I.wall[1][2][i3];
      else
        right = a.dir > 0 ? fdn[e] : gp[t];
      double rv = -sm.vpd[i1] * left + sm.vmd[i1] * right - Pj[e] * inv_eps;
      if (bj) rv -= bj[e];
      r[t] = rv;
    }
    if (tid < N) sm.den[tid] = 1.0 / (sm.c1[tid] + Acoef);

    // ---- M[g]: discrete Maxwellian of the current iterate
    if (wid == 0) {
      double th[5] = {0, 0, 0, 0, 0};
      MaxwEval ev;
      int it = -1;
      if (continuum_guess(mom, th)) it = maxwellian_newton(N, dv, w, false, 0.0, mom, th, I.newton_tol, I.newton_max, ev);
      if (it < 0) {
        status |= SGS_ST_NEWTON_FAIL;
        if (!continuum_guess(mom, th)) status |= SGS_ST_NONPOSITIVE;
        maxw_eval(N, dv, w, false, 0.0, mom, th, ev);
      } else {
        c_newton += it;
      }
      c_solves++;
      store_factors(sm, ev, N);
      if (lane < 5) sm.thg[lane] = th[lane];
    }
    __syncthreads();

    int it = 0;
    for (;;) {
      // ---- pass B: cell-equation residual and the step-1 target s (eq. (26) notation)
      double v6[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int t = 0; t < EPT; t++) {
        if (idx[t] < 0) continue;
        int i1 = idx[t] >> 16, i2 = (idx[t] >> 8) & 0xff, i3 = idx[t] & 0xff;
        double M = sm.E[0][i1] * sm.E[1][i2] * sm.E[2][i3];
        double c1 = sm.c1[i1];
        double d = M - g[t];
        double res = c1 * g[t] + r[t] - Acoef * d;
        v6[0] += res * res;
        double tt = c1 * d - r[t];
        v6[1] += tt;
        v6[2] += tt * sm.vv[i1];
        v6[3] += tt * sm.vv[i2];
        v6[4] += tt * sm.vv[i3];
        v6[5] += tt * (sm.vq[i1] + sm.vq[i2] + sm.vq[i3]);
      }
      cluster_reduce<6>(v6, sm, buf, cl, CS);
      const double res = sqrt(w * v6[0]);
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
      if (stop) break;

      // ---- step 1 (eq. (24)) or the plain fixed-point step (eq. (22))
      if (wid == 0) {
        double sv[5] = {w * v6[1], w * v6[2], w * v6[3], w * v6[4], w * v6[5]};
        bool used = false;
        if (pfp) {
          bool exists = sv[0] > 0.0 && sv[0] * sv[4] > sv[1] * sv[1] + sv[2] * sv[2] + sv[3] * sv[3];
          if (exists) {
            double th[5];
#pragma unroll
            for (int k = 0; k < 5; k++) th[k] = sm.thg[k];
            MaxwEval ev;
            int n1 = maxwellian_newton(N, dv, w, true, inv_dx, sv, th, I.newton_tol, I.newton_max, ev);
            c_solves++;
            if (n1 > 0) {
              c_newton += n1;
              __syncwarp();
              store_factors(sm, ev, N);
              used = true;
            }
          }
          if (!used) c_fallback++;
        }
      }
      __syncthreads();

      // ---- step 2 (eq. (25)) and the moments of the new iterate
      double m5[5] = {0, 0, 0, 0, 0};
#pragma unroll
      for (int t = 0; t < EPT; t++) {
        if (idx[t] < 0) continue;
        int i1 = idx[t] >> 16, i2 = (idx[t] >> 8) & 0xff, i3 = idx[t] & 0xff;
        double Mp = sm.E[0][i1] * sm.E[1][i2] * sm.E[2][i3];
        double x = (Acoef * Mp - r[t]) * sm.den[i1];
        g[t] = x;
        m5[0] += x;
        m5[1] += x * sm.vv[i1];
        m5[2] += x * sm.vv[i2];
        m5[3] += x * sm.vv[i3];
        m5[4] += x * (sm.vq[i1] + sm.vq[i2] + sm.vq[i3]);
      }
      cluster_reduce<5>(m5, sm, buf, cl, CS);
      it++;
      if (wid == 0) {
        double mm[5] = {w * m5[0], w * m5[1], w * m5[2], w * m5[3], w * m5[4]};
        double th[5] = {0, 0, 0, 0, 0};
        MaxwEval ev;
        int n2 = -1;
        if (continuum_guess(mm, th)) n2 = maxwellian_newton(N, dv, w, false, 0.0, mm, th, I.newton_tol, I.newton_max, ev);
        if (n2 < 0) {
          status |= SGS_ST_NEWTON_FAIL;
          if (!continuum_guess(mm, th)) {
            status |= SGS_ST_NONPOSITIVE;
#pragma unroll
            for (int k = 0; k < 5; k++) th[k] = sm.thg[k];
          }
          maxw_eval(N, dv, w, false, 0.0, mm, th, ev);
        } else {
          c_newton += n2;
        }
        c_solves++;
        __syncwarp();
        store_factors(sm, ev, N);
        if (lane < 5) sm.thg[lane] = th[lane];
      }
      __syncthreads();
    }

#pragma unroll
    for (int t = 0; t < EPT; t++) {
      if (idx[t] < 0) continue;
      fj[e0 + t * stride] = g[t];
      gp[t] = g[t];
    }
    c_inner += it;
    // every CTA must finish reading this cell's neighbours before the next cell's
    // writes can be observed: the first reduction of the next visit is a cluster barrier.
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

int sweep_cluster_for(int N) {
  if (N <= 8) return 1;
  if (N <= 16) return 4;
  if (N <= 24) return 8;
  return 16;
}

template <int EPT>
static cudaError_t launch_sweep_t(const SweepArgs& a, int cluster, int tpb, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_sweep<EPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.n_inst * cluster);
  cfg.blockDim = dim3(tpb);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_sweep<EPT>, a);
}

cudaError_t launch_sweep(const SweepArgs& a, int cluster, int tpb, cudaStream_t st) {
  int K = a.N * a.N * a.N;
  int need = (K + cluster * tpb - 1) / (cluster * tpb);
  if (need <= 1) return launch_sweep_t<1>(a, cluster, tpb, st);
  if (need <= 2) return launch_sweep_t<2>(a, cluster, tpb, st);
  if (need <= 4) return launch_sweep_t<4>(a, cluster, tpb, st);
  if (need <= 8) return launch_sweep_t<8>(a, cluster, tpb, st);
  if (need <= 16) return launch_sweep_t<16>(a, cluster, tpb, st);
  return cudaErrorInvalidConfiguration;
}

}  // namespace sgs
