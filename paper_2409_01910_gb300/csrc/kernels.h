// Launch interfaces between the host API (sgs_api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace sgs {

template <typename T>
struct CplxOf;
template <>
struct CplxOf<double> {
  typedef double2 type;
};
template <>
struct CplxOf<float> {
  typedef float2 type;
};
template <typename T>
struct VecOf;
template <>
struct VecOf<double> {
  typedef double2 type;
};
template <>
struct VecOf<float> {
  typedef float4 type;
};
__device__ __forceinline__ double vec_get(const double2& v, int i) { return i == 0 ? v.x : v.y; }
__device__ __forceinline__ float vec_get(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
int sum_pad(int H, int elem_bytes);
__host__ __device__ inline double2 make_cplx(double a, double b) { return make_double2(a, b); }
__host__ __device__ inline float2 make_cplx(float a, float b) { return make_float2(a, b); }

// Cell list of the collision step (all instances, same N).
struct CellTables {
  const InstDev* inst;
  const long long* cell_off;  // element offset of each cell's distribution
  const int* cell_inst;       // instance of each cell
  const int* active;          // per instance (nullable): 0 = converged, its cells are skipped
};

// Whether cell c belongs to an active instance (every cell when active is null). A converged
// instance's f no longer changes, so its last collision results stay valid.
__device__ __forceinline__ bool cell_active(const int* active, const int* cell_inst, int c) {
  return !active || active[cell_inst[c]] != 0;
}

template <typename T>
struct SpecBufs {
  typedef typename CplxOf<T>::type CT;
  const double* tw_cos;  // [n][N] cos(2 pi k j / N), k = row - h, j = i - N/2 + 1
  const double* tw_sin;  // [n][N] sin(2 pi k j / N)
  const T* twc;          // the same tables in T (precomputed: no conversion in the kernels)
  const T* tws;
  CT *st1a, *st1b;       // [C][N][N][n]
  CT *st2a, *st2b;       // [C][N][n][n]
  CT *ahat, *bhat;       // [G][n][n][n][32]
  CT* qhat;              // [G][n][n][n][32]
  const int* cell_inst;  // instance of each cell, and the per-instance activity (nullable):
  const int* active;     // the transforms skip the cells of converged instances
};

template <typename T>
struct SumArgs {
  typedef typename CplxOf<T>::type CT;
  const int4* units;            // k1, k2, m1_lo, m1_hi
  const long long* unit_step0;  // first step of each unit in the weight table
  const T* W;                   // [steps][PW]
  const CT* ahat;
  const CT* bhat;
  CT* partial;                  // [units][Gs][n][32]
  int G;                        // groups of this launch (ahat, bhat, partial start at its first group)
  int Gs;                       // group stride of partial (the handle's group count)
  Counters* cnt;
  long long spin_max;
  const int* cell_inst;         // cells of this launch's groups and the per-instance activity
  const int* active;            // (nullable): a block whose groups hold no active cell returns
  int C;                        // cells of this launch
};

// Inputs of the first DFT pass: mode 0 transforms (f - M, f + M); modes 1 and 2 transform
// increments against a reference state (f_ref, M[f_ref]): mode 1 gives (Da, f + M), mode 2 gives
// (unused, Db), where Da = (f - M) - (f_ref - M_ref) and Db = (f + M) - (f_ref + M_ref).
struct DftMode {
  int mode;
  const double* f_ref;
  const double* theta_ref;
};

template <typename T>
struct RedArgs {
  typedef typename CplxOf<T>::type CT;
  const int2* row_k;      // (k1, k2) of each half-space row
  const int* row_start;   // CSR over row_units
  const int* row_units;
  const CT* partial;
  const CT* partial2;     // optional second set of partials, summed after the first
  CT* qhat;
  int n, G, n_rows;  // G: groups of this launch
  int Gs;            // group stride of partial and partial2
};

// Double-float spectral sum: weights as (FP32 table, FP32 remainder table) in the packed
// layout of the FP32 sum; rows as (re_hi, re_lo, im_hi, im_lo); partials in FP64.
struct SumDfArgs {
  const int4* units;
  const long long* unit_step0;
  const float* Whi;   // [steps][PW32]
  const float* Wlo;   // [steps][PW32]
  const float4* ahat;
  const float4* bhat;
  double2* partial;   // [units][Gs][n][32]
  int G;              // groups of this launch (ahat, bhat, partial start at its first group)
  int Gs;             // group stride of partial
  Counters* cnt;
  long long spin_max;
  const int* cell_inst;
  const int* active;  // as in SumArgs
  int C;
};

template <typename T>
struct CollideCtx {
  int N, C, H, NW, n_units;
  double dv;
  CellTables ct;
  const double* theta;
  const double* nu;
  double* efac;           // [C][3][kMaxN] separable factors of each cell's Maxwellian
  double* efac_ref;       // the same for the reference state (increment modes)
  double* mom;            // [C][N][5] moments of Q per slab (conservation projection), or null
  const double* cproj;    // [5][5] inverse Gram matrix of (1, v, |v|^2) (projection mode 1)
  int cproj_mode;         // 0 none, 1 plain, 2 Maxwellian-weighted conservation projection
  SpecBufs<T> sb;
  SumArgs<T> sum;
  RedArgs<T> red;
};

struct SweepArgs {
  const InstDev* inst;
  int n_inst;
  double* f;
  const double* P;
  const double* rhs;
  const double* nu;       // per global cell
  Counters* cnt;          // per instance
  int N;
  double dv;
  int dir;                // +1 forward, -1 backward
  const int* active;      // per instance: 0 = converged, its scans are skipped
  const double* theta;    // per global cell: Maxwellian exponents of the last collision step
  int s0, s1;             // 1-D: the launch visits scan positions [s0, min(s1, J)) (cells in scan
                          // order; a whole scan is [0, J)), so that a scan can run in segments
};

struct AuxArgs {
  const InstDev* inst;
  int n_inst, N, C;
  double dv;
  const long long* cell_off;
  const int* cell_inst;
  double* scratch;        // per-cell partials, per-instance values
  const int* active;      // per instance: 0 = converged, its rescale is skipped
  int two_d;              // 2-D space (one instance): grid nx x ny
  int nx, ny;
  double* sflux;          // second-order scheme: slope fluxes of the walls, [2 n_inst] in 1-D, one per
                          // boundary face [2 (nx + ny)] in 2-D; null at first order
};

// Host side (sgs_api.cu): validation of one problem description (SGS_OK, SGS_ERR_ARG or
// SGS_ERR_UNSUPPORTED, as sgs_setup returns them) and its device description.
int check_problem(const sgs_problem& p);
void fill_inst(const sgs_problem& p, int N, double dv, InstDev& I);

// cudaFuncSetAttribute through a per-device cache: the call is made once per (kernel,
// attribute, value) and device, so launches stay free of it (also during stream capture).
cudaError_t func_attr(const void* fn, cudaFuncAttribute attr, int value);
cudaError_t launch_update_active(const double* res, int n, double tol, int* active, cudaStream_t st);
cudaError_t launch_fill_int(int* p, int n, int value, cudaStream_t st);

// Separable factors of every cell's discrete Maxwellian from theta (efac [C][3][kMaxN]).
cudaError_t launch_factors(const double* theta, int C, int N, double dv, double* efac, cudaStream_t st);
// Second-order scheme (1-D): out = rhs + the explicit slope terms of the scan and the
// face-value correction of the lagged wall densities, all from the state f before the scan.
cudaError_t launch_slope_rhs(const AuxArgs& a, const double* f, const double* rhs, double* out, cudaStream_t st);
// The same for one 2-D instance (slopes along x and y, four wall sides).
cudaError_t launch_slope_rhs2d(const AuxArgs& a, const double* f, const double* rhs, double* out, cudaStream_t st);
// Source iteration: wall fluxes of f, then the per-node transport march (1-D problems).
cudaError_t launch_si_transport(const AuxArgs& a, double* f, const double* P, const double* rhs, const double* efac,
                                const double* nu, cudaStream_t st);
cudaError_t launch_moments(const double* f, const CellTables& ct, int C, int N, double dv, double tol, int maxit,
                           double* theta, double* nu, Counters* cnt, cudaStream_t st);
cudaError_t launch_collide_bgk(const double* f, const CellTables& ct, int C, int N, double dv, const double* theta,
                               const double* nu, double* Q, double* P, cudaStream_t st);
template <typename T>
cudaError_t launch_dft(const double* f, const CollideCtx<T>& x, const DftMode& md, cudaStream_t st);
template <typename T>
cudaError_t launch_spectral_sum(const CollideCtx<T>& x, typename CplxOf<T>::type* partial, cudaStream_t st);
template <typename T>
// Qraw (with the conservation projection; needs Q): also receives the unprojected operator.
cudaError_t launch_reduce_idft(const double* f, double* Q, double* P, const CollideCtx<T>& x,
                               const typename CplxOf<T>::type* partial2, const double* Qadd, cudaStream_t st,
                               double* Qraw = nullptr);
cudaError_t launch_sum_df(const SumDfArgs& a, int H, int n_units, cudaStream_t st);
cudaError_t launch_split_spec(double2* x, long long count, cudaStream_t st);
cudaError_t launch_build_weights_lo(const int4* units, const long long* unit_step0, int n_units, int H, int PW,
                                    const double* G, long long nb, const double* Lo, float* W, cudaStream_t st);
template <typename T>
cudaError_t launch_build_weights(const int4* units, const long long* unit_step0, int n_units, int H, int PW,
                                 const double* G, long long nb, const double* Lo, T* W, cudaStream_t st);

struct SweepShape {
  int ept;      // velocity nodes per thread (divides N)
  int cluster;  // CTAs per instance
  int tpb;      // threads per CTA
};
// arithmetic of the sweep's elementwise work and reductions
constexpr int kSweepF64 = 0;   // native FP64
constexpr int kSweepDF64 = 1;  // double-float on the FP32 pipes (FP64-class accuracy)
constexpr int kSweepF32 = 2;   // plain FP32 (converges only to FP32 resolution)
SweepShape sweep_shape(int N, int arith);
bool sweep_shape_valid(int N, const SweepShape& sh);
// Sweep launch shapes: nodes per thread with a compiled kernel, and the number of clusters of
// the shape that fit on the device at once (0: the shape cannot run).
bool sweep_ept_compiled(int ept);
cudaError_t sweep_max_clusters(const SweepShape& sh, int arith, int* n);
// 2-D: one wavefront (anti-diagonal wf of ordering 0..3) of the single 2-D instance.
cudaError_t launch_sweep2d(const SweepArgs& a, const SweepShape& sh, int arith, int ordering, int wf, int ncells,
                           cudaStream_t st);
cudaError_t launch_sweep(const SweepArgs& a, const SweepShape& sh, int arith, cudaStream_t st);
// Fast (Carleman-form) spectral operator on the tensor cores (fast.cu): one chunk of S slots
// (half-sphere nodes, the loss slot last) for every cell.
struct FastArgs {
  int n, npad, P, C, S;         // modes per dimension, padded K modes, grid, cells, slots of the chunk
  int s0;                       // first global slot of the chunk
  int terms;
  const float* fhat;            // [C][n][npad][npad][2]
  const float* wtab;            // [slots][2][n][npad][npad]
  const float* wslot;           // [slots] weight of each slot's product
  const float* bt12;            // [2P][2 npad]: passes 1 and 2
  const float* bt3;             // [P][2 npad]: pass 3 (real part)
  // the pass-2 and pass-3 operands as BF16 planes (hi; lo for 3 terms) of 128-row tiles in the
  // K-major core-matrix layout (K = 2 npad): Y1 rows (b, x3, k1 < npad) in blocks of 8 x3 by
  // 4 k1 (the order of fast.cu's y1_row), K (k2, re/im); Y2 rows (b, x2, x3), K (k1, re/im)
  uint16_t* Y1h;
  uint16_t* Y1l;
  uint16_t* Y2h;
  uint16_t* Y2l;
  float* G;                     // [C][P][P][P]
  long long spin_max;
  unsigned int* status;         // TIMEOUT bit
};

cudaError_t launch_fast_fhat(const float2* ahat, const float2* bhat, int C, int n, int npad, float* out,
                             cudaStream_t st);
cudaError_t launch_fast_pass(int pass, const FastArgs& a, cudaStream_t st);
cudaError_t launch_fast_final(const float* G, const float2* tw, int C, int n, int P, float2* T1, float2* T2,
                              float2* qhat, cudaStream_t st);

// Tensor-core self-test (fast.cu): D = A Bt^T on tcgen05 and on the CUDA cores.
cudaError_t tc_selftest(const float* A, const float* Bt, float* D, float* Dref, int K, int N, int terms, int swap,
                        int* err, cudaStream_t st);
// Latency probe of the scan's building blocks in one cluster of the given shape: mode 0
// cluster reductions, mode 1 Newton iterations of the discrete Maxwellian (reps of each).
cudaError_t probe_scan(int N, double dv, int arith, int cluster, int threads, int mode, int reps, cudaStream_t st);

cudaError_t launch_rescale(const AuxArgs& a, double* f, cudaStream_t st);
// rho, U, T and the heat flux q of every cell: out[8 c + (0..7)]
cudaError_t launch_macroscopic(const AuxArgs& a, const double* f, double* out, cudaStream_t st);
// After launch_rescale: Q, P (nullable) *= lam^2, nu *= lam, alpha += ln lam for the cells
// [c_lo, c_hi) whose collision step was evaluated on the state before the rescale.
cudaError_t launch_rescale_fixup(const AuxArgs& a, int c_lo, int c_hi, double* Q, double* P, double* nu,
                                 double* theta, cudaStream_t st);
cudaError_t launch_dc_rhs(const AuxArgs& a, const double* Qhi, double* Qlo_b, cudaStream_t st);
cudaError_t launch_residual(const AuxArgs& a, const double* f, const double* Q, const double* rhs, double* res,
                            cudaStream_t st);
cudaError_t launch_restrict(const double* fine, double* coarse, long long K, int Jc, cudaStream_t st);
// 2 x 2 coarsening of an nx x ny grid (2-D)
cudaError_t launch_restrict2d(const double* fine, double* coarse, long long K, int nx, int ny, cudaStream_t st);
cudaError_t launch_prolong_add2d(double* fine, const double* fc, const double* fc0, long long K, int nx, int ny,
                                 cudaStream_t st);
cudaError_t launch_axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t st);
cudaError_t launch_prolong_add(double* fine, const double* fc, const double* fc0, long long K, int Jc,
                               cudaStream_t st);
cudaError_t launch_residual_field(const AuxArgs& a, const double* f, const double* Q, const double* rhs, double* R,
                                  cudaStream_t st);

}  // namespace sgs
