// Outer residual of one instance without any device allocation.
//
// sgs_residual() keeps its per-cell partial sums in the workspace that the caller allocates
// and binds. Some callers cannot allocate device memory at all: code running inside a host
// framework that owns every allocation (a custom allocator or memory pool that must not be
// bypassed), callers working under a hard device-memory budget, or code paths where an
// allocation could synchronise the device. This file gives them sgs_residual_noalloc(): the
// same computation for one instance, with its scratch in a file-scope static device array.
//
// The scratch array is part of the loaded library image: every GPU that loads the library
// keeps it (kNoAllocScratch doubles, 32 KiB + 64 bytes) until the process exits. All calls
// share it, so calls whose kernels overlap on the GPU (different streams, or different host
// threads without ordering) race on it; order such calls on one stream. Every slot a call
// reads is written earlier in the same call, so no clearing between calls is needed.
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace sgs {
namespace {

constexpr int kNoAllocMaxCells = 4096;
constexpr int kNoAllocScratch = kNoAllocMaxCells + 8;  // [0, 2): wall fluxes, [8, 8 + J): cell partials

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

// Device address of the scratch array, looked up once per device with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

__device__ inline double na_block_sum(double x, double* sh) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[k];
  __syncthreads();
  return t;
}

// Outgoing wall fluxes into scratch[0] (x_lo side, v1 < 0 of cell 0) and scratch[1]
// (x_hi side, v1 > 0 of cell J-1).
__global__ void __launch_bounds__(256) k_na_wall_flux(InstDev I, const double* __restrict__ f, int N, double dv,
                                                       double* scratch) {
  __shared__ double sh[32];
  int side = blockIdx.x;
  int K = N * N * N;
  const double* fa = f + (long long)(side ? I.J - 1 : 0) * K;
  double acc = 0.0;
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    double v1 = node(e / (N * N), N, dv);
    if ((side == 0 && v1 < 0.0) || (side == 1 && v1 > 0.0)) acc += v1 * fa[e];
  }
  double t = na_block_sum(acc, sh);
  if (threadIdx.x == 0) scratch[side] = dv * dv * dv * t;
}

// Per-cell sum of w R^2 into scratch[8 + j].
__global__ void __launch_bounds__(256) k_na_residual_cells(InstDev I, const double* __restrict__ f,
                                                            const double* __restrict__ Q,
                                                            const double* __restrict__ rhs, int N, double dv,
                                                            double* scratch) {
  __shared__ double sh[32];
  int j = blockIdx.x;
  int K = N * N * N;
  long long base = (long long)j * K;
  double w = dv * dv * dv;
  double inv_dx = 1.0 / I.dx, inv_eps = 1.0 / I.eps;
  double rho_l = I.bc_kind[0] == SGS_INFLOW ? I.bc_rho[0] : -scratch[0] / I.wall_denom[0];
  double rho_r = I.bc_kind[1] == SGS_INFLOW ? I.bc_rho[1] : -scratch[1] / I.wall_denom[1];
  double acc = 0.0;
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    int i1 = e / (N * N), i2 = (e / N) % N, i3 = e % N;
    double v1 = node(i1, N, dv);
    double fj = f[base + e];
    double fl = j == 0 ? rho_l * I.wall[0][0][i1] * I.wall[0][1][i2] * I.wall[0][2][i3] : f[base - K + e];
    double fr = j == I.J - 1 ? rho_r * I.wall[1][0][i1] * I.wall[1][1][i2] * I.wall[1][2][i3] : f[base + K + e];
    double R = (fmax(v1, 0.0) * (fj - fl) + fmin(v1, 0.0) * (fr - fj)) * inv_dx - Q[base + e] * inv_eps;
    if (rhs) R -= rhs[base + e];
    acc += R * R;
  }
  double t = na_block_sum(acc, sh);
  if (threadIdx.x == 0) scratch[8 + j] = w * t;
}

__global__ void k_na_residual_final(int J, double dx, const double* scratch, double* res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int j = 0; j < J; j++) s += scratch[8 + j];
  res[0] = sqrt(dx * s);
}

}  // namespace
}  // namespace sgs

extern "C" int sgs_residual_noalloc(const sgs_problem* p, const double* f, const double* Q, const double* rhs,
                                    double* res, void* stream) {
  using namespace sgs;
  if (!p || !f || !Q || !res) return SGS_ERR_ARG;
  // the same problems sgs_setup accepts, restricted to what this entry point computes
  int chk = check_problem(*p);
  if (chk != SGS_OK) return chk;
  if (p->space_dim != 1) return SGS_ERR_ARG;      // one 1-D instance
  if (p->order == 2) return SGS_ERR_UNSUPPORTED;  // the first-order residual only
  if (p->nx > kNoAllocMaxCells) {
    fprintf(stderr, "sgs_residual_noalloc: %d cells exceed the static scratch capacity of %d cells\n", p->nx,
            kNoAllocMaxCells);
    return SGS_ERR_ARG;
  }
  const int N = p->nv;
  const double dv = 2.0 * p->v_max / N;
  InstDev I;
  fill_inst(*p, N, dv, I);  // wall Maxwellians and their zero-flux normalisation, as sgs_setup
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    fprintf(stderr, "sgs_residual_noalloc: scratch lookup failed: %s\n", cudaGetErrorString(e));
    return SGS_ERR_CUDA;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_na_wall_flux<<<2, 256, 0, st>>>(I, f, N, dv, scratch);
  k_na_residual_cells<<<p->nx, 256, 0, st>>>(I, f, Q, rhs, N, dv, scratch);
  k_na_residual_final<<<1, 32, 0, st>>>(p->nx, I.dx, scratch, res);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "sgs_residual_noalloc: launch failed: %s\n", cudaGetErrorString(e));
    return SGS_ERR_CUDA;
  }
  return SGS_OK;
}
