// Peak-rate probes of the arithmetic pipes that bound the solver's kernels.
//
// The direct spectral sums run on the CUDA-core FMA pipes (FP32 FFMA, FP64 DFMA), not on
// the tensor cores, so their rooflines need the FMA throughput of the device the solver runs
// on. k_peak_fma runs independent FMA chains (eight per thread, enough in flight to cover
// the pipe latency) on every SM and reports the rate the pipes sustain, timed with CUDA
// events on the caller's stream. Nothing is allocated: the chains' results are kept alive
// through a store to a static device variable behind a runtime test that never passes.
#include <cstdio>

#include "common.cuh"

namespace sgs {
namespace {

__device__ double g_peak_sink;

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__device__ __forceinline__ float fma_t(float x, float a, float b) { return fmaf(x, a, b); }
__device__ __forceinline__ double fma_t(double x, double a, double b) { return fma(x, a, b); }

// sentinel: a runtime value the chains never reach (they stay positive and small), so the
// compiler cannot drop the chains as dead code
template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(long long iters, T a, T b, T sentinel) {
  T x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; q++) x[q] = (T)(threadIdx.x + q) * (T)1e-3;
  for (long long i = 0; i < iters; i++) {
#pragma unroll
    for (int q = 0; q < kChains; q++) x[q] = fma_t(x[q], a, b);
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < kChains; q++) s += x[q];
  if (s == sentinel) g_peak_sink = (double)s;
}

template <typename T>
cudaError_t time_fma(int blocks, long long iters, cudaStream_t st, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  const T a = (T)0.999999, b = (T)1e-7;
  k_peak_fma<T><<<blocks, kPeakThreads, 0, st>>>(iters / 8 + 1, a, b, (T)-1);  // warm-up
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    k_peak_fma<T><<<blocks, kPeakThreads, 0, st>>>(iters, a, b, (T)-1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace
}  // namespace sgs

extern "C" int sgs_peak_fma(int precision, long long iters, double* tflops, int* sms, float* ms, void* stream) {
  using namespace sgs;
  if ((precision != SGS_FP32 && precision != SGS_FP64) || iters < 1 || !tflops) return SGS_ERR_ARG;
  int dev = 0, n_sm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = precision == SGS_FP32
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak_fma<float>, kPeakThreads, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak_fma<double>, kPeakThreads, 0);
  if (e != cudaSuccess || per_sm < 1) {
    fprintf(stderr, "sgs_peak_fma: %s\n", cudaGetErrorString(e));
    return SGS_ERR_CUDA;
  }
  const int blocks = n_sm * per_sm;  // every SM fully occupied, one wave
  float t = 0.0f;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  e = precision == SGS_FP32 ? time_fma<float>(blocks, iters, st, &t) : time_fma<double>(blocks, iters, st, &t);
  if (e != cudaSuccess) {
    fprintf(stderr, "sgs_peak_fma: %s\n", cudaGetErrorString(e));
    return SGS_ERR_CUDA;
  }
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kPeakThreads;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (sms) *sms = n_sm;
  if (ms) *ms = t;
  return SGS_OK;
}
