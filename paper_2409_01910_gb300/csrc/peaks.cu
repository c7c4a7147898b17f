// Peak-rate probes of the arithmetic pipes that bound the solver's kernels.
//
// The direct spectral sums run on the CUDA-core FMA pipes (FP32 FFMA, FP64 DFMA), not on
// the tensor cores, so their rooflines need the FMA throughput of the device the solver runs
// on. k_peak_fma runs independent FMA chains (eight per thread, enough in flight to cover
// the pipe latency) on every SM and reports the rate the pipes sustain, timed with CUDA
// events on the caller's stream. Nothing is allocated: the chains' results are kept alive
// through a store to a static device variable behind a runtime test that never passes.
#include <cstdio>
#include <cstring>

#include "common.cuh"

namespace sgs {
namespace {

__device__ double g_peak_sink;

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__device__ __forceinline__ float fma_t(float x, float a, float b) { return fmaf(x, a, b); }
__device__ __forceinline__ double fma_t(double x, double a, double b) { return fma(x, a, b); }
// A pair of FP32 values in one 64-bit register pair, multiplied and added by the packed
// instruction fma.rn.f32x2 (both halves at once).
struct f32x2 {
  unsigned long long v;
  __host__ __device__ f32x2() : v(0ull) {}
  __host__ __device__ explicit f32x2(float x) {
    unsigned u;
    memcpy(&u, &x, sizeof(u));
    v = ((unsigned long long)u << 32) | u;
  }
  __device__ bool operator==(const f32x2& o) const { return v == o.v; }
};
__device__ __forceinline__ f32x2 fma_t(f32x2 x, f32x2 a, f32x2 b) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(x.v), "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ f32x2 operator+(f32x2 x, f32x2 y) { return fma_t(x, f32x2(1.0f), y); }
__device__ __forceinline__ f32x2& operator+=(f32x2& x, f32x2 y) { return x = x + y; }
__device__ __forceinline__ double to_double(f32x2 x) { return (double)__uint_as_float((unsigned)x.v); }
__device__ __forceinline__ double to_double(float x) { return (double)x; }
__device__ __forceinline__ double to_double(double x) { return x; }

// sentinel: a runtime value the chains never reach (they stay positive and small), so the
// compiler cannot drop the chains as dead code
template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(long long iters, T a, T b, T sentinel) {
  T x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; q++) x[q] = T((float)(threadIdx.x + q) * 1e-3f);
  for (long long i = 0; i < iters; i++) {
#pragma unroll
    for (int q = 0; q < kChains; q++) x[q] = fma_t(x[q], a, b);
  }
  T s = x[0];
#pragma unroll
  for (int q = 1; q < kChains; q++) s += x[q];
  if (s == sentinel) g_peak_sink = to_double(s);
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
  const T a = T(0.999999f), b = T(1e-7f);
  k_peak_fma<T><<<blocks, kPeakThreads, 0, st>>>(iters / 8 + 1, a, b, T(-1.0f));  // warm-up
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    k_peak_fma<T><<<blocks, kPeakThreads, 0, st>>>(iters, a, b, T(-1.0f));
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
  const bool packed = (precision & SGS_PEAK_PACKED) != 0;
  precision &= ~SGS_PEAK_PACKED;
  if ((precision != SGS_FP32 && precision != SGS_FP64) || (packed && precision != SGS_FP32) || iters < 1 || !tflops)
    return SGS_ERR_ARG;
  int dev = 0, n_sm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = packed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak_fma<f32x2>, kPeakThreads, 0)
        : precision == SGS_FP32
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak_fma<float>, kPeakThreads, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak_fma<double>, kPeakThreads, 0);
  if (e != cudaSuccess || per_sm < 1) {
    fprintf(stderr, "sgs_peak_fma: %s\n", cudaGetErrorString(e));
    return SGS_ERR_CUDA;
  }
  const int blocks = n_sm * per_sm;  // every SM fully occupied, one wave
  float t = 0.0f;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  e = packed                    ? time_fma<f32x2>(blocks, iters, st, &t)
      : precision == SGS_FP32 ? time_fma<float>(blocks, iters, st, &t)
                              : time_fma<double>(blocks, iters, st, &t);
  if (e != cudaSuccess) {
    fprintf(stderr, "sgs_peak_fma: %s\n", cudaGetErrorString(e));
    return SGS_ERR_CUDA;
  }
  const double flops = 2.0 * (packed ? 2 : 1) * kChains * (double)iters * (double)blocks * kPeakThreads;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (sms) *sms = n_sm;
  if (ms) *ms = t;
  return SGS_OK;
}
