// Fast (Carleman-form) Fourier spectral collision operator on the tensor cores.
//
// Self-test of the tensor-core path first: one CTA computes D = A B^T on tcgen05 (BF16
// operands split from FP32, FP32 accumulation in TMEM) and a plain CUDA-core product, so the
// operand layout and descriptors can be checked on the device before the operator uses them.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace sgs {
namespace {

constexpr int kTcRows = 128;  // M of every tcgen05.mma here (cta_group::1)

// D (128 x N) = A (128 x K) * Bt (N x K)^T. terms 1: Ah Bh; terms 3: Ah Bh + Al Bh + Ah Bl.
// swap exchanges the two byte offsets of the descriptors (a layout check). err[0] receives 1
// when the completion wait gave up. Dref receives the FP32 CUDA-core product of the same
// BF16 terms.
__global__ void __launch_bounds__(kTcRows) k_tc_selftest(const float* __restrict__ A, const float* __restrict__ Bt,
                                                         float* __restrict__ D, float* __restrict__ Dref, int K,
                                                         int N, int terms, int swap, long long spin_max, int* err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  uint16_t* Ahi = reinterpret_cast<uint16_t*>(smraw);
  uint16_t* Alo = Ahi + kTcRows * K;
  uint16_t* Bhi = Alo + kTcRows * K;
  uint16_t* Blo = Bhi + N * K;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int t = threadIdx.x, warp = t >> 5;
  if (warp == 0) tc::tmem_alloc(&tslot, 128);
  if (t == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  for (int k = 0; k < K; k++) {
    uint16_t h, l;
    tc::split_bf16(A[t * K + k], h, l);
    const uint32_t o = tc::kmajor_offset(t, k, K) / 2;
    Ahi[o] = h;
    Alo[o] = l;
  }
  for (int r = t; r < N; r += kTcRows)
    for (int k = 0; k < K; k++) {
      uint16_t h, l;
      tc::split_bf16(Bt[r * K + k], h, l);
      const uint32_t o = tc::kmajor_offset(r, k, K) / 2;
      Bhi[o] = h;
      Blo[o] = l;
    }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tslot;
  if (t == 0) {
    const uint32_t lbo = swap ? (uint32_t)(K / 8) * 128 : 128, sbo = swap ? 128 : (uint32_t)(K / 8) * 128;
    const uint32_t idesc = tc::idesc_bf16_f32(kTcRows, N);
    for (int ks = 0; ks < K / 16; ks++) {
      const uint32_t step = (uint32_t)ks * 256;
      const uint64_t ah = tc::smem_desc(smem_addr(Ahi) + step, lbo, sbo);
      const uint64_t al = tc::smem_desc(smem_addr(Alo) + step, lbo, sbo);
      const uint64_t bh = tc::smem_desc(smem_addr(Bhi) + step, lbo, sbo);
      const uint64_t bl = tc::smem_desc(smem_addr(Blo) + step, lbo, sbo);
      tc::mma_bf16(taddr, ah, bh, idesc, ks > 0 ? 1u : 0u);
      if (terms == 3) {
        tc::mma_bf16(taddr, al, bh, idesc, 1u);
        tc::mma_bf16(taddr, ah, bl, idesc, 1u);
      }
    }
    tc::mma_commit(&bar);
  }
  // every thread waits; the result is made uniform so that the warp-wide TMEM loads below
  // are executed by all or none of the threads
  bool ok = __syncthreads_and(mbar_wait(&bar, 0, spin_max) ? 1 : 0) != 0;
  if (!ok) {
    if (t == 0) err[0] = 1;
    // one more bounded wait, so that no MMA is still writing TMEM when it is freed
    ok = __syncthreads_and(mbar_wait(&bar, 0, spin_max) ? 1 : 0) != 0;
    ok = false;
  }
  tc::fence_after_sync();
  if (ok) {
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int i = 0; i < 16; i++) D[t * N + c0 + i] = v[i];
    }
  }
  // CUDA-core product of the same BF16 terms
  for (int c = 0; c < N; c++) {
    float acc = 0.0f;
    for (int k = 0; k < K; k++) {
      const uint32_t oa = tc::kmajor_offset(t, k, K) / 2, ob = tc::kmajor_offset(c, k, K) / 2;
      const float ah = __bfloat162float(__ushort_as_bfloat16(Ahi[oa]));
      const float al = __bfloat162float(__ushort_as_bfloat16(Alo[oa]));
      const float bh = __bfloat162float(__ushort_as_bfloat16(Bhi[ob]));
      const float bl = __bfloat162float(__ushort_as_bfloat16(Blo[ob]));
      acc = fmaf(ah, bh, acc);
      if (terms == 3) acc = fmaf(al, bh, fmaf(ah, bl, acc));
    }
    Dref[t * N + c] = acc;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(taddr, 128);
}


// ---------------------------------------------------------------------------------------
// The fast operator (hard spheres, Carleman form, 3-D velocity). For every cell c and every
// slot s of the half-sphere rule (plus one slot for the loss term) the two weighted spectra
// X_{s,a} = w_{s,a} fhat_c (a = 0, 1) are transformed to a zero-padded P^3 grid by three
// separable passes, each a GEMM on the tensor cores against the DFT matrix
// E[x, k] = exp(2 pi i x (k - h) / P) written as a real 2 x 2 block matrix:
//   pass 1 (k3 -> x3): rows (b, k1, k2), K = (k3, re/im), out (x3, re/im) -> Y1[b][x3][k1][k2]
//   pass 2 (k2 -> x2): rows (b, x3, k1), K = (k2, re/im), out (x2, re/im) -> Y2[b][x2][x3][k1]
//   pass 3 (k1 -> x1): rows (c, x2, x3), K = (k1, re/im), out x1 (real part) for a = 0 and
//     a = 1, multiplied and summed over the slots with their weights into G[c][x2][x3][x1]
// b = (c, s, a). Operands are FP32 in memory, split into BF16 hi + lo on the way into shared
// memory (terms 3: hi hi + lo hi + hi lo; terms 1: hi hi), accumulated in FP32 in TMEM.
// ---------------------------------------------------------------------------------------

// Four consecutive values (k % 4 == 0) of one row: one 8-byte shared store per BF16 tile.
__device__ inline void put4(uint16_t* hi, uint16_t* lo, int row, int k, int K, float4 v, int terms) {
  uint16_t h[4], l[4];
  tc::split_bf16(v.x, h[0], l[0]);
  tc::split_bf16(v.y, h[1], l[1]);
  tc::split_bf16(v.z, h[2], l[2]);
  tc::split_bf16(v.w, h[3], l[3]);
  const uint32_t o = tc::kmajor_offset(row, k, K) / 2;
  *reinterpret_cast<uint2*>(hi + o) =
      make_uint2((uint32_t)h[0] | ((uint32_t)h[1] << 16), (uint32_t)h[2] | ((uint32_t)h[3] << 16));
  if (terms == 3)
    *reinterpret_cast<uint2*>(lo + o) =
        make_uint2((uint32_t)l[0] | ((uint32_t)l[1] << 16), (uint32_t)l[2] | ((uint32_t)l[3] << 16));
}

// A contiguous tile of ROWS rows x K floats (rows from `valid` on read as zero) into the BF16
// hi / lo tiles: 16-byte loads, eight in flight per thread before they are converted.
template <int K, int ROWS>
__device__ inline void load_tile(const float* __restrict__ src, int valid, uint16_t* hi, uint16_t* lo, int terms) {
  static_assert(ROWS % 8 == 0 && K % 8 == 0, "whole core matrices");
  constexpr int kChunks = ROWS * K / 4;
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll 1
  for (int c0 = threadIdx.x; c0 < kChunks; c0 += kTcRows * 8) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const int c = c0 + u * kTcRows;
      v[u] = c < kChunks && (c * 4) / K < valid ? s4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const int c = c0 + u * kTcRows;
      if (c < kChunks) put4(hi, lo, (c * 4) / K, (c * 4) % K, K, v[u], terms);
    }
  }
}

// Issues the MMAs of one product (K / 16 steps, 1 or 3 terms) into TMEM column `col`.
__device__ inline void issue_product(uint32_t tmem, uint32_t ahi, uint32_t alo, uint32_t bhi, uint32_t blo, int K,
                                     int N, int terms) {
  const uint32_t sbo = (uint32_t)(K / 8) * 128;
  const uint32_t idesc = tc::idesc_bf16_f32(128, N);
  for (int ks = 0; ks < K / 16; ks++) {
    const uint32_t step = (uint32_t)ks * 256;
    tc::mma_bf16(tmem, tc::smem_desc(ahi + step, 128, sbo), tc::smem_desc(bhi + step, 128, sbo), idesc,
                 ks > 0 ? 1u : 0u);
    if (terms == 3) {
      tc::mma_bf16(tmem, tc::smem_desc(alo + step, 128, sbo), tc::smem_desc(bhi + step, 128, sbo), idesc, 1u);
      tc::mma_bf16(tmem, tc::smem_desc(ahi + step, 128, sbo), tc::smem_desc(blo + step, 128, sbo), idesc, 1u);
    }
  }
}

// Waits for the MMAs committed to `bar` (phase parity `par`), uniformly over the CTA. On a
// time-out it reports, waits once more (bounded) so that nothing still writes TMEM, and
// returns false.
__device__ inline bool wait_mma(uint64_t* bar, uint32_t par, const FastArgs& a) {
  bool ok = __syncthreads_and(mbar_wait(bar, par, a.spin_max) ? 1 : 0) != 0;
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(a.status, SGS_ST_TIMEOUT);
    __syncthreads_and(mbar_wait(bar, par, a.spin_max) ? 1 : 0);
  }
  tc::fence_after_sync();
  return ok;
}

// NP: padded mode count along K (16 or 32, K = 2 NP); PP: the padded grid P (32 or 48).
template <int PASS, int NP, int PP>
__global__ void __launch_bounds__(kTcRows) k_fast_pass(FastArgs a) {
  extern __shared__ __align__(128) unsigned char smraw[];
  constexpr int K = 2 * NP, P = PP, np = NP;
  constexpr int NB = PASS == 3 ? P : 2 * P;  // columns of one product
  const int n = a.n;
  uint16_t* Bhi = reinterpret_cast<uint16_t*>(smraw);
  uint16_t* Blo = Bhi + NB * K;
  uint16_t* Abuf = Blo + NB * K;              // [nA][hi, lo][128][K]
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int t = threadIdx.x, warp = t >> 5;
  if (warp == 0) tc::tmem_alloc(&tslot, 128);
  if (t == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  // the DFT matrix of this pass (NB rows of K floats, contiguous), split once per CTA
  load_tile<K, NB>(PASS == 3 ? a.bt3 : a.bt12, NB, Bhi, Blo, 3);
  const int B = a.C * a.S * 2;
  long long rows;
  if (PASS == 1) rows = (long long)B * n * np;
  else if (PASS == 2) rows = (long long)B * P * n;
  else rows = (long long)a.C * P * P;
  const long long tiles = (rows + kTcRows - 1) / kTcRows;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tslot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  uint32_t phase = 0;
  bool ok = true;
  for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
    const long long r = tile * kTcRows + t;  // this thread's row
    const bool live = r < rows;
    if (PASS != 3) {
      // ---- A tile: 128 rows of K values
      uint16_t* Ahi = Abuf;
      uint16_t* Alo = Abuf + kTcRows * K;
      if (PASS == 1) {
        // row (b, k1, k2): the weights of slot s and side ab times the cell's spectrum,
        // both rows contiguous; every load of the row is issued before the first use
        int b = 0, k1 = 0, k2 = 0;
        if (live) {
          b = (int)(r / (n * np));
          const int rem = (int)(r % (n * np));
          k1 = rem / np;
          k2 = rem % np;
        }
        const int ab = b & 1, sl = (b >> 1) % a.S, c = (b >> 1) / a.S;
        const float4* fr = reinterpret_cast<const float4*>(a.fhat + (((long long)c * n + k1) * np + k2) * np * 2);
        const float4* wr =
            reinterpret_cast<const float4*>(a.wtab + ((((long long)(a.s0 + sl) * 2 + ab) * n + k1) * np + k2) * np);
        float4 fv[NP / 2], wv[NP / 4];
#pragma unroll
        for (int i = 0; i < NP / 2; i++) fv[i] = live ? fr[i] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int i = 0; i < NP / 4; i++) wv[i] = live ? wr[i] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int i = 0; i < NP / 2; i++) {  // K elements 4 i .. 4 i + 3: modes k3 = 2 i, 2 i + 1
          const float4 w4 = wv[i / 2];
          const float w0 = (i & 1) ? w4.z : w4.x, w1 = (i & 1) ? w4.w : w4.y;
          put4(Ahi, Alo, t, 4 * i, K, make_float4(w0 * fv[i].x, w0 * fv[i].y, w1 * fv[i].z, w1 * fv[i].w), a.terms);
        }
      } else {
        // rows of Y1 are consecutive blocks of K floats
        load_tile<K, kTcRows>(a.Y1 + tile * kTcRows * K, (int)(rows - tile * kTcRows < kTcRows ? rows - tile * kTcRows : kTcRows), Ahi, Alo,
                     a.terms);
      }
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (t == 0) {
        issue_product(taddr, smem_addr(Ahi), smem_addr(Alo), smem_addr(Bhi), smem_addr(Blo), K, NB, a.terms);
        tc::mma_commit(&bar);
      }
      ok = wait_mma(&bar, phase, a);
      phase ^= 1u;
      if (!ok) break;
      // ---- epilogue: 2P columns (x, re/im) of this thread's row
      for (int c0 = 0; c0 < NB; c0 += 16) {
        float v[16];
        tc::tmem_ld16(taddr + lane_base + (uint32_t)c0, v);
        if (!live) continue;
        if (PASS == 1) {
          const int b = (int)(r / (n * np)), rem = (int)(r % (n * np)), k1 = rem / np, k2 = rem % np;
#pragma unroll
          for (int i = 0; i < 16; i += 2) {
            const int x3 = (c0 + i) >> 1;
            float2* o = reinterpret_cast<float2*>(a.Y1 + ((((long long)b * P + x3) * n + k1) * np + k2) * 2);
            *o = make_float2(v[i], v[i + 1]);
          }
        } else {
          const int b = (int)(r / (P * n)), rem = (int)(r % (P * n)), x3 = rem / n, k1 = rem % n;
#pragma unroll
          for (int i = 0; i < 16; i += 2) {
            const int x2 = (c0 + i) >> 1;
            float2* o = reinterpret_cast<float2*>(a.Y2 + ((((long long)b * P + x2) * P + x3) * np + k1) * 2);
            *o = make_float2(v[i], v[i + 1]);
          }
        }
      }
      tc::fence_before_sync();
      __syncthreads();
    } else {
      // ---- pass 3: rows (c, x2, x3) of one cell (P^2 is a multiple of 128)
      const int c = (int)(tile * kTcRows / ((long long)P * P));
      const int row0 = (int)(tile * kTcRows % ((long long)P * P));
      float g[P];
#pragma unroll
      for (int i = 0; i < P; i++) g[i] = 0.0f;
      for (int sl = 0; sl < a.S && ok; sl++) {
        for (int ab = 0; ab < 2; ab++) {
          uint16_t* Ahi = Abuf + (size_t)ab * 2 * kTcRows * K;
          uint16_t* Alo = Ahi + kTcRows * K;
          const long long b = ((long long)c * a.S + sl) * 2 + ab;
          load_tile<K, kTcRows>(a.Y2 + (b * P * P + row0) * K, kTcRows, Ahi, Alo, a.terms);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0) {
          for (int ab = 0; ab < 2; ab++) {
            uint16_t* Ahi = Abuf + (size_t)ab * 2 * kTcRows * K;
            issue_product(taddr + (uint32_t)(ab * P), smem_addr(Ahi), smem_addr(Ahi + kTcRows * K), smem_addr(Bhi),
                          smem_addr(Blo), K, NB, a.terms);
          }
          tc::mma_commit(&bar);
        }
        ok = wait_mma(&bar, phase, a);
        phase ^= 1u;
        if (!ok) break;
        const float ws = a.wslot[a.s0 + sl];
#pragma unroll
        for (int c0 = 0; c0 < P; c0 += 16) {
          float va[16], vb[16];
          tc::tmem_ld16(taddr + lane_base + (uint32_t)c0, va);
          tc::tmem_ld16(taddr + lane_base + (uint32_t)(P + c0), vb);
#pragma unroll
          for (int i = 0; i < 16; i++) g[c0 + i] = fmaf(ws * va[i], vb[i], g[c0 + i]);
        }
        tc::fence_before_sync();
        __syncthreads();
      }
      if (ok && live) {
        float4* o = reinterpret_cast<float4*>(a.G + ((long long)c * P * P + row0 + t) * P);
#pragma unroll
        for (int i = 0; i < P / 4; i++) {
          float4 v = o[i];
          v.x += g[4 * i];
          v.y += g[4 * i + 1];
          v.z += g[4 * i + 2];
          v.w += g[4 * i + 3];
          o[i] = v;
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(taddr, 128);
}

// Compact FP32 spectrum of every cell, fhat = (ahat + bhat) / 2 (the transforms of f - M and
// f + M), zero-padded to npad along k2 and k3: out[c][k1][k2][k3][re, im].
__global__ void k_fast_fhat(const double2* __restrict__ ahat, const double2* __restrict__ bhat, int C, int n,
                            int npad, float* __restrict__ out) {
  const long long total = (long long)C * n * npad * npad;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int k3 = (int)(i % npad), k2 = (int)((i / npad) % npad), k1 = (int)((i / ((long long)npad * npad)) % n);
    const int c = (int)(i / ((long long)npad * npad * n));
    float2 v = make_float2(0.0f, 0.0f);
    if (k2 < n && k3 < n) {
      const long long o = ((((long long)(c / kLanes) * n + k1) * n + k2) * n + k3) * kLanes + (c % kLanes);
      v = make_float2((float)(0.5 * (ahat[o].x + bhat[o].x)), (float)(0.5 * (ahat[o].y + bhat[o].y)));
    }
    reinterpret_cast<float2*>(out)[i] = v;
  }
}

// Forward transform of G (real, [c][x2][x3][x1]) to the modes |k_i| <= h, times P^-3, in three
// passes with FP64 accumulation; tw[k][x] = exp(-2 pi i (k - h) x / P).
// pass A: T1[c][x2][x3][k1] = sum_x1 G e^{..k1 x1}
__global__ void k_fast_final_a(const float* __restrict__ G, const double2* __restrict__ tw, int n, int P,
                               double2* __restrict__ T1) {
  const long long cx = blockIdx.x;  // (c, x2, x3)
  const float* g = G + cx * P;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int x = 0; x < P; x++) {
      const double2 w = tw[k * P + x];
      re += w.x * g[x];
      im += w.y * g[x];
    }
    T1[cx * n + k] = make_double2(re, im);
  }
}

// pass B: T2[c][x2][k3][k1] = sum_x3 T1[c][x2][x3][k1] e^{..k3 x3}
__global__ void k_fast_final_b(const double2* __restrict__ T1, const double2* __restrict__ tw, int n, int P,
                               double2* __restrict__ T2) {
  const long long cx2 = blockIdx.x;  // (c, x2)
  const double2* src = T1 + cx2 * P * n;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int k3 = i / n, k1 = i % n;
    double re = 0.0, im = 0.0;
    for (int x3 = 0; x3 < P; x3++) {
      const double2 w = tw[k3 * P + x3], v = src[x3 * n + k1];
      re += w.x * v.x - w.y * v.y;
      im += w.x * v.y + w.y * v.x;
    }
    T2[cx2 * n * n + i] = make_double2(re, im);
  }
}

// pass C: qhat[g][k1][k2][k3][lane] = P^-3 sum_x2 T2[c][x2][k3][k1] e^{..k2 x2}
__global__ void k_fast_final_c(const double2* __restrict__ T2, const double2* __restrict__ tw, int n, int P,
                               double2* __restrict__ qhat) {
  const int c = blockIdx.x;
  const double scale = 1.0 / ((double)P * P * P);
  for (int i = threadIdx.x; i < n * n * n; i += blockDim.x) {
    const int k1 = i / (n * n), k2 = (i / n) % n, k3 = i % n;
    double re = 0.0, im = 0.0;
    for (int x2 = 0; x2 < P; x2++) {
      const double2 w = tw[k2 * P + x2], v = T2[(((long long)c * P + x2) * n + k3) * n + k1];
      re += w.x * v.x - w.y * v.y;
      im += w.x * v.y + w.y * v.x;
    }
    const long long o = ((((long long)(c / kLanes) * n + k1) * n + k2) * n + k3) * kLanes + (c % kLanes);
    qhat[o] = make_double2(re * scale, im * scale);
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Launchers of the fast operator.
// ---------------------------------------------------------------------------------------
cudaError_t launch_fast_fhat(const double2* ahat, const double2* bhat, int C, int n, int npad, float* out,
                             cudaStream_t st) {
  const long long total = (long long)C * n * npad * npad;
  k_fast_fhat<<<(int)std::min<long long>((total + 255) / 256, 152 * 8), 256, 0, st>>>(ahat, bhat, C, n, npad, out);
  return cudaGetLastError();
}

template <int PASS, int NP, int PP>
static cudaError_t launch_pass_t(const FastArgs& a, cudaStream_t st) {
  constexpr int K = 2 * NP, NB = PASS == 3 ? PP : 2 * PP, nA = PASS == 3 ? 2 : 1;
  constexpr size_t smem = (size_t)2 * NB * K * sizeof(uint16_t) + (size_t)nA * 2 * kTcRows * K * sizeof(uint16_t);
  auto kern = k_fast_pass<PASS, NP, PP>;
  cudaError_t e = func_attr((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // the whole unified L1 as shared memory, so that several CTAs share an SM
  if (e == cudaSuccess) e = func_attr((const void*)kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  const long long B = (long long)a.C * a.S * 2;
  long long rows = PASS == 1 ? B * a.n * NP : (PASS == 2 ? B * PP * a.n : (long long)a.C * PP * PP);
  const long long tiles = (rows + kTcRows - 1) / kTcRows;
  int dev = 0, sms = 0, per = 0, sm_bytes = 0, reserved = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kTcRows, smem);
  if (e != cudaSuccess) return e;
  // CTAs an SM's shared memory holds (the occupancy query can assume a smaller carveout); the
  // tile loop is strided, so CTAs beyond the resident ones only wait for a slot
  const int by_smem = sm_bytes / (int)(smem + 256 + (size_t)reserved);
  per = std::max(1, std::min(std::max(per, by_smem), 4));  // 128 TMEM columns per CTA: at most 4 CTAs share 512
  const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)sms * per));
  kern<<<grid, kTcRows, smem, st>>>(a);
  return cudaGetLastError();
}

template <int PASS>
static cudaError_t launch_pass_p(const FastArgs& a, cudaStream_t st) {
  if (a.npad == 16 && a.P == 32) return launch_pass_t<PASS, 16, 32>(a, st);
  if (a.npad == 32 && a.P == 32) return launch_pass_t<PASS, 32, 32>(a, st);
  if (a.npad == 32 && a.P == 48) return launch_pass_t<PASS, 32, 48>(a, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_fast_pass(int pass, const FastArgs& a, cudaStream_t st) {
  if (pass == 1) return launch_pass_p<1>(a, st);
  if (pass == 2) return launch_pass_p<2>(a, st);
  if (pass == 3) return launch_pass_p<3>(a, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_fast_final(const float* G, const double2* tw, int C, int n, int P, double2* T1, double2* T2,
                              double2* qhat, cudaStream_t st) {
  k_fast_final_a<<<C * P * P, 32, 0, st>>>(G, tw, n, P, T1);
  k_fast_final_b<<<C * P, 256, 0, st>>>(T1, tw, n, P, T2);
  k_fast_final_c<<<C, 256, 0, st>>>(T2, tw, n, P, qhat);
  return cudaGetLastError();
}

cudaError_t tc_selftest(const float* A, const float* Bt, float* D, float* Dref, int K, int N, int terms, int swap,
                        int* err, cudaStream_t st) {
  if (K % 16 || K < 16 || K > 64 || N % 16 || N < 16 || N > 128 || (terms != 1 && terms != 3))
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)2 * (kTcRows + N) * K * sizeof(uint16_t);
  cudaError_t e = func_attr((const void*)k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tc_selftest<<<1, kTcRows, smem, st>>>(A, Bt, D, Dref, K, N, terms, swap, 1LL << 24, err);
  return cudaGetLastError();
}

}  // namespace sgs

// Self-test of the tensor-core path (no counterpart in the paper; a check of the operand
// layout and descriptors on the device): D = A B^T for a 128 x K operand A and an N x K operand
// Bt of seeded values, on tcgen05 and on the CUDA cores from the same BF16 terms.
extern "C" int sgs_tc_selftest(int K, int N, int terms, int swap, void* dev_scratch, size_t bytes, double* max_err,
                               double* max_ref, void* stream) {
  using namespace sgs;
  if (!dev_scratch || !max_err || !max_ref) return SGS_ERR_ARG;
  const size_t nA = (size_t)128 * K, nB = (size_t)N * K, nD = (size_t)128 * N;
  const size_t need = sizeof(float) * (nA + nB + 2 * nD) + 256;
  if (bytes < need) return SGS_ERR_WORKSPACE;
  float* A = static_cast<float*>(dev_scratch);
  float* B = A + nA;
  float* D = B + nB;
  float* Dr = D + nD;
  int* err = reinterpret_cast<int*>(Dr + nD);
  std::vector<float> hA(nA), hB(nB), hD(nD), hR(nD);
  unsigned long long x = 0x9E3779B97F4A7C15ULL;
  auto rnd = [&]() {  // xorshift64*, values in [-1, 1)
    x ^= x >> 12;
    x ^= x << 25;
    x ^= x >> 27;
    return (float)((double)((x * 0x2545F4914F6CDD1DULL) >> 11) / 9007199254740992.0 * 2.0 - 1.0);
  };
  for (auto& v : hA) v = rnd();
  for (auto& v : hB) v = rnd();
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(A, hA.data(), sizeof(float) * nA, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B, hB.data(), sizeof(float) * nB, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(D, 0, sizeof(float) * nD, st);
  if (e == cudaSuccess) e = tc_selftest(A, B, D, Dr, K, N, terms, swap, err, st);
  if (e == cudaErrorInvalidValue) return SGS_ERR_ARG;
  if (e == cudaSuccess) e = cudaMemcpyAsync(hD.data(), D, sizeof(float) * nD, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hR.data(), Dr, sizeof(float) * nD, cudaMemcpyDeviceToHost, st);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    fprintf(stderr, "sgs_tc_selftest: %s\n", cudaGetErrorString(e));
    return SGS_ERR_CUDA;
  }
  double me = 0.0, mr = 0.0;
  for (size_t i = 0; i < nD; i++) {
    me = std::max(me, (double)std::fabs(hD[i] - hR[i]));
    mr = std::max(mr, (double)std::fabs(hR[i]));
  }
  *max_err = herr ? -1.0 : me;
  *max_ref = mr;
  return SGS_OK;
}
