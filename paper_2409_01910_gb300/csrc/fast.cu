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
//   pass 1 (k3 -> x3): rows (b, k1, k2), K = (k3, re/im), out (x3, re/im) -> Y1 rows (b, x3, k1)
//   pass 2 (k2 -> x2): rows (b, x3, k1), K = (k2, re/im), out (x2, re/im) -> Y2 rows (b, x2, x3)
//   pass 3 (k1 -> x1): rows (c, x2, x3), K = (k1, re/im), out x1 (real part) for a = 0 and
//     a = 1, multiplied and summed over the slots with their weights into G[c][x2][x3][x1]
// b = (c, s, a). Pass 1 forms its operand from the FP32 spectra and weights and splits it into
// BF16 hi + lo (terms 3: products hi hi + lo hi + hi lo; terms 1: hi hi), accumulated in FP32
// in TMEM; the pass-2 and pass-3 operands (Y1, Y2) are stored by the previous pass's epilogue
// as BF16 planes already in the shared-memory layout of the tensor core and streamed by bulk
// copies; the DFT matrices are split once per CTA.
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

// Bounded wait on phase `par` of `bar`, uniform over the CTA (every thread polls; the result
// is the AND), so that the warp-wide TMEM instructions after it run in all threads or none.
__device__ inline bool wait_uniform(uint64_t* bar, uint32_t par, long long spin_max) {
  const bool ok = __syncthreads_and(mbar_wait(bar, par, spin_max) ? 1 : 0) != 0;
  tc::fence_after_sync();
  return ok;
}

// After a wait gave up: report, then wait (bounded) for every copy and MMA still in flight
// (uses next .. issued - 1 of each double-buffered barrier pair), so that nothing writes this
// CTA's shared memory or TMEM when it is released.
__device__ inline void drain(uint64_t* bar, int next, int issued, long long spin_max) {
  for (int q = next; q < issued; q++) mbar_wait(&bar[q & 1], (uint32_t)((q >> 1) & 1), spin_max);
}

// Intermediate operands (the outputs of passes 1 and 2) are stored as the next pass's A
// tiles: BF16 planes hi (and lo for 3 terms) of 128-row tiles in the K-major core-matrix
// layout of shared memory, tile t at element t * 128 * K, so that the next pass copies a
// tile into shared memory with one bulk copy per plane and hands it to the tensor core.
// (re, im) of one complex entry are adjacent along K: one 32-bit store per plane.
__device__ inline void store_pair(uint16_t* __restrict__ hi, uint16_t* __restrict__ lo, long long row, int k, int K,
                                  float re, float im, int terms) {
  uint16_t h0, l0, h1, l1;
  tc::split_bf16(re, h0, l0);
  tc::split_bf16(im, h1, l1);
  const long long o = (row >> 7) * (kTcRows * (long long)K) + tc::kmajor_offset((int)(row & 127), k, K) / 2;
  *reinterpret_cast<uint32_t*>(hi + o) = (uint32_t)h0 | ((uint32_t)h1 << 16);
  if (terms == 3) *reinterpret_cast<uint32_t*>(lo + o) = (uint32_t)l0 | ((uint32_t)l1 << 16);
}

// Row of Y1 (the pass-2 operand) holding (b, x3, k1): per b, blocks of 4 k1 (k1 padded to
// NP) by blocks of 8 x3, inside a block x3 major and k1 minor. A warp of pass 2 then holds 8
// consecutive x3 by 4 consecutive k1 of one b, so that for each x2 its 32 stores of the
// pass-3 operand fill one 128-byte core matrix (rows x3 .. x3 + 7, K entries of 4 k1):
// whole sectors, coalesced.
template <int NP, int P>
__device__ inline long long y1_row(int b, int x3, int k1) {
  return ((((long long)b * (NP / 4) + (k1 >> 2)) * (P / 8) + (x3 >> 3)) * 8 + (x3 & 7)) * 4 + (k1 & 3);
}

// ---- pass 1 (k3 -> x3): rows (b, k1, k2), A = w_{s,a} fhat_c formed by the threads from
// two contiguous rows of L2-resident tables; the epilogue writes the pass-2 operand Y1 (rows
// in y1_row order, K = (k2, re/im)). Software-pipelined: the loads of tile i + 1 are issued
// into registers before the epilogue of tile i - 1, A is double-buffered in shared memory
// and the accumulator in TMEM, so the loads' latency overlaps the epilogue and the MMAs.
template <int NP, int PP, int TERMS>
__global__ void __launch_bounds__(kTcRows) k_fast_pass1(FastArgs a) {
  constexpr int NPL = TERMS == 3 ? 2 : 1;  // BF16 planes of an operand (hi; lo for 3 products)
  extern __shared__ __align__(128) unsigned char smraw[];
  constexpr int K = 2 * NP, P = PP, np = NP, NB = 2 * P;
  constexpr int TILE = kTcRows * K;
  const int n = a.n;
  uint16_t* Bhi = reinterpret_cast<uint16_t*>(smraw);
  uint16_t* Blo = Bhi + NB * K;
  uint16_t* Abuf = Blo + NB * K;  // [2 buffers][NPL planes][TILE]
  __shared__ __align__(8) uint64_t bar_mma[2];
  __shared__ uint32_t tslot;
  const int t = threadIdx.x, warp = t >> 5;
  if (warp == 0) tc::tmem_alloc(&tslot, 256);  // two accumulators of NB columns, 128 apart
  if (t == 0) {
    mbar_init(&bar_mma[0], 1);
    mbar_init(&bar_mma[1], 1);
    fence_mbar_init();
  }
  load_tile<K, NB>(a.bt12, NB, Bhi, Blo, 3);  // the DFT matrix, split once per CTA
  // rows (b, k1 < NP, k2): per b, blocks of 4 k1 by blocks of 8 k2, inside a block k2 major
  // and k1 minor, so that for each x3 a warp's 32 epilogue stores fill two 64-byte runs of Y1
  // (rows of 4 consecutive k1, 16 consecutive K entries); rows with k1 >= n are zero
  const long long rows = (long long)a.C * a.S * 2 * NP * np;
  const long long tiles = (rows + kTcRows - 1) / kTcRows;
  const int nt = tiles > blockIdx.x ? (int)((tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tslot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  // this thread's row of tile i: (b, k1, k2); rows past the end read as zero
  auto row_of = [&](int i, int& b, int& k1, int& k2) {
    const long long r = (blockIdx.x + (long long)i * gridDim.x) * kTcRows + t;
    b = k1 = k2 = 0;
    if (r >= rows) return false;
    b = (int)(r / (NP * np));
    const int rem = (int)(r % (NP * np));  // ((k1 / 4) * (np / 8) + k2 / 8) * 32 + (k2 % 8) * 4 + k1 % 4
    const int blk = rem >> 5, in = rem & 31;
    k1 = (blk / (np / 8)) * 4 + (in & 3);
    k2 = (blk % (np / 8)) * 8 + (in >> 2);
    if (k1 >= n) {
      b = k1 = k2 = 0;
      return false;
    }
    return true;
  };
  float4 fv[NP / 2], wv[NP / 4];
  auto load_rows = [&](int i) {
    int b, k1, k2;
    const bool live = row_of(i, b, k1, k2);
    const int ab = b & 1, sl = (b >> 1) % a.S, c = (b >> 1) / a.S;
    const float4* fr = reinterpret_cast<const float4*>(a.fhat + (((long long)c * n + k1) * np + k2) * np * 2);
    const float4* wr =
        reinterpret_cast<const float4*>(a.wtab + ((((long long)(a.s0 + sl) * 2 + ab) * n + k1) * np + k2) * np);
#pragma unroll
    for (int q = 0; q < NP / 2; q++) fv[q] = live ? fr[q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NP / 4; q++) wv[q] = live ? wr[q] : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto epilogue = [&](int i) {
    int b, k1, k2;
    const bool live = row_of(i, b, k1, k2);
    const uint32_t acc = taddr + lane_base + (uint32_t)((i & 1) * 128);
#pragma unroll
    for (int c0 = 0; c0 < NB; c0 += 16) {
      float v[16];
      tc::tmem_ld16(acc + (uint32_t)c0, v);
      if (live) {
#pragma unroll
        for (int q = 0; q < 16; q += 2) {
          const int x3 = (c0 + q) >> 1;
          store_pair(a.Y1h, a.Y1l, y1_row<NP, P>(b, x3, k1), 2 * k2, K, v[q], v[q + 1], TERMS);
        }
      }
    }
  };
  int mma_next = 0, mma_wait = 0;
  bool ok = true;
  if (nt > 0) load_rows(0);
  for (int i = 0; i < nt; i++) {
    // A of tile i (its buffer was last read by MMA i - 2, waited for in iteration i - 1)
    uint16_t* Ahi = Abuf + (size_t)(i & 1) * NPL * TILE;
    uint16_t* Alo = Ahi + (NPL - 1) * TILE;
    // K elements 4 q .. 4 q + 3 hold modes k3 = 2 q, 2 q + 1. Lanes of one row position in the
    // core matrices (t, t + 8, t + 16, t + 24) share shared-memory banks; the odd groups of 8
    // lanes store the two halves of each 16-byte chunk in the other order (selected values and
    // addresses, no branch), which halves the bank conflicts of these stores.
    const bool swap = (t >> 3) & 1;
#pragma unroll
    for (int q = 0; q < NP / 2; q += 2) {
      float4 x[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const float4 w4 = wv[(q + u) / 2];
        const float w0 = u ? w4.z : w4.x, w1 = u ? w4.w : w4.y;
        x[u] = make_float4(w0 * fv[q + u].x, w0 * fv[q + u].y, w1 * fv[q + u].z, w1 * fv[q + u].w);
      }
      put4(Ahi, Alo, t, 4 * (q + (swap ? 1 : 0)), K, swap ? x[1] : x[0], TERMS);
      put4(Ahi, Alo, t, 4 * (q + (swap ? 0 : 1)), K, swap ? x[0] : x[1], TERMS);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
      issue_product(taddr + (uint32_t)((i & 1) * 128), smem_addr(Ahi), smem_addr(Alo), smem_addr(Bhi),
                    smem_addr(Blo), K, NB, TERMS);
      tc::mma_commit(&bar_mma[i & 1]);
    }
    mma_next = i + 1;
    if (i + 1 < nt) load_rows(i + 1);  // in flight during the epilogue below
    if (i >= 1) {
      ok = wait_uniform(&bar_mma[(i - 1) & 1], (uint32_t)(((i - 1) >> 1) & 1), a.spin_max);
      if (!ok) break;
      mma_wait = i;
      epilogue(i - 1);
      tc::fence_before_sync();
      __syncthreads();
    }
  }
  if (ok && nt > 0) {
    ok = wait_uniform(&bar_mma[(nt - 1) & 1], (uint32_t)(((nt - 1) >> 1) & 1), a.spin_max);
    if (ok) {
      mma_wait = nt;
      epilogue(nt - 1);
    }
  }
  if (!ok) {
    if (t == 0) atomicOr(a.status, SGS_ST_TIMEOUT);
    drain(bar_mma, mma_wait, mma_next, a.spin_max);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(taddr, 256);
}

// ---- pass 2 (k2 -> x2): A tiles of Y1 (rows (b, x3, k1)) streamed by bulk copies into
// double-buffered operand buffers; two TMEM accumulators, so that the copy of tile i + 1 and
// the MMAs of tile i run while the epilogue of tile i - 1 writes the pass-3 operand Y2 (rows
// (b, x2, x3), K = (k1, re/im)).
template <int NP, int PP, int TERMS>
__global__ void __launch_bounds__(kTcRows) k_fast_pass2(FastArgs a) {
  constexpr int NPL = TERMS == 3 ? 2 : 1;  // BF16 planes of an operand (hi; lo for 3 products)
  extern __shared__ __align__(128) unsigned char smraw[];
  constexpr int K = 2 * NP, P = PP, NB = 2 * P;
  constexpr int TILE = kTcRows * K;  // elements of one operand plane tile
  uint16_t* Bhi = reinterpret_cast<uint16_t*>(smraw);
  uint16_t* Blo = Bhi + NB * K;
  uint16_t* Abuf = Blo + NB * K;  // [2 buffers][NPL planes][TILE]
  __shared__ __align__(8) uint64_t bar_ld[2], bar_mma[2];
  __shared__ uint32_t tslot;
  const int t = threadIdx.x, warp = t >> 5;
  if (warp == 0) tc::tmem_alloc(&tslot, 256);  // two accumulators of NB columns, 128 apart
  if (t == 0) {
    for (int j = 0; j < 2; j++) {
      mbar_init(&bar_ld[j], 1);
      mbar_init(&bar_mma[j], 1);
    }
    fence_mbar_init();
  }
  load_tile<K, NB>(a.bt12, NB, Bhi, Blo, 3);
  const long long rows = (long long)a.C * a.S * 2 * NP * P;  // rows (b, k1 < NP, x3) in y1_row order
  const long long tiles = (rows + kTcRows - 1) / kTcRows;
  const int nt = tiles > blockIdx.x ? (int)((tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;  // this CTA's tiles
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tslot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t plane_bytes = TILE * sizeof(uint16_t);
  auto issue_ld = [&](int i) {  // thread 0: the operand planes of this CTA's i-th tile
    const long long tile = blockIdx.x + (long long)i * gridDim.x;
    uint16_t* dst = Abuf + (size_t)(i & 1) * NPL * TILE;
    mbar_arrive_expect_tx(&bar_ld[i & 1], plane_bytes * NPL);
    bulk_g2s(dst, a.Y1h + tile * TILE, plane_bytes, &bar_ld[i & 1]);
    if (TERMS == 3) bulk_g2s(dst + TILE, a.Y1l + tile * TILE, plane_bytes, &bar_ld[i & 1]);
  };
  auto epilogue = [&](int i) {
    const long long r = (blockIdx.x + (long long)i * gridDim.x) * kTcRows + t;
    const bool live = r < rows;
    int b = 0, x3 = 0, k1 = 0;
    if (live) {
      b = (int)(r / (NP * P));
      const int rem = (int)(r % (NP * P));  // ((k1 / 4) * (P / 8) + x3 / 8) * 32 + (x3 % 8) * 4 + k1 % 4
      const int blk = rem >> 5, in = rem & 31;
      k1 = (blk / (P / 8)) * 4 + (in & 3);
      x3 = (blk % (P / 8)) * 8 + (in >> 2);
    }
    const uint32_t acc = taddr + lane_base + (uint32_t)((i & 1) * 128);
#pragma unroll
    for (int c0 = 0; c0 < NB; c0 += 16) {
      float v[16];
      tc::tmem_ld16(acc + (uint32_t)c0, v);
      if (live) {
#pragma unroll
        for (int q = 0; q < 16; q += 2) {
          const int x2 = (c0 + q) >> 1;
          store_pair(a.Y2h, a.Y2l, ((long long)b * P + x2) * P + x3, 2 * k1, K, v[q], v[q + 1], TERMS);
        }
      }
    }
  };
  int ld_next = 0, ld_wait = 0, mma_next = 0, mma_wait = 0;
  if (t == 0)
    for (int i = 0; i < 2 && i < nt; i++) issue_ld(i);
  ld_next = nt < 2 ? nt : 2;
  bool ok = true;
  for (int i = 0; i < nt; i++) {
    ok = wait_uniform(&bar_ld[i & 1], (uint32_t)((i >> 1) & 1), a.spin_max);
    if (!ok) break;
    ld_wait = i + 1;
    if (t == 0) {
      uint16_t* A = Abuf + (size_t)(i & 1) * NPL * TILE;
      issue_product(taddr + (uint32_t)((i & 1) * 128), smem_addr(A), smem_addr(A + (NPL - 1) * TILE), smem_addr(Bhi),
                    smem_addr(Blo), K, NB, TERMS);
      tc::mma_commit(&bar_mma[i & 1]);
    }
    mma_next = i + 1;
    if (i >= 1) {
      ok = wait_uniform(&bar_mma[(i - 1) & 1], (uint32_t)(((i - 1) >> 1) & 1), a.spin_max);
      if (!ok) break;
      mma_wait = i;
      // MMA i - 1 has read its operand buffer: the copy of tile i + 1 goes there
      if (i + 1 < nt) {
        if (t == 0) issue_ld(i + 1);
        ld_next = i + 2;
      }
      epilogue(i - 1);
      tc::fence_before_sync();
      __syncthreads();
    }
  }
  if (ok && nt > 0) {
    ok = wait_uniform(&bar_mma[(nt - 1) & 1], (uint32_t)(((nt - 1) >> 1) & 1), a.spin_max);
    if (ok) {
      mma_wait = nt;
      epilogue(nt - 1);
    }
  }
  if (!ok) {
    if (t == 0) atomicOr(a.status, SGS_ST_TIMEOUT);
    drain(bar_ld, ld_wait, ld_next, a.spin_max);
    drain(bar_mma, mma_wait, mma_next, a.spin_max);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(taddr, 256);
}

// ---- pass 3 (k1 -> x1): units (tile of rows (c, x2, x3), slot s); a unit's two operands
// (sides a = 0, 1 of b = (c, s, a)) are Y2 tiles, streamed by bulk copies into
// double-buffered operand buffers; its two products (real part of the transform) go to a
// TMEM accumulator pair, double-buffered like pass 2; the epilogue multiplies the two sides,
// weights the slot and sums the slots of the tile in registers, then adds the sum to G.
template <int NP, int PP, int TERMS>
__global__ void __launch_bounds__(kTcRows) k_fast_pass3(FastArgs a) {
  constexpr int NPL = TERMS == 3 ? 2 : 1;  // BF16 planes of an operand (hi; lo for 3 products)
  extern __shared__ __align__(128) unsigned char smraw[];
  constexpr int K = 2 * NP, P = PP, NB = P;
  constexpr int TILE = kTcRows * K;
  constexpr int TPC = P * P / kTcRows;  // tiles per cell (P^2 is a multiple of 128)
  uint16_t* Bhi = reinterpret_cast<uint16_t*>(smraw);
  uint16_t* Blo = Bhi + NB * K;
  uint16_t* Abuf = Blo + NB * K;  // [2 buffers][side 2][NPL planes][TILE]
  __shared__ __align__(8) uint64_t bar_ld[2], bar_mma[2];
  __shared__ uint32_t tslot;
  const int t = threadIdx.x, warp = t >> 5;
  if (warp == 0) tc::tmem_alloc(&tslot, 256);  // two accumulator pairs (sides at +0, +P), 128 apart
  if (t == 0) {
    for (int j = 0; j < 2; j++) {
      mbar_init(&bar_ld[j], 1);
      mbar_init(&bar_mma[j], 1);
    }
    fence_mbar_init();
  }
  load_tile<K, NB>(a.bt3, NB, Bhi, Blo, 3);
  const int S = a.S;
  const long long tiles = (long long)a.C * TPC;
  const int nt = tiles > blockIdx.x ? (int)((tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  const int nu = nt * S;  // units of this CTA: tile-major, slots inner
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tslot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t plane_bytes = TILE * sizeof(uint16_t);
  auto issue_ld = [&](int u) {  // thread 0
    const long long tile = blockIdx.x + (long long)(u / S) * gridDim.x;
    const int s = u % S;
    const long long c = tile / TPC, tin = tile % TPC;
    uint16_t* dst = Abuf + (size_t)(u & 1) * 2 * NPL * TILE;
    mbar_arrive_expect_tx(&bar_ld[u & 1], plane_bytes * 2 * NPL);
    for (int ab = 0; ab < 2; ab++) {
      const long long src = ((c * S + s) * 2 + ab) * TPC + tin;  // tile of b = (c, s, ab)
      bulk_g2s(dst + (size_t)ab * NPL * TILE, a.Y2h + src * TILE, plane_bytes, &bar_ld[u & 1]);
      if (TERMS == 3) bulk_g2s(dst + (size_t)ab * NPL * TILE + TILE, a.Y2l + src * TILE, plane_bytes, &bar_ld[u & 1]);
    }
  };
  float g[P];
#pragma unroll
  for (int q = 0; q < P; q++) g[q] = 0.0f;
  auto epilogue = [&](int u) {
    const int s = u % S;
    const float ws = a.wslot[a.s0 + s];
    const uint32_t acc = taddr + lane_base + (uint32_t)((u & 1) * 128);
#pragma unroll
    for (int c0 = 0; c0 < P; c0 += 16) {
      float va[16], vb[16];
      tc::tmem_ld16(acc + (uint32_t)c0, va);
      tc::tmem_ld16(acc + (uint32_t)(P + c0), vb);
#pragma unroll
      for (int q = 0; q < 16; q++) g[c0 + q] = fmaf(ws * va[q], vb[q], g[c0 + q]);
    }
    if (s == S - 1) {  // the tile's last slot: add the slot sum to G and start the next tile
      const long long tile = blockIdx.x + (long long)(u / S) * gridDim.x;
      float4* o = reinterpret_cast<float4*>(a.G + (tile * kTcRows + t) * P);
#pragma unroll
      for (int q = 0; q < P / 4; q++) {
        float4 v = o[q];
        v.x += g[4 * q];
        v.y += g[4 * q + 1];
        v.z += g[4 * q + 2];
        v.w += g[4 * q + 3];
        o[q] = v;
      }
#pragma unroll
      for (int q = 0; q < P; q++) g[q] = 0.0f;
    }
  };
  int ld_next = 0, ld_wait = 0, mma_next = 0, mma_wait = 0;
  if (t == 0)
    for (int u = 0; u < 2 && u < nu; u++) issue_ld(u);
  ld_next = nu < 2 ? nu : 2;
  bool ok = true;
  for (int u = 0; u < nu; u++) {
    ok = wait_uniform(&bar_ld[u & 1], (uint32_t)((u >> 1) & 1), a.spin_max);
    if (!ok) break;
    ld_wait = u + 1;
    if (t == 0) {
      uint16_t* A = Abuf + (size_t)(u & 1) * 2 * NPL * TILE;
      for (int ab = 0; ab < 2; ab++)
        issue_product(taddr + (uint32_t)((u & 1) * 128 + ab * P), smem_addr(A + (size_t)ab * NPL * TILE),
                      smem_addr(A + (size_t)ab * NPL * TILE + (NPL - 1) * TILE), smem_addr(Bhi), smem_addr(Blo), K,
                      NB, TERMS);
      tc::mma_commit(&bar_mma[u & 1]);
    }
    mma_next = u + 1;
    if (u >= 1) {
      ok = wait_uniform(&bar_mma[(u - 1) & 1], (uint32_t)(((u - 1) >> 1) & 1), a.spin_max);
      if (!ok) break;
      mma_wait = u;
      if (u + 1 < nu) {
        if (t == 0) issue_ld(u + 1);
        ld_next = u + 2;
      }
      epilogue(u - 1);
      tc::fence_before_sync();
      __syncthreads();
    }
  }
  if (ok && nu > 0) {
    ok = wait_uniform(&bar_mma[(nu - 1) & 1], (uint32_t)(((nu - 1) >> 1) & 1), a.spin_max);
    if (ok) {
      mma_wait = nu;
      epilogue(nu - 1);
    }
  }
  if (!ok) {
    if (t == 0) atomicOr(a.status, SGS_ST_TIMEOUT);
    drain(bar_ld, ld_wait, ld_next, a.spin_max);
    drain(bar_mma, mma_wait, mma_next, a.spin_max);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(taddr, 256);
}

// Compact FP32 spectrum of every cell, fhat = (ahat + bhat) / 2 (the transforms of f - M and
// f + M), zero-padded to npad along k2 and k3: out[c][k1][k2][k3][re, im].
__global__ void k_fast_fhat(const float2* __restrict__ ahat, const float2* __restrict__ bhat, int C, int n, int npad,
                            float* __restrict__ out) {
  const long long total = (long long)C * n * npad * npad;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int k3 = (int)(i % npad), k2 = (int)((i / npad) % npad), k1 = (int)((i / ((long long)npad * npad)) % n);
    const int c = (int)(i / ((long long)npad * npad * n));
    float2 v = make_float2(0.0f, 0.0f);
    if (k2 < n && k3 < n) {
      const long long o = ((((long long)(c / kLanes) * n + k1) * n + k2) * n + k3) * kLanes + (c % kLanes);
      v = make_float2(0.5f * (ahat[o].x + bhat[o].x), 0.5f * (ahat[o].y + bhat[o].y));
    }
    reinterpret_cast<float2*>(out)[i] = v;
  }
}

// Forward transform of G (real, [c][x2][x3][x1]) to the modes |k_i| <= h, times P^-3, in three
// separable passes in FP32 (G itself carries FP32 sums of BF16 products);
// tw[k][x] = exp(-2 pi i (k - h) x / P).
// pass A: T1[c][x2][x3][k1] = sum_x1 G e^{..k1 x1}; one warp per row (c, x2, x3)
__global__ void k_fast_final_a(const float* __restrict__ G, const float2* __restrict__ tw, int n, int P,
                               long long rows, float2* __restrict__ T1) {
  const long long cx = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (cx >= rows) return;
  const float* g = G + cx * P;
  for (int k = lane; k < n; k += 32) {
    float re = 0.0f, im = 0.0f;
    for (int x = 0; x < P; x++) {
      const float2 w = tw[k * P + x];
      const float gv = g[x];
      re = fmaf(w.x, gv, re);
      im = fmaf(w.y, gv, im);
    }
    T1[cx * n + k] = make_float2(re, im);
  }
}

// pass B: T2[c][x2][k3][k1] = sum_x3 T1[c][x2][x3][k1] e^{..k3 x3}
__global__ void k_fast_final_b(const float2* __restrict__ T1, const float2* __restrict__ tw, int n, int P,
                               float2* __restrict__ T2) {
  const long long cx2 = blockIdx.x;  // (c, x2)
  const float2* src = T1 + cx2 * P * n;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int k3 = i / n, k1 = i % n;
    float re = 0.0f, im = 0.0f;
    for (int x3 = 0; x3 < P; x3++) {
      const float2 w = tw[k3 * P + x3], v = src[x3 * n + k1];
      re = fmaf(w.x, v.x, fmaf(-w.y, v.y, re));
      im = fmaf(w.x, v.y, fmaf(w.y, v.x, im));
    }
    T2[cx2 * n * n + i] = make_float2(re, im);
  }
}

// pass C: qhat[g][k1][k2][k3][lane] = P^-3 sum_x2 T2[c][x2][k3][k1] e^{..k2 x2}; grid (C, blocks
// over the n^3 modes)
__global__ void k_fast_final_c(const float2* __restrict__ T2, const float2* __restrict__ tw, int n, int P,
                               float2* __restrict__ qhat) {
  const int c = blockIdx.x;
  const float scale = 1.0f / ((float)P * P * P);
  const int i = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= n * n * n) return;
  const int k1 = i / (n * n), k2 = (i / n) % n, k3 = i % n;
  float re = 0.0f, im = 0.0f;
  for (int x2 = 0; x2 < P; x2++) {
    const float2 w = tw[k2 * P + x2], v = T2[(((long long)c * P + x2) * n + k3) * n + k1];
    re = fmaf(w.x, v.x, fmaf(-w.y, v.y, re));
    im = fmaf(w.x, v.y, fmaf(w.y, v.x, im));
  }
  const long long o = ((((long long)(c / kLanes) * n + k1) * n + k2) * n + k3) * kLanes + (c % kLanes);
  qhat[o] = make_float2(re * scale, im * scale);
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Launchers of the fast operator.
// ---------------------------------------------------------------------------------------
cudaError_t launch_fast_fhat(const float2* ahat, const float2* bhat, int C, int n, int npad, float* out,
                             cudaStream_t st) {
  const long long total = (long long)C * n * npad * npad;
  k_fast_fhat<<<(int)std::min<long long>((total + 255) / 256, 152 * 8), 256, 0, st>>>(ahat, bhat, C, n, npad, out);
  return cudaGetLastError();
}

// CTAs per SM for a pass kernel: what its shared memory allows (the occupancy query can
// assume a smaller carveout) and what its TMEM columns allow (512 per SM); the tile loops are
// strided, so CTAs beyond the resident ones only wait for a slot.
static cudaError_t pass_grid(const void* kern, size_t smem, int tmem_cols, long long work, int* grid) {
  cudaError_t e = func_attr(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = func_attr(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int dev = 0, sms = 0, per = 0, sm_bytes = 0, reserved = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kTcRows, smem);
  if (e != cudaSuccess) return e;
  const int by_smem = sm_bytes / (int)(smem + 256 + (size_t)reserved);
  per = std::max(1, std::min(std::max(per, by_smem), 512 / tmem_cols));
  *grid = (int)std::max<long long>(1, std::min<long long>(work, (long long)sms * per));
  return cudaSuccess;
}

template <int NP, int PP, int TERMS>
static cudaError_t launch_passes_t(int pass, const FastArgs& a, cudaStream_t st) {
  constexpr int K = 2 * NP, TILE = kTcRows * K;
  constexpr int NPL = TERMS == 3 ? 2 : 1;  // operand planes: 1 product needs no lo buffers
  const long long B = (long long)a.C * a.S * 2;
  int grid = 0;
  cudaError_t e;
  if (pass == 1) {
    constexpr size_t smem = sizeof(uint16_t) * ((size_t)2 * 2 * PP * K + (size_t)2 * NPL * TILE);
    const long long tiles = (B * NP * NP + kTcRows - 1) / kTcRows;
    e = pass_grid((const void*)k_fast_pass1<NP, PP, TERMS>, smem, 256, tiles, &grid);
    if (e == cudaSuccess) k_fast_pass1<NP, PP, TERMS><<<grid, kTcRows, smem, st>>>(a);
  } else if (pass == 2) {
    constexpr size_t smem = sizeof(uint16_t) * ((size_t)2 * 2 * PP * K + (size_t)2 * NPL * TILE);
    const long long tiles = (B * PP * NP + kTcRows - 1) / kTcRows;
    e = pass_grid((const void*)k_fast_pass2<NP, PP, TERMS>, smem, 256, tiles, &grid);
    if (e == cudaSuccess) k_fast_pass2<NP, PP, TERMS><<<grid, kTcRows, smem, st>>>(a);
  } else {
    constexpr size_t smem = sizeof(uint16_t) * ((size_t)2 * PP * K + (size_t)2 * 2 * NPL * TILE);
    const long long tiles = (long long)a.C * PP * PP / kTcRows;
    e = pass_grid((const void*)k_fast_pass3<NP, PP, TERMS>, smem, 256, tiles, &grid);
    if (e == cudaSuccess) k_fast_pass3<NP, PP, TERMS><<<grid, kTcRows, smem, st>>>(a);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int NP, int PP>
static cudaError_t launch_passes_t(int pass, const FastArgs& a, cudaStream_t st) {
  return a.terms == 3 ? launch_passes_t<NP, PP, 3>(pass, a, st) : launch_passes_t<NP, PP, 1>(pass, a, st);
}

cudaError_t launch_fast_pass(int pass, const FastArgs& a, cudaStream_t st) {
  if (pass < 1 || pass > 3) return cudaErrorInvalidValue;
  if (a.npad == 16 && a.P == 32) return launch_passes_t<16, 32>(pass, a, st);
  if (a.npad == 32 && a.P == 32) return launch_passes_t<32, 32>(pass, a, st);
  if (a.npad == 32 && a.P == 48) return launch_passes_t<32, 48>(pass, a, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_fast_final(const float* G, const float2* tw, int C, int n, int P, float2* T1, float2* T2,
                              float2* qhat, cudaStream_t st) {
  const long long rows = (long long)C * P * P;
  k_fast_final_a<<<(int)((rows + 7) / 8), 256, 0, st>>>(G, tw, n, P, rows, T1);
  k_fast_final_b<<<C * P, 256, 0, st>>>(T1, tw, n, P, T2);
  k_fast_final_c<<<dim3(C, (n * n * n + 255) / 256), 256, 0, st>>>(T2, tw, n, P, qhat);
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
