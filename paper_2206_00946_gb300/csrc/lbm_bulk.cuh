// Shared-memory staging of the populations with the Blackwell bulk-copy engine
// (cp.async.bulk, completion tracked by an mbarrier transaction count).
//
// A CTA owns a contiguous tile of T cells; the 26 population arrays (19 f, 7 g,
// structure of arrays) each contribute one contiguous segment of T floats, so a
// tile arrives as 26 one-dimensional bulk copies.  Tiles are double-buffered:
// while the CTA computes tile k from one buffer the copy engine fills the other
// with tile k+1, which keeps loads in flight during the long collision
// arithmetic.  Every wait on an mbarrier is bounded; on timeout the kernel
// raises ERRF_TIMEOUT, drains its own copies (again bounded) and returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_phases.cuh"

namespace lbm {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// one-dimensional global -> shared bulk copy; dst, src and bytes multiples of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ unsigned long long bulk_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait: false after ~1 s without completion
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = bulk_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (bulk_ns() - t0 > 1000000000ull) return false;
    __nanosleep(32);
  }
  return true;
}

// Issues the 26 segment copies of tile [c0, c0+n) into stage (19 + 7 rows of T floats).
template <int T>
__device__ __forceinline__ void stage_tile(const float* __restrict__ fA, const float* __restrict__ gA, long long N,
                                           int c0, int n, float* stage, uint64_t* bar) {
  const unsigned bytes = (unsigned)n * 4u;
  mbar_expect_tx(bar, 26u * bytes);
#pragma unroll 1
  for (int i = 0; i < 19; ++i) bulk_g2s(stage + i * T, fA + i * N + c0, bytes, bar);
#pragma unroll 1
  for (int i = 0; i < 7; ++i) bulk_g2s(stage + (19 + i) * T, gA + i * N + c0, bytes, bar);
}

// Phase C over the whole lattice with double-buffered bulk staging of the
// populations.  Requires N % 4 == 0 (16-byte aligned segments).
template <int T>
__global__ void __launch_bounds__(T) k_phaseC_bulk(Params P, const float* __restrict__ fA,
                                                    const float* __restrict__ gA, float* fB, float* gB, Aux X,
                                                    int* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* stage = reinterpret_cast<float*>(smem_raw);  // [2][26][T]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 2 * 26 * T * sizeof(float));
  __shared__ int s_fail;
  const int N = (int)P.N;
  const int ntiles = (N + T - 1) / T;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
    s_fail = 0;
  }
  __syncthreads();
  int tile = blockIdx.x;
  if (threadIdx.x == 0 && tile < ntiles) stage_tile<T>(fA, gA, P.N, tile * T, min(T, N - tile * T), stage, &bar[0]);
  int fail_k = -1, fail_next = 0;
  for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
    const int b = k & 1;
    const int next = tile + gridDim.x;
    if (threadIdx.x == 0 && next < ntiles) {
      fence_proxy_async();  // buffer b^1 was read by every thread before the last barrier
      stage_tile<T>(fA, gA, P.N, next * T, min(T, N - next * T), stage + (b ^ 1) * 26 * T, &bar[b ^ 1]);
    }
    if (!mbar_wait(&bar[b], (unsigned)(k >> 1) & 1u)) s_fail = 1;
    __syncthreads();
    if (s_fail) {
      fail_k = k;
      fail_next = next < ntiles;
      break;
    }
    const int c = tile * T + threadIdx.x;
    if (c < N) {
      const float* s = stage + b * 26 * T + threadIdx.x;
      float fl[19], gl[7];
#pragma unroll
      for (int i = 0; i < 19; ++i) fl[i] = s[i * T];
#pragma unroll
      for (int i = 0; i < 7; ++i) gl[i] = s[(19 + i) * T];
      phaseC_cell(P, c, fl, gl, gA, fB, gB, X);
    }
    __syncthreads();
  }
  if (fail_k >= 0 && threadIdx.x == 0) {
    // drain our own copies still in flight (bounded) before the CTA exits
    atomicOr(err, ERRF_TIMEOUT);
    mbar_wait(&bar[fail_k & 1], (unsigned)(fail_k >> 1) & 1u);
    if (fail_next) mbar_wait(&bar[(fail_k + 1) & 1], (unsigned)((fail_k + 1) >> 1) & 1u);
  }
}

}  // namespace lbm
