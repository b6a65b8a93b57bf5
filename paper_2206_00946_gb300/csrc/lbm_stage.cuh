// Shared-memory staging of the populations of the force + D3Q19 and D3Q7 passes, with the
// bulk-copy engine (cp.async.bulk; completion tracked by an mbarrier transaction count).
//
// A CTA of kStageT threads works through tiles of kStageT consecutive cells.  In the
// structure-of-arrays layout each population array holds a tile as one contiguous segment,
// so a tile arrives as 19 (D3Q19) or 7 (D3Q7) one-dimensional bulk copies issued by one
// thread.  Tiles are double-buffered: while the CTA computes tile k from one buffer, the
// copy engine fills the other with tile k+1, so the HBM latency of the cell's own
// populations overlaps the stencils, the collision and the push of the tile before.  The
// stencil reads (psi, u, the destinations of the relaxed push) stay plain loads.
//
// Every wait on an mbarrier is bounded (about one second).  On a timeout the kernel raises
// ERRF_TIMEOUT, waits (again bounded) for the copies it issued and returns.  A bulk copy of a
// valid global range into the CTA's own shared memory always completes, so a wait runs out
// only when the barrier expects more bytes than its copies bring (the stall that
// lbm_inject_stall requests); every copy issued has then landed before the CTA exits.  The
// drain is bounded all the same, so that no CTA can wait forever.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_phases.cuh"

namespace lbm {

constexpr int kStageT = kStaged;  // cells per tile = threads per CTA

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

// one-dimensional global -> shared bulk copy; both addresses and the size multiples of 16 B
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// orders this CTA's generic-proxy reads of a buffer before the next bulk copy into it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ unsigned long long stage_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait for the phase `parity` of bar: false after about one second
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = stage_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (stage_ns() - t0 > 1000000000ull) return false;
    __nanosleep(32);
  }
  return true;
}

// The NR segment copies of the tile starting at cell c (kStageT cells) into `buf`
// ([NR][kStageT] stored populations).
// (extra: bytes expected beyond the copies, nonzero only for an injected stall)
template <typename ST, int NR>
__device__ __forceinline__ void stage_tile(const ST* __restrict__ src, long long N, int c, ST* buf, uint64_t* bar,
                                           unsigned extra = 0) {
  constexpr unsigned bytes = kStageT * sizeof(ST);
  mbar_expect_tx(bar, NR * bytes + extra);
#pragma unroll 1
  for (int i = 0; i < NR; ++i) bulk_g2s(buf + i * kStageT, src + i * N + c, bytes, bar);
}

// The cells [c0, c1) in tiles of kStageT, with the NR population rows of each tile staged in
// shared memory (double-buffered) before body(c, x, y, z, s) runs for the thread's cell, s
// pointing at its population 0 (population i at s[i * kStageT]).  Requires (c1 - c0) and c0
// multiples of kStageT and N * sizeof(ST) a multiple of 16.  Dynamic shared memory:
// 2 * NR * kStageT * sizeof(ST) + 16 bytes.
template <typename ST, int NR, typename Body>
__device__ __forceinline__ void staged_tiles(const Params& P, const ST* __restrict__ src, int c0, int c1, int* err,
                                             Body body) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  ST* stage = reinterpret_cast<ST*>(smem_raw);  // [2][NR][kStageT]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 2 * NR * kStageT * sizeof(ST));
  __shared__ int s_fail;
  const int ntiles = (c1 - c0) / kStageT;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
    s_fail = 0;
  }
  __syncthreads();
  int tile = blockIdx.x;
  if (threadIdx.x == 0 && tile < ntiles) {
    // a stall request (failure-detection tests; the int after the error flags) is taken by
    // the first CTA 0 that sees it
    const unsigned extra = (blockIdx.x == 0 && atomicExch(err + 1, 0) != 0) ? 16u : 0u;
    stage_tile<ST, NR>(src, P.N, c0 + tile * kStageT, stage, &bar[0], extra);
  }
  int fail_k = -1, fail_next = 0;
  for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
    const int b = k & 1;
    const int next = tile + gridDim.x;
    if (threadIdx.x == 0 && next < ntiles) {
      fence_proxy_async();  // buffer b^1 was read by every thread before the last barrier
      stage_tile<ST, NR>(src, P.N, c0 + next * kStageT, stage + (b ^ 1) * NR * kStageT, &bar[b ^ 1]);
    }
    if (!mbar_wait(&bar[b], (unsigned)(k >> 1) & 1u)) s_fail = 1;
    __syncthreads();
    if (s_fail) {
      fail_k = k;
      fail_next = next < ntiles;
      break;
    }
    const int c = c0 + tile * kStageT + threadIdx.x;
    int x, y, z;
    cell_xyz(P, c, x, y, z);
    body(c, x, y, z, stage + b * NR * kStageT + threadIdx.x);
    __syncthreads();
  }
  if (fail_k >= 0 && threadIdx.x == 0) {
    // the copies this CTA issued and has not seen complete: wait for them (bounded) before
    // the CTA's shared memory is released
    atomicOr(err, ERRF_TIMEOUT);
    mbar_wait(&bar[fail_k & 1], (unsigned)(fail_k >> 1) & 1u);
    if (fail_next) mbar_wait(&bar[(fail_k + 1) & 1], (unsigned)((fail_k + 1) >> 1) & 1u);
  }
}

// err: the context's error flags, followed by its stall request (see lbm_inject_stall).
// Force + D3Q19 over [c0, c1) with the 19 populations staged
template <typename ST>
__global__ void __launch_bounds__(kStageT, 4) k_phaseBC19_staged(Params P, const ST* __restrict__ fA, ST* fB,
                                                                 AuxFor<ST> X, int c0, int c1, int* err) {
  staged_tiles<ST, 19>(P, fA, c0, c1, err, [&](int c, int x, int y, int z, const ST* s) {
    phaseBC19<ST, true>(P, c, x, y, z, fA, fB, X, s);
  });
}

// D3Q7 collision + relaxed push over [c0, c1) with the cell's 7 populations staged
template <typename ST, int VT>
__global__ void __launch_bounds__(kStageT, 4) k_phaseC7_staged(Params P, const ST* __restrict__ gA, ST* gB,
                                                               AuxFor<ST> X, int c0, int c1, int* err) {
  staged_tiles<ST, 7>(P, gA, c0, c1, err, [&](int c, int x, int y, int z, const ST* s) {
    phaseC7_staged<ST, VT>(P, c, x, y, z, s, gA, gB, X);
  });
}

}  // namespace lbm
