// One launch per time step: a persistent kernel that runs the four per-cell
// phases (A macro, B force, C collide+stream, D boundary) of every z-plane as a
// software pipeline.  Work items are (phase, plane, tile) triples dispensed in
// a fixed order by an atomic counter; before an item runs, its CTA waits (with
// a bounded spin) until the planes it reads were finished by earlier items:
//   B(z) <- A(z-1..z+1),  C(z) <- B(z-1..z+1),  D(z) <- C(z-2..z+2).
// Every dependency points to an item dispensed earlier, so the CTA holding the
// earliest unfinished item can always proceed.  Because phase A of a plane runs
// only a few planes ahead of phase C of the same plane, C's second read of the
// populations is served from L2 and each population crosses HBM once per step.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <vector>

#include "lbm_fused_plan.cuh"
#include "lbm_phases.cuh"

namespace lbm {

struct FusedArgs {
  const float* fA;
  const float* gA;
  float* fB;
  float* gB;
  const int* stages;
  const int* stage_first;
  const int* item_stage;
  unsigned* done;
  unsigned* ctr;
  int* abort;
  int* err;
  int tile, tiles_per_plane, total_items, grid;
  unsigned base;         // counter value at the start of this launch
  unsigned epoch;
  long long timeout_ns;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__host__ __device__ inline bool plane_has_boundary(const Params& P, int z) {
  if (P.tface[0] || P.tface[1] || P.tface[2] || P.tface[3]) return true;
  return (P.tface[4] || P.tface[5]) && (z == 0 || z == P.nz - 1);
}

// Planes a stage reads from the previous phase: radius 1 for B and C, 2 for D.
__host__ __device__ inline int dep_radius(int ph) { return ph == PH_D ? 2 : (ph == PH_A ? -1 : 1); }

__host__ __device__ inline int dep_plane(const Params& P, int z, int k, bool& valid) {
  int q = z + k;
  valid = true;
  if (q < 0 || q >= P.nz) {
    if (P.face_kind[4] == FACE_PERIODIC)
      q = (q % P.nz + P.nz) % P.nz;
    else
      valid = false;
  }
  return q;
}

__device__ __forceinline__ int fetch_item(const FusedArgs& A) {
  const unsigned old = atomicAdd(A.ctr, 1u);
  const int item = (int)(old - A.base);
  return (item < 0 || item >= A.total_items) ? -1 : item;
}

#ifndef LBM_FUSED_MINBLOCKS
#define LBM_FUSED_MINBLOCKS 2
#endif

__global__ void __launch_bounds__(256, LBM_FUSED_MINBLOCKS) k_fused(Params P, Aux X, FusedArgs A) {
  __shared__ int s_next;
  __shared__ int s_ok;
  int err = 0;
  const int plane = P.nx * P.ny;
  if (threadIdx.x == 0) s_next = fetch_item(A);
  __syncthreads();
  int item = s_next;
  while (item >= 0) {
    __syncthreads();  // everyone has read s_next
    const int s = A.item_stage[item];
    const int t = item - A.stage_first[s];
    const int code = A.stages[s];
    const int ph = code >> 24, z = code & 0xffffff;
    if (threadIdx.x == 0) {
      // the next item is claimed now, so its dispatch latency overlaps this item's work
      s_next = *(volatile int*)A.abort ? -1 : fetch_item(A);
      int ok = 1;
      const int r = dep_radius(ph);
      if (r > 0) {
        const unsigned target = (A.epoch + 1u) * (unsigned)A.tiles_per_plane;
        const unsigned long long t0 = global_ns();
        for (int k = -r; k <= r && ok; ++k) {
          bool valid;
          const int q = dep_plane(P, z, k, valid);
          if (!valid) continue;
          const unsigned* cnt = A.done + (ph - 1) * P.nz + q;
          while ((int)(ld_acquire(cnt) - target) < 0) {
            if (*(volatile int*)A.abort) {
              ok = 0;
              break;
            }
            if ((long long)(global_ns() - t0) > A.timeout_ns) {
              atomicExch(A.abort, 1);
              atomicOr(A.err, ERRF_TIMEOUT);
              ok = 0;
              break;
            }
            __nanosleep(64);
          }
        }
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    if (ph == PH_D) {
      const int cnt = boundary_count(P, z);
      for (int k = t * A.tile + threadIdx.x; k < min(cnt, (t + 1) * A.tile); k += blockDim.x) {
        int x, y;
        boundary_xy(P, z, k, x, y);
        const int m = node_tfaces(P, x, y, z);
        if (m) phaseD(P, cell_of(P, x, y, z), x, y, z, m, A.fB, A.gB, X);
      }
    } else {
      const int c0 = z * plane + t * A.tile;
      const int c1 = min(c0 + A.tile, (z + 1) * plane);
      if (ph == PH_A) {
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) phaseA(P, c, A.fA, A.gA, X, nullptr, err);
      } else if (ph == PH_B) {
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) phaseB(P, c, X);
      } else {
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) phaseC(P, c, A.fA, A.gA, A.fB, A.gB, X);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(A.done + ph * P.nz + z, 1u);
    }
    item = s_next;
  }
  if (err) atomicOr(A.err, err);
}

// ---------------------------------------------------------------- host ------

// Orders the (phase, plane) stages topologically.  A stage becomes eligible
// once every stage it depends on was placed at least `gap` positions earlier,
// which leaves the in-flight window of CTAs room before anyone waits; later
// phases are preferred so that a plane's collision follows its macro pass
// after a short, bounded distance.
inline std::vector<int> fused_order(const Params& P, int gap) {
  const int nz = P.nz;
  std::vector<int> pos(4 * nz, -1);
  std::vector<char> exists(4 * nz, 1);
  int total = 0;
  for (int z = 0; z < nz; ++z) {
    if (!plane_has_boundary(P, z)) exists[PH_D * nz + z] = 0;
    for (int ph = 0; ph < 4; ++ph) total += exists[ph * nz + z];
  }
  std::vector<int> order;
  order.reserve(total);
  std::vector<int> next(4, 0);  // lowest plane not yet placed, per phase (scan start)
  auto ready = [&](int ph, int z, int g) {
    const int r = dep_radius(ph);
    if (r < 0) return true;
    for (int k = -r; k <= r; ++k) {
      bool valid;
      const int q = dep_plane(P, z, k, valid);
      if (!valid) continue;
      const int p = pos[(ph - 1) * nz + q];
      if (p < 0 || (int)order.size() - p < g) return false;
    }
    return true;
  };
  while ((int)order.size() < total) {
    int pick = -1;
    for (int pass = 0; pass < 2 && pick < 0; ++pass) {
      const int g = pass == 0 ? gap : 0;
      for (int ph = 3; ph >= 1 && pick < 0; --ph)
        for (int z = next[ph]; z < nz; ++z) {
          const int id = ph * nz + z;
          if (!exists[id] || pos[id] >= 0) continue;
          if (ready(ph, z, g)) {
            pick = id;
            break;
          }
        }
      if (pick < 0 && pass == 0) {
        for (int z = next[0]; z < nz; ++z)
          if (pos[z] < 0) {
            pick = z;
            break;
          }
      }
    }
    if (pick < 0) break;  // cannot happen: some stage is always ready
    pos[pick] = (int)order.size();
    order.push_back(((pick / nz) << 24) | (pick % nz));
    const int ph = pick / nz;
    while (next[ph] < nz && (pos[ph * nz + next[ph]] >= 0 || !exists[ph * nz + next[ph]])) ++next[ph];
  }
  return order;
}

// Tuning knobs (environment, read at lbm_init): LBM_FUSED_CPT = cells per
// thread of one work item, LBM_FUSED_GAP = minimum distance in stages between a
// stage and the stages it depends on (0 = one in-flight window).
inline int fused_plan(const Params& P, FusedPlan* plan, int threads = 256, int cells_per_thread = 4) {
  if (const char* e = std::getenv("LBM_FUSED_CPT")) cells_per_thread = std::max(1, std::atoi(e));
  plan->threads = threads;
  const long long plane = (long long)P.nx * P.ny;
  long long tile = (long long)threads * cells_per_thread;
  if (tile > plane) tile = ((plane + threads - 1) / threads) * threads;
  plan->tile = (int)tile;
  plan->tiles_per_plane = (int)((plane + tile - 1) / tile);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused, threads, 0);
  if (sms <= 0) sms = 1;
  if (per_sm <= 0) per_sm = 1;
  plan->grid = sms * per_sm;
  const int inflight_stages = (plan->grid + plan->tiles_per_plane - 1) / plan->tiles_per_plane;
  int gap = inflight_stages + 1;
  if (const char* e = std::getenv("LBM_FUSED_GAP")) {
    const int g = std::atoi(e);
    if (g > 0) gap = g;
  }
  plan->stages_h = fused_order(P, gap);
  plan->nstages = (int)plan->stages_h.size();
  plan->stage_first_h.assign(plan->nstages, 0);
  plan->item_stage_h.clear();
  long long items = 0;
  for (int s = 0; s < plan->nstages; ++s) {
    const int ph = plan->stages_h[s] >> 24, z = plan->stages_h[s] & 0xffffff;
    long long n = plan->tiles_per_plane;
    if (ph == PH_D) {
      const long long cnt = ((P.tface[4] || P.tface[5]) && (z == 0 || z == P.nz - 1)) ? plane : P.bd_perim;
      n = std::max(1LL, (cnt + tile - 1) / tile);
    }
    plan->stage_first_h[s] = (int)items;
    items += n;
    if (items > 0x3fffffffLL) return -1;
    for (long long k = 0; k < n; ++k) plan->item_stage_h.push_back(s);
  }
  plan->total_items = items;
  if ((long long)plan->grid > plan->total_items) plan->grid = (int)plan->total_items;
  plan->epoch = 0;
  plan->stages_d = nullptr;
  plan->stage_first_d = nullptr;
  plan->item_stage_d = nullptr;
  plan->done_d = nullptr;
  plan->ctr_d = nullptr;
  plan->abort_d = nullptr;
  return 0;
}

inline int fused_alloc(FusedPlan* plan, const Params& P, cudaStream_t s) {
  if (cudaMalloc(&plan->stages_d, sizeof(int) * plan->nstages) != cudaSuccess) return -2;
  if (cudaMalloc(&plan->stage_first_d, sizeof(int) * plan->nstages) != cudaSuccess) return -2;
  if (cudaMalloc(&plan->item_stage_d, sizeof(int) * plan->total_items) != cudaSuccess) return -2;
  if (cudaMemcpyAsync(plan->stage_first_d, plan->stage_first_h.data(), sizeof(int) * plan->nstages,
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return -2;
  if (cudaMemcpyAsync(plan->item_stage_d, plan->item_stage_h.data(), sizeof(int) * plan->total_items,
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return -2;
  if (cudaMalloc(&plan->done_d, sizeof(unsigned) * 4 * P.nz) != cudaSuccess) return -2;
  if (cudaMalloc(&plan->ctr_d, sizeof(unsigned)) != cudaSuccess) return -2;
  if (cudaMalloc(&plan->abort_d, sizeof(int)) != cudaSuccess) return -2;
  if (cudaMemcpyAsync(plan->stages_d, plan->stages_h.data(), sizeof(int) * plan->nstages, cudaMemcpyHostToDevice,
                      s) != cudaSuccess)
    return -2;
  if (cudaMemsetAsync(plan->done_d, 0, sizeof(unsigned) * 4 * P.nz, s) != cudaSuccess) return -2;
  if (cudaMemsetAsync(plan->ctr_d, 0, sizeof(unsigned), s) != cudaSuccess) return -2;
  if (cudaMemsetAsync(plan->abort_d, 0, sizeof(int), s) != cudaSuccess) return -2;
  if (cudaStreamSynchronize(s) != cudaSuccess) return -2;  // stages_h is pageable
  plan->epoch = 0;
  return 0;
}

inline int fused_reset(FusedPlan* plan, const Params& P, cudaStream_t s) {
  if (!plan->done_d) return 0;
  if (cudaMemsetAsync(plan->done_d, 0, sizeof(unsigned) * 4 * P.nz, s) != cudaSuccess) return -2;
  if (cudaMemsetAsync(plan->ctr_d, 0, sizeof(unsigned), s) != cudaSuccess) return -2;
  if (cudaMemsetAsync(plan->abort_d, 0, sizeof(int), s) != cudaSuccess) return -2;
  plan->epoch = 0;
  return 0;
}

inline int fused_step(FusedPlan* plan, const Params& P, const float* fA, const float* gA, float* fB, float* gB,
                      const Aux& X, int* err, cudaStream_t s) {
  FusedArgs a;
  a.fA = fA;
  a.gA = gA;
  a.fB = fB;
  a.gB = gB;
  a.stages = plan->stages_d;
  a.stage_first = plan->stage_first_d;
  a.item_stage = plan->item_stage_d;
  a.done = plan->done_d;
  a.ctr = plan->ctr_d;
  a.abort = plan->abort_d;
  a.err = err;
  a.tile = plan->tile;
  a.tiles_per_plane = plan->tiles_per_plane;
  a.total_items = (int)plan->total_items;
  a.grid = plan->grid;
  a.epoch = plan->epoch;
  a.base = (unsigned)((unsigned long long)plan->epoch * (unsigned long long)(plan->total_items + plan->grid));
  a.timeout_ns = 2000000000LL;
  k_fused<<<plan->grid, plan->threads, 0, s>>>(P, X, a);
  plan->epoch += 1;
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

inline void fused_free(FusedPlan* plan) {
  cudaFree(plan->stages_d);
  cudaFree(plan->stage_first_d);
  cudaFree(plan->item_stage_d);
  plan->stage_first_d = nullptr;
  plan->item_stage_d = nullptr;
  cudaFree(plan->done_d);
  cudaFree(plan->ctr_d);
  cudaFree(plan->abort_d);
  plan->stages_d = nullptr;
  plan->stage_first_d = nullptr;
  plan->item_stage_d = nullptr;
  plan->done_d = nullptr;
  plan->ctr_d = nullptr;
  plan->abort_d = nullptr;
}

inline int fused_launches(const FusedPlan*) { return 1; }

}  // namespace lbm
