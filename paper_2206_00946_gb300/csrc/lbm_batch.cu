// Batched stepping of many independent lattices of uneven size: one persistent
// cooperative launch per time step runs the four phases over a work list of
// tiles that spans every domain, with a grid-wide barrier between phases;
// runs of steps are replayed from a CUDA graph.  The launch shape (threads per
// CTA, CTAs per SM, cells per tile) comes from a measured autotuner.
//
// The batch schedules contexts made by lbm_init (FP32 storage); they keep
// their buffers and remain usable through the single-lattice entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_ctx.cuh"

namespace {

struct BatchDomain {
  float* f[2];
  float* g[2];
  Aux X;
  int* err;
};

struct BatchArgs {
  const Params* P;          // [D]
  const BatchDomain* dom;   // [D]
  const int4* tiles;        // (domain, c0, c1, -): cell ranges of the lattice phases
  const int4* btiles;       // (domain, k0, k1, -): face-node candidate ranges of phase D
  int ntiles, nbtiles;
  int cur;                  // buffer parity of the current state (shared by every domain)
  unsigned* bar;            // [0] arrivals, [1] generation
  int* abort;               // set when a barrier wait gave up
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch (every CTA is resident), with a
// bounded wait: after ~2 s without progress it raises the abort flag and
// returns false, and every CTA leaves the launch at its next barrier.
__device__ bool grid_barrier(unsigned* bar, int* abort) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire_u32(bar + 1);
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = now_ns();
      while (ld_acquire_u32(bar + 1) == gen) {
        if (*(volatile int*)abort) {
          ok = 0;
          break;
        }
        if (now_ns() - t0 > 2000000000ull) {
          atomicExch(abort, 1);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  __threadfence();
  return s_ok != 0;
}

// copy of the domain's parameters in shared memory for the CTA's tile
__device__ __forceinline__ void load_params(const Params* src, Params* dst) {
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Params) / sizeof(int)); i += blockDim.x) d[i] = s[i];
}

__global__ void __launch_bounds__(256) k_batch_step(BatchArgs A) {
  __shared__ Params sP;
  __shared__ BatchDomain sD;
  const int a = A.cur, b = 1 - A.cur;
  for (int ph = 0; ph < 4; ++ph) {
    const int n = ph == 3 ? A.nbtiles : A.ntiles;
    const int4* list = ph == 3 ? A.btiles : A.tiles;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
      const int4 tl = list[t];
      __syncthreads();  // the previous tile's threads are done with sP, sD
      load_params(A.P + tl.x, &sP);
      if (threadIdx.x == 0) sD = A.dom[tl.x];
      __syncthreads();
      int e = 0;
      for (int c = tl.y + threadIdx.x; c < tl.z; c += blockDim.x) {
        if (ph == 0) {
          phaseA<float>(sP, c, sD.f[a], sD.g[a], sD.X, nullptr, e, false);
        } else if (ph == 1) {
          phaseBC19<float>(sP, c, sD.f[a], sD.f[b], sD.X);
        } else if (ph == 2) {
          phaseC7<float>(sP, c, sD.g[a], sD.g[b], sD.X);
        } else {
          int x, y, z;
          boundary_candidate(sP, c, x, y, z);
          const int m = node_tfaces(sP, x, y, z);
          if (m) phaseD<float>(sP, cell_of(sP, x, y, z), x, y, z, m, sD.f[b], sD.g[b], sD.X);
        }
      }
      if (e) atomicOr(sD.err, e);
    }
    if (ph < 3 && !grid_barrier(A.bar, A.abort)) return;
  }
}

// One phase over every domain's tiles (grid-stride over the tile list); the
// launch boundary between phases replaces the grid barrier.
template <int PH>
__global__ void __launch_bounds__(256, 4) k_batch_phase(BatchArgs A) {
  __shared__ Params sP;
  __shared__ BatchDomain sD;
  const int a = A.cur, b = 1 - A.cur;
  const int n = PH == 3 ? A.nbtiles : A.ntiles;
  const int4* list = PH == 3 ? A.btiles : A.tiles;
  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    const int4 tl = list[t];
    __syncthreads();
    load_params(A.P + tl.x, &sP);
    if (threadIdx.x == 0) sD = A.dom[tl.x];
    __syncthreads();
    int e = 0;
    for (int c = tl.y + threadIdx.x; c < tl.z; c += blockDim.x) {
      if (PH == 0) {
        phaseA<float>(sP, c, sD.f[a], sD.g[a], sD.X, nullptr, e, false);
      } else if (PH == 1) {
        phaseBC19<float>(sP, c, sD.f[a], sD.f[b], sD.X);
      } else if (PH == 2) {
        phaseC7<float>(sP, c, sD.g[a], sD.g[b], sD.X);
      } else {
        int x, y, z;
        boundary_candidate(sP, c, x, y, z);
        const int m = node_tfaces(sP, x, y, z);
        if (m) phaseD<float>(sP, cell_of(sP, x, y, z), x, y, z, m, sD.f[b], sD.g[b], sD.X);
      }
    }
    if (e) atomicOr(sD.err, e);
  }
}

}  // namespace

struct lbm_batch {
  std::vector<lbm_ctx*> ctx;
  cudaStream_t stream = nullptr;
  Params* P_d = nullptr;
  BatchDomain* dom_d = nullptr;
  int4* tiles_d = nullptr;
  int4* btiles_d = nullptr;
  int ntiles = 0, nbtiles = 0;
  unsigned* bar_d = nullptr;
  int* abort_d = nullptr;
  int threads = 256, ctas_per_sm = 2, tile = 2048, grid = 0, nsm = 0;
  int mode = 0;  // 0: one persistent cooperative launch per step; 1: one launch per phase
  int cur = 0;
  int graph_steps = 8;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  long long cells = 0;
};

namespace {

int cst(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

void drop_graphs(lbm_batch* b) {
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) {
      cudaGraphExecDestroy(b->graph[k]);
      b->graph[k] = nullptr;
    }
}

// Tile lists for the current tile size; grid from the shape and the occupancy.
int build_tiles(lbm_batch* b) {
  std::vector<int4> t, bt;
  for (int d = 0; d < (int)b->ctx.size(); ++d) {
    const Params& P = b->ctx[d]->P;
    for (long long c0 = 0; c0 < P.N; c0 += b->tile)
      t.push_back(make_int4(d, (int)c0, (int)std::min<long long>(c0 + b->tile, P.N), 0));
    for (long long k0 = 0; k0 < P.bd_total; k0 += b->threads)
      bt.push_back(make_int4(d, (int)k0, (int)std::min<long long>(k0 + b->threads, P.bd_total), 0));
  }
  cudaFree(b->tiles_d);
  cudaFree(b->btiles_d);
  b->tiles_d = b->btiles_d = nullptr;
  int st = cst(cudaMalloc(&b->tiles_d, sizeof(int4) * std::max<size_t>(1, t.size())));
  if (!st) st = cst(cudaMalloc(&b->btiles_d, sizeof(int4) * std::max<size_t>(1, bt.size())));
  if (!st && !t.empty())
    st = cst(cudaMemcpy(b->tiles_d, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice));
  if (!st && !bt.empty())
    st = cst(cudaMemcpy(b->btiles_d, bt.data(), sizeof(int4) * bt.size(), cudaMemcpyHostToDevice));
  b->ntiles = (int)t.size();
  b->nbtiles = (int)bt.size();
  int occ = 0;
  if (!st) st = cst(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_step, b->threads, 0));
  if (!st && occ < 1) st = LBM_ERR_ARG;
  if (!st) b->grid = std::min(b->ctas_per_sm, occ) * b->nsm;
  drop_graphs(b);
  return st;
}

int launch_one(lbm_batch* b, cudaStream_t s) {
  BatchArgs A;
  A.P = b->P_d;
  A.dom = b->dom_d;
  A.tiles = b->tiles_d;
  A.btiles = b->btiles_d;
  A.ntiles = b->ntiles;
  A.nbtiles = b->nbtiles;
  A.cur = b->cur;
  A.bar = b->bar_d;
  A.abort = b->abort_d;
  if (b->mode == 1) {
    const int g = b->nsm * 8;
    k_batch_phase<0><<<g, b->threads, 0, s>>>(A);
    k_batch_phase<1><<<g, b->threads, 0, s>>>(A);
    k_batch_phase<2><<<g, b->threads, 0, s>>>(A);
    k_batch_phase<3><<<g, b->threads, 0, s>>>(A);
    b->cur = 1 - b->cur;
    return cst(cudaGetLastError());
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)b->grid);
  cfg.blockDim = dim3((unsigned)b->threads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the grid barriers cannot starve
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const int st = cst(cudaLaunchKernelEx(&cfg, k_batch_step, A));
  b->cur = 1 - b->cur;
  return st;
}

// every context's parity follows the batch's
void sync_parity(lbm_batch* b) {
  for (lbm_ctx* c : b->ctx) c->cur = b->cur;
}

int capture(lbm_batch* b) {
  const int parity = b->cur;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return LBM_ERR_CUDA;
  cudaGraph_t g = nullptr;
  int st = cst(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < b->graph_steps && !st; ++k) st = launch_one(b, cs);
  const cudaError_t e = cudaStreamEndCapture(cs, &g);
  b->cur = parity;
  if (!st && e == cudaSuccess && g) st = cst(cudaGraphInstantiate(&b->graph[parity], g, 0));
  else st = LBM_ERR_CUDA;
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  cudaGetLastError();
  return st;
}

}  // namespace

extern "C" int lbm_batch_create(lbm_batch** out, lbm_ctx* const* ctxs, int n) {
  if (!out || !ctxs || n < 1) return LBM_ERR_ARG;
  *out = nullptr;
  for (int d = 0; d < n; ++d) {
    const lbm_ctx* c = ctxs[d];
    if (!c || c->hp.storage != LBM_STORE_F32 || c->hp.vartheta || c->stream != ctxs[0]->stream) return LBM_ERR_ARG;
    if (!c->has_state) return LBM_ERR_STATE;
  }
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ERR_ARG;
  b->ctx.assign(ctxs, ctxs + n);
  b->stream = ctxs[0]->stream;
  b->cur = ctxs[0]->cur;
  int dev = 0;
  int st = cst(cudaGetDevice(&dev));
  if (!st) st = cst(cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev));
  // a context at the other parity moves its state to the batch's
  std::vector<Params> P(n);
  std::vector<BatchDomain> D(n);
  for (int d = 0; d < n && !st; ++d) {
    lbm_ctx* c = ctxs[d];
    if (c->cur != b->cur) {
      st = cst(cudaMemcpyAsync(c->f[b->cur], c->f[c->cur], 19ull * c->N * sizeof(float), cudaMemcpyDeviceToDevice,
                               b->stream));
      if (!st)
        st = cst(cudaMemcpyAsync(c->g[b->cur], c->g[c->cur], 7ull * c->N * sizeof(float),
                                 cudaMemcpyDeviceToDevice, b->stream));
      c->cur = b->cur;
    }
    P[d] = c->P;
    for (int k = 0; k < 2; ++k) {
      D[d].f[k] = static_cast<float*>(c->f[k]);
      D[d].g[k] = static_cast<float*>(c->g[k]);
    }
    D[d].X = c->X;
    D[d].err = c->err_d;
    b->cells += c->N;
  }
  if (!st) st = cst(cudaMalloc(&b->P_d, sizeof(Params) * n));
  if (!st) st = cst(cudaMalloc(&b->dom_d, sizeof(BatchDomain) * n));
  if (!st) st = cst(cudaMemcpy(b->P_d, P.data(), sizeof(Params) * n, cudaMemcpyHostToDevice));
  if (!st) st = cst(cudaMemcpy(b->dom_d, D.data(), sizeof(BatchDomain) * n, cudaMemcpyHostToDevice));
  if (!st) st = cst(cudaMalloc(&b->bar_d, 2 * sizeof(unsigned)));
  if (!st) st = cst(cudaMalloc(&b->abort_d, sizeof(int)));
  if (!st) st = cst(cudaMemset(b->bar_d, 0, 2 * sizeof(unsigned)));
  if (!st) st = cst(cudaMemset(b->abort_d, 0, sizeof(int)));
  if (!st) st = build_tiles(b);
  if (st) {
    lbm_batch_destroy(b);
    return st;
  }
  *out = b;
  return LBM_OK;
}

extern "C" int lbm_batch_step(lbm_batch* b, int n) {
  if (!b || n < 0) return LBM_ERR_ARG;
  int st = LBM_OK, done = 0;
  while (b->graph_steps > 0 && n - done >= b->graph_steps && !st) {
    if (!b->graph[b->cur]) st = capture(b);
    if (st) {  // graphs unavailable: launch directly from now on
      b->graph_steps = 0;
      st = LBM_OK;
      break;
    }
    st = cst(cudaGraphLaunch(b->graph[b->cur], b->stream));
    done += b->graph_steps;  // an even count: the parity returns
  }
  for (; done < n && !st; ++done) st = launch_one(b, b->stream);
  sync_parity(b);
  return st;
}

extern "C" int lbm_batch_sync(lbm_batch* b) {
  if (!b) return LBM_ERR_ARG;
  int ab = 0;
  if (cudaMemcpyAsync(&ab, b->abort_d, sizeof(int), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (ab) {
    // a barrier gave up: reset the barrier and the abort flag so that the batch can
    // step again once the caller has set the domains' states anew (they are partial)
    if (cudaMemsetAsync(b->bar_d, 0, 2 * sizeof(unsigned), b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->abort_d, 0, sizeof(int), b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
      return LBM_ERR_CUDA;
    return LBM_ERR_TIMEOUT;
  }
  for (lbm_ctx* c : b->ctx) {
    const int s = lbm_sync(c);
    if (s) return s;
  }
  return LBM_OK;
}

extern "C" long long lbm_batch_cells(const lbm_batch* b) { return b ? b->cells : 0; }

// Test support: the arrival counter of the grid barrier is set to the grid size,
// so that no arrival of the next persistent launch completes it (each CTA's wait
// gives up after its bound and the launch ends).
extern "C" int lbm_batch_inject_stall(lbm_batch* b) {
  if (!b || b->mode != 0) return LBM_ERR_ARG;
  const unsigned v[2] = {(unsigned)b->grid, 0u};
  return cst(cudaMemcpyAsync(b->bar_d, v, sizeof(v), cudaMemcpyHostToDevice, b->stream)) ||
                 cst(cudaStreamSynchronize(b->stream))
             ? LBM_ERR_CUDA
             : LBM_OK;
}

// Measured choice of the launch shape: every candidate (threads per CTA, CTAs
// per SM, cells per tile) runs a few timed steps; the fastest is kept.  The
// domains' states are saved before and restored after.
extern "C" int lbm_batch_tune(lbm_batch* b, int* threads, int* ctas_per_sm, int* tile_cells) {
  if (!b) return LBM_ERR_ARG;
  std::vector<float*> save(b->ctx.size(), nullptr);
  std::vector<int> errs(b->ctx.size(), 0);
  int st = cst(cudaStreamSynchronize(b->stream));
  for (size_t d = 0; d < b->ctx.size() && !st; ++d)
    st = cst(cudaMemcpy(&errs[d], b->ctx[d]->err_d, sizeof(int), cudaMemcpyDeviceToHost));
  for (size_t d = 0; d < b->ctx.size() && !st; ++d) {
    lbm_ctx* c = b->ctx[d];
    st = cst(cudaMalloc(&save[d], 26ull * c->N * sizeof(float)));
    if (!st) st = cst(cudaMemcpyAsync(save[d], c->f[b->cur], 19ull * c->N * sizeof(float), cudaMemcpyDeviceToDevice,
                                      b->stream));
    if (!st) st = cst(cudaMemcpyAsync(save[d] + 19 * c->N, c->g[b->cur], 7ull * c->N * sizeof(float),
                                      cudaMemcpyDeviceToDevice, b->stream));
  }
  const int cur0 = b->cur;
  const int th0 = b->threads, cp0 = b->ctas_per_sm, ti0 = b->tile;
  const int gs = b->graph_steps;
  b->graph_steps = 0;
  float best = 1e30f;
  const int mo0 = b->mode;
  int bt = th0, bc = cp0, bi = ti0, bm = mo0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!st) st = cst(cudaEventCreate(&e0));
  if (!st) st = cst(cudaEventCreate(&e1));
  const int TH[2] = {128, 256}, TI[4] = {1024, 2048, 4096, 8192};
  for (int mo = 0; mo < 2 && !st; ++mo)
  for (int a = 0; a < 2 && !st; ++a)
    for (int cp = 1; cp <= 4 && !st; ++cp)
      for (int ti = 0; ti < 4 && !st; ++ti) {
        if (mo == 1 && cp > 1) continue;  // the phased launches size their own grids
        b->mode = mo;
        b->threads = TH[a];
        b->ctas_per_sm = cp;
        b->tile = TI[ti];
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_step, b->threads, 0);
        if (mo == 0 && cp > occ) continue;
        st = build_tiles(b);
        for (int w = 0; w < 2 && !st; ++w) st = launch_one(b, b->stream);
        if (!st) st = cst(cudaEventRecord(e0, b->stream));
        for (int k = 0; k < 4 && !st; ++k) st = launch_one(b, b->stream);
        if (!st) st = cst(cudaEventRecord(e1, b->stream));
        if (!st) st = cst(cudaEventSynchronize(e1));
        float ms = 0.f;
        if (!st) st = cst(cudaEventElapsedTime(&ms, e0, e1));
        if (!st && ms < best) {
          best = ms;
          bt = b->threads;
          bc = b->ctas_per_sm;
          bi = b->tile;
          bm = b->mode;
        }
      }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  b->threads = bt;
  b->ctas_per_sm = bc;
  b->tile = bi;
  b->mode = bm;
  b->graph_steps = gs;
  const int st2 = build_tiles(b);
  if (!st) st = st2;
  // restore the states at the original parity
  b->cur = cur0;
  for (size_t d = 0; d < b->ctx.size(); ++d) {
    lbm_ctx* c = b->ctx[d];
    if (save[d] && !st) {
      st = cst(cudaMemcpyAsync(c->f[cur0], save[d], 19ull * c->N * sizeof(float), cudaMemcpyDeviceToDevice,
                               b->stream));
      if (!st)
        st = cst(cudaMemcpyAsync(c->g[cur0], save[d] + 19 * c->N, 7ull * c->N * sizeof(float),
                                 cudaMemcpyDeviceToDevice, b->stream));
    }
  }
  cudaStreamSynchronize(b->stream);
  for (float* p : save) cudaFree(p);
  // the timing steps' error flags belong to no step of the caller's run
  for (size_t d = 0; d < b->ctx.size() && !st; ++d)
    st = cst(cudaMemcpy(b->ctx[d]->err_d, &errs[d], sizeof(int), cudaMemcpyHostToDevice));
  if (!st) st = cst(cudaMemset(b->bar_d, 0, 2 * sizeof(unsigned)));
  if (!st) st = cst(cudaMemset(b->abort_d, 0, sizeof(int)));
  sync_parity(b);
  if (threads) *threads = b->threads;
  if (ctas_per_sm) *ctas_per_sm = b->mode == 1 ? 0 : b->ctas_per_sm;  // 0: one launch per phase
  if (tile_cells) *tile_cells = b->tile;
  return st;
}

extern "C" void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  cudaFree(b->P_d);
  cudaFree(b->dom_d);
  cudaFree(b->tiles_d);
  cudaFree(b->btiles_d);
  cudaFree(b->bar_d);
  cudaFree(b->abort_d);
  delete b;
}
