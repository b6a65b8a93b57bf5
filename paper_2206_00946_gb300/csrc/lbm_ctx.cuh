// Internal: the context behind the opaque lbm_ctx handle, shared by the
// translation units of the library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "lbm.h"
#include "lbm_fused_plan.cuh"
#include "lbm_phases.cuh"

using namespace lbm;

struct AdjRec;  // recorded forward run of the discrete adjoint (lbm_adjoint.cu)
void adj_free(lbm_ctx* c);
int lbm_step_phases_internal(lbm_ctx* c);  // one step, one launch per phase

#define LBM_PROF_KINDS 6

// Slab-pipelined schedule: the lattice is cut into slabs of whole z-planes and
// every phase kernel runs per slab.  Stage (phase, slab) waits only for the
// stages of neighbouring slabs it reads, through events on a few streams, so
// the phases of different slabs overlap on the GPU and a slab's populations are
// read again (phase C) shortly after phase A read them, from L2.  Dependencies
// (s = slab, t = step): BC19(s) <- A(s-1..s+1) (force + D3Q19 pass);
// C7(s) <- BC19(s-1..s+1); D(s) <- BC19, C7 (s-1..s+1); and across steps
// A_t(s) <- BC19_{t-1}, C7_{t-1} (s-1..s+1), D_{t-1}(s).  Slabs hold at least
// three planes, so the inward neighbour of a face node lies in its own slab.
// A run of steps, and a single step, are captured once into CUDA graphs per
// buffer parity and replayed.
enum { SPH_A = 0, SPH_C19 = 1, SPH_C7 = 2, SPH_D = 3, SPH_N = 4 };
constexpr int kMaxSlabStreams = 8;

struct SlabPlan {
  int nslab = 0;
  std::vector<int> zb;                 // plane bounds of the slabs (nslab + 1)
  std::vector<int> order;              // stage codes phase * nslab + slab, topological
  std::vector<char> has_d;             // slab has boundary nodes
  int nstreams = 0;
  cudaStream_t st[kMaxSlabStreams] = {};
  std::vector<cudaEvent_t> ev;         // per stage code
  cudaEvent_t fork = nullptr, join[kMaxSlabStreams] = {};
  int graph_steps = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};   // graph_steps steps from buffer parity k
  cudaGraphExec_t graph1[2] = {nullptr, nullptr};  // one step from buffer parity k
};

struct lbm_ctx {
  lbm_params hp;
  Params P;
  cudaStream_t stream;
  int device;
  long long N;
  void* f[2];  // populations, element type per storage mode
  void* g[2];
  size_t esize;
  int cur;
  float* aux;
  float* hist;  // vartheta = 1: T at the two previous steps (2N floats, X.T1 and X.T2)
  float2* ref;  // FP16 storage with per-cell references: those of population buffer k at ref + k N
  Aux X;
  float* tface[6];
  long long tface_n[6];
  int* err_d;
  int* err_h;
  double* partial;
  double* red_out;
  double* red_h;
  int red_blocks;
  int grid;
  int stage19;      // force + D3Q19 with staged populations: tiles per CTA (0: off)
  int stage7;       // D3Q7 with staged populations: tiles per CTA (0: off)
  bool has_state;
  cudaStream_t side;  // second stream for the D3Q7 collision
  cudaEvent_t ev_fork, ev_join;
  SlabPlan* slabs;    // slab-pipelined schedule (LBM_SCHED_SLABS)
  // kernel timing: event pairs bracketing each launch while profiling is on
  bool profiling;
  struct Ev {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Ev>* evs;
  std::vector<cudaEvent_t>* pool;
  double prof_ms[LBM_PROF_KINDS];
  long long prof_n[LBM_PROF_KINDS];
  FusedPlan plan;
  AdjRec* adj;  // lbm_record / lbm_adjoint_step
};

