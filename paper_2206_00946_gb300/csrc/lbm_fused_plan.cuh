// Host-side plan of the persistent one-launch-per-step schedule (lbm_fused.cuh),
// separate from the kernel so that other translation units can hold one.
#pragma once

#include <vector>

namespace lbm {

enum { PH_A = 0, PH_B = 1, PH_C = 2, PH_D = 3 };

struct FusedPlan {
  int threads;           // threads per CTA
  int tile;              // cells per work item (multiple of threads)
  int tiles_per_plane;
  int nstages;
  int grid;              // persistent CTAs
  long long total_items;
  unsigned epoch;        // launches since the counters were cleared
  int* stages_d;         // [nstages] phase << 24 | z
  int* stage_first_d;    // [nstages] first item of each stage
  int* item_stage_d;     // [total_items] stage of each item
  std::vector<int> stage_first_h, item_stage_h;
  unsigned* done_d;      // [4 * nz] tiles finished per (phase, plane), cumulative over launches
  unsigned* ctr_d;       // dispatch counter, cumulative over launches
  int* abort_d;
  std::vector<int> stages_h;
};

}  // namespace lbm
