// Dispatch of the eigenvector product of Eq. (6) to its implementations (native
// FP64 with in-kernel Qhat tiles, or the split-precision tcgen05 path), and the
// workspace each implementation needs.
#pragma once

#include <vector>

#include "../../include/tdc.h"
#include "tdc_internal.cuh"

namespace tdc {

struct PathLevel {
  bool oz = false;
  bool hss = false;
  int gemm_cfg = 1;          // FP64 product tile shape (levels on the FP64 product)
  int64_t gemm_bound = 0;    // upper bound on its tiles (grid size)
  size_t tab_off = 0;        // OzJob array of the level in the table region
  size_t cum_off[3] = {0, 0, 0};
  int64_t nb[3] = {0, 0, 0}; // blocks: slice A, slice B, GEMM tiles
};

struct PathPlan {
  std::vector<PathLevel> levels;
  size_t arena_bytes = 0;    // slice arena (reused level after level)
  size_t table_bytes = 0;    // OzJob arrays + launch tables
  std::vector<uint64_t> table_store;   // host image of the table region (aligned below)
  unsigned char* table = nullptr;
  unsigned char* arena_dev = nullptr;
  unsigned char* table_dev = nullptr;
  int slices = 6;
};

// Merges of order below this use the FP64 product even on the split path.
constexpr int64_t kOzMinOrder = 256;

bool path_supported(const tdc_opts& o);
// Decides the product form per level and sizes its workspace (no device access).
void path_prepare(PathPlan& pp, const tdc_opts& o, const std::vector<const std::vector<MergeJob>*>& lv);
// Binds the carved device regions, encodes the tensor maps and uploads the tables.
bool path_bind(PathPlan& pp, unsigned char* arena, unsigned char* table_dev,
               const std::vector<const std::vector<MergeJob>*>& lv, cudaStream_t st);
// Launches the product for all merges of level l.  cum_tiles is the level's device
// scratch of njobs + 1 int64.  Returns 0, or 3 / 4 from the HSS path.
int launch_product(const PathPlan& pp, int l, const tdc_opts& o, const std::vector<MergeJob>& hjobs,
                   const MergeJob* jobs, int64_t* cum_tiles, QBufs qb, DevWs w, cudaStream_t st);

// FP64 product tile shapes per level.  The shape of a level is tile_cfg when that
// is >= 0; otherwise the autotuned choice recorded for the same level structure
// (tune_store), else a size rule (tile rows <= the merge halves, 32 or 64 columns).
void path_set_shape(PathPlan& pp, int l, int cfg, const std::vector<MergeJob>& jobs);
std::vector<int64_t> tune_key(const tdc_opts& o, const std::vector<const std::vector<MergeJob>*>& lv);
void tune_store(const std::vector<int64_t>& key, const std::vector<int>& cfg);
// While set, launch_product records an event pair around each FP64-product level.
struct LevelTimer {
  std::vector<cudaEvent_t> a, b;
  std::vector<bool> used;
};
void set_level_timer(LevelTimer* t);
void launch_copy_k(const MergeScalars* scal, int64_t* k_out, cudaStream_t st);

}  // namespace tdc
