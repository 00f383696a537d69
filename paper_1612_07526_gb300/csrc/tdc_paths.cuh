// Dispatch of the eigenvector product of Eq. (6) to its implementations, and the
// workspace each implementation needs.
#pragma once

#include <vector>

#include "../../include/tdc.h"
#include "tdc_internal.cuh"

namespace tdc {

struct PathSizes {
  size_t bytes = 0;          // extra workspace bytes of the chosen product path
};

struct PathWs {
  unsigned char* base = nullptr;
  size_t bytes = 0;
};

// Workspace of the product path for problems of order <= maxn whose largest merge
// has order maxm (nprob problems).
PathSizes path_sizes(const tdc_opts& o, int64_t maxn, int64_t maxm, int nprob);
// Carves the path workspace at base + *off (advancing *off); base may be null.
PathWs carve_paths(unsigned char* base, size_t& off, const PathSizes& ps);
bool path_supported(const tdc_opts& o);
// Launches the product for all merges of one level (host copy of the jobs in hjobs).
void launch_product(const tdc_opts& o, const std::vector<MergeJob>& hjobs, const MergeJob* jobs,
                    const int64_t* cum_tiles, int64_t ntiles, QBufs qb, DevWs w, PathWs pw,
                    cudaStream_t st);
void launch_copy_k(const MergeScalars* scal, int64_t* k_out, cudaStream_t st);

}  // namespace tdc
