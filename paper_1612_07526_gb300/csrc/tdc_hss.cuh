// HSS form of the eigenvector product (Algorithm 1 and the HSS multiply); see hss.cu.
#pragma once

#include <vector>

#include "../../include/tdc.h"
#include "tdc_internal.cuh"

namespace tdc {

struct HssCols {
  const double** col;         // kept-order columns of Q_sel, at the merge's row 0
  int32_t *lo, *hi;           // rows [lo, hi) where each can be nonzero
  int n1;
};

struct HIdJob {
  const double* phi;          // rows x rp, column-major, leading dimension ld
  int64_t ld;
  int rows;                   // static row count, or
  const int* rows_dev;        // device row count
  int rows_max;
  double* U;                  // rows x rank output, leading dimension rows_max
  int* rank_out;
  int* skel_local;
  double* scratch;            // rp x rows_max
};

struct HssNodeDev {
  int lo, hi, leaf, c1, c2, root;
  double *phi, *theta;        // Phi and Theta of the node (leading dimension ldphi)
  int64_t ldphi;
  double *U, *V;              // leading dimension ldU
  int64_t ldU;
  double *Yh, *Zh, *B;        // rp x rp blocks (leading dimension rp)
  double *G, *F;              // m x rp (multiply)
  int *I, *J;                 // global skeleton indices
  int *Iloc, *Jloc;           // local skeleton rows of Phi / Theta
  int *Icand, *Jcand;         // global indices of the parent's Phi / Theta rows
  int *kU, *kV, *rows_u, *rows_v;
};

size_t hss_arena_bytes(int64_t m, const tdc_opts& o);
// Runs Algorithm 1 and the HSS multiply for one merge whose deflation, roots,
// zhat and norms are in w; writes the K non-deflated output columns.  Reads K on the
// host (one stream synchronization).  Returns 0, 3 (arena too small) or 4.
// run_hss_merge's return when a node's ID rank reached the sample count (r + p) with
// more rows than samples: nothing has been written; the caller computes the merge's
// product densely instead.
constexpr int kHssSaturated = 100;
int run_hss_merge(const MergeJob& hJ, QBufs qb, DevWs w, unsigned char* arena, size_t arena_bytes,
                  const tdc_opts& o, cudaStream_t st);

}  // namespace tdc
