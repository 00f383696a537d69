// Batched dense FP64 GEMM on the FP64 pipe: C = alpha op(A) op(B) + beta C for a list of
// problems in one launch per operand layout (the backward's products Q^T G and Q M when
// the split-precision path is not selected); see dgemm.cu.
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace tdc {

// Element (r, c) of an operand: p[r + c ld] (column-major), or p[c + r ld] when trans
// (the transpose of a column-major array).
struct DMat {
  const double* p;
  int64_t ld;
  int trans;
};

struct DGemm {
  int M, N, K;
  DMat a, b;
  double* C;                  // column-major, leading dimension ldc
  int64_t ldc;
  double alpha, beta;
};

// Bytes of job table launch_dgemms stages for `njobs` problems.
size_t dgemm_table_bytes(size_t njobs);
// Stages the job tables at dev_tab + tab_off (advancing tab_off, within tab_bytes) and
// launches the products on st, one launch per combination of transposition flags.
// Returns 0, or 3 when the tables do not fit.
int launch_dgemms(const std::vector<DGemm>& g, unsigned char* dev_tab, size_t& tab_off, size_t tab_bytes,
                  cudaStream_t st);

}  // namespace tdc
