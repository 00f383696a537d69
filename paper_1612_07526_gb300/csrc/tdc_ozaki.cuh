// Split-precision (Ozaki-style) FP64 emulation of the eigenvector product of Eq. (6)
// on the bf16 tensor cores (tcgen05.mma kind::f16 with FP32 accumulation in TMEM).
//
// Splitting.  Every row r of Q_sel (restricted to the k-range its half uses) is
// scaled by a power of two sigma_r >= max_k |Q_sel[r, k]| and every column i of Qhat
// by tau_i >= max_k |Qhat[k, i]|.  The scaled values x in [-1, 1] are rounded to
// X = rint(x 2^(8S-1)) and written in balanced base 256:
//     x ~= sum_{p=1..S} 2^(-7-8(p-1)) a_p,   a_1 in [-128, 128], a_p in [-128, 127],
// each digit exact in bf16; the representation error is at most 2^(-8S) per entry.
// Then  (Q_sel Qhat)[r, i] = sigma_r tau_i sum_{p,q} 2^(-14-8(p+q-2)) (a_p . b_q)[r, i]
// and the sum is kept for levels L = p + q <= S + 2.
//
// Exactness.  |a_p b_q| <= 2^14, so a level-L sum of at most 4 pairs over 256 k is
// an integer of magnitude <= 2^24: levels 2..5 are accumulated in FP32 (exactly)
// over chunks of 256 k and each chunk is flushed into a 64-bit integer accumulator
// (LSB = the level-5 unit).  Levels 6..S+2 carry weights below 2^-46 relative and
// are accumulated in FP32 over the whole k range.
#pragma once

#include <cuda.h>

#include <vector>

#include "tdc_internal.cuh"

namespace tdc {

constexpr int kOzBM = 128;          // tile rows (one TMEM lane per row)
constexpr int kOzBN = 64;           // tile columns (one TMEM column block per level)
constexpr int kOzBK = 32;           // k per pipeline stage (64-byte swizzled rows)
constexpr int kOzChunk = 256;       // k per exact chunk
constexpr int kOzPad = 64;          // padding of the Gu groups in the k coordinate

struct OzJob {                      // CUtensorMap members force 64+ byte alignment
  CUtensorMap mapA[2];              // A slices of the T1 rows (0) and T2 rows (1)
  CUtensorMap mapB;                 // B slices (columns of Qhat)
  uint16_t* a[2];                   // a[h] + ((p * ldk / 32 + k / 32) * rows_h + r) * 32 + k % 32
  uint16_t* b;                      // b + ((q * ldk / 32 + k / 32) * m + i) * 32 + k % 32
  double* sigma;                    // per merge-local row: power-of-two row scale
  int32_t* texp;                    // per column: tau_i = 2^texp
  int64_t ldk;                      // padded k extent
  int32_t slices;
  int32_t pad_;
};

// Host side: bytes of the per-merge slice arena, and filling an OzJob for a merge
// whose arena starts at `base` (256-byte aligned).
size_t oz_job_bytes(const MergeJob& J, int slices);
bool oz_fill_job(OzJob& z, const MergeJob& J, unsigned char* base, int slices);

// Launches, for one level's merges, the schedule and slicing kernels (part 0) or the
// persistent tcgen05 GEMM (part 1).  cum_sb and cum_t are rewritten on the device from
// the merges' K; nb_sb and ntiles are host bounds (K = m) that size the grids.
void launch_ozaki_level(int part, const MergeJob* jobs, const OzJob* ozj, int njobs, const int64_t* cum_sa,
                        int64_t nb_sa, int64_t* cum_sb, int64_t nb_sb, int64_t* cum_t,
                        int64_t ntiles, int slices, QBufs qb, DevWs w, cudaStream_t st);
// bf16 slice products per FP64-equivalent product: pairs (p, q) with p + q <= S + 2.
int oz_slice_pairs(int slices);

// Products C = A B on the same split-precision tensor-core path (the backward's Q^T G and
// Q M; the HSS sampling and leaf-level products).  An operand is read element by element
// through one of these forms, (row, column) of the operand as the product uses it:
//   SG_DENSE     p[(r0 + row) + (c0 + col) ld]            (column-major)
//   SG_DENSE_T   p[(c0 + col) + (r0 + row) ld]            (the transpose of a column-major array)
//   SG_QHAT      wcol[c0 + col][r0 + row] sinv[c0 + col]  (the merge's Cauchy factor, generated)
//   SG_QHAT_T    wcol[r0 + row][c0 + col] sinv[r0 + row]  (its transpose)
//   SG_XCOLS     xcol[c0 + col][row] for xlo[c0 + col] <= row < xhi[c0 + col], else 0
//                (gathered eigenvector columns with their nonzero row ranges)
//   SG_STACK     [P P2]: p[(r0 + row) + col ld] for col < k1, else p2[(r0 + row) + (col - k1) ld2]
//   SG_STACK_ROWS [P; P2]: p[row + (c0 + col) ld] for row < k1, else p2[(row - k1) + (c0 + col) ld2]
//   SG_QHAT_RAW, SG_QHAT_T_RAW  SG_QHAT, SG_QHAT_T without the sinv factor (wcol only)
//   SG_DENSE_RS  SG_DENSE with row (r0 + row) scaled by rs[r0 + row]
// with k1 = *split (device).  In SG_DENSE_T, off_dev (optional, device) adds to c0.  In
// the SG_QHAT forms, lid (optional) gives a block index per Qhat index, and entries whose
// row and column share a block read as zero (Qhat without its diagonal blocks).
// C = alpha A B + beta C (or, with crow, C = diag(crow) A B), column-major with ldc, or through column pointers
// cptrs[cc0 + col][row].  Mdev, Ndev and Kdev (optional, device) hold the actual sizes
// (<= M, N, K): A's and B's entries past them count as zero, and C's rows and columns past
// them are not written.  A problem may name an earlier one of its batch with the same A
// (a_from), whose slices it then reads.  One call runs a batch: slicing of every A and B, then one
// persistent GEMM over all their tiles.  The workspace holds the slices (about
// 2 S (M + N) K bytes per problem) and the job table; split_gemm_bytes gives its size.
// Returns 0, -1 (an empty or null operand), 3 (workspace too small) or 4.
enum : int { SG_DENSE = 0, SG_DENSE_T = 1, SG_QHAT = 2, SG_QHAT_T = 3, SG_XCOLS = 4, SG_STACK = 5,
             SG_STACK_ROWS = 6, SG_QHAT_RAW = 7, SG_QHAT_T_RAW = 8, SG_DENSE_RS = 9 };
struct SgOp {
  int mode = SG_DENSE;
  int r0 = 0, c0 = 0;
  int k1 = 0;                       // resolved from split on the device
  const double* p = nullptr;
  int64_t ld = 0;
  const double* p2 = nullptr;
  int64_t ld2 = 0;
  const int* split = nullptr;
  const int* off_dev = nullptr;
  double* const* wcol = nullptr;
  const double* sinv = nullptr;
  const int32_t* lid = nullptr;
  const double* rs = nullptr;       // SG_DENSE_RS: row scales
  const double* const* xcol = nullptr;
  const int32_t* xlo = nullptr;
  const int32_t* xhi = nullptr;
};
struct SgProblem {
  int M = 0, N = 0, K = 0;
  SgOp a, b;
  double* C = nullptr;
  int64_t ldc = 0;
  double* const* cptrs = nullptr;
  int cc0 = 0;
  const int* Mdev = nullptr;
  const int* Ndev = nullptr;
  const int* Kdev = nullptr;
  double alpha = 1.0, beta = 0.0;
  const double* crow = nullptr;     // optional: C's row r scaled by crow[r] (with alpha = 1, beta = 0)
  int a_from = -1;            // an earlier problem of the batch with the same A (M, K, Mdev, Kdev): its slices are reused
};
inline SgOp sg_dense(const double* p, int64_t ld, bool trans = false) {
  SgOp o;
  o.mode = trans ? SG_DENSE_T : SG_DENSE;
  o.p = p;
  o.ld = ld;
  return o;
}
inline SgProblem sg_problem(int M, int N, int K, SgOp a, SgOp b, double* C, int64_t ldc) {
  SgProblem p;
  p.M = M;
  p.N = N;
  p.K = K;
  p.a = a;
  p.b = b;
  p.C = C;
  p.ldc = ldc;
  return p;
}
size_t split_gemm_bytes(const std::vector<SgProblem>& pr, int slices);
int split_gemm(const std::vector<SgProblem>& pr, int slices, unsigned char* ws, size_t ws_bytes, int* dev_err,
               cudaStream_t st);
// Units per job for the three launches (host).
int64_t oz_blocks_slice_a(const MergeJob& J);
int64_t oz_blocks_slice_b(const MergeJob& J);
int64_t oz_tiles(const MergeJob& J);

}  // namespace tdc
