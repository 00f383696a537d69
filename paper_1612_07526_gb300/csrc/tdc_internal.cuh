// Internal types and device helpers shared by the CUDA translation units of libtdc.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tdc {

constexpr double kEps = 1.1102230246251565e-16;     // 2^-53, unit roundoff
constexpr double kInvSqrt2 = 0.7071067811865476;    // correctly rounded 1/sqrt(2)

// Device status bits (OR-ed into the status word).
enum : int { ST_SECULAR = 1, ST_NONFINITE = 2, ST_LEAF = 4, ST_WAIT = 8 };

// Per-sorted-position flags written by the deflation kernel.
enum : int { F_T1 = 1, F_T2 = 2, F_ROT = 4 };

// Eigenvector storage.  A problem's top merge (or its only leaf) writes the caller's
// array in sorted order.  Everything below lives in the problem's pool: three n x n
// column blocks (ld n) in the workspace, 3n physical columns.  A slot table gives,
// for every eigenpair slot v of a problem (the eigenpair's index in its node's sorted
// order, offset by the node's first index), the column holding its eigenvector: a
// pointer to the column's row 0 of the problem and the rows [lo, hi) where it can be
// nonzero (the node that produced it).  A deflated column keeps its storage at every
// level above, so only the top merge moves it.

// One leaf of the DC tree: an nl x nl tridiagonal block.
struct LeafJob {
  int64_t v_off;     // first index of the leaf in the d / e / lambda vectors and the slot table
  int64_t q_off;     // element offset of the leaf block (0,0) in its output array
  int32_t ld;        // leading dimension of that array
  int32_t buf;       // 0: the caller's output (the leaf is a whole problem), 1: the pool
  int32_t nl;        // leaf order (1..32)
  int32_t prob;      // problem index
  int32_t root;      // 1 if the leaf is the whole problem (sign convention applied)
  int32_t lo;        // first row of the leaf within its problem
};

// One rank-one merge (Eqs. 3-6) of rows / columns [lo, lo + n1 + n2) of a problem.
struct MergeJob {
  int64_t v_off;     // first index of the merged block in the vectors and the slot table
  int64_t out_off;   // final merges: element offset of block (0,0) in the caller's output
  int64_t ld_out;    // leading dimension of the caller's output
  int64_t pool_off;  // element offset of the problem's pool (3n columns of n rows)
  int64_t in_off;    // ext merges: element offset of the caller's input block (0,0)
  int64_t ld_in;     // ext merges: its leading dimension
  int32_t pn;        // problem order n (the pool's leading dimension)
  int32_t lo;        // first row / column of the merge within its problem
  int32_t n1, n2;
  int32_t prob;
  int32_t fin;       // 1: outputs go to the caller's array in sorted order
  double beta;       // coupling entry b_k, used when e_idx < 0
  int64_t e_idx;     // index of b_k in the e vector, or -1
  int64_t mid;       // merge id (index into the per-merge scalars)
  int32_t root;      // 1: the output gets the sign convention (a problem's top merge)
  int32_t ext;       // 1: the inputs are the caller's block-diagonal Q (tdc_merge), not the slot table
};

// A problem of a batch as the persistent kernel sees it (the plan lists these largest
// first): its vectors, leaves, tear points and merges (in bottom-up level order).
struct PersistProb {
  int64_t v0, n;         // first index and order
  int64_t leaf0;         // first of its leaves in the plan's leaf list
  int64_t tear0, tear1;  // its tear points in the plan's tear list
  int64_t merge0;        // first of its merges in the persistent merge list
  int32_t nleaf, nmerge;
};

struct MergeScalars {
  int32_t K;         // non-deflated count
  int32_t c1, c3;    // Gu groups: columns touching rows of T1 only / both halves
  int32_t nd;        // deflated count
  int32_t nrot;      // plane rotations applied
  int32_t sorted;    // 1 if the deflated values came out ascending
  int32_t nchain;    // chains of rotations sharing a column
  int32_t pad_;
  double rho;        // 2 |beta|
  double tol;        // deflation tolerance
  unsigned long long evals;   // secular-function evaluations over the merge's roots
  unsigned long long live;    // rows the deflated columns can be nonzero in, summed
  unsigned long long mxbits;  // max(|d|, |z|) as magnitude bits (zeroed per solve)
  unsigned long long pad2_;
};

// Device workspace arrays; per-index arrays are addressed at job.v_off.
struct DevWs {
  double *ds, *zs;            // sorted d and z (updated by rotations)
  double *dbar, *zbar;        // non-deflated (K) values
  float2 *dbar32;             // d as FP32 pairs (hi, lo), d = hi + lo (the secular solver's FP32 phase)
  float *zbar32;              // z in FP32
  double *zhat, *tau, *sinv, *cmax;
  double *taulo;              // extended-precision eigenvectors: the roots' low parts (tau + taulo)
  double *lamnd;              // non-deflated eigenvalues d_org + tau
  double *dv;                 // deflated eigenvalues (sorted-position order)
  double *skey;               // 2n scratch keys for the fallback sort
  int32_t *srcs, *typ, *flag, *ev, *cand, *slot;
  int32_t *kidx, *kperm, *org, *dsrc, *dperm, *posK, *posD;
  int32_t *sval;              // 2n scratch values for the fallback sort
  const double **colptr;      // grouped (Gu order) non-deflated columns, at the merge's row 0
  const double **dcolptr;     // deflated columns, at the merge's row 0
  int32_t *klo, *khi;         // rows [klo, khi) of colptr[k] that can be nonzero (merge rows)
  int32_t *dlo, *dhi;         // the same for dcolptr[a]
  double **outptr;            // output column of kept eigenpair i, at the merge's row 0
  double **wptr;              // column i of the Cauchy factor zhat_j / (d_j - lambda_i), j < K (unscaled)
  const double **tptr;        // slot table: column pointer at the problem's row 0
  int32_t *tlo, *thi;         // slot table: nonzero rows [tlo, thi) (problem rows)
  int32_t *rj, *rk;           // rotation records (sorted positions)
  int32_t *chain;             // first rotation of each chain
  double *rc, *rs;
  MergeScalars *scal;         // per merge id
  unsigned long long *lroots; // per tree level: non-deflated roots of the level's merges, then (at
                              // kMaxLevels + level) the level's largest K (2 kMaxLevels)
  double *dmod;               // torn diagonal (Eq. 2 corner updates)
  double2 *lrot;              // leaf QL: recorded plane rotations (c, s), kLeafRot per leaf
  uint8_t *lroti;             // leaf QL: row index i of each rotation (rows i, i+1)
  int32_t *lrotn;             // leaf QL: rotations recorded, or -1: redo the leaf serially
  int *status;                // per problem
  int32_t ext;                // 1: extended-precision eigenvectors (tdc_opts.eigvec), else Loewner z
};

constexpr int kMaxLevels = 64;   // merge levels of one plan (log2 of the largest n / leaf, plus one)
constexpr int kLeafRot = 2048;   // rotations recorded per leaf (a 32-leaf needs about 1300)

struct QBufs {
  double *A;                  // the caller's output array
  double *P;                  // the pools (workspace)
  const double *In;           // ext merges: the caller's input array
};

// Input column j (0 <= j < n1 + n2, the children's sorted order) of a merge: a
// pointer at the merge's row 0 and the merge rows [lo, hi) where it can be nonzero.
struct ColRef {
  const double* p;
  int lo, hi;
};
__device__ __forceinline__ ColRef merge_input(const MergeJob& J, const QBufs& qb, const DevWs& w, int j) {
  ColRef c;
  const int m = J.n1 + J.n2;
  if (J.ext) {
    c.p = qb.In + J.in_off + (int64_t)j * J.ld_in;
    c.lo = j < J.n1 ? 0 : J.n1;
    c.hi = j < J.n1 ? J.n1 : m;
  } else {
    const int64_t v = J.v_off + j;
    c.p = w.tptr[v] + J.lo;
    c.lo = max(w.tlo[v] - J.lo, 0);
    c.hi = min(w.thi[v] - J.lo, m);
  }
  return c;
}
// Column pc (0 <= pc < 3n) of the merge's problem pool, at the merge's row 0.
__device__ __forceinline__ double* pool_col(const MergeJob& J, const QBufs& qb, int pc) {
  return qb.P + J.pool_off + (int64_t)pc * J.pn + J.lo;
}
// Pool column of a pointer at the merge's row 0, or -1 outside this problem's pool.
__device__ __forceinline__ int pool_index(const MergeJob& J, const QBufs& qb, const double* p) {
  const double* base = qb.P + J.pool_off + J.lo;
  if (p < base) return -1;
  const int64_t d = p - base;
  // d / pn without a 64-bit division: a float estimate (d < 3 pn^2 < 2^63, so it is off
  // by at most one), corrected with integer products
  const int64_t pn = J.pn;
  if (d >= 3 * pn * pn) return -1;
  int64_t q = (int64_t)((float)d * (1.0f / (float)pn));
  if (q * pn > d) --q;
  else if ((q + 1) * pn <= d) ++q;
  if (q < 0 || q * pn != d || q >= 3 * pn) return -1;
  return (int)q;
}

// Smallest j with cum[j+1] > b (cum has njobs+1 entries, cum[0] = 0).
__device__ __forceinline__ int find_job(const int64_t* __restrict__ cum, int njobs, int64_t b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (cum[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_prod(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Profiling hook (defined in api.cu): brackets a phase with CUDA events when the
// per-phase timing of tdc_profile_begin() is on; a no-op otherwise.
void phase_mark(int phase, bool begin, int nlaunch, cudaStream_t st);
// Phase id of tree level l's FP64 product (kLevelMark + l): timed per level.
constexpr int kLevelMark = 100;
// Event marks around one launch of the dense split GEMM kernel (begin carries the
// launch's bf16 slice-pair flops); summed into tdc_profile's sg_gemm fields.
void sg_gemm_mark(bool begin, double tensor_flops, cudaStream_t st);
// Counts HSS merges that fell back to the dense product (while profiling is on).
void hss_fallbacks_add(int n);
// Counts HSS compressions repeated with a doubled sample (while profiling is on).
void hss_regrowths_add(int n);
// Adds the sampling flops of one HSS compression (while profiling is on).
void hss_sampling_flops_add(double f);
// While an object constructed with `on` = true lives, phase_mark records nothing on
// the constructing thread (no CUDA events are created).
struct ProfileSuspend {
  explicit ProfileSuspend(bool on);
  ~ProfileSuspend();
  ProfileSuspend(const ProfileSuspend&) = delete;
  ProfileSuspend& operator=(const ProfileSuspend&) = delete;

 private:
  bool prev_;
};

// Grid size for a grid-stride kernel: min(nb, SMs x per_sm), at least 1.
unsigned grid_cap(int64_t nb, int per_sm);

// Kernel launchers (defined in the .cu files; all asynchronous on `st`).
void launch_tear(const int64_t* tear_list, const int64_t* tear_ptr, int nprob, int64_t ntear, int leaf,
                 const double* d, const double* e, double* dmod, int64_t ntot, cudaStream_t st);
void launch_leaves(const LeafJob* jobs, int njobs, const double* dmod, const double* e,
                   double* lam, QBufs qb, DevWs w, cudaStream_t st);
// Rank-one merges of one tree level (`lev`, 0 = the lowest; w.lroots and w.scal zeroed
// before the first level of a solve).  cum_cols: the prefix of the merges' orders.
// sec_lanes: lanes per secular root, 0 = chosen from the level's root count.
// cta: threads of the one-CTA-per-merge kernels, merge_cta_threads(largest merge).
int merge_cta_threads(int64_t maxm);
void launch_merge_level(int lev, const MergeJob* jobs, int njobs, const int64_t* cum_w8, int64_t nb_w8,
                        const int64_t* cum_rows, int64_t nb_rows, const int64_t* cum_cols,
                        int64_t nb_cols, double* lam, const double* e, QBufs qb, DevWs w,
                        int max_iter, int sec_lanes, int cta, cudaStream_t st, cudaEvent_t placed = nullptr);
// FP64 product, tile shape `cfg` (0 .. kGemmShapes-1): 128x128, 128x64, 64x64, 64x32,
// 32x32, 128x32, 64x16, 128x16, 16x16, 16x32, 16x64, 32x16 (rows x columns).
// cum_tiles (njobs + 1 entries of device memory) is rewritten with the
// tile prefix of the level's actual K; `bound` is the host's upper bound on tiles.
void launch_gemm_fp64(int cfg, const MergeJob* jobs, int njobs, int64_t* cum_tiles, int64_t bound,
                      QBufs qb, DevWs w, cudaStream_t st);
int gemm_shape_rows(int cfg);
int gemm_shape_cols(int cfg);
// Top merges' deflated-column gather and sign convention.  Levels whose largest merge
// (maxm rows) is below kWideColumn take one warp per column, eight columns per virtual
// block (the cdiv(m, 8) prefix of the level); larger ones a 256-thread block per column
// (the m prefix).
constexpr int64_t kWideColumn = 2048;
void launch_defl_copy(const MergeJob* jobs, int njobs, const int64_t* cum_w8, int64_t nb_w8,
                      const int64_t* cum_cols, int64_t nb_cols, int64_t maxm, QBufs qb, DevWs w,
                      bool any_root, cudaStream_t st);
// The same in two parts: the deflated columns' copy, and the sign convention of the
// problems' top merges (which needs the product's columns too).
void launch_defl_copy_cols(const MergeJob* jobs, int njobs, const int64_t* cum_w8, int64_t nb_w8,
                           const int64_t* cum_cols, int64_t nb_cols, int64_t maxm, QBufs qb, DevWs w,
                           cudaStream_t st);
void launch_sign(const MergeJob* jobs, int njobs, const int64_t* cum_w8, int64_t nb_w8, const int64_t* cum_cols,
                 int64_t nb_cols, int64_t maxm, QBufs qb, DevWs w, bool any_root, cudaStream_t st);


constexpr int kGemmShapes = 12;

// The persistent batched solve: one launch; every CTA takes whole problems from a work
// queue (largest first) and runs all of their phases itself, so no CTA waits on another.
// queue: a device counter the caller zeroes before the launch; w.scal zeroed likewise.
void launch_batched_persistent(const PersistProb* probs, int nprob, unsigned* queue, const LeafJob* leaves,
                               const int64_t* tear_list, const MergeJob* pmerges, const int32_t* pmlev,
                               const double* d, const double* e, double* lam, QBufs qb, DevWs w, int max_iter,
                               cudaStream_t st);

}  // namespace tdc
