// Eigenvector product of Eq. (6) in native FP64 with the Cauchy-like factor Qhat
// generated inside the kernel:
//     U[:, pos_i] = sum_k Q_sel[:, k] Qhat[k, i],
//     Qhat[k, i]  = zhat_j / ((d_j - d_org(i)) - tau_i) * sinv_i,   j = kperm[k],
// read from the unscaled columns the norm kernel keeps (one division per entry and
// merge, not per row tile) and scaled by sinv_i while the tile is loaded,
// where Q_sel are the non-deflated (possibly rotated) columns in Gu's order
// (columns touching rows of T1 only, both halves, rows of T2 only).  Rows of T1
// use the first two groups and rows of T2 the last two, so the zero blocks of
// diag(Q1, Q2) are never multiplied.
//
// Tile shapes BM x BN x 8 (BM in {16, 32, 64, 128}, BN in {16, 32, 64, 128}), 256 threads
// in a 16 x 16 grid,
// (BM/16) x (BN/16) FP64 accumulators per thread, double-buffered shared memory;
// the next slab of Qhat is loaded while the current one is consumed.  Every
// output element is one FMA chain over k in ascending order, whatever the shape,
// so all shapes give bit-identical results and the shape is a pure speed choice.
//
// Scheduling: K is known only on the device, so a one-block kernel first counts
// each merge's tiles from its K (k_gemm_sched) and the product kernel strides over
// exactly those tiles; tiles beyond K are never visited.
#include "tdc_gemm_tile.cuh"
#include "tdc_internal.cuh"

namespace tdc {

namespace {

struct Shape {
  int bm, bn;
};
constexpr Shape kShapes[kGemmShapes] = {{128, 128}, {128, 64}, {64, 64}, {64, 32}, {32, 32}, {128, 32},
                                        {64, 16},   {128, 16}, {16, 16}, {16, 32}, {16, 64}, {32, 16}};
using gemm::BK;
using gemm::NT;
using gemm::GemmSmem;
using gemm::gemm_tile;

// Tiles of each merge from its actual K: (row tiles of T1 + of T2) x ceil(K / BN);
// cum[j] = tiles of merges before j.  One block; thread t sums a contiguous run of
// merges, then the runs are scanned in shared memory.
__global__ __launch_bounds__(1024) void k_gemm_sched(const MergeJob* __restrict__ jobs, int njobs,
                                                     const MergeScalars* __restrict__ scal, int bm, int bn,
                                                     int64_t* __restrict__ cum) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int per = (njobs + 1023) / 1024;
  const int j0 = min(t * per, njobs), j1 = min(j0 + per, njobs);
  int64_t s = 0;
  for (int j = j0; j < j1; ++j) {
    const MergeJob& J = jobs[j];
    const int K = scal[J.mid].K;
    s += (int64_t)((J.n1 + bm - 1) / bm + (J.n2 + bm - 1) / bm) * ((K + bn - 1) / bn);
  }
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {      // inclusive Hillis-Steele scan
    const int64_t v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run = t > 0 ? part[t - 1] : 0;
  for (int j = j0; j < j1; ++j) {
    cum[j] = run;
    const MergeJob& J = jobs[j];
    const int K = scal[J.mid].K;
    run += (int64_t)((J.n1 + bm - 1) / bm + (J.n2 + bm - 1) / bm) * ((K + bn - 1) / bn);
  }
  if (t == 1023) cum[njobs] = part[1023];
}

template <int BM, int BN>
__global__ __launch_bounds__(NT) void k_gemm_fp64(const MergeJob* __restrict__ jobs, int njobs,
                                                  const int64_t* __restrict__ cum, QBufs qb, DevWs w) {
  __shared__ GemmSmem<BM, BN> sm;
  const int64_t ntiles = cum[njobs];
  for (int64_t vb = blockIdx.x; vb < ntiles; vb += gridDim.x) {
    gemm_tile<BM, BN>(vb, sm, jobs, njobs, cum, qb, w);
    __syncthreads();
  }
}

template <int BM, int BN>
void launch_shape(const MergeJob* jobs, int njobs, int64_t* cum, int64_t bound, QBufs qb, DevWs w,
                  cudaStream_t st) {
  static int per_sm = 0;
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_gemm_fp64<BM, BN>, NT, 0) != cudaSuccess || b < 1)
      b = 1;
    per_sm = b;
  }
  k_gemm_sched<<<1, 1024, 0, st>>>(jobs, njobs, w.scal, BM, BN, cum);
  k_gemm_fp64<BM, BN><<<grid_cap(bound, per_sm), NT, 0, st>>>(jobs, njobs, cum, qb, w);
}

}  // namespace

int gemm_shape_rows(int cfg) { return kShapes[cfg].bm; }
int gemm_shape_cols(int cfg) { return kShapes[cfg].bn; }

void launch_gemm_fp64(int cfg, const MergeJob* jobs, int njobs, int64_t* cum_tiles, int64_t bound,
                      QBufs qb, DevWs w, cudaStream_t st) {
  if (njobs == 0 || bound == 0) return;
  switch (cfg) {
    case 0: launch_shape<128, 128>(jobs, njobs, cum_tiles, bound, qb, w, st); break;
    case 1: launch_shape<128, 64>(jobs, njobs, cum_tiles, bound, qb, w, st); break;
    case 2: launch_shape<64, 64>(jobs, njobs, cum_tiles, bound, qb, w, st); break;
    case 3: launch_shape<64, 32>(jobs, njobs, cum_tiles, bound, qb, w, st); break;
    case 4: launch_shape<32, 32>(jobs, njobs, cum_tiles, bound, qb, w, st); break;
    case 5: launch_shape<128, 32>(jobs, njobs, cum_tiles, bound, qb, w, st); break;
    case 6: launch_shape<64, 16>(jobs, njobs, cum_tiles, bound, qb, w, st); break;
    case 7: launch_shape<128, 16>(jobs, njobs, cum_tiles, bound, qb, w, st); break;
    case 8: launch_shape<16, 16>(jobs, njobs, cum_tiles, bound, qb, w, st); break;
    case 9: launch_shape<16, 32>(jobs, njobs, cum_tiles, bound, qb, w, st); break;
    case 10: launch_shape<16, 64>(jobs, njobs, cum_tiles, bound, qb, w, st); break;
    default: launch_shape<32, 16>(jobs, njobs, cum_tiles, bound, qb, w, st); break;
  }
}

}  // namespace tdc
