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
#include "tdc_internal.cuh"

namespace tdc {

namespace {

constexpr int BK = 8, NT = 256;

struct Shape {
  int bm, bn;
};
constexpr Shape kShapes[kGemmShapes] = {{128, 128}, {128, 64}, {64, 64}, {64, 32}, {32, 32}, {128, 32},
                                        {64, 16},   {128, 16}, {16, 16}, {16, 32}, {16, 64}, {32, 16}};

template <int BM, int BN>
struct GemmSmem {
  double As[2][BK][BM];
  double Bs[2][BK][BN];
  double sinv[BN];
  const double* wcol[BN];
  int pos[BN];
};

template <int BM, int BN>
__device__ __forceinline__ void gemm_tile(int64_t vb, GemmSmem<BM, BN>& sm, const MergeJob* __restrict__ jobs,
                                          int njobs, const int64_t* __restrict__ cum, QBufs qb, DevWs w) {
  constexpr int TM = BM / 16, TN = BN / 16;         // accumulators per thread
  constexpr int NB = BN * BK;                       // Qhat entries per slab (128 for BN = 16)
  constexpr int NA = BM * BK;                       // Q_sel entries per slab (128 for BM = 16)
  constexpr int LA = NA >= NT ? NA / NT : 1, LB = NB >= NT ? NB / NT : 1;  // loads / generated entries per thread
  auto& As = sm.As;
  auto& Bs = sm.Bs;
  const int jb = find_job(cum, njobs, vb);
  const MergeJob J = jobs[jb];
  const int64_t tile = vb - cum[jb];
  const int n1 = J.n1, n2 = J.n2, m = n1 + n2;
  const int nrt1 = (n1 + BM - 1) / BM, nrt2 = (n2 + BM - 1) / BM;
  const int ct = (int)(tile / (nrt1 + nrt2));
  const int rt = (int)(tile % (nrt1 + nrt2));
  const MergeScalars S = w.scal[J.mid];
  const int K = S.K;
  const bool top = rt < nrt1;
  const int r0 = top ? rt * BM : n1 + (rt - nrt1) * BM;
  const int rend = top ? n1 : m;
  const int kbeg = top ? 0 : S.c1;
  const int kend = top ? S.c1 + S.c3 : K;
  const int64_t o = J.v_off;
  const int32_t* __restrict__ kperm = w.kperm + o;
  const double* const* __restrict__ colptr = w.colptr + o;

  const int tid = threadIdx.x;
  for (int c = tid; c < BN; c += NT) {
    const int i = ct * BN + c;
    if (i < K) {
      sm.sinv[c] = w.sinv[o + i];
      sm.wcol[c] = w.wptr[o + i];
      sm.pos[c] = w.posK[o + i];
    } else {
      sm.sinv[c] = 0.0;
      sm.wcol[c] = nullptr;
      sm.pos[c] = -1;
    }
  }
  __syncthreads();

  // loader mapping: thread t covers LA consecutive rows (LB columns) of one k row;
  // narrow slabs use their first NA (NB) threads
  const bool la_on = tid * LA < NA;
  const int la_k = la_on ? (tid * LA) / BM : 0, la_r = la_on ? (tid * LA) % BM : 0;
  const bool lb_on = tid * LB < NB;                // narrow slabs: the first NB threads
  const int lb_k = lb_on ? (tid * LB) / BN : 0, lb_c = lb_on ? (tid * LB) % BN : 0;
  double ra[LA], rb[LB];
  auto load_a = [&](int k0) {
    const int k = k0 + la_k;
    if (la_on && k < kend) {
      const double* col = colptr[k];
      const int lo = max(w.klo[o + k], r0), hi = min(w.khi[o + k], rend);   // rows that can be nonzero
#pragma unroll
      for (int u = 0; u < LA; ++u) {
        const int r = r0 + la_r + u;
        ra[u] = (r >= lo && r < hi) ? col[r] : 0.0;
      }
    } else {
#pragma unroll
      for (int u = 0; u < LA; ++u) ra[u] = 0.0;
    }
  };
  auto gen_b = [&](int k0) {
    const int k = k0 + lb_k;
    if (lb_on && k < kend) {
      const int j = kperm[k];
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        const int c = lb_c + u;
        rb[u] = (sm.pos[c] >= 0) ? sm.wcol[c][j] * sm.sinv[c] : 0.0;
      }
    } else {
#pragma unroll
      for (int u = 0; u < LB; ++u) rb[u] = 0.0;
    }
  };
  auto store = [&](int stg) {
    if (la_on)
#pragma unroll
      for (int u = 0; u < LA; ++u) As[stg][la_k][la_r + u] = ra[u];
    if (lb_on)
#pragma unroll
      for (int u = 0; u < LB; ++u) Bs[stg][lb_k][lb_c + u] = rb[u];
  };

  const int tx = tid & 15, ty = tid >> 4;
  double acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = 0.0;

  if (kbeg < kend) {
    load_a(kbeg);
    gen_b(kbeg);
    store(0);
    __syncthreads();
    int stg = 0;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
      const bool more = k0 + BK < kend;
      if (more) load_a(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double fa[TM], fb[TN];
#pragma unroll
        for (int a = 0; a < TM; ++a) fa[a] = As[stg][kk][tx + 16 * a];
#pragma unroll
        for (int b = 0; b < TN; ++b) fb[b] = Bs[stg][kk][ty + 16 * b];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TN; ++b) acc[a][b] = fma(fa[a], fb[b], acc[a][b]);
      }
      if (more) {
        gen_b(k0 + BK);
        store(stg ^ 1);
      }
      __syncthreads();
      stg ^= 1;
    }
  }

#pragma unroll
  for (int b = 0; b < TN; ++b) {
    const int c = ty + 16 * b;
    if (sm.pos[c] < 0) continue;
    double* col = w.outptr[o + ct * BN + c] + r0;
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      const int r = tx + 16 * a;
      if (r0 + r < rend) col[r] = acc[a][b];
    }
  }
}

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
