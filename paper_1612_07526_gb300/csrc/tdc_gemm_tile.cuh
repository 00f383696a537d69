// The FP64 eigenvector product's tile (Eq. 6 with Qhat generated in shared memory),
// shared by the level kernels (gemm_fp64.cu) and the persistent batched kernel
// (dc_kernels.cu).  See gemm_fp64.cu for the scheme.
#pragma once

#include "tdc_internal.cuh"

namespace tdc {
namespace gemm {

constexpr int BK = 8, NT = 256;


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

}  // namespace gemm
}  // namespace tdc
