// Eigenvector product of Eq. (6) in native FP64 with the Cauchy-like factor Qhat
// generated inside the kernel:
//     U[:, pos_i] = sum_k Q_sel[:, k] Qhat[k, i],
//     Qhat[k, i]  = zhat_j / ((d_j - d_org(i)) - tau_i) * sinv_i,   j = kperm[k],
// where Q_sel are the non-deflated (possibly rotated) columns in Gu's order
// (columns touching rows of T1 only, both halves, rows of T2 only).  Rows of T1
// use the first two groups and rows of T2 the last two, so the zero blocks of
// diag(Q1, Q2) are never multiplied.  Qhat is never stored.
//
// Tile 128 x 128 x 8, 256 threads, 8 x 8 FP64 accumulators per thread,
// double-buffered shared memory; the next tile of Qhat is generated while the
// current one is consumed.
#include "tdc_internal.cuh"

namespace tdc {

namespace {

constexpr int BM = kGemmBM, BN = kGemmBN, BK = 8, NT = 256;

struct GemmSmem {
  double As[2][BK][BM];
  double Bs[2][BK][BN];
  double dorg[BN], tau[BN], sinv[BN];
  int pos[BN];
};

__device__ __forceinline__ void gemm_tile(int64_t vb, GemmSmem& sm, const MergeJob* __restrict__ jobs,
                                          int njobs, const int64_t* __restrict__ cum, QBufs qb, DevWs w) {
  auto& As = sm.As;
  auto& Bs = sm.Bs;
  double* s_dorg = sm.dorg;
  double* s_tau = sm.tau;
  double* s_sinv = sm.sinv;
  int* s_pos = sm.pos;
  const int jb = find_job(cum, njobs, vb);
  const MergeJob J = jobs[jb];
  const int64_t tile = vb - cum[jb];
  const int n1 = J.n1, n2 = J.n2, m = n1 + n2;
  const int nrt1 = (n1 + BM - 1) / BM, nrt2 = (n2 + BM - 1) / BM;
  const int ct = (int)(tile / (nrt1 + nrt2));
  const int rt = (int)(tile % (nrt1 + nrt2));
  const MergeScalars S = w.scal[J.mid];
  const int K = S.K;
  if (ct * BN >= K) return;
  const bool top = rt < nrt1;
  const int r0 = top ? rt * BM : n1 + (rt - nrt1) * BM;
  const int rend = top ? n1 : m;
  const int kbeg = top ? 0 : S.c1;
  const int kend = top ? S.c1 + S.c3 : K;
  const int64_t o = J.v_off;
  const double* __restrict__ dbar = w.dbar + o;
  const double* __restrict__ zhat = w.zhat + o;
  const int32_t* __restrict__ kperm = w.kperm + o;
  const double* const* __restrict__ colptr = w.colptr + o;

  const int tid = threadIdx.x;
  for (int c = tid; c < BN; c += NT) {
    const int i = ct * BN + c;
    if (i < K) {
      s_dorg[c] = dbar[w.org[o + i]];
      s_tau[c] = w.tau[o + i];
      s_sinv[c] = w.sinv[o + i];
      s_pos[c] = w.posK[o + i];
    } else {
      s_dorg[c] = 0.0;
      s_tau[c] = 0.0;
      s_sinv[c] = 0.0;
      s_pos[c] = -1;
    }
  }
  __syncthreads();

  // loader mapping: 8 rows of k, 32 threads x 4 consecutive rows / columns each
  const int lk = tid >> 5;
  const int l4 = (tid & 31) * 4;
  double ra[4], rb[4];
  auto load_a = [&](int k0) {
    const int k = k0 + lk;
    if (k < kend) {
      const double* col = colptr[k] + r0;
#pragma unroll
      for (int u = 0; u < 4; ++u) ra[u] = (r0 + l4 + u < rend) ? col[l4 + u] : 0.0;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) ra[u] = 0.0;
    }
  };
  auto gen_b = [&](int k0) {
    const int k = k0 + lk;
    if (k < kend) {
      const int j = kperm[k];
      const double zj = zhat[j], dj = dbar[j];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = l4 + u;
        rb[u] = (s_pos[c] >= 0) ? (zj / ((dj - s_dorg[c]) - s_tau[c])) * s_sinv[c] : 0.0;
      }
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) rb[u] = 0.0;
    }
  };
  auto store = [&](int stg) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      As[stg][lk][l4 + u] = ra[u];
      Bs[stg][lk][l4 + u] = rb[u];
    }
  };

  const int tx = tid & 15, ty = tid >> 4;
  double acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0;

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
        double fa[8], fb[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) fa[a] = As[stg][kk][tx + 16 * a];
#pragma unroll
        for (int b = 0; b < 8; ++b) fb[b] = Bs[stg][kk][ty + 16 * b];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] = fma(fa[a], fb[b], acc[a][b]);
      }
      if (more) {
        gen_b(k0 + BK);
        store(stg ^ 1);
      }
      __syncthreads();
      stg ^= 1;
    }
  }

  int64_t ld;
  double* out = (J.src ? qb.A + J.off_a : qb.B + J.off_b);
  ld = J.src ? J.lda : J.ldb;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int c = ty + 16 * b;
    const int pos = s_pos[c];
    if (pos < 0) continue;
    double* col = out + (int64_t)pos * ld + r0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int r = tx + 16 * a;
      if (r0 + r < rend) col[r] = acc[a][b];
    }
  }
}

// Grid-stride over the level's tiles: tiles of columns beyond K cost a few loads.
__global__ __launch_bounds__(NT) void k_gemm_fp64(int64_t ntiles, const MergeJob* __restrict__ jobs,
                                                  int njobs, const int64_t* __restrict__ cum, QBufs qb,
                                                  DevWs w) {
  __shared__ GemmSmem sm;
  for (int64_t vb = blockIdx.x; vb < ntiles; vb += gridDim.x) {
    gemm_tile(vb, sm, jobs, njobs, cum, qb, w);
    __syncthreads();
  }
}

}  // namespace

void launch_gemm_fp64(const MergeJob* jobs, int njobs, const int64_t* cum_tiles, int64_t ntiles,
                      QBufs qb, DevWs w, cudaStream_t st) {
  if (ntiles == 0) return;
  k_gemm_fp64<<<grid_cap(ntiles, 1), NT, 0, st>>>(ntiles, jobs, njobs, cum_tiles, qb, w);
}

}  // namespace tdc
