// HSS form of the eigenvector product (Section 2, Algorithm 1 and the fast
// multiply): Qhat (K x K, never stored) is compressed by randomized sampling and
// interpolative decompositions, then U = Q_sel Qhat_hss is formed with an up-sweep
// through the nested bases U, the sibling couplings B and a down-sweep through V.
// Qhat stays in the order of the sorted d (no Gu grouping: it would break the
// off-diagonal low rank).  The decompositions run in FP64:
//   k_hss_omega   Gaussian sampling matrices (SplitMix64 + Box-Muller)
//   k_hss_id_cl   column-pivoted QR of Phi^T (row ID Phi ~= U Phi(I, :)), one
//                 cluster of 2-16 CTAs per decomposition with Phi^T held in their
//                 shared memory; k_hss_id, one CTA and global scratch, where it
//                 does not fit
//   k_hss_couple  per parent: sibling couplings B (Qhat at the skeletons)
//   k_hss_parent  per parent: its Phi and Theta from the children's
//   k_hss_skel    global skeleton indices
// Every product runs on the split-precision tensor-core GEMM (tdc_ozaki.cuh, 7 slices):
// the sampling Y = Qhat Omega1 and Z = Qhat^T Omega2 with Qhat's diagonal leaf blocks
// read as zero, the nodes' Yhat = V^T [Yhat_1; Yhat_2] and Zhat = U^T [Zhat_1; Zhat_2],
// and the multiply's up-sweep, couplings, down-sweep and leaf products.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "tdc_hss.cuh"
#include "tdc_ozaki.cuh"

namespace tdc {

namespace {

constexpr unsigned kFullMask = 0xffffffffu;

// ------------------------------------------------------------------ Qhat entries
struct QhatSrc {
  double* const* wcol;        // unscaled Cauchy columns kept by the norm kernel
  const double* sinv;
};
__device__ __forceinline__ double qhat(const QhatSrc& q, int j, int i) {
  return q.wcol[i][j] * q.sinv[i];
}

// ------------------------------------------------------------------ sampling matrices
__device__ __forceinline__ uint64_t splitmix(uint64_t seed, uint64_t idx) {
  uint64_t z = seed + (idx + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void k_hss_omega(double* __restrict__ om, int64_t rows, int cols, uint64_t seed, uint64_t stream) {
  const int64_t n = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t q = stream * (1ull << 40) + (uint64_t)e;   // e = c * rows + r
    const uint64_t z1 = splitmix(seed, 2 * q), z2 = splitmix(seed, 2 * q + 1);
    const double u1 = ((double)(z1 >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = (double)(z2 >> 11) * 0x1.0p-53;
    om[e] = sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
  }
}

// kept-order (sorted d) column pointers of Q_sel and their row-support types
__global__ void k_hss_cols(const MergeJob J, DevWs w, HssCols xc) {
  const int K = w.scal[J.mid].K;
  const int64_t o = J.v_off;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    const int j = w.kperm[o + k];
    xc.col[j] = w.colptr[o + k];
    xc.lo[j] = w.klo[o + k];
    xc.hi[j] = w.khi[o + k];
  }
}

// ------------------------------------------------------------------ interpolative decomposition
// Row ID of Phi (rows x rp, column-major, ld): Householder QR with column pivoting of
// M = Phi^T (rp x rows, built in scratch), stopped when the pivot column's remaining
// norm falls to tol times the first; then T = R11^-1 R12 and U[perm[t], :] = e_t,
// U[perm[rank + c], :] = T[:, c]^T.  One CTA per decomposition.
__global__ __launch_bounds__(256) void k_hss_id(const HIdJob* __restrict__ jobs, double tol, int rp) {
  extern __shared__ double sh[];
  const HIdJob Jb = jobs[blockIdx.x];
  const int rows = Jb.rows_dev ? *Jb.rows_dev : Jb.rows;
  double* nrm = sh;                        // rows
  double* v = sh + Jb.rows_max;            // rp
  int* perm = reinterpret_cast<int*>(v + rp);
  __shared__ double s_red[32];
  __shared__ int s_idx[32];
  __shared__ double s_r0;
  const int tid = threadIdx.x, NT = blockDim.x;
  double* Mx = Jb.scratch;                 // rp x rows_max, column c = row c of Phi
  for (int c = tid; c < rows; c += NT) {
    double s = 0.0;
    for (int r = 0; r < rp; ++r) {
      const double x = Jb.phi[(int64_t)r * Jb.ld + c];
      Mx[(int64_t)c * rp + r] = x;
      s += x * x;
    }
    nrm[c] = s;
    perm[c] = c;
  }
  __syncthreads();
  const int kmax = min(rp, rows);
  int rank = kmax;
  for (int k = 0; k < kmax; ++k) {
    // pivot: largest remaining column norm (first on ties)
    double bv = -1.0;
    int bi = 0x7fffffff;
    for (int c = k + tid; c < rows; c += NT)
      if (nrm[c] > bv) { bv = nrm[c]; bi = c; }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_xor_sync(kFullMask, bv, off);
      const int oi = __shfl_xor_sync(kFullMask, bi, off);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { s_red[tid >> 5] = bv; s_idx[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      for (int q = 1; q < NT / 32; ++q)
        if (s_red[q] > bv || (s_red[q] == bv && s_idx[q] < bi)) { bv = s_red[q]; bi = s_idx[q]; }
      s_idx[0] = bi;
      s_red[0] = bv;
    }
    __syncthreads();
    const int p = s_idx[0];
    const double pn = sqrt(fmax(s_red[0], 0.0));
    if (k == 0) {
      if (tid == 0) s_r0 = pn;
      __syncthreads();
    }
    if (!(pn > tol * s_r0)) { rank = k; break; }
    __syncthreads();
    if (p != k) {                            // swap columns k and p
      for (int r = tid; r < rp; r += NT) {
        const double a = Mx[(int64_t)k * rp + r];
        Mx[(int64_t)k * rp + r] = Mx[(int64_t)p * rp + r];
        Mx[(int64_t)p * rp + r] = a;
      }
      if (tid == 0) {
        const double a = nrm[k]; nrm[k] = nrm[p]; nrm[p] = a;
        const int b = perm[k]; perm[k] = perm[p]; perm[p] = b;
      }
    }
    __syncthreads();
    // Householder vector of M[k:, k] (warp 0, lanes over the rows of the sample)
    const int lane = tid & 31, wid = tid >> 5, nw = NT >> 5;
    if (wid == 0) {
      double* colk = Mx + (int64_t)k * rp;
      double s = 0.0;
      for (int r = k + lane; r < rp; r += 32) s = fma(colk[r], colk[r], s);
      s = warp_sum(s);
      const double x0 = colk[k];
      const double alpha = x0 >= 0.0 ? -sqrt(s) : sqrt(s);
      double vv = 0.0;
      for (int r = k + lane; r < rp; r += 32) {
        const double vr = colk[r] - (r == k ? alpha : 0.0);
        v[r] = vr;
        vv = fma(vr, vr, vv);
      }
      vv = warp_sum(vv);
      if (lane == 0) s_red[1] = vv > 0.0 ? 2.0 / vv : 0.0;
      for (int r = k + lane; r < rp; r += 32) colk[r] = r == k ? alpha : 0.0;
    }
    __syncthreads();
    const double beta = s_red[1];
    // the reflection of the remaining columns, a warp per column
    for (int c = k + 1 + wid; c < rows; c += nw) {
      double* col = Mx + (int64_t)c * rp;
      double wdot = 0.0;
      for (int r = k + lane; r < rp; r += 32) wdot = fma(v[r], col[r], wdot);
      wdot = warp_sum(wdot) * beta;
      double s = 0.0;
      for (int r = k + lane; r < rp; r += 32) {
        const double x = col[r] - wdot * v[r];
        col[r] = x;
        if (r > k) s = fma(x, x, s);
      }
      s = warp_sum(s);
      if (lane == 0) nrm[c] = s;
    }
    __syncthreads();
  }
  if (tid == 0) {
    *Jb.rank_out = rank;
    for (int t = 0; t < rank; ++t) Jb.skel_local[t] = perm[t];
  }
  // U (rows x rank, column-major, ld = rows_max)
  for (int e = tid; e < rows * rank; e += NT) {
    const int r = e % rows, c = e / rows;
    Jb.U[(int64_t)c * Jb.rows_max + r] = 0.0;
  }
  __syncthreads();
  for (int t = tid; t < rank; t += NT) Jb.U[(int64_t)t * Jb.rows_max + perm[t]] = 1.0;
  // T = R11^-1 R12, a warp per column c of R12 (back substitution, lanes over the
  // solved entries of each step)
  {
    const int lane = tid & 31, wid = tid >> 5, nw = NT >> 5;
    for (int c = rank + wid; c < rows; c += nw) {
      double* col = Mx + (int64_t)c * rp;   // R12 column, solved in place (rows 0..rank)
      for (int r = rank - 1; r >= 0; --r) {
        double s = 0.0;
        for (int q = r + 1 + lane; q < rank; q += 32) s = fma(Mx[(int64_t)q * rp + r], col[q], s);
        s = warp_sum(s);
        if (lane == 0) col[r] = (col[r] - s) / Mx[(int64_t)r * rp + r];
        __syncwarp();
      }
      for (int t = lane; t < rank; t += 32) Jb.U[(int64_t)t * Jb.rows_max + perm[c]] = col[t];
    }
  }
}

// The same row ID on a cluster of CS CTAs (2 to 16, chosen per launch so that all its
// clusters are resident together).  CTA q of the cluster holds the
// columns [q W, q W + W) of M = Phi^T (rows of Phi) in its shared memory (column c
// at M + c ldm, rows 0..rp-1), so every step works on shared memory, with one cluster
// barrier per step:
//   1. after the barrier every CTA reads the cluster's offers (each warp's unselected
//      column of largest remaining norm, double-buffered by step parity) and picks the
//      same pivot p (largest norm, then smallest index);
//   2. every CTA reads M(k:, p) from the shared memory of the CTA that holds it and forms
//      the same Householder vector from that column's exact norm (which also decides the
//      stop: |R_kk| <= tol |R_00|); the holder writes R_kk and the zeros below it into
//      the column only after the next barrier, when every CTA has read it;
//   3. every CTA reflects its unselected columns (four threads per column), downdates
//      their squared norms by R(k, c)^2 (recomputing a norm exactly when the downdate
//      has cancelled it to 2^-26 of its last exact value or below: the usual safeguard
//      of pivoted QR with norm downdating), and offers its next pivot.
// The pivot columns are not moved: R11 = M(0:rank, piv) is written to global scratch
// (row-major), and after a further barrier each CTA solves R11 T(:, c) = M(0:rank, c)
// for its other columns and writes its rows of U.
constexpr int kIdThreads = 256;

struct IdClShape {
  int W, ldm;                 // columns per CTA (a multiple of 8), leading dimension of M
  size_t smem;
};
IdClShape id_cl_shape(int rows_max, int rp, int cs) {
  IdClShape sh;
  sh.W = ((rows_max + cs - 1) / cs + 7) / 8 * 8;
  sh.ldm = (rp + 15) / 16 * 16 + 4;          // 4 mod 16 doubles: a warp's quads spread over the banks
  sh.smem = (size_t)sh.W * sh.ldm * 8 + (size_t)2 * sh.W * 8 + (size_t)rp * 8 + (size_t)rp * 4 +
            (size_t)sh.W * 4 + 64;
  return sh;
}

__global__ void __launch_bounds__(kIdThreads, 1)
    k_hss_id_cl(const HIdJob* __restrict__ jobs, double tol, int rp, int W, int ldm) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) double sm_id[];
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank();
  const int CS = (int)cl.num_blocks();         // the cluster size of this launch
  const HIdJob Jb = jobs[blockIdx.x / CS];
  const int rows = Jb.rows_dev ? *Jb.rows_dev : Jb.rows;
  double* M = sm_id;                          // W x ldm
  double* nrm = M + (size_t)W * ldm;          // downdated squared norms of M(k:, c)
  double* nref = nrm + W;                     // the same at their last exact computation
  double* v = nref + W;                       // this step's Householder vector (rows k..rp-1)
  int* piv = reinterpret_cast<int*>(v + rp);
  int* stc = piv + rp;                        // per column: -2 absent, -1 active, else its step
  __shared__ double s_wv[2][kIdThreads / 32];
  __shared__ int s_wi[2][kIdThreads / 32];
  __shared__ int s_p;
  __shared__ double s_beta, s_alpha, s_pn;
  const int tid = threadIdx.x, NT = kIdThreads, lane = tid & 31;
  const int quad = tid >> 2, ql = tid & 3, NQ = NT / 4;
  const int g0 = crank * W;

  for (int e = tid; e < W * rp; e += NT) {    // M(r, c) = Phi(g0 + c, r)
    const int c = e % W, r = e / W, g = g0 + c;
    M[(size_t)c * ldm + r] = g < rows ? Jb.phi[(int64_t)r * Jb.ld + g] : 0.0;
  }
  __syncthreads();
  for (int c = quad; c < W; c += NQ) {        // W is a multiple of 8: uniform per warp
    double s = 0.0;
    for (int r = ql; r < rp; r += 4) s = fma(M[(size_t)c * ldm + r], M[(size_t)c * ldm + r], s);
    s += __shfl_xor_sync(kFullMask, s, 1);
    s += __shfl_xor_sync(kFullMask, s, 2);
    if (ql == 0) {
      nrm[c] = s;
      nref[c] = s;
      stc[c] = g0 + c < rows ? -1 : -2;
    }
  }
  __syncthreads();
  // each warp's offer: its active column of largest remaining norm (first on ties),
  // double-buffered by step parity; the pivot is the best of the cluster's 8 x 8 offers
  auto offer = [&](int slot) {
    double bv = -1.0;
    int bi = 0x7fffffff;
    for (int c = tid; c < W; c += NT)
      if (stc[c] == -1 && nrm[c] > bv) { bv = nrm[c]; bi = g0 + c; }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_xor_sync(kFullMask, bv, off);
      const int oi = __shfl_xor_sync(kFullMask, bi, off);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) {
      s_wv[slot][tid >> 5] = bv;
      s_wi[slot][tid >> 5] = bi;
    }
  };
  offer(0);
  cl.sync();                                  // step 0's offers published

  const int kmax = min(rp, rows);
  int rank = kmax;
  double r0 = 0.0;
  int pend = -1;                              // this CTA's previous pivot column, R not yet written
  double pend_alpha = 0.0;
  for (int k = 0; k < kmax; ++k) {
    // the previous pivot's column: R_kk and zeros below (every CTA has read it)
    if (pend >= 0) {
      double* col = M + (size_t)pend * ldm;
      for (int r = k - 1 + tid; r < rp; r += NT) col[r] = r == k - 1 ? pend_alpha : 0.0;
      pend = -1;
    }
    // warp 0: the pivot, then the Householder vector of M(k:, p) read from its holder
    if (tid < 32) {
      double ov = -1.0;
      int oi = 0x7fffffff;
#pragma unroll
      for (int h = 0; h < (16 * (kIdThreads / 32) + 31) / 32; ++h) {
        const int q = lane + 32 * h;
        if (q < CS * (kIdThreads / 32)) {
          const int cta = q / (kIdThreads / 32), wq = q % (kIdThreads / 32);
          const double v2 = *cl.map_shared_rank(&s_wv[k & 1][wq], cta);
          const int i2 = *cl.map_shared_rank(&s_wi[k & 1][wq], cta);
          if (v2 > ov || (v2 == ov && i2 < oi)) { ov = v2; oi = i2; }
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double pv = __shfl_xor_sync(kFullMask, ov, off);
        const int pi = __shfl_xor_sync(kFullMask, oi, off);
        if (pv > ov || (pv == ov && pi < oi)) { ov = pv; oi = pi; }
      }
      const int p = oi;                        // the same in every lane and every CTA
      if (lane == 0) s_p = p;
      if (p != 0x7fffffff) {
        const int owner = p / W;
        const double* col = cl.map_shared_rank(M + (size_t)(p - owner * W) * ldm, owner);
        double s = 0.0;
        for (int r = k + lane; r < rp; r += 32) {
          const double x = col[r];
          v[r] = x;
          s = fma(x, x, s);
        }
        s = warp_sum(s);
        const double pn = sqrt(s);
        const double rr0 = k == 0 ? pn : r0;
        __syncwarp();
        const double alpha = v[k] >= 0.0 ? -pn : pn;
        __syncwarp();                         // every lane has read v[k]
        double vv = 0.0;
        for (int r = k + lane; r < rp; r += 32) {
          const double vr = v[r] - (r == k ? alpha : 0.0);
          v[r] = vr;
          vv = fma(vr, vr, vv);
        }
        vv = warp_sum(vv);
        if (lane == 0) {
          s_beta = !(pn > tol * rr0) ? -1.0 : (vv > 0.0 ? 2.0 / vv : 0.0);   // -1: stop
          s_alpha = alpha;
          s_pn = pn;
        }
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p == 0x7fffffff) { rank = k; break; }
    const double beta = s_beta;
    if (k == 0) r0 = s_pn;
    if (beta < 0.0) { rank = k; break; }
    if (p / W == crank) {
      pend = p - g0;
      pend_alpha = s_alpha;
      if (tid == 0) stc[pend] = k;            // read by the offers after the next barrier
    }
    if (tid == 0) piv[k] = p;
    // reflect the unselected columns (the pivot excluded by index: its mark may be in
    // flight), downdate their norms
    for (int c = quad; c < W; c += NQ) {
      const bool act = stc[c] == -1 && g0 + c != p;
      double* col = M + (size_t)c * ldm;
      double w = 0.0;
      if (act)
        for (int r = k + ql; r < rp; r += 4) w = fma(v[r], col[r], w);
      w += __shfl_xor_sync(kFullMask, w, 1);
      w += __shfl_xor_sync(kFullMask, w, 2);
      double rk = 0.0;
      if (act) {
        w *= beta;
        for (int r = k + ql; r < rp; r += 4) {
          const double x = fma(-w, v[r], col[r]);
          col[r] = x;
          if (r == k) rk = x;
        }
      }
      rk = __shfl_sync(kFullMask, rk, (tid & 31) & ~3);   // R(k, c), held by the quad's lane 0
      const double sd = nrm[c] - rk * rk;
      const bool redo = act && !(sd > 0x1p-26 * nref[c]);
      double s = 0.0;
      if (redo)                               // each lane rereads only the rows it wrote
        for (int r = k + ql; r < rp; r += 4)
          if (r > k) s = fma(col[r], col[r], s);
      s += __shfl_xor_sync(kFullMask, s, 1);
      s += __shfl_xor_sync(kFullMask, s, 2);
      if (act && ql == 0) {
        nrm[c] = redo ? s : sd;
        if (redo) nref[c] = s;
      }
    }
    __syncthreads();
    offer((k + 1) & 1);
    cl.sync();                                // step k + 1's offers published; step k's reads done
  }
  if (pend >= 0) {                            // the last pivot's column
    double* col = M + (size_t)pend * ldm;
    for (int r = rank - 1 + tid; r < rp; r += NT) col[r] = r == rank - 1 ? pend_alpha : 0.0;
  }
  __syncthreads();
  // R11 (rank x rank, row-major) to global scratch: R11(i, j) = M(i, piv[j])
  double* R11 = Jb.scratch;
  for (int e = tid; e < W * rank; e += NT) {
    const int c = e % W, i = e / W, j = stc[c];
    if (j >= 0) R11[(int64_t)i * rank + j] = M[(size_t)c * ldm + i];
  }
  if (crank == 0) {
    if (tid == 0) *Jb.rank_out = rank;
    for (int t = tid; t < rank; t += NT) Jb.skel_local[t] = piv[t];
  }
  cl.sync();                                  // R11 visible to the cluster; no shared reads after
  // T(:, c) = R11^-1 M(0:rank, c) for the other columns, in place
  for (int c = quad; c < W; c += NQ) {
    const bool act = stc[c] == -1;
    double* col = M + (size_t)c * ldm;
    for (int r = rank - 1; r >= 0; --r) {
      double s = 0.0;
      if (act)
        for (int q = r + 1 + ql; q < rank; q += 4) s = fma(R11[(int64_t)r * rank + q], col[q], s);
      s += __shfl_xor_sync(kFullMask, s, 1);
      s += __shfl_xor_sync(kFullMask, s, 2);
      if (act && ql == 0) col[r] = (col[r] - s) / R11[(int64_t)r * rank + r];
      __syncwarp();
    }
  }
  __syncthreads();
  // rows g0 .. g0 + W - 1 of U (rows x rank, column-major, ld rows_max)
  for (int e = tid; e < W * rank; e += NT) {
    const int c = e % W, t = e / W, g = g0 + c;
    if (g >= rows) continue;
    const int j = stc[c];
    Jb.U[(int64_t)t * Jb.rows_max + g] = j >= 0 ? (j == t ? 1.0 : 0.0) : M[(size_t)c * ldm + t];
  }
}

// The cluster size of one k_hss_id_cl launch of `nids` decompositions: the largest of
// 16, 8, 4 and 2 whose clusters are all resident at once (one wave), else 8 (or the
// largest that fits its shared memory); 0 when none does (then k_hss_id runs instead).
// Its shape goes to *sh.
constexpr size_t kIdClMaxSmem = 200u << 10;
int id_cl_max_clusters(int cs, size_t smem) {
  if (cudaFuncSetAttribute(k_hss_id_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      (cs > 8 && cudaFuncSetAttribute(k_hss_id_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)cs);
  cfg.blockDim = dim3(kIdThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void*)k_hss_id_cl, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}
int id_cl_pick(int nids, int rows_max, int rp, IdClShape* sh) {
  int fallback = 0;
  IdClShape fsh{};
  for (int cs = 16; cs >= 2; cs >>= 1) {
    const IdClShape s = id_cl_shape(rows_max, rp, cs);
    if (s.smem > kIdClMaxSmem) continue;
    const int n = id_cl_max_clusters(cs, s.smem);
    if (n <= 0) continue;
    if (nids <= n) {                          // the largest size whose clusters fit in one wave
      *sh = s;
      return cs;
    }
    if (fallback == 0 || cs == 8) {           // else 8 CTAs (more waves of the same clusters
      fallback = cs;                          // beat fewer, larger CTAs per decomposition)
      fsh = s;
    }
  }
  *sh = fsh;
  return fallback;
}
cudaError_t launch_id_cl(const HIdJob* jobs, int nids, int cs, const IdClShape& sh, double tol, int rp,
                         cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(nids * cs));
  cfg.blockDim = dim3(kIdThreads);
  cfg.dynamicSmemBytes = sh.smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_hss_id_cl, jobs, tol, rp, sh.W, sh.ldm);
}

// ------------------------------------------------------------------ parent steps
// B_{c1} = Qhat(I_c1, J_c2), B_{c2} = Qhat(I_c2, J_c1), and (unless root)
//   Phi_p   = [Phi_c1(Iloc_c1) - B_c1 Yhat_c2 ; Phi_c2(Iloc_c2) - B_c2 Yhat_c1]
//   Theta_p = [Theta_c1(Jloc_c1) - B_c2^T Zhat_c2 ; Theta_c2(Jloc_c2) - B_c1^T Zhat_c1]
// in two kernels (the second reads the first's B), each with kParentParts CTAs per
// parent (blockIdx.y) sharing its elements.
constexpr int kParentParts = 8;
__global__ __launch_bounds__(256) void k_hss_couple(const HssNodeDev* __restrict__ nodes,
                                                    const int* __restrict__ plist, int rp, QhatSrc q) {
  const HssNodeDev P = nodes[plist[blockIdx.x]];
  const HssNodeDev A = nodes[P.c1], Bn = nodes[P.c2];
  const int ku1 = *A.kU, kv1 = *A.kV, ku2 = *Bn.kU, kv2 = *Bn.kV;
  const int t0 = blockIdx.y * blockDim.x + threadIdx.x, NT = gridDim.y * blockDim.x;
  for (int e = t0; e < ku1 * kv2; e += NT) {
    const int r = e % ku1, c = e / ku1;
    A.B[(int64_t)c * rp + r] = qhat(q, A.I[r], Bn.J[c]);
  }
  for (int e = t0; e < ku2 * kv1; e += NT) {
    const int r = e % ku2, c = e / ku2;
    Bn.B[(int64_t)c * rp + r] = qhat(q, Bn.I[r], A.J[c]);
  }
  if (P.root) return;
  if (t0 == 0) {
    *P.rows_u = ku1 + ku2;
    *P.rows_v = kv1 + kv2;
  }
  // skeleton candidates of the parent (global indices), in row order of Phi_p
  for (int r = t0; r < ku1 + ku2; r += NT) P.Icand[r] = r < ku1 ? A.I[r] : Bn.I[r - ku1];
  for (int r = t0; r < kv1 + kv2; r += NT) P.Jcand[r] = r < kv1 ? A.J[r] : Bn.J[r - kv1];
}

__global__ __launch_bounds__(256) void k_hss_parent(const HssNodeDev* __restrict__ nodes,
                                                    const int* __restrict__ plist, int rp) {
  const HssNodeDev P = nodes[plist[blockIdx.x]];
  if (P.root) return;
  const HssNodeDev A = nodes[P.c1], Bn = nodes[P.c2];
  const int ku1 = *A.kU, kv1 = *A.kV, ku2 = *Bn.kU, kv2 = *Bn.kV;
  const int t0 = blockIdx.y * blockDim.x + threadIdx.x, NT = gridDim.y * blockDim.x;
  // Phi_p rows: first ku1 from child 1, then ku2 from child 2
  for (int e = t0; e < (ku1 + ku2) * rp; e += NT) {
    const int r = e % (ku1 + ku2), c = e / (ku1 + ku2);
    double s;
    if (r < ku1) {
      s = A.phi[(int64_t)c * A.ldphi + A.Iloc[r]];
      for (int t = 0; t < kv2; ++t) s -= A.B[(int64_t)t * rp + r] * Bn.Yh[(int64_t)c * rp + t];
    } else {
      const int rr = r - ku1;
      s = Bn.phi[(int64_t)c * Bn.ldphi + Bn.Iloc[rr]];
      for (int t = 0; t < kv1; ++t) s -= Bn.B[(int64_t)t * rp + rr] * A.Yh[(int64_t)c * rp + t];
    }
    P.phi[(int64_t)c * P.ldphi + r] = s;
  }
  for (int e = t0; e < (kv1 + kv2) * rp; e += NT) {
    const int r = e % (kv1 + kv2), c = e / (kv1 + kv2);
    double s;
    if (r < kv1) {
      s = A.theta[(int64_t)c * A.ldphi + A.Jloc[r]];
      for (int t = 0; t < ku2; ++t) s -= Bn.B[(int64_t)r * rp + t] * Bn.Zh[(int64_t)c * rp + t];
    } else {
      const int rr = r - kv1;
      s = Bn.theta[(int64_t)c * Bn.ldphi + Bn.Jloc[rr]];
      for (int t = 0; t < ku1; ++t) s -= A.B[(int64_t)rr * rp + t] * A.Zh[(int64_t)c * rp + t];
    }
    P.theta[(int64_t)c * P.ldphi + r] = s;
  }
}

// After a node's IDs: its global skeleton indices (a leaf's rows start at lo, a
// parent's are the candidates its children passed up).
__global__ void k_hss_skel(const HssNodeDev* __restrict__ nodes, const int* __restrict__ list) {
  const HssNodeDev N = nodes[list[blockIdx.x]];
  const int ku = *N.kU, kv = *N.kV;
  for (int t = threadIdx.x; t < ku; t += blockDim.x) N.I[t] = N.leaf ? N.lo + N.Iloc[t] : N.Icand[N.Iloc[t]];
  for (int t = threadIdx.x; t < kv; t += blockDim.x) N.J[t] = N.leaf ? N.lo + N.Jloc[t] : N.Jcand[N.Jloc[t]];
}

__global__ void k_read_k(const MergeScalars* scal, int64_t mid, int* out) { *out = scal[mid].K; }


}  // namespace

// ------------------------------------------------------------------ host orchestration
namespace {

struct Bump {
  unsigned char* p;
  size_t off = 0;
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* r = p ? reinterpret_cast<T*>(p + off) : nullptr;
    off += n * sizeof(T);
    return r;
  }
};

struct HNodeHost {
  int lo, hi, level, c1 = -1, c2 = -1, parent = -1;
};

int build_tree(std::vector<HNodeHost>& t, int lo, int hi, int level, int leaf) {
  HNodeHost nd;
  nd.lo = lo;
  nd.hi = hi;
  nd.level = level;
  if (hi - lo > leaf) {
    const int mid = lo + (hi - lo) / 2;
    const int a = build_tree(t, lo, mid, level + 1, leaf);
    const int b = build_tree(t, mid, hi, level + 1, leaf);
    nd.c1 = a;
    nd.c2 = b;
    t.push_back(nd);
    const int me = (int)t.size() - 1;
    t[a].parent = me;
    t[b].parent = me;
    return me;
  }
  t.push_back(nd);
  return (int)t.size() - 1;
}

constexpr size_t kTabBytes = 1u << 22;

struct HssLayout {
  int* dK;
  double *om1, *om2, *Y, *Z;
  HssCols xc;
  int32_t* lid;               // leaf of each Qhat index
  std::vector<HNodeHost> tree;
  int root = 0;
  std::vector<HssNodeDev> nd;
  HssNodeDev* dnodes;
  unsigned char* tab;
  double* idscratch;
  int* lists;
  size_t bytes = 0;
};

// The arena layout for K non-deflated columns of an order-m merge (base may be null
// to size it).
void hss_layout(HssLayout& L, unsigned char* base, int K, int m, const tdc_opts& o, int rp) {
  const int hl = std::max(o.hss_leaf, 2);
  const int rmax = std::max(hl, 2 * rp);
  Bump b{base};
  L.dK = b.take<int>(1);
  L.om1 = b.take<double>((size_t)K * rp);
  L.om2 = b.take<double>((size_t)K * rp);
  L.Y = b.take<double>((size_t)K * rp);
  L.Z = b.take<double>((size_t)K * rp);
  L.xc.col = b.take<const double*>(K);
  L.xc.lo = b.take<int32_t>(K);
  L.xc.hi = b.take<int32_t>(K);
  L.lid = b.take<int32_t>(K);
  L.tree.clear();
  L.root = build_tree(L.tree, 0, std::max(K, 1), 0, hl);
  const int nn = (int)L.tree.size();
  L.nd.assign(nn, HssNodeDev{});
  for (int i = 0; i < nn; ++i) {
    HssNodeDev& d = L.nd[i];
    const HNodeHost& h = L.tree[i];
    d.lo = h.lo;
    d.hi = h.hi;
    d.leaf = h.c1 < 0;
    d.c1 = h.c1;
    d.c2 = h.c2;
    d.root = i == L.root;
    if (d.leaf) {
      d.phi = L.Y ? L.Y + h.lo : nullptr;     // a leaf's Phi is formed in place in Y (ld = K)
      d.theta = L.Z ? L.Z + h.lo : nullptr;
      d.ldphi = K;
    } else {
      d.phi = b.take<double>((size_t)rmax * rp);
      d.theta = b.take<double>((size_t)rmax * rp);
      d.ldphi = rmax;
    }
    d.U = b.take<double>((size_t)rmax * rp);
    d.V = b.take<double>((size_t)rmax * rp);
    d.ldU = rmax;
    d.Yh = b.take<double>((size_t)rp * rp);
    d.Zh = b.take<double>((size_t)rp * rp);
    d.B = b.take<double>((size_t)rp * rp);
    d.G = b.take<double>((size_t)m * rp);
    d.F = b.take<double>((size_t)m * rp);
    d.I = b.take<int>(rp);
    d.J = b.take<int>(rp);
    d.Iloc = b.take<int>(rmax);
    d.Jloc = b.take<int>(rmax);
    d.Icand = b.take<int>(rmax);
    d.Jcand = b.take<int>(rmax);
    int* ints = b.take<int>(4);
    d.kU = ints;
    d.kV = ints ? ints + 1 : nullptr;
    d.rows_u = ints ? ints + 2 : nullptr;
    d.rows_v = ints ? ints + 3 : nullptr;
  }
  L.dnodes = b.take<HssNodeDev>(nn);
  L.tab = b.take<unsigned char>(kTabBytes);
  L.idscratch = b.take<double>((size_t)nn * 2 * rp * rmax);
  L.lists = b.take<int>((size_t)4 * nn + 8);
  L.bytes = b.off;
}

}  // namespace

// The largest sample an HSS merge may grow to: r + p doubled hss_grow times.
int hss_rp_max(const tdc_opts& o) { return o.hss_rp << std::max(0, std::min(o.hss_grow, 4)); }

// The split-precision GEMMs of an HSS merge (every product of the sampling, the
// compression and the multiply) use 7 slices: the sampled Y feeds rank decisions at the
// compression tolerance, and 6 slices left noise of about 2e-12 relative in Y at
// K = 16384; the multiply's products write the eigenvectors themselves.
constexpr int kHssSlices = 7;

// Workspace of the split GEMMs of one HSS merge of order m (K <= m kept columns, rp
// samples, leaves of at most hss_leaf): the largest of its batches, sized on the tree of
// K = m (which has the most nodes on every level) with every leaf at the full leaf size:
// the sampling (Qhat Omega1, Qhat^T Omega2), one level's hats (V^T S, U^T S), one level of
// the up-sweep (X(:, t) U_t or [G_1 G_2] U_p), one level's couplings (G B and F V^T), the
// leaves' X(:, t) D_t and their F_t V_t^T.
static size_t hss_split_bytes(int64_t m, const tdc_opts& o, int rp) {
  const int hl = std::max(o.hss_leaf, 2);
  const int mi = (int)m, kin = std::max(hl, 2 * rp);
  std::vector<HNodeHost> tree;
  build_tree(tree, 0, std::max(mi, 1), 0, hl);
  int maxlev = 0, nleaves = 0;
  for (const HNodeHost& h : tree) {
    maxlev = std::max(maxlev, h.level);
    nleaves += h.c1 < 0;
  }
  std::vector<int> nodes(maxlev + 1, 0), parents(maxlev + 1, 0);
  for (const HNodeHost& h : tree) {
    nodes[h.level] += 1;
    parents[h.level] += h.c1 >= 0;
  }
  auto batch = [&](int count, int M, int N, int K) {
    std::vector<SgProblem> v((size_t)std::max(count, 0), sg_problem(M, N, K, SgOp{}, SgOp{}, nullptr, 0));
    return v.empty() ? size_t(0) : split_gemm_bytes(v, kHssSlices);
  };
  size_t b = batch(2, mi, rp, mi);
  b = std::max(b, batch(nleaves, mi, hl, hl));
  b = std::max(b, batch(nleaves, mi, hl, rp));
  for (int l = 0; l <= maxlev; ++l) {
    b = std::max(b, batch(2 * nodes[l], rp, rp, kin));
    b = std::max(b, batch(nodes[l], mi, rp, kin) + batch(nodes[l] - parents[l], mi, hl, hl));
    b = std::max(b, batch(2 * parents[l], mi, rp, rp));
  }
  return b;
}

size_t hss_arena_bytes(int64_t m, const tdc_opts& o) {
  HssLayout L;
  hss_layout(L, nullptr, (int)m, (int)m, o, hss_rp_max(o));   // every layout fits in the largest
  return L.bytes + 4096 + hss_split_bytes(m, o, hss_rp_max(o)) + 256;
}

// 1 in *flag if a node's row or column ID used all rp samples while it had more rows
// than that: the sampled range may then miss part of the block, and the compression
// cannot be trusted at the tolerance (the root has no ID).
__global__ void k_hss_saturated(const HssNodeDev* __restrict__ nd, int nn, int rp, int* __restrict__ flag) {
  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const HssNodeDev& d = nd[i];
    if (d.root) continue;
    const int ru = d.leaf ? d.hi - d.lo : *d.rows_u;
    const int rv = d.leaf ? d.hi - d.lo : *d.rows_v;
    if ((*d.kU >= rp && ru > rp) || (*d.kV >= rp && rv > rp)) atomicOr(flag, 1);
  }
}

void k_hss_saturated_zero(int* flag, cudaStream_t st) { cudaMemsetAsync(flag, 0, sizeof(int), st); }

int run_hss_merge(const MergeJob& hJ, QBufs qb, DevWs w, unsigned char* arena, size_t arena_bytes,
                  const tdc_opts& o, cudaStream_t st) {
  // K is needed on the host to shape the HSS tree
  int* dK = reinterpret_cast<int*>(arena);
  k_read_k<<<1, 1, 0, st>>>(w.scal, hJ.mid, dK);
  int K = 0;
  cudaMemcpyAsync(&K, dK, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return 4;
  if (K == 0) return 0;
  const int m = hJ.n1 + hJ.n2;
  const int64_t o_v = hJ.v_off;
  QhatSrc q{w.wptr + o_v, w.sinv + o_v};
  double* const* outp = w.outptr + o_v;     // output column of each kept eigenpair
  HssLayout L;
  HssCols xc{};
  int nn = 0, maxlev = 0, rp = o.hss_rp, rmax = 0;
  size_t toff = 0;
  unsigned char* tab = nullptr;
  std::vector<std::vector<int>> byl;
  // Algorithm 1 with r + p = rp sample columns, then the check of the ID ranks against
  // the sample count.  Returns 0, kHssSaturated, 3 or 4.
  unsigned char* split_ws = nullptr;       // the split GEMMs' workspace, after the layout
  size_t split_bytes = 0;
  auto compress = [&]() -> int {
    rmax = std::max(std::max(o.hss_leaf, 2), 2 * rp);
    hss_layout(L, arena, K, m, o, rp);
    if (L.bytes > arena_bytes) return 3;
    const size_t so = (L.bytes + 4095) & ~size_t(255);
    split_ws = arena + so;
    split_bytes = arena_bytes > so ? arena_bytes - so : 0;
    nn = (int)L.tree.size();
    const auto& tree = L.tree;
    auto& nd = L.nd;
    xc = L.xc;
    xc.n1 = hJ.n1;
    cudaMemcpyAsync(L.dnodes, nd.data(), nn * sizeof(HssNodeDev), cudaMemcpyHostToDevice, st);
    toff = 0;
    tab = L.tab;

    // ---- sampling: Omega, Y = Qhat Omega1, Z = Qhat^T Omega2 (column c of Omega does
    // not depend on rp, so a grown sample extends the previous one)
    phase_mark(10, true, 0, st);
    hss_sampling_flops_add(4.0 * (double)K * (double)K * (double)rp);
    const uint64_t seed = 0x5EEDull + (uint64_t)hJ.mid;
    k_hss_omega<<<grid_cap((int64_t)K * rp / 256 + 1, 8), 256, 0, st>>>(L.om1, K, rp, seed, 1);
    k_hss_omega<<<grid_cap((int64_t)K * rp / 256 + 1, 8), 256, 0, st>>>(L.om2, K, rp, seed, 2);
    k_hss_cols<<<grid_cap(K / 256 + 1, 4), 256, 0, st>>>(hJ, w, xc);
    // on the split-precision tensor-core GEMM, with Qhat's diagonal leaf blocks read as
    // zero: Y and Z are then the leaves' Phi = Y(t) - D_t Omega1(t) and
    // Theta = Z(t) - D_t^T Omega2(t) without the subtraction
    maxlev = 0;
    for (int i = 0; i < nn; ++i) maxlev = std::max(maxlev, tree[i].level);
    byl.assign(maxlev + 1, {});
    for (int i = 0; i < nn; ++i) byl[tree[i].level].push_back(i);
    {
      std::vector<int32_t> lid(K);
      for (int i = 0; i < nn; ++i)
        if (nd[i].leaf)
          for (int j = tree[i].lo; j < tree[i].hi; ++j) lid[j] = i;
      cudaMemcpyAsync(L.lid, lid.data(), (size_t)K * 4, cudaMemcpyHostToDevice, st);
      // Qhat = W diag(sinv) (W the unscaled Cauchy columns): Y = W (diag(sinv) Omega1)
      // and Z = diag(sinv) W^T Omega2, so the K^2 slicing reads W alone and the
      // 1/||.|| factors go to Omega1's rows and Z's rows (K (r + p) products each)
      SgOp qa;
      qa.mode = SG_QHAT_RAW;
      qa.wcol = q.wcol;
      qa.lid = nn > 1 ? L.lid : nullptr;
      SgOp qt = qa;
      qt.mode = SG_QHAT_T_RAW;
      SgOp o1 = sg_dense(L.om1, K);
      o1.mode = SG_DENSE_RS;
      o1.rs = q.sinv;
      std::vector<SgProblem> g{sg_problem(K, rp, K, qa, o1, L.Y, K),
                               sg_problem(K, rp, K, qt, sg_dense(L.om2, K), L.Z, K)};
      g[1].crow = q.sinv;
      const int rc = split_gemm(g, kHssSlices, split_ws, split_bytes, w.status + hJ.prob, st);
      if (rc) return rc == 3 ? 3 : 4;
    }
    phase_mark(10, false, 6, st);
    phase_mark(11, true, 0, st);
    // ---- interpolative decompositions, leaves to root
    const size_t id_smem = (size_t)(rmax + rp) * 8 + (size_t)rmax * 4 + 64;
    int* lp = L.lists;
    for (int lev = maxlev; lev >= 1; --lev) {
      std::vector<int> parents, all;
      for (int i : byl[lev]) {
        all.push_back(i);
        if (!nd[i].leaf) parents.push_back(i);
      }
      if (!parents.empty()) {
        cudaMemcpyAsync(lp, parents.data(), parents.size() * 4, cudaMemcpyHostToDevice, st);
        const dim3 pg((unsigned)parents.size(), kParentParts);
        k_hss_couple<<<pg, 256, 0, st>>>(L.dnodes, lp, rp, q);
        k_hss_parent<<<pg, 256, 0, st>>>(L.dnodes, lp, rp);
        lp += parents.size();
      }
      std::vector<HIdJob> ids;
      for (int i : all) {
        HIdJob u;
        std::memset(&u, 0, sizeof(u));
        u.phi = nd[i].phi;
        u.ld = nd[i].ldphi;
        u.rows = nd[i].leaf ? tree[i].hi - tree[i].lo : 0;
        u.rows_dev = nd[i].leaf ? nullptr : nd[i].rows_u;
        u.rows_max = rmax;
        u.U = nd[i].U;
        u.rank_out = nd[i].kU;
        u.skel_local = nd[i].Iloc;
        u.scratch = L.idscratch + (size_t)(2 * i) * rp * rmax;
        ids.push_back(u);
        HIdJob v = u;
        v.phi = nd[i].theta;
        v.rows_dev = nd[i].leaf ? nullptr : nd[i].rows_v;
        v.U = nd[i].V;
        v.rank_out = nd[i].kV;
        v.skel_local = nd[i].Jloc;
        v.scratch = L.idscratch + (size_t)(2 * i + 1) * rp * rmax;
        ids.push_back(v);
      }
      toff = (toff + 255) & ~size_t(255);
      if (toff + ids.size() * sizeof(HIdJob) > kTabBytes) return 3;
      HIdJob* did = reinterpret_cast<HIdJob*>(tab + toff);
      cudaMemcpyAsync(did, ids.data(), ids.size() * sizeof(HIdJob), cudaMemcpyHostToDevice, st);
      toff += ids.size() * sizeof(HIdJob);
      IdClShape ish;
      const int cs = id_cl_pick((int)ids.size(), rmax, rp, &ish);
      if (cs == 0 || launch_id_cl(did, (int)ids.size(), cs, ish, o.hss_tol, rp, st) != cudaSuccess) {
        cudaGetLastError();
        k_hss_id<<<(unsigned)ids.size(), 256, id_smem, st>>>(did, o.hss_tol, rp);
      }
      cudaMemcpyAsync(lp, all.data(), all.size() * 4, cudaMemcpyHostToDevice, st);
      k_hss_skel<<<(unsigned)all.size(), 128, 0, st>>>(L.dnodes, lp);
      lp += all.size();
      // Yhat = V^T S1, Zhat = U^T S2 with S = the node's rows of Omega (leaf) or its
      // children's stacked Yhat / Zhat (parent)
      std::vector<SgProblem> hg;
      for (int i : all) {
        SgProblem y = sg_problem(rp, rp, 0, sg_dense(nd[i].V, nd[i].ldU, true), SgOp{}, nd[i].Yh, rp);
        y.Mdev = nd[i].kV;
        SgProblem z = y;
        z.a.p = nd[i].U;
        z.C = nd[i].Zh;
        z.Mdev = nd[i].kU;
        if (nd[i].leaf) {
          y.K = z.K = tree[i].hi - tree[i].lo;
          y.b = sg_dense(L.om1, K);
          z.b = sg_dense(L.om2, K);
          y.b.r0 = z.b.r0 = tree[i].lo;
        } else {
          const int c1 = tree[i].c1, c2 = tree[i].c2;
          y.K = z.K = 2 * rp;
          y.Kdev = nd[i].rows_v;
          z.Kdev = nd[i].rows_u;
          y.b.mode = z.b.mode = SG_STACK_ROWS;
          y.b.p = nd[c1].Yh; y.b.p2 = nd[c2].Yh; y.b.split = nd[c1].kV;
          z.b.p = nd[c1].Zh; z.b.p2 = nd[c2].Zh; z.b.split = nd[c1].kU;
          y.b.ld = y.b.ld2 = z.b.ld = z.b.ld2 = rp;
        }
        hg.push_back(y);
        hg.push_back(z);
      }
      const int rc = split_gemm(hg, kHssSlices, split_ws, split_bytes, w.status + hJ.prob, st);
      if (rc) return rc == 3 ? 3 : 4;
    }
    const int root = L.root;
    if (!nd[root].leaf) {                       // root: couplings of its children only
      cudaMemcpyAsync(lp, &root, 4, cudaMemcpyHostToDevice, st);
      k_hss_couple<<<dim3(1, kParentParts), 256, 0, st>>>(L.dnodes, lp, rp, q);
      lp += 1;
    }
    if (nn > 1) k_hss_saturated_zero(L.dK, st);
    if (nn > 1) k_hss_saturated<<<1, 256, 0, st>>>(L.dnodes, nn, rp, L.dK);
    phase_mark(11, false, 8 * maxlev + 2, st);
    if (nn > 1) {                               // ranks that reached the sample count
      int sat = 0;
      cudaMemcpyAsync(&sat, L.dK, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) return 4;
      if (sat) return kHssSaturated;
    }
    return 0;
  };
  // Adaptive sampling (Section 2.1): while an ID rank reaches the sample count, double
  // r + p and compress again, at most hss_grow times; then the caller's dense product.
  for (int g = 0;; ++g) {
    const int rc = compress();
    if (rc == 0) break;
    if (rc != kHssSaturated) return rc;
    if (g >= std::max(0, std::min(o.hss_grow, 4))) return kHssSaturated;
    hss_regrowths_add(1);
    rp *= 2;
  }
  const auto& tree = L.tree;
  auto& nd = L.nd;
  phase_mark(12, true, 0, st);

  // ---- multiply: Out = X Qhat_hss, X = Q_sel (m rows, K kept columns), every product
  // on the split-precision tensor-core GEMM
  int nmul = 0;
  auto run_split = [&](std::vector<SgProblem>& g) -> int {
    if (g.empty()) return 0;
    nmul += 3;
    const int rc = split_gemm(g, kHssSlices, split_ws, split_bytes, w.status + hJ.prob, st);
    return rc == 0 ? 0 : (rc == 3 ? 3 : 4);
  };
  SgOp xo;                                  // gathered columns of Q_sel (kept order)
  xo.mode = SG_XCOLS;
  xo.xcol = xc.col;
  xo.xlo = xc.lo;
  xo.xhi = xc.hi;
  // X(:, t) D_t, the leaf's own block of the output (overwritten here; the down-sweep's
  // F_t V_t^T is added at the end), reusing the slices of X(:, t) of its G = X(:, t) U
  auto leaf_d = [&](int i, SgOp xa) {
    SgOp db;
    db.mode = SG_QHAT;
    db.r0 = tree[i].lo;
    db.c0 = tree[i].lo;
    db.wcol = q.wcol;
    db.sinv = q.sinv;
    const int sz = tree[i].hi - tree[i].lo;
    SgProblem p = sg_problem(m, sz, sz, xa, db, nullptr, 0);
    p.cptrs = outp;
    p.cc0 = tree[i].lo;
    return p;
  };
  for (int lev = maxlev; lev >= 1; --lev) {   // up-sweep: G = X(:, t) U, G_p = [G_1 G_2] U_p
    std::vector<SgProblem> g;
    for (int i : byl[lev]) {
      SgProblem p;
      if (nd[i].leaf) {
        SgOp xa = xo;
        xa.c0 = tree[i].lo;
        p = sg_problem(m, rp, tree[i].hi - tree[i].lo, xa, sg_dense(nd[i].U, rmax), nd[i].G, m);
        p.Ndev = nd[i].kU;
        g.push_back(p);
        SgProblem dp = leaf_d(i, xa);
        dp.a_from = (int)g.size() - 1;
        g.push_back(dp);
        continue;
      } else {
        SgOp a;
        a.mode = SG_STACK;
        a.p = nd[tree[i].c1].G;
        a.p2 = nd[tree[i].c2].G;
        a.ld = a.ld2 = m;
        a.split = nd[tree[i].c1].kU;
        p = sg_problem(m, rp, 2 * rp, a, sg_dense(nd[i].U, rmax), nd[i].G, m);
        p.Kdev = nd[i].rows_u;
      }
      p.Ndev = nd[i].kU;
      g.push_back(p);
    }
    if (const int rc = run_split(g)) return rc;
  }
  for (int lev = 0; lev < maxlev; ++lev) {     // couplings and down-sweep, root to leaves
    std::vector<SgProblem> g1, g2;
    for (int p : byl[lev]) {
      if (nd[p].leaf) continue;
      const int c1 = tree[p].c1, c2 = tree[p].c2;
      for (int side = 0; side < 2; ++side) {
        const int dst = side ? c2 : c1, src = side ? c1 : c2;
        // F_dst = G_src B_src
        SgProblem a = sg_problem(m, rp, rp, sg_dense(nd[src].G, m), sg_dense(nd[src].B, rp), nd[dst].F, m);
        a.Ndev = nd[dst].kV;
        a.Kdev = nd[src].kU;
        g1.push_back(a);
        if (!nd[p].root) {                     // F_dst += F_p V_p(rows of dst)^T
          SgProblem b = sg_problem(m, rp, rp, sg_dense(nd[p].F, m), sg_dense(nd[p].V, rmax, true), nd[dst].F, m);
          b.b.off_dev = side ? nd[c1].kV : nullptr;
          b.Ndev = nd[dst].kV;
          b.Kdev = nd[p].kV;
          b.beta = 1.0;
          g2.push_back(b);
        }
      }
    }
    if (const int rc = run_split(g1)) return rc;
    if (const int rc = run_split(g2)) return rc;
  }
  {                                             // leaves: Out(:, pos(t)) += F_t V_t^T
    std::vector<SgProblem> g;
    for (int i = 0; i < nn; ++i) {
      if (!nd[i].leaf) continue;
      const int lo = tree[i].lo, sz = tree[i].hi - tree[i].lo;
      if (nn == 1) {                            // a single leaf: Out = X Qhat
        SgOp xa = xo;
        xa.c0 = lo;
        g.push_back(leaf_d(i, xa));
        continue;
      }
      SgProblem b = sg_problem(m, sz, rp, sg_dense(nd[i].F, m), sg_dense(nd[i].V, rmax, true), nullptr, 0);
      b.Kdev = nd[i].kV;
      b.cptrs = outp;
      b.cc0 = lo;
      b.beta = 1.0;
      g.push_back(b);
    }
    if (const int rc = run_split(g)) return rc;
  }
  phase_mark(12, false, nmul, st);
  return toff > kTabBytes ? 3 : 0;
}

}  // namespace tdc
