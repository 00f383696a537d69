// HSS form of the eigenvector product (Section 2, Algorithm 1 and the fast
// multiply): Qhat (K x K, never stored) is compressed by randomized sampling and
// interpolative decompositions, then U = Q_sel Qhat_hss is formed with an up-sweep
// through the nested bases U, the sibling couplings B and a down-sweep through V.
// Qhat stays in the order of the sorted d (no Gu grouping: it would break the
// off-diagonal low rank).  Everything runs in FP64:
//   k_hss_omega   Gaussian sampling matrices (SplitMix64 + Box-Muller)
//   k_hss_gemm    batched FP64 GEMM whose operands may be dense, transposed,
//                 Qhat blocks generated on the fly, gathered columns of Q_sel, or two
//                 stacked blocks; the output may be scattered to eigenvector columns
//   k_hss_id      batched column-pivoted QR of Phi^T: row ID Phi ~= U Phi(I, :)
//   k_hss_parent  per parent: sibling couplings B and the parent's Phi, Theta
//   k_hss_hat     per parent: Yhat = V^T [Yhat_1; Yhat_2], Zhat = U^T [Zhat_1; Zhat_2]
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

// ------------------------------------------------------------------ batched GEMM
__device__ __forceinline__ double fetch(const HOp& op, const QhatSrc& q, const HssCols& xc, int r, int c) {
  switch (op.mode) {
    case HOP_DENSE: return op.p[(int64_t)(op.c0 + c) * op.ld + op.r0 + r];
    case HOP_DENSE_T: {
      const int c0 = op.c0 + (op.row_off_dev ? *op.row_off_dev : 0);
      return op.p[(int64_t)(op.r0 + r) * op.ld + c0 + c];
    }
    case HOP_QHAT: {
      const int j = op.ridx ? op.ridx[r] : op.r0 + r;
      const int i = op.cidx ? op.cidx[c] : op.c0 + c;
      return qhat(q, j, i);
    }
    case HOP_QHAT_T: {
      const int j = op.cidx ? op.cidx[c] : op.c0 + c;
      const int i = op.ridx ? op.ridx[r] : op.r0 + r;
      return qhat(q, j, i);
    }
    case HOP_XCOLS: {
      const int j = op.c0 + c;                 // kept (sorted-d) column index
      return r >= xc.lo[j] && r < xc.hi[j] ? xc.col[j][r] : 0.0;
    }
    case HOP_STACK: {                          // columns [0, k1) from p, the rest from p2
      const int k1 = *op.split;
      return c < k1 ? op.p[(int64_t)c * op.ld + r] : op.p2[(int64_t)(c - k1) * op.ld2 + r];
    }
    case HOP_STACK_ROWS: {                     // rows [0, k1) from p, the rest from p2
      const int k1 = *op.split;
      return r < k1 ? op.p[(int64_t)c * op.ld + r] : op.p2[(int64_t)c * op.ld2 + (r - k1)];
    }
    default: return 0.0;
  }
}

constexpr int TB = 64, TK = 16;

// Whether consecutive k of an operand are adjacent in memory (then the tile loader
// walks k fastest across threads, else the row / column index), so that a warp's loads
// fall on few cache lines.  A is read as a(r, k), B as b(k, c).
__device__ __forceinline__ bool a_k_contiguous(int mode) { return mode == HOP_DENSE_T || mode == HOP_QHAT_T; }
__device__ __forceinline__ bool b_k_contiguous(int mode) { return mode != HOP_DENSE_T && mode != HOP_QHAT_T; }

__global__ __launch_bounds__(256) void k_hss_gemm(const HGemm* __restrict__ jobs, int njobs,
                                                  const int64_t* __restrict__ cum, QhatSrc q, HssCols xc) {
  __shared__ double As[TK][TB + 1];
  __shared__ double Bs[TK][TB + 1];
  const int jb = find_job(cum, njobs, blockIdx.x);
  const HGemm G = jobs[jb];
  const int64_t t = blockIdx.x - cum[jb];
  const int M = G.Mdev ? *G.Mdev : G.M;
  const int N = G.Ndev ? *G.Ndev : G.N;
  const int Kd = G.Kdev ? *G.Kdev : G.K;
  const int ntm = (G.M + TB - 1) / TB;
  const int tm = (int)(t % ntm), tn = (int)(t / ntm);
  const int r0 = tm * TB, c0 = tn * TB;
  if (r0 >= M || c0 >= N) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  const bool ak = a_k_contiguous(G.a.mode), bk = b_k_contiguous(G.b.mode);   // uniform per job
  for (int k0 = 0; k0 < Kd; k0 += TK) {
    for (int e = tid; e < TK * TB; e += 256) {
      const int kk = ak ? e % TK : e / TB, rr = ak ? e / TK : e % TB;
      const int r = r0 + rr, k = k0 + kk;
      As[kk][rr] = (r < M && k < Kd) ? fetch(G.a, q, xc, r, k) : 0.0;
    }
    for (int e = tid; e < TK * TB; e += 256) {
      const int kk = bk ? e % TK : e / TB, cc = bk ? e / TK : e % TB;
      const int c = c0 + cc, k = k0 + kk;
      Bs[kk][cc] = (c < N && k < Kd) ? fetch(G.b, q, xc, k, c) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double fa[4], fb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) fa[a] = As[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) fb[b] = Bs[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(fa[a], fb[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int c = c0 + ty + 16 * b;
    if (c >= N) continue;
    double* col;
    if (G.cmode == HC_SCATTER) col = G.C + (int64_t)G.cpos[G.cc0 + c] * G.ldc;
    else if (G.cmode == HC_PTRS) col = G.cptrs[G.cc0 + c];
    else col = G.C + (int64_t)c * G.ldc;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = r0 + tx + 16 * a;
      if (r >= M) continue;
      const double v = G.alpha * acc[a][b];
      col[r] = G.beta == 0.0 ? v : v + G.beta * col[r];
    }
  }
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

// ------------------------------------------------------------------ parent steps
// B_{c1} = Qhat(I_c1, J_c2), B_{c2} = Qhat(I_c2, J_c1), and (unless root)
//   Phi_p   = [Phi_c1(Iloc_c1) - B_c1 Yhat_c2 ; Phi_c2(Iloc_c2) - B_c2 Yhat_c1]
//   Theta_p = [Theta_c1(Jloc_c1) - B_c2^T Zhat_c2 ; Theta_c2(Jloc_c2) - B_c1^T Zhat_c1]
__global__ __launch_bounds__(256) void k_hss_parent(const HssNodeDev* __restrict__ nodes,
                                                    const int* __restrict__ plist, int rp, QhatSrc q) {
  const HssNodeDev P = nodes[plist[blockIdx.x]];
  const HssNodeDev A = nodes[P.c1], Bn = nodes[P.c2];
  const int ku1 = *A.kU, kv1 = *A.kV, ku2 = *Bn.kU, kv2 = *Bn.kV;
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int e = tid; e < ku1 * kv2; e += NT) {
    const int r = e % ku1, c = e / ku1;
    A.B[(int64_t)c * rp + r] = qhat(q, A.I[r], Bn.J[c]);
  }
  for (int e = tid; e < ku2 * kv1; e += NT) {
    const int r = e % ku2, c = e / ku2;
    Bn.B[(int64_t)c * rp + r] = qhat(q, Bn.I[r], A.J[c]);
  }
  __syncthreads();
  if (P.root) return;
  // Phi_p rows: first ku1 from child 1, then ku2 from child 2
  for (int e = tid; e < (ku1 + ku2) * rp; e += NT) {
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
  for (int e = tid; e < (kv1 + kv2) * rp; e += NT) {
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
  if (tid == 0) {
    *P.rows_u = ku1 + ku2;
    *P.rows_v = kv1 + kv2;
  }
  // skeleton candidates of the parent (global indices), in row order of Phi_p
  for (int r = tid; r < ku1 + ku2; r += NT) P.Icand[r] = r < ku1 ? A.I[r] : Bn.I[r - ku1];
  for (int r = tid; r < kv1 + kv2; r += NT) P.Jcand[r] = r < kv1 ? A.J[r] : Bn.J[r - kv1];
}

// After a node's IDs: global skeleton indices, and Yhat, Zhat.
//   leaf:   I = lo + Iloc,  Yhat = V^T Omega1(t),       Zhat = U^T Omega2(t)
//   parent: I = Icand(Iloc), Yhat = V^T [Yhat_1; Yhat_2], Zhat = U^T [Zhat_1; Zhat_2]
__global__ __launch_bounds__(256) void k_hss_hat(const HssNodeDev* __restrict__ nodes,
                                                 const int* __restrict__ list, int rp,
                                                 const double* __restrict__ om1,
                                                 const double* __restrict__ om2, int64_t K) {
  const HssNodeDev N = nodes[list[blockIdx.x]];
  const int tid = threadIdx.x, NT = blockDim.x;
  const int ku = *N.kU, kv = *N.kV;
  const int ru = N.leaf ? N.hi - N.lo : *N.rows_u;
  const int rv = N.leaf ? N.hi - N.lo : *N.rows_v;
  for (int t = tid; t < ku; t += NT) N.I[t] = N.leaf ? N.lo + N.Iloc[t] : N.Icand[N.Iloc[t]];
  for (int t = tid; t < kv; t += NT) N.J[t] = N.leaf ? N.lo + N.Jloc[t] : N.Jcand[N.Jloc[t]];
  int k1u = 0, k1v = 0;
  const double *y1 = nullptr, *y2 = nullptr, *z1 = nullptr, *z2 = nullptr;
  if (!N.leaf) {
    const HssNodeDev A = nodes[N.c1], Bn = nodes[N.c2];
    k1v = *A.kV;
    k1u = *A.kU;
    y1 = A.Yh; y2 = Bn.Yh; z1 = A.Zh; z2 = Bn.Zh;
  }
  for (int e = tid; e < kv * rp; e += NT) {       // Yhat = V^T (stack), kv x rp
    const int r = e % kv, c = e / kv;
    double s = 0.0;
    for (int t = 0; t < rv; ++t) {
      double x;
      if (N.leaf) x = om1[(int64_t)c * K + N.lo + t];
      else x = t < k1v ? y1[(int64_t)c * rp + t] : y2[(int64_t)c * rp + (t - k1v)];
      s += N.V[(int64_t)r * N.ldU + t] * x;
    }
    N.Yh[(int64_t)c * rp + r] = s;
  }
  for (int e = tid; e < ku * rp; e += NT) {       // Zhat = U^T (stack), ku x rp
    const int r = e % ku, c = e / ku;
    double s = 0.0;
    for (int t = 0; t < ru; ++t) {
      double x;
      if (N.leaf) x = om2[(int64_t)c * K + N.lo + t];
      else x = t < k1u ? z1[(int64_t)c * rp + t] : z2[(int64_t)c * rp + (t - k1u)];
      s += N.U[(int64_t)r * N.ldU + t] * x;
    }
    N.Zh[(int64_t)c * rp + r] = s;
  }
}

__global__ void k_read_k(const MergeScalars* scal, int64_t mid, int* out) { *out = scal[mid].K; }

int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

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

void launch_gemms(const std::vector<HGemm>& g, unsigned char* dev_tab, size_t& tab_off, QhatSrc q,
                  HssCols xc, cudaStream_t st) {
  if (g.empty()) return;
  std::vector<int64_t> cum(g.size() + 1, 0);
  for (size_t i = 0; i < g.size(); ++i) cum[i + 1] = cum[i] + cdiv64(g[i].M, TB) * cdiv64(g[i].N, TB);
  tab_off = (tab_off + 255) & ~size_t(255);
  HGemm* dj = reinterpret_cast<HGemm*>(dev_tab + tab_off);
  tab_off += g.size() * sizeof(HGemm);
  tab_off = (tab_off + 255) & ~size_t(255);
  int64_t* dc = reinterpret_cast<int64_t*>(dev_tab + tab_off);
  tab_off += cum.size() * 8;
  if (tab_off > kTabBytes) return;
  cudaMemcpyAsync(dj, g.data(), g.size() * sizeof(HGemm), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dc, cum.data(), cum.size() * 8, cudaMemcpyHostToDevice, st);
  if (cum.back() > 0) k_hss_gemm<<<(unsigned)cum.back(), 256, 0, st>>>(dj, (int)g.size(), dc, q, xc);
}

HGemm gemm0() {
  HGemm g;
  std::memset(&g, 0, sizeof(g));
  g.alpha = 1.0;
  return g;
}

}  // namespace

void launch_dense_gemms(const std::vector<HGemm>& g, unsigned char* dev_tab, size_t& tab_off,
                        cudaStream_t st) {
  QhatSrc q{};
  HssCols xc{};
  launch_gemms(g, dev_tab, tab_off, q, xc, st);
}

// The largest sample an HSS merge may grow to: r + p doubled hss_grow times.
int hss_rp_max(const tdc_opts& o) { return o.hss_rp << std::max(0, std::min(o.hss_grow, 4)); }

// The split-precision GEMMs of an HSS merge (sampling, and the leaf-level products of
// the multiply) use 7 slices: the sampled Y feeds rank decisions at the compression
// tolerance, and 6 slices left noise of about 2e-12 relative in Y at K = 16384.
constexpr int kHssSlices = 7;

// Workspace of the split GEMMs of one HSS merge of order m (K <= m kept columns, rp
// samples, leaves of at most hss_leaf): the larger of the sampling batch (Qhat Omega1,
// Qhat^T Omega2) and a leaf batch (X(:, t) D_t or X(:, t) U_t for every leaf t).
static size_t hss_split_bytes(int64_t m, const tdc_opts& o, int rp) {
  const int hl = std::max(o.hss_leaf, 2);
  std::vector<SgProblem> sampling(2, sg_problem((int)m, rp, (int)m, SgOp{}, SgOp{}, nullptr, 0));
  std::vector<SgProblem> leaves;
  for (int64_t lo = 0; lo < m; lo += hl) {
    const int sz = (int)std::min<int64_t>(hl, m - lo);
    leaves.push_back(sg_problem((int)m, std::max(sz, rp), sz, SgOp{}, SgOp{}, nullptr, 0));
  }
  return std::max(split_gemm_bytes(sampling, kHssSlices), split_gemm_bytes(leaves, kHssSlices));
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
    {                                           // on the split-precision tensor-core GEMM
      SgOp qa;
      qa.mode = SG_QHAT;
      qa.wcol = q.wcol;
      qa.sinv = q.sinv;
      SgOp qt = qa;
      qt.mode = SG_QHAT_T;
      std::vector<SgProblem> g{sg_problem(K, rp, K, qa, sg_dense(L.om1, K), L.Y, K),
                               sg_problem(K, rp, K, qt, sg_dense(L.om2, K), L.Z, K)};
      const int rc = split_gemm(g, kHssSlices, split_ws, split_bytes, w.status + hJ.prob, st);
      if (rc) return rc == 3 ? 3 : 4;
    }
    // ---- leaves: Phi = Y(t) - D Omega1(t), Theta = Z(t) - D^T Omega2(t), in place
    maxlev = 0;
    for (int i = 0; i < nn; ++i) maxlev = std::max(maxlev, tree[i].level);
    byl.assign(maxlev + 1, {});
    for (int i = 0; i < nn; ++i) byl[tree[i].level].push_back(i);
    if (nn > 1) {
      std::vector<HGemm> g;
      for (int i = 0; i < nn; ++i) {
        if (!nd[i].leaf) continue;
        const int lo = tree[i].lo, sz = tree[i].hi - tree[i].lo;
        HGemm a = gemm0();
        a.M = sz; a.N = rp; a.K = sz;
        a.a.mode = HOP_QHAT; a.a.r0 = lo; a.a.c0 = lo;
        a.b.mode = HOP_DENSE; a.b.p = L.om1; a.b.ld = K; a.b.r0 = lo;
        a.C = L.Y + lo; a.ldc = K; a.alpha = -1.0; a.beta = 1.0;
        g.push_back(a);
        HGemm b = a;
        b.a.mode = HOP_QHAT_T;
        b.b.p = L.om2;
        b.C = L.Z + lo;
        g.push_back(b);
      }
      launch_gemms(g, tab, toff, q, xc, st);
    }
    phase_mark(10, false, 5, st);
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
        k_hss_parent<<<(unsigned)parents.size(), 256, 0, st>>>(L.dnodes, lp, rp, q);
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
      k_hss_id<<<(unsigned)ids.size(), 256, id_smem, st>>>(did, o.hss_tol, rp);
      cudaMemcpyAsync(lp, all.data(), all.size() * 4, cudaMemcpyHostToDevice, st);
      k_hss_hat<<<(unsigned)all.size(), 256, 0, st>>>(L.dnodes, lp, rp, L.om1, L.om2, K);
      lp += all.size();
    }
    const int root = L.root;
    if (!nd[root].leaf) {                       // root: couplings of its children only
      cudaMemcpyAsync(lp, &root, 4, cudaMemcpyHostToDevice, st);
      k_hss_parent<<<1, 256, 0, st>>>(L.dnodes, lp, rp, q);
      lp += 1;
    }
    if (nn > 1) k_hss_saturated_zero(L.dK, st);
    if (nn > 1) k_hss_saturated<<<1, 256, 0, st>>>(L.dnodes, nn, rp, L.dK);
    phase_mark(11, false, 3 * maxlev + 2, st);
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

  // ---- multiply: Out = X Qhat_hss, X = Q_sel (m rows, K kept columns)
  SgOp xo;                                  // gathered columns of Q_sel (kept order)
  xo.mode = SG_XCOLS;
  xo.xcol = xc.col;
  xo.xlo = xc.lo;
  xo.xhi = xc.hi;
  for (int lev = maxlev; lev >= 1; --lev) {   // up-sweep: G = X(:, t) U, G_p = [G_1 G_2] U_p
    std::vector<HGemm> g;
    std::vector<SgProblem> gl;                // leaves: on the split-precision GEMM
    for (int i : byl[lev]) {
      if (nd[i].leaf) {
        SgOp xa = xo;
        xa.c0 = tree[i].lo;
        SgProblem p = sg_problem(m, rp, tree[i].hi - tree[i].lo, xa, sg_dense(nd[i].U, rmax), nd[i].G, m);
        p.Ndev = nd[i].kU;
        gl.push_back(p);
        continue;
      }
      HGemm a = gemm0();
      a.M = m; a.N = rp; a.Ndev = nd[i].kU;
      a.C = nd[i].G; a.ldc = m;
      a.b.mode = HOP_DENSE; a.b.p = nd[i].U; a.b.ld = rmax;
      a.K = 2 * rp; a.Kdev = nd[i].rows_u;
      a.a.mode = HOP_STACK; a.a.p = nd[tree[i].c1].G; a.a.ld = m;
      a.a.p2 = nd[tree[i].c2].G; a.a.ld2 = m; a.a.split = nd[tree[i].c1].kU;
      g.push_back(a);
    }
    if (!gl.empty()) {
      const int rc = split_gemm(gl, kHssSlices, split_ws, split_bytes, w.status + hJ.prob, st);
      if (rc) return rc == 3 ? 3 : 4;
    }
    launch_gemms(g, tab, toff, q, xc, st);
  }
  for (int lev = 0; lev < maxlev; ++lev) {     // couplings and down-sweep, root to leaves
    std::vector<HGemm> g1, g2;
    for (int p : byl[lev]) {
      if (nd[p].leaf) continue;
      const int c1 = tree[p].c1, c2 = tree[p].c2;
      for (int side = 0; side < 2; ++side) {
        const int dst = side ? c2 : c1, src = side ? c1 : c2;
        HGemm a = gemm0();                     // F_dst = G_src B_src
        a.M = m; a.N = rp; a.Ndev = nd[dst].kV; a.K = rp; a.Kdev = nd[src].kU;
        a.a.mode = HOP_DENSE; a.a.p = nd[src].G; a.a.ld = m;
        a.b.mode = HOP_DENSE; a.b.p = nd[src].B; a.b.ld = rp;
        a.C = nd[dst].F; a.ldc = m;
        g1.push_back(a);
        if (!nd[p].root) {                     // F_dst += F_p V_p(rows of dst)^T
          HGemm b = gemm0();
          b.M = m; b.N = rp; b.Ndev = nd[dst].kV; b.K = rp; b.Kdev = nd[p].kV;
          b.a.mode = HOP_DENSE; b.a.p = nd[p].F; b.a.ld = m;
          b.b.mode = HOP_DENSE_T; b.b.p = nd[p].V; b.b.ld = rmax;
          b.b.row_off_dev = side ? nd[c1].kV : nullptr;
          b.C = nd[dst].F; b.ldc = m; b.beta = 1.0;
          g2.push_back(b);
        }
      }
    }
    launch_gemms(g1, tab, toff, q, xc, st);
    launch_gemms(g2, tab, toff, q, xc, st);
  }
  {                                             // leaves: Out(:, pos(t)) = X(:, t) D + F V^T
    std::vector<HGemm> g2;
    std::vector<SgProblem> g1;                  // X(:, t) D_t on the split-precision GEMM
    for (int i = 0; i < nn; ++i) {
      if (!nd[i].leaf) continue;
      const int lo = tree[i].lo, sz = tree[i].hi - tree[i].lo;
      SgOp xa = xo;
      xa.c0 = lo;
      SgOp db;
      db.mode = SG_QHAT;
      db.r0 = lo;
      db.c0 = lo;
      db.wcol = q.wcol;
      db.sinv = q.sinv;
      SgProblem p = sg_problem(m, sz, sz, xa, db, nullptr, 0);
      p.cptrs = outp;
      p.cc0 = lo;
      g1.push_back(p);
      if (nn > 1) {
        HGemm b = gemm0();
        b.M = m; b.N = sz; b.K = rp; b.Kdev = nd[i].kV;
        b.a.mode = HOP_DENSE; b.a.p = nd[i].F; b.a.ld = m;
        b.b.mode = HOP_DENSE_T; b.b.p = nd[i].V; b.b.ld = rmax;
        b.cmode = HC_PTRS; b.cptrs = outp; b.cc0 = lo;
        b.beta = 1.0;
        g2.push_back(b);
      }
    }
    const int rc = split_gemm(g1, kHssSlices, split_ws, split_bytes, w.status + hJ.prob, st);
    if (rc) return rc == 3 ? 3 : 4;
    launch_gemms(g2, tab, toff, q, xc, st);
  }
  phase_mark(12, false, 4 * maxlev + 2, st);
  return toff > kTabBytes ? 3 : 0;
}

}  // namespace tdc
