// Adjoint of the eigendecomposition T = Q diag(lambda) Q^T with respect to the
// tridiagonal entries (d, e), formed on the band only:
//     Tbar = Q (diag(lambda_bar) + F o (Q^T Qbar)) Q^T,   F_ic = 1 / (lambda_c - lambda_i), F_ii = 0,
//     dbar_a = Tbar_aa,   ebar_a = Tbar_{a,a+1} + Tbar_{a+1,a}.
// Qbar is typically nonzero in a few columns S: then with P = Q^T Qbar_S,
// M_S = F(:, S) o P and W = Q M_S,
//     dbar_a = sum_i lambda_bar_i Q_ai^2 + sum_{c in S} W_ac Q_{a,c}
//     ebar_a = 2 sum_i lambda_bar_i Q_ai Q_{a+1,i}
//              + sum_{c in S} (W_ac Q_{a+1,c} + W_{a+1,c} Q_{a,c}),
// two n x n x |S| FP64 GEMMs and O(n^2) band sums.  Nothing of the forward merge
// tree is stored: (lambda, Q) are all the backward needs.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "../../include/tdc.h"
#include "tdc_dgemm.cuh"
#include "tdc_internal.cuh"
#include "tdc_ozaki.cuh"

namespace tdc {
namespace {

// Nonzero columns of Qbar (n x n, ld), compacted in ascending order.
__global__ void k_bw_flag(const double* __restrict__ gq, int64_t ld, int64_t n, int* __restrict__ flag) {
  const int64_t c = blockIdx.x;
  bool nz = false;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) nz |= gq[c * ld + r] != 0.0;
  nz = __syncthreads_or(nz);
  if (threadIdx.x == 0) flag[c] = nz ? 1 : 0;
}
__global__ void k_bw_compact(const int* __restrict__ flag, int64_t n, int* __restrict__ cols, int* __restrict__ ns) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int k = 0;
  for (int64_t c = 0; c < n; ++c)
    if (flag[c]) cols[k++] = (int)c;
  *ns = k;
}
// Gathers Qbar(:, S) into a dense n x s block.
__global__ void k_bw_gather(const double* __restrict__ gq, int64_t ld, int64_t n, const int* __restrict__ cols,
                            int s, double* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * s) return;
  const int64_t r = e % n, c = e / n;
  out[e] = gq[(int64_t)cols[c] * ld + r];
}
// M_S(i, c) = P(i, c) / (lambda_{S_c} - lambda_i), zero for i = S_c.
__global__ void k_bw_m(const double* __restrict__ P, const double* __restrict__ lam, const int* __restrict__ cols,
                       int64_t n, int s, double* __restrict__ M) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * s) return;
  const int64_t i = e % n, c = e / n;
  const int sc = cols[c];
  M[e] = (i == sc) ? 0.0 : P[e] / (lam[sc] - lam[i]);
}
// The band of Tbar, one row a per thread.
__global__ void k_bw_band(const double* __restrict__ Q, int64_t ld, int64_t n, const double* __restrict__ lam,
                          const double* __restrict__ glam, const double* __restrict__ W, const int* __restrict__ cols,
                          int s, double* __restrict__ gd, double* __restrict__ ge) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n) return;
  (void)lam;
  const bool has_next = a + 1 < n;
  double dsum = 0.0, esum = 0.0;
  if (glam) {
    for (int64_t i = 0; i < n; ++i) {
      const double qa = Q[i * ld + a];
      const double gl = glam[i];
      dsum += gl * qa * qa;
      if (has_next) esum += gl * qa * Q[i * ld + a + 1];
    }
    esum *= 2.0;
  }
  for (int c = 0; c < s; ++c) {
    const int64_t col = cols[c];
    const double wa = W[(int64_t)c * n + a];
    const double qa = Q[col * ld + a];
    dsum += wa * qa;
    if (has_next) esum += wa * Q[col * ld + a + 1] + W[(int64_t)c * n + a + 1] * qa;
  }
  gd[a] = dsum;
  if (has_next) ge[a] = esum;
}

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// ---------------------------------------------------------------- batched form
// Problem p of a batch: order n, its vectors at v (dense packing: prefix sums of n)
// and its n x n blocks at q (prefix sums of n^2, ld = n); after the column count, its
// s nonzero columns of Qbar are listed at c (prefix sums of n) and its n x s blocks
// G, P, W start at g (prefix sums of n s).
struct BwProb {
  int64_t n, v, q, g;
  int32_t s, pad_;
};

// Column j of the batch (prefix of n): 1 if Qbar's column is nonzero anywhere.
__global__ void k_bwb_flag(const BwProb* __restrict__ pr, int nb, const int64_t* __restrict__ cum_n,
                           const double* __restrict__ gq, int* __restrict__ flag) {
  const int p = find_job(cum_n, nb, blockIdx.x);
  const int64_t c = blockIdx.x - cum_n[p];
  const BwProb P = pr[p];
  bool nz = false;
  for (int64_t r = threadIdx.x; r < P.n; r += blockDim.x) nz |= gq[P.q + c * P.n + r] != 0.0;
  nz = __syncthreads_or(nz);
  if (threadIdx.x == 0) flag[P.v + c] = nz ? 1 : 0;
}

// One block per problem: the nonzero columns in ascending order and their count.
__global__ void k_bwb_compact(BwProb* __restrict__ pr, const int* __restrict__ flag, int* __restrict__ cols) {
  __shared__ int s_warp[32];
  __shared__ int s_base;
  BwProb& P = pr[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) s_base = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < P.n; c0 += blockDim.x) {
    const int64_t c = c0 + tid;
    const int f = c < P.n ? flag[P.v + c] : 0;
    const unsigned b = __ballot_sync(0xffffffffu, f);
    if (lane == 0) s_warp[wid] = __popc(b);
    __syncthreads();
    int before = 0, total = 0;
    for (int w2 = 0; w2 < nw; ++w2) {
      before += w2 < wid ? s_warp[w2] : 0;
      total += s_warp[w2];
    }
    if (f) cols[P.v + s_base + before + __popc(b & ((1u << lane) - 1u))] = (int)c;
    __syncthreads();
    if (tid == 0) s_base += total;
    __syncthreads();
  }
  if (tid == 0) P.s = s_base;
}

// G(:, k) = Qbar(:, cols[k]) for every problem: element e of the batch's n s prefix.
__global__ void k_bwb_gather(const BwProb* __restrict__ pr, int nb, const int64_t* __restrict__ cum_ns,
                             int64_t total, const double* __restrict__ gq, const int* __restrict__ cols,
                             double* __restrict__ G) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int p = find_job(cum_ns, nb, e);
    const BwProb P = pr[p];
    const int64_t l = e - cum_ns[p];
    const int64_t r = l % P.n, k = l / P.n;
    G[P.g + l] = gq[P.q + (int64_t)cols[P.v + k] * P.n + r];
  }
}

// M(i, k) = P(i, k) / (lambda_{cols[k]} - lambda_i), zero for i = cols[k] (overwrites G).
__global__ void k_bwb_m(const BwProb* __restrict__ pr, int nb, const int64_t* __restrict__ cum_ns, int64_t total,
                        const double* __restrict__ Pm, const double* __restrict__ lam, const int* __restrict__ cols,
                        double* __restrict__ M) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int p = find_job(cum_ns, nb, e);
    const BwProb P = pr[p];
    const int64_t l = e - cum_ns[p];
    const int64_t i = l % P.n, k = l / P.n;
    const int c = cols[P.v + k];
    M[P.g + l] = (i == c) ? 0.0 : Pm[P.g + l] / (lam[P.v + c] - lam[P.v + i]);
  }
}

// The band of Tbar, one row a of one problem per thread (the batch's n prefix).
__global__ void k_bwb_band(const BwProb* __restrict__ pr, int nb, const int64_t* __restrict__ cum_n, int64_t total,
                           const double* __restrict__ Q, const double* __restrict__ glam,
                           const double* __restrict__ W, const int* __restrict__ cols, double* __restrict__ gd,
                           double* __restrict__ ge) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int p = find_job(cum_n, nb, e);
  const BwProb P = pr[p];
  const int64_t a = e - cum_n[p], n = P.n;
  const double* Qp = Q + P.q;
  const bool has_next = a + 1 < n;
  double dsum = 0.0, esum = 0.0;
  if (glam) {
    const double* gl = glam + P.v;
    for (int64_t i = 0; i < n; ++i) {
      const double qa = Qp[i * n + a];
      dsum += gl[i] * qa * qa;
      if (has_next) esum += gl[i] * qa * Qp[i * n + a + 1];
    }
    esum *= 2.0;
  }
  const double* Wp = W + P.g;
  for (int k = 0; k < P.s; ++k) {
    const int64_t col = cols[P.v + k];
    const double wa = Wp[(int64_t)k * n + a];
    const double qa = Qp[col * n + a];
    dsum += wa * qa;
    if (has_next) esum += wa * Qp[col * n + a + 1] + Wp[(int64_t)k * n + a + 1] * qa;
  }
  gd[P.v + a] = dsum;
  if (has_next) ge[P.v + a] = esum;
}

constexpr size_t kBwTab = size_t(1) << 22;     // GEMM job tables (the batched GEMM's limit)

struct BwLayout {
  BwProb* prob;
  int64_t* cum;          // cum_n (nb + 1), then cum_ns (nb + 1)
  int* flag;
  int* cols;
  unsigned char* tab;
  double* G;             // sum n s each: G (then M), P, W
  double* P;
  double* W;
  int* status_scratch;   // the split products' wait status when the caller passes none
  size_t fixed;          // bytes before G
};

BwLayout bw_layout(unsigned char* b, int nb, int64_t vtot) {
  BwLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = b ? b + off : nullptr;
    off = al(off + bytes);
    return p;
  };
  L.prob = reinterpret_cast<BwProb*>(take(sizeof(BwProb) * nb));
  L.cum = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * 2 * (nb + 1)));
  L.flag = reinterpret_cast<int*>(take(sizeof(int) * vtot));
  L.cols = reinterpret_cast<int*>(take(sizeof(int) * vtot));
  L.tab = take(kBwTab);
  L.status_scratch = reinterpret_cast<int*>(take(16));
  L.fixed = off;
  return L;
}

}  // namespace
}  // namespace tdc

using namespace tdc;

namespace {
// The backward's two products run on the split-precision tensor-core path when the
// options select the split product (path TDC_PATH_DENSE_OZAKI), in FP64 otherwise.  They
// use 7 slices whatever opts->ozaki_slices says: the eigenvector term multiplies the
// error of Q^T Qbar by 1/(lambda_c - lambda_i), up to about 1e5 on the n = 4096
// configuration, and 6 slices (about 2e-14 per product) left 2e-9 relative in the
// gradient against 2e-10 with 7.
bool bw_split(const tdc_opts* opts) { return opts && opts->path == TDC_PATH_DENSE_OZAKI; }
int bw_slices(const tdc_opts*) { return 7; }
}  // namespace

extern "C" size_t tdc_backward_workspace_bytes(int64_t n, const tdc_opts* opts) {
  if (n < 1) return 0;
  size_t b = al(n * 4) + al(n * 4) + al(16) + 3 * al((size_t)n * n * 8) + al(1 << 20);
  if (bw_split(opts) && n <= INT32_MAX) {
    const std::vector<SgProblem> pr{sg_problem((int)n, (int)n, (int)n, SgOp{}, SgOp{}, nullptr, 0)};
    b += al(split_gemm_bytes(pr, bw_slices(opts)));
  }
  return b;
}

extern "C" int tdc_syev_tridiag_backward(int64_t n, const double* lambda, const double* Q, int64_t ldq,
                                         const double* g_lambda, const double* g_Q, int64_t ldg, double* g_d,
                                         double* g_e, const tdc_opts* opts, void* ws, size_t ws_bytes,
                                         int* dev_status, void* stream) {
  if (n < 1) return -1;
  if (!lambda) return -2;
  if (!Q) return -3;
  if (ldq < n) return -4;
  if (g_Q && ldg < n) return -7;
  if (!g_d) return -8;
  if (!g_e && n > 1) return -9;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return -11;
  if (ws_bytes < tdc_backward_workspace_bytes(n, opts)) return 3;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* b = reinterpret_cast<unsigned char*>(ws);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = b + off;
    off = al(off + bytes);
    return p;
  };
  int* flag = reinterpret_cast<int*>(take(n * 4));
  int* cols = reinterpret_cast<int*>(take(n * 4));
  int* ns_dev = reinterpret_cast<int*>(take(16));
  int s = 0;
  if (g_Q) {
    k_bw_flag<<<(unsigned)n, 256, 0, st>>>(g_Q, ldg, n, flag);
    k_bw_compact<<<1, 32, 0, st>>>(flag, n, cols, ns_dev);
    if (cudaMemcpyAsync(&s, ns_dev, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return 4;
    if (cudaStreamSynchronize(st) != cudaSuccess) return 4;
  }
  double* G = reinterpret_cast<double*>(take((size_t)n * (s > 0 ? s : 1) * 8));
  double* P = reinterpret_cast<double*>(take((size_t)n * (s > 0 ? s : 1) * 8));
  double* W = reinterpret_cast<double*>(take((size_t)n * (s > 0 ? s : 1) * 8));
  unsigned char* tab = take(1 << 20);
  if (off > ws_bytes) return 3;
  if (s > 0) {
    const int64_t ne = n * s;
    k_bw_gather<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(g_Q, ldg, n, cols, s, G);
    if (bw_split(opts)) {
      // the split-precision arena follows the FP64 path's buffers
      unsigned char* arena = b + off;
      const size_t abytes = ws_bytes > off ? ws_bytes - off : 0;
      std::vector<SgProblem> pr{sg_problem((int)n, s, (int)n, sg_dense(Q, ldq, true), sg_dense(G, n), P, n)};   // P = Q^T G
      int* err = dev_status ? dev_status : ns_dev + 1;      // a timed-out tensor-core wait sets bit 8 here
      int rc = split_gemm(pr, bw_slices(opts), arena, abytes, err, st);
      if (rc) return rc;
      k_bw_m<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(P, lambda, cols, n, s, G);   // M_S into G
      pr[0] = sg_problem((int)n, s, (int)n, sg_dense(Q, ldq), sg_dense(G, n), W, n);                  // W = Q M_S
      rc = split_gemm(pr, bw_slices(opts), arena, abytes, err, st);
      if (rc) return rc;
    } else {
      std::vector<DGemm> g(1);
      std::memset(g.data(), 0, sizeof(DGemm));
      g[0].M = (int)n; g[0].N = s; g[0].K = (int)n;          // P = Q^T G
      g[0].a = DMat{Q, ldq, 1};
      g[0].b = DMat{G, n, 0};
      g[0].C = P; g[0].ldc = n; g[0].alpha = 1.0;
      size_t toff = 0;
      if (launch_dgemms(g, tab, toff, 1 << 20, st)) return 3;
      k_bw_m<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(P, lambda, cols, n, s, G);   // M_S into G
      g[0].a = DMat{Q, ldq, 0};                                                           // W = Q M_S
      g[0].C = W;
      if (launch_dgemms(g, tab, toff, 1 << 20, st)) return 3;
    }
  }
  k_bw_band<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Q, ldq, n, lambda, g_lambda, W, cols, s, g_d, g_e);
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

extern "C" size_t tdc_backward_batched_workspace_bytes(int32_t batch, const int64_t* n_host, int64_t max_cols,
                                                       const tdc_opts* opts) {
  if (batch < 1 || !n_host) return 0;
  int64_t vtot = 0, ns = 0;
  for (int p = 0; p < batch; ++p) {
    if (n_host[p] < 1) return 0;
    vtot += n_host[p];
    const int64_t s = max_cols < 0 ? n_host[p] : std::min<int64_t>(max_cols, n_host[p]);
    ns += n_host[p] * std::max<int64_t>(s, 1);
  }
  const BwLayout L = bw_layout(nullptr, batch, vtot);
  size_t bytes = L.fixed + 3 * al((size_t)ns * 8) + 256;
  if (bw_split(opts)) {
    std::vector<SgProblem> pr;
    for (int p = 0; p < batch; ++p) {
      const int64_t s = max_cols < 0 ? n_host[p] : std::min<int64_t>(max_cols, n_host[p]);
      if (n_host[p] > INT32_MAX) return 0;
      pr.push_back(sg_problem((int)n_host[p], (int)std::max<int64_t>(s, 1), (int)n_host[p], SgOp{}, SgOp{}, nullptr,
                              0));
    }
    bytes += al(split_gemm_bytes(pr, bw_slices(opts)));
  }
  return bytes;
}

extern "C" int tdc_syev_tridiag_backward_batched(int32_t batch, const int64_t* n_host, const double* lambda_cat,
                                                 const double* Q_cat, const double* g_lambda_cat,
                                                 const double* g_Q_cat, double* g_d_cat, double* g_e_cat,
                                                 const tdc_opts* opts, void* ws, size_t ws_bytes, int* dev_status,
                                                 void* stream) {
  if (batch < 1) return -1;
  if (!n_host) return -2;
  if (!lambda_cat) return -3;
  if (!Q_cat) return -4;
  if (!g_d_cat) return -7;
  if (!g_e_cat) return -8;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return -10;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::vector<BwProb> pr(batch);
  std::vector<int64_t> cum(2 * (batch + 1), 0);
  int64_t vtot = 0, qtot = 0;
  for (int p = 0; p < batch; ++p) {
    const int64_t n = n_host[p];
    if (n < 1 || n > INT32_MAX) return -2;
    pr[p] = BwProb{n, vtot, qtot, 0, 0, 0};
    vtot += n;
    qtot += n * n;
    cum[p + 1] = cum[p] + n;
  }
  unsigned char* b = reinterpret_cast<unsigned char*>(ws);
  BwLayout L = bw_layout(b, batch, vtot);
  if (L.fixed + 256 > ws_bytes) return 3;
  if (g_Q_cat) {
    cudaMemcpyAsync(L.prob, pr.data(), sizeof(BwProb) * batch, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(L.cum, cum.data(), sizeof(int64_t) * (batch + 1), cudaMemcpyHostToDevice, st);
    if (vtot > 0x7FFFFFFF) return -2;
    k_bwb_flag<<<(unsigned)vtot, 256, 0, st>>>(L.prob, batch, L.cum, g_Q_cat, L.flag);
    k_bwb_compact<<<batch, 256, 0, st>>>(L.prob, L.flag, L.cols);
    if (cudaMemcpyAsync(pr.data(), L.prob, sizeof(BwProb) * batch, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return 4;
    if (cudaStreamSynchronize(st) != cudaSuccess) return 4;      // the column counts shape the GEMMs
  }
  int64_t ns = 0;
  for (int p = 0; p < batch; ++p) {
    if (!g_Q_cat) pr[p].s = 0;
    pr[p].g = ns;
    ns += pr[p].n * pr[p].s;
    cum[batch + 1 + p + 1] = ns;
  }
  size_t off = L.fixed;
  L.G = reinterpret_cast<double*>(b + off);
  off = al(off + (size_t)std::max<int64_t>(ns, 1) * 8);
  L.P = reinterpret_cast<double*>(b + off);
  off = al(off + (size_t)std::max<int64_t>(ns, 1) * 8);
  L.W = reinterpret_cast<double*>(b + off);
  off = al(off + (size_t)std::max<int64_t>(ns, 1) * 8);
  if (off > ws_bytes) return 3;
  cudaMemcpyAsync(L.prob, pr.data(), sizeof(BwProb) * batch, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(L.cum, cum.data(), sizeof(int64_t) * 2 * (batch + 1), cudaMemcpyHostToDevice, st);
  const int64_t* cum_n = L.cum;
  const int64_t* cum_ns = L.cum + batch + 1;
  if (ns > 0) {
    const unsigned gb = grid_cap((ns + 255) / 256, 8);
    k_bwb_gather<<<gb, 256, 0, st>>>(L.prob, batch, cum_ns, ns, g_Q_cat, L.cols, L.G);
    if (bw_split(opts)) {
      std::vector<SgProblem> pa, pw;
      for (int p = 0; p < batch; ++p) {
        if (pr[p].s == 0) continue;
        const int n = (int)pr[p].n;
        pa.push_back(sg_problem(n, pr[p].s, n, sg_dense(Q_cat + pr[p].q, n, true), sg_dense(L.G + pr[p].g, n),
                                L.P + pr[p].g, n));                                                       // Q^T G
        pw.push_back(sg_problem(n, pr[p].s, n, sg_dense(Q_cat + pr[p].q, n), sg_dense(L.G + pr[p].g, n),
                                L.W + pr[p].g, n));                                                       // Q M
      }
      unsigned char* arena = b + off;
      const size_t abytes = ws_bytes > off ? ws_bytes - off : 0;
      int* err = dev_status ? dev_status : L.status_scratch;
      int rc = split_gemm(pa, bw_slices(opts), arena, abytes, err, st);
      if (rc) return rc;
      k_bwb_m<<<gb, 256, 0, st>>>(L.prob, batch, cum_ns, ns, L.P, lambda_cat, L.cols, L.G);   // M into G
      rc = split_gemm(pw, bw_slices(opts), arena, abytes, err, st);
      if (rc) return rc;
      k_bwb_band<<<(unsigned)((vtot + 255) / 256), 256, 0, st>>>(L.prob, batch, cum_n, vtot, Q_cat, g_lambda_cat,
                                                                 L.W, L.cols, g_d_cat, g_e_cat);
      return cudaGetLastError() == cudaSuccess ? 0 : 4;
    }
    std::vector<DGemm> g;
    for (int p = 0; p < batch; ++p) {           // P = Q^T G
      if (pr[p].s == 0) continue;
      DGemm h;
      std::memset(&h, 0, sizeof(h));
      h.M = (int)pr[p].n; h.N = pr[p].s; h.K = (int)pr[p].n;
      h.a = DMat{Q_cat + pr[p].q, pr[p].n, 1};
      h.b = DMat{L.G + pr[p].g, pr[p].n, 0};
      h.C = L.P + pr[p].g; h.ldc = pr[p].n; h.alpha = 1.0;
      g.push_back(h);
    }
    size_t toff = 0;
    if (launch_dgemms(g, L.tab, toff, kBwTab, st)) return 3;
    k_bwb_m<<<gb, 256, 0, st>>>(L.prob, batch, cum_ns, ns, L.P, lambda_cat, L.cols, L.G);   // M into G
    for (DGemm& h : g) {                         // W = Q M: same shapes, same offsets
      const int64_t go = h.C - L.P;
      h.a.trans = 0;
      h.b.p = L.G + go;
      h.C = L.W + go;
    }
    if (launch_dgemms(g, L.tab, toff, kBwTab, st)) return 3;
  }
  k_bwb_band<<<(unsigned)((vtot + 255) / 256), 256, 0, st>>>(L.prob, batch, cum_n, vtot, Q_cat, g_lambda_cat,
                                                             L.W, L.cols, g_d_cat, g_e_cat);
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
