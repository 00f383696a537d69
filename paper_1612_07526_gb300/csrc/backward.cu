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

#include <cstring>
#include <vector>

#include "../../include/tdc.h"
#include "tdc_hss.cuh"

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

}  // namespace
}  // namespace tdc

using namespace tdc;

extern "C" size_t tdc_backward_workspace_bytes(int64_t n, const tdc_opts* opts) {
  (void)opts;
  if (n < 1) return 0;
  return al(n * 4) + al(n * 4) + al(16) + 3 * al((size_t)n * n * 8) + al(1 << 20);
}

extern "C" int tdc_syev_tridiag_backward(int64_t n, const double* lambda, const double* Q, int64_t ldq,
                                         const double* g_lambda, const double* g_Q, int64_t ldg, double* g_d,
                                         double* g_e, const tdc_opts* opts, void* ws, size_t ws_bytes,
                                         int* dev_status, void* stream) {
  (void)dev_status;
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
    std::vector<HGemm> g(1);
    std::memset(g.data(), 0, sizeof(HGemm));
    g[0].M = (int)n; g[0].N = s; g[0].K = (int)n;          // P = Q^T G
    g[0].a.mode = HOP_DENSE_T; g[0].a.p = Q; g[0].a.ld = ldq;
    g[0].b.mode = HOP_DENSE; g[0].b.p = G; g[0].b.ld = n;
    g[0].C = P; g[0].ldc = n; g[0].alpha = 1.0;
    size_t toff = 0;
    launch_dense_gemms(g, tab, toff, st);
    k_bw_m<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(P, lambda, cols, n, s, G);   // M_S into G
    g[0].a.mode = HOP_DENSE; g[0].a.p = Q; g[0].a.ld = ldq;                            // W = Q M_S
    g[0].b.p = G;
    g[0].C = W;
    launch_dense_gemms(g, tab, toff, st);
  }
  k_bw_band<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Q, ldq, n, lambda, g_lambda, W, cols, s, g_d, g_e);
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
