// Batched dense FP64 GEMM (see tdc_dgemm.cuh).  One CTA per 64 x 64 tile of C, k in
// steps of 16 through shared memory, a 4 x 4 block of C per thread.  The transposition
// flags are template parameters, so each operand tile is loaded with its own index
// order: lanes run along whichever of (row, k) or (k, column) is contiguous in memory.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "tdc_dgemm.cuh"
#include "tdc_internal.cuh"

namespace tdc {
namespace {

constexpr int TB = 64, TK = 16;

template <int AT, int BT>
__global__ __launch_bounds__(256) void k_dgemm(const DGemm* __restrict__ jobs, int njobs,
                                               const int64_t* __restrict__ cum) {
  __shared__ double As[TK][TB + 1];
  __shared__ double Bs[TK][TB + 1];
  const int jb = find_job(cum, njobs, blockIdx.x);
  const DGemm G = jobs[jb];
  const int64_t t = blockIdx.x - cum[jb];
  const int ntm = (G.M + TB - 1) / TB;
  const int r0 = (int)(t % ntm) * TB, c0 = (int)(t / ntm) * TB;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < G.K; k0 += TK) {
    for (int e = tid; e < TK * TB; e += 256) {       // A(r, k)
      const int kk = AT ? e % TK : e / TB, rr = AT ? e / TK : e % TB;
      const int r = r0 + rr, k = k0 + kk;
      double v = 0.0;
      if (r < G.M && k < G.K) v = AT ? G.a.p[(int64_t)k + (int64_t)r * G.a.ld] : G.a.p[(int64_t)r + (int64_t)k * G.a.ld];
      As[kk][rr] = v;
    }
    for (int e = tid; e < TK * TB; e += 256) {       // B(k, c)
      const int kk = BT ? e / TB : e % TK, cc = BT ? e % TB : e / TK;
      const int c = c0 + cc, k = k0 + kk;
      double v = 0.0;
      if (c < G.N && k < G.K) v = BT ? G.b.p[(int64_t)c + (int64_t)k * G.b.ld] : G.b.p[(int64_t)k + (int64_t)c * G.b.ld];
      Bs[kk][cc] = v;
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
    if (c >= G.N) continue;
    double* col = G.C + (int64_t)c * G.ldc;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = r0 + tx + 16 * a;
      if (r >= G.M) continue;
      const double v = G.alpha * acc[a][b];
      col[r] = G.beta == 0.0 ? v : v + G.beta * col[r];
    }
  }
}

int64_t tiles(const DGemm& g) { return (int64_t)((g.M + TB - 1) / TB) * ((g.N + TB - 1) / TB); }

}  // namespace

size_t dgemm_table_bytes(size_t njobs) { return 4 * (njobs * sizeof(DGemm) + (njobs + 1) * 8 + 512); }

int launch_dgemms(const std::vector<DGemm>& g, unsigned char* dev_tab, size_t& tab_off, size_t tab_bytes,
                  cudaStream_t st) {
  for (int form = 0; form < 4; ++form) {
    std::vector<DGemm> sel;
    for (const DGemm& x : g)
      if ((x.a.trans ? 1 : 0) + (x.b.trans ? 2 : 0) == form && x.M > 0 && x.N > 0) sel.push_back(x);
    if (sel.empty()) continue;
    std::vector<int64_t> cum(sel.size() + 1, 0);
    for (size_t i = 0; i < sel.size(); ++i) cum[i + 1] = cum[i] + tiles(sel[i]);
    tab_off = (tab_off + 255) & ~size_t(255);
    DGemm* dj = reinterpret_cast<DGemm*>(dev_tab + tab_off);
    tab_off += sel.size() * sizeof(DGemm);
    tab_off = (tab_off + 255) & ~size_t(255);
    int64_t* dc = reinterpret_cast<int64_t*>(dev_tab + tab_off);
    tab_off += cum.size() * 8;
    if (tab_off > tab_bytes) return 3;
    cudaMemcpyAsync(dj, sel.data(), sel.size() * sizeof(DGemm), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dc, cum.data(), cum.size() * 8, cudaMemcpyHostToDevice, st);
    const unsigned grid = (unsigned)cum.back();
    switch (form) {
      case 0: k_dgemm<0, 0><<<grid, 256, 0, st>>>(dj, (int)sel.size(), dc); break;
      case 1: k_dgemm<1, 0><<<grid, 256, 0, st>>>(dj, (int)sel.size(), dc); break;
      case 2: k_dgemm<0, 1><<<grid, 256, 0, st>>>(dj, (int)sel.size(), dc); break;
      default: k_dgemm<1, 1><<<grid, 256, 0, st>>>(dj, (int)sel.size(), dc); break;
    }
  }
  return 0;
}

}  // namespace tdc
