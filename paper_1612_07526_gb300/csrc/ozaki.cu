// Split-precision eigenvector product of Eq. (6) on tcgen05 tensor cores.
// See tdc_ozaki.cuh for the splitting and the exactness argument.
//
// Kernels (one launch each per tree level, over that level's merges):
//   k_oz_slice_a  rows of Q_sel (gathered columns, Gu order, padded groups): row
//                 scale, then S bf16 digit slices written k-major;
//   k_oz_slice_b  Qhat generated from (d, zhat, origin, tau, 1/norm) and split the
//                 same way, one column of Qhat per k-major row;
//   k_oz_gemm     128 x 64 output tiles: a TMA producer warp, an MMA warp and eight
//                 epilogue warps.  Six to eight FP32 accumulators of 64 TMEM
//                 columns (one per level p + q); one MMA per A slice and group of
//                 up to four B slices; exact levels are flushed every 256 k into
//                 64-bit integers held by the epilogue threads.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstring>
#include <mutex>

#include "tdc_ozaki.cuh"

namespace tdc {

namespace {

constexpr int kThreads = 320;       // warp 0: TMA, warp 1: MMA + TMEM owner, warps 2-9: epilogue
constexpr int kEpiWarps = 8;        // two per TMEM lane quadrant, each owning 32 of a level's 64 columns
constexpr long long kWaitNs = 2LL * 1000 * 1000 * 1000;    // bounded mbarrier waits (2 s)

__host__ __device__ constexpr int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// padded k (Gu groups each padded to kOzPad) -> grouped index in [0, K), or -1
__device__ __forceinline__ int padded_to_grouped(int k, int c1, int c3, int K, int P1, int P3) {
  if (k < P1) return k < c1 ? k : -1;
  if (k < P1 + P3) return (k - P1) < c3 ? c1 + (k - P1) : -1;
  const int r = k - P1 - P3;
  return r < K - c1 - c3 ? c1 + c3 + r : -1;
}

// Balanced base-256 digits of X (|X| <= 2^(8S-1)), most significant first, as bf16
// bits.  With Y = X + sum_{p < S-1} 128 * 256^p, the S-1 low bytes of Y are d_p + 128
// (d_p in [-128, 127] the balanced digits, least significant first) and the
// arithmetic shift Y >> 8(S-1) is the top digit, in [-128, 128].  A byte b becomes
// the float b - 128 by placing it in the mantissa of 2^23 and subtracting 2^23 + 128
// (both exact); an integer of at most 8 significant bits is exact in bf16, whose bits
// are the float's upper half.
template <int S>
__device__ __forceinline__ void digits_bf16(long long X, uint16_t (&out)[S]) {
  unsigned long long bias = 0;
#pragma unroll
  for (int q = 0; q < S - 1; ++q) bias |= 128ull << (8 * q);
  const unsigned long long Y = (unsigned long long)X + bias;
  const uint32_t lo = (uint32_t)Y, hi = (uint32_t)(Y >> 32);
#pragma unroll
  for (int q = 0; q < S - 1; ++q) {
    const uint32_t b = ((q < 4 ? lo >> (8 * q) : hi >> (8 * (q - 4)))) & 255u;
    const float f = __uint_as_float(0x4B000000u | b) - 8388736.0f;
    out[S - 1 - q] = (uint16_t)(__float_as_uint(f) >> 16);
  }
  const long long top = (long long)Y >> (8 * (S - 1));
  out[0] = (uint16_t)(__float_as_uint((float)(int)top) >> 16);
}

// round(x * 2^k) to the nearest integer, ties to even, for |x 2^k| < 2^62, in
// integer arithmetic on the bits of x (x = M 2^e2 with the integer significand M):
// the scaled significand is shifted right with the discarded bits rounded.
__device__ __forceinline__ long long round_scaled(double x, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  const unsigned long long F = b & 0xFFFFFFFFFFFFFull;
  const unsigned long long M = E ? (F | (1ull << 52)) : F;
  const int sh = -((E ? E - 1075 : -1074) + k);          // right shift of M
  unsigned long long q;
  if (sh <= 0) {
    q = M << (-sh);
  } else if (sh >= 64) {
    q = 0;
  } else {
    q = M >> sh;
    const unsigned long long rem = M & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
  }
  return (b >> 63) ? -(long long)q : (long long)q;
}

// ------------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.b32 %0, 1, 0, P;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity; gives up after limit_ns (kWaitNs by
// default) or when another role has aborted, setting the abort flag and the status bit.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err,
                          long long limit_ns = kWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = global_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255) == 255) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > limit_ns) {
        *abort_flag = 1;
        atomicOr(err, ST_WAIT);
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x,
                                            int y, int z, int v) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], [%2];"
      ::"r"(dst), "l"(map), "r"(bar), "r"(x), "r"(y), "r"(z), "r"(v)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, 8-row groups
// 512 bytes apart (SM100 descriptor: start >> 4, LBO, SBO >> 4, version 1, layout 4).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major,
// M = 128 and N = 64 nq (nq stacked B slices).
__host__ __device__ constexpr uint32_t idesc_n(int nq) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((kOzBN * nq) >> 3) << 17) |
         ((uint32_t)(kOzBM >> 4) << 24);
}
__device__ __forceinline__ void tmem_st32_zero(uint32_t taddr) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
      "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
      "r"(0u)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// The epilogue's conversions and power-of-two scalings on the integer pipes, from the
// IEEE-754 binary64/binary32 formats (GB300's FP64 pipe issues 2 lanes per clock per SM,
// and with five FP64 operations per output it, not the tensor pipe, bounded the GEMM).
// The int64 value v as the nearest double (ties to even): sign, the leading bit's
// position p, and the 52 bits after it, rounded when p > 52.
__device__ __forceinline__ double i64_to_double_bits(long long v) {
  if (v == 0) return 0.0;
  const unsigned long long s = (unsigned long long)v & 0x8000000000000000ull;
  const unsigned long long u = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  int p = 63 - __clzll((long long)u);
  unsigned long long q;
  if (p <= 52) {
    q = u << (52 - p);
  } else {
    const int sh = p - 52;
    q = u >> sh;
    const unsigned long long rem = u & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
    if (q >> 53) {                                       // rounded up to the next power of two
      q >>= 1;
      ++p;
    }
  }
  return __longlong_as_double((long long)(s | ((unsigned long long)(1023 + p) << 52) | (q & 0xFFFFFFFFFFFFFull)));
}
// The rare cases (subnormal, infinite or NaN operands or results) through ldexp, out of
// line: inlined, the compiler if-converts them, and their FP64 instructions then issue
// for every output although no lane takes them.
__device__ __noinline__ double f32_ldexp_slow(float f, int e) { return ldexp((double)f, e); }
__device__ __noinline__ double ldexp_slow(double x, int e) { return ldexp(x, e); }
// f 2^e exactly as a double, for a normal float f and a result in the normal range
// (the exponent field rebased, the 23 fraction bits moved up); other f through FP64.
__device__ __forceinline__ double f32_pow2_to_double(float f, int e) {
  const unsigned b = __float_as_uint(f);
  const int ex = (int)((b >> 23) & 0xFFu);
  if ((b & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)(b >> 31) << 63);   // signed zero
  if (ex == 0 || ex == 0xFF) return f32_ldexp_slow(f, e);  // subnormal, inf, NaN
  return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) |
                                          ((unsigned long long)(ex - 127 + 1023 + e) << 52) |
                                          ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}
// x 2^e exactly when the result stays normal (the exponent field moved by e), else
// through ldexp.
__device__ __forceinline__ double scale_pow2(double x, int e) {
  const long long b = __double_as_longlong(x);
  if ((b & 0x7FFFFFFFFFFFFFFFll) == 0) return x;       // signed zero
  const int ex = (int)((b >> 52) & 0x7FF);
  const int ne = ex + e;
  if (ex != 0 && ex != 0x7FF && ne >= 1 && ne <= 2046) return __longlong_as_double(b + ((long long)e << 52));
  return ldexp_slow(x, e);
}
// One output of the product: (acc + tsum 2^-8) 2^e, acc in level-5 units, tsum in
// level-6 units; one FP64 addition.
__device__ __forceinline__ double oz_combine(long long acc, float tsum, int e) {
  return scale_pow2(i64_to_double_bits(acc) + f32_pow2_to_double(tsum, -8), e);
}

struct JobView {
  int jb;
  int64_t local;
};
__device__ __forceinline__ JobView job_of(const int64_t* cum, int njobs) {
  JobView v;
  v.jb = find_job(cum, njobs, blockIdx.x);
  v.local = blockIdx.x - cum[v.jb];
  return v;
}

// ------------------------------------------------------------------------ slicing of Q_sel
template <int S>
__global__ __launch_bounds__(256) void k_oz_slice_a(const MergeJob* __restrict__ jobs,
                                                    const OzJob* __restrict__ ozj, int njobs,
                                                    const int64_t* __restrict__ cum, DevWs w) {
  __shared__ double tile[64][33];
  __shared__ unsigned long long s_max[8][32];
  __shared__ int s_exp[32];
  const JobView jv = job_of(cum, njobs);
  const MergeJob J = jobs[jv.jb];
  const OzJob& Z = ozj[jv.jb];
  const MergeScalars Sc = w.scal[J.mid];
  const int K = Sc.K, c1 = Sc.c1, c3 = Sc.c3;
  const int P1 = (int)rup(c1, kOzPad), P3 = (int)rup(c3, kOzPad), P2 = (int)rup(K - c1 - c3, kOzPad);
  const int nrt1 = (J.n1 + 31) / 32;
  const int h = jv.local < nrt1 ? 0 : 1;
  const int rt = h ? (int)jv.local - nrt1 : (int)jv.local;
  const int rows_h = h ? J.n2 : J.n1;
  const int rowbase = h ? J.n1 : 0;
  const int r0 = rt * 32;
  const int kb = h ? P1 : 0;
  const int klen = h ? P3 + P2 : P1 + P3;
  const double* const* colptr = w.colptr + J.v_off;
  const int tid = threadIdx.x;
  const int r = tid & 31, kq = tid >> 5;
  const bool rvalid = r0 + r < rows_h;
  // pass 1: row maxima, on the magnitude bits (integer order = order of |x|), four
  // independent loads in flight per thread
  unsigned long long mx = 0ull;
  const int row = rowbase + r0 + r;
  for (int k0 = kq; k0 < klen; k0 += 32) {
    unsigned long long v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + 8 * u;
      const int kg = k < klen ? padded_to_grouped(kb + k, c1, c3, K, P1, P3) : -1;
      v[u] = kg >= 0 && rvalid && row >= w.klo[J.v_off + kg] && row < w.khi[J.v_off + kg]
                 ? (unsigned long long)__double_as_longlong(colptr[kg][row]) & 0x7FFFFFFFFFFFFFFFull
                 : 0ull;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) mx = v[u] > mx ? v[u] : mx;
  }
  s_max[kq][r] = mx;
  __syncthreads();
  if (tid < 32) {
    unsigned long long mb = s_max[0][tid];
    for (int q = 1; q < 8; ++q) mb = s_max[q][tid] > mb ? s_max[q][tid] : mb;
    const double m = __longlong_as_double((long long)mb);
    int e = 0;
    if (m > 0.0) frexp(m, &e);     // m < 2^e
    s_exp[tid] = e;
    if (r0 + tid < rows_h) Z.sigma[rowbase + r0 + tid] = m > 0.0 ? ldexp(1.0, e) : 0.0;
  }
  __syncthreads();
  // pass 2: digits, 64 k at a time, transposed through shared memory
  const int wr = tid >> 3, wk = (tid & 7) * 8;
  const int shift = 8 * S - 1 - s_exp[wr];
  uint16_t* abase = Z.a[h];
  for (int k0 = 0; k0 < klen; k0 += 64) {
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const int k = kq * 8 + kk;
      const int kg = padded_to_grouped(kb + k0 + k, c1, c3, K, P1, P3);
      const int row = rowbase + r0 + r;
      tile[k][r] = (kg >= 0 && rvalid && k0 + k < klen && row >= w.klo[J.v_off + kg] &&
                    row < w.khi[J.v_off + kg]) ? colptr[kg][row] : 0.0;
    }
    __syncthreads();
    if (r0 + wr < rows_h) {
      uint16_t dg[8][S];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const double x = tile[wk + j][wr];
        const long long X = round_scaled(x, shift);
        uint16_t t[S];
        digits_bf16<S>(X, t);
#pragma unroll
        for (int p = 0; p < S; ++p) dg[j][p] = t[p];
      }
#pragma unroll
      for (int p = 0; p < S; ++p) {
        uint4 v;
        v.x = (uint32_t)dg[0][p] | ((uint32_t)dg[1][p] << 16);
        v.y = (uint32_t)dg[2][p] | ((uint32_t)dg[3][p] << 16);
        v.z = (uint32_t)dg[4][p] | ((uint32_t)dg[5][p] << 16);
        v.w = (uint32_t)dg[6][p] | ((uint32_t)dg[7][p] << 16);
        const int k = k0 + wk;                 // k-blocked: [slice][k / 32][row][k % 32]
        *reinterpret_cast<uint4*>(abase + (((int64_t)p * (Z.ldk / kOzBK) + k / kOzBK) * rows_h + r0 + wr) * kOzBK +
                                  (k % kOzBK)) = v;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------ generated, sliced Qhat
// Blocks strided over the level's schedule (cum from k_oz_sched): a merge's K x KP
// entries of Qhat (KP its padded length) as K KP / 8 vectors of 8 k, 256 vectors per
// block, thread f of the merge taking column f / (KP / 8) and k from 8 (f % (KP / 8)).
template <int S>
__global__ __launch_bounds__(256) void k_oz_slice_b(const MergeJob* __restrict__ jobs,
                                                    const OzJob* __restrict__ ozj, int njobs,
                                                    const int64_t* __restrict__ cum, DevWs w) {
  const int64_t total = cum[njobs];
  for (int64_t vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int jb = find_job(cum, njobs, vb);
    const MergeJob J = jobs[jb];
    const MergeScalars Sc = w.scal[J.mid];
    const int K = Sc.K, c1 = Sc.c1, c3 = Sc.c3;
    const int P1 = (int)rup(c1, kOzPad), P3 = (int)rup(c3, kOzPad), P2 = (int)rup(K - c1 - c3, kOzPad);
    const int KP = P1 + P3 + P2, nv = KP / 8;
    const int64_t f = (vb - cum[jb]) * 256 + threadIdx.x;
    if (f >= (int64_t)K * nv) continue;
    const int i = (int)(f / nv);
    const int k0 = (int)(f % nv) * 8;
    const OzJob& Z = ozj[jb];
    const int m = J.n1 + J.n2;
    const int64_t o = J.v_off;
    const int32_t* __restrict__ kperm = w.kperm + o;
    const double* __restrict__ wcol = w.wptr[o + i];     // unscaled column i of the Cauchy factor
    const double si = w.sinv[o + i];
    // tau_i = 2^e >= the column's largest entry: e from the exponent field (cmax normal), else frexp
    const long long cb = __double_as_longlong(w.cmax[o + i]);
    const int ce = (int)((cb >> 52) & 0x7FF);
    int e = 0;
    if (ce != 0 && ce != 0x7FF && cb > 0) e = ce - 1022;
    else if (cb > 0) frexp(w.cmax[o + i], &e);
    if (k0 == 0) Z.texp[i] = e;
    const int shift = 8 * S - 1 - e;
    uint16_t dg[8][S];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int kg = padded_to_grouped(k0 + j, c1, c3, K, P1, P3);
      double v = 0.0;
      if (kg >= 0) v = wcol[kperm[kg]] * si;
      uint16_t tt[S];
      digits_bf16<S>(round_scaled(v, shift), tt);
#pragma unroll
      for (int p = 0; p < S; ++p) dg[j][p] = tt[p];
    }
#pragma unroll
    for (int p = 0; p < S; ++p) {
      uint4 vv;
      vv.x = (uint32_t)dg[0][p] | ((uint32_t)dg[1][p] << 16);
      vv.y = (uint32_t)dg[2][p] | ((uint32_t)dg[3][p] << 16);
      vv.z = (uint32_t)dg[4][p] | ((uint32_t)dg[5][p] << 16);
      vv.w = (uint32_t)dg[6][p] | ((uint32_t)dg[7][p] << 16);
      *reinterpret_cast<uint4*>(Z.b + (((int64_t)p * (Z.ldk / kOzBK) + k0 / kOzBK) * m + i) * kOzBK +
                                (k0 % kOzBK)) = vv;
    }
  }
}

// The level's schedules from the merges' K (known only on the device): blocks of
// k_oz_slice_b (cdiv(K KP / 8, 256)) and tiles of k_oz_gemm ((row tiles of T1
// + of T2) x cdiv(K, kOzBN)); cum[j] = units of the merges before j.  One block of
// 1024 threads, each summing a contiguous run of merges, then a scan.
__global__ __launch_bounds__(1024) void k_oz_sched(const MergeJob* __restrict__ jobs, int njobs,
                                                   const MergeScalars* __restrict__ scal,
                                                   int64_t* __restrict__ cum_sb, int64_t* __restrict__ cum_t) {
  __shared__ int64_t part[2][1024];
  const int t = threadIdx.x;
  const int per = (njobs + 1023) / 1024;
  const int j0 = min(t * per, njobs), j1 = min(j0 + per, njobs);
  auto units = [&](int j, int64_t& sb, int64_t& tl) {
    const MergeJob& J = jobs[j];
    const MergeScalars& Sc = scal[J.mid];
    const int K = Sc.K;
    const int64_t KP = rup(Sc.c1, kOzPad) + rup(Sc.c3, kOzPad) + rup(K - Sc.c1 - Sc.c3, kOzPad);
    sb = ((int64_t)K * (KP / 8) + 255) / 256;
    tl = (int64_t)((J.n1 + kOzBM - 1) / kOzBM + (J.n2 + kOzBM - 1) / kOzBM) * ((K + kOzBN - 1) / kOzBN);
  };
  int64_t a = 0, b = 0;
  for (int j = j0; j < j1; ++j) {
    int64_t sb, tl;
    units(j, sb, tl);
    a += sb;
    b += tl;
  }
  part[0][t] = a;
  part[1][t] = b;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {      // inclusive Hillis-Steele scans
    const int64_t va = t >= off ? part[0][t - off] : 0, vb = t >= off ? part[1][t - off] : 0;
    __syncthreads();
    part[0][t] += va;
    part[1][t] += vb;
    __syncthreads();
  }
  int64_t ra = t > 0 ? part[0][t - 1] : 0, rb = t > 0 ? part[1][t - 1] : 0;
  for (int j = j0; j < j1; ++j) {
    cum_sb[j] = ra;
    cum_t[j] = rb;
    int64_t sb, tl;
    units(j, sb, tl);
    ra += sb;
    rb += tl;
  }
  if (t == 1023) {
    cum_sb[njobs] = part[0][1023];
    cum_t[njobs] = part[1][1023];
  }
}

// ------------------------------------------------------------------------ tcgen05 GEMM
// MMA schedule.  Level L = p + q accumulates at TMEM columns (L - 2) * 64, so for a
// fixed A slice p the products with the B slices q = qa .. qa + nq - 1 (stacked
// contiguously in shared memory) land in the contiguous columns starting at
// (p + qa - 2) * 64: one MMA of N = 64 nq covers them (nq <= 4, N <= 256).  Per 16-deep
// k step that is 2S - 2 MMAs instead of one per pair, and each A slice is read from
// shared memory once per group instead of once per pair.
template <int S>
struct OzCfg {
  static constexpr int NL = S + 1;                       // levels 2 .. S+2
  static constexpr int ST = S <= 6 ? 3 : 2;              // pipeline stages
  static constexpr int A_BYTES = kOzBM * kOzBK * 2 * S;
  static constexpr int B_BYTES = kOzBN * kOzBK * 2 * S;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int SMEM = ST * STAGE + 1024 + 256;
  static_assert(NL * kOzBN <= 512, "TMEM columns");
  static_assert(S >= 4, "the chunk-reset MMA covers levels 2..5");
  __host__ __device__ static constexpr int qmax(int p) { return S < S + 2 - p ? S : S + 2 - p; }
};

// One tile of the product: its merge, half (T1 or T2 rows), rows and columns, and the
// k range of the Gu groups that half uses.
struct OzTile {
  int jb, h, row0, rows_h, rowbase, ct, kb, nst, nchunks, K;
};
__device__ __forceinline__ OzTile oz_tile(const MergeJob* __restrict__ jobs, const int64_t* __restrict__ cum,
                                          int njobs, const DevWs& w, int64_t t) {
  OzTile v;
  v.jb = find_job(cum, njobs, t);
  const int64_t local = t - cum[v.jb];
  const MergeJob J = jobs[v.jb];
  const MergeScalars Sc = w.scal[J.mid];
  const int K = Sc.K, c1 = Sc.c1, c3 = Sc.c3;
  const int nct = (K + kOzBN - 1) / kOzBN;                 // >= 1: a merge with tiles has K > 0
  const int nrt1 = (J.n1 + kOzBM - 1) / kOzBM;
  v.K = K;
  v.ct = (int)(local % nct);
  const int rtl = (int)(local / nct);
  v.h = rtl < nrt1 ? 0 : 1;
  v.row0 = (v.h ? rtl - nrt1 : rtl) * kOzBM;               // within the half
  v.rows_h = v.h ? J.n2 : J.n1;
  v.rowbase = v.h ? J.n1 : 0;
  const int P1 = (int)rup(c1, kOzPad), P3 = (int)rup(c3, kOzPad), P2 = (int)rup(K - c1 - c3, kOzPad);
  const int klen = v.h ? P3 + P2 : P1 + P3;
  v.kb = v.h ? P1 : 0;
  v.nst = klen / kOzBK;
  v.nchunks = (v.nst + kOzChunk / kOzBK - 1) / (kOzChunk / kOzBK);
  return v;
}

// Persistent: each CTA (one per SM) takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// of the level's schedule (cum from k_oz_sched: each merge's tiles from its K).  The
// pipeline's stage and accumulator barriers keep counting across tiles; the epilogue
// re-zeroes the levels >= 6 after reading them and releases the accumulators (tfree)
// before the next tile's first MMA.
template <int S>
__global__ __launch_bounds__(kThreads, 1) void k_oz_gemm(const MergeJob* __restrict__ jobs,
                                                         const OzJob* __restrict__ ozj, int njobs,
                                                         const int64_t* __restrict__ cum, QBufs qb,
                                                         DevWs w) {
  using C = OzCfg<S>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::ST * C::STAGE);
  // bars[0..ST) full, [ST..2ST) empty, 2ST accfull, 2ST+1 accempty, 2ST+2 done, 2ST+3 tfree
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * C::ST + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int64_t total = cum[njobs];
  if ((int64_t)blockIdx.x >= total) return;               // uniform: no barrier touched yet

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (C::ST + s); };
  const uint32_t accfull = bar0 + 8u * (2 * C::ST);
  const uint32_t accempty = bar0 + 8u * (2 * C::ST + 1);
  const uint32_t done = bar0 + 8u * (2 * C::ST + 2);
  const uint32_t tfree = bar0 + 8u * (2 * C::ST + 3);
  int* err0 = w.status + jobs[find_job(cum, njobs, blockIdx.x)].prob;   // wait timeouts are reported here

  if (tid == 0) {
    for (int s = 0; s < C::ST; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(accfull, 1);
    mbar_init(accempty, kEpiWarps);
    mbar_init(done, 1);
    mbar_init(tfree, kEpiWarps);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // Every accumulator starts at zero, so that every MMA may accumulate; the exact
  // levels are restarted at each chunk by the one MMA that covers all of them, the
  // others are re-zeroed by the epilogue after each tile.
  if (warp >= 2) {
    const uint32_t tq = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(((warp - 2) >> 2) * 32);
#pragma unroll
    for (int L = 0; L < C::NL; ++L) tmem_st32_zero(tq + (uint32_t)(L * kOzBN));
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      uint32_t g = 0, issued_total = 0;
      for (int64_t t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x) {
        const OzTile T = oz_tile(jobs, cum, njobs, w, t);
        int* err = w.status + jobs[T.jb].prob;
        const CUtensorMap* mA = &ozj[T.jb].mapA[T.h];
        const CUtensorMap* mB = &ozj[T.jb].mapB;
        asm volatile("prefetch.tensormap [%0];" ::"l"(mA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(mB) : "memory");
        bool ok = true;
        for (int it = 0; it < T.nst; ++it, ++g) {
          const int s = (int)(g % C::ST);
          const uint32_t ph = (g / C::ST) & 1u;
          if (!mbar_wait(empty(s), ph ^ 1u, abort_flag, err)) { ok = false; break; }
          const uint32_t sa = smem_u32(smem + s * C::STAGE);
          mbar_expect_tx(full(s), C::STAGE);
          tma_load_4d(sa, mA, full(s), 0, T.row0, it, 0);
          tma_load_4d(sa + C::A_BYTES, mB, full(s), 0, T.ct * kOzBN, T.kb / kOzBK + it, 0);
          issued_total = g + 1;
        }
        if (!ok) break;
      }
      if (*abort_flag) {      // let the copies in flight land before the CTA exits
        const long long t0 = global_ns();
        for (uint32_t q = (issued_total > (uint32_t)C::ST ? issued_total - C::ST : 0u); q < issued_total; ++q) {
          const uint32_t ph = (q / C::ST) & 1u;
          while (!mbar_try(full((int)(q % C::ST)), ph) && global_ns() - t0 < kWaitNs) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      const int per_chunk = kOzChunk / kOzBK;
      uint32_t g = 0, cg = 0, ti = 0;
      int* err = err0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < total && ok; t += gridDim.x) {
        const OzTile T = oz_tile(jobs, cum, njobs, w, t);
        if (T.nst == 0) continue;
        err = w.status + jobs[T.jb].prob;
        if (ti > 0) {                                      // the previous tile's accumulators read and reset
          if (!mbar_wait(tfree, (ti - 1) & 1u, abort_flag, err)) { ok = false; break; }
          tc_fence_after();
        }
        for (int it = 0; it < T.nst; ++it, ++g) {
          const int s = (int)(g % C::ST);
          const uint32_t ph = (g / C::ST) & 1u;
          if (!mbar_wait(full(s), ph, abort_flag, err)) { ok = false; break; }
          tc_fence_after();
          const int chunk = it / per_chunk;
          const bool first = (it % per_chunk) == 0;
          const bool last = (it % per_chunk) == per_chunk - 1 || it == T.nst - 1;
          const uint32_t sa = smem_u32(smem + s * C::STAGE);
          const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < kOzBK / 16; ++kk) {
            // groups whose levels are all >= 6 (accumulated over the whole k range)
#pragma unroll
            for (int p = 1; p <= S; ++p) {
#pragma unroll
              for (int qa = 1; qa <= 5; qa += 4) {
                if (qa <= C::qmax(p) && p + qa >= 6) {
                  const int nq = C::qmax(p) - qa + 1 < 4 ? C::qmax(p) - qa + 1 : 4;
                  tc_mma(tmem + (uint32_t)((p + qa - 2) * kOzBN),
                         sdesc(sa + (p - 1) * (kOzBM * kOzBK * 2) + kk * 32),
                         sdesc(sb + (qa - 1) * (kOzBN * kOzBK * 2) + kk * 32), idesc_n(nq), 1u);
                }
              }
            }
            if (first && kk == 0 && chunk > 0) {           // the previous chunk's exact levels drained
              if (!mbar_wait(accempty, (cg - 1) & 1u, abort_flag, err)) { ok = false; break; }
              tc_fence_after();
            }
            // groups that touch the exact levels 2..5; (p = 1, q = 1..4) comes first and
            // overwrites all four at the start of a chunk
#pragma unroll
            for (int p = 1; p <= 4; ++p) {
              const int nq = C::qmax(p) < 4 ? C::qmax(p) : 4;
              const uint32_t acc = (p == 1 && first && kk == 0) ? 0u : 1u;
              tc_mma(tmem + (uint32_t)((p - 1) * kOzBN), sdesc(sa + (p - 1) * (kOzBM * kOzBK * 2) + kk * 32),
                     sdesc(sb + kk * 32), idesc_n(nq), acc);
            }
          }
          if (!ok) break;
          tc_commit(empty(s));
          if (last) {
            tc_commit(accfull);
            ++cg;
          }
        }
        if (!ok) break;
        tc_commit(done);
        ++ti;
      }
      if (*abort_flag) {                                   // the MMAs issued complete before the exit
        tc_commit(done);                                   // phases complete in order: the last
        const long long t0 = global_ns();                  // committed tile's, then this one
        if (ti > 0)
          while (!mbar_try(done, (ti - 1) & 1u) && global_ns() - t0 < kWaitNs) {
          }
        while (!mbar_try(done, ti & 1u) && global_ns() - t0 < kWaitNs) {
        }
      }
    }
  } else {
    // ---------------- epilogue: warps 2..9; TMEM lane quadrant = warp % 4, and the
    // warp owns columns [32 half, 32 half + 32) of every level.  Every tcgen05.ld is
    // executed by all 32 lanes (.sync.aligned); only the global stores are
    // predicated on the row being inside the half.
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quad * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 32);
    uint32_t cg = 0, ti = 0;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
      const OzTile T = oz_tile(jobs, cum, njobs, w, t);
      const MergeJob J = jobs[T.jb];
      const OzJob* Z = ozj + T.jb;
      int* err = w.status + J.prob;
      long long acc[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = 0;
      bool ok = true;
      for (int c = 0; c < T.nchunks; ++c) {
        const bool got = __all_sync(0xffffffffu, mbar_wait(accfull, cg & 1u, abort_flag, err));
        if (!got) { ok = false; break; }
        tc_fence_after();
#pragma unroll
        for (int L = 2; L <= 5; ++L) {
          uint32_t v[32];
          tmem_ld32(trow + (uint32_t)((L - 2) * kOzBN), v);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 32; ++j)
            acc[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << (8 * (5 - L));
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(accempty);
        ++cg;
      }
      // tail levels combined in FP32, smallest first: their rounding stays below the
      // FP32 accumulation error that level 6 already carries
      float tsum[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) tsum[j] = 0.0f;
      if (ok && T.nst > 0) {
        ok = __all_sync(0xffffffffu, mbar_wait(done, ti & 1u, abort_flag, err));
        if (ok) {
          tc_fence_after();
#pragma unroll
          for (int L = S + 2; L >= 6; --L) {
            uint32_t v[32];
            tmem_ld32(trow + (uint32_t)((L - 2) * kOzBN), v);
            tmem_wait_ld();
            const float wL = __int_as_float((127 - 8 * (L - 6)) << 23);     // 2^(-8 (L - 6))
#pragma unroll
            for (int j = 0; j < 32; ++j) tsum[j] = fmaf(__uint_as_float(v[j]), wL, tsum[j]);
          }
#pragma unroll
          for (int L = 6; L <= S + 2; ++L) tmem_st32_zero(trow + (uint32_t)((L - 2) * kOzBN));
          tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tfree);
          ++ti;
        }
      }
      if (!ok) break;
      const int grow = T.row0 + row;
      if (grow < T.rows_h) {
        // sigma is a power of two (or zero: a row with no entries in its k range)
        const long long sb = __double_as_longlong(Z->sigma[T.rowbase + grow]);
        const bool zrow = (sb & 0x7FFFFFFFFFFFFFFFll) == 0;
        const int es = (int)((sb >> 52) & 0x7FF) - 1023;
        double* const* outptr = w.outptr + J.v_off;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = T.ct * kOzBN + half * 32 + j;
          if (col < T.K) {
            // acc counts level-5 units (2^-38), tsum level-6 units (2^-46); times tau_i sigma_r
            outptr[col][T.rowbase + grow] = zrow ? 0.0 : oz_combine(acc[j], tsum[j], Z->texp[col] - 38 + es);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

template <int S>
void launch_s(int part, const MergeJob* jobs, const OzJob* ozj, int njobs, const int64_t* cum_sa, int64_t nb_sa,
              int64_t* cum_sb, int64_t nb_sb, int64_t* cum_t, int64_t ntiles, QBufs qb, DevWs w,
              cudaStream_t st) {
  using C = OzCfg<S>;
  // the shared-memory opt-in is a per-device attribute of the kernel: set it once on
  // every device that launches it (with the device's SM count for the persistent grid)
  static std::mutex mu;
  static bool attr[64] = {};
  static int sms[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int nsm = 148;
  {
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64 || !attr[dev]) {
      cudaFuncSetAttribute(k_oz_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
      int n = 0;
      if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 148;
      if (dev >= 0 && dev < 64) {
        attr[dev] = true;
        sms[dev] = n;
      }
      nsm = n;
    } else {
      nsm = sms[dev];
    }
  }
  // nb_sb and ntiles are the host's bounds (K = m); the kernels stride over the
  // schedules k_oz_sched writes from the actual K
  if (part == 0) {
    k_oz_sched<<<1, 1024, 0, st>>>(jobs, njobs, w.scal, cum_sb, cum_t);
    if (nb_sa) k_oz_slice_a<S><<<(unsigned)nb_sa, 256, 0, st>>>(jobs, ozj, njobs, cum_sa, w);
    if (nb_sb) k_oz_slice_b<S><<<grid_cap(nb_sb, 8), 256, 0, st>>>(jobs, ozj, njobs, cum_sb, w);
  } else if (ntiles) {
    const unsigned grid = (unsigned)(ntiles < nsm ? ntiles : nsm);
    k_oz_gemm<S><<<grid, kThreads, C::SMEM, st>>>(jobs, ozj, njobs, cum_t, qb, w);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Slices in k-blocked order, [slice][k / 32][row][k % 32]: a tile's box (32 k, its rows,
// one k block, every slice) is one contiguous run of rows x 64 bytes per slice, and
// lands in shared memory as [slice][row][32 k], as the MMA descriptors expect.
bool encode4d(CUtensorMap* map, void* base, int64_t ldk, int64_t rows, int slices, int box_rows) {
  auto fn = encoder();
  if (!fn) return false;
  const int64_t nkb = ldk / kOzBK;
  cuuint64_t dims[4] = {(cuuint64_t)kOzBK, (cuuint64_t)rows, (cuuint64_t)nkb, (cuuint64_t)slices};
  cuuint64_t strides[3] = {(cuuint64_t)kOzBK * 2, (cuuint64_t)(rows * kOzBK * 2), (cuuint64_t)(nkb * rows * kOzBK * 2)};
  cuuint32_t box[4] = {(cuuint32_t)kOzBK, (cuuint32_t)box_rows, 1u, (cuuint32_t)slices};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t job_ldk(const MergeJob& J) { return rup((int64_t)J.n1 + J.n2 + 3 * kOzPad, kOzPad); }

// ------------------------------------------------------------------------ dense split GEMM
// C_j = A_j B_j for a batch of dense column-major problems (A_j: M x K, or given as its
// transpose; B_j: K x N), with the merge product's splitting, tensor-core schedule and
// epilogue: A's rows and B's columns are scaled by powers of two (2^aexp[r], 2^bexp[c])
// and split into S bf16 digit slices in the k-blocked layout, and a persistent tcgen05
// kernel forms the 128 x 64 tiles.  Used for the backward's products.
struct SgJob {                       // CUtensorMap members force 64-byte alignment
  CUtensorMap mapA, mapB;            // slices: [slice][k / 32][row or column][32]
  SgOp a, b;                         // A (M x K) and B (K x N), element by element
  double* C;                         // C[r, c] = C[r + c ldc], or cptrs[cc0 + c][r]
  double* const* cptrs;
  const int *Mdev, *Ndev, *Kdev;     // actual sizes (device), or null
  double alpha, beta;
  const double* crow;                // row scales of C (with alpha = 1, beta = 0), or null
  uint16_t *as, *bs;
  int32_t *aexp, *bexp;              // INT32_MIN: a zero row / column
  unsigned long long *amax, *bmax;   // row / column maxima of |A|, |B| (magnitude bits)
  int64_t ldc;
  int32_t M, N, K, Kp;               // Kp: K rounded up to 64
  int32_t cc0, pad_;
};

// The operand with its device-held offsets read once: k1 of the stacked forms, the
// column offset of SG_DENSE_T.
__device__ __forceinline__ SgOp sg_resolve(const SgOp& o) {
  SgOp r = o;
  if (o.split) r.k1 = *o.split;
  if (o.off_dev) r.c0 += *o.off_dev;
  return r;
}
__device__ __forceinline__ int sg_size(const int* dev, int host) { return dev ? min(*dev, host) : host; }
// Element (row, col) of an operand in the SG_* form MODE (the forms are listed with
// SgOp), without branches (but for the live-row test of SG_XCOLS): an element outside the
// operand (ok false) is read at the operand's first element and replaced by zero, so that
// the loads of several elements can be in flight together.
template <int MODE>
__device__ __forceinline__ double sg_ld(const SgOp& o, int row, int col, bool ok) {
  row = ok ? row : 0;
  col = ok ? col : 0;
  double x;
  if constexpr (MODE == SG_DENSE) {
    x = o.p[(int64_t)(o.r0 + row) + (int64_t)(o.c0 + col) * o.ld];
  } else if constexpr (MODE == SG_DENSE_T) {
    x = o.p[(int64_t)(o.c0 + col) + (int64_t)(o.r0 + row) * o.ld];
  } else if constexpr (MODE == SG_QHAT || MODE == SG_QHAT_T || MODE == SG_QHAT_RAW || MODE == SG_QHAT_T_RAW) {
    constexpr bool tr = MODE == SG_QHAT_T || MODE == SG_QHAT_T_RAW;
    const int j = tr ? o.c0 + col : o.r0 + row;                 // Qhat(j, i)
    const int i = tr ? o.r0 + row : o.c0 + col;
    if constexpr (MODE == SG_QHAT || MODE == SG_QHAT_T) x = o.wcol[i][j] * o.sinv[i];
    else x = o.wcol[i][j];
    if (o.lid) ok = ok && o.lid[i] != o.lid[j];
  } else if constexpr (MODE == SG_DENSE_RS) {
    x = o.p[(int64_t)(o.r0 + row) + (int64_t)(o.c0 + col) * o.ld] * o.rs[o.r0 + row];
  } else if constexpr (MODE == SG_XCOLS) {
    const int j = o.c0 + col;
    ok = ok && row >= o.xlo[j] && row < o.xhi[j];
    x = ok ? o.xcol[j][row] : 0.0;             // rows outside the live range are not read
  } else if constexpr (MODE == SG_STACK) {
    const bool first = col < o.k1;
    x = first ? o.p[(int64_t)(o.r0 + row) + (int64_t)col * o.ld]
              : o.p2[(int64_t)(o.r0 + row) + (int64_t)(col - o.k1) * o.ld2];
  } else {                                  // SG_STACK_ROWS
    const bool first = row < o.k1;
    x = first ? o.p[(int64_t)row + (int64_t)(o.c0 + col) * o.ld]
              : o.p2[(int64_t)(row - o.k1) + (int64_t)(o.c0 + col) * o.ld2];
  }
  return ok ? x : 0.0;
}

// Slicing of the operands, in two launches each so that every block has a bounded
// share of k and the grid covers the device whatever the operand's shape:
//   k_sg_amax / k_sg_bmax  partial row (column) maxima of |A| (|B|) over one chunk of k,
//                          combined with atomicMax on the magnitude bits (integer order =
//                          order of |x|) into amax / bmax, zeroed before;
//   k_sg_slice_a / _b      the row's (column's) power of two from that maximum, then the
//                          digits of the chunk.
// A: blocks of 32 rows x kSgChunkA k; lanes run along whichever index is contiguous in
// memory, through shared memory.  B: blocks of 8 columns (a warp each) x kSgChunkB k.
constexpr int kSgChunkA = 512;
constexpr int kSgChunkB = 2048;
__device__ __forceinline__ unsigned long long sg_mag(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ int sg_exp_of(unsigned long long mb) {   // 2^(e-1) <= m < 2^e
  int e = 0;
  const double m = __longlong_as_double((long long)mb);
  if (m > 0.0) frexp(m, &e);
  return e;
}
struct SgABlock {
  int jb, r0, k0;
};
__device__ __forceinline__ SgABlock sg_ablock(const SgJob* __restrict__ jobs, const int64_t* __restrict__ cum,
                                              int njobs) {
  SgABlock b;
  b.jb = find_job(cum, njobs, blockIdx.x);
  const int64_t local = blockIdx.x - cum[b.jb];
  const int nkc = (jobs[b.jb].Kp + kSgChunkA - 1) / kSgChunkA;
  b.r0 = (int)(local / nkc) * 32;
  b.k0 = (int)(local % nkc) * kSgChunkA;
  return b;
}

template <int MODE>
__global__ __launch_bounds__(256) void k_sg_amax(const SgJob* __restrict__ jobs, int njobs,
                                                 const int64_t* __restrict__ cum) {
  __shared__ unsigned long long s_max[8][32];
  const SgABlock blk = sg_ablock(jobs, cum, njobs);
  const SgJob& J = jobs[blk.jb];
  const int r0 = blk.r0, tid = threadIdx.x;
  const int Me = sg_size(J.Mdev, J.M), kend = min(sg_size(J.Kdev, J.K), blk.k0 + kSgChunkA);
  const SgOp A = sg_resolve(J.a);
  auto at = [&](int r, int k) -> double { return sg_ld<MODE>(A, r0 + r, k, r0 + r < Me && k < kend); };
  constexpr bool rowc = MODE != SG_DENSE_T && MODE != SG_QHAT_T && MODE != SG_QHAT_T_RAW;   // consecutive rows adjacent in memory
  if constexpr (rowc) {                             // lanes along rows, 8 consecutive k per warp
    const int r = tid & 31, kq = tid >> 5;
    unsigned long long mx = 0ull;
    for (int k0 = blk.k0 + kq * 8; k0 < kend; k0 += 64) {
      unsigned long long v[8];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) v[kk] = sg_mag(at(r, k0 + kk));
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) mx = v[kk] > mx ? v[kk] : mx;
    }
    s_max[kq][r] = mx;
  } else {                                          // a warp per four rows, lanes along k
    const int lane = tid & 31, wq = tid >> 5;
    unsigned long long m[4] = {0ull, 0ull, 0ull, 0ull};
    for (int k = blk.k0 + lane; k < kend; k += 64) {
      unsigned long long v[4][2];
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        v[rr][0] = sg_mag(at(wq * 4 + rr, k));
        v[rr][1] = sg_mag(at(wq * 4 + rr, k + 32));
      }
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        m[rr] = v[rr][0] > m[rr] ? v[rr][0] : m[rr];
        m[rr] = v[rr][1] > m[rr] ? v[rr][1] : m[rr];
      }
    }
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, m[rr], off);
        m[rr] = o > m[rr] ? o : m[rr];
      }
      if (lane == 0) s_max[0][wq * 4 + rr] = m[rr];
    }
    if (tid < 32)
      for (int q = 1; q < 8; ++q) s_max[q][tid] = 0ull;
  }
  __syncthreads();
  if (tid < 32 && r0 + tid < Me) {
    unsigned long long mb = s_max[0][tid];
    for (int q = 1; q < 8; ++q) mb = s_max[q][tid] > mb ? s_max[q][tid] : mb;
    if (mb) atomicMax(J.amax + r0 + tid, mb);
  }
}

template <int S, int MODE>
__global__ __launch_bounds__(256) void k_sg_slice_a(const SgJob* __restrict__ jobs, int njobs,
                                                    const int64_t* __restrict__ cum) {
  __shared__ double tile[64][33];
  __shared__ int s_exp[32];
  const SgABlock blk = sg_ablock(jobs, cum, njobs);
  const SgJob& J = jobs[blk.jb];
  const int r0 = blk.r0, tid = threadIdx.x;
  const int M = J.M, K = sg_size(J.Kdev, J.K), Me = sg_size(J.Mdev, J.M), Kp = J.Kp;
  uint16_t* const as = J.as;
  const SgOp A = sg_resolve(J.a);
  auto at = [&](int r, int k) -> double { return sg_ld<MODE>(A, r0 + r, k, r0 + r < Me && k < K); };
  constexpr bool rowc = MODE != SG_DENSE_T && MODE != SG_QHAT_T && MODE != SG_QHAT_T_RAW;
  if (tid < 32) {
    const unsigned long long mb = r0 + tid < M ? J.amax[r0 + tid] : 0ull;
    const int e = sg_exp_of(mb);
    s_exp[tid] = e;
    if (blk.k0 == 0 && r0 + tid < M) J.aexp[r0 + tid] = mb ? e : INT32_MIN;
  }
  __syncthreads();
  const int wr = tid >> 3, wk = (tid & 7) * 8;
  const int shift = 8 * S - 1 - s_exp[wr];
  const int kstop = min(Kp, blk.k0 + kSgChunkA);
  for (int k0 = blk.k0; k0 < kstop; k0 += 64) {
    if constexpr (rowc) {
      const int r = tid & 31, kq = tid >> 5;
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) tile[kq * 8 + kk][r] = at(r, k0 + kq * 8 + kk);
    } else {
      const int k = tid & 63, rq = tid >> 6;
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) tile[k][rq * 8 + rr] = at(rq * 8 + rr, k0 + k);
    }
    __syncthreads();
    if (r0 + wr < M) {
      uint16_t dg[8][S];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint16_t t[S];
        digits_bf16<S>(round_scaled(tile[wk + j][wr], shift), t);
#pragma unroll
        for (int p = 0; p < S; ++p) dg[j][p] = t[p];
      }
      const int k = k0 + wk;
#pragma unroll
      for (int p = 0; p < S; ++p) {
        uint4 v;
        v.x = (uint32_t)dg[0][p] | ((uint32_t)dg[1][p] << 16);
        v.y = (uint32_t)dg[2][p] | ((uint32_t)dg[3][p] << 16);
        v.z = (uint32_t)dg[4][p] | ((uint32_t)dg[5][p] << 16);
        v.w = (uint32_t)dg[6][p] | ((uint32_t)dg[7][p] << 16);
        *reinterpret_cast<uint4*>(as + (((int64_t)p * (Kp / kOzBK) + k / kOzBK) * M + r0 + wr) * kOzBK +
                                  (k % kOzBK)) = v;
      }
    }
    __syncthreads();
  }
}

struct SgBBlock {
  int jb, c, k0;
};
__device__ __forceinline__ SgBBlock sg_bblock(const SgJob* __restrict__ jobs, const int64_t* __restrict__ cum,
                                              int njobs) {
  SgBBlock b;
  b.jb = find_job(cum, njobs, blockIdx.x);
  const int64_t local = blockIdx.x - cum[b.jb];
  const int nkc = (jobs[b.jb].Kp + kSgChunkB - 1) / kSgChunkB;
  b.c = (int)(local / nkc) * 8 + (int)(threadIdx.x >> 5);
  b.k0 = (int)(local % nkc) * kSgChunkB;
  return b;
}

template <int MODE>
__global__ __launch_bounds__(256) void k_sg_bmax(const SgJob* __restrict__ jobs, int njobs,
                                                 const int64_t* __restrict__ cum) {
  const SgBBlock blk = sg_bblock(jobs, cum, njobs);
  const SgJob& J = jobs[blk.jb];
  const int lane = threadIdx.x & 31, c = blk.c;
  if (c >= J.N) return;                             // uniform over the warp
  const bool live = !J.Ndev || c < *J.Ndev;         // columns past the actual count are zero
  const int kend = min(sg_size(J.Kdev, J.K), blk.k0 + kSgChunkB);
  const SgOp B = sg_resolve(J.b);
  unsigned long long m = 0ull;
  for (int k0 = blk.k0 + lane; k0 < kend; k0 += 128) {   // four independent loads in flight
    unsigned long long v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = sg_mag(sg_ld<MODE>(B, k0 + 32 * u, c, live && k0 + 32 * u < kend));
#pragma unroll
    for (int u = 0; u < 4; ++u) m = v[u] > m ? v[u] : m;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, off);
    m = o > m ? o : m;
  }
  if (lane == 0 && m) atomicMax(J.bmax + c, m);
}

template <int S, int MODE>
__global__ __launch_bounds__(256) void k_sg_slice_b(const SgJob* __restrict__ jobs, int njobs,
                                                    const int64_t* __restrict__ cum) {
  const SgBBlock blk = sg_bblock(jobs, cum, njobs);
  const SgJob& J = jobs[blk.jb];
  const int lane = threadIdx.x & 31, c = blk.c;
  if (c >= J.N) return;                             // uniform over the warp
  const bool live = !J.Ndev || c < *J.Ndev;
  const int K = sg_size(J.Kdev, J.K), Kp = J.Kp, N = J.N;
  uint16_t* const bs = J.bs;
  const SgOp B = sg_resolve(J.b);
  const unsigned long long mb = J.bmax[c];
  const int e = sg_exp_of(mb);
  if (lane == 0 && blk.k0 == 0) J.bexp[c] = mb ? e : INT32_MIN;
  const int shift = 8 * S - 1 - e;
  const int kstop = min(Kp, blk.k0 + kSgChunkB);
  for (int k0 = blk.k0 + lane * 8; k0 < kstop; k0 += 256) {
    uint16_t dg[8][S];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint16_t t[S];
      digits_bf16<S>(round_scaled(sg_ld<MODE>(B, k0 + j, c, live && k0 + j < K), shift), t);
#pragma unroll
      for (int p = 0; p < S; ++p) dg[j][p] = t[p];
    }
#pragma unroll
    for (int p = 0; p < S; ++p) {
      uint4 v;
      v.x = (uint32_t)dg[0][p] | ((uint32_t)dg[1][p] << 16);
      v.y = (uint32_t)dg[2][p] | ((uint32_t)dg[3][p] << 16);
      v.z = (uint32_t)dg[4][p] | ((uint32_t)dg[5][p] << 16);
      v.w = (uint32_t)dg[6][p] | ((uint32_t)dg[7][p] << 16);
      *reinterpret_cast<uint4*>(bs + (((int64_t)p * (Kp / kOzBK) + k0 / kOzBK) * N + c) * kOzBK +
                                (k0 % kOzBK)) = v;
    }
  }
}

// The persistent GEMM over the batch's 128 x 64 tiles (cum: tiles of the jobs before
// j).  Same roles, barriers, MMA schedule and epilogue combination as k_oz_gemm; the
// k range is the whole padded K of the job.
struct SgTile {
  int jb, row0, ct, nst, nchunks;
};
__device__ __forceinline__ SgTile sg_tile(const SgJob* __restrict__ jobs, const int64_t* __restrict__ cum,
                                          int njobs, int64_t t) {
  SgTile v;
  v.jb = find_job(cum, njobs, t);
  const int64_t local = t - cum[v.jb];
  const int nct = (jobs[v.jb].N + kOzBN - 1) / kOzBN;
  v.ct = (int)(local % nct);
  v.row0 = (int)(local / nct) * kOzBM;
  v.nst = jobs[v.jb].Kp / kOzBK;
  v.nchunks = (v.nst + kOzChunk / kOzBK - 1) / (kOzChunk / kOzBK);
  return v;
}

template <int S>
__global__ __launch_bounds__(kThreads, 1) void k_sg_gemm(const SgJob* __restrict__ jobs, int njobs,
                                                         const int64_t* __restrict__ cum, int* err0) {
  using C = OzCfg<S>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::ST * C::STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * C::ST + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int64_t total = cum[njobs];
  if ((int64_t)blockIdx.x >= total) return;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (C::ST + s); };
  const uint32_t accfull = bar0 + 8u * (2 * C::ST);
  const uint32_t accempty = bar0 + 8u * (2 * C::ST + 1);
  const uint32_t done = bar0 + 8u * (2 * C::ST + 2);
  const uint32_t tfree = bar0 + 8u * (2 * C::ST + 3);
  int* err = err0;

  if (tid == 0) {
    for (int s = 0; s < C::ST; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(accfull, 1);
    mbar_init(accempty, kEpiWarps);
    mbar_init(done, 1);
    mbar_init(tfree, kEpiWarps);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (warp >= 2) {
    const uint32_t tq = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(((warp - 2) >> 2) * 32);
#pragma unroll
    for (int L = 0; L < C::NL; ++L) tmem_st32_zero(tq + (uint32_t)(L * kOzBN));
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      uint32_t g = 0, issued_total = 0;
      for (int64_t t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x) {
        const SgTile T = sg_tile(jobs, cum, njobs, t);
        const CUtensorMap* mA = &jobs[T.jb].mapA;
        const CUtensorMap* mB = &jobs[T.jb].mapB;
        asm volatile("prefetch.tensormap [%0];" ::"l"(mA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(mB) : "memory");
        bool ok = true;
        for (int it = 0; it < T.nst; ++it, ++g) {
          const int s = (int)(g % C::ST);
          const uint32_t ph = (g / C::ST) & 1u;
          if (!mbar_wait(empty(s), ph ^ 1u, abort_flag, err)) { ok = false; break; }
          const uint32_t sa = smem_u32(smem + s * C::STAGE);
          mbar_expect_tx(full(s), C::STAGE);
          tma_load_4d(sa, mA, full(s), 0, T.row0, it, 0);
          tma_load_4d(sa + C::A_BYTES, mB, full(s), 0, T.ct * kOzBN, it, 0);
          issued_total = g + 1;
        }
        if (!ok) break;
      }
      if (*abort_flag) {
        const long long t0 = global_ns();
        for (uint32_t q = (issued_total > (uint32_t)C::ST ? issued_total - C::ST : 0u); q < issued_total; ++q) {
          const uint32_t ph = (q / C::ST) & 1u;
          while (!mbar_try(full((int)(q % C::ST)), ph) && global_ns() - t0 < kWaitNs) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      const int per_chunk = kOzChunk / kOzBK;
      uint32_t g = 0, cg = 0, ti = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < total && ok; t += gridDim.x) {
        const SgTile T = sg_tile(jobs, cum, njobs, t);
        if (T.nst == 0) continue;
        if (ti > 0) {
          if (!mbar_wait(tfree, (ti - 1) & 1u, abort_flag, err)) { ok = false; break; }
          tc_fence_after();
        }
        for (int it = 0; it < T.nst; ++it, ++g) {
          const int s = (int)(g % C::ST);
          const uint32_t ph = (g / C::ST) & 1u;
          if (!mbar_wait(full(s), ph, abort_flag, err)) { ok = false; break; }
          tc_fence_after();
          const int chunk = it / per_chunk;
          const bool first = (it % per_chunk) == 0;
          const bool last = (it % per_chunk) == per_chunk - 1 || it == T.nst - 1;
          const uint32_t sa = smem_u32(smem + s * C::STAGE);
          const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < kOzBK / 16; ++kk) {
#pragma unroll
            for (int p = 1; p <= S; ++p) {
#pragma unroll
              for (int qa = 1; qa <= 5; qa += 4) {
                if (qa <= C::qmax(p) && p + qa >= 6) {
                  const int nq = C::qmax(p) - qa + 1 < 4 ? C::qmax(p) - qa + 1 : 4;
                  tc_mma(tmem + (uint32_t)((p + qa - 2) * kOzBN),
                         sdesc(sa + (p - 1) * (kOzBM * kOzBK * 2) + kk * 32),
                         sdesc(sb + (qa - 1) * (kOzBN * kOzBK * 2) + kk * 32), idesc_n(nq), 1u);
                }
              }
            }
            if (first && kk == 0 && chunk > 0) {
              if (!mbar_wait(accempty, (cg - 1) & 1u, abort_flag, err)) { ok = false; break; }
              tc_fence_after();
            }
#pragma unroll
            for (int p = 1; p <= 4; ++p) {
              const int nq = C::qmax(p) < 4 ? C::qmax(p) : 4;
              const uint32_t acc = (p == 1 && first && kk == 0) ? 0u : 1u;
              tc_mma(tmem + (uint32_t)((p - 1) * kOzBN), sdesc(sa + (p - 1) * (kOzBM * kOzBK * 2) + kk * 32),
                     sdesc(sb + kk * 32), idesc_n(nq), acc);
            }
          }
          if (!ok) break;
          tc_commit(empty(s));
          if (last) {
            tc_commit(accfull);
            ++cg;
          }
        }
        if (!ok) break;
        tc_commit(done);
        ++ti;
      }
      if (*abort_flag) {
        tc_commit(done);
        const long long t0 = global_ns();
        if (ti > 0)
          while (!mbar_try(done, (ti - 1) & 1u) && global_ns() - t0 < kWaitNs) {
          }
        while (!mbar_try(done, ti & 1u) && global_ns() - t0 < kWaitNs) {
        }
      }
    }
  } else {
    // ---------------- epilogue (as k_oz_gemm's)
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quad * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 32);
    uint32_t cg = 0, ti = 0;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
      const SgTile T = sg_tile(jobs, cum, njobs, t);
      const SgJob& J = jobs[T.jb];
      long long acc[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = 0;
      bool ok = true;
      for (int c = 0; c < T.nchunks; ++c) {
        const bool got = __all_sync(0xffffffffu, mbar_wait(accfull, cg & 1u, abort_flag, err));
        if (!got) { ok = false; break; }
        tc_fence_after();
#pragma unroll
        for (int L = 2; L <= 5; ++L) {
          uint32_t v[32];
          tmem_ld32(trow + (uint32_t)((L - 2) * kOzBN), v);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 32; ++j)
            acc[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << (8 * (5 - L));
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(accempty);
        ++cg;
      }
      float tsum[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) tsum[j] = 0.0f;
      if (ok && T.nst > 0) {
        ok = __all_sync(0xffffffffu, mbar_wait(done, ti & 1u, abort_flag, err));
        if (ok) {
          tc_fence_after();
#pragma unroll
          for (int L = S + 2; L >= 6; --L) {
            uint32_t v[32];
            tmem_ld32(trow + (uint32_t)((L - 2) * kOzBN), v);
            tmem_wait_ld();
            const float wL = __int_as_float((127 - 8 * (L - 6)) << 23);
#pragma unroll
            for (int j = 0; j < 32; ++j) tsum[j] = fmaf(__uint_as_float(v[j]), wL, tsum[j]);
          }
#pragma unroll
          for (int L = 6; L <= S + 2; ++L) tmem_st32_zero(trow + (uint32_t)((L - 2) * kOzBN));
          tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tfree);
          ++ti;
        }
      }
      if (!ok) break;
      // the job's fields in registers first (the stores below could otherwise alias the
      // job table for the compiler and force it to reload them), then the output
      // addresses, exponents and (with beta) old values eight columns at a time, so that
      // their loads are in flight together
      const int grow = T.row0 + row;
      const int ncol = sg_size(J.Ndev, J.N), mrow = sg_size(J.Mdev, J.M);
      double* const* const cptrs = J.cptrs;
      double* const Cb = J.C;
      const int64_t ldc = J.ldc;
      const int cc0 = J.cc0;
      const double alpha = J.alpha, beta = J.beta;
      // the update's form, uniform per job: branches around whole groups (an FP64
      // operation under a per-output predicate would still issue on the 2-lane FP64 pipe)
      const double* const crow = J.crow;
      const int emode = crow ? 3 : ((alpha == 1.0 && beta == 0.0) ? 0 : ((alpha == 1.0 && beta == 1.0) ? 1 : 2));
      const int32_t* const bexp = J.bexp;
      if (grow < mrow) {
        const int ea = J.aexp[grow];
        const int colb = T.ct * kOzBN + half * 32;
#pragma unroll
        for (int g = 0; g < 32; g += 8) {
          double* dst[8];
          int eb[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int col = colb + g + j;
            const bool in = col < ncol;
            eb[j] = in ? bexp[col] : INT32_MIN;
            dst[j] = !in ? nullptr : (cptrs ? cptrs[cc0 + col] + grow : Cb + (int64_t)grow + (int64_t)col * ldc);
          }
          if (emode == 0) {                      // C = A B
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (dst[j]) *dst[j] = (ea == INT32_MIN || eb[j] == INT32_MIN) ? 0.0 : oz_combine(acc[g + j], tsum[g + j], eb[j] - 38 + ea);
          } else if (emode == 3) {               // C = diag(crow) A B
            const double cr = crow[grow];
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (dst[j])
                *dst[j] = cr * ((ea == INT32_MIN || eb[j] == INT32_MIN) ? 0.0
                                : oz_combine(acc[g + j], tsum[g + j], eb[j] - 38 + ea));
          } else {                               // C = alpha A B + beta C
            double old[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) old[j] = dst[j] ? *dst[j] : 0.0;
            if (emode == 1) {                      // C += A B
#pragma unroll
              for (int j = 0; j < 8; ++j)
                if (dst[j])
                  *dst[j] = old[j] + ((ea == INT32_MIN || eb[j] == INT32_MIN) ? 0.0
                                      : oz_combine(acc[g + j], tsum[g + j], eb[j] - 38 + ea));
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j)
                if (dst[j])
                  *dst[j] = fma(alpha, (ea == INT32_MIN || eb[j] == INT32_MIN) ? 0.0
                                       : oz_combine(acc[g + j], tsum[g + j], eb[j] - 38 + ea), beta * old[j]);
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

}  // namespace

size_t oz_job_bytes(const MergeJob& J, int slices) {
  const int64_t m = J.n1 + J.n2, ldk = job_ldk(J);
  size_t b = 0;
  b += rup(slices * (int64_t)J.n1 * ldk * 2, 256);
  b += rup(slices * (int64_t)J.n2 * ldk * 2, 256);
  b += rup(slices * m * ldk * 2, 256);
  b += rup(m * 8, 256);
  b += rup(m * 4, 256);
  return b;
}

bool oz_fill_job(OzJob& z, const MergeJob& J, unsigned char* base, int slices) {
  std::memset(&z, 0, sizeof(z));
  const int64_t m = J.n1 + J.n2, ldk = job_ldk(J);
  size_t off = 0;
  z.a[0] = reinterpret_cast<uint16_t*>(base + off);
  off += rup(slices * (int64_t)J.n1 * ldk * 2, 256);
  z.a[1] = reinterpret_cast<uint16_t*>(base + off);
  off += rup(slices * (int64_t)J.n2 * ldk * 2, 256);
  z.b = reinterpret_cast<uint16_t*>(base + off);
  off += rup(slices * m * ldk * 2, 256);
  z.sigma = reinterpret_cast<double*>(base + off);
  off += rup(m * 8, 256);
  z.texp = reinterpret_cast<int32_t*>(base + off);
  z.ldk = ldk;
  z.slices = slices;
  bool ok = encode4d(&z.mapA[0], z.a[0], ldk, J.n1, slices, kOzBM);
  ok = ok && encode4d(&z.mapA[1], z.a[1], ldk, J.n2, slices, kOzBM);
  ok = ok && encode4d(&z.mapB, z.b, ldk, m, slices, kOzBN);
  return ok;
}

int64_t oz_blocks_slice_a(const MergeJob& J) { return (J.n1 + 31) / 32 + (J.n2 + 31) / 32; }
int64_t oz_blocks_slice_b(const MergeJob& J) {
  return (int64_t)(J.n1 + J.n2) * ((job_ldk(J) + 2047) / 2048);
}
int64_t oz_tiles(const MergeJob& J) {
  const int64_t m = J.n1 + J.n2;
  return ((J.n1 + kOzBM - 1) / kOzBM + (J.n2 + kOzBM - 1) / kOzBM) * ((m + kOzBN - 1) / kOzBN);
}

void launch_ozaki_level(int part, const MergeJob* jobs, const OzJob* ozj, int njobs, const int64_t* cum_sa,
                        int64_t nb_sa, int64_t* cum_sb, int64_t nb_sb, int64_t* cum_t,
                        int64_t ntiles, int slices, QBufs qb, DevWs w, cudaStream_t st) {
  switch (slices) {
    case 5: launch_s<5>(part, jobs, ozj, njobs, cum_sa, nb_sa, cum_sb, nb_sb, cum_t, ntiles, qb, w, st); break;
    case 7: launch_s<7>(part, jobs, ozj, njobs, cum_sa, nb_sa, cum_sb, nb_sb, cum_t, ntiles, qb, w, st); break;
    default: launch_s<6>(part, jobs, ozj, njobs, cum_sa, nb_sa, cum_sb, nb_sb, cum_t, ntiles, qb, w, st); break;
  }
}

namespace {
constexpr int kSgForms = 10;                    // the SG_* forms: one slicing launch each
}  // namespace

// The job table, the per-form block counts of A and B and the tile counts (as
// split_gemm_s takes them), then each problem's slices, exponents and maxima.
size_t split_gemm_bytes(const std::vector<SgProblem>& pr, int slices) {
  const int S = slices < 5 ? 5 : (slices > 7 ? 7 : slices);
  const int64_t cum = ((int64_t)pr.size() + 1) * 8;
  size_t b = rup((int64_t)pr.size() * (int64_t)sizeof(SgJob), 256) + 2 * rup(kSgForms * cum, 256) + rup(cum, 256);
  int64_t nmax = 0;
  for (const SgProblem& p : pr) {
    const int64_t Kp = rup(p.K, 64);
    b += rup((int64_t)S * p.M * Kp * 2, 256) + rup((int64_t)S * p.N * Kp * 2, 256) + rup((int64_t)p.M * 4, 256) +
         rup((int64_t)p.N * 4, 256);
    nmax += p.M + p.N;
  }
  return b + rup(nmax * 8, 256) + 512;
}

namespace {
// The maxima launch of a form, then its digits launch (same blocks).
template <int MODE>
void launch_max(bool a, unsigned grid, const SgJob* jobs, int nj, const int64_t* cum, cudaStream_t st) {
  if (a) k_sg_amax<MODE><<<grid, 256, 0, st>>>(jobs, nj, cum);
  else k_sg_bmax<MODE><<<grid, 256, 0, st>>>(jobs, nj, cum);
}
void launch_maxima(bool a, int form, unsigned grid, const SgJob* jobs, int nj, const int64_t* cum, cudaStream_t st) {
  switch (form) {
    case SG_DENSE: launch_max<SG_DENSE>(a, grid, jobs, nj, cum, st); break;
    case SG_DENSE_T: launch_max<SG_DENSE_T>(a, grid, jobs, nj, cum, st); break;
    case SG_QHAT: launch_max<SG_QHAT>(a, grid, jobs, nj, cum, st); break;
    case SG_QHAT_T: launch_max<SG_QHAT_T>(a, grid, jobs, nj, cum, st); break;
    case SG_XCOLS: launch_max<SG_XCOLS>(a, grid, jobs, nj, cum, st); break;
    case SG_STACK: launch_max<SG_STACK>(a, grid, jobs, nj, cum, st); break;
    case SG_QHAT_RAW: launch_max<SG_QHAT_RAW>(a, grid, jobs, nj, cum, st); break;
    case SG_QHAT_T_RAW: launch_max<SG_QHAT_T_RAW>(a, grid, jobs, nj, cum, st); break;
    case SG_DENSE_RS: launch_max<SG_DENSE_RS>(a, grid, jobs, nj, cum, st); break;
    default: launch_max<SG_STACK_ROWS>(a, grid, jobs, nj, cum, st); break;
  }
}
template <int S>
void launch_slice_a(int form, unsigned grid, const SgJob* jobs, int nj, const int64_t* cum, cudaStream_t st) {
  switch (form) {
    case SG_DENSE: k_sg_slice_a<S, SG_DENSE><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_DENSE_T: k_sg_slice_a<S, SG_DENSE_T><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_QHAT: k_sg_slice_a<S, SG_QHAT><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_QHAT_T: k_sg_slice_a<S, SG_QHAT_T><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_XCOLS: k_sg_slice_a<S, SG_XCOLS><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_STACK: k_sg_slice_a<S, SG_STACK><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_QHAT_RAW: k_sg_slice_a<S, SG_QHAT_RAW><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_QHAT_T_RAW: k_sg_slice_a<S, SG_QHAT_T_RAW><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_DENSE_RS: k_sg_slice_a<S, SG_DENSE_RS><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    default: k_sg_slice_a<S, SG_STACK_ROWS><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
  }
}
template <int S>
void launch_slice_b(int form, unsigned grid, const SgJob* jobs, int nj, const int64_t* cum, cudaStream_t st) {
  switch (form) {
    case SG_DENSE: k_sg_slice_b<S, SG_DENSE><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_DENSE_T: k_sg_slice_b<S, SG_DENSE_T><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_QHAT: k_sg_slice_b<S, SG_QHAT><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_QHAT_T: k_sg_slice_b<S, SG_QHAT_T><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_XCOLS: k_sg_slice_b<S, SG_XCOLS><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_STACK: k_sg_slice_b<S, SG_STACK><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_QHAT_RAW: k_sg_slice_b<S, SG_QHAT_RAW><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_QHAT_T_RAW: k_sg_slice_b<S, SG_QHAT_T_RAW><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    case SG_DENSE_RS: k_sg_slice_b<S, SG_DENSE_RS><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
    default: k_sg_slice_b<S, SG_STACK_ROWS><<<grid, 256, 0, st>>>(jobs, nj, cum); break;
  }
}

template <int S>
int split_gemm_s(const std::vector<SgProblem>& pr, unsigned char* ws, size_t ws_bytes, int* err, cudaStream_t st) {
  using C = OzCfg<S>;
  static std::mutex mu;
  static bool attr[64] = {};
  static int sms[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int nsm = 148;
  {
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64 || !attr[dev]) {
      cudaFuncSetAttribute(k_sg_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
      int n = 0;
      if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 148;
      if (dev >= 0 && dev < 64) {
        attr[dev] = true;
        sms[dev] = n;
      }
      nsm = n;
    } else {
      nsm = sms[dev];
    }
  }
  const size_t nj = pr.size();
  size_t off = (256 - (reinterpret_cast<uintptr_t>(ws) & 255)) & 255;
  auto take = [&](size_t bytes) {
    unsigned char* p = ws + off;
    off = (size_t)rup((int64_t)(off + bytes), 256);
    return p;
  };
  SgJob* djobs = reinterpret_cast<SgJob*>(take(nj * sizeof(SgJob)));
  int64_t* dca = reinterpret_cast<int64_t*>(take(kSgForms * (nj + 1) * 8));   // per form of A
  int64_t* dcb = reinterpret_cast<int64_t*>(take(kSgForms * (nj + 1) * 8));   // per form of B
  int64_t* dct = reinterpret_cast<int64_t*>(take((nj + 1) * 8));
  size_t nmax = 0;                               // row and column maxima, one zeroed region
  for (size_t j = 0; j < nj; ++j)
    nmax += (pr[j].a_from >= 0 && (size_t)pr[j].a_from < j ? 0 : (size_t)pr[j].M) + (size_t)pr[j].N;
  unsigned long long* maxima = reinterpret_cast<unsigned long long*>(take(nmax * 8));
  size_t moff = 0;
  std::vector<SgJob> jobs(nj);
  std::vector<int64_t> ca(kSgForms * (nj + 1), 0), cb(kSgForms * (nj + 1), 0), ct(nj + 1, 0);
  for (size_t j = 0; j < nj; ++j) {
    const SgProblem& p = pr[j];
    SgJob& J = jobs[j];
    J = SgJob{};
    J.M = p.M;
    J.N = p.N;
    J.K = p.K;
    J.Kp = (int32_t)rup(p.K, 64);
    J.a = p.a;
    J.b = p.b;
    J.C = p.C;
    J.ldc = p.ldc;
    J.cptrs = p.cptrs;
    J.cc0 = p.cc0;
    J.Mdev = p.Mdev;
    J.Ndev = p.Ndev;
    J.Kdev = p.Kdev;
    J.alpha = p.alpha;
    J.beta = p.beta;
    J.crow = p.crow;
    if (p.crow && (p.alpha != 1.0 || p.beta != 0.0)) return -1;
    const bool shared = p.a_from >= 0 && (size_t)p.a_from < j;
    if (shared) {
      const SgJob& src = jobs[p.a_from];
      if (src.M != J.M || src.Kp != J.Kp) return -1;
      J.as = src.as;
      J.aexp = src.aexp;
      J.amax = src.amax;
      J.mapA = src.mapA;
    } else {
      J.as = reinterpret_cast<uint16_t*>(take((size_t)S * p.M * J.Kp * 2));
      J.aexp = reinterpret_cast<int32_t*>(take((size_t)p.M * 4));
      J.amax = maxima + moff;
      moff += (size_t)p.M;
      if (!encode4d(&J.mapA, J.as, J.Kp, p.M, S, kOzBM)) return 4;
    }
    J.bs = reinterpret_cast<uint16_t*>(take((size_t)S * p.N * J.Kp * 2));
    J.bexp = reinterpret_cast<int32_t*>(take((size_t)p.N * 4));
    J.bmax = maxima + moff;
    moff += (size_t)p.N;
    if (!encode4d(&J.mapB, J.bs, J.Kp, p.N, S, kOzBN)) return 4;
    if (p.a.mode < 0 || p.a.mode >= kSgForms || p.b.mode < 0 || p.b.mode >= kSgForms) return -1;
    const int64_t na = (int64_t)((p.M + 31) / 32) * ((J.Kp + kSgChunkA - 1) / kSgChunkA);
    const int64_t nb = (int64_t)((p.N + 7) / 8) * ((J.Kp + kSgChunkB - 1) / kSgChunkB);
    for (int f = 0; f < kSgForms; ++f) {
      const size_t o = (size_t)f * (nj + 1);
      ca[o + j + 1] = ca[o + j] + (f == p.a.mode && !shared ? na : 0);
      cb[o + j + 1] = cb[o + j] + (f == p.b.mode ? nb : 0);
    }
    ct[j + 1] = ct[j] + (int64_t)((p.M + kOzBM - 1) / kOzBM) * ((p.N + kOzBN - 1) / kOzBN);
  }
  if (off > ws_bytes) return 3;
  cudaMemcpyAsync(djobs, jobs.data(), nj * sizeof(SgJob), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dca, ca.data(), ca.size() * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dcb, cb.data(), cb.size() * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dct, ct.data(), (nj + 1) * 8, cudaMemcpyHostToDevice, st);
  if (nmax) cudaMemsetAsync(maxima, 0, nmax * 8, st);
  for (int f = 0; f < kSgForms; ++f) {          // maxima, then digits, per form present
    const size_t o = (size_t)f * (nj + 1);
    if (ca[o + nj]) {
      launch_maxima(true, f, (unsigned)ca[o + nj], djobs, (int)nj, dca + o, st);
      launch_slice_a<S>(f, (unsigned)ca[o + nj], djobs, (int)nj, dca + o, st);
    }
    if (cb[o + nj]) {
      launch_maxima(false, f, (unsigned)cb[o + nj], djobs, (int)nj, dcb + o, st);
      launch_slice_b<S>(f, (unsigned)cb[o + nj], djobs, (int)nj, dcb + o, st);
    }
  }
  if (ct[nj]) {
    const unsigned grid = (unsigned)(ct[nj] < nsm ? ct[nj] : nsm);
    double tf = 0.0;
    for (const SgProblem& p : pr) tf += 2.0 * p.M * (double)p.N * (double)p.K;
    sg_gemm_mark(true, tf * oz_slice_pairs(S), st);
    k_sg_gemm<S><<<grid, kThreads, C::SMEM, st>>>(djobs, (int)nj, dct, err);
    sg_gemm_mark(false, 0.0, st);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
}  // namespace

int split_gemm(const std::vector<SgProblem>& pr, int slices, unsigned char* ws, size_t ws_bytes, int* dev_err,
               cudaStream_t st) {
  if (pr.empty()) return 0;
  for (const SgProblem& p : pr)
    if (p.M < 1 || p.N < 1 || p.K < 1 || (!p.C && !p.cptrs)) return -1;
  if (ws_bytes < split_gemm_bytes(pr, slices)) return 3;
  switch (slices < 5 ? 5 : (slices > 7 ? 7 : slices)) {
    case 5: return split_gemm_s<5>(pr, ws, ws_bytes, dev_err, st);
    case 7: return split_gemm_s<7>(pr, ws, ws_bytes, dev_err, st);
    default: return split_gemm_s<6>(pr, ws, ws_bytes, dev_err, st);
  }
}

int oz_slice_pairs(int slices) {
  int n = 0;
  for (int p = 1; p <= slices; ++p) n += slices < slices + 2 - p ? slices : slices + 2 - p;
  return n;
}

}  // namespace tdc

namespace tdc {
namespace {
// The product epilogue's combination of one output (integer-pipe conversions, one FP64
// addition), element by element.
__global__ void k_diag_combine(const long long* __restrict__ acc, const float* __restrict__ ts,
                               const int* __restrict__ e, double* __restrict__ r, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = oz_combine(acc[i], ts[i], e[i]);
}
// The product kernel's bounded wait, on an mbarrier that nothing arrives on: after
// limit_ns it sets the abort flag and ST_WAIT in *err and returns (no copy or MMA is
// in flight, no tensor memory is held).  out[0] = 1 if the wait ended by itself.
__global__ void k_diag_wait(long long limit_ns, int* err, int* out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) out[0] = mbar_wait(smem_u32(&bar), 0u, &abort_flag, err, limit_ns) ? 1 : 0;
}
}  // namespace
}  // namespace tdc

extern "C" int tdc_diag_wait_timeout(int64_t limit_ns, int* dev_status, int* dev_out, void* stream) {
  if (limit_ns < 1000 || limit_ns > tdc::kWaitNs) return -1;
  if (!dev_status) return -2;
  if (!dev_out) return -3;
  tdc::k_diag_wait<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>((long long)limit_ns, dev_status, dev_out);
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

extern "C" int tdc_diag_split_combine(const int64_t* acc, const float* tsum, const int32_t* e2, double* r, int64_t n,
                                      void* stream) {
  if (n < 0) return -5;
  if (n == 0) return 0;
  if (!acc) return -1;
  if (!tsum) return -2;
  if (!e2) return -3;
  if (!r) return -4;
  tdc::k_diag_combine<<<tdc::grid_cap((n + 255) / 256, 8), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const long long*>(acc), tsum, e2, r, n);
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
