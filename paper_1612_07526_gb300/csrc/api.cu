// C ABI of libtdc: argument checks, the DC tree plan, workspace layout and the
// level-by-level launch sequence.  See include/tdc.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/tdc.h"
#include "tdc_internal.cuh"
#include "tdc_ozaki.cuh"
#include "tdc_paths.cuh"

namespace tdc {

// ---------------------------------------------------------------------------
// Plan: the DC trees of all problems, leaves and merges grouped by height (a
// merge runs after both children; all merges of one height run together).
// ---------------------------------------------------------------------------
struct ProblemDesc {
  int64_t n;
  int64_t vbase;            // vector offset
  int64_t qa, lda;          // the caller's output: offset of (0,0), leading dimension
  int64_t pool;             // offset of the problem's pool (3n columns of n rows) in the pools
};

struct LevelPlan {
  std::vector<MergeJob> jobs;
  std::vector<int64_t> cw8, crows, ccols, ctiles;
  size_t o_jobs = 0, o_cw8 = 0, o_crows = 0, o_ccols = 0, o_ctiles = 0;
};

struct Plan {
  std::vector<LeafJob> leaves;
  std::vector<int64_t> tear_list, tear_ptr;
  std::vector<LevelPlan> levels;
  std::vector<int64_t> sign_qoff, sign_n, sign_ld, sign_cum;
  // the persistent kernel's view: problems largest first, each problem's merges bottom-up
  std::vector<PersistProb> pprobs;
  std::vector<MergeJob> pmerges;
  std::vector<int32_t> pmlev;
  int64_t nmerges = 0;
  int64_t maxm = 0;
  size_t o_leaves = 0, o_tlist = 0, o_tptr = 0, o_sq = 0, o_sn = 0, o_sl = 0, o_sc = 0;
  size_t o_pprobs = 0, o_pmerges = 0, o_pmlev = 0;
  std::vector<unsigned char> blob;
};

// Per problem: its leaves (contiguous in the leaf list: the tree is built problem by
// problem), tear points and merges in level order; problems sorted by order,
// largest first, so the persistent kernel's work queue ends on small problems.
static void persistent_lists(Plan& P, int nprob, const std::vector<int64_t>& vbase, const std::vector<int64_t>& nvec) {
  std::vector<std::vector<std::pair<MergeJob, int32_t>>> per(nprob);
  for (size_t l = 0; l < P.levels.size(); ++l)
    for (const MergeJob& J : P.levels[l].jobs) per[J.prob].push_back({J, (int32_t)l});
  std::vector<int64_t> leaf0(nprob, -1), nleaf(nprob, 0);
  for (size_t i = 0; i < P.leaves.size(); ++i) {
    const int p = P.leaves[i].prob;
    if (leaf0[p] < 0) leaf0[p] = (int64_t)i;
    ++nleaf[p];
  }
  P.pprobs.clear();
  P.pmerges.clear();
  P.pmlev.clear();
  for (int p = 0; p < nprob; ++p) {
    PersistProb q{};
    q.v0 = vbase[p];
    q.n = nvec[p];
    q.leaf0 = leaf0[p] < 0 ? 0 : leaf0[p];
    q.nleaf = (int32_t)nleaf[p];
    q.tear0 = P.tear_ptr[p];
    q.tear1 = P.tear_ptr[p + 1];
    q.merge0 = (int64_t)P.pmerges.size();
    q.nmerge = (int32_t)per[p].size();
    for (const auto& jm : per[p]) {
      P.pmerges.push_back(jm.first);
      P.pmlev.push_back(jm.second);
    }
    P.pprobs.push_back(q);
  }
  std::stable_sort(P.pprobs.begin(), P.pprobs.end(),
                   [](const PersistProb& a, const PersistProb& b) { return a.n > b.n; });
}

static int build_node(Plan& P, const ProblemDesc& pd, int prob, int64_t lo, int64_t n, int depth,
                      int leaf) {
  if (n <= leaf) {
    LeafJob L{};
    L.v_off = pd.vbase + lo;
    L.buf = depth == 0 ? 0 : 1;                 // a whole problem writes the caller's array
    L.q_off = L.buf ? pd.pool + lo * pd.n + lo : pd.qa + lo * pd.lda + lo;
    L.ld = (int32_t)(L.buf ? pd.n : pd.lda);
    L.nl = (int32_t)n;
    L.prob = prob;
    L.root = depth == 0 ? 1 : 0;
    L.lo = (int32_t)lo;
    P.leaves.push_back(L);
    return 0;
  }
  const int64_t n1 = n / 2;
  P.tear_list.push_back(pd.vbase + lo + n1 - 1);
  const int h1 = build_node(P, pd, prob, lo, n1, depth + 1, leaf);
  const int h2 = build_node(P, pd, prob, lo + n1, n - n1, depth + 1, leaf);
  const int h = std::max(h1, h2) + 1;
  MergeJob J{};
  J.v_off = pd.vbase + lo;
  J.out_off = pd.qa + lo * pd.lda + lo;
  J.ld_out = pd.lda;
  J.pool_off = pd.pool;
  J.pn = (int32_t)pd.n;
  J.lo = (int32_t)lo;
  J.n1 = (int32_t)n1;
  J.n2 = (int32_t)(n - n1);
  J.prob = prob;
  J.fin = depth == 0 ? 1 : 0;
  J.e_idx = pd.vbase + lo + n1 - 1;
  J.beta = 0.0;
  J.mid = P.nmerges++;
  J.root = depth == 0 ? 1 : 0;
  J.ext = 0;
  if ((int)P.levels.size() < h) P.levels.resize(h);
  P.levels[h - 1].jobs.push_back(J);
  P.maxm = std::max(P.maxm, n);
  return h;
}

static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <class T>
static size_t blob_put(std::vector<unsigned char>& blob, const std::vector<T>& v) {
  size_t off = (blob.size() + 255) & ~size_t(255);
  blob.resize(off + v.size() * sizeof(T));
  if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
  return off;
}

static void finish_plan(Plan& P) {
  for (auto& L : P.levels) {
    const size_t nj = L.jobs.size();
    L.cw8.assign(nj + 1, 0);
    L.crows.assign(nj + 1, 0);
    L.ccols.assign(nj + 1, 0);
    L.ctiles.assign(nj + 1, 0);
    for (size_t j = 0; j < nj; ++j) {
      const MergeJob& J = L.jobs[j];
      const int64_t m = J.n1 + J.n2;
      L.cw8[j + 1] = L.cw8[j] + cdiv(m, 8);
      L.crows[j + 1] = L.crows[j] + cdiv(m, 256) * cdiv(m, 64);
      L.ccols[j + 1] = L.ccols[j] + m;
      // ctiles is device scratch: the product rewrites it from the actual K
    }
  }
  P.blob.clear();
  P.o_leaves = blob_put(P.blob, P.leaves);
  P.o_tlist = blob_put(P.blob, P.tear_list);
  P.o_tptr = blob_put(P.blob, P.tear_ptr);
  P.o_sq = blob_put(P.blob, P.sign_qoff);
  P.o_sn = blob_put(P.blob, P.sign_n);
  P.o_sl = blob_put(P.blob, P.sign_ld);
  P.o_sc = blob_put(P.blob, P.sign_cum);
  P.o_pprobs = blob_put(P.blob, P.pprobs);
  P.o_pmerges = blob_put(P.blob, P.pmerges);
  P.o_pmlev = blob_put(P.blob, P.pmlev);
  for (auto& L : P.levels) {
    L.o_jobs = blob_put(P.blob, L.jobs);
    L.o_cw8 = blob_put(P.blob, L.cw8);
    L.o_crows = blob_put(P.blob, L.crows);
    L.o_ccols = blob_put(P.blob, L.ccols);
    L.o_ctiles = blob_put(P.blob, L.ctiles);
  }
  P.blob.resize((P.blob.size() + 255) & ~size_t(255));
}

static void build_plan(Plan& P, const std::vector<ProblemDesc>& probs, int leaf) {
  P.tear_ptr.push_back(0);
  P.sign_cum.push_back(0);
  std::vector<int64_t> vbase(probs.size()), nvec(probs.size());
  for (size_t p = 0; p < probs.size(); ++p) {
    const ProblemDesc& pd = probs[p];
    if (pd.n > 0) build_node(P, pd, (int)p, 0, pd.n, 0, leaf);
    P.tear_ptr.push_back((int64_t)P.tear_list.size());
    P.sign_qoff.push_back(pd.qa);
    P.sign_n.push_back(pd.n);
    P.sign_ld.push_back(pd.lda);
    P.sign_cum.push_back(P.sign_cum.back() + pd.n);
    vbase[p] = pd.vbase;
    nvec[p] = pd.n;
  }
  persistent_lists(P, (int)probs.size(), vbase, nvec);
  finish_plan(P);
}

// ---------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------
struct Carver {
  unsigned char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
};

struct Layout {
  DevWs w{};
  unsigned* queue = nullptr;  // the persistent kernel's work counter
  double* pool = nullptr;     // the problems' pools: 3 n x n per problem
  unsigned char* plan = nullptr;
  unsigned char* arena = nullptr;
  unsigned char* table = nullptr;
  size_t bytes = 0;
};

static Layout carve(void* ws, int64_t nvec, int64_t qwords, int64_t nmerges, int nprob,
                    size_t plan_bytes, const PathPlan& ps, int64_t nleaf) {
  Carver c{reinterpret_cast<unsigned char*>(ws)};
  Layout L;
  const size_t N = (size_t)std::max<int64_t>(nvec, 1);
  L.pool = c.take<double>(3 * (size_t)qwords);
  DevWs& w = L.w;
  w.ds = c.take<double>(N);
  w.zs = c.take<double>(N);
  w.dbar = c.take<double>(N);
  w.zbar = c.take<double>(N);
  w.dbar32 = c.take<float2>(N);
  w.zbar32 = c.take<float>(N);
  w.zhat = c.take<double>(N);
  w.tau = c.take<double>(N);
  w.taulo = c.take<double>(N);
  w.sinv = c.take<double>(N);
  w.cmax = c.take<double>(N);
  w.lamnd = c.take<double>(N);
  w.dv = c.take<double>(N);
  w.dmod = c.take<double>(N);
  w.rc = c.take<double>(N);
  w.rs = c.take<double>(N);
  w.skey = c.take<double>(2 * N);
  w.srcs = c.take<int32_t>(N);
  w.typ = c.take<int32_t>(N);
  w.flag = c.take<int32_t>(N);
  w.ev = c.take<int32_t>(N);
  w.cand = c.take<int32_t>(N);
  w.slot = c.take<int32_t>(N);
  w.kidx = c.take<int32_t>(N);
  w.kperm = c.take<int32_t>(N);
  w.org = c.take<int32_t>(N);
  w.dsrc = c.take<int32_t>(N);
  w.dperm = c.take<int32_t>(N);
  w.posK = c.take<int32_t>(N);
  w.posD = c.take<int32_t>(N);
  w.rj = c.take<int32_t>(N);
  w.rk = c.take<int32_t>(N);
  w.chain = c.take<int32_t>(N);
  w.sval = c.take<int32_t>(2 * N);
  w.colptr = c.take<const double*>(N);
  w.dcolptr = c.take<const double*>(N);
  w.klo = c.take<int32_t>(N);
  w.khi = c.take<int32_t>(N);
  w.dlo = c.take<int32_t>(N);
  w.dhi = c.take<int32_t>(N);
  w.outptr = c.take<double*>(N);
  w.wptr = c.take<double*>(N);
  w.tptr = c.take<const double*>(N);
  w.tlo = c.take<int32_t>(N);
  w.thi = c.take<int32_t>(N);
  w.scal = c.take<MergeScalars>((size_t)std::max<int64_t>(nmerges, 1));
  w.lroots = c.take<unsigned long long>(2 * kMaxLevels);
  const size_t NL = (size_t)std::max<int64_t>(nleaf, 1);
  w.lrot = c.take<double2>(NL * kLeafRot);
  w.lroti = c.take<uint8_t>(NL * kLeafRot);
  w.lrotn = c.take<int32_t>(NL);
  w.status = c.take<int>((size_t)std::max(nprob, 1));
  L.queue = c.take<unsigned>(64);
  L.plan = c.take<unsigned char>(plan_bytes);
  L.table = c.take<unsigned char>(ps.table_bytes);
  L.arena = c.take<unsigned char>(ps.arena_bytes);
  L.bytes = c.off;
  return L;
}

static tdc_opts resolve_opts(const tdc_opts* o) {
  tdc_opts r;
  tdc_default_opts(&r);
  if (o) r = *o;
  return r;
}

static bool opts_valid(const tdc_opts& o) {
  return o.path >= TDC_PATH_DENSE_FP64 && o.path <= TDC_PATH_AUTO && o.leaf >= 1 && o.leaf <= 32 &&
         o.max_secular_iter >= 1 && o.ozaki_slices >= 5 && o.ozaki_slices <= 7 && o.hss_leaf >= 16 &&
         o.hss_rp >= 8 && o.hss_tol > 0.0 &&
         (o.secular_lanes == 0 || o.secular_lanes == 1 || o.secular_lanes == 2 || o.secular_lanes == 4 ||
          o.secular_lanes == 8 || o.secular_lanes == 16 || o.secular_lanes == 32) &&
         (o.eigvec == TDC_EIGVEC_LOWNER || o.eigvec == TDC_EIGVEC_EXTENDED) && o.hss_grow >= 0 &&
         o.hss_grow <= 4;
}

template <class T>
static const T* P_(const Layout& L, size_t off) {
  return reinterpret_cast<const T*>(L.plan + off);
}
template <class T>
static T* PM_(const Layout& L, size_t off) {        // device scratch inside the plan region
  return reinterpret_cast<T*>(L.plan + off);
}

// Launch the whole level sequence of a plan whose blob is already on the device.
static std::vector<const std::vector<MergeJob>*> level_jobs(const Plan& P) {
  std::vector<const std::vector<MergeJob>*> v;
  for (const LevelPlan& lv : P.levels) v.push_back(&lv.jobs);
  return v;
}

// A second stream and two events per host thread and device, for running the top
// merges' deflated-column copy beside their Loewner, norm and product kernels (created on
// first use; never released while the thread lives).
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
static SideStream* side_stream() {
  static thread_local SideStream r[16];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return nullptr;
  SideStream& x = r[dev];
  if (!x.s) {
    if (cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking) != cudaSuccess) {
      x.s = nullptr;
      return nullptr;
    }
    if (cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming) != cudaSuccess) {
      cudaStreamDestroy(x.s);
      x.s = nullptr;
      return nullptr;
    }
  }
  return &x;
}

static bool phases_profiled();   // per-phase event timing on (the phases then run one after another)

static int run_plan(const Plan& P, const PathPlan& pp, const Layout& L_in, const tdc_opts& o,
                    const double* d, const double* e, double* lam, QBufs qb, int64_t nvec, int nprob,
                    bool sign_norm, double* qa_for_sign, cudaStream_t st, bool overlap = true) {
  if (phases_profiled()) overlap = false;
  Layout L = L_in;
  L.w.ext = o.eigvec == TDC_EIGVEC_EXTENDED ? 1 : 0;
  // leaves of one element and n < 2^31 give at most 31 merge levels
  static_assert(kMaxLevels >= 32, "level table too small");
  cudaMemsetAsync(L.w.lroots, 0, 2 * kMaxLevels * sizeof(unsigned long long), st);
  cudaMemsetAsync(L.w.scal, 0, std::max<int64_t>(P.nmerges, 1) * sizeof(MergeScalars), st);
  phase_mark(0, true, 0, st);
  launch_tear(P_<int64_t>(L, P.o_tlist), P_<int64_t>(L, P.o_tptr), nprob, (int64_t)P.tear_list.size(),
              o.leaf, d, e, L.w.dmod, nvec, st);
  launch_leaves(P_<LeafJob>(L, P.o_leaves), (int)P.leaves.size(), L.w.dmod, e, lam, qb, L.w, st);
  phase_mark(0, false, 4, st);
  for (size_t li = 0; li < P.levels.size(); ++li) {
    const LevelPlan& lv = P.levels[li];
    const int nj = (int)lv.jobs.size();
    if (nj == 0) continue;
    const MergeJob* jobs = P_<MergeJob>(L, lv.o_jobs);
    bool any_root = false, any_fin = false;
    int64_t maxm = 0;
    for (const MergeJob& J : lv.jobs) {
      any_root |= J.root != 0;
      any_fin |= J.fin != 0;
      maxm = std::max<int64_t>(maxm, J.n1 + J.n2);
    }
    // Deflated columns move only in a problem's top merge (below, the slot table keeps
    // them in place).  Their copy needs the placement only, and touches none of the
    // columns the Loewner, norm and product kernels read or write, so it runs beside
    // them on a side stream (HBM-bound beside FP64- or tensor-bound work); the sign
    // convention waits for both.
    SideStream* side = (any_fin && overlap) ? side_stream() : nullptr;
    launch_merge_level((int)li, jobs, nj, P_<int64_t>(L, lv.o_cw8), lv.cw8.back(), P_<int64_t>(L, lv.o_crows),
                       lv.crows.back(), P_<int64_t>(L, lv.o_ccols), lv.ccols.back(), lam, e, qb, L.w,
                       o.max_secular_iter, o.secular_lanes, merge_cta_threads(maxm), st,
                       side ? side->fork : nullptr);
    if (side) {
      cudaStreamWaitEvent(side->s, side->fork, 0);
      launch_defl_copy_cols(jobs, nj, P_<int64_t>(L, lv.o_cw8), lv.cw8.back(), P_<int64_t>(L, lv.o_ccols),
                            lv.ccols.back(), maxm, qb, L.w, side->s);
      cudaEventRecord(side->join, side->s);
    }
    const int prc = launch_product(pp, (int)li, o, lv.jobs, jobs, PM_<int64_t>(L, lv.o_ctiles), qb, L.w, st);
    if (side) cudaStreamWaitEvent(st, side->join, 0);
    if (prc) return prc;
    if (any_fin) {
      if (!side)
        launch_defl_copy_cols(jobs, nj, P_<int64_t>(L, lv.o_cw8), lv.cw8.back(), P_<int64_t>(L, lv.o_ccols),
                              lv.ccols.back(), maxm, qb, L.w, st);
      launch_sign(jobs, nj, P_<int64_t>(L, lv.o_cw8), lv.cw8.back(), P_<int64_t>(L, lv.o_ccols), lv.ccols.back(),
                  maxm, qb, L.w, sign_norm && any_root, st);
    }
  }
  (void)qa_for_sign;
  return 0;
}

// ---------------------------------------------------------------------------
// Autotuning of the FP64 product tile shape per tree level: the whole plan runs
// once per shape (every FP64-product level on that shape), each level's product is
// timed with CUDA events, best of two rounds, and the fastest shape per level is
// kept in the plan and recorded for plans of the same level structure.  All shapes
// give bit-identical results, so tuning changes speed only.
// ---------------------------------------------------------------------------
static int autotune_plan(const Plan& P, PathPlan& pp, const Layout& L, const tdc_opts& o, const double* d,
                         const double* e, double* lam, QBufs qb, int64_t nvec, int nprob, cudaStream_t st,
                         std::vector<int>& best) {
  const int nl = (int)P.levels.size();
  LevelTimer T;
  T.a.assign(nl, nullptr);
  T.b.assign(nl, nullptr);
  T.used.assign(nl, false);
  for (int l = 0; l < nl; ++l) {
    cudaEventCreate(&T.a[l]);
    cudaEventCreate(&T.b[l]);
  }
  std::vector<std::vector<float>> t(kGemmShapes, std::vector<float>(nl, 3.0e38f));
  std::vector<int> keep(nl);
  for (int l = 0; l < nl; ++l) keep[l] = pp.levels[l].gemm_cfg;
  std::vector<bool> timed(nl, false);
  int rc = 0;
  for (int rep = 0; rep < 2 && rc == 0; ++rep) {
    for (int c = 0; c < kGemmShapes && rc == 0; ++c) {
      for (int l = 0; l < nl; ++l) path_set_shape(pp, l, c, P.levels[l].jobs);
      std::fill(T.used.begin(), T.used.end(), false);
      cudaMemsetAsync(L.w.status, 0, sizeof(int) * std::max(nprob, 1), st);
      set_level_timer(&T);
      rc = run_plan(P, pp, L, o, d, e, lam, qb, nvec, nprob, true, nullptr, st);
      set_level_timer(nullptr);
      if (rc == 0 && cudaStreamSynchronize(st) != cudaSuccess) rc = 4;
      if (rc) break;
      for (int l = 0; l < nl; ++l) {
        if (!T.used[l]) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, T.a[l], T.b[l]) == cudaSuccess) t[c][l] = std::min(t[c][l], ms);
        timed[l] = true;
      }
    }
  }
  best.assign(nl, 0);
  for (int l = 0; l < nl; ++l) {
    int b = keep[l];
    if (timed[l]) {
      b = 0;
      for (int c = 1; c < kGemmShapes; ++c)
        if (t[c][l] < t[b][l]) b = c;
    }
    best[l] = b;
    path_set_shape(pp, l, b, P.levels[l].jobs);
  }
  for (int l = 0; l < nl; ++l) {
    cudaEventDestroy(T.a[l]);
    cudaEventDestroy(T.b[l]);
  }
  if (rc == 0) tune_store(tune_key(o, level_jobs(P)), best);
  return rc;
}

static void copy_shapes(const std::vector<int>& best, int32_t* out, int32_t max_levels, int32_t* n_out) {
  if (n_out) *n_out = (int32_t)best.size();
  if (!out) return;
  for (int l = 0; l < (int)best.size() && l < max_levels; ++l) out[l] = best[l];
}

// ---------------------------------------------------------------------------
// Per-phase profiling (tdc_profile_begin / tdc_profile_end)
// ---------------------------------------------------------------------------
struct ProfRec {
  int ph;
  cudaEvent_t a, b;
};
struct ProfState {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<ProfRec> recs;
  // open event per phase (the HSS phases nest inside phase 5), then per tree level of
  // the FP64 product (phase ids kLevelMark + level)
  cudaEvent_t open_ev[TDC_NPHASE + TDC_PROFILE_LEVELS] = {};
  int64_t launches[TDC_NPHASE] = {};
  double flops = 0.0, bytes = 0.0, fp64_flops = 0.0, split_flops = 0.0, tensor_flops = 0.0, copy_bytes = 0.0;
  double secular_flops = 0.0;
  int64_t secular_evals = 0;
  int64_t merges = 0, ktot = 0, calls = 0, hss_fallbacks = 0, hss_regrowths = 0;
  double hss_sampling_flops = 0.0, sg_tensor_flops = 0.0;
  cudaEvent_t sg_open = nullptr;
  double lvl_bytes[TDC_PROFILE_LEVELS] = {}, lvl_flops[TDC_PROFILE_LEVELS] = {};
  MergeScalars* hscal = nullptr;
  size_t hscal_n = 0;
};
static ProfState g_prof;

// Calls that must not create events (the allocation-free entry) suspend the per-phase
// marks on their thread for their duration.
static thread_local bool t_prof_suspended = false;
ProfileSuspend::ProfileSuspend(bool on) : prev_(t_prof_suspended) { t_prof_suspended = prev_ || on; }
static bool phases_profiled() { return g_prof.on && !t_prof_suspended; }
ProfileSuspend::~ProfileSuspend() { t_prof_suspended = prev_; }


void hss_fallbacks_add(int n) {
  if (g_prof.on && !t_prof_suspended) g_prof.hss_fallbacks += n;
}
void hss_regrowths_add(int n) {
  if (g_prof.on && !t_prof_suspended) g_prof.hss_regrowths += n;
}
void hss_sampling_flops_add(double f) {
  if (g_prof.on && !t_prof_suspended) g_prof.hss_sampling_flops += f;
}

static cudaEvent_t prof_event() {
  if (g_prof.used == g_prof.pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    g_prof.pool.push_back(e);
  }
  return g_prof.pool[g_prof.used++];
}

void phase_mark(int phase, bool begin, int nlaunch, cudaStream_t st) {
  if (!g_prof.on || t_prof_suspended) return;
  int slot = phase;
  if (phase >= kLevelMark && phase < kLevelMark + TDC_PROFILE_LEVELS) slot = TDC_NPHASE + (phase - kLevelMark);
  else if (phase < 0 || phase >= TDC_NPHASE) return;
  if (begin) {
    g_prof.open_ev[slot] = prof_event();
    cudaEventRecord(g_prof.open_ev[slot], st);
  } else if (g_prof.open_ev[slot]) {
    cudaEvent_t b = prof_event();
    cudaEventRecord(b, st);
    g_prof.recs.push_back(ProfRec{phase, g_prof.open_ev[slot], b});
    g_prof.open_ev[slot] = nullptr;
    if (phase < TDC_NPHASE) g_prof.launches[phase] += nlaunch;
  }
}

constexpr int kSgMark = 200;   // ProfRec id of the split GEMM kernel's launches
void sg_gemm_mark(bool begin, double tensor_flops, cudaStream_t st) {
  if (!g_prof.on || t_prof_suspended) return;
  if (begin) {
    g_prof.sg_open = prof_event();
    cudaEventRecord(g_prof.sg_open, st);
    g_prof.sg_tensor_flops += tensor_flops;
  } else if (g_prof.sg_open) {
    cudaEvent_t b = prof_event();
    cudaEventRecord(b, st);
    g_prof.recs.push_back(ProfRec{kSgMark, g_prof.sg_open, b});
    g_prof.sg_open = nullptr;
  }
}

// After a profiled solve: read the per-merge counts and add up the product's work.
static void prof_account(const Plan& P, const PathPlan& pp, const MergeScalars* dscal, cudaStream_t st) {
  if (!g_prof.on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;   // no sync
  const size_t nm = (size_t)std::max<int64_t>(P.nmerges, 1);
  if (g_prof.hscal_n < nm) {
    if (g_prof.hscal) cudaFreeHost(g_prof.hscal);
    cudaMallocHost(&g_prof.hscal, nm * sizeof(MergeScalars));
    g_prof.hscal_n = nm;
  }
  cudaMemcpyAsync(g_prof.hscal, dscal, nm * sizeof(MergeScalars), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  const double pairs = oz_slice_pairs(pp.slices);
  for (size_t l = 0; l < P.levels.size(); ++l) {
    const bool oz = l < pp.levels.size() && pp.levels[l].oz;
    const bool hss = l < pp.levels.size() && pp.levels[l].hss;
    for (const MergeJob& J : P.levels[l].jobs) {
      const MergeScalars& S = g_prof.hscal[J.mid];
      const double K = S.K, c1 = S.c1, c3 = S.c3, c2 = S.K - S.c1 - S.c3;
      const double m = (double)J.n1 + J.n2;
      const double f = 2.0 * K * (J.n1 * (c1 + c3) + J.n2 * (c3 + c2));
      g_prof.flops += f;
      if (oz) {
        g_prof.split_flops += f;
        g_prof.tensor_flops += pairs * f;
      } else if (!hss) {
        g_prof.fp64_flops += f;
        if (l < TDC_PROFILE_LEVELS) {
          g_prof.lvl_flops[l] += f;
          g_prof.lvl_bytes[l] += 8.0 * (J.n1 * (c1 + c3) + J.n2 * (c3 + c2) + m * K);
        }
      }
      g_prof.bytes += 8.0 * (J.n1 * (c1 + c3) + J.n2 * (c3 + c2) + m * K);
      if (J.fin) g_prof.copy_bytes += 8.0 * m * (m - K) + 8.0 * (double)S.live;   // columns written, live rows read
      g_prof.secular_flops += 10.0 * K * (double)S.evals;     // K terms per evaluation: 1 division, 4 FMA, 1 mul
      g_prof.secular_evals += (int64_t)S.evals;
      g_prof.merges += 1;
      g_prof.ktot += S.K;
    }
  }
  g_prof.calls += 1;
}

static int launch_status() {
  const cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? 0 : 4;
}

// single-problem plan helper
static void single_problem_plan(Plan& P, int64_t n, int64_t ldq, int leaf) {
  ProblemDesc pd{};
  pd.n = n;
  pd.vbase = 0;
  pd.qa = 0;
  pd.lda = ldq;
  pd.pool = 0;
  build_plan(P, {pd}, leaf);
}

static size_t syev_bytes(int64_t n, const tdc_opts& o, const Plan& P) {
  PathPlan pp;
  path_prepare(pp, o, level_jobs(P));
  Layout L = carve(nullptr, n, n * n, P.nmerges, 1, P.blob.size(), pp, (int64_t)P.leaves.size());
  return L.bytes;
}

int syev_core(int64_t n, const double* d, const double* e, double* lambda, double* Q, int64_t ldq,
              const tdc_opts* opts, void* ws, size_t ws_bytes, int* dev_status, void* stream,
              bool profile_accounting) {
  if (n < 1) return -1;
  if (!d) return -2;
  if (!e && n > 1) return -3;
  if (!lambda) return -4;
  if (!Q) return -5;
  if (ldq < n) return -6;
  const tdc_opts o = resolve_opts(opts);
  if (!opts_valid(o) || !path_supported(o)) return -7;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return -8;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const ProfileSuspend no_events(!profile_accounting);   // no per-phase events either
  Plan P;
  single_problem_plan(P, n, ldq, o.leaf);
  PathPlan pp;
  const auto lj = level_jobs(P);
  path_prepare(pp, o, lj);
  Layout L = carve(ws, n, n * n, P.nmerges, 1, P.blob.size(), pp, (int64_t)P.leaves.size());
  if (L.bytes > ws_bytes) return 3;
  if (dev_status) L.w.status = dev_status;
  cudaMemsetAsync(L.w.status, 0, sizeof(int), st);
  cudaMemcpyAsync(L.plan, P.blob.data(), P.blob.size(), cudaMemcpyHostToDevice, st);
  if (!path_bind(pp, L.arena, L.table, lj, st)) return 4;
  QBufs qb{Q, L.pool, nullptr};
  const int prc = run_plan(P, pp, L, o, d, e ? e : d, lambda, qb, n, 1, true, Q, st, profile_accounting);
  if (prc) return prc;
  if (profile_accounting) prof_account(P, pp, L.w.scal, st);
  return launch_status();
}

// Intermediate values of one merge (tdc_merge_inspect): the per-merge counts from the
// merge scalars and the type-1 flags, and copies of the per-index arrays, all read
// from the workspace after the merge's kernels (in stream order).
__global__ void k_trace_counts(const MergeScalars* __restrict__ scal, const int32_t* __restrict__ flag,
                               int m, int64_t* __restrict__ out) {
  __shared__ int s_t1;
  if (threadIdx.x == 0) s_t1 = 0;
  __syncthreads();
  int c = 0;
  for (int p = threadIdx.x; p < m; p += blockDim.x) c += (flag[p] & F_T1) != 0;
  atomicAdd(&s_t1, c);
  __syncthreads();
  if (threadIdx.x == 0) {
    const MergeScalars S = scal[0];
    out[0] = S.K;
    out[1] = S.nd;
    out[2] = S.nrot;
    out[3] = S.c1;
    out[4] = S.c3;
    out[5] = s_t1;
    out[6] = 0;
    out[7] = 0;
  }
}

template <class T>
static void trace_copy(T* dst, const T* src, int64_t n, cudaStream_t st) {
  if (dst) cudaMemcpyAsync(dst, src, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, st);
}

static void copy_trace(const tdc_merge_trace& t, const DevWs& w, int64_t n, cudaStream_t st) {
  if (t.counts) k_trace_counts<<<1, 256, 0, st>>>(w.scal, w.flag, (int)n, t.counts);
  trace_copy(t.perm, w.srcs, n, st);
  trace_copy(t.d_sorted, w.ds, n, st);
  trace_copy(t.z_sorted, w.zs, n, st);
  trace_copy(t.kept, w.kidx, n, st);
  trace_copy(t.deflated, w.dsrc, n, st);
  trace_copy(t.rot_j, w.rj, n, st);
  trace_copy(t.rot_k, w.rk, n, st);
  trace_copy(t.rot_c, w.rc, n, st);
  trace_copy(t.rot_s, w.rs, n, st);
  trace_copy(t.dbar, w.dbar, n, st);
  trace_copy(t.zbar, w.zbar, n, st);
  trace_copy(t.origin, w.org, n, st);
  trace_copy(t.tau, w.tau, n, st);
  trace_copy(t.zhat, w.zhat, n, st);
  trace_copy(t.sinv, w.sinv, n, st);
  if (w.ext) trace_copy(t.tau_lo, w.taulo, n, st);
}

}  // namespace tdc

static_assert(sizeof(tdc_opts) == 56, "tdc_opts layout is part of the ABI");

using namespace tdc;

extern "C" {

void tdc_default_opts(tdc_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->path = TDC_PATH_DENSE_FP64;
  o->leaf = 32;
  o->hss_tol = 1e-12;
  o->hss_leaf = 512;
  o->hss_rp = 128;
  o->k_threshold = 8192;
  o->ozaki_slices = 6;
  o->max_secular_iter = 64;
  o->tile_cfg = -1;
  o->hss_grow = 1;
}

const char* tdc_version(void) { return "tdc 0.2 (sm_103a)"; }

size_t tdc_struct_bytes(int which) {
  switch (which) {
    case 0: return sizeof(tdc_opts);
    case 1: return sizeof(tdc_profile);
    case 2: return sizeof(tdc_merge_trace);
    default: return 0;
  }
}

size_t tdc_workspace_bytes(int64_t n, const tdc_opts* opts) {
  const tdc_opts o = resolve_opts(opts);
  if (n < 1 || !opts_valid(o)) return 0;
  Plan P;
  single_problem_plan(P, n, n, o.leaf);
  return syev_bytes(n, o, P);
}

int tdc_syev_tridiag(int64_t n, const double* d, const double* e, double* lambda, double* Q,
                     int64_t ldq, const tdc_opts* opts, void* ws, size_t ws_bytes, int* dev_status,
                     void* stream) {
  return tdc::syev_core(n, d, e, lambda, Q, ldq, opts, ws, ws_bytes, dev_status, stream, true);
}

int tdc_autotune(int64_t n, const double* d, const double* e, double* lambda, double* Q, int64_t ldq,
                 const tdc_opts* opts, void* ws, size_t ws_bytes, int32_t* shape_per_level,
                 int32_t max_levels, int32_t* n_levels, int* dev_status, void* stream) {
  if (n < 1) return -1;
  if (!d) return -2;
  if (!e && n > 1) return -3;
  if (!lambda) return -4;
  if (!Q) return -5;
  if (ldq < n) return -6;
  const tdc_opts o = resolve_opts(opts);
  if (!opts_valid(o) || !path_supported(o)) return -7;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return -8;
  if (shape_per_level && max_levels < 0) return -11;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Plan P;
  single_problem_plan(P, n, ldq, o.leaf);
  PathPlan pp;
  const auto lj = level_jobs(P);
  path_prepare(pp, o, lj);
  Layout L = carve(ws, n, n * n, P.nmerges, 1, P.blob.size(), pp, (int64_t)P.leaves.size());
  if (L.bytes > ws_bytes) return 3;
  if (dev_status) L.w.status = dev_status;
  cudaMemcpyAsync(L.plan, P.blob.data(), P.blob.size(), cudaMemcpyHostToDevice, st);
  if (!path_bind(pp, L.arena, L.table, lj, st)) return 4;
  QBufs qb{Q, L.pool, nullptr};
  std::vector<int> best;
  const int rc = autotune_plan(P, pp, L, o, d, e ? e : d, lambda, qb, n, 1, st, best);
  if (rc) return rc;
  copy_shapes(best, shape_per_level, max_levels, n_levels);
  return launch_status();
}

size_t tdc_host_buffer_bytes(int64_t n, const tdc_opts* opts) {
  const size_t ws = tdc_workspace_bytes(n, opts);
  if (ws == 0) return 0;
  const size_t vec = ((size_t)n * 8 + 255) & ~size_t(255);
  const size_t mat = ((size_t)n * n * 8 + 255) & ~size_t(255);
  return ws + 3 * vec + mat + 256;
}

// Checks the host entry's arguments and enqueues copy-in, solve and copy-out on the
// stream; the status word goes to *status_dst.  Returns 0 or the argument / launch code.
static int host_enqueue(int64_t n, const double* d_host, const double* e_host, double* lambda_host,
                        double* Q_host, int64_t ldq, const tdc_opts* opts, void* dev_buf, size_t dev_buf_bytes,
                        int* status_dst, void* stream) {
  if (n < 1) return -1;
  if (!d_host) return -2;
  if (!e_host && n > 1) return -3;
  if (!lambda_host) return -4;
  if (!Q_host) return -5;
  if (ldq < n) return -6;
  const size_t need = tdc_host_buffer_bytes(n, opts);
  if (need == 0) return -7;
  if (!dev_buf || (reinterpret_cast<uintptr_t>(dev_buf) & 255)) return -8;
  if (dev_buf_bytes < need) return 3;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* b = reinterpret_cast<unsigned char*>(dev_buf);
  const size_t vec = ((size_t)n * 8 + 255) & ~size_t(255);
  const size_t mat = ((size_t)n * n * 8 + 255) & ~size_t(255);
  double* dd = reinterpret_cast<double*>(b);
  double* de = reinterpret_cast<double*>(b + vec);
  double* dl = reinterpret_cast<double*>(b + 2 * vec);
  double* dq = reinterpret_cast<double*>(b + 3 * vec);
  int* dstat = reinterpret_cast<int*>(b + 3 * vec + mat);
  void* ws = b + 3 * vec + mat + 256;
  cudaMemcpyAsync(dd, d_host, n * 8, cudaMemcpyHostToDevice, st);
  if (n > 1) cudaMemcpyAsync(de, e_host, (n - 1) * 8, cudaMemcpyHostToDevice, st);
  const int rc = tdc_syev_tridiag(n, dd, de, dl, dq, n, opts, ws, dev_buf_bytes - (3 * vec + mat + 256),
                                  dstat, stream);
  if (rc != 0) return rc;
  cudaMemcpyAsync(lambda_host, dl, n * 8, cudaMemcpyDeviceToHost, st);
  cudaMemcpy2DAsync(Q_host, ldq * 8, dq, n * 8, n * 8, n, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(status_dst, dstat, sizeof(int), cudaMemcpyDeviceToHost, st);
  return launch_status();
}

int tdc_syev_tridiag_host(int64_t n, const double* d_host, const double* e_host, double* lambda_host,
                          double* Q_host, int64_t ldq, const tdc_opts* opts, void* dev_buf,
                          size_t dev_buf_bytes, void* stream) {
  int hs = 0;
  const int rc = host_enqueue(n, d_host, e_host, lambda_host, Q_host, ldq, opts, dev_buf, dev_buf_bytes, &hs,
                              stream);
  if (rc != 0) return rc;
  if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return 4;
  return hs;
}

int tdc_syev_tridiag_host_async(int64_t n, const double* d_host, const double* e_host, double* lambda_host,
                                double* Q_host, int64_t ldq, const tdc_opts* opts, void* dev_buf,
                                size_t dev_buf_bytes, int* status_host, void* stream) {
  if (!status_host) return -10;
  return host_enqueue(n, d_host, e_host, lambda_host, Q_host, ldq, opts, dev_buf, dev_buf_bytes, status_host,
                      stream);
}

size_t tdc_merge_workspace_bytes(int64_t n, const tdc_opts* opts) {
  const tdc_opts o = resolve_opts(opts);
  if (n < 2 || !opts_valid(o)) return 0;
  Plan P;
  P.levels.resize(1);
  P.levels[0].jobs.resize(1);
  P.nmerges = 1;
  P.maxm = n;
  P.tear_ptr = {0, 0};
  P.levels[0].jobs[0].n1 = (int32_t)(n / 2);
  P.levels[0].jobs[0].n2 = (int32_t)(n - n / 2);
  finish_plan(P);
  PathPlan pp;
  path_prepare(pp, o, level_jobs(P));
  Layout L = carve(nullptr, n, n * n, 1, 1, P.blob.size(), pp, 0);
  return L.bytes;
}

static int merge_core(int64_t n1, int64_t n2, const double* D, const double* Q, int64_t ldq, double beta,
                      double* lambda, double* Q_out, int64_t ldqo, int64_t* K_out, const tdc_opts* opts,
                      void* ws, size_t ws_bytes, int* dev_status, void* stream, const tdc_merge_trace* tr) {
  if (n1 < 1) return -1;
  if (n2 < 1) return -2;
  if (!D) return -3;
  if (!Q) return -4;
  const int64_t n = n1 + n2;
  if (ldq < n) return -5;
  if (!lambda) return -7;
  if (!Q_out) return -8;
  if (ldqo < n) return -9;
  const tdc_opts o = resolve_opts(opts);
  if (!opts_valid(o) || !path_supported(o)) return -11;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return -12;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Plan P;
  P.levels.resize(1);
  MergeJob J{};
  J.v_off = 0;
  J.out_off = 0;
  J.ld_out = ldqo;
  J.pool_off = 0;
  J.pn = (int32_t)n;
  J.lo = 0;
  J.in_off = 0;
  J.ld_in = ldq;
  J.ext = 1;                     // inputs: the caller's Q
  J.fin = 1;                     // outputs: the caller's Q_out in sorted order, no sign convention
  J.root = 0;
  J.n1 = (int32_t)n1;
  J.n2 = (int32_t)n2;
  J.prob = 0;
  J.beta = beta;
  J.e_idx = -1;
  J.mid = 0;
  P.levels[0].jobs.push_back(J);
  P.nmerges = 1;
  P.maxm = n;
  P.tear_ptr = {0, 0};
  finish_plan(P);
  PathPlan pp;
  const auto lj = level_jobs(P);
  path_prepare(pp, o, lj);
  Layout L = carve(ws, n, n * n, 1, 1, P.blob.size(), pp, 0);
  if (L.bytes > ws_bytes) return 3;
  if (dev_status) L.w.status = dev_status;
  cudaMemsetAsync(L.w.status, 0, sizeof(int), st);
  cudaMemcpyAsync(L.plan, P.blob.data(), P.blob.size(), cudaMemcpyHostToDevice, st);
  if (!path_bind(pp, L.arena, L.table, lj, st)) return 4;
  cudaMemcpyAsync(lambda, D, n * 8, cudaMemcpyDeviceToDevice, st);
  QBufs qb{Q_out, L.pool, Q};
  L.w.ext = o.eigvec == TDC_EIGVEC_EXTENDED ? 1 : 0;
  const LevelPlan& lv = P.levels[0];
  const MergeJob* jobs = P_<MergeJob>(L, lv.o_jobs);
  cudaMemsetAsync(L.w.lroots, 0, 2 * kMaxLevels * sizeof(unsigned long long), st);
  cudaMemsetAsync(L.w.scal, 0, sizeof(MergeScalars), st);
  launch_merge_level(0, jobs, 1, P_<int64_t>(L, lv.o_cw8), lv.cw8.back(), P_<int64_t>(L, lv.o_crows),
                     lv.crows.back(), P_<int64_t>(L, lv.o_ccols), lv.ccols.back(), lambda, nullptr,
                     qb, L.w, o.max_secular_iter, o.secular_lanes, merge_cta_threads(n), st);
  const int prc = launch_product(pp, 0, o, lv.jobs, jobs, PM_<int64_t>(L, lv.o_ctiles), qb, L.w, st);
  if (prc) return prc;
  launch_defl_copy(jobs, 1, P_<int64_t>(L, lv.o_cw8), lv.cw8.back(), P_<int64_t>(L, lv.o_ccols),
                   lv.ccols.back(), n, qb, L.w, false, st);
  if (K_out) launch_copy_k(L.w.scal, K_out, st);
  if (tr) copy_trace(*tr, L.w, n, st);       // L.w.ext set above
  prof_account(P, pp, L.w.scal, st);
  return launch_status();
}

int tdc_merge(int64_t n1, int64_t n2, const double* D, const double* Q, int64_t ldq, double beta,
              double* lambda, double* Q_out, int64_t ldqo, int64_t* K_out, const tdc_opts* opts,
              void* ws, size_t ws_bytes, int* dev_status, void* stream) {
  return merge_core(n1, n2, D, Q, ldq, beta, lambda, Q_out, ldqo, K_out, opts, ws, ws_bytes, dev_status,
                    stream, nullptr);
}

int tdc_merge_inspect(int64_t n1, int64_t n2, const double* D, const double* Q, int64_t ldq, double beta,
                      double* lambda, double* Q_out, int64_t ldqo, int64_t* K_out, const tdc_opts* opts,
                      void* ws, size_t ws_bytes, int* dev_status, void* stream, const tdc_merge_trace* trace) {
  if (!trace) return -16;
  return merge_core(n1, n2, D, Q, ldq, beta, lambda, Q_out, ldqo, K_out, opts, ws, ws_bytes, dev_status,
                    stream, trace);
}

size_t tdc_batched_workspace_bytes(int32_t batch, const int64_t* n_host, const tdc_opts* opts) {
  const tdc_opts o = resolve_opts(opts);
  if (batch < 1 || !n_host || !opts_valid(o)) return 0;
  std::vector<ProblemDesc> probs(batch);
  int64_t vtot = 0, qtot = 0, maxn = 0;
  for (int p = 0; p < batch; ++p) {
    const int64_t n = n_host[p];
    if (n < 1) return 0;
    probs[p] = ProblemDesc{n, vtot, qtot, n, 3 * qtot};
    vtot += n;
    qtot += n * n;
    maxn = std::max(maxn, n);
  }
  Plan P;
  build_plan(P, probs, o.leaf);
  PathPlan pp;
  path_prepare(pp, o, level_jobs(P));
  Layout L = carve(nullptr, vtot, qtot, P.nmerges, batch, P.blob.size(), pp, (int64_t)P.leaves.size());
  return L.bytes;
}

int tdc_syev_tridiag_batched(int32_t batch, const int64_t* n_host, const int64_t* off_de,
                             const int64_t* off_q, const double* d_cat, const double* e_cat,
                             double* lambda_cat, double* Q_cat, const tdc_opts* opts, void* ws,
                             size_t ws_bytes, int* dev_status_per_problem, void* stream) {
  if (batch < 1) return -1;
  if (!n_host) return -2;
  if (!off_de) return -3;
  if (!off_q) return -4;
  if (!d_cat) return -5;
  if (!e_cat) return -6;
  if (!lambda_cat) return -7;
  if (!Q_cat) return -8;
  const tdc_opts o = resolve_opts(opts);
  if (!opts_valid(o) || !path_supported(o)) return -9;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return -10;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // Internal vectors and the B / side buffers use a dense packing; the caller's
  // offsets address d, e, lambda and Q only.  Map: problem p's internal vector base
  // is its packed offset; the kernels index d/e/lambda by v_off, so the packed and
  // caller offsets must coincide -> require off_de to be the dense packing.
  std::vector<ProblemDesc> probs(batch);
  int64_t vtot = 0, qtot = 0, maxn = 0;
  for (int p = 0; p < batch; ++p) {
    const int64_t n = n_host[p];
    if (n < 1) return -2;
    if (off_de[p] != vtot) return -3;
    if (off_q[p] < 0) return -4;
    probs[p] = ProblemDesc{n, vtot, off_q[p], n, 3 * qtot};
    vtot += n;
    qtot += n * n;
    maxn = std::max(maxn, n);
  }
  Plan P;
  build_plan(P, probs, o.leaf);
  PathPlan pp;
  const auto lj = level_jobs(P);
  path_prepare(pp, o, lj);
  Layout L = carve(ws, vtot, qtot, P.nmerges, batch, P.blob.size(), pp, (int64_t)P.leaves.size());
  if (L.bytes > ws_bytes) return 3;
  if (dev_status_per_problem) L.w.status = dev_status_per_problem;
  cudaMemsetAsync(L.w.status, 0, sizeof(int) * batch, st);
  cudaMemcpyAsync(L.plan, P.blob.data(), P.blob.size(), cudaMemcpyHostToDevice, st);
  if (!path_bind(pp, L.arena, L.table, lj, st)) return 4;
  QBufs qb{Q_cat, L.pool, nullptr};
  const int prc = run_plan(P, pp, L, o, d_cat, e_cat, lambda_cat, qb, vtot, batch, true, Q_cat, st);
  if (prc) return prc;
  prof_account(P, pp, L.w.scal, st);
  return launch_status();
}

void tdc_profile_begin(void) {
  g_prof.on = true;
  g_prof.used = 0;
  g_prof.recs.clear();
  for (int i = 0; i < TDC_NPHASE; ++i) g_prof.launches[i] = 0;
  g_prof.flops = g_prof.bytes = g_prof.fp64_flops = g_prof.split_flops = g_prof.tensor_flops = 0.0;
  g_prof.copy_bytes = g_prof.secular_flops = 0.0;
  g_prof.secular_evals = 0;
  g_prof.merges = g_prof.ktot = g_prof.calls = g_prof.hss_fallbacks = g_prof.hss_regrowths = 0;
  g_prof.hss_sampling_flops = g_prof.sg_tensor_flops = 0.0;
  g_prof.sg_open = nullptr;
  for (int i = 0; i < TDC_NPHASE + TDC_PROFILE_LEVELS; ++i) g_prof.open_ev[i] = nullptr;
  for (int l = 0; l < TDC_PROFILE_LEVELS; ++l) g_prof.lvl_bytes[l] = g_prof.lvl_flops[l] = 0.0;
}

int tdc_profile_end(tdc_profile* out) {
  if (!out) return -1;
  std::memset(out, 0, sizeof(*out));
  if (cudaDeviceSynchronize() != cudaSuccess) return 4;
  for (const ProfRec& r : g_prof.recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    if (r.ph == kSgMark) out->sg_gemm_ms += ms;
    else if (r.ph >= kLevelMark) out->level_fp64_product_ms[r.ph - kLevelMark] += ms;
    else out->ms[r.ph] += ms;
  }
  for (int i = 0; i < TDC_NPHASE; ++i) out->launches[i] = g_prof.launches[i];
  out->product_flops = g_prof.flops;
  out->product_min_bytes = g_prof.bytes;
  out->merges = g_prof.merges;
  out->K_total = g_prof.ktot;
  out->calls = g_prof.calls;
  out->fp64_product_flops = g_prof.fp64_flops;
  out->split_product_flops = g_prof.split_flops;
  out->split_tensor_flops = g_prof.tensor_flops;
  out->defl_copy_bytes = g_prof.copy_bytes;
  out->secular_flops = g_prof.secular_flops;
  out->secular_evals = g_prof.secular_evals;
  out->hss_fallbacks = g_prof.hss_fallbacks;
  out->hss_regrowths = g_prof.hss_regrowths;
  out->hss_sampling_flops = g_prof.hss_sampling_flops;
  out->sg_tensor_flops = g_prof.sg_tensor_flops;
  for (int l = 0; l < TDC_PROFILE_LEVELS; ++l) {
    out->level_fp64_min_bytes[l] = g_prof.lvl_bytes[l];
    out->level_fp64_flops[l] = g_prof.lvl_flops[l];
  }
  g_prof.on = false;
  g_prof.recs.clear();
  g_prof.used = 0;
  return 0;
}

struct tdc_batched_plan {
  tdc::Plan P;
  tdc::PathPlan pp;
  tdc::Layout L;
  tdc_opts o;
  int32_t batch = 0;
  int64_t vtot = 0;
  int64_t qtot = 0;
};

int tdc_batched_plan_create(int32_t batch, const int64_t* n_host, const tdc_opts* opts, void* ws,
                            size_t ws_bytes, void* stream, tdc_batched_plan** out) {
  if (batch < 1) return -1;
  if (!n_host) return -2;
  if (!out) return -7;
  const tdc_opts o = resolve_opts(opts);
  if (!opts_valid(o) || !path_supported(o) || o.path == TDC_PATH_HSS || o.path == TDC_PATH_AUTO) return -3;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return -4;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  tdc_batched_plan* h = new tdc_batched_plan();
  h->o = o;
  h->batch = batch;
  std::vector<ProblemDesc> probs(batch);
  int64_t vtot = 0, qtot = 0;
  for (int p = 0; p < batch; ++p) {
    const int64_t n = n_host[p];
    if (n < 1) {
      delete h;
      return -2;
    }
    probs[p] = ProblemDesc{n, vtot, qtot, n, 3 * qtot};
    vtot += n;
    qtot += n * n;
  }
  h->vtot = vtot;
  h->qtot = qtot;
  build_plan(h->P, probs, o.leaf);
  const auto lj = level_jobs(h->P);
  path_prepare(h->pp, o, lj);
  h->L = carve(ws, vtot, qtot, h->P.nmerges, batch, h->P.blob.size(), h->pp, (int64_t)h->P.leaves.size());
  if (h->L.bytes > ws_bytes) {
    delete h;
    return 3;
  }
  cudaMemcpyAsync(h->L.plan, h->P.blob.data(), h->P.blob.size(), cudaMemcpyHostToDevice, st);
  if (!path_bind(h->pp, h->L.arena, h->L.table, lj, st)) {
    delete h;
    return 4;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    delete h;
    return 4;
  }
  *out = h;
  return 0;
}

int tdc_batched_plan_execute(const tdc_batched_plan* h, const double* d_cat, const double* e_cat,
                             double* lambda_cat, double* Q_cat, int* dev_status_per_problem, void* stream) {
  if (!h) return -1;
  if (!d_cat) return -2;
  if (!e_cat) return -3;
  if (!lambda_cat) return -4;
  if (!Q_cat) return -5;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Layout L = h->L;
  if (dev_status_per_problem) L.w.status = dev_status_per_problem;
  cudaMemsetAsync(L.w.status, 0, sizeof(int) * h->batch, st);
  QBufs qb{Q_cat, L.pool, nullptr};
  const int prc = run_plan(h->P, h->pp, L, h->o, d_cat, e_cat, lambda_cat, qb, h->vtot, h->batch, true, Q_cat, st);
  if (prc) return prc;
  prof_account(h->P, h->pp, L.w.scal, st);
  return launch_status();
}

int tdc_batched_plan_execute_host(const tdc_batched_plan* h, const double* d_host, const double* e_host,
                                  double* lambda_host, double* Q_host, int* status_host, double* d_dev,
                                  double* e_dev, double* lambda_dev, double* Q_dev, int* dev_status,
                                  void* stream) {
  if (!h) return -1;
  if (!d_host) return -2;
  if (!e_host) return -3;
  if (!lambda_host) return -4;
  if (!Q_host) return -5;
  if (!status_host) return -6;
  if (!d_dev) return -7;
  if (!e_dev) return -8;
  if (!lambda_dev) return -9;
  if (!Q_dev) return -10;
  if (!dev_status) return -11;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaMemcpyAsync(d_dev, d_host, h->vtot * sizeof(double), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(e_dev, e_host, h->vtot * sizeof(double), cudaMemcpyHostToDevice, st);
  const int rc = tdc_batched_plan_execute(h, d_dev, e_dev, lambda_dev, Q_dev, dev_status, stream);
  if (rc != 0) return rc;
  cudaMemcpyAsync(lambda_host, lambda_dev, h->vtot * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(Q_host, Q_dev, h->qtot * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(status_host, dev_status, h->batch * sizeof(int), cudaMemcpyDeviceToHost, st);
  return launch_status();
}

int tdc_batched_plan_autotune(tdc_batched_plan* h, const double* d_cat, const double* e_cat,
                              double* lambda_cat, double* Q_cat, int32_t* shape_per_level, int32_t max_levels,
                              int32_t* n_levels, void* stream) {
  if (!h) return -1;
  if (!d_cat) return -2;
  if (!e_cat) return -3;
  if (!lambda_cat) return -4;
  if (!Q_cat) return -5;
  if (shape_per_level && max_levels < 0) return -7;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  QBufs qb{Q_cat, h->L.pool, nullptr};
  std::vector<int> best;
  const int rc = autotune_plan(h->P, h->pp, h->L, h->o, d_cat, e_cat, lambda_cat, qb, h->vtot, h->batch, st, best);
  if (rc) return rc;
  copy_shapes(best, shape_per_level, max_levels, n_levels);
  return launch_status();
}

int tdc_batched_plan_execute_persistent(const tdc_batched_plan* h, const double* d_cat, const double* e_cat,
                                        double* lambda_cat, double* Q_cat, int* dev_status_per_problem,
                                        void* stream) {
  if (!h) return -1;
  if (!d_cat) return -2;
  if (!e_cat) return -3;
  if (!lambda_cat) return -4;
  if (!Q_cat) return -5;
  if (h->o.path != TDC_PATH_DENSE_FP64) return -1;   // the FP64 product only
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Layout L = h->L;
  if (dev_status_per_problem) L.w.status = dev_status_per_problem;
  L.w.ext = h->o.eigvec == TDC_EIGVEC_EXTENDED ? 1 : 0;
  const Plan& P = h->P;
  cudaMemsetAsync(L.w.status, 0, sizeof(int) * h->batch, st);
  cudaMemsetAsync(L.w.lroots, 0, 2 * kMaxLevels * sizeof(unsigned long long), st);
  cudaMemsetAsync(L.w.scal, 0, std::max<int64_t>(P.nmerges, 1) * sizeof(MergeScalars), st);
  cudaMemsetAsync(L.queue, 0, sizeof(unsigned), st);
  QBufs qb{Q_cat, L.pool, nullptr};
  launch_batched_persistent(P_<PersistProb>(L, P.o_pprobs), (int)P.pprobs.size(), L.queue,
                            P_<LeafJob>(L, P.o_leaves), P_<int64_t>(L, P.o_tlist), P_<MergeJob>(L, P.o_pmerges),
                            P_<int32_t>(L, P.o_pmlev), d_cat, e_cat, lambda_cat, qb, L.w, h->o.max_secular_iter, st);
  return launch_status();
}

void tdc_batched_plan_destroy(tdc_batched_plan* h) { delete h; }

int tdc_read_status(const int* dev_status, void* stream) {
  if (!dev_status) return -1;
  int h = 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&h, dev_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return -2;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -2;
  return h;
}

}  // extern "C"
