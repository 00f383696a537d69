// Product-path dispatch (see tdc_paths.cuh).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>

#include "tdc_hss.cuh"
#include "tdc_ozaki.cuh"
#include "tdc_paths.cuh"

namespace tdc {

namespace {
__global__ void k_copy_k(const MergeScalars* scal, int64_t* k_out) { *k_out = scal[0].K; }

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

std::mutex g_tune_mu;
std::map<std::vector<int64_t>, std::vector<int>> g_tune;
LevelTimer* g_timer = nullptr;

// Size rule: tile rows no larger than the merge halves, 16 or 32 columns for the
// smallest merges, else 64 (K is known only on the device).
int default_shape(int64_t maxm) {
  if (maxm <= 32) return 8;
  if (maxm <= 64) return 11;
  if (maxm <= 128) return 3;
  return 1;
}
}  // namespace

void path_set_shape(PathPlan& pp, int l, int cfg, const std::vector<MergeJob>& jobs) {
  PathLevel& L = pp.levels[l];
  L.gemm_cfg = cfg < 0 ? 0 : (cfg >= kGemmShapes ? kGemmShapes - 1 : cfg);
  const int64_t bm = gemm_shape_rows(L.gemm_cfg), bn = gemm_shape_cols(L.gemm_cfg);
  int64_t b = 0;
  for (const MergeJob& J : jobs)
    b += ((J.n1 + bm - 1) / bm + (J.n2 + bm - 1) / bm) * ((J.n1 + J.n2 + bn - 1) / bn);
  L.gemm_bound = b;
}

std::vector<int64_t> tune_key(const tdc_opts& o, const std::vector<const std::vector<MergeJob>*>& lv) {
  std::vector<int64_t> k{(int64_t)o.path, (int64_t)o.leaf, (int64_t)lv.size()};
  for (const auto* jobs : lv) {
    int64_t maxm = 0, sum = 0;
    for (const MergeJob& J : *jobs) {
      maxm = std::max<int64_t>(maxm, J.n1 + J.n2);
      sum += J.n1 + J.n2;
    }
    k.push_back((int64_t)jobs->size());
    k.push_back(maxm);
    k.push_back(sum);
  }
  return k;
}

void tune_store(const std::vector<int64_t>& key, const std::vector<int>& cfg) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune[key] = cfg;
}

void set_level_timer(LevelTimer* t) { g_timer = t; }

bool path_supported(const tdc_opts& o) {
  return o.path == TDC_PATH_DENSE_FP64 || o.path == TDC_PATH_DENSE_OZAKI || o.path == TDC_PATH_HSS ||
         o.path == TDC_PATH_AUTO;
}

// Level choice: HSS for levels whose merges reach the HSS size (HSS path: two HSS
// leaves; AUTO: k_threshold), the split product for large dense merges (split and
// AUTO paths), FP64 otherwise.
static int level_kind(const tdc_opts& o, int64_t maxm) {
  if (o.path == TDC_PATH_HSS && maxm >= 2 * (int64_t)o.hss_leaf) return 2;
  if (o.path == TDC_PATH_AUTO && maxm >= o.k_threshold) return 2;
  if ((o.path == TDC_PATH_DENSE_OZAKI || o.path == TDC_PATH_AUTO) && maxm >= kOzMinOrder) return 1;
  return 0;
}

void path_prepare(PathPlan& pp, const tdc_opts& o, const std::vector<const std::vector<MergeJob>*>& lv) {
  pp.levels.assign(lv.size(), PathLevel{});
  std::vector<int> tuned;
  if (o.tile_cfg < 0) {
    const std::vector<int64_t> key = tune_key(o, lv);
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end() && it->second.size() == lv.size()) tuned = it->second;
  }
  pp.slices = o.ozaki_slices < 5 ? 5 : (o.ozaki_slices > 7 ? 7 : o.ozaki_slices);
  pp.arena_bytes = 0;
  size_t tab = 0;
  for (size_t l = 0; l < lv.size(); ++l) {
    const auto& jobs = *lv[l];
    int64_t maxm = 0;
    for (const MergeJob& J : jobs) maxm = std::max<int64_t>(maxm, J.n1 + J.n2);
    PathLevel& L = pp.levels[l];
    if (jobs.empty()) continue;
    path_set_shape(pp, (int)l, o.tile_cfg >= 0 ? o.tile_cfg : (tuned.empty() ? default_shape(maxm) : tuned[l]),
                   jobs);
    const int kind = level_kind(o, maxm);
    if (kind == 2) {
      L.hss = true;
      pp.arena_bytes = std::max(pp.arena_bytes, al(hss_arena_bytes(maxm, o)));
      continue;
    }
    if (kind != 1) continue;
    L.oz = true;
    size_t arena = 0;
    for (const MergeJob& J : jobs) arena += al(oz_job_bytes(J, pp.slices));
    pp.arena_bytes = std::max(pp.arena_bytes, arena);
    L.tab_off = tab;
    tab = al(tab + jobs.size() * sizeof(OzJob));
    for (int c = 0; c < 3; ++c) {
      L.cum_off[c] = tab;
      tab = al(tab + (jobs.size() + 1) * sizeof(int64_t));
    }
  }
  pp.table_bytes = tab;
}

bool path_bind(PathPlan& pp, unsigned char* arena, unsigned char* table_dev,
               const std::vector<const std::vector<MergeJob>*>& lv, cudaStream_t st) {
  pp.arena_dev = arena;
  pp.table_dev = table_dev;
  (void)lv;
  if (pp.table_bytes == 0) return true;
  pp.table_store.assign(pp.table_bytes / 8 + 64, 0);
  pp.table = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(pp.table_store.data()) + 255) & ~uintptr_t(255));
  bool ok = true;
  for (size_t l = 0; l < lv.size(); ++l) {
    PathLevel& L = pp.levels[l];
    if (!L.oz) continue;
    const auto& jobs = *lv[l];
    OzJob* z = reinterpret_cast<OzJob*>(pp.table + L.tab_off);
    int64_t* cum[3];
    for (int c = 0; c < 3; ++c) {
      cum[c] = reinterpret_cast<int64_t*>(pp.table + L.cum_off[c]);
      cum[c][0] = 0;
    }
    size_t off = 0;
    for (size_t j = 0; j < jobs.size(); ++j) {
      ok = ok && oz_fill_job(z[j], jobs[j], arena + off, pp.slices);
      off += al(oz_job_bytes(jobs[j], pp.slices));
      cum[0][j + 1] = cum[0][j] + oz_blocks_slice_a(jobs[j]);
      cum[1][j + 1] = cum[1][j] + oz_blocks_slice_b(jobs[j]);
      cum[2][j + 1] = cum[2][j] + oz_tiles(jobs[j]);
    }
    for (int c = 0; c < 3; ++c) L.nb[c] = cum[c][jobs.size()];
  }
  cudaMemcpyAsync(table_dev, pp.table, pp.table_bytes, cudaMemcpyHostToDevice, st);
  return ok;
}

int launch_product(const PathPlan& pp, int l, const tdc_opts& o, const std::vector<MergeJob>& hjobs,
                   const MergeJob* jobs, int64_t* cum_tiles, QBufs qb, DevWs w, cudaStream_t st) {
  const PathLevel* L = (l >= 0 && l < (int)pp.levels.size()) ? &pp.levels[l] : nullptr;
  if (!(L && L->oz)) phase_mark(5, true, 0, st);
  if (L && L->hss) {
    int rc = 0;
    for (size_t j = 0; j < hjobs.size(); ++j) {
      rc = run_hss_merge(hjobs[j], qb, w, pp.arena_dev, pp.arena_bytes, o, st);
      if (rc == kHssSaturated) {             // samples too few for the ranks: the exact dense product
        launch_gemm_fp64(L->gemm_cfg, jobs + j, 1, cum_tiles, L->gemm_bound, qb, w, st);
        hss_fallbacks_add(1);
        rc = 0;
      }
      if (rc) break;
    }
    phase_mark(5, false, 1, st);
    return rc;
  }
  if (L && L->oz) {
    const OzJob* z = reinterpret_cast<const OzJob*>(pp.table_dev + L->tab_off);
    const int64_t* c0 = reinterpret_cast<const int64_t*>(pp.table_dev + L->cum_off[0]);
    int64_t* c1 = reinterpret_cast<int64_t*>(pp.table_dev + L->cum_off[1]);
    int64_t* c2 = reinterpret_cast<int64_t*>(pp.table_dev + L->cum_off[2]);
    phase_mark(9, true, 0, st);
    launch_ozaki_level(0, jobs, z, (int)hjobs.size(), c0, L->nb[0], c1, L->nb[1], c2, L->nb[2], pp.slices, qb,
                       w, st);
    phase_mark(9, false, 2, st);
    phase_mark(8, true, 0, st);
    launch_ozaki_level(1, jobs, z, (int)hjobs.size(), c0, L->nb[0], c1, L->nb[1], c2, L->nb[2], pp.slices, qb,
                       w, st);
    phase_mark(8, false, 1, st);
  } else {
    const bool timed = g_timer && l >= 0 && l < (int)g_timer->a.size();
    if (timed) cudaEventRecord(g_timer->a[l], st);
    phase_mark(kLevelMark + l, true, 0, st);
    launch_gemm_fp64(L ? L->gemm_cfg : 1, jobs, (int)hjobs.size(), cum_tiles, L ? L->gemm_bound : 0, qb, w, st);
    phase_mark(kLevelMark + l, false, 0, st);
    if (timed) {
      cudaEventRecord(g_timer->b[l], st);
      g_timer->used[l] = true;
    }
    phase_mark(5, false, 2, st);
  }
  return 0;
}

void launch_copy_k(const MergeScalars* scal, int64_t* k_out, cudaStream_t st) {
  k_copy_k<<<1, 1, 0, st>>>(scal, k_out);
}

}  // namespace tdc
