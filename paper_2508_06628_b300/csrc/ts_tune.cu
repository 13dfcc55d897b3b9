// ts_tune.cu -- the autotuner of the hot path's launch and list parameters
// (ts_tuning: pair work-item size, cell-list bin edge, skin scale,
// inner-list radius, re-list hysteresis).  Each candidate is timed in situ: the batch's MD step
// (as the caller runs it) replayed as a CUDA graph, CUDA events around whole
// calls on the caller's stream.  The fields are tuned one after another, each
// over its candidate values with the others at their best so far.  Results
// are cached in a text file keyed by (potential kinds, log2 of the atom and
// system capacities, precision), one line per tuning:
//   key item_warps inner_fraction relist_soon bin_factor skin_scale
// (a line without skin_scale reads as 1), and the last line matching a
// batch's key is applied at ts_batch_create.
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "ts_kernels.cuh"

namespace ts {

static std::string tune_key(const ts_batch* b) {
  std::ostringstream k;
  k << "pots=";
  for (int q = 0; q < b->n_pots; q++) k << b->pots[q].kind;
  int na = 0, ns = 0;
  for (int64_t n = b->cfg.atom_capacity; n > 1; n >>= 1) na++;
  for (int64_t n = b->cfg.system_capacity; n > 1; n >>= 1) ns++;
  k << ";log2atoms=" << na << ";log2systems=" << ns << ";fp64=" << (b->f64 ? 1 : 0);
  return k.str();
}

bool tuning_valid(const ts_tuning& t) {
  return (t.item_warps == 4 || t.item_warps == 8) && t.inner_fraction > 0 && t.inner_fraction <= 1 &&
         t.relist_soon > 0 && t.relist_soon <= 1 && (t.bin_factor == 1.0 || t.bin_factor == 0.5) &&
         t.skin_scale > 0 && t.skin_scale <= 1;
}

// the last cache line whose key matches, if any
static bool read_cache(const std::string& path, const std::string& key, ts_tuning& out) {
  std::ifstream f(path);
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream ls(line);
    std::string k;
    ts_tuning t;
    t.skin_scale = 1.0;
    if (!(ls >> k >> t.item_warps >> t.inner_fraction >> t.relist_soon >> t.bin_factor)) continue;
    double sc;
    if (ls >> sc) t.skin_scale = sc;
    if (k == key && tuning_valid(t)) {
      out = t;
      found = true;
    }
  }
  return found;
}

void autotune_load(ts_batch* b) {
  b->pair_threads = 128;
  if (b->cache_path.empty()) return;
  ts_tuning t;
  if (read_cache(b->cache_path, tune_key(b), t)) b->tune = t;
}

// Make t the batch's parameters: new potential table, and a fresh layout
// (work items) and listing of every system on the next call.
ts_status apply_tuning(ts_batch* b, const ts_tuning& t) {
  b->tune = t;
  DevPot dp[kMaxPots];
  fill_devpots(b, dp);
  b->dp_host.assign(dp, dp + kMaxPots);
  cudaSetDevice(b->cfg.device);
  if (!cuda_ok(b, cudaMemcpy(b->d_pots, dp, sizeof dp, cudaMemcpyHostToDevice), "potential table")) return TS_ERR_CUDA;
  b->topo_valid = false;      // items follow item_warps; the bins follow bin_factor
  b->graphs_valid = false;
  return TS_OK;
}

}  // namespace ts

using namespace ts;

extern "C" ts_status ts_batch_tuning(const ts_batch* b, ts_tuning* out) {
  if (!b || !out) return TS_ERR_INVALID_ARG;
  *out = b->tune;
  return TS_OK;
}

extern "C" ts_status ts_batch_set_tuning(ts_batch* b, const ts_tuning* t) {
  if (!b || !t) return TS_ERR_INVALID_ARG;
  if (!tuning_valid(*t)) return fail(b, TS_ERR_INVALID_ARG, "tuning outside its ranges");
  if (!cuda_ok(b, cudaDeviceSynchronize(), "synchronise")) return TS_ERR_CUDA;
  return apply_tuning(b, *t);
}

extern "C" ts_status ts_autotune(ts_batch* b, ts_state* s, const ts_md_params* p, int n_steps, void* stream) {
  ts_status r = check_state(b, s, true);
  if (r != TS_OK) return r;
  if (!p || n_steps < 1 || n_steps > 1000) return fail(b, TS_ERR_INVALID_ARG, "bad MD parameters or step count");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (!cuda_ok(b, cudaEventCreate(&e0), "event") || !cuda_ok(b, cudaEventCreate(&e1), "event")) return TS_ERR_CUDA;
  ts_md_params q = *p;
  // Every trial starts from the same state: the caller's, advanced by an
  // equilibrating run of 4 n_steps (trials then time the dynamics that
  // follow, not the start-up transient of a freshly built state), saved on
  // the device and restored, with the same noise counter, before each trial.
  const bool npt = p->kind == TS_NPT_LANGEVIN, nhc = p->kind == TS_NVT_NHC;
  const size_t nx = 3 * (size_t)s->n_atoms, nb = (size_t)s->n_systems;
  const size_t nsave = 2 * nx + (npt ? 10 * nb : 0) + (nhc ? 6 * nb : 0);
  double* save = nullptr;
  if (!cuda_ok(b, cudaMalloc(&save, 8 * nsave), "tuning state copy")) return TS_ERR_CUDA;
  auto copy_state = [&](bool restore) -> bool {
    struct { double* a; size_t n; } parts[5] = {{s->pos, nx}, {s->vel, nx}, {npt ? s->cell : nullptr, 9 * nb},
                                                {npt ? p->baro : nullptr, nb}, {nhc ? p->nhc : nullptr, 6 * nb}};
    size_t off = 0;
    for (auto& pt : parts) {
      if (!pt.a) continue;
      cudaError_t e = restore ? cudaMemcpyAsync(pt.a, save + off, 8 * pt.n, cudaMemcpyDeviceToDevice, st)
                              : cudaMemcpyAsync(save + off, pt.a, 8 * pt.n, cudaMemcpyDeviceToDevice, st);
      if (!cuda_ok(b, e, "tuning state copy")) return false;
      off += pt.n;
    }
    return true;
  };
  r = ts_md_step(b, s, &q, 4 * n_steps, nullptr, nullptr, st);
  q.step0 += 4 * (uint64_t)n_steps;
  if (r == TS_OK && !copy_state(false)) r = TS_ERR_CUDA;
  const uint64_t step_start = q.step0;
  // milliseconds per MD step of configuration t: a warm-up call (layout,
  // listing, graph capture), then three timed calls of n_steps
  auto trial = [&](const ts_tuning& t, double& ms_out) -> ts_status {
    if (!copy_state(true)) return TS_ERR_CUDA;
    q.step0 = step_start;
    ts_status rr = apply_tuning(b, t);
    if (rr != TS_OK) return rr;
    if ((rr = ts_md_step(b, s, &q, n_steps, nullptr, nullptr, st)) != TS_OK) return rr;
    q.step0 += (uint64_t)n_steps;
    if (!cuda_ok(b, cudaEventRecord(e0, st), "event record")) return TS_ERR_CUDA;
    for (int c = 0; c < 3; c++) {
      if ((rr = ts_md_step(b, s, &q, n_steps, nullptr, nullptr, st)) != TS_OK) return rr;
      q.step0 += (uint64_t)n_steps;
    }
    if (!cuda_ok(b, cudaEventRecord(e1, st), "event record") || !cuda_ok(b, cudaEventSynchronize(e1), "event sync"))
      return TS_ERR_CUDA;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms_out = ms / (3.0 * n_steps);
    if (getenv("TS_TUNE_LOG"))
      fprintf(stderr, "ts_autotune: item_warps %d inner %.3g soon %.3g bins %.3g skin %.3g: %.5f ms/step\n",
              t.item_warps, t.inner_fraction, t.relist_soon, t.bin_factor, t.skin_scale, ms_out);
    return ts_batch_poll(b, st, -1);   // a trial that overflowed a list or met bad input fails the tuning
  };
  ts_tuning best = b->tune;
  double best_ms = 0;
  if (r == TS_OK) r = trial(best, best_ms);
  if (r != TS_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(save);
    return r;
  }
  // the fields in turn, each over its candidates with the others at their best
  const double bins[2] = {1.0, 0.5};
  const int items[2] = {8, 4};
  const double skins[3] = {1.0, 0.9, 0.8};
  const double inner[5] = {0.2, 0.3, 0.45, 0.5, 1.0};   // 1: the inner list is the Verlet list
  const double soon[3] = {0.4, 0.5, 0.6};
  const int ncand[5] = {2, 2, 3, 5, 3};
  for (int field = 0; field < 5 && r == TS_OK; field++) {
    for (int c = 0; c < ncand[field] && r == TS_OK; c++) {
      ts_tuning t = best;
      if (field == 0) t.bin_factor = bins[c];
      if (field == 1) t.item_warps = items[c];
      if (field == 2) t.skin_scale = skins[c];
      if (field == 3) t.inner_fraction = inner[c];
      if (field == 4) t.relist_soon = soon[c];
      if (t.bin_factor == best.bin_factor && t.item_warps == best.item_warps && t.skin_scale == best.skin_scale &&
          t.inner_fraction == best.inner_fraction && t.relist_soon == best.relist_soon)
        continue;   // the current best, timed already
      double ms = 0;
      r = trial(t, ms);
      if (r == TS_OK && ms < best_ms) { best_ms = ms; best = t; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(save);
  ts_status ra = apply_tuning(b, best);
  if (r != TS_OK) return r;
  if (ra != TS_OK) return ra;
  if (!b->cache_path.empty()) {
    FILE* f = fopen(b->cache_path.c_str(), "a");
    if (f) {
      fprintf(f, "%s %d %.17g %.17g %.17g %.17g\n", tune_key(b).c_str(), best.item_warps, best.inner_fraction,
              best.relist_soon, best.bin_factor, best.skin_scale);
      fclose(f);
    }
  }
  return cuda_ok(b, cudaGetLastError(), "ts_autotune") ? TS_OK : TS_ERR_CUDA;
}
