// ts_sched.cpp -- host-side batching logic (TorchSim, Sec. 3): the memory
// probe of Fig. 2, the admission queue of the InFlightAutobatcher and the bin
// packing of the BinningAutobatcher (Fig. 3).  No device memory is touched here.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/ts.h"

// Fig. 2: for each probe system grow a batch of copies until the fit test
// fails; max scaler = min over probes of (systems that fit) * scaler.
extern "C" ts_status ts_estimate_max_scaler(const double* scaler, int n, int (*fits)(double, int, void*), void* ctx,
                                            int max_systems, int* n_fit_out, double* max_scaler_out) {
  if (!scaler || n < 1 || !fits || max_systems < 1 || !max_scaler_out) return TS_ERR_INVALID_ARG;
  double best = INFINITY;
  for (int k = 0; k < n; k++) {
    if (!(scaler[k] > 0)) return TS_ERR_INVALID_ARG;
    int m = 0;
    while (m < max_systems && fits(scaler[k] * (m + 1), m + 1, ctx)) m++;
    if (n_fit_out) n_fit_out[k] = m;
    if (m == 0) return TS_ERR_BUDGET;
    double v = m * scaler[k];
    if (v < best) best = v;
  }
  *max_scaler_out = best;
  return TS_OK;
}

struct ts_sched {
  double max_scaler = 0;
  int32_t max_active = 0;
  std::deque<std::pair<int64_t, double>> pending;
  std::unordered_map<int64_t, double> active;
  double active_scaler = 0;
};

extern "C" ts_status ts_sched_create(double max_scaler, int32_t max_active, ts_sched** out) {
  if (!out || !(max_scaler > 0) || max_active < 1) return TS_ERR_INVALID_ARG;
  ts_sched* q = new (std::nothrow) ts_sched();
  if (!q) return TS_ERR_BUDGET;
  q->max_scaler = max_scaler;
  q->max_active = max_active;
  *out = q;
  return TS_OK;
}

extern "C" ts_status ts_sched_destroy(ts_sched* q) {
  if (!q) return TS_ERR_INVALID_ARG;
  delete q;
  return TS_OK;
}

extern "C" ts_status ts_sched_push(ts_sched* q, int64_t id, double scaler) {
  if (!q || !(scaler > 0)) return TS_ERR_INVALID_ARG;
  if (scaler > q->max_scaler) return TS_ERR_BUDGET;   // could never be admitted
  q->pending.emplace_back(id, scaler);
  return TS_OK;
}

// Sample systems from the stream, in order, until memory (the scaler budget)
// or the active-slot limit is full.
extern "C" ts_status ts_sched_fill(ts_sched* q, int64_t* ids_out, int cap, int* n_out) {
  if (!q || !n_out || cap < 0 || (cap > 0 && !ids_out)) return TS_ERR_INVALID_ARG;
  int n = 0;
  while (!q->pending.empty() && n < cap && (int32_t)q->active.size() < q->max_active) {
    auto [id, sc] = q->pending.front();
    if (q->active_scaler + sc > q->max_scaler * (1 + 1e-12)) break;
    q->pending.pop_front();
    q->active.emplace(id, sc);
    q->active_scaler += sc;
    ids_out[n++] = id;
  }
  *n_out = n;
  return TS_OK;
}

extern "C" ts_status ts_sched_retire(ts_sched* q, const int64_t* ids, int n) {
  if (!q || n < 0 || (n > 0 && !ids)) return TS_ERR_INVALID_ARG;
  for (int k = 0; k < n; k++) {
    auto it = q->active.find(ids[k]);
    if (it == q->active.end()) return TS_ERR_INVALID_ARG;
    q->active_scaler -= it->second;
    q->active.erase(it);
  }
  if (q->active.empty()) q->active_scaler = 0;
  return TS_OK;
}

extern "C" ts_status ts_sched_stats(const ts_sched* q, int32_t* n_active, int64_t* n_pending, double* active_scaler) {
  if (!q) return TS_ERR_INVALID_ARG;
  if (n_active) *n_active = (int32_t)q->active.size();
  if (n_pending) *n_pending = (int64_t)q->pending.size();
  if (active_scaler) *active_scaler = q->active_scaler;
  return TS_OK;
}

// BinningAutobatcher: 1-D bin packing by first fit decreasing (the paper asks
// for as few bins as possible and names no algorithm; exact packing is
// NP-hard, and FFD uses at most 11/9 OPT + 6/9 bins).
extern "C" ts_status ts_bin_pack(const double* sizes, int n, double capacity, int32_t* bin_out,
                                 int32_t* n_bins_out) {
  if (n < 0 || (n > 0 && (!sizes || !bin_out)) || !(capacity > 0) || !std::isfinite(capacity) || !n_bins_out)
    return TS_ERR_INVALID_ARG;
  for (int k = 0; k < n; k++) {
    if (!(sizes[k] > 0) || !std::isfinite(sizes[k])) return TS_ERR_INVALID_ARG;
    if (sizes[k] > capacity) return TS_ERR_BUDGET;
  }
  std::vector<int> order(n);
  for (int k = 0; k < n; k++) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sizes[a] > sizes[b]; });
  std::vector<double> room;
  for (int k : order) {
    size_t c = 0;
    while (c < room.size() && room[c] < sizes[k]) c++;
    if (c == room.size()) room.push_back(capacity);
    room[c] -= sizes[k];
    bin_out[k] = (int32_t)c;
  }
  *n_bins_out = (int32_t)room.size();
  return TS_OK;
}
