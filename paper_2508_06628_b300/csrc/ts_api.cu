// ts_api.cu -- the batch object and the C ABI entry points of libts.so
// (declared in include/ts.h).  Host code only orchestrates: every step of the
// path runs in the kernels of ts_neighbor.cu, ts_pair.cu, ts_md.cu,
// ts_fire.cu and ts_adjoint.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ts_api.h"

using namespace ts;

namespace ts {

const char* kNoError = "";

bool cuda_ok(ts_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  if (b) {
    b->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    b->sticky = TS_ERR_CUDA;
  }
  return false;
}

ts_status fail(ts_batch* b, ts_status st, const std::string& msg) {
  if (b) b->last_error = msg;
  return st;
}

static int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 148 * 16) g = 148 * 16;
  return (int)g;
}

template <typename T>
static bool alloc(ts_batch* b, T*& p, size_t count) {
  p = nullptr;
  if (count == 0) count = 1;
  size_t bytes = sizeof(T) * count;
  if (!cuda_ok(b, cudaMalloc((void**)&p, bytes), "cudaMalloc")) return false;
  b->allocations.push_back((void*)p);
  b->bytes_allocated += bytes;
  return true;
}

size_t scratch_bytes(int64_t Ncap, int64_t Bcap, int64_t Ccap, int32_t max_nbrs, bool f64) {
  size_t per_slot = f64 ? (3 * 8 /*xd*/ + 3 * 8 /*vd*/ + 3 * 8 /*Fd*/ + 8 /*minv*/ + 3 * 8 /*xrd*/ +
                           3 * 8 * 3 /*tmp d0,d1*/ + 4 * 8 /*tmp d2*/ + 2 * 3 * 8 /*gd*/)
                        : (2 * 16 /*x*/ + 2 * 16 /*v*/ + 16 /*F*/ + 2 * 16 /*xr*/ + 2 * 16 + 2 * 16 /*tmp f*/ +
                           2 * 16 /*g*/);
  per_slot += (f64 ? 3 * 8 : 2 * 16) /*prune reference*/ + 4 /*nn_in*/ + (size_t)(max_nbrs + 3) / 4 * 16 /*inner list*/;
  per_slot += 4 * 4 /*perm sys bin nn*/ + 3 * 4 /*tmp i*/ + (size_t)max_nbrs * 4 + 8 * 8 / 32 /*partials*/ + (4 /*warp_sys*/ + 16 /*pair work items*/ + 4 * kItemWarps /*their warps' systems*/ + 31) / 32;
  size_t per_sys = 4 /*inner-list format*/ + 8 * 4 + 9 * 8 * 3 + 9 * 4 + 6 * 4 + 4 * 4 + 8 + 12 /*list-build work table*/ + 8 /*piston*/ + 4 /*geometry state*/ + 8 /*table bounds*/ + 32 * 4 /*FIRE FP32 coefficients*/ +
                   (size_t)kNCodes * (32 + 24 + 16);
  return per_slot * (size_t)Ncap + per_sys * (size_t)Bcap + (size_t)Ccap * 8;
}

// The device potential table from the potentials and the tuned parameters:
// cutoffs and shifts, list radius rc + skin (the potential's skin times the
// tuned scale), bin edge (the list radius times the tuned bin factor), re-list
// hysteresis, inner (pruned) list radius.
void fill_devpots(ts_batch* b, DevPot* dp) {
  memset(dp, 0, sizeof(DevPot) * kMaxPots);
  b->use_small_pair = true;
  for (int q = 0; q < b->n_pots; q++) {
    const ts_potential& P = b->pots[q];
    DevPot& D = dp[q];
    D.kind = P.kind; D.shift = P.shift;
    for (int c = 0; c < 3; c++) { D.pd[c] = P.p[c]; D.pf[c] = (float)P.p[c]; }
    double rc = P.kind == TS_SOFT_SPHERE ? P.p[0] : P.cutoff;
    D.rc2d = rc * rc; D.rc2f = (float)(rc * rc);
    D.sinvf = (float)(1.0 / P.p[0]);
    double phic = 0;
    if (P.shift && P.kind == TS_LJ) { double s = P.p[0] / rc, s6 = s * s * s * s * s * s; phic = 4 * P.p[1] * (s6 * s6 - s6); }
    if (P.shift && P.kind == TS_MORSE) { double e = exp(-P.p[1] * (rc - P.p[2])); phic = P.p[0] * (e * e - 2 * e); }
    D.phicd = phic; D.phicf = (float)phic;
    const double skin = P.skin * b->tune.skin_scale;   // the tuned skin
    D.skin = skin;
    D.rlist = rc + skin; D.rlist2d = D.rlist * D.rlist; D.rlist2f = (float)D.rlist2d;
    D.binw = D.rlist * b->tune.bin_factor;
    D.soon2 = b->tune.relist_soon * b->tune.relist_soon;
    {   // inner skin of the pruned list: a fraction of the skin (1 = no pruning)
      double sin = b->tune.inner_fraction * skin, ri = rc + sin + kListBand;
      D.rin2d = ri * ri; D.rin2f = (float)D.rin2d;
      D.half_in2d = 0.25 * sin * sin; D.half_in2f = (float)D.half_in2d;
    }
    D.rlist_in2f = (float)((D.rlist - kListBand) * (D.rlist - kListBand));
    D.rlist_out2f = (float)((D.rlist + kListBand) * (D.rlist + kListBand));
    D.half_skin2f = (float)(0.25 * skin * skin);
    D.soon_half_skin2f = (float)(D.soon2 * 0.25 * skin * skin);
    b->rc[q] = rc;
    if (D.rlist >= kFixMaxList) b->use_small_pair = false;   // beyond the fixed-point range of k_pair_small
  }
}

}  // namespace ts

// ---------------------------------------------------------------------------
extern "C" ts_status ts_batch_create(const ts_batch_config* cfg, const ts_potential* pots, int n_pots, ts_batch** out) {
  if (!out) return TS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg || !pots || n_pots < 1 || n_pots > kMaxPots) return TS_ERR_INVALID_ARG;
  if (cfg->atom_capacity < 1 || cfg->system_capacity < 1 || cfg->max_neighbors < 0 ||
      (cfg->precision != TS_MIXED && cfg->precision != TS_FP64))
    return TS_ERR_INVALID_ARG;
  for (int q = 0; q < n_pots; q++) {
    const ts_potential& P = pots[q];
    if (P.kind < 0 || P.kind > 2 || !(P.skin >= 0) || !(P.cutoff > 0 || P.kind == TS_SOFT_SPHERE)) return TS_ERR_INVALID_ARG;
    if (P.kind == TS_SOFT_SPHERE && !(P.p[0] > 0 && P.p[2] >= 1.0)) return TS_ERR_INVALID_ARG;
    if (P.kind == TS_LJ && !(P.p[0] > 0)) return TS_ERR_INVALID_ARG;
  }
  ts_batch* b = new ts_batch();
  b->cfg = *cfg;
  if (cfg->autotune_cache) { b->cache_path = cfg->autotune_cache; b->cfg.autotune_cache = b->cache_path.c_str(); }
  b->f64 = cfg->precision == TS_FP64;
  b->n_pots = n_pots;
  for (int q = 0; q < n_pots; q++) b->pots[q] = pots[q];
  b->max_nbrs = cfg->max_neighbors > 0 ? cfg->max_neighbors : 160;
  b->Bcap = cfg->system_capacity;
  b->Ncap = ((cfg->atom_capacity + 31LL * cfg->system_capacity) + 31) / 32 * 32;
  b->Wcap = b->Ncap / 32;
  b->Ccap = cfg->atom_capacity + 27LL * cfg->system_capacity;
  if (b->Ncap >= (1LL << 31) || b->Ccap >= (1LL << 31)) { delete b; return TS_ERR_UNSUPPORTED; }
  size_t need = scratch_bytes(b->Ncap, b->Bcap, b->Ccap, b->max_nbrs, b->f64);
  if (cfg->memory_budget_bytes && need > cfg->memory_budget_bytes) { delete b; return TS_ERR_BUDGET; }
  if (!cuda_ok(b, cudaSetDevice(cfg->device), "cudaSetDevice")) { delete b; return TS_ERR_CUDA; }
  if (!cuda_ok(b, cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, cfg->device), "SM count")) {
    delete b;
    return TS_ERR_CUDA;
  }
  // tuned launch and list parameters: defaults (TS_SOON / TS_INNER override),
  // then the cache entry for this configuration, if any
  {
    const char* e = getenv("TS_SOON");
    if (e) { double f = atof(e); b->tune.relist_soon = (f > 0 && f <= 1) ? f : 1.0; }
    e = getenv("TS_INNER");
    if (e) { double f = atof(e); b->tune.inner_fraction = (f > 0 && f <= 1) ? f : 1.0; }
  }
  autotune_load(b);
  // device potential table
  DevPot dp[kMaxPots];
  fill_devpots(b, dp);
  bool ok = true;
  SysArrays& S = b->S;
  SlotArrays& A = b->A;
  int64_t N = b->Ncap, B = b->Bcap;
  ok = ok && alloc(b, b->d_pots, kMaxPots) && alloc(b, b->d_err, 4) && alloc(b, b->d_counters, 4) &&

       alloc(b, b->d_step, 2) && alloc(b, b->d_rec, 1);
  ok = ok && alloc(b, S.seg_start, B) && alloc(b, S.n_atoms, B) && alloc(b, S.caller_off, B + 1) && alloc(b, S.pot, B) &&
       alloc(b, S.uid, B) && alloc(b, S.bin_off, B) && alloc(b, S.bin_cap, B) && alloc(b, S.warp_start, B) &&
       alloc(b, S.warp_end, B) && alloc(b, S.h, 9 * B) && alloc(b, S.hinv, 9 * B) && alloc(b, S.hinvf, 9 * B) && alloc(b, S.href, 9 * B) &&
       alloc(b, S.nb, 3 * B) && alloc(b, S.reach, 3 * B) && alloc(b, S.pmask, B) && alloc(b, S.relist, B) && alloc(b, S.prune, B) && alloc(b, S.dirty, B) &&
       alloc(b, S.soon, B) && alloc(b, S.infmt, B) && alloc(b, S.any, 1) && alloc(b, S.geom, B) && alloc(b, S.tbound, B) && alloc(b, S.lbound, B) &&
       alloc(b, S.kT, B) && alloc(b, S.shift, 2 * B * kNCodes) && alloc(b, S.shiftd, 3 * B * kNCodes) && alloc(b, S.shiftq, B * kNCodes);
  ok = ok && alloc(b, A.perm, N) && alloc(b, A.sys, N) && alloc(b, A.bin, N) && alloc(b, A.nn, N) &&
       alloc(b, A.nbr, (size_t)b->max_nbrs * N) && alloc(b, A.nbr_in, (size_t)(b->max_nbrs + 3) / 4 * 4 * N) && alloc(b, A.nn_in, N) && alloc(b, A.tmp_i0, N) && alloc(b, A.tmp_i1, N) &&
       alloc(b, A.tmp_i2, N);
  if (b->f64) {
    ok = ok && alloc(b, A.xpd, 3 * N) && alloc(b, A.xd, 3 * N) && alloc(b, A.vd, 3 * N) && alloc(b, A.Fd, 3 * N) && alloc(b, A.minvd, N) &&
         alloc(b, A.xrd, 3 * N) && alloc(b, A.tmp_d0, 3 * N) && alloc(b, A.tmp_d1, 3 * N) &&
         alloc(b, A.tmp_d2, 4 * N) && alloc(b, A.gd0, 3 * N) && alloc(b, A.gd1, 3 * N);
  } else {
    ok = ok && alloc(b, A.xph, N) && alloc(b, A.xpl, N) && alloc(b, A.xh, N) && alloc(b, A.xl, N) && alloc(b, A.vh, N) && alloc(b, A.vl, N) && alloc(b, A.F, N) &&
         alloc(b, A.xrh, N) && alloc(b, A.xrl, N) && alloc(b, A.tmp_f0, 2 * N) && alloc(b, A.tmp_f1, N) &&
         alloc(b, A.tmp_f2, N) && alloc(b, A.tmp_f3, N) && alloc(b, A.g0, N) && alloc(b, A.g1, N);
  }
  ok = ok && alloc(b, b->d_partial, (size_t)kPartialStride * b->Wcap) && alloc(b, b->d_warp_sys, b->Wcap) &&
       alloc(b, b->d_count, b->Ccap) && alloc(b, b->d_cstart, b->Ccap) &&
       alloc(b, b->d_bsum, (b->Ccap + 1023) / 1024 + 1) && alloc(b, b->d_starts, B + 1) &&
       alloc(b, b->d_Eint, B) && alloc(b, b->d_Wint, 9 * B) && alloc(b, b->d_scal, 32 * B) && alloc(b, b->d_fcoef, 32 * B) && alloc(b, b->d_nhc, 6 * B) && alloc(b, b->d_baro, B) &&
       alloc(b, b->d_gparam_part, 4 * b->Wcap) && alloc(b, b->d_gacc, 3 * kMaxPots) &&
       alloc(b, b->d_items, b->Wcap) && alloc(b, b->d_item_sys, (size_t)kItemWarps * b->Wcap) && alloc(b, b->d_tab_sys, B) && alloc(b, b->d_tab_base, B + 1) && alloc(b, b->d_tab_base_a, B + 1) &&
       alloc(b, b->d_tab_n, 3);
  if (ok) ok = cuda_ok(b, cudaMemcpy(b->d_pots, dp, sizeof dp, cudaMemcpyHostToDevice), "copy pots");
  if (ok) ok = cuda_ok(b, cudaMemset(b->d_err, 0, 16), "memset") && cuda_ok(b, cudaMemset(b->d_counters, 0, 32), "memset");
  if (ok) ok = cuda_ok(b, cudaMemset(A.perm, 0xff, sizeof(int32_t) * N), "memset") &&
               cuda_ok(b, cudaMemset(A.sys, 0xff, sizeof(int32_t) * N), "memset") &&
               cuda_ok(b, cudaMemset(A.nn, 0, sizeof(int32_t) * N), "memset") &&
               cuda_ok(b, cudaMemset(A.nn_in, 0, sizeof(int32_t) * N), "memset") &&
               cuda_ok(b, cudaMemset(S.infmt, 0, sizeof(int32_t) * B), "memset") &&
               cuda_ok(b, cudaMemset(b->d_partial, 0, sizeof(double) * kPartialStride * b->Wcap), "memset");
  if (ok) ok = cuda_ok(b, cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming), "event");
  if (ok) {
    int least = 0, greatest = 0;
    ok = cuda_ok(b, cudaDeviceGetStreamPriorityRange(&least, &greatest), "priority range") &&
         cuda_ok(b, cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, greatest), "side stream") &&
         cuda_ok(b, cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming), "event") &&
         cuda_ok(b, cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming), "event") &&
         cuda_ok(b, cudaEventCreateWithFlags(&b->ev_pruned, cudaEventDisableTiming), "event");
    b->prio_hi = greatest;
    const char* e = getenv("TS_OVERLAP_RELIST");
    if (e && atoi(e) == 0) b->overlap_relist = false;
    e = getenv("TS_BWD_SMALL");
    if (e && atoi(e) == 0) b->bwd_small = false;
  }
  if (ok) ok = cuda_ok(b, cudaFuncSetAttribute(k_relist_small<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sizeof(SmallSmem)), "smem attribute") &&
               cuda_ok(b, cudaFuncSetAttribute(k_relist_small<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sizeof(SmallSmem)), "smem attribute") &&
               cuda_ok(b, cudaFuncSetAttribute(k_pair_small<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(kPairTabBytes + kSmallRecord * kSmallMax)), "smem attribute") &&
               cuda_ok(b, cudaFuncSetAttribute(k_pair_small<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(kPairTabBytes + kSmallRecord * kSmallMax)), "smem attribute") &&
               bwd_attributes(b);
  if (!ok) { ts_batch_destroy(b); return TS_ERR_CUDA; }
  b->dp_host.assign(dp, dp + kMaxPots);
  *out = b;
  return TS_OK;
}

extern "C" ts_status ts_batch_set_potentials(ts_batch* b, const ts_potential* pots, int n_pots) {
  if (!b || !pots || n_pots != b->n_pots) return TS_ERR_INVALID_ARG;
  for (int q = 0; q < n_pots; q++) {
    const ts_potential& P = pots[q];
    const ts_potential& O = b->pots[q];
    if (P.kind != O.kind || P.shift != O.shift || P.cutoff != O.cutoff || P.skin != O.skin ||
        (P.kind == TS_SOFT_SPHERE && P.p[0] != O.p[0]))
      return fail(b, TS_ERR_INVALID_ARG, "only the parameters p may change (and not the soft-sphere sigma)");
  }
  for (int q = 0; q < n_pots; q++) {
    const ts_potential& P = pots[q];
    DevPot& D = b->dp_host[q];
    for (int c = 0; c < 3; c++) { D.pd[c] = P.p[c]; D.pf[c] = (float)P.p[c]; }
    double rc = b->rc[q], phic = 0;
    if (P.shift && P.kind == TS_LJ) { double s = P.p[0] / rc, s6 = s * s * s * s * s * s; phic = 4 * P.p[1] * (s6 * s6 - s6); }
    if (P.shift && P.kind == TS_MORSE) { double e = exp(-P.p[1] * (rc - P.p[2])); phic = P.p[0] * (e * e - 2 * e); }
    D.phicd = phic; D.phicf = (float)phic;
    b->pots[q] = P;
  }
  cudaSetDevice(b->cfg.device);
  if (!cuda_ok(b, cudaMemcpy(b->d_pots, b->dp_host.data(), sizeof(DevPot) * kMaxPots, cudaMemcpyHostToDevice), "pots"))
    return TS_ERR_CUDA;
  if (b->topo_valid) {   // forces at the current positions are stale for every system
    std::vector<int32_t> ones(b->B, 1);
    if (!cuda_ok(b, cudaMemcpy(b->S.dirty, ones.data(), 4 * b->B, cudaMemcpyHostToDevice), "dirty")) return TS_ERR_CUDA;
  }
  return TS_OK;
}

extern "C" ts_status ts_batch_destroy(ts_batch* b) {
  if (!b) return TS_ERR_INVALID_ARG;
  cudaSetDevice(b->cfg.device);
  cudaDeviceSynchronize();
  for (void* p : b->allocations) cudaFree(p);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->ev_pruned) cudaEventDestroy(b->ev_pruned);
  if (b->side) cudaStreamDestroy(b->side);
  for (auto& g : b->graphs) if (g.exec) cudaGraphExecDestroy(g.exec);
  delete b;
  return TS_OK;
}

extern "C" const char* ts_last_error(const ts_batch* b) {
  if (!b) return "null batch";
  return b->last_error.c_str();
}

extern "C" ts_status ts_batch_counters(const ts_batch* b, int64_t* launches, int64_t* relists) {
  if (!b) return TS_ERR_INVALID_ARG;
  if (launches) *launches = b->launches;
  if (relists) {
    int64_t c[4] = {0, 0, 0, 0};
    cudaMemcpy(c, b->d_counters, sizeof c, cudaMemcpyDeviceToHost);
    *relists = c[0];
  }
  return TS_OK;
}

extern "C" ts_status ts_batch_prunes(const ts_batch* b, int64_t* prunes) {
  if (!b || !prunes) return TS_ERR_INVALID_ARG;
  int64_t c[2] = {0, 0};
  if (!cuda_ok(const_cast<ts_batch*>(b), cudaMemcpy(c, b->d_counters, sizeof c, cudaMemcpyDeviceToHost), "d2h"))
    return TS_ERR_CUDA;
  *prunes = c[1];
  return TS_OK;
}

extern "C" ts_status ts_batch_memory_model(const ts_batch* b, double* bytes_per_atom, double* bytes_per_system) {
  if (!b) return TS_ERR_INVALID_ARG;
  size_t a = scratch_bytes(1, 0, 0, b->max_nbrs, b->f64) + 8;   // + one bin per atom
  size_t s = scratch_bytes(0, 1, 27, b->max_nbrs, b->f64) + scratch_bytes(31, 0, 0, b->max_nbrs, b->f64);
  if (bytes_per_atom) *bytes_per_atom = (double)a;
  if (bytes_per_system) *bytes_per_system = (double)s;
  return TS_OK;
}

extern "C" ts_status ts_batch_poll(ts_batch* b, void* stream, int timeout_ms) {
  if (!b) return TS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (!cuda_ok(b, cudaEventRecord(b->ev, st), "event record")) return TS_ERR_CUDA;
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t q = cudaEventQuery(b->ev);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) { cuda_ok(b, q, "event query"); return TS_ERR_CUDA; }
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_ms >= 0 && ms > timeout_ms) return TS_ERR_NOT_READY;
  }
  int32_t e = 0;
  if (!cuda_ok(b, cudaMemcpy(&e, b->d_err, sizeof e, cudaMemcpyDeviceToHost), "read error word")) return TS_ERR_CUDA;
  if (e) cudaMemset(b->d_err, 0, sizeof e);
  ts_status st2 = b->sticky;
  b->sticky = TS_OK;
  if (st2 != TS_OK) return st2;
  if (e & kErrBadSystemIdx) return fail(b, TS_ERR_INVALID_ARG, "system_idx is not non-decreasing or a system is empty");
  if (e & kErrNeighborOverflow) return fail(b, TS_ERR_NEIGHBOR_OVERFLOW, "an atom has more neighbours than max_neighbors");
  if (e & kErrUnsupported)
    return fail(b, TS_ERR_UNSUPPORTED, "cell outside the supported range, or variable-cell FIRE with a non-periodic axis");
  if (e & kErrNonFinite) return fail(b, TS_ERR_NONFINITE, "non-finite or out-of-range position or cell");
  if (e & kErrTimeout) return fail(b, TS_ERR_TIMEOUT, "a bounded device wait ran out");
  return TS_OK;
}

// ---------------------------------------------------------------------------
namespace ts {

// Derive the batch layout from system_idx: per-system caller offsets, padded
// segments, warp ranges and bin reservations.  One device->host copy.
ts_status derive_topology(ts_batch* b, const ts_state* s, cudaStream_t st) {
  int32_t B = s->n_systems;
  int64_t N = s->n_atoms;
  if (B < 1 || N < 1 || B > b->Bcap || N > b->cfg.atom_capacity)
    return fail(b, TS_ERR_BUDGET, "state exceeds the batch capacity");
  if (!cuda_ok(b, cudaMemsetAsync(b->d_starts, 0xff, sizeof(int64_t) * (B + 1), st), "memset")) return TS_ERR_CUDA;
  k_sys_bounds<<<grid_for(N, 256), 256, 0, st>>>(N, s->system_idx, B, b->d_starts, b->d_err);
  b->launches++;
  std::vector<int64_t> starts(B);
  std::vector<int32_t> pot(B);
  int32_t err = 0;
  if (!cuda_ok(b, cudaMemcpyAsync(starts.data(), b->d_starts, sizeof(int64_t) * B, cudaMemcpyDeviceToHost, st), "d2h") ||
      !cuda_ok(b, cudaMemcpyAsync(pot.data(), s->pot_idx, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, st), "d2h") ||
      !cuda_ok(b, cudaMemcpyAsync(&err, b->d_err, sizeof err, cudaMemcpyDeviceToHost, st), "d2h") ||
      !cuda_ok(b, cudaStreamSynchronize(st), "sync"))
    return TS_ERR_CUDA;
  if (err & kErrBadSystemIdx) {
    cudaMemset(b->d_err, 0, 4);
    return fail(b, TS_ERR_INVALID_ARG, "system_idx must be non-decreasing, in range, with every system non-empty");
  }
  std::vector<int64_t> caller_off(B + 1), seg(B);
  std::vector<int32_t> n(B), bin_off(B), bin_cap(B), ws(B), we(B);
  for (int k = 0; k < B; k++) {
    if (starts[k] < 0) return fail(b, TS_ERR_INVALID_ARG, "empty system");
    caller_off[k] = starts[k];
  }
  caller_off[B] = N;
  int64_t slot = 0, bins = 0;
  std::vector<int32_t> warp_sys;
  for (int k = 0; k < B; k++) {
    n[k] = (int32_t)(caller_off[k + 1] - caller_off[k]);
    if (n[k] < 1) return fail(b, TS_ERR_INVALID_ARG, "empty system");
    if (n[k] > (int64_t)kJMask) return fail(b, TS_ERR_UNSUPPORTED, "system larger than 2^22 atoms");
    if (pot[k] < 0 || pot[k] >= b->n_pots) return fail(b, TS_ERR_INVALID_ARG, "pot_idx out of range");
    bin_off[k] = (int32_t)bins;
    bin_cap[k] = std::max<int32_t>(27, n[k]);
    bins += bin_cap[k];
  }
  // Slot layout order: by potential, larger systems first.  The pair
  // kernel's work items are runs of consecutive warps, so they then hold
  // warps of one potential and similar cost.  A system's results do not
  // depend on where its segment lies.
  std::vector<int32_t> lay(B);
  for (int k = 0; k < B; k++) lay[k] = k;
  std::stable_sort(lay.begin(), lay.end(), [&](int a, int c) { return pot[a] != pot[c] ? pot[a] < pot[c] : n[a] > n[c]; });
  for (int k : lay) {
    seg[k] = slot;
    int64_t npad = (n[k] + 31) / 32 * 32;
    ws[k] = (int32_t)(slot / 32);
    slot += npad;
    we[k] = (int32_t)(slot / 32);
    for (int w = ws[k]; w < we[k]; w++) warp_sys.push_back(k);
  }
  if (slot > b->Ncap || bins > b->Ccap) return fail(b, TS_ERR_BUDGET, "padded layout exceeds capacity");
  b->B = B; b->N = N; b->Npad = slot; b->nwarps = (int32_t)(slot / 32); b->nbins = bins;
  b->n_large = 0;
  for (int k = 0; k < B; k++) b->n_large += n[k] > kSmallMax;
  // work items of the shared-memory pair kernel (systems up to kSmallMax atoms):
  // the warps of those systems, in order, cut into runs of at most 8; a run
  // may straddle systems, and stages every system it touches, as long as
  // that staged range stays within kSmallMax slots (otherwise it is cut at
  // the system boundary)
  const int wpi = b->tune.item_warps, cap = kSmallMax / kWarp;
  std::vector<int4> items;
  std::vector<double> work, wmax;
  b->nst_max = 0;
  {
    int first = -1, count = 0, s0 = -1;
    double wk = 0, wm = 0;
    auto flush = [&](int s_last) {
      if (count == 0) return;
      items.push_back(make_int4(ws[s0], we[s_last] - ws[s0], first, count));
      work.push_back(wk);
      wmax.push_back(wm);
      b->nst_max = std::max(b->nst_max, (we[s_last] - ws[s0]) * kWarp);
      count = 0; wk = 0; wm = 0;
    };
    int s_prev = -1;
    for (int k : lay) {   // systems in slot order
      if (n[k] > kSmallMax) { flush(s_prev); continue; }
      // relative cost of a warp-entry: soft-sphere lists are about half as long
      double c = b->pots[pot[k]].kind == TS_SOFT_SPHERE ? 0.5 : (b->pots[pot[k]].kind == TS_MORSE ? 1.1 : 1.0);
      for (int w = ws[k]; w < we[k]; w++) {
        if (count > 0 && (count == wpi || we[k] - ws[s0] > cap)) flush(s_prev);
        if (count == 0) { first = w; s0 = k; }
        count++;
        wk += c * std::min(kWarp, n[k] - (w - ws[k]) * kWarp);
        wm = std::max(wm, c);
        s_prev = k;
      }
    }
    flush(s_prev);
  }
  b->n_items = (int32_t)items.size();
  if (b->n_items > b->Wcap) return fail(b, TS_ERR_BUDGET, "pair work table exceeds capacity");
  {   // The warps of an item run side by side, so a CTA lasts as long as its
      // costliest warp: items with the longest per-atom lists first (any
      // size), then by total work (atoms, soft spheres weighted by half for
      // their shorter lists), so that the launch ends on cheap items
    std::vector<int32_t> order(b->n_items);
    for (int c = 0; c < b->n_items; c++) order[c] = c;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int c) { return wmax[a] != wmax[c] ? wmax[a] > wmax[c] : work[a] > work[c]; });
    std::vector<int4> sorted(b->n_items);
    for (int c = 0; c < b->n_items; c++) sorted[c] = items[order[c]];
    items.swap(sorted);
  }
  // each item's warps' systems, read by a CTA beside its item (not through
  // the item's first warp, which would add a dependent load to the prologue)
  std::vector<int32_t> item_sys((size_t)kItemWarps * b->n_items, 0);
  for (int c = 0; c < b->n_items; c++)
    for (int w = 0; w < items[c].w; w++) item_sys[(size_t)kItemWarps * c + w] = warp_sys[items[c].z + w];
  b->h_caller_off = caller_off; b->h_n = n; b->h_pot = pot; b->h_seg = seg;
  SysArrays& S = b->S;
  bool ok = cuda_ok(b, cudaMemcpyAsync(S.seg_start, seg.data(), 8 * B, cudaMemcpyHostToDevice, st), "h2d") &&
            cuda_ok(b, cudaMemcpyAsync(S.n_atoms, n.data(), 4 * B, cudaMemcpyHostToDevice, st), "h2d") &&
            cuda_ok(b, cudaMemcpyAsync(S.caller_off, caller_off.data(), 8 * (B + 1), cudaMemcpyHostToDevice, st), "h2d") &&
            cuda_ok(b, cudaMemcpyAsync(S.pot, pot.data(), 4 * B, cudaMemcpyHostToDevice, st), "h2d") &&
            cuda_ok(b, cudaMemcpyAsync(S.bin_off, bin_off.data(), 4 * B, cudaMemcpyHostToDevice, st), "h2d") &&
            cuda_ok(b, cudaMemcpyAsync(S.bin_cap, bin_cap.data(), 4 * B, cudaMemcpyHostToDevice, st), "h2d") &&
            cuda_ok(b, cudaMemcpyAsync(S.warp_start, ws.data(), 4 * B, cudaMemcpyHostToDevice, st), "h2d") &&
            cuda_ok(b, cudaMemcpyAsync(S.warp_end, we.data(), 4 * B, cudaMemcpyHostToDevice, st), "h2d") &&
            cuda_ok(b, cudaMemcpyAsync(b->d_warp_sys, warp_sys.data(), 4 * warp_sys.size(), cudaMemcpyHostToDevice, st), "h2d");
  if (ok && b->n_items > 0)
    ok = cuda_ok(b, cudaMemcpyAsync(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, st), "h2d") &&
         cuda_ok(b, cudaMemcpyAsync(b->d_item_sys, item_sys.data(), 4 * item_sys.size(), cudaMemcpyHostToDevice, st), "h2d");
  if (s->uid) {
    ok = ok && cuda_ok(b, cudaMemcpyAsync(S.uid, s->uid, 4 * B, cudaMemcpyDeviceToDevice, st), "d2d");
  } else {
    std::vector<uint32_t> u(B);
    for (int k = 0; k < B; k++) u[k] = (uint32_t)k;
    ok = ok && cuda_ok(b, cudaMemcpyAsync(S.uid, u.data(), 4 * B, cudaMemcpyHostToDevice, st), "h2d") &&
         cuda_ok(b, cudaStreamSynchronize(st), "sync");
  }
  ok = ok && cuda_ok(b, cudaMemsetAsync(b->A.perm, 0xff, 4 * b->Ncap, st), "memset") &&
       cuda_ok(b, cudaMemsetAsync(b->A.sys, 0xff, 4 * b->Ncap, st), "memset");
  if (!ok) return TS_ERR_CUDA;
  k_init_slots<<<B, 128, 0, st>>>(B, S, b->A);
  b->launches++;
  std::vector<int32_t> ones(B, 1);
  ok = cuda_ok(b, cudaMemcpyAsync(S.relist, ones.data(), 4 * B, cudaMemcpyHostToDevice, st), "h2d") &&
       cuda_ok(b, cudaMemcpyAsync(S.dirty, ones.data(), 4 * B, cudaMemcpyHostToDevice, st), "h2d") &&
       cuda_ok(b, cudaMemsetAsync(S.soon, 0, 4 * B, st), "memset") && cuda_ok(b, cudaMemsetAsync(S.any, 0, 4, st), "memset") &&
       cuda_ok(b, cudaMemsetAsync(S.prune, 0, 4 * B, st), "memset") &&
       cuda_ok(b, cudaMemsetAsync(S.geom, 0, 4 * B, st), "memset") &&
       cuda_ok(b, cudaMemsetAsync(b->d_count, 0, 4 * b->Ccap, st), "memset") &&
       cuda_ok(b, cudaStreamSynchronize(st), "sync");
  if (!ok) return TS_ERR_CUDA;
  b->topo_valid = true;
  b->first_import = true;
  b->graphs_valid = false;
  return TS_OK;
}

ts_status check_state(ts_batch* b, const ts_state* s, bool need_vel) {
  if (!b || !s) return TS_ERR_INVALID_ARG;
  if (!s->pos || !s->mass || !s->cell || !s->system_idx || !s->pot_idx || (need_vel && !s->vel))
    return fail(b, TS_ERR_INVALID_ARG, "null state pointer");
  if (s->n_systems < 1 || s->n_atoms < 1) return fail(b, TS_ERR_INVALID_ARG, "empty state");
  return TS_OK;
}

// Per-call prologue: topology (if needed), cell geometry, image shifts,
// position import with dirty / skin flags.
ts_status prologue(ts_batch* b, ts_state* s, cudaStream_t st, bool import_vel, bool fire, bool geometry) {
  cudaSetDevice(b->cfg.device);
  if (!b->topo_valid || s->n_systems != b->B || s->n_atoms != b->N) {
    ts_status r = derive_topology(b, s, st);
    if (r != TS_OK) return r;
  }
  int B = b->B;
  // A cell other than the one the lists were built for: every call but FIRE
  // checks against the listing cell (its skin test has no room for a cell
  // change); FIRE, whose own test budgets the cell change since the listing,
  // checks only for a change made by the caller since the last call.
  // (geometry = false: the caller knows the cell is the one of its previous
  // import, so the geometry and the image shifts stand)
  const int cell_check = b->first_import ? 0 : (fire ? 1 : 2);
  if (geometry || b->first_import) {
    k_geometry<<<(B + 31) / 32, 32, 0, st>>>(B, b->S, s->cell, s->pbc, b->d_pots, b->d_err, cell_check);
    k_shift_table<<<B, 128, 0, st>>>(B, b->S);
    b->launches += 2;
  }
  int g = grid_for(b->Npad, 256);
  const int wv = import_vel ? 1 : 0;   // velocities in the same pass
  if (b->f64) k_import_pos<true><<<g, 256, 0, st>>>(b->Npad, b->S, b->A, s->pos, b->d_pots, !b->first_import, b->d_err, wv, s->vel, s->mass);
  else k_import_pos<false><<<g, 256, 0, st>>>(b->Npad, b->S, b->A, s->pos, b->d_pots, !b->first_import, b->d_err, wv, s->vel, s->mass);
  b->launches++;
  b->first_import = false;
  return cuda_ok(b, cudaGetLastError(), "prologue launch") ? TS_OK : TS_ERR_CUDA;
}

// Re-list every flagged system: bin, counting sort (canonical order inside a
// bin), state move, explicit list.  Kernels skip unflagged systems, so the
// sequence is safe to issue every step (and to capture in a graph).
void relist_sort(ts_batch* b, cudaStream_t st, bool move_fire, int prio) {
  int B = b->B;
  // systems of up to kSmallMax atoms: bin and sort, one CTA per system, plus
  // one CTA that writes the list-build work table
  if (b->f64)
    launch_k(st, prio, B + 1, kSmallThreads, sizeof(SmallSmem), k_relist_small<true>, B, b->S, b->A, b->Ncap,
             (int)move_fire, b->d_cstart, b->d_count, (const DevPot*)b->d_pots, b->max_nbrs, b->d_err, b->d_tab_sys,
             b->d_tab_base, b->d_tab_base_a, b->d_tab_n);
  else
    launch_k(st, prio, B + 1, kSmallThreads, sizeof(SmallSmem), k_relist_small<false>, B, b->S, b->A, b->Ncap,
             (int)move_fire, b->d_cstart, b->d_count, (const DevPot*)b->d_pots, b->max_nbrs, b->d_err, b->d_tab_sys,
             b->d_tab_base, b->d_tab_base_a, b->d_tab_n);
  b->launches++;
  if (b->n_large > 0) relist_large_sort(b, st, move_fire);
}

void relist_build(ts_batch* b, cudaStream_t st, int prio) {
  // Verlet lists of the table's warps: a resident grid taking warps from a counter
  int grid = b->n_sm * kBuildCtasPerSm;
  if (b->f64)
    launch_k(st, prio, grid, 128, 0, k_build_list_warp<true>, b->S, b->A, (const int32_t*)b->d_tab_sys,
             (const int32_t*)b->d_tab_base, (const int32_t*)b->d_tab_base_a, b->d_tab_n, (const int32_t*)b->d_cstart, (const int32_t*)b->d_count,
             (const DevPot*)b->d_pots, b->max_nbrs, b->Ncap, b->d_err);
  else
    launch_k(st, prio, grid, 128, 0, k_build_list_warp<false>, b->S, b->A, (const int32_t*)b->d_tab_sys,
             (const int32_t*)b->d_tab_base, (const int32_t*)b->d_tab_base_a, b->d_tab_n, (const int32_t*)b->d_cstart, (const int32_t*)b->d_count,
             (const DevPot*)b->d_pots, b->max_nbrs, b->Ncap, b->d_err);
  b->launches++;
}

void relist_lists(ts_batch* b, cudaStream_t st, bool move_fire, int prio) {
  relist_sort(b, st, move_fire, prio);
  relist_build(b, st, prio);
}

// end of a re-listing pass: flag bookkeeping.  md_pass: the pass's pair
// launches ran in inner-list mode and refreshed every flagged system.
void relist_finish(ts_batch* b, cudaStream_t st, bool md_pass, bool overlap) {
  // one CTA up to 1024 systems (the end-of-pass flag clear then needs no
  // cross-CTA arrival), CTAs of 128 above; after a programmatically
  // serialized pair launch, launched the same way: resident early, it waits
  // in griddepcontrol.wait for that launch to complete
  const int t = b->B <= 1024 ? std::max(32, (b->B + 31) / 32 * 32) : 128;
  if (overlap)
    launch_k_overlap(st, (b->B + t - 1) / t, t, 0, k_after_relist, b->B, b->S, b->d_counters, md_pass ? 1 : 0);
  else
    k_after_relist<<<(b->B + t - 1) / t, t, 0, st>>>(b->B, b->S, b->d_counters, md_pass ? 1 : 0);
  b->launches++;
}

void relist(ts_batch* b, cudaStream_t st, bool move_fire) {
  relist_lists(b, st, move_fire);
  relist_finish(b, st, false);
}

// Re-listing pass and pair forces with the re-listing off the critical path.
// The systems that keep their lists get their forces on `st` while the
// flagged ones are re-sorted, re-listed and get theirs on the side stream
// (highest priority, so that its latency-bound kernels are dispatched ahead
// of the pair kernel's pending CTAs).  The two halves touch disjoint systems:
// the sort moves only flagged systems' slots, and a pair CTA that stages a
// flagged neighbour system's positions while they move never reads them.  In
// a step that re-lists nothing the side stream's launches find no work, and
// they overlap the pair forces.  Returns false (nothing issued) when the
// overlap is off or `st` is the legacy default stream.
// In MD steps (inner lists) the systems that keep their lists split once
// more: those that re-filter their inner list in this step run the longer
// Verlet-list loop, so they are launched first and the steady systems'
// launch follows with programmatic serialization: its CTAs are dispatched
// once every CTA of the first launch is resident, so the long warps start in
// the first wave instead of ending the step.  The bookkeeping waits for both
// through an event recorded after the first.
bool relist_pair_overlapped(ts_batch* b, cudaStream_t st, bool move_fire, bool ew, bool inner) {
  if (!b->overlap_relist || !b->side || st == nullptr) return false;
  if (!cuda_ok(b, cudaEventRecord(b->ev_fork, st), "event record") ||
      !cuda_ok(b, cudaStreamWaitEvent(b->side, b->ev_fork, 0), "stream wait"))
    return false;
  relist_sort(b, b->side, move_fire, b->prio_hi);
  relist_build(b, b->side, b->prio_hi);
  pair(b, b->side, ew, kPairRelisted, b->prio_hi, inner);
  cuda_ok(b, cudaEventRecord(b->ev_join, b->side), "event record");
  if (inner && b->ev_pruned) {
    pair(b, st, ew, kPairPruned, 0, inner);
    cuda_ok(b, cudaEventRecord(b->ev_pruned, st), "event record");
    pair(b, st, ew, kPairSteady, 0, inner, true);
    cuda_ok(b, cudaStreamWaitEvent(st, b->ev_pruned, 0), "stream wait");
  } else {
    pair(b, st, ew, kPairKept, 0, inner);
  }
  cuda_ok(b, cudaStreamWaitEvent(st, b->ev_join, 0), "stream wait");
  relist_finish(b, st, inner, inner && b->ev_pruned);
  return true;
}

// systems above kSmallMax atoms: global counting sort over all bins
void relist_large_sort(ts_batch* b, cudaStream_t st, bool move_fire) {
  int B = b->B;
  int64_t Np = b->Npad, nb = b->nbins;
  int g = grid_for(Np, 256);
  k_zero_bins<<<B, 256, 0, st>>>(B, b->S, b->d_count);
  if (b->f64) k_bin_atoms<true><<<g, 256, 0, st>>>(Np, b->S, b->A, b->d_count);
  else k_bin_atoms<false><<<g, 256, 0, st>>>(Np, b->S, b->A, b->d_count);
  int nblk = (int)((nb + 1023) / 1024);
  k_scan_block<<<nblk, 1024, 0, st>>>(nb, b->d_count, b->d_cstart, b->d_bsum);
  k_scan_sums<<<1, 1024, 0, st>>>(nblk, b->d_bsum);
  k_scan_add<<<nblk, 1024, 0, st>>>(nb, b->d_cstart, b->d_bsum);
  k_scatter_ids<<<g, 256, 0, st>>>(Np, b->S, b->A, b->d_cstart);
  if (b->f64) {
    k_final_slot<true><<<g, 256, 0, st>>>(Np, b->S, b->A, b->d_cstart, b->d_count, move_fire);
    k_copy_back<true><<<g, 256, 0, st>>>(Np, b->S, b->A, move_fire);
  } else {
    k_final_slot<false><<<g, 256, 0, st>>>(Np, b->S, b->A, b->d_cstart, b->d_count, move_fire);
    k_copy_back<false><<<g, 256, 0, st>>>(Np, b->S, b->A, move_fire);
  }
  b->launches += 9;
}

void pair(ts_batch* b, cudaStream_t st, bool ew, int filter, int prio, bool inner, bool overlap) {
  const int in = inner ? 1 : 0;
  int threads = b->pair_threads;
  int blocks = (int)(((int64_t)b->nwarps * 32 + threads - 1) / threads);
  const DevPot* pots = b->d_pots;
  const int32_t* ws = b->d_warp_sys;
  if (b->f64) {
    if (overlap) {
      if (ew) launch_k_overlap(st, blocks, threads, 0, k_pair<true, true>, b->nwarps, ws, b->S, b->A, pots, b->Ncap, filter, b->d_partial, 0, in);
      else launch_k_overlap(st, blocks, threads, 0, k_pair<true, false>, b->nwarps, ws, b->S, b->A, pots, b->Ncap, filter, b->d_partial, 0, in);
    } else {
      if (ew) launch_k(st, prio, blocks, threads, 0, k_pair<true, true>, b->nwarps, ws, b->S, b->A, pots, b->Ncap, filter, b->d_partial, 0, in);
      else launch_k(st, prio, blocks, threads, 0, k_pair<true, false>, b->nwarps, ws, b->S, b->A, pots, b->Ncap, filter, b->d_partial, 0, in);
    }
    b->launches++;
    return;
  }
  // mixed precision: systems up to kSmallMax atoms from shared memory, larger ones gathered through L1
  bool small = b->use_small_pair && b->n_items > 0;
  if (small) {
    size_t shm = kPairTabBytes + (size_t)kSmallRecord * b->nst_max;
    const int4* it = b->d_items;
    if (overlap) {
      if (ew) launch_k_overlap(st, b->n_items, 32 * b->tune.item_warps, shm, k_pair_small<true>, b->n_items, it, b->d_item_sys, b->S, b->A, pots, b->Ncap, filter, b->d_partial, in);
      else launch_k_overlap(st, b->n_items, 32 * b->tune.item_warps, shm, k_pair_small<false>, b->n_items, it, b->d_item_sys, b->S, b->A, pots, b->Ncap, filter, b->d_partial, in);
    } else {
      if (ew) launch_k(st, prio, b->n_items, 32 * b->tune.item_warps, shm, k_pair_small<true>, b->n_items, it, b->d_item_sys, b->S, b->A, pots, b->Ncap, filter, b->d_partial, in);
      else launch_k(st, prio, b->n_items, 32 * b->tune.item_warps, shm, k_pair_small<false>, b->n_items, it, b->d_item_sys, b->S, b->A, pots, b->Ncap, filter, b->d_partial, in);
    }
    b->launches++;
  }
  if (!small || b->n_large > 0) {
    int sk = small ? 1 : 0;
    if (overlap && !small) {
      if (ew) launch_k_overlap(st, blocks, threads, 0, k_pair<false, true>, b->nwarps, ws, b->S, b->A, pots, b->Ncap, filter, b->d_partial, sk, in);
      else launch_k_overlap(st, blocks, threads, 0, k_pair<false, false>, b->nwarps, ws, b->S, b->A, pots, b->Ncap, filter, b->d_partial, sk, in);
    } else {
      if (ew) launch_k(st, prio, blocks, threads, 0, k_pair<false, true>, b->nwarps, ws, b->S, b->A, pots, b->Ncap, filter, b->d_partial, sk, in);
      else launch_k(st, prio, blocks, threads, 0, k_pair<false, false>, b->nwarps, ws, b->S, b->A, pots, b->Ncap, filter, b->d_partial, sk, in);
    }
    b->launches++;
  }
}

void reduce_sys(ts_batch* b, cudaStream_t st, double* E, double* stress, double* KE) {
  int B = b->B;
  k_reduce_sys<<<(B * 32 + 127) / 128, 128, 0, st>>>(B, b->S, b->d_partial, E, stress, KE, b->d_Eint, b->d_Wint);
  b->launches++;
}

void clear_dirty(ts_batch* b, cudaStream_t st) {
  k_clear_dirty<<<(b->B + 127) / 128, 128, 0, st>>>(b->B, b->S);
  b->launches++;
}

void export_state(ts_batch* b, cudaStream_t st, double* pos, double* vel) {
  int g = grid_for(b->Npad, 256);
  if (b->f64) k_export_state<true><<<g, 256, 0, st>>>(b->Npad, b->A, pos, vel);
  else k_export_state<false><<<g, 256, 0, st>>>(b->Npad, b->A, pos, vel);
  b->launches++;
}

void export_forces(ts_batch* b, cudaStream_t st, double* F) {
  int g = grid_for(b->Npad, 256);
  if (b->f64) k_export_forces<true><<<g, 256, 0, st>>>(b->Npad, b->A, F);
  else k_export_forces<false><<<g, 256, 0, st>>>(b->Npad, b->A, F);
  b->launches++;
}

// forces current for every system at the current positions
void ensure_forces(ts_batch* b, cudaStream_t st) {
  relist(b, st, false);
  pair(b, st, true, true);
  clear_dirty(b, st);
}

}  // namespace ts

extern "C" ts_status ts_neighbor_build(ts_batch* b, ts_state* s, int force_rebuild, void* stream) {
  ts_status r = check_state(b, s, false);
  if (r != TS_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  if (force_rebuild) b->topo_valid = false;
  r = prologue(b, s, st, false);
  if (r != TS_OK) return r;
  relist(b, st, false);
  export_state(b, st, s->pos, nullptr);
  return cuda_ok(b, cudaGetLastError(), "ts_neighbor_build") ? TS_OK : TS_ERR_CUDA;
}

extern "C" ts_status ts_pair_forces(ts_batch* b, ts_state* s, double* F, double* E, double* stress, void* stream) {
  ts_status r = check_state(b, s, false);
  if (r != TS_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  r = prologue(b, s, st, false);
  if (r != TS_OK) return r;
  relist(b, st, false);
  pair(b, st, true, false);
  reduce_sys(b, st, E, stress, nullptr);
  if (F) export_forces(b, st, F);
  export_state(b, st, s->pos, nullptr);
  clear_dirty(b, st);
  return cuda_ok(b, cudaGetLastError(), "ts_pair_forces") ? TS_OK : TS_ERR_CUDA;
}

namespace ts {

// ts_md_step, and ts_md_record with frames != nullptr
static ts_status md_call(ts_batch* b, ts_state* s, const ts_md_params* p, int n_steps, double* E, double* KE,
                         double* frames, void* stream) {
  ts_status r = check_state(b, s, true);
  if (r != TS_OK) return r;
  if (!p || n_steps < 0 || !(p->dt > 0) ||
      (p->kind != TS_NVE && p->kind != TS_LANGEVIN && p->kind != TS_NVT_NHC && p->kind != TS_NPT_LANGEVIN) ||
      (p->kind == TS_LANGEVIN && (!p->kT || !(p->gamma >= 0))) ||
      (p->kind == TS_NVT_NHC && (!p->kT || !p->nhc || !(p->tau > 0))) ||
      (p->kind == TS_NPT_LANGEVIN &&
       (!p->kT || !p->baro || !(p->tau > 0) || !(p->gamma >= 0) || !std::isfinite(p->p_ext))))
    return fail(b, TS_ERR_INVALID_ARG, "bad MD parameters");
  const bool npt = p->kind == TS_NPT_LANGEVIN;
  cudaStream_t st = (cudaStream_t)stream;
  r = prologue(b, s, st, true);
  if (r != TS_OK) return r;
  if (p->kind != TS_NVE &&
      !cuda_ok(b, cudaMemcpyAsync(b->S.kT, p->kT, 8 * b->B, cudaMemcpyDeviceToDevice, st), "kT"))
    return TS_ERR_CUDA;
  // the chain state lives in batch memory during the call (the step loop is
  // captured once as a graph, with fixed pointers)
  if (p->kind == TS_NVT_NHC &&
      !cuda_ok(b, cudaMemcpyAsync(b->d_nhc, p->nhc, 48 * b->B, cudaMemcpyDeviceToDevice, st), "nhc"))
    return TS_ERR_CUDA;
  if (npt) {   // the piston velocities live in batch memory during the call; every axis periodic
    if (!cuda_ok(b, cudaMemcpyAsync(b->d_baro, p->baro, 8 * b->B, cudaMemcpyDeviceToDevice, st), "baro"))
      return TS_ERR_CUDA;
    k_require_periodic<<<(b->B + 127) / 128, 128, 0, st>>>(b->B, b->S, b->d_err);
    b->launches++;
  }
  double c1 = exp(-p->gamma * p->dt);
  r = md_loop(b, st, p, n_steps, c1, E != nullptr || KE != nullptr, frames);
  if (r != TS_OK) return r;
  if (p->kind == TS_NVT_NHC &&
      !cuda_ok(b, cudaMemcpyAsync(p->nhc, b->d_nhc, 48 * b->B, cudaMemcpyDeviceToDevice, st), "nhc"))
    return TS_ERR_CUDA;
  if (npt && (!cuda_ok(b, cudaMemcpyAsync(p->baro, b->d_baro, 8 * b->B, cudaMemcpyDeviceToDevice, st), "baro") ||
              !cuda_ok(b, cudaMemcpyAsync(s->cell, b->S.h, 72 * b->B, cudaMemcpyDeviceToDevice, st), "cell")))
    return TS_ERR_CUDA;
  reduce_sys(b, st, E, nullptr, KE);
  export_state(b, st, s->pos, s->vel);
  return cuda_ok(b, cudaGetLastError(), frames ? "ts_md_record" : "ts_md_step") ? TS_OK : TS_ERR_CUDA;
}

}  // namespace ts

extern "C" ts_status ts_md_step(ts_batch* b, ts_state* s, const ts_md_params* p, int n_steps, double* E, double* KE,
                                void* stream) {
  return md_call(b, s, p, n_steps, E, KE, nullptr, stream);
}

extern "C" ts_status ts_md_record(ts_batch* b, ts_state* s, const ts_md_params* p, int n_steps, double* frames,
                                  void* stream) {
  if (!b) return TS_ERR_INVALID_ARG;
  if (!frames || n_steps < 1) return fail(b, TS_ERR_INVALID_ARG, "null frames or no steps");
  if (p && p->kind == TS_NPT_LANGEVIN) return fail(b, TS_ERR_INVALID_ARG, "NPT changes the cell: not recorded");
  return md_call(b, s, p, n_steps, nullptr, nullptr, frames, stream);
}

extern "C" ts_status ts_neighbor_export(ts_batch* b, int32_t* j_out, int32_t* img_out, int32_t* count_out, void* stream) {
  if (!b || !j_out || !img_out || !count_out) return TS_ERR_INVALID_ARG;
  if (!b->topo_valid) return fail(b, TS_ERR_INVALID_ARG, "no neighbour lists yet");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t blocks = (b->Npad + 127) / 128;
  k_export_list<<<(int)(blocks < 1 ? 1 : blocks), 128, 0, st>>>(b->Npad, b->S, b->A, b->max_nbrs, b->Ncap, j_out,
                                                                 img_out, count_out);
  b->launches++;
  return cuda_ok(b, cudaGetLastError(), "ts_neighbor_export") ? TS_OK : TS_ERR_CUDA;
}

extern "C" int32_t ts_batch_max_neighbors(const ts_batch* b) { return b ? b->max_nbrs : 0; }

extern "C" ts_status ts_profile_pair(ts_batch* b, ts_state* s, int reps, void* flush_buf, size_t flush_bytes,
                                     double* ms_out, int64_t* pairs_out, int64_t* atoms_out, void* stream) {
  ts_status r = check_state(b, s, false);
  if (r != TS_OK) return r;
  if (reps < 1 || !ms_out) return fail(b, TS_ERR_INVALID_ARG, "reps < 1 or null output");
  cudaStream_t st = (cudaStream_t)stream;
  r = prologue(b, s, st, false);
  if (r != TS_OK) return r;
  ensure_forces(b, st);
  // inner lists at the current positions for every system (one refreshing launch)
  if (!cuda_ok(b, cudaMemsetAsync(b->S.prune, 1, 4 * (size_t)b->B, st), "memset")) return TS_ERR_CUDA;
  pair(b, st, false, kPairAll, 0, true);
  if (!cuda_ok(b, cudaMemsetAsync(b->S.prune, 0, 4 * (size_t)b->B, st), "memset")) return TS_ERR_CUDA;
  // every launch between its own pair of events, all enqueued before the
  // first is waited for: the stream is busy (the refreshing launch above, the
  // previous launch or the flush) while the host submits the next, so no
  // event pair includes the host's launch latency
  std::vector<cudaEvent_t> ev(2 * (size_t)reps, nullptr);
  bool ok = true;
  for (auto& e : ev) ok = ok && cuda_ok(b, cudaEventCreate(&e), "event");
  for (int k = 0; ok && k < reps; k++) {
    if (flush_buf && flush_bytes) cudaMemsetAsync(flush_buf, k & 0xff, flush_bytes, st);
    cudaEventRecord(ev[2 * k], st);
    pair(b, st, false, kPairAll, 0, true);
    cudaEventRecord(ev[2 * k + 1], st);
  }
  double total = 0;
  if (ok) ok = cuda_ok(b, cudaEventSynchronize(ev[2 * (size_t)reps - 1]), "event sync");
  for (int k = 0; ok && k < reps; k++) {
    float ms = 0;
    ok = cuda_ok(b, cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]), "event time");
    total += ms;
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (!ok) return TS_ERR_CUDA;
  *ms_out = total / reps;
  if (pairs_out) {
    unsigned long long* d = (unsigned long long*)b->d_counters + 2;
    unsigned long long h = 0;
    cudaMemsetAsync(d, 0, 8, st);
    k_count_pairs<<<(int)(((int64_t)b->nwarps * 32 + 127) / 128), 128, 0, st>>>(b->nwarps, b->d_warp_sys, b->S, b->A,
                                                                                 b->d_pots, b->Ncap, b->f64, d);
    b->launches++;
    if (!cuda_ok(b, cudaMemcpyAsync(&h, d, 8, cudaMemcpyDeviceToHost, st), "d2h") ||
        !cuda_ok(b, cudaStreamSynchronize(st), "sync"))
      return TS_ERR_CUDA;
    *pairs_out = (int64_t)h;
  }
  if (atoms_out) *atoms_out = b->N;
  return cuda_ok(b, cudaGetLastError(), "ts_profile_pair") ? TS_OK : TS_ERR_CUDA;
}
