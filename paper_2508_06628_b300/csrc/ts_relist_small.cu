// ts_relist_small.cu -- re-listing in two launches for every flagged system:
// (A) k_relist_small: one CTA per flagged small system (n <= kSmallMax) bins
//     and sorts the system in shared memory:
//   1. wrap positions into the cell (by a whole lattice vector, from the
//      image-shift table), bin them, count per bin;
//   2. exclusive scan of the bin counts; provisional scatter; canonical rank
//      inside each bin (ascending caller index, the same order as the
//      multi-kernel path of ts_neighbor.cu used for larger systems);
//   3. move the per-slot state into the new order (the CTA owns the whole
//      segment, so a barrier separates all reads from all writes) and
//      publish the bin starts in the layout the multi-kernel path uses.
//     One extra CTA writes the work table of (B): the flagged systems in
//     system order, with the exclusive prefix of their warps.
// (B) k_build_list_warp: the Verlet list of every atom of those systems, one
//     warp per 32 sorted atoms: the warp walks the union of its lanes'
//     stencils, stages each bin's atoms through shared memory in coalesced
//     chunks of 32, and every lane tests its own atom against each staged
//     candidate (broadcast reads, so the loads and the image shift of a
//     candidate are shared by 32 atoms).  Each lane visits its stencil bins
//     in the same order as a per-atom loop would, so the list order is
//     canonical.
#include "ts_kernels.cuh"

namespace ts {

constexpr int kSmallThreads = 512;
constexpr int kBuildCtasPerSm = 5;   // grid of k_build_list_warp: resident CTAs of 128 threads per SM (96 registers)
// Passes that re-list at most this many atoms build one warp per atom (short
// dependency chains); larger passes one warp per 32 atoms (fewer instructions).
constexpr int kAtomModeMaxAtoms = 32768;

struct SmallSmem {
  int32_t bin_old[kSmallMax];
  int32_t pid[kSmallMax];   // caller index, old order
  int32_t start[kSmallMax + 1];
  int32_t fill[kSmallMax];
  int32_t tmp[kSmallMax];   // provisional order, then bin of the new slot
  int32_t warp_tot[kSmallThreads / 32];
};

// block-wide exclusive scan of n <= kSmallMax counts held in `a` (in place);
// returns the total
__device__ int block_exclusive_scan(int32_t* a, int n, int32_t* warp_tot) {
  constexpr int per = kSmallMax / kSmallThreads;   // 8 entries per thread
  int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  int base = t * per;
  int loc[per], sum = 0;
#pragma unroll
  for (int q = 0; q < per; q++) { loc[q] = (base + q < n) ? a[base + q] : 0; sum += loc[q]; }
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) { int v = __shfl_up_sync(0xffffffffu, incl, o); if (lane >= o) incl += v; }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int v = lane < kSmallThreads / 32 ? warp_tot[lane] : 0, inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) { int u = __shfl_up_sync(0xffffffffu, inc, o); if (lane >= o) inc += u; }
    if (lane < kSmallThreads / 32) warp_tot[lane] = inc - v;
  }
  __syncthreads();
  int run = warp_tot[wid] + incl - sum;
#pragma unroll
  for (int q = 0; q < per; q++) { if (base + q < n) a[base + q] = run; run += loc[q]; }
  __syncthreads();
  int total = 0;
  if (n > 0) total = a[n - 1] + ((n - 1) / per == t ? loc[(n - 1) % per] : 0);
  // broadcast the total from the owner of the last entry
  __shared__ int s_total;
  if (n > 0 && (n - 1) / per == t) s_total = total;
  __syncthreads();
  return n > 0 ? s_total : 0;
}

// Work table of k_build_list_warp (one CTA): entries e = 0..ne-1 are the
// flagged systems in system order; tab_base[e] / tab_base_a[e] count their
// warps (32-slot groups) / atoms before entry e, [ne] the totals;
// tab_n = {ne, work counter of the build, build mode}.
__device__ void relist_table(int32_t B, const SysArrays& S, SmallSmem& sm, int32_t* tab_sys, int32_t* tab_base,
                             int32_t* tab_base_a, int32_t* tab_n) {
  const int t = threadIdx.x;
  int ecarry = 0, wcarry = 0, acarry = 0;
  for (int c0 = 0; c0 < B; c0 += kSmallMax) {
    const int m = min(kSmallMax, B - c0);
    for (int i = t; i < m; i += kSmallThreads) {
      int s = c0 + i;
      bool f = need_relist(S, s);
      sm.tmp[i] = f;
      sm.start[i] = f;
      sm.fill[i] = f ? S.warp_end[s] - S.warp_start[s] : 0;
      sm.pid[i] = f ? S.n_atoms[s] : 0;
    }
    __syncthreads();
    int ne = block_exclusive_scan(sm.start, m, sm.warp_tot);
    int nw = block_exclusive_scan(sm.fill, m, sm.warp_tot);
    int na = block_exclusive_scan(sm.pid, m, sm.warp_tot);
    for (int i = t; i < m; i += kSmallThreads)
      if (sm.tmp[i]) {
        tab_sys[ecarry + sm.start[i]] = c0 + i;
        tab_base[ecarry + sm.start[i]] = wcarry + sm.fill[i];
        tab_base_a[ecarry + sm.start[i]] = acarry + sm.pid[i];
      }
    ecarry += ne;
    wcarry += nw;
    acarry += na;
    __syncthreads();
  }
  if (t == 0) {
    tab_base[ecarry] = wcarry;
    tab_base_a[ecarry] = acarry;
    tab_n[0] = ecarry;
    tab_n[1] = 0;                               // work counter of the build
    tab_n[2] = acarry <= kAtomModeMaxAtoms;     // build mode: one warp per atom for small passes
  }
}

template <bool F64>
__global__ void __launch_bounds__(kSmallThreads, 2)   // at most 64 registers: fits beside pair CTAs
k_relist_small(int32_t B, SysArrays S, SlotArrays A, int64_t stride, int move_fire, int32_t* cstart, int32_t* count,
               const DevPot* __restrict__ pots, int32_t max_nbrs, int32_t* err, int32_t* tab_sys, int32_t* tab_base,
               int32_t* tab_base_a, int32_t* tab_n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmallSmem& sm = *reinterpret_cast<SmallSmem*>(smem_raw);
  int s = blockIdx.x;
  if (s == B) { relist_table(B, S, sm, tab_sys, tab_base, tab_base_a, tab_n); return; }   // the extra CTA
  if (s > B || !need_relist(S, s)) return;
  int n = S.n_atoms[s];
  if (n > kSmallMax) return;
  int t = threadIdx.x;
  int64_t seg = S.seg_start[s];
  const double* g = S.hinv + 9 * s;
  const double* h = S.h + 9 * s;
  const int nb0 = S.nb[3 * s], nb1 = S.nb[3 * s + 1], nb2 = S.nb[3 * s + 2];
  int nbins = nb0 * nb1 * nb2;
  int boff = S.bin_off[s];
  for (int c = t; c < nbins; c += kSmallThreads) sm.start[c] = 0;
  __syncthreads();
  // 1. wrap, bin, count
  for (int i = t; i < n; i += kSmallThreads) {
    int64_t k = seg + i;
    int kb[3], nbv[3] = {nb0, nb1, nb2};
    bool done = false;
    if constexpr (!F64) {
      float4 hi = A.xh[k], lo = A.xl[k];
      if (wrap_bin_mixed(S, s, hi, lo, kb)) {
        A.tmp_f0[k] = hi; A.tmp_f1[k] = lo;
        done = true;
      }
    }
    if (!done) {
      // FP64 route: FP64 positions, or an atom further out than the image table covers
      double x[3];
      if constexpr (F64) {
        for (int c = 0; c < 3; c++) x[c] = A.xd[3 * k + c];
      } else {
        float4 hi = A.xh[k], lo = A.xl[k];
        x[0] = (double)hi.x + lo.x; x[1] = (double)hi.y + lo.y; x[2] = (double)hi.z + lo.z;
      }
      double f[3];
      const int pm = S.pmask[s];
      for (int a = 0; a < 3; a++) {
        double v = x[0] * g[a] + x[1] * g[3 + a] + x[2] * g[6 + a];
        if (pm >> a & 1) {
          v -= floor(v);
          if (v >= 1.0) v = 0.0;
        }
        f[a] = v;
        int q = (int)floor(v * nbv[a]);
        kb[a] = q >= nbv[a] ? nbv[a] - 1 : (q < 0 ? 0 : q);
      }
      double xw[3];
      for (int c = 0; c < 3; c++) xw[c] = f[0] * h[c] + f[1] * h[3 + c] + f[2] * h[6 + c];
      if constexpr (F64) {
        for (int c = 0; c < 3; c++) A.tmp_d0[3 * k + c] = xw[c];
      } else {
        float4 hi, lo;
        split_pos(xw[0], hi.x, lo.x); split_pos(xw[1], hi.y, lo.y); split_pos(xw[2], hi.z, lo.z);
        hi.w = 0.f; lo.w = 0.f;
        A.tmp_f0[k] = hi; A.tmp_f1[k] = lo;
      }
    }
    int b = (kb[2] * nb1 + kb[1]) * nb0 + kb[0];
    sm.bin_old[i] = b;
    sm.pid[i] = A.perm[k];
    atomicAdd(&sm.start[b], 1);
  }
  __syncthreads();
  // 2. scan, provisional scatter, canonical rank
  block_exclusive_scan(sm.start, nbins, sm.warp_tot);
  if (t == 0) sm.start[nbins] = n;
  for (int c = t; c < nbins; c += kSmallThreads) sm.fill[c] = 0;
  __syncthreads();
  for (int i = t; i < n; i += kSmallThreads) {
    int b = sm.bin_old[i];
    sm.tmp[sm.start[b] + atomicAdd(&sm.fill[b], 1)] = i;
  }
  __syncthreads();
  int newslot[kSmallMax / kSmallThreads];
  int nmine = 0;
  for (int i = t; i < n; i += kSmallThreads) {
    int b = sm.bin_old[i], p = sm.pid[i], r = 0;
    for (int q = sm.start[b]; q < sm.start[b + 1]; q++) r += sm.pid[sm.tmp[q]] < p;
    newslot[nmine++] = sm.start[b] + r;
  }
  __syncthreads();
  // 3. move state: reads of the old order, then writes of the new order
  nmine = 0;
  for (int i = t; i < n; i += kSmallThreads) {
    int d = newslot[nmine++];
    int64_t ko = seg + i, kd = seg + d;
    sm.tmp[d] = sm.bin_old[i];
    A.tmp_i1[kd] = sm.pid[i];
    if constexpr (F64) {
      for (int c = 0; c < 3; c++) A.tmp_d1[3 * kd + c] = A.vd[3 * ko + c];
      A.tmp_d2[kd] = A.minvd[ko];
      if (move_fire) for (int c = 0; c < 3; c++) A.tmp_d2[stride + 3 * kd + c] = A.gd0[3 * ko + c];
    } else {
      A.tmp_f2[kd] = A.vh[ko];
      A.tmp_f3[kd] = A.vl[ko];
      if (move_fire) A.tmp_f0[stride + kd] = A.g0[ko];
      A.xh[kd] = A.tmp_f0[ko];
      A.xl[kd] = A.tmp_f1[ko];
    }
  }
  __syncthreads();
  for (int d = t; d < n; d += kSmallThreads) {
    int64_t kd = seg + d;
    A.perm[kd] = A.tmp_i1[kd];
    A.bin[kd] = boff + sm.tmp[d];
    if constexpr (F64) {
      for (int c = 0; c < 3; c++) A.vd[3 * kd + c] = A.tmp_d1[3 * kd + c];
      A.minvd[kd] = A.tmp_d2[kd];
      if (move_fire) for (int c = 0; c < 3; c++) A.gd0[3 * kd + c] = A.tmp_d2[stride + 3 * kd + c];
    } else {
      A.vh[kd] = A.tmp_f2[kd];
      A.vl[kd] = A.tmp_f3[kd];
      if (move_fire) A.g0[kd] = A.tmp_f0[stride + kd];
    }
  }
  if constexpr (F64) {
    // FP64 positions: new order from the wrapped copy (old-order tmp_d0); the
    // loop above read no xd, so write them after the barrier
    __syncthreads();
    nmine = 0;
    for (int i = t; i < n; i += kSmallThreads) {
      int d = newslot[nmine++];
      for (int c = 0; c < 3; c++) A.xd[3 * (seg + d) + c] = A.tmp_d0[3 * (seg + i) + c];
    }
  }
  // bin starts and counts in the multi-kernel layout: the scan at a
  // system's first bin equals its caller offset
  int64_t coff = S.caller_off[s];
  for (int c = t; c < nbins; c += kSmallThreads) {
    cstart[boff + c] = (int32_t)(coff + sm.start[c]);
    count[boff + c] = sm.start[c + 1] - sm.start[c];
  }
}

// floor(a / b) for b > 0; stencil coordinates lie within a cell width or
// two of the cell, so the common cases take no integer division
__device__ __forceinline__ int floor_div(int a, int b) {
  if (a >= 0) return a < b ? 0 : (a < 2 * b ? 1 : a / b);
  return a >= -b ? -1 : -((-a + b - 1) / b);
}

// One warp: the lists of the 32 slots of warp `wi` of system `s` (a flagged
// system).  sh_h / sh_d: this warp's staging area.
template <bool F64>
__device__ void build_warp(int s, int wi, const SysArrays& S, const SlotArrays& A, const int32_t* __restrict__ cstart,
                           const int32_t* __restrict__ count, const DevPot* __restrict__ pots, int32_t max_nbrs,
                           int64_t stride, int32_t* err, float4* sh_h, double (*sh_d)[3]) {
  const int lane = threadIdx.x & 31;
  const int w = S.warp_start[s] + wi;
  int64_t k = (int64_t)w * kWarp + lane;
  bool valid = A.perm[k] >= 0;   // lane 0 of a warp is always a real atom
  const DevPot& P = pots[S.pot[s]];
  const int nb0 = S.nb[3 * s], nb1 = S.nb[3 * s + 1], nb2 = S.nb[3 * s + 2];
  const int m0 = S.reach[3 * s], m1 = S.reach[3 * s + 1], m2 = S.reach[3 * s + 2];
  const int pm = S.pmask[s];
  int64_t seg = S.seg_start[s];
  int boff = S.bin_off[s];
  int lbr = A.bin[k] - boff;                                   // padding lanes: any value
  int lb = __shfl_sync(0xffffffffu, lbr, valid ? lane : 0);    // ... replaced by lane 0's bin
  int kx = lb % nb0, ky = (lb / nb0) % nb1, kz = lb / (nb0 * nb1);
  // union of the lanes' stencils, in unwrapped bin coordinates
  int x0 = __reduce_min_sync(0xffffffffu, kx) - m0, x1 = __reduce_max_sync(0xffffffffu, kx) + m0;
  int y0 = __reduce_min_sync(0xffffffffu, ky) - m1, y1 = __reduce_max_sync(0xffffffffu, ky) + m1;
  int z0 = __reduce_min_sync(0xffffffffu, kz) - m2, z1 = __reduce_max_sync(0xffffffffu, kz) + m2;
  float4 hi = make_float4(0, 0, 0, 0), lo = hi;
  double xi[3] = {0, 0, 0};
  if (valid) {
    if constexpr (F64) { for (int c = 0; c < 3; c++) xi[c] = A.xd[3 * k + c]; }
    else { hi = A.xh[k]; lo = A.xl[k]; }
  }
  int cnt = 0;
  const int nx = x1 - x0 + 1, ny = y1 - y0 + 1, ncell = nx * ny * (z1 - z0 + 1);
  const int64_t coff = S.caller_off[s];
  // bounding box of the warp's atoms (hi parts; padding lanes take lane 0's
  // atom): a staged candidate farther than r_list + 1e-3 A from it is no
  // lane's neighbour and is dropped before the per-lane tests
  float3 bb_lo = make_float3(0.f, 0.f, 0.f), bb_hi = bb_lo;
  if constexpr (!F64) {
    float bx = __shfl_sync(0xffffffffu, hi.x, valid ? lane : 0), by = __shfl_sync(0xffffffffu, hi.y, valid ? lane : 0),
          bz = __shfl_sync(0xffffffffu, hi.z, valid ? lane : 0);
    bb_lo = make_float3(bx, by, bz); bb_hi = bb_lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      bb_lo.x = fminf(bb_lo.x, __shfl_xor_sync(0xffffffffu, bb_lo.x, o));
      bb_lo.y = fminf(bb_lo.y, __shfl_xor_sync(0xffffffffu, bb_lo.y, o));
      bb_lo.z = fminf(bb_lo.z, __shfl_xor_sync(0xffffffffu, bb_lo.z, o));
      bb_hi.x = fmaxf(bb_hi.x, __shfl_xor_sync(0xffffffffu, bb_hi.x, o));
      bb_hi.y = fmaxf(bb_hi.y, __shfl_xor_sync(0xffffffffu, bb_hi.y, o));
      bb_hi.z = fmaxf(bb_hi.z, __shfl_xor_sync(0xffffffffu, bb_hi.z, o));
    }
  }
  const unsigned lanes_below = (1u << lane) - 1u;
  // cells in (z, y, x) order, 32 at a time: each lane resolves one cell's
  // bin start, count, image code and shift, then the warp walks them in order
  for (int cb = 0; cb < ncell; cb += 32) {
    int my_start = 0, my_count = 0, my_code = 0;
    float4 my_sh = make_float4(0, 0, 0, 0), my_sl = my_sh;
    {
      int ci = cb + lane;
      if (ci < ncell) {
        int cx = x0 + ci % nx, cy = y0 + (ci / nx) % ny, cz = z0 + ci / (nx * ny);
        int ix = floor_div(cx, nb0), iy = floor_div(cy, nb1), iz = floor_div(cz, nb2);
        int gb = boff + ((cz - iz * nb2) * nb1 + (cy - iy * nb1)) * nb0 + (cx - ix * nb0);
        my_code = img_code(ix, iy, iz);
        // a cell beyond the edge of a non-periodic axis is empty
        const bool open_edge = ((pm & 1) == 0 && ix != 0) || ((pm & 2) == 0 && iy != 0) || ((pm & 4) == 0 && iz != 0);
        my_start = open_edge ? 0 : (int)((int64_t)cstart[gb] - coff);
        my_count = open_edge ? 0 : count[gb];
        if constexpr (!F64) {
          int64_t ti = (int64_t)s * kNCodes + my_code;
          my_sh = S.shift[2 * ti];
          my_sl = S.shift[2 * ti + 1];
        }
      }
    }
    const int ncb = min(32, ncell - cb);
    // coordinates of cell cb, then stepped in (z, y, x) order
    int cx = x0 + cb % nx, cy = y0 + (cb / nx) % ny, cz = z0 + cb / (nx * ny);
    for (int tc = 0; tc < ncb; tc++) {
      if (tc > 0 && ++cx > x1) {
        cx = x0;
        if (++cy > y1) { cy = y0; ++cz; }
      }
      bool in = valid && abs(cz - kz) <= m2 && abs(cy - ky) <= m1 && abs(cx - kx) <= m0;
      int code = __shfl_sync(0xffffffffu, my_code, tc);
      int64_t b0 = seg + __shfl_sync(0xffffffffu, my_start, tc);
      int c = __shfl_sync(0xffffffffu, my_count, tc);
      float a0 = 0, a1 = 0, a2 = 0, e0 = 0, e1 = 0, e2 = 0, cs0 = 0, cs1 = 0, cs2 = 0;
      double s0 = 0, s1 = 0, s2 = 0;
      if constexpr (F64) {
        const double* sd = S.shiftd + 3 * ((int64_t)s * kNCodes + code);
        s0 = sd[0] - xi[0]; s1 = sd[1] - xi[1]; s2 = sd[2] - xi[2];
      } else {
        cs0 = __shfl_sync(0xffffffffu, my_sh.x, tc);   // the cell's image shift (hi)
        cs1 = __shfl_sync(0xffffffffu, my_sh.y, tc);
        cs2 = __shfl_sync(0xffffffffu, my_sh.z, tc);
        a0 = cs0 - hi.x;   // exact (2^-12 grid)
        a1 = cs1 - hi.y;
        a2 = cs2 - hi.z;
        e0 = __shfl_sync(0xffffffffu, my_sl.x, tc) - lo.x;
        e1 = __shfl_sync(0xffffffffu, my_sl.y, tc) - lo.y;
        e2 = __shfl_sync(0xffffffffu, my_sl.z, tc) - lo.z;
      }
      if (!__any_sync(0xffffffffu, in) || c == 0) continue;
      {
        for (int base = 0; base < c; base += 32) {
          int q = base + lane;
          int nc = min(32, c - base);
          unsigned km = 0;   // staged candidates kept by the box test (bit = index in the chunk)
          if constexpr (F64) {
            if (q < c) { for (int cc = 0; cc < 3; cc++) sh_d[lane][cc] = A.xd[3 * (b0 + q) + cc]; }
          } else {
            // stage the candidates near the warp's box, in order, with their
            // list entry in w (lo parts only for the rare undecided tests)
            float4 cj = make_float4(0.f, 0.f, 0.f, 0.f);
            bool keep = false;
            if (q < c) {
              cj = A.xh[b0 + q];
              const float px = cj.x + cs0, py = cj.y + cs1, pz = cj.z + cs2;   // exact (2^-12 grid)
              const float ux = fmaxf(fmaxf(bb_lo.x - px, px - bb_hi.x), 0.f),
                          uy = fmaxf(fmaxf(bb_lo.y - py, py - bb_hi.y), 0.f),
                          uz = fmaxf(fmaxf(bb_lo.z - pz, pz - bb_hi.z), 0.f);
              keep = fmaf(ux, ux, fmaf(uy, uy, uz * uz)) < P.rlist_out2f;
            }
            km = __ballot_sync(0xffffffffu, keep);
            nc = __popc(km);
            if (keep) {
              cj.w = __uint_as_float((uint32_t)(b0 - seg + q) | ((uint32_t)code << kJBits));
              sh_h[__popc(km & lanes_below)] = cj;
            }
          }
          __syncwarp();
          if (in) {
            const uint32_t cbits = (uint32_t)code << kJBits;
            const int j0 = (int)(b0 - seg) + base;                            // local index of candidate 0
            const int self = code == kCenter ? (int)(k - b0) - base : -1;     // the atom itself, if staged here
            auto append = [&](bool hit, int tq) {
              if (hit) {
                if (cnt < max_nbrs) A.nbr[cnt * stride + k] = (uint32_t)(j0 + tq) | cbits;
                cnt++;
              }
            };
            if constexpr (F64) {
              auto test = [&](int tq) -> bool {
                double d0 = sh_d[tq][0] + s0, d1 = sh_d[tq][1] + s1, d2 = sh_d[tq][2] + s2;
                return d0 * d0 + d1 * d1 + d2 * d2 < P.rlist2d && tq != self;
              };
              for (int tq = 0; tq < nc; tq++) append(test(tq), tq);
            } else {
              // hi parts (exact sum on the 2^-12 grid) decide every test but
              // those in a thin shell around the list radius, which take the
              // double-float test; four tests per round, straight-line unless
              // one of them is undecided
              // staged entry t: hi position, index in the chunk in w
              auto rh2 = [&](const float4 xj) {
                const float h0 = xj.x + a0, h1 = xj.y + a1, h2 = xj.z + a2;
                return fmaf(h0, h0, fmaf(h1, h1, h2 * h2));
              };
              auto exact = [&](const float4 xj) {
                const float4 lj = A.xl[seg + (__float_as_uint(xj.w) & kJMask)];
                const float d0 = (xj.x + a0) + (lj.x + e0), d1 = (xj.y + a1) + (lj.y + e1),
                            d2 = (xj.z + a2) + (lj.z + e2);
                return d0 * d0 + d1 * d1 + d2 * d2 < P.rlist2f;
              };
              const float in2 = P.rlist_in2f, out2 = P.rlist_out2f;
              // hits as a bit mask over the staged entries (the rare entries in
              // the 1e-3 A shell take the exact test), then appended in order
              unsigned hm = 0, ho = 0;
#pragma unroll 4
              for (int t = 0; t < nc; t++) {
                const float r = rh2(sh_h[t]);
                hm |= (unsigned)(r < in2) << t;
                ho |= (unsigned)(r <= out2) << t;
              }
              for (unsigned um = ho & ~hm; um; um &= um - 1) {   // the shell
                const int t = __ffs(um) - 1;
                if (exact(sh_h[t])) hm |= 1u << t;
              }
              if (self >= 0 && self < 32) hm &= ~(1u << __popc(km & ((1u << self) - 1u)));   // the atom itself
              const int nh = __popc(hm);
              if (cnt + nh <= max_nbrs) {
                uint32_t* out = A.nbr + k + (int64_t)cnt * stride;
                for (; hm; hm &= hm - 1, out += stride) *out = __float_as_uint(sh_h[__ffs(hm) - 1].w);
              } else {
                for (int c2 = cnt; hm; hm &= hm - 1, c2++)
                  if (c2 < max_nbrs) A.nbr[(int64_t)c2 * stride + k] = __float_as_uint(sh_h[__ffs(hm) - 1].w);
              }
              cnt += nh;
            }
          }
          __syncwarp();
        }
      }
    }
  }
  if (valid) {
    if (cnt > max_nbrs) { atomicOr(err, kErrNeighborOverflow); cnt = max_nbrs; }
    A.nn[k] = cnt;
    if constexpr (F64) { for (int c = 0; c < 3; c++) A.xrd[3 * k + c] = xi[c]; }
    else { A.xrh[k] = hi; A.xrl[k] = lo; }
  }
}

// One warp: the list of atom `a` of system `s` (sorted order), the lanes
// taking 32 consecutive candidates at a time.  For each stencil row (dz, dy)
// the bins kx-m..kx+m that share one image index are consecutive in the
// sorted order, so their atoms form one contiguous slot range; a ballot and
// prefix count append the hits in candidate order, which is the order of
// build_warp's per-lane loop.  Short dependency chains: the mode for passes
// that re-list few atoms, where build_warp's long per-warp loops would set
// the pass's latency.
template <bool F64>
__device__ void build_atom(int s, int a, const SysArrays& S, const SlotArrays& A, const int32_t* __restrict__ cstart,
                           const int32_t* __restrict__ count, const DevPot* __restrict__ pots, int32_t max_nbrs,
                           int64_t stride, int32_t* err) {
  const int lane = threadIdx.x & 31;
  const int64_t seg = S.seg_start[s];
  const int64_t k = seg + a;
  const DevPot& P = pots[S.pot[s]];
  const int nb0 = S.nb[3 * s], nb1 = S.nb[3 * s + 1], nb2 = S.nb[3 * s + 2];
  const int m0 = S.reach[3 * s], m1 = S.reach[3 * s + 1], m2 = S.reach[3 * s + 2];
  const int boff = S.bin_off[s];
  const int64_t coff = S.caller_off[s];
  const int lb = A.bin[k] - boff;
  const int kx = lb % nb0, ky = (lb / nb0) % nb1, kz = lb / (nb0 * nb1);
  float4 hi = make_float4(0, 0, 0, 0), lo = hi;
  double xi[3] = {0, 0, 0};
  if constexpr (F64) { for (int c = 0; c < 3; c++) xi[c] = A.xd[3 * k + c]; }
  else { hi = A.xh[k]; lo = A.xl[k]; }
  int cnt = 0;
  const int pm = S.pmask[s];
  // along a non-periodic axis the stencil stops at the edges (no images)
  const int xlo = (pm & 1) ? kx - m0 : max(kx - m0, 0), xhi = (pm & 1) ? kx + m0 : min(kx + m0, nb0 - 1);
  for (int dz = -m2; dz <= m2; dz++) {
    const int zz = kz + dz, iz = floor_div(zz, nb2), cz = zz - iz * nb2;
    if (!(pm & 4) && iz != 0) continue;
    for (int dy = -m1; dy <= m1; dy++) {
      const int yy = ky + dy, iy = floor_div(yy, nb1), cy = yy - iy * nb1;
      if (!(pm & 2) && iy != 0) continue;
      const int rowb = boff + (cz * nb1 + cy) * nb0;
      for (int xx = xlo; xx <= xhi;) {
        const int ix = floor_div(xx, nb0);
        const int xe = min(xhi, (ix + 1) * nb0 - 1);
        const int gb0 = rowb + (xx - ix * nb0), gb1 = rowb + (xe - ix * nb0);
        const int q0 = (int)(cstart[gb0] - coff), q1 = (int)(cstart[gb1] - coff) + count[gb1];
        const int code = img_code(ix, iy, iz);
        const int64_t ti = (int64_t)s * kNCodes + code;
        float a0 = 0, a1 = 0, a2 = 0, e0 = 0, e1 = 0, e2 = 0;
        double s0 = 0, s1 = 0, s2 = 0;
        if constexpr (F64) {
          const double* sd = S.shiftd + 3 * ti;
          s0 = sd[0] - xi[0]; s1 = sd[1] - xi[1]; s2 = sd[2] - xi[2];
        } else {
          const float4 sh = S.shift[2 * ti], sl = S.shift[2 * ti + 1];
          a0 = sh.x - hi.x; a1 = sh.y - hi.y; a2 = sh.z - hi.z;   // exact (2^-12 grid)
          e0 = sl.x - lo.x; e1 = sl.y - lo.y; e2 = sl.z - lo.z;
        }
        for (int qb = q0; qb < q1; qb += 32) {
          const int q = qb + lane;
          bool hit = false;
          if (q < q1 && !(q == a && code == kCenter)) {
            if constexpr (F64) {
              const double* xj = A.xd + 3 * (seg + q);
              const double d0 = xj[0] + s0, d1 = xj[1] + s1, d2 = xj[2] + s2;
              hit = d0 * d0 + d1 * d1 + d2 * d2 < P.rlist2d;
            } else {
              const float4 xj = A.xh[seg + q];
              const float h0 = xj.x + a0, h1 = xj.y + a1, h2 = xj.z + a2;
              const float rh2 = fmaf(h0, h0, fmaf(h1, h1, h2 * h2));
              hit = rh2 < P.rlist_in2f;
              if (!hit && rh2 <= P.rlist_out2f) {   // within 1e-3 A of the list radius
                const float4 lj = A.xl[seg + q];
                const float d0 = h0 + (lj.x + e0), d1 = h1 + (lj.y + e1), d2 = h2 + (lj.z + e2);
                hit = d0 * d0 + d1 * d1 + d2 * d2 < P.rlist2f;
              }
            }
          }
          const unsigned bal = __ballot_sync(0xffffffffu, hit);
          if (hit) {
            const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
            if (pos < max_nbrs) A.nbr[pos * stride + k] = (uint32_t)q | ((uint32_t)code << kJBits);
          }
          cnt += __popc(bal);
        }
        xx = xe + 1;
      }
    }
  }
  if (lane == 0) {
    if (cnt > max_nbrs) { atomicOr(err, kErrNeighborOverflow); cnt = max_nbrs; }
    A.nn[k] = cnt;
    if constexpr (F64) { for (int c = 0; c < 3; c++) A.xrd[3 * k + c] = xi[c]; }
    else { A.xrh[k] = hi; A.xrl[k] = lo; }
  }
}

// (B) Verlet lists of the work table's warps: one warp per 32 sorted atoms,
// warps taken from a counter (a fixed, resident grid; consecutive grabs are
// neighbouring atoms, and CTAs that start late beside another kernel just
// take less work).
template <bool F64>
__global__ void __launch_bounds__(128, kBuildCtasPerSm) k_build_list_warp(
    SysArrays S, SlotArrays A, const int32_t* __restrict__ tab_sys, const int32_t* __restrict__ tab_base,
    const int32_t* __restrict__ tab_base_a, int32_t* __restrict__ tab_n, const int32_t* __restrict__ cstart,
    const int32_t* __restrict__ count, const DevPot* __restrict__ pots, int32_t max_nbrs, int64_t stride,
    int32_t* err) {
  __shared__ float4 sh_h[4][32];
  __shared__ double sh_d[4][32][3];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int ne = tab_n[0];
  const bool per_atom = tab_n[2] != 0;   // chosen by the table CTA from the pass's size
  const int32_t* base = per_atom ? tab_base_a : tab_base;
  const int total = base[ne];
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(tab_n + 1, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= total) break;
    int e0 = 0, e1 = ne - 1;   // last entry with base[e] <= t (warp-uniform search)
    while (e0 < e1) {
      int mid = (e0 + e1 + 1) >> 1;
      if (base[mid] <= t) e0 = mid; else e1 = mid - 1;
    }
    if (per_atom) build_atom<F64>(tab_sys[e0], t - base[e0], S, A, cstart, count, pots, max_nbrs, stride, err);
    else build_warp<F64>(tab_sys[e0], t - base[e0], S, A, cstart, count, pots, max_nbrs, stride, err, sh_h[wib],
                         sh_d[wib]);
  }
}

}  // namespace ts
