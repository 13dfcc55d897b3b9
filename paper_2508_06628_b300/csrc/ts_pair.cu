// ts_pair.cu -- fused pair energy / force / virial kernel and the per-system
// FP64 reduction behind ts_pair_forces.
//
// Definitions (forces, energy and stress as the model output, Sec. 2 of the
// TorchSim paper): with d = x_j + n h - x_i over the full neighbour list,
//   F_i = sum_j phi'(r) d / r,  E_i = 1/2 sum_j [phi(r) - phi(rc)],
//   W = 1/2 sum_ij phi'(r) d (x) d / r,  stress = W / V.
// One thread per atom gathers its neighbours (no scatter atomics: the full
// list gives every atom its own force); a warp holds 32 atoms of one system,
// so energy and virial go through warp shuffles into one FP64 partial per
// warp, and a second kernel sums each system's warps in a fixed order.
#include <type_traits>

#include "ts_kernels.cuh"

namespace ts {

template <bool F64, bool EW>
__global__ void __launch_bounds__(256) k_pair(int32_t n_warps, const int32_t* __restrict__ warp_sys, SysArrays S,
                                              SlotArrays A, const DevPot* __restrict__ pots, int64_t stride,
                                              int filter, double* __restrict__ partial, int skip_small, int inner) {
  int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (w >= n_warps) return;
  int s = warp_sys[w];
  if (pair_skip(S, s, filter)) return;
  if (skip_small && S.n_atoms[s] <= kSmallMax) return;   // handled by k_pair_small
  // inner-list mode (MD steps): a system flagged for pruning, or re-listed in
  // this pass, runs its full list and writes the inner list on the way
  const bool refresh = inner && (S.prune[s] || need_relist(S, s));   // warp-uniform
  const uint32_t* NB = inner && !refresh ? A.nbr_in : A.nbr;
  int64_t k = (int64_t)w * kWarp + lane;
  const DevPot P = pots[S.pot[s]];
  bool valid = A.perm[k] >= 0;
  int nn = valid ? (inner && !refresh ? A.nn_in : A.nn)[k] : 0;
  int cin = 0;
  uint32_t* out_in = A.nbr_in + k;
  int64_t seg = S.seg_start[s];
  if constexpr (F64) {
    const double* tab = S.shiftd + 3 * (int64_t)s * kNCodes;
    double xi0 = A.xd[3 * k], xi1 = A.xd[3 * k + 1], xi2 = A.xd[3 * k + 2];
    double f0 = 0, f1 = 0, f2 = 0, e = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    for (int q = 0; q < nn; q++) {
      uint32_t ent = __ldg(NB + q * stride + k);
      int64_t j = seg + (ent & kJMask);
      int code = (int)(ent >> kJBits);
      double d0 = A.xd[3 * j] - xi0, d1 = A.xd[3 * j + 1] - xi1, d2 = A.xd[3 * j + 2] - xi2;
      if (code != kCenter) { d0 += tab[3 * code]; d1 += tab[3 * code + 1]; d2 += tab[3 * code + 2]; }
      double r2 = d0 * d0 + d1 * d1 + d2 * d2;
      if (refresh && r2 < P.rin2d) out_in[(int64_t)(cin++) * stride] = ent;
      if (r2 < P.rc2d) {
        double phi, fr;
        PotMath<double>::eval(P, r2, phi, fr);
        f0 += fr * d0; f1 += fr * d1; f2 += fr * d2;
        if (EW) {
          e += 0.5 * (phi - P.phicd);
          double hf = 0.5 * fr;
          w0 += hf * d0 * d0; w1 += hf * d1 * d1; w2 += hf * d2 * d2;
          w3 += hf * d0 * d1; w4 += hf * d0 * d2; w5 += hf * d1 * d2;
        }
      }
    }
    if (valid) { A.Fd[3 * k] = f0; A.Fd[3 * k + 1] = f1; A.Fd[3 * k + 2] = f2; }
    if (refresh && valid) {
      A.nn_in[k] = cin;
      A.xpd[3 * k] = xi0; A.xpd[3 * k + 1] = xi1; A.xpd[3 * k + 2] = xi2;
    }
    if (EW) {
      double v[7] = {e, w0, w1, w2, w3, w4, w5};
#pragma unroll
      for (int c = 0; c < 7; c++) {
        double t = warp_sum(v[c]);
        if (lane == 0) partial[(int64_t)w * kPartialStride + c] = t;
      }
    }
  } else {
    const float4* tab = S.shift + 2 * (int64_t)s * kNCodes;
    float4 xi = A.xh[k], li = A.xl[k];
    float f0 = 0.f, f1 = 0.f, f2 = 0.f, e = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f, w4 = 0.f, w5 = 0.f;
    auto one = [&](uint32_t ent, float4 xj, float4 lj) {
      int code = (int)(ent >> kJBits);
      // hi parts on the 2^-12 grid: exact; lo parts tiny
      float a0 = xj.x - xi.x, a1 = xj.y - xi.y, a2 = xj.z - xi.z;
      float b0 = lj.x - li.x, b1 = lj.y - li.y, b2 = lj.z - li.z;
      if (code != kCenter) {
        float4 sh = __ldg(tab + 2 * code), sl = __ldg(tab + 2 * code + 1);
        a0 += sh.x; a1 += sh.y; a2 += sh.z;
        b0 += sl.x; b1 += sl.y; b2 += sl.z;
      }
      float d0 = a0 + b0, d1 = a1 + b1, d2 = a2 + b2;
      float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
      if (refresh && r2 < P.rin2f) out_in[(int64_t)(cin++) * stride] = ent;
      if (r2 < P.rc2f) {
        float phi, fr;
        PotMath<float>::eval(P, r2, phi, fr);
        f0 = fmaf(fr, d0, f0); f1 = fmaf(fr, d1, f1); f2 = fmaf(fr, d2, f2);
        if (EW) {
          e += 0.5f * (phi - P.phicf);
          float hf = 0.5f * fr;
          float h0 = hf * d0, h1 = hf * d1;
          w0 = fmaf(h0, d0, w0); w1 = fmaf(h1, d1, w1); w2 = fmaf(hf * d2, d2, w2);
          w3 = fmaf(h0, d1, w3); w4 = fmaf(h0, d2, w4); w5 = fmaf(h1, d2, w5);
        }
      }
    };
    // Four independent gathers in flight per lane, and the next four list
    // entries fetched before this block's gathers: the loop is otherwise
    // latency bound on the streamed index loads (evict-first, so they do not
    // push neighbour positions out of L1).  Same summation order as a plain
    // loop, so results do not depend on the unrolling.
    const float4* ph = A.xh + seg;
    const float4* pl = A.xl + seg;
    const uint32_t* lp = NB + k;
    int q = 0;
    uint32_t n0 = 0, n1 = 0, n2 = 0, n3 = 0;
    if (nn >= 4) {
      n0 = __ldcs(lp); n1 = __ldcs(lp + stride); n2 = __ldcs(lp + 2 * stride); n3 = __ldcs(lp + 3 * stride);
    }
    for (; q + 4 <= nn; q += 4) {
      uint32_t e0 = n0, e1 = n1, e2 = n2, e3 = n3;
      if (q + 8 <= nn) {
        const uint32_t* np = lp + (int64_t)(q + 4) * stride;
        n0 = __ldcs(np); n1 = __ldcs(np + stride); n2 = __ldcs(np + 2 * stride); n3 = __ldcs(np + 3 * stride);
      }
      float4 x0 = __ldg(ph + (e0 & kJMask)), l0 = __ldg(pl + (e0 & kJMask));
      float4 x1 = __ldg(ph + (e1 & kJMask)), l1 = __ldg(pl + (e1 & kJMask));
      float4 x2 = __ldg(ph + (e2 & kJMask)), l2 = __ldg(pl + (e2 & kJMask));
      float4 x3 = __ldg(ph + (e3 & kJMask)), l3 = __ldg(pl + (e3 & kJMask));
      one(e0, x0, l0); one(e1, x1, l1); one(e2, x2, l2); one(e3, x3, l3);
    }
    for (; q < nn; q++) {
      uint32_t ent = __ldg(NB + q * stride + k);
      int64_t j = seg + (ent & kJMask);
      one(ent, __ldg(A.xh + j), __ldg(A.xl + j));
    }
    if (valid) A.F[k] = make_float4(f0, f1, f2, e);
    if (refresh && valid) { A.nn_in[k] = cin; A.xph[k] = xi; A.xpl[k] = li; }
    if (EW) {
      double v[7] = {(double)e, (double)w0, (double)w1, (double)w2, (double)w3, (double)w4, (double)w5};
#pragma unroll
      for (int c = 0; c < 7; c++) {
        double t = warp_sum(v[c]);
        if (lane == 0) partial[(int64_t)w * kPartialStride + c] = t;
      }
    }
  }
}

// Mixed-precision pair kernel for systems of up to kSmallMax atoms.  One CTA
// per work item (built on the host, int4 in warp units):
//   x = first staged warp, y = staged warps, z = first computed warp,
//   w = computed warps (at most 8).
// An item is a run of consecutive warps that may straddle systems; its staged
// range holds every system those warps belong to (at most kSmallMax slots),
// so every neighbour gather is a shared-memory read.  Staged record per atom:
// 16 B, the fixed-point coordinates (units of 2^-26 A, modulo 2^32), so that
// a gather is one 16-byte read and a 2048-atom system takes 32 KB; a pair
// vector is the exact integer difference plus the fixed-point image shift,
// converted once to FP32.  List entries stream from global memory
// (coalesced, evict-first, prefetched two blocks of four ahead).  The potential
// arithmetic and summation order are those of k_pair; the pair vectors carry
// the same single FP32 rounding but a different quantisation of the
// coordinates, so the two kernels agree within the mixed-precision tolerance,
// not bit for bit.
constexpr int kPairSmallThreads = 256;
constexpr int kSmallRecord = 16;   // staged bytes per atom

template <bool EW>
__global__ void __launch_bounds__(kPairSmallThreads) k_pair_small(
    int32_t n_items, const int4* __restrict__ items, const int32_t* __restrict__ warp_sys, SysArrays S,
    SlotArrays A, const DevPot* __restrict__ pots, int64_t stride, int filter, double* __restrict__ partial,
    int inner) {
  extern __shared__ __align__(16) uint4 sq[];   // [staged] fixed-point (x, y, z, -)
  if ((int)blockIdx.x >= n_items) return;
  const int4 W = items[blockIdx.x];
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // leave before staging when no warp of the item is selected
  const bool mine = wl < W.w && !pair_skip(S, warp_sys[W.z + wl], filter);
  if (!__syncthreads_or(mine)) return;
  const int64_t st0 = (int64_t)W.x * kWarp;
  const int nst = W.y * kWarp;
#pragma unroll 4
  for (int t = threadIdx.x; t < nst; t += kPairSmallThreads) {
    float4 h = __ldg(A.xh + st0 + t), l = __ldg(A.xl + st0 + t);
    sq[t] = make_uint4(fix_coord(h.x, l.x), fix_coord(h.y, l.y), fix_coord(h.z, l.z), 0u);
  }
  __syncthreads();
  if (!mine) return;
  const int wg = W.z + wl;
  const int s = warp_sys[wg];
  const int64_t seg = S.seg_start[s];
  const int64_t k = (int64_t)wg * kWarp + lane;
  const int i = (int)(k - seg);
  const int n = S.n_atoms[s];
  const bool valid = i < n;
  const uint4* hq = sq + (seg - st0);
  const DevPot P = pots[S.pot[s]];
  const uint4* tab = S.shiftq + (int64_t)s * kNCodes;
  // inner-list mode (MD steps): a system flagged for pruning, or re-listed in
  // this pass, runs its full list and writes the inner list on the way
  const bool refresh = inner && (S.prune[s] || need_relist(S, s));   // warp-uniform
  const bool use_in = inner && !refresh;
  const int nn = valid ? (use_in ? A.nn_in : A.nn)[k] : 0;
  const uint4 xi = valid ? hq[i] : make_uint4(0, 0, 0, 0);
  int cin = 0;
  float f0 = 0.f, f1 = 0.f, f2 = 0.f, e = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f, w4 = 0.f, w5 = 0.f;
  // The potential kind is uniform over a warp (one system): one loop per kind,
  // with no branch inside an entry.  Every entry evaluates the potential and
  // selects a zero force factor beyond rc (fmaf(0, d, f) == f, so the sums are
  // those of the branching form), which lets the four entries of a round
  // overlap.
  auto run = [&](auto kind, auto refresh_c) {
    constexpr int K = decltype(kind)::value;
    constexpr bool R = decltype(refresh_c)::value;
    auto one = [&](uint32_t ent) {
      const int code = (int)(ent >> kJBits);
      const int j = (int)(ent & kJMask);
      const bool img = code != kCenter;
      const uint4 sh = img ? __ldg(tab + code) : make_uint4(0, 0, 0, 0);
      const uint4 xj = hq[j];
      // exact integer pair vector (modulo 2^32), one rounding to FP32; kept in
      // fixed-point units, the power-of-two scale applied once to r^2 and once
      // to the force factor (scaling by 2^k commutes with FP32 rounding, so
      // r^2 and the force sums are bit-identical to scaling each component)
      const float u0 = (float)(int)(xj.x - xi.x + sh.x);
      const float u1 = (float)(int)(xj.y - xi.y + sh.y);
      const float u2 = (float)(int)(xj.z - xi.z + sh.z);
      const float r2 = fmaf(u0, u0, fmaf(u1, u1, u2 * u2)) * (kFixInv * kFixInv);
      const bool in = r2 < P.rc2f;
      if (R) {   // inner list: within rc + inner skin (+ 1e-3 A), in list order
        if (r2 < P.rin2f) A.nbr_in[(int64_t)cin * stride + k] = ent;
        cin += r2 < P.rin2f;
      }
      float phi, fr;
      PotMath<float>::eval_k<K>(P, r2, phi, fr);
      fr = in ? fr : 0.f;
      const float fu = fr * kFixInv;
      f0 = fmaf(fu, u0, f0); f1 = fmaf(fu, u1, f1); f2 = fmaf(fu, u2, f2);
      if (EW) {
        const float d0 = u0 * kFixInv, d1 = u1 * kFixInv, d2 = u2 * kFixInv;
        e += in ? 0.5f * (phi - P.phicf) : 0.f;
        float hf = 0.5f * fr;
        float h0 = hf * d0, h1 = hf * d1;
        w0 = fmaf(h0, d0, w0); w1 = fmaf(h1, d1, w1); w2 = fmaf(hf * d2, d2, w2);
        w3 = fmaf(h0, d1, w3); w4 = fmaf(h0, d2, w4); w5 = fmaf(h1, d2, w5);
      }
    };
    const uint32_t* lp = (use_in ? A.nbr_in : A.nbr) + k;
    int q = 0;
    // list entries stream two blocks of four ahead of use (n: the next
    // block, m: the one after)
    uint32_t n0 = 0, n1 = 0, n2 = 0, n3 = 0, m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    if (nn >= 4) { n0 = __ldcs(lp); n1 = __ldcs(lp + stride); n2 = __ldcs(lp + 2 * stride); n3 = __ldcs(lp + 3 * stride); }
    if (nn >= 8) {
      const uint32_t* np = lp + 4 * stride;
      m0 = __ldcs(np); m1 = __ldcs(np + stride); m2 = __ldcs(np + 2 * stride); m3 = __ldcs(np + 3 * stride);
    }
    for (; q + 4 <= nn; q += 4) {
      uint32_t e0 = n0, e1 = n1, e2 = n2, e3 = n3;
      n0 = m0; n1 = m1; n2 = m2; n3 = m3;
      if (q + 12 <= nn) {
        const uint32_t* np = lp + (int64_t)(q + 8) * stride;
        m0 = __ldcs(np); m1 = __ldcs(np + stride); m2 = __ldcs(np + 2 * stride); m3 = __ldcs(np + 3 * stride);
      }
      one(e0); one(e1); one(e2); one(e3);
    }
    for (; q < nn; q++) one(__ldcs(lp + (int64_t)q * stride));
  };
  using Off = std::false_type;
  using On = std::true_type;
  if (!refresh) {
    if (P.kind == TS_LJ) run(std::integral_constant<int, TS_LJ>{}, Off{});
    else if (P.kind == TS_MORSE) run(std::integral_constant<int, TS_MORSE>{}, Off{});
    else run(std::integral_constant<int, TS_SOFT_SPHERE>{}, Off{});
  } else {
    if (P.kind == TS_LJ) run(std::integral_constant<int, TS_LJ>{}, On{});
    else if (P.kind == TS_MORSE) run(std::integral_constant<int, TS_MORSE>{}, On{});
    else run(std::integral_constant<int, TS_SOFT_SPHERE>{}, On{});
    if (valid) { A.nn_in[k] = cin; A.xph[k] = __ldg(A.xh + k); A.xpl[k] = __ldg(A.xl + k); }
  }
  if (valid) A.F[k] = make_float4(f0, f1, f2, e);
  if (EW) {   // one FP64 partial per warp (every computed warp lies inside its system's padded segment)
    double v[7] = {(double)e, (double)w0, (double)w1, (double)w2, (double)w3, (double)w4, (double)w5};
#pragma unroll
    for (int cc = 0; cc < 7; cc++) {
      double t = warp_sum(v[cc]);
      if (lane == 0) partial[(int64_t)wg * kPartialStride + cc] = t;
    }
  }
}

// One warp per system: FP64 sum of the system's warp partials in warp order
// (deterministic, independent of the batch around the system).
// partial slots: 0 energy, 1..6 virial (xx yy zz xy xz yz), 7 kinetic energy.
__global__ void k_reduce_sys(int32_t B, SysArrays S, const double* __restrict__ partial, double* E, double* stress,
                             double* KE, double* Eint, double* Wint) {
  int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (s >= B) return;
  int w0 = S.warp_start[s], w1 = S.warp_end[s];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int w = w0 + lane; w < w1; w += 32)
    for (int c = 0; c < 8; c++) acc[c] += partial[(int64_t)w * kPartialStride + c];
  for (int c = 0; c < 8; c++) acc[c] = warp_sum(acc[c]);
  if (lane != 0) return;
  const double* h = S.h + 9 * s;
  double V = fabs(h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                  h[2] * (h[3] * h[7] - h[4] * h[6]));
  double W[9] = {acc[1], acc[4], acc[5], acc[4], acc[2], acc[6], acc[5], acc[6], acc[3]};
  if (E) E[s] = acc[0];
  if (Eint) Eint[s] = acc[0];
  if (stress) for (int q = 0; q < 9; q++) stress[9 * (int64_t)s + q] = W[q] / V;
  if (Wint) for (int q = 0; q < 9; q++) Wint[9 * (int64_t)s + q] = W[q];
  if (KE) KE[s] = acc[7];
}

__global__ void k_clear_dirty(int32_t B, SysArrays S) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < B) S.dirty[s] = 0;
}

// ordered pairs within the cutoff (work of one pair launch)
__global__ void k_count_pairs(int32_t n_warps, const int32_t* __restrict__ warp_sys, SysArrays S, SlotArrays A,
                              const DevPot* __restrict__ pots, int64_t stride, int f64,
                              unsigned long long* out) {
  int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (w >= n_warps) return;
  int s = warp_sys[w];
  int64_t k = (int64_t)w * kWarp + lane;
  const DevPot P = pots[S.pot[s]];
  int nn = A.perm[k] >= 0 ? A.nn[k] : 0;
  int64_t seg = S.seg_start[s];
  unsigned long long c = 0;
  for (int q = 0; q < nn; q++) {
    uint32_t ent = A.nbr[q * stride + k];
    int64_t j = seg + (ent & kJMask);
    int code = (int)(ent >> kJBits);
    double d0, d1, d2;
    if (f64) {
      const double* sh = S.shiftd + 3 * ((int64_t)s * kNCodes + code);
      d0 = A.xd[3 * j] - A.xd[3 * k] + sh[0]; d1 = A.xd[3 * j + 1] - A.xd[3 * k + 1] + sh[1];
      d2 = A.xd[3 * j + 2] - A.xd[3 * k + 2] + sh[2];
    } else {
      int64_t t = (int64_t)s * kNCodes + code;
      float4 a = A.xh[j], b = A.xl[j], ia = A.xh[k], ib = A.xl[k], sh = S.shift[2 * t], sl = S.shift[2 * t + 1];
      d0 = (double)((a.x - ia.x + sh.x) + (b.x - ib.x + sl.x));
      d1 = (double)((a.y - ia.y + sh.y) + (b.y - ib.y + sl.y));
      d2 = (double)((a.z - ia.z + sh.z) + (b.z - ib.z + sl.z));
    }
    c += (d0 * d0 + d1 * d1 + d2 * d2) < P.rc2d;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0 && c) atomicAdd(out, c);
}


}  // namespace ts
