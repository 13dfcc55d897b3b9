// ts_adjoint.cu -- differentiable path (the paper's Sec. 2: gradients of a
// trajectory observable, a radial distribution function, with respect to
// potential parameters): the pair-force adjoint, the smeared RDF and its
// position gradient, and the reverse step of velocity Verlet.
//
// Pair adjoint, with d = x_j + n h - x_i over the full list and upstream
// gF = dL/dF, gE = dL/dE, gS = dL/dstress:
//   gx_i = sum_j K(d_ij) (gF_j - gF_i) - gE F_i - (1/V) sum_j dT(d_ij) : gS
//   K(d) = phi'' u u^T + (phi'/r)(I - u u^T),  u = d/r
//   T(d)_ab = (phi'/r) d_a d_b
//   gtheta_p = sum_ij (dphi'/dp) u.gF_i + gE/2 sum (dphi/dp - dphi(rc)/dp)
//              + 1/(2V) sum (dphi'/dp)/r (d.gS.d)
// Each atom gathers gF of its neighbours (full list), so no scatter atomics;
// parameter gradients go warp -> system -> potential in a fixed order.
#include <type_traits>

#include "ts_kernels.cuh"

namespace ts {

// STRESS: gS given (the stress terms are compiled out of the common case, which
// keeps the mixed variant within 64 registers: 8 CTAs of 128 threads per SM)
template <bool F64, bool STRESS>
__global__ void __launch_bounds__(128, F64 ? 4 : 8) k_pair_bwd(int32_t n_warps, const int32_t* __restrict__ warp_sys, SysArrays S,
                                                  SlotArrays A, const DevPot* __restrict__ pots, int64_t stride,
                                                  const double* __restrict__ gE, const double* __restrict__ gS,
                                                  double* gpart, int accum_part, int skip_small) {
  int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (w >= n_warps) return;
  int s = warp_sys[w];
  if (skip_small && S.n_atoms[s] <= kSmallMax) return;   // k_pair_bwd_small takes it
  int64_t k = (int64_t)w * kWarp + lane;
  const DevPot P = pots[S.pot[s]];
  bool valid = A.perm[k] >= 0;
  // the inner (pruned) list holds every pair within rc while the system is
  // neither flagged for a refresh nor re-listed since: every caller re-lists
  // flagged systems first, and a non-MD re-listing flags the system, so the
  // test is warp-uniform and needs no host state; the inner list keeps the
  // outer list's order, so the sums are the same either way
  const bool use_in = !S.prune[s] && !need_relist(S, s);
  const int ifmt = use_in ? S.infmt[s] : kInnerVerlet;
  int nn = valid ? (use_in ? A.nn_in : A.nn)[k] : 0;
  const int64_t seg = S.seg_start[s];
  // entry q of the list read, and its (slot of j, image code) in either format
  auto entry = [&](int q) -> uint32_t {
    return use_in ? __ldg(A.nbr_in + inner_at(q, k, stride)) : __ldg(A.nbr + (int64_t)q * stride + k);
  };
  // staged-table index -> image code of this warp's inner-list format, looked up in shared memory
  __shared__ uint16_t tab_code[4][kTabEntries + 2];
  const int wib = threadIdx.x >> 5;
  if (fmt_kind(ifmt) == kInnerTab) {
    const TabDecode tdec(ifmt);
    for (int c = lane; c < kTabCodes; c += kWarp) tab_code[wib][c] = (uint16_t)tdec.code(c);
  }
  __syncwarp();
  auto decode = [&](uint32_t e, int64_t& j, int& code) {
    const int kind = fmt_kind(ifmt);
    if (kind == kInnerVerlet) {
      j = seg + (e & kJMask);
      code = (int)(e >> kJBits);
    } else {
      j = seg + ((e & 0xffffu) >> 4);
      code = kind == kInnerTab ? (int)tab_code[wib][e >> 20] : (int)(e >> 16);
    }
  };
  constexpr bool stress = STRESS;
  double Vinv = 0.0, Sg[9];
  if constexpr (stress) {
    const double* h = S.h + 9 * s;
    Vinv = 1.0 / fabs(h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                      h[2] * (h[3] * h[7] - h[4] * h[6]));
  }
  for (int q = 0; q < 9; q++) Sg[q] = stress ? gS[9 * (int64_t)s + q] : 0.0;
  double gEs = gE ? gE[s] : 0.0;
  // the energy term needs the shift derivative dphi(rc)/dp (in the loop's
  // precision: the FP64 pipe is a small fraction of the FP32 one)
  const bool shift_e = P.shift && P.kind != TS_SOFT_SPHERE && gEs != 0.0;
  if constexpr (F64) {
    double dphic[3] = {0, 0, 0};
    if (shift_e) {
      double r, d1, d2, dd1[3];
      PotMath<double>::eval2(P, P.rc2d, r, d1, d2, dphic, dd1);
    }
    double gx[3] = {0, 0, 0}, gth[3] = {0, 0, 0};
    const double* tab = S.shiftd + 3 * (int64_t)s * kNCodes;
    const double* xi = A.xd + 3 * k;
    const double* gi = A.gd1 + 3 * k;
    for (int q = 0; q < nn; q++) {
      int64_t j;
      int code;
      decode(entry(q), j, code);
      double d[3];
      for (int c = 0; c < 3; c++) d[c] = A.xd[3 * j + c] - xi[c] + tab[3 * code + c];
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (!(r2 < P.rc2d)) continue;
      double r, d1, d2, dphi[3], dd1[3];
      PotMath<double>::eval2(P, r2, r, d1, d2, dphi, dd1);
      double u[3] = {d[0] / r, d[1] / r, d[2] / r};
      double g[3];
      for (int c = 0; c < 3; c++) g[c] = A.gd1[3 * j + c] - gi[c];
      double ug = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
      double ugi = u[0] * gi[0] + u[1] * gi[1] + u[2] * gi[2];
      for (int c = 0; c < 3; c++) gx[c] += d2 * ug * u[c] + d1 / r * (g[c] - ug * u[c]);
      for (int p = 0; p < 3; p++) gth[p] += dd1[p] * ugi + 0.5 * gEs * (dphi[p] - dphic[p]);
      if constexpr (stress) {
        double Aq = (d2 - d1 / r) / (r * r), dSd = 0;
        for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) dSd += d[a] * Sg[3 * a + b] * d[b];
        for (int c = 0; c < 3; c++) {
          double Sd = Sg[3 * c] * d[0] + Sg[3 * c + 1] * d[1] + Sg[3 * c + 2] * d[2];
          double dS = d[0] * Sg[c] + d[1] * Sg[3 + c] + d[2] * Sg[6 + c];
          gx[c] -= Vinv * (Aq * d[c] * dSd + d1 / r * (Sd + dS));
        }
        for (int p = 0; p < 3; p++) gth[p] += 0.5 * Vinv * dd1[p] / r * dSd;
      }
    }
    if (valid) {
      for (int c = 0; c < 3; c++) A.gd0[3 * k + c] = gx[c] - gEs * A.Fd[3 * k + c];
    }
    for (int p = 0; p < 3; p++) {
      double t = warp_sum(gth[p]);
      if (lane == 0) gpart[4 * (int64_t)w + p] = accum_part ? gpart[4 * (int64_t)w + p] + t : t;
    }
  } else {
    const float4* tab = S.shift + 2 * (int64_t)s * kNCodes;
    float4 xi = A.xh[k], li = A.xl[k], gi = A.g1[k];
    // parameter gradients: compensated (Kahan) FP32 sums per thread -- the
    // FP64 pipe of this part runs at a small fraction of the FP32 rate --
    // then FP64 sums over the warp, the system and the batch
    float gxf[3] = {0.f, 0.f, 0.f}, gtf[3] = {0.f, 0.f, 0.f}, gtc[3] = {0.f, 0.f, 0.f};
    float gEf = (float)gEs, Vf = (float)Vinv;
    float Sf[9];
    for (int q = 0; q < 9; q++) Sf[q] = (float)Sg[q];
    float dpc[3] = {0.f, 0.f, 0.f};
    if (shift_e) {
      float r, d1, d2, dd1[3];
      PotMath<float>::eval2(P, P.rc2f, r, d1, d2, dpc, dd1);
    }
    // entries four at a time, the next four in flight: one 16-byte group of
    // the inner list, or four loads of the Verlet list
    auto group = [&](int g) -> uint4 {
      if (use_in) return __ldg(reinterpret_cast<const uint4*>(A.nbr_in) + (int64_t)g * stride + k);
      const int q = 4 * g;
      return make_uint4(q < nn ? entry(q) : 0u, q + 1 < nn ? entry(q + 1) : 0u, q + 2 < nn ? entry(q + 2) : 0u,
                        q + 3 < nn ? entry(q + 3) : 0u);
    };
    uint4 cur = nn > 0 ? group(0) : make_uint4(0u, 0u, 0u, 0u), nxt = make_uint4(0u, 0u, 0u, 0u);
    for (int q = 0; q < nn; q++) {
      const int c = q & 3;
      if (c == 0) {
        if (q > 0) cur = nxt;
        if (q + 4 < nn) nxt = group((q >> 2) + 1);
      }
      const uint32_t ent = c == 0 ? cur.x : (c == 1 ? cur.y : (c == 2 ? cur.z : cur.w));
      int64_t j;
      int code;
      decode(ent, j, code);
      float4 xj = __ldg(A.xh + j), lj = __ldg(A.xl + j);
      float4 sh = __ldg(tab + 2 * code), sl = __ldg(tab + 2 * code + 1);
      float d[3] = {((xj.x - xi.x) + sh.x) + ((lj.x - li.x) + sl.x), ((xj.y - xi.y) + sh.y) + ((lj.y - li.y) + sl.y),
                    ((xj.z - xi.z) + sh.z) + ((lj.z - li.z) + sl.z)};
      float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (!(r2 < P.rc2f)) continue;
      float r, d1, d2, dphi[3], dd1[3];
      PotMath<float>::eval2(P, r2, r, d1, d2, dphi, dd1);
      float ri = 1.0f / r;
      float u[3] = {d[0] * ri, d[1] * ri, d[2] * ri};
      float4 gj = __ldg(A.g1 + j);
      float g[3] = {gj.x - gi.x, gj.y - gi.y, gj.z - gi.z};
      float ug = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
      float ugi = u[0] * gi.x + u[1] * gi.y + u[2] * gi.z;
      for (int c = 0; c < 3; c++) gxf[c] += d2 * ug * u[c] + d1 * ri * (g[c] - ug * u[c]);
      for (int p = 0; p < 3; p++) {
        const float y = (dd1[p] * ugi + 0.5f * gEf * (dphi[p] - dpc[p])) - gtc[p];
        const float t = gtf[p] + y;
        gtc[p] = (t - gtf[p]) - y;
        gtf[p] = t;
      }
      if constexpr (stress) {
        float Aq = (d2 - d1 * ri) * ri * ri, dSd = 0.f;
        for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) dSd += d[a] * Sf[3 * a + b] * d[b];
        for (int c = 0; c < 3; c++) {
          float Sd = Sf[3 * c] * d[0] + Sf[3 * c + 1] * d[1] + Sf[3 * c + 2] * d[2];
          float dS = d[0] * Sf[c] + d[1] * Sf[3 + c] + d[2] * Sf[6 + c];
          gxf[c] -= Vf * (Aq * d[c] * dSd + d1 * ri * (Sd + dS));
        }
        for (int p = 0; p < 3; p++) gtf[p] += 0.5f * Vf * dd1[p] * ri * dSd;
      }
    }
    if (valid) {
      float4 F = A.F[k];
      A.g0[k] = make_float4(gxf[0] - gEf * F.x, gxf[1] - gEf * F.y, gxf[2] - gEf * F.z, 0.f);
    }
    for (int p = 0; p < 3; p++) {
      const double t = warp_sum((double)gtf[p] - (double)gtc[p]);
      if (lane == 0) gpart[4 * (int64_t)w + p] = accum_part ? gpart[4 * (int64_t)w + p] + t : t;
    }
  }
}

// Mixed-precision pair backward for the systems of up to kSmallMax atoms
// (no stress upstream): one CTA per pair work item of the forward kernel,
// the item's systems staged in shared memory as the same fixed-point records
// (and, for inner lists in the table format, the same per-warp image tables),
// so that a pair vector is the exact integer difference converted once to
// FP32, as in the forward pass; the upstream gF is staged with them (24 bytes per atom, 3 CTAs per SM).  Same sums as
// k_pair_bwd: list order per atom, compensated FP32 parameter sums per thread,
// FP64 over the warp.
// staged bytes per atom: the fixed-point position with gF_x in its fourth word (16 B), gF_y and gF_z (8 B)
constexpr int kBwdRecord = 24;
__global__ void __launch_bounds__(kPairSmallThreads, 3) k_pair_bwd_small(
    int32_t n_items, const int4* __restrict__ items, const int32_t* __restrict__ item_sys, SysArrays S,
    SlotArrays A, const DevPot* __restrict__ pots, int64_t stride, const double* __restrict__ gE, double* gpart,
    int accum_part) {
  extern __shared__ __align__(16) uint4 smem[];
  uint4* tabs = smem;                                   // [kItemWarps][kTabEntries] image shifts
  uint4* sq = smem + kItemWarps * kTabEntries;          // [staged] fixed-point (x, y, z, -)
  if ((int)blockIdx.x >= n_items) return;
  // the prologue's dependent loads as in k_pair_small: item and its warps'
  // systems, then the system and slot words (and the first inner-list group)
  // together, ahead of the staging loop
  const int4 W = items[blockIdx.x];
  float2* sg = reinterpret_cast<float2*>(sq + W.y * kWarp);   // [staged] upstream gF_y, gF_z
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = item_sys[(int64_t)blockIdx.x * kItemWarps + wl];   // 0 past the item's warps
  const int wg = W.z + wl;
  const bool mine = wl < W.w;
  const int64_t k = (int64_t)wg * kWarp + lane;
  const uint4* lp = reinterpret_cast<const uint4*>(A.nbr_in) + k;
  const int fmt_s = S.infmt[s];
  const int64_t seg = S.seg_start[s];
  const int n_s = S.n_atoms[s];
  const int pot_s = S.pot[s];
  const double gEs = gE ? gE[s] : 0.0;
  int nn_first = 0;
  uint4 g_first = make_uint4(0u, 0u, 0u, 0u);
  if (mine) { nn_first = A.nn_in[k]; g_first = __ldcs(lp); }   // group 0 exists for every slot
  // the inner list holds every pair within rc unless the system was flagged or re-listed since its filtering
  const bool use_in = mine && !S.prune[s] && !need_relist(S, s);
  const int fmt = use_in ? fmt_s : kInnerVerlet;
  const bool staged_tab = use_in && fmt_kind(fmt) == kInnerTab;
  const int64_t st0 = (int64_t)W.x * kWarp;
  const int nst = W.y * kWarp;
  const int i = (int)(k - seg);
  const bool valid = mine && i < n_s;
  if (!(use_in && valid)) nn_first = 0;
  uint4* tab = tabs + wl * kTabEntries;
  const uint4* gtab = S.shiftq + (int64_t)s * kNCodes;
#pragma unroll 4
  for (int t = threadIdx.x; t < nst; t += blockDim.x) {
    float4 h = __ldg(A.xh + st0 + t), l = __ldg(A.xl + st0 + t);
    const float4 g = __ldg(A.g1 + st0 + t);
    sq[t] = make_uint4(fix_coord(h.x, l.x), fix_coord(h.y, l.y), fix_coord(h.z, l.z), __float_as_uint(g.x));
    sg[t] = make_float2(g.y, g.z);
  }
  if (staged_tab) {
    const int ntab = (2 * fmt_bound(fmt, 0) + 1) * (2 * fmt_bound(fmt, 1) + 1) * (2 * fmt_bound(fmt, 2) + 1);
    const TabDecode td(fmt);
    for (int c = lane; c < ntab; c += kWarp) tab[c] = __ldg(gtab + td.code(c));
    if (lane == 0) tab[kTabFar] = make_uint4(kFarShift, 0u, 0u, 0u);
  }
  __syncthreads();
  if (!mine) return;
  const uint4* hq = sq + (seg - st0);
  const DevPot P = pots[pot_s];
  const float2* g1s = sg + (seg - st0);
  const uint4 xi = valid ? hq[i] : make_uint4(0, 0, 0, 0);
  const float2 gyz = valid ? g1s[i] : make_float2(0.f, 0.f);
  const float4 gi = make_float4(__uint_as_float(xi.w), gyz.x, gyz.y, 0.f);
  const float gEf = (float)gEs;
  float dpc[3] = {0.f, 0.f, 0.f};
  if (P.shift && P.kind != TS_SOFT_SPHERE && gEs != 0.0) {
    float r, d1, d2, dd1[3];
    PotMath<float>::eval2(P, P.rc2f, r, d1, d2, dpc, dd1);
  }
  float gxf[3] = {0.f, 0.f, 0.f}, gtf[3] = {0.f, 0.f, 0.f}, gtc[3] = {0.f, 0.f, 0.f};
  auto kahan = [&](int p, float v) {
    const float y = v - gtc[p];
    const float t = gtf[p] + y;
    gtc[p] = (t - gtf[p]) - y;
    gtf[p] = t;
  };
  // LJ constants: with s = sigma / r, A = phi'/r = -24 eps (2 s^12 - s^6) / r^2 and
  // Bc = (phi'' - phi'/r) / r^2 = 24 eps (28 s^12 - 8 s^6) / r^4 need no square root
  const float sig2 = P.pf[0] * P.pf[0], eps24 = 24.0f * P.pf[1], isig = 1.0f / P.pf[0];
  const float hgE = 0.5f * gEf;
  // one entry: neighbour record xj (slot j of the system), image shift sh;
  // gx_i += (phi'/r) g + (phi'' - phi'/r) (d.g) d / r^2 with g = gF_j - gF_i,
  // gtheta += (dphi'/dtheta) (d.gF_i) / r + gE/2 (dphi/dtheta - dphi(rc)/dtheta)
  auto one = [&](auto kind, const uint4& xj, const uint4& sh, int j) {
    constexpr int K = decltype(kind)::value;
    const float d0 = (float)(int)(xj.x - xi.x + sh.x) * kFixInv;
    const float d1v = (float)(int)(xj.y - xi.y + sh.y) * kFixInv;
    const float d2v = (float)(int)(xj.z - xi.z + sh.z) * kFixInv;
    const float r2 = fmaf(d0, d0, fmaf(d1v, d1v, d2v * d2v));
    if (!(r2 < P.rc2f)) return;
    const float2 gjyz = g1s[j];
    const float4 gj = make_float4(__uint_as_float(xj.w), gjyz.x, gjyz.y, 0.f);
    const float g0 = gj.x - gi.x, g1v = gj.y - gi.y, g2v = gj.z - gi.z;
    const float dg = fmaf(d0, g0, fmaf(d1v, g1v, d2v * g2v));
    const float dgi = fmaf(d0, gi.x, fmaf(d1v, gi.y, d2v * gi.z));
    if constexpr (K == TS_LJ) {
      const float ri2 = __frcp_rn(r2);
      const float s2 = sig2 * ri2, s6 = s2 * s2 * s2, s12 = s6 * s6;
      const float A = -eps24 * fmaf(2.0f, s12, -s6) * ri2;
      const float Bc = eps24 * fmaf(28.0f, s12, -8.0f * s6) * ri2 * ri2;
      const float Bd = Bc * dg;
      gxf[0] = fmaf(A, g0, fmaf(Bd, d0, gxf[0]));
      gxf[1] = fmaf(A, g1v, fmaf(Bd, d1v, gxf[1]));
      gxf[2] = fmaf(A, g2v, fmaf(Bd, d2v, gxf[2]));
      // dphi'/dsigma = -144 eps (4 s^12 - s^6) / (r sigma), dphi'/deps = phi'/eps;
      // dphi/dsigma = 24 eps (2 s^12 - s^6) / sigma, dphi/deps = 4 (s^12 - s^6)
      const float w = dgi * ri2;
      kahan(0, fmaf(-6.0f * eps24 * isig * fmaf(4.0f, s12, -s6), w,
                    hgE * (eps24 * isig * fmaf(2.0f, s12, -s6) - dpc[0])));
      kahan(1, fmaf(-24.0f * fmaf(2.0f, s12, -s6), w, hgE * (4.0f * (s12 - s6) - dpc[1])));
    } else {
      float r, p1, p2, dphi[3], dd1[3];
      PotMath<float>::eval2(P, r2, r, p1, p2, dphi, dd1);
      const float ri = 1.0f / r;
      const float A = p1 * ri;
      const float Bd = (p2 - A) * ri * ri * dg;
      gxf[0] = fmaf(A, g0, fmaf(Bd, d0, gxf[0]));
      gxf[1] = fmaf(A, g1v, fmaf(Bd, d1v, gxf[1]));
      gxf[2] = fmaf(A, g2v, fmaf(Bd, d2v, gxf[2]));
      const float ugi = dgi * ri;
      for (int p = 0; p < 3; p++) kahan(p, fmaf(dd1[p], ugi, hgE * (dphi[p] - dpc[p])));
    }
  };
  auto run = [&](auto kind) {
  if (use_in) {
    // four entries per 16-byte load, the next group in flight ahead of use
    const char* hb = reinterpret_cast<const char*>(hq);
    const char* tb = reinterpret_cast<const char*>(tab);
    const int ng = (nn_first + 3) >> 2;
    auto ent1 = [&](uint32_t ent) {
      const uint32_t off = ent & 0xffffu;
      const uint4 xj = *reinterpret_cast<const uint4*>(hb + off);
      uint4 sh;
      if (staged_tab) {
        sh = *reinterpret_cast<const uint4*>(tb + (ent >> 16));
      } else {
        const uint32_t code = ent >> 16;
        sh = code == kRawFar ? make_uint4(kFarShift, 0u, 0u, 0u)
                             : (code != (uint32_t)kCenter ? __ldg(gtab + code) : make_uint4(0u, 0u, 0u, 0u));
      }
      one(kind, xj, sh, (int)(off >> 4));
    };
    uint4 n0 = g_first;
    for (int gq = 0; gq < ng; gq++) {
      const uint4 e = n0;
      if (gq + 1 < ng) n0 = __ldcs(lp + (int64_t)(gq + 1) * stride);
      ent1(e.x); ent1(e.y); ent1(e.z); ent1(e.w);
    }
  } else {
    const int nn = valid ? A.nn[k] : 0;
    const uint32_t* lp = A.nbr + k;
    auto ent1 = [&](uint32_t ent) {
      const int code = (int)(ent >> kJBits);
      const int j = (int)(ent & kJMask);
      const uint4 sh = code != kCenter ? __ldg(gtab + code) : make_uint4(0, 0, 0, 0);
      one(kind, hq[j], sh, j);
    };
    int q = 0;
    uint32_t n0 = 0, n1 = 0, n2 = 0, n3 = 0;
    if (nn >= 4) { n0 = __ldcs(lp); n1 = __ldcs(lp + stride); n2 = __ldcs(lp + 2 * stride); n3 = __ldcs(lp + 3 * stride); }
    for (; q + 4 <= nn; q += 4) {
      uint32_t e0 = n0, e1 = n1, e2 = n2, e3 = n3;
      if (q + 8 <= nn) {
        const uint32_t* np = lp + (int64_t)(q + 4) * stride;
        n0 = __ldcs(np); n1 = __ldcs(np + stride); n2 = __ldcs(np + 2 * stride); n3 = __ldcs(np + 3 * stride);
      }
      ent1(e0); ent1(e1); ent1(e2); ent1(e3);
    }
    for (; q < nn; q++) ent1(__ldcs(lp + (int64_t)q * stride));
  }
  };
  // one loop per potential kind (uniform over the warp)
  if (P.kind == TS_LJ) run(std::integral_constant<int, TS_LJ>{});
  else if (P.kind == TS_MORSE) run(std::integral_constant<int, TS_MORSE>{});
  else run(std::integral_constant<int, TS_SOFT_SPHERE>{});
  if (valid) {
    const float4 F = A.F[k];
    A.g0[k] = make_float4(gxf[0] - gEf * F.x, gxf[1] - gEf * F.y, gxf[2] - gEf * F.z, 0.f);
  }
  for (int p = 0; p < 3; p++) {
    const double t = warp_sum((double)gtf[p] - (double)gtc[p]);
    if (lane == 0) gpart[4 * (int64_t)wg + p] = accum_part ? gpart[4 * (int64_t)wg + p] + t : t;
  }
}

// upstream gF (caller order, FP64) -> slots (g1 / gd1), scaled per atom by
// scale_dt_over_2m * (1/m) when scale > 0 (the velocity-Verlet kick factor)
template <bool F64>
__global__ void k_import_grad(int64_t Npad, SlotArrays A, const double* __restrict__ g, double kick) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    double c = 1.0;
    if (kick > 0) c = kick * (F64 ? A.minvd[k] : (double)A.vh[k].w);
    double v0 = c * g[3 * (int64_t)p], v1 = c * g[3 * (int64_t)p + 1], v2 = c * g[3 * (int64_t)p + 2];
    if constexpr (F64) { A.gd1[3 * k] = v0; A.gd1[3 * k + 1] = v1; A.gd1[3 * k + 2] = v2; }
    else A.g1[k] = make_float4((float)v0, (float)v1, (float)v2, 0.f);
  }
}

// gPos[p] (+)= gx (slots g0 / gd0)
template <bool F64>
__global__ void k_export_grad(int64_t Npad, SlotArrays A, double* gPos, int accumulate) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    double v[3];
    if constexpr (F64) { for (int c = 0; c < 3; c++) v[c] = A.gd0[3 * k + c]; }
    else { float4 g = A.g0[k]; v[0] = g.x; v[1] = g.y; v[2] = g.z; }
    for (int c = 0; c < 3; c++) gPos[3 * (int64_t)p + c] = (accumulate ? gPos[3 * (int64_t)p + c] : 0.0) + v[c];
  }
}

// parameter gradients: warp partials -> per system (one warp each) -> per potential
__global__ void k_gparam_sys(int32_t B, SysArrays S, const double* __restrict__ gpart, double* gsys) {
  int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (s >= B) return;
  double a[3] = {0, 0, 0};
  for (int w = S.warp_start[s] + lane; w < S.warp_end[s]; w += 32)
    for (int p = 0; p < 3; p++) a[p] += gpart[4 * (int64_t)w + p];
  for (int p = 0; p < 3; p++) a[p] = warp_sum(a[p]);
  if (lane == 0) for (int p = 0; p < 3; p++) gsys[3 * (int64_t)s + p] = a[p];
}
// one warp per potential (at most kMaxPots = 16 warps, one CTA): lanes stride
// over the systems, then a fixed-order warp sum, so the result is deterministic
__global__ void k_gparam_pot(int32_t B, int32_t n_pots, SysArrays S, const double* __restrict__ gsys, double* gParams,
                             int accumulate) {
  int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= n_pots) return;
  double a[3] = {0, 0, 0};
  // a lane's systems s = lane, lane + 32, ... in order, their loads issued
  // eight at a time (one latency per eight systems instead of per system)
  constexpr int kU = 8;
  for (int s0 = lane; s0 < B; s0 += 32 * kU) {
    int pq[kU];
    double g[kU][3];
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const int s = s0 + 32 * u;
      pq[u] = s < B ? S.pot[s] : -1;
      for (int p = 0; p < 3; p++) g[u][p] = s < B ? gsys[3 * (int64_t)s + p] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; u++)
      if (pq[u] == q) for (int p = 0; p < 3; p++) a[p] += g[u][p];
  }
  for (int p = 0; p < 3; p++) a[p] = warp_sum(a[p]);
  if (lane == 0)
    for (int p = 0; p < 3; p++) gParams[3 * q + p] = (accumulate ? gParams[3 * q + p] : 0.0) + a[p];
}

// ---- smeared RDF ---------------------------------------------------------------
// g_k = V/(N(N-1)) sum_{ordered pairs, r < rmax + 4D} exp(-(r-r_k)^2/2D^2) / (sqrt(2 pi) D 4 pi r_k^2)
// Pairs add their Gaussian (|r - r_k| <= 8 D) into a per-warp shared
// histogram; warps add into the system's FP64 row.
template <bool F64>
__global__ void k_rdf(int32_t n_warps, const int32_t* __restrict__ warp_sys, SysArrays S, SlotArrays A,
                      int64_t stride, double rmax, int K, double* g) {
  using T = typename std::conditional<F64, double, float>::type;
  extern __shared__ __align__(8) unsigned char hist_raw[];
  int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  T* hs = reinterpret_cast<T*>(hist_raw) + wib * K;
  for (int q = lane; q < K; q += 32) hs[q] = T(0);
  __syncwarp();
  if (w >= n_warps) return;
  int s = warp_sys[w];
  int64_t k = (int64_t)w * kWarp + lane;
  int nn = A.perm[k] >= 0 ? A.nn[k] : 0;
  int64_t seg = S.seg_start[s];
  T D = (T)(rmax / K), cut2 = (T)((rmax + 4 * rmax / K) * (rmax + 4 * rmax / K));
  for (int q = 0; q < nn; q++) {
    uint32_t ent = A.nbr[q * stride + k];
    int64_t j = seg + (ent & kJMask);
    int code = (int)(ent >> kJBits);
    T r2;
    if constexpr (F64) {
      const double* sh = S.shiftd + 3 * ((int64_t)s * kNCodes + code);
      double d0 = A.xd[3 * j] - A.xd[3 * k] + sh[0], d1 = A.xd[3 * j + 1] - A.xd[3 * k + 1] + sh[1],
             d2 = A.xd[3 * j + 2] - A.xd[3 * k + 2] + sh[2];
      r2 = d0 * d0 + d1 * d1 + d2 * d2;
    } else {
      int64_t t = (int64_t)s * kNCodes + code;
      float4 a = A.xh[j], b = A.xl[j], ia = A.xh[k], ib = A.xl[k], sh = S.shift[2 * t], sl = S.shift[2 * t + 1];
      float d0 = ((a.x - ia.x) + sh.x) + ((b.x - ib.x) + sl.x), d1 = ((a.y - ia.y) + sh.y) + ((b.y - ib.y) + sl.y),
            d2 = ((a.z - ia.z) + sh.z) + ((b.z - ib.z) + sl.z);
      r2 = d0 * d0 + d1 * d1 + d2 * d2;
    }
    if (!(r2 < cut2)) continue;
    T r = sqrt(r2);
    int c = (int)(r / D);
    for (int b = c - 8; b <= c + 8; b++) {
      if (b < 0 || b >= K) continue;
      T rk = (b + T(0.5)) * D, t = (r - rk) / D;
      atomicAdd(&hs[b], exp(T(-0.5) * t * t) / (rk * rk));
    }
  }
  __syncwarp();
  for (int q = lane; q < K; q += 32)
    if (hs[q] != T(0)) atomicAdd(&g[(int64_t)s * K + q], (double)hs[q]);
}

__global__ void k_rdf_norm(int32_t B, SysArrays S, double rmax, int K, double* g) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * K) return;
  int s = (int)(t / K);
  const double* h = S.h + 9 * s;
  double V = fabs(h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) + h[2] * (h[3] * h[7] - h[4] * h[6]));
  double n = S.n_atoms[s], D = rmax / K;
  g[t] *= V / (n * (n - 1)) / (sqrt(2.0 * M_PI) * D * 4.0 * M_PI);
}

// gx_i = -2 sum_j dG(r_ij) u_ij,  dG(r) = sum_k gg_k pref exp(-t^2/2) (-t/D) / r_k^2
template <bool F64>
__global__ void k_rdf_bwd(int32_t n_warps, const int32_t* __restrict__ warp_sys, SysArrays S, SlotArrays A,
                          int64_t stride, double rmax, int K, const double* __restrict__ gg) {
  extern __shared__ __align__(8) unsigned char coef_raw[];
  int wib = threadIdx.x >> 5;
  int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (w >= n_warps) return;
  int s = warp_sys[w];
  int64_t k = (int64_t)w * kWarp + lane;
  bool valid = A.perm[k] >= 0;
  int nn = valid ? A.nn[k] : 0;
  int64_t seg = S.seg_start[s];
  const double* h = S.h + 9 * s;
  double V = fabs(h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) + h[2] * (h[3] * h[7] - h[4] * h[6]));
  double n = S.n_atoms[s], D = rmax / K;
  double pref = V / (n * (n - 1)) / (sqrt(2.0 * M_PI) * D * 4.0 * M_PI);
  const double* ggs = gg + (int64_t)s * K;
  double cut2 = (rmax + 4 * D) * (rmax + 4 * D);
  double gx[3] = {0, 0, 0};
  if constexpr (F64) {
    for (int q = 0; q < nn; q++) {
      uint32_t ent = A.nbr[q * stride + k];
      int64_t j = seg + (ent & kJMask);
      int code = (int)(ent >> kJBits);
      double d[3];
      const double* sh = S.shiftd + 3 * ((int64_t)s * kNCodes + code);
      for (int c = 0; c < 3; c++) d[c] = A.xd[3 * j + c] - A.xd[3 * k + c] + sh[c];
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (!(r2 < cut2)) continue;
      double r = sqrt(r2);
      int c = (int)(r / D);
      double dG = 0;
      for (int b = c - 8; b <= c + 8; b++) {
        if (b < 0 || b >= K) continue;
        double rk = (b + 0.5) * D, t = (r - rk) / D;
        dG += ggs[b] * pref * exp(-0.5 * t * t) / (rk * rk) * (-t / D);
      }
      for (int cc = 0; cc < 3; cc++) gx[cc] -= 2.0 * dG * d[cc] / r;
    }
    if (valid) for (int c = 0; c < 3; c++) A.gd0[3 * k + c] = gx[c];
  } else {
    // FP32: the per-bin factor gg_b pref / (r_b^2 D) is staged once per warp
    // in shared memory, so a pair's 17 bins cost one exponential each and no
    // FP64 arithmetic (a small fraction of the FP32 rate on this part)
    float* cf = reinterpret_cast<float*>(coef_raw) + wib * K;
    for (int b = lane; b < K; b += 32) {
      double rk = (b + 0.5) * D;
      cf[b] = (float)(ggs[b] * pref / (rk * rk * D));
    }
    __syncwarp();
    const float Df = (float)D, iD = (float)(1.0 / D), cut2f = (float)cut2;
    float gxf[3] = {0.f, 0.f, 0.f};
    for (int q = 0; q < nn; q++) {
      uint32_t ent = __ldg(A.nbr + q * stride + k);
      int64_t j = seg + (ent & kJMask);
      int code = (int)(ent >> kJBits);
      int64_t t = (int64_t)s * kNCodes + code;
      float4 a = A.xh[j], b = A.xl[j], ia = A.xh[k], ib = A.xl[k], sh = S.shift[2 * t], sl = S.shift[2 * t + 1];
      float d0 = ((a.x - ia.x) + sh.x) + ((b.x - ib.x) + sl.x);
      float d1 = ((a.y - ia.y) + sh.y) + ((b.y - ib.y) + sl.y);
      float d2 = ((a.z - ia.z) + sh.z) + ((b.z - ib.z) + sl.z);
      float r2 = d0 * d0 + d1 * d1 + d2 * d2;
      if (!(r2 < cut2f)) continue;
      float r = sqrtf(r2);
      int c = (int)(r * iD);
      float dG = 0.f;
      for (int bb = c - 8; bb <= c + 8; bb++) {
        if (bb < 0 || bb >= K) continue;
        float tt = (r - (bb + 0.5f) * Df) * iD;
        dG -= cf[bb] * expf(-0.5f * tt * tt) * tt;
      }
      float f = 2.0f * dG / r;
      gxf[0] -= f * d0; gxf[1] -= f * d1; gxf[2] -= f * d2;
    }
    if (valid) A.g0[k] = make_float4(gxf[0], gxf[1], gxf[2], 0.f);
  }
}

// velocity-Verlet reverse step, caller-order vectors:
// stage 1: ub = ax + tmp; vh = av + dt ub (ub kept in ax, vh in av)
// stage 2: ax = ub + tmp
template <bool F64>
__global__ void k_vv_adj(int64_t Npad, SlotArrays A, double* ax, double* av, double dt, int stage) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    double t[3];
    if constexpr (F64) { for (int c = 0; c < 3; c++) t[c] = A.gd0[3 * k + c]; }
    else { float4 g = A.g0[k]; t[0] = g.x; t[1] = g.y; t[2] = g.z; }
    for (int c = 0; c < 3; c++) {
      int64_t o = 3 * (int64_t)p + c;
      double ub = ax[o] + t[c];
      ax[o] = ub;
      if (stage == 1) av[o] = av[o] + dt * ub;
    }
  }
}

}  // namespace ts

using namespace ts;

namespace ts {

static int egrid(ts_batch* b) {
  int64_t g = (b->Npad + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 148 * 16 ? 148 * 16 : g));
}

bool bwd_attributes(ts_batch* b) {
  return cuda_ok(b, cudaFuncSetAttribute(k_pair_bwd_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kPairTabBytes + kBwdRecord * kSmallMax)), "smem attribute");
}

// parameter gradients of the per-warp partials into gParams
static void gparam_reduce(ts_batch* b, cudaStream_t st, double* gParams, int accumulate_params) {
  k_gparam_sys<<<(b->B * 32 + 127) / 128, 128, 0, st>>>(b->B, b->S, b->d_gparam_part, b->d_scal);
  k_gparam_pot<<<1, 32 * b->n_pots, 0, st>>>(b->B, b->n_pots, b->S, b->d_scal, gParams, accumulate_params);
  b->launches += 2;
}

// gx of the current gF (in g1 / gd1) into slots g0 / gd0; per-warp parameter
// partials written (accum_part = 0) or added to (1); with gParams, reduced into it
static void backward_core(ts_batch* b, cudaStream_t st, const double* gE, const double* gS, double* gParams,
                          int accumulate_params, int accum_part = 0) {
  int blocks = (int)(((int64_t)b->nwarps * 32 + 127) / 128);
  // mixed precision without a stress upstream: systems up to kSmallMax atoms from shared memory
  const size_t shm = kPairTabBytes + (size_t)kBwdRecord * b->nst_max;
  const bool small = !b->f64 && !gS && b->use_small_pair && b->bwd_small && b->n_items > 0;
  if (small) {
    k_pair_bwd_small<<<b->n_items, 32 * b->tune.item_warps, shm, st>>>(
        b->n_items, b->d_items, b->d_item_sys, b->S, b->A, b->d_pots, b->Ncap, gE, b->d_gparam_part, accum_part);
    b->launches++;
  }
  if (!small || b->n_large > 0) {
    auto kern = b->f64 ? (gS ? k_pair_bwd<true, true> : k_pair_bwd<true, false>)
                       : (gS ? k_pair_bwd<false, true> : k_pair_bwd<false, false>);
    kern<<<blocks, 128, 0, st>>>(b->nwarps, b->d_warp_sys, b->S, b->A, b->d_pots, b->Ncap, gE, gS,
                                 b->d_gparam_part, accum_part, small ? 1 : 0);
    b->launches++;
  }
  if (gParams) gparam_reduce(b, st, gParams, accumulate_params);
}

static ts_status rdf_check(ts_batch* b, double rmax, int K) {
  if (!(rmax > 0) || K < 1 || K > 4096) return fail(b, TS_ERR_INVALID_ARG, "bad rmax or K");
  for (int q = 0; q < b->n_pots; q++)
    if (b->rc[q] + b->pots[q].skin * b->tune.skin_scale < rmax + 4.0 * rmax / K)
      return fail(b, TS_ERR_INVALID_ARG, "neighbour lists shorter than rmax + 4 D: raise the skin");
  return TS_OK;
}

}  // namespace ts

extern "C" ts_status ts_pair_forces_backward(ts_batch* b, ts_state* s, const double* gF, const double* gE,
                                             const double* gStress, double* gPos, double* gParams, int accumulate,
                                             void* stream) {
  ts_status r = check_state(b, s, false);
  if (r != TS_OK) return r;
  if (!gF || (!gPos && !gParams)) return fail(b, TS_ERR_INVALID_ARG, "null gradient pointer");
  cudaStream_t st = (cudaStream_t)stream;
  r = prologue(b, s, st, false);
  if (r != TS_OK) return r;
  ensure_forces(b, st);
  int g = egrid(b);
  if (b->f64) k_import_grad<true><<<g, 256, 0, st>>>(b->Npad, b->A, gF, 0.0);
  else k_import_grad<false><<<g, 256, 0, st>>>(b->Npad, b->A, gF, 0.0);
  b->launches++;
  backward_core(b, st, gE, gStress, gParams, accumulate);
  if (gPos) {
    if (b->f64) k_export_grad<true><<<g, 256, 0, st>>>(b->Npad, b->A, gPos, accumulate);
    else k_export_grad<false><<<g, 256, 0, st>>>(b->Npad, b->A, gPos, accumulate);
    b->launches++;
  }
  export_state(b, st, s->pos, nullptr);
  return cuda_ok(b, cudaGetLastError(), "ts_pair_forces_backward") ? TS_OK : TS_ERR_CUDA;
}

extern "C" ts_status ts_rdf(ts_batch* b, ts_state* s, double rmax, int K, double* g, void* stream) {
  ts_status r = check_state(b, s, false);
  if (r != TS_OK) return r;
  if (!g) return fail(b, TS_ERR_INVALID_ARG, "null output");
  if ((r = rdf_check(b, rmax, K)) != TS_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  r = prologue(b, s, st, false);
  if (r != TS_OK) return r;
  relist(b, st, false);
  if (!cuda_ok(b, cudaMemsetAsync(g, 0, sizeof(double) * K * (size_t)b->B, st), "memset")) return TS_ERR_CUDA;
  int threads = 128;
  size_t shm = (b->f64 ? sizeof(double) : sizeof(float)) * K * (threads / 32);
  if (shm > 48 * 1024) return fail(b, TS_ERR_INVALID_ARG, "K too large");
  int blocks = (int)(((int64_t)b->nwarps * 32 + threads - 1) / threads);
  if (b->f64) k_rdf<true><<<blocks, threads, shm, st>>>(b->nwarps, b->d_warp_sys, b->S, b->A, b->Ncap, rmax, K, g);
  else k_rdf<false><<<blocks, threads, shm, st>>>(b->nwarps, b->d_warp_sys, b->S, b->A, b->Ncap, rmax, K, g);
  k_rdf_norm<<<(int)(((int64_t)b->B * K + 255) / 256), 256, 0, st>>>(b->B, b->S, rmax, K, g);
  b->launches += 2;
  export_state(b, st, s->pos, nullptr);
  return cuda_ok(b, cudaGetLastError(), "ts_rdf") ? TS_OK : TS_ERR_CUDA;
}

extern "C" ts_status ts_rdf_backward(ts_batch* b, ts_state* s, double rmax, int K, const double* gg, double* gPos,
                                     void* stream) {
  ts_status r = check_state(b, s, false);
  if (r != TS_OK) return r;
  if (!gg || !gPos) return fail(b, TS_ERR_INVALID_ARG, "null pointer");
  if ((r = rdf_check(b, rmax, K)) != TS_OK) return r;
  const size_t shm = b->f64 ? 0 : sizeof(float) * (size_t)K * 4;   // per-bin factors, one row per warp
  if (shm > 48 * 1024) return fail(b, TS_ERR_INVALID_ARG, "K too large");
  cudaStream_t st = (cudaStream_t)stream;
  r = prologue(b, s, st, false);
  if (r != TS_OK) return r;
  relist(b, st, false);
  int blocks = (int)(((int64_t)b->nwarps * 32 + 127) / 128);
  if (b->f64) k_rdf_bwd<true><<<blocks, 128, 0, st>>>(b->nwarps, b->d_warp_sys, b->S, b->A, b->Ncap, rmax, K, gg);
  else k_rdf_bwd<false><<<blocks, 128, shm, st>>>(b->nwarps, b->d_warp_sys, b->S, b->A, b->Ncap, rmax, K, gg);
  int g = egrid(b);
  if (b->f64) k_export_grad<true><<<g, 256, 0, st>>>(b->Npad, b->A, gPos, 1);
  else k_export_grad<false><<<g, 256, 0, st>>>(b->Npad, b->A, gPos, 1);
  b->launches += 2;
  export_state(b, st, s->pos, nullptr);
  return cuda_ok(b, cudaGetLastError(), "ts_rdf_backward") ? TS_OK : TS_ERR_CUDA;
}

extern "C" ts_status ts_vv_adjoint_step(ts_batch* b, ts_state* s, const double* x_next, double dt, double* ax,
                                        double* av, double* gParams, void* stream) {
  ts_status r = check_state(b, s, false);
  if (r != TS_OK) return r;
  if (!x_next || !ax || !av || !gParams || !(dt > 0)) return fail(b, TS_ERR_INVALID_ARG, "bad adjoint arguments");
  cudaStream_t st = (cudaStream_t)stream;
  int g = egrid(b);
  // (1) at u = x_{t+1}: ubar = ax + c J(u)^T av
  ts_state su = *s;
  su.pos = const_cast<double*>(x_next);
  r = prologue(b, &su, st, true);
  if (r != TS_OK) return r;
  relist(b, st, false);
  if (b->f64) k_import_grad<true><<<g, 256, 0, st>>>(b->Npad, b->A, av, 0.5 * dt);
  else k_import_grad<false><<<g, 256, 0, st>>>(b->Npad, b->A, av, 0.5 * dt);
  b->launches++;
  backward_core(b, st, nullptr, nullptr, gParams, 1);
  if (b->f64) k_vv_adj<true><<<g, 256, 0, st>>>(b->Npad, b->A, ax, av, dt, 1);
  else k_vv_adj<false><<<g, 256, 0, st>>>(b->Npad, b->A, ax, av, dt, 1);
  b->launches++;
  // (2) at x_t: ax = ubar + c J(x_t)^T vh, av = vh
  r = prologue(b, s, st, false);
  if (r != TS_OK) return r;
  relist(b, st, false);
  if (b->f64) k_import_grad<true><<<g, 256, 0, st>>>(b->Npad, b->A, av, 0.5 * dt);
  else k_import_grad<false><<<g, 256, 0, st>>>(b->Npad, b->A, av, 0.5 * dt);
  b->launches++;
  backward_core(b, st, nullptr, nullptr, gParams, 1);
  if (b->f64) k_vv_adj<true><<<g, 256, 0, st>>>(b->Npad, b->A, ax, av, dt, 2);
  else k_vv_adj<false><<<g, 256, 0, st>>>(b->Npad, b->A, ax, av, dt, 2);
  b->launches++;
  return cuda_ok(b, cudaGetLastError(), "ts_vv_adjoint_step") ? TS_OK : TS_ERR_CUDA;
}

namespace ts {

// The reverse sweep of ts_vv_adjoint_segment.  With ax, av the adjoints of
// (x, v) at frame t0+n, the n reverse velocity-Verlet steps issued one at a
// time take at every interior frame m two products c J(x_m)^T av with the same
// av (the closing half of the reverse of step m+1 and the opening half of the
// reverse of step m, c = dt/2).  The sweep takes that product once, with weight
// dt, as the forward loop merges the half kicks of adjacent steps:
//   frame n:          ax += (dt/2) J(x_n)^T av;  av += dt ax
//   frames n-1 .. 1:  ax += dt J(x_m)^T av;      av += dt ax
//   frame 0:          ax += (dt/2) J(x_0)^T av
// (J^T av of the pair backward; its parameter part is summed per warp over
// the frames and reduced into gParams once; the RDF gradient at an observed
// frame m >= 1 is added to ax first).  The cell is the same at every frame,
// so only the first import computes the geometry and image shifts.
static ts_status adjoint_sweep(ts_batch* b, const ts_state* s, const double* frames, int n, int64_t t0, double dt,
                               double* ax, double* av, double* gParams, int rdf_every, double rmax, int K,
                               const double* gg, cudaStream_t st) {
  const int64_t stride = 3 * (int64_t)s->n_atoms;
  const int g = egrid(b);
  const int blocks = (int)(((int64_t)b->nwarps * 32 + 127) / 128);
  const size_t rshm = b->f64 ? 0 : sizeof(float) * (size_t)K * 4;
  for (int m = n; m >= 0; m--) {
    ts_state sm = *s;
    sm.pos = const_cast<double*>(frames + (int64_t)m * stride);
    sm.vel = nullptr;
    ts_status r = prologue(b, &sm, st, false, false, m == n);
    if (r != TS_OK) return r;
    relist(b, st, false);
    if (rdf_every > 0 && m >= 1 && (t0 + m) % rdf_every == 0) {
      if (b->f64) k_rdf_bwd<true><<<blocks, 128, 0, st>>>(b->nwarps, b->d_warp_sys, b->S, b->A, b->Ncap, rmax, K, gg);
      else k_rdf_bwd<false><<<blocks, 128, rshm, st>>>(b->nwarps, b->d_warp_sys, b->S, b->A, b->Ncap, rmax, K, gg);
      if (b->f64) k_export_grad<true><<<g, 256, 0, st>>>(b->Npad, b->A, ax, 1);
      else k_export_grad<false><<<g, 256, 0, st>>>(b->Npad, b->A, ax, 1);
      b->launches += 2;
    }
    const double c = (m == n || m == 0) ? 0.5 * dt : dt;
    if (b->f64) k_import_grad<true><<<g, 256, 0, st>>>(b->Npad, b->A, av, c);
    else k_import_grad<false><<<g, 256, 0, st>>>(b->Npad, b->A, av, c);
    b->launches++;
    backward_core(b, st, nullptr, nullptr, nullptr, 1, m < n ? 1 : 0);
    const int stage = m > 0 ? 1 : 2;
    if (b->f64) k_vv_adj<true><<<g, 256, 0, st>>>(b->Npad, b->A, ax, av, dt, stage);
    else k_vv_adj<false><<<g, 256, 0, st>>>(b->Npad, b->A, ax, av, dt, stage);
    b->launches++;
  }
  gparam_reduce(b, st, gParams, 1);
  return cuda_ok(b, cudaGetLastError(), "adjoint sweep") ? TS_OK : TS_ERR_CUDA;
}

}  // namespace ts

extern "C" ts_status ts_vv_adjoint_segment(ts_batch* b, ts_state* s, const double* frames, int n, int64_t t0,
                                           double dt, double* ax, double* av, double* gParams, int rdf_every,
                                           double rmax, int K, const double* gg, void* stream) {
  ts_status r = check_state(b, s, false);
  if (r != TS_OK) return r;
  if (!frames || n < 1 || !ax || !av || !gParams || !(dt > 0) || (rdf_every > 0 && !gg))
    return fail(b, TS_ERR_INVALID_ARG, "bad adjoint segment arguments");
  if (rdf_every > 0) {
    if ((r = rdf_check(b, rmax, K)) != TS_OK) return r;
    if (!b->f64 && sizeof(float) * (size_t)K * 4 > 48 * 1024) return fail(b, TS_ERR_INVALID_ARG, "K too large");
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(b->cfg.device);
  // replayed as a CUDA graph once the layout is settled: the sweep's launches
  // depend only on the arguments in the key (and on which frames are observed)
  const bool settled = b->topo_valid && !b->first_import && s->n_systems == b->B && s->n_atoms == b->N;
  if (!(b->use_graphs && st != nullptr && settled))
    return adjoint_sweep(b, s, frames, n, t0, dt, ax, av, gParams, rdf_every, rmax, K, gg, st);
  graph_cache_check(b);
  ts_graph_entry key;
  key.kind = 1;
  key.n_steps = n;
  key.stream = st;
  const void* ptrs[8] = {frames, ax, av, gParams, gg, s->cell, s->pbc, nullptr};
  for (int q = 0; q < 8; q++) key.ptr[q] = ptrs[q];
  key.ival[0] = rdf_every;
  key.ival[1] = rdf_every > 0 ? ((t0 % rdf_every) + rdf_every) % rdf_every : 0;
  key.dval[0] = dt;
  key.dval[1] = rdf_every > 0 ? rmax : 0.0;
  key.md_kind = rdf_every > 0 ? K : 0;
  auto same = [&](const ts_graph_entry& e) {
    if (e.kind != 1 || e.n_steps != n || e.stream != st || e.md_kind != key.md_kind) return false;
    for (int q = 0; q < 8; q++) if (e.ptr[q] != key.ptr[q]) return false;
    return e.ival[0] == key.ival[0] && e.ival[1] == key.ival[1] && e.dval[0] == key.dval[0] && e.dval[1] == key.dval[1];
  };
  // a key seen for the first time is only remembered (a one-off sweep, such
  // as one over a whole stored trajectory, is issued directly: its launches
  // are queued far ahead of the device); its second call is captured
  int seen = -1;
  for (size_t q = 0; q < b->graphs.size(); q++) {
    ts_graph_entry& e = b->graphs[q];
    if (!same(e)) continue;
    if (!e.exec) { seen = (int)q; break; }
    if (!cuda_ok(b, cudaGraphLaunch(e.exec, st), "cudaGraphLaunch")) return TS_ERR_CUDA;
    b->launches += e.kernels;
    return TS_OK;
  }
  if (seen < 0) {
    graph_store(b, key);
    return adjoint_sweep(b, s, frames, n, t0, dt, ax, av, gParams, rdf_every, rmax, K, gg, st);
  }
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return adjoint_sweep(b, s, frames, n, t0, dt, ax, av, gParams, rdf_every, rmax, K, gg, st);
  }
  const int64_t l0 = b->launches;
  r = adjoint_sweep(b, s, frames, n, t0, dt, ax, av, gParams, rdf_every, rmax, K, gg, st);
  const int64_t nk = b->launches - l0;
  b->launches = l0;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (r != TS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return r;
  }
  cudaGraphExec_t exec = nullptr;
  if (e != cudaSuccess || cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return adjoint_sweep(b, s, frames, n, t0, dt, ax, av, gParams, rdf_every, rmax, K, gg, st);
  }
  cudaGraphDestroy(graph);
  b->graphs[seen].exec = exec;
  b->graphs[seen].kernels = nk;
  if (!cuda_ok(b, cudaGraphLaunch(exec, st), "cudaGraphLaunch")) return TS_ERR_CUDA;
  b->launches += nk;
  return TS_OK;
}
