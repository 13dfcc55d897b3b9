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
  asm volatile("griddepcontrol.launch_dependents;");   // as in k_pair_small
  int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (w >= n_warps) return;
  int s = warp_sys[w];
  if (pair_skip(S, s, filter)) return;
  if (skip_small && S.n_atoms[s] <= kSmallMax) return;   // handled by k_pair_small
  // inner-list mode (MD steps): a system flagged for pruning, or re-listed in
  // this pass, runs its full list and writes the inner list on the way
  const bool refresh = inner && (S.prune[s] || need_relist(S, s));   // warp-uniform
  const bool use_in = inner && !refresh;
  int64_t k = (int64_t)w * kWarp + lane;
  const DevPot P = pots[S.pot[s]];
  bool valid = A.perm[k] >= 0;
  int nn = valid ? (use_in ? A.nn_in : A.nn)[k] : 0;
  int cin = 0;
  // entry q of the list read (the inner list in its grouped layout, Verlet-list format here)
  auto entry = [&](int q) -> uint32_t {
    return use_in ? __ldcs(A.nbr_in + inner_at(q, k, stride)) : __ldcs(A.nbr + (int64_t)q * stride + k);
  };
  auto keep = [&](uint32_t ent) { A.nbr_in[inner_at(cin++, k, stride)] = ent; };
  if (refresh && lane == 0) S.infmt[s] = kInnerVerlet;
  int64_t seg = S.seg_start[s];
  if constexpr (F64) {
    const double* tab = S.shiftd + 3 * (int64_t)s * kNCodes;
    double xi0 = A.xd[3 * k], xi1 = A.xd[3 * k + 1], xi2 = A.xd[3 * k + 2];
    double f0 = 0, f1 = 0, f2 = 0, e = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    for (int q = 0; q < nn; q++) {
      uint32_t ent = entry(q);
      int64_t j = seg + (ent & kJMask);
      int code = (int)(ent >> kJBits);
      double d0 = A.xd[3 * j] - xi0, d1 = A.xd[3 * j + 1] - xi1, d2 = A.xd[3 * j + 2] - xi2;
      if (code != kCenter) { d0 += tab[3 * code]; d1 += tab[3 * code + 1]; d2 += tab[3 * code + 2]; }
      double r2 = d0 * d0 + d1 * d1 + d2 * d2;
      if (refresh && r2 < P.rin2d) keep(ent);
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
      if (refresh && r2 < P.rin2f) keep(ent);
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
    int q = 0;
    uint32_t n0 = 0, n1 = 0, n2 = 0, n3 = 0;
    if (nn >= 4) { n0 = entry(0); n1 = entry(1); n2 = entry(2); n3 = entry(3); }
    for (; q + 4 <= nn; q += 4) {
      uint32_t e0 = n0, e1 = n1, e2 = n2, e3 = n3;
      if (q + 8 <= nn) { n0 = entry(q + 4); n1 = entry(q + 5); n2 = entry(q + 6); n3 = entry(q + 7); }
      float4 x0 = __ldg(ph + (e0 & kJMask)), l0 = __ldg(pl + (e0 & kJMask));
      float4 x1 = __ldg(ph + (e1 & kJMask)), l1 = __ldg(pl + (e1 & kJMask));
      float4 x2 = __ldg(ph + (e2 & kJMask)), l2 = __ldg(pl + (e2 & kJMask));
      float4 x3 = __ldg(ph + (e3 & kJMask)), l3 = __ldg(pl + (e3 & kJMask));
      one(e0, x0, l0); one(e1, x1, l1); one(e2, x2, l2); one(e3, x3, l3);
    }
    for (; q < nn; q++) {
      uint32_t ent = entry(q);
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
//   w = computed warps (at most the CTA's warps, 4 or 8: the tuned item size).
// An item is a run of consecutive warps that may straddle systems; its staged
// range holds every system those warps belong to (at most kSmallMax slots),
// so every neighbour gather is a shared-memory read.  Staged record per atom:
// 16 B, the fixed-point coordinates (units of 2^-26 A, modulo 2^32); a pair
// vector is the exact integer difference plus the fixed-point image shift,
// converted once to FP32 (one rounding, the same as the double-float form).
//
// Three list modes per warp (a warp belongs to one system):
//  * inner list, kInnerTab (MD steps, the common case): the system's image
//    shifts that its lists reference (|n_a| <= b_a per axis, at most 125
//    images) are staged in shared memory (one table per warp),
//    and an entry holds the byte offsets of the neighbour's record and of its
//    shift, so an entry costs a 16-byte share of a vector load, two shared
//    loads, the integer pair vector and the potential;
//  * inner list, kInnerRaw (lists reaching more images than a table holds):
//    the same loop, the entries holding the image code and the shift read
//    through L1;
//  * Verlet list (non-MD calls, and MD steps in which the system is re-listed
//    or an atom moved half the inner skin since the last filtering): the full
//    list with global image shifts; in MD steps the launch writes the inner
//    list on the way (entries within rc + inner skin, in list order, padded
//    to a multiple of four with entries whose shift is 32 A).
// Every mode evaluates a pair with the same function (pair_fixed) from the
// same bits and sums the entries of the inner list in list order; pairs
// beyond rc add exactly zero, so forces do not depend on which list was read.
constexpr int kPairSmallThreads = 256;
constexpr int kItemWarps = kPairSmallThreads / kWarp;
constexpr int kSmallRecord = 16;                                    // staged bytes per atom
constexpr size_t kPairTabBytes = (size_t)kItemWarps * kTabEntries * 16;   // image tables, one per warp
constexpr float kFix2 = 4503599627370496.0f;                       // 2^52: r^2 in fixed-point units
constexpr uint32_t kFarShift = 0x7fffffffu;                        // 32 A: beyond every cutoff this kernel takes
constexpr uint32_t kRawFar = 0xffffu;                              // kInnerRaw padding entry

// Per-warp constants of the potential in fixed-point units (u = 2^26 d):
// F_i += fu u with fu = phi'(r) / (r 2^26), r2u = u.u = 2^52 r^2.
struct PairFix {
  float rc2u;      // rc^2 2^52
  float a, b, c;   // LJ: sigma^2 2^52, -24 eps 2^26, 4 eps;  Morse: alpha, r0, 2 alpha D;  SS: 1/(sigma 2^26), -eps/sigma, eps/alpha
  float d, e;      // Morse: D, 2^-26;  SS: alpha
};

template <int K>
__device__ __forceinline__ PairFix pair_fix(const DevPot& P) {
  PairFix C;
  C.rc2u = P.rc2f * kFix2;
  if constexpr (K == TS_LJ) {
    C.a = (P.pf[0] * P.pf[0]) * kFix2; C.b = -24.0f * P.pf[1] * kFix; C.c = 4.0f * P.pf[1]; C.d = 0.f; C.e = 0.f;
  } else if constexpr (K == TS_MORSE) {
    C.a = P.pf[1]; C.b = P.pf[2]; C.c = 2.0f * P.pf[1] * P.pf[0]; C.d = P.pf[0]; C.e = kFixInv;
  } else {
    C.a = P.sinvf * kFixInv; C.b = -P.pf[1] * P.sinvf; C.c = P.pf[1] / P.pf[2]; C.d = P.pf[2]; C.e = 0.f;
  }
  return C;
}

// fu and (EW) the unshifted pair energy phi of a pair with r2u = u.u > 0;
// fu is zero beyond the cutoff (selected, so that out-of-range entries add
// exactly zero and a round of entries has no branch).  Every rounding is
// spelled out (fmaf, __fmul_rn), so that the two-entry form below, whose
// lanes repeat these operations in packed f32x2 instructions, gives the same
// bits as this one whatever the compiler contracts.
template <int K, bool EW>
__device__ __forceinline__ float pair_fixed(const PairFix& C, float r2u, float& phi) {
  float fu;
  if constexpr (K == TS_LJ) {
    float ri2;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ri2) : "f"(r2u));   // ~1 ulp; the LJ terms are well conditioned
    const float s2 = C.a * ri2, s6 = s2 * s2 * s2;
    fu = fmaf(s6, 2.0f * C.b, -C.b) * (s6 * ri2);      // -24 eps s6 (2 s6 - 1) / r^2 / 2^26
    if (EW) phi = C.c * fmaf(s6, s6, -s6);
  } else if constexpr (K == TS_MORSE) {
    // r correctly rounded: it sets the exponent's argument, where the stiff
    // Morse force amplifies any error; 1/r only scales the result
    const float r = __fmul_rn(sqrtf(r2u), C.e);
    const float e = __expf(C.a * fmaf(r, -1.0f, C.b));
    fu = C.c * e * fmaf(e, -1.0f, 1.0f) * rsqrtf(r2u);
    if (EW) phi = C.d * fmaf(e, e, -2.0f * e);
  } else {
    const float ri = rsqrtf(r2u);
    const float t = fmaf(r2u * ri, -C.a, 1.0f);         // 1 - r/sigma in one fused operation
    const float ta1 = (C.d == 2.0f) ? t : __powf(t, C.d - 1.0f);
    fu = C.b * ta1 * ri;
    if (EW) phi = C.c * ta1 * t;
  }
  return r2u < C.rc2u ? fu : 0.f;
}

// Two entries at once: each lane of a packed f32x2 instruction rounds as the
// scalar operation does, so (fa, fb) are pair_fixed(ra) and pair_fixed(rb)
// bit for bit; the FP32 arithmetic takes about half the issue slots.
template <int K, bool EW>
__device__ __forceinline__ void pair_fixed2(const PairFix& C, float ra, float rb, float& fa, float& fb, float& pa,
                                            float& pb) {
  const unsigned long long R2 = f2_pack(ra, rb);
  unsigned long long FU, PHI = 0;
  if constexpr (K == TS_LJ) {
    float ia, ib;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ia) : "f"(ra));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ib) : "f"(rb));
    const unsigned long long RI = f2_pack(ia, ib);
    const unsigned long long S2 = f2_mul(f2_splat(C.a), RI);
    const unsigned long long S6 = f2_mul(f2_mul(S2, S2), S2);
    FU = f2_mul(f2_fma(S6, f2_splat(2.0f * C.b), f2_splat(-C.b)), f2_mul(S6, RI));
    if (EW) PHI = f2_mul(f2_splat(C.c), f2_fma(S6, S6, f2_mul(S6, f2_splat(-1.0f))));
  } else if constexpr (K == TS_MORSE) {
    const unsigned long long R = f2_mul(f2_pack(sqrtf(ra), sqrtf(rb)), f2_splat(C.e));
    const unsigned long long X = f2_mul(f2_splat(C.a), f2_fma(R, f2_splat(-1.0f), f2_splat(C.b)));
    float xa, xb;
    f2_unpack(X, xa, xb);
    const unsigned long long E = f2_pack(__expf(xa), __expf(xb));
    FU = f2_mul(f2_mul(f2_mul(f2_splat(C.c), E), f2_fma(E, f2_splat(-1.0f), f2_splat(1.0f))),
                f2_pack(rsqrtf(ra), rsqrtf(rb)));
    if (EW) PHI = f2_mul(f2_splat(C.d), f2_fma(E, E, f2_mul(E, f2_splat(-2.0f))));
  } else {
    const unsigned long long RI = f2_pack(rsqrtf(ra), rsqrtf(rb));
    const unsigned long long T = f2_fma(f2_mul(R2, RI), f2_splat(-C.a), f2_splat(1.0f));
    unsigned long long TA1 = T;
    if (C.d != 2.0f) {
      float ta, tb;
      f2_unpack(T, ta, tb);
      TA1 = f2_pack(__powf(ta, C.d - 1.0f), __powf(tb, C.d - 1.0f));
    }
    FU = f2_mul(f2_mul(f2_splat(C.b), TA1), RI);
    if (EW) PHI = f2_mul(f2_mul(f2_splat(C.c), TA1), T);
  }
  f2_unpack(FU, fa, fb);
  if (EW) f2_unpack(PHI, pa, pb);
  fa = ra < C.rc2u ? fa : 0.f;
  fb = rb < C.rc2u ? fb : 0.f;
}

template <bool EW>
struct PairSums {
  float f0 = 0.f, f1 = 0.f, f2 = 0.f, e = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f, w4 = 0.f, w5 = 0.f;
};

// integer pair vector of staged record xj, image shift sh (fixed point), against atom xi
__device__ __forceinline__ void pair_vec(const uint4& xi, const uint4& xj, const uint4& sh, float& u0, float& u1,
                                         float& u2) {
  u0 = (float)(int)(xj.x - xi.x + sh.x);
  u1 = (float)(int)(xj.y - xi.y + sh.y);
  u2 = (float)(int)(xj.z - xi.z + sh.z);
}

// one entry's contribution, summed in list order
template <bool EW>
__device__ __forceinline__ void pair_acc(const PairFix& C, float phic, float u0, float u1, float u2, float r2u,
                                         float fu, float phi, PairSums<EW>& A) {
  A.f0 = fmaf(fu, u0, A.f0); A.f1 = fmaf(fu, u1, A.f1); A.f2 = fmaf(fu, u2, A.f2);
  if (EW) {
    A.e += r2u < C.rc2u ? 0.5f * (phi - phic) : 0.f;
    const float hf = fu * (0.5f * kFixInv);            // W += 1/2 (phi'/r) d d = 1/2 fu 2^-26 u u
    const float h0 = hf * u0, h1 = hf * u1;
    A.w0 = fmaf(h0, u0, A.w0); A.w1 = fmaf(h1, u1, A.w1); A.w2 = fmaf(hf * u2, u2, A.w2);
    A.w3 = fmaf(h0, u1, A.w3); A.w4 = fmaf(h0, u2, A.w4); A.w5 = fmaf(h1, u2, A.w5);
  }
}

// one entry: staged record xj, image shift sh (fixed point) against atom xi
template <int K, bool EW>
__device__ __forceinline__ float pair_add(const PairFix& C, float phic, const uint4& xi, const uint4& xj,
                                          const uint4& sh, PairSums<EW>& A) {
  float u0, u1, u2;
  pair_vec(xi, xj, sh, u0, u1, u2);
  const float r2u = fmaf(u0, u0, fmaf(u1, u1, u2 * u2));
  float phi = 0.f;
  const float fu = pair_fixed<K, EW>(C, r2u, phi);
  pair_acc<EW>(C, phic, u0, u1, u2, r2u, fu, phi, A);
  return r2u;
}

// two entries (a, then b): the same bits as two pair_add calls in that order
template <int K, bool EW>
__device__ __forceinline__ void pair_add2(const PairFix& C, float phic, const uint4& xi, const uint4& xa,
                                          const uint4& sa, const uint4& xb, const uint4& sb, PairSums<EW>& A,
                                          float& r2a, float& r2b) {
  float a0, a1, a2, b0, b1, b2;
  pair_vec(xi, xa, sa, a0, a1, a2);
  pair_vec(xi, xb, sb, b0, b1, b2);
  const unsigned long long U0 = f2_pack(a0, b0), U1 = f2_pack(a1, b1), U2 = f2_pack(a2, b2);
  f2_unpack(f2_fma(U0, U0, f2_fma(U1, U1, f2_mul(U2, U2))), r2a, r2b);
  float fa, fb, pa = 0.f, pb = 0.f;
  pair_fixed2<K, EW>(C, r2a, r2b, fa, fb, pa, pb);
  pair_acc<EW>(C, phic, a0, a1, a2, r2a, fa, pa, A);
  pair_acc<EW>(C, phic, b0, b1, b2, r2b, fb, pb, A);
}

template <bool EW>
__global__ void __launch_bounds__(kPairSmallThreads, EW ? 3 : 4) k_pair_small(
    int32_t n_items, const int4* __restrict__ items, const int32_t* __restrict__ item_sys, SysArrays S,
    SlotArrays A, const DevPot* __restrict__ pots, int64_t stride, int filter, double* __restrict__ partial,
    int inner) {
  // a launch that follows this one with programmatic serialization (the MD
  // step's steady systems after the re-filtering ones) may be dispatched as
  // soon as every CTA of this grid is resident: it reads nothing this grid writes
  asm volatile("griddepcontrol.launch_dependents;");
  extern __shared__ __align__(16) uint4 smem[];
  uint4* tabs = smem;                                   // [kItemWarps][kTabEntries] image shifts
  uint4* sq = smem + kItemWarps * kTabEntries;          // [staged] fixed-point (x, y, z, -)
  if ((int)blockIdx.x >= n_items) return;
  // The prologue is a chain of dependent loads (item -> system words ->
  // list words and image shifts -> staged positions): each level's loads go
  // out together, and every load that needs no shared memory leaves before
  // the staging loop, so that its latency overlaps it.
  const int4 W = items[blockIdx.x];
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = item_sys[(int64_t)blockIdx.x * kItemWarps + wl];   // 0 past the item's warps
  const bool inw = wl < W.w;
  const int wg = W.z + wl;
  const int64_t k = (int64_t)wg * kWarp + lane;
  const uint4* lp = reinterpret_cast<const uint4*>(A.nbr_in) + k;
  // the system's words and the slot's inner-list count and first group (the
  // group exists for every slot; both are used only with a standing inner list)
  const int fmt_s = S.infmt[s];
  const int64_t seg = S.seg_start[s];
  const int n_s = S.n_atoms[s];
  const int pot_s = S.pot[s];
  int nn_first = 0;
  uint4 g_first = make_uint4(0u, 0u, 0u, 0u);
  if (inw && inner) { nn_first = A.nn_in[k]; g_first = __ldcs(lp); }
  // list mode of this warp: inner lists in MD steps unless the system is
  // re-listed in this pass or flagged for filtering
  const bool sel = inw && !pair_skip(S, s, filter);
  const bool refresh = sel && inner && (S.prune[s] || need_relist(S, s));
  // leave before staging when no warp of the item is selected
  const bool mine = sel;
  if (!__syncthreads_or(mine)) return;
  const int fmt = mine && inner && !refresh ? fmt_s : kInnerVerlet;
  const bool use_in = mine && inner && !refresh;
  const bool staged_tab = use_in && fmt_kind(fmt) == kInnerTab;   // warp-uniform
  const int64_t st0 = (int64_t)W.x * kWarp;
  const int nst = W.y * kWarp;
  const int i = (int)(k - seg);
  const bool valid = mine && i < n_s;
  if (!(use_in && valid)) nn_first = 0;
  // the warp's image shifts (|n_a| <= b_a as the format word says; at most
  // 125, four per lane), held in registers across the staging loop
  uint4* tab = tabs + wl * kTabEntries;
  const uint4* gt = S.shiftq + (int64_t)s * kNCodes;
  const int ntab = staged_tab ? (2 * fmt_bound(fmt, 0) + 1) * (2 * fmt_bound(fmt, 1) + 1) * (2 * fmt_bound(fmt, 2) + 1) : 0;
  uint4 tv[4];
  {
    const TabDecode td(fmt);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int c = lane + q * kWarp;
      if (c < ntab) tv[q] = __ldg(gt + td.code(c));
    }
  }
#pragma unroll 4
  for (int t = threadIdx.x; t < nst; t += blockDim.x) {
    float4 h = __ldg(A.xh + st0 + t), l = __ldg(A.xl + st0 + t);
    sq[t] = make_uint4(fix_coord(h.x, l.x), fix_coord(h.y, l.y), fix_coord(h.z, l.z), 0u);
  }
  if (staged_tab) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int c = lane + q * kWarp;
      if (c < ntab) tab[c] = tv[q];
    }
    if (lane == 0) tab[kTabFar] = make_uint4(kFarShift, 0u, 0u, 0u);
  }
  // a warp that filters its inner list (into the table format) reads no
  // staged table: its region holds the image code -> table index lookup
  const int ofmt = refresh ? tab_format(S, s) : kInnerVerlet;
  if (refresh && fmt_kind(ofmt) == kInnerTab) {   // only the codes of the format's images occur
    uint8_t* lut = reinterpret_cast<uint8_t*>(tab);
    const int ntab = (2 * fmt_bound(ofmt, 0) + 1) * (2 * fmt_bound(ofmt, 1) + 1) * (2 * fmt_bound(ofmt, 2) + 1);
    const TabDecode td(ofmt);
    for (int c = lane; c < ntab; c += kWarp) lut[td.code(c)] = (uint8_t)c;
  }
  __syncthreads();
  if (!mine) return;
  const uint4* hq = sq + (seg - st0);
  const DevPot P = pots[pot_s];
  const uint4* gtab = S.shiftq + (int64_t)s * kNCodes;
  const uint4 xi = valid ? hq[i] : make_uint4(0, 0, 0, 0);
  PairSums<EW> acc;
  // one loop per potential kind (uniform over the warp) and list mode
  auto run = [&](auto kind) {
    constexpr int K = decltype(kind)::value;
    const PairFix C = pair_fix<K>(P);
    if (use_in) {
      // four entries per 16-byte load, the next group in flight ahead of use
      const char* hb = reinterpret_cast<const char*>(hq);
      const char* tb = reinterpret_cast<const char*>(tab);
      const int ng = (nn_first + 3) >> 2;
      auto shift = [&](uint32_t ent) {
        if (staged_tab) return *reinterpret_cast<const uint4*>(tb + (ent >> 16));
        // kInnerRaw: the image code, or kRawFar for padding
        const uint32_t code = ent >> 16;
        return code == kRawFar ? make_uint4(kFarShift, 0u, 0u, 0u)
                               : (code != (uint32_t)kCenter ? __ldg(gtab + code) : make_uint4(0u, 0u, 0u, 0u));
      };
      auto two = [&](uint32_t ea, uint32_t eb) {
        const uint4 xa = *reinterpret_cast<const uint4*>(hb + (ea & 0xffffu));
        const uint4 xb = *reinterpret_cast<const uint4*>(hb + (eb & 0xffffu));
        float ra, rb;
        pair_add2<K, EW>(C, P.phicf, xi, xa, shift(ea), xb, shift(eb), acc, ra, rb);
      };
      // one group of four in flight ahead of use
      uint4 n0 = g_first;
      for (int g = 0; g < ng; g++) {
        const uint4 e = n0;
        if (g + 1 < ng) n0 = __ldcs(lp + (int64_t)(g + 1) * stride);
        two(e.x, e.y); two(e.z, e.w);
      }
    } else {   // Verlet list; in MD steps, filter it into the inner list
      const int nn = valid ? A.nn[k] : 0;
      const uint32_t* lp = A.nbr + k;
      // the images the Verlet list can hold: those of the geometry it was
      // built for, which is the current one (in MD steps a system whose cell
      // changed since its listing is re-listed first)
      const bool otab = fmt_kind(ofmt) == kInnerTab;
      const uint8_t* lut = reinterpret_cast<const uint8_t*>(tab);
      const float rin2u = P.rin2f * kFix2;
      int cin = 0;
      // inner entries stored one by one into their groups of four (one
      // 4-byte store per kept entry beats collecting a group in registers)
      auto keep = [&](uint32_t e) {
        A.nbr_in[inner_at(cin, k, stride)] = e;
        cin++;
      };
      auto one = [&](uint32_t ent) {
        const int code = (int)(ent >> kJBits);
        const int j = (int)(ent & kJMask);
        const uint4 sh = code != kCenter ? __ldg(gtab + code) : make_uint4(0, 0, 0, 0);
        const float r2u = pair_add<K, EW>(C, P.phicf, xi, hq[j], sh, acc);
        if (refresh && r2u < rin2u) {
          const uint32_t hi = otab ? (uint32_t)lut[code] << 4 : (uint32_t)code;
          keep((hi << 16) | ((uint32_t)j << 4));
        }
      };
      // list entries stream two blocks of four ahead of use (n: the next
      // block, m: the one after): one 4-byte load per entry, so the loop
      // needs more loads in flight than the inner-list loop
      int q = 0;
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
      if (refresh) {
        if (valid) {
          // pad the last group with entries whose shift is beyond every cutoff
          const int n_in = cin;
          const uint32_t far = otab ? (uint32_t)kTabFar << 20 : kRawFar << 16;
          while (cin & 3) keep(far | ((uint32_t)i << 4));
          A.nn_in[k] = n_in;
          A.xph[k] = __ldg(A.xh + k); A.xpl[k] = __ldg(A.xl + k);
        }
        if (lane == 0) S.infmt[s] = ofmt;   // every warp of the system writes the same value
      }
    }
  };
  if (P.kind == TS_LJ) run(std::integral_constant<int, TS_LJ>{});
  else if (P.kind == TS_MORSE) run(std::integral_constant<int, TS_MORSE>{});
  else run(std::integral_constant<int, TS_SOFT_SPHERE>{});
  if (valid) A.F[k] = make_float4(acc.f0, acc.f1, acc.f2, acc.e);
  if (EW) {   // one FP64 partial per warp (every computed warp lies inside its system's padded segment)
    double v[7] = {(double)acc.e, (double)acc.w0, (double)acc.w1, (double)acc.w2, (double)acc.w3, (double)acc.w4,
                   (double)acc.w5};
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
