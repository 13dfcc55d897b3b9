// ts_internal.cuh -- device-side data layout and helpers of libts.so.
//
// Layout (B300-first): every system occupies a contiguous segment of
// "slots" padded to a multiple of 32, so a warp never straddles two systems:
// the potential, cell and image table of a warp are uniform, and per-system
// energy/virial reduce with warp shuffles into one FP64 partial per warp (no
// scatter atomics).  Inside a segment, atoms are sorted by cell-list bin
// (re-sorted at every re-listing), so neighbour gathers stay local in L1/L2.
//
// Mixed precision stores a position as hi + lo: hi on a 2^-12 A grid (exact
// in FP32 for |x| < 2048 A), lo = x - hi (|lo| <= 2^-13).  A pair vector
// d = x_j + n h - x_i is then formed as (hi_j + S_hi - hi_i) -- exact, all
// terms on the grid -- plus (lo_j + S_lo - lo_i), so d carries one rounding
// only, independent of the box size.  The lattice image shift S = n h is
// stored the same way per (system, image code).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ts.h"

namespace ts {

constexpr int kWarp = 32;
constexpr float kGrid = 4096.0f;          // 2^12
// Half-width of the shell around the list radius where the hi-only distance
// (off by at most 3 * 2^-13 * sqrt(3) = 6.3e-4 A) cannot decide a list test.
constexpr double kListBand = 1e-3;
// Default inner skin of the pruned pair list, as a fraction of the skin.
constexpr double kInnerSkinFraction = 0.3;
// NPT: per-system factors written by k_npt_sys for the step's atom updates
// (stride in doubles and slots): atom kicks v <- v eb + fb F/m at the step's
// opening and closing, half drifts x <- x + x ea + fa v (ea = e^{v_e dt/2} - 1)
// before and after the O step, the displacement allowance and lambda - 1, the
// isotropic scale of the cell since the listing.
constexpr int kNptStride = 32;
enum NptFactor : int { kNptEbOpen = 0, kNptFbOpen, kNptEa1, kNptFa1, kNptEa2, kNptFa2, kNptEbClose, kNptFbClose,
                       kNptAllow, kNptLam };
constexpr float kInvGrid = 1.0f / 4096.0f;
constexpr double kMaxCoord = 2000.0;      // |x| bound of the hi/lo representation
constexpr int kJBits = 22;                // neighbour entry: j (22 bits) | image code (10 bits)
constexpr uint32_t kJMask = (1u << kJBits) - 1u;
constexpr int kMaxReach = 4;              // images n_a in [-4, 4]
constexpr int kImgSide = 2 * kMaxReach + 1;
constexpr int kNCodes = kImgSide * kImgSide * kImgSide;   // 729
constexpr int kCenter = kMaxReach + kImgSide * kMaxReach + kImgSide * kImgSide * kMaxReach;
constexpr int kMaxPots = 16;
constexpr int kSmallMax = 2048;           // systems up to this size are sorted by one CTA

// Re-list hysteresis: a system whose atoms moved more than skin/2 must be
// re-listed; one past soon * skin/2 (soon per potential, 1 = off) is
// re-listed in the same pass whenever any system must, so re-listings gather
// into fewer, wider launches.
constexpr int kPartialStride = 8;         // doubles per warp partial

// error word bits (sticky, OR-ed)
constexpr int kErrNeighborOverflow = 1;
constexpr int kErrBadSystemIdx = 2;
constexpr int kErrUnsupported = 4;
constexpr int kErrNonFinite = 8;
constexpr int kErrTimeout = 16;

__host__ __device__ inline int img_code(int nx, int ny, int nz) {
  return (nx + kMaxReach) + kImgSide * (ny + kMaxReach) + kImgSide * kImgSide * (nz + kMaxReach);
}

// ---------------------------------------------------------------------------
// Inner (pruned) lists.  Layout: groups of four entries per slot,
// [q / 4][slot][4], so that a thread loads four entries with one 16-byte load.
// Entry format, per system: the format word SysArrays::infmt, written by the
// launch that filters the list (kind in bits 0-3, and for kInnerTab the image
// bounds b_x, b_y, b_z of the staged shift table in bits 4-6, 7-9, 10-12):
//   kInnerVerlet  the Verlet-list format, j | code << kJBits (FP64 mode and
//                 systems above kSmallMax atoms);
//   kInnerTab     low 16 bits j * 16, the byte offset of neighbour j's staged
//                 record in the shared-memory pair kernel; high 16 bits 16 x
//                 the image's index in the staged shift table, which holds
//                 the (2 b_x + 1)(2 b_y + 1)(2 b_z + 1) <= kTabCodes images
//                 with |n_a| <= b_a, x fastest; kTabFar marks padding
//                 entries (lists padded to a multiple of four);
//   kInnerRaw     low 16 bits j * 16; high 16 bits the image code, or 0xffff
//                 for padding entries (lists reaching more images than the
//                 staged table holds).
enum InnerFmt : int32_t { kInnerVerlet = 0, kInnerTab = 1, kInnerRaw = 2 };
constexpr int kTabCodes = 125;                              // images of one staged table
constexpr int kTabFar = kTabCodes;                          // shift entry of padding entries
constexpr int kTabEntries = kTabCodes + 1;
__host__ __device__ inline int64_t inner_at(int q, int64_t k, int64_t stride) {
  return (((int64_t)(q >> 2) * stride + k) << 2) | (int64_t)(q & 3);
}
__host__ __device__ inline int fmt_kind(int f) { return f & 15; }
__host__ __device__ inline int fmt_bound(int f, int a) { return (f >> (4 + 3 * a)) & 7; }
__host__ __device__ inline int fmt_tab(int bx, int by, int bz) {
  return kInnerTab | bx << 4 | by << 7 | bz << 10;
}
// Image code of staged-table index c (c < kTabEntries) under format word f:
// table digits by multiply-shift division (m = floor(2^16 / side) + 1 is exact
// for numerators below 2^16 / side^2 > 126), constants set once per warp.
struct TabDecode {
  int bx, by, bz, sx, sy, mx, my;
  __host__ __device__ explicit TabDecode(int f)
      : bx(fmt_bound(f, 0)), by(fmt_bound(f, 1)), bz(fmt_bound(f, 2)), sx(2 * bx + 1), sy(2 * by + 1),
        mx(65536 / sx + 1), my(65536 / sy + 1) {}
  __host__ __device__ int code(int c) const {
    const int q1 = (c * mx) >> 16, q2 = (q1 * my) >> 16;
    return img_code(c - sx * q1 - bx, q1 - sy * q2 - by, q2 - bz);
  }
};
__host__ __device__ inline int tab_to_code(int c, int f) { return TabDecode(f).code(c); }
// staged-table index of image code `code` (base-9 digits by multiply-shift
// division, exact for code < 729); clamped into the table, which holds every
// image the lists of a system with this format word can reference
__host__ __device__ inline int code_to_tab(int code, int f) {
  const int q1 = (code * 7282) >> 16, q2 = (q1 * 7282) >> 16;
  const int nx = code - 9 * q1 - kMaxReach, ny = q1 - 9 * q2 - kMaxReach, nz = q2 - kMaxReach;
  const int bx = fmt_bound(f, 0), by = fmt_bound(f, 1), bz = fmt_bound(f, 2);
  const int c = (nx + bx) + (2 * bx + 1) * ((ny + by) + (2 * by + 1) * (nz + bz));
  return c < 0 ? 0 : (c >= kTabCodes ? kTabCodes - 1 : c);
}
// (j, image code) of an inner-list entry under format word f (not a padding
// entry); D = TabDecode(f)
__host__ __device__ inline void inner_decode(uint32_t e, int f, const TabDecode& D, int& j, int& code) {
  const int kind = fmt_kind(f);
  if (kind == kInnerVerlet) { j = (int)(e & kJMask); code = (int)(e >> kJBits); return; }
  j = (int)((e & 0xffffu) >> 4);
  code = kind == kInnerTab ? D.code((int)(e >> 20)) : (int)(e >> 16);
}

struct DevPot {
  int kind, shift;
  float pf[3];
  float rc2f, phicf, rlist2f;
  float sinvf;    // 1/sigma in FP32 (soft sphere)
  float half_skin2f, soon_half_skin2f;   // (skin/2)^2 and soon^2 (skin/2)^2, FP32 (mixed skin check)
  float rlist_in2f, rlist_out2f;         // (rlist -+ 1e-3 A)^2: certain hit / miss of the hi-only list test
  // dynamic pruning: the inner list keeps the entries within rc + inner skin
  // (squared, with a 1e-3 A margin: the test may keep a few more); a system's
  // list is refreshed once an atom moved more than half the inner skin
  float rin2f; double rin2d;
  float half_in2f; double half_in2d;
  double pd[3];
  double rc2d, phicd, rlist, rlist2d, skin;
  double binw;    // cell-list bin edge (at least rlist / 2; the stencil reach follows)
  double soon2;   // squared hysteresis factor
};

// Per-system data the device reads (SoA, capacity Bcap).
struct SysArrays {
  int64_t* seg_start;     // padded slot start
  int32_t* n_atoms;       // atoms of the system
  int64_t* caller_off;    // first caller index of the system
  int32_t* pot;           // potential index
  uint32_t* uid;          // RNG key
  int32_t* bin_off;       // first bin of the system
  int32_t* bin_cap;       // bins reserved for the system
  int32_t* warp_start;    // first warp
  int32_t* warp_end;      // one past last warp
  double* h;              // [9] cell rows
  double* hinv;           // [9]
  float* hinvf;           // [9] FP32 copy (bin choice)
  double* href;           // [9] cell at the last listing (FIRE)
  int32_t* nb;            // [3] bins per axis (at last listing)
  int32_t* reach;         // [3]
  int32_t* pmask;         // periodic axes, bit a set when axis a is periodic
  float4* shift;          // [kNCodes][2] (hi xyz, lo xyz) mixed
  double* shiftd;         // [kNCodes][3] fp64
  uint4* shiftq;          // [kNCodes] (x, y, z) in units of 2^-26 A, modulo 2^32 (shared-memory pair kernel)
  int32_t* relist;        // per-system re-list flag
  int32_t* prune;         // per-system flag: the next MD pair launch refreshes the inner list (an atom
                          // moved half the inner skin since the last refresh, or the list is stale)
  int32_t* soon;          // atoms past kSoon * skin/2: re-list along with any forced pass
  int32_t* any;           // [1] some system must re-list in this pass
  int32_t* geom;          // bit 0: geometry and image tables current for h and pmask; bit 1: just recomputed
  int32_t* tbound;        // image codes with every |n_a| <= tbound are current in the shift tables
  int32_t* lbound;        // largest |n_a| the system's Verlet list can hold (set when it is listed)
  int32_t* dirty;         // forces stale for this system
  int32_t* infmt;         // entry format of the system's inner list (InnerFmt)
  double* kT;             // per-system kT (MD)
};

// Largest |n_a| of an image code that a list built for the current geometry
// can hold: a stencil of reach m over nb cells wraps at most ceil(m / nb)
// times along a periodic axis (open axes hold no images), and at least 1, so
// that an atom one cell outside is wrapped from the table.
__device__ __forceinline__ int image_bound(const SysArrays& S, int s) {
  int r = 1;
  for (int a = 0; a < 3; a++)
    if (S.pmask[s] >> a & 1) {
      int nb = S.nb[3 * s + a], m = S.reach[3 * s + a];
      r = max(r, (m + nb - 1) / nb);
    }
  return min(r, kMaxReach);
}

// Largest |n_a| along axis a of an image code in a list built for the
// current geometry (0 along an open axis); the format word of a staged shift
// table that covers them, or kInnerRaw when they are more than the table holds.
__device__ __forceinline__ int axis_bound(const SysArrays& S, int s, int a) {
  if (!(S.pmask[s] >> a & 1)) return 0;
  const int nb = S.nb[3 * s + a], m = S.reach[3 * s + a];
  return min((m + nb - 1) / nb, kMaxReach);
}
__device__ __forceinline__ int tab_format(const SysArrays& S, int s) {
  const int bx = axis_bound(S, s, 0), by = axis_bound(S, s, 1), bz = axis_bound(S, s, 2);
  return (2 * bx + 1) * (2 * by + 1) * (2 * bz + 1) <= kTabCodes ? fmt_tab(bx, by, bz) : (int)kInnerRaw;
}

__device__ __forceinline__ bool need_relist(const SysArrays& S, int s) {
  return S.relist[s] || (S.soon[s] && S.any[0]);
}

// Which systems a pair launch covers: all, those flagged dirty, or (while a
// re-listing pass runs beside it) those keeping their lists or those being
// re-listed; in MD steps the systems keeping their lists split further into
// those whose inner list stands (kPairSteady) and those that re-filter it
// from the Verlet list in this step (kPairPruned).  The flags stay fixed
// until the pass's bookkeeping kernel runs after every part.
enum PairFilter : int { kPairAll = 0, kPairDirty = 1, kPairKept = 2, kPairRelisted = 3, kPairSteady = 4,
                        kPairPruned = 5 };
__device__ __forceinline__ bool pair_skip(const SysArrays& S, int s, int filter) {
  if (filter == kPairAll) return false;
  if (filter == kPairDirty) return !S.dirty[s];
  const bool re = need_relist(S, s);
  if (filter == kPairRelisted) return !re;
  if (filter == kPairKept) return re;
  return re || ((S.prune[s] != 0) == (filter == kPairSteady));
}

struct SlotArrays {
  float4* xh; float4* xl;     // mixed positions hi/lo (w unused)
  float4* vh; float4* vl;     // mixed velocities hi/lo; vh.w = 1/m
  float4* F;                  // mixed forces (w = per-atom energy)
  double* xd;                 // fp64 positions [3]
  double* vd;                 // fp64 velocities [3]
  double* Fd;                 // fp64 forces [3]
  double* minvd;              // fp64 inverse mass
  float4* xrh; float4* xrl;   // positions at last listing (mixed)
  double* xrd;                // positions at last listing (fp64) [3]
  int32_t* perm;              // slot -> caller index (-1 padding)
  int32_t* sys;               // slot -> system (-1 padding)
  int32_t* bin;               // slot -> global bin (valid after a listing)
  int32_t* nn;                // neighbour count
  uint32_t* nbr;              // [max_nbrs][Ncap] (transposed ELL)
  // inner list (dynamic pruning): the entries of nbr within rc + inner skin at
  // the last refresh, in the same order; positions at that refresh
  int32_t* nn_in;
  uint32_t* nbr_in;           // [max_nbrs rounded up to 4 / 4][Ncap][4], see inner_at
  float4* xph; float4* xpl;   // mixed
  double* xpd;                // fp64 [3]
  // reorder scratch
  int32_t* tmp_i0; int32_t* tmp_i1; int32_t* tmp_i2;
  float4* tmp_f0; float4* tmp_f1; float4* tmp_f2; float4* tmp_f3;
  double* tmp_d0; double* tmp_d1; double* tmp_d2;
  // FIRE / adjoint per-slot vectors (mixed: float4; fp64: double[3])
  float4* g0; float4* g1;
  double* gd0; double* gd1;
};

// ---------------------------------------------------------------------------
// double-float helpers (FP32 pairs) for positions and velocities
// ---------------------------------------------------------------------------
// Fixed-point coordinates of the shared-memory pair kernel: units of 2^-26 A,
// kept modulo 2^32.  A pair vector is the exact integer x_j - x_i + S (exact
// as long as it is shorter than 2^31 units = 32 A) and then one conversion
// to FP32: the same single rounding as the double-float form, plus the
// quantisation of each coordinate (at most 2^-27 A = 7.5e-9 A).
constexpr float kFix = 67108864.0f;               // 2^26
constexpr float kFixInv = 1.4901161193847656e-8f; // 2^-26
constexpr double kFixMaxList = 30.0;             // list radii at or above this use the general kernel
__device__ __forceinline__ uint32_t fix_coord(float hi, float lo) {
  // hi * 2^26 is an integer (hi lies on the 2^-12 grid); lo * 2^26 is rounded
  return (uint32_t)(unsigned long long)__float2ll_rn(hi * kFix) + (uint32_t)__float2int_rn(lo * kFix);
}

// Two FP32 lanes in one 64-bit register pair, for the packed f32x2
// instructions of sm_100+ (each lane rounds exactly as the scalar operation).
__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ unsigned long long f2_splat(float a) { return f2_pack(a, a); }

__device__ __forceinline__ void split_pos(double x, float& hi, float& lo) {
  double h = rint(x * 4096.0) * (1.0 / 4096.0);
  hi = (float)h;
  lo = (float)(x - h);
}
__device__ __forceinline__ void pos_add(float& hi, float& lo, float d) {
  lo += d;
  if (fabsf(lo) > 0.5f * kInvGrid) {
    float q = rintf(lo * kGrid) * kInvGrid;
    hi += q;
    lo -= q;
  }
}
// (h, l) <- c (h, l) as a double-float: the product of the high part exactly
// (fma residual), then renormalised
__device__ __forceinline__ void df_scale(float& h, float& l, float c) {
  const float p = c * h;
  const float e = fmaf(c, h, -p) + c * l;
  h = p + e;
  l = e - (h - p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_add(float& hi, float& lo, float a) {
  float s, e;
  two_sum(hi, a, s, e);
  e += lo;
  hi = s + e;
  lo = e - (hi - s);
}

// ---------------------------------------------------------------------------
// Pair potentials.  fr = phi'(r)/r; phi unshifted.  d2 = phi''(r).
// ---------------------------------------------------------------------------
template <typename T> struct PotMath;

template <> struct PotMath<float> {
  // one potential kind, no branches (K known at compile time)
  template <int K>
  static __device__ __forceinline__ void eval_k(const DevPot& P, float r2, float& phi, float& fr) {
    if constexpr (K == TS_LJ) {
      float ri2 = __fdividef(1.0f, r2);   // ~2 ulp; the LJ terms are well conditioned
      float s2 = P.pf[0] * P.pf[0] * ri2;
      float s6 = s2 * s2 * s2, s12 = s6 * s6;
      phi = 4.0f * P.pf[1] * (s12 - s6);
      fr = -24.0f * P.pf[1] * ri2 * (2.0f * s12 - s6);
    } else if constexpr (K == TS_MORSE) {
      float r = sqrtf(r2);
      float e = __expf(P.pf[1] * (P.pf[2] - r));
      phi = P.pf[0] * (e * e - 2.0f * e);
      fr = 2.0f * P.pf[1] * P.pf[0] * e * (1.0f - e) * rsqrtf(r2);
    } else {
      float ri = rsqrtf(r2);
      float t = fmaf(-r2 * ri, P.sinvf, 1.0f);
      float al = P.pf[2];
      float ta1 = (al == 2.0f) ? t : __powf(t, al - 1.0f);
      phi = P.pf[1] / al * ta1 * t;
      fr = -P.pf[1] * P.sinvf * ta1 * ri;
    }
  }
  static __device__ __forceinline__ void eval(const DevPot& P, float r2, float& phi, float& fr) {
    if (P.kind == TS_LJ) {
      float ri2 = __fdividef(1.0f, r2);   // ~2 ulp; the LJ terms are well conditioned
      float s2 = P.pf[0] * P.pf[0] * ri2;
      float s6 = s2 * s2 * s2, s12 = s6 * s6;
      phi = 4.0f * P.pf[1] * (s12 - s6);
      fr = -24.0f * P.pf[1] * ri2 * (2.0f * s12 - s6);
    } else if (P.kind == TS_MORSE) {
      // r correctly rounded: it sets the exponent's argument, where the
      // stiff Morse force amplifies any error; 1/r only scales the result
      float r = sqrtf(r2);
      float e = __expf(P.pf[1] * (P.pf[2] - r));
      phi = P.pf[0] * (e * e - 2.0f * e);
      fr = 2.0f * P.pf[1] * P.pf[0] * e * (1.0f - e) * rsqrtf(r2);
    } else {
      float ri = rsqrtf(r2);
      float t = fmaf(-r2 * ri, P.sinvf, 1.0f);   // 1 - r/sigma in one fused operation
      float al = P.pf[2];
      float ta1 = (al == 2.0f) ? t : __powf(t, al - 1.0f);
      phi = P.pf[1] / al * ta1 * t;
      fr = -P.pf[1] * P.sinvf * ta1 * ri;
    }
  }
  // phi'/r and phi'' (for the adjoint), plus parameter derivatives of phi and phi'
  static __device__ __forceinline__ void eval2(const DevPot& P, float r2, float& r, float& d1, float& d2,
                                               float dphi[3], float dd1[3]) {
    r = sqrtf(r2);
    dphi[0] = dphi[1] = dphi[2] = 0.f; dd1[0] = dd1[1] = dd1[2] = 0.f;
    if (P.kind == TS_LJ) {
      float sg = P.pf[0], ep = P.pf[1];
      float ri = __frcp_rn(r);
      float s = sg * ri, s2 = s * s, s6 = s2 * s2 * s2, s12 = s6 * s6;
      d1 = -24.0f * ep * ri * (2.0f * s12 - s6);
      d2 = 24.0f * ep * ri * ri * (26.0f * s12 - 7.0f * s6);
      dphi[0] = 24.0f * ep / sg * (2.0f * s12 - s6);
      dphi[1] = 4.0f * (s12 - s6);
      dd1[0] = -144.0f * ep * ri / sg * (4.0f * s12 - s6);
      dd1[1] = -24.0f * ri * (2.0f * s12 - s6);
    } else if (P.kind == TS_MORSE) {
      float D = P.pf[0], a = P.pf[1], r0 = P.pf[2];
      float x = r - r0, e = expf(-a * x);
      d1 = 2.0f * a * D * (e - e * e);
      d2 = 2.0f * a * a * D * (2.0f * e * e - e);
      dphi[0] = e * e - 2.0f * e;
      dphi[1] = 2.0f * D * x * (e - e * e);
      dphi[2] = 2.0f * a * D * (e * e - e);
      dd1[0] = 2.0f * a * (e - e * e);
      dd1[1] = 2.0f * D * (e - e * e) + 2.0f * a * D * x * (2.0f * e * e - e);
      dd1[2] = -d2;
    } else {
      float sg = P.pf[0], ep = P.pf[1], al = P.pf[2];
      float t = 1.0f - r / sg;
      float lt = logf(t);
      float ta = __powf(t, al), ta1 = __powf(t, al - 1.0f), ta2 = __powf(t, al - 2.0f);
      d1 = -ep / sg * ta1;
      d2 = ep / (sg * sg) * (al - 1.0f) * ta2;
      dphi[0] = ep * ta1 * r / (sg * sg);
      dphi[1] = ta / al;
      dphi[2] = -ep / (al * al) * ta + ep / al * ta * lt;
      dd1[0] = ep / (sg * sg) * ta1 - ep / sg * (al - 1.0f) * ta2 * r / (sg * sg);
      dd1[1] = -ta1 / sg;
      dd1[2] = -ep / sg * ta1 * lt;
    }
  }
};

template <> struct PotMath<double> {
  static __device__ __forceinline__ void eval(const DevPot& P, double r2, double& phi, double& fr) {
    if (P.kind == TS_LJ) {
      double ri2 = 1.0 / r2;
      double s2 = P.pd[0] * P.pd[0] * ri2;
      double s6 = s2 * s2 * s2, s12 = s6 * s6;
      phi = 4.0 * P.pd[1] * (s12 - s6);
      fr = -24.0 * P.pd[1] * ri2 * (2.0 * s12 - s6);
    } else if (P.kind == TS_MORSE) {
      double r = sqrt(r2);
      double e = exp(-P.pd[1] * (r - P.pd[2]));
      phi = P.pd[0] * (e * e - 2.0 * e);
      fr = 2.0 * P.pd[1] * P.pd[0] * (e - e * e) / r;
    } else {
      double r = sqrt(r2);
      double t = 1.0 - r / P.pd[0];
      double al = P.pd[2];
      double ta1 = (al == 2.0) ? t : pow(t, al - 1.0);
      phi = P.pd[1] / al * ta1 * t;
      fr = -P.pd[1] / P.pd[0] * ta1 / r;
    }
  }
  static __device__ __forceinline__ void eval2(const DevPot& P, double r2, double& r, double& d1, double& d2,
                                               double dphi[3], double dd1[3]) {
    r = sqrt(r2);
    dphi[0] = dphi[1] = dphi[2] = 0; dd1[0] = dd1[1] = dd1[2] = 0;
    if (P.kind == TS_LJ) {
      double sg = P.pd[0], ep = P.pd[1];
      double s = sg / r, s2 = s * s, s6 = s2 * s2 * s2, s12 = s6 * s6;
      d1 = -24.0 * ep / r * (2.0 * s12 - s6);
      d2 = 24.0 * ep / (r * r) * (26.0 * s12 - 7.0 * s6);
      dphi[0] = 24.0 * ep / sg * (2.0 * s12 - s6);
      dphi[1] = 4.0 * (s12 - s6);
      dd1[0] = -144.0 * ep / (r * sg) * (4.0 * s12 - s6);
      dd1[1] = -24.0 / r * (2.0 * s12 - s6);
    } else if (P.kind == TS_MORSE) {
      double D = P.pd[0], a = P.pd[1], r0 = P.pd[2];
      double x = r - r0, e = exp(-a * x);
      d1 = 2.0 * a * D * (e - e * e);
      d2 = 2.0 * a * a * D * (2.0 * e * e - e);
      dphi[0] = e * e - 2.0 * e;
      dphi[1] = 2.0 * D * x * (e - e * e);
      dphi[2] = 2.0 * a * D * (e * e - e);
      dd1[0] = 2.0 * a * (e - e * e);
      dd1[1] = 2.0 * D * (e - e * e) + 2.0 * a * D * x * (2.0 * e * e - e);
      dd1[2] = -d2;
    } else {
      double sg = P.pd[0], ep = P.pd[1], al = P.pd[2];
      double t = 1.0 - r / sg, lt = log(t);
      double ta = pow(t, al), ta1 = pow(t, al - 1.0), ta2 = pow(t, al - 2.0);
      d1 = -ep / sg * ta1;
      d2 = ep / (sg * sg) * (al - 1.0) * ta2;
      dphi[0] = ep * ta1 * r / (sg * sg);
      dphi[1] = ta / al;
      dphi[2] = -ep / (al * al) * ta + ep / al * ta * lt;
      dd1[0] = ep / (sg * sg) * ta1 - ep / sg * (al - 1.0) * ta2 * r / (sg * sg);
      dd1[1] = -ta1 / sg;
      dd1[2] = -ep / sg * ta1 * lt;
    }
  }
};

// warp-level reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

}  // namespace ts
