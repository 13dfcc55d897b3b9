// ts_neighbor.cu -- topology, import/export and the per-system cell-list
// neighbour build (triclinic, multi-image) behind ts_neighbor_build.
//
// Method: for every system, bins per lattice direction
// n_a = max(1, floor(w_a / r_list)) with w_a = V / |h_b x h_c| the
// perpendicular width, fractional coordinates wrapped to [0,1), and a
// stencil reach m_a = ceil(r_list n_a / w_a) bins, stencil bins outside the
// grid mapping back with a lattice image shift.  Several images of one bin
// (small cells, the general multi-image case) are distinct stencil entries.
// The explicit list at r_list = rc + skin (transposed ELL, one 32-bit entry
// per neighbour: local index | image code) is rebuilt per system when one of
// its atoms moved more than skin/2.
#include "ts_kernels.cuh"

namespace ts {

// --- topology --------------------------------------------------------------
// starts[s] = first caller index of system s; validates system_idx.
__global__ void k_sys_bounds(int64_t N, const int32_t* __restrict__ sidx, int32_t B, int64_t* starts,
                             int32_t* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int s = sidx[i];
    if (s < 0 || s >= B) { atomicOr(err, kErrBadSystemIdx); continue; }
    int p = (i == 0) ? -1 : sidx[i - 1];
    if (p > s || (p != s && p != s - 1)) atomicOr(err, kErrBadSystemIdx);
    if (p != s) starts[s] = i;
    if (i == N - 1 && s != B - 1) atomicOr(err, kErrBadSystemIdx);
  }
}

// slot tables: perm/sys for every padded slot of every system (identity order)
__global__ void k_init_slots(int32_t B, SysArrays S, SlotArrays A) {
  int s = blockIdx.x;
  if (s >= B) return;
  if (threadIdx.x == 0) S.lbound[s] = kMaxReach;   // no list yet: the first tables are complete
  int64_t st = S.seg_start[s];
  int n = S.n_atoms[s];
  int npad = (n + kWarp - 1) / kWarp * kWarp;
  for (int k = threadIdx.x; k < npad; k += blockDim.x) {
    A.perm[st + k] = k < n ? (int32_t)(S.caller_off[s] + k) : -1;
    A.sys[st + k] = k < n ? s : -1;
    A.nn[st + k] = 0;
    A.nn_in[st + k] = 0;
  }
}

// --- import / export ---------------------------------------------------------
// Positions from the caller; marks systems whose positions changed (forces
// stale), systems whose atoms left the skin (re-list) and systems whose atoms
// moved half the inner skin since their last prune (whoever moved them: the
// caller, or FIRE, which keeps no inner list).  check_skin = 0 on the first
// import after a topology change (everything is re-listed anyway).
template <bool F64>
__device__ __forceinline__ void import_vel_slot(SlotArrays& A, int64_t k, int p, const double* __restrict__ vel,
                                                const double* __restrict__ mass) {
  double m = mass[p];
  double v0 = vel ? vel[3 * (int64_t)p] : 0.0, v1 = vel ? vel[3 * (int64_t)p + 1] : 0.0,
         v2 = vel ? vel[3 * (int64_t)p + 2] : 0.0;
  if constexpr (F64) {
    double* vd = A.vd + 3 * k;
    vd[0] = v0; vd[1] = v1; vd[2] = v2;
    A.minvd[k] = 1.0 / m;
  } else {
    float4 h, l;
    h.x = (float)v0; l.x = (float)(v0 - (double)h.x);
    h.y = (float)v1; l.y = (float)(v1 - (double)h.y);
    h.z = (float)v2; l.z = (float)(v2 - (double)h.z);
    h.w = 1.0f / (float)m; l.w = 0.f;   // FP32 divide: no FP64 on the mixed import
    A.vh[k] = h; A.vl[k] = l;
  }
}

// Along periodic axes a position is defined modulo the lattice.  For an
// imported position that lies beyond the skin of its listing reference (e its
// displacement from it), take the image nearest the reference: unwrapped
// coordinates (a stored trajectory, a caller's own integrator) are the same
// configuration and cost no re-listing.  The lattice vector is chosen in FP32
// and applied to x in FP64; returns whether x moved.
__device__ __forceinline__ bool lattice_image(const SysArrays& S, int s, float e0, float e1, float e2, double& x0,
                                              double& x1, double& x2) {
  const int pm = S.pmask[s];
  if (!pm) return false;
  const float* g = S.hinvf + 9 * s;
  int n[3];
  for (int a = 0; a < 3; a++)
    n[a] = (pm >> a & 1) ? (int)rintf(fmaf(e0, g[a], fmaf(e1, g[3 + a], e2 * g[6 + a]))) : 0;
  if (!(n[0] | n[1] | n[2])) return false;
  const double* h = S.h + 9 * s;
  x0 -= n[0] * h[0] + n[1] * h[3] + n[2] * h[6];
  x1 -= n[0] * h[1] + n[1] * h[4] + n[2] * h[7];
  x2 -= n[0] * h[2] + n[1] * h[5] + n[2] * h[8];
  return true;
}

// with_vel: velocities and inverse masses too (MD calls), in the same pass
template <bool F64>
__global__ void k_import_pos(int64_t Npad, SysArrays S, SlotArrays A, const double* __restrict__ pos,
                             const DevPot* __restrict__ pots, int check_skin, int32_t* err, int with_vel = 0,
                             const double* __restrict__ vel = nullptr, const double* __restrict__ mass = nullptr) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    if (with_vel) import_vel_slot<F64>(A, k, p, vel, mass);
    int s = A.sys[k];
    double x0 = pos[3 * (int64_t)p], x1 = pos[3 * (int64_t)p + 1], x2 = pos[3 * (int64_t)p + 2];
    if (!(isfinite(x0) && isfinite(x1) && isfinite(x2)) || fabs(x0) > kMaxCoord || fabs(x1) > kMaxCoord ||
        fabs(x2) > kMaxCoord) {
      atomicOr(err, kErrNonFinite);
      continue;
    }
    bool changed;
    const DevPot& P = pots[S.pot[s]];
    if constexpr (F64) {
      double* xd = A.xd + 3 * k;
      changed = (xd[0] != x0) || (xd[1] != x1) || (xd[2] != x2);
      if (changed) { xd[0] = x0; xd[1] = x1; xd[2] = x2; }
      if (check_skin) {
        const double* xr = A.xrd + 3 * k;
        double dx = x0 - xr[0], dy = x1 - xr[1], dz = x2 - xr[2];
        double sk = 0.5 * P.skin, d2 = dx * dx + dy * dy + dz * dz;
        if (d2 > sk * sk && lattice_image(S, s, (float)dx, (float)dy, (float)dz, x0, x1, x2)) {
          xd[0] = x0; xd[1] = x1; xd[2] = x2;
          dx = x0 - xr[0]; dy = x1 - xr[1]; dz = x2 - xr[2];
          d2 = dx * dx + dy * dy + dz * dz;
        }
        if (d2 > sk * sk) { S.relist[s] = 1; S.any[0] = 1; }
        else if (d2 > P.soon2 * sk * sk) S.soon[s] = 1;
        const double* xp = A.xpd + 3 * k;
        double p0 = x0 - xp[0], p1 = x1 - xp[1], p2 = x2 - xp[2];
        if (p0 * p0 + p1 * p1 + p2 * p2 > P.half_in2d) S.prune[s] = 1;
      }
    } else {
      // unchanged when the caller's value is the one the slot holds (the
      // double the export wrote), whatever its hi/lo split
      float4 h = A.xh[k], l = A.xl[k];
      changed = (x0 != (double)h.x + (double)l.x) || (x1 != (double)h.y + (double)l.y) ||
                (x2 != (double)h.z + (double)l.z);
      if (changed) {
        split_pos(x0, h.x, l.x); split_pos(x1, h.y, l.y); split_pos(x2, h.z, l.z);
        h.w = 0.f; l.w = 0.f;
        A.xh[k] = h; A.xl[k] = l;
      }
      if (check_skin) {
        // the skin and refresh tests in FP32, with the thresholds the kick uses
        const float4 rh = A.xrh[k], rl = A.xrl[k];
        float ex = (h.x - rh.x) + (l.x - rl.x), ey = (h.y - rh.y) + (l.y - rl.y), ez = (h.z - rh.z) + (l.z - rl.z);
        float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
        if (d2 > P.half_skin2f && lattice_image(S, s, ex, ey, ez, x0, x1, x2)) {
          split_pos(x0, h.x, l.x); split_pos(x1, h.y, l.y); split_pos(x2, h.z, l.z);
          A.xh[k] = h; A.xl[k] = l;
          ex = (h.x - rh.x) + (l.x - rl.x); ey = (h.y - rh.y) + (l.y - rl.y); ez = (h.z - rh.z) + (l.z - rl.z);
          d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
        }
        if (d2 > P.half_skin2f) { S.relist[s] = 1; S.any[0] = 1; }
        else if (d2 > P.soon_half_skin2f) S.soon[s] = 1;
        const float4 ph = A.xph[k], pl = A.xpl[k];
        const float q0 = (h.x - ph.x) + (l.x - pl.x), q1 = (h.y - ph.y) + (l.y - pl.y), q2 = (h.z - ph.z) + (l.z - pl.z);
        if (fmaf(q0, q0, fmaf(q1, q1, q2 * q2)) > P.half_in2f) S.prune[s] = 1;
      }
    }
    if (changed) S.dirty[s] = 1;
  }
}


template <bool F64>
__global__ void k_export_state(int64_t Npad, SlotArrays A, double* pos, double* vel) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    if constexpr (F64) {
      if (pos) for (int c = 0; c < 3; c++) pos[3 * (int64_t)p + c] = A.xd[3 * k + c];
      if (vel) for (int c = 0; c < 3; c++) vel[3 * (int64_t)p + c] = A.vd[3 * k + c];
    } else {
      if (pos) {
        float4 h = A.xh[k], l = A.xl[k];
        pos[3 * (int64_t)p] = (double)h.x + (double)l.x;
        pos[3 * (int64_t)p + 1] = (double)h.y + (double)l.y;
        pos[3 * (int64_t)p + 2] = (double)h.z + (double)l.z;
      }
      if (vel) {
        float4 h = A.vh[k], l = A.vl[k];
        vel[3 * (int64_t)p] = (double)h.x + (double)l.x;
        vel[3 * (int64_t)p + 1] = (double)h.y + (double)l.y;
        vel[3 * (int64_t)p + 2] = (double)h.z + (double)l.z;
      }
    }
  }
}

// positions into row `row` of the frames whose base address is *base
// (caller order, rows of 3 * n_atoms doubles): the base is read on the device,
// so that a captured step loop writes wherever the latest call points it
template <bool F64>
__global__ void k_export_frame(int64_t Npad, SlotArrays A, const uint64_t* __restrict__ base, int64_t row,
                               int64_t n_atoms) {
  double* pos = reinterpret_cast<double*>(*base) + row * 3 * n_atoms;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    if constexpr (F64) {
      for (int c = 0; c < 3; c++) pos[3 * (int64_t)p + c] = A.xd[3 * k + c];
    } else {
      float4 h = A.xh[k], l = A.xl[k];
      pos[3 * (int64_t)p] = (double)h.x + (double)l.x;
      pos[3 * (int64_t)p + 1] = (double)h.y + (double)l.y;
      pos[3 * (int64_t)p + 2] = (double)h.z + (double)l.z;
    }
  }
}

template <bool F64>
__global__ void k_export_forces(int64_t Npad, SlotArrays A, double* F) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    if constexpr (F64) {
      for (int c = 0; c < 3; c++) F[3 * (int64_t)p + c] = A.Fd[3 * k + c];
    } else {
      float4 f = A.F[k];
      F[3 * (int64_t)p] = f.x; F[3 * (int64_t)p + 1] = f.y; F[3 * (int64_t)p + 2] = f.z;
    }
  }
}

// --- per-system geometry -----------------------------------------------------
__device__ inline double det3(const double* h) {
  return h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) + h[2] * (h[3] * h[7] - h[4] * h[6]);
}

// Cell import, inverse, bins and reach (bins clamped to the system's bin
// reservation), periodic axes.  Along a non-periodic axis there are no
// images and no wrapping: the cell spans the bins, atoms beyond it fall into
// the edge bins (bins are at least r_list wide, so every pair within r_list
// still lies in neighbouring bins), and the stencil stops at the edges.
__global__ void k_geometry(int32_t B, SysArrays S, const double* __restrict__ cell, const uint8_t* __restrict__ pbc,
                           const DevPot* __restrict__ pots, int32_t* err, int cell_check, int keep_pmask = 0,
                           int force = 0) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  double h[9];
  for (int q = 0; q < 9; q++) h[q] = cell[9 * (int64_t)s + q];
  if (cell_check) {   // lists built for another cell: re-list (see the prologue for the two checks)
    const double* ref = cell_check == 1 ? S.h + 9 * s : S.href + 9 * s;
    bool moved = false;
    for (int q = 0; q < 9; q++) moved |= h[q] != ref[q];
    if (moved) { S.relist[s] = 1; S.any[0] = 1; }
  }
  const int pm = keep_pmask ? S.pmask[s] : pbc ? ((pbc[3 * s] ? 1 : 0) | (pbc[3 * s + 1] ? 2 : 0) | (pbc[3 * s + 2] ? 4 : 0)) : 7;
  // lists built with another periodicity hold images along an axis that is
  // now open (or miss those of one now periodic): re-list
  if (cell_check && pm != S.pmask[s]) { S.relist[s] = 1; S.any[0] = 1; }
  // the same cell and periodicity as at the last (error-free) computation:
  // geometry and image tables stand (S.geom bit 0: valid, bit 1: recomputed
  // by this launch, so k_shift_table rebuilds the tables)
  if (!force && (S.geom[s] & 1) && pm == S.pmask[s]) {
    bool same = true;
    for (int q = 0; q < 9; q++) same &= h[q] == S.h[9 * s + q];
    if (same) { S.geom[s] = 1; return; }
  }
  S.geom[s] = 2;
  for (int q = 0; q < 9; q++) S.h[9 * s + q] = h[q];
  S.pmask[s] = pm;
  double d = det3(h);
  if (!(fabs(d) > 0) || !isfinite(d)) { atomicOr(err, kErrNonFinite); return; }
  // inverse cell by one reciprocal (an FP64 divide is a long sequence on this
  // part); it only places atoms in bins and wraps them, which tolerate ulps
  const double id = 1.0 / d;
  double g[9];
  g[0] = (h[4] * h[8] - h[5] * h[7]) * id; g[1] = (h[2] * h[7] - h[1] * h[8]) * id;
  g[2] = (h[1] * h[5] - h[2] * h[4]) * id; g[3] = (h[5] * h[6] - h[3] * h[8]) * id;
  g[4] = (h[0] * h[8] - h[2] * h[6]) * id; g[5] = (h[2] * h[3] - h[0] * h[5]) * id;
  g[6] = (h[3] * h[7] - h[4] * h[6]) * id; g[7] = (h[1] * h[6] - h[0] * h[7]) * id;
  g[8] = (h[0] * h[4] - h[1] * h[3]) * id;
  for (int q = 0; q < 9; q++) { S.hinv[9 * s + q] = g[q]; S.hinvf[9 * s + q] = (float)g[q]; }
  // widths w_a = V / |b x c| between opposite faces, and their reciprocals
  // |b x c| / V from the reciprocal already taken: one divide per axis
  double V = fabs(d), w[3], iw[3];
  double ext = 0;
  for (int a = 0; a < 3; a++) {
    const double* b = h + 3 * ((a + 1) % 3);
    const double* c = h + 3 * ((a + 2) % 3);
    double cx = b[1] * c[2] - b[2] * c[1], cy = b[2] * c[0] - b[0] * c[2], cz = b[0] * c[1] - b[1] * c[0];
    const double nc = sqrt(cx * cx + cy * cy + cz * cz);
    w[a] = V / nc;
    iw[a] = nc * fabs(id);
    ext += fabs(h[3 * a]) + fabs(h[3 * a + 1]) + fabs(h[3 * a + 2]);
  }
  double rl = pots[S.pot[s]].rlist, bw = pots[S.pot[s]].binw;
  const double ibw = 1.0 / bw;
  int nb[3], m[3];
  bool bad = false;
  for (int a = 0; a < 3; a++) {
    double f = floor(w[a] * ibw);
    nb[a] = f < 1.0 ? 1 : (f > 1024.0 ? 1024 : (int)f);
  }
  int cap = S.bin_cap[s];
  while ((int64_t)nb[0] * nb[1] * nb[2] > cap) {
    int a = (nb[0] >= nb[1] && nb[0] >= nb[2]) ? 0 : (nb[1] >= nb[2] ? 1 : 2);
    nb[a] = nb[a] > 1 ? nb[a] - 1 : 1;
    if (nb[0] == 1 && nb[1] == 1 && nb[2] == 1) break;
  }
  for (int a = 0; a < 3; a++) {
    m[a] = (int)ceil(rl * nb[a] * iw[a]);
    if (m[a] < 1) m[a] = 1;
    if (!(pm >> a & 1)) m[a] = m[a] < nb[a] ? m[a] : nb[a];   // open axis: no images, the stencil stops at the edges
    else if (m[a] > kMaxReach) { m[a] = kMaxReach; atomicOr(err, kErrUnsupported); bad = true; }
    S.nb[3 * s + a] = nb[a];
    S.reach[3 * s + a] = m[a];
  }
  // the image tables are rebuilt for the codes the current lists hold and the
  // codes a list built for this geometry can hold
  S.tbound[s] = max(S.lbound[s], image_bound(S, s));
  // positions wrapped into the cell plus the skin must stay inside the hi/lo range
  if (ext + 2.0 * rl > 0.5 * kMaxCoord) { atomicOr(err, kErrUnsupported); bad = true; }
  S.geom[s] = bad ? 2 : 3;   // an error is raised again by every call until the cell changes
}

// Image shift table S = n h for every image code within the system's table
// bound (S.tbound), stored hi/lo (mixed), FP64 and fixed point.  One CTA per
// system, its threads over the codes (up to 729 for a small cell, whose FP64
// work per code would otherwise set the launch's length); a system whose cell
// did not change keeps its tables.
__global__ void k_shift_table(int32_t B, SysArrays S) {
  const int s = blockIdx.x;
  if (s >= B || !(S.geom[s] & 2)) return;   // cell unchanged: the tables stand
  const int tb = S.tbound[s], side = 2 * tb + 1;
  const double* h = S.h + 9 * s;
  for (int i = threadIdx.x; i < side * side * side; i += blockDim.x) {
    const int nx = i % side - tb, ny = (i / side) % side - tb, nz = i / (side * side) - tb;
    const int64_t t = (int64_t)s * kNCodes + img_code(nx, ny, nz);
    double v[3];
    for (int c = 0; c < 3; c++) v[c] = nx * h[c] + ny * h[3 + c] + nz * h[6 + c];
    float4 hi, lo;
    split_pos(v[0], hi.x, lo.x); split_pos(v[1], hi.y, lo.y); split_pos(v[2], hi.z, lo.z);
    hi.w = 0.f; lo.w = 0.f;
    S.shift[2 * t] = hi; S.shift[2 * t + 1] = lo;
    for (int c = 0; c < 3; c++) S.shiftd[3 * t + c] = v[c];
    S.shiftq[t] = make_uint4((uint32_t)(unsigned long long)llrint(v[0] * (double)kFix),
                             (uint32_t)(unsigned long long)llrint(v[1] * (double)kFix),
                             (uint32_t)(unsigned long long)llrint(v[2] * (double)kFix), 0u);
  }
}

// Wrap a double-float position into its cell by a whole lattice vector (along
// periodic axes) and find its bin.  FP32 fractional coordinates choose the lattice vector and the
// bin (an atom within ~1e-7 of a face may end up a few 1e-6 A outside its bin,
// far inside any skin); the shift itself is the system's double-float image
// shift, added exactly to hi and with one FP32 rounding to lo, so an atom that
// stays inside its cell is left bit-identical.  No FP64 arithmetic (slow on
// this part).  Returns false when the atom lies more cells away than the image
// table currently covers (S.tbound, at least 1)
// (the caller then takes the FP64 route).
__device__ __forceinline__ bool wrap_bin_mixed(const SysArrays& S, int s, float4& hi, float4& lo, int kb[3]) {
  const float* g = S.hinvf + 9 * s;
  const float x0 = hi.x + lo.x, x1 = hi.y + lo.y, x2 = hi.z + lo.z;
  const int pm = S.pmask[s];
  int n[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    float v = fmaf(x0, g[a], fmaf(x1, g[3 + a], x2 * g[6 + a]));
    int nb = S.nb[3 * s + a];
    float fl = 0.f;
    if (pm >> a & 1) {   // periodic: whole lattice vectors back into the cell
      fl = floorf(v);
      if (!(fabsf(fl) <= (float)S.tbound[s])) return false;   // beyond the current table entries
    } else if (!(fabsf(v) <= 4096.f)) {
      return false;
    }
    n[a] = (int)fl;
    int q = (int)floorf((v - fl) * (float)nb);   // open axis: atoms beyond the cell go to the edge bins
    kb[a] = q >= nb ? nb - 1 : (q < 0 ? 0 : q);
  }
  if (n[0] | n[1] | n[2]) {
    int64_t ti = (int64_t)s * kNCodes + img_code(-n[0], -n[1], -n[2]);
    float4 sh = S.shift[2 * ti], sl = S.shift[2 * ti + 1];
    hi.x += sh.x; hi.y += sh.y; hi.z += sh.z;   // exact: both on the 2^-12 grid
    pos_add(hi.x, lo.x, sl.x); pos_add(hi.y, lo.y, sl.y); pos_add(hi.z, lo.z, sl.z);
  }
  return true;
}

// --- counting sort by (system, bin) ------------------------------------------
__global__ void k_zero_bins(int32_t B, SysArrays S, int32_t* count) {
  int s = blockIdx.x;
  if (s >= B || !need_relist(S, s) || S.n_atoms[s] <= kSmallMax) return;
  int off = S.bin_off[s], cap = S.bin_cap[s];
  for (int k = threadIdx.x; k < cap; k += blockDim.x) count[off + k] = 0;
}

// wrap positions into the cell, bin them, claim a (provisional) rank in the bin
template <bool F64>
__global__ void k_bin_atoms(int64_t Npad, SysArrays S, SlotArrays A, int32_t* count) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    int s = A.sys[k];
    if (!need_relist(S, s) || S.n_atoms[s] <= kSmallMax) continue;
    int kb[3];
    if constexpr (!F64) {
      float4 hi = A.xh[k], lo = A.xl[k];
      if (wrap_bin_mixed(S, s, hi, lo, kb)) {
        A.tmp_f0[k] = hi; A.tmp_f1[k] = lo;
        int gb = S.bin_off[s] + (kb[2] * S.nb[3 * s + 1] + kb[1]) * S.nb[3 * s] + kb[0];
        A.tmp_i0[k] = gb;
        A.tmp_i1[k] = atomicAdd(&count[gb], 1);
        continue;
      }
    }
    double x[3];
    if constexpr (F64) {
      for (int c = 0; c < 3; c++) x[c] = A.xd[3 * k + c];
    } else {
      float4 h = A.xh[k], l = A.xl[k];
      x[0] = (double)h.x + l.x; x[1] = (double)h.y + l.y; x[2] = (double)h.z + l.z;
    }
    const double* g = S.hinv + 9 * s;
    const double* h = S.h + 9 * s;
    double f[3];
    const int pm = S.pmask[s];
    for (int a = 0; a < 3; a++) {
      double v = x[0] * g[a] + x[1] * g[3 + a] + x[2] * g[6 + a];
      if (pm >> a & 1) {
        v -= floor(v);
        if (v >= 1.0) v = 0.0;
      }
      f[a] = v;
      int nb = S.nb[3 * s + a];
      int q = (int)floor(v * nb);
      kb[a] = q >= nb ? nb - 1 : (q < 0 ? 0 : q);
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
    int gb = S.bin_off[s] + (kb[2] * S.nb[3 * s + 1] + kb[1]) * S.nb[3 * s] + kb[0];
    A.tmp_i0[k] = gb;
    A.tmp_i1[k] = atomicAdd(&count[gb], 1);
  }
}

// exclusive scan of bin counts: block sums, scan of sums, add
__global__ void k_scan_block(int64_t n, const int32_t* __restrict__ in, int32_t* out, int32_t* bsum) {
  __shared__ int32_t sh[1024];
  int64_t i = blockIdx.x * 1024ll + threadIdx.x;
  int v = i < n ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = sh[threadIdx.x] - v;
  if (threadIdx.x == 1023) bsum[blockIdx.x] = sh[1023];
}
__global__ void k_scan_sums(int32_t nb, int32_t* bsum) {   // one block, sequential chunks
  __shared__ int32_t carry;
  __shared__ int32_t sh[1024];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < nb ? bsum[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) bsum[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
}
__global__ void k_scan_add(int64_t n, int32_t* out, const int32_t* __restrict__ bsum) {
  int64_t i = blockIdx.x * 1024ll + threadIdx.x;
  if (i < n) out[i] += bsum[blockIdx.x];
}

// first slot of a bin: seg_start + (scan[bin] - scan[first bin]) and the
// scan at a system's first bin equals its caller offset (counts are n_s)
__device__ __forceinline__ int64_t bin_slot(const SysArrays& S, const int32_t* cstart, int s, int gb) {
  return S.seg_start[s] + (int64_t)cstart[gb] - S.caller_off[s];
}

__global__ void k_scatter_ids(int64_t Npad, SysArrays S, SlotArrays A, const int32_t* __restrict__ cstart) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    int s = A.sys[k];
    if (!need_relist(S, s) || S.n_atoms[s] <= kSmallMax) continue;
    int gb = A.tmp_i0[k];
    A.tmp_i2[bin_slot(S, cstart, s, gb) + A.tmp_i1[k]] = p;
  }
}

// canonical order inside a bin (ascending caller index) -> final slot; move
// the per-slot state into the destination buffers
template <bool F64>
__global__ void k_final_slot(int64_t Npad, SysArrays S, SlotArrays A, const int32_t* __restrict__ cstart,
                             const int32_t* __restrict__ count, int move_fire) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    int s = A.sys[k];
    if (!need_relist(S, s) || S.n_atoms[s] <= kSmallMax) continue;
    int gb = A.tmp_i0[k];
    int64_t base = bin_slot(S, cstart, s, gb);
    int cnt = count[gb], r = 0;
    for (int q = 0; q < cnt; q++) r += A.tmp_i2[base + q] < p;
    int64_t d = base + r;
    A.bin[d] = gb;
    A.tmp_i1[d] = p;   // new perm (copied back below)
    if constexpr (F64) {
      for (int c = 0; c < 3; c++) A.xd[3 * d + c] = A.tmp_d0[3 * k + c];
      for (int c = 0; c < 3; c++) A.tmp_d1[3 * d + c] = A.vd[3 * k + c];
      A.tmp_d2[d] = A.minvd[k];
      if (move_fire) for (int c = 0; c < 3; c++) A.tmp_d2[Npad + 3 * d + c] = A.gd0[3 * k + c];
    } else {
      A.xh[d] = A.tmp_f0[k];
      A.xl[d] = A.tmp_f1[k];
      A.tmp_f2[d] = A.vh[k];
      A.tmp_f3[d] = A.vl[k];
      if (move_fire) A.tmp_f0[Npad + d] = A.g0[k];
    }
  }
}

template <bool F64>
__global__ void k_copy_back(int64_t Npad, SysArrays S, SlotArrays A, int move_fire) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int s = A.sys[k];
    if (s < 0 || !need_relist(S, s) || S.n_atoms[s] <= kSmallMax) continue;
    A.perm[k] = A.tmp_i1[k];
    if constexpr (F64) {
      for (int c = 0; c < 3; c++) A.vd[3 * k + c] = A.tmp_d1[3 * k + c];
      A.minvd[k] = A.tmp_d2[k];
      if (move_fire) for (int c = 0; c < 3; c++) A.gd0[3 * k + c] = A.tmp_d2[Npad + 3 * k + c];
    } else {
      A.vh[k] = A.tmp_f2[k];
      A.vl[k] = A.tmp_f3[k];
      if (move_fire) A.g0[k] = A.tmp_f0[Npad + k];
    }
  }
}

// per-system flag bookkeeping after a listing: the re-listed systems' forces are stale
__global__ void k_after_relist(int32_t B, SysArrays S, int64_t* counters, int md_pass) {
  // launched with programmatic serialization after a pair launch: nothing
  // before that launch has completed (no-op otherwise)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  bool refreshed = false, re = false;
  if (s < B) {
    // inner lists: an MD pass's pair launches refreshed every flagged or
    // re-listed system (counted in counters[1]); after any other pass a
    // re-listed system's inner list is stale until the next MD pass
    re = need_relist(S, s);
    if (md_pass) {
      refreshed = S.prune[s] || re;
      S.prune[s] = 0;
    } else if (re) {
      S.prune[s] = 1;
    }
    if (re) {
      S.lbound[s] = image_bound(S, s);   // the lists just built hold codes up to this bound
      S.dirty[s] = 1;
      S.relist[s] = 0;
      S.soon[s] = 0;
      for (int q = 0; q < 9; q++) S.href[9 * s + q] = S.h[9 * s + q];
    }
  }
  // the counts, one atomic per warp (a mass re-listing flags most systems)
  const unsigned nref = __popc(__ballot_sync(0xffffffffu, refreshed)), nre = __popc(__ballot_sync(0xffffffffu, re));
  if ((threadIdx.x & 31) == 0) {
    if (nref) atomicAdd((unsigned long long*)(counters + 1), (unsigned long long)nref);
    if (nre) atomicAdd((unsigned long long*)counters, (unsigned long long)nre);
  }
  // end of the pass: the last block to finish clears the batch-wide flag,
  // once every block has read it (counters[3]: a wrapping block counter); a
  // single block (batches up to 1024 systems) has read it at the barrier
  __syncthreads();
  if (threadIdx.x == 0) {
    if (gridDim.x == 1) {
      S.any[0] = 0;
    } else {
      __threadfence();
      if (atomicInc((unsigned*)(counters + 3), gridDim.x - 1) == gridDim.x - 1) S.any[0] = 0;
    }
  }
}

// list export in caller order (j as caller index, image n per axis)
__global__ void k_export_list(int64_t Npad, SysArrays S, SlotArrays A, int32_t max_nbrs, int64_t stride,
                              int32_t* j_out, int32_t* img_out, int32_t* count_out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    int s = A.sys[k];
    int64_t seg = S.seg_start[s];
    int nn = A.nn[k];
    count_out[p] = nn;
    for (int q = 0; q < max_nbrs; q++) {
      int64_t o = (int64_t)p * max_nbrs + q;
      if (q < nn) {
        uint32_t e = A.nbr[q * stride + k];
        int code = (int)(e >> kJBits);
        j_out[o] = A.perm[seg + (e & kJMask)];
        img_out[3 * o] = code % kImgSide - kMaxReach;
        img_out[3 * o + 1] = (code / kImgSide) % kImgSide - kMaxReach;
        img_out[3 * o + 2] = code / (kImgSide * kImgSide) - kMaxReach;
      } else {
        j_out[o] = -1;
        img_out[3 * o] = img_out[3 * o + 1] = img_out[3 * o + 2] = 0;
      }
    }
  }
}


}  // namespace ts
