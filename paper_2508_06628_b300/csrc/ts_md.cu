// ts_md.cu -- velocity Verlet and BAOAB Langevin steps behind ts_md_step
// (the paper's batched Langevin MD, Sec. 4).
//
// One step:  v += (dt/2m) F;  [VV]  x += dt v
//                            [BAOAB] x += dt/2 v;  v = c1 v + sqrt((1-c1^2) kT/m) xi;  x += dt/2 v
//            F = F(x);  v += (dt/2m) F.
// Consecutive half kicks of adjacent steps are merged into one full kick, so
// a step is one elementwise kernel plus the pair kernel.  The noise xi is
// Philox4x32-10 (Salmon et al., SC'11) keyed by (seed, system uid) with
// counter (step, atom index within its system), then Box-Muller, so it does
// not depend on where the system sits in the batch.
#include <type_traits>

#include "ts_kernels.cuh"

namespace ts {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
}

// three standard normals for (step, local atom, seed, uid); T = double in
// FP64 mode, float in mixed mode (no FP64 arithmetic or conversions there)
template <bool F64, typename T>
__device__ __forceinline__ void normals3(uint64_t step, uint32_t la, uint32_t seed, uint32_t uid, T z[3]) {
  uint32_t c[4] = {(uint32_t)step, la, (uint32_t)(step >> 32), 0u};
  philox4x32_10(c, seed, uid);
  if constexpr (F64) {
    const double two_pi = 6.283185307179586476925286766559;
    double u0 = ((double)c[0] + 0.5) * 2.3283064365386962890625e-10;
    double u1 = ((double)c[1] + 0.5) * 2.3283064365386962890625e-10;
    double u2 = ((double)c[2] + 0.5) * 2.3283064365386962890625e-10;
    double u3 = ((double)c[3] + 0.5) * 2.3283064365386962890625e-10;
    double R0 = sqrt(-2.0 * log(u0)), R1 = sqrt(-2.0 * log(u2));
    double sn, cs;
    sincos(two_pi * u1, &sn, &cs);
    z[0] = R0 * cs; z[1] = R0 * sn;
    z[2] = R1 * cos(two_pi * u3);
  } else {
    // u = (c + 1/2) 2^-32 as in FP64; small words convert exactly, so the
    // logarithm's tail matches the FP64 draw to FP32 rounding
    const float s32 = 2.3283064365386962890625e-10f, h32 = 1.16415321826934814453125e-10f;
    float u0 = fminf(fmaf((float)c[0], s32, h32), 0.99999994f);
    float u1 = fmaf((float)c[1], s32, h32);
    float u2 = fminf(fmaf((float)c[2], s32, h32), 0.99999994f);
    float u3 = fmaf((float)c[3], s32, h32);
    float R0 = sqrtf(-2.0f * logf(u0)), R1 = sqrtf(-2.0f * logf(u2));
    float sn, cs;
    sincospif(2.0f * u1, &sn, &cs);
    z[0] = R0 * cs; z[1] = R0 * sn;
    z[2] = R1 * cospif(2.0f * u3);
  }
}

// KIND 0: VV (kick, full drift); KIND 1: BAOAB (kick, half drift, O, half drift);
// KIND 2: NVT chain (scale, kick, full drift); KIND 3: NPT (barostat-coupled
// kick, scaled half drift, O, scaled half drift, with the per-system factors
// of k_npt_sys in sysf[kNptStride * s + ...]).
// kick = dt/2 on the first step of a call, dt when merged with the previous
// step's closing half kick (KIND 0, 1).  Also flags systems whose atoms left
// the skin (KIND 3: moved beyond the cell's isotropic scaling by more than
// the allowance k_npt_sys left), or moved half the inner skin since the last
// inner-list refresh (KIND 0-2).
template <bool F64, int KIND>
__global__ void k_md_kick_drift(int64_t Npad, SysArrays S, SlotArrays A, const DevPot* __restrict__ pots, double kick,
                                double dt, double c1, uint32_t seed, const uint64_t* __restrict__ step_base,
                                uint64_t koff, const double* __restrict__ sysf) {
  const uint64_t step = *step_base + koff;
  const float omc2f = (float)(1.0 - c1 * c1);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    int s = A.sys[k];
    using Real = typename std::conditional<F64, double, float>::type;
    Real z[3] = {0, 0, 0};
    if (KIND == 1 || KIND == 3) {
      normals3<F64>(step, (uint32_t)(p - S.caller_off[s]), seed, S.uid[s], z);
    }
    const double* q = KIND == 3 ? sysf + kNptStride * (int64_t)s : nullptr;
    double dx = 0, dy = 0, dz = 0;
    if constexpr (F64) {
      double mi = A.minvd[k];
      double* v = A.vd + 3 * k;
      double* x = A.xd + 3 * k;
      const double* f = A.Fd + 3 * k;
      const double osc = sqrt((1.0 - c1 * c1) * S.kT[s] * mi);
      if (KIND == 3) {
        for (int c = 0; c < 3; c++) v[c] = v[c] * q[kNptEbOpen] + q[kNptFbOpen] * mi * f[c];
        for (int c = 0; c < 3; c++) x[c] += x[c] * q[kNptEa1] + q[kNptFa1] * v[c];
        for (int c = 0; c < 3; c++) v[c] = c1 * v[c] + osc * z[c];
        for (int c = 0; c < 3; c++) x[c] += x[c] * q[kNptEa2] + q[kNptFa2] * v[c];
      } else {
        if (KIND == 2) { const double c = sysf[s]; for (int m = 0; m < 3; m++) v[m] *= c; }   // chain scaling
        for (int c = 0; c < 3; c++) v[c] += kick * mi * f[c];
        if (KIND != 1) {
          for (int c = 0; c < 3; c++) x[c] += dt * v[c];
        } else {
          for (int c = 0; c < 3; c++) x[c] += 0.5 * dt * v[c];
          for (int c = 0; c < 3; c++) v[c] = c1 * v[c] + osc * z[c];
          for (int c = 0; c < 3; c++) x[c] += 0.5 * dt * v[c];
        }
      }
      const double* xr = A.xrd + 3 * k;
      dx = x[0] - xr[0]; dy = x[1] - xr[1]; dz = x[2] - xr[2];
      if (KIND == 3) {   // displacement beyond the cell's isotropic scaling since the listing
        const double l = q[kNptLam];
        dx -= l * xr[0]; dy -= l * xr[1]; dz -= l * xr[2];
      }
    } else {
      float4 vh = A.vh[k], vl = A.vl[k], xh = A.xh[k], xl = A.xl[k], f = A.F[k];
      // O step, v <- c1 v + so z in double-float: scale the pair, then add the noise
      auto ou = [&]() {
        const float cc = (float)c1;
        const float so = sqrtf(omc2f * (float)S.kT[s] * vh.w);
        float nx = cc * vh.x, ny = cc * vh.y, nz = cc * vh.z;
        float ex = fmaf(cc, vh.x, -nx) + cc * vl.x, ey = fmaf(cc, vh.y, -ny) + cc * vl.y,
              ez = fmaf(cc, vh.z, -nz) + cc * vl.z;
        vh.x = nx + ex; vl.x = ex - (vh.x - nx);
        vh.y = ny + ey; vl.y = ey - (vh.y - ny);
        vh.z = nz + ez; vl.z = ez - (vh.z - nz);
        df_add(vh.x, vl.x, so * z[0]); df_add(vh.y, vl.y, so * z[1]); df_add(vh.z, vl.z, so * z[2]);
      };
      auto drift = [&](float t) {
        pos_add(xh.x, xl.x, t * vh.x + t * vl.x);
        pos_add(xh.y, xl.y, t * vh.y + t * vl.y);
        pos_add(xh.z, xl.z, t * vh.z + t * vl.z);
      };
      // NPT half drift: x <- x + x (e^{v_e dt/2} - 1) + fa v (the increment in FP32)
      auto scaled_drift = [&](float em1, float fa) {
        pos_add(xh.x, xl.x, fmaf(xh.x, em1, xl.x * em1) + fa * vh.x + fa * vl.x);
        pos_add(xh.y, xl.y, fmaf(xh.y, em1, xl.y * em1) + fa * vh.y + fa * vl.y);
        pos_add(xh.z, xl.z, fmaf(xh.z, em1, xl.z * em1) + fa * vh.z + fa * vl.z);
      };
      if (KIND == 3) {
        const float eb = (float)q[kNptEbOpen], a = (float)q[kNptFbOpen] * vh.w;
        df_scale(vh.x, vl.x, eb); df_scale(vh.y, vl.y, eb); df_scale(vh.z, vl.z, eb);
        df_add(vh.x, vl.x, a * f.x); df_add(vh.y, vl.y, a * f.y); df_add(vh.z, vl.z, a * f.z);
        scaled_drift((float)q[kNptEa1], (float)q[kNptFa1]);
        ou();
        scaled_drift((float)q[kNptEa2], (float)q[kNptFa2]);
      } else {
        if (KIND == 2) {   // chain scaling of the double-float velocity
          const float c = (float)sysf[s];
          df_scale(vh.x, vl.x, c); df_scale(vh.y, vl.y, c); df_scale(vh.z, vl.z, c);
        }
        float a = (float)kick * vh.w;
        df_add(vh.x, vl.x, a * f.x); df_add(vh.y, vl.y, a * f.y); df_add(vh.z, vl.z, a * f.z);
        if (KIND != 1) {
          drift((float)dt);
        } else {
          drift((float)(0.5 * dt));
          ou();
          drift((float)(0.5 * dt));
        }
      }
      A.vh[k] = vh; A.vl[k] = vl; A.xh[k] = xh; A.xl[k] = xl;
      // skin check in FP32 (a threshold decision; FP64 is slow on this part)
      float4 rh = A.xrh[k], rl = A.xrl[k];
      float ex = (xh.x - rh.x) + (xl.x - rl.x), ey = (xh.y - rh.y) + (xl.y - rl.y), ez = (xh.z - rh.z) + (xl.z - rl.z);
      if (KIND == 3) {   // displacement beyond the cell's isotropic scaling since the listing
        const float l = (float)q[kNptLam];
        ex = fmaf(-l, rh.x, ex); ey = fmaf(-l, rh.y, ey); ez = fmaf(-l, rh.z, ez);
      }
      float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
      const DevPot& P = pots[S.pot[s]];
      if (KIND == 3) {
        const float se = (float)q[kNptAllow], se2 = se * se;
        if (se <= 0.f || d2 > se2) { S.relist[s] = 1; S.any[0] = 1; }
        else if (d2 > (float)P.soon2 * se2) S.soon[s] = 1;
        continue;
      }
      if (d2 > P.half_skin2f) { S.relist[s] = 1; S.any[0] = 1; }
      else if (d2 > P.soon_half_skin2f) S.soon[s] = 1;
      // inner list: refreshed in this step's pair launch once an atom moved half the inner skin
      float4 ph = A.xph[k], pl = A.xpl[k];
      float px = (xh.x - ph.x) + (xl.x - pl.x), py = (xh.y - ph.y) + (xl.y - pl.y), pz = (xh.z - ph.z) + (xl.z - pl.z);
      if (fmaf(px, px, fmaf(py, py, pz * pz)) > P.half_in2f) S.prune[s] = 1;
      continue;
    }
    const double sk = KIND == 3 ? q[kNptAllow] : 0.5 * pots[S.pot[s]].skin, d2 = dx * dx + dy * dy + dz * dz;
    if (sk <= 0 || d2 > sk * sk) { S.relist[s] = 1; S.any[0] = 1; }
    else if (d2 > pots[S.pot[s]].soon2 * sk * sk) S.soon[s] = 1;
    if constexpr (F64) {
      if (KIND != 3) {
        const double* x = A.xd + 3 * k;
        const double* xp = A.xpd + 3 * k;
        const double p0 = x[0] - xp[0], p1 = x[1] - xp[1], p2 = x[2] - xp[2];
        if (p0 * p0 + p1 * p1 + p2 * p2 > pots[S.pot[s]].half_in2d) S.prune[s] = 1;
      }
    }
  }
}

// Variable-cell filters and the barostat need a stress along every axis: a
// system with a non-periodic axis is refused (device error word, read at poll).
__global__ void k_require_periodic(int32_t B, SysArrays S, int32_t* err) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < B && S.pmask[s] != 7) atomicOr(err, kErrUnsupported);
}

// closing half kick of the last step; kinetic energy per warp (partial slot 7).
// npt (NPT steps): the closing kick is the barostat-coupled one of k_npt_sys,
// v <- v eb + fb F/m, instead of v += kick F/m.
template <bool F64>
__global__ void k_md_final(int32_t n_warps, SysArrays S, SlotArrays A, double kick, double* partial,
                           const double* __restrict__ vscale, const double* __restrict__ npt) {
  int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (w >= n_warps) return;
  int64_t k = (int64_t)w * kWarp + lane;
  double ke = 0;
  if (A.perm[k] >= 0) {
    const double* q = npt ? npt + kNptStride * (int64_t)A.sys[k] : nullptr;
    if constexpr (F64) {
      double mi = A.minvd[k];
      double* v = A.vd + 3 * k;
      const double* f = A.Fd + 3 * k;
      if (q) { for (int c = 0; c < 3; c++) v[c] = v[c] * q[kNptEbClose] + q[kNptFbClose] * mi * f[c]; }
      else { for (int c = 0; c < 3; c++) v[c] += kick * mi * f[c]; }
      if (vscale) { const double c = vscale[A.sys[k]]; for (int q = 0; q < 3; q++) v[q] *= c; }
      ke = 0.5 / mi * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    } else {
      float4 vh = A.vh[k], vl = A.vl[k], f = A.F[k];
      float a = (float)kick * vh.w;
      if (q) {
        const float eb = (float)q[kNptEbClose];
        df_scale(vh.x, vl.x, eb); df_scale(vh.y, vl.y, eb); df_scale(vh.z, vl.z, eb);
        a = (float)q[kNptFbClose] * vh.w;
      }
      df_add(vh.x, vl.x, a * f.x); df_add(vh.y, vl.y, a * f.y); df_add(vh.z, vl.z, a * f.z);
      if (vscale) {
        const float c = (float)vscale[A.sys[k]];
        df_scale(vh.x, vl.x, c); df_scale(vh.y, vl.y, c); df_scale(vh.z, vl.z, c);
      }
      A.vh[k] = vh; A.vl[k] = vl;
      double v0 = (double)vh.x + vl.x, v1 = (double)vh.y + vl.y, v2 = (double)vh.z + vl.z;
      // the mass as the correctly rounded FP32 reciprocal of the stored FP32
      // inverse mass (half an FP32 ulp, the size of the error the stored
      // inverse already carries): no FP64 division per atom, which is slow on
      // this part and runs every step under the chain and the barostat
      ke = 0.5 * (double)__frcp_rn(vh.w) * (v0 * v0 + v1 * v1 + v2 * v2);
    }
  }
  ke = warp_sum(ke);
  if (lane == 0) partial[(int64_t)w * kPartialStride + 7] = ke;
}


__global__ void k_set_u64(uint64_t* p, uint64_t v) { *p = v; }

// NVT Nose-Hoover chain (Martyna, Klein and Tuckerman 1992), chain of three
// per system, with the time-reversible factorisation of Martyna, Tuckerman,
// Tobias and Klein 1996: C(dt/2) B A (forces) B C(dt/2).  One chain half-step
// C(h), K the kinetic energy, Nf = 3n - 3, Q1 = Nf kT tau^2, Qk = kT tau^2:
// the last thermostat velocity takes a quarter kick from its force, the
// others (from the top down) are damped by the next one over h/4, kicked by
// h/2 and damped again; the thermostat positions advance by h w; the atoms'
// velocities scale by exp(-h w1); the same sweep runs bottom up with the new
// K.  Returns the velocity scale.
// The state lives in registers (xi, w by reference to the caller's locals) and
// the masses' reciprocals are taken once, so that the serial chain of FP64
// operations (slow on this part) holds no division and no memory round trip.
struct NhcConst {
  double nf, kT, q1, qk, iq1, iqk;   // Nf, kT, Q1 = Nf kT tau^2, Qk = kT tau^2, 1/Q1, 1/Qk
};
__device__ __forceinline__ double nhc_half_step(double h, double K, const NhcConst& c, double (&xi)[3],
                                                double (&w)[3]) {
  constexpr int M = 3;
  auto force = [&](int k, double Kin) {   // G_k
    return k == 0 ? (2.0 * Kin - c.nf * c.kT) * c.iq1 : ((k == 1 ? c.q1 : c.qk) * w[k - 1] * w[k - 1] - c.kT) * c.iqk;
  };
  w[M - 1] += 0.5 * h * force(M - 1, K);
#pragma unroll
  for (int k = M - 2; k >= 0; k--) {
    const double d = exp(-0.25 * h * w[k + 1]);
    w[k] = (w[k] * d + 0.5 * h * force(k, K)) * d;
  }
#pragma unroll
  for (int k = 0; k < M; k++) xi[k] += h * w[k];
  const double sc = exp(-h * w[0]);
  K *= sc * sc;
  // the closing sweep's factors use w_2, w_3 as they stand now (the sweep
  // updates w_1 and w_2 only afterwards): both exponentials go out together
  const double d0 = exp(-0.25 * h * w[1]), d1 = exp(-0.25 * h * w[2]);
  w[0] = (w[0] * d0 + 0.5 * h * force(0, K)) * d0;
  w[1] = (w[1] * d1 + 0.5 * h * force(1, K)) * d1;
  w[M - 1] += 0.5 * h * force(M - 1, K);
  return sc;
}

// One warp per system: the kinetic energy from the per-warp partials (slot 7,
// fixed order), `halves` chain half-steps of dt/2 (two between consecutive
// steps, one at the ends of a call), the product of their velocity scales.
// nhc: [B][6] (xi_1..3, w_1..3).
__global__ void k_nhc_update(int32_t B, SysArrays S, const double* __restrict__ partial, double dt, double tau,
                             int halves, double* nhc, double* vscale) {
  const int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= B) return;
  double K = 0;
  for (int w = S.warp_start[s] + lane; w < S.warp_end[s]; w += 32) K += partial[(int64_t)w * kPartialStride + 7];
  K = warp_sum(K);
  if (lane != 0) return;
  NhcConst c;
  c.nf = fmax(3.0 * S.n_atoms[s] - 3.0, 1.0);
  c.kT = S.kT[s];
  c.qk = c.kT * tau * tau;
  c.q1 = c.nf * c.qk;
  c.iq1 = 1.0 / c.q1;
  c.iqk = 1.0 / c.qk;
  double* st = nhc + 6 * (int64_t)s;
  double xi[3] = {st[0], st[1], st[2]}, w[3] = {st[3], st[4], st[5]};
  double sc = 1.0;
  for (int q = 0; q < halves; q++) {
    const double f = nhc_half_step(0.5 * dt, K, c, xi, w);
    K *= f * f;
    sc *= f;
  }
  for (int q = 0; q < 3; q++) { st[q] = xi[q]; st[3 + q] = w[q]; }
  vscale[s] = sc;
}

// NPT (isotropic barostat of Martyna, Tobias and Klein 1994, Langevin
// friction and noise on atoms and piston).  One warp per system: the kinetic
// energy K (partial slot 7) and the pair virial Xi = -tr W (slots 1-3) summed
// over the system's warps in order; then, with Nf = 3n, a = 1 + 3/Nf,
// W = (Nf + 3) kT tau^2, V = |det h| and G = (a 2K + Xi - 3 V p_ext) / W:
//   close: the closing piston half kick of a step, v_e += dt/2 G;
//   open:  the opening piston half kick of the next step, v_e += dt/2 G, and
//          that step's factors: the atom kick with c = a v_e (eb = e^{-c dt/2},
//          fb = dt/2 e^{-c dt/4} shc(c dt/4)); the half drift before the O
//          step with v_e (ea = e^{v_e dt/2} - 1, fa = dt/2 e^{v_e dt/4}
//          shc(v_e dt/4)); the piston's O step v_e' = c1 v_e +
//          sqrt((1 - c1^2) kT / W) xi (xi: first normal of counter (step,
//          0xffffffff)); the half drift after it with v_e'; the closing atom
//          kick with a v_e'; the new cell h e^{v_e dt/2} e^{v_e' dt/2}; and the
//          re-list allowance.  Under isotropic scaling by lambda since the
//          listing (h = lambda h_ref) a listed pair vector is lambda d_0 plus
//          the atoms' non-affine displacements u = x - lambda x_ref, so the
//          lists stay valid while 2 max |u| + |lambda - 1| r_list < skin:
//          allowance (skin - |lambda - 1| r_list) / 2 on |u|, lambda - 1 kept
//          for the kick's test; a system with no allowance left re-lists.
// baro[s] holds v_e between launches (after an open: v_e', the piston
// velocity after the O step).  A piston mass that is not positive (kT <= 0)
// or a non-finite force sets the non-finite error (read at poll) and leaves
// the piston unkicked.
enum NptMode : int { kNptOpen = 1, kNptClose = 2 };

__device__ __forceinline__ double shc(double y) {   // sinh(y) / y
  if (fabs(y) < 1e-3) { const double y2 = y * y; return 1.0 + y2 / 6.0 * (1.0 + y2 / 20.0); }
  return sinh(y) / y;
}

__global__ void k_npt_sys(int32_t B, SysArrays S, const DevPot* __restrict__ pots, const double* __restrict__ partial,
                          double dt, double c1, double tau, double p_ext, uint32_t seed,
                          const uint64_t* __restrict__ step_base, uint64_t koff, int mode, double* baro, double* f,
                          int32_t* err) {
  const int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= B) return;
  double K = 0, trw = 0;
  for (int w = S.warp_start[s] + lane; w < S.warp_end[s]; w += 32) {
    const double* pw = partial + (int64_t)w * kPartialStride;
    K += pw[7];
    trw += pw[1] + pw[2] + pw[3];
  }
  K = warp_sum(K);
  trw = warp_sum(trw);
  if (lane != 0) return;
  const double nf = 3.0 * S.n_atoms[s], al = 1.0 + 3.0 / nf, kT = S.kT[s];
  const double Wp = (nf + 3.0) * kT * tau * tau;
  double* h = S.h + 9 * s;
  const double V = fabs(h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                        h[2] * (h[3] * h[7] - h[4] * h[6]));
  double G = (al * 2.0 * K - trw - 3.0 * V * p_ext) / Wp;
  if (!(Wp > 0) || !isfinite(G)) { atomicOr(err, kErrNonFinite); G = 0; }   // kT <= 0, or a blown-up system
  double ve = baro[s];
  if (mode & kNptClose) ve += 0.5 * dt * G;
  if (!(mode & kNptOpen)) { baro[s] = ve; return; }
  ve += 0.5 * dt * G;
  double* q = f + kNptStride * (int64_t)s;
  auto kick = [&](double v, double& eb, double& fb) {
    const double c = al * v;
    eb = exp(-0.5 * c * dt);
    fb = 0.5 * dt * exp(-0.25 * c * dt) * shc(0.25 * c * dt);
  };
  auto drift = [&](double v, double& ea, double& fa) {
    ea = expm1(0.5 * v * dt);
    fa = 0.5 * dt * exp(0.25 * v * dt) * shc(0.25 * v * dt);
  };
  kick(ve, q[kNptEbOpen], q[kNptFbOpen]);
  drift(ve, q[kNptEa1], q[kNptFa1]);
  double z[3];
  normals3<true>(*step_base + koff, 0xffffffffu, seed, S.uid[s], z);
  const double ve2 = c1 * ve + sqrt((1.0 - c1 * c1) * kT / Wp) * z[0];
  drift(ve2, q[kNptEa2], q[kNptFa2]);
  kick(ve2, q[kNptEbClose], q[kNptFbClose]);
  const double e1 = exp(0.5 * ve * dt), e2 = exp(0.5 * ve2 * dt);
  for (int m = 0; m < 9; m++) h[m] = h[m] * e1 * e2;
  const double* hr = S.href + 9 * s;
  const double Vr = fabs(hr[0] * (hr[4] * hr[8] - hr[5] * hr[7]) - hr[1] * (hr[3] * hr[8] - hr[5] * hr[6]) +
                         hr[2] * (hr[3] * hr[7] - hr[4] * hr[6]));
  const double Vn = V * e1 * e1 * e1 * e2 * e2 * e2;
  const double lm1 = expm1(log(Vn / Vr) / 3.0);
  const DevPot& P = pots[S.pot[s]];
  const double se = 0.5 * (P.skin - fabs(lm1) * P.rlist);
  q[kNptAllow] = se;
  q[kNptLam] = lm1;
  if (se <= 0) { S.relist[s] = 1; S.any[0] = 1; }
  baro[s] = ve2;
}

}  // namespace ts
