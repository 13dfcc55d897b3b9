// ts_fire.cu -- batched variable-cell FIRE (Bitzek et al., PRL 97, 170201,
// 2006) behind ts_fire_step: the paper's structural relaxation under
// in-flight batching (Sec. 3).
//
// Generalised coordinates per system (UnitCellFilter-style reading):
// xt_i = x_i Fd^-T for the atoms and Q = c Fd (c = number of atoms) for the
// cell, with h = h0 Fd^T.  Generalised forces ft_i = F_i Fd and
// G = -V (sigma + p I) Fd^-T / c.  One step per system, unit masses:
//   P = f.v; P > 0: v <- (1-a) v + a |v| f/|f|, after Nmin positive steps
//   dt <- min(dt finc, dtmax), a <- a fa; P <= 0: v <- 0, dt <- dt fdec,
//   a <- a0 (the first step skips the test); v <- v + dt f; dq = dt v
//   clamped to |dq| <= maxstep over the whole system vector; q <- q + dq.
// The new velocity is v' = A v + g f with per-system scalars A, g, so |v'|^2
// follows from the reduced f.v, v.v, f.f and the clamp needs no second pass:
// kernel 1 reduces per warp, kernel 2 updates per system (FP64 cell state), kernel 3
// moves the atoms.
#include <type_traits>

#include "ts_kernels.cuh"

namespace ts {

constexpr int kFireCoef = 32;   // doubles of per-system coefficients
constexpr int kFireSysWarps = 16;   // warps of a k_fire_sys CTA (32 systems per CTA)

__device__ inline void inv_T3(const double* A, double* out) {   // out = A^-T
  double d = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
  // one division: an FP64 divide is a long instruction sequence on this part
  const double id = 1.0 / d;
  double g[9];
  g[0] = (A[4] * A[8] - A[5] * A[7]) * id; g[1] = (A[2] * A[7] - A[1] * A[8]) * id;
  g[2] = (A[1] * A[5] - A[2] * A[4]) * id; g[3] = (A[5] * A[6] - A[3] * A[8]) * id;
  g[4] = (A[0] * A[8] - A[2] * A[6]) * id; g[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  g[6] = (A[3] * A[7] - A[4] * A[6]) * id; g[7] = (A[1] * A[6] - A[0] * A[7]) * id;
  g[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) out[3 * a + b] = g[3 * b + a];
}

__global__ void k_fire_init(int32_t B, const double* __restrict__ cell, const ts_fire_params p, ts_fire_state* fs) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  ts_fire_state t;
  t.dt = p.dt0; t.alpha = p.alpha0; t.npos = 0; t.started = 0; t.converged = 0; t.nsteps = 0;
  for (int q = 0; q < 9; q++) { t.Fd[q] = (q == 0 || q == 4 || q == 8) ? 1.0 : 0.0; t.h0[q] = cell[9 * (int64_t)s + q]; }
  fs[s] = t;
}

// atom FIRE velocities: caller rows (offset(s) + 3 s + local) <-> slots
template <bool F64>
__global__ void k_fire_vel_io(int64_t Npad, SlotArrays A, double* fvel, int to_slots) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    int64_t row = (int64_t)p + 3 * (int64_t)A.sys[k];
    double* v = fvel + 3 * row;
    if constexpr (F64) {
      for (int c = 0; c < 3; c++) {
        if (to_slots) A.gd0[3 * k + c] = v[c]; else v[c] = A.gd0[3 * k + c];
      }
    } else {
      if (to_slots) A.g0[k] = make_float4((float)v[0], (float)v[1], (float)v[2], 0.f);
      else { float4 g = A.g0[k]; v[0] = g.x; v[1] = g.y; v[2] = g.z; }
    }
  }
}

// per warp: P = ft.v, v.v, ft.ft, max |F|^2 over the warp's atoms
template <bool F64>
__global__ void k_fire_reduce(int32_t n_warps, const int32_t* __restrict__ warp_sys, SlotArrays A,
                              const ts_fire_state* __restrict__ fs, double* part) {
  int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (w >= n_warps) return;
  int s = warp_sys[w];
  int64_t k = (int64_t)w * kWarp + lane;
  // the mixed variant works in FP32 (its forces and velocities are FP32; the
  // FP64 pipe is a small fraction of the FP32 one) and hands FP64 partials on
  using R = typename std::conditional<F64, double, float>::type;
  R P = 0, vv = 0, ff = 0, fm = 0;
  if (A.perm[k] >= 0) {
    const double* Fd = fs[s].Fd;
    R F[3], v[3];
    if constexpr (F64) {
      for (int c = 0; c < 3; c++) { F[c] = A.Fd[3 * k + c]; v[c] = A.gd0[3 * k + c]; }
    } else {
      float4 f = A.F[k], g = A.g0[k];
      F[0] = f.x; F[1] = f.y; F[2] = f.z; v[0] = g.x; v[1] = g.y; v[2] = g.z;
    }
    for (int b = 0; b < 3; b++) {
      R ft = F[0] * (R)Fd[b] + F[1] * (R)Fd[3 + b] + F[2] * (R)Fd[6 + b];
      P += ft * v[b]; vv += v[b] * v[b]; ff += ft * ft;
    }
    fm = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
  }
  for (int o = 16; o > 0; o >>= 1) {
    P += __shfl_xor_sync(0xffffffffu, P, o);
    vv += __shfl_xor_sync(0xffffffffu, vv, o);
    ff += __shfl_xor_sync(0xffffffffu, ff, o);
    fm = fmax(fm, __shfl_xor_sync(0xffffffffu, fm, o));
  }
  if (lane == 0) {
    part[4 * (int64_t)w] = P; part[4 * (int64_t)w + 1] = vv; part[4 * (int64_t)w + 2] = ff; part[4 * (int64_t)w + 3] = fm;
  }
}

// per system: convergence test, FIRE scalars, cell update; writes the
// coefficients the atom kernel applies.  final_mode: outputs only.
//
// A CTA of kFireSysWarps warps takes 32 systems: each warp reduces the
// partials of some of them (lanes over the system's warps), then one thread
// per system takes the system's step.  That step is a serial dependency chain,
// and a dependent FP64 operation costs tens of cycles on this part, so the
// mixed variant keeps FP64 only where the state needs it (the deformation
// gradient, the cell, the atom map and the skin budget) and takes the
// stress, the cell force and the FIRE scalars in FP32.
template <bool F64>
__global__ void __launch_bounds__(32 * kFireSysWarps) k_fire_sys(int32_t B, SysArrays S, ts_fire_state* fs, double* fvel, const double* __restrict__ Wint,
                           const double* __restrict__ Eint, const double* __restrict__ part, const ts_fire_params p,
                           const DevPot* __restrict__ pots, double* cell, double* coef, float* fcoef, uint8_t* conv_out,
                           double* E_out, double* fmax_out, double* smax_out, int final_mode) {
  using R = typename std::conditional<F64, double, float>::type;
  __shared__ double red[32][4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s0 = blockIdx.x * 32;
  for (int i = warp; i < 32 && s0 + i < B; i += kFireSysWarps) {
    const int sr = s0 + i;
    double P = 0, vv = 0, ff = 0, fm2 = 0;
    for (int w = S.warp_start[sr] + lane; w < S.warp_end[sr]; w += 32) {
      P += part[4 * (int64_t)w]; vv += part[4 * (int64_t)w + 1]; ff += part[4 * (int64_t)w + 2];
      fm2 = fmax(fm2, part[4 * (int64_t)w + 3]);
    }
    P = warp_sum(P); vv = warp_sum(vv); ff = warp_sum(ff);
    for (int o = 16; o > 0; o >>= 1) fm2 = fmax(fm2, __shfl_xor_sync(0xffffffffu, fm2, o));
    if (lane == 0) { red[i][0] = P; red[i][1] = vv; red[i][2] = ff; red[i][3] = fm2; }
  }
  __syncthreads();
  const int s = s0 + lane;
  if (warp != 0 || s >= B) return;
  R P = (R)red[lane][0], vv = (R)red[lane][1], ff = (R)red[lane][2];
  const double fm2 = red[lane][3];
  ts_fire_state st = fs[s];
  double* h = cell + 9 * (int64_t)s;
  double V = fabs(h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) + h[2] * (h[3] * h[7] - h[4] * h[6]));
  const R iV = (R)1 / (R)V;
  R sig[9], sm = 0;
  for (int q = 0; q < 9; q++) sig[q] = (R)Wint[9 * (int64_t)s + q] * iV;
  for (int q = 0; q < 9; q++) sm = fmax(sm, fabs(sig[q]));
  const R fm = sqrt((R)fm2);
  if (E_out) E_out[s] = Eint[s];
  if (fmax_out) fmax_out[s] = fm;
  if (smax_out) smax_out[s] = sm;
  double* cf = coef + kFireCoef * (int64_t)s;
  float* fc = fcoef + kFireCoef * (int64_t)s;
  if (final_mode) { if (conv_out) conv_out[s] = (uint8_t)st.converged; return; }
  cf[0] = 0.0;
  fc[0] = 0.f;
  if (!st.converged && fm <= (R)p.fmax && (!p.variable_cell || sm <= (R)p.smax)) st.converged = 1;
  if (conv_out) conv_out[s] = (uint8_t)st.converged;
  if (st.converged) { fs[s] = st; return; }
  int n = S.n_atoms[s];
  const R ic = (R)1 / (R)n;
  int64_t row0 = S.caller_off[s] + 3 * (int64_t)s + n;
  double* vc = fvel + 3 * row0;
  double FiT[9];
  inv_T3(st.Fd, FiT);
  R G[9], vcr[9];
  for (int q = 0; q < 9; q++) { G[q] = 0; vcr[q] = (R)vc[q]; }
  if (p.variable_cell) {
    R sp[9];
    for (int q = 0; q < 9; q++) sp[q] = sig[q];
    sp[0] += (R)p.p_ext; sp[4] += (R)p.p_ext; sp[8] += (R)p.p_ext;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        R acc = 0;
        for (int q = 0; q < 3; q++) acc += sp[3 * a + q] * (R)FiT[3 * q + b];
        G[3 * a + b] = -(R)V * acc * ic;
      }
    for (int q = 0; q < 9; q++) { P += G[q] * vcr[q]; vv += vcr[q] * vcr[q]; ff += G[q] * G[q]; }
  }
  R Ac = 1, bc = 0;
  if (st.started) {
    if (P > 0) {
      Ac = (R)1 - (R)st.alpha;
      bc = ff > 0 ? (R)st.alpha * sqrt(vv / ff) : (R)0;
      if (st.npos > p.nmin) { st.dt = fmin(st.dt * p.finc, p.dt_max); st.alpha *= p.falpha; }
      st.npos++;
    } else {
      Ac = 0; bc = 0;
      st.dt *= p.fdec; st.alpha = p.alpha0; st.npos = 0;
    }
  }
  st.started = 1;
  const R dt = (R)st.dt;
  R g = bc + dt;
  R vn2 = Ac * Ac * vv + g * g * ff + (R)2 * Ac * g * P;
  R nrm = dt * sqrt(fmax(vn2, (R)0));
  R scale = nrm > (R)p.maxstep ? (R)p.maxstep / nrm : (R)1;
  R sdt = scale * dt;
  double Fn[9];
  for (int q = 0; q < 9; q++) Fn[q] = st.Fd[q];
  if (p.variable_cell) {
    for (int q = 0; q < 9; q++) {
      R vn = Ac * vcr[q] + g * G[q];
      vc[q] = (double)vn;
      Fn[q] = st.Fd[q] + (double)(sdt * vn * ic);
    }
  }
  // h = h0 Fn^T
  double hn[9];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) hn[3 * a + b] = st.h0[3 * a] * Fn[3 * b] + st.h0[3 * a + 1] * Fn[3 * b + 1] + st.h0[3 * a + 2] * Fn[3 * b + 2];
  for (int q = 0; q < 9; q++) h[q] = hn[q];
  // atom map: x' = x (Fd^-T Fn^T) + dq Fn^T ;  M = Fd^-T Fn^T - I,  T = Fn^T
  cf[0] = 1.0; cf[1] = (double)Ac; cf[2] = (double)g; cf[3] = (double)sdt;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double m = 0;
      for (int q = 0; q < 3; q++) m += FiT[3 * a + q] * Fn[3 * b + q];
      cf[4 + 3 * a + b] = m - (a == b ? 1.0 : 0.0);
      cf[13 + 3 * a + b] = Fn[3 * b + a];
      cf[22 + 3 * a + b] = st.Fd[3 * a + b];
    }
  // skin left for atom motion after the cell change since the last listing:
  // image shifts move by |n dh| <= sum_a reach_a |dh_a|
  double dh = 0;
  for (int a = 0; a < 3; a++) {
    double r2 = 0;
    for (int b = 0; b < 3; b++) { double t = hn[3 * a + b] - S.href[9 * s + 3 * a + b]; r2 += t * t; }
    dh += S.reach[3 * s + a] * sqrt(r2);
  }
  double se = 0.5 * (pots[S.pot[s]].skin - dh);
  cf[31] = se;
  for (int q = 0; q < kFireCoef; q++) fc[q] = (float)cf[q];   // the mixed atom kernel's copy
  if (se <= 0) { S.relist[s] = 1; S.any[0] = 1; }
  for (int q = 0; q < 9; q++) st.Fd[q] = Fn[q];
  st.nsteps++;
  fs[s] = st;
}

template <bool F64>
__global__ void k_fire_update(int64_t Npad, SysArrays S, SlotArrays A, const double* __restrict__ coef,
                              const float* __restrict__ fcoef, const DevPot* __restrict__ pots) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Npad; k += (int64_t)gridDim.x * blockDim.x) {
    int p = A.perm[k];
    if (p < 0) continue;
    int s = A.sys[k];
    if constexpr (F64) {
      const double* cf = coef + kFireCoef * (int64_t)s;
      if (cf[0] == 0.0) continue;
      double Ac = cf[1], g = cf[2], sdt = cf[3];
      const double* M = cf + 4;
      const double* T = cf + 13;
      const double* Fd = cf + 22;
      double* x = A.xd + 3 * k;
      double* v = A.gd0 + 3 * k;
      const double* F = A.Fd + 3 * k;
      double dq[3], nx[3];
      for (int b = 0; b < 3; b++) {
        double ft = F[0] * Fd[b] + F[1] * Fd[3 + b] + F[2] * Fd[6 + b];
        v[b] = Ac * v[b] + g * ft;
        dq[b] = sdt * v[b];
      }
      for (int c = 0; c < 3; c++)
        nx[c] = x[c] + (x[0] * M[c] + x[1] * M[3 + c] + x[2] * M[6 + c]) + (dq[0] * T[c] + dq[1] * T[3 + c] + dq[2] * T[6 + c]);
      for (int c = 0; c < 3; c++) x[c] = nx[c];
      const double* xr = A.xrd + 3 * k;
      double dx2 = 0;
      for (int c = 0; c < 3; c++) dx2 += (x[c] - xr[c]) * (x[c] - xr[c]);
      double se = cf[31];
      if (se <= 0 || dx2 > se * se) { S.relist[s] = 1; S.any[0] = 1; }
      else if (dx2 > pots[S.pot[s]].soon2 * se * se) S.soon[s] = 1;
    } else {
      // FP32 throughout, from the FP32 copy of the coefficients
      const float* cf = fcoef + kFireCoef * (int64_t)s;
      if (cf[0] == 0.f) continue;
      const float Ac = cf[1], g = cf[2], sdt = cf[3];
      const float* M = cf + 4;
      const float* T = cf + 13;
      const float* Fd = cf + 22;
      float4 xh = A.xh[k], xl = A.xl[k], f = A.F[k], v = A.g0[k];
      float F[3] = {f.x, f.y, f.z}, vv[3] = {v.x, v.y, v.z}, dq[3];
      for (int b = 0; b < 3; b++) {
        float ft = F[0] * Fd[b] + F[1] * Fd[3 + b] + F[2] * Fd[6 + b];
        vv[b] = Ac * vv[b] + g * ft;
        dq[b] = sdt * vv[b];
      }
      float x0 = xh.x + xl.x, x1 = xh.y + xl.y, x2 = xh.z + xl.z;
      float d[3];
      for (int c = 0; c < 3; c++)
        d[c] = (x0 * M[c] + x1 * M[3 + c] + x2 * M[6 + c]) + (dq[0] * T[c] + dq[1] * T[3 + c] + dq[2] * T[6 + c]);
      pos_add(xh.x, xl.x, d[0]); pos_add(xh.y, xl.y, d[1]); pos_add(xh.z, xl.z, d[2]);
      A.xh[k] = xh; A.xl[k] = xl;
      A.g0[k] = make_float4(vv[0], vv[1], vv[2], 0.f);
      float4 rh = A.xrh[k], rl = A.xrl[k];
      float e0 = (xh.x - rh.x) + (xl.x - rl.x), e1 = (xh.y - rh.y) + (xl.y - rl.y), e2 = (xh.z - rh.z) + (xl.z - rl.z);
      const float dx2 = e0 * e0 + e1 * e1 + e2 * e2, se = cf[31], se2 = se * se;
      if (se <= 0.f || dx2 > se2) { S.relist[s] = 1; S.any[0] = 1; }
      else if (dx2 > (float)pots[S.pot[s]].soon2 * se2) S.soon[s] = 1;
    }
  }
}


}  // namespace ts

using namespace ts;

extern "C" ts_status ts_fire_init(ts_batch* b, ts_state* s, const ts_fire_params* p, ts_fire_state* fs, double* fvel,
                                  void* stream) {
  ts_status r = check_state(b, s, false);
  if (r != TS_OK) return r;
  if (!p || !fs || !fvel) return fail(b, TS_ERR_INVALID_ARG, "null FIRE argument");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(b->cfg.device);
  k_fire_init<<<(s->n_systems + 127) / 128, 128, 0, st>>>(s->n_systems, s->cell, *p, fs);
  b->launches++;
  if (!cuda_ok(b, cudaMemsetAsync(fvel, 0, sizeof(double) * 3 * (s->n_atoms + 3 * (int64_t)s->n_systems), st), "memset"))
    return TS_ERR_CUDA;
  return cuda_ok(b, cudaGetLastError(), "ts_fire_init") ? TS_OK : TS_ERR_CUDA;
}

extern "C" ts_status ts_fire_step(ts_batch* b, ts_state* s, ts_fire_state* fs, double* fvel, const ts_fire_params* p,
                                  int n_steps, uint8_t* converged, double* E, double* fmax, double* smax, void* stream) {
  ts_status r = check_state(b, s, false);
  if (r != TS_OK) return r;
  if (!p || !fs || !fvel || n_steps < 0 || !(p->dt0 > 0) || !(p->maxstep > 0))
    return fail(b, TS_ERR_INVALID_ARG, "bad FIRE arguments");
  cudaStream_t st = (cudaStream_t)stream;
  r = prologue(b, s, st, false, true);
  if (r != TS_OK) return r;
  if (p->variable_cell) {
    k_require_periodic<<<(b->B + 127) / 128, 128, 0, st>>>(b->B, b->S, b->d_err);
    b->launches++;
  }
  int g = (int)std::min<int64_t>(std::max<int64_t>((b->Npad + 255) / 256, 1), 148 * 16);
  if (b->f64) k_fire_vel_io<true><<<g, 256, 0, st>>>(b->Npad, b->A, fvel, 1);
  else k_fire_vel_io<false><<<g, 256, 0, st>>>(b->Npad, b->A, fvel, 1);
  b->launches++;
  // forces, energy and virial current at the starting configuration
  relist(b, st, true);
  pair(b, st, true, false);
  reduce_sys(b, st, nullptr, nullptr, nullptr);
  clear_dirty(b, st);
  int wblocks = (int)(((int64_t)b->nwarps * 32 + 127) / 128);
  int sblocks = (b->B + 31) / 32;
  for (int k = 0; k <= n_steps; k++) {
    if (b->f64) k_fire_reduce<true><<<wblocks, 128, 0, st>>>(b->nwarps, b->d_warp_sys, b->A, fs, b->d_gparam_part);
    else k_fire_reduce<false><<<wblocks, 128, 0, st>>>(b->nwarps, b->d_warp_sys, b->A, fs, b->d_gparam_part);
    (b->f64 ? k_fire_sys<true> : k_fire_sys<false>)<<<sblocks, 32 * kFireSysWarps, 0, st>>>(b->B, b->S, fs, fvel, b->d_Wint, b->d_Eint, b->d_gparam_part, *p, b->d_pots,
                                        s->cell, b->d_scal, b->d_fcoef, converged, E, fmax, smax, k == n_steps);
    b->launches += 2;
    if (k == n_steps) break;
    if (b->f64) k_fire_update<true><<<g, 256, 0, st>>>(b->Npad, b->S, b->A, b->d_scal, b->d_fcoef, b->d_pots);
    else k_fire_update<false><<<g, 256, 0, st>>>(b->Npad, b->S, b->A, b->d_scal, b->d_fcoef, b->d_pots);
    k_geometry<<<(b->B + 31) / 32, 32, 0, st>>>(b->B, b->S, s->cell, s->pbc, b->d_pots, b->d_err, 0);
    k_shift_table<<<b->B, 128, 0, st>>>(b->B, b->S);
    b->launches += 3;
    relist(b, st, true);
    pair(b, st, true, false);
    reduce_sys(b, st, nullptr, nullptr, nullptr);
    clear_dirty(b, st);
  }
  export_state(b, st, s->pos, nullptr);
  if (b->f64) k_fire_vel_io<true><<<g, 256, 0, st>>>(b->Npad, b->A, fvel, 0);
  else k_fire_vel_io<false><<<g, 256, 0, st>>>(b->Npad, b->A, fvel, 0);
  b->launches++;
  return cuda_ok(b, cudaGetLastError(), "ts_fire_step") ? TS_OK : TS_ERR_CUDA;
}
