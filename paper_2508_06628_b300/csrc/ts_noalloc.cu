// ts_noalloc.cu -- ts_pair_forces_noalloc: energies, forces and stress of a
// small batch with no device allocation, for callers that cannot call
// cudaMalloc: a host program that hands this library a fixed set of buffers
// and forbids allocation after start-up, code running inside another
// framework that owns the device allocator, or a loop that cannot afford
// cudaMalloc's implicit device synchronisation.
//
// It computes the same quantities as ts_pair_forces in FP64, but directly
// from the caller's arrays: for every atom, an all-pairs sum over the atoms
// of its system and over every lattice image that can lie within the cutoff
// (no neighbour list, no batch object).  Its only scratch is the table of
// per-CTA energy/virial partials below: a file-scope device array of fixed
// size, so the entry point never allocates.
//
// Each system is covered by kNoAllocChunks CTAs that stride over its atoms;
// every CTA reduces its threads' energy and virial in a fixed order and
// writes one row of the table (plain stores, no atomics), and a second kernel
// sums a system's rows in row order.  Results are therefore bit-reproducible
// and do not depend on the rest of the batch.
//
// The table is shared by every call on a device and keeps the last call's
// contents; each call overwrites every row it reads.  Calls that overlap on
// the GPU (two streams, or two host threads) race on it and must be
// serialised by the caller.
#include "ts_kernels.cuh"

namespace ts {

constexpr int kNoAllocMaxSystems = 4096;
constexpr int kNoAllocChunks = 2;                 // CTAs (table rows) per system
constexpr int kNoAllocThreads = 128;
constexpr int kNoAllocMaxPots = 4;
constexpr int kNoAllocMaxDevices = 64;
constexpr double kNoAllocMaxFrac = 1e6;           // |fractional separation| beyond this: invalid input

// 4096 systems x 2 rows x 8 doubles = 512 KiB per device that loads the library
static __device__ __align__(256) double g_noalloc_rows[kNoAllocMaxSystems * kNoAllocChunks * 8];

struct NoAllocPots {
  DevPot p[kNoAllocMaxPots];
};

// The system's cell and atom range, or false when the input cannot be
// evaluated: a potential index outside [0, n_pots), offsets out of order or
// outside [0, N], a singular or non-finite cell, or a cell so thin that an
// image more than kMaxReach cells away could lie within the cutoff (the
// limit of the batch path too).  range_ok: the offsets at least delimit atoms
// of the batch.
__device__ __forceinline__ bool noalloc_system(int s, int64_t N, int n_pots, const double* __restrict__ cell,
                                               const int32_t* __restrict__ pot_idx,
                                               const int64_t* __restrict__ offsets, const NoAllocPots& P,
                                               int64_t& a, int64_t& e, int& q, bool& range_ok, double rw[3],
                                               double g[9]) {
  q = pot_idx[s];
  a = offsets[s];
  e = offsets[s + 1];
  range_ok = a >= 0 && e <= N && a <= e;
  if (q < 0 || q >= n_pots || !range_ok) return false;
  const double* h = cell + 9 * (int64_t)s;
  const double det = h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                     h[2] * (h[3] * h[7] - h[4] * h[6]);
  const double V = fabs(det);
  if (!(V > 0) || !isfinite(V)) return false;
  const double rc = sqrt(P.p[q].rc2d);
  // perpendicular width w_a = V / |b x c|: an image n_a further than rc / w_a
  // cells from the fractional separation cannot lie within rc
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const double* u = h + 3 * ((c + 1) % 3);
    const double* v = h + 3 * ((c + 2) % 3);
    const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
    rw[c] = rc * sqrt(cx * cx + cy * cy + cz * cz) / V;
    if (!(rw[c] <= (double)kMaxReach)) return false;
  }
  g[0] = (h[4] * h[8] - h[5] * h[7]) / det; g[1] = (h[2] * h[7] - h[1] * h[8]) / det;
  g[2] = (h[1] * h[5] - h[2] * h[4]) / det; g[3] = (h[5] * h[6] - h[3] * h[8]) / det;
  g[4] = (h[0] * h[8] - h[2] * h[6]) / det; g[5] = (h[2] * h[3] - h[0] * h[5]) / det;
  g[6] = (h[3] * h[7] - h[4] * h[6]) / det; g[7] = (h[1] * h[6] - h[0] * h[7]) / det;
  g[8] = (h[0] * h[4] - h[1] * h[3]) / det;
  return true;
}

// grid (kNoAllocChunks, B): CTA (c, s) takes atoms off[s] + c*T + t, stepping
// by kNoAllocChunks*T, and writes table row s*kNoAllocChunks + c
__global__ void __launch_bounds__(kNoAllocThreads) k_noalloc_pair(int64_t N, int n_pots,
    const double* __restrict__ pos, const double* __restrict__ cell, const int32_t* __restrict__ sidx,
    const int32_t* __restrict__ pot_idx, const int64_t* __restrict__ offsets, const NoAllocPots P,
    double* __restrict__ F, double* __restrict__ rows) {
  const int s = blockIdx.y, t = threadIdx.x;
  int64_t a, e;
  int q;
  bool range_ok;
  double rw[3], g[9];
  const bool ok = noalloc_system(s, N, n_pots, cell, pot_idx, offsets, P, a, e, q, range_ok, rw, g);
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  bool bad = !ok;
  if (!ok && range_ok && F) {   // a system that cannot be evaluated: NaN forces on its atoms
    for (int64_t i = a + (int64_t)blockIdx.x * kNoAllocThreads + t; i < e;
         i += (int64_t)kNoAllocChunks * kNoAllocThreads)
      F[3 * i] = F[3 * i + 1] = F[3 * i + 2] = nan;
  }
  if (ok) {
    const DevPot& pp = P.p[q];
    const double* h = cell + 9 * (int64_t)s;
    for (int64_t i = a + (int64_t)blockIdx.x * kNoAllocThreads + t; i < e;
         i += (int64_t)kNoAllocChunks * kNoAllocThreads) {
      const double xi0 = pos[3 * i], xi1 = pos[3 * i + 1], xi2 = pos[3 * i + 2];
      // an atom whose system index disagrees with the offsets, or whose
      // position is not finite, invalidates the system
      bool atom_ok = sidx[i] == s && isfinite(xi0) && isfinite(xi1) && isfinite(xi2);
      double f0 = 0, f1 = 0, f2 = 0, en = 0, w[6] = {0, 0, 0, 0, 0, 0};
      for (int64_t j = a; j < e && atom_ok; j++) {
        const double b0 = pos[3 * j] - xi0, b1 = pos[3 * j + 1] - xi1, b2 = pos[3 * j + 2] - xi2;
        int lo[3], hi[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const double ds = b0 * g[c] + b1 * g[3 + c] + b2 * g[6 + c];
          if (!(fabs(ds) < kNoAllocMaxFrac)) { atom_ok = false; break; }   // non-finite or absurdly far
          lo[c] = (int)floor(-ds - rw[c]);
          hi[c] = (int)ceil(-ds + rw[c]);
        }
        if (!atom_ok) break;
        for (int nz = lo[2]; nz <= hi[2]; nz++)
          for (int ny = lo[1]; ny <= hi[1]; ny++)
            for (int nx = lo[0]; nx <= hi[0]; nx++) {
              if (j == i && nx == 0 && ny == 0 && nz == 0) continue;
              const double d0 = b0 + nx * h[0] + ny * h[3] + nz * h[6];
              const double d1 = b1 + nx * h[1] + ny * h[4] + nz * h[7];
              const double d2 = b2 + nx * h[2] + ny * h[5] + nz * h[8];
              const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
              if (!(r2 < pp.rc2d)) continue;
              double phi, fr;
              PotMath<double>::eval(pp, r2, phi, fr);
              f0 += fr * d0; f1 += fr * d1; f2 += fr * d2;
              en += 0.5 * (phi - pp.phicd);
              const double hf = 0.5 * fr;
              w[0] += hf * d0 * d0; w[1] += hf * d1 * d1; w[2] += hf * d2 * d2;
              w[3] += hf * d0 * d1; w[4] += hf * d0 * d2; w[5] += hf * d1 * d2;
            }
      }
      if (!atom_ok) { bad = true; f0 = f1 = f2 = nan; }
      if (F) { F[3 * i] = f0; F[3 * i + 1] = f1; F[3 * i + 2] = f2; }
      acc[0] += en;
      for (int c = 0; c < 6; c++) acc[1 + c] += w[c];
    }
  }
  // fixed-order block reduction: warp shuffles, then warp 0 over the warps
  __shared__ double red[kNoAllocThreads / kWarp][8];
  const int lane = t & 31, wid = t >> 5;
  const int anybad = __syncthreads_or(bad);
  for (int c = 0; c < 7; c++) {
    const double v = warp_sum(acc[c]);
    if (lane == 0) red[wid][c] = v;
  }
  __syncthreads();
  if (t < 7) {
    double v = 0;
    for (int k = 0; k < kNoAllocThreads / kWarp; k++) v += red[k][t];
    rows[((int64_t)s * kNoAllocChunks + blockIdx.x) * 8 + t] = anybad ? nan : v;
  }
}

// one thread per system: E and stress from the system's rows, in row order
__global__ void k_noalloc_finish(int32_t B, const double* __restrict__ cell, const double* __restrict__ rows,
                                 double* E, double* stress) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int c = 0; c < kNoAllocChunks; c++)
    for (int k = 0; k < 7; k++) acc[k] += rows[((int64_t)s * kNoAllocChunks + c) * 8 + k];
  const double* h = cell + 9 * (int64_t)s;
  const double V = fabs(h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                        h[2] * (h[3] * h[7] - h[4] * h[6]));
  if (E) E[s] = acc[0];
  if (stress) {
    const double W[9] = {acc[1], acc[4], acc[5], acc[4], acc[2], acc[6], acc[5], acc[6], acc[3]};
    for (int k = 0; k < 9; k++) stress[9 * (int64_t)s + k] = W[k] / V;
  }
}

// device address of the static table, looked up once per device
static double* g_noalloc_ptr[kNoAllocMaxDevices];

}  // namespace ts

using namespace ts;

extern "C" ts_status ts_pair_forces_noalloc(const ts_potential* pots, int n_pots, const ts_state* s,
                                            const int64_t* offsets, double* F, double* E, double* stress,
                                            void* stream) {
  if (!pots || n_pots < 1 || n_pots > kNoAllocMaxPots || !s || !offsets || !s->pos || !s->cell || !s->system_idx ||
      !s->pot_idx || s->n_atoms < 1 || s->n_systems < 1)
    return TS_ERR_INVALID_ARG;
  if (s->n_systems > kNoAllocMaxSystems) return TS_ERR_BUDGET;   // more systems than the table holds
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return TS_ERR_CUDA;
  if (!g_noalloc_ptr[dev]) {   // set-up on this device's first call
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_rows) != cudaSuccess || !p) { cudaGetLastError(); return TS_ERR_CUDA; }
    g_noalloc_ptr[dev] = (double*)p;
  }
  NoAllocPots P;
  memset(&P, 0, sizeof P);
  for (int q = 0; q < n_pots; q++) {
    const ts_potential& Q = pots[q];
    if (Q.kind < 0 || Q.kind > 2) return TS_ERR_INVALID_ARG;
    if (Q.kind == TS_SOFT_SPHERE && !(Q.p[2] >= 1.0)) return TS_ERR_INVALID_ARG;
    DevPot& D = P.p[q];
    D.kind = Q.kind; D.shift = Q.shift;
    for (int c = 0; c < 3; c++) { D.pd[c] = Q.p[c]; D.pf[c] = (float)Q.p[c]; }
    const double rc = Q.kind == TS_SOFT_SPHERE ? Q.p[0] : Q.cutoff;
    if (!(rc > 0) || !std::isfinite(rc)) return TS_ERR_INVALID_ARG;
    D.rc2d = rc * rc;
    double phic = 0;
    if (Q.shift && Q.kind == TS_LJ) { double t = Q.p[0] / rc, t6 = t * t * t * t * t * t; phic = 4 * Q.p[1] * (t6 * t6 - t6); }
    if (Q.shift && Q.kind == TS_MORSE) { double e = exp(-Q.p[1] * (rc - Q.p[2])); phic = Q.p[0] * (e * e - 2 * e); }
    D.phicd = phic;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* rows = g_noalloc_ptr[dev];
  const int B = s->n_systems;
  k_noalloc_pair<<<dim3(kNoAllocChunks, B), kNoAllocThreads, 0, st>>>(s->n_atoms, n_pots, s->pos, s->cell,
                                                                      s->system_idx, s->pot_idx, offsets, P, F, rows);
  k_noalloc_finish<<<(B + 127) / 128, 128, 0, st>>>(B, s->cell, rows, E, stress);
  return cudaGetLastError() == cudaSuccess ? TS_OK : TS_ERR_CUDA;
}
