// ts_noalloc.cu -- ts_pair_forces_noalloc: energies, forces and stress of a
// small batch with no device allocation, for callers that cannot call
// cudaMalloc (a host program that hands this library a fixed set of buffers
// and forbids allocation after start-up, code that runs while another
// component owns the device allocator, or work issued into a captured
// stream, where an allocation would break the capture).
//
// It computes the same quantities as ts_pair_forces in FP64, but directly
// from the caller's arrays: for every atom, an all-pairs sum over the atoms
// of its system and over every lattice image that can lie within the cutoff
// (no neighbour list, no batch object).  Its only scratch is the per-system
// energy/virial accumulator below: a file-scope device array of fixed size,
// so the entry point never allocates.
//
// The accumulator is shared by every call on a device and keeps the last
// call's contents; each call clears the rows it uses before accumulating.
// Calls that overlap on the GPU (two streams, or two host threads) race on
// it and must be serialised by the caller.
#include "ts_kernels.cuh"

namespace ts {

constexpr int kNoAllocMaxSystems = 4096;       // rows of the static accumulator
constexpr int kNoAllocMaxPots = 4;
constexpr int kNoAllocMaxDevices = 64;

// 4096 systems x 8 doubles = 256 KiB per device that loads the library
static __device__ __align__(256) double g_noalloc_acc[kNoAllocMaxSystems * 8];

struct NoAllocPots {
  DevPot p[kNoAllocMaxPots];
};

__global__ void k_noalloc_clear(int32_t B, double* acc) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < B * 8) acc[t] = 0.0;
}

// one thread per atom: all-pairs over the atom's system and its images
__global__ void k_noalloc_pair(int64_t N, int32_t B, const double* __restrict__ pos, const double* __restrict__ cell,
                               const int32_t* __restrict__ sidx, const int32_t* __restrict__ pot_idx,
                               const int64_t* __restrict__ offsets, const NoAllocPots P, double* F, double* acc) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int s = sidx[i];
  if (s < 0 || s >= B) return;
  const DevPot& pp = P.p[pot_idx[s]];
  const double* h = cell + 9 * (int64_t)s;
  double V = fabs(h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) + h[2] * (h[3] * h[7] - h[4] * h[6]));
  double rc = sqrt(pp.rc2d);
  // perpendicular widths and the inverse cell: for a pair with fractional
  // difference ds, |d| >= |ds_a + n_a| w_a, so n_a outside
  // [floor(-ds_a - rc/w_a), ceil(-ds_a + rc/w_a)] cannot be within rc
  double rw[3], g[9];
  for (int a = 0; a < 3; a++) {
    const double* b = h + 3 * ((a + 1) % 3);
    const double* c = h + 3 * ((a + 2) % 3);
    double cx = b[1] * c[2] - b[2] * c[1], cy = b[2] * c[0] - b[0] * c[2], cz = b[0] * c[1] - b[1] * c[0];
    rw[a] = rc * sqrt(cx * cx + cy * cy + cz * cz) / V;
  }
  {
    double dt = h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) + h[2] * (h[3] * h[7] - h[4] * h[6]);
    g[0] = (h[4] * h[8] - h[5] * h[7]) / dt; g[1] = (h[2] * h[7] - h[1] * h[8]) / dt;
    g[2] = (h[1] * h[5] - h[2] * h[4]) / dt; g[3] = (h[5] * h[6] - h[3] * h[8]) / dt;
    g[4] = (h[0] * h[8] - h[2] * h[6]) / dt; g[5] = (h[2] * h[3] - h[0] * h[5]) / dt;
    g[6] = (h[3] * h[7] - h[4] * h[6]) / dt; g[7] = (h[1] * h[6] - h[0] * h[7]) / dt;
    g[8] = (h[0] * h[4] - h[1] * h[3]) / dt;
  }
  double xi0 = pos[3 * i], xi1 = pos[3 * i + 1], xi2 = pos[3 * i + 2];
  double f0 = 0, f1 = 0, f2 = 0, e = 0, w[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t j = offsets[s]; j < offsets[s + 1]; j++) {
    double b0 = pos[3 * j] - xi0, b1 = pos[3 * j + 1] - xi1, b2 = pos[3 * j + 2] - xi2;
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
      double ds = b0 * g[a] + b1 * g[3 + a] + b2 * g[6 + a];
      lo[a] = (int)floor(-ds - rw[a]);
      hi[a] = (int)ceil(-ds + rw[a]);
    }
    for (int nz = lo[2]; nz <= hi[2]; nz++)
      for (int ny = lo[1]; ny <= hi[1]; ny++)
        for (int nx = lo[0]; nx <= hi[0]; nx++) {
          if (j == i && nx == 0 && ny == 0 && nz == 0) continue;
          double d0 = b0 + nx * h[0] + ny * h[3] + nz * h[6];
          double d1 = b1 + nx * h[1] + ny * h[4] + nz * h[7];
          double d2 = b2 + nx * h[2] + ny * h[5] + nz * h[8];
          double r2 = d0 * d0 + d1 * d1 + d2 * d2;
          if (!(r2 < pp.rc2d)) continue;
          double phi, fr;
          PotMath<double>::eval(pp, r2, phi, fr);
          f0 += fr * d0; f1 += fr * d1; f2 += fr * d2;
          e += 0.5 * (phi - pp.phicd);
          double hf = 0.5 * fr;
          w[0] += hf * d0 * d0; w[1] += hf * d1 * d1; w[2] += hf * d2 * d2;
          w[3] += hf * d0 * d1; w[4] += hf * d0 * d2; w[5] += hf * d1 * d2;
        }
  }
  if (F) { F[3 * i] = f0; F[3 * i + 1] = f1; F[3 * i + 2] = f2; }
  atomicAdd(&acc[8 * s], e);
  for (int c = 0; c < 6; c++) atomicAdd(&acc[8 * s + 1 + c], w[c]);
}

__global__ void k_noalloc_finish(int32_t B, const double* __restrict__ cell, const double* __restrict__ acc, double* E,
                                 double* stress) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  const double* h = cell + 9 * (int64_t)s;
  double V = fabs(h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) + h[2] * (h[3] * h[7] - h[4] * h[6]));
  const double* a = acc + 8 * (int64_t)s;
  if (E) E[s] = a[0];
  if (stress) {
    double W[9] = {a[1], a[4], a[5], a[4], a[2], a[6], a[5], a[6], a[3]};
    for (int q = 0; q < 9; q++) stress[9 * (int64_t)s + q] = W[q] / V;
  }
}

// device address of the static accumulator, fetched once per device
static double* g_noalloc_ptr[kNoAllocMaxDevices];

}  // namespace ts

using namespace ts;

extern "C" ts_status ts_pair_forces_noalloc(const ts_potential* pots, int n_pots, const ts_state* s,
                                            const int64_t* offsets, double* F, double* E, double* stress,
                                            void* stream) {
  if (!pots || n_pots < 1 || n_pots > kNoAllocMaxPots || !s || !offsets || !s->pos || !s->cell || !s->system_idx ||
      !s->pot_idx || s->n_atoms < 1 || s->n_systems < 1)
    return TS_ERR_INVALID_ARG;
  if (s->n_systems > kNoAllocMaxSystems) return TS_ERR_BUDGET;   // more systems than accumulator rows
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return TS_ERR_CUDA;
  if (!g_noalloc_ptr[dev]) {   // set-up on this device's first call (must precede any stream capture)
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_acc) != cudaSuccess || !p) { cudaGetLastError(); return TS_ERR_CUDA; }
    g_noalloc_ptr[dev] = (double*)p;
  }
  NoAllocPots P;
  memset(&P, 0, sizeof P);
  for (int q = 0; q < n_pots; q++) {
    const ts_potential& Q = pots[q];
    if (Q.kind < 0 || Q.kind > 2) return TS_ERR_INVALID_ARG;
    DevPot& D = P.p[q];
    D.kind = Q.kind; D.shift = Q.shift;
    for (int c = 0; c < 3; c++) { D.pd[c] = Q.p[c]; D.pf[c] = (float)Q.p[c]; }
    double rc = Q.kind == TS_SOFT_SPHERE ? Q.p[0] : Q.cutoff;
    if (!(rc > 0)) return TS_ERR_INVALID_ARG;
    D.rc2d = rc * rc;
    double phic = 0;
    if (Q.shift && Q.kind == TS_LJ) { double t = Q.p[0] / rc, t6 = t * t * t * t * t * t; phic = 4 * Q.p[1] * (t6 * t6 - t6); }
    if (Q.shift && Q.kind == TS_MORSE) { double e = exp(-Q.p[1] * (rc - Q.p[2])); phic = Q.p[0] * (e * e - 2 * e); }
    D.phicd = phic;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* acc = g_noalloc_ptr[dev];
  int B = s->n_systems;
  k_noalloc_clear<<<(B * 8 + 255) / 256, 256, 0, st>>>(B, acc);
  k_noalloc_pair<<<(int)((s->n_atoms + 127) / 128), 128, 0, st>>>(s->n_atoms, B, s->pos, s->cell, s->system_idx,
                                                                  s->pot_idx, offsets, P, F, acc);
  k_noalloc_finish<<<(B + 127) / 128, 128, 0, st>>>(B, s->cell, acc, E, stress);
  return cudaGetLastError() == cudaSuccess ? TS_OK : TS_ERR_CUDA;
}
