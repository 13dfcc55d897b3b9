// ts_inflight.cu -- retire/admit step of the in-flight batching runtime
// (TorchSim Sec. 3, Fig. 3: converged systems leave the batch and systems
// sampled from the stream take their place while memory allows).
//
// ts_batch_compact_admit writes a new batched state: the kept systems, in
// order, gathered by one kernel from the old state through a small map built
// on the host, then the admitted systems copied from host arrays (one copy
// per array).  FIRE state follows the kept systems and is initialised fresh
// for admitted ones.  The batch re-derives its layout on the next call.
#include "ts_kernels.cuh"

namespace ts {

// map rows: (src atom offset, dst atom offset, atoms, src system, dst system)
__global__ void k_compact(int32_t n_keep, const int64_t* __restrict__ map, const double* __restrict__ pos_s,
                          const double* __restrict__ vel_s, const double* __restrict__ mass_s,
                          const double* __restrict__ cell_s, const uint8_t* __restrict__ pbc_s,
                          const int32_t* __restrict__ pot_s, const uint32_t* __restrict__ uid_s, double* pos_d,
                          double* vel_d, double* mass_d, double* cell_d, uint8_t* pbc_d, int32_t* sidx_d,
                          int32_t* pot_d, uint32_t* uid_d, const ts_fire_state* __restrict__ fs_s,
                          const double* __restrict__ fv_s, ts_fire_state* fs_d, double* fv_d) {
  int r = blockIdx.x;
  if (r >= n_keep) return;
  const int64_t* m = map + 5 * r;
  int64_t so = m[0], dof = m[1], n = m[2];
  int ss = (int)m[3], ds = (int)m[4];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    for (int c = 0; c < 3; c++) pos_d[3 * (dof + i) + c] = pos_s[3 * (so + i) + c];
    if (vel_s && vel_d) for (int c = 0; c < 3; c++) vel_d[3 * (dof + i) + c] = vel_s[3 * (so + i) + c];
    mass_d[dof + i] = mass_s[so + i];
    sidx_d[dof + i] = ds;
  }
  if (fv_s && fv_d) {   // generalised velocity rows: atoms then the 3 cell rows
    int64_t rs = so + 3 * (int64_t)ss, rd = dof + 3 * (int64_t)ds;
    for (int64_t i = threadIdx.x; i < 3 * (n + 3); i += blockDim.x) fv_d[3 * rd + i] = fv_s[3 * rs + i];
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < 9; q++) cell_d[9 * (int64_t)ds + q] = cell_s[9 * (int64_t)ss + q];
    for (int q = 0; q < 3; q++) pbc_d[3 * (int64_t)ds + q] = pbc_s ? pbc_s[3 * (int64_t)ss + q] : 1;
    pot_d[ds] = pot_s[ss];
    if (uid_d) uid_d[ds] = uid_s ? uid_s[ss] : (uint32_t)ss;
    if (fs_s && fs_d) fs_d[ds] = fs_s[ss];
  }
}

// admitted systems: system index, pbc and fresh FIRE state
__global__ void k_admit_fill(int32_t first_sys, int32_t n_new, int64_t first_atom, const int64_t* __restrict__ starts,
                             int32_t* sidx_d, uint8_t* pbc_d, const double* __restrict__ cell_d,
                             const ts_fire_params p, ts_fire_state* fs_d, double* fv_d, int fire) {
  int k = blockIdx.x;
  if (k >= n_new) return;
  int ds = first_sys + k;
  int64_t a0 = first_atom + starts[k], a1 = first_atom + starts[k + 1];
  for (int64_t i = a0 + threadIdx.x; i < a1; i += blockDim.x) sidx_d[i] = ds;
  if (fire && fv_d) {
    int64_t rd = a0 + 3 * (int64_t)ds;
    for (int64_t i = threadIdx.x; i < 3 * (a1 - a0 + 3); i += blockDim.x) fv_d[3 * rd + i] = 0.0;
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < 3; q++) pbc_d[3 * (int64_t)ds + q] = 1;
    if (fire && fs_d) {
      ts_fire_state t;
      t.dt = p.dt0; t.alpha = p.alpha0; t.npos = 0; t.started = 0; t.converged = 0; t.nsteps = 0;
      for (int q = 0; q < 9; q++) { t.Fd[q] = (q == 0 || q == 4 || q == 8) ? 1.0 : 0.0; t.h0[q] = cell_d[9 * (int64_t)ds + q]; }
      fs_d[ds] = t;
    }
  }
}

}  // namespace ts

using namespace ts;

extern "C" ts_status ts_batch_compact_admit(ts_batch* b, const ts_state* src, const uint8_t* keep,
                                            const ts_host_systems* add, ts_state* dst, const ts_fire_state* fs_src,
                                            const double* fvel_src, ts_fire_state* fs_dst, double* fvel_dst,
                                            const ts_fire_params* fire, void* stream) {
  if (!b || !dst || !dst->pos || !dst->mass || !dst->cell || !dst->pbc || !dst->system_idx || !dst->pot_idx)
    return TS_ERR_INVALID_ARG;
  if (src && src->n_systems > 0 && (!keep || !src->pos || !src->mass || !src->cell || !src->pot_idx))
    return fail(b, TS_ERR_INVALID_ARG, "compact: null source array or keep mask");
  if ((fs_dst || fvel_dst) && !fire) return fail(b, TS_ERR_INVALID_ARG, "compact: FIRE state without parameters");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(b->cfg.device);
  // kept systems: atom counts from the source topology (host copy of offsets)
  std::vector<int64_t> map;
  int32_t nsys = 0;
  int64_t natoms = 0;
  if (src && src->n_systems > 0) {
    if (!b->topo_valid || src->n_systems != b->B || src->n_atoms != b->N) {
      ts_status r = derive_topology(b, src, st);
      if (r != TS_OK) return r;
    }
    for (int k = 0; k < src->n_systems; k++) {
      if (!keep[k]) continue;
      int64_t n = b->h_caller_off[k + 1] - b->h_caller_off[k];
      map.insert(map.end(), {b->h_caller_off[k], natoms, n, (int64_t)k, (int64_t)nsys});
      natoms += n;
      nsys++;
    }
  }
  int32_t n_new = add ? add->n_systems : 0;
  int64_t add_atoms = add ? add->n_atoms : 0;
  if (nsys + n_new > b->Bcap || natoms + add_atoms > b->cfg.atom_capacity)
    return fail(b, TS_ERR_BUDGET, "compact: batch capacity exceeded");
  if (nsys + n_new == 0) return fail(b, TS_ERR_INVALID_ARG, "compact: empty result");
  int64_t* dmap = nullptr;
  int64_t* dstarts = nullptr;
  // scratch for the maps: the batch's per-system FIRE coefficient area (32 doubles per system)
  size_t need = sizeof(int64_t) * (map.size() + n_new + 1);
  if (need > sizeof(double) * 32 * (size_t)b->Bcap) return fail(b, TS_ERR_BUDGET, "compact: map too large");
  dmap = (int64_t*)b->d_scal;
  dstarts = dmap + map.size();
  std::vector<int64_t> starts(n_new + 1, 0);
  for (int k = 0; k < n_new; k++) {
    if (add->n_per_system[k] < 1) return fail(b, TS_ERR_INVALID_ARG, "compact: empty admitted system");
    starts[k + 1] = starts[k] + add->n_per_system[k];
  }
  if (add && starts[n_new] != add_atoms) return fail(b, TS_ERR_INVALID_ARG, "compact: atom counts disagree");
  bool ok = true;
  if (!map.empty())
    ok = ok && cuda_ok(b, cudaMemcpyAsync(dmap, map.data(), 8 * map.size(), cudaMemcpyHostToDevice, st), "h2d");
  if (n_new) ok = ok && cuda_ok(b, cudaMemcpyAsync(dstarts, starts.data(), 8 * (n_new + 1), cudaMemcpyHostToDevice, st), "h2d");
  if (!ok) return TS_ERR_CUDA;
  if (nsys) {
    k_compact<<<nsys, 128, 0, st>>>(nsys, dmap, src->pos, src->vel, src->mass, src->cell, src->pbc, src->pot_idx,
                                    src->uid, dst->pos, dst->vel, const_cast<double*>(dst->mass), dst->cell,
                                    const_cast<uint8_t*>(dst->pbc),
                                    const_cast<int32_t*>(dst->system_idx), const_cast<int32_t*>(dst->pot_idx),
                                    const_cast<uint32_t*>(dst->uid), fs_src, fvel_src, fs_dst, fvel_dst);
    b->launches++;
  }
  if (n_new) {
    ok = cuda_ok(b, cudaMemcpyAsync(dst->pos + 3 * natoms, add->pos, 24 * add_atoms, cudaMemcpyHostToDevice, st), "h2d") &&
         cuda_ok(b, cudaMemcpyAsync(const_cast<double*>(dst->mass) + natoms, add->mass, 8 * add_atoms, cudaMemcpyHostToDevice, st), "h2d") &&
         cuda_ok(b, cudaMemcpyAsync(dst->cell + 9 * (int64_t)nsys, add->cell, 72 * (size_t)n_new, cudaMemcpyHostToDevice, st), "h2d") &&
         cuda_ok(b, cudaMemcpyAsync(const_cast<int32_t*>(dst->pot_idx) + nsys, add->pot_idx, 4 * (size_t)n_new, cudaMemcpyHostToDevice, st), "h2d");
    if (ok && dst->uid && add->uid)
      ok = cuda_ok(b, cudaMemcpyAsync(const_cast<uint32_t*>(dst->uid) + nsys, add->uid, 4 * (size_t)n_new, cudaMemcpyHostToDevice, st), "h2d");
    if (ok && dst->vel) ok = cuda_ok(b, cudaMemsetAsync(dst->vel + 3 * natoms, 0, 24 * add_atoms, st), "memset");
    if (!ok) return TS_ERR_CUDA;
    ts_fire_params fp{};
    if (fire) fp = *fire;
    k_admit_fill<<<n_new, 128, 0, st>>>(nsys, n_new, natoms, dstarts, const_cast<int32_t*>(dst->system_idx),
                                        const_cast<uint8_t*>(dst->pbc), dst->cell, fp, fs_dst, fvel_dst,
                                        fire != nullptr);
    b->launches++;
  }
  dst->n_systems = nsys + n_new;
  dst->n_atoms = natoms + add_atoms;
  // the maps live in batch scratch: finish before anything else reuses it
  if (!cuda_ok(b, cudaStreamSynchronize(st), "compact sync")) return TS_ERR_CUDA;
  b->topo_valid = false;
  return cuda_ok(b, cudaGetLastError(), "ts_batch_compact_admit") ? TS_OK : TS_ERR_CUDA;
}
