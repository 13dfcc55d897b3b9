// ts_kernels.cuh -- declarations of the device kernels of libts.so.
#pragma once
#include "ts_internal.cuh"

namespace ts {

// topology / import / export (ts_neighbor.cu)
__global__ void k_sys_bounds(int64_t N, const int32_t* sidx, int32_t B, int64_t* starts, int32_t* err);
__global__ void k_init_slots(int32_t B, SysArrays S, SlotArrays A);
template <bool F64>
__global__ void k_import_pos(int64_t Npad, SysArrays S, SlotArrays A, const double* pos, const DevPot* pots,
                             int check_skin, int32_t* err);
template <bool F64>
__global__ void k_import_vel(int64_t Npad, SlotArrays A, const double* vel, const double* mass);
template <bool F64>
__global__ void k_export_state(int64_t Npad, SlotArrays A, double* pos, double* vel);
template <bool F64>
__global__ void k_export_forces(int64_t Npad, SlotArrays A, double* F);
__global__ void k_geometry(int32_t B, SysArrays S, const double* cell, const uint8_t* pbc, const DevPot* pots,
                           int32_t* err);
__global__ void k_shift_table(int32_t B, SysArrays S);
__global__ void k_zero_bins(int32_t B, SysArrays S, int32_t* count);
template <bool F64>
__global__ void k_bin_atoms(int64_t Npad, SysArrays S, SlotArrays A, int32_t* count);
__global__ void k_scan_block(int64_t n, const int32_t* in, int32_t* out, int32_t* bsum);
__global__ void k_scan_sums(int32_t nb, int32_t* bsum);
__global__ void k_scan_add(int64_t n, int32_t* out, const int32_t* bsum);
__global__ void k_scatter_ids(int64_t Npad, SysArrays S, SlotArrays A, const int32_t* cstart);
template <bool F64>
__global__ void k_final_slot(int64_t Npad, SysArrays S, SlotArrays A, const int32_t* cstart, const int32_t* count,
                             int move_fire);
template <bool F64>
__global__ void k_copy_back(int64_t Npad, SysArrays S, SlotArrays A, int move_fire);
template <bool F64>
__global__ void k_build_list(int64_t Npad, SysArrays S, SlotArrays A, const int32_t* cstart, const int32_t* count,
                             const DevPot* pots, int32_t max_nbrs, int64_t stride, int32_t* err);
__global__ void k_after_relist(int32_t B, SysArrays S, int64_t* relist_counter);
__global__ void k_export_list(int64_t Npad, SysArrays S, SlotArrays A, int32_t max_nbrs, int64_t stride,
                              int32_t* j_out, int32_t* img_out, int32_t* count_out);

// pair forces (ts_pair.cu)
template <bool F64, bool EW>
__global__ void k_pair(int32_t n_warps, const int32_t* warp_sys, SysArrays S, SlotArrays A, const DevPot* pots,
                       int64_t stride, int only_dirty, double* partial);
__global__ void k_reduce_sys(int32_t B, SysArrays S, const double* partial, double* E, double* stress, double* KE,
                             double* Eint, double* Wint);
__global__ void k_clear_dirty(int32_t B, SysArrays S);
__global__ void k_count_pairs(int32_t n_warps, const int32_t* warp_sys, SysArrays S, SlotArrays A, const DevPot* pots,
                              int64_t stride, int f64, unsigned long long* out);

// MD (ts_md.cu)
template <bool F64, int KIND>
__global__ void k_md_kick_drift(int64_t Npad, SysArrays S, SlotArrays A, const DevPot* pots, double kick, double dt,
                                double c1, uint32_t seed, const uint64_t* step_base, uint64_t koff);
__global__ void k_set_u64(uint64_t* p, uint64_t v);
template <bool F64>
__global__ void k_md_final(int32_t n_warps, SysArrays S, SlotArrays A, double kick, double* partial);

}  // namespace ts
