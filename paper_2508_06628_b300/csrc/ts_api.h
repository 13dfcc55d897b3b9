// ts_api.h -- the batch object shared by the host-side translation units.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "ts_kernels.cuh"

struct ts_graph_entry {
  int kind = -1;            // 0 = MD loop, 1 = adjoint segment
  int n_steps = 0;
  const void* ptr[8] = {};  // further key: the caller's pointers the graph's nodes hold
  int64_t ival[2] = {};     //   ... and integer / real arguments
  double dval[2] = {};
  int md_kind = 0;
  bool need_e = false;
  double dt = 0, c1 = 0;
  uint32_t seed = 0;
  double tau = 0, p_ext = 0;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;      // kernel nodes in the graph
};

struct ts_batch {
  ts_batch_config cfg{};
  std::string cache_path;
  bool f64 = false;
  int n_pots = 0;
  ts_potential pots[ts::kMaxPots];
  double rc[ts::kMaxPots];
  std::vector<ts::DevPot> dp_host;
  int32_t max_nbrs = 128;
  int64_t Ncap = 0, Wcap = 0, Ccap = 0;
  int32_t Bcap = 0;
  // topology
  bool topo_valid = false, first_import = true;
  int32_t B = 0, nwarps = 0, n_large = 0, n_items = 0, nst_max = 0;
  bool use_small_pair = true;
  int4* d_items = nullptr;        // work items of k_pair_small
  int32_t* d_item_sys = nullptr;  // system of each warp of each work item [Wcap][kItemWarps]
  int32_t* d_tab_sys = nullptr;   // list-build work table (k_relist_small writes it)
  int32_t* d_tab_base = nullptr;
  int32_t* d_tab_base_a = nullptr;
  int32_t* d_tab_n = nullptr;
  int n_sm = 148;
  int64_t N = 0, Npad = 0, nbins = 0;
  std::vector<int64_t> h_caller_off, h_seg;
  std::vector<int32_t> h_n, h_pot;
  // device
  ts::SysArrays S{};
  ts::SlotArrays A{};
  ts::DevPot* d_pots = nullptr;
  int32_t* d_err = nullptr;
  int64_t* d_counters = nullptr;
  uint64_t* d_step = nullptr;
  uint64_t* d_rec = nullptr;      // base address of the frames ts_md_record writes (read by the step graph)
  double* d_partial = nullptr;
  int32_t* d_warp_sys = nullptr;
  int32_t* d_count = nullptr;
  int32_t* d_cstart = nullptr;
  int32_t* d_bsum = nullptr;
  int64_t* d_starts = nullptr;
  double* d_Eint = nullptr;
  double* d_Wint = nullptr;
  double* d_scal = nullptr;         // per-system FIRE / scratch scalars [32 B]
  float* d_fcoef = nullptr;         // FP32 copy of the per-system FIRE step coefficients [32 B]
  double* d_nhc = nullptr;          // Nose-Hoover chain state during a call [6 per system]
  double* d_baro = nullptr;         // NPT piston velocities during a call [1 per system]
  double* d_gparam_part = nullptr;  // per-warp parameter-gradient partials [4 Wcap]
  double* d_gacc = nullptr;
  std::vector<void*> allocations;
  size_t bytes_allocated = 0;
  cudaEvent_t ev = nullptr;
  // second stream (highest priority) and fork/join events: a re-listing pass
  // runs beside the pair forces of the systems that keep their lists
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_pruned = nullptr;   // after the MD step's re-filtering pair launch
  bool overlap_relist = true;
  bool bwd_small = true;          // pair backward of small systems from shared memory (mixed precision)
  int prio_hi = 0;                // numerically greatest-priority value of the device
  // launch shapes and list parameters (autotuned, ts_tune.cu)
  int pair_threads = 128;
  ts_tuning tune = {8, 0.3, 0.5, 1.0, 1.0};
  bool use_graphs = true;
  std::vector<ts_graph_entry> graphs;
  bool graphs_valid = false;
  // bookkeeping
  int64_t launches = 0;
  ts_status sticky = TS_OK;
  std::string last_error;
};

namespace ts {
bool cuda_ok(ts_batch* b, cudaError_t e, const char* what);
ts_status fail(ts_batch* b, ts_status st, const std::string& msg);
size_t scratch_bytes(int64_t Ncap, int64_t Bcap, int64_t Ccap, int32_t max_nbrs, bool f64);
ts_status derive_topology(ts_batch* b, const ts_state* s, cudaStream_t st);
ts_status check_state(ts_batch* b, const ts_state* s, bool need_vel);
ts_status prologue(ts_batch* b, ts_state* s, cudaStream_t st, bool import_vel, bool fire = false,
                   bool geometry = true);
// Kernel launch with a scheduling priority (0: the stream's own).  Stream
// capture keeps the launch attribute as the kernel node's priority.
template <typename... KArgs, typename... Args>
inline void launch_k(cudaStream_t st, int prio, dim3 grid, dim3 block, size_t shm, void (*kern)(KArgs...),
                     Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = shm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = prio;
  cfg.attrs = at;
  cfg.numAttrs = prio != 0 ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, args...);
}
// a launch with programmatic stream serialization: it may start once every
// CTA of the preceding kernel on the stream has issued
// griddepcontrol.launch_dependents (it must not read that kernel's results)
template <typename... KArgs, typename... Args>
inline void launch_k_overlap(cudaStream_t st, dim3 grid, dim3 block, size_t shm, void (*kern)(KArgs...),
                             Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = shm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
}
void relist(ts_batch* b, cudaStream_t st, bool move_fire);
void relist_lists(ts_batch* b, cudaStream_t st, bool move_fire, int prio = 0);
void relist_sort(ts_batch* b, cudaStream_t st, bool move_fire, int prio);
void relist_build(ts_batch* b, cudaStream_t st, int prio);
void relist_finish(ts_batch* b, cudaStream_t st, bool md_pass, bool overlap = false);
bool relist_pair_overlapped(ts_batch* b, cudaStream_t st, bool move_fire, bool ew, bool inner);
void relist_large_sort(ts_batch* b, cudaStream_t st, bool move_fire);
void pair(ts_batch* b, cudaStream_t st, bool ew, int filter, int prio = 0, bool inner = false, bool overlap = false);
void reduce_sys(ts_batch* b, cudaStream_t st, double* E, double* stress, double* KE);
void clear_dirty(ts_batch* b, cudaStream_t st);
void export_state(ts_batch* b, cudaStream_t st, double* pos, double* vel);
void export_forces(ts_batch* b, cudaStream_t st, double* F);
void ensure_forces(ts_batch* b, cudaStream_t st);
ts_status md_loop(ts_batch* b, cudaStream_t st, const ts_md_params* p, int n_steps, double c1, bool need_e,
                  double* rec = nullptr);
void graph_cache_check(ts_batch* b);
bool bwd_attributes(ts_batch* b);
bool graph_store(ts_batch* b, const ts_graph_entry& ge);
void autotune_load(ts_batch* b);
void fill_devpots(ts_batch* b, DevPot* dp);
bool tuning_valid(const ts_tuning& t);
}  // namespace ts
