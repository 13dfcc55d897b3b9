// ts_run.cu -- the persistent MD step loop behind ts_md_step.  The forces at
// the call's start and the K-step loop (kick/drift/noise + skin check,
// conditional per-system re-listing, pair forces; the chain or the piston
// between steps under NVT-NHC and NPT) are issued once into a CUDA graph per
// (K, parameters, stream) and replayed on later calls, so the host crosses to
// the device once per call instead of once per kernel.  Kernels read sizes and the Langevin
// step counter from device memory, so one graph serves every call with the
// same batch layout.
#include "ts_api.h"

namespace ts {

static void md_body(ts_batch* b, cudaStream_t st, const ts_md_params* p, int n_steps, double c1, bool need_e,
                    bool rec) {
  // forces current for every system (re-listing what the import flagged),
  // inside the step graph so that an unchanged state costs a few empty launches
  ensure_forces(b, st);
  // recorded frames (base address in b->d_rec): row k = positions after k steps
  auto record = [&](int64_t row) {
    const int64_t blk = (b->Npad + 255) / 256;
    const int gr = (int)(blk < 1 ? 1 : (blk > 148 * 16 ? 148 * 16 : blk));
    if (b->f64) k_export_frame<true><<<gr, 256, 0, st>>>(b->Npad, b->A, b->d_rec, row, b->N);
    else k_export_frame<false><<<gr, 256, 0, st>>>(b->Npad, b->A, b->d_rec, row, b->N);
    b->launches++;
  };
  if (rec) record(0);
  if (p->kind == TS_NPT_LANGEVIN) pair(b, st, true, kPairAll);   // the virial of every system for the first piston kick
  int g = 0;
  {
    int64_t blocks = (b->Npad + 255) / 256;
    g = (int)(blocks < 148 * 16 ? (blocks < 1 ? 1 : blocks) : 148 * 16);
  }
  const int wblocks = (int)(((int64_t)b->nwarps * 32 + 127) / 128);
  const int sblocks = (int)(((int64_t)b->B * 32 + 127) / 128);
  const bool nhc = p->kind == TS_NVT_NHC;
  const bool npt = p->kind == TS_NPT_LANGEVIN;
  const bool inner = !npt;      // NPT: full lists (the inner lists' refresh test has no cell term)
  double* vscale = b->d_scal;   // per-system velocity scale of the chain, or the NPT factors
  auto final_ke = [&](double kick, const double* scale, const double* nptf) {   // kick, scale, KE partials
    if (b->f64) k_md_final<true><<<wblocks, 128, 0, st>>>(b->nwarps, b->S, b->A, kick, b->d_partial, scale, nptf);
    else k_md_final<false><<<wblocks, 128, 0, st>>>(b->nwarps, b->S, b->A, kick, b->d_partial, scale, nptf);
    b->launches++;
  };
  auto chain = [&](int halves) {
    k_nhc_update<<<sblocks, 128, 0, st>>>(b->B, b->S, b->d_partial, p->dt, p->tau, halves, b->d_nhc, vscale);
    b->launches++;
  };
  auto piston = [&](int mode, int koff) {
    k_npt_sys<<<sblocks, 128, 0, st>>>(b->B, b->S, b->d_pots, b->d_partial, p->dt, c1, p->tau, p->p_ext, p->seed,
                                       b->d_step, (uint64_t)koff, mode, b->d_baro, b->d_scal, b->d_err);
    b->launches++;
  };
  if (nhc && n_steps > 0) {   // the opening chain half-step of the first step
    final_ke(0.0, nullptr, nullptr);
    chain(1);
  }
  if (npt && n_steps > 0) {   // the opening piston half kick and the first step's factors
    final_ke(0.0, nullptr, nullptr);
    piston(kNptOpen, 0);
  }
  for (int k = 0; k < n_steps; k++) {
    // BAOAB and NVE merge the closing half kick of a step with the opening
    // one of the next; the chain sits between them, so NHC kicks by dt/2
    double kick = (k == 0 || nhc) ? 0.5 * p->dt : p->dt;
    if (b->f64) {
      if (p->kind == TS_NVE)
        k_md_kick_drift<true, 0><<<g, 256, 0, st>>>(b->Npad, b->S, b->A, b->d_pots, kick, p->dt, c1, p->seed, b->d_step, k, nullptr);
      else if (p->kind == TS_LANGEVIN)
        k_md_kick_drift<true, 1><<<g, 256, 0, st>>>(b->Npad, b->S, b->A, b->d_pots, kick, p->dt, c1, p->seed, b->d_step, k, nullptr);
      else if (nhc)
        k_md_kick_drift<true, 2><<<g, 256, 0, st>>>(b->Npad, b->S, b->A, b->d_pots, kick, p->dt, c1, p->seed, b->d_step, k, vscale);
      else
        k_md_kick_drift<true, 3><<<g, 256, 0, st>>>(b->Npad, b->S, b->A, b->d_pots, kick, p->dt, c1, p->seed, b->d_step, k, vscale);
    } else {
      if (p->kind == TS_NVE)
        k_md_kick_drift<false, 0><<<g, 256, 0, st>>>(b->Npad, b->S, b->A, b->d_pots, kick, p->dt, c1, p->seed, b->d_step, k, nullptr);
      else if (p->kind == TS_LANGEVIN)
        k_md_kick_drift<false, 1><<<g, 256, 0, st>>>(b->Npad, b->S, b->A, b->d_pots, kick, p->dt, c1, p->seed, b->d_step, k, nullptr);
      else if (nhc)
        k_md_kick_drift<false, 2><<<g, 256, 0, st>>>(b->Npad, b->S, b->A, b->d_pots, kick, p->dt, c1, p->seed, b->d_step, k, vscale);
      else
        k_md_kick_drift<false, 3><<<g, 256, 0, st>>>(b->Npad, b->S, b->A, b->d_pots, kick, p->dt, c1, p->seed, b->d_step, k, vscale);
    }
    b->launches++;
    if (npt) {   // geometry and image shifts of the new cell (k_npt_sys scaled it)
      k_geometry<<<(b->B + 31) / 32, 32, 0, st>>>(b->B, b->S, b->S.h, nullptr, b->d_pots, b->d_err, 0, 1, 1);
      k_shift_table<<<b->B, 128, 0, st>>>(b->B, b->S);
      b->launches += 2;
    }
    bool ew = npt || (need_e && k == n_steps - 1);   // NPT: the virial drives the piston
    // forces from the inner lists; systems flagged for pruning or re-listed
    // in this pass refresh theirs in the same launch
    if (!relist_pair_overlapped(b, st, false, ew, inner)) {
      relist_lists(b, st, false);
      pair(b, st, ew, kPairAll, 0, inner);
      relist_finish(b, st, inner);
    }
    if (nhc) {   // closing half kick and the kinetic energy, then the chain (two half-steps between steps)
      final_ke(0.5 * p->dt, nullptr, nullptr);
      chain(k == n_steps - 1 ? 1 : 2);
    }
    if (npt) {   // closing atom kick and the kinetic energy, then the piston (closing + next opening)
      final_ke(0.0, nullptr, vscale);
      piston(kNptClose | (k < n_steps - 1 ? kNptOpen : 0), k + 1);
    }
    if (rec) record(k + 1);
  }
  if (nhc) final_ke(0.0, n_steps > 0 ? vscale : nullptr, nullptr);   // the last chain scaling, kinetic energy
  else if (!npt || n_steps == 0) final_ke(n_steps > 0 ? 0.5 * p->dt : 0.0, nullptr, nullptr);
  clear_dirty(b, st);
}

// Drop every cached graph once the layout they were captured for is gone.
void graph_cache_check(ts_batch* b) {
  if (!b->graphs_valid) {
    for (auto& g : b->graphs) if (g.exec) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
    b->graphs_valid = true;
  }
}

// Keep a graph entry (an instantiated graph, or the marker of a key seen
// once); the oldest of more than 16 is dropped.
bool graph_store(ts_batch* b, const ts_graph_entry& ge) {
  if (b->graphs.size() > 16) {
    if (b->graphs.front().exec) cudaGraphExecDestroy(b->graphs.front().exec);
    b->graphs.erase(b->graphs.begin());
  }
  b->graphs.push_back(ge);
  return true;
}

ts_status md_loop(ts_batch* b, cudaStream_t st, const ts_md_params* p, int n_steps, double c1, bool need_e,
                  double* rec) {
  k_set_u64<<<1, 1, 0, st>>>(b->d_step, p->step0);
  b->launches++;
  if (rec) {
    k_set_u64<<<1, 1, 0, st>>>(b->d_rec, (uint64_t)(uintptr_t)rec);
    b->launches++;
  }
  graph_cache_check(b);
  const void* rkey = rec ? b->d_rec : nullptr;   // recording graphs serve every frames address
  bool capturable = b->use_graphs && st != nullptr && n_steps > 0;
  if (capturable) {
    for (auto& g : b->graphs) {
      if (g.kind == 0 && g.n_steps == n_steps && g.md_kind == p->kind && g.need_e == need_e && g.dt == p->dt &&
          g.c1 == c1 && g.seed == p->seed && g.tau == p->tau && g.p_ext == p->p_ext && g.stream == st &&
          g.ptr[0] == rkey && g.exec) {
        if (!cuda_ok(b, cudaGraphLaunch(g.exec, st), "cudaGraphLaunch")) return TS_ERR_CUDA;
        b->launches += g.kernels;
        return TS_OK;
      }
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      int64_t l0 = b->launches;
      md_body(b, st, p, n_steps, c1, need_e, rec != nullptr);
      int64_t nk = b->launches - l0;
      b->launches = l0;
      cudaError_t e = cudaStreamEndCapture(st, &graph);
      cudaGraphExec_t exec = nullptr;
      if (e == cudaSuccess && cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority) == cudaSuccess) {
        cudaGraphDestroy(graph);
        ts_graph_entry ge;
        ge.kind = 0; ge.n_steps = n_steps; ge.md_kind = p->kind; ge.need_e = need_e; ge.dt = p->dt; ge.c1 = c1;
        ge.seed = p->seed; ge.tau = p->tau; ge.p_ext = p->p_ext; ge.stream = st; ge.exec = exec; ge.kernels = nk;
        ge.ptr[0] = rkey;
        graph_store(b, ge);
        if (!cuda_ok(b, cudaGraphLaunch(exec, st), "cudaGraphLaunch")) return TS_ERR_CUDA;
        b->launches += nk;
        return TS_OK;
      }
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
    } else {
      cudaGetLastError();
    }
  }
  md_body(b, st, p, n_steps, c1, need_e, rec != nullptr);
  return cuda_ok(b, cudaGetLastError(), "md loop") ? TS_OK : TS_ERR_CUDA;
}

}  // namespace ts
