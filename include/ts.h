/*
 * ts.h -- C ABI of libts.so, a batched pair-potential MD / FIRE / adjoint
 * engine for NVIDIA B300 (sm_103a).
 *
 * The data model is TorchSim's SimState (arXiv 2508.06628, Sec. 3): many
 * periodic systems of uneven size evolve together; atom-wise arrays
 * (positions, velocities, masses) are concatenated over systems and
 * system-wise arrays (cells, stress) are stacked; a non-decreasing per-atom
 * system index ties atoms to systems.  The model output schema is energies,
 * forces and stress (Sec. 2).  The paper names Lennard-Jones, Morse and
 * soft-sphere potentials, MD integrators (Langevin MD, Sec. 4), structural
 * relaxation optimisers (Sec. 1), memory-aware batching with in-flight
 * admission (Sec. 3, Figs. 2-3) and differentiable trajectories (Sec. 2).
 *
 * Conventions (every entry point):
 *  - Units: Angstrom, eV, amu.  Time unit t0 = sqrt(amu A^2/eV) = 10.1805 fs;
 *    callers convert dt.  Temperatures are passed as kT in eV.
 *  - Cells are row-major [3][3] with rows = lattice vectors (x = s h for a
 *    fractional row vector s).  pbc[a] = 0 makes axis a non-periodic: no
 *    images and no wrapping along it (atoms may lie outside the cell, which
 *    then only sets the binning).  Variable-cell FIRE needs pbc = {1,1,1}
 *    (other systems report TS_ERR_UNSUPPORTED at poll).
 *  - Every array pointer in ts_state and every output pointer is DEVICE
 *    memory owned by the caller, unless the comment says "host".  The library
 *    never frees caller memory; it owns only its scratch, sized at
 *    ts_batch_create.
 *  - Calls are asynchronous and ordered on the given stream (a cudaStream_t
 *    passed as void*, NULL = legacy default stream).  Argument errors are
 *    returned immediately; device-side errors (neighbour overflow, invalid
 *    system_idx, non-finite values, timeouts) set a sticky per-batch error
 *    word that ts_batch_poll returns.  No exception crosses
 *    the ABI.  One host thread per batch.
 *  - Positions are wrapped into the cell whenever a system's neighbour list
 *    is rebuilt, so returned positions may differ from the inputs by lattice
 *    vectors.
 */
#ifndef TS_H_
#define TS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TS_OK = 0,
  TS_ERR_INVALID_ARG = 1,        /* bad pointer, size or ordering                 */
  TS_ERR_UNSUPPORTED = 2,        /* non-periodic axis, cell too small/large       */
  TS_ERR_BUDGET = 3,             /* capacity or memory budget exceeded            */
  TS_ERR_CUDA = 4,               /* a CUDA runtime call failed (ts_last_error)   */
  TS_ERR_NEIGHBOR_OVERFLOW = 5,  /* an atom has more neighbours than max_neighbors */
  TS_ERR_TIMEOUT = 6,            /* a bounded wait ran out                        */
  TS_ERR_NONFINITE = 7,          /* NaN/Inf met in positions or forces            */
  TS_ERR_NOT_READY = 8           /* poll: work still in flight                    */
} ts_status;

typedef enum { TS_LJ = 0, TS_MORSE = 1, TS_SOFT_SPHERE = 2 } ts_pot_kind;

/* A pair potential (the paper lists LJ, Morse and soft sphere, Sec. 1; the
 * forms are the textbook ones):
 *   LJ          p = {sigma, eps, -}:   phi = 4 eps [(sigma/r)^12 - (sigma/r)^6]
 *   Morse       p = {D, alpha, r0}:    phi = D [e^{-2 alpha (r-r0)} - 2 e^{-alpha (r-r0)}]
 *   soft sphere p = {sigma, eps, alpha}: phi = (eps/alpha)(1 - r/sigma)^alpha, r < sigma
 * cutoff: pair cutoff rc (soft sphere: ignored, rc = sigma).
 * shift: 1 subtracts phi(rc) from every pair energy (forces unchanged).
 * skin: Verlet skin of this potential's neighbour lists (list radius
 * rc + skin; a system is re-listed when one of its atoms moved more than
 * skin/2 since its last build). */
typedef struct {
  int32_t kind;
  int32_t shift;
  double p[3];
  double cutoff;
  double skin;
} ts_potential;

typedef enum { TS_MIXED = 0, TS_FP64 = 1 } ts_precision;

/* Batch configuration.
 * atom_capacity / system_capacity: the largest total atom count and system
 *   count any state passed to this batch may have (in-flight admission
 *   included).  All scratch is allocated at create for these capacities.
 * max_neighbors: per-atom neighbour-list capacity; 0 picks 160
 *   (an atom beyond it sets TS_ERR_NEIGHBOR_OVERFLOW).
 * memory_budget_bytes: 0 = no limit; otherwise create fails with
 *   TS_ERR_BUDGET if the scratch would exceed it, and in-flight admission
 *   admits systems only while their memory scaler fits (Sec. 3).
 * precision: TS_MIXED = FP32 pair arithmetic, FP64 per-system energy/virial
 *   accumulation, compensated (double-float) positions and velocities;
 *   TS_FP64 = FP64 everywhere.
 * device: CUDA device ordinal the batch lives on.
 * autotune_cache: host path of a text file caching tuned launch parameters,
 *   or NULL. */
typedef struct {
  int64_t atom_capacity;
  int32_t system_capacity;
  int32_t max_neighbors;
  size_t memory_budget_bytes;
  int32_t precision;
  int32_t device;
  const char* autotune_cache;
} ts_batch_config;

/* A batched state (SimState, Sec. 3).  All pointers are caller-owned DEVICE
 * memory; sizes in elements:
 *   pos [n_atoms][3] f64 (read/write), vel [n_atoms][3] f64 (A/t0, read/write;
 *   may be NULL for calls that do not integrate), mass [n_atoms] f64 (amu),
 *   cell [n_systems][3][3] f64 (read/write: FIRE moves it), pbc [n_systems][3] u8,
 *   system_idx [n_atoms] i32 (non-decreasing, every system non-empty),
 *   pot_idx [n_systems] i32 (index into the batch's potentials),
 *   uid [n_systems] u32 stable system ids keying the Langevin noise (NULL =
 *   the system's index).
 * system_idx, pot_idx and uid set the batch topology (the engine's slot
 * layout and noise keys), read when it is derived: on a batch's first call,
 * when n_systems or n_atoms differ from the last call's, and on
 * ts_neighbor_build with force_rebuild != 0.  A caller that changes one of
 * them with the same counts calls ts_neighbor_build(force_rebuild = 1) first.  pos, vel, mass,
 * cell and pbc may change freely between calls (changed cells and
 * periodicity re-list their systems). */
typedef struct {
  int32_t n_systems;
  int64_t n_atoms;
  double* pos;
  double* vel;
  const double* mass;
  double* cell;
  const uint8_t* pbc;
  const int32_t* system_idx;
  const int32_t* pot_idx;
  const uint32_t* uid;
} ts_state;

typedef struct ts_batch ts_batch;

/* Create a batch: allocate all scratch on cfg->device for the capacities.
 * pots: host array of n_pots (1..16) potentials, copied.
 * Returns TS_ERR_INVALID_ARG, TS_ERR_BUDGET or TS_ERR_CUDA on failure
 * (*out = NULL). */
ts_status ts_batch_create(const ts_batch_config* cfg, const ts_potential* pots, int n_pots, ts_batch** out);

/* Replace the potentials' parameters p[3] in place (kinds, cutoffs, shifts
 * and skins must stay as created: TS_ERR_INVALID_ARG otherwise).  Used to
 * evaluate a loss at new parameters, e.g. in a fitting loop (Sec. 2).
 * Host array of n_pots entries; synchronous. */
ts_status ts_batch_set_potentials(ts_batch* b, const ts_potential* pots, int n_pots);

/* Free all scratch of the batch (synchronises the device first).  The paper
 * has no counterpart (its batches are PyTorch tensors freed by the garbage
 * collector); the library never frees caller memory. */
ts_status ts_batch_destroy(ts_batch* b);

/* Neighbour build (per-system triclinic cell list with multi-image stencil,
 * then an explicit Verlet list at rc + skin).  Derives the batch topology
 * from system_idx when force_rebuild != 0 or on the first call (one
 * device->host copy of the per-system offsets and a stream synchronisation);
 * otherwise re-lists only systems whose atoms moved more than skin/2.
 * Wraps positions into the cell (in place) for re-listed systems.
 * The paper attributes the remaining cost differences between models to
 * graph construction (Sec. 4). */
ts_status ts_neighbor_build(ts_batch* b, ts_state* s, int force_rebuild, void* stream);

/* Copy the current neighbour lists out, in caller order (for checks and
 * analysis; the neighbour graph whose construction Sec. 4 names as the
 * cost that separates models): j_out [n_atoms][max_neighbors] i32 caller index of each
 * neighbour, img_out [n_atoms][max_neighbors][3] i32 lattice image n of the
 * pair (x_j + n h - x_i, relative to the positions returned by the last
 * call), count_out [n_atoms] i32.  Unused entries are -1 / 0.  All device.
 * ts_batch_max_neighbors gives the row length. */
ts_status ts_neighbor_export(ts_batch* b, int32_t* j_out, int32_t* img_out, int32_t* count_out, void* stream);
int32_t ts_batch_max_neighbors(const ts_batch* b);

/* Energies, forces and stress (Sec. 2 output schema) at the current
 * positions, using the current lists (re-listing systems past their skin).
 * F [n_atoms][3] f64, E [n_systems] f64, stress [n_systems][3][3] f64
 * (sigma = (1/V) dE/d strain; negative under compression); any may be NULL.
 * E and stress are summed per system in FP64, deterministically. */
ts_status ts_pair_forces(ts_batch* b, ts_state* s, double* F, double* E, double* stress, void* stream);

typedef enum { TS_NVE = 0, TS_LANGEVIN = 1, TS_NVT_NHC = 2, TS_NPT_LANGEVIN = 3 } ts_md_kind;

/* MD parameters (Sec. 1 lists NVE, NVT and Langevin integrators).
 * NVE: velocity Verlet.  LANGEVIN: BAOAB with friction gamma (1/t0) and
 * per-system kT (device array [n_systems], eV); the noise is Philox4x32-10
 * keyed by (seed, uid) with counter (step, atom index within its system), so
 * it is independent of batch layout.  step0 is the counter of the first step
 * of this call.  NVT_NHC: Nose-Hoover chain of three per system (Martyna,
 * Klein and Tuckerman 1992; time-reversible factorisation C(dt/2) B A B
 * C(dt/2) of Martyna, Tuckerman, Tobias and Klein 1996), thermostat time
 * constant tau (t0), masses Q1 = Nf kT tau^2 and Qk = kT tau^2 with
 * Nf = 3n - 3; nhc is the chain state, device [n_systems][6] f64 (xi_1..3,
 * then the thermostat velocities w_1..3; zeros to start), read and written.
 * The extended energy K + U + sum Q_k w_k^2/2 + Nf kT xi_1 + kT (xi_2 + xi_3)
 * is conserved.
 * NPT_LANGEVIN (Sec. 1 lists NPT): isotropic barostat of Martyna, Tobias and
 * Klein (1994) with Langevin friction gamma and noise on the atoms and on the
 * piston.  Per system the cell scales as dh/dt = v_e h; piston mass
 * W = (Nf + 3) kT tau^2 with Nf = 3n and barostat time tau (t0); external
 * pressure p_ext (eV/A^3); the atoms couple through a = 1 + 3/Nf:
 *   dx/dt = v + v_e x, dv/dt = F/m - a v_e v,
 *   W dv_e/dt = a 2K + Xi - 3 V p_ext   (Xi = -sum over pairs phi'(r) r).
 * One step: piston half kick, atom half kick, half drift, O step of atoms
 * and piston (the piston's normal is the first of the atom-index counter
 * 0xffffffff), half drift, forces, atom half kick, piston half kick; every
 * sub-flow is solved exactly.  baro: device [n_systems] f64, the piston
 * velocities v_e (zeros to start), read and written; s->cell is updated in
 * place.  Every system must be periodic along all three axes
 * (TS_ERR_UNSUPPORTED otherwise).  Without friction K + U + W v_e^2/2 +
 * p_ext V is conserved.  MD steps of this kind compute forces from the full
 * neighbour lists (no inner lists) and re-list a system when its atoms'
 * displacement plus the image shifts' movement under the cell change could
 * reach the skin. */
typedef struct {
  int32_t kind;
  double dt;
  double gamma;
  const double* kT;
  uint32_t seed;
  uint64_t step0;
  double tau;      /* NVT_NHC: thermostat time; NPT_LANGEVIN: barostat time */
  double* nhc;     /* NVT_NHC only */
  double p_ext;    /* NPT_LANGEVIN only */
  double* baro;    /* NPT_LANGEVIN only */
} ts_md_params;

/* Run n_steps MD steps on the whole batch (Sec. 4 runs Langevin MD).  The
 * per-step loop (kick/drift/noise, skin check, conditional per-system
 * re-listing, pair forces) runs on the device without host round trips.
 * E, KE [n_systems] f64 (may be NULL): potential and kinetic energy after
 * the last step.  pos and vel are updated in place. */
ts_status ts_md_step(ts_batch* b, ts_state* s, const ts_md_params* p, int n_steps, double* E, double* KE,
                     void* stream);

/* ts_md_step that also records the trajectory's positions, for the adjoint's
 * recomputed segments (Sec. 2: differentiable simulation; the reverse needs
 * every frame of a checkpointed segment).  frames [n_steps+1][n_atoms][3]
 * f64 (device, caller order; caller-owned): row 0 receives the positions at
 * the start of the call (as the library holds them: each atom in the lattice
 * image nearest its listing reference, so a row may differ from s->pos by
 * lattice vectors), row k those after k steps.  The last row equals s->pos on
 * return.  Row k equals the positions after a ts_md_step call of k steps from
 * the same state and lists.  Kinds TS_NVE, TS_LANGEVIN and TS_NVT_NHC;
 * TS_ERR_INVALID_ARG for TS_NPT_LANGEVIN (the cell changes every step and is
 * not recorded), a NULL frames pointer or n_steps < 1; otherwise errors as
 * ts_md_step.  On a stream other than the legacy default stream the loop is a
 * CUDA graph cached per (n_steps, parameters, stream) as in ts_md_step; the
 * frames address is read on the device, so one graph serves every buffer. */
ts_status ts_md_record(ts_batch* b, ts_state* s, const ts_md_params* p, int n_steps, double* frames,
                       void* stream);

/* FIRE parameters (Bitzek et al. 2006), with the stopping test of the
 * relaxation: max_i |F_i| <= fmax and (variable cell) max_ab |sigma_ab| <= smax. */
typedef struct {
  double dt0, dt_max, finc, fdec, alpha0, falpha, maxstep, fmax, smax, p_ext;
  int32_t nmin;
  int32_t variable_cell;
} ts_fire_params;

/* Per-system FIRE state, caller-owned DEVICE memory, one per system:
 * fs [n_systems] (zero-filled plus dt = dt0, alpha = alpha0, Fd = identity,
 * h0 = the starting cell is the fresh state; ts_fire_init writes it),
 * fvel [n_atoms + 3 n_systems][3] f64 generalised velocities (the 3 cell rows
 * of system k follow its atoms, at row offset(k) + 3k). */
typedef struct {
  double dt, alpha;
  int32_t npos, started, converged, nsteps;
  double Fd[9];
  double h0[9];
} ts_fire_state;

/* Write the fresh FIRE state for every system (fvel zeroed). */
ts_status ts_fire_init(ts_batch* b, ts_state* s, const ts_fire_params* p, ts_fire_state* fs, double* fvel,
                       void* stream);

/* Run n_steps variable-cell FIRE steps (the paper's structural relaxation,
 * run under in-flight batching, Sec. 3).  Converged systems are frozen;
 * converged [n_systems] u8 (device, may be NULL) receives the flags, and
 * E / fmax / smax [n_systems] f64 (device, may be NULL) the values at the
 * final configuration. */
ts_status ts_fire_step(ts_batch* b, ts_state* s, ts_fire_state* fs, double* fvel, const ts_fire_params* p,
                       int n_steps, uint8_t* converged, double* E, double* fmax, double* smax, void* stream);

/* Adjoint of ts_pair_forces (Sec. 2: gradients of trajectory observables with
 * respect to model parameters).  Inputs: gF [n_atoms][3] = dL/dF, gE
 * [n_systems] = dL/dE (may be NULL), gStress [n_systems][3][3] = dL/dstress
 * (may be NULL).  Outputs: gPos [n_atoms][3] = dL/dpos through F, E and
 * stress; gParams [n_pots][3] = dL/dp of each potential's parameters
 * (cutoffs held fixed).  accumulate != 0 adds into gPos and gParams instead of
 * overwriting them.  Uses the current neighbour lists (positions must be
 * within the skin of the last build; the call re-lists otherwise). */
ts_status ts_pair_forces_backward(ts_batch* b, ts_state* s, const double* gF, const double* gE,
                                  const double* gStress, double* gPos, double* gParams, int accumulate,
                                  void* stream);

/* Gaussian-smeared radial distribution function of each system (the
 * trajectory observable of Sec. 2): K bins on [0, rmax), centres
 * r_k = (k + 1/2) D, D = rmax / K, width D;
 * g_k = V/(N(N-1)) sum over ordered neighbour pairs with r < rmax + 4D of
 * exp(-(r - r_k)^2 / 2D^2) / (sqrt(2 pi) D 4 pi r_k^2).
 * g [n_systems][K] f64.  Needs rc + skin >= rmax + 4D for every potential.
 * TS_ERR_INVALID_ARG for K outside [1, 4096] or above what four warps' rows
 * of shared memory hold (48 KB): K <= 3072 in mixed precision, K <= 1536 in
 * FP64 (forward), K <= 3072 for the mixed-precision backward. */
ts_status ts_rdf(ts_batch* b, ts_state* s, double rmax, int K, double* g, void* stream);

/* gPos [n_atoms][3] += d(sum_{s,k} gg[s][k] g[s][k]) / d pos. */
ts_status ts_rdf_backward(ts_batch* b, ts_state* s, double rmax, int K, const double* gg, double* gPos,
                          void* stream);

/* One reverse step of velocity Verlet (the discrete adjoint used to
 * differentiate an NVE trajectory, Sec. 2).  Forward step from (x_t, v_t):
 * vh = v_t + c F(x_t), x_{t+1} = x_t + dt vh, v_{t+1} = vh + c F(x_{t+1}),
 * c = dt / (2 m).  Given s->pos = x_t, x_next = x_{t+1} [n_atoms][3] (device)
 * and the adjoints ax = dL/dx_{t+1}, av = dL/dv_{t+1} (device, in/out), this
 * overwrites them with dL/dx_t, dL/dv_t and adds c J_theta^T terms into
 * gParams [n_pots][3]. */
ts_status ts_vv_adjoint_step(ts_batch* b, ts_state* s, const double* x_next, double dt, double* ax, double* av,
                             double* gParams, void* stream);

/* The reverse of n NVE steps over stored frames: the result of n calls of
 * ts_vv_adjoint_step (up to rounding), issued from the library with the half
 * kicks of adjacent reverse steps merged as the forward loop merges them:
 * the two products (dt/2) J(x_m)^T av that the reverse steps out of and into
 * an interior frame m take with the same av become one product with weight
 * dt, so each frame costs one pair backward pass instead of two.
 * frames [n+1][n_atoms][3] f64 (device, caller order) hold x_{t0}, ...,
 * x_{t0+n}; ax, av (device, in/out) hold dL/dx, dL/dv at t0+n on entry and at
 * t0 on return; gParams [n_pots][3] (device) accumulates.  With rdf_every > 0,
 * at every frame t0+m (m = n ... 1) with (t0+m) % rdf_every == 0 the gradient
 * of sum_{s,k} gg[s][k] g_k(x_{t0+m}) (ts_rdf_backward with rmax, K; gg
 * [n_systems][K] f64, device) is added to ax before that frame's product.
 * s supplies masses, cells, pbc and the topology; s->pos and s->vel are not
 * read.  On a stream other than the legacy default stream, once the batch's
 * layout is settled, a call whose arguments (n, frames, ax, av, gParams, gg,
 * cell and pbc pointers, dt, rdf_every, t0 mod rdf_every, rmax, K, stream)
 * repeat those of an earlier call is captured as a CUDA graph and replayed by
 * later such calls; a first call is issued directly (a one-off sweep over a
 * long stored trajectory is queued far ahead of the device anyway).  Errors
 * as ts_vv_adjoint_step and ts_rdf_backward; n >= 1. */
ts_status ts_vv_adjoint_segment(ts_batch* b, ts_state* s, const double* frames, int n, int64_t t0, double dt,
                                double* ax, double* av, double* gParams, int rdf_every, double rmax, int K,
                                const double* gg, void* stream);

/* ---- in-flight batching runtime (Sec. 3, Figs. 2-3) ---------------------- */

/* Memory scaler of one system: n_atoms (model memory fixed per atom) or
 * n_atoms * number density (radial-cutoff models), Sec. 3. */
typedef enum { TS_SCALE_N_ATOMS = 0, TS_SCALE_N_ATOMS_X_DENSITY = 1 } ts_memory_scaling;

/* Memory probe of Fig. 2 (host only): for each probe system k (its memory
 * scaler scaler[k]), grow a batch of copies of it one system at a time
 * until fits(total_scaler, n_systems, ctx) returns 0 (the out-of-memory
 * signal), and take max_scaler = min_k (n_fit_k * scaler[k]).
 * n_fit_out [n] (host, may be NULL) receives the counts.  Returns
 * TS_ERR_BUDGET if some probe system does not fit even once.
 * max_systems bounds each probe. */
ts_status ts_estimate_max_scaler(const double* scaler, int n, int (*fits)(double, int, void*), void* ctx,
                                 int max_systems, int* n_fit_out, double* max_scaler_out);

/* Bytes of batch scratch per atom and per system for this configuration
 * (the analytic memory model the admission budget uses). */
ts_status ts_batch_memory_model(const ts_batch* b, double* bytes_per_atom, double* bytes_per_system);

/* In-flight scheduler (host only, no device memory): a queue of pending
 * systems (by scaler) and a set of active slots under max_scaler and
 * max_active.  ts_sched_fill pops pending systems in order while their
 * scaler fits (Sec. 3: "samples systems from the stream until memory is
 * full"); ts_sched_retire frees slots.  ids are caller-chosen. */
typedef struct ts_sched ts_sched;
ts_status ts_sched_create(double max_scaler, int32_t max_active, ts_sched** out);
ts_status ts_sched_destroy(ts_sched* q);
ts_status ts_sched_push(ts_sched* q, int64_t id, double scaler);
/* Admit pending systems; writes up to cap admitted ids to ids_out (host) and
 * their count to n_out. */
ts_status ts_sched_fill(ts_sched* q, int64_t* ids_out, int cap, int* n_out);
ts_status ts_sched_retire(ts_sched* q, const int64_t* ids, int n);
ts_status ts_sched_stats(const ts_sched* q, int32_t* n_active, int64_t* n_pending, double* active_scaler);

/* BinningAutobatcher (Sec. 3, Fig. 3, fixed-length runs): pack n systems of
 * memory footprint sizes[k] (host, in the units of the maximum memory, e.g.
 * atoms) into as few bins of `capacity` as the first-fit-decreasing
 * heuristic finds (systems by decreasing size, ties by index; each into the
 * first bin with room).  Writes bin_out[k] (host, [n]) and the bin count.
 * A size above capacity returns TS_ERR_BUDGET; a size <= 0 or a bad argument
 * TS_ERR_INVALID_ARG.  Pure host code. */
ts_status ts_bin_pack(const double* sizes, int n, double capacity, int32_t* bin_out, int32_t* n_bins_out);

/* Compact a batched device state: keep the systems whose keep[k] != 0
 * (host mask [n_systems]) and append n_new staged systems from host arrays
 * (pinned or pageable), writing the new state into dst (device arrays sized
 * for the batch capacity).  Used by the in-flight loop to retire converged
 * systems and admit new ones between FIRE calls; topology is re-derived on
 * the next call (force rebuild).  The FIRE state arrays (fs, fvel) follow
 * the same compaction when not NULL. */
typedef struct {
  int32_t n_systems;
  int64_t n_atoms;
  const double* pos;        /* host [n_atoms][3] */
  const double* mass;       /* host [n_atoms]    */
  const double* cell;       /* host [n_systems][9] */
  const int32_t* n_per_system; /* host [n_systems] */
  const int32_t* pot_idx;   /* host [n_systems] */
  const uint32_t* uid;      /* host [n_systems] */
} ts_host_systems;

ts_status ts_batch_compact_admit(ts_batch* b, const ts_state* src, const uint8_t* keep, const ts_host_systems* add,
                                 ts_state* dst, const ts_fire_state* fs_src, const double* fvel_src,
                                 ts_fire_state* fs_dst, double* fvel_dst, const ts_fire_params* fire,
                                 void* stream);

/* Block until all work queued on the stream is done, or timeout_ms passes
 * (TS_ERR_NOT_READY; nothing is lost, poll again).  Returns the sticky
 * device error word, then clears it.  The paper has no counterpart: PyTorch
 * raises errors synchronously, whereas this library runs asynchronously on
 * streams and reports device-side errors (neighbour overflow, invalid
 * system_idx, non-finite input) here.  No kernel of this library waits on a
 * flag, so TS_ERR_TIMEOUT is never raised by the current kernels. */
ts_status ts_batch_poll(ts_batch* b, void* stream, int timeout_ms);

/* Launch and list parameters of the hot path (the paper has no counterpart:
 * they shape how this engine maps the batched method onto the GPU and do
 * not change what it computes beyond rounding order):
 *   item_warps      warps (of 32 atoms) per CTA work item of the
 *                   shared-memory pair kernel: 4 or 8 (the tile size);
 *   inner_fraction  inner (pruned) list radius rc + inner_fraction * skin,
 *                   (0, 1] (1 = no pruning);
 *   relist_soon     re-list hysteresis: once any system re-lists, systems
 *                   whose atoms moved more than relist_soon * skin/2 re-list
 *                   in the same pass, (0, 1] (1 = off);
 *   bin_factor      cell-list bin edge = bin_factor * (rc + skin): 1 or 0.5
 *                   (the stencil then reaches two bins);
 *   skin_scale      every potential's skin is used times skin_scale, (0, 1]
 *                   (shorter Verlet lists and more frequent re-listing; the
 *                   lists never outgrow the capacity sized for the skins
 *                   given at create; ts_rdf refuses an rmax + 4D beyond
 *                   rc + skin * skin_scale). */
typedef struct {
  int32_t item_warps;
  double inner_fraction;
  double relist_soon;
  double bin_factor;
  double skin_scale;
} ts_tuning;

/* Autotuner (the paper has no counterpart).  Times the MD step of p (n_steps
 * per timed call, CUDA events around CUDA-graph replays on `stream`) for
 * candidate values of each ts_tuning field in turn -- bin_factor {1, 0.5},
 * item_warps {8, 4}, skin_scale {1, 0.9, 0.8}, inner_fraction {0.2, 0.3, 0.45,
 * 0.5, 1}, relist_soon {0.4, 0.5, 0.6} -- keeping the fastest value of each
 * before tuning the next, applies the result and appends it to
 * cfg->autotune_cache (host text file, one "key item_warps inner_fraction
 * relist_soon bin_factor skin_scale" line; key = potential kinds, log2 of the
 * atom and system capacities, precision; a line without skin_scale reads as
 * 1) when a path was given.  ts_batch_create applies the last matching cache
 * line.  The state
 * is first advanced by 4 n_steps (so that trials time the dynamics that
 * follow, not the start-up transient), then saved in a temporary device copy
 * (positions, velocities; the cell and piston velocities under NPT, the chain
 * state under NHC) that is restored, with the same noise counter, before each
 * trial.  s is left at the end of the last trial: pass a copy of the state to
 * keep the original.  Allocates that copy, synchronises.  n_steps in
 * [1, 1000]. */
ts_status ts_autotune(ts_batch* b, ts_state* s, const ts_md_params* p, int n_steps, void* stream);

/* The batch's current parameters, or set them (TS_ERR_INVALID_ARG outside the
 * ranges above).  Setting them re-derives the layout and re-lists every system
 * on the next call (synchronous; the paper has no counterpart). */
ts_status ts_batch_tuning(const ts_batch* b, ts_tuning* out);
ts_status ts_batch_set_tuning(ts_batch* b, const ts_tuning* t);

/* Measurement hook: launch the pair-force kernel alone (forces only, from the
 * inner lists, the form an MD step uses) reps times, after re-listing flagged
 * systems and re-filtering every inner list, each launch preceded by
 * a write of flush_bytes to flush_buf (device scratch, may be NULL) to evict
 * L2, timing each launch with its own pair of CUDA events on the stream (all
 * launches are enqueued before the first is waited for, so that no event pair
 * includes the host's launch latency).  Synchronises.
 * ms_out (host): mean launch duration in ms; pairs_out (host, may be NULL):
 * ordered pairs within the cutoff (the algorithmic work of one launch);
 * atoms_out (host, may be NULL): atoms per launch. */
ts_status ts_profile_pair(ts_batch* b, ts_state* s, int reps, void* flush_buf, size_t flush_bytes, double* ms_out,
                          int64_t* pairs_out, int64_t* atoms_out, void* stream);

/* Energies, forces and stress without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc -- a host program that hands the library a fixed set
 * of buffers and forbids allocation after start-up, code running inside
 * another framework that owns the device allocator, or a loop that cannot
 * afford cudaMalloc's implicit device synchronisation.
 * It needs no ts_batch: it takes the potentials (host array, 1..4 entries),
 * a state whose pos, cell, system_idx and pot_idx are read (vel, mass, pbc,
 * uid are ignored; all systems fully periodic) and offsets [n_systems + 1]
 * (device i64, first atom of each system, then n_atoms), and writes F
 * [n_atoms][3], E [n_systems], stress [n_systems][3][3] (device f64; E and
 * stress may be NULL).  Arithmetic is FP64: an all-pairs sum over each
 * system's atoms and every lattice image within the cutoff, so the cost is
 * O(n^2) per system -- meant for small systems.  Energies and stress are
 * reduced in a fixed order (bit-reproducible, independent of the batch).
 * A system that cannot be evaluated gets NaN in E, stress and (when its
 * offsets delimit atoms of the batch) the F rows of its atoms: pot_idx
 * outside [0, n_pots), offsets decreasing or outside [0, n_atoms], a
 * singular or non-finite cell, a cell so thin that an image more than 4
 * cells away could lie within the cutoff, an atom whose system_idx
 * disagrees with the offsets, or a non-finite position.
 * Scratch: a fixed device table of per-CTA partial sums (4096 systems x 2
 * rows x 8 doubles = 512 KiB) that every GPU loading the library holds until
 * exit.  More than 4096 systems returns TS_ERR_BUDGET.  The first call on a
 * device looks up that table's address (cudaGetSymbolAddress); make it
 * before capturing a stream.  All calls share the table and each call
 * overwrites the rows it reads, so calls that overlap on the GPU (several
 * streams or host threads) race and must be serialised by the caller. */
ts_status ts_pair_forces_noalloc(const ts_potential* pots, int n_pots, const ts_state* s, const int64_t* offsets,
                                 double* F, double* E, double* stress, void* stream);

/* Human-readable text of the last host-side error of this batch (never NULL).
 * The paper has no counterpart (Python exceptions carry the text there). */
const char* ts_last_error(const ts_batch* b);

/* Counters for reporting: kernel launches issued so far by this batch, and
 * neighbour-list rebuilds (system re-listings) so far.  The paper has no
 * counterpart; the re-listing count measures the neighbour-graph work that
 * Sec. 4 names as a cost. */
ts_status ts_batch_counters(const ts_batch* b, int64_t* launches, int64_t* relists);

/* Inner-list refreshes so far (one per system and refresh).  MD steps compute
 * forces from an inner list, the entries of the Verlet list within
 * rc + f * skin (f = 0.3, or TS_INNER at batch creation; 1 turns pruning
 * off).  A system's inner list is re-filtered from its Verlet list by the
 * pair launch of the MD step in which it was re-listed or one of its atoms
 * had moved f * skin / 2 since the last filtering; that launch runs the full
 * list.  Pairs beyond rc contribute exactly zero, so results are
 * bit-identical with pruning on or off; this count is for reporting.
 * Synchronises the device; TS_ERR_INVALID_ARG on a null argument. */
ts_status ts_batch_prunes(const ts_batch* b, int64_t* prunes);

#ifdef __cplusplus
}
#endif
#endif /* TS_H_ */
