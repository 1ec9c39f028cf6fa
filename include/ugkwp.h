/*
 * ugkwp.h -- C ABI of the GB300 (sm_103a) implementation of the per-time-step
 * particle phase of the unified gas-kinetic wave-particle (UGKWP) method for
 * the frequency-dependent radiation transport equation, with the wave-part
 * flux and the matrix-free source iteration around it.
 *
 * Method: Yang, Zhu, Liu, Xu, "Unified gas-kinetic wave-particle method for
 * frequency-dependent radiation transport equation" -- Algorithm 1 (the time
 * step), Eqs. particle-tf-formula, IhpFormula, wfrpFormula, macroSysFinal,
 * the interface-reset remark, Eqs. Blinear/kg with App. A (frequency of a
 * particle), App. B with Algorithm 2 (source iteration).
 *
 * Conventions shared by every entry point:
 *  - Every call returns UGKWP_OK (0) or a negative UGKWP_ERR_* code.  Nothing
 *    throws across the ABI.  ugkwp_last_error() gives a message.
 *  - The library never allocates device memory: the caller passes one device
 *    workspace (size from ugkwp_workspace_size) and keeps ownership of it; the
 *    handle itself is a small host allocation freed by ugkwp_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued asynchronously; only ugkwp_tallies, ugkwp_get_state and
 *    ugkwp_set_state synchronise the stream.
 *  - Layout: cells c = (iz*ny + iy)*nx + ix (ny = 1 in 1D, nz = 1 below 3D);
 *    per (cell, group) arrays [c*G + g]; x-faces f = (iz*ny + iy)*(nx+1) + fx
 *    (at x = fx*dx), then y-faces nxface + (iz*(ny+1) + fy)*nx + ix, then
 *    z-faces nxface + nyface + (fz*ny + iy)*nx + ix; sides 0 = x-, 1 = x+,
 *    2 = y-, 3 = y+, 4 = z-, 5 = z+.  Normalised units h = k = 1.
 *  - Errors found on the device during a step (particle capacity exceeded,
 *    source iteration not converged, non-finite state, a bounded wait that
 *    timed out) are latched in a status word and returned by ugkwp_tallies.
 */
#ifndef UGKWP_H
#define UGKWP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define UGKWP_OK 0
#define UGKWP_ERR_ARG (-1)          /* invalid argument or inconsistent problem */
#define UGKWP_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define UGKWP_ERR_CAPACITY (-3)     /* more surviving particles than capacity, or a bin overflowed */
#define UGKWP_ERR_NOCONV (-4)       /* source iteration hit si_max_iters */
#define UGKWP_ERR_NONFINITE (-5)    /* NaN/Inf in the macroscopic state */
#define UGKWP_ERR_TIMEOUT (-6)      /* a bounded device-side wait gave up */
#define UGKWP_ERR_WORKSPACE (-7)    /* workspace too small or misaligned */
#define UGKWP_ERR_UNSUPPORTED (-8)  /* a combination this build does not implement */

/* device status bits (ugkwp_tallies.status_bits) */
#define UGKWP_ST_CAPACITY 1u
#define UGKWP_ST_NOCONV 2u
#define UGKWP_ST_NONFINITE 4u
#define UGKWP_ST_TIMEOUT 8u
#define UGKWP_ST_IDSPACE 16u   /* step past 2^20 - 1: a newborn's identity (birth step << 44 |
                                  bin << 20 | k) has no room, so nothing was sampled */

enum { UGKWP_BC_REFLECT = 0, UGKWP_BC_VACUUM = 1, UGKWP_BC_BLACKBODY = 2 };
enum { UGKWP_FP64 = 0, UGKWP_MIXED = 1 };
/* Method (Sec. 2.2): UGKWP samples the collisionless part e^{-dt/tau} I^h of
 * the wave part with t_f = dt; UGKP samples all of I^h, every newborn draws
 * its own free time, and a sampled half carries no wave flux (the particles
 * carry its whole free transport).  Black-body sides are sampled the UGKWP
 * way in both.  The adjoint entry points accept UGKWP only. */
enum { UGKWP_METHOD_UGKWP = 0, UGKWP_METHOD_UGKP = 1 };

/* Problem statement (Sec. 3 numerical set-up; all pointers are HOST pointers,
 * read during ugkwp_init only; the caller keeps ownership).
 *   sigma(nu, T) = sigma0[c] * nu^sig_p * T^sig_q, capped at sig_cap (> 0)
 *   (Eq. sigmaMarsharkMF: sig_p = -3, sig_q = -1/2); with sig_law = 1 times the
 *   photo-ionisation factor (1 - e^{-nu/T}) of the Larsen case (Sec. 3.3:
 *   sig_p = -3, sig_q = 0); group opacity by Simpson's
 *   rule on the edges and midpoint of each group.  grey = 1: one group, no
 *   frequency dependence, Phi = a c T^4.
 *   Boundary sides: REFLECT (mirror), VACUUM (no inflow), BLACKBODY at bcT
 *   (1D only in this build).  src_T: a cell with src_T > 0 receives
 *   src_on * src_amp[c] * c * dt * Phi_g(src_T) in rho_g each step while
 *   t^n = n dt < src_t_end (src_amp NULL: 1; src_t_end <= 0: always); the
 *   Olson case (Sec. 3.5) has Q = B(0.5 keV) e^{-693 x^3} for ct <= 2.
 *   sig_law = 2: the carbon-hydrogen foam of the Olson case, sigma = sigma0
 *   kappa(nu, T) with kappa = min(1e7, 1e9 T^2) for nu <= 0.008,
 *   3e6 (0.008/nu)^2/(1 + 200 T^1.5) for 0.008 < nu <= 0.3, and that times
 *   (0.3/nu)^0.5 plus 4e4 (0.3/nu)^2.5/(1 + 8000 T^2) above (nu, T in keV;
 *   sig_p and sig_q are not used).
 *   cv_law = 1: the foam's heat capacity (Eq. cvolson), cv[c] (1 + alpha +
 *   (T + chi) dalpha/dT) with alpha = (1/2) e^{-chi/T} (sqrt(1 + 4 e^{chi/T})
 *   - 1), chi = cv_chi; the material energy is cv[c] (T + (T + chi) alpha).
 *   tau_num_C: the numerical collision time of the heterogeneous cases
 *   (Sec. 3.2), tau_num = tau + C J dt with J the largest temperature contrast
 *   |T_c - T_n|/(T_c + T_n) over a cell's interior faces, replaces tau in the
 *   sampled fraction e = exp(-dt/tau_num) (births and wave flux); 0 keeps tau. */
typedef struct ugkwp_problem {
  int32_t dim;            /* 1, 2 or 3 */
  int32_t nx, ny;         /* cells; ny ignored (1) in 1D */
  int32_t G;              /* groups, 1..64 */
  int32_t grey;           /* 1: grey (G == 1) */
  int32_t wave_order;     /* 1: cell averages, 2: van Leer reconstruction of rho_h */
  int32_t si_max_iters;   /* source-iteration cap */
  int32_t precision;      /* UGKWP_FP64 or UGKWP_MIXED (particle state in FP32) */
  int32_t bc[4];
  int32_t sig_law;        /* 0: sigma0 nu^p T^q; 1: times (1 - e^{-nu/T}) (Larsen case); 2: Olson foam */
  double dx, dy;
  double sig_p, sig_q, sig_cap;
  double a, c, eps, dt;
  double omega_ref;       /* reference particle energy (rho*V units), <= 0: no particles */
  double si_tol;          /* source-iteration tolerance (relative, max norm) */
  double src_on;
  double tau_num_C;       /* thin/thick joint sampling: tau_num = tau + C J dt (0: off) */
  double bcT[4];
  uint64_t seed;          /* Philox key = (seed_lo, seed_hi ^ instance) */
  uint32_t instance;
  int32_t method;         /* UGKWP_METHOD_UGKWP (0) or UGKWP_METHOD_UGKP (1) */
  int64_t particle_capacity;   /* particles one step may process (survivors in + newborns): each of
                                  the two particle buffers holds that many; a particle beyond it
                                  is dropped (UGKWP_ST_CAPACITY), its energy left to the wave part */
  const double* nu_edges;      /* [G+1] increasing, > 0 (ignored when grey) */
  const double* sigma0;        /* [ncell] */
  const double* cv;            /* [ncell] */
  const double* T0;            /* [ncell] initial material temperature */
  const double* rho0;          /* [ncell*G] initial rho_g, or NULL: Phi_g(T0) */
  const double* src_T;         /* [ncell] or NULL */
  const double* src_amp;       /* [ncell] source profile factor, or NULL (1) */
  double src_t_end;            /* source active while t^n < src_t_end (<= 0: always) */
  int32_t cv_law;              /* 0: constant cv; 1: Olson foam heat capacity (Eq. cvolson) */
  int32_t _pad2;
  double cv_chi;               /* chi of cv_law 1 */
  /* 3D (dim 3): cells along z, the z sides (4: z-, 5: z+; reflecting or
   * vacuum) and the cell height.  Ignored for dim 1 and 2. */
  int32_t nz;
  int32_t bc_z[2];
  int32_t _pad3;
  double dz;
  double bcT_z[2];
  /* Wave/particle split after the source iteration (Sec. 2.2, I^h = I^{n+1}
   * - I^p).  0 (default): where the collisionless survivors of a (cell,
   * group) hold more than rho^{n+1} V, their weights are scaled down to it,
   * so rho^h never goes below min(rho^{n+1}, 0) (a reading where the paper is
   * silent; the scaled bins are counted in n_scaled_bins).  1: the split as
   * written, rho^h = rho^{n+1} - E_surv/V, nothing scaled. */
  int32_t split_literal;
  /* Source iteration of a UGKWP_MIXED problem (App. B, Algorithm 2): FP32
   * iterates of the same linearised update first, from T^n until the change
   * of T is near FP32 resolution, then FP64 iterates from there to si_tol --
   * the fixed point reached is the FP64 one, only the starting point differs.
   * 0 (default): on where the iteration has at least 2^17 (cell, group)
   * pairs (over all ensemble members); 1: on; -1: off.  Ignored in FP64. */
  int32_t si_warm32;
  /* Source iteration of a single 1D problem of at most two cells per SM
   * (without the FP32 warm start): 0 (default): two warps per cell, which
   * share each iterate's work (the same results, bit for bit); -1: one warp
   * per cell. */
  int32_t si_pair;
  int32_t _pad6;
} ugkwp_problem;

typedef struct ugkwp_handle ugkwp_handle;

/* Device pointers into the workspace (valid until the next step) and host
 * copies of the per-step counters and energy ledger. */
typedef struct ugkwp_tally_report {
  const double* T;        /* [ncell]   material temperature T^{n+1} */
  const double* rho;      /* [ncell*G] rho^{n+1} */
  const double* rho_h;    /* [ncell*G] wave part rho^{n+1} - rho^p */
  const double* rho_p;    /* [ncell*G] particle part (collisionless survivors / V) */
  const double* W;        /* [ncell*G] w^{fr,p}, particle energy in minus out (Eq. wfrpFormula) */
  const double* Fwave;    /* [nface*G] wave-part flux F^{fr,wave} */
  const double* Feq;      /* [nface*G] equilibrium flux of the last source iterate */
  const double* esc;      /* [6*G] particle energy escaped per side (x-, x+, y-, y+, z-, z+) */
  const double* inflow;   /* [6*G] particle energy entering per side */
  int64_t step;           /* steps completed */
  int64_t n_particles;    /* particles alive after the last step */
  int64_t n_in, n_born, n_survived, n_absorbed, n_escaped, n_removed, n_segments;
  int32_t si_iters;
  uint32_t status_bits;   /* UGKWP_ST_* latched since init */
  double E_rad0, E_mat0, E_rad1, E_mat1;      /* sum V rho/c, sum V Cv T before/after */
  double bnd_in_macro, bnd_in_part, bnd_out_part, src_in;
  int64_t n_scaled_bins;  /* (cell, group) bins whose survivors' weights were scaled (split_literal 0) */
  int32_t si_iters32;     /* FP32 warm-start iterates before the si_iters FP64 ones (si_warm32) */
  int32_t _pad5;
} ugkwp_tally_report;

/* Host-side structure-of-arrays particle buffers for ugkwp_get_state /
 * ugkwp_set_state (parity checks, checkpoints).  1D: ox holds mu; y, oy are 0. */
typedef struct ugkwp_particles_host {
  double *x, *y, *ox, *oy, *nu, *w;
  uint64_t* id;
  int32_t *cell, *grp;
  double *z, *oz;         /* dim 3 only (may be NULL otherwise) */
} ugkwp_particles_host;

/* Per-particle end record written when a record buffer is attached
 * (ugkwp_set_records): one per particle processed in a step, at its position
 * in the step's processing order (survivors first, then newborns). */
typedef struct ugkwp_record {
  uint64_t id;
  int32_t fate;           /* 0 survived, 1 absorbed (collided), 2 escaped, 3 removed */
  int32_t cell0, cell1, grp, nseg, _pad;
  double x, y, ox, oy, nu, w, t_end;
  double z, oz;           /* dim 3 (0 otherwise) */
} ugkwp_record;

/* Workspace bytes for problem p (256-byte aligned pieces). */
int ugkwp_workspace_size(const ugkwp_problem* p, size_t* bytes);

/* Copy the problem into the device workspace, set the initial state
 * (T0, rho0 or Phi_g(T0), no particles) and return a handle.  The workspace
 * must stay allocated until ugkwp_destroy. */
int ugkwp_init(const ugkwp_problem* p, void* d_workspace, size_t bytes, void* stream,
               ugkwp_handle** out);

/* Advance nsteps time steps (Algorithm 1), asynchronously on `stream`:
 * birth counts and scan (Eq. IhpFormula), streaming of survivors and
 * newborns with t_f reset and tallies (Eqs. particle-tf-formula, wfrpFormula),
 * wave flux (Sec. 2.2), source iteration (App. B), removal of the collided
 * particles with the survivors sorted by (cell, group) bin.  Each step is
 * one replay of a CUDA graph captured on the first call. */
int ugkwp_step(ugkwp_handle* h, int nsteps, void* stream);

/* One step like ugkwp_step, launched kernel by kernel and bracketed by CUDA
 * events on `stream`, then synchronise: phase_ms[0] the whole step, [1]
 * birth counts and their scan, [2] wave flux, [3] particle kernel, [4] source
 * iteration, [5] end of step (the survivor sort, which ugkwp_step runs
 * beside the source iteration, then the weight scaling and counters)
 * (device milliseconds).  For measurement; the events are created and
 * destroyed per call. */
int ugkwp_step_timed(ugkwp_handle* h, void* stream, float* phase_ms);

/* Synchronise `stream` and fill *out (device pointers + host counters). */
int ugkwp_tallies(ugkwp_handle* h, ugkwp_tally_report* out, void* stream);

/* Copy the state to host arrays: T [ncell], rho, rho_h, rho_p [ncell*G] (any
 * may be NULL) and up to `cap` particles; *n receives the particle count.
 * After a step the particles are sorted by bin (cell c, group g: c*G + g);
 * the order inside a bin is set by atomics, so identify particles by `id`.
 * (After ugkwp_set_state they are in the order given.)  Synchronises
 * `stream`. */
int ugkwp_get_state(ugkwp_handle* h, double* T, double* rho, double* rho_h, double* rho_p,
                    ugkwp_particles_host* parts, int64_t cap, int64_t* n, void* stream);

/* Replace the state from host arrays (T, rho, rho_h required; parts may be
 * NULL when n == 0) and set the step counter.  Synchronises `stream`. */
int ugkwp_set_state(ugkwp_handle* h, const double* T, const double* rho, const double* rho_h,
                    const ugkwp_particles_host* parts, int64_t n, int64_t step, void* stream);

/* Attach (or detach with NULL) a DEVICE buffer of `cap` ugkwp_record entries
 * that the next steps fill; records beyond cap are dropped. */
int ugkwp_set_records(ugkwp_handle* h, ugkwp_record* d_records, int64_t cap);

/* ---- ensembles: independent problems advanced together ----
 * Members share dim, precision and si_max_iters but may differ in every
 * other field (cells, groups, opacities, boundaries, weights, seeds,
 * instance numbers).  One ugkwp_step advances all of them with the same
 * kernels as a single problem: one launch per phase over every member's
 * bins, faces and cells, one persistent particle launch whose tiles run over
 * all members' particles (so uneven members share the GPU), and one
 * cooperative source iteration in which each member stops at its own
 * convergence.  A member's results equal those of the same problem run
 * alone (same identities and random streams, up to the summation order of
 * FP64 atomics).  At most 4096 members; records are not available. */
int ugkwp_workspace_size_ensemble(const ugkwp_problem* probs, int n, size_t* bytes);
int ugkwp_init_ensemble(const ugkwp_problem* probs, int n, void* d_workspace, size_t bytes, void* stream,
                        ugkwp_handle** out);
/* Per-member forms of ugkwp_tallies / ugkwp_get_state / ugkwp_set_state
 * (the plain calls address member 0). */
int ugkwp_tallies_member(ugkwp_handle* h, int member, ugkwp_tally_report* out, void* stream);
int ugkwp_get_state_member(ugkwp_handle* h, int member, double* T, double* rho, double* rho_h,
                           double* rho_p, ugkwp_particles_host* parts, int64_t cap, int64_t* n,
                           void* stream);
int ugkwp_set_state_member(ugkwp_handle* h, int member, const double* T, const double* rho,
                           const double* rho_h, const ugkwp_particles_host* parts, int64_t n,
                           int64_t step, void* stream);

/* ---- checkpoint / restore ----
 * The state of every member (T, rho, rho_h, rho_p, the live particles and
 * the control block with the step counter) copied device-to-device into a
 * caller-owned DEVICE buffer of ugkwp_checkpoint_size bytes (256-byte
 * aligned), asynchronously on `stream`.  Identities and counter-based random
 * streams make a restored run repeat the same steps, up to the summation
 * order of FP64 atomics. */
int ugkwp_checkpoint_size(const ugkwp_handle* h, size_t* bytes);
int ugkwp_checkpoint(ugkwp_handle* h, void* d_buf, size_t bytes, void* stream);
int ugkwp_restore(ugkwp_handle* h, const void* d_buf, size_t bytes, void* stream);

/* ---- launch shape of the particle kernel ----
 * block: 128, 256 or 512 threads; particles_per_thread: 1, 2 or 4 (the
 * mixed-precision kernel streams chunks of 32 x particles_per_thread
 * particles per warp, the FP64 kernel tiles of block x min(it, 2));
 * blocks_per_sm: 0 for as many as fit. */
int ugkwp_set_launch(ugkwp_handle* h, int block, int particles_per_thread, int blocks_per_sm);
/* ---- bounded waits ----
 * The source iteration's grid barrier polls at most `spins` times (0: the
 * default 2^25) before it gives up, sets UGKWP_ST_TIMEOUT and returns, so a
 * lost arrival never hangs the device.  extra_arrivals > 0 is a failure
 * injection for tests: every barrier then also waits for that many arrivals
 * that never come, so each wait runs out and the step reports the timeout
 * (the state it leaves is not meaningful; the context stays usable).
 * Enqueued on `stream`; takes effect from the next step.  No counterpart in
 * the paper. */
int ugkwp_set_wait_limit(ugkwp_handle* h, uint32_t spins, uint32_t extra_arrivals, void* stream);
/* Time every launch shape on `steps` identical steps (the state is saved in
 * d_ckpt, a buffer of ugkwp_checkpoint_size bytes, and restored before each
 * candidate and at the end), keep the fastest particle phase, and report it
 * in best[3] = {block, particles_per_thread, blocks_per_sm} and *best_ms.
 * Synchronises `stream`. */
int ugkwp_autotune(ugkwp_handle* h, void* d_ckpt, size_t bytes, int steps, void* stream, int* best,
                   float* best_ms);

/* ---- adjoint: gradient of a function of the final state with respect to
 * the per-cell log-opacity scales s_c (sigma0_c -> sigma0_c e^{s_c}) ----
 * The paper has no adjoint; this is the reverse mode of the step of
 * Algorithm 1 as implemented here.  The derivative is pathwise: every Monte
 * Carlo decision of a step (birth counts N, face crossings, collision,
 * survival, escape) is held as the forward step took it, with the same
 * Philox draws (common random numbers).  Along that path the particle
 * tallies are linear in the weights, a newborn's weight is E/N at fixed N
 * (Eq. IhpFormula), a survivor keeps its weight; the Simpson group opacity,
 * the wave flux (Sec. 2.2) and the converged source iteration (App. B,
 * differentiated through its fixed point) carry the rest.  Single-problem
 * FP64 handles only (UGKWP_ERR_UNSUPPORTED otherwise).
 *
 * Usage: checkpoint the forward run every k steps (ugkwp_checkpoint); for
 * the backward pass, restore a checkpoint and re-run its k steps with
 * ugkwp_step_taped (one tape per step), then call ugkwp_adjoint_step on the
 * tapes in reverse order, after ugkwp_adjoint_seed for the last step.
 * Restored steps repeat the forward ones up to the summation order of FP64
 * atomics.  All buffers are caller-owned DEVICE memory, 256-byte aligned. */

/* Bytes of one step's tape holding up to rec_cap processed particles (the
 * step's survivors in plus its newborns; a step with more sets
 * UGKWP_ST_CAPACITY in the forward status and in the adjoint's). */
int ugkwp_tape_size(ugkwp_handle* h, int64_t rec_cap, size_t* bytes);
/* One step (like ugkwp_step with nsteps = 1, without the captured graph)
 * that also writes its tape: T^n, rho_h^n, T^{n+1}, rho^{n+1}, the birth
 * counts, the step's counts, and per processed particle its start cell, end
 * cell, output slot and group.  Asynchronous on `stream`. */
int ugkwp_step_taped(ugkwp_handle* h, void* d_tape, size_t bytes, int64_t rec_cap, void* stream);
/* Bytes of the adjoint workspace (adjoint state, dL/ds, per-step work). */
int ugkwp_adjoint_workspace_size(ugkwp_handle* h, size_t* bytes);
/* Start the reverse pass: zero the workspace and set the adjoint of the
 * final temperature to d_dL_dT [ncell] (device; NULL leaves it 0). */
int ugkwp_adjoint_seed(ugkwp_handle* h, void* d_adj, size_t bytes, const double* d_dL_dT, void* stream);
/* Reverse one step from its tape: maps the adjoints of the step's outputs to
 * those of its inputs and adds the step's explicit part to dL/ds.  The
 * adjoint source iteration stops at max |d mu| <= si_tol max |mu| (cap
 * si_max_iters, else UGKWP_ST_NOCONV).  Asynchronous on `stream`. */
int ugkwp_adjoint_step(ugkwp_handle* h, const void* d_tape, size_t tape_bytes, int64_t rec_cap, void* d_adj,
                       size_t adj_bytes, void* stream);
/* Before reversing a recomputed segment whose end is the start of the
 * segment reversed last: the order of survivors inside a bin depends on
 * thread timing, so re-index the particles' weight adjoints from the order held in
 * d_ckpt (that later segment's checkpoint) to the handle's current particle
 * order (the recomputed segment's end), matching particle identities.  A
 * particle present on one side only gets 0 and is counted in the result's
 * `unmatched`.  Asynchronous on `stream`. */
int ugkwp_adjoint_remap(ugkwp_handle* h, void* d_adj, size_t adj_bytes, const void* d_ckpt, size_t ckpt_bytes,
                        void* stream);
/* Copy dL/ds [ncell] and dL/dT of the first reversed step's input [ncell]
 * (either pointer may be NULL; device destinations), and report the adjoint's
 * latched UGKWP_ST_* bits, the last step's adjoint source iterations and the
 * particles left unmatched by ugkwp_adjoint_remap (any pointer may be NULL).
 * Synchronises `stream`. */
int ugkwp_adjoint_result(ugkwp_handle* h, const void* d_adj, size_t bytes, double* d_dL_ds, double* d_dL_dT0,
                         uint32_t* status_bits, int32_t* si_iters, uint64_t* unmatched, void* stream);

const char* ugkwp_last_error(const ugkwp_handle* h);
void ugkwp_destroy(ugkwp_handle* h);

/* ---- kernel-level entry points (device pointers; parity tests of single
 * building blocks).  Each is asynchronous on `stream`. ---- */

/* Philox4x32-10 (Salmon et al., SC'11) of n counters [n*4] under key (k0, k1). */
int ugkwp_philox(const uint32_t* d_ctr, uint32_t k0, uint32_t k1, uint32_t* d_out, int64_t n,
                 void* stream);

/* Group Planck fractions b_g(T) = (15/pi^4) int_{nu_g/T}^{nu_{g+1}/T} t^3/(e^t-1) dt and
 * the derivative fractions d_g(T) with dPhi_g/dT = a c T^3 d_g(T), for n temperatures:
 * d_b, d_d are [n*G] (d_d may be NULL).  d_nu_edges is a DEVICE array [G+1]. */
int ugkwp_planck(const double* d_T, int64_t n, const double* d_nu_edges, int G, double* d_b,
                 double* d_d, void* stream);

/* Time-integrated coefficients at x = dt/tau for n values: d_out [n*4] =
 * (C2/tau, C4 - e, (C5 + dt e/2)/tau, C4) (Eq. C2Formula and the UGKS free-flux
 * coefficients). */
int ugkwp_coefs(const double* d_x, int64_t n, double* d_out, void* stream);

/* Exclusive prefix sum of per-bin birth counts (the birth ordinals of
 * Eq. IhpFormula's sampled particles): d_offsets[i] = sum_{j<i} d_counts[j]
 * for i = 0..n (n + 1 values, d_offsets[n] = the total).  n <= 2^24 and the
 * total must fit in 32 bits.  d_scratch: a DEVICE buffer of at least
 * UGKWP_SCAN_SCRATCH_BYTES(n) bytes for the per-block partial sums. */
#define UGKWP_SCAN_SCRATCH_BYTES(n) (4 * (((n) + 4095) / 4096) + 4)
int ugkwp_exclusive_scan(const uint32_t* d_counts, int64_t n, uint32_t* d_offsets, void* d_scratch,
                         size_t scratch_bytes, void* stream);

/* The same exclusive scan, allocating nothing: for callers that cannot get
 * device memory -- a program whose GPU memory is all held by its own pool
 * allocator, a plug-in whose host framework forbids cudaMalloc/cudaFree
 * inside its time step (they can synchronise the whole device), or code
 * that only holds pointers to buffers allocated by someone else.  It has no
 * counterpart in the paper.  The scratch (per-block partial sums) is a
 * fixed 16 KiB device array compiled into the library, resident on every GPU
 * that loads the library until the process exits; n is limited to
 * UGKWP_NOALLOC_SCAN_MAX_N and larger n is rejected with UGKWP_ERR_ARG
 * (message from ugkwp_last_error(NULL)).  The caller still passes the
 * counts and the n + 1 offsets (DEVICE pointers).  The first call on a
 * device looks up the array's device address with that device current
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array, so calls that overlap on the GPU (on
 * different streams, or from different host threads) race and must not be
 * issued; each call overwrites the partials it reads, so nothing is left to
 * clear between calls.  No cudaMalloc, cudaFree or allocating library
 * routine is called. */
#define UGKWP_NOALLOC_SCAN_MAX_N (1ll << 24)
int ugkwp_exclusive_scan_noalloc(const uint32_t* d_counts, int64_t n, uint32_t* d_offsets, void* stream);

/* Frequency of a particle from uniforms d_eta [n] for group [nlo, nhi] at
 * temperature T (App. A, linear-frequency sampling) into d_nu [n]. */
int ugkwp_sample_nu(const double* d_eta, int64_t n, double nlo, double nhi, double T, double* d_nu,
                    void* stream);

#ifdef __cplusplus
}
#endif
#endif
