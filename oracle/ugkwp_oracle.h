/*
 * ugkwp_oracle.h -- CPU FP64 oracle of the UGKWP particle phase, the wave flux
 * and the source iteration (Yang, Zhu, Liu, Xu, "Unified gas-kinetic
 * wave-particle method for frequency-dependent radiation transport equation").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may include,
 * link or call this code; only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark use it.  It shares no source with the
 * CUDA path: it is a plain, slow, step-by-step restatement of the method.
 *
 * Conventions (same meaning as the C ABI of the product, declared separately):
 *   cells are indexed c = (iz*ny + iy)*nx + ix; (cell, group) arrays are [c*G + g];
 *   x-faces f = (iz*ny + iy)*(nx+1) + fx (face fx sits at x = fx*dx);
 *   y-faces f = nxf + (iz*(ny+1) + fy)*nx + ix (face fy sits at y = fy*dy);
 *   z-faces f = nxf + nyf + (fz*ny + iy)*nx + ix;
 *   sides: 0 = x-, 1 = x+, 2 = y-, 3 = y+, 4 = z-, 5 = z+.
 */
#ifndef UGKWP_ORACLE_H
#define UGKWP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_BC_REFLECT = 0, OR_BC_VACUUM = 1, OR_BC_BLACKBODY = 2 };
enum { OR_UGKWP = 0, OR_UGKP = 1 };
enum { OR_SURVIVED = 0, OR_ABSORBED = 1, OR_ESCAPED = 2, OR_REMOVED = 3 };
enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_CAPACITY = -3, OR_ERR_NOCONV = -4,
       OR_ERR_NONFINITE = -5, OR_ERR_IDSPACE = -9 };
/* A newborn's identity is (birth step << 44) | (bin << 20) | k: the birth
 * step has 20 bits.  A step past OR_MAX_STEP samples no particle and returns
 * OR_ERR_IDSPACE (its identities, and with them its random streams, would
 * repeat those of an earlier step). */
#define OR_MAX_STEP ((int64_t)((1 << 20) - 1))

typedef struct {
  int32_t dim, nx, ny, G;
  int32_t grey;          /* 1: one grey group, b = 1, particles carry no frequency */
  int32_t wave_order;    /* 1: cell-average upwind values, 2: van Leer linear reconstruction */
  int32_t si_max_iters;
  int32_t bc[4];
  int32_t sig_law;       /* 0: sigma0 nu^p T^q; 1: sigma0 nu^p T^q (1 - e^{-nu/T}) (Larsen case) */
  double dx, dy;
  double sig_p, sig_q, sig_cap;   /* sigma = sigma0 * nu^p * T^q, capped (cap <= 0: none) */
  double a, c, eps, dt;
  double omega_ref;               /* reference particle energy (rho*V units) */
  double si_tol;
  double src_on;                  /* multiplies the patch source */
  double tau_num_C;               /* C of the numerical collision time (0: tau_num = tau) */
  double bcT[4];
  uint64_t seed;
  uint32_t instance;
  int32_t method;                 /* OR_UGKWP (0) or OR_UGKP (1, Sec. 2.2: all of I^h as particles) */
  const double* nu_edges;         /* [G+1] */
  const double* sigma0;           /* [ncell] */
  const double* cv;               /* [ncell] */
  const double* src_T;            /* [ncell] or NULL */
  const double* src_amp;          /* [ncell] source profile factor, or NULL (1) */
  double src_t_end;               /* the source acts while t^n = step dt < src_t_end (<= 0: always) */
  int32_t cv_law;                 /* 0: constant cv; 1: Olson CH foam, cv (1 + alpha + (T + chi) alpha') */
  int32_t _pad2;
  double cv_chi;                  /* chi of cv_law 1 */
  int32_t nz;                     /* 3D: cells along z (dim 3) */
  int32_t bc_z[2];                /* sides 4 (z-) and 5 (z+) */
  int32_t _pad3;
  double dz;
  double bcT_z[2];
  int32_t split_literal;          /* 1: rho^h = rho^{n+1} - E_surv/V as written; 0: survivors scaled */
  int32_t _pad4;
} or_problem;

/* Structure-of-arrays particle set.  In 1D, ox holds mu and y, oy are 0. */
typedef struct {
  double *x, *y, *ox, *oy, *nu, *w;
  uint64_t* id;
  int32_t *cell, *grp;
  double *z, *oz;                 /* 3D only (may be NULL otherwise) */
} or_particles;

/* One record per particle processed in a step (survivors in, then newborns). */
typedef struct {
  uint64_t id;
  int32_t fate, cell0, cell1, grp, nseg, _pad;
  double x, y, ox, oy, nu, w, t_end;
  double z, oz;
} or_record;

typedef struct {
  /* arrays owned by the caller */
  double* W;       /* [ncell*G] particle net energy w^{fr,p} (in minus out) */
  double* E_surv;  /* [ncell*G] energy of collisionless survivors by end cell */
  double* E_abs;   /* [ncell*G] energy of collided particles by collision cell */
  double* esc;     /* [4*G] particle energy leaving through each side */
  double* inflow;  /* [4*G] particle energy entering from each side's ghost */
  double* Fwave;   /* [nface*G] wave flux (x-faces then y-faces) */
  double* Feq;     /* [nface*G] equilibrium flux of the last source iteration */
  int32_t* N;      /* [nbins] birth counts, nbins = (ncell+4)*G */
  double* omega;   /* [nbins] */
  double* e_eff;   /* [nbins] */
  /* scalars written by the oracle */
  int64_t n_in, n_born, n_survived, n_absorbed, n_escaped, n_removed, n_segments;
  int32_t si_iters, status;
  double E_rad0, E_mat0, E_rad1, E_mat1;   /* sum V (rho/c) and sum V Cv T, before/after */
  double bnd_in_macro, bnd_out_macro;      /* through boundary faces, energy units */
  double bnd_in_part, bnd_out_part;        /* particles, energy units */
  double src_in;
  int64_t n_scaled_bins;                   /* (cell, group) bins whose survivors were scaled */
} or_tallies;

/* --- building blocks (each is pinned separately by the tests) --- */
void   or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_uniform(uint32_t wa, uint32_t wb);
double or_draw(const or_problem* P, uint64_t id, int64_t step, int64_t j);
double or_sigma(const or_problem* P, int c, double nu, double T);
double or_sigma_group(const or_problem* P, int c, int g, double T);
double or_mat_energy(const or_problem* P, int c, double T);   /* material energy per volume e(T) */
double or_heat_capacity(const or_problem* P, int c, double T); /* de/dT */
double or_planck_integral(double x1, double x2);      /* (15/pi^4) int_x1^x2 t^3/(e^t-1) dt */
double or_planck_dintegral(double x1, double x2);     /* (15/pi^4) int_x1^x2 t^4 e^t/(e^t-1)^2 dt */
double or_phi(const or_problem* P, int g, double T);  /* angle-integrated group equilibrium */
double or_dphi(const or_problem* P, int g, double T); /* its T-derivative */
void   or_coefs(double x, double* f2, double* f4, double* f5, double* c4);
double or_nu_cdf(double nlo, double nhi, double T, double nu);
double or_sample_nu(double nlo, double nhi, double T, double eta);

/* Stream one particle (Algorithm 1, steps 3-5).  If draws != NULL the
 * uniforms are taken from it in order (n_draws of them) instead of Philox.
 * Returns the fate.  trace_x/trace_t (nullable, cap trace_cap) receive the
 * position and elapsed time at the end of every flight segment. */
int or_stream_particle(const or_problem* P, const double* T, int64_t step,
                       double* x, double* y, double* ox, double* oy, double nu,
                       double w, uint64_t id, int32_t* cell, int32_t g,
                       int newborn, int64_t first_draw,
                       const double* draws, int64_t n_draws,
                       or_tallies* tal, int32_t* nseg, double* t_end,
                       double* trace_x, double* trace_t, int trace_cap, int* n_trace);
/* The same in 3D (z and Omega_z too; 1D and 2D leave them untouched). */
int or_stream_particle3(const or_problem* P, const double* T, int64_t step,
                       double* x, double* y, double* z, double* ox, double* oy, double* oz, double nu,
                       double w, uint64_t id, int32_t* cell, int32_t g,
                       int newborn, int64_t first_draw,
                       const double* draws, int64_t n_draws,
                       or_tallies* tal, int32_t* nseg, double* t_end,
                       double* trace_x, double* trace_t, int trace_cap, int* n_trace);

/* Delta t / tau_num for cell c, group g at T (Sec. 3.2, thin/thick joint):
 * tau_num = tau + C J Delta t with J the largest |T_c - T_n|/(T_c + T_n) over
 * the cell's interior faces; equals Delta t / tau when C = 0. */
double or_x_num(const or_problem* P, const double* T, int c, int g);

int or_birth_counts(const or_problem* P, const double* T, const double* rho_h,
                    or_tallies* tal, int64_t* n_new);

int or_wave_flux(const or_problem* P, const double* T, const double* rho_h,
                 const double* e_eff, double* Fwave);

int or_source_iteration(const or_problem* P, const double* T_n, const double* rho_n,
                        const double* R, double* T_out, double* rho_out,
                        double* Feq_out, int* iters);

/* One full time step (Algorithm 1).  Inputs T, rho, rho_h ([ncell], [ncell*G]) and
 * n_in particles; outputs the new macroscopic state, the surviving particles
 * (capacity cap_out) and, if rec != NULL, one record per processed particle. */
int or_step(const or_problem* P, int64_t step,
            const double* T, const double* rho, const double* rho_h,
            int64_t n_in, const or_particles* pin,
            double* T_out, double* rho_out, double* rho_h_out, double* rho_p_out,
            or_particles* pout, int64_t cap_out, int64_t* n_out,
            or_record* rec, int64_t rec_cap,
            or_tallies* tal);

/* or_step with an optional second weight per particle: when tal2 != NULL
 * every particle is streamed once more along the same path carrying w2_in[i]
 * (survivors in) or w2_bins[b] (newborns of bin b) into tal2 (W, E_surv,
 * E_abs, esc, inflow; zeroed by the caller), and survivors carry their
 * second weight to w2_out in output order (before the end-of-step weight
 * scaling, whose factors per (cell, group) go to w2_scale when it is not
 * NULL).  The tangent step uses it: the particle tallies are linear in the
 * weights along a fixed path. */
int or_step_core(const or_problem* P, int64_t step,
                 const double* T, const double* rho, const double* rho_h,
                 int64_t n_in, const or_particles* pin,
                 double* T_out, double* rho_out, double* rho_h_out, double* rho_p_out,
                 or_particles* pout, int64_t cap_out, int64_t* n_out,
                 or_record* rec, int64_t rec_cap,
                 or_tallies* tal,
                 const double* w2_in, const double* w2_bins, double* w2_out, or_tallies* tal2,
                 double* w2_scale);

/* --- tangent (forward-mode pathwise derivative), ugkwp_oracle_tangent.c ---
 * Directions: ds[c] changes the log of sigma0_c; dT, drho, drho_h and the
 * particles' weight tangents change the incoming state.  Every discrete
 * decision of the step is held fixed (common random numbers). */
double or_dsigma_group(const or_problem* P, int c, int g, double T, double ds, double dT);
void   or_dcoefs(double x, double* df2, double* df4, double* df5, double* dc4);
int    or_wave_flux_tangent(const or_problem* P, const double* T, const double* dT,
                            const double* ds, const double* rho_h, const double* drho_h,
                            const double* e_eff, double* dFwave);
/* T, rho: the converged solution of the source iteration; dR: tangent of its
 * constant part R. */
int    or_source_iteration_tangent(const or_problem* P, const double* dT_n, const double* ds,
                                   const double* dR, const double* T, const double* rho,
                                   double* dT_out, double* drho_out, int* iters);
/* (tau_num_C must be 0: OR_ERR_ARG otherwise.) */
int    or_step_tangent(const or_problem* P, int64_t step, const double* ds,
                       const double* T, const double* dT, const double* rho, const double* drho,
                       const double* rho_h, const double* drho_h,
                       int64_t n_in, const or_particles* pin, const double* dw_in,
                       double* T_out, double* dT_out, double* rho_out, double* drho_out,
                       double* rho_h_out, double* drho_h_out, double* rho_p_out,
                       or_particles* pout, double* dw_out, int64_t cap_out, int64_t* n_out,
                       or_tallies* tal);

/* Initial equilibrium rho_g = Phi_g(T0) per cell. */
void or_init_rho(const or_problem* P, const double* T0, double* rho);

#ifdef __cplusplus
}
#endif
#endif
