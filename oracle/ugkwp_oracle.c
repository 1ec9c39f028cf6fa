/*
 * ugkwp_oracle.c -- plain, slow, step-by-step CPU FP64 oracle of the UGKWP
 * method for the frequency-dependent (multigroup) radiation transport
 * equation: Yang, Zhu, Liu, Xu, "Unified gas-kinetic wave-particle method for
 * frequency-dependent radiation transport equation".
 *
 * TEST INFRASTRUCTURE ONLY: used by the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the product library, with which
 * it shares no code.  Every function states the passage of the paper it
 * follows.  Where the paper is silent or garbled the reading taken is stated
 * at the function (the same readings are listed in the design document).
 *
 * Normalised units: h = k = 1, so the Planck argument is nu/T.
 */
#include "ugkwp_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846264338327950288
#define PLANCK_NORM (15.0 / (PI * PI * PI * PI))   /* 15/pi^4 */
#define MAX_K_PER_BIN ((1 << 20) - 1)

/* Grid: cells c = (iz ny + iy) nx + ix; faces along axis a between the line
 * cells k-1 and k (k = 0..n_a): x-faces (iz ny + iy)(nx+1) + k, y-faces
 * nxf + (iz (ny+1) + k) nx + ix, z-faces nxf + nyf + (k ny + iy) nx + ix.  A
 * "line" of axis a is the set of cells sharing the other two coordinates,
 * numbered with the lower remaining axis fastest.  1D and 2D are the cases
 * ny = nz = 1 and nz = 1.                                                   */
static int ny_of(const or_problem* P) { return P->dim >= 2 ? P->ny : 1; }
static int nz_of(const or_problem* P) { return P->dim == 3 ? P->nz : 1; }
static int ncell_of(const or_problem* P) { return P->nx * ny_of(P) * nz_of(P); }
static int nxface_of(const or_problem* P) { return (P->nx + 1) * ny_of(P) * nz_of(P); }
static int nyface_of(const or_problem* P) { return P->dim >= 2 ? P->nx * (ny_of(P) + 1) * nz_of(P) : 0; }
static int nface_of(const or_problem* P) {
  return nxface_of(P) + nyface_of(P) + (P->dim == 3 ? P->nx * ny_of(P) * (nz_of(P) + 1) : 0);
}
static double vol_of(const or_problem* P) {
  return P->dx * (P->dim >= 2 ? P->dy : 1.0) * (P->dim == 3 ? P->dz : 1.0);
}
static int bc_of(const or_problem* P, int side) { return side < 4 ? P->bc[side] : P->bc_z[side - 4]; }
static double bcT_of(const or_problem* P, int side) { return side < 4 ? P->bcT[side] : P->bcT_z[side - 4]; }
static double h_of(const or_problem* P, int axis) { return axis == 0 ? P->dx : (axis == 1 ? P->dy : P->dz); }
/* area of a face normal to `axis` (1D: 1; 2D: the other cell width) */
static double area_of(const or_problem* P, int axis) {
  if (P->dim == 1) return 1.0;
  if (P->dim == 2) return axis == 0 ? P->dy : P->dx;
  return axis == 0 ? P->dy * P->dz : (axis == 1 ? P->dx * P->dz : P->dx * P->dy);
}
static int n_along(const or_problem* P, int axis) { return axis == 0 ? P->nx : (axis == 1 ? ny_of(P) : nz_of(P)); }
static int n_lines(const or_problem* P, int axis) { return ncell_of(P) / n_along(P, axis); }
static int line_cell(const or_problem* P, int axis, int line, int k) {
  const int nx = P->nx, ny = ny_of(P);
  if (axis == 0) return line * nx + k;
  if (axis == 1) return ((line / nx) * ny + k) * nx + line % nx;
  return k * nx * ny + line;
}
static int line_face(const or_problem* P, int axis, int line, int k) {
  const int nx = P->nx, ny = ny_of(P);
  if (axis == 0) return line * (nx + 1) + k;
  if (axis == 1) return nxface_of(P) + ((line / nx) * (ny + 1) + k) * nx + line % nx;
  return nxface_of(P) + nyface_of(P) + k * nx * ny + line;
}
static void cell_coords(const or_problem* P, int c, int* ix, int* iy, int* iz) {
  const int nx = P->nx, ny = ny_of(P);
  *ix = c % nx;
  *iy = (c / nx) % ny;
  *iz = c / (nx * ny);
}
/* the face of cell c on `axis`, lower (dir < 0) or upper side */
static int cell_face(const or_problem* P, int c, int axis, int dir) {
  int i[3];
  cell_coords(P, c, &i[0], &i[1], &i[2]);
  const int nx = P->nx;
  const int line = axis == 0 ? i[1] + ny_of(P) * i[2] : (axis == 1 ? i[0] + nx * i[2] : i[0] + nx * i[1]);
  return line_face(P, axis, line, i[axis] + (dir > 0 ? 1 : 0));
}

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers: Philox4x32-10 as published by Salmon,
 * Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
 * Each round multiplies lanes 0 and 2 by the two round multipliers, swaps
 * the high halves across and xors in the counter and the round key; the key
 * is bumped by the two Weyl constants between rounds.                       */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A uniform in (0,1) from two 32-bit words: the top 52 bits m, then
 * (m + 1/2) 2^-52, which is exact in binary64 and never 0 or 1, so ln u is
 * always finite.                                                            */
double or_uniform(uint32_t wa, uint32_t wb) {
  uint64_t m = ((uint64_t)wa << 20) | (uint64_t)(wb >> 12);
  return ((double)m + 0.5) * 0x1p-52;
}

/* Draw number j of particle `id` in time step `step`: Philox block j/2 of
 * counter (id_lo, id_hi, step, j/2) under key (seed_lo, seed_hi ^ instance);
 * even j uses words 0,1 and odd j words 2,3.                                */
double or_draw(const or_problem* P, uint64_t id, int64_t step, int64_t j) {
  uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)step, (uint32_t)(j >> 1)};
  uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32) ^ P->instance};
  uint32_t w[4];
  or_philox4x32_10(ctr, key, w);
  return (j & 1) ? or_uniform(w[2], w[3]) : or_uniform(w[0], w[1]);
}

/* ------------------------------------------------------------------------ */
/* Opacity.  The paper takes sigma_g^a = sigma_g^e = sigma_g(nu) (Sec. 2.1);
 * the tests use sigma(nu, T) = sigma0 nu^p T^q (Eq. sigmaMarsharkMF has
 * p = -3, q = -1/2), capped pointwise.  sig_law 1 adds the photo-ionisation
 * factor (1 - e^{-nu/T}) of the Larsen case (Sec. 3.3: gamma0 (1 -
 * e^{-h nu/kT})/(h nu)^3, i.e. p = -3, q = 0).  Particles use sigma at their
 * own frequency and the cell temperature.                                   */
/* sig_law 2: the carbon-hydrogen foam of the Olson case (Sec. 3.5),
 * sigma = rho kappa with sigma0 = rho and kappa in three frequency bands
 * (T and h nu in keV):
 *   h nu <= 0.008: min(1e7, 1e9 T^2);
 *   0.008 < h nu <= 0.3: 3e6 (0.008/h nu)^2 / (1 + 200 T^1.5);
 *   h nu > 0.3: the same times (0.3/h nu)^0.5, plus 4e4 (0.3/h nu)^2.5 / (1 + 8000 T^2). */
static double olson_kappa(double nu, double T) {
  if (nu <= 0.008) return fmin(1e7, 1e9 * T * T);
  const double a = 0.008 / nu;
  const double b = 3e6 * a * a / (1.0 + 200.0 * pow(T, 1.5));
  if (nu <= 0.3) return b;
  const double r = 0.3 / nu;
  return b * sqrt(r) + 4e4 * pow(r, 2.5) / (1.0 + 8000.0 * T * T);
}

double or_sigma(const or_problem* P, int c, double nu, double T) {
  double s;
  if (!P->grey && P->sig_law == 2) {
    s = P->sigma0[c] * olson_kappa(nu, T);
  } else {
    s = P->sigma0[c] * pow(T, P->sig_q);
    if (!P->grey) s *= pow(nu, P->sig_p);
    if (!P->grey && P->sig_law == 1) s *= -expm1(-nu / T);
  }
  if (P->sig_cap > 0.0 && !(s <= P->sig_cap)) s = P->sig_cap;
  return s;
}

/* Heat capacity and material energy per volume.  cv_law 0: e = cv T.
 * cv_law 1, the Olson foam (Eq. cvolson): rho C_v = K [1 + alpha + (T + chi)
 * alpha'], K = cv[c] (the a T_keV^3 H of the paper), with
 *   alpha = (1/2) e^{-chi/T} (sqrt(1 + 4 e^{chi/T}) - 1)
 *         = (1/2) (sqrt(u^2 + 4u) - u),  u = e^{-chi/T}   (no overflow as T -> 0),
 *   alpha' = (chi/T^2) (alpha - 1/sqrt(1 + 4 e^{chi/T})),
 * whose antiderivative vanishing at T = 0 is e(T) = K [T + (T + chi) alpha]
 * ((T + chi) alpha has derivative alpha + (T + chi) alpha', and alpha -> 0). */
static double olson_alpha(double chi, double T, double* dalpha) {
  const double u = exp(-chi / T);
  const double al = 0.5 * (sqrt(u * u + 4.0 * u) - u);
  if (dalpha) *dalpha = chi / (T * T) * (al - sqrt(u / (u + 4.0)));
  return al;
}

double or_mat_energy(const or_problem* P, int c, double T) {
  if (P->cv_law != 1) return P->cv[c] * T;
  return P->cv[c] * (T + (T + P->cv_chi) * olson_alpha(P->cv_chi, T, NULL));
}

double or_heat_capacity(const or_problem* P, int c, double T) {
  if (P->cv_law != 1) return P->cv[c];
  double da;
  const double al = olson_alpha(P->cv_chi, T, &da);
  return P->cv[c] * (1.0 + al + (T + P->cv_chi) * da);
}

/* Group opacity by Simpson's rule on nu_{g-1/2}, nu_mid, nu_{g+1/2}
 * (Sec. 3, numerical set-up), nu_mid the arithmetic midpoint (App. A).     */
double or_sigma_group(const or_problem* P, int c, int g, double T) {
  if (P->grey) return or_sigma(P, c, 0.0, T);
  double a = P->nu_edges[g], b = P->nu_edges[g + 1], m = 0.5 * (a + b);
  return (or_sigma(P, c, a, T) + 4.0 * or_sigma(P, c, m, T) + or_sigma(P, c, b, T)) / 6.0;
}

/* ------------------------------------------------------------------------ */
/* Planck group integrals.  B_g(T) is the integral of B(nu,T) over the group
 * (Sec. 2.1); its angle-integrated value is Phi_g(T) = a c T^4 b_g(T) with
 * b_g = (15/pi^4) int_{nu-/T}^{nu+/T} t^3/(e^t - 1) dt, so that the sum over
 * all frequencies is a c T^4.  Computed by adaptive 20-point Gauss-Legendre
 * quadrature with fixed breakpoints so no peak is missed.                   */
static double gl_x[20], gl_w[20];
static int gl_ready = 0;

static void gl_init(void) {
  const int n = 20;
  for (int i = 0; i < n; ++i) {
    long double z = cosl((long double)PI * (i + 0.75L) / (n + 0.5L)), z1, pp = 1.0L;
    for (int it = 0; it < 100; ++it) {
      long double p1 = 1.0L, p2 = 0.0L;
      for (int j = 1; j <= n; ++j) {
        long double p3 = p2;
        p2 = p1;
        p1 = ((2.0L * j - 1.0L) * z * p2 - (j - 1.0L) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0L);
      z1 = z;
      z = z1 - p1 / pp;
      if (fabsl(z - z1) <= 1e-17L) break;
    }
    gl_x[i] = (double)z;
    gl_w[i] = (double)(2.0L / ((1.0L - z * z) * pp * pp));
  }
  gl_ready = 1;
}

typedef double (*integrand_fn)(double);

static double gl_panel(integrand_fn f, double a, double b) {
  double m = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
  for (int i = 0; i < 20; ++i) s += gl_w[i] * f(m + h * gl_x[i]);
  return s * h;
}

/* Composite rule on n equal panels, n doubled until two successive values
 * agree to 1e-14; the finer one is then correct to rounding, since the
 * 20-point rule's error falls like h^40 on these analytic integrands.      */
static double gl_composite(integrand_fn f, double a, double b) {
  double prev = gl_panel(f, a, b);
  for (int n = 2; n <= 4096; n *= 2) {
    double h = (b - a) / n, s = 0.0;
    for (int i = 0; i < n; ++i) s += gl_panel(f, a + i * h, i == n - 1 ? b : a + (i + 1) * h);
    if (fabs(s - prev) <= 1e-14 * fabs(s)) return s;
    prev = s;
  }
  return prev;
}

static double integrate(integrand_fn f, double x1, double x2) {
  static const double brk[] = {0.25, 1.0, 2.0, 4.0, 8.0, 16.0, 32.0, 64.0, 128.0, 256.0, 800.0};
  if (!gl_ready) gl_init();
  if (!(x2 > x1)) return 0.0;
  double total = 0.0, a = x1;
  for (int i = 0; i < (int)(sizeof brk / sizeof brk[0]) && a < x2; ++i) {
    if (brk[i] <= a) continue;
    double b = brk[i] < x2 ? brk[i] : x2;
    total += gl_composite(f, a, b);
    a = b;
  }
  /* beyond t = 800 both integrands are below 1e-340: zero in binary64 */
  return total;
}

/* t^3/(e^t - 1), written with e^{-t} above t = 1 so that it does not overflow
 * to zero at t ~ 709.8 (which would truncate the tail of deep-Wien groups). */
static double planck_t3(double t) {
  if (t > 1.0) {
    double em = exp(-t);
    return t * t * t * em / (1.0 - em);
  }
  return t * t * t / expm1(t);
}

static double planck_t4(double t) {
  if (t > 1.0) {
    double em = exp(-t), d = 1.0 - em;
    return t * t * t * t * em / (d * d);
  }
  double d = expm1(t);
  return t * t * t * t * exp(t) / (d * d);
}

double or_planck_integral(double x1, double x2) { return PLANCK_NORM * integrate(planck_t3, x1, x2); }
double or_planck_dintegral(double x1, double x2) { return PLANCK_NORM * integrate(planck_t4, x1, x2); }

double or_phi(const or_problem* P, int g, double T) {
  if (!(T > 0.0)) return 0.0;
  double T4 = T * T * T * T;
  if (P->grey) return P->a * P->c * T4;
  return P->a * P->c * T4 * or_planck_integral(P->nu_edges[g] / T, P->nu_edges[g + 1] / T);
}

/* dPhi_g/dT = a c T^3 (15/pi^4) int t^4 e^t/(e^t-1)^2 dt over the same range
 * (differentiating the group integral of B(nu,T) under the integral sign). */
double or_dphi(const or_problem* P, int g, double T) {
  if (!(T > 0.0)) return 0.0;
  double T3 = T * T * T;
  if (P->grey) return 4.0 * P->a * P->c * T3;
  return P->a * P->c * T3 * or_planck_dintegral(P->nu_edges[g] / T, P->nu_edges[g + 1] / T);
}

/* ------------------------------------------------------------------------ */
/* Time-integrated flux coefficients, x = dt/tau, e = exp(-x):
 *   C2 / tau          = (2/x)(1-e) - 1 - e          (Eq. C2Formula)
 *   C4                = (1-e)/x                     (UGKS free flux, C4)
 *   C4 - e                                           (wave flux, Sec. 2.2)
 *   (C5 + dt e/2)/tau = e (1 + x/2) - (1-e)/x       (C5 = tau e - (tau^2/dt)(1-e))
 * The closed forms lose all digits as x -> 0, so below x = 1/2 the Taylor
 * series of the same functions is summed instead; both in long double.     */
void or_coefs(double x, double* f2, double* f4, double* f5, double* c4) {
  long double X = x;
  if (!(x > 0.0)) { *f2 = 0; *f4 = 0; *f5 = 0; *c4 = 1; return; }
  if (x < 0.5) {
    long double s2 = 0, s4 = 0, s5 = 0, c = 1, p = 1;   /* p = x^k, fact = (k+1)! */
    long double fact = 1, sgn = 1;
    for (int k = 1; k <= 60; ++k) {
      p *= X;
      fact *= (k + 1);
      sgn = -sgn;                          /* (-1)^k */
      long double t = p / fact;
      s2 += sgn * (1 - k) * t;             /* sum_{k>=2} (-1)^k (1-k) x^k/(k+1)! */
      s4 += -sgn * k * t;                  /* sum_{k>=1} (-1)^{k+1} k x^k/(k+1)! */
      s5 += sgn * k * (1 - k) * t / 2;     /* sum_{k>=2} (-1)^k k(1-k) x^k/(2 (k+1)!) */
      c += sgn * t;                        /* (1-e^{-x})/x = sum (-1)^k x^k/(k+1)! */
    }
    *f2 = (double)s2; *f4 = (double)s4; *f5 = (double)s5; *c4 = (double)c;
    return;
  }
  long double e = expl(-X), E1 = -expm1l(-X);
  *c4 = (double)(E1 / X);
  *f2 = (double)(2 * E1 / X - 1 - e);
  *f4 = (double)(E1 / X - e);
  *f5 = (double)(e * (1 + X / 2) - E1 / X);
}

/* ------------------------------------------------------------------------ */
/* Frequency of a particle (Remark on particle frequency, Eqs. Blinear, kg and
 * App. A).  Within group [nlo, nhi] the Planck shape is replaced by the line
 * B_mid + k (nu - nu_mid), k = (B(nhi) - B(nlo))/(nhi - nlo).  Readings: the
 * numerator of App. A's G has B_mid (nu - nu_lo) (the printed
 * B_mid (nhi - nlo) is a typo, as a, b, c of Eq. SquareEq confirm); k is
 * clamped to |k| <= 2 B_mid / (nhi - nlo) so the density is never negative.
 * B is only needed relative to B_mid; the ratio is taken in logarithms.     */
static double log_expm1(double z) { return z > 30.0 ? z + log1p(-exp(-z)) : log(expm1(z)); }

static double planck_ratio(double nu, double nmid, double T) {
  double l = 3.0 * log(nu / nmid) + log_expm1(nmid / T) - log_expm1(nu / T);
  if (l > 700.0) l = 700.0;
  return exp(l);
}

static double slope_hat(double nlo, double nhi, double T) {
  double dnu = nhi - nlo, nmid = 0.5 * (nlo + nhi);
  if (!(T > 0.0)) return 0.0;
  double k = (planck_ratio(nhi, nmid, T) - planck_ratio(nlo, nmid, T)) / dnu;
  double kmax = 2.0 / dnu;
  if (k > kmax) k = kmax;
  if (k < -kmax) k = -kmax;
  if (k != k) k = 0.0;
  return k;
}

/* G(nu): the cumulative distribution of Eq. Gformula under the line. */
double or_nu_cdf(double nlo, double nhi, double T, double nu) {
  double dnu = nhi - nlo, nmid = 0.5 * (nlo + nhi), k = slope_hat(nlo, nhi, T);
  double num = (nu - nlo) + 0.5 * k * ((nu - nmid) * (nu - nmid) - (nlo - nmid) * (nlo - nmid));
  return num / dnu;
}

/* G(nu) = eta, solved by bisection on the monotone CDF. */
double or_sample_nu(double nlo, double nhi, double T, double eta) {
  double lo = nlo, hi = nhi;
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (or_nu_cdf(nlo, nhi, T, mid) < eta) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------ */
/* Streaming of one particle (Algorithm 1 steps 3-5 with the t_f reset of the
 * interface remark).  Free time t_f = min(-tau ln eta, dt) (Eq. particle tf
 * formula) for a particle alive at step start; t_f = dt in the birth cell for
 * a newborn (Eq. IhpFormula samples collisionless particles only), except in
 * the UGKP variant (Sec. 2.2), whose newborns sample all of I^h and so draw
 * their t_f like every other particle (after their position, direction and
 * frequency draws; a black-body ghost's entering particles keep t_f = dt); on
 * entering a new cell t_f2 = min(-tau_new ln eta, dt - t_tra).  Trajectory
 * x = x^n + (c/eps) Omega t (Sec. 2.2).  Readings: a face is crossed only if
 * the time to reach it is strictly below the remaining free time; at a
 * reflecting wall the direction flips and t_f is not reset; a particle that
 * leaves through a vacuum or black-body side escapes; a particle born in a
 * black-body ghost cell that does not reach the domain is removed; on a tie
 * between faces of different axes the lower axis (x, then y, then z) is
 * taken first.  Energy crossing
 * faces is tallied as in Eq. wfrpFormula (in minus out).                    */
static double draw_j(const or_problem* P, uint64_t id, int64_t step, int64_t j,
                     const double* draws, int64_t n_draws, int* bad) {
  if (draws) {
    if (j >= n_draws) { *bad = 1; return 0.5; }
    return draws[j];
  }
  return or_draw(P, id, step, j);
}

int or_stream_particle3(const or_problem* P, const double* T, int64_t step,
                        double* px, double* py, double* pz, double* pox, double* poy, double* poz,
                        double nu, double w, uint64_t id, int32_t* pcell, int32_t g,
                        int newborn, int64_t first_draw,
                        const double* draws, int64_t n_draws,
                        or_tallies* tal, int32_t* nseg_out, double* t_end,
                        double* trace_x, double* trace_t, int trace_cap, int* n_trace) {
  const int nx = P->nx, ny = ny_of(P), nz = nz_of(P), G = P->G;
  const double v = P->c / P->eps, dt = P->dt;
  const double inv_rate = P->eps * P->eps / P->c;   /* tau = eps^2/(c sigma) */
  double p[3] = {*px, *py, *pz}, o[3] = {*pox, *poy, *poz};
  const double h[3] = {P->dx, P->dy, P->dz};
  const int n[3] = {nx, ny, nz};
  int cell = *pcell;
  int ic[3] = {0, 0, 0};
  if (P->dim == 1) ic[0] = cell;
  else cell_coords(P, cell, &ic[0], &ic[1], &ic[2]);
  int ghost = (P->dim == 1) && (cell < 0 || cell >= nx);
  int ghost_side = (cell < 0) ? 0 : 1;
  int bad = 0, nseg = 0, fate;
  int64_t j = first_draw;
  double t_tra = 0.0, t_rem;
  int collided;
  if (n_trace) *n_trace = 0;

  if (newborn && (P->method != OR_UGKP || ghost)) {
    t_rem = dt;
    collided = 0;
  } else {
    double u = draw_j(P, id, step, j++, draws, n_draws, &bad);
    double tc = -log(u) * inv_rate / or_sigma(P, cell, nu, T[cell]);
    collided = tc < dt;
    t_rem = collided ? tc : dt;
  }

  for (;;) {
    /* time to the nearest face along each axis; ties go to the lower axis */
    int axis = 0;
    double tf = INFINITY;
    for (int a = 0; a < P->dim; ++a) {
      const double lo = ic[a] * h[a], hi = (ic[a] + 1) * h[a];
      double ta = INFINITY;
      if (o[a] > 0) ta = fmax(hi - p[a], 0.0) / (v * o[a]);
      else if (o[a] < 0) ta = fmax(p[a] - lo, 0.0) / (v * -o[a]);
      if (a == 0 || ta < tf) { tf = ta; axis = a; }
    }
    if (tf < t_rem) {
      ++nseg;
      t_tra += tf;
      t_rem -= tf;
      const int dir = o[axis] > 0 ? 1 : -1;
      for (int a = 0; a < 3; ++a) {
        if (a == axis) p[a] = dir > 0 ? (ic[a] + 1) * h[a] : ic[a] * h[a];
        else if (a < P->dim || a == 1) p[a] += v * o[a] * tf;
      }
      if (trace_x && n_trace && *n_trace < trace_cap) { trace_x[*n_trace] = p[0]; trace_t[*n_trace] = t_tra; ++*n_trace; }
      int ni[3] = {ic[0], ic[1], ic[2]};
      ni[axis] += dir;
      const int outside = ni[axis] < 0 || ni[axis] >= n[axis];
      if (outside) {
        const int side = axis * 2 + (dir > 0 ? 1 : 0);
        if (bc_of(P, side) == OR_BC_REFLECT) {
          o[axis] = -o[axis];
          continue;
        }
        if (tal) {
          tal->esc[side * G + g] += w;
          tal->W[cell * G + g] -= w;
        }
        fate = OR_ESCAPED;
        break;
      }
      const int ncell = (ni[2] * ny + ni[1]) * nx + ni[0];
      if (tal) {
        if (ghost) tal->inflow[ghost_side * G + g] += w;
        else tal->W[cell * G + g] -= w;
        tal->W[ncell * G + g] += w;
      }
      ghost = 0;
      cell = ncell;
      ic[0] = ni[0]; ic[1] = ni[1]; ic[2] = ni[2];
      double u = draw_j(P, id, step, j++, draws, n_draws, &bad);
      double tc = -log(u) * inv_rate / or_sigma(P, cell, nu, T[cell]);
      double avail = dt - t_tra;
      collided = tc < avail;
      t_rem = collided ? tc : avail;
      continue;
    }
    ++nseg;
    p[0] += v * o[0] * t_rem;
    p[1] += v * o[1] * t_rem;
    if (P->dim == 3) p[2] += v * o[2] * t_rem;
    t_tra += t_rem;
    t_rem = 0.0;
    if (trace_x && n_trace && *n_trace < trace_cap) { trace_x[*n_trace] = p[0]; trace_t[*n_trace] = t_tra; ++*n_trace; }
    if (ghost) fate = OR_REMOVED;
    else if (collided) { fate = OR_ABSORBED; if (tal) tal->E_abs[cell * G + g] += w; }
    else { fate = OR_SURVIVED; if (tal) tal->E_surv[cell * G + g] += w; }
    break;
  }
  *px = p[0]; *py = p[1]; *pz = p[2]; *pox = o[0]; *poy = o[1]; *poz = o[2]; *pcell = cell;
  if (nseg_out) *nseg_out = nseg;
  if (t_end) *t_end = t_tra;
  return bad ? -1 : fate;
}

int or_stream_particle(const or_problem* P, const double* T, int64_t step,
                       double* px, double* py, double* pox, double* poy, double nu,
                       double w, uint64_t id, int32_t* pcell, int32_t g,
                       int newborn, int64_t first_draw,
                       const double* draws, int64_t n_draws,
                       or_tallies* tal, int32_t* nseg_out, double* t_end,
                       double* trace_x, double* trace_t, int trace_cap, int* n_trace) {
  double z = 0.0, oz = 0.0;
  return or_stream_particle3(P, T, step, px, py, &z, pox, poy, &oz, nu, w, id, pcell, g, newborn, first_draw,
                             draws, n_draws, tal, nseg_out, t_end, trace_x, trace_t, trace_cap, n_trace);
}

/* ------------------------------------------------------------------------ */
/* Birth counts (Eq. IhpFormula and the weight formula of Sec. 2.2): the
 * collisionless part of the wave, E = e^{-dt/tau} max(rho_h, 0) V, is carried
 * by N = floor(E/omega_ref + 1/2) particles of energy E/N (omega_ref the
 * reference weight of Sec. 3).  tau from the Simpson group opacity at T^n.
 * N = 0 gives e_eff = 0, so the wave flux falls back to the UGKS flux (the
 * remark on unsampled particles).  Black-body sides in 1D have a ghost cell
 * at T_b holding rho_h = Phi_g(T_b); of its collisionless particles only
 * those that reach the wall within dt matter, and they carry
 * E = e (c/eps)/4 Phi_g(T_b) dt through the wall (the half-range flux of an
 * isotropic ghost).  They are sampled directly (see or_step).  Bins are
 * ordered interior cells (c*G + g) then ghosts ((ncell + side)*G + g).
 * UGKP variant (Sec. 2.2, the specific intensity fully represented by
 * particles): an interior bin samples all of its wave part, E = max(rho_h, 0)
 * V, and marks it with e_eff = -1 (the wave flux then carries none of it);
 * black-body ghosts are sampled as in UGKWP.                                 */
/* Numerical collision time for the thin/thick joint (Sec. 3.2, heterogeneous
 * cases): tau_num = tau + C (T^l - T^r)/(T^l + T^r) dt is written per
 * interface.  Readings: the magnitude of the temperature contrast (the stated
 * aim is more sampled particles, tau_num >= tau), and a cell takes the
 * largest contrast over its interior faces.  Returns dt/tau_num =
 * x/(1 + C J x) with x = dt/tau. */
double or_x_num(const or_problem* P, const double* T, int c, int g) {
  const double rate_f = P->c / (P->eps * P->eps);
  const double x = P->dt * rate_f * or_sigma_group(P, c, g, T[c]);
  if (!(P->tau_num_C > 0.0)) return x;
  const int nx = P->nx, ny = ny_of(P), nz = nz_of(P);
  int ix, iy, iz;
  cell_coords(P, c, &ix, &iy, &iz);
  double J = 0.0;
  const int nb[6][3] = {{ix - 1, iy, iz}, {ix + 1, iy, iz}, {ix, iy - 1, iz},
                        {ix, iy + 1, iz}, {ix, iy, iz - 1}, {ix, iy, iz + 1}};
  for (int k = 0; k < 2 * P->dim; ++k) {
    const int jx = nb[k][0], jy = nb[k][1], jz = nb[k][2];
    if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
    const double Tn = T[(jz * ny + jy) * nx + jx];
    const double j = fabs(T[c] - Tn) / (T[c] + Tn);
    if (j > J) J = j;
  }
  return x / (1.0 + P->tau_num_C * J * x);
}

int or_birth_counts(const or_problem* P, const double* T, const double* rho_h,
                    or_tallies* tal, int64_t* n_new) {
  const int ncell = ncell_of(P), G = P->G, nbins = (ncell + 4) * G;
  const double V = vol_of(P), rate_f = P->c / (P->eps * P->eps);
  int64_t total = 0;
  int status = OR_OK;
  for (int b = 0; b < nbins; ++b) { tal->N[b] = 0; tal->omega[b] = 0.0; tal->e_eff[b] = 0.0; }
  for (int b = 0; b < nbins; ++b) {
    int cell = b / G, g = b % G;
    double Tb, E;
    int src_cell;
    if (cell < ncell) {
      src_cell = cell;
      Tb = T[cell];
      double rh = rho_h[b] > 0.0 ? rho_h[b] : 0.0;
      E = rh * V;
    } else {
      int side = cell - ncell;
      if (P->dim != 1 || side > 1 || P->bc[side] != OR_BC_BLACKBODY) continue;
      src_cell = side == 0 ? 0 : P->nx - 1;
      Tb = P->bcT[side];
      E = 0.25 * (P->c / P->eps) * or_phi(P, g, Tb) * P->dt;
    }
    double x;
    if (cell < ncell) x = or_x_num(P, T, cell, g);
    else x = P->dt * rate_f * or_sigma_group(P, src_cell, g, Tb);
    double e = exp(-x);
    const int all = P->method == OR_UGKP && cell < ncell;   /* UGKP: the whole wave part */
    if (!all) E *= e;
    if (!(P->omega_ref > 0.0) || !(E > 0.0)) continue;
    double q = floor(E / P->omega_ref + 0.5);
    if (q > (double)MAX_K_PER_BIN) { status = OR_ERR_CAPACITY; q = MAX_K_PER_BIN; }
    int N = (int)q;
    tal->N[b] = N;
    if (N > 0) { tal->omega[b] = E / N; tal->e_eff[b] = all ? -1.0 : e; }
    total += N;
  }
  *n_new = total;
  return status;
}

/* ------------------------------------------------------------------------ */
/* Wave-part free-transport flux (Sec. 2.2):
 *   F^{fr,wave} = int (c/eps) Omega.n [ (C4 - e) I^h + (C5 + dt e/2) (c/eps) Omega.grad I^h ] dOmega.
 * Readings: F^{fr,UGKS} takes its coefficients C4, C5 from the face opacity
 * (harmonic mean of the two sides' group opacities at T^n, as App. B does for
 * C2), so a uniform Planck field carries no flux across an opacity jump; the
 * subtracted DVM flux of the sampled part uses the sampled fraction e of the
 * upwind cell (e = 0 where no particle was sampled, the remark on unsampled
 * particles).  Half-range integrals: the outward half of each side uses that
 * side's I^h; for isotropic I^h = rho_h/2 (1D) or rho_h/4pi (2D) the moments
 * give (c/eps)/4 and (c/eps)^2/6.  wave_order 2 evaluates I^h on the face
 * from a van Leer limited linear reconstruction and uses the upwind cell's
 * slope as the gradient (the second-order statement opening the construction
 * of the equilibrium part); wave_order 1 uses cell averages and the central
 * difference across the face.  Reflecting walls carry no flux; a black-body
 * ghost holds rho_h = Phi_g(T_b) at opacity sigma_g(T_b), a vacuum ghost
 * rho_h = 0 at the inner cell's opacity.                                    */
static double van_leer(double dl, double dr) {
  return dl * dr > 0.0 ? 2.0 * dl * dr / (dl + dr) : 0.0;
}

/* Coefficients of one half: A = C4_f - e_h, B = C5_f + dt e_h/2, where
 * e_h = exp(-x_h) of the upwind cell (or 0), written without cancellation;
 * A = B = 0 for a half whose whole wave part was sampled (UGKP, e_eff < 0). */
static void half_coefs(double x_f, double tau_f, double x_h, double e_eff, double dt,
                       double* A, double* B) {
  double f2, f4, f5, c4;
  or_coefs(x_f, &f2, &f4, &f5, &c4);
  if (e_eff < 0.0) {
    /* UGKP: the particles carry the whole free transport F^{fr,UGKS}(I^h) of
     * this half, so the wave part contributes nothing */
    *A = 0.0;
    *B = 0.0;
  } else if (e_eff > 0.0) {
    /* e_f - e_h, without cancellation when x_h ~ x_f and without overflow */
    double d = x_h - x_f;
    double ef_minus_eh = fabs(d) < 0.5 ? exp(-x_h) * expm1(d) : exp(-x_f) - exp(-x_h);
    *A = f4 + ef_minus_eh;
    *B = tau_f * f5 - 0.5 * dt * ef_minus_eh;
  } else {
    *A = c4;
    *B = -tau_f * f4;
  }
}

int or_wave_flux(const or_problem* P, const double* T, const double* rho_h,
                 const double* e_eff, double* Fwave) {
  const int G = P->G, ncell = ncell_of(P);
  const double v = P->c / P->eps, rate_f = P->c / (P->eps * P->eps), dt = P->dt;
  for (int axis = 0; axis < P->dim; ++axis) {
    const double h = h_of(P, axis);
    const int nk = n_along(P, axis);                   /* cells along the axis */
    const int nlines = n_lines(P, axis);
    const int sideL = axis * 2, sideR = axis * 2 + 1;
    for (int line = 0; line < nlines; ++line) {
      for (int f = 0; f <= nk; ++f) {
        int fidx = line_face(P, axis, line, f);
        for (int g = 0; g < G; ++g) {
#define CELL_AT(k) line_cell(P, axis, line, (k))
          int kL = f - 1, kR = f;
          int lin = kL >= 0, rin = kR < nk;
          if ((!lin && bc_of(P, sideL) == OR_BC_REFLECT) || (!rin && bc_of(P, sideR) == OR_BC_REFLECT)) {
            Fwave[fidx * G + g] = 0.0;
            continue;
          }
          /* rho_h at line index k, ghosts included */
#define RHO_AT(k, out) do {                                                          \
            int kk_ = (k);                                                           \
            if (kk_ >= 0 && kk_ < nk) out = rho_h[CELL_AT(kk_) * G + g];            \
            else {                                                                   \
              int s_ = kk_ < 0 ? sideL : sideR;                                      \
              int kin_ = kk_ < 0 ? 0 : nk - 1;                                       \
              if (bc_of(P, s_) == OR_BC_REFLECT) out = rho_h[CELL_AT(kin_) * G + g];  \
              else if (bc_of(P, s_) == OR_BC_BLACKBODY) out = or_phi(P, g, bcT_of(P, s_)); \
              else out = 0.0;                                                        \
            }                                                                        \
          } while (0)
          double rl, rr, rll, rrr, sl, sr, fl, fr;
          RHO_AT(kL, rl); RHO_AT(kR, rr);
          if (P->wave_order >= 2) {
            RHO_AT(kL - 1, rll); RHO_AT(kR + 1, rrr);
            sl = lin ? van_leer((rl - rll) / h, (rr - rl) / h) : 0.0;
            sr = rin ? van_leer((rr - rl) / h, (rrr - rr) / h) : 0.0;
            fl = rl + 0.5 * h * sl;
            fr = rr - 0.5 * h * sr;
          } else {
            sl = sr = (rr - rl) / h;
            fl = rl; fr = rr;
          }
#undef RHO_AT
          /* side opacities and sampled fractions */
          double sgl, sgr, el, er, xhl = 0.0, xhr = 0.0;
          if (lin) {
            sgl = or_sigma_group(P, CELL_AT(kL), g, T[CELL_AT(kL)]); el = e_eff[CELL_AT(kL) * G + g];
            xhl = or_x_num(P, T, CELL_AT(kL), g);
          } else if (bc_of(P, sideL) == OR_BC_BLACKBODY) {
            sgl = or_sigma_group(P, CELL_AT(0), g, bcT_of(P, sideL)); el = e_eff[(ncell + sideL) * G + g];
            xhl = dt * rate_f * sgl;
          } else { sgl = -1.0; el = 0.0; }
          if (rin) {
            sgr = or_sigma_group(P, CELL_AT(kR), g, T[CELL_AT(kR)]); er = e_eff[CELL_AT(kR) * G + g];
            xhr = or_x_num(P, T, CELL_AT(kR), g);
          } else if (bc_of(P, sideR) == OR_BC_BLACKBODY) {
            sgr = or_sigma_group(P, CELL_AT(nk - 1), g, bcT_of(P, sideR)); er = e_eff[(ncell + sideR) * G + g];
            xhr = dt * rate_f * sgr;
          } else { sgr = -1.0; er = 0.0; }
          if (sgl < 0.0) sgl = sgr;          /* vacuum ghost: inner opacity */
          if (sgr < 0.0) sgr = sgl;
#undef CELL_AT
          double sf = 2.0 * sgl * sgr / (sgl + sgr);
          double tau_f = 1.0 / (rate_f * sf);
          double x_f = dt / tau_f;
          double AL, BL, AR, BR;
          half_coefs(x_f, tau_f, xhl, el, dt, &AL, &BL);
          half_coefs(x_f, tau_f, xhr, er, dt, &AR, &BR);
          Fwave[fidx * G + g] = AL * (v / 4.0) * fl - AR * (v / 4.0) * fr
                              + (BL * sl + BR * sr) * (v * v / 6.0);
        }
      }
    }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Source iteration for Eq. macroSysFinal (App. B, Eq. macroSysAppendixIte and
 * Algorithm 2), in 1D and 2D.  Each iterate k:
 *   sigma^k, Phi^k = Phi_g(T^k) from T^k;
 *   F^eq on every face = C2 (c/eps)^2 (1/3) (Phi_R - Phi_L)/h with C2 from the
 *   harmonic-mean face opacity (App. B) -- the K_g B_i - M_g term, both
 *   neighbours and the cell itself at iterate k (Jacobi);
 *   rho^{k+1}, T^{k+1} from the two equations with the emission linearised,
 *   Phi_g(T^{k+1}) ~ Phi^k + Phi'^k (T^{k+1} - T^k) (reading: the literal
 *   update of T from the lagged emission diverges when
 *   sum_g dt sigma_g Phi'_g / (Cv (1 + c dt sigma_g)) > 1, as it is for
 *   a = c = Cv = 1 and T ~ 1; the fixed point is the same).
 * With a_g = c dt sigma_g/eps^2 the two equations give the closed form
 *   T^{k+1} = [Cv T^n + sum_g (a_g/c)(Q_g - Phi_g + Phi'_g T^k)/(1 + a_g)]
 *           / [Cv + sum_g (a_g/c) Phi'_g/(1 + a_g)],
 *   rho_g^{k+1} = (Q_g + a_g (Phi_g + Phi'_g (T^{k+1} - T^k)))/(1 + a_g),
 * Q_g = R_g + (dt/h)(F^eq_in - F^eq_out).  In 1D the paper's "2 B_g" and in
 * 3D "4 pi B_g" are both Phi_g.  Stopping rule (Algorithm 2, tolerances
 * unstated): max over cells of |dT|/T and of max_g |d rho_g| / sum_g |rho_g|
 * both <= si_tol.                                                           */
int or_source_iteration(const or_problem* P, const double* T_n, const double* rho_n,
                        const double* R, double* T_out, double* rho_out,
                        double* Feq_out, int* iters) {
  const int G = P->G, ncell = ncell_of(P);
  const int nface = nface_of(P);
  const double v = P->c / P->eps, dt = P->dt;
  const double rate_f = P->c / (P->eps * P->eps);
  double* Tk = malloc(sizeof(double) * ncell);
  double* rk = malloc(sizeof(double) * ncell * G);
  double* sig = malloc(sizeof(double) * ncell * G);
  double* phi = malloc(sizeof(double) * ncell * G);
  double* dphi = malloc(sizeof(double) * ncell * G);
  double* Feq = Feq_out ? Feq_out : malloc(sizeof(double) * nface * G);
  int status = OR_ERR_NOCONV, k;
  memcpy(Tk, T_n, sizeof(double) * ncell);
  memcpy(rk, rho_n, sizeof(double) * ncell * G);
  for (k = 0; k < P->si_max_iters; ++k) {
    for (int c = 0; c < ncell; ++c)
      for (int g = 0; g < G; ++g) {
        sig[c * G + g] = or_sigma_group(P, c, g, Tk[c]);
        phi[c * G + g] = or_phi(P, g, Tk[c]);
        dphi[c * G + g] = or_dphi(P, g, Tk[c]);
      }
    /* equilibrium flux on every face */
    for (int axis = 0; axis < P->dim; ++axis) {
      const double h = h_of(P, axis);
      const int nk = n_along(P, axis), nlines = n_lines(P, axis);
      for (int line = 0; line < nlines; ++line)
        for (int f = 0; f <= nk; ++f) {
          int fidx = line_face(P, axis, line, f);
          for (int g = 0; g < G; ++g) {
            int cl = f - 1 >= 0 ? line_cell(P, axis, line, f - 1) : -1;
            int cr = f < nk ? line_cell(P, axis, line, f) : -1;
            double sl, sr, pl, pr;
            if (cl < 0 || cr < 0) {
              int side = axis * 2 + (cl < 0 ? 0 : 1);
              int cin = cl < 0 ? cr : cl;
              if (bc_of(P, side) == OR_BC_REFLECT) { Feq[fidx * G + g] = 0.0; continue; }
              double sg, pg;
              if (bc_of(P, side) == OR_BC_BLACKBODY) {
                sg = or_sigma_group(P, cin, g, bcT_of(P, side));
                pg = or_phi(P, g, bcT_of(P, side));
              } else { sg = sig[cin * G + g]; pg = 0.0; }
              if (cl < 0) { sl = sg; pl = pg; sr = sig[cr * G + g]; pr = phi[cr * G + g]; }
              else        { sr = sg; pr = pg; sl = sig[cl * G + g]; pl = phi[cl * G + g]; }
            } else {
              sl = sig[cl * G + g]; sr = sig[cr * G + g];
              pl = phi[cl * G + g]; pr = phi[cr * G + g];
            }
            double sf = 2.0 * sl * sr / (sl + sr);
            double tau = 1.0 / (rate_f * sf);
            double f2, f4, f5, c4;
            or_coefs(dt / tau, &f2, &f4, &f5, &c4);
            Feq[fidx * G + g] = tau * f2 * (v * v / 3.0) * (pr - pl) / h;
          }
        }
    }
    /* per-cell linearised update */
    double errT = 0.0, errR = 0.0;
    for (int c = 0; c < ncell; ++c) {
      /* e(T^{k+1}) ~ e(T^k) + C_v(T^k) (T^{k+1} - T^k) for a T-dependent heat
       * capacity (the same fixed point); cv_law 0 is the constant case */
      double num, den;
      if (P->cv_law == 1) {
        const double cvk = or_heat_capacity(P, c, Tk[c]);
        num = or_mat_energy(P, c, T_n[c]) - or_mat_energy(P, c, Tk[c]) + cvk * Tk[c];
        den = cvk;
      } else {
        num = P->cv[c] * T_n[c];
        den = P->cv[c];
      }
      double Q[256];
      double a[256];
      for (int g = 0; g < G; ++g) {
        double q = R[c * G + g];
        for (int axis = 0; axis < P->dim; ++axis) {
          const int fl = cell_face(P, c, axis, -1), fu = cell_face(P, c, axis, +1);
          q += (dt / h_of(P, axis)) * (Feq[fl * G + g] - Feq[fu * G + g]);
        }
        Q[g] = q;
        a[g] = dt * rate_f * sig[c * G + g];
        double ap = a[g] / P->c / (1.0 + a[g]);
        num += ap * (q - phi[c * G + g] + dphi[c * G + g] * Tk[c]);
        den += ap * dphi[c * G + g];
      }
      double Tnew = num / den;
      if (!(Tnew > 1e-30)) Tnew = 1e-30;
      double dmax = 0.0, rsum = 0.0;
      for (int g = 0; g < G; ++g) {
        double r = (Q[g] + a[g] * (phi[c * G + g] + dphi[c * G + g] * (Tnew - Tk[c]))) / (1.0 + a[g]);
        double d = fabs(r - rk[c * G + g]);
        if (d > dmax) dmax = d;
        rsum += fabs(r);
        rk[c * G + g] = r;
      }
      double eT = fabs(Tnew - Tk[c]) / Tnew;
      if (eT > errT) errT = eT;
      double eR = rsum > 0.0 ? dmax / rsum : 0.0;
      if (eR > errR) errR = eR;
      T_out[c] = Tnew;
    }
    memcpy(Tk, T_out, sizeof(double) * ncell);
    if (!(errT == errT) || !(errR == errR)) { status = OR_ERR_NONFINITE; ++k; break; }
    if (errT <= P->si_tol && errR <= P->si_tol) { status = OR_OK; ++k; break; }
  }
  memcpy(rho_out, rk, sizeof(double) * ncell * G);
  memcpy(T_out, Tk, sizeof(double) * ncell);
  *iters = k;
  free(Tk); free(rk); free(sig); free(phi); free(dphi);
  if (!Feq_out) free(Feq);
  return status;
}

/* ------------------------------------------------------------------------ */
void or_init_rho(const or_problem* P, const double* T0, double* rho) {
  const int ncell = ncell_of(P), G = P->G;
  for (int c = 0; c < ncell; ++c)
    for (int g = 0; g < G; ++g) rho[c * G + g] = or_phi(P, g, T0[c]);
}

/* One UGKWP time step, in the order of Algorithm 1:
 *   t_f for remaining particles, sampling of new collisionless particles,
 *   streaming with tallies, source iteration for Eq. macroSysFinal,
 *   removal of collided particles, then the wave/particle split
 *   I^h = I^{n+1} - I^p (Sec. 2.2).  The source of a patch cell adds
 *   src_on amp c dt Phi_g(T_s) to rho_g each step while t^n < src_t_end
 *   (reading for the Olson-type source, Q = B(T_s) e^{-693 x^3} for ct <= 2:
 *   amp the profile at the cell centre).                                    */
int or_step(const or_problem* P, int64_t step,
            const double* T, const double* rho, const double* rho_h,
            int64_t n_in, const or_particles* pin,
            double* T_out, double* rho_out, double* rho_h_out, double* rho_p_out,
            or_particles* pout, int64_t cap_out, int64_t* n_out,
            or_record* rec, int64_t rec_cap,
            or_tallies* tal) {
  return or_step_core(P, step, T, rho, rho_h, n_in, pin, T_out, rho_out, rho_h_out, rho_p_out,
                      pout, cap_out, n_out, rec, rec_cap, tal, NULL, NULL, NULL, NULL, NULL);
}

/* A particle streamed a second time from the same start (same identity,
 * step and draws, hence the same path) carrying another weight into another
 * set of tallies. */
static void restream(const or_problem* P, const double* T, int64_t step, double x, double y,
                     double ox, double oy, double nu, double w, uint64_t id, int32_t cell,
                     int32_t g, int newborn, int64_t first_draw, or_tallies* tal) {
  int32_t nseg;
  double tend;
  or_stream_particle(P, T, step, &x, &y, &ox, &oy, nu, w, id, &cell, g, newborn, first_draw,
                     NULL, 0, tal, &nseg, &tend, NULL, NULL, 0, NULL);
}

int or_step_core(const or_problem* P, int64_t step,
                 const double* T, const double* rho, const double* rho_h,
                 int64_t n_in, const or_particles* pin,
                 double* T_out, double* rho_out, double* rho_h_out, double* rho_p_out,
                 or_particles* pout, int64_t cap_out, int64_t* n_out,
                 or_record* rec, int64_t rec_cap,
                 or_tallies* tal,
                 const double* w2_in, const double* w2_bins, double* w2_out, or_tallies* tal2,
                 double* w2_scale) {
  const int nx = P->nx, G = P->G, ncell = ncell_of(P);
  const int nface = nface_of(P);
  const double V = vol_of(P), dt = P->dt;
  int status = OR_OK;
  if (P->dim < 1 || P->dim > 3) return OR_ERR_ARG;
  if (G < 1 || G > 256 || (P->grey && G != 1)) return OR_ERR_ARG;
  if (P->dim >= 2)
    for (int s = 0; s < 2 * P->dim; ++s)
      if (bc_of(P, s) == OR_BC_BLACKBODY) return OR_ERR_ARG;

  memset(tal->W, 0, sizeof(double) * ncell * G);
  memset(tal->E_surv, 0, sizeof(double) * ncell * G);
  memset(tal->E_abs, 0, sizeof(double) * ncell * G);
  memset(tal->esc, 0, sizeof(double) * 6 * G);
  memset(tal->inflow, 0, sizeof(double) * 6 * G);
  tal->n_in = n_in;
  tal->n_born = tal->n_survived = tal->n_absorbed = tal->n_escaped = tal->n_removed = 0;
  tal->n_segments = 0;

  /* energy before */
  tal->E_rad0 = tal->E_mat0 = 0.0;
  for (int c = 0; c < ncell; ++c) {
    for (int g = 0; g < G; ++g) tal->E_rad0 += V * rho[c * G + g] / P->c;
    tal->E_mat0 += V * or_mat_energy(P, c, T[c]);
  }

  /* steps 2: birth counts from the wave part at t^n */
  int64_t n_new = 0;
  int st = or_birth_counts(P, T, rho_h, tal, &n_new);
  if (st) status = st;
  if (step > OR_MAX_STEP) {   /* identities exhausted: nothing is sampled */
    for (int b = 0; b < (ncell + 4) * G; ++b) { tal->N[b] = 0; tal->omega[b] = 0.0; tal->e_eff[b] = 0.0; }
    n_new = 0;
    status = OR_ERR_IDSPACE;
  }
  tal->n_born = n_new;

  /* steps 1, 3: remaining particles, then newborns */
  int64_t nrec = 0, nout = 0;
  for (int64_t i = 0; i < n_in; ++i) {
    double x = pin->x[i], y = pin->y[i], ox = pin->ox[i], oy = pin->oy[i];
    double z = pin->z ? pin->z[i] : 0.0, oz = pin->oz ? pin->oz[i] : 0.0;
    int32_t cell = pin->cell[i], cell0 = cell, nseg;
    double tend;
    if (tal2)
      restream(P, T, step, x, y, ox, oy, pin->nu[i], w2_in[i], pin->id[i], cell, pin->grp[i], 0, 0, tal2);
    int fate = or_stream_particle3(P, T, step, &x, &y, &z, &ox, &oy, &oz, pin->nu[i], pin->w[i], pin->id[i],
                                   &cell, pin->grp[i], 0, 0, NULL, 0, tal, &nseg, &tend,
                                   NULL, NULL, 0, NULL);
    tal->n_segments += nseg;
    if (fate == OR_SURVIVED) {
      ++tal->n_survived;
      if (nout < cap_out) {
        pout->x[nout] = x; pout->y[nout] = y; pout->ox[nout] = ox; pout->oy[nout] = oy;
        if (pout->z) { pout->z[nout] = z; pout->oz[nout] = oz; }
        pout->nu[nout] = pin->nu[i]; pout->w[nout] = pin->w[i]; pout->id[nout] = pin->id[i];
        pout->cell[nout] = cell; pout->grp[nout] = pin->grp[i];
        if (w2_out) w2_out[nout] = w2_in[i];
      } else status = OR_ERR_CAPACITY;
      ++nout;
    } else if (fate == OR_ABSORBED) ++tal->n_absorbed;
    else if (fate == OR_ESCAPED) ++tal->n_escaped;
    else ++tal->n_removed;
    if (rec && nrec < rec_cap) {
      or_record* r = &rec[nrec];
      r->id = pin->id[i]; r->fate = fate; r->cell0 = cell0; r->cell1 = cell; r->grp = pin->grp[i];
      r->nseg = nseg; r->_pad = 0; r->x = x; r->y = y; r->ox = ox; r->oy = oy; r->nu = pin->nu[i];
      r->w = pin->w[i]; r->t_end = tend; r->z = z; r->oz = oz;
    }
    ++nrec;
  }
  const int nbins = (ncell + 4) * G;
  for (int b = 0; b < nbins; ++b) {
    int bc_cell = b / G, g = b % G;
    for (int k = 0; k < tal->N[b]; ++k) {
      uint64_t id = ((uint64_t)step << 44) | ((uint64_t)b << 20) | (uint64_t)k;
      int64_t j = 0;
      double x, y = 0.0, z = 0.0, ox, oy = 0.0, oz = 0.0, nu = 0.0, Tb;
      int32_t cell;
      if (bc_cell < ncell) {
        int ix, iy, iz;
        cell_coords(P, bc_cell, &ix, &iy, &iz);
        x = ix * P->dx + or_draw(P, id, step, j++) * P->dx;
        if (P->dim >= 2) y = iy * P->dy + or_draw(P, id, step, j++) * P->dy;
        if (P->dim == 3) z = iz * P->dz + or_draw(P, id, step, j++) * P->dz;
        if (P->dim == 1) {
          ox = 2.0 * or_draw(P, id, step, j++) - 1.0;
        } else {
          /* 3D isotropic directions (2D keeps their x and y components) */
          double muz = 2.0 * or_draw(P, id, step, j++) - 1.0;
          double phi = 2.0 * PI * or_draw(P, id, step, j++);
          double s = sqrt(fmax(0.0, 1.0 - muz * muz));
          ox = s * cos(phi);
          oy = s * sin(phi);
          if (P->dim == 3) oz = muz;
        }
        cell = bc_cell;
        Tb = T[bc_cell];
      } else {
        /* A collisionless ghost particle (uniform in the ghost cell, isotropic
         * inward) reaches the wall within dt iff its distance d < v mu dt.
         * Restricted to those, mu has density 2 mu on (0,1) and d is uniform
         * on (0, v mu dt): sample exactly that set.                          */
        int side = bc_cell - ncell;
        double u = or_draw(P, id, step, j++);
        double m = sqrt(or_draw(P, id, step, j++));
        double d = u * (P->c / P->eps) * m * P->dt;
        x = side == 0 ? -d : nx * P->dx + d;
        ox = side == 0 ? m : -m;
        cell = side == 0 ? -1 : nx;
        Tb = P->bcT[side];
      }
      if (!P->grey) nu = or_sample_nu(P->nu_edges[g], P->nu_edges[g + 1], Tb, or_draw(P, id, step, j++));
      int32_t cell0 = cell, nseg;
      double tend, w = tal->omega[b];
      if (tal2) restream(P, T, step, x, y, ox, oy, nu, w2_bins[b], id, cell, g, 1, j, tal2);
      int fate = or_stream_particle3(P, T, step, &x, &y, &z, &ox, &oy, &oz, nu, w, id, &cell, g, 1, j,
                                     NULL, 0, tal, &nseg, &tend, NULL, NULL, 0, NULL);
      tal->n_segments += nseg;
      if (fate == OR_SURVIVED) {
        ++tal->n_survived;
        if (nout < cap_out) {
          pout->x[nout] = x; pout->y[nout] = y; pout->ox[nout] = ox; pout->oy[nout] = oy;
          if (pout->z) { pout->z[nout] = z; pout->oz[nout] = oz; }
          pout->nu[nout] = nu; pout->w[nout] = w; pout->id[nout] = id;
          pout->cell[nout] = cell; pout->grp[nout] = g;
          if (w2_out) w2_out[nout] = w2_bins[b];
        } else status = OR_ERR_CAPACITY;
        ++nout;
      } else if (fate == OR_ABSORBED) ++tal->n_absorbed;
      else if (fate == OR_ESCAPED) ++tal->n_escaped;
      else ++tal->n_removed;
      if (rec && nrec < rec_cap) {
        or_record* r = &rec[nrec];
        r->id = id; r->fate = fate; r->cell0 = cell0; r->cell1 = cell; r->grp = g; r->nseg = nseg;
        r->_pad = 0; r->x = x; r->y = y; r->ox = ox; r->oy = oy; r->nu = nu; r->w = w; r->t_end = tend;
        r->z = z; r->oz = oz;
      }
      ++nrec;
    }
  }
  *n_out = nout;

  /* wave flux from the wave part at t^n */
  or_wave_flux(P, T, rho_h, tal->e_eff, tal->Fwave);

  /* constant part of the rho equation */
  double* R = malloc(sizeof(double) * ncell * G);
  tal->src_in = 0.0;
  for (int c = 0; c < ncell; ++c) {
    for (int g = 0; g < G; ++g) {
      double r = rho[c * G + g];
      for (int axis = 0; axis < P->dim; ++axis) {
        const int fl = cell_face(P, c, axis, -1), fu = cell_face(P, c, axis, +1);
        r += (dt / h_of(P, axis)) * (tal->Fwave[fl * G + g] - tal->Fwave[fu * G + g]);
      }
      r += tal->W[c * G + g] / V;
      if (P->src_T && P->src_T[c] > 0.0 && P->src_on != 0.0 &&
          (!(P->src_t_end > 0.0) || (double)step * dt < P->src_t_end)) {
        double s = P->src_on * (P->src_amp ? P->src_amp[c] : 1.0) * P->c * dt * or_phi(P, g, P->src_T[c]);
        r += s;
        tal->src_in += V * s / P->c;
      }
      R[c * G + g] = r;
    }
  }

  /* step 4: source iteration */
  int iters = 0;
  st = or_source_iteration(P, T, rho, R, T_out, rho_out, tal->Feq, &iters);
  if (st && !status) status = st;
  tal->si_iters = iters;
  free(R);

  /* wave / particle split and energy ledger.  Reading (the paper is silent
   * on it): the collisionless survivors of a (cell, group) never hold more
   * energy than rho^{n+1} leaves there.  Where E_surv/V > rho^{n+1} their
   * weights are scaled by f = max(rho^{n+1}, 0) V / E_surv, so that
   * rho^p = max(rho^{n+1}, 0) and rho^h = rho^{n+1} - rho^p >= min(rho^{n+1}, 0);
   * rho^{n+1} and the energy are unchanged.  Without it a cold cell crossed by
   * many survivors accumulates a negative wave part that the source
   * iteration takes out of the material, until T^{n+1} has no positive
   * solution.  With split_literal the split is I^h = I^{n+1} - I^p as the
   * paper writes it (Sec. 2.2) and nothing is scaled. */
  double* fscale = malloc(sizeof(double) * (size_t)ncell * G);
  int any_scaled = 0;
  tal->n_scaled_bins = 0;
  tal->E_rad1 = tal->E_mat1 = 0.0;
  for (int c = 0; c < ncell; ++c) {
    for (int g = 0; g < G; ++g) {
      const int i = c * G + g;
      double rp = tal->E_surv[i] / V, r = rho_out[i];
      fscale[i] = 1.0;
      if (!P->split_literal && rp > 0.0 && r < rp) {
        fscale[i] = r > 0.0 ? r / rp : 0.0;
        rp = r > 0.0 ? r : 0.0;
        any_scaled = 1;
        ++tal->n_scaled_bins;
      }
      rho_p_out[i] = rp;
      rho_h_out[i] = r - rp;
      tal->E_rad1 += V * r / P->c;
    }
    tal->E_mat1 += V * or_mat_energy(P, c, T_out[c]);
  }
  if (any_scaled) {
    const int64_t m = nout < cap_out ? nout : cap_out;
    for (int64_t k = 0; k < m; ++k) {
      const double f = fscale[pout->cell[k] * G + pout->grp[k]];
      if (f != 1.0) pout->w[k] *= f;
    }
  }
  if (w2_scale) memcpy(w2_scale, fscale, sizeof(double) * (size_t)ncell * G);
  free(fscale);
  double bin = 0.0;
  for (int axis = 0; axis < P->dim; ++axis) {
    const int nk = n_along(P, axis), nlines = n_lines(P, axis);
    const double S = area_of(P, axis);
    for (int line = 0; line < nlines; ++line)
      for (int g = 0; g < G; ++g) {
        int f0 = line_face(P, axis, line, 0);
        int f1 = line_face(P, axis, line, nk);
        bin += dt * S * ((tal->Feq[f0 * G + g] + tal->Fwave[f0 * G + g]) -
                         (tal->Feq[f1 * G + g] + tal->Fwave[f1 * G + g])) / P->c;
      }
  }
  tal->bnd_in_macro = bin;
  tal->bnd_out_macro = 0.0;
  double pin_e = 0.0, pout_e = 0.0;
  for (int i = 0; i < 6 * G; ++i) { pin_e += tal->inflow[i]; pout_e += tal->esc[i]; }
  tal->bnd_in_part = pin_e / P->c;
  tal->bnd_out_part = pout_e / P->c;
  (void)nface;
  for (int c = 0; c < ncell; ++c)
    if (!(T_out[c] == T_out[c])) { status = OR_ERR_NONFINITE; break; }
  tal->status = status;
  return status;
}
