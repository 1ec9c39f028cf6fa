/*
 * ugkwp_oracle_tangent.c -- forward-mode (tangent) derivative of one oracle
 * step with respect to the per-cell log-opacity scales s_c
 * (sigma0_c -> sigma0_c e^{s_c}) and to the incoming state.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of the oracle.
 *
 * The step is a Monte Carlo step, so "the derivative" is the pathwise one:
 * every discrete decision (birth counts N = floor(E/omega_ref + 1/2), which
 * face a particle crosses, whether it collides, survives or escapes) is held
 * at the value the step took, with the same Philox draws (common random
 * numbers).  Along such a fixed path the particle tallies are linear in the
 * particle weights, a newborn's weight is E/N with N fixed, a survivor keeps
 * its weight, and positions, free times and frequencies only decide the path.
 * What remains is smooth: the Simpson group opacity at T^n, the sampled
 * fraction e = exp(-dt c sigma/eps^2), the wave flux (Sec. 2.2 with the
 * face-opacity reading), and the implicit source iteration (App. B) whose
 * converged solution is differentiated through its own fixed-point map.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ugkwp_oracle.h"

static int ncell_of(const or_problem* P) { return P->nx * (P->dim == 2 ? P->ny : 1); }
static int nxface_of(const or_problem* P) { return (P->nx + 1) * (P->dim == 2 ? P->ny : 1); }
static int nface_of(const or_problem* P) {
  return P->dim == 2 ? (P->nx + 1) * P->ny + P->nx * (P->ny + 1) : P->nx + 1;
}
static double vol_of(const or_problem* P) { return P->dim == 2 ? P->dx * P->dy : P->dx; }

/* d sigma(nu, T)/ds and dT at one frequency: sigma = sigma0 e^s nu^p T^q, so
 * d sigma = sigma (ds + q dT/T) below the cap and 0 where the cap is taken. */
static double dsigma_point(const or_problem* P, int c, double nu, double T, double ds, double dT) {
  double s = P->sigma0[c] * pow(T, P->sig_q);
  if (!P->grey) s *= pow(nu, P->sig_p);
  if (P->sig_cap > 0.0 && !(s <= P->sig_cap)) return 0.0;
  return s * (ds + P->sig_q * dT / T);
}

double or_dsigma_group(const or_problem* P, int c, int g, double T, double ds, double dT) {
  if (P->grey) return dsigma_point(P, c, 0.0, T, ds, dT);
  double a = P->nu_edges[g], b = P->nu_edges[g + 1], m = 0.5 * (a + b);
  return (dsigma_point(P, c, a, T, ds, dT) + 4.0 * dsigma_point(P, c, m, T, ds, dT) +
          dsigma_point(P, c, b, T, ds, dT)) / 6.0;
}

/* x-derivatives of the flux coefficients of or_coefs: term by term on the
 * same Taylor series below x = 1/2, and from the closed forms above it,
 * with e = exp(-x):  c4' = (e - c4)/x,  f4' = c4' + e,  f2' = 2 c4' + e,
 * f5' = -e (1 + x)/2 - c4'.                                                 */
void or_dcoefs(double x, double* df2, double* df4, double* df5, double* dc4) {
  if (!(x > 0.0)) { *df2 = 0.0; *df4 = 0.5; *df5 = 0.0; *dc4 = -0.5; return; }
  long double X = x;
  if (x < 0.5) {
    long double s2 = 0, s4 = 0, s5 = 0, c = 0, p = 1;   /* p = x^(k-1) */
    long double fact = 1, sgn = 1;
    for (int k = 1; k <= 60; ++k) {
      if (k > 1) p *= X;
      fact *= (k + 1);
      sgn = -sgn;                          /* (-1)^k */
      long double t = k * p / fact;        /* d/dx x^k/(k+1)! */
      s2 += sgn * (1 - k) * t;
      s4 += -sgn * k * t;
      s5 += sgn * k * (1 - k) * t / 2;
      c += sgn * t;
    }
    *df2 = (double)s2; *df4 = (double)s4; *df5 = (double)s5; *dc4 = (double)c;
    return;
  }
  long double e = expl(-X), c4 = -expm1l(-X) / X;
  long double d4 = (e - c4) / X;
  *dc4 = (double)d4;
  *df4 = (double)(d4 + e);
  *df2 = (double)(2 * d4 + e);
  *df5 = (double)(-e * (1 + X) / 2 - d4);
}

/* ------------------------------------------------------------------------ */
/* Tangent of or_wave_flux.  Same face loop and the same readings (upwind
 * halves, face opacity from the harmonic mean of the side opacities at T^n,
 * e of the upwind cell or 0, van Leer slopes); each quantity is carried with
 * its derivative.  The branch taken at every face (limiter active or not,
 * sampled or unsampled upwind cell) is the forward one.                      */
static void van_leer_t(double a, double da, double b, double db, double* v, double* dv) {
  if (a * b > 0.0) {
    double s = a + b;
    *v = 2.0 * a * b / s;
    *dv = (2.0 * b * b * da + 2.0 * a * a * db) / (s * s);
  } else {
    *v = 0.0;
    *dv = 0.0;
  }
}

static void half_coefs_t(const or_problem* P, double x_f, double dx_f, double tau_f, double dtau_f,
                         double x_h, double dx_h, double e_eff,
                         double* A, double* dA, double* B, double* dB) {
  const double dt = P->dt;
  double f2, f4, f5, c4, df2, df4, df5, dc4;
  or_coefs(x_f, &f2, &f4, &f5, &c4);
  or_dcoefs(x_f, &df2, &df4, &df5, &dc4);
  if (e_eff > 0.0) {
    double ef = exp(-x_f), eh = exp(-x_h);
    double d = x_h - x_f;
    double ef_minus_eh = fabs(d) < 0.5 ? exp(-x_h) * expm1(d) : ef - eh;
    double dem = -ef * dx_f + eh * dx_h;
    *A = f4 + ef_minus_eh;
    *dA = df4 * dx_f + dem;
    *B = tau_f * f5 - 0.5 * dt * ef_minus_eh;
    *dB = dtau_f * f5 + tau_f * df5 * dx_f - 0.5 * dt * dem;
  } else {
    *A = c4;
    *dA = dc4 * dx_f;
    *B = -tau_f * f4;
    *dB = -(dtau_f * f4 + tau_f * df4 * dx_f);
  }
}

int or_wave_flux_tangent(const or_problem* P, const double* T, const double* dT, const double* ds,
                         const double* rho_h, const double* drho_h, const double* e_eff,
                         double* dFwave) {
  const int nx = P->nx, ny = P->dim == 2 ? P->ny : 1, G = P->G, ncell = nx * ny;
  const double v = P->c / P->eps, rate_f = P->c / (P->eps * P->eps), dt = P->dt;
  const int nxf = nxface_of(P);
  for (int axis = 0; axis < P->dim; ++axis) {
    const double h = axis == 0 ? P->dx : P->dy;
    const int nk = axis == 0 ? nx : ny;
    const int nlines = axis == 0 ? ny : nx;
    const int sideL = axis * 2, sideR = axis * 2 + 1;
    for (int line = 0; line < nlines; ++line) {
      for (int f = 0; f <= nk; ++f) {
        int fidx = axis == 0 ? line * (nx + 1) + f : nxf + f * nx + line;
        for (int g = 0; g < G; ++g) {
#define CELL_AT(k) (axis == 0 ? line * nx + (k) : (k) * nx + line)
          int kL = f - 1, kR = f;
          int lin = kL >= 0, rin = kR < nk;
          if ((!lin && P->bc[sideL] == OR_BC_REFLECT) || (!rin && P->bc[sideR] == OR_BC_REFLECT)) {
            dFwave[fidx * G + g] = 0.0;
            continue;
          }
          /* value and derivative of rho_h at line index k, ghosts included */
#define RHO_AT(k, out, dout) do {                                                   \
            int kk_ = (k);                                                           \
            if (kk_ >= 0 && kk_ < nk) {                                              \
              out = rho_h[CELL_AT(kk_) * G + g]; dout = drho_h[CELL_AT(kk_) * G + g]; \
            } else {                                                                 \
              int s_ = kk_ < 0 ? sideL : sideR;                                      \
              int kin_ = kk_ < 0 ? 0 : nk - 1;                                       \
              if (P->bc[s_] == OR_BC_REFLECT) {                                      \
                out = rho_h[CELL_AT(kin_) * G + g]; dout = drho_h[CELL_AT(kin_) * G + g]; \
              } else if (P->bc[s_] == OR_BC_BLACKBODY) {                             \
                out = or_phi(P, g, P->bcT[s_]); dout = 0.0;                          \
              } else { out = 0.0; dout = 0.0; }                                      \
            }                                                                        \
          } while (0)
          double rl, rr, rll, rrr, drl, drr, drll, drrr, sl, sr, dsl, dsr, fl, fr, dfl, dfr;
          RHO_AT(kL, rl, drl); RHO_AT(kR, rr, drr);
          if (P->wave_order >= 2) {
            RHO_AT(kL - 1, rll, drll); RHO_AT(kR + 1, rrr, drrr);
            if (lin) van_leer_t((rl - rll) / h, (drl - drll) / h, (rr - rl) / h, (drr - drl) / h, &sl, &dsl);
            else { sl = 0.0; dsl = 0.0; }
            if (rin) van_leer_t((rr - rl) / h, (drr - drl) / h, (rrr - rr) / h, (drrr - drr) / h, &sr, &dsr);
            else { sr = 0.0; dsr = 0.0; }
            fl = rl + 0.5 * h * sl; dfl = drl + 0.5 * h * dsl;
            fr = rr - 0.5 * h * sr; dfr = drr - 0.5 * h * dsr;
          } else {
            sl = sr = (rr - rl) / h;
            dsl = dsr = (drr - drl) / h;
            fl = rl; fr = rr; dfl = drl; dfr = drr;
          }
#undef RHO_AT
          double sgl, sgr, dsgl, dsgr, el, er;
          if (lin) {
            int c = CELL_AT(kL);
            sgl = or_sigma_group(P, c, g, T[c]);
            dsgl = or_dsigma_group(P, c, g, T[c], ds[c], dT[c]);
            el = e_eff[c * G + g];
          } else if (P->bc[sideL] == OR_BC_BLACKBODY) {
            int c = CELL_AT(0);
            sgl = or_sigma_group(P, c, g, P->bcT[sideL]);
            dsgl = or_dsigma_group(P, c, g, P->bcT[sideL], ds[c], 0.0);
            el = e_eff[(ncell + sideL) * G + g];
          } else { sgl = -1.0; dsgl = 0.0; el = 0.0; }
          if (rin) {
            int c = CELL_AT(kR);
            sgr = or_sigma_group(P, c, g, T[c]);
            dsgr = or_dsigma_group(P, c, g, T[c], ds[c], dT[c]);
            er = e_eff[c * G + g];
          } else if (P->bc[sideR] == OR_BC_BLACKBODY) {
            int c = CELL_AT(nk - 1);
            sgr = or_sigma_group(P, c, g, P->bcT[sideR]);
            dsgr = or_dsigma_group(P, c, g, P->bcT[sideR], ds[c], 0.0);
            er = e_eff[(ncell + sideR) * G + g];
          } else { sgr = -1.0; dsgr = 0.0; er = 0.0; }
          if (sgl < 0.0) { sgl = sgr; dsgl = dsgr; }
          if (sgr < 0.0) { sgr = sgl; dsgr = dsgl; }
#undef CELL_AT
          double sum = sgl + sgr;
          double sf = 2.0 * sgl * sgr / sum;
          double dsf = 2.0 * (sgr * sgr * dsgl + sgl * sgl * dsgr) / (sum * sum);
          double tau_f = 1.0 / (rate_f * sf), dtau_f = -tau_f * dsf / sf;
          double x_f = dt / tau_f, dx_f = dt * rate_f * dsf;
          double AL, dAL, BL, dBL, AR, dAR, BR, dBR;
          half_coefs_t(P, x_f, dx_f, tau_f, dtau_f, dt * rate_f * sgl, dt * rate_f * dsgl, el,
                       &AL, &dAL, &BL, &dBL);
          half_coefs_t(P, x_f, dx_f, tau_f, dtau_f, dt * rate_f * sgr, dt * rate_f * dsgr, er,
                       &AR, &dAR, &BR, &dBR);
          dFwave[fidx * G + g] = (dAL * fl + AL * dfl - dAR * fr - AR * dfr) * (v / 4.0)
                               + (dBL * sl + BL * dsl + dBR * sr + BR * dsr) * (v * v / 6.0);
        }
      }
    }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Tangent of the converged source iteration.  The iteration map of
 * or_source_iteration, T^{k+1} = num(T^k)/den(T^k) and
 * rho^{k+1} = (Q + a (Phi + Phi' (T^{k+1} - T^k)))/(1 + a), differentiated at
 * its fixed point T* (where T^{k+1} = T^k, so every term carrying the
 * derivative of Phi' is multiplied by T^{k+1} - T^k = 0):
 *   dT^{k+1} = (Cv dT^n + sum_g [da'_g (Q_g - Phi_g) + a'_g dQ_g]) / den,
 *   drho_g   = (dQ_g + da_g (Phi_g - rho_g) + a_g Phi'_g dT^{k+1}) / (1 + a_g),
 * with a = dt c sigma/eps^2, a' = a/(c (1 + a)), dQ = dR + (dt/h)(dF_in - dF_out)
 * and dF the tangent of the equilibrium face flux at iterate k.  Iterated from
 * dT^0 = dT^n like the forward iteration (same contraction), until the
 * largest change of dT is <= si_tol times the largest |dT|.  Q at the fixed
 * point is rho*(1 + a) - a Phi(T*), which is the rho equation solved for Q.  */
int or_source_iteration_tangent(const or_problem* P, const double* dT_n, const double* ds,
                                const double* dR, const double* T, const double* rho,
                                double* dT_out, double* drho_out, int* iters) {
  const int nx = P->nx, ny = P->dim == 2 ? P->ny : 1, G = P->G, ncell = nx * ny;
  const int nxf = nxface_of(P), nface = nface_of(P);
  const double v = P->c / P->eps, dt = P->dt;
  const double rate_f = P->c / (P->eps * P->eps);
  const size_t ncg = (size_t)ncell * G;
  double* sig = malloc(sizeof(double) * ncg);
  double* phi = malloc(sizeof(double) * ncg);
  double* dphi = malloc(sizeof(double) * ncg);
  double* Q = malloc(sizeof(double) * ncg);
  double* dsig = malloc(sizeof(double) * ncg);
  double* dF = malloc(sizeof(double) * (size_t)nface * G);
  double* dTk = malloc(sizeof(double) * ncell);
  for (int c = 0; c < ncell; ++c)
    for (int g = 0; g < G; ++g) {
      size_t i = (size_t)c * G + g;
      sig[i] = or_sigma_group(P, c, g, T[c]);
      phi[i] = or_phi(P, g, T[c]);
      dphi[i] = or_dphi(P, g, T[c]);
      double a = dt * rate_f * sig[i];
      Q[i] = rho[i] * (1.0 + a) - a * phi[i];
    }
  memcpy(dTk, dT_n, sizeof(double) * ncell);
  int status = OR_ERR_NOCONV, k;
  for (k = 0; k < P->si_max_iters; ++k) {
    for (int c = 0; c < ncell; ++c)
      for (int g = 0; g < G; ++g)
        dsig[(size_t)c * G + g] = or_dsigma_group(P, c, g, T[c], ds[c], dTk[c]);
    /* tangent of the equilibrium flux on every face */
    for (int axis = 0; axis < P->dim; ++axis) {
      const double h = axis == 0 ? P->dx : P->dy;
      const int nk = axis == 0 ? nx : ny, nlines = axis == 0 ? ny : nx;
      for (int line = 0; line < nlines; ++line)
        for (int f = 0; f <= nk; ++f) {
          int fidx = axis == 0 ? line * (nx + 1) + f : nxf + f * nx + line;
          for (int g = 0; g < G; ++g) {
            int cl = f - 1 >= 0 ? (axis == 0 ? line * nx + f - 1 : (f - 1) * nx + line) : -1;
            int cr = f < nk ? (axis == 0 ? line * nx + f : f * nx + line) : -1;
            double sl, sr, pl, pr, dsl, dsr, dpl, dpr;
            if (cl < 0 || cr < 0) {
              int side = axis * 2 + (cl < 0 ? 0 : 1);
              int cin = cl < 0 ? cr : cl;
              if (P->bc[side] == OR_BC_REFLECT) { dF[fidx * G + g] = 0.0; continue; }
              double sg, pg, dsg;
              if (P->bc[side] == OR_BC_BLACKBODY) {
                sg = or_sigma_group(P, cin, g, P->bcT[side]);
                dsg = or_dsigma_group(P, cin, g, P->bcT[side], ds[cin], 0.0);
                pg = or_phi(P, g, P->bcT[side]);
              } else { sg = sig[cin * G + g]; dsg = dsig[cin * G + g]; pg = 0.0; }
              size_t ii = (size_t)cin * G + g;
              if (cl < 0) {
                sl = sg; dsl = dsg; pl = pg; dpl = 0.0;
                sr = sig[ii]; dsr = dsig[ii]; pr = phi[ii]; dpr = dphi[ii] * dTk[cin];
              } else {
                sr = sg; dsr = dsg; pr = pg; dpr = 0.0;
                sl = sig[ii]; dsl = dsig[ii]; pl = phi[ii]; dpl = dphi[ii] * dTk[cin];
              }
            } else {
              size_t il = (size_t)cl * G + g, ir = (size_t)cr * G + g;
              sl = sig[il]; sr = sig[ir]; dsl = dsig[il]; dsr = dsig[ir];
              pl = phi[il]; pr = phi[ir];
              dpl = dphi[il] * dTk[cl]; dpr = dphi[ir] * dTk[cr];
            }
            double sum = sl + sr;
            double sf = 2.0 * sl * sr / sum;
            double dsf = 2.0 * (sr * sr * dsl + sl * sl * dsr) / (sum * sum);
            double tau = 1.0 / (rate_f * sf), dtau = -tau * dsf / sf;
            double f2, f4, f5, c4, df2, df4, df5, dc4;
            or_coefs(dt / tau, &f2, &f4, &f5, &c4);
            or_dcoefs(dt / tau, &df2, &df4, &df5, &dc4);
            double C2 = tau * f2, dC2 = dtau * f2 + tau * df2 * dt * rate_f * dsf;
            dF[fidx * G + g] = (dC2 * (pr - pl) + C2 * (dpr - dpl)) * (v * v / 3.0) / h;
          }
        }
    }
    double dmax = 0.0, amax = 0.0;
    for (int c = 0; c < ncell; ++c) {
      int ix = c % nx, iy = c / nx;
      double num = P->cv[c] * dT_n[c], den = P->cv[c];
      for (int g = 0; g < G; ++g) {
        size_t i = (size_t)c * G + g;
        int fxl = iy * (nx + 1) + ix, fxr = fxl + 1;
        double dq = dR[i] + (dt / P->dx) * (dF[fxl * G + g] - dF[fxr * G + g]);
        if (P->dim == 2) {
          int fyl = nxf + iy * nx + ix, fyr = nxf + (iy + 1) * nx + ix;
          dq += (dt / P->dy) * (dF[fyl * G + g] - dF[fyr * G + g]);
        }
        double a = dt * rate_f * sig[i], da = dt * rate_f * dsig[i];
        double ap = a / P->c / (1.0 + a), dap = da / P->c / ((1.0 + a) * (1.0 + a));
        num += dap * (Q[i] - phi[i]) + ap * dq;
        den += ap * dphi[i];
        /* rho tangent uses this iterate's dQ, da and the new dT (below) */
        drho_out[i] = dq;          /* provisional: dQ */
        dsig[i] = da;              /* reuse: da */
      }
      double dTn = num / den;
      for (int g = 0; g < G; ++g) {
        size_t i = (size_t)c * G + g;
        double a = dt * rate_f * sig[i];
        drho_out[i] = (drho_out[i] + dsig[i] * (phi[i] - rho[i]) + a * dphi[i] * dTn) / (1.0 + a);
      }
      double d = fabs(dTn - dTk[c]);
      if (d > dmax) dmax = d;
      if (fabs(dTn) > amax) amax = fabs(dTn);
      dT_out[c] = dTn;
    }
    memcpy(dTk, dT_out, sizeof(double) * ncell);
    if (!(dmax == dmax)) { status = OR_ERR_NONFINITE; ++k; break; }
    if (dmax <= P->si_tol * amax || amax == 0.0) { status = OR_OK; ++k; break; }
  }
  *iters = k;
  free(sig); free(phi); free(dphi); free(Q); free(dsig); free(dF); free(dTk);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Tangent of one full step (Algorithm 1) along ds, dT, drho, drho_h and the
 * weight tangents dw_in of the incoming particles.  Runs the step itself
 * (same outputs as or_step) and returns the tangents of T^{n+1}, rho^{n+1},
 * rho_h^{n+1} and of the survivors' weights (in output order).             */
int or_step_tangent(const or_problem* P, int64_t step, const double* ds,
                    const double* T, const double* dT, const double* rho, const double* drho,
                    const double* rho_h, const double* drho_h,
                    int64_t n_in, const or_particles* pin, const double* dw_in,
                    double* T_out, double* dT_out, double* rho_out, double* drho_out,
                    double* rho_h_out, double* drho_h_out, double* rho_p_out,
                    or_particles* pout, double* dw_out, int64_t cap_out, int64_t* n_out,
                    or_tallies* tal) {
  const int nx = P->nx, ny = P->dim == 2 ? P->ny : 1, G = P->G, ncell = nx * ny;
  const int nxf = nxface_of(P), nface = nface_of(P), nbins = (ncell + 4) * G;
  const double V = vol_of(P), dt = P->dt, rate_f = P->c / (P->eps * P->eps);
  const size_t ncg = (size_t)ncell * G;
  if (P->tau_num_C > 0.0) return OR_ERR_ARG;   /* tangent of tau = tau_num only */
  if (P->sig_law != 0) return OR_ERR_ARG;      /* and of the power-law opacity */
  if (P->method != OR_UGKWP) return OR_ERR_ARG;  /* and of the UGKWP sampling */
  if (P->dim == 3) return OR_ERR_ARG;           /* in 1D and 2D */
  if (P->cv_law != 0) return OR_ERR_ARG;        /* and of a constant heat capacity */

  /* births: N and e as the step takes them, and d(E/N) per bin */
  int64_t n_new = 0;
  or_birth_counts(P, T, rho_h, tal, &n_new);
  double* dw_bins = calloc(nbins, sizeof(double));
  for (int b = 0; b < nbins; ++b) {
    if (tal->N[b] <= 0) continue;
    int cell = b / G, g = b % G;
    double e = tal->e_eff[b], dsig, dE;
    if (cell < ncell) {
      dsig = or_dsigma_group(P, cell, g, T[cell], ds[cell], dT[cell]);
      double de = -e * dt * rate_f * dsig;
      double rh = rho_h[b];
      dE = (de * (rh > 0.0 ? rh : 0.0) + (rh > 0.0 ? e * drho_h[b] : 0.0)) * V;
    } else {
      int side = cell - ncell;
      int src_cell = side == 0 ? 0 : P->nx - 1;
      dsig = or_dsigma_group(P, src_cell, g, P->bcT[side], ds[src_cell], 0.0);
      double de = -e * dt * rate_f * dsig;
      dE = 0.25 * (P->c / P->eps) * or_phi(P, g, P->bcT[side]) * dt * de;
    }
    dw_bins[b] = dE / tal->N[b];
  }

  /* the step, every particle streamed a second time with its weight tangent */
  or_tallies dtal;
  memset(&dtal, 0, sizeof dtal);
  dtal.W = calloc(ncg, sizeof(double));
  dtal.E_surv = calloc(ncg, sizeof(double));
  dtal.E_abs = calloc(ncg, sizeof(double));
  dtal.esc = calloc(4 * G, sizeof(double));
  dtal.inflow = calloc(4 * G, sizeof(double));
  double* fscale = malloc(sizeof(double) * ncg);
  int status = or_step_core(P, step, T, rho, rho_h, n_in, pin, T_out, rho_out, rho_h_out, rho_p_out,
                            pout, cap_out, n_out, NULL, 0, tal, dw_in, dw_bins, dw_out, &dtal, fscale);

  /* wave flux and the constant part of the rho equation */
  double* dFw = calloc((size_t)nface * G, sizeof(double));
  or_wave_flux_tangent(P, T, dT, ds, rho_h, drho_h, tal->e_eff, dFw);
  double* dR = malloc(sizeof(double) * ncg);
  for (int c = 0; c < ncell; ++c) {
    int ix = c % nx, iy = c / nx;
    for (int g = 0; g < G; ++g) {
      int fxl = iy * (nx + 1) + ix, fxr = fxl + 1;
      double r = drho[c * G + g] + (dt / P->dx) * (dFw[fxl * G + g] - dFw[fxr * G + g]);
      if (P->dim == 2) {
        int fyl = nxf + iy * nx + ix, fyr = nxf + (iy + 1) * nx + ix;
        r += (dt / P->dy) * (dFw[fyl * G + g] - dFw[fyr * G + g]);
      }
      dR[c * G + g] = r + dtal.W[c * G + g] / V;
    }
  }

  int iters = 0;
  int st = or_source_iteration_tangent(P, dT, ds, dR, T_out, rho_out, dT_out, drho_out, &iters);
  if (st && !status) status = st;
  /* wave / particle split with the survivors' scaling: where f != 1 the
   * particle part is max(rho^{n+1}, 0), each survivor's weight w f with
   * f = rho^{n+1} V / E_surv (or 0), so df = drho^{n+1} V/E_surv
   * - rho^{n+1} V dE_surv/E_surv^2. */
  double* df = calloc(ncg, sizeof(double));
  for (size_t i = 0; i < ncg; ++i) {
    if (fscale[i] == 1.0) {
      drho_h_out[i] = drho_out[i] - dtal.E_surv[i] / V;
    } else if (fscale[i] > 0.0) {
      drho_h_out[i] = 0.0;
      double Es = tal->E_surv[i];
      df[i] = drho_out[i] * V / Es - rho_out[i] * V * dtal.E_surv[i] / (Es * Es);
    } else {
      drho_h_out[i] = drho_out[i];
    }
  }
  {
    const int64_t m = *n_out < cap_out ? *n_out : cap_out;
    for (int64_t k = 0; k < m; ++k) {
      const size_t i = (size_t)pout->cell[k] * G + pout->grp[k];
      const double f = fscale[i];
      if (f == 1.0) continue;
      dw_out[k] = f > 0.0 ? dw_out[k] * f + (pout->w[k] / f) * df[i] : 0.0;
    }
  }

  free(df); free(fscale);
  free(dw_bins); free(dFw); free(dR);
  free(dtal.W); free(dtal.E_surv); free(dtal.E_abs); free(dtal.esc); free(dtal.inflow);
  return status;
}
