// ugkwp_adjoint.cu -- reverse-mode (adjoint) pass of one UGKWP step on sm_103a,
// for the gradient of a function of the final state with respect to the
// per-cell log-opacity scales s_c (sigma0_c -> sigma0_c e^{s_c}).
//
// The derivative is the pathwise one: the step's Monte Carlo decisions (birth
// counts N, which faces a particle crosses, collision, survival, escape) are
// held as the forward step took them, with the same Philox draws.  Along that
// path the particle tallies are linear in the weights; a newborn's weight is
// E/N at fixed N with E = e max(rho_h, 0) V and e = exp(-dt c sigma_g/eps^2);
// a survivor keeps its weight into the next step.  The smooth parts are the
// Simpson group opacity at T^n (births, wave flux), the wave flux of Sec. 2.2
// (face-opacity reading, van Leer reconstruction) and the converged source
// iteration of App. B, whose adjoint solves the transposed linear system of
// its fixed point with the same Jacobi splitting the forward iteration uses.
//
// The end-of-step scaling of survivors (where they would hold more than
// rho^{n+1} of their cell and group, their weights are scaled by
// f = rho^{n+1} V/E_surv) is differentiated too: f depends on rho^{n+1} and, via
// E_surv, on every survivor of the bin.
//
// One adjoint step reads the tape the forward step wrote (T^n, rho_h^n, N,
// T^{n+1}, rho^{n+1}, the scaling factors and E_surv, and one record per
// processed particle: start cell, end cell, output slot, group, weight) and
// maps the adjoints of the step's outputs (T^{n+1}, rho^{n+1}, rho_h^{n+1},
// survivors' weights) to those of its inputs (T^n, rho^n, rho_h^n, incoming
// particles' weights), adding the explicit s-dependence to dL/ds.  Kernels:
//   k_adj_scale_sums one thread per processed particle: per scaled bin the
//                   sum of next-step weight adjoints times weights;
//   k_adj_si        cooperative, one warp per cell: adjoint source iteration,
//                   adjoint of R and the SI's part of dL/ds and dL/dT^n;
//   k_adj_wave      one thread per (face, group): wave-flux adjoint;
//   k_adj_particles one thread per processed particle: weight adjoints;
//   k_adj_birth     one warp per cell: newborn weights and group opacities at
//                   T^n, then the new adjoint state.
#include "ugkwp_device.cuh"
#include "ugkwp_grid.cuh"
#include "ugkwp_launch.h"

namespace ugkwp {

// --------------------------------------------------------------------------
// Layouts (host side)

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t hash_size(const Dev& d) {
  size_t h = 1024;
  while (h < 2 * (size_t)d.capacity) h <<= 1;
  return h;
}

TapeLayout tape_layout(const Dev& d, long long rec_cap) {
  TapeLayout L;
  const size_t ncg = (size_t)d.ncell * d.G;
  size_t o = 0;
  L.hdr = o;    o += up256(sizeof(Ctrl));
  L.T0 = o;     o += up256(sizeof(double) * d.ncell);
  L.T1 = o;     o += up256(sizeof(double) * d.ncell);
  L.rho1 = o;   o += up256(sizeof(double) * ncg);
  L.rho_h0 = o; o += up256(sizeof(double) * ncg);
  L.wscale = o; o += up256(sizeof(double) * ncg);
  L.Esurv = o;  o += up256(sizeof(double) * ncg);
  L.N = o;      o += up256(sizeof(uint32_t) * d.nbins);
  L.rec = o;    o += up256(sizeof(TapeRec) * (size_t)(rec_cap > 0 ? rec_cap : 0));
  L.total = o;
  return L;
}

TapeView tape_view(const Dev& d, const void* base, long long rec_cap) {
  const TapeLayout L = tape_layout(d, rec_cap);
  const char* b = static_cast<const char*>(base);
  TapeView t;
  t.hdr = reinterpret_cast<const Ctrl*>(b + L.hdr);
  t.T0 = reinterpret_cast<const double*>(b + L.T0);
  t.T1 = reinterpret_cast<const double*>(b + L.T1);
  t.rho1 = reinterpret_cast<const double*>(b + L.rho1);
  t.rho_h0 = reinterpret_cast<const double*>(b + L.rho_h0);
  t.wscale = reinterpret_cast<const double*>(b + L.wscale);
  t.Esurv = reinterpret_cast<const double*>(b + L.Esurv);
  t.N = reinterpret_cast<const uint32_t*>(b + L.N);
  t.rec = reinterpret_cast<const TapeRec*>(b + L.rec);
  t.rec_cap = rec_cap;
  return t;
}

size_t adjoint_bytes(const Dev& d) {
  const size_t ncg = (size_t)d.ncell * d.G, nc = d.ncell, cap = (size_t)d.capacity;
  size_t o = up256(sizeof(AdjCtrl));
  o += 4 * up256(sizeof(double) * nc);            // lamT, lamS, lamT0, ls
  o += 2 * up256(sizeof(double) * ncg);           // lamRho, lamRhoH
  o += 2 * up256(sizeof(double) * cap);           // lamW[2]
  o += 4 * up256(sizeof(double) * ncg);           // lamR, lamRhoH0, lamSig0, Sb
  o += up256(sizeof(double) * d.nbins);           // lamE
  o += 5 * up256(sizeof(double) * nc);            // mu[2], gT, D, Jl
  o += 6 * up256(sizeof(double) * ncg);           // sig1, sig1s, phi1, dphi1, sig0, sig0s
  o += up256(sizeof(double) * ncg * 2 * d.dim);   // dFdT
  const size_t hs = hash_size(d);
  o += up256(sizeof(unsigned long long) * hs) + up256(sizeof(double) * hs);   // hkeys, hvals
  return o;
}

AdjView adjoint_view(const Dev& d, void* base) {
  const size_t ncg = (size_t)d.ncell * d.G, nc = d.ncell, cap = (size_t)d.capacity;
  char* b = static_cast<char*>(base);
  size_t o = 0;
  auto take = [&](size_t bytes) { char* p = b + o; o += up256(bytes); return p; };
  AdjView a;
  a.ctrl = reinterpret_cast<AdjCtrl*>(take(sizeof(AdjCtrl)));
  a.lamT = reinterpret_cast<double*>(take(sizeof(double) * nc));
  a.lamS = reinterpret_cast<double*>(take(sizeof(double) * nc));
  a.lamT0 = reinterpret_cast<double*>(take(sizeof(double) * nc));
  a.ls = reinterpret_cast<double*>(take(sizeof(double) * nc));
  a.lamRho = reinterpret_cast<double*>(take(sizeof(double) * ncg));
  a.lamRhoH = reinterpret_cast<double*>(take(sizeof(double) * ncg));
  a.lamW[0] = reinterpret_cast<double*>(take(sizeof(double) * cap));
  a.lamW[1] = reinterpret_cast<double*>(take(sizeof(double) * cap));
  a.lamR = reinterpret_cast<double*>(take(sizeof(double) * ncg));
  a.lamRhoH0 = reinterpret_cast<double*>(take(sizeof(double) * ncg));
  a.lamSig0 = reinterpret_cast<double*>(take(sizeof(double) * ncg));
  a.lamE = reinterpret_cast<double*>(take(sizeof(double) * d.nbins));
  a.Sb = reinterpret_cast<double*>(take(sizeof(double) * ncg));
  a.mu[0] = reinterpret_cast<double*>(take(sizeof(double) * nc));
  a.mu[1] = reinterpret_cast<double*>(take(sizeof(double) * nc));
  a.gT = reinterpret_cast<double*>(take(sizeof(double) * nc));
  a.D = reinterpret_cast<double*>(take(sizeof(double) * nc));
  a.Jl = reinterpret_cast<double*>(take(sizeof(double) * nc));
  a.sig1 = reinterpret_cast<double*>(take(sizeof(double) * ncg));
  a.sig1s = reinterpret_cast<double*>(take(sizeof(double) * ncg));
  a.phi1 = reinterpret_cast<double*>(take(sizeof(double) * ncg));
  a.dphi1 = reinterpret_cast<double*>(take(sizeof(double) * ncg));
  a.sig0 = reinterpret_cast<double*>(take(sizeof(double) * ncg));
  a.sig0s = reinterpret_cast<double*>(take(sizeof(double) * ncg));
  a.dFdT = reinterpret_cast<double*>(take(sizeof(double) * ncg * 2 * d.dim));
  a.hsize = (long long)hash_size(d);
  a.hkeys = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * a.hsize));
  a.hvals = reinterpret_cast<double*>(take(sizeof(double) * a.hsize));
  a.cap = d.capacity;
  return a;
}

// --------------------------------------------------------------------------
// Device helpers

// Bounded grid barrier of the cooperative adjoint kernel (monotone arrival
// counter; on timeout the status bit is set and every block returns).
__device__ __forceinline__ bool adj_barrier(AdjCtrl* ctrl, unsigned int limit, unsigned int target) {
  __shared__ int s_timeout;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&ctrl->bar_count, 1u);
    const unsigned int lim = limit ? limit : (1u << 25);
    unsigned int spins = 0;
    int to = 0;
    while (true) {
      if (load_acquire_u32(&ctrl->bar_count) >= target) break;
      if (++spins > lim) { to = 1; break; }
      __nanosleep(64);
    }
    if (to) atomicOr(&ctrl->status, ST_TIMEOUT);
    __threadfence();
    s_timeout = to;
  }
  __syncthreads();
  return s_timeout == 0;
}

__device__ __forceinline__ void adj_max(unsigned long long* slot, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

// The other side of a face of cell c for the source iteration at T^{n+1}:
// its opacity and Phi, and their derivatives with respect to T_c and s_c
// (non-zero only for ghosts that take the cell's own opacity).
struct Nb {
  int kind;        // 0: reflecting wall (no flux), 1: cell n, 2: black-body ghost, 3: vacuum ghost
  int n;
  double s, sT, sS, phi;
};

__device__ __forceinline__ Nb adj_neighbour(const Dev& d, const AdjView& a, int c, int axis, int dir, int g,
                                            double sc, double scT, double scS) {
  Nb r;
  const int ix = c % d.nx, iy = c / d.nx;
  const int jx = ix + (axis == 0 ? dir : 0), jy = iy + (axis == 1 ? dir : 0);
  const int nyy = d.dim == 2 ? d.ny : 1;
  r.n = -1;
  r.sT = 0.0;
  r.sS = 0.0;
  if (jx < 0 || jx >= d.nx || jy < 0 || jy >= nyy) {
    const int side = axis * 2 + (dir > 0 ? 1 : 0);
    if (d.bc[side] == BC_REFLECT) { r.kind = 0; r.s = sc; r.phi = 0.0; return r; }
    if (d.bc[side] == BC_BLACKBODY) {
      r.kind = 2;
      r.s = d.ghost_sig[side * d.G + g];
      r.sS = sigma_group_ds(d, sigma_T(d, c, d.bcT[side]), g);
      r.phi = d.ghost_phi[side * d.G + g];
      return r;
    }
    r.kind = 3;
    r.s = sc; r.sT = scT; r.sS = scS; r.phi = 0.0;
    return r;
  }
  r.kind = 1;
  r.n = jy * d.nx + jx;
  r.s = __ldcg(a.sig1 + (size_t)r.n * d.G + g);
  r.phi = __ldcg(a.phi1 + (size_t)r.n * d.G + g);
  return r;
}

// Derivatives of the equilibrium flux F = C2 (v^2/3)(Phi_u - Phi_l)/h on the
// face (axis, dir) of cell c with respect to T_c and s_c.  C2 = tau f2(x),
// tau = 1/(rate sigma_f), x = dt/tau, sigma_f = 2 s_l s_u/(s_l + s_u).
__device__ __forceinline__ void face_grad(const Dev& d, double h, int dir, double sc, double scT, double scS,
                                          double pc, double dpc, const Nb& nb, double* dT, double* dS) {
  const double sl = dir < 0 ? nb.s : sc, su = dir < 0 ? sc : nb.s;
  const double pl = dir < 0 ? nb.phi : pc, pu = dir < 0 ? pc : nb.phi;
  const double sum = sl + su;
  const double sf = 2.0 * sl * su / sum;
  const double tau = 1.0 / (d.rate_f * sf);
  const double x = d.dt / tau;
  const double f2 = coef_f2(x);
  const double df2 = coef_derivs(x).f2;
  const double C = tau * f2;
  const double dC = -tau / sf * f2 + tau * df2 * d.dt * d.rate_f;
  const double K = d.v * d.v / 3.0 / h;
  const double dPhi = pu - pl;
  const double inv = 1.0 / (sum * sum);
  const double dFsl = dC * 2.0 * su * su * inv * K * dPhi;
  const double dFsu = dC * 2.0 * sl * sl * inv * K * dPhi;
  const double dFsc = dir < 0 ? dFsu : dFsl, dFsn = dir < 0 ? dFsl : dFsu;
  const double dFpc = dir < 0 ? C * K : -C * K;
  *dT = dFsc * scT + dFsn * nb.sT + dFpc * dpc;
  *dS = dFsc * scS + dFsn * nb.sS;
}

// --------------------------------------------------------------------------
// Where the step scaled a (cell, group)'s survivors by f = rho V/E_surv, the
// weights depend on each other through E_surv: S_b = sum over the bin's
// survivors of lambda_w(next step) x w (the weight before scaling).
__global__ void __launch_bounds__(256) k_adj_scale_sums(const __grid_constant__ Dev d, const TapeView t,
                                                        const AdjView a) {
  if (!t.hdr->scaled) return;
  const long long n = (long long)t.hdr->n_in + (long long)t.hdr->n_new;
  if (n > t.rec_cap) return;   // reported by k_adj_particles
  const double* __restrict__ lw_next = a.lamW[a.ctrl->cur];
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const TapeRec tr = t.rec[k];
    if (tr.slot < 0) continue;
    const size_t b = (size_t)tr.c1 * d.G + tr.g;
    const double f = t.wscale[b];
    if (f != 1.0 && f > 0.0) atomicAdd(a.Sb + b, lw_next[tr.slot] * tr.w);
  }
}

// --------------------------------------------------------------------------
// Adjoint of the converged source iteration.  The fixed point solves
//   F_c(T) = Cv (T_c - T^n_c) - sum_g a'_g (Q_g - Phi_g(T_c)) = 0,
//   rho_g = (Q_g + a_g Phi_g)/(1 + a_g),
// a = dt c sigma_g(T_c, s_c)/eps^2, a' = a/(c (1 + a)),
// Q = R + (dt/h)(F_in - F_out) with the equilibrium face fluxes at T.
// Given adjoints lT (of T) and lr (of rho, including rho_h = rho - rho_p):
//   v = lr/(1+a) is the adjoint of Q through rho;
//   g_T = lT + sum_g lr (a Phi' + (Phi - rho) a_T)/(1+a) + sum_faces (dt/h)(v_u - v_l) dF/dT_c;
//   J^T mu = g_T solved by mu <- mu + (g_T - J^T mu)/D, D the forward's
//   denominator Cv + sum_g a' Phi' (the forward iteration's splitting, so the
//   same contraction), J^T mu = (Cv - sum_g [a'_T (Q - Phi) - a' Phi']) mu
//   - sum_faces (dt/h)(w_u - w_l) dF/dT_c, w = a' mu;
// then lambda_R = v + a' mu, dL/dT^n += Cv mu and
//   dL/ds_c += sum_g [lr (Phi - rho) a_s/(1+a) + a'_s (Q - Phi) mu]
//            + sum_faces (dt/h)(lambda_R,u - lambda_R,l) dF/ds_c.
template <int NC>
__global__ void __launch_bounds__(256) k_adj_si(const __grid_constant__ Dev d, const TapeView t, const AdjView a) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  const long long gw = blockIdx.x * (long long)nwb + wib, nw = (long long)gridDim.x * nwb;
  const int G = d.G, ncell = d.ncell, nslot = 2 * d.dim;
  const double dt = d.dt, rate = d.rate_f;
  const unsigned int spin_limit = a.ctrl->bar_limit;
  __shared__ double s_red[8][2];
  unsigned int bar = 0;

  // ---- prologue: caches at T^{n+1} and T^n, local parts, zeroed accumulators
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < 4 * G; i += blockDim.x) a.lamE[(size_t)ncell * G + i] = 0.0;
  for (long long cc = gw; cc < ncell; cc += nw) {
    const int c = (int)cc;
    const double T1 = t.T1[c], T0 = t.T0[c], cv = d.cv[c];
    double sg[NC], ph[NC], dp[NC];
    cell_planck<NC>(d, c, T1, sg, ph, dp);
    const double sT1 = sigma_T(d, c, T1), sT0 = sigma_T(d, c, T0);
    double lT = 0.0, lS = 0.0, jl = 0.0, den = 0.0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const int g = lane + 32 * j;
      if (g >= G) continue;
      const size_t i = (size_t)c * G + g;
      const double s1 = sg[j], s1s = sigma_group_ds(d, sT1, g), s1T = d.sig_q / T1 * s1s;
      __stcg(a.sig1 + i, s1);
      __stcg(a.sig1s + i, s1s);
      __stcg(a.phi1 + i, ph[j]);
      __stcg(a.dphi1 + i, dp[j]);
      a.sig0[i] = sigma_group(d, sT0, g);
      a.sig0s[i] = sigma_group_ds(d, sT0, g);
      a.lamRhoH0[i] = 0.0;
      a.lamSig0[i] = 0.0;
      a.lamE[i] = 0.0;
      const double rho1 = t.rho1[i];
      // adjoint of rho^{n+1}: directly, through rho_h = rho - rho_p, and, where
      // the survivors were scaled by f = rho V/E_surv, through their weights
      const double f = t.wscale[i];
      const double lr = a.lamRho[i] + (f == 1.0 || f <= 0.0 ? a.lamRhoH[i] : a.Sb[i] * d.vol / t.Esurv[i]);
      const double A = dt * rate * s1, AT = dt * rate * s1T, AS = dt * rate * s1s, op = 1.0 + A;
      const double Q = rho1 * op - A * ph[j];
      __stcg(a.lamR + i, lr / op);                    // v, the adjoint of Q through rho
      lT += lr * (A * dp[j] + (ph[j] - rho1) * AT) / op;
      lS += lr * (ph[j] - rho1) * AS / op;
      const double ap = A / (d.c * op), apT = AT / (d.c * op * op);
      den += ap * dp[j];
      jl -= apT * (Q - ph[j]) - ap * dp[j];
    }
    lT = warp_sum(lT);
    lS = warp_sum(lS);
    den = warp_sum(den);
    jl = warp_sum(jl);
    if (lane == 0) {
      a.gT[c] = a.lamT[c] + lT;
      a.ls[c] = lS;
      a.D[c] = cv + den;
      a.Jl[c] = cv + jl;
    }
  }
  if (!adj_barrier(a.ctrl, spin_limit, (++bar) * gridDim.x)) return;

  // ---- face part of g_T; dF/dT_c per face cached for the iterations
  for (long long cc = gw; cc < ncell; cc += nw) {
    const int c = (int)cc;
    const double T1 = t.T1[c];
    double gf = 0.0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const int g = lane + 32 * j;
      if (g >= G) continue;
      const size_t i = (size_t)c * G + g;
      const double sc = __ldcg(a.sig1 + i), scS = __ldcg(a.sig1s + i), scT = d.sig_q / T1 * scS;
      const double pc = __ldcg(a.phi1 + i), dpc = __ldcg(a.dphi1 + i);
      const double vc = __ldcg(a.lamR + i);
      for (int axis = 0; axis < d.dim; ++axis) {
        const double h = axis == 0 ? d.dx : d.dy;
        for (int dir = -1; dir <= 1; dir += 2) {
          const int slot = axis * 2 + (dir > 0 ? 1 : 0);
          const Nb nb = adj_neighbour(d, a, c, axis, dir, g, sc, scT, scS);
          double dT = 0.0, dS = 0.0;
          if (nb.kind != 0) face_grad(d, h, dir, sc, scT, scS, pc, dpc, nb, &dT, &dS);
          __stcg(a.dFdT + ((size_t)c * nslot + slot) * G + g, dT);
          const double vn = nb.kind == 1 ? __ldcg(a.lamR + (size_t)nb.n * G + g) : 0.0;
          const double lf = dir < 0 ? (dt / h) * (vc - vn) : (dt / h) * (vn - vc);
          gf += lf * dT;
        }
      }
    }
    gf = warp_sum(gf);
    if (lane == 0) {
      const double gt = a.gT[c] + gf;
      a.gT[c] = gt;
      __stcg(a.mu[0] + c, gt / a.D[c]);
    }
  }
  if (!adj_barrier(a.ctrl, spin_limit, (++bar) * gridDim.x)) return;

  // ---- iterations
  int it = 0, done = 0;
  for (; it < d.si_max_iters; ++it) {
    const int cur = it & 1, nxt = cur ^ 1;
    double werr = 0.0, wmag = 0.0;
    for (long long cc = gw; cc < ncell; cc += nw) {
      const int c = (int)cc;
      const double mc = __ldcg(a.mu[cur] + c);
      double jt = 0.0;
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const int g = lane + 32 * j;
        if (g >= G) continue;
        const size_t i = (size_t)c * G + g;
        const double sc = __ldcg(a.sig1 + i);
        const double Ac = dt * rate * sc;
        const double wc = Ac / (d.c * (1.0 + Ac)) * mc;
        const int ix = c % d.nx, iy = c / d.nx;
        for (int axis = 0; axis < d.dim; ++axis) {
          const double h = axis == 0 ? d.dx : d.dy;
          for (int dir = -1; dir <= 1; dir += 2) {
            const int jx = ix + (axis == 0 ? dir : 0), jy = iy + (axis == 1 ? dir : 0);
            const int nyy = d.dim == 2 ? d.ny : 1;
            double wn = 0.0;
            if (jx >= 0 && jx < d.nx && jy >= 0 && jy < nyy) {
              const int n = jy * d.nx + jx;
              const double An = dt * rate * __ldcg(a.sig1 + (size_t)n * G + g);
              wn = An / (d.c * (1.0 + An)) * __ldcg(a.mu[cur] + n);
            }
            const int slot = axis * 2 + (dir > 0 ? 1 : 0);
            const double lf = dir < 0 ? (dt / h) * (wc - wn) : (dt / h) * (wn - wc);
            jt -= lf * __ldcg(a.dFdT + ((size_t)c * nslot + slot) * G + g);
          }
        }
      }
      jt = warp_sum(jt) + a.Jl[c] * mc;
      const double mn = mc + (a.gT[c] - jt) / a.D[c];
      if (lane == 0) __stcg(a.mu[nxt] + c, mn);
      const double err = fabs(mn - mc), mag = fabs(mn);
      werr = fmax(werr, (err == err) ? err : 1e300);
      wmag = fmax(wmag, (mag == mag) ? mag : 1e300);
    }
    if (lane == 0) { s_red[wib][0] = werr; s_red[wib][1] = wmag; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double e = 0.0, m = 0.0;
      for (int w = 0; w < nwb; ++w) { e = fmax(e, s_red[w][0]); m = fmax(m, s_red[w][1]); }
      adj_max(&a.ctrl->err_slot[it % 3][0], e);
      adj_max(&a.ctrl->err_slot[it % 3][1], m);
      if (blockIdx.x == 0) { a.ctrl->err_slot[(it + 1) % 3][0] = 0ull; a.ctrl->err_slot[(it + 1) % 3][1] = 0ull; }
    }
    if (!adj_barrier(a.ctrl, spin_limit, (++bar) * gridDim.x)) return;
    const double e = __longlong_as_double((long long)load_acquire_u64(&a.ctrl->err_slot[it % 3][0]));
    const double m = __longlong_as_double((long long)load_acquire_u64(&a.ctrl->err_slot[it % 3][1]));
    if (e <= d.si_tol * m || m == 0.0) { done = 1; ++it; break; }
  }
  const int fin = it & 1;   // buffer written by the last iterate (mu[0] if none ran)

  // ---- epilogue: lambda_R, dL/dT^n (SI part), local dL/ds
  for (long long cc = gw; cc < ncell; cc += nw) {
    const int c = (int)cc;
    const double mu = __ldcg(a.mu[fin] + c);
    double lS = 0.0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const int g = lane + 32 * j;
      if (g >= G) continue;
      const size_t i = (size_t)c * G + g;
      const double s1 = __ldcg(a.sig1 + i), s1s = __ldcg(a.sig1s + i), ph = __ldcg(a.phi1 + i);
      const double A = dt * rate * s1, AS = dt * rate * s1s, op = 1.0 + A;
      const double Q = t.rho1[i] * op - A * ph;
      const double ap = A / (d.c * op), apS = AS / (d.c * op * op);
      __stcg(a.lamR + i, __ldcg(a.lamR + i) + ap * mu);
      lS += apS * (Q - ph) * mu;
    }
    lS = warp_sum(lS);
    if (lane == 0) {
      a.lamT0[c] = d.cv[c] * mu;
      a.ls[c] += lS;
    }
  }
  if (!adj_barrier(a.ctrl, spin_limit, (++bar) * gridDim.x)) return;
  for (long long cc = gw; cc < ncell; cc += nw) {
    const int c = (int)cc;
    const double T1 = t.T1[c];
    double lS = 0.0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const int g = lane + 32 * j;
      if (g >= G) continue;
      const size_t i = (size_t)c * G + g;
      const double sc = __ldcg(a.sig1 + i), scS = __ldcg(a.sig1s + i), scT = d.sig_q / T1 * scS;
      const double pc = __ldcg(a.phi1 + i), dpc = __ldcg(a.dphi1 + i);
      const double lc = __ldcg(a.lamR + i);
      for (int axis = 0; axis < d.dim; ++axis) {
        const double h = axis == 0 ? d.dx : d.dy;
        for (int dir = -1; dir <= 1; dir += 2) {
          const Nb nb = adj_neighbour(d, a, c, axis, dir, g, sc, scT, scS);
          if (nb.kind == 0) continue;
          double dT, dS;
          face_grad(d, h, dir, sc, scT, scS, pc, dpc, nb, &dT, &dS);
          const double ln = nb.kind == 1 ? __ldcg(a.lamR + (size_t)nb.n * G + g) : 0.0;
          const double lf = dir < 0 ? (dt / h) * (lc - ln) : (dt / h) * (ln - lc);
          lS += lf * dS;
        }
      }
    }
    lS = warp_sum(lS);
    if (lane == 0) a.lamS[c] += a.ls[c] + lS;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctrl->iters = (unsigned int)it;
    if (!done) atomicOr(&a.ctrl->status, ST_NOCONV);
  }
}

// --------------------------------------------------------------------------
// Adjoint of the wave flux (one thread per face and group).  lambda_F =
// (dt/h)(lambda_R,u - lambda_R,l) since the face's flux enters R of the upper
// cell with + and of the lower cell with -.  The forward flux is recomputed
// from the tape's rho_h^n and the opacities at T^n; the branches (limiter,
// sampled or unsampled upwind cell) are the forward ones.  Contributions go
// to lambda(rho_h^n) along the reconstruction stencil, to lambda(sigma_g(T^n))
// of both sides, and, for a black-body ghost side, to dL/ds of the cell whose
// sigma0 the ghost uses.
__device__ __forceinline__ double rho_h_tape(const Dev& d, const TapeView& t, const FaceRef& r, int k, int g) {
  if (k >= 0 && k < r.nk) return t.rho_h0[(size_t)line_cell(d, r, k) * d.G + g];
  const int side = r.axis * 2 + (k < 0 ? 0 : 1);
  if (d.bc[side] == BC_REFLECT) return t.rho_h0[(size_t)line_cell(d, r, k < 0 ? 0 : r.nk - 1) * d.G + g];
  if (d.bc[side] == BC_BLACKBODY) return d.ghost_phi[side * d.G + g];
  return 0.0;
}

// add lambda to rho_h at stencil position k (mirror ghosts map to the inner cell)
__device__ __forceinline__ void add_rho_h(const Dev& d, const AdjView& a, const FaceRef& r, int k, int g, double l) {
  if (l == 0.0) return;
  int cell = -1;
  if (k >= 0 && k < r.nk) cell = line_cell(d, r, k);
  else {
    const int side = r.axis * 2 + (k < 0 ? 0 : 1);
    if (d.bc[side] == BC_REFLECT) cell = line_cell(d, r, k < 0 ? 0 : r.nk - 1);
  }
  if (cell >= 0) atomicAdd(a.lamRhoH0 + (size_t)cell * d.G + g, l);
}

// A, B of one half and their partial derivatives in x_f, tau_f, x_h.
struct HalfD {
  double A, B, A_xf, A_xh, B_tf, B_xf, B_xh;
};

__device__ __forceinline__ HalfD half_coefs_d(double xf, double tauf, double xh, bool sampled, double dt) {
  HalfD r;
  const CoefDeriv cd = coef_derivs(xf);
  if (sampled) {
    const double dd = xh - xf;
    const double ef = exp(-xf), eh = exp(-xh);
    const double efh = fabs(dd) < 0.5 ? exp(-xh) * expm1(dd) : ef - eh;
    const double f5 = coef_f5(xf);
    r.A = coef_f4(xf) + efh;
    r.B = tauf * f5 - 0.5 * dt * efh;
    r.A_xf = cd.f4 - ef;
    r.A_xh = eh;
    r.B_tf = f5;
    r.B_xf = tauf * cd.f5 + 0.5 * dt * ef;
    r.B_xh = -0.5 * dt * eh;
  } else {
    const double f4 = coef_f4(xf);
    r.A = coef_c4(xf);
    r.B = -tauf * f4;
    r.A_xf = cd.c4;
    r.A_xh = 0.0;
    r.B_tf = -f4;
    r.B_xf = -tauf * cd.f4;
    r.B_xh = 0.0;
  }
  return r;
}

__global__ void k_adj_wave(const __grid_constant__ Dev d, const TapeView t, const AdjView a) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long total = (long long)d.nface * d.G;
  const int G = d.G;
  const double v = d.v, dt = d.dt, rate = d.rate_f;
  for (long long gi = tid; gi < total; gi += stride) {
    const int f = (int)(gi / G), g = (int)(gi - (long long)f * G);
    const FaceRef r = face_ref(d, f);
    const int sideL = r.axis * 2, sideR = sideL + 1;
    const bool lin = r.k - 1 >= 0, rin = r.k < r.nk;
    if ((!lin && d.bc[sideL] == BC_REFLECT) || (!rin && d.bc[sideR] == BC_REFLECT)) continue;
    const int cl = lin ? line_cell(d, r, r.k - 1) : -1, cr = rin ? line_cell(d, r, r.k) : -1;
    const double lRl = lin ? a.lamR[(size_t)cl * G + g] : 0.0;
    const double lRr = rin ? a.lamR[(size_t)cr * G + g] : 0.0;
    const double lF = (dt / r.h) * (lRr - lRl);
    if (lF == 0.0) continue;
    // forward reconstruction
    const double rl = rho_h_tape(d, t, r, r.k - 1, g), rr = rho_h_tape(d, t, r, r.k, g);
    double sl, sr, fl, fr, rll = 0.0, rrr = 0.0;
    if (d.wave_order >= 2) {
      rll = rho_h_tape(d, t, r, r.k - 2, g);
      rrr = rho_h_tape(d, t, r, r.k + 1, g);
      sl = lin ? van_leer((rl - rll) / r.h, (rr - rl) / r.h) : 0.0;
      sr = rin ? van_leer((rr - rl) / r.h, (rrr - rr) / r.h) : 0.0;
      fl = rl + 0.5 * r.h * sl;
      fr = rr - 0.5 * r.h * sr;
    } else {
      sl = sr = (rr - rl) / r.h;
      fl = rl;
      fr = rr;
    }
    // side opacities at T^n and whether the upwind cell was sampled
    double sgl = -1.0, sgr = -1.0, sgl_s = 0.0, sgr_s = 0.0;
    bool el = false, er = false;
    int ghost_l = -1, ghost_r = -1;
    if (lin) {
      sgl = a.sig0[(size_t)cl * G + g];
      el = t.N[(size_t)cl * G + g] > 0;
    } else if (d.bc[sideL] == BC_BLACKBODY) {
      const int cin = line_cell(d, r, 0);
      sgl = d.ghost_sig[sideL * G + g];
      sgl_s = sigma_group_ds(d, sigma_T(d, cin, d.bcT[sideL]), g);
      el = t.N[(size_t)(d.ncell + sideL) * G + g] > 0;
      ghost_l = cin;
    }
    if (rin) {
      sgr = a.sig0[(size_t)cr * G + g];
      er = t.N[(size_t)cr * G + g] > 0;
    } else if (d.bc[sideR] == BC_BLACKBODY) {
      const int cin = line_cell(d, r, r.nk - 1);
      sgr = d.ghost_sig[sideR * G + g];
      sgr_s = sigma_group_ds(d, sigma_T(d, cin, d.bcT[sideR]), g);
      er = t.N[(size_t)(d.ncell + sideR) * G + g] > 0;
      ghost_r = cin;
    }
    const bool vac_l = sgl < 0.0, vac_r = sgr < 0.0;
    if (vac_l) sgl = sgr;
    if (vac_r) sgr = sgl;
    const double sum = sgl + sgr;
    const double sf = 2.0 * sgl * sgr / sum;
    const double tauf = 1.0 / (rate * sf);
    const double xf = dt / tauf;
    const HalfD L = half_coefs_d(xf, tauf, dt * rate * sgl, el, dt);
    const HalfD R = half_coefs_d(xf, tauf, dt * rate * sgr, er, dt);
    // F = AL (v/4) fl - AR (v/4) fr + (BL sl + BR sr) v^2/6
    const double lAL = lF * 0.25 * v * fl, lAR = -lF * 0.25 * v * fr;
    const double lBL = lF * sl * v * v / 6.0, lBR = lF * sr * v * v / 6.0;
    const double l_xf = lAL * L.A_xf + lBL * L.B_xf + lAR * R.A_xf + lBR * R.B_xf;
    const double l_tf = lBL * L.B_tf + lBR * R.B_tf;
    const double l_sf = l_xf * dt * rate + l_tf * (-tauf / sf);
    double l_sl = (lAL * L.A_xh + lBL * L.B_xh) * dt * rate + l_sf * 2.0 * sgr * sgr / (sum * sum);
    double l_sr = (lAR * R.A_xh + lBR * R.B_xh) * dt * rate + l_sf * 2.0 * sgl * sgl / (sum * sum);
    if (vac_l) { l_sr += l_sl; l_sl = 0.0; }
    if (vac_r) { l_sl += l_sr; l_sr = 0.0; }
    if (lin) atomicAdd(a.lamSig0 + (size_t)cl * G + g, l_sl);
    else if (ghost_l >= 0) atomicAdd(a.lamS + ghost_l, l_sl * sgl_s);
    if (rin) atomicAdd(a.lamSig0 + (size_t)cr * G + g, l_sr);
    else if (ghost_r >= 0) atomicAdd(a.lamS + ghost_r, l_sr * sgr_s);
    // rho_h through the reconstruction
    const double lfl = lF * L.A * 0.25 * v, lfr = -lF * R.A * 0.25 * v;
    double lsl = lF * L.B * v * v / 6.0, lsr = lF * R.B * v * v / 6.0;
    double lrl = 0.0, lrr = 0.0, lrll = 0.0, lrrr = 0.0;
    if (d.wave_order >= 2) {
      lrl += lfl;
      lsl += 0.5 * r.h * lfl;
      lrr += lfr;
      lsr -= 0.5 * r.h * lfr;
      if (lin) {
        const double a1 = (rl - rll) / r.h, b1 = (rr - rl) / r.h;
        if (a1 * b1 > 0.0) {
          const double s2 = (a1 + b1) * (a1 + b1);
          const double la = lsl * 2.0 * b1 * b1 / s2, lb = lsl * 2.0 * a1 * a1 / s2;
          lrl += (la - lb) / r.h;
          lrll -= la / r.h;
          lrr += lb / r.h;
        }
      }
      if (rin) {
        const double a2 = (rr - rl) / r.h, b2 = (rrr - rr) / r.h;
        if (a2 * b2 > 0.0) {
          const double s2 = (a2 + b2) * (a2 + b2);
          const double la = lsr * 2.0 * b2 * b2 / s2, lb = lsr * 2.0 * a2 * a2 / s2;
          lrr += (la - lb) / r.h;
          lrl -= la / r.h;
          lrrr += lb / r.h;
        }
      }
    } else {
      lrl += lfl - (lsl + lsr) / r.h;
      lrr += lfr + (lsl + lsr) / r.h;
    }
    add_rho_h(d, a, r, r.k - 1, g, lrl);
    add_rho_h(d, a, r, r.k, g, lrr);
    if (d.wave_order >= 2) {
      add_rho_h(d, a, r, r.k - 2, g, lrll);
      add_rho_h(d, a, r, r.k + 1, g, lrrr);
    }
  }
}

// --------------------------------------------------------------------------
// Weight adjoints of the processed particles.  Along its path a particle of
// weight w adds w to W of its end cell (survived or collided), takes w from W
// of its start cell (started inside), and adds w to E_surv of its end cell
// if it survived, where it also becomes input particle `slot` of the next
// step.  With lambda_W = lambda_R/V and lambda_Esurv = -lambda(rho_h^{n+1})/V:
//   lambda_w = [end] lambda_W(c1) - [start inside] lambda_W(c0)
//            + [survived] (lambda_Esurv(c1) + lambda_w^{next}(slot)).
// Incoming particles keep lambda_w for the previous step; a newborn of bin b
// passes lambda_w / N_b to lambda_E(b).
__device__ __forceinline__ void warp_run_add_adj(double* base, long long key, double v) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long prev = __shfl_up_sync(full, key, 1);
  const bool head = lane == 0 || prev != key;
  const unsigned heads = __ballot_sync(full, head);
  const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double tv = __shfl_up_sync(full, v, o);
    if (lane - o >= start) v += tv;
  }
  const long long nxt = __shfl_down_sync(full, key, 1);
  const bool tail = lane == 31 || nxt != key;
  if (tail && key >= 0) atomicAdd(base + key, v);
}

__global__ void __launch_bounds__(256) k_adj_particles(const __grid_constant__ Dev d, const TapeView t,
                                                       const AdjView a) {
  const long long n_in = (long long)t.hdr->n_in, n_new = (long long)t.hdr->n_new;
  const long long n = n_in + n_new;
  if (n > t.rec_cap || n_in > a.cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctrl->status, ST_CAPACITY);
    return;
  }
  const unsigned int cur = a.ctrl->cur;
  const double* __restrict__ lw_next = a.lamW[cur];
  double* __restrict__ lw_out = a.lamW[cur ^ 1u];
  const int G = d.G;
  const double invV = 1.0 / d.vol;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // whole warps iterate together (the run aggregation needs all lanes)
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
    const long long k = base + threadIdx.x;
    long long key = -1;
    double l = 0.0;
    if (k < n) {
      const TapeRec tr = t.rec[k];
      const int g = tr.g;
      if (tr.c1 >= 0) l += a.lamR[(size_t)tr.c1 * G + g] * invV;
      if (tr.c0 >= 0) l -= a.lamR[(size_t)tr.c0 * G + g] * invV;
      if (tr.slot >= 0) {
        const size_t b = (size_t)tr.c1 * G + g;
        const double f = t.wscale[b];
        if (f == 1.0) l += -a.lamRhoH[b] * invV + lw_next[tr.slot];
        else if (f > 0.0) l += lw_next[tr.slot] * f - t.rho1[b] * d.vol / (t.Esurv[b] * t.Esurv[b]) * a.Sb[b];
      }
      if (k < n_in) {
        lw_out[k] = l;
      } else {
        const int cb = tr.c0 >= 0 ? tr.c0 : d.ncell + (-1 - tr.c0);
        key = (long long)cb * G + g;
        const uint32_t N = t.N[key];
        l = N ? l / (double)N : 0.0;
      }
    }
    warp_run_add_adj(a.lamE, key, key >= 0 ? l : 0.0);
  }
}

// --------------------------------------------------------------------------
// Births and group opacities at T^n (one warp per cell), then the new
// adjoint state.  E = e max(rho_h, 0) V with e = exp(-dt rate sigma_g):
//   lambda(rho_h^n) += lambda_E e V [rho_h > 0],
//   lambda(sigma_g) += lambda_E max(rho_h, 0) V (-e dt rate);
// black-body ghost bins (1D) carry E = e (v/4) Phi_g(T_b) dt with the ghost
// opacity from the inner cell's sigma0.  Then
//   lambda(T^n) = Cv mu + sum_g lambda(sigma_g) dsigma_g/dT,
//   dL/ds_c    += sum_g lambda(sigma_g) dsigma_g/ds.
template <int NC>
__global__ void __launch_bounds__(256) k_adj_birth(const __grid_constant__ Dev d, const TapeView t,
                                                   const AdjView a) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  const long long gw = blockIdx.x * (long long)nwb + wib, nw = (long long)gridDim.x * nwb;
  const int G = d.G, ncell = d.ncell;
  const double dt = d.dt, rate = d.rate_f, V = d.vol;
  for (long long cc = gw; cc < ncell; cc += nw) {
    const int c = (int)cc;
    const double T0 = t.T0[c];
    double lT = 0.0, lS = 0.0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const int g = lane + 32 * j;
      if (g >= G) continue;
      const size_t i = (size_t)c * G + g;
      double lsig = a.lamSig0[i], lrh = a.lamRhoH0[i];
      if (t.N[i] > 0) {
        const double e = exp(-dt * rate * a.sig0[i]);
        const double rh = t.rho_h0[i];
        const double lE = a.lamE[i];
        lsig += lE * (rh > 0.0 ? rh : 0.0) * V * (-e * dt * rate);
        if (rh > 0.0) lrh += lE * e * V;
      }
      const double s0s = a.sig0s[i];
      lT += lsig * d.sig_q / T0 * s0s;
      lS += lsig * s0s;
      a.lamRhoH[i] = lrh;
      a.lamRho[i] = a.lamR[i];
      // black-body ghost bins fed through this boundary cell (1D)
      if (d.dim == 1) {
        for (int side = 0; side < 2; ++side) {
          const int cin = side == 0 ? 0 : d.nx - 1;
          if (c != cin || d.bc[side] != BC_BLACKBODY) continue;
          const size_t b = (size_t)(ncell + side) * G + g;
          if (t.N[b] == 0) continue;
          const double sg = d.ghost_sig[side * G + g];
          const double e = exp(-dt * rate * sg);
          const double lsg = a.lamE[b] * 0.25 * d.v * d.ghost_phi[side * G + g] * dt * (-e * dt * rate);
          lS += lsg * sigma_group_ds(d, sigma_T(d, c, d.bcT[side]), g);
        }
      }
    }
    lT = warp_sum(lT);
    lS = warp_sum(lS);
    if (lane == 0) {
      a.lamT[c] = a.lamT0[c] + lT;
      a.lamS[c] += lS;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->cur ^= 1u;
}

// --------------------------------------------------------------------------
// Re-indexing across a checkpoint boundary.  Survivors are compacted in a
// thread-order-dependent order, so the particles a checkpoint holds and the
// same particles at the end of the recomputed previous segment are in
// different orders.  The weight adjoints of the checkpoint's order go into an
// open-addressing hash keyed by particle identity and are read back in the
// handle's current order; a particle found on one side only (a Monte Carlo
// decision that flipped under the roundoff of the recomputation) gets 0 and
// is counted.
constexpr unsigned long long kEmpty = ~0ull;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  // SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA'14)
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_hash_clear(AdjView a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.hsize;
       i += (long long)gridDim.x * blockDim.x)
    a.hkeys[i] = kEmpty;
}

__global__ void k_hash_insert(AdjView a, const Ctrl* saved, const unsigned long long* ids) {
  const long long n = (long long)saved->n_part[saved->cur];
  const double* lam = a.lamW[a.ctrl->cur];
  const unsigned long long mask = (unsigned long long)a.hsize - 1ull;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n && i < a.cap;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long key = ids[i];
    unsigned long long h = mix64(key) & mask;
    for (long long probe = 0; probe < a.hsize; ++probe, h = (h + 1) & mask) {
      const unsigned long long prev = atomicCAS(a.hkeys + h, kEmpty, key);
      if (prev == kEmpty || prev == key) { a.hvals[h] = lam[i]; break; }
    }
  }
}

__global__ void k_hash_lookup(const __grid_constant__ Dev d, AdjView a) {
  const Ctrl* ctrl = d.ctrl;
  const unsigned cur = ctrl->cur;
  const long long n = (long long)ctrl->n_part[cur];
  const unsigned long long* ids = d.pid[cur];
  double* out = a.lamW[a.ctrl->cur ^ 1u];
  const unsigned long long mask = (unsigned long long)a.hsize - 1ull;
  unsigned long long miss = 0;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
       s += (long long)gridDim.x * blockDim.x) {
    const unsigned long long key = ids[s];
    unsigned long long h = mix64(key) & mask;
    double v = 0.0;
    bool found = false;
    for (long long probe = 0; probe < a.hsize; ++probe, h = (h + 1) & mask) {
      const unsigned long long k = a.hkeys[h];
      if (k == key) { v = a.hvals[h]; found = true; break; }
      if (k == kEmpty) break;
    }
    if (!found) ++miss;
    out[s] = v;
  }
  if (miss) atomicAdd(&a.ctrl->unmatched, miss);
}

__global__ void k_adj_flip(AdjView a) { a.ctrl->cur ^= 1u; }

cudaError_t launch_adjoint_remap(const Dev& d, const AdjView& a, const char* ckpt_member, cudaStream_t s) {
  const Ctrl* saved = reinterpret_cast<const Ctrl*>(ckpt_member + ckpt_ctrl_offset(d));
  const unsigned long long* ids = reinterpret_cast<const unsigned long long*>(ckpt_member + ckpt_ids_offset(d));
  k_hash_clear<<<sm_count() * 8, 256, 0, s>>>(a);
  k_hash_insert<<<sm_count() * 8, 256, 0, s>>>(a, saved, ids);
  k_hash_lookup<<<sm_count() * 8, 256, 0, s>>>(d, a);
  k_adj_flip<<<1, 1, 0, s>>>(a);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// host launchers

static int g_adj_si_per[2][2] = {};

template <int NC>
static cudaError_t launch_adj_si_t(const Dev& d, const TapeView& t, const AdjView& a, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int small = d.ncell <= 8 * sms;
  const int threads = small ? 32 : 256;
  int& per = g_adj_si_per[NC - 1][small];
  if (!per) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_adj_si<NC>, threads, 0);
    if (per < 1) per = 1;
  }
  const long long want = ((long long)d.ncell * 32 + threads - 1) / threads;
  const long long maxb = (long long)sms * per;
  int blocks = (int)(want < maxb ? want : maxb);
  if (blocks < 1) blocks = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_adj_si<NC>, d, t, a);
}

cudaError_t launch_adjoint_step(const Dev& d, const TapeView& t, const AdjView& a, cudaStream_t s) {
  cudaError_t r = cudaMemsetAsync(&a.ctrl->bar_count, 0, sizeof(unsigned int), s);
  if (r) return r;
  r = cudaMemsetAsync(a.ctrl->err_slot, 0, sizeof(a.ctrl->err_slot), s);
  if (r) return r;
  r = cudaMemsetAsync(a.Sb, 0, sizeof(double) * (size_t)d.ncell * d.G, s);
  if (r) return r;
  k_adj_scale_sums<<<sm_count() * 4, 256, 0, s>>>(d, t, a);
  r = d.G > 32 ? launch_adj_si_t<2>(d, t, a, s) : launch_adj_si_t<1>(d, t, a, s);
  if (r) return r;
  const long long nfg = (long long)d.nface * d.G;
  long long wb = (nfg + 127) / 128;
  if (wb > sm_count() * 32) wb = sm_count() * 32;
  k_adj_wave<<<(int)(wb > 0 ? wb : 1), 128, 0, s>>>(d, t, a);
  k_adj_particles<<<sm_count() * 8, 256, 0, s>>>(d, t, a);
  long long cb = ((long long)d.ncell * 32 + 255) / 256;
  if (cb > sm_count() * 16) cb = sm_count() * 16;
  if (d.G > 32) k_adj_birth<2><<<(int)cb, 256, 0, s>>>(d, t, a);
  else k_adj_birth<1><<<(int)cb, 256, 0, s>>>(d, t, a);
  return cudaGetLastError();
}

}  // namespace ugkwp
