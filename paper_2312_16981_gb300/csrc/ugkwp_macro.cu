// ugkwp_macro.cu -- cell/face kernels of the UGKWP step on sm_103a:
// birth counts and their scan (Eq. IhpFormula), the wave-part flux (Sec. 2.2),
// the matrix-free source iteration (App. B, Algorithm 2) as one cooperative
// persistent kernel, the end-of-step bookkeeping, initialisation, and the
// kernel-level entry points used by the parity tests.
#include "ugkwp_device.cuh"
#include "ugkwp_grid.cuh"
#include "ugkwp_launch.h"
#include "ugkwp_si.cuh"

namespace ugkwp {

// --------------------------------------------------------------------------
// Initialisation: Phi_g(T0) where rho0 is not given, ghost tables, source.
__device__ void phi_dphi_cell(const Dev& d, double T, int g, double* phi, double* dphi) {
  // Phi_g(T) = a c T^4 b_g(T), dPhi_g/dT = a c T^3 (4 b_g + ...); grey: b = 1
  if (!(T > 0.0)) { *phi = 0.0; if (dphi) *dphi = 0.0; return; }
  const double ac = d.a * d.c, T3 = T * T * T;
  if (d.grey) { *phi = ac * T3 * T; if (dphi) *dphi = 4.0 * ac * T3; return; }
  const EdgeVal lo = planck_edge(d.nu_edges[g] / T), hi = planck_edge(d.nu_edges[g + 1] / T);
  const double b = planck_fraction(lo, hi);
  *phi = ac * T3 * T * b;
  if (dphi) *dphi = ac * T3 * planck_dfraction(b, lo, hi);
}

__global__ void k_init_pow(Dev d) {
  // nu^p at the Simpson points and FP32 edges; before anything uses sigma_group
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (int g = tid; g < d.G; g += stride) {
    const double a = d.nu_edges[g], b = d.nu_edges[g + 1], m = 0.5 * (a + b);
    double* np = const_cast<double*>(d.nu_pow);
    np[3 * g] = d.grey ? 1.0 : pow_fast(a, d.sig_p);
    np[3 * g + 1] = d.grey ? 1.0 : pow_fast(m, d.sig_p);
    np[3 * g + 2] = d.grey ? 1.0 : pow_fast(b, d.sig_p);
  }
  for (int g = tid; g <= d.G; g += stride)
    if (d.nu_edges_f) d.nu_edges_f[g] = (float)d.nu_edges[g];
  // FP32 copies of the interpolant tables (the same on every call)
  for (int i = tid; i < (kPlanckRows + 1) * (kPlanckDeg + 1); i += stride) {
    kP1TabF[i] = (float)kPlanckTab[2 * i];
    kG4TabF[i] = (float)kPlanckTab[2 * i + 1];
    kC2TabF[i] = (float)kC2Tab[i];
  }
  if (d.nu_pow_f)
    for (int g = tid; g < d.G; g += stride) {
      const double a = d.nu_edges[g], b = d.nu_edges[g + 1], m = 0.5 * (a + b);
      d.nu_pow_f[3 * g] = d.grey ? 1.0f : (float)pow_fast(a, d.sig_p);
      d.nu_pow_f[3 * g + 1] = d.grey ? 1.0f : (float)pow_fast(m, d.sig_p);
      d.nu_pow_f[3 * g + 2] = d.grey ? 1.0f : (float)pow_fast(b, d.sig_p);
    }
  // foam opacity nu factors at the Simpson points (sig_law 2)
  if (d.olson_nu)
    for (int g = tid; g < d.G; g += stride) {
      const double a = d.nu_edges[g], b = d.nu_edges[g + 1], pts[3] = {a, 0.5 * (a + b), b};
      for (int k = 0; k < 3; ++k) {
        double* t = d.olson_nu + 9 * g + 3 * k;
        foam_nu(pts[k], t, t + 1, t + 2);
        if (d.olson_nu_f)
          for (int q = 0; q < 3; ++q) d.olson_nu_f[9 * g + 3 * k + q] = (float)t[q];
      }
    }
}

__global__ void k_init_tables(Dev d, const double* src_T, const double* src_amp, int init_rho) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const int n = d.ncell * d.G;
  for (int i = tid; i < n; i += stride) {
    const int c = i / d.G, g = i - c * d.G;
    if (init_rho) {
      double p;
      phi_dphi_cell(d, d.T[c], g, &p, nullptr);
      d.rho[i] = p;
      d.rho_h[i] = p;
      d.rho_p[i] = 0.0;
    }
    if (d.src) {
      double p = 0.0;
      if (src_T && src_T[c] > 0.0) phi_dphi_cell(d, src_T[c], g, &p, nullptr);
      const_cast<double*>(d.src)[i] = d.src_on * (src_amp ? src_amp[c] : 1.0) * d.c * d.dt * p;
    }
  }
  for (int i = tid; i < 6 * d.G; i += stride) {
    const int side = i / d.G, g = i - side * d.G;
    double p = 0.0, s = 0.0;
    if (d.bc[side] == BC_BLACKBODY) {
      const int cin = side == 0 ? 0 : (side == 1 ? d.nx - 1 : 0);
      phi_dphi_cell(d, d.bcT[side], g, &p, nullptr);
      s = sigma_group_at(d, sigma_T(d, cin, d.bcT[side]), d.bcT[side], g);
    }
    const_cast<double*>(d.ghost_phi)[i] = p;
    const_cast<double*>(d.ghost_sig)[i] = s;
  }
}

// --------------------------------------------------------------------------
// Birth counts (Eq. IhpFormula, weight formula of Sec. 2.2): per bin the
// collisionless part E = e^{-dt/tau} max(rho_h, 0) V, tau from the Simpson
// group opacity at T^n, N = floor(E/omega_ref + 1/2), omega = E/N, e_eff = e
// if N > 0 else 0 (UGKP: an interior bin samples E = max(rho_h, 0) V and
// marks e_eff = -1).  Black-body ghost bins (1D) carry the entering part of the
// ghost's collisionless particles, E = e (c/eps)/4 Phi_g(T_b) dt.  Also
// stores sigma_g(T^n), sigma0 T^q per cell, the sampler slope per bin, zeroes
// this step's tallies and resets the per-step counters.
template <bool ENS>
__global__ void k_birth(const __grid_constant__ Dev d0, const Ens e) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long total = ENS ? e.total_bins : (long long)d0.nbins;
  for (long long gb = tid; gb < total; gb += stride) {
  const int m = ENS ? find_member(e.bin0, e.M, gb) : 0;
  const Dev& d = ENS ? e.devs[m] : d0;
  const int b = (int)(ENS ? gb - e.bin0[m] : gb);
  Ctrl* ctrl = d.ctrl;
  if (b == 0) {
    ctrl->n_new = 0;
    ctrl->n_out = 0;
    ctrl->n_in = ctrl->n_part[ctrl->cur];
    ctrl->n_born = ctrl->n_survived = ctrl->n_absorbed = ctrl->n_escaped = 0;
    ctrl->n_removed = ctrl->n_segments = 0;
    ctrl->bar_count = 0;
    ctrl->scaled = 0;
    ctrl->tile_next = 0;
    ctrl->n_scaled_bins = 0;
    for (int s = 0; s < 3; ++s) ctrl->err_slot[s][0] = ctrl->err_slot[s][1] = 0ull;
    ctrl->E_rad0 = ctrl->E_mat0 = ctrl->E_rad1 = ctrl->E_mat1 = 0.0;
    ctrl->bnd_in_macro = ctrl->bnd_in_part = ctrl->bnd_out_part = ctrl->src_in = 0.0;
  }
  const int G = d.G;
  d.sort_cnt[b] = 0u;   // the particle kernel counts the survivors it stores per bin
  {
    const int cell = b / G, g = b - cell * G;
    double E, sig, Tb;
    if (cell < d.ncell) {
      Tb = d.T[cell];
      const double sT = sigma_T(d, cell, Tb);
      if (g == 0) {
        d.sT[cell] = sT;
        d.sTinv[cell] = 1.0 / sT;
        if (d.sT_f) {
          d.sT_f[cell] = (float)sT;
          d.sTinv_f[cell] = (float)(1.0 / sT);
          d.invT_f[cell] = (float)(1.0 / Tb);
        }
        if (d.olson_c) {   // foam opacity T factors at T^n for the particles
          const FoamT f = foam_T(Tb);
          d.olson_c[3 * cell] = f.A; d.olson_c[3 * cell + 1] = f.B; d.olson_c[3 * cell + 2] = f.C;
          if (d.olson_cf) {
            d.olson_cf[3 * cell] = (float)f.A; d.olson_cf[3 * cell + 1] = (float)f.B;
            d.olson_cf[3 * cell + 2] = (float)f.C;
          }
        }
      }
      sig = sigma_group_at(d, sT, Tb, g);
      d.sigT[b] = sig;
      d.W[b] = 0.0;
      d.E_surv[b] = 0.0;
      d.Wq[2 * b] = 0ull; d.Wq[2 * b + 1] = 0ull;
      d.Esq[2 * b] = 0ull; d.Esq[2 * b + 1] = 0ull;
      const double rh = d.rho_h[b];
      E = (rh > 0.0 ? rh : 0.0) * d.vol;
    } else {
      const int side = cell - d.ncell;
      d.esc[side * G + g] = 0.0;
      d.inflow[side * G + g] = 0.0;
      if (side < 2) {   // the z sides' tallies (bins hold four ghost slots)
        d.esc[(side + 4) * G + g] = 0.0;
        d.inflow[(side + 4) * G + g] = 0.0;
      }
      if (d.dim != 1 || side > 1 || d.bc[side] != BC_BLACKBODY) {
        d.N[b] = 0; d.omega[b] = 0.0; d.e_eff[b] = 0.0; d.khat[b] = 0.0;
        if (d.omega_f) { d.omega_f[b] = 0.0f; d.khat_f[b] = 0.0f; }
        continue;
      }
      sig = d.ghost_sig[side * G + g];
      Tb = d.bcT[side];
      E = 0.25 * d.v * d.ghost_phi[side * G + g] * d.dt;
    }
    // sampled fraction e = exp(-dt/tau_num): tau_num = tau + C J dt at thin/thick
    // joints (Sec. 3.2), J the largest |T_c - T_n|/(T_c + T_n) over the cell's
    // interior faces; x = dt/tau when C = 0
    double x = d.dt * d.rate_f * sig;
    if (cell < d.ncell && d.tau_num_C > 0.0) {
      int ix, iy, iz;
      cell_xyz(d, cell, &ix, &iy, &iz);
      double J = 0.0;
      for (int k = 0; k < 2 * d.dim; ++k) {
        const int s = (k & 1) ? 1 : -1;
        const int jx = ix + (k < 2 ? s : 0), jy = iy + (k >> 1 == 1 ? s : 0), jz = iz + (k >> 1 == 2 ? s : 0);
        if (jx < 0 || jx >= d.nx || jy < 0 || jy >= d.ny || jz < 0 || jz >= d.nz) continue;
        const double Tn = d.T[(jz * d.ny + jy) * d.nx + jx];
        J = fmax(J, fabs(Tb - Tn) / (Tb + Tn));
      }
      x = x / (1.0 + d.tau_num_C * J * x);
    }
    d.xnum[b] = x;
    const double e = exp(-x);
    const bool all = d.method == 1 && cell < d.ncell;   // UGKP: the whole wave part
    if (!all) E *= e;
    uint32_t N = 0;
    double w = 0.0, ee = 0.0;
    // a newborn's identity holds its birth step in 20 bits: past that no
    // particle is sampled (the step is flagged)
    const bool id_ok = d.ctrl->step <= kMaxStep;
    if (!id_ok && b == 0) atomicOr(&ctrl->status, ST_IDSPACE);
    if (id_ok && d.omega_ref > 0.0 && E > 0.0) {
      double q = floor(E / d.omega_ref + 0.5);
      if (q > (double)kMaxPerBin) { q = (double)kMaxPerBin; atomicOr(&ctrl->status, ST_CAPACITY); }
      N = (uint32_t)q;
      if (N) { w = E / (double)N; ee = all ? -1.0 : e; }
    }
    d.N[b] = N;
    d.omega[b] = w;
    d.e_eff[b] = ee;
    // the sampler slope: FP64 for the FP64 particle kernel; the FP32 kernel
    // samples in FP32 and takes it from FP32 arithmetic (the FP64 exp and
    // expm1 cost tens of FP64 instructions each on this chip)
    if (d.omega_f) {
      d.khat[b] = 0.0;
      d.omega_f[b] = (float)w;
      d.khat_f[b] = (N && !d.grey) ? sampler_khat_f(d.nu_edges_f[g], d.nu_edges_f[g + 1], (float)Tb) : 0.0f;
    } else {
      d.khat[b] = (N && !d.grey) ? sampler_khat(d.nu_edges[g], d.nu_edges[g + 1], Tb) : 0.0;
    }
  }
  }
}

// --------------------------------------------------------------------------
// Exclusive scan of the birth counts: per-block sums, a one-block scan of
// the sums, then per-block scans with their offsets.  Tile = 4096 bins.
constexpr int kScanThreads = 1024, kScanPer = 4, kScanTile = kScanThreads * kScanPer;
static_assert(kScanTile == kScanTileCounts, "scan tile and the scratch size it implies");

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_tot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_warp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t x = lane < nw ? s_warp[lane] : 0u, xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += t;
    }
    if (lane < nw) s_warp[lane] = xi - x;
    if (lane == nw - 1) s_tot = xi;   // block total
  }
  __syncthreads();
  const uint32_t res = s_warp[wid] + inc - v;
  if (total) *total = s_tot;
  __syncthreads();
  return res;
}

__device__ __forceinline__ void scan_reduce_body(const uint32_t* __restrict__ N, long long n,
                                                 uint32_t* __restrict__ part, int blk) {
  const long long base = (long long)blk * kScanTile + (long long)threadIdx.x * kScanPer;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k)
    if (base + k < n) s += N[base + k];
  uint32_t tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) part[blk] = tot;
}

// one block: exclusive scan of nparts (<= kScanTile) block sums in place; the
// grand total goes to off[n] and, when given, to two 64-bit counters
__device__ __forceinline__ void scan_partials_body(uint32_t* __restrict__ part, int nparts,
                                                   uint32_t* __restrict__ off_total,
                                                   unsigned long long* total_a, unsigned long long* total_b) {
  const int base = threadIdx.x * kScanPer;
  uint32_t v[kScanPer], s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) { v[k] = base + k < nparts ? part[base + k] : 0u; s += v[k]; }
  uint32_t tot;
  uint32_t ex = block_exclusive_scan(s, &tot);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < nparts) part[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) {
    *off_total = tot;
    if (total_a) *total_a = tot;
    if (total_b) *total_b = tot;
  }
}

__device__ __forceinline__ void scan_apply_body(const uint32_t* __restrict__ N, long long n,
                                                const uint32_t* __restrict__ part, uint32_t* __restrict__ off,
                                                int blk) {
  const long long base = (long long)blk * kScanTile + (long long)threadIdx.x * kScanPer;
  uint32_t v[kScanPer], s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) { v[k] = base + k < n ? N[base + k] : 0u; s += v[k]; }
  uint32_t ex = block_exclusive_scan(s, nullptr) + part[blk];
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < n) off[base + k] = ex;
    ex += v[k];
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ N, long long n,
                                                             uint32_t* __restrict__ part) {
  scan_reduce_body(N, n, part, blockIdx.x);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partials(uint32_t* __restrict__ part, int nparts,
                                                               uint32_t* __restrict__ off_total,
                                                               unsigned long long* total_a,
                                                               unsigned long long* total_b) {
  scan_partials_body(part, nparts, off_total, total_a, total_b);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t* __restrict__ N, long long n,
                                                            const uint32_t* __restrict__ part,
                                                            uint32_t* __restrict__ off) {
  scan_apply_body(N, n, part, off, blockIdx.x);
}

// Ensemble: one scan per member, member = blockIdx.y; which = 0 scans the
// birth counts (totals to n_new, n_born), which = 1 the survivors per bin of
// the sort (total to n_out).
struct ScanArrays {
  const uint32_t* cnt;
  uint32_t *off, *part;
  unsigned long long *total_a, *total_b;
};

__device__ __forceinline__ ScanArrays scan_arrays(const Dev& d, int which) {
  if (which) return ScanArrays{d.sort_cnt, d.sort_off, d.sort_part, &d.ctrl->n_out, nullptr};
  return ScanArrays{d.N, d.off, d.part, &d.ctrl->n_new, &d.ctrl->n_born};
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce_ens(const Ens e, int which) {
  const Dev& d = e.devs[blockIdx.y];
  if ((long long)blockIdx.x * kScanTile >= d.nbins) return;
  const ScanArrays a = scan_arrays(d, which);
  scan_reduce_body(a.cnt, d.nbins, a.part, blockIdx.x);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partials_ens(const Ens e, int which) {
  const Dev& d = e.devs[blockIdx.y];
  const ScanArrays a = scan_arrays(d, which);
  scan_partials_body(a.part, (d.nbins + kScanTile - 1) / kScanTile, a.off + d.nbins, a.total_a, a.total_b);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply_ens(const Ens e, int which) {
  const Dev& d = e.devs[blockIdx.y];
  if ((long long)blockIdx.x * kScanTile >= d.nbins) return;
  const ScanArrays a = scan_arrays(d, which);
  scan_apply_body(a.cnt, d.nbins, a.part, a.off, blockIdx.x);
}

// Ensemble: prefix over members of this step's particle tiles (survivors +
// newborns, tiles of e.tile particles), one block; also resets the barrier.
__global__ void __launch_bounds__(1024) k_tiles(const Ens e) {
  const unsigned long long kParticleTile = (unsigned long long)e.tile;
  __shared__ int s_carry;
  if (threadIdx.x == 0) { s_carry = 0; *e.bar = 0u; *e.tile_next = 0ull; }
  __syncthreads();
  for (int base = 0; base < e.M; base += blockDim.x) {
    const int m = base + threadIdx.x;
    uint32_t t = 0;
    if (m < e.M) {
      const Ctrl* c = e.devs[m].ctrl;
      const unsigned long long n = c->n_part[c->cur] + c->n_new;
      t = (uint32_t)((n + kParticleTile - 1) / kParticleTile);
    }
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan(t, &tot);
    if (m < e.M) e.tile0[m] = s_carry + (int)ex;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += (int)tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) e.tile0[e.M] = s_carry;
}

// A = C4_f - e_h, B = C5_f + dt e_h/2 of one half (face coefficients f4, f5,
// c4 at x_f shared by both halves; upwind e).  e_eff > 0 is exp(-x_h) itself
// (the birth kernel's value), so e_f - e_h = e_h expm1(x_h - x_f) takes one
// expm1, or uses e_f = exp(-x_f) (ef, when the face coefficients computed it;
// ef < 0 otherwise).
__device__ __forceinline__ void half_coefs(double xf, double ef, double tauf, double xh, double e_eff,
                                           double dt, double f4, double f5, double c4,
                                           double* A, double* B) {
  if (e_eff < 0.0) {
    // UGKP: the particles carry this half's whole free transport
    *A = 0.0;
    *B = 0.0;
  } else if (e_eff > 0.0) {
    const double dd = xh - xf;
    const double efh = fabs(dd) < 0.5 ? e_eff * expm1(dd) : (ef >= 0.0 ? ef : exp(-xf)) - e_eff;
    *A = f4 + efh;
    *B = tauf * f5 - 0.5 * dt * efh;
  } else {
    *A = c4;
    *B = -tauf * f4;
  }
}

// Wave-part flux F^{fr,wave} on every (face, group) (Sec. 2.2): upwind
// half-range integrals with C4, C5 from the harmonic-mean face opacity and the
// sampled fraction e of the upwind cell; wave_order 2 reconstructs rho_h with
// van Leer slopes.  Reflecting walls carry none.
template <bool ENS>
__global__ void k_wave(const __grid_constant__ Dev d0, const Ens e) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long total = ENS ? e.total_fg : (long long)d0.nface * d0.G;
  for (long long gi = tid; gi < total; gi += stride) {
    const int m = ENS ? find_member(e.fg0, e.M, gi) : 0;
    const Dev& d = ENS ? e.devs[m] : d0;
    const int i = (int)(ENS ? gi - e.fg0[m] : gi);
    const int G = d.G;
    const double v = d.v;
    const int f = i / G, g = i - f * G;
    const FaceRef r = face_ref(d, f);
    const int sideL = r.axis * 2, sideR = sideL + 1;
    const bool lin = r.k - 1 >= 0, rin = r.k < r.nk;
    if ((!lin && d.bc[sideL] == BC_REFLECT) || (!rin && d.bc[sideR] == BC_REFLECT)) {
      d.Fwave[i] = 0.0;
      continue;
    }
    const double rl = rho_h_at(d, r, r.k - 1, g), rr = rho_h_at(d, r, r.k, g);
    double sl, sr, fl, fr;
    if (d.wave_order >= 2) {
      const double rll = rho_h_at(d, r, r.k - 2, g), rrr = rho_h_at(d, r, r.k + 1, g);
      const double ih = inv_h_of(d, r.axis);
      sl = lin ? van_leer((rl - rll) * ih, (rr - rl) * ih) : 0.0;
      sr = rin ? van_leer((rr - rl) * ih, (rrr - rr) * ih) : 0.0;
      fl = rl + 0.5 * r.h * sl;
      fr = rr - 0.5 * r.h * sr;
    } else {
      sl = sr = (rr - rl) / r.h;
      fl = rl;
      fr = rr;
    }
    double sgl = -1.0, sgr = -1.0, el = 0.0, er = 0.0, xhl = 0.0, xhr = 0.0;
    if (lin) {
      const int cl = line_cell(d, r, r.k - 1);
      sgl = d.sigT[cl * G + g];
      el = d.e_eff[cl * G + g];
      xhl = d.xnum[cl * G + g];
    } else if (d.bc[sideL] == BC_BLACKBODY) {
      sgl = d.ghost_sig[sideL * G + g];
      el = d.e_eff[(d.ncell + sideL) * G + g];
      xhl = d.xnum[(d.ncell + sideL) * G + g];
    }
    if (rin) {
      const int cr = line_cell(d, r, r.k);
      sgr = d.sigT[cr * G + g];
      er = d.e_eff[cr * G + g];
      xhr = d.xnum[cr * G + g];
    } else if (d.bc[sideR] == BC_BLACKBODY) {
      sgr = d.ghost_sig[sideR * G + g];
      er = d.e_eff[(d.ncell + sideR) * G + g];
      xhr = d.xnum[(d.ncell + sideR) * G + g];
    }
    if (sgl < 0.0) sgl = sgr;
    if (sgr < 0.0) sgr = sgl;
    // harmonic-mean face opacity: x_f = dt rate 2 sl sr/(sl + sr), tau_f = dt/x_f
    const double xf = d.dt * d.rate_f * (2.0 * sgl * sgr) / (sgl + sgr);
    const double tauf = d.dt / xf;
    double AL, BL, AR, BR, f4, f5, c4;
    const double ef = coef_f4_f5_c4(xf, &f4, &f5, &c4);
    half_coefs(xf, ef, tauf, xhl, el, d.dt, f4, f5, c4, &AL, &BL);
    half_coefs(xf, ef, tauf, xhr, er, d.dt, f4, f5, c4, &AR, &BR);
    d.Fwave[i] = AL * (v * 0.25) * fl - AR * (v * 0.25) * fr + (BL * sl + BR * sr) * (v * v / 6.0);
  }
}

// The wave-part flux of the mixed-precision build in FP32: the same upwind
// half-range expression as k_wave, from FP32 copies of rho^h, sigma_g(T^n),
// the sampled fractions and dt/tau_num, with the C4, C5 series (below x = 1,
// 12 terms) or closed forms in FP32; stored as a double.  Each face keeps
// one flux that both cells use, so the energy ledger still closes to
// roundoff; the flux itself carries FP32 rounding (relative error about
// 1e-6 where C5's closed form cancels near x = 1).
constexpr int kSerF = 12;
__device__ constexpr float kA4F[kSerF + 1] = {(float)a4(0), (float)a4(1), (float)a4(2), (float)a4(3), (float)a4(4),
                                              (float)a4(5), (float)a4(6), (float)a4(7), (float)a4(8), (float)a4(9),
                                              (float)a4(10), (float)a4(11), (float)a4(12)};
__device__ constexpr float kA5F[kSerF + 1] = {(float)a5(0), (float)a5(1), (float)a5(2), (float)a5(3), (float)a5(4),
                                              (float)a5(5), (float)a5(6), (float)a5(7), (float)a5(8), (float)a5(9),
                                              (float)a5(10), (float)a5(11), (float)a5(12)};
__device__ constexpr float kAC4F[kSerF + 1] = {(float)ac4(0), (float)ac4(1), (float)ac4(2), (float)ac4(3), (float)ac4(4),
                                               (float)ac4(5), (float)ac4(6), (float)ac4(7), (float)ac4(8), (float)ac4(9),
                                               (float)ac4(10), (float)ac4(11), (float)ac4(12)};

__device__ __forceinline__ float coef_f4_f5_c4_f(float x, float* f4, float* f5, float* c4) {
  if (x < 1.0f) {
    float s4 = kA4F[kSerF], s5 = kA5F[kSerF], sc = kAC4F[kSerF];
#pragma unroll
    for (int k = kSerF - 1; k >= 2; --k) {
      s4 = fmaf(s4, x, kA4F[k]);
      s5 = fmaf(s5, x, kA5F[k]);
      sc = fmaf(sc, x, kAC4F[k]);
    }
    s4 = fmaf(s4, x, kA4F[1]);
    sc = fmaf(fmaf(sc, x, kAC4F[1]), x, kAC4F[0]);
    *f4 = s4 * x;
    *f5 = s5 * x * x;
    *c4 = sc;
    return -1.0f;
  }
  const float e = __expf(-x);
  *c4 = (1.0f - e) / x;   // 1 - e has no cancellation for x >= 1
  *f4 = *c4 - e;
  *f5 = e * (1.0f + 0.5f * x) - *c4;
  return e;
}

__device__ __forceinline__ void half_coefs_f(float xf, float ef, float tauf, float xh, float e_eff, float dt, float f4,
                                             float f5, float c4, float* A, float* B) {
  if (e_eff < 0.0f) {
    *A = 0.0f;
    *B = 0.0f;
  } else if (e_eff > 0.0f) {
    const float dd = xh - xf;
    const float efh = fabsf(dd) < 0.5f ? e_eff * expm1f(dd) : (ef >= 0.0f ? ef : __expf(-xf)) - e_eff;
    *A = f4 + efh;
    *B = tauf * f5 - 0.5f * dt * efh;
  } else {
    *A = c4;
    *B = -tauf * f4;
  }
}

__device__ __forceinline__ float van_leer_f(float a, float b) {
  return a * b > 0.0f ? 2.0f * a * (b / (a + b)) : 0.0f;
}

__device__ __forceinline__ float rho_h_at_f(const Dev& d, const FaceRef& r, int k, int g) {
  return d2f_trunc(rho_h_at(d, r, k, g));
}

template <bool ENS>
__global__ void k_wave32(const __grid_constant__ Dev d0, const Ens e) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long total = ENS ? e.total_fg : (long long)d0.nface * d0.G;
  for (long long gi = tid; gi < total; gi += stride) {
    const int m = ENS ? find_member(e.fg0, e.M, gi) : 0;
    const Dev& d = ENS ? e.devs[m] : d0;
    const int i = (int)(ENS ? gi - e.fg0[m] : gi);
    const int G = d.G;
    const float v = d.vf, dt = d.dtf;
    const int f = i / G, g = i - f * G;
    const FaceRef r = face_ref(d, f);
    const int sideL = r.axis * 2, sideR = sideL + 1;
    const bool lin = r.k - 1 >= 0, rin = r.k < r.nk;
    if ((!lin && d.bc[sideL] == BC_REFLECT) || (!rin && d.bc[sideR] == BC_REFLECT)) {
      d.Fwave[i] = 0.0;
      continue;
    }
    const float rl = rho_h_at_f(d, r, r.k - 1, g), rr = rho_h_at_f(d, r, r.k, g);
    const float h = d2f_trunc(r.h);
    float sl, sr, fl, fr;
    if (d.wave_order >= 2) {
      const float rll = rho_h_at_f(d, r, r.k - 2, g), rrr = rho_h_at_f(d, r, r.k + 1, g);
      const float ih = __frcp_rn(h);
      sl = lin ? van_leer_f((rl - rll) * ih, (rr - rl) * ih) : 0.0f;
      sr = rin ? van_leer_f((rr - rl) * ih, (rrr - rr) * ih) : 0.0f;
      fl = rl + 0.5f * h * sl;
      fr = rr - 0.5f * h * sr;
    } else {
      sl = sr = (rr - rl) / h;
      fl = rl;
      fr = rr;
    }
    float sgl = -1.0f, sgr = -1.0f, el = 0.0f, er = 0.0f, xhl = 0.0f, xhr = 0.0f;
    if (lin) {
      const int cl = line_cell(d, r, r.k - 1);
      sgl = d2f_trunc(d.sigT[cl * G + g]);
      el = d2f_trunc(d.e_eff[cl * G + g]);
      xhl = d2f_trunc(d.xnum[cl * G + g]);
    } else if (d.bc[sideL] == BC_BLACKBODY) {
      sgl = d2f_trunc(d.ghost_sig[sideL * G + g]);
      el = d2f_trunc(d.e_eff[(d.ncell + sideL) * G + g]);
      xhl = d2f_trunc(d.xnum[(d.ncell + sideL) * G + g]);
    }
    if (rin) {
      const int cr = line_cell(d, r, r.k);
      sgr = d2f_trunc(d.sigT[cr * G + g]);
      er = d2f_trunc(d.e_eff[cr * G + g]);
      xhr = d2f_trunc(d.xnum[cr * G + g]);
    } else if (d.bc[sideR] == BC_BLACKBODY) {
      sgr = d2f_trunc(d.ghost_sig[sideR * G + g]);
      er = d2f_trunc(d.e_eff[(d.ncell + sideR) * G + g]);
      xhr = d2f_trunc(d.xnum[(d.ncell + sideR) * G + g]);
    }
    if (sgl < 0.0f) sgl = sgr;
    if (sgr < 0.0f) sgr = sgl;
    // harmonic-mean face opacity: x_f = dt rate 2 sl sr/(sl + sr), tau_f = dt/x_f
    const float xf = dt * d.ratef * 2.0f * sgl * (sgr / (sgl + sgr));
    const float tauf = dt / xf;
    float AL, BL, AR, BR, f4, f5, c4;
    const float ef = coef_f4_f5_c4_f(xf, &f4, &f5, &c4);
    half_coefs_f(xf, ef, tauf, xhl, el, dt, f4, f5, c4, &AL, &BL);
    half_coefs_f(xf, ef, tauf, xhr, er, dt, f4, f5, c4, &AR, &BR);
    const float F = AL * (v * 0.25f) * fl - AR * (v * 0.25f) * fr + (BL * sl + BR * sr) * (v * v * (1.0f / 6.0f));
    d.Fwave[i] = f2d_bits(F);
  }
}

// --------------------------------------------------------------------------
// Grid-wide barrier for the cooperative source-iteration kernel: a
// monotonically increasing arrival counter polled with acquire loads, bounded
// spin.  On timeout the
// status bit is set and the caller returns.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, Ctrl* status_ctrl, unsigned int limit_in,
                                             unsigned int target) {
  __shared__ int s_timeout;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    const unsigned int limit = limit_in ? limit_in : (1u << 25);
    target += status_ctrl->bar_extra;   // failure injection: arrivals that never come
    unsigned int spins = 0;
    int to = 0;
    while (true) {
      const unsigned int c = load_acquire_u32(count);
      if (c >= target) break;
      if (++spins > limit) { to = 1; break; }
      if (spins > 256) __nanosleep(64);   // back off only on a long wait
    }
    if (to) atomicOr(&status_ctrl->status, ST_TIMEOUT);
    __threadfence();
    s_timeout = to;
  }
  __syncthreads();
  return s_timeout == 0;
}

// Stopping rule of the source iteration after an iterate whose largest
// relative changes of T and rho are (eT, eR), the previous iterate's (pT,
// pR): the changes are within tol (reading of the unstated tolerances), or
// the iteration contracts fast (ratio r = e/p <= 1/10 in both) and the
// geometric tail of the changes still to come, e r/(1 - r), is within tol:
// the iterate is then within tol of the fixed point, as the plain rule
// allows, and the iterate that would only confirm it is saved (a slab
// contracts by about 1e-3 an iterate, the 2D checkerboard by about 3e-2).
// Slowly contracting iterations keep the plain rule.
__device__ __forceinline__ bool si_converged(double eT, double eR, double pT, double pR, double tol, bool prev) {
  if (eT <= tol && eR <= tol) return true;
  if (!prev || !(pT > 0.0) || !(pR > 0.0)) return false;
  const double rT = eT / pT, rR = eR / pR;
  if (!(rT <= 0.1) || !(rR <= 0.1)) return false;
  return eT * rT <= tol * (1.0 - rT) && eR * rR <= tol * (1.0 - rR);
}

// Neighbour values across one face of the cell at (ix, iy, iz): relaxation
// time and Phi at iterate k, or the ghost's.  Returns false for a reflecting
// wall (no flux).
__device__ __forceinline__ bool neighbour(const Dev& d, int ix, int iy, int iz, int axis, int dir, int g, int cur,
                                          double tau_c, double* tn, double* pn, int* nc) {
  const int jx = ix + (axis == 0 ? dir : 0), jy = iy + (axis == 1 ? dir : 0), jz = iz + (axis == 2 ? dir : 0);
  if (jx < 0 || jx >= d.nx || jy < 0 || jy >= d.ny || jz < 0 || jz >= d.nz) {
    const int side = axis * 2 + (dir > 0 ? 1 : 0);
    *nc = -1 - side;
    if (d.bc[side] == BC_REFLECT) return false;
    if (d.bc[side] == BC_BLACKBODY) {
      *tn = 1.0 / (d.rate_f * d.ghost_sig[side * d.G + g]);
      *pn = d.ghost_phi[side * d.G + g];
    } else {
      *tn = tau_c;
      *pn = 0.0;
    }
    return true;
  }
  const int n = (jz * d.ny + jy) * d.nx + jx;
  *nc = n;
  *tn = __ldcg(d.tauk[cur] + n * d.G + g);
  *pn = __ldcg(d.phik[cur] + n * d.G + g);
  return true;
}

// F^eq on face f at iterate k (lower side l, upper side u), or 0 at a
// reflecting wall; a black-body ghost takes tau = 1/(rate sigma_g(T_b)) and
// Phi_g(T_b), a vacuum ghost the inner cell's tau and Phi = 0.  The same
// expression, with the same operands, as a cell's own evaluation through
// neighbour(): the two agree bitwise.
__device__ __forceinline__ double face_feq(const Dev& d, int f, int g, int cur) {
  const FaceRef r = face_ref(d, f);
  const int sideL = r.axis * 2, sideR = sideL + 1;
  const bool lin = r.k - 1 >= 0, rin = r.k < r.nk;
  if ((!lin && d.bc[sideL] == BC_REFLECT) || (!rin && d.bc[sideR] == BC_REFLECT)) return 0.0;
  double tl = 0.0, tu = 0.0, pl = 0.0, pu = 0.0;
  if (lin) {
    const int i = line_cell(d, r, r.k - 1) * d.G + g;
    tl = __ldcg(d.tauk[cur] + i);
    pl = __ldcg(d.phik[cur] + i);
  }
  if (rin) {
    const int i = line_cell(d, r, r.k) * d.G + g;
    tu = __ldcg(d.tauk[cur] + i);
    pu = __ldcg(d.phik[cur] + i);
  }
  if (!lin) {
    if (d.bc[sideL] == BC_BLACKBODY) {
      tl = 1.0 / (d.rate_f * d.ghost_sig[sideL * d.G + g]);
      pl = d.ghost_phi[sideL * d.G + g];
    } else {
      tl = tu;
    }
  }
  if (!rin) {
    if (d.bc[sideR] == BC_BLACKBODY) {
      tu = 1.0 / (d.rate_f * d.ghost_sig[sideR * d.G + g]);
      pu = d.ghost_phi[sideR * d.G + g];
    } else {
      tu = tl;
    }
  }
  return feq_face_si(d, tl, tu, pl, pu, r.axis);
}

// Source iteration (App. B, Algorithm 2) in 1D, 2D and 3D, one warp per cell and
// one lane per group.  Iterate k: equilibrium fluxes from sigma^k, Phi^k of
// the cell and its neighbours (Jacobi), then the linearised closed-form update
//   T^{k+1} = [Cv T^n + sum_g (a_g/c)(Q_g - Phi_g + Phi'_g T^k)/(1 + a_g)]
//           / [Cv + sum_g (a_g/c) Phi'_g/(1 + a_g)],
//   rho^{k+1}_g = (Q_g + a_g (Phi_g + Phi'_g (T^{k+1} - T^k)))/(1 + a_g),
// a_g = c dt sigma_g/eps^2, Q_g = R_g + (dt/h)(F^eq_in - F^eq_out), and
// sigma^{k+1}, Phi^{k+1}, Phi'^{k+1} at T^{k+1} for the next iterate; one
// grid barrier per iterate.  Stopping rule: max over cells of |dT|/T and of
// max_g |d rho_g| / sum_g |rho_g| both <= si_tol.  The prologue assembles
// R = rho^n + wave-flux divergence + w^{fr,p}/V + source; the epilogue writes
// T^{n+1}, rho^{n+1}, rho^p = E_surv/V, rho^h = rho^{n+1} - rho^p and the
// energy ledger.
// Members of an ensemble converge separately: a member whose errors met the
// rule stops updating while the others go on (every block keeps the same
// per-member record, so all blocks leave the loop together).

// 1/T and sigma0 T^q of cell c: one rsqrt where the opacity law has T^{-1/2},
// else a reciprocal.  Every evaluation of the iterate state takes them from
// here, so a state computed at a temperature is bitwise the same whichever
// pass computed it.
__device__ __forceinline__ void inv_and_sigma_T(const Dev& d, int c, double T, double* invT, double* sT) {
  if (d.sig_q == -0.5) {
    const double rs = rsqrt(T);
    *invT = rs * rs;
    *sT = d.sigma0[c] * rs;
  } else {
    *invT = rcp_nr(T);
    *sT = sigma_T(d, c, T);
  }
}

// FP64 state of cell c at temperature T for the next iterate (slot): T^k,
// tau = 1/(rate sigma_g), q = 1/(tau + dt), Phi_g, dPhi_g/dT (FP32).
// PART 1: T^k, Phi_g, dPhi_g/dT; 2: tau, q (two warps of a cell share it).
// L: the cell's lanes; G: its group count, 0 for a segment past the last cell.
template <int NC, int PART = 0>
__device__ __forceinline__ void si_state(const Dev& d, int c, double T, double invT, double sT, int slot,
                                         const Lanes& L, int G) {
  double sg[NC], ph[NC];
  float dp[NC];
  si_planck<NC, PART>(d, T, invT, sT, sg, ph, dp, L, G);
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const int g = L.sl + L.seg * j;
    if (g < G) {
      if (PART != 1) {
        double tau, qv;
        tau_and_q(d, sg[j], &tau, &qv);
        __stcg(d.tauk[slot] + c * G + g, tau);
        __stcg(d.qk + c * G + g, qv);
      }
      if (PART != 2) {
        __stcg(d.phik[slot] + c * G + g, ph[j]);
        __stcg(d.dphik + c * G + g, dp[j]);
      }
    }
  }
  if (L.sl == 0 && G > 0 && PART != 2) __stcg(d.Tk[slot] + c, T);
}

// ---- FP32 warm start (mixed precision)
constexpr double kWarmTol = 3e-6;   // largest |dT|/T at which the FP32 iterates hand over
constexpr int kWarmMaxIters = 100;

// the same state in FP32
template <int NC>
__device__ __forceinline__ void si_state_f(const Dev& d, int c, float T, int slot, const Lanes& L, int G) {
  const float invT = __frcp_rn(T);
  const float sT = d2f_trunc(d.sigma0[c]) * pow_fast_f(T, d2f_trunc(d.sig_q));
  float sg[NC], ph[NC], dp[NC];
  si_planck_f<NC>(d, T, invT, sT, sg, ph, dp, L, G);
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const int g = L.sl + L.seg * j;
    if (g < G) {
      float tau, qv;
      tau_and_q_f(d, sg[j], &tau, &qv);
      __stcg(d.tau_f[slot] + c * G + g, tau);
      __stcg(d.q_f + c * G + g, qv);
      __stcg(d.phi_f[slot] + c * G + g, ph[j]);
      __stcg(d.dphik + c * G + g, dp[j]);
    }
  }
  if (L.sl == 0 && G > 0) __stcg(d.Tk_f[slot] + c, T);
}

// neighbour values across one face in FP32 (as neighbour()); false at a reflecting wall
__device__ __forceinline__ bool neighbour_f(const Dev& d, int ix, int iy, int iz, int axis, int dir, int g, int cur,
                                            float tau_c, float* tn, float* pn) {
  const int jx = ix + (axis == 0 ? dir : 0), jy = iy + (axis == 1 ? dir : 0), jz = iz + (axis == 2 ? dir : 0);
  if (jx < 0 || jx >= d.nx || jy < 0 || jy >= d.ny || jz < 0 || jz >= d.nz) {
    const int side = axis * 2 + (dir > 0 ? 1 : 0);
    if (d.bc[side] == BC_REFLECT) return false;
    if (d.bc[side] == BC_BLACKBODY) {
      *tn = __frcp_rn(d.ratef * d2f_trunc(d.ghost_sig[side * d.G + g]));
      *pn = d2f_trunc(d.ghost_phi[side * d.G + g]);
    } else {
      *tn = tau_c;
      *pn = 0.0f;
    }
    return true;
  }
  const int n = (jz * d.ny + jy) * d.nx + jx;
  *tn = __ldcg(d.tau_f[cur] + n * d.G + g);
  *pn = __ldcg(d.phi_f[cur] + n * d.G + g);
  return true;
}

// F^eq on face f in FP32 (as face_feq)
__device__ __forceinline__ float face_feq_f(const Dev& d, int f, int g, int cur) {
  const FaceRef r = face_ref(d, f);
  const int sideL = r.axis * 2, sideR = sideL + 1;
  const bool lin = r.k - 1 >= 0, rin = r.k < r.nk;
  if ((!lin && d.bc[sideL] == BC_REFLECT) || (!rin && d.bc[sideR] == BC_REFLECT)) return 0.0f;
  float tl = 0.0f, tu = 0.0f, pl = 0.0f, pu = 0.0f;
  if (lin) {
    const int i = line_cell(d, r, r.k - 1) * d.G + g;
    tl = __ldcg(d.tau_f[cur] + i);
    pl = __ldcg(d.phi_f[cur] + i);
  }
  if (rin) {
    const int i = line_cell(d, r, r.k) * d.G + g;
    tu = __ldcg(d.tau_f[cur] + i);
    pu = __ldcg(d.phi_f[cur] + i);
  }
  if (!lin) {
    if (d.bc[sideL] == BC_BLACKBODY) {
      tl = __frcp_rn(d.ratef * d2f_trunc(d.ghost_sig[sideL * d.G + g]));
      pl = d2f_trunc(d.ghost_phi[sideL * d.G + g]);
    } else {
      tl = tu;
    }
  }
  if (!rin) {
    if (d.bc[sideR] == BC_BLACKBODY) {
      tu = __frcp_rn(d.ratef * d2f_trunc(d.ghost_sig[sideR * d.G + g]));
      pu = d2f_trunc(d.ghost_phi[sideR * d.G + g]);
    } else {
      tu = tl;
    }
  }
  return feq_face_f(d, tl, tu, pl, pu, r.axis);
}

// One FP32 iterate of cell c (the linearised update of the FP64 iterate, no
// rho written): T^{k+1} and the cell's state at it into slot cur ^ 1.
// Returns |dT|/T (+inf where not finite; 0 for a segment past the last
// cell, G = 0).
template <int NC>
__device__ __forceinline__ float si_iterate_f(const Dev& d, int c, int cur, bool face_pass, const Lanes& L, int G) {
  const int nxt = cur ^ 1;
  const float dt = d.dtf;
  const float Tc = __ldcg(d.Tk_f[cur] + c);
  float num = 0.0f, den = 0.0f;
  int ix, iy, iz;
  cell_xyz(d, c, &ix, &iy, &iz);
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const int g = L.sl + L.seg * j;
    if (g >= G) continue;
    const int i = c * G + g;
    const float tc = __ldcg(d.tau_f[cur] + i), phc = __ldcg(d.phi_f[cur] + i), dpc = __ldcg(d.dphik + i);
    float q = d.R_f[i];
    for (int axis = 0; axis < d.dim; ++axis) {
      float Fin = 0.0f, Fout = 0.0f;
      if (face_pass) {
        Fin = __ldcg(d.Feq_f + face_index_xyz(d, ix, iy, iz, axis, -1) * G + g);
        Fout = __ldcg(d.Feq_f + face_index_xyz(d, ix, iy, iz, axis, +1) * G + g);
      } else {
        float tn, pn;
        if (neighbour_f(d, ix, iy, iz, axis, -1, g, cur, tc, &tn, &pn)) Fin = feq_face_f(d, tn, tc, pn, phc, axis);
        if (neighbour_f(d, ix, iy, iz, axis, +1, g, cur, tc, &tn, &pn)) Fout = feq_face_f(d, tc, tn, phc, pn, axis);
      }
      q = fmaf(d2f_trunc(d.dt_h[axis]), Fin - Fout, q);
    }
    const float qi = __ldcg(d.q_f + i);
    const float ap = dt * qi * d.inv_cf;
    num = fmaf(ap, fmaf(dpc, Tc, q - phc), num);
    den = fmaf(ap, dpc, den);
  }
  num = seg_sum_f(num, L);
  den = seg_sum_f(den, L);
  float Tnew;
  if (d.cv_law == 1) {
    const double Tcd = f2d_bits(Tc), Tnd = d.T[c];
    const double ck = heat_capacity(d, c, Tcd);
    Tnew = d2f_trunc((mat_energy(d, c, Tnd) - mat_energy(d, c, Tcd) + ck * Tcd + f2d_bits(num)) /
                     (ck + f2d_bits(den)));
  } else {
    const float cv = d2f_trunc(d.cv[c]);
    Tnew = __fdiv_rn(fmaf(cv, d2f_trunc(d.T[c]), num), cv + den);
  }
  if (!(Tnew > 1e-30f)) Tnew = (Tnew == Tnew) ? 1e-30f : Tnew;
  float eT = __fdiv_rn(fabsf(Tnew - Tc), Tnew);
  if (!(eT <= 3.0e38f)) eT = INFINITY;
  // a T^{k+1} that is not finite is stored as it is, without a state (the
  // hand-over falls back to T^n there); every segment takes the call, whose
  // shuffles need the whole warp
  const bool fin = Tnew == Tnew && Tnew < INFINITY;
  si_state_f<NC>(d, c, fin ? Tnew : 1.0f, nxt, L, fin ? G : 0);
  if (!fin && L.sl == 0 && G > 0) __stcg(d.Tk_f[nxt] + c, Tnew);
  return G > 0 ? eT : 0.0f;
}

// PAIR (single 1D problems of at most two cells per SM, FP64 iterates
// only): two warps per cell, one block each, so that a cell's chain of
// dependent FP64 instructions is split over two SM sub-partitions.  In an
// iterate each warp evaluates one of the cell's two faces and they exchange
// the fluxes through shared memory; both form Q, the sums and T^{k+1} (the
// same operations, so the same bits); then warp 0 evaluates the Planck
// values while warp 1 updates rho and evaluates the opacities, tau and q.
// The prologue and epilogue are split the same way (warp 0: R, T and the
// rho^p/rho^h split; warp 1: the ledger sums and the kept state).  The
// results are bitwise those of one warp per cell.
// The cell a lane serves in work item q: an item is one warp's 32/seg
// cells of one member (seg from the member's G, 32 in pair mode); a segment
// past the member's last cell gets its last cell and G = 0 (no group work,
// nothing stored).
struct SiCell {
  int m, c, G;
  Lanes L;
};

template <bool ENS, bool PAIR>
__device__ __forceinline__ SiCell si_cell(const Dev& d0, const Ens& e, long long q) {
  SiCell r;
  r.m = ENS ? find_member(e.item0, e.M, q) : 0;
  const Dev& d = ENS ? e.devs[r.m] : d0;
  r.L = lanes_of(PAIR ? 32 : seg_width(d.G));
  const long long t = ENS ? q - (long long)e.item0[r.m] : q;
  const long long c = t * (32 / r.L.seg) + r.L.sub;
  r.c = c < d.ncell ? (int)c : d.ncell - 1;
  r.G = c < d.ncell ? d.G : 0;
  return r;
}

template <int NC, bool ENS, bool PAIR>
__global__ void __launch_bounds__(256) k_si(const __grid_constant__ Dev d0, const Ens e) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  const long long gw = PAIR ? (long long)blockIdx.x : blockIdx.x * (long long)nwb + wib;
  const long long nw = PAIR ? (long long)gridDim.x : (long long)gridDim.x * nwb;
  // work items: one warp's cells (several per warp where G <= 16)
  const int cpw0 = PAIR ? 1 : 32 / seg_width(d0.G);
  const long long nitems = ENS ? e.total_items : ((long long)d0.ncell + cpw0 - 1) / cpw0;
  const int M = ENS ? e.M : 1;
  unsigned int* bar_count = ENS ? e.bar : &d0.ctrl->bar_count;
  Ctrl* st_ctrl = ENS ? e.devs[0].ctrl : d0.ctrl;
  const unsigned int spin_limit = st_ctrl->bar_timeout_spins;
  const bool warm = ENS ? e.devs[0].si_warm : d0.si_warm;
  __shared__ float s_err[8][2];
  __shared__ int s_conv[ENS ? kMaxEnsemble : 1];   // iterate count at convergence, 0 = still running
  __shared__ int s_any;
  __shared__ double s_pair[PAIR ? 2 : 1][PAIR ? 32 * NC : 1];   // PAIR: the two faces' fluxes
  unsigned int bar = 0;

  // The first iterate's inputs into L2 while the prologue runs: the Planck
  // and C2 interpolant tables (a share per block) and, where the previous
  // step left the iterate state, each cell's own rows of it (the neighbours'
  // rows are their own cells')
  {
    constexpr int kLp = (int)((sizeof(kPlanckTab) + 127) / 128), kLc = (int)((sizeof(kC2Tab) + 127) / 128);
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < kLp + kLc;
         l += (long long)gridDim.x * blockDim.x)
      prefetch_l2(l < kLp ? (const void*)((const char*)kPlanckTab + 128 * l)
                          : (const void*)((const char*)kC2Tab + 128 * (l - kLp)));
    if (!ENS && !warm && d0.ctrl->si_state_ok) {
      for (long long gq = gw; gq < nitems; gq += nw) {
        const SiCell sc = si_cell<ENS, PAIR>(d0, e, gq);
        const long long i = (long long)sc.c * sc.G + sc.L.sl;
        if (sc.L.sl < sc.G && (sc.L.sl & 15) == 0) {   // one lane per 128-byte line
          prefetch_l2(d0.tauk[0] + i);
          prefetch_l2(d0.phik[0] + i);
          prefetch_l2(d0.qk + i);
          prefetch_l2(d0.dphik + i);
        }
      }
    }
  }

  // ---- prologue.  A pair splits it: warp 0 forms R (and the state on a
  // first step), warp 1 the energy sums of the ledger.
  const bool roleA = !PAIR || wib == 0, roleB = !PAIR || wib == 1;
  {
    double e_rad0 = 0.0, e_mat0 = 0.0, e_src = 0.0;
    int acc_m = -1;
    for (long long gq = gw; gq < nitems; gq += nw) {
      const SiCell sc = si_cell<ENS, PAIR>(d0, e, gq);
      const int m = sc.m;
      if (ENS && m != acc_m && acc_m >= 0) {
        warp_sum2(e_rad0, e_src);
        e_mat0 = warp_sum(e_mat0);   // a warp carries several cells where G <= 16
        if (lane == 0) {
          Ctrl* cc = e.devs[acc_m].ctrl;
          atomicAdd(&cc->E_rad0, e_rad0);
          atomicAdd(&cc->E_mat0, e_mat0);
          if (e_src != 0.0) atomicAdd(&cc->src_in, e_src);
        }
        e_rad0 = e_mat0 = e_src = 0.0;
      }
      acc_m = m;
      const Dev& d = ENS ? e.devs[m] : d0;
      const int c = sc.c, G = sc.G;
      const Lanes& L = sc.L;
      const double dt = d.dt, V = d.vol;
      // the source acts while t^n = n dt < src_t_end (src_t_end <= 0: always)
      const bool src_on = d.src && (!(d.src_t_end > 0.0) || (double)d.ctrl->step * dt < d.src_t_end);
      int ix, iy, iz;
      cell_xyz(d, c, &ix, &iy, &iz);
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const int g = L.sl + L.seg * j;
        if (g < G) {
          const int i = c * G + g;
          const double r0 = d.rho[i];
          if (roleA) {
            double r = r0;
            for (int axis = 0; axis < d.dim; ++axis) {
              const int fl = face_index_xyz(d, ix, iy, iz, axis, -1), fr = face_index_xyz(d, ix, iy, iz, axis, +1);
              r += (dt * inv_h_of(d, axis)) * (d.Fwave[fl * G + g] - d.Fwave[fr * G + g]);
            }
            const double Wd = from_fixed(d.Wq + 2 * i, d.tq);
            d.W[i] = Wd;
            r += Wd * d.inv_vol;
            if (src_on) r += d.src[i];
            d.R[i] = r;
            if (warm) d.R_f[i] = d2f_trunc(r);
          }
          if (roleB) {
            if (src_on) e_src += V * d.src[i] * d.inv_c;
            e_rad0 += V * r0 * d.inv_c;
          }
        }
      }
      const double T = d.T[c];
      if (roleB && L.sl == 0 && G > 0) e_mat0 += V * mat_energy(d, c, T);
      if (roleA) {
        if (warm) si_state_f<NC>(d, c, d2f_trunc(T), 0, L, G);
        else if (!d.ctrl->si_state_ok) {
          double invT, sT;
          inv_and_sigma_T(d, c, T, &invT, &sT);
          si_state<NC>(d, c, T, invT, sT, 0, L, G);
        }
      }
    }
    if (roleB) {   // (warp-uniform)
      warp_sum2(e_rad0, e_src);
      e_mat0 = warp_sum(e_mat0);   // a warp carries several cells where G <= 16
    }
    if (roleB && lane == 0 && acc_m >= 0) {
      Ctrl* cc = ENS ? e.devs[acc_m].ctrl : d0.ctrl;
      atomicAdd(&cc->E_rad0, e_rad0);
      atomicAdd(&cc->E_mat0, e_mat0);
      if (e_src != 0.0) atomicAdd(&cc->src_in, e_src);
    }
  }
  for (int k = threadIdx.x; k < (ENS ? M : 1); k += blockDim.x) s_conv[k] = 0;
  // The first iterate reads the neighbours' state at T^n.  Where the
  // previous step left it, the prologue wrote nothing another cell reads (R
  // is the cell's own), so no grid barrier is needed before the iterates.
  if (ENS || warm || !d0.ctrl->si_state_ok) {
    if (!grid_barrier(bar_count, st_ctrl, spin_limit, (++bar) * gridDim.x)) return;
  } else {
    __syncthreads();
  }

  // ---- iterations.  `it` counts all iterates (it indexes the error slots),
  // itA the FP32 warm-start iterates, itB the FP64 ones.
  const int max_it = ENS ? e.devs[0].si_max_iters : d0.si_max_iters;
  int it = 0, itA = 0, itB = 0, all_done = 0;
  // 2D and 3D: every face's F^eq once per iterate (one warp per face, one lane per
  // group), then a grid barrier, instead of each cell evaluating its 2 dim
  // faces (a face costs a division and the C2 interpolant in FP64, the
  // scarce unit on this chip; in 1D the extra barrier costs more than the
  // second evaluation of a face saves)
  const bool face_pass = !ENS && d0.dim >= 2;
  if (warm && !PAIR) {
    // FP32 iterates from T^n while the largest |dT|/T falls: until it is
    // within kWarmTol, stalls near FP32 resolution, or kWarmMaxIters pass
    Ctrl* const ctrlA = ENS ? e.devs[0].ctrl : d0.ctrl;
    const int maxA = max_it < kWarmMaxIters ? max_it : kWarmMaxIters;
    for (; itA < maxA; ++itA, ++it) {
      const int cur = itA & 1;
      if (face_pass) {
        const int G = d0.G;
        const Lanes L = lanes_of(seg_width(G));
        const long long nfi = ((long long)d0.nface + cpw0 - 1) / cpw0;
        for (long long gq = gw; gq < nfi; gq += nw) {
          const long long f = gq * cpw0 + L.sub;
          if (f >= d0.nface) continue;
#pragma unroll
          for (int j = 0; j < NC; ++j) {
            const int g = L.sl + L.seg * j;
            if (g < G) d0.Feq_f[f * G + g] = face_feq_f(d0, (int)f, g, cur);
          }
        }
        if (!grid_barrier(bar_count, st_ctrl, spin_limit, (++bar) * gridDim.x)) return;
      }
      float werr = 0.0f;
      for (long long gq = gw; gq < nitems; gq += nw) {
        const SiCell sc = si_cell<ENS, PAIR>(d0, e, gq);
        const Dev& d = ENS ? e.devs[sc.m] : d0;
        werr = fmaxf(werr, si_iterate_f<NC>(d, sc.c, cur, face_pass, sc.L, sc.G));
      }
      werr = warp_max_nonneg_f(werr);
      if (lane == 0) s_err[wib][0] = werr;
      __syncthreads();
      if (threadIdx.x == 0) {
        float mx = 0.0f;
        for (int w = 0; w < nwb; ++w) mx = fmaxf(mx, s_err[w][0]);
        atomic_max_nonneg(&ctrlA->err_slot[it % 3][0], f2d_bits(mx));
      }
      if (blockIdx.x == 0)
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
          Ctrl* cc = ENS ? e.devs[k].ctrl : d0.ctrl;
          cc->err_slot[(it + 1) % 3][0] = 0ull;
          cc->err_slot[(it + 1) % 3][1] = 0ull;
        }
      if (!grid_barrier(bar_count, st_ctrl, spin_limit, (++bar) * gridDim.x)) return;
      const ErrPair ep = load_err_slots(ctrlA->err_slot, it);
      const double eA = ep.eT, pA = ep.pT;
      const bool stalled = itA > 0 && eA <= 1e-4 && eA > 0.5 * pA;
      if (!(eA <= 1e30) || eA <= kWarmTol || stalled || itA + 1 >= maxA) { ++itA; ++it; break; }
    }
    // hand-over: the FP64 state at the last FP32 temperature (at T^n in a
    // cell where that is not finite and positive)
    for (long long gq = gw; gq < nitems; gq += nw) {
      const SiCell sc = si_cell<ENS, PAIR>(d0, e, gq);
      const Dev& d = ENS ? e.devs[sc.m] : d0;
      const int c = sc.c;
      const float Tf = __ldcg(d.Tk_f[itA & 1] + c);
      const double T0 = (Tf > 0.0f && Tf < INFINITY) ? f2d_bits(Tf) : d.T[c];
      double invT, sT;
      inv_and_sigma_T(d, c, T0, &invT, &sT);
      si_state<NC>(d, c, T0, invT, sT, 0, sc.L, sc.G);
    }
    if (!grid_barrier(bar_count, st_ctrl, spin_limit, (++bar) * gridDim.x)) return;
  }
  for (; itB < max_it; ++itB, ++it) {
    const int cur = itB & 1, nxt = cur ^ 1;
    float werrT = 0.0f, werrR = 0.0f;
    if (face_pass) {
      const int G = d0.G;
      const Lanes L = lanes_of(seg_width(G));
      const long long nfi = ((long long)d0.nface + cpw0 - 1) / cpw0;
      for (long long gq = gw; gq < nfi; gq += nw) {
        const long long f = gq * cpw0 + L.sub;
        if (f >= d0.nface) continue;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          const int g = L.sl + L.seg * j;
          if (g < G) d0.Feq[f * G + g] = face_feq(d0, (int)f, g, cur);
        }
      }
      if (!grid_barrier(bar_count, st_ctrl, spin_limit, (++bar) * gridDim.x)) return;
    }
    for (long long gq = gw; gq < nitems; gq += nw) {
      const SiCell sc = si_cell<ENS, PAIR>(d0, e, gq);
      const int m = sc.m;
      if (ENS && s_conv[m]) continue;
      const Dev& d = ENS ? e.devs[m] : d0;
      const int c = sc.c, G = sc.G;
      const Lanes& L = sc.L;
      const double dt = d.dt;
      const double Tc = __ldcg(d.Tk[cur] + c), Tn = d.T[c], cv = d.cv[c];
      // with q = 1/(tau + dt): 1/(1 + a_g) = tau q and a_g/(1 + a_g) = dt q
      double Q[NC], ar[NC], r1[NC], phc[NC], dpc[NC];
      double num = 0.0, den = 0.0;
      int ix, iy, iz;
      cell_xyz(d, c, &ix, &iy, &iz);
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const int g = L.sl + L.seg * j;
        Q[j] = 0.0; ar[j] = 0.0; r1[j] = 1.0; phc[j] = 0.0; dpc[j] = 0.0;
        if (g >= G) continue;
        const int i = c * G + g;
        const double tc = __ldcg(d.tauk[cur] + i);
        phc[j] = __ldcg(d.phik[cur] + i);
        dpc[j] = f2d_bits(__ldcg(d.dphik + i));
        double q = d.R[i];
        if (face_pass) {
          for (int axis = 0; axis < d.dim; ++axis) {
            const double Fin = __ldcg(d.Feq + face_index_xyz(d, ix, iy, iz, axis, -1) * G + g);
            const double Fout = __ldcg(d.Feq + face_index_xyz(d, ix, iy, iz, axis, +1) * G + g);
            q = fma(d.dt_h[axis], Fin - Fout, q);
          }
        }
        if (PAIR) {
          // this warp's face: warp 0 the lower, warp 1 the upper
          const int dir = wib ? 1 : -1;
          double tn, pn;
          int nc;
          double F = 0.0;
          if (neighbour(d, ix, iy, iz, 0, dir, g, cur, tc, &tn, &pn, &nc))
            F = dir < 0 ? feq_face_si(d, tn, tc, pn, phc[j], 0) : feq_face_si(d, tc, tn, phc[j], pn, 0);
          if (dir > 0 || nc < 0) d.Feq[face_index_xyz(d, ix, iy, iz, 0, dir) * G + g] = F;
          s_pair[PAIR ? wib : 0][PAIR ? g : 0] = F;
        }
        for (int axis = 0; axis < ((face_pass || PAIR) ? 0 : d.dim); ++axis) {
          double Fin = 0.0, Fout = 0.0;
          for (int dir = -1; dir <= 1; dir += 2) {
            double tn, pn;
            int nc;
            double F = 0.0;
            if (neighbour(d, ix, iy, iz, axis, dir, g, cur, tc, &tn, &pn, &nc)) {
              F = dir < 0 ? feq_face_si(d, tn, tc, pn, phc[j], axis) : feq_face_si(d, tc, tn, phc[j], pn, axis);
            }
            const bool owner = dir > 0 ? true : (nc < 0);   // upper face, or a boundary face
            if (owner) d.Feq[face_index_xyz(d, ix, iy, iz, axis, dir) * G + g] = F;
            if (dir < 0) Fin = F; else Fout = F;
          }
          q = fma(d.dt_h[axis], Fin - Fout, q);
        }
        Q[j] = q;
        const double qi = __ldcg(d.qk + i);   // 1/(tau + dt), stored with tau
        r1[j] = tc * qi;
        ar[j] = dt * qi;
        if (!PAIR) {
          const double ap = ar[j] * d.inv_c;
          num = fma(ap, fma(dpc[j], Tc, q - phc[j]), num);
          den = fma(ap, dpc[j], den);
        }
      }
      if (PAIR) {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          const int k = PAIR ? L.sl + L.seg * j : 0;
          if (k >= G) continue;
          Q[j] = fma(d.dt_h[0], s_pair[0][k] - s_pair[PAIR ? 1 : 0][k], Q[j]);
          const double ap = ar[j] * d.inv_c;
          num = fma(ap, fma(dpc[j], Tc, Q[j] - phc[j]), num);
          den = fma(ap, dpc[j], den);
        }
        __syncthreads();   // both warps have read the exchange before a next cell writes it
      }
      seg_sum2(num, den, L);
      // a T-dependent heat capacity: e(T^{k+1}) ~ e(T^k) + C_v(T^k) (T^{k+1} - T^k)
      double Tnew;
      if (d.cv_law == 1) {
        const double ck = heat_capacity(d, c, Tc);
        Tnew = (mat_energy(d, c, Tn) - mat_energy(d, c, Tc) + ck * Tc + num) / (ck + den);
      } else {
        Tnew = fma(cv, Tn, num) * rcp_nr(cv + den);
      }
      {
        // T >= 1e-30 (NaN kept), compared as bit patterns
        const long long tb = __double_as_longlong(Tnew);
        const bool nan = (tb & 0x7fffffffffffffffll) > 0x7ff0000000000000ll;
        if (!nan && tb < kBits1em30) Tnew = 1e-30;
      }
      const double dT = Tnew - Tc;
      double invTn, sTn;
      inv_and_sigma_T(d, c, Tnew, &invTn, &sTn);
      if (PAIR && !wib) {
        // warp 0 of the pair: Phi, dPhi/dT and T at T^{k+1}
        si_state<NC, 1>(d, c, Tnew, invTn, sTn, nxt, L, G);
        continue;
      }
      double r[NC], dr[NC];
      int ex = 0;
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const int g = L.sl + L.seg * j;
        r[j] = 0.0; dr[j] = 0.0;
        if (g >= G) continue;
        const int i = c * G + g;
        r[j] = fma(Q[j], r1[j], ar[j] * fma(dpc[j], dT, phc[j]));
        dr[j] = r[j] - __ldcg(d.rho + i);
        __stcg(d.rho + i, r[j]);
        ex = max(ex, biased_exp(r[j]));
      }
      // max_g |d rho_g| / sum_g |rho_g| in FP32, both scaled by the cell's largest |rho_g|
      const int E = (int)seg_max_u((unsigned)ex, L);
      float dmax = 0.0f, rsum = 0.0f;
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        dmax = fmaxf(dmax, scaled_mag(dr[j], E));
        rsum += scaled_mag(r[j], E);
      }
      dmax = __uint_as_float(seg_max_u(__float_as_uint(dmax), L));
      rsum = seg_sum_f(rsum, L);
      float eR = rsum > 0.0f ? dmax / rsum : 0.0f;
      const int ET = biased_exp(Tnew);
      const float fT = scaled_mag(Tnew, ET);
      float eT = fT < INFINITY ? scaled_mag(dT, ET) / fT : INFINITY;
      if (!(eT <= 3.0e38f)) eT = INFINITY;
      if (!(eR <= 3.0e38f)) eR = INFINITY;
      if (G == 0) eT = eR = 0.0f;   // a segment past the last cell
      if (ENS) {
        // members differ between warps (a warp's cells are one member's):
        // each warp reports to its own member
        const float wT = warp_max_nonneg_f(eT), wR = warp_max_nonneg_f(eR);
        if (lane == 0) {
          atomic_max_nonneg(&d.ctrl->err_slot[it % 3][0], f2d_bits(wT));
          atomic_max_nonneg(&d.ctrl->err_slot[it % 3][1], f2d_bits(wR));
        }
      } else {
        werrT = fmaxf(werrT, eT);
        werrR = fmaxf(werrR, eR);
      }
      // warp 1 of a pair: the opacities, tau and q
      if (PAIR) si_state<NC, 2>(d, c, Tnew, invTn, sTn, nxt, L, G);
      else si_state<NC>(d, c, Tnew, invTn, sTn, nxt, L, G);
    }
    if (!ENS) {
      Ctrl* ctrl = d0.ctrl;
      werrT = warp_max_nonneg_f(werrT);
      werrR = warp_max_nonneg_f(werrR);
      if (lane == 0) { s_err[wib][0] = werrT; s_err[wib][1] = werrR; }
      __syncthreads();
      if (threadIdx.x == 0) {
        float mT = 0.0f, mR = 0.0f;
        for (int w = 0; w < nwb; ++w) { mT = fmaxf(mT, s_err[w][0]); mR = fmaxf(mR, s_err[w][1]); }
        atomic_max_nonneg(&ctrl->err_slot[it % 3][0], f2d_bits(mT));
        atomic_max_nonneg(&ctrl->err_slot[it % 3][1], f2d_bits(mR));
        if (blockIdx.x == 0) {
          ctrl->err_slot[(it + 1) % 3][0] = 0ull;
          ctrl->err_slot[(it + 1) % 3][1] = 0ull;
        }
      }
    } else if (blockIdx.x == 0) {
      for (int k = threadIdx.x; k < M; k += blockDim.x) {
        Ctrl* cc = e.devs[k].ctrl;
        cc->err_slot[(it + 1) % 3][0] = 0ull;
        cc->err_slot[(it + 1) % 3][1] = 0ull;
      }
    }
    if (!grid_barrier(bar_count, st_ctrl, spin_limit, (++bar) * gridDim.x)) return;
    if (!ENS) {
      Ctrl* ctrl = d0.ctrl;
      const ErrPair ep = load_err_slots(ctrl->err_slot, it);
      if (si_converged(ep.eT, ep.eR, ep.pT, ep.pR, d0.si_tol, itB > 0)) { s_conv[0] = itB + 1; all_done = 1; ++itB; ++it; break; }
    } else {
      if (threadIdx.x == 0) s_any = 0;
      __syncthreads();
      int running = 0;
      for (int k = threadIdx.x; k < M; k += blockDim.x) {
        if (s_conv[k]) continue;
        Ctrl* cc = e.devs[k].ctrl;
        const ErrPair ep = load_err_slots(cc->err_slot, it);
        if (si_converged(ep.eT, ep.eR, ep.pT, ep.pR, e.devs[k].si_tol, itB > 0)) s_conv[k] = itB + 1; else running = 1;
      }
      if (running) s_any = 1;
      __syncthreads();
      if (!s_any) { all_done = 1; ++itB; ++it; break; }
    }
  }

  // ---- epilogue: member m's last iterate wrote Tk[s_conv[m] & 1] (or
  // Tk[itB & 1]).  A pair splits it: warp 0 stores T and splits rho into
  // rho^p and rho^h, warp 1 keeps the last iterate's state and sums the
  // ledger.
  {
    double e_rad1 = 0.0, e_mat1 = 0.0, b_in = 0.0;
    int bad = 0, scaled = 0, acc_m = -1;
    for (long long gq = gw; gq < nitems; gq += nw) {
      const SiCell sc = si_cell<ENS, PAIR>(d0, e, gq);
      const int m = sc.m;
      if (ENS && m != acc_m && acc_m >= 0) {
        warp_sum2(e_rad1, b_in);
        e_mat1 = warp_sum(e_mat1);
        const unsigned sc_n = __reduce_add_sync(0xffffffffu, (unsigned)scaled);
        bad = __any_sync(0xffffffffu, bad) ? 1 : 0;
        if (lane == 0) {
          Ctrl* cc = e.devs[acc_m].ctrl;
          atomicAdd(&cc->E_rad1, e_rad1);
          atomicAdd(&cc->E_mat1, e_mat1);
          if (b_in != 0.0) atomicAdd(&cc->bnd_in_macro, b_in);
          if (bad) atomicOr(&cc->status, ST_NONFINITE);
          if (sc_n) { atomicOr(&cc->scaled, 1u); atomicAdd(&cc->n_scaled_bins, sc_n); }
        }
        e_rad1 = e_mat1 = b_in = 0.0;
        bad = 0;
        scaled = 0;
      }
      acc_m = m;
      const Dev& d = ENS ? e.devs[m] : d0;
      const int c = sc.c, G = sc.G;
      const Lanes& L = sc.L;
      const double dt = d.dt, V = d.vol;
      const int ran = s_conv[ENS ? m : 0] ? s_conv[ENS ? m : 0] : itB;
      const int fin = ran > 0 ? (ran & 1) : 0;
      const double T = __ldcg(d.Tk[fin] + c);
      // the last iterate's state (at T^{n+1}) into slot 0, where the next
      // step's iteration starts from it instead of re-evaluating it
      if (roleB && fin == 1 && !warm) {
        if (L.sl == 0 && G > 0) __stcg(d.Tk[0] + c, T);
        for (int g = L.sl; g < G; g += L.seg) {
          __stcg(d.tauk[0] + c * G + g, __ldcg(d.tauk[1] + c * G + g));
          __stcg(d.phik[0] + c * G + g, __ldcg(d.phik[1] + c * G + g));
        }
      }
      if (roleA) {
        if (G > 0 && (!(T == T) || T > 1e300)) bad = 1;
        if (L.sl == 0 && G > 0) d.T[c] = T;
      }
      if (roleB && L.sl == 0 && G > 0) e_mat1 += V * mat_energy(d, c, T);
      int ixyz[3];
      cell_xyz(d, c, &ixyz[0], &ixyz[1], &ixyz[2]);
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const int g = L.sl + L.seg * j;
        if (g >= G) continue;
        const int i = c * G + g;
        const double r = __ldcg(d.rho + i);
        if (roleA) {
          // survivors never hold more than rho^{n+1} leaves in their (cell,
          // group): their weights are scaled to it (rho and the energy unchanged)
          const double Es = from_fixed(d.Esq + 2 * i, d.tq);
          d.E_surv[i] = Es;
          double rp = Es * d.inv_vol, f = 1.0;
          if (!d.split_literal && rp > 0.0 && r < rp) {
            f = r > 0.0 ? r / rp : 0.0;
            rp = r > 0.0 ? r : 0.0;
            scaled += 1;
          }
          d.wscale[i] = f;
          d.rho_p[i] = rp;
          d.rho_h[i] = r - rp;
        }
        if (roleB) {
          e_rad1 += V * r * d.inv_c;
          // boundary faces: energy entering the domain
          for (int axis = 0; axis < d.dim; ++axis) {
            const double S = d.area[axis];
            const int k = ixyz[axis], nk = axis == 0 ? d.nx : (axis == 1 ? d.ny : d.nz);
            if (k == 0) {
              const int f = face_index(d, c, axis, -1);
              b_in += dt * S * (d.Feq[f * G + g] + d.Fwave[f * G + g]) * d.inv_c;
            }
            if (k == nk - 1) {
              const int f = face_index(d, c, axis, +1);
              b_in -= dt * S * (d.Feq[f * G + g] + d.Fwave[f * G + g]) * d.inv_c;
            }
          }
        }
      }
    }
    if (roleB) {   // (warp-uniform)
      warp_sum2(e_rad1, b_in);
      e_mat1 = warp_sum(e_mat1);
      if (lane == 0 && acc_m >= 0) {
        Ctrl* cc = ENS ? e.devs[acc_m].ctrl : d0.ctrl;
        atomicAdd(&cc->E_rad1, e_rad1);
        atomicAdd(&cc->E_mat1, e_mat1);
        if (b_in != 0.0) atomicAdd(&cc->bnd_in_macro, b_in);
      }
    }
    if (roleA) {
      bad = __any_sync(0xffffffffu, bad) ? 1 : 0;
      const unsigned sc_n = __reduce_add_sync(0xffffffffu, (unsigned)scaled);
      if (lane == 0 && acc_m >= 0) {
        Ctrl* cc = ENS ? e.devs[acc_m].ctrl : d0.ctrl;
        if (bad) atomicOr(&cc->status, ST_NONFINITE);
        if (sc_n) {
          atomicOr(&cc->scaled, 1u);
          atomicAdd(&cc->n_scaled_bins, sc_n);
        }
      }
    }
  }
  if (blockIdx.x == 0) {
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
      Ctrl* cc = ENS ? e.devs[k].ctrl : d0.ctrl;
      const int ran = s_conv[ENS ? k : 0];
      cc->si_iters = (unsigned int)(ran ? ran : itB);
      cc->si_iters32 = (unsigned int)itA;
      cc->si_state_ok = warm ? 0u : 1u;
      if (!ran) atomicOr(&cc->status, ST_NOCONV);
    }
  }
  (void)all_done;
}

// End of step (ensembles): the sorted survivors are back in the input buffer,
// which stays the live one; advance the step counter, particle ledger from
// the side tallies.
template <bool ENS>
__global__ void k_end_step(const __grid_constant__ Dev d0, const Ens e) {
  const Dev& d = ENS ? e.devs[blockIdx.y] : d0;
  Ctrl* ctrl = d.ctrl;
  if (threadIdx.x == 0) {
    const unsigned long long n = ctrl->n_out;
    const unsigned long long cap = (unsigned long long)d.capacity;
    const unsigned live = ctrl->cur;
    ctrl->n_part[live] = n < cap ? n : cap;
    ctrl->n_part[live ^ 1u] = 0;
    ctrl->step += 1;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double pin = 0.0, pout = 0.0;
    for (int i = threadIdx.x; i < 6 * d.G; i += 32) { pin += d.inflow[i]; pout += d.esc[i]; }
    pin = warp_sum(pin);
    pout = warp_sum(pout);
    if (threadIdx.x == 0) {
      ctrl->bnd_in_part = pin / d.c;
      ctrl->bnd_out_part = pout / d.c;
    }
  }
}

// Survivors' weights scaled by the factor the source-iteration epilogue set
// for their (cell, group) (a reading where the paper is silent: the particle
// part never exceeds rho^{n+1}).  Runs after the survivor sort; a member with
// nothing to scale returns at once.
// Scale the first n survivors of buffer b by their bins' factors, four
// particles a thread (one 16-byte key load, four independent factor
// gathers); only the particles whose factor is not 1 are written.  For
// ensembles: many members, each with many scaled bins of a few particles.
__device__ __forceinline__ void scale_weights_flat(const Dev& d, unsigned b, long long n) {
  const uint32_t* __restrict__ key = d.pkey[b];
  const bool mixed = d.precision == 1;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; 4 * q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const long long i0 = 4 * q;
    uint32_t k[4];
    if (i0 + 3 < n) {
      const uint4 kk = *reinterpret_cast<const uint4*>(key + i0);
      k[0] = kk.x; k[1] = kk.y; k[2] = kk.z; k[3] = kk.w;
    } else {
      for (int r = 0; r < 4; ++r) k[r] = i0 + r < n ? key[i0 + r] : 0u;
    }
    double f[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) f[r] = i0 + r < n ? __ldg(d.wscale + k[r]) : 1.0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (f[r] == 1.0) continue;
      if (mixed) d.fw[b][i0 + r] = (float)((double)d.fw[b][i0 + r] * f[r]);
      else d.pw[b][i0 + r] *= f[r];
    }
  }
}

// Scale the weights of buffer b's survivors by their bins' factors.  The
// survivors are sorted by bin: after the scatter, bin k holds the slots
// [sort_off[k] - sort_cnt[k], sort_off[k]), so only the bins whose factor
// is not 1 are touched (a warp checks 32 bins, then scales each such bin's
// run with all its lanes).  Warp w of nw over the problem's bins; for a
// single problem, whose grid has thousands of warps and few scaled bins.
__device__ __forceinline__ void scale_weights(const Dev& d, unsigned b, long long w, long long nw) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long nb = (long long)d.ncell * d.G;
  const bool mixed = d.precision == 1;
  for (long long k0 = 32 * w; k0 < nb; k0 += 32 * nw) {
    const long long k = k0 + lane;
    const double f = k < nb ? d.wscale[k] : 1.0;
    unsigned todo = __ballot_sync(full, f != 1.0);
    while (todo) {
      const int l = __ffs(todo) - 1;
      todo &= todo - 1;
      const double fk = __shfl_sync(full, f, l);
      const long long end = (long long)d.sort_off[k0 + l], begin = end - (long long)d.sort_cnt[k0 + l];
      // 256 weights a pass, their loads issued together (a run is a few
      // hundred survivors; one load round trip per weight would serialise)
      for (long long i0 = begin + lane; i0 < end; i0 += 256) {
        if (mixed) {
          float v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] = i0 + 32 * u < end ? d.fw[b][i0 + 32 * u] : 0.0f;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (i0 + 32 * u < end) d.fw[b][i0 + 32 * u] = (float)((double)v[u] * fk);
        } else {
          double v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] = i0 + 32 * u < end ? d.pw[b][i0 + 32 * u] : 0.0;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (i0 + 32 * u < end) d.pw[b][i0 + 32 * u] = v[u] * fk;
        }
      }
    }
  }
}

template <bool ENS>
__global__ void __launch_bounds__(256) k_scale_survivors(const __grid_constant__ Dev d0, const Ens e) {
  const Dev& d = ENS ? e.devs[blockIdx.y] : d0;
  const Ctrl* ctrl = d.ctrl;
  if (!ctrl->scaled) return;
  scale_weights_flat(d, ctrl->cur, (long long)ctrl->n_part[ctrl->cur]);
}

// End of step of a single problem in one launch: the sorted survivors'
// weights are scaled in the input buffer (the bins the split capped), and
// block 0 records their count, advances the step and sums the particle
// ledger.  The other blocks read only the live-buffer index and the scaled
// flag of the control block, which block 0 does not write, so no block
// waits for another.
__global__ void __launch_bounds__(256) k_finish_step(const __grid_constant__ Dev d) {
  Ctrl* ctrl = d.ctrl;
  const unsigned live = ctrl->cur;
  // block 0: the counts and the particle ledger (nothing else in this
  // kernel reads the words it writes, so it needs no other block)
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    double pin = 0.0, pout = 0.0;
    for (int i = threadIdx.x; i < 6 * d.G; i += 32) { pin += d.inflow[i]; pout += d.esc[i]; }
    pin = warp_sum(pin);
    pout = warp_sum(pout);
    if (threadIdx.x == 0) {
      const unsigned long long no = ctrl->n_out, cap = (unsigned long long)d.capacity;
      ctrl->n_part[live] = no < cap ? no : cap;
      ctrl->n_part[live ^ 1u] = 0;
      ctrl->step += 1;
      ctrl->bnd_in_part = pin / d.c;
      ctrl->bnd_out_part = pout / d.c;
    }
  }
  if (ctrl->scaled)
    scale_weights(d, live, (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5,
                  ((long long)gridDim.x * blockDim.x) >> 5);
}

// --------------------------------------------------------------------------
// Survivor sort by bin (cell, group), every step and in every build.  The
// particle kernel left each particle of the step in its slot of the other
// buffer, survivors with their end bin and the rest marked kDeadKey, and
// counted the stored survivors per bin; the counts are scanned into write
// cursors (their total is the step's survivor count, n_out), and this
// scatter moves every survivor into the input buffer at its bin's cursor.
// It runs beside the source iteration, which touches no particle; the end
// of step then scales the sorted survivors.  The order inside a bin follows
// the cursor atomics: nothing depends on it (random streams are keyed by
// particle identity, tallies are integer sums).  A taped FP64 step also
// records each survivor's new slot in its tape entry (where the adjoint
// finds the particle in the next step's input).

// Runs of equal keys among the warp's lanes: start lane of this lane's run
// and its length (at every lane of the run).
__device__ __forceinline__ void warp_runs(uint32_t key, int* start, int* len) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const uint32_t prev = __shfl_up_sync(full, key, 1);
  const unsigned heads = __ballot_sync(full, lane == 0 || prev != key);
  *start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
  const unsigned after = heads & ~(0xffffffffu >> (31 - lane));   // heads above this lane
  *len = (after ? __ffs(after) - 1 : 32) - *start;
}

template <typename F>
struct PartBufs {
  F *x, *ox, *nu, *w, *y, *oy, *z, *oz;
  unsigned long long* id;
  uint32_t* key;
};

template <typename F>
__device__ __forceinline__ PartBufs<F> part_bufs(const Dev& d, unsigned b);
template <>
__device__ __forceinline__ PartBufs<float> part_bufs<float>(const Dev& d, unsigned b) {
  return PartBufs<float>{d.fx[b], d.fox[b], d.fnu[b], d.fw[b], d.fy[b], d.foy[b], d.fz[b], d.foz[b],
                         d.pid[b], d.pkey[b]};
}
template <>
__device__ __forceinline__ PartBufs<double> part_bufs<double>(const Dev& d, unsigned b) {
  return PartBufs<double>{d.px[b], d.pox[b], d.pnu[b], d.pw[b], d.py[b], d.poy[b], d.pz[b], d.poz[b],
                          d.pid[b], d.pkey[b]};
}

// Two 32-slices [i0, i0 + 64) of the step's slots (below n): loads of both
// first, then both cursor atomics, then the stores, so a warp has two
// round trips in flight.
template <typename F, int DIM>
__device__ __forceinline__ void scatter_two(const Dev& d, unsigned cur, long long i0, long long n) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const PartBufs<F> src = part_bufs<F>(d, cur ^ 1u), dst = part_bufs<F>(d, cur);
  uint32_t k[2];
  unsigned long long id[2];
  F a[2][8];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const long long i = i0 + 32 * q + lane;
    k[q] = i < n ? __ldcs(src.key + i) : kDeadKey;
    id[q] = 0ull;
#pragma unroll
    for (int f = 0; f < 8; ++f) a[q][f] = F(0);
    if (k[q] != kDeadKey) {
      id[q] = __ldcs(src.id + i);
      a[q][0] = __ldcs(src.x + i); a[q][1] = __ldcs(src.ox + i);
      a[q][2] = __ldcs(src.nu + i); a[q][3] = __ldcs(src.w + i);
      if (DIM >= 2) { a[q][4] = __ldcs(src.y + i); a[q][5] = __ldcs(src.oy + i); }
      if (DIM == 3) { a[q][6] = __ldcs(src.z + i); a[q][7] = __ldcs(src.oz + i); }
    }
  }
  long long o[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int start, len;
    warp_runs(k[q], &start, &len);
    unsigned b = 0u;
    if (lane == start && k[q] != kDeadKey) b = atomicAdd(d.sort_off + k[q], (unsigned)len);
    b = __shfl_sync(full, b, start);
    o[q] = (long long)b + (lane - start);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (k[q] == kDeadKey) continue;
    if (o[q] >= d.capacity) {   // counts and slots disagree: never expected
      atomicOr(&d.ctrl->status, ST_CAPACITY);
      continue;
    }
    const long long j = o[q];
    dst.x[j] = a[q][0]; dst.ox[j] = a[q][1]; dst.nu[j] = a[q][2]; dst.w[j] = a[q][3];
    if (DIM >= 2) { dst.y[j] = a[q][4]; dst.oy[j] = a[q][5]; }
    if (DIM == 3) { dst.z[j] = a[q][6]; dst.oz[j] = a[q][7]; }
    dst.id[j] = id[q];
    dst.key[j] = k[q];
    const long long i = i0 + 32 * q + lane;
    if (d.tape && i < d.tape_cap) d.tape[i].slot = (int)j;
  }
}

template <typename F, int DIM, bool ENS>
__global__ void __launch_bounds__(256) k_sort_scatter(const __grid_constant__ Dev d0, const Ens e) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  if (!ENS) {
    const Ctrl* ctrl = d0.ctrl;
    const unsigned cur = ctrl->cur;
    const unsigned long long nt = ctrl->n_part[cur] + ctrl->n_new, cap = (unsigned long long)d0.capacity;
    const long long n = (long long)(nt < cap ? nt : cap);
    // one contiguous chunk of whole 64-slot pairs per warp, so warps running
    // at the same time work on different bins of the (nearly sorted) slots
    const long long per = ((n + nw - 1) / nw + 63) & ~63ll;
    const long long lo = w * per, hi = lo + per < n ? lo + per : n;
    for (long long i0 = lo; i0 < hi; i0 += 64) scatter_two<F, DIM>(d0, cur, i0, hi);
    return;
  }
  // ensembles: the particle kernel's tiles (e.tile slots each), one warp per
  // 64-slot pair of a tile
  const long long tile = e.tile, pairs = (tile + 63) / 64;
  const long long ntiles = (long long)e.tile0[e.M];
  for (long long u = w; u < ntiles * pairs; u += nw) {
    const long long t = u / pairs, pr = u - t * pairs;
    const int m = find_member(e.tile0, e.M, t);
    const Dev& d = e.devs[m];
    const Ctrl* ctrl = d.ctrl;
    const unsigned cur = ctrl->cur;
    const unsigned long long nt = ctrl->n_part[cur] + ctrl->n_new, cap = (unsigned long long)d.capacity;
    const long long n = (long long)(nt < cap ? nt : cap);
    const long long base = (t - (long long)e.tile0[m]) * tile, i0 = base + 64 * pr;
    const long long hi = base + tile < n ? base + tile : n;
    if (i0 < hi) scatter_two<F, DIM>(d, cur, i0, hi);
  }
}

// --------------------------------------------------------------------------
// Checkpoint / restore of a member's state in a caller buffer laid out as
// [Ctrl][T][rho][rho_h][rho_p][particle arrays, capacity entries each].
// Only the particles alive in the current buffer are copied; their count is
// read on the device (from the live control block when saving, from the
// saved one when restoring), so neither direction synchronises the host.
struct CkptLayout {
  size_t ctrl, T, rho, rho_h, rho_p, part[10], total;
};

__host__ __device__ inline size_t ckpt_align(size_t x) { return (x + 255) & ~size_t(255); }

__host__ __device__ inline CkptLayout ckpt_layout(const Dev& d) {
  CkptLayout L;
  const size_t nc = (size_t)d.ncell, ncg = (size_t)d.ncell * d.G, P = (size_t)d.capacity;
  const size_t fs = d.precision == 1 ? 4 : 8;
  size_t o = 0;
  L.ctrl = o; o = ckpt_align(o + sizeof(Ctrl));
  L.T = o; o = ckpt_align(o + 8 * nc);
  L.rho = o; o = ckpt_align(o + 8 * ncg);
  L.rho_h = o; o = ckpt_align(o + 8 * ncg);
  L.rho_p = o; o = ckpt_align(o + 8 * ncg);
  for (int k = 0; k < 6; ++k) { L.part[k] = o; o = ckpt_align(o + fs * P); }   // x y ox oy nu w
  L.part[6] = o; o = ckpt_align(o + 8 * P);                                   // id
  L.part[7] = o; o = ckpt_align(o + 4 * P);                                   // key
  const size_t zs = d.dim == 3 ? fs * P : 0;
  L.part[8] = o; o = ckpt_align(o + zs);                                      // z (3D)
  L.part[9] = o; o = ckpt_align(o + zs);                                      // oz (3D)
  L.total = o;
  return L;
}

size_t ckpt_bytes(const Dev& d) { return ckpt_layout(d).total; }
size_t ckpt_ids_offset(const Dev& d) { return ckpt_layout(d).part[6]; }
size_t ckpt_ctrl_offset(const Dev& d) { return ckpt_layout(d).ctrl; }

template <typename TT>
__device__ __forceinline__ void copy_n(TT* dst, const TT* src, long long n) {
  if (!dst || !src) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// save = 1: state -> buf; save = 0: buf -> state.  Member = blockIdx.y.
__global__ void k_checkpoint(const Ens e, const __grid_constant__ Dev d0, char* buf, const size_t* offs, int save) {
  const Dev& d = e.M > 1 ? e.devs[blockIdx.y] : d0;
  char* b = buf + offs[blockIdx.y];
  const CkptLayout L = ckpt_layout(d);
  Ctrl* saved = reinterpret_cast<Ctrl*>(b + L.ctrl);
  const Ctrl* src_ctrl = save ? d.ctrl : saved;
  const unsigned cur = src_ctrl->cur;
  const long long n = (long long)src_ctrl->n_part[cur];
  const long long nc = d.ncell, ncg = (long long)d.ncell * d.G;
  double* T = reinterpret_cast<double*>(b + L.T);
  double* rho = reinterpret_cast<double*>(b + L.rho);
  double* rho_h = reinterpret_cast<double*>(b + L.rho_h);
  double* rho_p = reinterpret_cast<double*>(b + L.rho_p);
  if (save) {
    copy_n(T, (const double*)d.T, nc);
    copy_n(rho, (const double*)d.rho, ncg);
    copy_n(rho_h, (const double*)d.rho_h, ncg);
    copy_n(rho_p, (const double*)d.rho_p, ncg);
  } else {
    copy_n(d.T, (const double*)T, nc);
    copy_n(d.rho, (const double*)rho, ncg);
    copy_n(d.rho_h, (const double*)rho_h, ncg);
    copy_n(d.rho_p, (const double*)rho_p, ncg);
  }
  if (d.precision == 1) {
    float* live[8] = {d.fx[cur], d.fy[cur], d.fox[cur], d.foy[cur], d.fnu[cur], d.fw[cur], d.fz[cur], d.foz[cur]};
    for (int k = 0; k < 8; ++k) {
      float* c = reinterpret_cast<float*>(b + L.part[k < 6 ? k : k + 2]);
      if (save) copy_n(c, (const float*)live[k], n); else copy_n(live[k], (const float*)c, n);
    }
  } else {
    double* live[8] = {d.px[cur], d.py[cur], d.pox[cur], d.poy[cur], d.pnu[cur], d.pw[cur], d.pz[cur], d.poz[cur]};
    for (int k = 0; k < 8; ++k) {
      double* c = reinterpret_cast<double*>(b + L.part[k < 6 ? k : k + 2]);
      if (save) copy_n(c, (const double*)live[k], n); else copy_n(live[k], (const double*)c, n);
    }
  }
  unsigned long long* cid = reinterpret_cast<unsigned long long*>(b + L.part[6]);
  uint32_t* ckey = reinterpret_cast<uint32_t*>(b + L.part[7]);
  if (save) {
    copy_n(cid, (const unsigned long long*)d.pid[cur], n);
    copy_n(ckey, (const uint32_t*)d.pkey[cur], n);
  } else {
    copy_n(d.pid[cur], (const unsigned long long*)cid, n);
    copy_n(d.pkey[cur], (const uint32_t*)ckey, n);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (save) *saved = *d.ctrl;
    else {
      *d.ctrl = *saved;
      d.ctrl->si_state_ok = 0;   // the iterate state is not part of a checkpoint
    }
  }
}

cudaError_t launch_checkpoint(const Dev& d, const Ens* e, char* buf, const size_t* d_offs, int save,
                              cudaStream_t s) {
  const Ens none{};
  const int M = e && e->M > 1 ? e->M : 1;
  k_checkpoint<<<dim3(sm_count() * 4, M), 256, 0, s>>>(e && e->M > 1 ? *e : none, d, buf, d_offs, save);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// kernel-level entry points
__global__ void k_unit_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 o = philox4x32_10(c, k0, k1);
    out[4 * i] = o.x; out[4 * i + 1] = o.y; out[4 * i + 2] = o.z; out[4 * i + 3] = o.w;
  }
}

__global__ void k_unit_planck(const double* T, long long n, const double* nu, int G, double* b,
                              double* dd) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * G;
       i += (long long)gridDim.x * blockDim.x) {
    const long long t = i / G;
    const int g = (int)(i - t * G);
    const double TT = T[t];
    const EdgeVal lo = planck_edge(nu[g] / TT), hi = planck_edge(nu[g + 1] / TT);
    const double bb = planck_fraction(lo, hi);
    b[i] = bb;
    if (dd) dd[i] = planck_dfraction(bb, lo, hi);
  }
}

__global__ void k_unit_coefs(const double* x, long long n, double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double xx = x[i];
    out[4 * i] = coef_f2(xx);
    out[4 * i + 1] = coef_f4(xx);
    out[4 * i + 2] = coef_f5(xx);
    out[4 * i + 3] = coef_c4(xx);
  }
}

__global__ void k_unit_sample(const double* eta, long long n, double nlo, double nhi, double T,
                              double* nu) {
  const double kh = sampler_khat(nlo, nhi, T);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    nu[i] = sample_nu(nlo, nhi, kh, eta[i]);
}

// --------------------------------------------------------------------------
// host launchers
int sm_count() {
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  if (dev < kMaxDevices) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  if (n < 1) n = 1;
  if (dev < kMaxDevices) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

// blocks for n items of `threads` each, at most `per_sm` blocks per SM
static int grid_for(long long n, int threads, int per_sm = 16) {
  long long b = (n + threads - 1) / threads;
  const long long cap = (long long)sm_count() * per_sm;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

cudaError_t launch_init_tables(const Dev& d, const double* src_T, const double* src_amp, int init_rho, cudaStream_t s) {
  k_init_pow<<<1, 64, 0, s>>>(d);
  k_init_tables<<<grid_for((long long)d.ncell * d.G, 256), 256, 0, s>>>(d, src_T, src_amp, init_rho);
  return cudaGetLastError();
}

int scan_parts(long long n) { return (int)((n + kScanTile - 1) / kScanTile); }

cudaError_t launch_scan(const uint32_t* N, long long n, uint32_t* part, uint32_t* off,
                        unsigned long long* total_a, unsigned long long* total_b, cudaStream_t s) {
  const int nparts = scan_parts(n);
  if (nparts > 0) k_scan_reduce<<<nparts, kScanThreads, 0, s>>>(N, n, part);
  k_scan_partials<<<1, kScanThreads, 0, s>>>(part, nparts, off + n, total_a, total_b);
  if (nparts > 0) k_scan_apply<<<nparts, kScanThreads, 0, s>>>(N, n, part, off);
  return cudaGetLastError();
}

// One-block exclusive scan of n <= 16 tiles of counts (grids of modest size):
// one launch instead of three; the total goes to off[n] and the two counters.
__global__ void __launch_bounds__(kScanThreads) k_scan_small(const uint32_t* __restrict__ N, long long n,
                                                            uint32_t* __restrict__ off,
                                                            unsigned long long* total_a,
                                                            unsigned long long* total_b) {
  // a kernel launched after this one as its programmatic dependent may set
  // itself up now (it waits for this kernel's results before reading them)
  asm volatile("griddepcontrol.launch_dependents;");
  uint32_t carry = 0;
  for (long long t = 0; t * kScanTile < n; ++t) {
    const long long base = t * kScanTile + (long long)threadIdx.x * kScanPer;
    uint32_t v[kScanPer], s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) { v[k] = base + k < n ? N[base + k] : 0u; s += v[k]; }
    uint32_t tot;
    uint32_t ex = block_exclusive_scan(s, &tot) + carry;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      if (base + k < n) off[base + k] = ex;
      ex += v[k];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) {
    off[n] = carry;
    if (total_a) *total_a = carry;
    if (total_b) *total_b = carry;
  }
}

cudaError_t launch_birth_and_scan(const Dev& d, const Ens* e, cudaStream_t s) {
  if (e && e->M > 1) {
    k_birth<true><<<grid_for(e->total_bins, 64, 64), 64, 0, s>>>(d, *e);
    const dim3 g(e->max_parts, e->M);
    k_scan_reduce_ens<<<g, kScanThreads, 0, s>>>(*e, 0);
    k_scan_partials_ens<<<dim3(1, e->M), kScanThreads, 0, s>>>(*e, 0);
    k_scan_apply_ens<<<g, kScanThreads, 0, s>>>(*e, 0);
    k_tiles<<<1, 1024, 0, s>>>(*e);
    return cudaGetLastError();
  }
  const Ens none{};
  k_birth<false><<<grid_for(d.nbins, 64), 64, 0, s>>>(d, none);
  if (d.nbins <= 16 * kScanTile) {
    k_scan_small<<<1, kScanThreads, 0, s>>>(d.N, d.nbins, d.off, &d.ctrl->n_new, &d.ctrl->n_born);
    return cudaGetLastError();
  }
  return launch_scan(d.N, d.nbins, d.part, d.off, &d.ctrl->n_new, &d.ctrl->n_born, s);
}

cudaError_t launch_wave(const Dev& d, const Ens* e, cudaStream_t s) {
  const bool f32 = d.precision == 1;   // mixed precision
  if (e && e->M > 1) {
    if (f32) k_wave32<true><<<grid_for(e->total_fg, 128, 64), 128, 0, s>>>(d, *e);
    else k_wave<true><<<grid_for(e->total_fg, 64, 64), 64, 0, s>>>(d, *e);
  } else {
    const Ens none{};
    if (f32) k_wave32<false><<<grid_for((long long)d.nface * d.G, 128), 128, 0, s>>>(d, none);
    else k_wave<false><<<grid_for((long long)d.nface * d.G, 64), 64, 0, s>>>(d, none);
  }
  return cudaGetLastError();
}

static int g_si_blocks[2][2][3] = {};

// One warp per cell.  On GB300 the FP64 pipe of an SM is the limit of this
// kernel, so a small grid is spread one warp per block over all SMs; a large
// grid uses 8-warp blocks (fewer arrivals at the grid barrier).
// items: the kernel's work items (a warp's cells each; pair mode: one cell
// per two-warp block)
template <int NC, bool ENS, bool PAIR>
static cudaError_t launch_si_t(const Dev& d, const Ens& e, long long items, cudaStream_t s) {
  const int sms = sm_count();
  const int small = items <= 8 * sms;
  const int threads = PAIR ? 64 : (small ? 32 : 256);
  int& per = g_si_blocks[NC - 1][ENS][PAIR ? 2 : small];
  if (!per) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_si<NC, ENS, PAIR>, threads, 0);
    if (per < 1) per = 1;
  }
  const long long want = PAIR ? items : (items * 32 + threads - 1) / threads;
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
  return cudaLaunchKernelEx(&cfg, k_si<NC, ENS, PAIR>, d, e);
}

cudaError_t launch_si(const Dev& d, const Ens* e, cudaStream_t s) {
  if (e && e->M > 1) {
    if (e->M > kMaxEnsemble) return cudaErrorInvalidValue;
    if (e->max_G > 32) return launch_si_t<2, true, false>(d, *e, e->total_items, s);
    return launch_si_t<1, true, false>(d, *e, e->total_items, s);
  }
  const Ens none{};
  // a 1D grid of at most two cells per SM, FP64 iterates only: two warps per
  // cell (one warp per cell would leave most SM sub-partitions idle)
  const bool pair = d.dim == 1 && !d.si_warm && d.ncell <= 2 * sm_count() && d.pair_si;
  const int cpw = 32 / seg_width(d.G);
  const long long items = ((long long)d.ncell + cpw - 1) / cpw;
  if (d.G > 32) {
    if (pair) return launch_si_t<2, false, true>(d, none, d.ncell, s);
    return launch_si_t<2, false, false>(d, none, items, s);
  }
  if (pair) return launch_si_t<1, false, true>(d, none, d.ncell, s);
  return launch_si_t<1, false, false>(d, none, items, s);
}

cudaError_t launch_end_step(const Dev& d, const Ens* e, cudaStream_t s) {
  if (e && e->M > 1) {
    k_end_step<true><<<dim3(1, e->M), 32, 0, s>>>(d, *e);
    k_scale_survivors<true><<<dim3(8, e->M), 256, 0, s>>>(d, *e);
  } else {
    // a warp per 32 bins (a scaled bin's run is scaled by the warp that
    // finds it), so the blocks' arrivals at the end stay few
    const long long nb = (long long)d.ncell * d.G;
    const long long blocks = (nb + 255) / 256;
    k_finish_step<<<(int)(blocks < sm_count() * 4 ? (blocks > 0 ? blocks : 1) : sm_count() * 4), 256, 0, s>>>(d);
  }
  return cudaGetLastError();
}

template <typename F, bool ENS>
static void launch_scatter(const Dev& d, const Ens& e, int blocks, cudaStream_t s) {
  if (d.dim == 3) k_sort_scatter<F, 3, ENS><<<blocks, 256, 0, s>>>(d, e);
  else if (d.dim == 2) k_sort_scatter<F, 2, ENS><<<blocks, 256, 0, s>>>(d, e);
  else k_sort_scatter<F, 1, ENS><<<blocks, 256, 0, s>>>(d, e);
}

cudaError_t launch_sort(const Dev& d, const Ens* e, cudaStream_t s) {
  // a quarter of the SM threads: the scatter runs beside the source iteration,
  // whose cooperative blocks must find room on every SM
  const int blocks = sm_count() * 2;
  const bool mixed = d.precision == 1;
  if (e && e->M > 1) {
    const dim3 g(e->max_parts, e->M);
    k_scan_reduce_ens<<<g, kScanThreads, 0, s>>>(*e, 1);
    k_scan_partials_ens<<<dim3(1, e->M), kScanThreads, 0, s>>>(*e, 1);
    k_scan_apply_ens<<<g, kScanThreads, 0, s>>>(*e, 1);
    if (mixed) launch_scatter<float, true>(d, *e, blocks, s);
    else launch_scatter<double, true>(d, *e, blocks, s);
    return cudaGetLastError();
  }
  if (d.nbins <= 16 * kScanTile) {
    k_scan_small<<<1, kScanThreads, 0, s>>>(d.sort_cnt, d.nbins, d.sort_off, &d.ctrl->n_out, nullptr);
  } else {
    cudaError_t r = launch_scan(d.sort_cnt, d.nbins, d.sort_part, d.sort_off, &d.ctrl->n_out, nullptr, s);
    if (r) return r;
  }
  const Ens none{};
  if (mixed) launch_scatter<float, false>(d, none, blocks, s);
  else launch_scatter<double, false>(d, none, blocks, s);
  return cudaGetLastError();
}

cudaError_t launch_unit_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, long long n,
                               cudaStream_t s) {
  k_unit_philox<<<grid_for(n, 256), 256, 0, s>>>(ctr, k0, k1, out, n);
  return cudaGetLastError();
}
cudaError_t launch_unit_planck(const double* T, long long n, const double* nu, int G, double* b,
                               double* dd, cudaStream_t s) {
  k_unit_planck<<<grid_for(n * G, 256), 256, 0, s>>>(T, n, nu, G, b, dd);
  return cudaGetLastError();
}
cudaError_t launch_unit_coefs(const double* x, long long n, double* out, cudaStream_t s) {
  k_unit_coefs<<<grid_for(n, 256), 256, 0, s>>>(x, n, out);
  return cudaGetLastError();
}
cudaError_t launch_unit_sample(const double* eta, long long n, double nlo, double nhi, double T,
                               double* nu, cudaStream_t s) {
  k_unit_sample<<<grid_for(n, 256), 256, 0, s>>>(eta, n, nlo, nhi, T, nu);
  return cudaGetLastError();
}

}  // namespace ugkwp
