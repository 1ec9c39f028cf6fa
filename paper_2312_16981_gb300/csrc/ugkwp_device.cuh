// ugkwp_device.cuh -- device building blocks of the UGKWP particle phase on
// sm_103a: counter-based random numbers, opacities, Planck group fractions,
// time-integrated flux coefficients and the linear-frequency sampler.
//
// Method: Yang, Zhu, Liu, Xu, "Unified gas-kinetic wave-particle method for
// frequency-dependent radiation transport equation".
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ugkwp_c2_table.h"
#include "ugkwp_log_table.h"
#include "ugkwp_planck_table.h"

namespace ugkwp {

constexpr int kMaxG = 64;
constexpr int kMaxEnsemble = 4096;   // members advanced together in one step
constexpr double kPi = 3.14159265358979323846;
constexpr double kPi4over15 = kPi * kPi * kPi * kPi / 15.0;   // int_0^inf t^3/(e^t-1) dt
constexpr double k15overPi4 = 15.0 / (kPi * kPi * kPi * kPi);

enum { BC_REFLECT = 0, BC_VACUUM = 1, BC_BLACKBODY = 2 };
enum { FATE_SURVIVED = 0, FATE_ABSORBED = 1, FATE_ESCAPED = 2, FATE_REMOVED = 3 };
enum : uint32_t { ST_CAPACITY = 1u, ST_NOCONV = 2u, ST_NONFINITE = 4u, ST_TIMEOUT = 8u, ST_IDSPACE = 16u };

// Bits of a newborn's 64-bit identity: (birth step << 44) | (bin << 20) | k.
// The step takes the top 20 bits: a handle refuses to step past 2^20 - 1
// (identities, and with them the random streams, would repeat).
constexpr int kIdBinShift = 20;
constexpr int kIdStepShift = 44;
constexpr uint32_t kMaxPerBin = (1u << 20) - 1u;
constexpr unsigned long long kMaxStep = (1ull << 20) - 1ull;

// Key of a slot the particle kernel leaves empty (a particle that did not
// survive, written in place); the survivor sort skips it.
constexpr uint32_t kDeadKey = 0xffffffffu;

// --------------------------------------------------------------------------
// Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// The key schedule (k0 + r W0, k1 + r W1 for rounds r = 0..9) is the same
// for every draw of a problem, so the particle kernels read it from the
// problem constants instead of adding the Weyl increments per round.
struct PhiloxKeys {
  uint32_t a[10], b[10];
};

__host__ __device__ inline PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
  PhiloxKeys k;
  for (int r = 0; r < 10; ++r) {
    k.a[r] = k0;
    k.b[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return k;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ k.a[r], lo1, hi0 ^ c.w ^ k.b[r], lo0);
  }
  return c;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
  return philox4x32_10(c, philox_keys(k0, k1));
}

// Uniform in (0,1): the 52 top bits m of (a, b), then m 2^-52 + 2^-53 (exact).
__device__ __forceinline__ double u01(uint32_t a, uint32_t b) {
  const unsigned long long m = ((unsigned long long)a << 20) | (unsigned long long)(b >> 12);
  return __ll2double_rn((long long)m) * 0x1p-52 + 0x1p-53;
}

// -ln u for u in (0, 1) in FP64 without the library logarithm (the FP64
// particle kernel is bound by its FP64 instructions, and a library log costs
// about thirty FMAs there): ln(1 + x) by the table-driven method of Tang
// (ACM TOMS 16, 1990) on one argument per lane -- x = u - 1 (exact) for
// u > 1/2, else u = 2^k m with m in [1/sqrt 2, sqrt 2] and x = m - 1 (exact)
// -- with breakpoints c_j = 1 + j/128 from ugkwp_log_table.h, r = (x -
// j/128)/c_j, |r| <= 1/128, ln(1 + r) by its series to r^7, and k ln 2 in two
// parts.  Within about an ulp of -ln u.
constexpr double kLn2Hi = 0x1.62e42fefa3800p-1, kLn2Lo = 0x1.ef35793c76730p-45;

__device__ __forceinline__ double neg_log_u64(double u) {
  double x, kd;
  if (u > 0.5) {
    x = u - 1.0;
    kd = 0.0;
  } else {
    const long long b = __double_as_longlong(u);
    int k = (int)((b >> 52) & 0x7ff) - 1023;
    long long mb = (b & 0x000fffffffffffffll) | 0x3ff0000000000000ll;   // m in [1, 2)
    if (mb > 0x3ff6a09e667f3bcdll) { mb -= 0x0010000000000000ll; ++k; }  // m > sqrt 2: halve
    x = __longlong_as_double(mb) - 1.0;
    kd = (double)k;
  }
  const double jd = rint(x * 128.0);
  const double2 t = __ldg(reinterpret_cast<const double2*>(kLogTab) + ((int)jd - kLogJMin));
  const double r = (x - jd * (1.0 / 128.0)) * t.x;
  double p = 1.0 / 7.0;
  p = fma(p, r, -1.0 / 6.0);
  p = fma(p, r, 1.0 / 5.0);
  p = fma(p, r, -0.25);
  p = fma(p, r, 1.0 / 3.0);
  p = fma(p, r, -0.5);
  const double l1p = fma(r * r, p, r);
  return -fma(kd, kLn2Hi, t.y + fma(kd, kLn2Lo, l1p));
}

// The draw sequence of one particle in one step: draw j comes from Philox
// block j/2 of counter (id_lo, id_hi, step, j/2), words (0,1) for even j and
// (2,3) for odd j; one Philox evaluation serves two draws.
struct Draws {
  uint32_t id_lo, id_hi, step, j, held;   // held = 1 + index of the Philox block in blk
  uint4 blk;
  __device__ __forceinline__ void init(unsigned long long id, uint32_t s, uint32_t first) {
    id_lo = (uint32_t)id;
    id_hi = (uint32_t)(id >> 32);
    step = s;
    j = first;
    held = 0;
  }
  __device__ __forceinline__ double next(const PhiloxKeys& pk) {
    const uint32_t b = j >> 1;
    if (held != b + 1u) {
      blk = philox4x32_10(make_uint4(id_lo, id_hi, step, b), pk);
      held = b + 1u;
    }
    const double u = (j & 1u) ? u01(blk.z, blk.w) : u01(blk.x, blk.y);
    ++j;
    return u;
  }
};

// FP32 uniforms from the same two words as the FP64 draw
// u = (m + 1/2) 2^-52, m = (a << 20) | (b >> 12): u and 1 - u are each formed
// with 2^-24 relative precision (so -ln u stays accurate both for small u and
// for u near 1), both in (0, 1).  -ln u uses log1p(-(1-u)) above u = 1/2.
struct UPair {
  float u, v;   // u and 1 - u
};

__device__ __forceinline__ UPair u01f(uint32_t a, uint32_t b) {
  UPair r;
  r.u = __uint2float_rz(a) * 0x1p-32f + (__uint2float_rz(b >> 12) + 0.5f) * 0x1p-52f;
  r.v = __uint2float_rz(~a) * 0x1p-32f + (__uint2float_rz((~b) >> 12) + 0.5f) * 0x1p-52f;
  return r;
}

// -ln u from the pair (u, 1 - u) without branching: ln(1 + x) = 2 atanh(t),
// t = x/(2 + x), on one argument chosen per lane -- x = -(1 - u) when
// 1 - u < 1/2 (so u near 1 keeps its relative precision), else u = 2^k m
// with m in [sqrt(1/2), sqrt(2)) and x = m - 1 (exact) -- and
// 2 atanh(t) = 2t (1 + t^2/3 + t^4/5 + ... + t^14/15) for |t| <= 1/3
// (truncation below 2^-24 relative); -ln u = -(k ln 2 + ln(1 + x)).
__device__ __forceinline__ float neg_log_u(const UPair& p) {
  const bool near1 = p.v < 0.5f;
  const unsigned b = __float_as_uint(p.u);
  int k = (int)((b >> 23) & 0xffu) - 127;
  unsigned mb = (b & 0x7fffffu) | 0x3f800000u;           // m in [1, 2)
  if (mb > 0x3fb504f3u) { mb -= 0x00800000u; ++k; }      // m in [sqrt(1/2), sqrt(2))
  const float x = near1 ? -p.v : __uint_as_float(mb) - 1.0f;
  const float kf = near1 ? 0.0f : (float)k;
  const float t = __fdividef(x, 2.0f + x);
  const float t2 = t * t;
  float s = 1.0f / 15.0f;
  s = fmaf(s, t2, 1.0f / 13.0f);
  s = fmaf(s, t2, 1.0f / 11.0f);
  s = fmaf(s, t2, 1.0f / 9.0f);
  s = fmaf(s, t2, 1.0f / 7.0f);
  s = fmaf(s, t2, 1.0f / 5.0f);
  s = fmaf(s, t2, 1.0f / 3.0f);
  s = fmaf(s, t2, 1.0f);
  // ln 2 split so that k ln 2 is exact in the first product
  return -fmaf(kf, 0x1.62e400p-1f, fmaf(kf, 0x1.7f7d1cp-20f, 2.0f * t * s));
}

// q = n / d for n < 2^24 with n/d < 2^22 (the caller checks Dev::fastdiv): an
// FP32 estimate from the reciprocal, within one of the quotient, corrected.
__device__ __forceinline__ uint32_t div_small(uint32_t n, uint32_t d, float inv_d) {
  uint32_t q = __float2uint_rz(__uint2float_rn(n) * inv_d);
  int r = (int)(n - q * d);
  if (r < 0) { --q; r += (int)d; }
  if (r >= (int)d) ++q;
  return q;
}

struct DrawsF {
  uint32_t id_lo, id_hi, step, j, held;
  uint4 blk;
  __device__ __forceinline__ void init(unsigned long long id, uint32_t s, uint32_t first) {
    id_lo = (uint32_t)id;
    id_hi = (uint32_t)(id >> 32);
    step = s;
    j = first;
    held = 0;
  }
  __device__ __forceinline__ UPair next2(const PhiloxKeys& pk) {
    const uint32_t b = j >> 1;
    if (held != b + 1u) {
      blk = philox4x32_10(make_uint4(id_lo, id_hi, step, b), pk);
      held = b + 1u;
    }
    const UPair u = (j & 1u) ? u01f(blk.z, blk.w) : u01f(blk.x, blk.y);
    ++j;
    return u;
  }
  __device__ __forceinline__ float next(const PhiloxKeys& pk) { return next2(pk).u; }
};

// --------------------------------------------------------------------------
// Problem constants and device pointers, passed to every kernel by value.
struct Dev {
  // geometry / model
  int dim, nx, ny, G, ncell, nbins, nface, nxface;
  int nz, nyface;    // nz = 1 below 3D; nyface = 0 in 1D
  int grey, wave_order, si_max_iters, precision, sig_law;
  int method;        // 0 UGKWP, 1 UGKP (all of I^h sampled; newborns draw t_f)
  int cv_law;        // 0 constant cv; 1 Olson foam heat capacity
  int split_literal; // 1: rho^h = rho^{n+1} - E_surv/V as written (no survivor scaling)
  double cv_chi, src_t_end;
  int bc[6];          // sides x-, x+, y-, y+, z-, z+
  double dx, dy, dz, vol, sig_p, sig_q, sig_cap, a, c, eps, dt;
  double v;          // c/eps, particle speed
  double rate_f;     // c/eps^2: 1/tau = rate_f * sigma
  double omega_ref, si_tol, src_on, tau_num_C;
  double bcT[6];
  double area[3];    // face area normal to each axis (1D: 1; 2D: the other width)
  uint32_t key0, key1;
  PhiloxKeys pk;     // Philox round keys of (key0, key1)
  long long capacity;
  // constant inputs
  const double* nu_edges;   // [G+1]
  const double* sigma0;     // [ncell]
  const double* cv;         // [ncell]
  const double* src;        // [ncell*G] per-step source increment of rho (or null)
  const double* ghost_phi;  // [6*G] Phi_g(T_b) per side
  const double* ghost_sig;  // [6*G] sigma_g(T_b) per side (sigma0 of the adjacent cell)
  // state
  double* T;        // [ncell]   T^n, then T^{n+1}
  double* rho;      // [ncell*G] rho^n, then rho^{n+1}
  double* rho_h;    // [ncell*G]
  double* rho_p;    // [ncell*G]
  // per-step work arrays
  double* sigT;     // [ncell*G] sigma_g(T^n)
  double* sT;       // [ncell]   sigma0 T^q
  double* sTinv;    // [ncell]   1/(sigma0 T^q)
  uint32_t* N;      // [nbins]
  uint32_t* off;    // [nbins+1] exclusive scan of N
  uint32_t* part;   // [scan partials]
  // counting sort of the survivors by bin (every step)
  uint32_t* sort_cnt;   // [nbins] survivors per bin this step
  uint32_t* sort_off;   // [nbins+1] their exclusive scan, then the bins' write cursors
  uint32_t* sort_part;  // [scan partials]
  double* omega;    // [nbins]
  double* xnum;     // [nbins] dt/tau_num of the bin (dt/tau where tau_num_C = 0)
  double* e_eff;    // [nbins]
  double* khat;     // [nbins] sampler slope in units of B(nu_mid)
  double* W;        // [ncell*G] (FP64 copy written by the source iteration)
  double* E_surv;   // [ncell*G] (FP64 copy written by the source iteration)
  unsigned long long* Wq;    // [ncell*G][2] W in fixed point (accumulated, see atomic_add_fixed)
  unsigned long long* Esq;   // [ncell*G][2] E_surv in fixed point (accumulated)
  double inv_dx, inv_dy, inv_dz, inv_c, inv_vol;
  double inv_2dt;             // 1/(2 dt)
  double two_dt;              // 2 dt
  double feq_k[3];            // dt (v^2/3)/h per axis: F^eq = C2/dt feq_k (Phi_u - Phi_l)
  double dt_h[3];             // dt/h per axis
  double tq, tq_inv;         // fixed-point quantum 2^-tq_shift (about omega_ref 2^-48) and its inverse
  int tq_shift;
  // FP32 copies of scalars (mixed-precision particle kernel)
  float dxf, dyf, dzf, vf, dtf, inv_rate_f, capf, spf, inv_capf;
  int fastdiv;               // ncell*G < 2^24: divide by G and nx with div_small
  float invG_f, inv_nx_f;    // 1/G, 1/nx in FP32
  double inv_cap;            // 1/sig_cap, or 0 without a cap
  double* esc;      // [6*G]
  double* inflow;   // [6*G]
  double* Fwave;    // [nface*G]
  double* Feq;      // [nface*G]
  double* R;        // [ncell*G] constant part of the rho equation
  double* wscale;   // [ncell*G] end-of-step scaling of the survivors' weights (1: none)
  double* Tk[2];    // [ncell] iterates
  double* tauk[2];  // [ncell*G] relaxation time 1/(rate_f sigma_g(T^k)) of the iterate
  double* qk;       // [ncell*G] 1/(tau + dt) of the iterate (read by the cell's own warp)
  double* phik[2];  // [ncell*G]
  float* dphik;     // [ncell*G] dPhi_g/dT of the iterate (FP32: it sets only the contraction rate)
  // FP32 warm start of the source iteration (mixed precision; null otherwise)
  int si_warm;      // 1: FP32 iterates before the FP64 ones this step
  int pair_si;      // 1: two warps per cell where the source iteration allows it
  float* Tk_f[2];   // [ncell]
  float* tau_f[2];  // [ncell*G]
  float* phi_f[2];  // [ncell*G]
  float* q_f;       // [ncell*G]
  float* R_f;       // [ncell*G]
  float* Feq_f;     // [nface*G] (2D and 3D face pass)
  float* nu_pow_f;  // [3G]
  float* olson_nu_f;  // [9G] (sig_law 2)
  float feq_kf[3], two_dtf, inv_2dtf, ratef, acf, inv_cf;
  // particles: two structure-of-arrays buffers, selected by ctrl->cur
  double* px[2];
  double* py[2];
  double* pox[2];
  double* poy[2];
  double* pz[2];        // 3D only
  double* poz[2];
  double* pnu[2];
  double* pw[2];
  unsigned long long* pid[2];
  uint32_t* pkey[2];    // bin c*G + g
  // mixed precision: FP32 state, positions local to the cell (0 <= xi <= dx)
  float* fx[2];
  float* fy[2];
  float* fox[2];
  float* foy[2];
  float* fz[2];         // 3D only
  float* foz[2];
  float* fnu[2];
  float* fw[2];
  double* olson_c;  // [3 ncell] foam opacity T factors A, B, C at T^n (sig_law 2)
  double* olson_nu; // [9 G] foam opacity nu factors at each Simpson point (sig_law 2)
  float* olson_cf;  // [3 ncell] A, B, C in FP32 (mixed precision)
  float* sT_f;      // [ncell] sigma0 T^q
  float* sTinv_f;   // [ncell] 1/(sigma0 T^q)
  float* invT_f;    // [ncell] 1/T^n (photo-ionisation factor of sig_law 1)
  float* omega_f;   // [nbins]
  float* khat_f;    // [nbins]
  float* nu_edges_f;       // [G+1] group edges in FP32
  const double* nu_pow;    // [3*G] nu^p at the lower edge, midpoint and upper edge of each group
  void* particles_begin;   // first particle buffer (start of the part left uninitialised)
  // control block and optional records
  struct Ctrl* ctrl;
  struct RecordOut* rec;
  long long rec_cap;
  // optional adjoint tape: one entry per processed particle (taped steps only)
  struct TapeRec* tape;
  long long tape_cap;
};

// Material energy per volume and heat capacity: cv[c] T and cv[c], or the
// Olson foam (cv_law 1, Eq. cvolson): cv[c] (T + (T + chi) alpha) and cv[c]
// (1 + alpha + (T + chi) alpha'), alpha = (sqrt(u^2 + 4u) - u)/2 with
// u = e^{-chi/T} (the paper's form without its overflow at small T),
// alpha' = (chi/T^2) (alpha - sqrt(u/(u + 4))).
__device__ __forceinline__ double foam_alpha(double chi, double T, double* dalpha) {
  const double u = exp(-chi / T);
  const double al = 0.5 * (sqrt(fma(u, u, 4.0 * u)) - u);
  if (dalpha) *dalpha = chi / (T * T) * (al - sqrt(u / (u + 4.0)));
  return al;
}

__device__ __forceinline__ double mat_energy(const Dev& d, int c, double T) {
  if (d.cv_law != 1) return d.cv[c] * T;
  return d.cv[c] * (T + (T + d.cv_chi) * foam_alpha(d.cv_chi, T, nullptr));
}

__device__ __forceinline__ double heat_capacity(const Dev& d, int c, double T) {
  if (d.cv_law != 1) return d.cv[c];
  double da;
  const double al = foam_alpha(d.cv_chi, T, &da);
  return d.cv[c] * (1.0 + al + (T + d.cv_chi) * da);
}

// Bin -> cell and cell -> grid row, for indices the problem holds.
__device__ __forceinline__ uint32_t div_bin(const Dev& d, uint32_t key) {
  return d.fastdiv ? div_small(key, (uint32_t)d.G, d.invG_f) : key / (uint32_t)d.G;
}
__device__ __forceinline__ uint32_t div_nx(const Dev& d, uint32_t cell) {
  return d.fastdiv ? div_small(cell, (uint32_t)d.nx, d.inv_nx_f) : cell / (uint32_t)d.nx;
}

// Ensemble view (independent problems advanced together): per-member
// descriptors and prefix tables over the members' index spaces.  Member m
// owns global indices [tab[m], tab[m+1]).  A single problem uses M = 1 and the
// kernels' non-ensemble instantiation, which never reads these tables.
// Lanes per cell in the source iteration: the smallest of 8, 16, 32 that
// holds G groups (32 above 16); a warp serves 32 / seg_width(G) cells.
__host__ __device__ inline int seg_width(int G) { return G <= 8 ? 8 : (G <= 16 ? 16 : 32); }

struct Ens {
  int M;
  const Dev* devs;        // [M] member descriptors (device copy)
  const int* cell0;       // [M+1] prefix of ncell
  const int* bin0;        // [M+1] prefix of nbins
  const int* fg0;         // [M+1] prefix of nface*G
  const int* item0;       // [M+1] prefix of the source iteration's work items (warps' cells)
  int* tile0;             // [M+1] prefix of this step's particle tiles (written on the device)
  unsigned int* bar;      // grid-barrier arrivals of the ensemble source iteration
  unsigned long long* tile_next;   // next particle tile to hand out (reset with bar each step)
  // totals known on the host (launch shapes)
  long long total_bins, total_fg, total_cells, total_items;
  int max_parts, max_G;
  int tile;               // particles per tile of the particle kernel's tile table
};

// Launch shape of the particle kernel (picked by the autotuner).  The
// mixed-precision kernel streams chunks of 32 x ppt particles per warp, the
// FP64 kernel tiles of block x ppt.
struct StreamShape {
  int block = 256;        // threads per block: 128, 256 or 512
  int ppt = 4;            // particles per thread per tile: 1, 2 or 4 (the FP64 kernel takes 2 for 4)
  int blocks_per_sm = 0;  // 0: as many as fit
};

// Member owning global index i: largest m with tab[m] <= i.
__device__ __forceinline__ int find_member(const int* __restrict__ tab, int M, long long i) {
  int lo = 0, hi = M;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((long long)__ldg(tab + mid) <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// Record layout identical to ugkwp_record in the public header.
struct RecordOut {
  unsigned long long id;
  int fate, cell0, cell1, grp, nseg, pad;
  double x, y, ox, oy, nu, w, t_end;
  double z, oz;
};

// Adjoint tape entry of one processed particle: where its weight was counted
// in this step.  c0 = start cell, or -1 - side for a black-body ghost birth;
// c1 = end cell of a survivor or the collision cell of an absorbed particle,
// else -1 (escaped, removed); slot = its index in the next step's input if it
// survived, else -1; g = group; w = its weight in this step (before the
// end-of-step scaling of survivors).
struct TapeRec {
  int c0, c1, slot, g;
  double w;
};

// Deterministic tallies.  W and E_surv are sums of particle weights added by
// many threads in an order that changes from run to run; in FP64 that order
// shows in the last bits, and through T in every later decision.  Each
// weight is instead rounded once to a fixed quantum q (a power of two between
// omega_ref 2^-49 and omega_ref 2^-48, a few 1e-15 of a reference weight) and
// the integers are added with integer atomics (a 32-bit low part and a
// signed high part per tally, atomic_add_fixed), which commute: a run is
// bitwise reproducible.  Weights up to 2^57 q (at least 256 omega_ref)
// are representable; a larger one sets the non-finite status bit.
constexpr double kFixedRange = 0x1p57;   // |w/q| below this: a warp's 32 add up without overflow

__device__ __forceinline__ long long to_fixed(double v, double q_inv, unsigned int* status) {
  const double x = v * q_inv;
  if (!(fabs(x) < kFixedRange)) {
    atomicOr(status, 4u);   // ST_NONFINITE: weight out of the tally range
    return 0;
  }
  return __double2ll_rn(x);
}

// The same conversion for an FP32 weight without FP64 arithmetic: w = m 2^(e-150)
// with a 24-bit integer m, so w/q = m 2^(e-150+shift) is formed with integer
// shifts (exact while q is finer than w's last bit, else rounded half up).
__device__ __forceinline__ long long to_fixed_f(float w, int shift, unsigned int* status) {
  const unsigned b = __float_as_uint(w);
  const int ex = (int)((b >> 23) & 0xffu);
  if (ex == 0) return 0;                  // zero (or a subnormal weight, below any quantum)
  const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
  const int sh = ex - 150 + shift;
  long long r;
  if (ex == 255 || sh > 33) {             // non-finite or |w/q| >= 2^57
    atomicOr(status, 4u);
    return 0;
  }
  if (sh >= 0) r = m << sh;
  else r = sh < -40 ? 0 : ((m + (1ll << (-sh - 1))) >> (-sh));
  return (b >> 31) ? -r : r;
}

// Carry-free 96-bit accumulation of signed 64-bit increments x = xh 2^32 + xl
// (xl = the low 32 bits, unsigned; xh = x >> 32, signed): c[0] sums the xl
// (below 2^32 each, so 2^32 of them cannot overflow 64 bits) and c[1] the xh
// in two's complement.  Both adds are fire-and-forget reductions: nothing
// waits for an old value, and the integer sums still commute, so a run stays
// bitwise reproducible.  The value is c[1] 2^32 + c[0].
__device__ __forceinline__ void atomic_add_fixed(unsigned long long* c, long long x) {
  if (x == 0) return;
  const unsigned long long lo = (unsigned long long)x & 0xffffffffull;
  const unsigned long long hi = (unsigned long long)(x >> 32);
  if (lo) atomicAdd(c, lo);
  if (hi) atomicAdd(c + 1, hi);
}

// The accumulated value times q, rounded once: c[1] 2^32 + c[0] is formed
// exactly as H 2^32 + L with L < 2^32 (H = c[1] + (c[0] >> 32), |H| < 2^53 for
// any tally this code holds), so only the final addition rounds.
__device__ __forceinline__ double from_fixed(const unsigned long long* c, double q) {
  const unsigned long long lo = __ldcg(c), hi = __ldcg(c + 1);
  const long long H = (long long)hi + (long long)(lo >> 32);
  const double L = (double)(lo & 0xffffffffull);
  return fma((double)H, 0x1p32, L) * q;
}

// Device control block: counters, status, barrier and reduction slots.
struct Ctrl {
  unsigned long long step;
  unsigned long long n_part[2];   // particles held in buffer 0/1
  unsigned int cur;               // buffer holding this step's input
  unsigned int status;            // ST_* bits, latched
  unsigned long long n_new, n_out;
  unsigned long long n_in, n_born, n_survived, n_absorbed, n_escaped, n_removed, n_segments;
  unsigned int si_iters;
  unsigned int bar_count;         // grid barrier arrivals (monotone)
  unsigned int bar_timeout_spins; // bounded-wait limit (0: default)
  unsigned int bar_extra;         // arrivals a barrier also waits for (failure injection; 0)
  unsigned int scaled;            // some survivors' weights need scaling this step
  unsigned int pad4_;
  unsigned long long tile_next;   // next particle tile to hand out (particle kernel; 0 at step start)
  unsigned long long pad3_;
  unsigned int n_scaled_bins;     // (cell, group) bins whose survivors were scaled this step
  unsigned int si_iters32;        // FP32 warm-start iterates of the last source iteration
  unsigned int si_state_ok;       // 1: slot 0 of the iterate state holds T^n's (the last iteration's
                                  // final state; cleared where T changes outside the step)
  unsigned int pad2_;
  unsigned long long err_slot[3][2];  // per-iteration max errors (double bit patterns)
  double E_rad0, E_mat0, E_rad1, E_mat1, bnd_in_macro, bnd_in_part, bnd_out_part, src_in;
};

// --------------------------------------------------------------------------
// Opacity sigma(nu, T) = sigma0 nu^p T^q, capped (Eq. sigmaMarsharkMF form).
__device__ __forceinline__ double pow_fast(double b, double e) {
  if (e == 0.0) return 1.0;
  if (e == -3.0) return 1.0 / (b * b * b);
  if (e == 3.0) return b * b * b;
  if (e == -0.5) return rsqrt(b);
  if (e == 1.0) return b;
  return pow(b, e);
}

// min(s, cap) for s >= 0 (or NaN: the cap), compared as bit patterns (the
// order of non-negative doubles) on the integer pipes: an FP64 compare costs
// an FP64 instruction, the scarce unit on this chip
__device__ __forceinline__ double cap_sigma(const Dev& d, double s) {
  const long long cap_bits = d.sig_cap > 0.0 ? __double_as_longlong(d.sig_cap) : 0x7fffffffffffffffll;
  return __double_as_longlong(s) > cap_bits ? d.sig_cap : s;
}

// 1/x for finite x > 0 away from the under- and overflow limits, to about an
// ulp: the hardware reciprocal approximation (rcp.approx.ftz.f64, relative
// error below 2^-19.9 as measured on sm_103a) and one third-order step:
// with e = 1 - x r, r (1 + e + e^2) = (1 - e^3)/x, an error below 2^-59.
// Three FP64 FMAs where a correctly rounded division takes about three times
// as many FP64 instructions; the source iteration's fixed point does not
// need the last bit.
__device__ __forceinline__ double rcp_nr(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// sigma0*T^q for cell c at temperature T
__device__ __forceinline__ double sigma_T(const Dev& d, int c, double T) {
  return d.sigma0[c] * pow_fast(T, d.sig_q);
}

// Simpson group opacity (Sec. 3: edges and midpoint, weights 1-4-1), with
// nu^p at the three points taken from a table built once.
__device__ __forceinline__ double sigma_group(const Dev& d, double sT, int g) {
  if (d.grey) return cap_sigma(d, sT);
  const double sa = cap_sigma(d, sT * __ldg(d.nu_pow + 3 * g));
  const double sm = cap_sigma(d, sT * __ldg(d.nu_pow + 3 * g + 1));
  const double sb = cap_sigma(d, sT * __ldg(d.nu_pow + 3 * g + 2));
  return (sa + 4.0 * sm + sb) * (1.0 / 6.0);
}

// Group opacity at temperature T: with sig_law 1 each Simpson point carries
// the photo-ionisation factor (1 - e^{-nu/T}) of the Larsen case (Sec. 3.3)
// before the cap.
// Olson foam opacity (sig_law 2, Sec. 3.5): kappa(nu, T) is A(T) for
// nu <= 0.008, B(T) (0.008/nu)^2 for nu <= 0.3, and B(T) (0.008/nu)^2
// (0.3/nu)^0.5 + C(T) (0.3/nu)^2.5 above, with A = min(1e7, 1e9 T^2),
// B = 3e6/(1 + 200 T^1.5), C = 4e4/(1 + 8000 T^2); sigma = sigma0 kappa.
struct FoamT {
  double A, B, C;
};

__device__ __forceinline__ FoamT foam_T(double T) {
  FoamT f;
  f.A = fmin(1e7, 1e9 * T * T);
  f.B = 3e6 / (1.0 + 200.0 * T * sqrt(T));
  f.C = 4e4 / (1.0 + 8000.0 * T * T);
  return f;
}

// nu factors (0.008/nu)^2, (0.008/nu)^2 (0.3/nu)^0.5, (0.3/nu)^2.5
__device__ __forceinline__ void foam_nu(double nu, double* f1, double* f2, double* f3) {
  const double inv = 1.0 / nu, a = 0.008 * inv, r = 0.3 * inv, sq = sqrt(r);
  *f1 = a * a;
  *f2 = a * a * sq;
  *f3 = r * r * sq;
}

__device__ __forceinline__ double foam_kappa(double nu, double A, double B, double C, double f1, double f2,
                                             double f3) {
  if (nu <= 0.008) return A;
  if (nu <= 0.3) return B * f1;
  return B * f2 + C * f3;
}

__device__ __forceinline__ double sigma_group_at(const Dev& d, double sT, double T, double invT, int g) {
  if (d.grey || d.sig_law == 0) return sigma_group(d, sT, g);
  const double a = d.nu_edges[g], b = d.nu_edges[g + 1], m = 0.5 * (a + b);
  if (d.sig_law == 2) {
    const FoamT f = foam_T(T);
    const double* t = d.olson_nu + 9 * g;
    const double sa = cap_sigma(d, sT * foam_kappa(a, f.A, f.B, f.C, __ldg(t), __ldg(t + 1), __ldg(t + 2)));
    const double sm = cap_sigma(d, sT * foam_kappa(m, f.A, f.B, f.C, __ldg(t + 3), __ldg(t + 4), __ldg(t + 5)));
    const double sb = cap_sigma(d, sT * foam_kappa(b, f.A, f.B, f.C, __ldg(t + 6), __ldg(t + 7), __ldg(t + 8)));
    return (sa + 4.0 * sm + sb) * (1.0 / 6.0);
  }
  const double sa = cap_sigma(d, sT * __ldg(d.nu_pow + 3 * g) * -expm1(-a * invT));
  const double sm = cap_sigma(d, sT * __ldg(d.nu_pow + 3 * g + 1) * -expm1(-m * invT));
  const double sb = cap_sigma(d, sT * __ldg(d.nu_pow + 3 * g + 2) * -expm1(-b * invT));
  return (sa + 4.0 * sm + sb) * (1.0 / 6.0);
}

__device__ __forceinline__ double sigma_group_at(const Dev& d, double sT, double T, int g) {
  return sigma_group_at(d, sT, T, 1.0 / T, g);
}

// 1/sigma(nu, T^n) of a particle in `cell`: max(1/(sigma0 T^q nu^p [1 - e^{-nu/T}]), 1/cap)
// from the per-cell 1/(sigma0 T^q) and 1/nu^p (inup); multiplications except
// for the photo-ionisation factor.
__device__ __forceinline__ double inv_sigma_particle(const Dev& d, int cell, double nu, double inup) {
  if (d.sig_law == 2 && !d.grey) {
    double f1, f2, f3;
    foam_nu(nu, &f1, &f2, &f3);
    const double* c = d.olson_c + 3 * cell;
    const double k = foam_kappa(nu, c[0], c[1], c[2], f1, f2, f3);
    return fmax(d.sTinv[cell] / k, d.inv_cap);
  }
  double si = d.sTinv[cell] * inup;
  if (d.sig_law == 1 && !d.grey) si /= -expm1(-nu / d.T[cell]);
  return fmax(si, d.inv_cap);
}

__device__ __forceinline__ float inv_sigma_particle_f(const Dev& d, int cell, float nu, float inup) {
  if (d.sig_law == 2 && !d.grey) {
    const float inv = __frcp_rn(nu), a = 0.008f * inv, r = 0.3f * inv, sq = sqrtf(r);
    const float* c = d.olson_cf + 3 * cell;
    float k;
    if (nu <= 0.008f) k = __ldg(c);
    else if (nu <= 0.3f) k = __ldg(c + 1) * (a * a);
    else k = __ldg(c + 1) * (a * a * sq) + __ldg(c + 2) * (r * r * sq);
    return fmaxf(__fdividef(__ldg(d.sTinv_f + cell), k), d.inv_capf);
  }
  float si = __ldg(d.sTinv_f + cell) * inup;
  if (d.sig_law == 1 && !d.grey) si /= -expm1f(-nu * __ldg(d.invT_f + cell));
  return fmaxf(si, d.inv_capf);
}

// d sigma_g / d s for sigma0 -> sigma0 e^s: the Simpson sum of the point
// values below the cap (a capped point does not depend on s).  The
// T-derivative is q/T times the same sum.
__device__ __forceinline__ double sigma_group_ds(const Dev& d, double sT, int g) {
  auto pt = [&](double s) { return (d.sig_cap > 0.0 && !(s <= d.sig_cap)) ? 0.0 : s; };
  if (d.grey) return pt(sT);
  const double sa = pt(sT * __ldg(d.nu_pow + 3 * g));
  const double sm = pt(sT * __ldg(d.nu_pow + 3 * g + 1));
  const double sb = pt(sT * __ldg(d.nu_pow + 3 * g + 2));
  return (sa + 4.0 * sm + sb) * (1.0 / 6.0);
}

// --------------------------------------------------------------------------
// Planck integrals per group edge x = nu/T.  The lower part
//   L(x) = int_0^x t^3/(e^t-1) dt = x^3/3 - x^4/8 + sum_m B_2m x^{2m+3}/((2m+3)(2m)!)
// and the upper part
//   U(x) = int_x^inf t^3/(e^t-1) dt = sum_n e^{-nx} (x^3/n + 3x^2/n^2 + 6x/n^3 + 6/n^4),
// with g4(x) = x^4/(e^x - 1), are read from piecewise degree-10 interpolants
// of these series (ugkwp_planck_table.h, written in 60-digit arithmetic by
// gen_tables.py; relative error 2e-16): one Horner pass over one row
// for every lane, whatever its x, so a warp whose groups straddle x = 2 no
// longer runs both series (the upper one needs up to 20 terms near x = 2).
//   x < 2:       L = x^3 p1(s),  g4 = x^3 p2(s)
//   2 <= x < 40: U = p1(s),      g4 = p2(s)
//   x >= 40:     U = e^{-x} (x^3 + 3x^2 + 6x + 6),  g4 = e^{-x} x^4

// Per edge: value V (L(x) if x < 2 else U(x)), flag lower, and x^4/(e^x - 1).
struct EdgeVal {
  double V, g4;
  bool lower;
};

__device__ __forceinline__ EdgeVal planck_edge(double x) {
  EdgeVal r;
  if (!(x > 0.0)) { r.V = 0.0; r.g4 = 0.0; r.lower = true; return r; }
  if (x > 740.0) { r.V = 0.0; r.g4 = 0.0; r.lower = false; return r; }
  const bool tail = x >= 40.0;
  const int j = tail ? kPlanckRows : (int)(x * 2.0);
  const double s = tail ? x : (x - (0.25 + 0.5 * j)) * 4.0;
  const double2* row = reinterpret_cast<const double2*>(kPlanckTab) + j * (kPlanckDeg + 1);
  double2 a = __ldg(row + kPlanckDeg);
  double p1 = a.x, p2 = a.y;
#pragma unroll
  for (int k = kPlanckDeg - 1; k >= 0; --k) {
    a = __ldg(row + k);
    p1 = fma(p1, s, a.x);
    p2 = fma(p2, s, a.y);
  }
  r.lower = j < kPlanckLowerRows;
  double m = 1.0;
  if (r.lower) m = x * x * x;
  else if (tail) m = exp(-x);
  r.V = m * p1;
  r.g4 = m * p2;
  return r;
}

// b = (15/pi^4) int_{x_lo}^{x_hi} t^3/(e^t-1) dt from the two edge values.
__device__ __forceinline__ double planck_fraction(const EdgeVal& lo, const EdgeVal& hi) {
  double I;
  if (hi.lower) I = hi.V - lo.V;
  else if (!lo.lower) I = lo.V - hi.V;
  else I = (kPi4over15 - lo.V) - hi.V;
  return k15overPi4 * I;
}

// dPhi_g/dT = a c T^3 [4 b + (15/pi^4)(g4(x_lo) - g4(x_hi))]: returns the bracket.
__device__ __forceinline__ double planck_dfraction(double b, const EdgeVal& lo, const EdgeVal& hi) {
  return 4.0 * b + k15overPi4 * (lo.g4 - hi.g4);
}

// --------------------------------------------------------------------------
// Time-integrated coefficients at x = dt/tau (Eq. C2Formula; C4, C5 of the
// UGKS free flux).  Below x = 1 the Taylor series (22 terms), else closed
// forms with expm1.
//   f2 = C2/tau          = sum_{k>=2} (-1)^k (1-k) x^k/(k+1)!
//   f4 = C4 - e          = sum_{k>=1} (-1)^{k+1} k x^k/(k+1)!
//   f5 = (C5 + dt e/2)/tau = sum_{k>=2} (-1)^k k(1-k) x^k/(2 (k+1)!)
//   c4 = C4              = sum_{k>=0} (-1)^k x^k/(k+1)!
__host__ __device__ constexpr double fact_d(int n) { return n <= 1 ? 1.0 : n * fact_d(n - 1); }
constexpr int kSer = 22;
__host__ __device__ constexpr double sgn(int k) { return (k & 1) ? -1.0 : 1.0; }
__host__ __device__ constexpr double a2(int k) { return sgn(k) * (1.0 - k) / fact_d(k + 1); }
__host__ __device__ constexpr double a4(int k) { return -sgn(k) * k / fact_d(k + 1); }
__host__ __device__ constexpr double a5(int k) { return sgn(k) * k * (1.0 - k) / (2.0 * fact_d(k + 1)); }
__host__ __device__ constexpr double ac4(int k) { return sgn(k) / fact_d(k + 1); }
// compile-time tables (k = 0..22)
#define UGKWP_SER_TABLE(f)                                                                   \
  {f(0),  f(1),  f(2),  f(3),  f(4),  f(5),  f(6),  f(7),  f(8),  f(9),  f(10), f(11),      \
   f(12), f(13), f(14), f(15), f(16), f(17), f(18), f(19), f(20), f(21), f(22)}
__device__ constexpr double kA2[kSer + 1] = UGKWP_SER_TABLE(a2);
__device__ constexpr double kA4[kSer + 1] = UGKWP_SER_TABLE(a4);
__device__ constexpr double kA5[kSer + 1] = UGKWP_SER_TABLE(a5);
__device__ constexpr double kAC4[kSer + 1] = UGKWP_SER_TABLE(ac4);
#undef UGKWP_SER_TABLE

__device__ __forceinline__ double coef_f2(double x) {
  if (x < 1.0) {
    double s = kA2[kSer];
#pragma unroll
    for (int k = kSer - 1; k >= 2; --k) s = fma(s, x, kA2[k]);
    return s * x * x;
  }
  const double e = exp(-x), E1 = -expm1(-x);
  return 2.0 * E1 / x - 1.0 - e;
}

// f2(x)/x (= C2/dt): the same series shifted by one power, or the closed form.
__device__ __forceinline__ double coef_g2(double x) {
  if (x < 1.0) {
    double s = kA2[kSer];
#pragma unroll
    for (int k = kSer - 1; k >= 2; --k) s = fma(s, x, kA2[k]);
    return s * x;
  }
  const double e = exp(-x), E1 = -expm1(-x);
  return (2.0 * E1 / x - 1.0 - e) / x;
}

// f2(x)/x (= C2/(tau x), C2 of Eq. C2Formula) for the source-iteration faces,
// given x and 1/x (the caller has both from the face's tau sum, x = 2 dt/(tau_l
// + tau_u)), from piecewise degree-10 interpolants (ugkwp_c2_table.h, written
// by gen_tables.py in 60-digit arithmetic; relative error 2e-16): one Horner
// pass for every lane, with no exp and no branch between the series and the
// closed form.  Rows 0..3 hold f2(x)/x^2, rows 4..79 g2 itself, row 80
// (x >= 40) (2/x - 1)/x as a polynomial in 1/x.
__device__ __forceinline__ double coef_g2_fast(double x, double ix) {
  const bool tail = x >= 40.0;
  const int j = tail ? kPlanckRows : (int)(x * 2.0);
  const double s = tail ? ix : (x - (0.25 + 0.5 * j)) * 4.0;
  const double* row = kC2Tab + j * (kPlanckDeg + 1);
  double p = __ldg(row + kPlanckDeg);
#pragma unroll
  for (int k = kPlanckDeg - 1; k >= 0; --k) p = fma(p, s, __ldg(row + k));
  return j < kPlanckLowerRows ? p * x : p;
}

__device__ __forceinline__ double coef_f4(double x) {
  if (x < 1.0) {
    double s = kA4[kSer];
#pragma unroll
    for (int k = kSer - 1; k >= 1; --k) s = fma(s, x, kA4[k]);
    return s * x;
  }
  return -expm1(-x) / x - exp(-x);
}

__device__ __forceinline__ double coef_f5(double x) {
  if (x < 1.0) {
    double s = kA5[kSer];
#pragma unroll
    for (int k = kSer - 1; k >= 2; --k) s = fma(s, x, kA5[k]);
    return s * x * x;
  }
  const double e = exp(-x);
  return e * (1.0 + 0.5 * x) + expm1(-x) / x;
}

__device__ __forceinline__ double coef_c4(double x) {
  if (x < 1.0) {
    double s = kAC4[kSer];
#pragma unroll
    for (int k = kSer - 1; k >= 0; --k) s = fma(s, x, kAC4[k]);
    return s;
  }
  return -expm1(-x) / x;
}

// x-derivatives of the same coefficients: the differentiated series below
// x = 1, and from the closed forms above it with e = exp(-x):
//   c4' = (e - c4)/x,  f4' = c4' + e,  f2' = 2 c4' + e,  f5' = -e (1 + x)/2 - c4'.
__host__ __device__ constexpr double da2(int k) { return k * a2(k); }
__host__ __device__ constexpr double da4(int k) { return k * a4(k); }
__host__ __device__ constexpr double da5(int k) { return k * a5(k); }
__host__ __device__ constexpr double dac4(int k) { return k * ac4(k); }
#define UGKWP_SER_TABLE(f)                                                                   \
  {f(0),  f(1),  f(2),  f(3),  f(4),  f(5),  f(6),  f(7),  f(8),  f(9),  f(10), f(11),      \
   f(12), f(13), f(14), f(15), f(16), f(17), f(18), f(19), f(20), f(21), f(22)}
__device__ constexpr double kD2[kSer + 1] = UGKWP_SER_TABLE(da2);
__device__ constexpr double kD4[kSer + 1] = UGKWP_SER_TABLE(da4);
__device__ constexpr double kD5[kSer + 1] = UGKWP_SER_TABLE(da5);
__device__ constexpr double kDC4[kSer + 1] = UGKWP_SER_TABLE(dac4);
#undef UGKWP_SER_TABLE

struct CoefDeriv {
  double f2, f4, f5, c4;
};

// sum_{k>=1} t[k] x^(k-1) by Horner
__device__ __forceinline__ double dser(const double* t, double x) {
  double s = t[kSer];
#pragma unroll
  for (int k = kSer - 1; k >= 1; --k) s = fma(s, x, t[k]);
  return s;
}

__device__ __forceinline__ CoefDeriv coef_derivs(double x) {
  CoefDeriv r;
  if (x < 1.0) {
    r.f2 = dser(kD2, x);
    r.f4 = dser(kD4, x);
    r.f5 = dser(kD5, x);
    r.c4 = dser(kDC4, x);
    return r;
  }
  const double e = exp(-x), c4 = -expm1(-x) / x;
  const double d4 = (e - c4) / x;
  r.c4 = d4;
  r.f4 = d4 + e;
  r.f2 = 2.0 * d4 + e;
  r.f5 = -0.5 * e * (1.0 + x) - d4;
  return r;
}

// f4, f5 and c4 at one x together (the wave flux needs all three per face):
// one Horner loop with three accumulators (terms to x^16) below x = 1/2, one
// exp/expm1 above (cancellation in f5 there costs at most ~30 ulp).
// Returns e = exp(-x) where it was computed (x >= 1/2), else -1.
constexpr int kSerW = 16;
__device__ __forceinline__ double coef_f4_f5_c4(double x, double* f4, double* f5, double* c4) {
  if (x < 0.5) {
    double s4 = kA4[kSerW], s5 = kA5[kSerW], sc = kAC4[kSerW];
#pragma unroll
    for (int k = kSerW - 1; k >= 2; --k) {
      s4 = fma(s4, x, kA4[k]);
      s5 = fma(s5, x, kA5[k]);
      sc = fma(sc, x, kAC4[k]);
    }
    s4 = fma(s4, x, kA4[1]);
    sc = fma(fma(sc, x, kAC4[1]), x, kAC4[0]);
    *f4 = s4 * x;
    *f5 = s5 * x * x;
    *c4 = sc;
    return -1.0;
  }
  const double e = exp(-x), m1 = expm1(-x);   // m1 = e - 1
  *c4 = -m1 / x;
  *f4 = *c4 - e;
  *f5 = e * (1.0 + 0.5 * x) - *c4;
  return e;
}

// --------------------------------------------------------------------------
// Linear-frequency sampling (Eqs. Blinear, kg; App. A).  With B in units of
// B(nu_mid) and slope khat clamped to |khat| <= 2/dnu (non-negative density),
// G(nu_lo + u) = eta is the quadratic (khat/2) u^2 + A u - eta dnu = 0 with
// A = 1 - khat dnu/2 >= 0; its root in [0, dnu] is taken in the form
// u = 2 eta dnu / (A + sqrt(A^2 + 2 khat eta dnu)), free of cancellation.
__device__ __forceinline__ double planck_ratio(double nu, double nmid, double T) {
  // B(nu)/B(nmid) = (nu/nmid)^3 e^{(nmid-nu)/T} (1 - e^{-nmid/T}) / (1 - e^{-nu/T})
  const double r = nu / nmid;
  double ex = (nmid - nu) / T;
  if (ex > 700.0) ex = 700.0;
  return r * r * r * exp(ex) * (expm1(-nmid / T) / expm1(-nu / T));
}

__device__ __forceinline__ double sampler_khat(double nlo, double nhi, double T) {
  if (!(T > 0.0)) return 0.0;
  const double dnu = nhi - nlo, nmid = 0.5 * (nlo + nhi);
  double k = (planck_ratio(nhi, nmid, T) - planck_ratio(nlo, nmid, T)) / dnu;
  const double kmax = 2.0 / dnu;
  k = fmin(fmax(k, -kmax), kmax);
  return k == k ? k : 0.0;
}

// The same slope in FP32 for the mixed-precision build, whose sampler runs
// in FP32 (the exponent is clamped where FP32 e^x overflows; the clamp on
// |khat| saturates first there).
__device__ __forceinline__ float planck_ratio_f(float nu, float nmid, float T) {
  const float r = __fdividef(nu, nmid);
  float ex = __fdividef(nmid - nu, T);
  if (ex > 80.0f) ex = 80.0f;
  return r * r * r * expf(ex) * __fdividef(expm1f(-nmid / T), expm1f(-nu / T));
}

__device__ __forceinline__ float sampler_khat_f(float nlo, float nhi, float T) {
  if (!(T > 0.0f)) return 0.0f;
  const float dnu = nhi - nlo, nmid = 0.5f * (nlo + nhi);
  float k = (planck_ratio_f(nhi, nmid, T) - planck_ratio_f(nlo, nmid, T)) / dnu;
  const float kmax = 2.0f / dnu;
  k = fminf(fmaxf(k, -kmax), kmax);
  return k == k ? k : 0.0f;
}

__device__ __forceinline__ double sample_nu(double nlo, double nhi, double khat, double eta) {
  const double dnu = nhi - nlo;
  const double A = fma(-0.5 * khat, dnu, 1.0);
  const double q = eta * dnu;
  const double u = 2.0 * q / (A + sqrt(fma(A, A, 2.0 * khat * q)));
  return fmin(nlo + u, nhi);
}

__device__ __forceinline__ float sample_nu_f(float nlo, float nhi, float khat, float eta) {
  const float dnu = nhi - nlo;
  const float A = fmaf(-0.5f * khat, dnu, 1.0f);
  const float q = eta * dnu;
  const float u = 2.0f * q / (A + sqrtf(fmaf(A, A, 2.0f * khat * q)));
  return fminf(nlo + u, nhi);
}

__device__ __forceinline__ float pow_fast_f(float b, float e) {
  if (e == 0.0f) return 1.0f;
  if (e == -3.0f) return __frcp_rn(b * b * b);
  if (e == 3.0f) return b * b * b;
  if (e == -0.5f) return rsqrtf(b);
  if (e == 1.0f) return b;
  return __powf(b, e);
}

// --------------------------------------------------------------------------
// Acquire loads of words other blocks update with atomics: plain L2 reads for
// spin-waits and for reading reduction slots after a grid barrier (polling
// with an atomic would queue behind the arrivals' read-modify-writes on the
// same address, and every thread of every block reads the slots).
__device__ __forceinline__ unsigned int load_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long load_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Hint: bring the 128-byte line holding p into L2.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// The error slots (T and rho) of the iterate just finished and of its
// predecessor, read after a grid barrier: relaxed GPU-scope loads (coherent
// at L2), all four in flight at once.  The barrier's acquire and block
// barrier already order them after every block's updates; acquire loads
// here would make each wait for the one before it.
struct ErrPair {
  double eT, eR, pT, pR;
};
__device__ __forceinline__ ErrPair load_err_slots(const unsigned long long (*slot)[2], int it) {
  unsigned long long a, b, c, e;
  const unsigned long long* s0 = slot[it % 3];
  const unsigned long long* s1 = slot[(it + 2) % 3];
  asm volatile(
      "ld.relaxed.gpu.global.u64 %0, [%4];\n\t"
      "ld.relaxed.gpu.global.u64 %1, [%5];\n\t"
      "ld.relaxed.gpu.global.u64 %2, [%6];\n\t"
      "ld.relaxed.gpu.global.u64 %3, [%7];"
      : "=l"(a), "=l"(b), "=l"(c), "=l"(e)
      : "l"(s0), "l"(s0 + 1), "l"(s1), "l"(s1 + 1)
      : "memory");
  ErrPair r;
  r.eT = __longlong_as_double((long long)a);
  r.eR = __longlong_as_double((long long)b);
  r.pT = __longlong_as_double((long long)c);
  r.pR = __longlong_as_double((long long)e);
  return r;
}

// --------------------------------------------------------------------------
// atomics on non-negative doubles ordered as their bit patterns
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* slot, double v) {
  if (v != v) v = __longlong_as_double(0x7FF0000000000000LL);  // NaN -> +inf
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

}  // namespace ugkwp
