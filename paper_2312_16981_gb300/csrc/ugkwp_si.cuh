// Arithmetic of the source iteration (App. B, Algorithm 2) arranged for the
// FP64 pipe of sm_103a, the scarce unit of that kernel: a warp instruction of
// FP64 add, multiply, FMA, compare, min/max or f64->f32 conversion holds the
// pipe for 64 cycles whatever the number of active lanes.
//
// What fixes the iteration's fixed point stays FP64, in the same operations
// as before: sigma_g, Phi_g (the Planck group integrals), the face fluxes
// F^eq, Q, the T and rho updates.  What does not is moved off the pipe:
//   - dPhi_g/dT, the slope of the linearised emission, only sets the
//     contraction rate (at T^{k+1} = T^k the slope cancels from both
//     updates), so it is evaluated and stored in FP32;
//   - the convergence measures |dT|/T and max_g |d rho_g| / sum_g |rho_g|
//     are formed in FP32 from the doubles' bit fields (relative error below
//     2^-20 in a measure compared with si_tol);
//   - table rows, range tests and the clamp of T are integer operations on
//     bit patterns.
#pragma once

#include "ugkwp_device.cuh"
#include "ugkwp_grid.cuh"

namespace ugkwp {

// bit patterns of the constants the range tests compare with (positive doubles
// order as their bit patterns)
constexpr long long kBits40 = 0x4044000000000000ll;     // 40.0
constexpr long long kBits740 = 0x4087200000000000ll;    // 740.0
constexpr long long kBits1em30 = 0x39b4484bfeebc2a0ll;  // 1e-30

// biased exponent field of a double
__device__ __forceinline__ int biased_exp(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }

// x as a float, mantissa truncated to 23 bits; below the float range +-0,
// above it (and inf, NaN) +-inf.  Integer operations only.
__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int ef = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  if (ef <= 0) return __uint_as_float(sign);
  if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)ef << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// a float as a double, exactly (subnormal floats as zero).  Integer operations only.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ex = (b >> 23) & 0xffu, sign = b & 0x80000000u, m = b & 0x7fffffu;
  if (ex == 0u) return __hiloint2double((int)sign, 0);
  const unsigned e64 = ex == 0xffu ? 0x7ffu : ex + 896u;   // 896 = 1023 - 127
  return __hiloint2double((int)(sign | (e64 << 20) | (m >> 3)), (int)(m << 29));
}

// |x| 2^(1023 - E) as a float, for a scale E (a biased exponent) at or above
// that of most operands: mantissa truncated to 23 bits, zero below the float
// range (and for zero or subnormal x), +inf above it and for inf or NaN.
__device__ __forceinline__ float scaled_mag(double x, int E) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int ex = (int)((hi >> 20) & 0x7ffu);
  if (ex == 0) return 0.0f;
  const int ef = ex - E + 127;
  if (ex == 0x7ff || ef >= 255) return __uint_as_float(0x7f800000u);
  if (ef <= 0) return 0.0f;
  return __uint_as_float(((unsigned)ef << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// floor(2 x) for 0 <= x < 2^50 from the bit pattern (the row of the
// half-unit-wide interpolant tables)
__device__ __forceinline__ int half_index(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;   // x = 1.m 2^e
  if (e < -1) return 0;
  const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
  return (int)(m >> (51 - e));
}

// -(2 j + 1) as a double, exactly, for 0 <= j < 2^30
__device__ __forceinline__ double neg_odd(int j) {
  const unsigned n = 2u * (unsigned)j + 1u;
  const int p = 31 - __clz(n);   // 2^p <= n < 2^(p+1)
  const unsigned long long mant = ((unsigned long long)n << (52 - p)) & 0xfffffffffffffull;
  return __longlong_as_double((long long)((1ull << 63) | ((unsigned long long)(p + 1023) << 52) | mant));
}

// sums of a and b over the warp with one FP64 add per level: after the first
// exchange the even lanes carry partial sums of a and the odd lanes of b;
// every lane returns both totals (bitwise the same in all lanes)
__device__ __forceinline__ void warp_sum2(double& a, double& b) {
  const bool odd = threadIdx.x & 1;
  double keep = odd ? b : a;
  const double send = odd ? a : b;
  keep += __shfl_xor_sync(0xffffffffu, send, 1);
#pragma unroll
  for (int o = 2; o < 32; o <<= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
  a = __shfl_sync(0xffffffffu, keep, 0);
  b = __shfl_sync(0xffffffffu, keep, 1);
}

// The lanes that serve one cell: a segment of `seg` lanes (8, 16 or 32, the
// smallest that holds the problem's G groups; 32 above 16), so that a warp
// carries 32/seg cells at once and an FP64 warp instruction, which costs the
// same whatever the number of active lanes, does the work of several cells
// where G is small.  Lane sl of a segment takes groups g = sl + seg j.  With
// seg = 32 every reduction below runs in the order of the whole-warp one.
struct Lanes {
  int seg, sub, sl, base;   // width, segment index in the warp, lane in it, its first lane
};

__device__ __forceinline__ Lanes lanes_of(int seg) {
  Lanes L;
  const int lane = threadIdx.x & 31;
  L.seg = seg;
  L.sl = lane & (seg - 1);
  L.base = lane - L.sl;
  L.sub = L.base / seg;
  return L;
}

// warp_sum2 within each segment (every lane of a segment gets its totals)
__device__ __forceinline__ void seg_sum2(double& a, double& b, const Lanes& L) {
  const bool odd = threadIdx.x & 1;
  double keep = odd ? b : a;
  const double send = odd ? a : b;
  keep += __shfl_xor_sync(0xffffffffu, send, 1);
  for (int o = 2; o < L.seg; o <<= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
  a = __shfl_sync(0xffffffffu, keep, L.base);
  b = __shfl_sync(0xffffffffu, keep, L.base + 1);
}

__device__ __forceinline__ float seg_sum_f(float v, const Lanes& L) {
  for (int o = L.seg >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned seg_max_u(unsigned v, const Lanes& L) {
  if (L.seg == 32) return __reduce_max_sync(0xffffffffu, v);
  for (int o = 1; o < L.seg; o <<= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max_nonneg_f(float v) {
  return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(v)));
}

// the g4 column of the Planck interpolant table in FP32 (filled once from the
// FP64 table by k_init_pow)
static __device__ float kG4TabF[(kPlanckRows + 1) * (kPlanckDeg + 1)];

// Planck edge value (as planck_edge) with g4 = x^4/(e^x - 1) in FP32
struct EdgeSI {
  double V;
  float g4;
  bool lower;
};

__device__ __forceinline__ EdgeSI planck_edge_si(double x) {
  EdgeSI r;
  const long long xb = __double_as_longlong(x);
  if (xb <= 0) { r.V = 0.0; r.g4 = 0.0f; r.lower = true; return r; }
  if (xb > kBits740) { r.V = 0.0; r.g4 = 0.0f; r.lower = false; return r; }
  const bool tail = xb >= kBits40;
  const int j = tail ? kPlanckRows : half_index(x);
  const double s = tail ? x : fma(x, 4.0, neg_odd(j));   // (x - (j/2 + 1/4)) 4
  const double* row = kPlanckTab + 2 * j * (kPlanckDeg + 1);
  const float* rowf = kG4TabF + j * (kPlanckDeg + 1);
  const float sf = d2f_trunc(s);
  double p1 = __ldg(row + 2 * kPlanckDeg);
  float p2 = __ldg(rowf + kPlanckDeg);
#pragma unroll
  for (int k = kPlanckDeg - 1; k >= 0; --k) {
    p1 = fma(p1, s, __ldg(row + 2 * k));
    p2 = fmaf(p2, sf, __ldg(rowf + k));
  }
  r.lower = j < kPlanckLowerRows;
  double m = 1.0;
  if (r.lower) m = x * x * x;
  else if (tail) m = exp(-x);
  r.V = m * p1;
  r.g4 = d2f_trunc(m) * p2;
  return r;
}

// Planck quantities of one cell at temperature T (> 0 or not) for the lane's
// groups g = sl + seg j of the cell's segment L (G: the cell's group count,
// 0 for a segment past the last cell): sigma_g and Phi_g in FP64, dPhi_g/dT
// in FP32.
// The same operations as cell_planck for sigma_g and Phi_g.  PART 1: Phi_g
// and dPhi_g/dT only; 2: sigma_g only (two warps of a cell share the work).
template <int NC, int PART = 0>
__device__ __forceinline__ void si_planck(const Dev& d, double T, double invT, double sT, double* sig,
                                          double* phi, float* dphi, const Lanes& L, int G) {
  const bool Tpos = __double_as_longlong(T) > 0;
  const double ac = d.a * d.c, T3 = T * T * T;
  const double acT3 = ac * T3, acT4 = acT3 * T;
  const float acT3f = d2f_trunc(acT3);
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const int g = L.sl + L.seg * j;
    if (d.grey) {
      sig[j] = cap_sigma(d, sT);
      phi[j] = Tpos ? acT4 : 0.0;
      dphi[j] = Tpos ? 4.0f * acT3f : 0.0f;
      continue;
    }
    if (PART == 2) {
      sig[j] = g < G ? sigma_group_at(d, sT, T, invT, g) : 1.0;
      continue;
    }
    EdgeSI lo;
    if (g <= G && Tpos) lo = planck_edge_si(d.nu_edges[g] * invT);
    else { lo.V = 0.0; lo.g4 = 0.0f; lo.lower = true; }
    EdgeSI hi;
    hi.V = __shfl_down_sync(0xffffffffu, lo.V, 1, L.seg);
    hi.g4 = __shfl_down_sync(0xffffffffu, lo.g4, 1, L.seg);
    hi.lower = __shfl_down_sync(0xffffffffu, (int)lo.lower, 1, L.seg) != 0;
    if (L.sl == L.seg - 1 && g + 1 <= G && Tpos) hi = planck_edge_si(d.nu_edges[g + 1] * invT);
    if (g < G) {
      sig[j] = PART == 1 ? 1.0 : sigma_group_at(d, sT, T, invT, g);
      if (Tpos) {
        double I;
        if (hi.lower) I = hi.V - lo.V;
        else if (!lo.lower) I = lo.V - hi.V;
        else I = (kPi4over15 - lo.V) - hi.V;
        const double b = k15overPi4 * I;
        phi[j] = acT4 * b;
        dphi[j] = acT3f * fmaf((float)k15overPi4, lo.g4 - hi.g4, 4.0f * d2f_trunc(b));
      } else {
        phi[j] = 0.0;
        dphi[j] = 0.0f;
      }
    } else {
      sig[j] = 1.0; phi[j] = 0.0; dphi[j] = 0.0f;
    }
  }
}

// C2(x)/dt of the face flux (as coef_g2_fast) with the row chosen on the integer pipes
__device__ __forceinline__ double coef_g2_si(double x, double ix) {
  const bool tail = __double_as_longlong(x) >= kBits40;
  const int j = tail ? kPlanckRows : half_index(x);
  const double s = tail ? ix : fma(x, 4.0, neg_odd(j));
  const double* row = kC2Tab + j * (kPlanckDeg + 1);
  double p = __ldg(row + kPlanckDeg);
#pragma unroll
  for (int k = kPlanckDeg - 1; k >= 0; --k) p = fma(p, s, __ldg(row + k));
  return j < kPlanckLowerRows ? p * x : p;
}

// F^eq on a face between relaxation times tl, tu and Phi values pl, pu (lower,
// upper side) along `axis`: C2 (v^2/3) (Phi_u - Phi_l)/h with the harmonic-mean
// face opacity, tau_f = (tl + tu)/2 (App. B).  A pure function of its
// operands, so the two cells of a face evaluate it bitwise alike.
__device__ __forceinline__ double feq_face_si(const Dev& d, double tl, double tu, double pl, double pu, int axis) {
  const double st = tl + tu;
  const double x = d.two_dt * rcp_nr(st);
  return coef_g2_si(x, st * d.inv_2dt) * (d.feq_k[axis] * (pu - pl));
}

// --------------------------------------------------------------------------
// FP32 warm start (mixed precision).  The same linearised Jacobi update in
// FP32 gives the FP64 iterates a starting temperature within about 1e-6 of
// the fixed point; the FP64 iterates then converge to si_tol exactly as from
// T^n, and the fixed point they reach is the FP64 one.  FP32 copies of the
// interpolant tables (filled once from the FP64 tables by k_init_pow):
static __device__ float kP1TabF[(kPlanckRows + 1) * (kPlanckDeg + 1)];
static __device__ float kC2TabF[(kPlanckRows + 1) * (kPlanckDeg + 1)];

struct EdgeF {
  float V, g4;
  bool lower;
};

__device__ __forceinline__ EdgeF planck_edge_f(float x) {
  EdgeF r;
  if (!(x > 0.0f)) { r.V = 0.0f; r.g4 = 0.0f; r.lower = true; return r; }
  if (x > 740.0f) { r.V = 0.0f; r.g4 = 0.0f; r.lower = false; return r; }
  const bool tail = x >= 40.0f;
  const int j = tail ? kPlanckRows : (int)(2.0f * x);
  const float s = tail ? x : fmaf(x, 4.0f, -(float)(2 * j + 1));
  const float* r1 = kP1TabF + j * (kPlanckDeg + 1);
  const float* r2 = kG4TabF + j * (kPlanckDeg + 1);
  float p1 = __ldg(r1 + kPlanckDeg), p2 = __ldg(r2 + kPlanckDeg);
#pragma unroll
  for (int k = kPlanckDeg - 1; k >= 0; --k) {
    p1 = fmaf(p1, s, __ldg(r1 + k));
    p2 = fmaf(p2, s, __ldg(r2 + k));
  }
  r.lower = j < kPlanckLowerRows;
  float m = 1.0f;
  if (r.lower) m = x * x * x;
  else if (tail) m = __expf(-x);
  r.V = m * p1;
  r.g4 = m * p2;
  return r;
}

// group opacity in FP32 (the three laws of sigma_group_at)
__device__ __forceinline__ float sigma_group_f(const Dev& d, float sT, float T, float invT, int g) {
  const float cap = d.capf;
  if (d.grey) return fminf(sT, cap);
  const float a = __ldg(d.nu_edges_f + g), b = __ldg(d.nu_edges_f + g + 1), m = 0.5f * (a + b);
  if (d.sig_law == 2) {
    const float A = fminf(1e7f, 1e9f * T * T);
    const float B = __fdividef(3e6f, 1.0f + 200.0f * T * sqrtf(T));
    const float C = __fdividef(4e4f, 1.0f + 8000.0f * T * T);
    const float* t = d.olson_nu_f + 9 * g;
    auto kap = [&](float nu, const float* f) {
      if (nu <= 0.008f) return A;
      if (nu <= 0.3f) return B * __ldg(f);
      return B * __ldg(f + 1) + C * __ldg(f + 2);
    };
    const float sa = fminf(sT * kap(a, t), cap), sm = fminf(sT * kap(m, t + 3), cap), sb = fminf(sT * kap(b, t + 6), cap);
    return (sa + 4.0f * sm + sb) * (1.0f / 6.0f);
  }
  const float* np = d.nu_pow_f + 3 * g;
  float fa = 1.0f, fm = 1.0f, fb = 1.0f;
  if (d.sig_law == 1) { fa = -expm1f(-a * invT); fm = -expm1f(-m * invT); fb = -expm1f(-b * invT); }
  const float sa = fminf(sT * __ldg(np) * fa, cap), sm = fminf(sT * __ldg(np + 1) * fm, cap);
  const float sb = fminf(sT * __ldg(np + 2) * fb, cap);
  return (sa + 4.0f * sm + sb) * (1.0f / 6.0f);
}

// sigma_g, Phi_g, dPhi_g/dT of one cell at T in FP32 (lanes as si_planck)
template <int NC>
__device__ __forceinline__ void si_planck_f(const Dev& d, float T, float invT, float sT, float* sig, float* phi,
                                            float* dphi, const Lanes& L, int G) {
  const bool Tpos = T > 0.0f;
  const float acT3 = d.acf * (T * T * T), acT4 = acT3 * T;
  const float k15 = (float)k15overPi4, kpi = (float)kPi4over15;
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const int g = L.sl + L.seg * j;
    if (d.grey) {
      sig[j] = fminf(sT, d.capf);
      phi[j] = Tpos ? acT4 : 0.0f;
      dphi[j] = Tpos ? 4.0f * acT3 : 0.0f;
      continue;
    }
    EdgeF lo;
    if (g <= G && Tpos) lo = planck_edge_f(__ldg(d.nu_edges_f + g) * invT);
    else { lo.V = 0.0f; lo.g4 = 0.0f; lo.lower = true; }
    EdgeF hi;
    hi.V = __shfl_down_sync(0xffffffffu, lo.V, 1, L.seg);
    hi.g4 = __shfl_down_sync(0xffffffffu, lo.g4, 1, L.seg);
    hi.lower = __shfl_down_sync(0xffffffffu, (int)lo.lower, 1, L.seg) != 0;
    if (L.sl == L.seg - 1 && g + 1 <= G && Tpos) hi = planck_edge_f(__ldg(d.nu_edges_f + g + 1) * invT);
    if (g < G) {
      sig[j] = sigma_group_f(d, sT, T, invT, g);
      if (Tpos) {
        float I;
        if (hi.lower) I = hi.V - lo.V;
        else if (!lo.lower) I = lo.V - hi.V;
        else I = (kpi - lo.V) - hi.V;
        const float b = k15 * I;
        phi[j] = acT4 * b;
        dphi[j] = acT3 * fmaf(k15, lo.g4 - hi.g4, 4.0f * b);
      } else {
        phi[j] = 0.0f;
        dphi[j] = 0.0f;
      }
    } else {
      sig[j] = 1.0f; phi[j] = 0.0f; dphi[j] = 0.0f;
    }
  }
}

// tau = 1/(rate sigma) and q = 1/(tau + dt) = A/(1 + dt A), A = rate sigma, in FP32
__device__ __forceinline__ void tau_and_q_f(const Dev& d, float sig, float* tau, float* q) {
  const float A = d.ratef * sig;
  *tau = __frcp_rn(A);
  *q = A * __frcp_rn(fmaf(d.dtf, A, 1.0f));
}

__device__ __forceinline__ float coef_g2_f(float x, float ix) {
  const bool tail = x >= 40.0f;
  const int j = tail ? kPlanckRows : (int)(2.0f * x);
  const float s = tail ? ix : fmaf(x, 4.0f, -(float)(2 * j + 1));
  const float* row = kC2TabF + j * (kPlanckDeg + 1);
  float p = __ldg(row + kPlanckDeg);
#pragma unroll
  for (int k = kPlanckDeg - 1; k >= 0; --k) p = fmaf(p, s, __ldg(row + k));
  return j < kPlanckLowerRows ? p * x : p;
}

// F^eq of a face in FP32 (feq_face_si)
__device__ __forceinline__ float feq_face_f(const Dev& d, float tl, float tu, float pl, float pu, int axis) {
  const float st = tl + tu;
  const float x = d.two_dtf * __frcp_rn(st);
  return coef_g2_f(x, st * d.inv_2dtf) * (d.feq_kf[axis] * (pu - pl));
}

}  // namespace ugkwp
