// ugkwp_api.cu -- host runtime behind the C ABI declared in include/ugkwp.h:
// workspace layout, problem upload, the per-step launch sequence of
// Algorithm 1, state and tally transfer, and the kernel-level entry points.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ugkwp.h"
#include "ugkwp_device.cuh"
#include "ugkwp_launch.h"

using ugkwp::Ctrl;
using ugkwp::Dev;

// (cell, group) pairs from which a mixed-precision source iteration starts
// with FP32 iterates by default (si_warm32 = 0)
constexpr long long kWarmMinPairs = 1ll << 17;

struct ugkwp_handle {
  Dev d;                        // member 0 (what the single-problem calls address)
  std::vector<Dev> members;     // every member's descriptor (host copy of the device table)
  ugkwp::Ens ens{};             // device view of the ensemble (used when M > 1)
  int M = 1;
  ugkwp::StreamShape shape;     // launch shape of the particle kernel
  ugkwp_problem p;     // scalars of member 0; host pointers cleared after init
  void* ws = nullptr;
  size_t ws_bytes = 0;
  char err[512];
  // one step captured as a CUDA graph, replayed by ugkwp_step
  cudaStream_t cap_stream = nullptr;
  // the wave flux runs beside the particle kernel in the captured step
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // the survivor sort runs beside the source iteration
  cudaStream_t sort_stream = nullptr;
  cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

thread_local char g_err[512] = "";

// Particles per tile of an ensemble's tile table: the FP32 kernel streams
// chunks of 32 x ppt particles per warp, the FP64 kernel tiles of block x ppt.
int ens_tile(const ugkwp_handle* h) {
  const int prec = h->members.empty() ? h->d.precision : h->members[0].precision;
  return prec == UGKWP_MIXED ? 32 * h->shape.ppt : h->shape.block * (h->shape.ppt >= 2 ? 2 : 1);
}

int fail(ugkwp_handle* h, int code, const char* msg) {
  char* dst = h ? h->err : g_err;
  snprintf(dst, 512, "%s", msg);
  return code;
}

int cuda_fail(ugkwp_handle* h, cudaError_t e, const char* where) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
  return fail(h, UGKWP_ERR_CUDA, buf);
}

#define CK(call, h)                                  \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

long long ny_of(const ugkwp_problem* p) { return p->dim >= 2 ? p->ny : 1; }
long long nz_of(const ugkwp_problem* p) { return p->dim == 3 ? p->nz : 1; }
long long ncell_of(const ugkwp_problem* p) { return (long long)p->nx * ny_of(p) * nz_of(p); }
long long nxface_of(const ugkwp_problem* p) { return (long long)(p->nx + 1) * ny_of(p) * nz_of(p); }
long long nyface_of(const ugkwp_problem* p) {
  return p->dim >= 2 ? (long long)p->nx * (ny_of(p) + 1) * nz_of(p) : 0;
}
long long nface_of(const ugkwp_problem* p) {
  return nxface_of(p) + nyface_of(p) + (p->dim == 3 ? (long long)p->nx * ny_of(p) * (nz_of(p) + 1) : 0);
}

int validate(const ugkwp_problem* p, ugkwp_handle* h) {
  if (!p) return fail(h, UGKWP_ERR_ARG, "problem is NULL");
  if (p->dim < 1 || p->dim > 3) return fail(h, UGKWP_ERR_ARG, "dim must be 1, 2 or 3");
  if (p->nx < 1 || (p->dim >= 2 && p->ny < 1) || (p->dim == 3 && p->nz < 1))
    return fail(h, UGKWP_ERR_ARG, "nx, ny, nz must be >= 1");
  if (ncell_of(p) * (long long)(p->G > 0 ? p->G : 1) >= (1ll << 31))
    return fail(h, UGKWP_ERR_ARG, "ncell*G must be < 2^31");
  if (p->G < 1 || p->G > ugkwp::kMaxG) return fail(h, UGKWP_ERR_ARG, "G must be in 1..64");
  if (p->grey && p->G != 1) return fail(h, UGKWP_ERR_ARG, "grey requires G == 1");
  if (!(p->dx > 0) || (p->dim >= 2 && !(p->dy > 0)) || (p->dim == 3 && !(p->dz > 0)))
    return fail(h, UGKWP_ERR_ARG, "dx, dy, dz must be > 0");
  if (!(p->dt > 0) || !(p->c > 0) || !(p->eps > 0) || !(p->a > 0))
    return fail(h, UGKWP_ERR_ARG, "dt, c, eps, a must be > 0");
  if (!p->sigma0 || !p->cv || !p->T0) return fail(h, UGKWP_ERR_ARG, "sigma0, cv, T0 are required");
  if (!p->grey && !p->nu_edges) return fail(h, UGKWP_ERR_ARG, "nu_edges required unless grey");
  for (int s = 0; s < 4; ++s) {
    if (p->bc[s] < 0 || p->bc[s] > 2) return fail(h, UGKWP_ERR_ARG, "bad boundary condition");
    if (p->dim == 1 && s < 2 && p->bc[s] == UGKWP_BC_BLACKBODY && !(p->bcT[s] > 0))
      return fail(h, UGKWP_ERR_ARG, "black-body side needs bcT > 0");
    if (p->dim >= 2 && p->bc[s] == UGKWP_BC_BLACKBODY)
      return fail(h, UGKWP_ERR_UNSUPPORTED, "black-body sides are 1D only in this build");
  }
  if (p->dim == 3)
    for (int s = 0; s < 2; ++s) {
      if (p->bc_z[s] < 0 || p->bc_z[s] > 2) return fail(h, UGKWP_ERR_ARG, "bad boundary condition");
      if (p->bc_z[s] == UGKWP_BC_BLACKBODY)
        return fail(h, UGKWP_ERR_UNSUPPORTED, "black-body sides are 1D only in this build");
    }
  if (p->wave_order != 1 && p->wave_order != 2) return fail(h, UGKWP_ERR_ARG, "wave_order must be 1 or 2");
  if (p->si_max_iters < 1) return fail(h, UGKWP_ERR_ARG, "si_max_iters must be >= 1");
  if (p->precision != UGKWP_FP64 && p->precision != UGKWP_MIXED)
    return fail(h, UGKWP_ERR_ARG, "precision must be UGKWP_FP64 or UGKWP_MIXED");
  if (p->particle_capacity < 1) return fail(h, UGKWP_ERR_ARG, "particle_capacity must be >= 1");
  if (p->si_warm32 < -1 || p->si_warm32 > 1) return fail(h, UGKWP_ERR_ARG, "si_warm32 must be -1, 0 or 1");
  if (p->si_pair != 0 && p->si_pair != -1) return fail(h, UGKWP_ERR_ARG, "si_pair must be 0 or -1");
  if (!(p->tau_num_C >= 0.0)) return fail(h, UGKWP_ERR_ARG, "tau_num_C must be >= 0");
  if (p->sig_law < 0 || p->sig_law > 2) return fail(h, UGKWP_ERR_ARG, "sig_law must be 0, 1 or 2");
  if (p->sig_law == 2 && p->grey) return fail(h, UGKWP_ERR_ARG, "sig_law 2 (Olson foam) needs groups (grey = 0)");
  if (p->cv_law != 0 && p->cv_law != 1) return fail(h, UGKWP_ERR_ARG, "cv_law must be 0 or 1");
  if (p->cv_law == 1 && !(p->cv_chi > 0.0)) return fail(h, UGKWP_ERR_ARG, "cv_law 1 needs cv_chi > 0");
  if (p->method != UGKWP_METHOD_UGKWP && p->method != UGKWP_METHOD_UGKP)
    return fail(h, UGKWP_ERR_ARG, "method must be 0 (UGKWP) or 1 (UGKP)");
  const long long nbins = (ncell_of(p) + 4) * p->G;
  if (nbins >= (1ll << 24)) return fail(h, UGKWP_ERR_ARG, "(ncell+4)*G must be < 2^24 (particle id layout)");
  return UGKWP_OK;
}

// Bump allocator over the workspace; with base == nullptr it only sizes.
struct Carver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(long long n) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += sizeof(T) * (size_t)(n > 0 ? n : 0);
    return p;
  }
};

void carve(const ugkwp_problem* p, Carver& cv, Dev& d, double** src_T_tmp) {
  const long long nc = ncell_of(p), G = p->G, ncg = nc * G, nb = (nc + 4) * G;
  const long long nf = nface_of(p), P = p->particle_capacity;
  d.nu_edges = cv.take<double>(G + 1);
  d.nu_edges_f = cv.take<float>(G + 1);
  d.nu_pow = cv.take<double>(3 * G);
  d.sigma0 = cv.take<double>(nc);
  d.cv = cv.take<double>(nc);
  d.src = p->src_T ? cv.take<double>(ncg) : nullptr;
  d.ghost_phi = cv.take<double>(6 * G);
  d.ghost_sig = cv.take<double>(6 * G);
  d.T = cv.take<double>(nc);
  d.rho = cv.take<double>(ncg);
  d.rho_h = cv.take<double>(ncg);
  d.rho_p = cv.take<double>(ncg);
  d.sigT = cv.take<double>(ncg);
  d.sT = cv.take<double>(nc);
  d.sTinv = cv.take<double>(nc);
  d.N = cv.take<uint32_t>(nb);
  d.off = cv.take<uint32_t>(nb + 1);
  d.part = cv.take<uint32_t>(ugkwp::scan_parts(nb) + 1);
  d.sort_cnt = cv.take<uint32_t>(nb);
  d.sort_off = cv.take<uint32_t>(nb + 1);
  d.sort_part = cv.take<uint32_t>(ugkwp::scan_parts(nb) + 1);
  d.omega = cv.take<double>(nb);
  d.xnum = cv.take<double>(nb);
  d.e_eff = cv.take<double>(nb);
  d.khat = cv.take<double>(nb);
  d.W = cv.take<double>(ncg);
  d.E_surv = cv.take<double>(ncg);
  d.Wq = cv.take<unsigned long long>(2 * ncg);
  d.Esq = cv.take<unsigned long long>(2 * ncg);
  d.esc = cv.take<double>(6 * G);
  d.inflow = cv.take<double>(6 * G);
  d.Fwave = cv.take<double>(nf * G);
  d.Feq = cv.take<double>(nf * G);
  d.R = cv.take<double>(ncg);
  d.wscale = cv.take<double>(ncg);
  d.Tk[0] = cv.take<double>(nc);
  d.Tk[1] = cv.take<double>(nc);
  d.tauk[0] = cv.take<double>(ncg);
  d.tauk[1] = cv.take<double>(ncg);
  d.qk = cv.take<double>(ncg);
  d.phik[0] = cv.take<double>(ncg);
  d.phik[1] = cv.take<double>(ncg);
  d.dphik = cv.take<float>(ncg);
  d.ctrl = cv.take<Ctrl>(1);
  *src_T_tmp = d.R;   // scratch during init only
  const bool mixed = p->precision == UGKWP_MIXED;
  d.olson_c = p->sig_law == 2 ? cv.take<double>(3 * nc) : nullptr;
  d.olson_nu = p->sig_law == 2 ? cv.take<double>(9 * G) : nullptr;
  d.olson_cf = (p->sig_law == 2 && mixed) ? cv.take<float>(3 * nc) : nullptr;
  d.sT_f = mixed ? cv.take<float>(nc) : nullptr;
  d.sTinv_f = mixed ? cv.take<float>(nc) : nullptr;
  d.invT_f = mixed ? cv.take<float>(nc) : nullptr;
  d.omega_f = mixed ? cv.take<float>(nb) : nullptr;
  d.khat_f = mixed ? cv.take<float>(nb) : nullptr;
  for (int k = 0; k < 2; ++k) {
    d.Tk_f[k] = mixed ? cv.take<float>(nc) : nullptr;
    d.tau_f[k] = mixed ? cv.take<float>(ncg) : nullptr;
    d.phi_f[k] = mixed ? cv.take<float>(ncg) : nullptr;
  }
  d.q_f = mixed ? cv.take<float>(ncg) : nullptr;
  d.R_f = mixed ? cv.take<float>(ncg) : nullptr;
  d.Feq_f = (mixed && p->dim >= 2) ? cv.take<float>(nf * G) : nullptr;
  d.nu_pow_f = mixed ? cv.take<float>(3 * G) : nullptr;
  d.olson_nu_f = (mixed && p->sig_law == 2) ? cv.take<float>(9 * G) : nullptr;
  d.particles_begin = nullptr;
  for (int b = 0; b < 2; ++b) {
    if (mixed) {
      d.fx[b] = cv.take<float>(P);
      if (!b) d.particles_begin = d.fx[0];
      d.fox[b] = cv.take<float>(P);
      d.fy[b] = p->dim >= 2 ? cv.take<float>(P) : nullptr;
      d.foy[b] = p->dim >= 2 ? cv.take<float>(P) : nullptr;
      d.fz[b] = p->dim == 3 ? cv.take<float>(P) : nullptr;
      d.foz[b] = p->dim == 3 ? cv.take<float>(P) : nullptr;
      d.fnu[b] = cv.take<float>(P);
      d.fw[b] = cv.take<float>(P);
      d.px[b] = d.pox[b] = d.py[b] = d.poy[b] = d.pz[b] = d.poz[b] = d.pnu[b] = d.pw[b] = nullptr;
    } else {
      d.px[b] = cv.take<double>(P);
      if (!b) d.particles_begin = d.px[0];
      d.pox[b] = cv.take<double>(P);
      d.py[b] = p->dim >= 2 ? cv.take<double>(P) : nullptr;
      d.poy[b] = p->dim >= 2 ? cv.take<double>(P) : nullptr;
      d.pz[b] = p->dim == 3 ? cv.take<double>(P) : nullptr;
      d.poz[b] = p->dim == 3 ? cv.take<double>(P) : nullptr;
      d.pnu[b] = cv.take<double>(P);
      d.pw[b] = cv.take<double>(P);
      d.fx[b] = d.fox[b] = d.fy[b] = d.foy[b] = d.fz[b] = d.foz[b] = d.fnu[b] = d.fw[b] = nullptr;
    }
    d.pid[b] = cv.take<unsigned long long>(P);
    d.pkey[b] = cv.take<uint32_t>(P);
  }
  // tail pad: the particle kernel's bulk copies round a tile's survivor count
  // up to whole 16-byte chunks and may read up to 12 bytes past an array
  cv.take<char>(256);
}

void fill_scalars(const ugkwp_problem* p, Dev& d) {
  d.dim = p->dim;
  d.nx = p->nx;
  d.ny = (int)ny_of(p);
  d.nz = (int)nz_of(p);
  d.nyface = (int)nyface_of(p);
  d.G = p->G;
  d.ncell = (int)ncell_of(p);
  d.nbins = (d.ncell + 4) * p->G;
  d.nface = (int)nface_of(p);
  d.nxface = (int)nxface_of(p);
  d.grey = p->grey;
  d.wave_order = p->wave_order;
  d.si_max_iters = p->si_max_iters;
  d.precision = p->precision;
  for (int s = 0; s < 4; ++s) { d.bc[s] = p->bc[s]; d.bcT[s] = p->bcT[s]; }
  for (int s = 0; s < 2; ++s) {
    d.bc[4 + s] = p->dim == 3 ? p->bc_z[s] : ugkwp::BC_REFLECT;
    d.bcT[4 + s] = p->dim == 3 ? p->bcT_z[s] : 0.0;
  }
  d.dx = p->dx;
  d.dy = p->dim >= 2 ? p->dy : 1.0;
  d.dz = p->dim == 3 ? p->dz : 1.0;
  d.vol = p->dx * (p->dim >= 2 ? p->dy : 1.0) * (p->dim == 3 ? p->dz : 1.0);
  if (p->dim == 1) { d.area[0] = d.area[1] = d.area[2] = 1.0; }
  else if (p->dim == 2) { d.area[0] = d.dy; d.area[1] = d.dx; d.area[2] = 1.0; }
  else { d.area[0] = d.dy * d.dz; d.area[1] = d.dx * d.dz; d.area[2] = d.dx * d.dy; }
  d.sig_p = p->grey ? 0.0 : p->sig_p;
  d.sig_q = p->sig_law == 2 ? 0.0 : p->sig_q;   // the foam law has no T^q factor
  d.sig_cap = p->sig_cap;
  d.a = p->a;
  d.c = p->c;
  d.eps = p->eps;
  d.dt = p->dt;
  d.inv_2dt = 0.5 / p->dt;
  d.two_dt = 2.0 * p->dt;
  d.v = p->c / p->eps;
  d.inv_dx = 1.0 / d.dx;
  d.inv_dy = 1.0 / d.dy;
  d.inv_dz = 1.0 / d.dz;
  d.inv_c = 1.0 / p->c;
  {
    const double inv_h[3] = {d.inv_dx, d.inv_dy, d.inv_dz};
    for (int a = 0; a < 3; ++a) {
      d.feq_k[a] = p->dt * (d.v * d.v / 3.0) * inv_h[a];
      d.dt_h[a] = p->dt * inv_h[a];
    }
  }
  d.inv_vol = 1.0 / d.vol;
  d.rate_f = p->c / (p->eps * p->eps);
  d.omega_ref = p->omega_ref;
  d.si_tol = p->si_tol;
  d.src_on = p->src_on;
  d.tau_num_C = p->tau_num_C;
  d.sig_law = p->sig_law;
  d.cv_law = p->cv_law;
  d.split_literal = p->split_literal ? 1 : 0;
  d.cv_chi = p->cv_chi;
  d.src_t_end = p->src_t_end;
  d.method = p->method;
  d.key0 = (uint32_t)p->seed;
  d.key1 = (uint32_t)(p->seed >> 32) ^ p->instance;
  d.pk = ugkwp::philox_keys(d.key0, d.key1);
  d.capacity = p->particle_capacity;
  // fixed-point quantum of the tallies: the power of two just below omega_ref 2^-48
  d.tq_shift = 48 - (p->omega_ref > 0.0 ? std::ilogb(p->omega_ref) : 0);
  d.tq = std::ldexp(1.0, -d.tq_shift);
  d.tq_inv = std::ldexp(1.0, d.tq_shift);
  // FP32 copies for the mixed-precision particle kernel
  d.dxf = (float)d.dx;
  d.dyf = (float)d.dy;
  d.dzf = (float)d.dz;
  d.vf = (float)d.v;
  d.dtf = (float)d.dt;
  d.inv_rate_f = (float)(p->eps * p->eps / p->c);
  d.capf = p->sig_cap > 0.0 ? (float)p->sig_cap : INFINITY;
  d.spf = (float)d.sig_p;
  d.inv_cap = p->sig_cap > 0.0 ? 1.0 / p->sig_cap : 0.0;
  d.inv_capf = (float)d.inv_cap;
  d.two_dtf = (float)d.two_dt;
  d.inv_2dtf = (float)d.inv_2dt;
  d.ratef = (float)d.rate_f;
  d.acf = (float)(d.a * d.c);
  d.inv_cf = (float)d.inv_c;
  for (int a = 0; a < 3; ++a) d.feq_kf[a] = (float)d.feq_k[a];
  d.si_warm = 0;   // set once the ensemble's size is known
  d.pair_si = p->si_pair == -1 ? 0 : 1;
  // bin and cell indices below 2^24 divide by G and nx through an FP32 reciprocal
  d.fastdiv = (long long)d.ncell * d.G < (1ll << 24) ? 1 : 0;
  d.invG_f = 1.0f / (float)d.G;
  d.inv_nx_f = 1.0f / (float)d.nx;
  d.rec = nullptr;
  d.rec_cap = 0;
  d.tape = nullptr;
  d.tape_cap = 0;
}

}  // namespace

void ugkwp::set_global_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

extern "C" {

}  // extern "C"

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t member_bytes(const ugkwp_problem* p) {
  Carver cv{nullptr};
  Dev d{};
  double* tmp;
  carve(p, cv, d, &tmp);
  return align256(cv.off);
}

size_t table_bytes(int M) {
  return align256(sizeof(Dev) * (size_t)M) + 5 * align256(sizeof(int) * (size_t)(M + 1)) + 256;
}

int validate_members(const ugkwp_problem* probs, int M) {
  if (!probs || M < 1) return fail(nullptr, UGKWP_ERR_ARG, "need at least one problem");
  if (M > ugkwp::kMaxEnsemble) return fail(nullptr, UGKWP_ERR_ARG, "too many ensemble members (max 4096)");
  for (int m = 0; m < M; ++m) {
    int st = validate(&probs[m], nullptr);
    if (st) return st;
    if (probs[m].dim != probs[0].dim || probs[m].precision != probs[0].precision)
      return fail(nullptr, UGKWP_ERR_ARG, "ensemble members must share dim and precision");
    if (probs[m].si_max_iters != probs[0].si_max_iters)
      return fail(nullptr, UGKWP_ERR_ARG, "ensemble members must share si_max_iters");
    if (M > 1 && probs[m].dim == 3)
      return fail(nullptr, UGKWP_ERR_UNSUPPORTED, "ensembles are built for 1D and 2D members");
  }
  return UGKWP_OK;
}

// Copy member m's problem into its workspace region and set its initial state.
cudaError_t init_member(const ugkwp_problem* p, char* base, Dev& d, cudaStream_t s, const char** where) {
  Carver cv{base};
  d = Dev{};
  double* src_T_tmp = nullptr;
  carve(p, cv, d, &src_T_tmp);
  fill_scalars(p, d);
  const long long nc = d.ncell, G = d.G, ncg = nc * G;
  // zero everything but the particle buffers
  const size_t head = (size_t)((char*)d.particles_begin - base);
  cudaError_t e;
  *where = "memset";
  if ((e = cudaMemsetAsync(base, 0, head, s))) return e;
  std::vector<double> edges(G + 1);
  if (p->grey) { edges[0] = 0.0; edges[1] = 1.0; }
  else for (int g = 0; g <= G; ++g) edges[g] = p->nu_edges[g];
  *where = "problem upload";
  if ((e = cudaMemcpyAsync((void*)d.nu_edges, edges.data(), sizeof(double) * (G + 1), cudaMemcpyHostToDevice, s))) return e;
  if ((e = cudaMemcpyAsync((void*)d.sigma0, p->sigma0, sizeof(double) * nc, cudaMemcpyHostToDevice, s))) return e;
  if ((e = cudaMemcpyAsync((void*)d.cv, p->cv, sizeof(double) * nc, cudaMemcpyHostToDevice, s))) return e;
  if ((e = cudaMemcpyAsync(d.T, p->T0, sizeof(double) * nc, cudaMemcpyHostToDevice, s))) return e;
  if (p->rho0) {
    if ((e = cudaMemcpyAsync(d.rho, p->rho0, sizeof(double) * ncg, cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(d.rho_h, p->rho0, sizeof(double) * ncg, cudaMemcpyHostToDevice, s))) return e;
  }
  if (p->src_T)
    if ((e = cudaMemcpyAsync(src_T_tmp, p->src_T, sizeof(double) * nc, cudaMemcpyHostToDevice, s))) return e;
  double* src_amp_tmp = (p->src_T && p->src_amp) ? d.W : nullptr;   // scratch during init only
  if (src_amp_tmp)
    if ((e = cudaMemcpyAsync(src_amp_tmp, p->src_amp, sizeof(double) * nc, cudaMemcpyHostToDevice, s))) return e;
  *where = "init kernel";
  if ((e = ugkwp::launch_init_tables(d, p->src_T ? src_T_tmp : nullptr, src_amp_tmp, p->rho0 ? 0 : 1, s))) return e;
  // the source temperatures sat in R; wait before the next member's upload reuses host data
  *where = "init sync";
  return cudaStreamSynchronize(s);
}

}  // namespace

extern "C" {

int ugkwp_workspace_size_ensemble(const ugkwp_problem* probs, int n, size_t* bytes) {
  int st = validate_members(probs, n);
  if (st) return st;
  if (!bytes) return fail(nullptr, UGKWP_ERR_ARG, "bytes is NULL");
  size_t tot = 0;
  for (int m = 0; m < n; ++m) tot += member_bytes(&probs[m]);
  *bytes = tot + table_bytes(n) + 256;
  return UGKWP_OK;
}

int ugkwp_workspace_size(const ugkwp_problem* p, size_t* bytes) {
  return ugkwp_workspace_size_ensemble(p, 1, bytes);
}

int ugkwp_init_ensemble(const ugkwp_problem* probs, int n, void* d_workspace, size_t bytes, void* stream,
                        ugkwp_handle** out) {
  if (!out) return fail(nullptr, UGKWP_ERR_ARG, "out is NULL");
  *out = nullptr;
  size_t need = 0;
  int st = ugkwp_workspace_size_ensemble(probs, n, &need);
  if (st) return st;
  if (!d_workspace || bytes < need)
    return fail(nullptr, UGKWP_ERR_WORKSPACE, "workspace missing or smaller than the required size");
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256)
    return fail(nullptr, UGKWP_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  ugkwp_handle* h = new (std::nothrow) ugkwp_handle;
  if (!h) return fail(nullptr, UGKWP_ERR_ARG, "out of host memory");
  h->err[0] = 0;
  h->p = probs[0];
  h->M = n;
  h->ws = d_workspace;
  h->ws_bytes = bytes;
  h->members.resize(n);
  cudaStream_t s = (cudaStream_t)stream;
  auto bad = [&](cudaError_t e, const char* w) {
    int r = cuda_fail(h, e, w);
    snprintf(g_err, 512, "%s", h->err);
    delete h;
    return r;
  };
  char* base = static_cast<char*>(d_workspace);
  std::vector<int> cell0(n + 1, 0), bin0(n + 1, 0), fg0(n + 1, 0), item0(n + 1, 0);
  long long max_bins = 0;
  int max_G = 0;
  for (int m = 0; m < n; ++m) {
    const char* where = "";
    cudaError_t e = init_member(&probs[m], base, h->members[m], s, &where);
    if (e) return bad(e, where);
    base += member_bytes(&probs[m]);
    const Dev& d = h->members[m];
    cell0[m + 1] = cell0[m] + d.ncell;
    bin0[m + 1] = bin0[m] + d.nbins;
    fg0[m + 1] = fg0[m] + d.nface * d.G;
    const int cpw = 32 / ugkwp::seg_width(d.G);
    item0[m + 1] = item0[m] + (d.ncell + cpw - 1) / cpw;
    if (d.nbins > max_bins) max_bins = d.nbins;
    if (d.G > max_G) max_G = d.G;
  }
  // FP32 warm start of the source iteration: mixed precision, and on by
  // default where the iteration has enough (cell, group) pairs to be bound by
  // the FP64 pipe (about 2^17: 24 per lane of every SM); a small latency-bound
  // iteration gains nothing from it
  {
    long long ncg = 0;
    for (int m = 0; m < n; ++m) ncg += (long long)h->members[m].ncell * h->members[m].G;
    const int want = probs[0].si_warm32;
    const bool on = probs[0].precision == UGKWP_MIXED && (want == 1 || (want == 0 && ncg >= kWarmMinPairs));
    for (int m = 0; m < n; ++m) h->members[m].si_warm = on ? 1 : 0;
  }
  // device tables
  Carver cv{base};
  Dev* d_devs = cv.take<Dev>(n);
  int* d_cell0 = cv.take<int>(n + 1);
  int* d_bin0 = cv.take<int>(n + 1);
  int* d_fg0 = cv.take<int>(n + 1);
  int* d_item0 = cv.take<int>(n + 1);
  int* d_tile0 = cv.take<int>(n + 1);
  unsigned int* d_bar = cv.take<unsigned int>(4);   // barrier arrivals, then the tile counter (8-byte aligned)
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_devs, h->members.data(), sizeof(Dev) * n, cudaMemcpyHostToDevice, s))) return bad(e, "member table");
  if ((e = cudaMemcpyAsync(d_cell0, cell0.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s))) return bad(e, "tables");
  if ((e = cudaMemcpyAsync(d_bin0, bin0.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s))) return bad(e, "tables");
  if ((e = cudaMemcpyAsync(d_fg0, fg0.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s))) return bad(e, "tables");
  if ((e = cudaMemcpyAsync(d_item0, item0.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s))) return bad(e, "tables");
  if ((e = cudaMemsetAsync(d_tile0, 0, sizeof(int) * (n + 1), s))) return bad(e, "tables");
  if ((e = cudaMemsetAsync(d_bar, 0, 4 * sizeof(unsigned int), s))) return bad(e, "tables");
  if ((e = cudaStreamSynchronize(s))) return bad(e, "init sync");
  ugkwp::Ens& E = h->ens;
  E.M = n;
  E.devs = d_devs;
  E.cell0 = d_cell0;
  E.bin0 = d_bin0;
  E.fg0 = d_fg0;
  E.item0 = d_item0;
  E.tile0 = d_tile0;
  E.bar = d_bar;
  E.tile_next = reinterpret_cast<unsigned long long*>(d_bar + 2);
  E.total_bins = bin0[n];
  E.total_fg = fg0[n];
  E.total_cells = cell0[n];
  E.total_items = item0[n];
  E.max_parts = ugkwp::scan_parts(max_bins);
  E.max_G = max_G;
  E.tile = ens_tile(h);
  h->d = h->members[0];
  h->p.nu_edges = h->p.sigma0 = h->p.cv = h->p.T0 = h->p.rho0 = h->p.src_T = h->p.src_amp = nullptr;
  *out = h;
  return UGKWP_OK;
}

int ugkwp_init(const ugkwp_problem* p, void* d_workspace, size_t bytes, void* stream,
               ugkwp_handle** out) {
  return ugkwp_init_ensemble(p, 1, d_workspace, bytes, stream, out);
}

}  // extern "C"

namespace {

// Side branches of a captured step: the wave flux (it needs only the birth
// kernel's sampled fractions) beside the particle kernel, and the survivor
// sort (it needs only the particle kernel's slots and counts) beside the
// source iteration, which touches no particle.
struct Branches {
  cudaStream_t side = nullptr, sort = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, fork2 = nullptr, join2 = nullptr;
};

// One step (in stream order without branches).
cudaError_t enqueue_step_dev(const Dev& d, const ugkwp::Ens* e, const ugkwp::StreamShape& sh,
                             cudaStream_t s, const Branches& b = Branches()) {
  cudaError_t r = ugkwp::launch_birth_and_scan(d, e, s);
  if (b.side) {
    // beside the particle kernel: the wave flux
    if (!r) r = cudaEventRecord(b.fork, s);
    if (!r) r = cudaStreamWaitEvent(b.side, b.fork, 0);
    if (!r) r = ugkwp::launch_wave(d, e, b.side);
    if (!r) r = cudaEventRecord(b.join, b.side);
    if (!r) r = ugkwp::launch_stream(d, e, sh, s);
    if (!r) r = cudaStreamWaitEvent(s, b.join, 0);
  } else {
    if (!r) r = ugkwp::launch_wave(d, e, s);
    if (!r) r = ugkwp::launch_stream(d, e, sh, s);
  }
  if (b.sort) {
    if (!r) r = cudaEventRecord(b.fork2, s);
    if (!r) r = cudaStreamWaitEvent(b.sort, b.fork2, 0);
    if (!r) r = ugkwp::launch_sort(d, e, b.sort);
    if (!r) r = cudaEventRecord(b.join2, b.sort);
    if (!r) r = ugkwp::launch_si(d, e, s);
    if (!r) r = cudaStreamWaitEvent(s, b.join2, 0);
  } else {
    if (!r) r = ugkwp::launch_si(d, e, s);
    if (!r) r = ugkwp::launch_sort(d, e, s);
  }
  if (!r) r = ugkwp::launch_end_step(d, e, s);
  return r;
}

void drop_graph(ugkwp_handle* h) {
  if (h->exec) cudaGraphExecDestroy(h->exec);
  h->exec = nullptr;
}

// Capture one step (every kernel reads the step's counts from the device
// control block, so the same graph serves every step).
int capture_one(ugkwp_handle* h, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), h);
  Branches b;
  b.side = h->side_stream; b.fork = h->ev_fork; b.join = h->ev_join;
  b.sort = h->sort_stream; b.fork2 = h->ev_fork2; b.join2 = h->ev_join2;
  cudaError_t e = enqueue_step_dev(h->d, h->M > 1 ? &h->ens : nullptr, h->shape, h->cap_stream, b);
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
  if (e) { if (g) cudaGraphDestroy(g); return cuda_fail(h, e, "capturing the step"); }
  if (e2) return cuda_fail(h, e2, "end of capture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e) { *out = nullptr; return cuda_fail(h, e, "instantiating the step graph"); }
  return UGKWP_OK;
}

int capture_step(ugkwp_handle* h) {
  if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), h);
  if (!h->side_stream) {
    CK(cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking), h);
    CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), h);
    CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming), h);
    CK(cudaStreamCreateWithFlags(&h->sort_stream, cudaStreamNonBlocking), h);
    CK(cudaEventCreateWithFlags(&h->ev_fork2, cudaEventDisableTiming), h);
    CK(cudaEventCreateWithFlags(&h->ev_join2, cudaEventDisableTiming), h);
  }
  int st = capture_one(h, &h->exec);
  if (st) drop_graph(h);
  return st;
}

}  // namespace

extern "C" {

int ugkwp_step(ugkwp_handle* h, int nsteps, void* stream) {
  if (!h) return fail(nullptr, UGKWP_ERR_ARG, "handle is NULL");
  if (nsteps < 0) return fail(h, UGKWP_ERR_ARG, "nsteps < 0");
  cudaStream_t s = (cudaStream_t)stream;
  if (!h->exec) {
    int st = capture_step(h);
    if (st) return st;
  }
  for (int n = 0; n < nsteps; ++n) CK(cudaGraphLaunch(h->exec, s), h);
  return UGKWP_OK;
}

int ugkwp_step_timed(ugkwp_handle* h, void* stream, float* phase_ms) {
  if (!h || !phase_ms) return fail(h, UGKWP_ERR_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t ev[6];
  for (int i = 0; i < 6; ++i) CK(cudaEventCreate(&ev[i]), h);
  int rc = UGKWP_OK;
  const ugkwp::Ens* en = h->M > 1 ? &h->ens : nullptr;
  cudaError_t e = cudaEventRecord(ev[0], s);
  if (!e) e = ugkwp::launch_birth_and_scan(h->d, en, s);
  if (!e) e = cudaEventRecord(ev[1], s);
  if (!e) e = ugkwp::launch_wave(h->d, en, s);
  if (!e) e = cudaEventRecord(ev[2], s);
  if (!e) e = ugkwp::launch_stream(h->d, en, h->shape, s);
  if (!e) e = cudaEventRecord(ev[3], s);
  if (!e) e = ugkwp::launch_si(h->d, en, s);
  if (!e) e = cudaEventRecord(ev[4], s);
  if (!e) e = ugkwp::launch_sort(h->d, en, s);
  if (!e) e = ugkwp::launch_end_step(h->d, en, s);
  if (!e) e = cudaEventRecord(ev[5], s);
  if (!e) e = cudaEventSynchronize(ev[5]);
  if (!e) {
    cudaEventElapsedTime(&phase_ms[0], ev[0], ev[5]);
    for (int i = 1; i < 6; ++i) cudaEventElapsedTime(&phase_ms[i], ev[i - 1], ev[i]);
  } else {
    rc = cuda_fail(h, e, "timed step");
  }
  for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
  return rc;
}

int ugkwp_tallies_member(ugkwp_handle* h, int m, ugkwp_tally_report* out, void* stream) {
  if (!h || !out) return fail(h, UGKWP_ERR_ARG, "NULL argument");
  if (m < 0 || m >= h->M) return fail(h, UGKWP_ERR_ARG, "member index out of range");
  cudaStream_t s = (cudaStream_t)stream;
  const Dev& d = h->members[m];
  Ctrl c;
  CK(cudaMemcpyAsync(&c, d.ctrl, sizeof c, cudaMemcpyDeviceToHost, s), h);
  CK(cudaStreamSynchronize(s), h);
  out->T = d.T; out->rho = d.rho; out->rho_h = d.rho_h; out->rho_p = d.rho_p; out->W = d.W;
  out->Fwave = d.Fwave; out->Feq = d.Feq; out->esc = d.esc; out->inflow = d.inflow;
  out->step = (int64_t)c.step;
  out->n_particles = (int64_t)c.n_part[c.cur];
  out->n_in = (int64_t)c.n_in; out->n_born = (int64_t)c.n_born; out->n_survived = (int64_t)c.n_survived;
  out->n_absorbed = (int64_t)c.n_absorbed; out->n_escaped = (int64_t)c.n_escaped;
  out->n_removed = (int64_t)c.n_removed; out->n_segments = (int64_t)c.n_segments;
  out->si_iters = (int32_t)c.si_iters;
  out->n_scaled_bins = (int64_t)c.n_scaled_bins;
  out->si_iters32 = (int32_t)c.si_iters32;
  out->status_bits = c.status;
  out->E_rad0 = c.E_rad0; out->E_mat0 = c.E_mat0; out->E_rad1 = c.E_rad1; out->E_mat1 = c.E_mat1;
  out->bnd_in_macro = c.bnd_in_macro; out->bnd_in_part = c.bnd_in_part;
  out->bnd_out_part = c.bnd_out_part; out->src_in = c.src_in;
  return UGKWP_OK;
}

int ugkwp_tallies(ugkwp_handle* h, ugkwp_tally_report* out, void* stream) {
  return ugkwp_tallies_member(h, 0, out, stream);
}

int ugkwp_get_state_member(ugkwp_handle* h, int member, double* T, double* rho, double* rho_h,
                           double* rho_p, ugkwp_particles_host* parts, int64_t cap, int64_t* n,
                           void* stream) {
  if (!h) return fail(nullptr, UGKWP_ERR_ARG, "handle is NULL");
  if (member < 0 || member >= h->M) return fail(h, UGKWP_ERR_ARG, "member index out of range");
  cudaStream_t s = (cudaStream_t)stream;
  const Dev& d = h->members[member];
  const size_t ncg = (size_t)d.ncell * d.G;
  Ctrl c;
  CK(cudaMemcpyAsync(&c, d.ctrl, sizeof c, cudaMemcpyDeviceToHost, s), h);
  CK(cudaStreamSynchronize(s), h);
  if (T) CK(cudaMemcpyAsync(T, d.T, sizeof(double) * d.ncell, cudaMemcpyDeviceToHost, s), h);
  if (rho) CK(cudaMemcpyAsync(rho, d.rho, sizeof(double) * ncg, cudaMemcpyDeviceToHost, s), h);
  if (rho_h) CK(cudaMemcpyAsync(rho_h, d.rho_h, sizeof(double) * ncg, cudaMemcpyDeviceToHost, s), h);
  if (rho_p) CK(cudaMemcpyAsync(rho_p, d.rho_p, sizeof(double) * ncg, cudaMemcpyDeviceToHost, s), h);
  const long long np = (long long)c.n_part[c.cur];
  if (n) *n = np;
  if (parts && cap > 0) {
    const long long m = np < cap ? np : cap;
    const unsigned b = c.cur;
    std::vector<uint32_t> key(m > 0 ? m : 1);
    const bool mixed = d.precision == UGKWP_MIXED;
    if (d.dim == 3 && (!parts->z || !parts->oz)) return fail(h, UGKWP_ERR_ARG, "3D particles need z and oz");
    std::vector<float> fb(mixed && m > 0 ? (size_t)m * 8 : 1);
    if (m > 0 && !mixed) {
      CK(cudaMemcpyAsync(parts->x, d.px[b], sizeof(double) * m, cudaMemcpyDeviceToHost, s), h);
      CK(cudaMemcpyAsync(parts->ox, d.pox[b], sizeof(double) * m, cudaMemcpyDeviceToHost, s), h);
      CK(cudaMemcpyAsync(parts->nu, d.pnu[b], sizeof(double) * m, cudaMemcpyDeviceToHost, s), h);
      CK(cudaMemcpyAsync(parts->w, d.pw[b], sizeof(double) * m, cudaMemcpyDeviceToHost, s), h);
      if (d.dim >= 2) {
        CK(cudaMemcpyAsync(parts->y, d.py[b], sizeof(double) * m, cudaMemcpyDeviceToHost, s), h);
        CK(cudaMemcpyAsync(parts->oy, d.poy[b], sizeof(double) * m, cudaMemcpyDeviceToHost, s), h);
      }
      if (d.dim == 3) {
        CK(cudaMemcpyAsync(parts->z, d.pz[b], sizeof(double) * m, cudaMemcpyDeviceToHost, s), h);
        CK(cudaMemcpyAsync(parts->oz, d.poz[b], sizeof(double) * m, cudaMemcpyDeviceToHost, s), h);
      }
    } else if (m > 0) {
      float* f = fb.data();
      CK(cudaMemcpyAsync(f, d.fx[b], sizeof(float) * m, cudaMemcpyDeviceToHost, s), h);
      CK(cudaMemcpyAsync(f + m, d.fox[b], sizeof(float) * m, cudaMemcpyDeviceToHost, s), h);
      CK(cudaMemcpyAsync(f + 2 * m, d.fnu[b], sizeof(float) * m, cudaMemcpyDeviceToHost, s), h);
      CK(cudaMemcpyAsync(f + 3 * m, d.fw[b], sizeof(float) * m, cudaMemcpyDeviceToHost, s), h);
      if (d.dim >= 2) {
        CK(cudaMemcpyAsync(f + 4 * m, d.fy[b], sizeof(float) * m, cudaMemcpyDeviceToHost, s), h);
        CK(cudaMemcpyAsync(f + 5 * m, d.foy[b], sizeof(float) * m, cudaMemcpyDeviceToHost, s), h);
      }
      if (d.dim == 3) {
        CK(cudaMemcpyAsync(f + 6 * m, d.fz[b], sizeof(float) * m, cudaMemcpyDeviceToHost, s), h);
        CK(cudaMemcpyAsync(f + 7 * m, d.foz[b], sizeof(float) * m, cudaMemcpyDeviceToHost, s), h);
      }
    }
    if (m > 0) {
      CK(cudaMemcpyAsync(parts->id, d.pid[b], sizeof(uint64_t) * m, cudaMemcpyDeviceToHost, s), h);
      CK(cudaMemcpyAsync(key.data(), d.pkey[b], sizeof(uint32_t) * m, cudaMemcpyDeviceToHost, s), h);
    }
    CK(cudaStreamSynchronize(s), h);
    for (long long i = 0; i < m; ++i) {
      const int cell = (int)(key[i] / (uint32_t)d.G);
      parts->cell[i] = (int32_t)cell;
      parts->grp[i] = (int32_t)(key[i] % (uint32_t)d.G);
      if (mixed) {
        const float* f = fb.data();
        const int ix = cell % d.nx, iy = (cell / d.nx) % d.ny, iz = cell / (d.nx * d.ny);
        parts->x[i] = ix * d.dx + (double)f[i];
        parts->ox[i] = f[m + i];
        parts->nu[i] = f[2 * m + i];
        parts->w[i] = f[3 * m + i];
        parts->y[i] = d.dim >= 2 ? iy * d.dy + (double)f[4 * m + i] : 0.0;
        parts->oy[i] = d.dim >= 2 ? (double)f[5 * m + i] : 0.0;
        if (d.dim == 3) {
          parts->z[i] = iz * d.dz + (double)f[6 * m + i];
          parts->oz[i] = (double)f[7 * m + i];
        }
      } else if (d.dim == 1) {
        parts->y[i] = 0.0;
        parts->oy[i] = 0.0;
      }
      if (d.dim < 3) {
        if (parts->z) parts->z[i] = 0.0;
        if (parts->oz) parts->oz[i] = 0.0;
      }
    }
  }
  CK(cudaStreamSynchronize(s), h);
  return UGKWP_OK;
}

int ugkwp_get_state(ugkwp_handle* h, double* T, double* rho, double* rho_h, double* rho_p,
                    ugkwp_particles_host* parts, int64_t cap, int64_t* n, void* stream) {
  return ugkwp_get_state_member(h, 0, T, rho, rho_h, rho_p, parts, cap, n, stream);
}

int ugkwp_set_state_member(ugkwp_handle* h, int member, const double* T, const double* rho,
                           const double* rho_h, const ugkwp_particles_host* parts, int64_t n,
                           int64_t step, void* stream) {
  if (!h || !T || !rho || !rho_h) return fail(h, UGKWP_ERR_ARG, "NULL argument");
  if (member < 0 || member >= h->M) return fail(h, UGKWP_ERR_ARG, "member index out of range");
  if (n < 0 || n > h->members[member].capacity) return fail(h, UGKWP_ERR_CAPACITY, "n exceeds particle capacity");
  if (step < 0 || (unsigned long long)step > ugkwp::kMaxStep)
    return fail(h, UGKWP_ERR_ARG, "step must be in 0..2^20-1 (a newborn's identity holds its birth step in 20 bits)");
  if (n > 0 && !parts) return fail(h, UGKWP_ERR_ARG, "particles missing");
  cudaStream_t s = (cudaStream_t)stream;
  const Dev& d = h->members[member];
  const size_t ncg = (size_t)d.ncell * d.G;
  CK(cudaMemcpyAsync(d.T, T, sizeof(double) * d.ncell, cudaMemcpyHostToDevice, s), h);
  CK(cudaMemcpyAsync(d.rho, rho, sizeof(double) * ncg, cudaMemcpyHostToDevice, s), h);
  CK(cudaMemcpyAsync(d.rho_h, rho_h, sizeof(double) * ncg, cudaMemcpyHostToDevice, s), h);
  std::vector<uint32_t> key(n > 0 ? n : 1);
  for (long long i = 0; i < n; ++i) {
    if (parts->cell[i] < 0 || parts->cell[i] >= d.ncell || parts->grp[i] < 0 || parts->grp[i] >= d.G)
      return fail(h, UGKWP_ERR_ARG, "particle cell or group out of range");
    key[i] = (uint32_t)(parts->cell[i] * d.G + parts->grp[i]);
  }
  if (n > 0 && d.dim == 3 && (!parts->z || !parts->oz)) return fail(h, UGKWP_ERR_ARG, "3D particles need z and oz");
  std::vector<float> fb(d.precision == UGKWP_MIXED && n > 0 ? (size_t)n * 8 : 1);
  if (n > 0 && d.precision != UGKWP_MIXED) {
    CK(cudaMemcpyAsync(d.px[0], parts->x, sizeof(double) * n, cudaMemcpyHostToDevice, s), h);
    CK(cudaMemcpyAsync(d.pox[0], parts->ox, sizeof(double) * n, cudaMemcpyHostToDevice, s), h);
    CK(cudaMemcpyAsync(d.pnu[0], parts->nu, sizeof(double) * n, cudaMemcpyHostToDevice, s), h);
    CK(cudaMemcpyAsync(d.pw[0], parts->w, sizeof(double) * n, cudaMemcpyHostToDevice, s), h);
    if (d.dim >= 2) {
      CK(cudaMemcpyAsync(d.py[0], parts->y, sizeof(double) * n, cudaMemcpyHostToDevice, s), h);
      CK(cudaMemcpyAsync(d.poy[0], parts->oy, sizeof(double) * n, cudaMemcpyHostToDevice, s), h);
    }
    if (d.dim == 3) {
      CK(cudaMemcpyAsync(d.pz[0], parts->z, sizeof(double) * n, cudaMemcpyHostToDevice, s), h);
      CK(cudaMemcpyAsync(d.poz[0], parts->oz, sizeof(double) * n, cudaMemcpyHostToDevice, s), h);
    }
  } else if (n > 0) {
    // positions relative to the particle's cell, in FP32
    float* f = fb.data();
    for (long long i = 0; i < n; ++i) {
      const int cell = parts->cell[i];
      const int ix = cell % d.nx, iy = (cell / d.nx) % d.ny, iz = cell / (d.nx * d.ny);
      f[i] = (float)(parts->x[i] - ix * d.dx);
      f[n + i] = (float)parts->ox[i];
      f[2 * n + i] = (float)parts->nu[i];
      f[3 * n + i] = (float)parts->w[i];
      f[4 * n + i] = d.dim >= 2 ? (float)(parts->y[i] - iy * d.dy) : 0.0f;
      f[5 * n + i] = d.dim >= 2 ? (float)parts->oy[i] : 0.0f;
      f[6 * n + i] = d.dim == 3 ? (float)(parts->z[i] - iz * d.dz) : 0.0f;
      f[7 * n + i] = d.dim == 3 ? (float)parts->oz[i] : 0.0f;
    }
    CK(cudaMemcpyAsync(d.fx[0], f, sizeof(float) * n, cudaMemcpyHostToDevice, s), h);
    CK(cudaMemcpyAsync(d.fox[0], f + n, sizeof(float) * n, cudaMemcpyHostToDevice, s), h);
    CK(cudaMemcpyAsync(d.fnu[0], f + 2 * n, sizeof(float) * n, cudaMemcpyHostToDevice, s), h);
    CK(cudaMemcpyAsync(d.fw[0], f + 3 * n, sizeof(float) * n, cudaMemcpyHostToDevice, s), h);
    if (d.dim >= 2) {
      CK(cudaMemcpyAsync(d.fy[0], f + 4 * n, sizeof(float) * n, cudaMemcpyHostToDevice, s), h);
      CK(cudaMemcpyAsync(d.foy[0], f + 5 * n, sizeof(float) * n, cudaMemcpyHostToDevice, s), h);
    }
    if (d.dim == 3) {
      CK(cudaMemcpyAsync(d.fz[0], f + 6 * n, sizeof(float) * n, cudaMemcpyHostToDevice, s), h);
      CK(cudaMemcpyAsync(d.foz[0], f + 7 * n, sizeof(float) * n, cudaMemcpyHostToDevice, s), h);
    }
  }
  if (n > 0) {
    CK(cudaMemcpyAsync(d.pid[0], parts->id, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, s), h);
    CK(cudaMemcpyAsync(d.pkey[0], key.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, s), h);
  }
  Ctrl c;
  CK(cudaMemcpyAsync(&c, d.ctrl, sizeof c, cudaMemcpyDeviceToHost, s), h);
  CK(cudaStreamSynchronize(s), h);
  c.cur = 0;
  c.n_part[0] = (unsigned long long)n;
  c.n_part[1] = 0;
  c.step = (unsigned long long)step;
  c.si_state_ok = 0;   // T changed: the stored iterate state is stale
  CK(cudaMemcpyAsync(d.ctrl, &c, sizeof c, cudaMemcpyHostToDevice, s), h);
  CK(cudaStreamSynchronize(s), h);
  return UGKWP_OK;
}

int ugkwp_set_state(ugkwp_handle* h, const double* T, const double* rho, const double* rho_h,
                    const ugkwp_particles_host* parts, int64_t n, int64_t step, void* stream) {
  return ugkwp_set_state_member(h, 0, T, rho, rho_h, parts, n, step, stream);
}

int ugkwp_set_records(ugkwp_handle* h, ugkwp_record* d_records, int64_t cap) {
  if (!h) return fail(nullptr, UGKWP_ERR_ARG, "handle is NULL");
  if (h->M > 1) return fail(h, UGKWP_ERR_UNSUPPORTED, "records are for single-problem handles");
  static_assert(sizeof(ugkwp_record) == sizeof(ugkwp::RecordOut), "record layout");
  h->d.rec = reinterpret_cast<ugkwp::RecordOut*>(d_records);
  h->d.rec_cap = d_records ? cap : 0;
  h->members[0] = h->d;
  drop_graph(h);   // the captured step holds the old record pointer
  return UGKWP_OK;
}

int ugkwp_set_launch(ugkwp_handle* h, int block, int particles_per_thread, int blocks_per_sm) {
  if (!h) return fail(nullptr, UGKWP_ERR_ARG, "handle is NULL");
  if ((block != 128 && block != 256 && block != 512) ||
      (particles_per_thread != 1 && particles_per_thread != 2 && particles_per_thread != 4) || blocks_per_sm < 0)
    return fail(h, UGKWP_ERR_ARG, "block must be 128, 256 or 512; particles per thread 1, 2 or 4");
  h->shape.block = block;
  h->shape.ppt = particles_per_thread;
  h->shape.blocks_per_sm = blocks_per_sm;
  h->ens.tile = ens_tile(h);
  drop_graph(h);
  return UGKWP_OK;
}

int ugkwp_set_wait_limit(ugkwp_handle* h, uint32_t spins, uint32_t extra_arrivals, void* stream) {
  if (!h) return fail(nullptr, UGKWP_ERR_ARG, "handle is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned int v[2] = {spins, extra_arrivals};
  for (int m = 0; m < h->M; ++m) {
    Ctrl* c = h->members[m].ctrl;
    CK(cudaMemcpyAsync(&c->bar_timeout_spins, &v[0], sizeof(unsigned int), cudaMemcpyHostToDevice, s), h);
    CK(cudaMemcpyAsync(&c->bar_extra, &v[1], sizeof(unsigned int), cudaMemcpyHostToDevice, s), h);
  }
  CK(cudaStreamSynchronize(s), h);   // the host values live on this frame
  return UGKWP_OK;
}

int ugkwp_checkpoint_size(const ugkwp_handle* h, size_t* bytes) {
  if (!h || !bytes) return fail(nullptr, UGKWP_ERR_ARG, "NULL argument");
  size_t tot = align256(sizeof(size_t) * (size_t)h->M);
  for (int m = 0; m < h->M; ++m) tot += ugkwp::ckpt_bytes(h->members[m]);
  *bytes = tot;
  return UGKWP_OK;
}

namespace {
int checkpoint_io(ugkwp_handle* h, void* d_buf, size_t bytes, void* stream, int save) {
  size_t need = 0;
  ugkwp_checkpoint_size(h, &need);
  if (!d_buf || bytes < need) return fail(h, UGKWP_ERR_WORKSPACE, "checkpoint buffer smaller than ugkwp_checkpoint_size");
  if (reinterpret_cast<uintptr_t>(d_buf) % 256) return fail(h, UGKWP_ERR_WORKSPACE, "checkpoint buffer must be 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<size_t> offs(h->M);
  size_t o = align256(sizeof(size_t) * (size_t)h->M);
  for (int m = 0; m < h->M; ++m) { offs[m] = o; o += ugkwp::ckpt_bytes(h->members[m]); }
  // the member offsets live in the buffer's head (copied from pageable memory: staged before return)
  CK(cudaMemcpyAsync(d_buf, offs.data(), sizeof(size_t) * h->M, cudaMemcpyHostToDevice, s), h);
  CK(ugkwp::launch_checkpoint(h->d, h->M > 1 ? &h->ens : nullptr, static_cast<char*>(d_buf),
                              static_cast<const size_t*>(d_buf), save, s), h);
  return UGKWP_OK;
}
}  // namespace

int ugkwp_checkpoint(ugkwp_handle* h, void* d_buf, size_t bytes, void* stream) {
  if (!h) return fail(nullptr, UGKWP_ERR_ARG, "handle is NULL");
  return checkpoint_io(h, d_buf, bytes, stream, 1);
}

int ugkwp_restore(ugkwp_handle* h, const void* d_buf, size_t bytes, void* stream) {
  if (!h) return fail(nullptr, UGKWP_ERR_ARG, "handle is NULL");
  return checkpoint_io(h, const_cast<void*>(d_buf), bytes, stream, 0);
}

int ugkwp_autotune(ugkwp_handle* h, void* d_ckpt, size_t bytes, int steps, void* stream, int* best,
                   float* best_ms) {
  if (!h || !best) return fail(h, UGKWP_ERR_ARG, "NULL argument");
  if (steps < 1) return fail(h, UGKWP_ERR_ARG, "steps must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  int st = ugkwp_checkpoint(h, d_ckpt, bytes, stream);
  if (st) return st;
  const ugkwp::StreamShape keep = h->shape;
  const int blocks[3] = {128, 256, 512}, ppts[3] = {1, 2, 4}, pers[2] = {0, -1};
  float best_t = 1e30f;
  ugkwp::StreamShape best_s = keep;
  for (int bi = 0; bi < 3; ++bi)
    for (int pi = 0; pi < 3; ++pi)
      for (int qi = 0; qi < 2; ++qi) {
        ugkwp::StreamShape sh;
        sh.block = blocks[bi];
        sh.ppt = ppts[pi];
        // -1: half of what fits (longer persistent loops, fewer resident warps)
        int occ = 0;
        if (pers[qi] < 0) {
          int dev = 0;
          cudaGetDevice(&dev);
          occ = 2048 / sh.block / 2;
          if (occ < 1) occ = 1;
        }
        sh.blocks_per_sm = pers[qi] < 0 ? occ : 0;
        h->shape = sh;
        h->ens.tile = ens_tile(h);
        if ((st = ugkwp_restore(h, d_ckpt, bytes, stream))) return st;
        float total = 0.f;
        for (int k = 0; k < steps; ++k) {
          float ms[6];
          if ((st = ugkwp_step_timed(h, stream, ms))) return st;
          total += ms[3];
        }
        if (total < best_t) { best_t = total; best_s = sh; }
      }
  h->shape = best_s;
  h->ens.tile = ens_tile(h);
  drop_graph(h);
  if ((st = ugkwp_restore(h, d_ckpt, bytes, stream))) return st;
  CK(cudaStreamSynchronize(s), h);
  best[0] = best_s.block;
  best[1] = best_s.ppt;
  best[2] = best_s.blocks_per_sm;
  if (best_ms) *best_ms = best_t / steps;
  (void)keep;
  return UGKWP_OK;
}

// ---- adjoint: tape of a forward step, reverse steps, result
namespace {
int adjoint_check(ugkwp_handle* h) {
  if (!h) return fail(nullptr, UGKWP_ERR_ARG, "handle is NULL");
  if (h->M > 1) return fail(h, UGKWP_ERR_UNSUPPORTED, "the adjoint is for single-problem handles");
  if (h->d.precision != UGKWP_FP64)
    return fail(h, UGKWP_ERR_UNSUPPORTED, "the adjoint tape is written by the FP64 particle kernel");
  if (h->d.tau_num_C != 0.0)
    return fail(h, UGKWP_ERR_UNSUPPORTED, "the adjoint differentiates tau, not tau_num (tau_num_C = 0)");
  if (h->d.split_literal)
    return fail(h, UGKWP_ERR_UNSUPPORTED, "the adjoint is checked with the default wave/particle split (split_literal = 0)");
  if (h->d.sig_law != 0)
    return fail(h, UGKWP_ERR_UNSUPPORTED, "the adjoint differentiates the power-law opacity (sig_law = 0)");
  if (h->d.cv_law != 0)
    return fail(h, UGKWP_ERR_UNSUPPORTED, "the adjoint takes a constant heat capacity (cv_law = 0)");
  if (h->d.method != UGKWP_METHOD_UGKWP)
    return fail(h, UGKWP_ERR_UNSUPPORTED, "the adjoint differentiates the UGKWP sampling (method = 0)");
  if (h->d.dim == 3) return fail(h, UGKWP_ERR_UNSUPPORTED, "the adjoint is built for 1D and 2D grids");
  return UGKWP_OK;
}
}  // namespace

int ugkwp_tape_size(ugkwp_handle* h, int64_t rec_cap, size_t* bytes) {
  int st = adjoint_check(h);
  if (st) return st;
  if (!bytes || rec_cap < 0) return fail(h, UGKWP_ERR_ARG, "bad arguments");
  *bytes = ugkwp::tape_layout(h->d, rec_cap).total;
  return UGKWP_OK;
}

int ugkwp_step_taped(ugkwp_handle* h, void* d_tape, size_t bytes, int64_t rec_cap, void* stream) {
  int st = adjoint_check(h);
  if (st) return st;
  if (!d_tape || rec_cap < 0) return fail(h, UGKWP_ERR_ARG, "bad arguments");
  const ugkwp::TapeLayout L = ugkwp::tape_layout(h->d, rec_cap);
  if (bytes < L.total) return fail(h, UGKWP_ERR_WORKSPACE, "tape smaller than ugkwp_tape_size");
  if (reinterpret_cast<uintptr_t>(d_tape) % 256) return fail(h, UGKWP_ERR_WORKSPACE, "tape must be 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const Dev& d = h->d;
  char* b = static_cast<char*>(d_tape);
  const size_t ncg = (size_t)d.ncell * d.G;
  CK(cudaMemcpyAsync(b + L.T0, d.T, sizeof(double) * d.ncell, cudaMemcpyDeviceToDevice, s), h);
  CK(cudaMemcpyAsync(b + L.rho_h0, d.rho_h, sizeof(double) * ncg, cudaMemcpyDeviceToDevice, s), h);
  Dev dt = d;
  dt.tape = reinterpret_cast<ugkwp::TapeRec*>(b + L.rec);
  dt.tape_cap = rec_cap;
  CK(enqueue_step_dev(dt, nullptr, h->shape, s), h);
  CK(cudaMemcpyAsync(b + L.T1, d.T, sizeof(double) * d.ncell, cudaMemcpyDeviceToDevice, s), h);
  CK(cudaMemcpyAsync(b + L.rho1, d.rho, sizeof(double) * ncg, cudaMemcpyDeviceToDevice, s), h);
  CK(cudaMemcpyAsync(b + L.wscale, d.wscale, sizeof(double) * ncg, cudaMemcpyDeviceToDevice, s), h);
  CK(cudaMemcpyAsync(b + L.Esurv, d.E_surv, sizeof(double) * ncg, cudaMemcpyDeviceToDevice, s), h);
  CK(cudaMemcpyAsync(b + L.N, d.N, sizeof(uint32_t) * d.nbins, cudaMemcpyDeviceToDevice, s), h);
  CK(cudaMemcpyAsync(b + L.hdr, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToDevice, s), h);
  return UGKWP_OK;
}

int ugkwp_adjoint_workspace_size(ugkwp_handle* h, size_t* bytes) {
  int st = adjoint_check(h);
  if (st) return st;
  if (!bytes) return fail(h, UGKWP_ERR_ARG, "NULL argument");
  *bytes = ugkwp::adjoint_bytes(h->d);
  return UGKWP_OK;
}

namespace {
int adjoint_ws_check(ugkwp_handle* h, const void* d_adj, size_t bytes) {
  if (!d_adj || bytes < ugkwp::adjoint_bytes(h->d))
    return fail(h, UGKWP_ERR_WORKSPACE, "adjoint workspace smaller than ugkwp_adjoint_workspace_size");
  if (reinterpret_cast<uintptr_t>(d_adj) % 256)
    return fail(h, UGKWP_ERR_WORKSPACE, "adjoint workspace must be 256-byte aligned");
  return UGKWP_OK;
}
}  // namespace

int ugkwp_adjoint_seed(ugkwp_handle* h, void* d_adj, size_t bytes, const double* d_dL_dT, void* stream) {
  int st = adjoint_check(h);
  if (st || (st = adjoint_ws_check(h, d_adj, bytes))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemsetAsync(d_adj, 0, ugkwp::adjoint_bytes(h->d), s), h);
  const ugkwp::AdjView a = ugkwp::adjoint_view(h->d, d_adj);
  CK(cudaMemcpyAsync(&a.ctrl->bar_limit, &h->d.ctrl->bar_timeout_spins, sizeof(unsigned int),
                     cudaMemcpyDeviceToDevice, s), h);
  if (d_dL_dT)
    CK(cudaMemcpyAsync(a.lamT, d_dL_dT, sizeof(double) * h->d.ncell, cudaMemcpyDeviceToDevice, s), h);
  return UGKWP_OK;
}

int ugkwp_adjoint_step(ugkwp_handle* h, const void* d_tape, size_t tape_bytes, int64_t rec_cap, void* d_adj,
                       size_t adj_bytes, void* stream) {
  int st = adjoint_check(h);
  if (st || (st = adjoint_ws_check(h, d_adj, adj_bytes))) return st;
  if (!d_tape || rec_cap < 0) return fail(h, UGKWP_ERR_ARG, "bad arguments");
  if (tape_bytes < ugkwp::tape_layout(h->d, rec_cap).total)
    return fail(h, UGKWP_ERR_WORKSPACE, "tape smaller than ugkwp_tape_size");
  const ugkwp::TapeView t = ugkwp::tape_view(h->d, d_tape, rec_cap);
  const ugkwp::AdjView a = ugkwp::adjoint_view(h->d, d_adj);
  CK(ugkwp::launch_adjoint_step(h->d, t, a, (cudaStream_t)stream), h);
  return UGKWP_OK;
}

int ugkwp_adjoint_remap(ugkwp_handle* h, void* d_adj, size_t adj_bytes, const void* d_ckpt, size_t ckpt_bytes,
                        void* stream) {
  int st = adjoint_check(h);
  if (st || (st = adjoint_ws_check(h, d_adj, adj_bytes))) return st;
  size_t need = 0;
  ugkwp_checkpoint_size(h, &need);
  if (!d_ckpt || ckpt_bytes < need) return fail(h, UGKWP_ERR_WORKSPACE, "checkpoint buffer smaller than ugkwp_checkpoint_size");
  const ugkwp::AdjView a = ugkwp::adjoint_view(h->d, d_adj);
  // single-problem checkpoint: member 0 starts after the 256-byte offset table
  const char* member = static_cast<const char*>(d_ckpt) + align256(sizeof(size_t));
  CK(ugkwp::launch_adjoint_remap(h->d, a, member, (cudaStream_t)stream), h);
  return UGKWP_OK;
}

int ugkwp_adjoint_result(ugkwp_handle* h, const void* d_adj, size_t bytes, double* d_dL_ds, double* d_dL_dT0,
                         uint32_t* status_bits, int32_t* si_iters, uint64_t* unmatched, void* stream) {
  int st = adjoint_check(h);
  if (st || (st = adjoint_ws_check(h, d_adj, bytes))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const ugkwp::AdjView a = ugkwp::adjoint_view(h->d, const_cast<void*>(d_adj));
  if (d_dL_ds) CK(cudaMemcpyAsync(d_dL_ds, a.lamS, sizeof(double) * h->d.ncell, cudaMemcpyDeviceToDevice, s), h);
  if (d_dL_dT0) CK(cudaMemcpyAsync(d_dL_dT0, a.lamT, sizeof(double) * h->d.ncell, cudaMemcpyDeviceToDevice, s), h);
  ugkwp::AdjCtrl c;
  CK(cudaMemcpyAsync(&c, a.ctrl, sizeof c, cudaMemcpyDeviceToHost, s), h);
  CK(cudaStreamSynchronize(s), h);
  if (status_bits) *status_bits = c.status;
  if (si_iters) *si_iters = (int32_t)c.iters;
  if (unmatched) *unmatched = (uint64_t)c.unmatched;
  return UGKWP_OK;
}

const char* ugkwp_last_error(const ugkwp_handle* h) { return h ? h->err : g_err; }

void ugkwp_destroy(ugkwp_handle* h) {
  if (!h) return;
  drop_graph(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side_stream) cudaStreamDestroy(h->side_stream);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->sort_stream) cudaStreamDestroy(h->sort_stream);
  if (h->ev_fork2) cudaEventDestroy(h->ev_fork2);
  if (h->ev_join2) cudaEventDestroy(h->ev_join2);
  delete h;
}

int ugkwp_philox(const uint32_t* d_ctr, uint32_t k0, uint32_t k1, uint32_t* d_out, int64_t n,
                 void* stream) {
  if (n < 0 || (n > 0 && (!d_ctr || !d_out))) return fail(nullptr, UGKWP_ERR_ARG, "bad arguments");
  if (n == 0) return UGKWP_OK;
  CK(ugkwp::launch_unit_philox(d_ctr, k0, k1, d_out, n, (cudaStream_t)stream), nullptr);
  return UGKWP_OK;
}

int ugkwp_planck(const double* d_T, int64_t n, const double* d_nu_edges, int G, double* d_b,
                 double* d_d, void* stream) {
  if (n < 0 || G < 1 || (n > 0 && (!d_T || !d_nu_edges || !d_b)))
    return fail(nullptr, UGKWP_ERR_ARG, "bad arguments");
  if (n == 0) return UGKWP_OK;
  CK(ugkwp::launch_unit_planck(d_T, n, d_nu_edges, G, d_b, d_d, (cudaStream_t)stream), nullptr);
  return UGKWP_OK;
}

int ugkwp_coefs(const double* d_x, int64_t n, double* d_out, void* stream) {
  if (n < 0 || (n > 0 && (!d_x || !d_out))) return fail(nullptr, UGKWP_ERR_ARG, "bad arguments");
  if (n == 0) return UGKWP_OK;
  CK(ugkwp::launch_unit_coefs(d_x, n, d_out, (cudaStream_t)stream), nullptr);
  return UGKWP_OK;
}

int ugkwp_exclusive_scan(const uint32_t* d_counts, int64_t n, uint32_t* d_offsets, void* d_scratch,
                         size_t scratch_bytes, void* stream) {
  if (n < 0 || n > (1ll << 24) || !d_offsets || (n > 0 && !d_counts))
    return fail(nullptr, UGKWP_ERR_ARG, "bad arguments (0 <= n <= 2^24, counts and offsets required)");
  if (!d_scratch || scratch_bytes < (size_t)UGKWP_SCAN_SCRATCH_BYTES(n))
    return fail(nullptr, UGKWP_ERR_WORKSPACE, "scratch smaller than UGKWP_SCAN_SCRATCH_BYTES(n)");
  CK(ugkwp::launch_scan(d_counts, n, static_cast<uint32_t*>(d_scratch), d_offsets, nullptr, nullptr,
                        (cudaStream_t)stream), nullptr);
  return UGKWP_OK;
}

int ugkwp_sample_nu(const double* d_eta, int64_t n, double nlo, double nhi, double T, double* d_nu,
                    void* stream) {
  if (n < 0 || !(nhi > nlo) || (n > 0 && (!d_eta || !d_nu))) return fail(nullptr, UGKWP_ERR_ARG, "bad arguments");
  if (n == 0) return UGKWP_OK;
  CK(ugkwp::launch_unit_sample(d_eta, n, nlo, nhi, T, d_nu, (cudaStream_t)stream), nullptr);
  return UGKWP_OK;
}

}  // extern "C"
