// ugkwp_launch.h -- host-side launchers of the device kernels (internal).
#pragma once
#include <atomic>
#include <cuda_runtime.h>
#include "ugkwp_device.cuh"

namespace ugkwp {

constexpr int kMaxDevices = 64;
// multiprocessors of the current device (looked up once per device)
int sm_count();
// counts per block of the three-kernel scan (launch_scan): its scratch holds
// one partial sum per (n + kScanTileCounts - 1) / kScanTileCounts
constexpr long long kScanTileCounts = 4096;

cudaError_t launch_init_tables(const Dev& d, const double* src_T, const double* src_amp, int init_rho,
                               cudaStream_t s);
cudaError_t launch_birth_and_scan(const Dev& d, const Ens* e, cudaStream_t s);
int scan_parts(long long n);
cudaError_t launch_scan(const uint32_t* N, long long n, uint32_t* part, uint32_t* off,
                        unsigned long long* total_a, unsigned long long* total_b, cudaStream_t s);
cudaError_t launch_wave(const Dev& d, const Ens* e, cudaStream_t s);
// The particle kernels of a step: one launch.  A mixed-precision 1D single
// problem with few face crossings takes the survivor kernel (which also
// streams the newborns), every other problem the general kernel of its
// precision.
cudaError_t launch_stream(const Dev& d, const Ens* e, const StreamShape& sh, cudaStream_t s);
cudaError_t launch_si(const Dev& d, const Ens* e, cudaStream_t s);
cudaError_t launch_end_step(const Dev& d, const Ens* e, cudaStream_t s);
// survivor sort of every step: scan of the survivors per bin, scatter back
// into the input buffer in bin order
cudaError_t launch_sort(const Dev& d, const Ens* e, cudaStream_t s);

size_t ckpt_bytes(const Dev& d);
cudaError_t launch_checkpoint(const Dev& d, const Ens* e, char* buf, const size_t* d_offs, int save,
                              cudaStream_t s);

// ---- adjoint (ugkwp_adjoint.cu)
// Tape of one forward step, in a caller buffer: the control block after the
// step (counts), T^n, T^{n+1}, rho^{n+1}, rho_h^n, the survivors' scaling
// factors and E_surv per (cell, group), the birth counts N and one TapeRec
// per processed particle.
struct TapeLayout {
  size_t hdr, T0, T1, rho1, rho_h0, wscale, Esurv, N, rec, total;
};
struct TapeView {
  const Ctrl* hdr;
  const double *T0, *T1, *rho1, *rho_h0, *wscale, *Esurv;
  const uint32_t* N;
  const TapeRec* rec;
  long long rec_cap;
};
// Control block of the adjoint workspace.
struct AdjCtrl {
  unsigned int bar_count;       // grid barrier arrivals (reset before each adjoint step)
  unsigned int status;          // ST_* bits, latched since the seed
  unsigned int cur;             // which lamW buffer holds the next step's weight adjoints
  unsigned int iters;           // adjoint source iterations of the last step
  unsigned int bar_limit;       // bounded-wait limit (0: default)
  unsigned int pad;
  unsigned long long err_slot[3][2];
  unsigned long long unmatched; // particles without a partner across a checkpoint boundary
};
// Adjoint workspace: the adjoint state (of T^n, rho^n, rho_h^n and the
// incoming particles' weights), the accumulated dL/ds and per-step work.
struct AdjView {
  AdjCtrl* ctrl;
  double *lamT, *lamS, *lamT0, *ls, *lamRho, *lamRhoH;
  double* lamW[2];
  double *lamR, *lamRhoH0, *lamSig0, *lamE, *Sb;
  double *mu[2], *gT, *D, *Jl;
  double *sig1, *sig1s, *phi1, *dphi1, *sig0, *sig0s, *dFdT;
  unsigned long long* hkeys;    // id -> weight-adjoint hash (remap across checkpoints)
  double* hvals;
  long long hsize;              // power of two >= 2 x capacity
  long long cap;
};
TapeLayout tape_layout(const Dev& d, long long rec_cap);
TapeView tape_view(const Dev& d, const void* base, long long rec_cap);
size_t adjoint_bytes(const Dev& d);
AdjView adjoint_view(const Dev& d, void* base);
cudaError_t launch_adjoint_step(const Dev& d, const TapeView& t, const AdjView& a, cudaStream_t s);
// Re-index the weight adjoints from a checkpoint's particle order (ids and
// count read from the checkpoint buffer of member 0) to the handle's current
// particle order, matching by particle identity.
cudaError_t launch_adjoint_remap(const Dev& d, const AdjView& a, const char* ckpt_member, cudaStream_t s);
size_t ckpt_ids_offset(const Dev& d);
size_t ckpt_ctrl_offset(const Dev& d);

// message returned by ugkwp_last_error(NULL)
void set_global_error(const char* msg);

cudaError_t launch_unit_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out,
                               long long n, cudaStream_t s);
cudaError_t launch_unit_planck(const double* T, long long n, const double* nu, int G, double* b,
                               double* dd, cudaStream_t s);
cudaError_t launch_unit_coefs(const double* x, long long n, double* out, cudaStream_t s);
cudaError_t launch_unit_sample(const double* eta, long long n, double nlo, double nhi, double T,
                               double* nu, cudaStream_t s);

}  // namespace ugkwp
