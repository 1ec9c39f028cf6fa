// ugkwp_launch.h -- host-side launchers of the device kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include "ugkwp_device.cuh"

namespace ugkwp {

cudaError_t launch_init_tables(const Dev& d, const double* src_T, int init_rho, cudaStream_t s);
cudaError_t launch_birth_and_scan(const Dev& d, const Ens* e, cudaStream_t s);
int scan_parts(long long n);
cudaError_t launch_scan(const uint32_t* N, long long n, uint32_t* part, uint32_t* off,
                        unsigned long long* total_a, unsigned long long* total_b, cudaStream_t s);
cudaError_t launch_wave(const Dev& d, const Ens* e, cudaStream_t s);
cudaError_t launch_stream(const Dev& d, const Ens* e, const StreamShape& sh, cudaStream_t s);
cudaError_t launch_si(const Dev& d, const Ens* e, cudaStream_t s);
cudaError_t launch_end_step(const Dev& d, const Ens* e, cudaStream_t s);

size_t ckpt_bytes(const Dev& d);
cudaError_t launch_checkpoint(const Dev& d, const Ens* e, char* buf, const size_t* d_offs, int save,
                              cudaStream_t s);

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
