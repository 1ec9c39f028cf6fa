// ugkwp_grid.cuh -- cell and face helpers shared by the step kernels and
// their adjoint: face indexing along grid lines, the van Leer limiter, warp
// reductions and the per-cell opacity/Planck evaluation of the source
// iteration (one warp per cell, one lane per group).
#pragma once
#include "ugkwp_device.cuh"

namespace ugkwp {

// --------------------------------------------------------------------------
// Face walk helpers: face f -> axis, the line of cells through it and its
// position along the line.  A line of axis a is the set of cells sharing the
// other two coordinates; its cells are base + k*stride, k = 0..nk-1.
struct FaceRef {
  int axis, k, nk;   // face between line cells k-1 and k, 0..nk
  int base, stride;
  double h;
};

__device__ __forceinline__ FaceRef face_ref(const Dev& d, int f) {
  FaceRef r;
  if (f < d.nxface) {
    const int line = f / (d.nx + 1);
    r.axis = 0; r.k = f - line * (d.nx + 1); r.nk = d.nx; r.h = d.dx;
    r.base = line * d.nx; r.stride = 1;
  } else if (f < d.nxface + d.nyface) {
    // y-faces (iz (ny+1) + k) nx + ix
    const int q = f - d.nxface;
    const int t = q / d.nx, ix = q - t * d.nx;
    const int iz = d.nz > 1 ? t / (d.ny + 1) : 0;
    r.axis = 1; r.k = t - iz * (d.ny + 1); r.nk = d.ny; r.h = d.dy;
    r.base = iz * d.nx * d.ny + ix; r.stride = d.nx;
  } else {
    // z-faces k nx ny + (iy nx + ix)
    const int q = f - d.nxface - d.nyface, nxy = d.nx * d.ny;
    r.axis = 2; r.k = q / nxy; r.nk = d.nz; r.h = d.dz;
    r.base = q - r.k * nxy; r.stride = nxy;
  }
  return r;
}

__device__ __forceinline__ int line_cell(const Dev& d, const FaceRef& r, int k) {
  (void)d;
  return r.base + k * r.stride;
}

__device__ __forceinline__ double inv_h_of(const Dev& d, int axis) {
  return axis == 0 ? d.inv_dx : (axis == 1 ? d.inv_dy : d.inv_dz);
}

// cell c -> (ix, iy, iz)
__device__ __forceinline__ void cell_xyz(const Dev& d, int c, int* ix, int* iy, int* iz) {
  if (d.nz > 1) {
    const int nxy = d.nx * d.ny;
    *iz = c / nxy;
    c -= *iz * nxy;
  } else {
    *iz = 0;
  }
  *iy = c / d.nx;
  *ix = c - *iy * d.nx;
}

// rho_h at line position k including ghosts (mirror / black body / vacuum)
__device__ __forceinline__ double rho_h_at(const Dev& d, const FaceRef& r, int k, int g) {
  if (k >= 0 && k < r.nk) return d.rho_h[line_cell(d, r, k) * d.G + g];
  const int side = r.axis * 2 + (k < 0 ? 0 : 1);
  if (d.bc[side] == BC_REFLECT) return d.rho_h[line_cell(d, r, k < 0 ? 0 : r.nk - 1) * d.G + g];
  if (d.bc[side] == BC_BLACKBODY) return d.ghost_phi[side * d.G + g];
  return 0.0;
}

__device__ __forceinline__ double van_leer(double a, double b) {
  return a * b > 0.0 ? 2.0 * a * b / (a + b) : 0.0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Planck and opacity of one cell at temperature T for the lane's groups:
// sigma_g, Phi_g and dPhi_g/dT, g = lane + 32 j.  Edge values are shared
// between neighbouring lanes by shuffles.
template <int NC>
__device__ __forceinline__ void cell_planck(const Dev& d, int c, double T, double* sig, double* phi,
                                            double* dphi, double invT, double sT) {
  const int lane = threadIdx.x & 31, G = d.G;
  const double ac = d.a * d.c, T3 = T * T * T;
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const int g = lane + 32 * j;
    if (d.grey) {
      sig[j] = cap_sigma(d, sT);
      phi[j] = T > 0.0 ? ac * T3 * T : 0.0;
      dphi[j] = T > 0.0 ? 4.0 * ac * T3 : 0.0;
      continue;
    }
    EdgeVal lo;
    if (g <= G && T > 0.0) lo = planck_edge(d.nu_edges[g] * invT);
    else { lo.V = 0.0; lo.g4 = 0.0; lo.lower = true; }
    EdgeVal hi;
    hi.V = __shfl_down_sync(0xffffffffu, lo.V, 1);
    hi.g4 = __shfl_down_sync(0xffffffffu, lo.g4, 1);
    hi.lower = __shfl_down_sync(0xffffffffu, (int)lo.lower, 1) != 0;
    if (lane == 31 && g + 1 <= G && T > 0.0) hi = planck_edge(d.nu_edges[g + 1] * invT);
    if (g < G) {
      sig[j] = sigma_group_at(d, sT, T, invT, g);
      if (T > 0.0) {
        const double b = planck_fraction(lo, hi);
        phi[j] = ac * T3 * T * b;
        dphi[j] = ac * T3 * planck_dfraction(b, lo, hi);
      } else {
        phi[j] = 0.0;
        dphi[j] = 0.0;
      }
    } else {
      sig[j] = 1.0; phi[j] = 0.0; dphi[j] = 0.0;
    }
  }
}

template <int NC>
__device__ __forceinline__ void cell_planck(const Dev& d, int c, double T, double* sig, double* phi,
                                            double* dphi, double invT) {
  cell_planck<NC>(d, c, T, sig, phi, dphi, invT, sigma_T(d, c, T));
}

template <int NC>
__device__ __forceinline__ void cell_planck(const Dev& d, int c, double T, double* sig, double* phi,
                                            double* dphi) {
  cell_planck<NC>(d, c, T, sig, phi, dphi, 1.0 / T);
}

// tau = 1/(rate sigma) and q = 1/(tau + dt) of the source iteration with one
// reciprocal: A = rate sigma, D = 1 + dt A, P = 1/(A D), tau = D P, q = A^2 P.
__device__ __forceinline__ void tau_and_q(const Dev& d, double sig, double* tau, double* q) {
  const double A = d.rate_f * sig, D = fma(d.dt, A, 1.0);
  const double P = rcp_nr(A * D);
  *tau = D * P;
  *q = A * A * P;
}

// the face on `axis` of the cell at (ix, iy, iz), lower (dir < 0) or upper side
__device__ __forceinline__ int face_index_xyz(const Dev& d, int ix, int iy, int iz, int axis, int dir) {
  const int up = dir > 0 ? 1 : 0;
  if (axis == 0) return (iz * d.ny + iy) * (d.nx + 1) + ix + up;
  if (axis == 1) return d.nxface + (iz * (d.ny + 1) + iy + up) * d.nx + ix;
  return d.nxface + d.nyface + ((iz + up) * d.ny + iy) * d.nx + ix;
}

__device__ __forceinline__ int face_index(const Dev& d, int c, int axis, int dir) {
  int ix, iy, iz;
  cell_xyz(d, c, &ix, &iy, &iz);
  return face_index_xyz(d, ix, iy, iz, axis, dir);
}

}  // namespace ugkwp
