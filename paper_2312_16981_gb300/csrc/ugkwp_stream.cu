// ugkwp_stream.cu -- the particle kernels of the UGKWP step on sm_103a.
//
// One persistent launch processes a virtual index space [0, n_surv + n_new):
// first the particles that survived the previous step (Algorithm 1: a free
// time t_f = min(-tau ln eta, dt), Eq. particle-tf-formula), then the
// particles sampled this step from the wave part's collisionless fraction
// (Eq. IhpFormula; born in registers with t_f = dt; in the UGKP variant all
// of the wave part is sampled and a newborn draws its free time after its
// birth draws).  Each particle streams cell by cell with the free time reset
// on entering a new cell (interface remark: t_f2 = min(-tau_i ln eta,
// dt - t_tra)), reflects at mirror walls, escapes through open sides.
// Tallies: the net particle energy per (cell, group) w^{fr,p} (Eq.
// wfrpFormula, accumulated as end minus start, which telescopes the face
// crossings), the energy of the collisionless survivors per end bin, escapes
// and inflow per side.
//
// Every processed particle is written in place: particle i of the step goes
// to slot i of the other buffer, a particle that collided, escaped or left a
// ghost leaves its slot marked dead (kDeadKey).  There is no compaction here,
// so no atomics and no block barrier decide where a survivor goes; instead
// the kernel counts the survivors per end bin, and the survivor sort (a scan
// of the counts and a scatter, beside the source iteration) moves them back
// into the input buffer in bin order.  That is Algorithm 1's last step
// (collided particles removed) with the survivors kept cell-sorted.
//
// The FP32 kernel streams chunks of survivors staged in shared memory: each
// warp starts bulk copies (cp.async.bulk, completion counted on an mbarrier)
// of its next chunks' arrays into a ring of three stages of its own while it
// streams the current one, so no warp waits for another.  Per-cell opacity
// factors of single problems are held in shared memory when they fit.
#include "ugkwp_device.cuh"
#include "ugkwp_launch.h"

namespace ugkwp {


// largest b with off[b] <= j, for off[0] = 0 <= j < off[nbins]
__device__ __forceinline__ int find_bin(const uint32_t* __restrict__ off, int nbins, uint32_t j) {
  int lo = 0, hi = nbins;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= j) lo = mid; else hi = mid;
  }
  return lo;
}

// Sum the fixed-point weights v over runs of equal keys among consecutive
// lanes and add each run's total once (keys < 0 contribute nothing), and each
// run's length to cnt[key] (the survivors per bin that the sort moves).
// Particles are held sorted by (cell, group), so a warp usually issues one
// add per run.  Integer sums: the result does not depend on which lanes meet
// in a warp.  Common case first: every lane with a key holds the same key and
// v >= 0; then the warp sums v in three 21-bit pieces with integer warp
// reductions (each piece's sum stays below 2^26; v < 2^57 by the fixed-point
// range) instead of the segmented scan.
__device__ __forceinline__ void warp_run_add_fixed(unsigned long long* base, int key, long long v,
                                                   uint32_t* cnt) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned keyed = __ballot_sync(full, key >= 0);
  if (!keyed) return;
  const int first = __ffs(keyed) - 1;
  const int k0 = __shfl_sync(full, key, first);
  if (__all_sync(full, key < 0 || (key == k0 && v >= 0))) {
    const unsigned long long u = key >= 0 ? (unsigned long long)v : 0ull;
    const unsigned long long s0 = __reduce_add_sync(full, (unsigned)(u & 0x1fffffull));
    const unsigned long long s1 = __reduce_add_sync(full, (unsigned)((u >> 21) & 0x1fffffull));
    const unsigned long long s2 = __reduce_add_sync(full, (unsigned)(u >> 42));
    if (lane == first) {
      atomic_add_fixed(base + 2 * (long long)k0, (long long)(s0 + (s1 << 21) + (s2 << 42)));
      atomicAdd(cnt + k0, (unsigned)__popc(keyed));
    }
    return;
  }
  const int prev = __shfl_up_sync(full, key, 1);
  const bool head = lane == 0 || prev != key;
  const unsigned heads = __ballot_sync(full, head);
  const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(full, v, o);
    if (lane - o >= start) v += t;
  }
  const int nxt = __shfl_down_sync(full, key, 1);
  const bool tail = lane == 31 || nxt != key;
  if (tail && key >= 0) {
    atomic_add_fixed(base + 2 * (long long)key, v);
    atomicAdd(cnt + key, (unsigned)(lane - start + 1));
  }
}

// The same with a count per lane (n survivors summed in v by this lane):
// each run adds its v total to base[key] and its n total to cnt[key].
__device__ __forceinline__ void warp_run_add_fixed_n(unsigned long long* base, int key, long long v, unsigned n,
                                                     uint32_t* cnt) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned keyed = __ballot_sync(full, key >= 0);
  if (!keyed) return;
  const int first = __ffs(keyed) - 1;
  const int k0 = __shfl_sync(full, key, first);
  if (__all_sync(full, key < 0 || (key == k0 && v >= 0))) {
    const unsigned long long u = key >= 0 ? (unsigned long long)v : 0ull;
    const unsigned long long s0 = __reduce_add_sync(full, (unsigned)(u & 0x1fffffull));
    const unsigned long long s1 = __reduce_add_sync(full, (unsigned)((u >> 21) & 0x1fffffull));
    const unsigned long long s2 = __reduce_add_sync(full, (unsigned)(u >> 42));
    const unsigned sn = __reduce_add_sync(full, key >= 0 ? n : 0u);
    if (lane == first) {
      atomic_add_fixed(base + 2 * (long long)k0, (long long)(s0 + (s1 << 21) + (s2 << 42)));
      atomicAdd(cnt + k0, sn);
    }
    return;
  }
  const int prev = __shfl_up_sync(full, key, 1);
  const bool head = lane == 0 || prev != key;
  const unsigned heads = __ballot_sync(full, head);
  const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(full, v, o);
    const unsigned tn = __shfl_up_sync(full, n, o);
    if (lane - o >= start) { v += t; n += tn; }
  }
  const int nxt = __shfl_down_sync(full, key, 1);
  const bool tail = lane == 31 || nxt != key;
  if (tail && key >= 0) {
    atomic_add_fixed(base + 2 * (long long)key, v);
    atomicAdd(cnt + key, n);
  }
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// --------------------------------------------------------------------------
// Bulk asynchronous copies (cp.async.bulk, completion on an mbarrier) that
// stage tiles of particle arrays in shared memory.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for phase `parity` of `bar`; false if it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (unsigned k = 0; k < (1u << 22); ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Shared-memory stage of one tile of FP32 survivors: id (8 B), then x, ox,
// nu, w, key (, y, oy (, z, oz)) (4 B each), `tile` entries per array.
template <int DIM>
struct StageF {
  static constexpr int kArr4 = 5 + (DIM >= 2 ? 2 : 0) + (DIM == 3 ? 2 : 0);
  static constexpr int kBytesPer = 8 + 4 * kArr4;
  unsigned long long* id;
  float *x, *ox, *nu, *w, *y, *oy, *z, *oz;
  uint32_t* key;
  __device__ __forceinline__ StageF(unsigned char* base, int tile) {
    id = reinterpret_cast<unsigned long long*>(base);
    float* f = reinterpret_cast<float*>(base + 8 * (size_t)tile);
    x = f; ox = f + tile; nu = f + 2 * tile; w = f + 3 * tile;
    key = reinterpret_cast<uint32_t*>(f + 4 * tile);
    y = f + 5 * tile; oy = f + 6 * tile; z = f + 7 * tile; oz = f + 8 * tile;
  }
};

constexpr int kStages = 3;          // shared-memory stages of the FP32 kernel
constexpr int kSmemCells = 4096;    // per-cell opacity factors held in shared memory up to this many cells

static size_t stream32_stage_bytes(int dim, int tile) {
  const int per = dim == 3 ? StageF<3>::kBytesPer : (dim == 2 ? StageF<2>::kBytesPer : StageF<1>::kBytesPer);
  return (size_t)tile * per;
}

// Shared-memory opacity table of a single problem: 1/(sigma0 T^q) per cell,
// then 1/T per cell for the photo-ionisation law; none for the foam law or
// grids above kSmemCells.
static int stream32_table_floats(const Dev& d) {
  if (d.sig_law == 2 || d.ncell > kSmemCells) return 0;
  return d.ncell * (d.sig_law == 1 && !d.grey ? 2 : 1);
}

// The survivor kernel's table: 1/(sigma0 T^q) per cell, then every 32nd
// birth offset (off[32 s], the segments the newborns' bin search starts
// from) when there are at most kSegMax of them.
constexpr int kSegMax = 1024;
__host__ __device__ inline int fast_segments(int nbins) {
  const int ns = (nbins + 31) / 32;
  return ns <= kSegMax ? ns : 0;
}
__host__ __device__ inline size_t fast_table_bytes(int ncell, int nbins) {
  return (4 * (size_t)ncell + 4 * (size_t)fast_segments(nbins) + 127) & ~(size_t)127;
}

struct Counters {   // per thread; a thread sees far fewer than 2^32 events
  unsigned seg = 0, abs = 0, esc = 0, surv = 0, rem = 0;
};

__device__ __forceinline__ void flush_counters(Ctrl* ctrl, Counters& c) {
  const unsigned long long seg = warp_sum_u64(c.seg), abs = warp_sum_u64(c.abs), esc = warp_sum_u64(c.esc);
  const unsigned long long surv = warp_sum_u64(c.surv), rem = warp_sum_u64(c.rem);
  if ((threadIdx.x & 31) == 0) {
    if (seg) atomicAdd(&ctrl->n_segments, seg);
    if (abs) atomicAdd(&ctrl->n_absorbed, abs);
    if (esc) atomicAdd(&ctrl->n_escaped, esc);
    if (surv) atomicAdd(&ctrl->n_survived, surv);
    if (rem) atomicAdd(&ctrl->n_removed, rem);
  }
  c = Counters();
}

// The same once per block: the warps' sums meet in shared memory and one
// thread adds them to the control block (many warps adding to the same five
// words serialise at the L2).  Every thread of the block must call it.
__device__ __forceinline__ void flush_counters_block(Ctrl* ctrl, Counters& c) {
  __shared__ unsigned long long s_c[5];
  if (threadIdx.x < 5) s_c[threadIdx.x] = 0ull;
  __syncthreads();
  const unsigned long long seg = warp_sum_u64(c.seg), abs = warp_sum_u64(c.abs), esc = warp_sum_u64(c.esc);
  const unsigned long long surv = warp_sum_u64(c.surv), rem = warp_sum_u64(c.rem);
  if ((threadIdx.x & 31) == 0) {
    if (seg) atomicAdd(&s_c[0], seg);
    if (abs) atomicAdd(&s_c[1], abs);
    if (esc) atomicAdd(&s_c[2], esc);
    if (surv) atomicAdd(&s_c[3], surv);
    if (rem) atomicAdd(&s_c[4], rem);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_c[0]) atomicAdd(&ctrl->n_segments, s_c[0]);
    if (s_c[1]) atomicAdd(&ctrl->n_absorbed, s_c[1]);
    if (s_c[2]) atomicAdd(&ctrl->n_escaped, s_c[2]);
    if (s_c[3]) atomicAdd(&ctrl->n_survived, s_c[3]);
    if (s_c[4]) atomicAdd(&ctrl->n_removed, s_c[4]);
  }
  c = Counters();
}

// Step-constant fields of a single problem's control block, read once per
// thread.
struct StepHead {
  unsigned cur;
  long long n_surv, n_tot;
  uint32_t step;
};

__device__ __forceinline__ StepHead step_head(const Dev& d) {
  const Ctrl* c = d.ctrl;
  StepHead h;
  h.cur = c->cur;
  h.n_surv = (long long)c->n_part[h.cur];
  h.n_tot = h.n_surv + (long long)c->n_new;
  h.step = (uint32_t)c->step;
  return h;
}

__device__ __forceinline__ long long tiles_of(const Dev& d, long long tile) {
  const Ctrl* ctrl = d.ctrl;
  const long long n = (long long)ctrl->n_part[ctrl->cur] + (long long)ctrl->n_new;
  return (n + tile - 1) / tile;
}

template <int DIM, bool ENS, int PPT>
__global__ void __launch_bounds__(512, 1) k_stream64(const __grid_constant__ Dev d0, const Ens e) {
  Counters cnt;
  int acc_m = 0;
  const long long tile = (long long)blockDim.x * PPT;   // PPT sub-tiles of one particle per thread
  const long long ntiles = ENS ? (long long)e.tile0[e.M] : tiles_of(d0, tile);
  const StepHead h0 = ENS ? StepHead{} : step_head(d0);
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
  const int m = ENS ? find_member(e.tile0, e.M, t) : 0;
  if (ENS && m != acc_m) { flush_counters(e.devs[acc_m].ctrl, cnt); acc_m = m; }
  const Dev& d = ENS ? e.devs[m] : d0;
  const long long lt = ENS ? t - (long long)e.tile0[m] : t;
  Ctrl* ctrl = d.ctrl;
  const unsigned cur = ENS ? ctrl->cur : h0.cur, nxb = cur ^ 1u;
  const long long n_surv = ENS ? (long long)ctrl->n_part[cur] : h0.n_surv;
  const long long n_tot = ENS ? n_surv + (long long)ctrl->n_new : h0.n_tot;
  const uint32_t step = ENS ? (uint32_t)ctrl->step : h0.step;
  const int G = d.G, nx = d.nx, ny = DIM >= 2 ? d.ny : 1, nz = DIM == 3 ? d.nz : 1;
  const double v = d.v, dt = d.dt, inv_rate = d.eps * d.eps / d.c;
  const double* __restrict__ in_x = d.px[cur];
  const double* __restrict__ in_y = d.py[cur];
  const double* __restrict__ in_ox = d.pox[cur];
  const double* __restrict__ in_oy = d.poy[cur];
  const double* __restrict__ in_z = d.pz[cur];
  const double* __restrict__ in_oz = d.poz[cur];
  const double* __restrict__ in_nu = d.pnu[cur];
  const double* __restrict__ in_w = d.pw[cur];
  const unsigned long long* __restrict__ in_id = d.pid[cur];
  const uint32_t* __restrict__ in_key = d.pkey[cur];
  for (int sub = 0; sub < PPT; ++sub) {
    const long long i = lt * tile + (long long)sub * blockDim.x + threadIdx.x;
    const bool valid = i < n_tot;
    double x = 0.0, y = 0.0, z = 0.0, ox = 0.0, oy = 0.0, oz = 0.0, nu = 0.0, w = 0.0;
    unsigned long long id = 0ull;
    int cell = 0, g = 0, gside = -1;
    bool newborn = false;
    Draws rng;
    rng.init(0ull, step, 0u);
    if (valid) {
      if (i < n_surv) {
        x = in_x[i];
        ox = in_ox[i];
        if (DIM >= 2) { y = in_y[i]; oy = in_oy[i]; }
        if (DIM == 3) { z = in_z[i]; oz = in_oz[i]; }
        nu = in_nu[i];
        w = in_w[i];
        id = in_id[i];
        const uint32_t key = in_key[i];
        cell = (int)div_bin(d, key);
        g = (int)(key - (uint32_t)cell * (uint32_t)G);
        rng.init(id, step, 0u);
      } else {
        newborn = true;
        const uint32_t j = (uint32_t)(i - n_surv);
        const int bin = find_bin(d.off, d.nbins, j);
        const uint32_t k = j - __ldg(d.off + bin);
        id = ((unsigned long long)step << kIdStepShift) | ((unsigned long long)bin << kIdBinShift) |
             (unsigned long long)k;
        rng.init(id, step, 0u);
        const int cb = (int)div_bin(d, (uint32_t)bin);
        g = bin - cb * G;
        double Tb;
        if (cb < d.ncell) {
          int cx, cy, cz = 0;
          if (DIM == 3) {
            cz = cb / (nx * ny);
            const int rem = cb - cz * nx * ny;
            cy = rem / nx;
            cx = rem - cy * nx;
          } else {
            cy = DIM == 2 ? (int)div_nx(d, (uint32_t)cb) : 0;
            cx = cb - cy * nx;
          }
          x = cx * d.dx + rng.next(d.pk) * d.dx;
          if (DIM >= 2) y = cy * d.dy + rng.next(d.pk) * d.dy;
          if (DIM == 3) z = cz * d.dz + rng.next(d.pk) * d.dz;
          if (DIM == 1) {
            ox = 2.0 * rng.next(d.pk) - 1.0;
          } else {
            const double muz = 2.0 * rng.next(d.pk) - 1.0;
            const double ph = rng.next(d.pk);
            double sp, cp;
            sincospi(2.0 * ph, &sp, &cp);
            const double s = sqrt(fmax(0.0, 1.0 - muz * muz));
            ox = s * cp;
            oy = s * sp;
            if (DIM == 3) oz = muz;
          }
          cell = cb;
          Tb = d.T[cb];
        } else {
          // black-body ghost (1D): the entering set, mu ~ 2 mu dmu, distance
          // uniform within reach v mu dt
          const int side = cb - d.ncell;
          const double u = rng.next(d.pk);
          const double m = sqrt(rng.next(d.pk));
          const double dd = u * v * m * dt;
          x = side == 0 ? -dd : nx * d.dx + dd;
          ox = side == 0 ? m : -m;
          cell = side == 0 ? -1 : nx;
          gside = side;
          Tb = d.bcT[side];
        }
        (void)Tb;
        if (!d.grey)
          nu = sample_nu(d.nu_edges[g], d.nu_edges[g + 1], __ldg(d.khat + bin), rng.next(d.pk));
        w = __ldg(d.omega + bin);
      }
    }

    // ---- streaming
    int fate = FATE_REMOVED, nseg = 0, eside = -1;
    const int cell0 = cell;
    double t_tra = 0.0;
    if (valid) {
      const double inup = d.grey ? 1.0 : pow_fast(nu, -d.sig_p);
      double t_rem;
      bool collided;
      if (newborn && (d.method == 0 || gside >= 0)) {   // UGKP newborns draw t_f too
        t_rem = dt;
        collided = false;
      } else {
        const double u = rng.next(d.pk);
        const double sig_inv = inv_sigma_particle(d, cell, nu, inup);
        const double tc = neg_log_u64(u) * inv_rate * sig_inv;
        collided = tc < dt;
        t_rem = collided ? tc : dt;
      }
      bool ghost = gside >= 0;
      int cx, cy, cz = 0;
      if (DIM == 3) {
        cz = cell / (nx * ny);
        const int rem = cell - cz * nx * ny;
        cy = rem / nx;
        cx = rem - cy * nx;
      } else {
        cy = DIM == 2 ? (int)div_nx(d, (uint32_t)cell) : 0;
        cx = DIM == 2 ? cell - cy * nx : cell;
      }
      const double ivx = ox != 0.0 ? 1.0 / (v * fabs(ox)) : 0.0;
      const double ivy = (DIM >= 2 && oy != 0.0) ? 1.0 / (v * fabs(oy)) : 0.0;
      const double ivz = (DIM == 3 && oz != 0.0) ? 1.0 / (v * fabs(oz)) : 0.0;
      for (int guard = 0;; ++guard) {
        if (guard >= 4096) {            // defensive bound (NaN state)
          atomicOr(&ctrl->status, ST_NONFINITE);
          fate = FATE_REMOVED;
          break;
        }
        const double xL = cx * d.dx, xR = (cx + 1) * d.dx;
        double tx = INFINITY, ty = INFINITY;
        if (ox > 0.0) tx = fmax(xR - x, 0.0) * ivx;
        else if (ox < 0.0) tx = fmax(x - xL, 0.0) * ivx;
        double yB = 0.0, yT = 0.0, zB = 0.0, zT = 0.0, tz = INFINITY;
        if (DIM >= 2) {
          yB = cy * d.dy;
          yT = (cy + 1) * d.dy;
          if (oy > 0.0) ty = fmax(yT - y, 0.0) * ivy;
          else if (oy < 0.0) ty = fmax(y - yB, 0.0) * ivy;
        }
        if (DIM == 3) {
          zB = cz * d.dz;
          zT = (cz + 1) * d.dz;
          if (oz > 0.0) tz = fmax(zT - z, 0.0) * ivz;
          else if (oz < 0.0) tz = fmax(z - zB, 0.0) * ivz;
        }
        // nearest face; ties go to the lower axis
        int axis = (tx <= ty) ? 0 : 1;
        double tf = axis == 0 ? tx : ty;
        if (DIM == 3 && tz < tf) { axis = 2; tf = tz; }
        if (tf < t_rem) {
          ++nseg;
          t_tra += tf;
          t_rem -= tf;
          int dir;
          if (axis == 0) {
            dir = ox > 0.0 ? 1 : -1;
            x = dir > 0 ? xR : xL;
            if (DIM >= 2) y += v * oy * tf;
            if (DIM == 3) z += v * oz * tf;
          } else if (DIM < 3 || axis == 1) {
            dir = oy > 0.0 ? 1 : -1;
            y = dir > 0 ? yT : yB;
            x += v * ox * tf;
            if (DIM == 3) z += v * oz * tf;
          } else {
            dir = oz > 0.0 ? 1 : -1;
            z = dir > 0 ? zT : zB;
            x += v * ox * tf;
            y += v * oy * tf;
          }
          const int nxc = cx + (axis == 0 ? dir : 0), nyc = cy + (axis == 1 ? dir : 0);
          const int nzc = cz + (axis == 2 ? dir : 0);
          if (nxc < 0 || nxc >= nx || nyc < 0 || nyc >= ny || (DIM == 3 && (nzc < 0 || nzc >= nz))) {
            const int side = axis * 2 + (dir > 0 ? 1 : 0);
            if (d.bc[side] == BC_REFLECT) {
              if (axis == 0) ox = -ox; else if (axis == 1) oy = -oy; else oz = -oz;
              continue;
            }
            fate = FATE_ESCAPED;
            eside = side;
            break;
          }
          ghost = false;
          cx = nxc;
          cy = nyc;
          cz = nzc;
          cell = (cz * ny + cy) * nx + cx;
          const double u = rng.next(d.pk);
          const double sig_inv = inv_sigma_particle(d, cell, nu, inup);
          const double tc = neg_log_u64(u) * inv_rate * sig_inv;
          const double avail = dt - t_tra;
          collided = tc < avail;
          t_rem = collided ? tc : avail;
          continue;
        }
        ++nseg;
        x += v * ox * t_rem;
        if (DIM >= 2) y += v * oy * t_rem;
        if (DIM == 3) z += v * oz * t_rem;
        t_tra += t_rem;
        t_rem = 0.0;
        fate = ghost ? FATE_REMOVED : (collided ? FATE_ABSORBED : FATE_SURVIVED);
        break;
      }
    }

    // ---- in place: slot i of the other buffer (kDeadKey unless it survived)
    const bool keep = valid && fate == FATE_SURVIVED;
    const bool room = i < d.capacity;
    const bool stored = keep && room;
    if (valid && room) {
      d.px[nxb][i] = x;
      d.pox[nxb][i] = ox;
      if (DIM >= 2) { d.py[nxb][i] = y; d.poy[nxb][i] = oy; }
      if (DIM == 3) { d.pz[nxb][i] = z; d.poz[nxb][i] = oz; }
      d.pnu[nxb][i] = nu;
      d.pw[nxb][i] = w;
      d.pid[nxb][i] = id;
      d.pkey[nxb][i] = stored ? (uint32_t)(cell * G + g) : kDeadKey;
    }
    if (keep && !room) atomicOr(&ctrl->status, ST_CAPACITY);

    // ---- tallies (W and E_surv in fixed point, see to_fixed).  A survivor
    // that found no slot is counted in W but not in E_surv: its energy stays
    // with the wave part.
    const int lane = threadIdx.x & 31;
    const long long wq = valid ? to_fixed(w, d.tq_inv, &ctrl->status) : 0ll;
    warp_run_add_fixed(d.Esq, stored ? cell * G + g : -1 - lane, wq, d.sort_cnt);
    if (valid && fate != FATE_REMOVED) {
      const bool start_in = gside < 0;
      const bool end_in = fate == FATE_SURVIVED || fate == FATE_ABSORBED;
      if (!(start_in && end_in && cell0 == cell)) {
        if (start_in) atomic_add_fixed(d.Wq + 2 * (cell0 * G + g), -wq);
        if (end_in) atomic_add_fixed(d.Wq + 2 * (cell * G + g), wq);
      }
      if (!start_in) atomicAdd(d.inflow + gside * G + g, w);
      if (fate == FATE_ESCAPED) atomicAdd(d.esc + eside * G + g, w);
    }
    if (valid) {
      cnt.seg += (unsigned)nseg;
      cnt.abs += fate == FATE_ABSORBED;
      cnt.esc += fate == FATE_ESCAPED;
      cnt.surv += fate == FATE_SURVIVED;
      cnt.rem += fate == FATE_REMOVED;
      if (d.rec && i < d.rec_cap) {
        RecordOut& r = d.rec[i];
        r.id = id; r.fate = fate; r.cell0 = cell0; r.cell1 = cell; r.grp = g; r.nseg = nseg; r.pad = 0;
        r.x = x; r.y = y; r.ox = ox; r.oy = oy; r.nu = nu; r.w = w; r.t_end = t_tra;
        r.z = z; r.oz = oz;
      }
    }
    // adjoint tape: where this particle's weight was counted (its slot in the
    // next step's input is filled in by the survivor sort)
    if (!ENS && d.tape && valid) {
      if (i < d.tape_cap) {
        TapeRec tr;
        tr.c0 = gside >= 0 ? -1 - gside : cell0;
        tr.c1 = (fate == FATE_SURVIVED || fate == FATE_ABSORBED) ? cell : -1;
        tr.slot = -1;
        tr.g = g;
        tr.w = w;
        d.tape[i] = tr;
      } else {
        atomicOr(&ctrl->status, ST_CAPACITY);
      }
    }
  }
  }
  flush_counters(ENS ? e.devs[acc_m].ctrl : d0.ctrl, cnt);
}

// --------------------------------------------------------------------------
// Mixed precision (FP32 particle state and arithmetic, fixed-point tallies):
// the same algorithm as k_stream64 with positions held relative to the cell
// (0 <= xi <= dx) and FP32 uniforms from the same Philox words.  A survivor
// costs 28 B read and 28 B written in 1D.
//
// A warp streams chunks of 32 x rounds consecutive particles (so its lanes
// share bins and its stores are whole 128-byte lines).

// State of one particle in the FP32 kernel.
struct P32 {
  float xi, eta, zeta, ox, oy, oz, nu, w, t_rem, t_tra;
  unsigned long long id;
  int cx, cy, cz, g, gside, fate, nseg, eside, cell0;
  bool collided, ghost, newborn;
};

// 1/sigma(nu, T^n) of a particle in cell c: the per-cell factors from shared
// memory when the problem's table is there (tab_n > 0), else from the device
__device__ __forceinline__ float inv_sigma32(const Dev& d, int c, float nu, float inup, int tab_n,
                                             bool tab_invT, const float* s_sinv, const float* s_invT) {
  if (tab_n) {
    float si = s_sinv[c] * inup;
    if (tab_invT) si /= -expm1f(-nu * s_invT[c]);
    return fmaxf(si, d.inv_capf);
  }
  return inv_sigma_particle_f(d, c, nu, inup);
}

// The streaming loop from a particle's current state (free time t_rem in its
// cell) to the end of the step: faces crossed with the free time reset,
// reflections, escapes, the final flight.
template <int DIM>
__device__ __forceinline__ void stream_loop32(const Dev& d, P32& q, DrawsF& rng, float inup, int tab_n,
                                              bool tab_invT, const float* s_sinv, const float* s_invT) {
  const int nx = d.nx, ny = DIM >= 2 ? d.ny : 1, nz = DIM == 3 ? d.nz : 1;
  const float dxf = d.dxf, dyf = d.dyf, dzf = d.dzf, vf = d.vf, dtf = d.dtf, inv_rate = d.inv_rate_f;
  const float ivx = q.ox != 0.0f ? __frcp_rn(vf * fabsf(q.ox)) : 0.0f;
  const float ivy = (DIM >= 2 && q.oy != 0.0f) ? __frcp_rn(vf * fabsf(q.oy)) : 0.0f;
  const float ivz = (DIM == 3 && q.oz != 0.0f) ? __frcp_rn(vf * fabsf(q.oz)) : 0.0f;
  for (int guard = 0;; ++guard) {
    if (guard >= 4096) {
      atomicOr(&d.ctrl->status, ST_NONFINITE);
      q.fate = FATE_REMOVED;
      break;
    }
    float tx = INFINITY, ty = INFINITY, tz = INFINITY;
    if (q.ox > 0.0f) tx = fmaxf(dxf - q.xi, 0.0f) * ivx;
    else if (q.ox < 0.0f) tx = fmaxf(q.xi, 0.0f) * ivx;
    if (DIM >= 2) {
      if (q.oy > 0.0f) ty = fmaxf(dyf - q.eta, 0.0f) * ivy;
      else if (q.oy < 0.0f) ty = fmaxf(q.eta, 0.0f) * ivy;
    }
    if (DIM == 3) {
      if (q.oz > 0.0f) tz = fmaxf(dzf - q.zeta, 0.0f) * ivz;
      else if (q.oz < 0.0f) tz = fmaxf(q.zeta, 0.0f) * ivz;
    }
    // nearest face; ties go to the lower axis
    int axis = (tx <= ty) ? 0 : 1;
    float tf = axis == 0 ? tx : ty;
    if (DIM == 3 && tz < tf) { axis = 2; tf = tz; }
    if (tf < q.t_rem) {
      ++q.nseg;
      q.t_tra += tf;
      q.t_rem -= tf;
      int dir;
      if (axis == 0) {
        dir = q.ox > 0.0f ? 1 : -1;
        q.xi = dir > 0 ? dxf : 0.0f;
        if (DIM >= 2) q.eta = fminf(fmaxf(fmaf(vf * q.oy, tf, q.eta), 0.0f), dyf);
        if (DIM == 3) q.zeta = fminf(fmaxf(fmaf(vf * q.oz, tf, q.zeta), 0.0f), dzf);
      } else if (DIM < 3 || axis == 1) {
        dir = q.oy > 0.0f ? 1 : -1;
        q.eta = dir > 0 ? dyf : 0.0f;
        q.xi = fminf(fmaxf(fmaf(vf * q.ox, tf, q.xi), 0.0f), dxf);
        if (DIM == 3) q.zeta = fminf(fmaxf(fmaf(vf * q.oz, tf, q.zeta), 0.0f), dzf);
      } else {
        dir = q.oz > 0.0f ? 1 : -1;
        q.zeta = dir > 0 ? dzf : 0.0f;
        q.xi = fminf(fmaxf(fmaf(vf * q.ox, tf, q.xi), 0.0f), dxf);
        q.eta = fminf(fmaxf(fmaf(vf * q.oy, tf, q.eta), 0.0f), dyf);
      }
      const int nxc = q.cx + (axis == 0 ? dir : 0), nyc = q.cy + (axis == 1 ? dir : 0);
      const int nzc = q.cz + (axis == 2 ? dir : 0);
      if (nxc < 0 || nxc >= nx || nyc < 0 || nyc >= ny || (DIM == 3 && (nzc < 0 || nzc >= nz))) {
        const int side = axis * 2 + (dir > 0 ? 1 : 0);
        if (d.bc[side] == BC_REFLECT) {
          if (axis == 0) q.ox = -q.ox; else if (axis == 1) q.oy = -q.oy; else q.oz = -q.oz;
          continue;
        }
        q.fate = FATE_ESCAPED;
        q.eside = side;
        break;
      }
      q.ghost = false;
      if (axis == 0) q.xi = dir > 0 ? 0.0f : dxf;
      else if (axis == 1) q.eta = dir > 0 ? 0.0f : dyf;
      else q.zeta = dir > 0 ? 0.0f : dzf;
      q.cx = nxc;
      q.cy = nyc;
      q.cz = nzc;
      const UPair u = rng.next2(d.pk);
      const float sig_inv = inv_sigma32(d, (q.cz * ny + q.cy) * nx + q.cx, q.nu, inup, tab_n, tab_invT, s_sinv, s_invT);
      const float tc = neg_log_u(u) * inv_rate * sig_inv;
      const float avail = dtf - q.t_tra;
      q.collided = tc < avail;
      q.t_rem = q.collided ? tc : avail;
      continue;
    }
    ++q.nseg;
    q.xi = fminf(fmaxf(fmaf(vf * q.ox, q.t_rem, q.xi), 0.0f), dxf);
    if (DIM >= 2) q.eta = fminf(fmaxf(fmaf(vf * q.oy, q.t_rem, q.eta), 0.0f), dyf);
    if (DIM == 3) q.zeta = fminf(fmaxf(fmaf(vf * q.oz, q.t_rem, q.zeta), 0.0f), dzf);
    q.t_tra += q.t_rem;
    q.fate = q.ghost ? FATE_REMOVED : (q.collided ? FATE_ABSORBED : FATE_SURVIVED);
    break;
  }
}

// The W and side tallies of a particle that changed cell, entered from a
// ghost or escaped (end minus start of Eq. wfrpFormula; FP64 side tallies).
__device__ __forceinline__ void cross_tallies32(const Dev& d, const P32& q, int cell, long long wq) {
  if (q.fate != FATE_REMOVED && (q.gside >= 0 || q.fate == FATE_ESCAPED || q.cell0 != cell)) {
    const int G = d.G;
    const double wd = (double)q.w;
    const bool start_in = q.gside < 0;
    const bool end_in = q.fate == FATE_SURVIVED || q.fate == FATE_ABSORBED;
    if (start_in) atomic_add_fixed(d.Wq + 2 * (q.cell0 * G + q.g), -wq);
    if (end_in) atomic_add_fixed(d.Wq + 2 * (cell * G + q.g), wq);
    if (!start_in) atomicAdd(d.inflow + q.gside * G + q.g, wd);
    if (q.fate == FATE_ESCAPED) atomicAdd(d.esc + q.eside * G + q.g, wd);
  }
}

template <int DIM>
__device__ __forceinline__ void record32(const Dev& d, const P32& q, long long i, int cell) {
  if (d.rec && i < d.rec_cap) {
    RecordOut& rr = d.rec[i];
    rr.id = q.id; rr.fate = q.fate; rr.cell0 = q.cell0;
    rr.cell1 = (q.fate == FATE_REMOVED && q.gside >= 0) ? q.cx : cell;
    rr.grp = q.g; rr.nseg = q.nseg; rr.pad = 0;
    rr.x = q.cx * d.dx + (double)q.xi;
    rr.y = DIM >= 2 ? q.cy * d.dy + (double)q.eta : 0.0;
    rr.ox = q.ox; rr.oy = q.oy; rr.nu = q.nu; rr.w = (double)q.w; rr.t_end = q.t_tra;
    rr.z = DIM == 3 ? q.cz * d.dz + (double)q.zeta : 0.0;
    rr.oz = q.oz;
  }
}

// Slot i of the other buffer (kDeadKey unless the particle survived); false
// for a survivor that found no slot (counted in W but not in E_surv: its
// energy stays with the wave part).
template <int DIM>
__device__ __forceinline__ bool store32(const Dev& d, unsigned nxb, const P32& q, long long i, int cell) {
  const bool keep = q.fate == FATE_SURVIVED;
  if (i >= d.capacity) {
    if (keep) atomicOr(&d.ctrl->status, ST_CAPACITY);
    return false;
  }
  d.fx[nxb][i] = q.xi;
  d.fox[nxb][i] = q.ox;
  if (DIM >= 2) { d.fy[nxb][i] = q.eta; d.foy[nxb][i] = q.oy; }
  if (DIM == 3) { d.fz[nxb][i] = q.zeta; d.foz[nxb][i] = q.oz; }
  d.fnu[nxb][i] = q.nu;
  d.fw[nxb][i] = q.w;
  d.pid[nxb][i] = q.id;
  d.pkey[nxb][i] = keep ? (uint32_t)(cell * d.G + q.g) : kDeadKey;
  return keep;
}

// A newborn of the virtual index j = i - n_surv (Eq. IhpFormula): its bin
// from the birth scan, identity, position uniform in its cell (or, in a
// black-body ghost, the entering set), isotropic direction, frequency by
// the linear sampler (App. A) and weight.
template <int DIM>
__device__ __forceinline__ void birth32_in(const Dev& d, P32& q, DrawsF& rng, uint32_t j, uint32_t step,
                                          int bin, uint32_t off_bin) {
  const int G = d.G, nx = d.nx, ny = DIM >= 2 ? d.ny : 1;
  q.newborn = true;
  const uint32_t kk = j - off_bin;
  q.id = ((unsigned long long)step << kIdStepShift) | ((unsigned long long)bin << kIdBinShift) |
         (unsigned long long)kk;
  rng.init(q.id, step, 0u);
  const int cb = (int)div_bin(d, (uint32_t)bin);
  q.g = bin - cb * G;
  if (cb < d.ncell) {
    if (DIM == 3) {
      q.cz = cb / (nx * ny);
      const int rem = cb - q.cz * nx * ny;
      q.cy = rem / nx;
      q.cx = rem - q.cy * nx;
    } else {
      q.cy = DIM == 2 ? (int)div_nx(d, (uint32_t)cb) : 0;
      q.cx = cb - q.cy * nx;
    }
    q.xi = rng.next(d.pk) * d.dxf;
    if (DIM >= 2) q.eta = rng.next(d.pk) * d.dyf;
    if (DIM == 3) q.zeta = rng.next(d.pk) * d.dzf;
    if (DIM == 1) {
      q.ox = 2.0f * rng.next(d.pk) - 1.0f;
    } else {
      const float muz = 2.0f * rng.next(d.pk) - 1.0f;
      const float ph = rng.next(d.pk);
      float sp, cp;
      sincospif(2.0f * ph, &sp, &cp);
      const float sq = sqrtf(fmaxf(0.0f, 1.0f - muz * muz));
      q.ox = sq * cp;
      q.oy = sq * sp;
      if (DIM == 3) q.oz = muz;
    }
  } else {
    const int side = cb - d.ncell;
    const float u = rng.next(d.pk);
    const float mm = sqrtf(rng.next(d.pk));
    const float dd = u * d.vf * mm * d.dtf;
    q.cx = side == 0 ? -1 : nx;
    q.xi = side == 0 ? d.dxf - dd : dd;
    q.ox = side == 0 ? mm : -mm;
    q.gside = side;
  }
  if (!d.grey)
    q.nu = sample_nu_f(__ldg(d.nu_edges_f + q.g), __ldg(d.nu_edges_f + q.g + 1), __ldg(d.khat_f + bin),
                       rng.next(d.pk));
  q.w = __ldg(d.omega_f + bin);
}

template <int DIM>
__device__ __forceinline__ void birth32(const Dev& d, P32& q, DrawsF& rng, uint32_t j, uint32_t step,
                                       const uint32_t* off) {
  int lo = 0, hi = d.nbins;   // largest bin with off[bin] <= j
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= j) lo = mid; else hi = mid;
  }
  birth32_in<DIM>(d, q, rng, j, step, lo, off[lo]);
}

// Birth bins of a warp's 32 consecutive ordinals j (lanes with `need`): the
// largest bin with off[bin] <= j.  The segment of 32 bins holding it comes
// from a table of every 32nd offset (s_seg, ns entries, in shared memory);
// then the warp loads one segment's 32 offsets at a time (a segment that
// some unresolved lane needs) and each of its lanes finds its bin among them
// by a five-step search over the warp's registers.  Consecutive ordinals
// share segments, so a warp usually loads one or two.
__device__ __forceinline__ int birth_bin32(const Dev& d, const uint32_t* s_seg, int ns, uint32_t j, bool need,
                                          uint32_t* off_bin) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = ns;   // largest segment s with off[32 s] <= j
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (s_seg[mid] <= j) lo = mid; else hi = mid;
  }
  const int seg = lo;
  int bin = 0;
  uint32_t ob = 0u;
  unsigned pend = __ballot_sync(full, need);
  while (pend) {
    const int s = __shfl_sync(full, seg, __ffs(pend) - 1);
    const int b = 32 * s + lane;
    const uint32_t o = b < d.nbins ? __ldg(d.off + b) : 0xffffffffu;
    int t = 0;   // largest t with o_t <= j (o_0 <= j for the lanes of this segment)
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
      const uint32_t ov = __shfl_sync(full, o, t + step);
      if (ov <= j) t += step;
    }
    const uint32_t ot = __shfl_sync(full, o, t);
    if (need && seg == s) {
      bin = 32 * s + t;
      ob = ot;
      need = false;
    }
    pend = __ballot_sync(full, need);
  }
  *off_bin = ob;
  return bin;
}

// Cell coordinates of a survivor from its bin key (cell c * G + group g).
template <int DIM>
__device__ __forceinline__ void decode_key32(const Dev& d, uint32_t key, P32& q) {
  const int nx = d.nx, ny = DIM >= 2 ? d.ny : 1;
  if (key >= (uint32_t)d.nbins) key = 0u;   // only after a failed wait (flagged): stay in range
  const int cell = (int)div_bin(d, key);
  q.g = (int)(key - (uint32_t)cell * (uint32_t)d.G);
  if (DIM == 3) {
    q.cz = cell / (nx * ny);
    const int rem = cell - q.cz * nx * ny;
    q.cy = rem / nx;
    q.cx = rem - q.cy * nx;
  } else {
    q.cy = DIM == 2 ? (int)div_nx(d, (uint32_t)cell) : 0;
    q.cx = cell - q.cy * nx;
  }
}

__device__ __forceinline__ void clear32(P32& q) {
  q.xi = q.eta = q.zeta = q.ox = q.oy = q.oz = q.nu = q.w = 0.f;
  q.t_rem = q.t_tra = 0.0f;
  q.id = 0ull;
  q.cx = q.cy = q.cz = q.g = 0;
  q.gside = -1;
  q.newborn = false;
  q.collided = false;
  q.fate = FATE_REMOVED;
  q.nseg = 0;
  q.eside = -1;
}

// Free time of the particle in its cell (a survivor draws it; a UGKWP
// newborn has t_f = dt) and its first flight: if that flight ends the step
// (no face first), finish it and return false; else return true with t_rem
// and collided set for stream_loop32 (the same arithmetic as its first pass).
template <int DIM>
__device__ __forceinline__ bool first_flight32(const Dev& d, P32& q, DrawsF& rng, float inup, int tab_n,
                                               bool tab_invT, const float* s_sinv, const float* s_invT) {
  const int nx = d.nx, ny = DIM >= 2 ? d.ny : 1;
  const float dxf = d.dxf, dyf = d.dyf, dzf = d.dzf, vf = d.vf, dtf = d.dtf;
  if (q.newborn && (d.method == 0 || q.gside >= 0)) {   // UGKP newborns draw t_f too
    q.t_rem = dtf;
    q.collided = false;
  } else {
    const UPair u = rng.next2(d.pk);
    const float sig_inv = inv_sigma32(d, (q.cz * ny + q.cy) * nx + q.cx, q.nu, inup, tab_n, tab_invT, s_sinv, s_invT);
    const float tc = neg_log_u(u) * d.inv_rate_f * sig_inv;
    q.collided = tc < dtf;
    q.t_rem = q.collided ? tc : dtf;
  }
  const float ivx = q.ox != 0.0f ? __frcp_rn(vf * fabsf(q.ox)) : 0.0f;
  const float ivy = (DIM >= 2 && q.oy != 0.0f) ? __frcp_rn(vf * fabsf(q.oy)) : 0.0f;
  const float ivz = (DIM == 3 && q.oz != 0.0f) ? __frcp_rn(vf * fabsf(q.oz)) : 0.0f;
  float tx = INFINITY, ty = INFINITY, tz = INFINITY;
  if (q.ox > 0.0f) tx = fmaxf(dxf - q.xi, 0.0f) * ivx;
  else if (q.ox < 0.0f) tx = fmaxf(q.xi, 0.0f) * ivx;
  if (DIM >= 2) {
    if (q.oy > 0.0f) ty = fmaxf(dyf - q.eta, 0.0f) * ivy;
    else if (q.oy < 0.0f) ty = fmaxf(q.eta, 0.0f) * ivy;
  }
  if (DIM == 3) {
    if (q.oz > 0.0f) tz = fmaxf(dzf - q.zeta, 0.0f) * ivz;
    else if (q.oz < 0.0f) tz = fmaxf(q.zeta, 0.0f) * ivz;
  }
  const float tf = fminf(fminf(tx, ty), tz);
  if (tf < q.t_rem) return true;
  q.nseg = 1;
  q.xi = fminf(fmaxf(fmaf(vf * q.ox, q.t_rem, q.xi), 0.0f), dxf);
  if (DIM >= 2) q.eta = fminf(fmaxf(fmaf(vf * q.oy, q.t_rem, q.eta), 0.0f), dyf);
  if (DIM == 3) q.zeta = fminf(fmaxf(fmaf(vf * q.oz, q.t_rem, q.zeta), 0.0f), dzf);
  q.t_tra = q.t_rem;
  q.fate = q.ghost ? FATE_REMOVED : (q.collided ? FATE_ABSORBED : FATE_SURVIVED);
  return false;
}

// Shared set-up of the FP32 kernels of a single problem: the per-cell opacity
// factors in shared memory (when they fit) at the start of the dynamic area.
struct Tab32 {
  int n;
  bool invT;
  float *sinv, *sinvT;
};

template <bool ENS>
__device__ __forceinline__ Tab32 load_tab32(const Dev& d0, unsigned char* s_dyn) {
  Tab32 t;
  t.n = ENS ? 0 : ((d0.sig_law == 2 || d0.ncell > kSmemCells) ? 0 : d0.ncell);
  t.invT = !ENS && t.n && d0.sig_law == 1 && !d0.grey;
  t.sinv = reinterpret_cast<float*>(s_dyn);
  t.sinvT = t.sinv + t.n;
  if (!ENS) {
    for (int c = threadIdx.x; c < t.n; c += blockDim.x) {
      t.sinv[c] = __ldg(d0.sTinv_f + c);
      if (t.invT) t.sinvT[c] = __ldg(d0.invT_f + c);
    }
  }
  return t;
}

__device__ __forceinline__ size_t tab32_bytes(const Tab32& t) {
  return (4 * (size_t)t.n * (t.invT ? 2 : 1) + 127) & ~(size_t)127;
}

// Every warp stages its own chunks: chunk k of global warp gw is chunk
// gw + k * (warps in the grid) of the kernel's particles (C = 32 x rounds
// particles each), so no warp waits for another and no atomic hands out work.
// Lane 0 keeps kStages chunks in flight: it starts the bulk copies of a
// chunk's survivors into a stage of the warp's ring (completion counted on
// that stage's mbarrier), and after the warp has streamed a chunk it reuses
// the stage for the chunk kStages further on.
template <int DIM, bool ENS>
struct Ring32 {
  unsigned char* ring;
  uint64_t* bar;
  int C;
  size_t stage_sz;
  // lane 0: expect the bytes of chunk c's survivors (below n_surv of member
  // dm's buffer cb) on stage s and start their copies
  __device__ __forceinline__ void issue(const Dev* dm, unsigned cb, long long lc, long long n_surv, int s) const {
    const long long first = lc * C;
    long long n = n_surv - first;
    n = n < 0 ? 0 : (n > C ? C : n);
    issue_at(dm, cb, first, n, s);
  }
  // the same for the n (<= C) survivors from slot `first` (a multiple of 4)
  __device__ __forceinline__ void issue_at(const Dev* dm, unsigned cb, long long first, long long n, int s) const {
    const unsigned c4 = (unsigned)((n + 3) & ~3ll), c2 = (unsigned)((n + 1) & ~1ll);
    const unsigned bytes = n ? c4 * 4u * StageF<DIM>::kArr4 + c2 * 8u : 0u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(&bar[s], bytes);
    if (bytes) {
      const StageF<DIM> sg(ring + s * stage_sz, C);
      bulk_g2s(sg.id, dm->pid[cb] + first, c2 * 8u, &bar[s]);
      bulk_g2s(sg.x, dm->fx[cb] + first, c4 * 4u, &bar[s]);
      bulk_g2s(sg.ox, dm->fox[cb] + first, c4 * 4u, &bar[s]);
      bulk_g2s(sg.nu, dm->fnu[cb] + first, c4 * 4u, &bar[s]);
      bulk_g2s(sg.w, dm->fw[cb] + first, c4 * 4u, &bar[s]);
      bulk_g2s(sg.key, dm->pkey[cb] + first, c4 * 4u, &bar[s]);
      if (DIM >= 2) {
        bulk_g2s(sg.y, dm->fy[cb] + first, c4 * 4u, &bar[s]);
        bulk_g2s(sg.oy, dm->foy[cb] + first, c4 * 4u, &bar[s]);
      }
      if (DIM == 3) {
        bulk_g2s(sg.z, dm->fz[cb] + first, c4 * 4u, &bar[s]);
        bulk_g2s(sg.oz, dm->foz[cb] + first, c4 * 4u, &bar[s]);
      }
    }
  }
};

// A survivor from slot li of a staged chunk.
template <int DIM>
__device__ __forceinline__ void from_stage32(const Dev& d, const StageF<DIM>& sg, int li, P32& q) {
  q.xi = sg.x[li];
  q.ox = sg.ox[li];
  if (DIM >= 2) { q.eta = sg.y[li]; q.oy = sg.oy[li]; }
  if (DIM == 3) { q.zeta = sg.z[li]; q.oz = sg.oz[li]; }
  q.nu = sg.nu[li];
  q.w = sg.w[li];
  q.id = sg.id[li];
  decode_key32<DIM>(d, sg.key[li], q);
}

// The general FP32 kernel: every particle of the step (survivors staged,
// newborns born in registers), first flight and streaming loop in place.
template <int DIM, bool ENS, int NT>
__global__ void __launch_bounds__(NT, (ENS || DIM == 3) ? (NT >= 512 ? 1 : (NT >= 256 ? 2 : 4)) : (NT >= 512 ? 2 : (NT >= 256 ? 4 : 8)))
    k_stream32(const __grid_constant__ Dev d0, const Ens e, int rounds) {
  extern __shared__ __align__(128) unsigned char s_dyn[];
  __shared__ uint64_t s_full[NT / 32][kStages];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Tab32 tab = load_tab32<ENS>(d0, s_dyn);
  Ring32<DIM, ENS> rg;
  rg.C = 32 * rounds;
  rg.stage_sz = (size_t)rg.C * StageF<DIM>::kBytesPer;
  rg.ring = s_dyn + tab32_bytes(tab) + (size_t)warp * kStages * rg.stage_sz;
  rg.bar = s_full[warp];
  const int C = rg.C;
  if (lane == 0) {
    for (int k = 0; k < kStages; ++k) mbar_init(&rg.bar[k], 1);
    mbar_init_fence();
  }
  __syncthreads();
  const StepHead h0 = ENS ? StepHead{} : step_head(d0);
  const long long gw = (long long)blockIdx.x * (NT / 32) + warp, tw = (long long)gridDim.x * (NT / 32);
  const long long nchunks = ENS ? (long long)e.tile0[e.M] : (h0.n_tot + C - 1) / C;
  unsigned* status0 = ENS ? &e.devs[0].ctrl->status : &d0.ctrl->status;
  auto issue = [&](long long c, int s) {
    if (ENS) {
      const int m = find_member(e.tile0, e.M, c);
      const Dev* dm = &e.devs[m];
      const unsigned cb = dm->ctrl->cur;
      rg.issue(dm, cb, c - (long long)e.tile0[m], (long long)dm->ctrl->n_part[cb], s);
    } else {
      rg.issue(&d0, h0.cur, c, h0.n_surv, s);
    }
  };
  int issued = 0;   // chunks of this warp whose copies were started
  for (; issued < kStages && gw + issued * tw < nchunks; ++issued)
    if (lane == 0) issue(gw + issued * tw, issued);
  __syncwarp();

  Counters cnt;
  int acc_m = 0;
  int k = 0, st = 0;
  unsigned par = 0u;   // stage st of chunk k, and the phase parity it waits for
  for (long long c = gw; c < nchunks; c += tw, ++k, st = st + 1 == kStages ? 0 : st + 1, par ^= st == 0 ? 1u : 0u) {
    if (!mbar_wait_bounded(&rg.bar[st], par)) {
      atomicOr(status0, ST_TIMEOUT);
      break;
    }
    const StageF<DIM> sgt(rg.ring + st * rg.stage_sz, C);
    const int m = ENS ? find_member(e.tile0, e.M, c) : 0;
    if (ENS && m != acc_m) { flush_counters(e.devs[acc_m].ctrl, cnt); acc_m = m; }
    const Dev& d = ENS ? e.devs[m] : d0;
    const long long lc = ENS ? c - (long long)e.tile0[m] : c;
    Ctrl* ctrl = d.ctrl;
    const unsigned cur = ENS ? ctrl->cur : h0.cur, nxb = cur ^ 1u;
    const long long n_surv = ENS ? (long long)ctrl->n_part[cur] : h0.n_surv;
    const long long n_tot = ENS ? n_surv + (long long)ctrl->n_new : h0.n_tot;
    const uint32_t step = ENS ? (uint32_t)ctrl->step : h0.step;
    const int G = d.G, nx = d.nx, ny = DIM >= 2 ? d.ny : 1;
    for (int r = 0; r < rounds; ++r) {
      const int li = r * 32 + lane;
      const long long i = lc * C + li;
      // every lane of this pass holds a survivor of the previous step (the
      // common case: no newborn code, every lane valid)
      const bool surv_pass = lc * C + (long long)r * 32 + 32 <= n_surv;
      const bool valid = i < n_tot;
      P32 q;
      clear32(q);
      DrawsF rng;
      if (surv_pass || (valid && i < n_surv)) {
        from_stage32<DIM>(d, sgt, li, q);
        rng.init(q.id, step, 0u);
      } else if (valid) {
        birth32<DIM>(d, q, rng, (uint32_t)(i - n_surv), step, d.off);
      } else {
        rng.init(0ull, step, 0u);
      }
      q.cell0 = q.gside >= 0 ? q.cx : (q.cz * ny + q.cy) * nx + q.cx;
      q.ghost = q.gside >= 0;
      // ---- streaming
      float inup = 1.0f;
      bool more = false;
      if (valid) {
        inup = d.grey ? 1.0f : pow_fast_f(q.nu, -d.spf);
        more = first_flight32<DIM>(d, q, rng, inup, ENS ? 0 : tab.n, tab.invT, tab.sinv, tab.sinvT);
      }
      if (more) stream_loop32<DIM>(d, q, rng, inup, ENS ? 0 : tab.n, tab.invT, tab.sinv, tab.sinvT);
      const int cell = (q.cz * ny + q.cy) * nx + q.cx;
      bool stored = false;
      if (valid) stored = store32<DIM>(d, nxb, q, i, cell);
      // ---- tallies (W and E_surv in fixed point, see to_fixed_f)
      const long long wq = valid ? to_fixed_f(q.w, d.tq_shift, &ctrl->status) : 0ll;
      warp_run_add_fixed(d.Esq, stored ? cell * G + q.g : -1 - lane, wq, d.sort_cnt);
      if (valid) {
        cross_tallies32(d, q, cell, wq);
        cnt.seg += (unsigned)q.nseg;
        cnt.abs += q.fate == FATE_ABSORBED;
        cnt.esc += q.fate == FATE_ESCAPED;
        cnt.surv += q.fate == FATE_SURVIVED;
        cnt.rem += q.fate == FATE_REMOVED;
        if (!ENS) record32<DIM>(d, q, i, cell);
      }
    }
    // the stage is free: the chunk kStages further on goes into it
    __syncwarp();
    if (c + kStages * tw < nchunks) {
      if (lane == 0) issue(c + kStages * tw, st);
      ++issued;
    }
    __syncwarp();
  }
  // after a failed wait: no copy may still be landing when the warp leaves
  if (lane == 0)
    for (int kk = k; kk < issued; ++kk) mbar_wait_bounded(&rg.bar[kk % kStages], (unsigned)(kk / kStages) & 1u);
  flush_counters(ENS ? e.devs[acc_m].ctrl : d0.ctrl, cnt);
}

// 1/x to about an ulp (rcp.approx): for the survivor kernel's face test,
// a decision that needs no correct rounding
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Survivor kernel of a 1D problem whose particles seldom reach a face in a
// step (v dt / dx small: the slabs), with the power-law opacity and its
// per-cell factors in shared memory: every survivor draws its free time
// (Eq. particle-tf-formula) and takes its first flight; one that ends the
// step there is finished in place (no face crossed, so only E_surv and the
// counters are tallied); one that reaches a face first is set aside (slot,
// remaining free time) in a per-warp buffer in shared memory.  The code of
// that first flight has no crossing loop, no birth sampling and no
// per-particle branching on the problem's options, so a warp's lanes stay
// together; after each chunk, while 32 or more survivors are set aside, the
// warp streams 32 of them through their faces, one per lane (and the rest
// after its last chunk).  A chunk's R x 32 first flights are computed before
// any of them is stored or tallied, so their dependent chains (Philox, the
// logarithm) interleave.  The step's newborns (born in registers, the
// general per-particle path) are streamed first, a chunk of 32 per warp,
// while the warps' first survivor chunks are landing.
// P3: sigma ~ nu^-3; R: 32-particle rounds per chunk.
template <int NT, bool P3, int R>
__global__ void __launch_bounds__(NT, NT >= 512 ? 1 : (NT >= 256 ? 2 : 4))
    k_stream32_fast(const __grid_constant__ Dev d) {
  constexpr int C = 32 * R;
  constexpr int kBuf = 32 + C;   // set-aside entries: fewer than 32 left over, plus one chunk
  extern __shared__ __align__(128) unsigned char s_dyn[];
  __shared__ uint64_t s_full[NT / 32][kStages];
  __shared__ uint32_t s_li[NT / 32][kBuf];
  __shared__ float s_lt[NT / 32][kBuf];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  const int ncell = d.ncell;
  float* s_sinv = reinterpret_cast<float*>(s_dyn);
  uint32_t* s_seg = reinterpret_cast<uint32_t*>(s_sinv + ncell);
  const int ns = fast_segments(d.nbins);
  Ring32<1, false> rg;
  rg.C = C;
  rg.stage_sz = (size_t)C * StageF<1>::kBytesPer;
  rg.ring = s_dyn + fast_table_bytes(ncell, d.nbins) + (size_t)warp * kStages * rg.stage_sz;
  rg.bar = s_full[warp];
  Ctrl* ctrl = d.ctrl;
  // Set-up that needs nothing from the kernels before this one in the
  // stream (launched as a programmatic dependent of the birth scan, it may
  // run while the scan finishes): the rings' barriers and the copies of the
  // warps' first survivor chunks (the previous step's survivors; the live
  // buffer and its count were set by the previous step's end).
  const unsigned cur = ctrl->cur;
  const long long n_surv = (long long)ctrl->n_part[cur];
  // a contiguous range of chunks per warp (bins run on across its chunks),
  // the counts differing by at most one between warps (with whole chunks
  // rounded up per warp, a step of a few chunks per warp would leave the
  // last warps, and the SMs holding them, without survivors)
  const long long gw = (long long)blockIdx.x * (NT / 32) + warp, tw = (long long)gridDim.x * (NT / 32);
  const long long nall = (n_surv + C - 1) / C;
  const long long c0 = gw * nall / tw, nchunks = (gw + 1) * nall / tw;
  const long long p0 = 0, p1 = n_surv;
  auto issue_chunk = [&](long long c, int s) { rg.issue(&d, cur, c, n_surv, s); };
  int issued = 0;
  if (lane == 0) {
    for (int k = 0; k < kStages; ++k) mbar_init(&rg.bar[k], 1);
    mbar_init_fence();
    for (; issued < kStages && c0 + issued < nchunks; ++issued) issue_chunk(c0 + issued, issued);
  }
  issued = __shfl_sync(full, issued, 0);
  __syncwarp();
  // the birth kernel's tables and the scan's offsets and count
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int c = threadIdx.x; c < ncell; c += NT) s_sinv[c] = __ldg(d.sTinv_f + c);
  for (int s = threadIdx.x; s < ns; s += NT) s_seg[s] = __ldg(d.off + 32 * s);
  __syncthreads();
  const StepHead h0 = step_head(d);
  const unsigned nxb = h0.cur ^ 1u;
  const uint32_t G = (uint32_t)d.G;
  const float invG = d.invG_f;
  const float dxf = d.dxf, vf = d.vf, dtf = d.dtf, inv_rate = d.inv_rate_f, inv_capf = d.inv_capf, spf = d.spf;
  const int tq_shift = d.tq_shift;
  const bool grey = d.grey;

  int acc_key = -1;
  long long acc_w = 0;
  unsigned acc_n = 0u;
  unsigned nl = 0;   // entries in the warp's buffer of set-aside survivors (same in every lane)
  Counters cnt;
  auto run_set_aside = [&](unsigned k) {
    const bool act = (unsigned)lane < k;
    P32 q;
    clear32(q);
    DrawsF rng;
    long long i = 0;
    if (act) {
      i = (long long)s_li[warp][lane];
      const float tl = s_lt[warp][lane];
      q.xi = d.fx[h0.cur][i];
      q.ox = d.fox[h0.cur][i];
      q.nu = d.fnu[h0.cur][i];
      q.w = d.fw[h0.cur][i];
      q.id = d.pid[h0.cur][i];
      decode_key32<1>(d, d.pkey[h0.cur][i], q);
      q.collided = tl < 0.0f;
      q.t_rem = fabsf(tl);
      rng.init(q.id, h0.step, 1u);
    } else {
      rng.init(0ull, h0.step, 0u);
    }
    q.cell0 = q.cx;
    const float inup = (!act || grey) ? 1.0f : pow_fast_f(q.nu, -spf);
    if (act) stream_loop32<1>(d, q, rng, inup, ncell, false, s_sinv, s_sinv + ncell);
    const int cell = q.cx;
    bool stored = false;
    if (act) stored = store32<1>(d, nxb, q, i, cell);
    const long long wq = act ? to_fixed_f(q.w, tq_shift, &ctrl->status) : 0ll;
    warp_run_add_fixed(d.Esq, stored ? cell * (int)G + q.g : -1 - lane, wq, d.sort_cnt);
    if (act) {
      cross_tallies32(d, q, cell, wq);
      cnt.seg += (unsigned)q.nseg;
      cnt.abs += q.fate == FATE_ABSORBED;
      cnt.esc += q.fate == FATE_ESCAPED;
      cnt.surv += q.fate == FATE_SURVIVED;
      cnt.rem += q.fate == FATE_REMOVED;
      record32<1>(d, q, i, cell);
    }
    // the rest of the buffer moves to the front, 32 entries a pass (each pass
    // reads entries at least k beyond those it writes)
    __syncwarp();
    for (unsigned b = 0; b + k < nl; b += 32u) {
      const bool mv = b + lane + k < nl;
      uint32_t a = 0u;
      float t = 0.0f;
      if (mv) { a = s_li[warp][b + k + lane]; t = s_lt[warp][b + k + lane]; }
      __syncwarp();
      if (mv) { s_li[warp][b + lane] = a; s_lt[warp][b + lane] = t; }
      __syncwarp();
    }
    nl -= k;
  };

  // ---- the newborns of the step (Eq. IhpFormula), while the first survivor
  // chunks land: chunks of 32 consecutive birth ordinals, chunk k to block
  // k mod (blocks), one warp of each block before the next
  {
    const long long n_new = h0.n_tot - h0.n_surv;
    const long long nnc = (n_new + 31) / 32;
    const int G = (int)d.G;
    for (long long kc = blockIdx.x + (long long)gridDim.x * warp; kc < nnc; kc += (long long)gridDim.x * (NT / 32)) {
      const long long jj = kc * 32 + lane;
      const bool valid = jj < n_new;
      const long long i = h0.n_surv + jj;
      P32 q;
      clear32(q);
      DrawsF rng;
      if (ns) {
        uint32_t ob;
        const int bin = birth_bin32(d, s_seg, ns, (uint32_t)jj, valid, &ob);
        if (valid) birth32_in<1>(d, q, rng, (uint32_t)jj, h0.step, bin, ob);
        else rng.init(0ull, h0.step, 0u);
      } else {
        if (valid) birth32<1>(d, q, rng, (uint32_t)jj, h0.step, d.off);
        else rng.init(0ull, h0.step, 0u);
      }
      q.cell0 = q.cx;
      q.ghost = q.gside >= 0;
      const float inup = (!valid || grey) ? 1.0f : pow_fast_f(q.nu, -spf);
      bool more = false;
      if (valid) more = first_flight32<1>(d, q, rng, inup, ncell, false, s_sinv, s_sinv + ncell);
      if (more) stream_loop32<1>(d, q, rng, inup, ncell, false, s_sinv, s_sinv + ncell);
      const int cell = q.cx;
      bool stored = false;
      if (valid) stored = store32<1>(d, nxb, q, i, cell);
      const long long wq = valid ? to_fixed_f(q.w, tq_shift, &ctrl->status) : 0ll;
      warp_run_add_fixed(d.Esq, stored ? cell * G + q.g : -1 - lane, wq, d.sort_cnt);
      if (valid) {
        cross_tallies32(d, q, cell, wq);
        cnt.seg += (unsigned)q.nseg;
        cnt.abs += q.fate == FATE_ABSORBED;
        cnt.esc += q.fate == FATE_ESCAPED;
        cnt.surv += q.fate == FATE_SURVIVED;
        cnt.rem += q.fate == FATE_REMOVED;
        record32<1>(d, q, i, cell);
      }
    }
  }

  int k = 0, st = 0;
  unsigned par = 0u;   // stage st of chunk k, and the phase parity it waits for
  for (long long c = c0; c < nchunks; ++c, ++k, st = st + 1 == kStages ? 0 : st + 1, par ^= st == 0 ? 1u : 0u) {
    if (!mbar_wait_bounded(&rg.bar[st], par)) {
      atomicOr(&ctrl->status, ST_TIMEOUT);
      break;
    }
    const StageF<1> sg(rg.ring + st * rg.stage_sz, C);
    const long long base = p0 + c * C;
    const int nval = (int)(p1 - base < C ? p1 - base : C);
    // ---- the first flights of the chunk's R x 32 survivors, independent of
    // one another (so their dependent chains interleave)
    float a_x[R], a_ox[R], a_nu[R], a_w[R], a_tr[R];
    unsigned long long a_id[R];
    uint32_t a_key[R], a_cell[R];
    bool a_col[R], a_later[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int li = r * 32 + lane;
      const bool valid = li < nval;
      const float xi = sg.x[li], ox = sg.ox[li], nu = sg.nu[li];
      const unsigned long long id = sg.id[li];
      const uint32_t key = valid ? sg.key[li] : 0u;
      a_w[r] = sg.w[li];
      // cell = key / G through an FP32 reciprocal, corrected (key < 2^24)
      uint32_t cell = __float2uint_rz(__uint2float_rn(key) * invG);
      const int rem = (int)(key - cell * G);
      cell = rem < 0 ? cell - 1u : (rem >= (int)G ? cell + 1u : cell);
      // free time: draw 0 of this step's stream of the particle
      const uint4 blk = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), h0.step, 0u), d.pk);
      const UPair u = u01f(blk.x, blk.y);
      // 1/sigma carries nu^{-p}: nu^3 for the nu^-3 law
      float inup;
      if (P3) inup = nu * nu * nu;
      else inup = grey ? 1.0f : pow_fast_f(nu, -spf);
      const float sig_inv = fmaxf(s_sinv[cell] * inup, inv_capf);
      const float tc = neg_log_u(u) * inv_rate * sig_inv;
      const bool collided = tc < dtf;
      const float t_rem = collided ? tc : dtf;
      // first flight: the face ahead comes first?
      const float dist = ox > 0.0f ? dxf - xi : xi;
      const float tf = fmaxf(dist, 0.0f) * rcp_approx(vf * fabsf(ox));
      a_later[r] = valid && tf < t_rem;
      a_x[r] = fminf(fmaxf(fmaf(vf * ox, t_rem, xi), 0.0f), dxf);
      a_ox[r] = ox;
      a_nu[r] = nu;
      a_tr[r] = t_rem;
      a_id[r] = id;
      a_key[r] = valid ? key : kDeadKey;
      a_cell[r] = cell;
      a_col[r] = collided;
    }
    // the stage is consumed: the chunk kStages further on goes into it
    __syncwarp();
    if (c + kStages < nchunks) {
      if (lane == 0) issue_chunk(c + kStages, st);
      ++issued;
    }
    float* __restrict__ o_x = d.fx[nxb] + base;
    float* __restrict__ o_ox = d.fox[nxb] + base;
    float* __restrict__ o_nu = d.fnu[nxb] + base;
    float* __restrict__ o_w = d.fw[nxb] + base;
    unsigned long long* __restrict__ o_id = d.pid[nxb] + base;
    uint32_t* __restrict__ o_key = d.pkey[nxb] + base;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int li = r * 32 + lane;
      const bool valid = a_key[r] != kDeadKey;
      // set aside: the slot and t_rem, negative when the flight ends in a collision
      const unsigned lmask = __ballot_sync(full, a_later[r]);
      if (a_later[r]) {
        const unsigned pos = nl + __popc(lmask & ((1u << lane) - 1u));
        s_li[warp][pos] = (uint32_t)(base + li);
        s_lt[warp][pos] = a_col[r] ? -a_tr[r] : a_tr[r];
      }
      nl += __popc(lmask);
      const bool fin = valid && !a_later[r];
      const bool collided = a_col[r];
      if (fin) {   // in place: slot i of the other buffer (i < n_surv <= capacity)
        o_x[li] = a_x[r];
        o_ox[li] = a_ox[r];
        o_nu[li] = a_nu[r];
        o_w[li] = a_w[r];
        o_id[li] = a_id[r];
        o_key[li] = collided ? kDeadKey : a_key[r];
      }
      // E_surv and the sort counts of the survivors (the particle stayed in
      // its cell, so W is unchanged), summed per thread while its bin stays
      // the same: a lane's successive particles are 32 slots apart in the
      // bin-sorted input, so nearly always in one bin
      if (fin && !collided) {
        const long long wq = to_fixed_f(a_w[r], tq_shift, &ctrl->status);
        if ((int)a_key[r] != acc_key || acc_n == 32u) {
          if (acc_n) {
            atomic_add_fixed(d.Esq + 2 * (long long)acc_key, acc_w);
            atomicAdd(d.sort_cnt + acc_key, acc_n);
          }
          acc_key = (int)a_key[r];
          acc_w = 0;
          acc_n = 0u;
        }
        acc_w += wq;
        ++acc_n;
      }
      cnt.seg += fin;
      cnt.abs += fin && collided;
      cnt.surv += fin && !collided;
      if (d.rec && fin && base + li < d.rec_cap) {
        P32 q;
        clear32(q);
        const uint32_t cell = a_cell[r];
        q.xi = a_x[r]; q.ox = a_ox[r]; q.nu = a_nu[r]; q.w = a_w[r]; q.id = a_id[r];
        q.cx = (int)cell; q.g = (int)(a_key[r] - cell * G);
        q.fate = collided ? FATE_ABSORBED : FATE_SURVIVED; q.nseg = 1; q.t_tra = a_tr[r]; q.cell0 = (int)cell;
        record32<1>(d, q, base + li, (int)cell);
      }
    }
    __syncwarp();
    while (nl >= 32u) run_set_aside(32u);
  }
  while (nl >= 32u) run_set_aside(32u);   // (only after a failed wait)
  if (nl) run_set_aside(nl);
  // the last runs: the warp's lanes mostly end in the same bin
  warp_run_add_fixed_n(d.Esq, acc_n ? acc_key : -1 - lane, acc_w, acc_n, d.sort_cnt);
  if (lane == 0)
    for (int kk = k; kk < issued; ++kk) mbar_wait_bounded(&rg.bar[kk % kStages], (unsigned)(kk / kStages) & 1u);
  flush_counters_block(ctrl, cnt);
}

static int g_stream64_occ[4][2][3][3] = {};   // [dim][ens][ppt][block index]
static int g_stream32_occ[4][2][3] = {};      // [dim][ens][block index] (at the table size last used)
static int g_stream32_occ_dyn[4][2][3] = {};

template <int DIM, bool ENS, int PPT>
static cudaError_t launch_stream64_t(const Dev& d, const Ens& e, const StreamShape& sh, cudaStream_t s) {
  const int sms = sm_count();
  const void* fn = (const void*)k_stream64<DIM, ENS, PPT>;
  const int bi = sh.block == 128 ? 0 : (sh.block == 512 ? 2 : 1);
  int& occ = g_stream64_occ[DIM][ENS][PPT][bi];
  if (!occ) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, sh.block, 0);
    if (occ < 1) occ = 1;
  }
  const int per = sh.blocks_per_sm > 0 && sh.blocks_per_sm < occ ? sh.blocks_per_sm : occ;
  k_stream64<DIM, ENS, PPT><<<sms * per, sh.block, 0, s>>>(d, e);
  return cudaGetLastError();
}

static size_t table32_bytes(const Dev& d) { return (4 * (size_t)stream32_table_floats(d) + 127) & ~(size_t)127; }

// 1D problems that take the survivor kernel (see launch_stream32_t)
static bool split32(const Dev& d) {
  return d.dim == 1 && d.v * d.dt / d.dx < 0.25 && d.sig_law == 0 && d.ncell <= kSmemCells;
}

template <int NT>
static const void* fast_fn(bool p3, int ppt) {
  if (p3) {
    if (ppt >= 4) return (const void*)k_stream32_fast<NT, true, 4>;
    if (ppt == 2) return (const void*)k_stream32_fast<NT, true, 2>;
    return (const void*)k_stream32_fast<NT, true, 1>;
  }
  if (ppt >= 4) return (const void*)k_stream32_fast<NT, false, 4>;
  if (ppt == 2) return (const void*)k_stream32_fast<NT, false, 2>;
  return (const void*)k_stream32_fast<NT, false, 1>;
}

template <int DIM, bool ENS, int NT>
static cudaError_t launch_stream32_t(const Dev& d, const Ens& e, const StreamShape& sh, cudaStream_t s) {
  const int sms = sm_count();
  const int C = 32 * sh.ppt;
  // a 1D problem whose particles seldom reach a face in a step (a particle
  // crosses at most v dt / dx cells) with the power-law opacity held in
  // shared memory: the survivor kernel (newborns included)
  const bool split = !ENS && DIM == 1 && split32(d);
  const size_t tab = ENS ? 0 : (split ? fast_table_bytes(d.ncell, d.nbins) : table32_bytes(d));
  const size_t dyn = tab + (size_t)(NT / 32) * kStages * stream32_stage_bytes(DIM, C);
  const int bi = NT == 128 ? 0 : (NT == 512 ? 2 : 1);
  const bool p3 = !d.grey && d.sig_p == -3.0;
  const void* fn = !split ? (const void*)k_stream32<DIM, ENS, NT> : fast_fn<NT>(p3, sh.ppt);
  int& occ = g_stream32_occ[DIM][ENS][bi];
  int& occ_dyn = g_stream32_occ_dyn[DIM][ENS][bi];
  const int key = ((int)dyn * 4 + (split ? 1 : 0) + (p3 ? 2 : 0)) * 8 + sh.ppt;
  if (!occ || occ_dyn != key) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, NT, dyn);
    if (occ < 1) occ = 1;
    occ_dyn = key;
  }
  const int per = sh.blocks_per_sm > 0 && sh.blocks_per_sm < occ ? sh.blocks_per_sm : occ;
  if (!split) {
    k_stream32<DIM, ENS, NT><<<sms * per, NT, dyn, s>>>(d, e, sh.ppt);
    return cudaGetLastError();
  }
  // a programmatic dependent of the kernel before it in the stream (the
  // birth scan): its set-up and first copies overlap that kernel's end, and
  // it waits for the kernel's results before it reads them
  void* args[] = {(void*)&d};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sms * per);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t r = cudaLaunchKernelExC(&cfg, fn, args);
  if (!r) r = cudaGetLastError();
  return r;
}

template <int DIM, bool ENS>
static cudaError_t launch_stream32_nt(const Dev& d, const Ens& e, const StreamShape& sh, cudaStream_t s) {
  if (sh.block == 128) return launch_stream32_t<DIM, ENS, 128>(d, e, sh, s);
  if (sh.block == 512) return launch_stream32_t<DIM, ENS, 512>(d, e, sh, s);
  return launch_stream32_t<DIM, ENS, 256>(d, e, sh, s);
}

template <bool ENS>
static cudaError_t launch_stream_dim(const Dev& d, const Ens& e, int mixed, const StreamShape& sh, cudaStream_t s) {
  if (d.dim == 3) {   // single problems only (ensembles are 1D/2D)
    if (ENS) return cudaErrorNotSupported;
    return mixed ? launch_stream32_nt<3, false>(d, e, sh, s) : launch_stream64_t<3, false, 1>(d, e, sh, s);
  }
  if (d.dim == 2) {
    if (mixed) return launch_stream32_nt<2, ENS>(d, e, sh, s);
    if (sh.ppt >= 2) return launch_stream64_t<2, ENS, 2>(d, e, sh, s);
    return launch_stream64_t<2, ENS, 1>(d, e, sh, s);
  }
  if (mixed) return launch_stream32_nt<1, ENS>(d, e, sh, s);
  if (sh.ppt >= 2) return launch_stream64_t<1, ENS, 2>(d, e, sh, s);
  return launch_stream64_t<1, ENS, 1>(d, e, sh, s);
}

cudaError_t launch_stream(const Dev& d, const Ens* e, const StreamShape& sh, cudaStream_t s) {
  const int mixed = d.precision == 1;
  if (e && e->M > 1) return launch_stream_dim<true>(d, *e, mixed, sh, s);
  const Ens none{};
  return launch_stream_dim<false>(d, none, mixed, sh, s);
}

}  // namespace ugkwp
