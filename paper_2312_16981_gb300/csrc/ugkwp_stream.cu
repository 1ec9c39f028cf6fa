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
// The FP32 kernel streams tiles of survivors staged in shared memory: one
// producer warp per block takes the next tile from a global counter and
// starts bulk copies (cp.async.bulk, completion counted on an mbarrier) of
// its arrays into one of three stages; the streaming warps wait on a stage's
// "full" barrier, process it and arrive on its "empty" barrier, so no warp
// waits for another.  Per-cell opacity factors of single problems are held
// in shared memory when they fit.
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
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
// Block = NT streaming threads + one producer warp.  Tiles of NT x rounds
// particles; a streaming warp takes 32 x rounds consecutive particles of a
// tile (so its lanes share bins and its stores are whole 128-byte lines).
template <int DIM, bool ENS, int NT>
__global__ void __launch_bounds__(NT + 32, NT >= 512 ? 1 : (NT >= 256 ? 3 : 6))
    k_stream32(const __grid_constant__ Dev d0, const Ens e, int rounds) {
  extern __shared__ __align__(128) unsigned char s_dyn[];
  __shared__ uint64_t s_full[kStages], s_empty[kStages];
  __shared__ long long s_tile[kStages];
  const long long tile = (long long)NT * rounds;
  const size_t stage_sz = (size_t)tile * StageF<DIM>::kBytesPer;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per-cell opacity factors of a single problem in shared memory
  const int tab_n = ENS ? 0 : ((d0.sig_law == 2 || d0.ncell > kSmemCells) ? 0 : d0.ncell);
  const bool tab_invT = !ENS && tab_n && d0.sig_law == 1 && !d0.grey;
  float* s_sinv = reinterpret_cast<float*>(s_dyn + kStages * stage_sz);
  float* s_invT = s_sinv + tab_n;
  if (threadIdx.x == 0) {
    for (int k = 0; k < kStages; ++k) {
      mbar_init(&s_full[k], 1);
      mbar_init(&s_empty[k], NT / 32);
    }
    mbar_init_fence();
  }
  if (!ENS) {
    for (int c = threadIdx.x; c < tab_n; c += blockDim.x) {
      s_sinv[c] = __ldg(d0.sTinv_f + c);
      if (tab_invT) s_invT[c] = __ldg(d0.invT_f + c);
    }
  }
  __syncthreads();
  const StepHead h0 = ENS ? StepHead{} : step_head(d0);

  if (warp == NT / 32) {
    // ---- producer: hand out tiles, stage their survivors
    if (lane != 0) return;
    unsigned long long* ctr = ENS ? e.tile_next : &d0.ctrl->tile_next;
    unsigned int* status = ENS ? &e.devs[0].ctrl->status : &d0.ctrl->status;
    const long long ntiles = ENS ? (long long)e.tile0[e.M] : (h0.n_tot + tile - 1) / tile;
    bool gave_up = false;
    unsigned issued = 0, lastpar = 0;
    for (int it = 0;; ++it) {
      const int s = it % kStages;
      if (it >= kStages) {
        const unsigned par = (unsigned)((it / kStages) - 1) & 1u;
        // the previous copy into this stage has landed (it needs no other warp) ...
        if (!mbar_wait_bounded(&s_full[s], par)) { atomicOr(status, ST_TIMEOUT); gave_up = true; }
        // ... and every streaming warp is done with it
        if (!gave_up && !mbar_wait_bounded(&s_empty[s], par)) { atomicOr(status, ST_TIMEOUT); gave_up = true; }
      }
      long long t = (long long)atomicAdd(ctr, 1ull);
      if (t >= ntiles) t = -1;
      s_tile[s] = t;
      unsigned bytes = 0;
      const Dev* dm = &d0;
      long long first = 0, n = 0;
      unsigned cb = h0.cur;
      if (t >= 0) {
        long long lt = t, n_surv = h0.n_surv;
        if (ENS) {
          const int m = find_member(e.tile0, e.M, t);
          dm = &e.devs[m];
          lt = t - (long long)e.tile0[m];
          cb = dm->ctrl->cur;
          n_surv = (long long)dm->ctrl->n_part[cb];
        }
        first = lt * tile;
        n = n_surv - first;
        n = n < 0 ? 0 : (n > tile ? tile : n);
        const unsigned c4 = (unsigned)((n + 3) & ~3ll), c2 = (unsigned)((n + 1) & ~1ll);
        bytes = n ? c4 * 4u * StageF<DIM>::kArr4 + c2 * 8u : 0u;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive_expect_tx(&s_full[s], bytes);
      issued |= 1u << s;
      lastpar = (lastpar & ~(1u << s)) | ((unsigned)((it / kStages) & 1) << s);
      if (bytes) {
        const StageF<DIM> sg(s_dyn + s * stage_sz, (int)tile);
        const unsigned c4 = (unsigned)((n + 3) & ~3ll), c2 = (unsigned)((n + 1) & ~1ll);
        bulk_g2s(sg.id, dm->pid[cb] + first, c2 * 8u, &s_full[s]);
        bulk_g2s(sg.x, dm->fx[cb] + first, c4 * 4u, &s_full[s]);
        bulk_g2s(sg.ox, dm->fox[cb] + first, c4 * 4u, &s_full[s]);
        bulk_g2s(sg.nu, dm->fnu[cb] + first, c4 * 4u, &s_full[s]);
        bulk_g2s(sg.w, dm->fw[cb] + first, c4 * 4u, &s_full[s]);
        bulk_g2s(sg.key, dm->pkey[cb] + first, c4 * 4u, &s_full[s]);
        if (DIM >= 2) {
          bulk_g2s(sg.y, dm->fy[cb] + first, c4 * 4u, &s_full[s]);
          bulk_g2s(sg.oy, dm->foy[cb] + first, c4 * 4u, &s_full[s]);
        }
        if (DIM == 3) {
          bulk_g2s(sg.z, dm->fz[cb] + first, c4 * 4u, &s_full[s]);
          bulk_g2s(sg.oz, dm->foz[cb] + first, c4 * 4u, &s_full[s]);
        }
      }
      if (t < 0) break;
    }
    // no copy may still be landing when the block's last warp leaves
    for (int s = 0; s < kStages; ++s)
      if ((issued >> s) & 1u) mbar_wait_bounded(&s_full[s], (lastpar >> s) & 1u);
    return;
  }

  // ---- streaming warps
  Counters cnt;
  int acc_m = 0;
  for (int it = 0;; ++it) {
    const int st = it % kStages;
    if (!mbar_wait_bounded(&s_full[st], (unsigned)(it / kStages) & 1u)) {
      atomicOr(ENS ? &e.devs[0].ctrl->status : &d0.ctrl->status, ST_TIMEOUT);
      break;
    }
    const long long t = *reinterpret_cast<volatile long long*>(&s_tile[st]);
    if (t < 0) break;
    const StageF<DIM> sgt(s_dyn + st * stage_sz, (int)tile);
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
    const float dxf = d.dxf, dyf = d.dyf, dzf = d.dzf, vf = d.vf, dtf = d.dtf;
    const float inv_rate = d.inv_rate_f, spf = d.spf;
    for (int r = 0; r < rounds; ++r) {
    const int li = (warp * rounds + r) * 32 + lane;
    const long long i = lt * tile + li;
    const bool valid = i < n_tot;
    float xi = 0.f, eta = 0.f, zeta = 0.f, ox = 0.f, oy = 0.f, oz = 0.f, nu = 0.f, w = 0.f;
    unsigned long long id = 0ull;
    int cx = 0, cy = 0, cz = 0, g = 0, gside = -1;
    bool newborn = false;
    DrawsF rng;
    rng.init(0ull, step, 0u);
    if (valid) {
      if (i < n_surv) {
        xi = sgt.x[li];
        ox = sgt.ox[li];
        if (DIM >= 2) { eta = sgt.y[li]; oy = sgt.oy[li]; }
        if (DIM == 3) { zeta = sgt.z[li]; oz = sgt.oz[li]; }
        nu = sgt.nu[li];
        w = sgt.w[li];
        id = sgt.id[li];
        uint32_t key = sgt.key[li];
        if (key >= (uint32_t)d.nbins) key = 0u;   // only after a failed wait (flagged): stay in range
        const int cell = (int)div_bin(d, key);
        g = (int)(key - (uint32_t)cell * (uint32_t)G);
        if (DIM == 3) {
          cz = cell / (nx * ny);
          const int rem = cell - cz * nx * ny;
          cy = rem / nx;
          cx = rem - cy * nx;
        } else {
          cy = DIM == 2 ? (int)div_nx(d, (uint32_t)cell) : 0;
          cx = cell - cy * nx;
        }
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
        if (cb < d.ncell) {
          if (DIM == 3) {
            cz = cb / (nx * ny);
            const int rem = cb - cz * nx * ny;
            cy = rem / nx;
            cx = rem - cy * nx;
          } else {
            cy = DIM == 2 ? (int)div_nx(d, (uint32_t)cb) : 0;
            cx = cb - cy * nx;
          }
          xi = rng.next(d.pk) * dxf;
          if (DIM >= 2) eta = rng.next(d.pk) * dyf;
          if (DIM == 3) zeta = rng.next(d.pk) * dzf;
          if (DIM == 1) {
            ox = 2.0f * rng.next(d.pk) - 1.0f;
          } else {
            const float muz = 2.0f * rng.next(d.pk) - 1.0f;
            const float ph = rng.next(d.pk);
            float sp, cp;
            sincospif(2.0f * ph, &sp, &cp);
            const float s = sqrtf(fmaxf(0.0f, 1.0f - muz * muz));
            ox = s * cp;
            oy = s * sp;
            if (DIM == 3) oz = muz;
          }
        } else {
          const int side = cb - d.ncell;
          const float u = rng.next(d.pk);
          const float m = sqrtf(rng.next(d.pk));
          const float dd = u * vf * m * dtf;
          cx = side == 0 ? -1 : nx;
          xi = side == 0 ? dxf - dd : dd;
          ox = side == 0 ? m : -m;
          gside = side;
        }
        if (!d.grey)
          nu = sample_nu_f(__ldg(d.nu_edges_f + g), __ldg(d.nu_edges_f + g + 1), __ldg(d.khat_f + bin),
                           rng.next(d.pk));
        w = __ldg(d.omega_f + bin);
      }
    }
    const int cell0 = gside >= 0 ? cx : (cz * ny + cy) * nx + cx;

    // 1/sigma(nu, T^n) in the particle's cell: the per-cell factors from
    // shared memory when the problem's table is there
    auto inv_sigma = [&](int c, float inup) -> float {
      if (!ENS && tab_n) {
        float si = s_sinv[c] * inup;
        if (tab_invT) si /= -expm1f(-nu * s_invT[c]);
        return fmaxf(si, d.inv_capf);
      }
      return inv_sigma_particle_f(d, c, nu, inup);
    };

    // ---- streaming
    int fate = FATE_REMOVED, nseg = 0, eside = -1;
    float t_tra = 0.0f;
    if (valid) {
      const float inup = d.grey ? 1.0f : pow_fast_f(nu, -spf);
      float t_rem;
      bool collided;
      if (newborn && (d.method == 0 || gside >= 0)) {   // UGKP newborns draw t_f too
        t_rem = dtf;
        collided = false;
      } else {
        const UPair u = rng.next2(d.pk);
        const float sig_inv = inv_sigma((cz * ny + cy) * nx + cx, inup);
        const float tc = neg_log_u(u) * inv_rate * sig_inv;
        collided = tc < dtf;
        t_rem = collided ? tc : dtf;
      }
      bool ghost = gside >= 0;
      const float ivx = ox != 0.0f ? __frcp_rn(vf * fabsf(ox)) : 0.0f;
      const float ivy = (DIM >= 2 && oy != 0.0f) ? __frcp_rn(vf * fabsf(oy)) : 0.0f;
      const float ivz = (DIM == 3 && oz != 0.0f) ? __frcp_rn(vf * fabsf(oz)) : 0.0f;
      for (int guard = 0;; ++guard) {
        if (guard >= 4096) {
          atomicOr(&ctrl->status, ST_NONFINITE);
          fate = FATE_REMOVED;
          break;
        }
        float tx = INFINITY, ty = INFINITY, tz = INFINITY;
        if (ox > 0.0f) tx = fmaxf(dxf - xi, 0.0f) * ivx;
        else if (ox < 0.0f) tx = fmaxf(xi, 0.0f) * ivx;
        if (DIM >= 2) {
          if (oy > 0.0f) ty = fmaxf(dyf - eta, 0.0f) * ivy;
          else if (oy < 0.0f) ty = fmaxf(eta, 0.0f) * ivy;
        }
        if (DIM == 3) {
          if (oz > 0.0f) tz = fmaxf(dzf - zeta, 0.0f) * ivz;
          else if (oz < 0.0f) tz = fmaxf(zeta, 0.0f) * ivz;
        }
        // nearest face; ties go to the lower axis
        int axis = (tx <= ty) ? 0 : 1;
        float tf = axis == 0 ? tx : ty;
        if (DIM == 3 && tz < tf) { axis = 2; tf = tz; }
        if (tf < t_rem) {
          ++nseg;
          t_tra += tf;
          t_rem -= tf;
          int dir;
          if (axis == 0) {
            dir = ox > 0.0f ? 1 : -1;
            xi = dir > 0 ? dxf : 0.0f;
            if (DIM >= 2) eta = fminf(fmaxf(fmaf(vf * oy, tf, eta), 0.0f), dyf);
            if (DIM == 3) zeta = fminf(fmaxf(fmaf(vf * oz, tf, zeta), 0.0f), dzf);
          } else if (DIM < 3 || axis == 1) {
            dir = oy > 0.0f ? 1 : -1;
            eta = dir > 0 ? dyf : 0.0f;
            xi = fminf(fmaxf(fmaf(vf * ox, tf, xi), 0.0f), dxf);
            if (DIM == 3) zeta = fminf(fmaxf(fmaf(vf * oz, tf, zeta), 0.0f), dzf);
          } else {
            dir = oz > 0.0f ? 1 : -1;
            zeta = dir > 0 ? dzf : 0.0f;
            xi = fminf(fmaxf(fmaf(vf * ox, tf, xi), 0.0f), dxf);
            eta = fminf(fmaxf(fmaf(vf * oy, tf, eta), 0.0f), dyf);
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
          if (axis == 0) xi = dir > 0 ? 0.0f : dxf;
          else if (axis == 1) eta = dir > 0 ? 0.0f : dyf;
          else zeta = dir > 0 ? 0.0f : dzf;
          cx = nxc;
          cy = nyc;
          cz = nzc;
          const UPair u = rng.next2(d.pk);
          const float sig_inv = inv_sigma((cz * ny + cy) * nx + cx, inup);
          const float tc = neg_log_u(u) * inv_rate * sig_inv;
          const float avail = dtf - t_tra;
          collided = tc < avail;
          t_rem = collided ? tc : avail;
          continue;
        }
        ++nseg;
        xi = fminf(fmaxf(fmaf(vf * ox, t_rem, xi), 0.0f), dxf);
        if (DIM >= 2) eta = fminf(fmaxf(fmaf(vf * oy, t_rem, eta), 0.0f), dyf);
        if (DIM == 3) zeta = fminf(fmaxf(fmaf(vf * oz, t_rem, zeta), 0.0f), dzf);
        t_tra += t_rem;
        fate = ghost ? FATE_REMOVED : (collided ? FATE_ABSORBED : FATE_SURVIVED);
        break;
      }
    }
    const int cell = (cz * ny + cy) * nx + cx;

    // ---- in place: slot i of the other buffer (kDeadKey unless it survived)
    const bool keep = valid && fate == FATE_SURVIVED;
    const bool room = i < d.capacity;
    const bool stored = keep && room;
    if (valid && room) {
      d.fx[nxb][i] = xi;
      d.fox[nxb][i] = ox;
      if (DIM >= 2) { d.fy[nxb][i] = eta; d.foy[nxb][i] = oy; }
      if (DIM == 3) { d.fz[nxb][i] = zeta; d.foz[nxb][i] = oz; }
      d.fnu[nxb][i] = nu;
      d.fw[nxb][i] = w;
      d.pid[nxb][i] = id;
      d.pkey[nxb][i] = stored ? (uint32_t)(cell * G + g) : kDeadKey;
    }
    if (keep && !room) atomicOr(&ctrl->status, ST_CAPACITY);

    // ---- tallies (W and E_surv in fixed point, see to_fixed_f; FP64 side
    // tallies).  A survivor that found no slot is counted in W but not in
    // E_surv: its energy stays with the wave part.
    const long long wq = valid ? to_fixed_f(w, d.tq_shift, &ctrl->status) : 0ll;
    warp_run_add_fixed(d.Esq, stored ? cell * G + g : -1 - lane, wq, d.sort_cnt);
    if (valid && fate != FATE_REMOVED && (gside >= 0 || fate == FATE_ESCAPED || cell0 != cell)) {
      const double wd = (double)w;
      const bool start_in = gside < 0;
      const bool end_in = fate == FATE_SURVIVED || fate == FATE_ABSORBED;
      if (start_in) atomic_add_fixed(d.Wq + 2 * (cell0 * G + g), -wq);
      if (end_in) atomic_add_fixed(d.Wq + 2 * (cell * G + g), wq);
      if (!start_in) atomicAdd(d.inflow + gside * G + g, wd);
      if (fate == FATE_ESCAPED) atomicAdd(d.esc + eside * G + g, wd);
    }
    if (valid) {
      cnt.seg += (unsigned)nseg;
      cnt.abs += fate == FATE_ABSORBED;
      cnt.esc += fate == FATE_ESCAPED;
      cnt.surv += fate == FATE_SURVIVED;
      cnt.rem += fate == FATE_REMOVED;
      if (!ENS && d.rec && i < d.rec_cap) {
        RecordOut& rr = d.rec[i];
        rr.id = id; rr.fate = fate; rr.cell0 = cell0; rr.cell1 = (fate == FATE_REMOVED && gside >= 0) ? cx : cell;
        rr.grp = g; rr.nseg = nseg; rr.pad = 0;
        rr.x = cx * d.dx + (double)xi;
        rr.y = DIM >= 2 ? cy * d.dy + (double)eta : 0.0;
        rr.ox = ox; rr.oy = oy; rr.nu = nu; rr.w = (double)w; rr.t_end = t_tra;
        rr.z = DIM == 3 ? cz * d.dz + (double)zeta : 0.0;
        rr.oz = oz;
      }
    }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&s_empty[st]);
  }
  flush_counters(ENS ? e.devs[acc_m].ctrl : d0.ctrl, cnt);
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

template <int DIM, bool ENS, int NT>
static cudaError_t launch_stream32_t(const Dev& d, const Ens& e, const StreamShape& sh, cudaStream_t s) {
  const int sms = sm_count();
  const void* fn = (const void*)k_stream32<DIM, ENS, NT>;
  const int tile = NT * sh.ppt;
  const size_t dyn = kStages * stream32_stage_bytes(DIM, tile) + (ENS ? 0 : 4 * (size_t)stream32_table_floats(d));
  const int bi = NT == 128 ? 0 : (NT == 512 ? 2 : 1);
  int& occ = g_stream32_occ[DIM][ENS][bi];
  int& occ_dyn = g_stream32_occ_dyn[DIM][ENS][bi];
  if (!occ || occ_dyn != (int)dyn) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, NT + 32, dyn);
    if (occ < 1) occ = 1;
    occ_dyn = (int)dyn;
  }
  const int per = sh.blocks_per_sm > 0 && sh.blocks_per_sm < occ ? sh.blocks_per_sm : occ;
  k_stream32<DIM, ENS, NT><<<sms * per, NT + 32, dyn, s>>>(d, e, sh.ppt);
  return cudaGetLastError();
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
    if (sh.ppt == 2) return launch_stream64_t<2, ENS, 2>(d, e, sh, s);
    return launch_stream64_t<2, ENS, 1>(d, e, sh, s);
  }
  if (mixed) return launch_stream32_nt<1, ENS>(d, e, sh, s);
  if (sh.ppt == 2) return launch_stream64_t<1, ENS, 2>(d, e, sh, s);
  return launch_stream64_t<1, ENS, 1>(d, e, sh, s);
}

cudaError_t launch_stream(const Dev& d, const Ens* e, const StreamShape& sh, cudaStream_t s) {
  const int mixed = d.precision == 1;
  if (e && e->M > 1) return launch_stream_dim<true>(d, *e, mixed, sh, s);
  const Ens none{};
  return launch_stream_dim<false>(d, none, mixed, sh, s);
}

}  // namespace ugkwp
