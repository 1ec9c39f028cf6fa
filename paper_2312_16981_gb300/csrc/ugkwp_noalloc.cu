// ugkwp_noalloc.cu -- an exclusive scan of birth counts that allocates
// nothing, for callers that cannot obtain device memory.
//
// Who needs it: code that runs where device allocation is unavailable or
// not allowed -- a host program whose GPU memory is entirely owned by its
// own pool allocator, a plug-in invoked by a framework that forbids
// cudaMalloc/cudaFree during its time step (those calls can synchronise the
// whole device), or a caller that only holds pointers to buffers someone
// else allocated.  Such a caller cannot provide the scratch buffer that
// ugkwp_exclusive_scan asks for; this variant keeps that scratch (the
// per-block partial sums) in a fixed device array compiled into the library.
//
// The array holds UGKWP_NOALLOC_SCAN_MAX_N / 4096 + 1 words (16 KiB) and stays
// resident on every GPU that loads the library until the process exits.
#include <atomic>
#include <cstdio>

#include "../../include/ugkwp.h"
#include "ugkwp_launch.h"

namespace {

// one partial sum per block of the scan kernels (ugkwp::kScanTileCounts
// counts each, the tile launch_scan splits the counts by), plus one
constexpr long long kMaxParts = UGKWP_NOALLOC_SCAN_MAX_N / ugkwp::kScanTileCounts + 1;
static_assert((UGKWP_NOALLOC_SCAN_MAX_N + ugkwp::kScanTileCounts - 1) / ugkwp::kScanTileCounts < kMaxParts,
              "the static scratch holds the partials of the largest accepted n");

// Per-block partial sums of the scan.  Every call overwrites the entries it
// reads before reading them, so nothing has to start at zero.
static __device__ __align__(256) uint32_t g_scan_partials[kMaxParts];

// Device address of g_scan_partials per device.  In host code the symbol is
// only a host-side stand-in, so the address is looked up once per device
// with that device current.  Host threads may make their first calls at the
// same time: the cache is atomic (each would store the same address).
std::atomic<uint32_t*> g_partials_addr[ugkwp::kMaxDevices];

int fail(int code, const char* fmt, const char* detail) {
  char buf[256];
  snprintf(buf, sizeof buf, fmt, detail);
  ugkwp::set_global_error(buf);   // read back with ugkwp_last_error(NULL)
  return code;
}

}  // namespace

extern "C" int ugkwp_exclusive_scan_noalloc(const uint32_t* d_counts, int64_t n, uint32_t* d_offsets,
                                            void* stream) {
  if (n < 0 || n > UGKWP_NOALLOC_SCAN_MAX_N || !d_offsets || (n > 0 && !d_counts))
    return fail(UGKWP_ERR_ARG, "%s",
                "bad arguments: need 0 <= n <= UGKWP_NOALLOC_SCAN_MAX_N (2^24, the size of the "
                "static scratch), and counts and offsets");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= ugkwp::kMaxDevices)
    return fail(UGKWP_ERR_CUDA, "no usable current device (%s)", cudaGetErrorString(e));
  uint32_t* part = g_partials_addr[dev].load(std::memory_order_acquire);
  if (!part) {
    e = cudaGetSymbolAddress((void**)&part, g_scan_partials);
    if (e != cudaSuccess || !part) return fail(UGKWP_ERR_CUDA, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    g_partials_addr[dev].store(part, std::memory_order_release);
  }
  e = ugkwp::launch_scan(d_counts, n, part, d_offsets, nullptr, nullptr, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(UGKWP_ERR_CUDA, "scan launch failed: %s", cudaGetErrorString(e));
  return UGKWP_OK;
}
