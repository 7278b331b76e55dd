// noalloc.cu -- dg_lower_bound_noalloc: the lower bound of dg_lower_bound
// computed without any scratch memory from the caller.
//
// Some callers cannot allocate device memory at the time they want a bound:
// code running inside a CUDA graph capture that forbids cudaMalloc, embedders
// whose allocator is owned by another runtime, or a serving loop with a
// fixed, pre-planned memory budget.  dg_lower_bound writes its intermediates
// (E^j per row, S_i and S_i / |J_i| per variable, one FP64 partial sum per
// reduction chunk, the path costs of long BDDs) into the scratch area of the
// caller's arena buffer; this
// variant keeps them in one file-scope __device__ array instead, so the
// caller passes only the inputs (lambda, M) and the output (bound per
// instance).  The arena's own scratch area is left untouched.
//
// Limits and sharing:
//  * the array holds kNoallocScratchBytes (4 MiB); arenas whose intermediates
//    need more (4 m + 8 n + 8 chunks + 4 per node of the long BDDs bytes) are
//    rejected with DG_EINVAL;
//  * every GPU that loads libdg holds the array until the process exits;
//  * all calls share it: two calls whose kernels overlap on the GPU (on
//    different streams, or from different host threads) race on it.  Calls
//    ordered on one stream are safe.  Every kernel overwrites every
//    intermediate it later reads, so nothing needs to start at zero.
//  * the first call on a device looks up the array's device address (host
//    code only sees a stand-in for it) with that device current; make that
//    first call before any stream capture.  The address is cached per device
//    ordinal for the life of the process, so a cudaDeviceReset (which
//    destroys the context holding the array) leaves the cache stale: do not
//    call this entry point after resetting the device.
#include <mutex>
#include <string>

#include "kernels.h"

namespace dg {

constexpr size_t kNoallocScratchBytes = size_t(4) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[128] = {nullptr};

// Device address of g_noalloc_scratch on the current device (looked up once
// per device).
dg_status noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(DG_ECUDA, std::string("dg_lower_bound_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 128) return fail(DG_EINVAL, "dg_lower_bound_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(DG_ECUDA, std::string("dg_lower_bound_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return DG_OK;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

dg_status lower_bound_noalloc(const DevArena& arena, const LaunchGroup* groups, int num_groups, int threads,
                              const StreamSet& ss, const float* lam, const float* M, double* lb) {
  cudaStream_t st = ss.main;
  const size_t bE = up256((size_t)arena.m * 4), bS = up256((size_t)arena.n * 4);
  const size_t bP = up256((size_t)arena.num_lb_chunks * 8);
  const size_t bL = up256((size_t)arena.long_cost_size * 4);
  const size_t need = bE + 2 * bS + bP + bL;
  if (need > kNoallocScratchBytes)
    return fail(DG_EINVAL, "dg_lower_bound_noalloc: this arena needs " + std::to_string(need) +
                               " bytes of scratch, more than the " + std::to_string(kNoallocScratchBytes) +
                               " bytes of the static array (4 m + 8 n + 8 chunks + 4 per long-BDD node must fit)");
  void* base = nullptr;
  if (dg_status s = noalloc_scratch(&base)) return s;
  char* p = static_cast<char*>(base);
  DevArena A = arena;  // same structure, intermediates redirected
  A.E = reinterpret_cast<float*>(p);
  A.S = reinterpret_cast<float*>(p + bE);
  A.Sbar = reinterpret_cast<float*>(p + bE + bS);
  A.slot_avg = nullptr;  // the bound's S reduction leaves the per-slot terms alone
  A.lb_part = reinterpret_cast<double*>(p + bE + 2 * bS);
  A.long_t = reinterpret_cast<float*>(p + bE + 2 * bS + bP);  // SP(., T) of the long BDDs' nodes
  A.long_d = nullptr;                                         // not read by the energy pass
  SweepArgs a{};
  a.lam = const_cast<float*>(lam);
  a.E = A.E;
  launch_sweep(kEnergy, A, a, threads, groups, num_groups, ss);
  launch_reduce_S(A, M, nullptr, nullptr, 0, false, st, false);
  launch_lower_bound(A, lb, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DG_ECUDA, std::string("dg_lower_bound_noalloc: ") + cudaGetErrorString(e));
  return DG_OK;
}

}  // namespace dg
