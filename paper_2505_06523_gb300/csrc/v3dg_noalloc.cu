// v3dg_sort_pairs_noalloc: the pair sort for callers that cannot allocate device memory.
//
// Some hosts own all device memory themselves: an engine or renderer that reserves its pools at
// start-up and forbids later allocations, or a real-time frame loop where cudaMalloc / cudaFree
// would stall the frame (both can synchronise the device) or fail under a fixed memory budget.
// This entry point serves them: it calls no cudaMalloc, cudaFree or other allocating routine.
// Its scratch (the ping-pong buffers, histograms and look-back status words of the radix sort)
// lives in one file-scope device array, g_scratch, sized for V3DG_SORT_NOALLOC_MAX_PAIRS pairs
// (about 8.5 MB).  Every GPU that loads the library holds that array until the process exits.
//
// In host code the name g_scratch is only a host-side stand-in for the device symbol, not a
// device address.  The first call on each device (with that device current) resolves the address
// with cudaGetSymbolAddress and caches it; that first call should come before any stream capture,
// and the cached address does not survive a device reset (cudaDeviceReset), after which the entry
// point must not be used in the same process.
// All calls share the one array and its contents persist between calls: each call clears the
// words that must start at zero, and calls whose work overlaps on the GPU race with each other.
// The look-back status words are not cleared per call; each call tags them with fresh epochs
// from a 64-bit call counter, and the whole status area is cleared whenever the 30-bit epoch
// sequence starts over, so a stale word from an earlier call never carries a current epoch.
#include <atomic>
#include <mutex>

#include <cuda_runtime.h>

#include "v3dg.h"
#include "v3dg_internal.h"

using namespace v3dg;

namespace {

constexpr uint64_t kMaxPairs = V3DG_SORT_NOALLOC_MAX_PAIRS;
constexpr uint32_t kTiles = uint32_t((kMaxPairs + kSortTile - 1) / kSortTile);
constexpr size_t kOffKeys = 0;
constexpr size_t kOffVals = kOffKeys + 4 * kMaxPairs;
constexpr size_t kOffStatus = kOffVals + 4 * kMaxPairs;
constexpr size_t kOffHist = kOffStatus + 8 * size_t(kTiles) * 256;
constexpr size_t kOffMisc = kOffHist + 2 * 4 * 256 * 4;   // [0] n, [1..4] tile counters, [5] timeout flag
constexpr size_t kBytes = kOffMisc + 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kBytes];

std::mutex g_mu;
void* g_base[kMaxDevices] = {};
std::atomic<uint64_t> g_calls{0};
// each call takes 8 consecutive epochs (the sort uses at most 4); the sequence has this period
constexpr uint64_t kEpochCalls = ((1u << 30) - 16u) / 8u;

__global__ void k_store_n(uint32_t* p, uint32_t v) { *p = v; }

}  // namespace

extern "C" v3dg_status v3dg_sort_pairs_noalloc(uint32_t* keys, uint32_t* vals, uint64_t n, int begin_bit, int end_bit,
                                               void* cuda_stream) {
  if (n == 0) return V3DG_OK;
  if (!keys || !vals) return V3DG_EINVAL;
  if (begin_bit < 0 || end_bit > 32 || begin_bit >= end_bit) return V3DG_EINVAL;
  if (n > kMaxPairs) return V3DG_EOVERFLOW;  // beyond the fixed scratch: nothing is done
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return V3DG_ECUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return V3DG_ECUDA;
      g_base[dev] = p;
    }
    base = g_base[dev];
  }
  int sm = 0;
  if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return V3DG_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* b = static_cast<unsigned char*>(base);
  uint32_t* misc = reinterpret_cast<uint32_t*>(b + kOffMisc);
  if (cudaMemsetAsync(misc, 0, 64, st) != cudaSuccess) return V3DG_ECUDA;
  k_store_n<<<1, 1, 0, st>>>(misc, uint32_t(n));
  SortScratch sc;
  sc.hist = reinterpret_cast<uint32_t*>(b + kOffHist);
  sc.status = reinterpret_cast<uint64_t*>(b + kOffStatus);
  sc.max_tiles = kTiles;
  sc.tile_counters = misc + 1;
  // fresh epochs for the look-back status words, which keep earlier calls' contents; when the
  // sequence starts over, clear them so that no word left by an earlier call matches an epoch
  const uint64_t call = g_calls.fetch_add(1);
  uint32_t epoch = uint32_t(8u * (call % kEpochCalls)) + 1u;
  if (call % kEpochCalls == 0 &&
      cudaMemsetAsync(b + kOffStatus, 0, 8 * size_t(kTiles) * 256, st) != cudaSuccess)
    return V3DG_ECUDA;
  bool in1 = false;
  int launches = 0;
  uint32_t* tk = reinterpret_cast<uint32_t*>(b + kOffKeys);
  uint32_t* tv = reinterpret_cast<uint32_t*>(b + kOffVals);
  if (launch_sort(keys, vals, tk, tv, misc, uint32_t(n), begin_bit, end_bit, false, sc, misc + 5, epoch, sm, st, &in1,
                  &launches) != cudaSuccess)
    return V3DG_ECUDA;
  if (in1) {
    if (cudaMemcpyAsync(keys, tk, 4 * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return V3DG_ECUDA;
    if (cudaMemcpyAsync(vals, tv, 4 * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return V3DG_ECUDA;
  }
  uint32_t timeout = 0;
  if (cudaMemcpyAsync(&timeout, misc + 5, sizeof timeout, cudaMemcpyDeviceToHost, st) != cudaSuccess) return V3DG_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return V3DG_ECUDA;
  return timeout ? V3DG_ETIMEOUT : V3DG_OK;
}
