// Stable LSD radix sort of (uint32 key, uint32 value) pairs, onesweep style.
//
// One histogram kernel reads the keys once and counts all digit passes (as many passes as 8-bit
// digits need, the key's bits then spread evenly over them: 13 tile bits as 7 + 6); then each
// pass is a single kernel: a block takes the next 4096-key tile (virtual id from an atomic counter),
// ranks its keys per digit within each warp (stable: item-major then lane order within a warp,
// warps in order), publishes its per-digit counts (the sums of the warps' counts), reorders the
// tile by digit in shared memory (so that the global writes come out in runs), and looks back
// across earlier tiles per digit (one thread per digit, 4 status words per round, bounded waits)
// to find its global offsets.
#include <algorithm>

#include "dev_common.cuh"

namespace v3dg {
namespace {

constexpr int kBins = 256;
constexpr int kLookback = 4;   // status words read per look-back round
constexpr int kWarps = kSortThreads / 32;
static_assert(kSortThreads >= kBins, "one thread per digit");

// Digit counts of every pass in one read of the keys (one shared histogram per pass and block).
// A thread counts a run of kHistRun consecutive keys and adds each pass's digit to the shared
// histogram only when it changes (runs of equal digits are common: the high digits of nearby
// keys -- depths of one cluster, tiles of one Gaussian -- coincide), which keeps shared-memory
// atomics on the few hot bins of the high digits from serialising.
constexpr int kHistRun = 16;

__global__ void __launch_bounds__(256)
k_hist(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ n_dev, uint32_t cap, int begin_bit,
       int end_bit, int passes, int width, uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[4][kBins];
  for (int i = threadIdx.x; i < 4 * kBins; i += blockDim.x) sh[i / kBins][i % kBins] = 0;
  __syncthreads();
  const uint32_t n = min(*n_dev, cap);
  int sh_[4];
  uint32_t m[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    sh_[p] = begin_bit + width * p;
    m[p] = (1u << min(max(end_bit - sh_[p], 0), width)) - 1u;
  }
  const uint32_t runs = (n + kHistRun - 1) / kHistRun;
  const bool aligned = (reinterpret_cast<uintptr_t>(keys) & 15u) == 0;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < runs; r += gridDim.x * blockDim.x) {
    const uint32_t i0 = r * kHistRun;
    uint32_t cur[4], cnt[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      cur[p] = 0xFFFFFFFFu;
      cnt[p] = 0;
    }
    if (aligned && i0 + kHistRun <= n) {   // a full run: four 16-byte loads
      const uint4* v = reinterpret_cast<const uint4*>(keys + i0);
#pragma unroll
      for (int q = 0; q < kHistRun / 4; ++q) {
        const uint4 k4 = v[q];
        const uint32_t kk[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            if (p >= passes) break;
            const uint32_t d = (kk[t] >> sh_[p]) & m[p];
            if (d != cur[p]) {
              if (cnt[p]) atomicAdd(&sh[p][cur[p]], cnt[p]);
              cur[p] = d;
              cnt[p] = 0;
            }
            ++cnt[p];
          }
      }
    } else {
      for (uint32_t i = i0; i < min(i0 + kHistRun, n); ++i) {
        const uint32_t k = keys[i];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          if (p >= passes) break;
          const uint32_t d = (k >> sh_[p]) & m[p];
          if (d != cur[p]) {
            if (cnt[p]) atomicAdd(&sh[p][cur[p]], cnt[p]);
            cur[p] = d;
            cnt[p] = 0;
          }
          ++cnt[p];
        }
      }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
      if (cnt[p]) atomicAdd(&sh[p][cur[p]], cnt[p]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kBins; i += blockDim.x) {
    const uint32_t c = sh[i / kBins][i % kBins];
    if (c) atomicAdd(hist + i, c);
  }
}

// Exclusive scan over digits of each pass's global histogram: the first output position of each
// digit (one block, one thread per digit).
__global__ void __launch_bounds__(kBins) k_hist_scan(const uint32_t* __restrict__ hist, int passes,
                                                     uint32_t* __restrict__ excl) {
  __shared__ uint32_t s_scan[kBins / 32 + 1];
  for (int p = 0; p < passes; ++p) {
    uint32_t total;
    excl[p * kBins + threadIdx.x] = block_exclusive_scan<kBins / 32>(hist[p * kBins + threadIdx.x], s_scan, &total);
  }
}

template <bool kImplicit>
__global__ void __launch_bounds__(kSortThreads, 4)
k_onesweep(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
           uint32_t* __restrict__ vout, const uint32_t* __restrict__ n_dev, uint32_t cap, int shift, uint32_t dmask,
           const uint32_t* __restrict__ gexcl, uint64_t* __restrict__ status, uint32_t* __restrict__ tile_counter,
           uint32_t epoch, uint32_t* __restrict__ err) {
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ uint32_t s_vals[kSortTile];
  __shared__ uint16_t s_wh[kWarps][kBins];   // per-warp digit counts, then per-warp exclusive offsets
  __shared__ uint32_t s_start[kBins];        // block-local start of each digit
  __shared__ uint32_t s_goff[kBins];         // global destination offset minus local start (mod 2^32)
  __shared__ uint32_t s_cnt[kBins];          // the tile's digit counts
  __shared__ uint32_t s_scan[kWarps + 1];
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_match[kWarps][kBins];   // per warp, the lanes holding each digit (zero between items)

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t n = min(*n_dev, cap);
  const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
  for (int i = tid; i < kWarps * kBins; i += kSortThreads) (&s_match[0][0])[i] = 0u;
  // persistent blocks: tiles in the order of an atomic counter, so every tile a look-back waits
  // for is held by a running block
  for (;;) {
  if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  if (tile >= ntiles) return;
  for (int i = tid; i < kWarps * kBins / 2; i += kSortThreads) reinterpret_cast<uint32_t*>(&s_wh[0][0])[i] = 0;
  __syncthreads();
  const uint32_t base = tile * kSortTile + warp * (kSortItems * 32);

  uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t idx = base + i * 32 + lane;
    const bool ok = idx < n;
    key[i] = ok ? kin[idx] : 0xFFFFFFFFu;
    val[i] = kImplicit ? idx : (ok ? vin[idx] : 0u);
  }
  // warp-level stable ranking: item-major, then lane order.  The lanes that share a digit come
  // from a shared-memory OR of lane bits (measured faster than match.any), or are the whole warp
  // when every lane has the same digit (common in the high digits of the depth keys, where the
  // OR would serialise on one word).
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t idx = base + i * 32 + lane;
    const bool ok = idx < n;
    const uint32_t live = __ballot_sync(0xffffffffu, ok);
    rank[i] = 0;
    if (ok) {
      const uint32_t d = (key[i] >> shift) & dmask;
      const uint32_t d0 = __shfl_sync(live, d, __ffs(live) - 1);
      const bool same = __all_sync(live, d == d0);   // (uniform over the live lanes)
      uint32_t peers = live;
      if (!same) {
        atomicOr(&s_match[warp][d], 1u << lane);
        __syncwarp(live);
        peers = s_match[warp][d];
      }
      const uint32_t before = __popc(peers & lanemask_lt());
      const uint32_t cur = s_wh[warp][d];
      __syncwarp(live);
      if (before == 0) {   // the digit's first lane: advance the warp's count, clear the lane bits
        s_wh[warp][d] = uint16_t(cur + __popc(peers));
        if (!same) s_match[warp][d] = 0u;
      }
      __syncwarp(live);
      rank[i] = cur + before;
    }
  }
  __syncthreads();
  // per digit (threads 0..255): exclusive offsets across warps, the block count, and the chain
  uint32_t cnt = 0;
  if (tid < kBins) {
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = s_wh[w][tid];
      s_wh[w][tid] = uint16_t(cnt);
      cnt += c;
    }
  }
  if (tid <= dmask) {   // the tile's digit counts, published as soon as they are known
    chain_publish(status + tid, kBins, tile, cnt, epoch);
    s_cnt[tid] = cnt;
  }
  uint32_t total;
  const uint32_t start = block_exclusive_scan<kWarps>(cnt, s_scan, &total);
  if (tid < kBins) s_start[tid] = start;
  __syncthreads();
  // reorder the tile by digit in shared memory (before the look-back, which needs none of the
  // tile's registers and gets the earlier tiles more time to publish)
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t idx = base + i * 32 + lane;
    if (idx < n) {
      const uint32_t dg = (key[i] >> shift) & dmask;
      const uint32_t pos = s_start[dg] + s_wh[warp][dg] + rank[i];
      s_keys[pos] = key[i];
      s_vals[pos] = val[i];
    }
  }
  if (tid <= dmask) {   // (the digit's count and start reloaded: no registers held over the reorder)
    const uint32_t excl = chain_lookback<kLookback>(status + tid, kBins, tile, s_cnt[tid], epoch, err);
    s_goff[tid] = gexcl[tid] + excl - s_start[tid];   // wraps; dst = s_goff + p is exact below 2^32
  }
  __syncthreads();
  const uint32_t valid = min(uint32_t(kSortTile), n - tile * kSortTile);
#pragma unroll 4
  for (uint32_t p = tid; p < valid; p += kSortThreads) {
    const uint32_t k = s_keys[p];
    const uint32_t dst = s_goff[(k >> shift) & dmask] + p;
    kout[dst] = k;
    vout[dst] = s_vals[p];
  }
  __syncthreads();   // the tile's shared data is consumed before the next tile reuses it
  }  // next tile
}

// Diagnostic of the bounded waits: warp 0 runs the radix-sort passes' look-back (one thread,
// kLookback words per round), warp 1 the warp-wide look-back of the compaction and expansion
// kernels, each as tile 1 of its own two-word chain whose tile 0 publishes the prefix 1000 + warp
// (publish != 0) or never publishes (its word keeps an epoch that is not `epoch`).
__global__ void k_check_wait(uint64_t* __restrict__ status, uint32_t epoch, uint32_t spin_limit, int publish,
                             uint32_t* __restrict__ out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t* chain = status + 2 * warp;
  if (lane == 0 && publish) chain_publish(chain, 1, 0, 1000u + uint32_t(warp), epoch);
  __syncwarp();
  if (warp == 0) {
    if (lane == 0) out[0] = chain_lookback<kLookback>(chain, 1, 1, 1u, epoch, out + 2, spin_limit);
  } else {
    const uint32_t e = chained_exclusive_warp(chain, 1, 1u, epoch, out + 2, spin_limit);
    if (lane == 0) out[1] = e;
  }
}

}  // namespace

int g_sort_blocks_per_sm = 4;   // resident onesweep blocks per SM (set with the attributes)

cudaError_t sort_set_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_onesweep<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_onesweep<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep<false>, kSortThreads, 0);
  if (e == cudaSuccess && per_sm > 0) g_sort_blocks_per_sm = per_sm;
  return e;
}

cudaError_t launch_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const uint32_t* n_dev,
                        uint32_t cap, int begin_bit, int end_bit, bool implicit_vals, const SortScratch& sc,
                        uint32_t* err_flag, uint32_t& epoch, int sm_count, cudaStream_t st, bool* result_in_1,
                        int* launches) {
  const int passes = (end_bit - begin_bit + 7) / 8;
  const int width = passes > 0 ? (end_bit - begin_bit + passes - 1) / passes : 8;   // balanced digits
  *result_in_1 = false;
  if (passes <= 0 || cap == 0) return cudaSuccess;
  if (passes > 4) return cudaErrorInvalidValue;
  const uint32_t max_tiles = (cap + kSortTile - 1) / kSortTile;
  if (max_tiles > sc.max_tiles) return cudaErrorInvalidValue;
  // persistent grid: the resident blocks, whatever the capacity (surplus blocks cost launches)
  const uint32_t grid = std::min<uint32_t>(max_tiles, uint32_t(sm_count) * uint32_t(g_sort_blocks_per_sm));
  cudaError_t e = cudaMemsetAsync(sc.hist, 0, sizeof(uint32_t) * kBins * passes, st);
  if (e != cudaSuccess) return e;
  k_hist<<<sm_count * 4, 256, 0, st>>>(k0, n_dev, cap, begin_bit, end_bit, passes, width, sc.hist);
  k_hist_scan<<<1, kBins, 0, st>>>(sc.hist, passes, sc.hist + 4 * kBins);
  *launches += 2;
  uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
  for (int p = 0; p < passes; ++p) {
    const int shift = begin_bit + width * p;
    const uint32_t dmask = (1u << std::min(end_bit - shift, width)) - 1u;
    epoch = (epoch + 1) & 0x3FFFFFFFu;
    if (epoch == 0) epoch = 1;
    const uint32_t ep = epoch;
    if (p == 0 && implicit_vals)
      k_onesweep<true><<<grid, kSortThreads, 0, st>>>(ki, vi, ko, vo, n_dev, cap, shift, dmask, sc.hist + 4 * kBins + kBins * p,
                                                           sc.status, sc.tile_counters + p, ep, err_flag);
    else
      k_onesweep<false><<<grid, kSortThreads, 0, st>>>(ki, vi, ko, vo, n_dev, cap, shift, dmask, sc.hist + 4 * kBins + kBins * p,
                                                            sc.status, sc.tile_counters + p, ep, err_flag);
    ++*launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  *result_in_1 = (passes & 1) != 0;
  return cudaSuccess;
}

cudaError_t launch_check_wait(uint64_t* status, uint32_t epoch, uint32_t spin_limit, int publish, uint32_t* out,
                              cudaStream_t st) {
  k_check_wait<<<1, 64, 0, st>>>(status, epoch, spin_limit, publish, out);
  return cudaGetLastError();
}

}  // namespace v3dg
