// Tile binning: pair offsets, duplication of each visible Gaussian into its tiles, tile ranges.
//
// The Gaussians arrive sorted by depth (stage one of the two-stage (tile, depth) sort), so the
// pairs are emitted in depth order; a stable sort on the tile id then yields (tile, depth, id)
// order, and each tile's range of the sorted pairs is found by boundary detection.
#include "dev_common.cuh"

namespace v3dg {
namespace {

constexpr int kScanThreads = 256, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t rect_area(const uint2 r) {
  const uint32_t w = (r.x >> 16) - (r.x & 0xFFFFu) + 1u;
  const uint32_t h = (r.y >> 16) - (r.y & 0xFFFFu) + 1u;
  return w * h;
}

__global__ void __launch_bounds__(kScanThreads)
k_pair_scan(const uint32_t* __restrict__ slots, const uint2* __restrict__ rect, uint32_t cap,
            uint32_t* __restrict__ offsets, uint32_t* __restrict__ frame, uint32_t tc_slot,
            uint64_t* __restrict__ status, uint32_t epoch) {
  __shared__ uint32_t s_tile, s_excl;
  __shared__ uint32_t s_scan[kScanThreads / 32 + 1];
  if (threadIdx.x == 0) s_tile = atomicAdd(frame + kTileCounters + tc_slot, 1u);
  __syncthreads();
  const uint32_t n = min(frame[kVisible], cap);
  const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
  const uint32_t tile = s_tile;
  if (tile >= ntiles) return;
  const uint32_t i0 = tile * kScanTile + threadIdx.x * kScanItems;
  uint32_t c[kScanItems], sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    c[i] = (i0 + i < n) ? rect_area(rect[slots[i0 + i]]) : 0u;
    sum += c[i];
  }
  uint32_t total;
  uint32_t ex = block_exclusive_scan<kScanThreads / 32>(sum, s_scan, &total);
  if (threadIdx.x == 0) s_excl = chained_exclusive(status, 1, tile, total, epoch, frame + kTimeout);
  __syncthreads();
  ex += s_excl;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (i0 + i < n) offsets[i0 + i] = ex;
    ex += c[i];
  }
  if (threadIdx.x == 0 && tile == ntiles - 1) frame[kPairs] = s_excl + total;
}

__global__ void __launch_bounds__(256)
k_duplicate(const uint32_t* __restrict__ slots, const uint2* __restrict__ rect, const uint32_t* __restrict__ offsets,
            uint32_t cap, uint32_t cap_pairs, int tiles_x, uint32_t* __restrict__ pk, uint32_t* __restrict__ pv,
            uint32_t* __restrict__ frame) {
  const uint32_t n = min(frame[kVisible], cap);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t slot = slots[k];
    const uint2 r = rect[slot];
    const uint32_t tx0 = r.x & 0xFFFFu, tx1 = r.x >> 16, ty0 = r.y & 0xFFFFu, ty1 = r.y >> 16;
    uint32_t o = offsets[k];
    if (uint64_t(o) + rect_area(r) > cap_pairs) {
      atomicOr(frame + kOverflow, 1u);
      continue;
    }
    if (ty1 < ty0 || tx1 < tx0 || ty1 >= 0xFFFFu || tx1 >= uint32_t(tiles_x)) continue;
    for (uint32_t ty = ty0; ty <= ty1; ++ty)
      for (uint32_t tx = tx0; tx <= tx1; ++tx, ++o) {
        pk[o] = ty * uint32_t(tiles_x) + tx;
        pv[o] = slot;
      }
  }
}

// After duplication: the pair count that later stages use (none when the frame overflowed, so
// that no stage reads pair slots that were not written).
__global__ void k_pairs_eff(uint32_t* frame, uint32_t cap_pairs) {
  frame[kPairsEff] = frame[kOverflow] ? 0u : min(frame[kPairs], cap_pairs);
}

__global__ void __launch_bounds__(256)
k_ranges(const uint32_t* __restrict__ tk, uint32_t cap_pairs, const uint32_t* __restrict__ frame,
         uint2* __restrict__ ranges, uint32_t n_tiles) {
  const uint32_t n = min(frame[kPairsEff], cap_pairs);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t t = tk[k];
    if (t >= n_tiles) continue;
    if (k == 0 || tk[k - 1] != t) ranges[t].x = k;
    if (k + 1 == n || tk[k + 1] != t) ranges[t].y = k + 1;
  }
}

}  // namespace

cudaError_t launch_pair_scan(const uint32_t* slots, const uint2* rect, uint32_t cap, uint32_t* offsets,
                             uint32_t* frame, uint32_t tc_slot, uint64_t* status, uint32_t epoch, cudaStream_t st) {
  const uint32_t blocks = (cap + kScanTile - 1) / kScanTile;
  if (blocks == 0) return cudaSuccess;
  k_pair_scan<<<blocks, kScanThreads, 0, st>>>(slots, rect, cap, offsets, frame, tc_slot, status, epoch);
  return cudaGetLastError();
}

cudaError_t launch_duplicate(const uint32_t* slots, const uint2* rect, const uint32_t* offsets, uint32_t cap,
                             uint32_t cap_pairs, int tiles_x, uint32_t* pk, uint32_t* pv, uint32_t* frame,
                             int sm_count, cudaStream_t st) {
  k_duplicate<<<sm_count * 8, 256, 0, st>>>(slots, rect, offsets, cap, cap_pairs, tiles_x, pk, pv, frame);
  k_pairs_eff<<<1, 1, 0, st>>>(frame, cap_pairs);
  return cudaGetLastError();
}

cudaError_t launch_ranges(const uint32_t* tk, uint32_t cap_pairs, const uint32_t* frame, uint2* ranges, int n_tiles,
                          int sm_count, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * size_t(n_tiles), st);
  if (e != cudaSuccess) return e;
  k_ranges<<<sm_count * 8, 256, 0, st>>>(tk, cap_pairs, frame, ranges, uint32_t(n_tiles));
  return cudaGetLastError();
}

}  // namespace v3dg
