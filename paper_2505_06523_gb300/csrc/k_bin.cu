// Tile binning: expansion of each visible Gaussian into its (tile, Gaussian) pairs, tile ranges.
//
// The Gaussians arrive sorted by depth (stage one of the two-stage (tile, depth) sort), so the
// pairs are emitted in depth order; a stable sort on the tile id then yields (tile, depth, id)
// order, and each tile's range of the sorted pairs is found by boundary detection.  A pair key
// carries, above the 20-bit tile id, the Gaussian's pixel box clipped to that tile (so that the
// blend can skip pairs by their keys alone).
#include <algorithm>

#include "dev_common.cuh"

namespace v3dg {
namespace {

// Tiles covered by a Gaussian's pixel box (x0 | x1 << 16, y0 | y1 << 16, inclusive pixels).
__device__ __forceinline__ uint32_t rect_area(const uint2 b) {
  const uint32_t w = ((b.x >> 16) >> 4) - ((b.x & 0xFFFFu) >> 4) + 1u;
  const uint32_t h = ((b.y >> 16) >> 4) - ((b.y & 0xFFFFu) >> 4) + 1u;
  return w * h;
}

constexpr int kExpThreads = 256, kExpItems = 4, kExpTile = kExpThreads * kExpItems;
constexpr uint32_t kExpWarps = kExpThreads / 32;

// One pass over the depth-sorted visible Gaussians: each block takes 1024 of them, scans their
// tile counts, finds its first pair position with a bounded look-back and then writes its pairs
// cooperatively: output position p belongs to the Gaussian j with off[j] <= p < off[j + 1], each
// warp takes one contiguous range of positions and follows the owners forward (one binary search
// per warp and tile), so large Gaussians are spread over the whole block and the writes are
// contiguous.
__global__ void __launch_bounds__(kExpThreads)
k_expand(const uint32_t* __restrict__ slots, const uint2* __restrict__ rect, uint32_t cap, uint32_t cap_pairs,
         int tiles_x, const uint2* __restrict__ list, const InstFrame* __restrict__ inst_views, uint32_t tiles_per_view,
         uint32_t* __restrict__ pk, uint32_t* __restrict__ pv, uint32_t* __restrict__ frame, uint32_t tc_slot,
         uint64_t* __restrict__ status, uint32_t epoch) {
  __shared__ uint32_t s_off[kExpTile + 1];
  __shared__ uint2 s_rect[kExpTile];
  __shared__ uint32_t s_slot[kExpTile];
  __shared__ uint32_t s_tbase[kExpTile];   // first (view, tile) id of the Gaussian's view
  __shared__ uint32_t s_scan[kExpThreads / 32 + 1];
  __shared__ uint32_t s_tile, s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t n = min(frame[kVisible], cap);
  const uint32_t ntiles = (n + kExpTile - 1) / kExpTile;
  for (;;) {   // persistent blocks: tiles in the order of an atomic counter
  if (threadIdx.x == 0) s_tile = atomicAdd(frame + kTileCounters + tc_slot, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  if (tile >= ntiles) return;
  const uint32_t first = tile * kExpTile;
  const uint32_t items = min(uint32_t(kExpTile), n - first);
  uint32_t c[kExpItems], sum = 0;
#pragma unroll
  for (int i = 0; i < kExpItems; ++i) {
    const uint32_t j = threadIdx.x * kExpItems + i;
    c[i] = 0;
    if (j < items) {
      const uint32_t slot = slots[first + j];
      const uint2 r = rect[slot];
      s_slot[j] = slot;
      s_rect[j] = r;
      s_tbase[j] = inst_views ? inst_views[list[slot / kSlots].x].view * tiles_per_view : 0u;
      c[i] = rect_area(r);
    }
    sum += c[i];
  }
  uint32_t total;
  uint32_t ex = block_exclusive_scan<kExpThreads / 32>(sum, s_scan, &total);
#pragma unroll
  for (int i = 0; i < kExpItems; ++i) {
    s_off[threadIdx.x * kExpItems + i] = ex;
    ex += c[i];
  }
  if (threadIdx.x < 32) {   // warp 0: the look-back, 32 tiles per round
    const uint32_t b = chained_exclusive_warp(status, tile, total, epoch, frame + kTimeout);
    if (threadIdx.x == 0) {
      s_off[kExpTile] = total;
      s_base = b;
      if (tile == ntiles - 1) frame[kPairs] = b + total;
    }
  }
  __syncthreads();
  const uint32_t base = s_base;
  if (threadIdx.x == 0 && total) atomicAdd(reinterpret_cast<unsigned long long*>(frame + kPairs64), total);
  const bool fits = uint64_t(base) + total <= cap_pairs;   // else the frame overflows: count, write nothing
  if (!fits && threadIdx.x == 0) atomicOr(frame + kOverflow, 1u);
  // Each warp writes one contiguous range of the tile's pairs, 32 positions per step.  The owner
  // of position p is the last item j with s_off[j] <= p.  Items start at distinct positions (each
  // Gaussian has at least one pair), so at most 32 items start within a step: with `ob` the owner
  // of the position before the step, lane i checks item ob + 1 + i, the warp ORs the start
  // offsets that fall in the step into one mask, and a lane's owner is ob plus the starts at or
  // before its position.
  const uint32_t per_warp = ((total + kExpWarps * 32u - 1u) / (kExpWarps * 32u)) * 32u;
  const uint32_t pw0 = min(uint32_t(warp) * per_warp, total), pw1 = min(pw0 + per_warp, total);
  int ob = -1;   // owner of pw0 - 1 (none before position 0)
  if (fits && pw0 > 0) {   // binary search, the same in every lane: s_off[lo] <= pw0 - 1 < s_off[hi]
    uint32_t lo = 0, hi = items;   // (s_off[0] = 0, s_off[items] = total)
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_off[mid] <= pw0 - 1u) lo = mid; else hi = mid;
    }
    ob = int(lo);
  }
  for (uint32_t p0 = pw0; fits && p0 < pw1; p0 += 32u) {
    const uint32_t p = p0 + uint32_t(lane);
    const int kk = ob + 1 + lane;
    uint32_t bit = 0;
    if (kk < int(items)) {
      const uint32_t v = s_off[kk] - p0;   // >= 0: item ob + 1 starts after position p0 - 1
      if (v < 32u) bit = 1u << v;
    }
    const uint32_t starts = __reduce_or_sync(0xffffffffu, bit);
    const uint32_t upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);   // positions p0 .. p
    const int owner = ob + __popc(starts & upto);
    ob = __shfl_sync(0xffffffffu, owner, 31);
    if (p >= pw1) continue;
    const uint32_t lo = uint32_t(owner);
    const uint2 r = s_rect[lo];
    const uint32_t x0 = r.x & 0xFFFFu, x1 = r.x >> 16, y0 = r.y & 0xFFFFu, y1 = r.y >> 16;
    const uint32_t tx0 = x0 >> 4, ty0 = y0 >> 4;
    const uint32_t w = (x1 >> 4) - tx0 + 1u;
    const uint32_t k = p - s_off[lo];
    const uint32_t dy = k / w;
    const uint32_t tx = tx0 + (k - dy * w), ty = ty0 + dy;
    // above the tile id: the box clipped to this tile, tile-local (rows exact, columns in quads)
    const uint32_t bx0 = x0 > 16 * tx ? x0 - 16 * tx : 0u, bx1 = min(x1 - 16 * tx, 15u);
    const uint32_t by0 = y0 > 16 * ty ? y0 - 16 * ty : 0u, by1 = min(y1 - 16 * ty, 15u);
    pk[base + p] = (s_tbase[lo] + ty * uint32_t(tiles_x) + tx) | (by0 << 20) | (by1 << 24) | ((bx0 >> 2) << 28) | ((bx1 >> 2) << 30);
    pv[base + p] = s_slot[lo];
  }
  __syncthreads();   // the tile's shared data is consumed before the next tile reuses it
  }  // next tile
}

// After duplication: the pair count that later stages use (none when the frame overflowed, so
// that no stage reads pair slots that were not written).
__global__ void k_pairs_eff(uint32_t* frame, uint32_t cap_pairs) {
  // a total beyond the capacity (counted in 64 bits, so also one beyond 2^32) overflows the frame
  const unsigned long long total = *reinterpret_cast<const unsigned long long*>(frame + kPairs64);
  if (total > cap_pairs) {
    frame[kOverflow] = 1u;
    frame[kPairs] = total > 0xFFFFFFFFull ? 0xFFFFFFFFu : uint32_t(total);
  }
  frame[kPairsEff] = frame[kOverflow] ? 0u : min(frame[kPairs], cap_pairs);
}

// Tile ranges by boundary detection: each thread takes four consecutive sorted keys at a time
// (one 16-byte load when the array is 16-byte aligned) and compares each with its neighbours.
__global__ void __launch_bounds__(256)
k_ranges(const uint32_t* __restrict__ tk, uint32_t cap_pairs, const uint32_t* __restrict__ frame,
         uint2* __restrict__ ranges, uint32_t n_tiles) {
  const uint32_t n = min(frame[kPairsEff], cap_pairs);
  const uint32_t groups = (n + 3) / 4;
  const bool aligned = (reinterpret_cast<uintptr_t>(tk) & 15u) == 0;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += gridDim.x * blockDim.x) {
    const uint32_t k0 = 4 * g;
    uint32_t t[6];   // tiles of keys k0 - 1 .. k0 + 4 (0xFFFFFFFF outside [0, n))
    t[0] = k0 > 0 ? tk[k0 - 1] & kPairTileMask : 0xFFFFFFFFu;
    if (aligned && k0 + 4 <= n) {
      const uint4 v = *reinterpret_cast<const uint4*>(tk + k0);
      t[1] = v.x & kPairTileMask;
      t[2] = v.y & kPairTileMask;
      t[3] = v.z & kPairTileMask;
      t[4] = v.w & kPairTileMask;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) t[1 + i] = k0 + i < n ? tk[k0 + i] & kPairTileMask : 0xFFFFFFFFu;
    }
    t[5] = k0 + 4 < n ? tk[k0 + 4] & kPairTileMask : 0xFFFFFFFFu;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t k = k0 + i, tt = t[1 + i];
      if (k >= n || tt >= n_tiles) continue;
      if (t[i] != tt) ranges[tt].x = k;
      if (t[i + 2] != tt) ranges[tt].y = k + 1;
    }
  }
}

}  // namespace

cudaError_t launch_expand(const uint32_t* slots, const uint2* rect, uint32_t cap, uint32_t cap_pairs, int tiles_x,
                          const uint2* list, const InstFrame* inst_views, uint32_t tiles_per_view, uint32_t* pk,
                          uint32_t* pv, uint32_t* frame, uint32_t tc_slot, uint64_t* status, uint32_t epoch,
                          int sm_count, cudaStream_t st) {
  // persistent grid: at most the resident blocks (8 of 256 threads per SM), whatever the capacity
  const uint32_t blocks = std::min<uint32_t>((cap + kExpTile - 1) / kExpTile, uint32_t(sm_count) * 8u);
  if (blocks)
    k_expand<<<blocks, kExpThreads, 0, st>>>(slots, rect, cap, cap_pairs, tiles_x, list, inst_views, tiles_per_view,
                                             pk, pv, frame, tc_slot, status, epoch);
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
