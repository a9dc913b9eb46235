// Device helpers shared by the kernels: acquire/release accesses and the bounded chained scan.
#pragma once

#include <cstdint>

#include "v3dg_internal.h"

namespace v3dg {

// A status word carries its flag and its value in one aligned 64-bit word, so a reader that sees
// the flag sees the value with it: relaxed (uncached, single-copy atomic) accesses suffice and no
// fence is needed.
__device__ __forceinline__ uint64_t ld_status(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_status(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t pack_status(uint32_t epoch, uint64_t flag, uint32_t value) {
  return (uint64_t(epoch) << 34) | (flag << 32) | uint64_t(value);
}

// Decoupled look-back.  Tile t owns the status word status[t * stride]; a word whose epoch differs
// from `epoch` counts as not yet written, so the array never needs clearing between launches.
// chain_publish makes the tile's aggregate visible (tile 0 publishes its inclusive prefix);
// chain_lookback then sums the earlier tiles' words back to the first inclusive prefix and
// publishes the tile's own.  Every wait is bounded: after kSpinLimit polls the thread sets *err,
// publishes what it has (so that later tiles do not wait in turn) and returns.
__device__ __forceinline__ void chain_publish(uint64_t* status, uint32_t stride, uint32_t tile, uint32_t agg,
                                              uint32_t epoch) {
  st_status(status + size_t(tile) * stride, pack_status(epoch, tile == 0 ? kFlagPrefix : kFlagAgg, agg));
}

//
// The walk reads kW earlier tiles' words per round with independent loads, so a walk over n
// tiles costs about n / kW memory latencies instead of n: walks are long when tiles reach their
// look-back out of order (a tile passes every earlier one that has only its aggregate).
template <int kW = 1>
__device__ __forceinline__ uint32_t chain_lookback(uint64_t* status, uint32_t stride, uint32_t tile, uint32_t agg,
                                                   uint32_t epoch, uint32_t* err, uint32_t spin_limit = kSpinLimit) {
  if (tile == 0) return 0;
  uint32_t excl = 0;
  int64_t j = int64_t(tile) - 1;
  uint32_t spins = 0;
  while (j >= 0) {
    uint64_t s[kW];
#pragma unroll
    for (int w = 0; w < kW; ++w) s[w] = j - w >= 0 ? ld_status(status + size_t(j - w) * stride) : 0;
    // consume the words in order, up to the first inclusive prefix or the first unwritten word
    int used = 0;
    bool done = false, wait = false;
#pragma unroll
    for (int w = 0; w < kW; ++w) {
      if (done || wait || j - w < 0) continue;
      const uint32_t flag = uint32_t(s[w] >> 32) & 3u;
      if (uint32_t(s[w] >> 34) != epoch || flag == 0) {
        wait = true;
        continue;
      }
      excl += uint32_t(s[w]);
      ++used;
      done = flag == kFlagPrefix;
    }
    if (done) break;
    j -= used;
    if (wait) {
      if (++spins > spin_limit) {
        atomicOr(err, 1u);
        break;
      }
      if (spins > 32) __nanosleep(32);
    }
  }
  st_status(status + size_t(tile) * stride, pack_status(epoch, kFlagPrefix, excl + agg));
  return excl;
}

// The look-back of one chain by a whole warp (all 32 lanes call it, converged): lane i reads the
// word of tile j - i, so each round covers 32 tiles; the nearest inclusive prefix or unwritten
// word ends the round.  Returns the exclusive prefix in every lane; lane 0 publishes.
__device__ __forceinline__ uint32_t chained_exclusive_warp(uint64_t* status, uint32_t tile, uint32_t agg,
                                                           uint32_t epoch, uint32_t* err,
                                                           uint32_t spin_limit = kSpinLimit) {
  const uint32_t lane = threadIdx.x & 31u;
  if (lane == 0) chain_publish(status, 1, tile, agg, epoch);
  if (tile == 0) return 0;
  uint32_t excl = 0, spins = 0;
  int64_t j = int64_t(tile) - 1;
  for (;;) {
    const int64_t q = j - int64_t(lane);
    // before tile 0 (never reached: tile 0 publishes an inclusive prefix) reads as a zero prefix
    const uint64_t s = q >= 0 ? ld_status(status + q) : pack_status(epoch, kFlagPrefix, 0);
    const uint32_t flag = uint32_t(s >> 32) & 3u;
    const bool ready = uint32_t(s >> 34) == epoch && flag != 0;
    const uint32_t not_ready = __ballot_sync(0xffffffffu, !ready);
    const uint32_t prefix = __ballot_sync(0xffffffffu, ready && flag == kFlagPrefix);
    const uint32_t first_wait = not_ready ? uint32_t(__ffs(not_ready) - 1) : 32u;
    const uint32_t first_prefix = prefix ? uint32_t(__ffs(prefix) - 1) : 32u;
    const uint32_t take = first_prefix < first_wait ? first_prefix + 1 : first_wait;
    uint32_t v = lane < take ? uint32_t(s) : 0u;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    excl += v;
    if (first_prefix < first_wait) break;
    j -= take;
    if (take == 0) {
      if (++spins > spin_limit) {
        if (lane == 0) atomicOr(err, 1u);
        break;
      }
      if (spins > 32) __nanosleep(32);
    }
  }
  if (lane == 0) st_status(status + tile, pack_status(epoch, kFlagPrefix, excl + agg));
  return excl;
}

// Exclusive prefix of `agg` over all tiles before `tile`: publish, then look back.
__device__ __forceinline__ uint32_t chained_exclusive(uint64_t* status, uint32_t stride, uint32_t tile,
                                                      uint32_t agg, uint32_t epoch, uint32_t* err) {
  chain_publish(status, stride, tile, agg, epoch);
  return chain_lookback(status, stride, tile, agg, epoch, err);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Block-wide exclusive scan of one uint32 per thread (blockDim.x == 32 * NW); returns the
// exclusive prefix and writes the block total to *total.  `scratch` holds NW + 1 words.
template <int NW>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* scratch, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < NW ? scratch[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += t;
    }
    if (lane < NW) scratch[lane] = wi - w;
    if (lane == NW - 1) scratch[NW] = wi;
  }
  __syncthreads();
  const uint32_t r = scratch[warp] + incl - v;
  *total = scratch[NW];
  __syncthreads();
  return r;
}

}  // namespace v3dg
