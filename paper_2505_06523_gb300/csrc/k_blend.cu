// Per-tile front-to-back alpha blending (Sec. 2.1): C = sum_i c_i a_i prod_{j<i} (1 - a_j).
//
// One 256-thread block per 16x16 tile; warp w owns the 4x8 pixel block at rows 4 (w / 2) .. +3,
// columns 8 (w % 2) .. +7, one pixel per lane.  The tile's depth-ordered records are staged
// through shared memory in batches of 256; a batch starts only while some pixel of the tile is
// still accumulating (block-wide early exit).  Per pixel and Gaussian:
//   log2 a = na dx^2 + nb dx dy + nc dy^2 + log2 o, a = min(0.999, 2^(log2 a)),
//   skip a < 1/255, stop before T (1 - a) < 1e-4.
// Each record's mean is stored relative to the pixel origin of its first tile, so dx, dy are
// differences of small numbers.  Each record also carries the pixel box of its alpha >= 1/255
// ellipse (outside it alpha < 1/255, so skipping there changes nothing).  At staging, the box
// gives the record's row and column masks in this tile and the set of warp blocks it touches;
// ballots turn the latter into one bit list per warp, so a warp visits only the records that
// reach its pixels, still in depth order, and stops as soon as all its pixels are done.  Once some
// warps are done, a batch is filled by scanning ahead: only each record's pixel box is read, and
// only records that reach a live warp are staged, so a tile whose list is long but whose few
// unfinished pixels are rarely touched costs little more than reading its list.
// Tiles differ in cost by orders of magnitude (long lists of tiny distant Gaussians rarely
// saturate a pixel), so the grid is persistent and blocks take tiles heaviest-first: k_tile_order
// buckets the tiles by log2 of their pair count, and blocks pull the next tile of that order.
#include <algorithm>

#include "dev_common.cuh"

namespace v3dg {
namespace {

constexpr int kBlendThreads = 256;
constexpr int kBlendWarps = kBlendThreads / 32;
constexpr float kLog2MinAlpha = -7.9943534f;  // log2(1/255)

// Tile order, heaviest first: one block buckets the tiles by floor(log2(pairs + 1)) (descending).
__global__ void __launch_bounds__(1024) k_tile_order(const uint2* __restrict__ ranges, int n_tiles,
                                                     uint32_t* __restrict__ order) {
  __shared__ uint32_t s_hist[32];
  if (threadIdx.x < 32) s_hist[threadIdx.x] = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) {
    const uint2 r = ranges[t];
    atomicAdd(&s_hist[__clz(r.y - r.x + 1u)], 1u);   // clz: 0 for the heaviest bucket
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const uint32_t v = s_hist[threadIdx.x];
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
      if (threadIdx.x >= d) incl += t;
    }
    s_hist[threadIdx.x] = incl - v;   // cursor: first position of the bucket
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) {
    const uint2 r = ranges[t];
    order[atomicAdd(&s_hist[__clz(r.y - r.x + 1u)], 1u)] = uint32_t(t);
  }
}

// Warp-block mask of a record's pixel box in tile (tx, ty): bit w is set when the box reaches the
// 4x8 block of warp w; *cm / *rm receive the box's column and row masks within the tile.
__device__ __forceinline__ uint32_t box_masks(const float4 r2, int tx, int ty, uint32_t* cm, uint32_t* rm) {
  const uint32_t bx = __float_as_uint(r2.z), by = __float_as_uint(r2.w);
  const int cx0 = max(int(bx & 0xFFFFu) - 16 * tx, 0), cx1 = min(int(bx >> 16) - 16 * tx, 15);
  const int cy0 = max(int(by & 0xFFFFu) - 16 * ty, 0), cy1 = min(int(by >> 16) - 16 * ty, 15);
  const uint32_t c = cx0 <= cx1 ? ((0xFFFFu >> (15 - cx1)) & (0xFFFFu << cx0)) : 0u;
  const uint32_t r = cy0 <= cy1 ? ((0xFFFFu >> (15 - cy1)) & (0xFFFFu << cy0)) : 0u;
  *cm = c;
  *rm = r;
  uint32_t w = 0;
#pragma unroll
  for (int k = 0; k < kBlendWarps; ++k) w |= uint32_t((r & (0xFu << (4 * (k >> 1)))) && (c & (0xFFu << (8 * (k & 1))))) << k;
  return w;
}

template <bool kCount>
__global__ void __launch_bounds__(kBlendThreads, 4)
k_blend(const uint2* __restrict__ ranges, const uint32_t* __restrict__ order, uint32_t* __restrict__ tile_counter,
        int n_tiles, const uint32_t* __restrict__ pv, const float4* __restrict__ rec, uint32_t cap_slots, int width,
        int height, int tiles_x, float* __restrict__ rgb, float* __restrict__ t_out,
        unsigned long long* __restrict__ work, const uint32_t* __restrict__ frame, uint32_t* __restrict__ sticky) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (frame[kOverflow]) atomicOr(sticky, 1u);
    if (frame[kTimeout]) atomicOr(sticky + 1, 1u);
  }
  __shared__ float4 s_g[kBlendThreads];             // (u, v, na, nb) in this tile's pixel frame
  __shared__ float4 s_c[kBlendThreads];             // (nc, log2 o, r, g)
  __shared__ float2 s_b[kBlendThreads];             // (b, row mask << 16 | column mask)
  __shared__ uint32_t s_list[kBlendWarps][kBlendWarps];  // [warp block][staging warp]: record bits
  __shared__ uint32_t s_qslot[kBlendThreads];       // the batch: slots of the records to stage, in order
  __shared__ uint32_t s_scan[kBlendWarps + 1];
  __shared__ uint32_t s_active[kBlendWarps];
  __shared__ uint32_t s_next, s_resume;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = 8 * (warp & 1) + (lane & 7), ly = 4 * (warp >> 1) + (lane >> 3);
  const float fx = float(lx) + 0.5f, fy = float(ly) + 0.5f;
  const uint32_t mybits = (1u << lx) | (1u << (16 + ly));
  uint32_t n_eval = 0, n_contrib = 0;
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t next = s_next;
    __syncthreads();
    if (next >= uint32_t(n_tiles)) break;
    const int tile = int(order[next]);
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int px = tx * 16 + lx, py = ty * 16 + ly;
    const bool inside = px < width && py < height;
    const uint2 range = ranges[tile];
    float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f;
    bool done = !inside;
    uint32_t sp = range.x;   // next list position to look at (uniform across the block)
    for (;;) {
      // warps that still have a pixel to fill
      const bool live = !__all_sync(0xffffffffu, done);
      if (lane == 0) s_active[warp] = live;
      __syncthreads();
      uint32_t act = 0;
#pragma unroll
      for (int w = 0; w < kBlendWarps; ++w) act |= s_active[w] << w;
      if (act == 0 || sp >= range.y) break;
      // fill the batch with the next records whose pixel box reaches a live warp, in list order
      uint32_t q = 0;
      if (act == (1u << kBlendWarps) - 1u) {   // every warp live: every record is relevant
        q = min(uint32_t(kBlendThreads), range.y - sp);
        if (threadIdx.x < q) s_qslot[threadIdx.x] = pv[sp + threadIdx.x];
        sp += q;
      } else {
        while (q < uint32_t(kBlendThreads) && sp < range.y) {
          constexpr int kScan = 4;   // records tested per thread and step
          const uint32_t i0 = sp + threadIdx.x * kScan;
          uint32_t sl[kScan], hits = 0;
#pragma unroll
          for (int k = 0; k < kScan; ++k) {
            sl[k] = 0xFFFFFFFFu;
            if (i0 + k < range.y) {
              sl[k] = pv[i0 + k];
              if (sl[k] < cap_slots) {
                uint32_t cm, rm;
                if (box_masks(rec[3 * size_t(sl[k]) + 2], tx, ty, &cm, &rm) & act) hits |= 1u << k;
              }
            }
          }
          uint32_t total;
          uint32_t pos = q + block_exclusive_scan<kBlendWarps>(__popc(hits), s_scan, &total);
#pragma unroll
          for (int k = 0; k < kScan; ++k) {
            if ((hits >> k) & 1u) {
              if (pos < uint32_t(kBlendThreads)) s_qslot[pos] = sl[k];
              else if (pos == uint32_t(kBlendThreads)) s_resume = i0 + k;   // first record left over
              ++pos;
            }
          }
          __syncthreads();
          if (q + total > uint32_t(kBlendThreads)) {
            sp = s_resume;
            q = kBlendThreads;
          } else {
            sp = min(sp + uint32_t(kBlendThreads * kScan), range.y);
            q += total;
          }
        }
      }
      __syncthreads();
      if (q == 0) break;
      // stage the batch
      uint32_t wmask = 0;
      if (threadIdx.x < q) {
        const uint32_t slot = s_qslot[threadIdx.x];
        if (slot < cap_slots) {
          const float4* r = rec + 3 * size_t(slot);
          const float4 r0 = r[0], r1 = r[1], r2 = r[2];
          const uint32_t org = __float_as_uint(r2.y);
          const float ox = float(16 * (tx - int(org & 0xFFFFu))), oy = float(16 * (ty - int(org >> 16)));
          s_g[threadIdx.x] = make_float4(r0.x - ox, r0.y - oy, r0.z, r0.w);
          s_c[threadIdx.x] = r1;
          uint32_t cm, rm;
          wmask = box_masks(r2, tx, ty, &cm, &rm) & act;
          s_b[threadIdx.x] = make_float2(r2.x, __uint_as_float(cm | (rm << 16)));
        }
      }
#pragma unroll
      for (int w = 0; w < kBlendWarps; ++w) {
        const uint32_t bits = __ballot_sync(0xffffffffu, (wmask >> w) & 1u);
        if (lane == 0) s_list[w][warp] = bits;
      }
      __syncthreads();
      bool warp_done = !((act >> warp) & 1u);
      for (int sw = 0; sw < kBlendWarps && !warp_done; ++sw) {
        uint32_t bits = s_list[warp][sw];
        while (bits) {
          const int j = sw * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          if (!done) {
            const float2 bm = s_b[j];
            if ((__float_as_uint(bm.y) & mybits) == mybits) {
              const float4 g = s_g[j];
              if (kCount) ++n_eval;
              const float dx = fx - g.x, dy = fy - g.y;
              const float4 c = s_c[j];
              const float l2a = fmaf(dx, fmaf(g.z, dx, g.w * dy), fmaf(c.x * dy, dy, c.y));
              if (l2a >= kLog2MinAlpha) {
                const float alpha = fminf(0.999f, exp2f(l2a));
                if (alpha >= 1.f / 255.f) {
                  const float tn = T * (1.f - alpha);
                  if (tn < 1e-4f) {
                    done = true;
                  } else {
                    if (kCount) ++n_contrib;
                    const float w = alpha * T;
                    cr = fmaf(w, c.z, cr);
                    cg = fmaf(w, c.w, cg);
                    cb = fmaf(w, bm.x, cb);
                    T = tn;
                  }
                }
              }
            }
          }
          if (__all_sync(0xffffffffu, done)) {
            warp_done = true;
            break;
          }
        }
      }
      __syncthreads();
    }
    if (inside) {
      const size_t p = size_t(py) * width + px;
      rgb[3 * p + 0] = cr;
      rgb[3 * p + 1] = cg;
      rgb[3 * p + 2] = cb;
      if (t_out) t_out[p] = T;
    }
  }  // next tile
  if (kCount) {
    unsigned long long e = n_eval, cnt = n_contrib;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, d);
      cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    }
    if (lane == 0) {
      atomicAdd(work, e);
      atomicAdd(work + 1, cnt);
    }
  }
}

}  // namespace

cudaError_t launch_blend(const uint2* ranges, uint32_t* order, uint32_t* tile_counter, const uint32_t* pv,
                         const float4* rec, uint32_t cap_slots, const CamConst& cam, float* rgb, float* t_out,
                         unsigned long long* work, const uint32_t* frame, uint32_t* sticky, int sm_count,
                         cudaStream_t st) {
  const int n_tiles = cam.tiles_x * cam.tiles_y;
  if (n_tiles == 0) return cudaSuccess;
  k_tile_order<<<1, 1024, 0, st>>>(ranges, n_tiles, order);
  const int grid = std::min(n_tiles, sm_count * 4);   // 4 resident blocks per SM (56 registers)
  if (work)
    k_blend<true><<<grid, kBlendThreads, 0, st>>>(ranges, order, tile_counter, n_tiles, pv, rec, cap_slots, cam.width,
                                                  cam.height, cam.tiles_x, rgb, t_out, work, frame, sticky);
  else
    k_blend<false><<<grid, kBlendThreads, 0, st>>>(ranges, order, tile_counter, n_tiles, pv, rec, cap_slots, cam.width,
                                                   cam.height, cam.tiles_x, rgb, t_out, nullptr, frame, sticky);
  return cudaGetLastError();
}

}  // namespace v3dg
