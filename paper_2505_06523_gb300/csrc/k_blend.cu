// Per-tile front-to-back alpha blending (Sec. 2.1): C = sum_i c_i a_i prod_{j<i} (1 - a_j).
//
// One 256-thread block per 16x16 tile, or per 8x8 quadrant of a tile with a long list
// (persistent blocks take work items heaviest-first: tiles differ in cost by orders of magnitude).
// The tile's depth-ordered records are taken in batches (128, 256 or 512 records); each batch runs
// in two phases:
//  - record-parallel test: each thread stages its own records and evaluates each at the pixels of
//    its alpha >= 1/255 box that are still accumulating; a pixel where the skip rule passes gets
//    the record's bit in its mask (one bit per record of the batch);
//  - pixel-parallel blend: each thread walks its pixel's mask in record (= depth) order and
//    blends exactly those records: a = min(0.999, 2^(na dx^2 + nb dx dy + nc dy^2 + log2 o)),
//    stopping before T (1 - a) < 1e-4.
// So sequential work is spent only where a Gaussian contributes, and small Gaussians (a few
// pixels each) no longer occupy whole warps.  Records are staged through shared memory; a batch
// is filled only with records whose box holds a pixel that is still accumulating, found by
// scanning ahead in the sorted pair keys, which carry each Gaussian's box within the tile (so
// skipped records cost one coalesced 4-byte read).  Each record's mean is stored relative to the
// pixel origin of its first tile, so dx, dy are differences of small numbers.
#include <algorithm>

#include "dev_common.cuh"

namespace v3dg {
namespace {

constexpr int kBlendThreads = 256;
constexpr int kBlendWarps = kBlendThreads / 32;
constexpr float kLog2MinAlpha = -7.9943534f;  // log2(1/255)

// log2(alpha) of a staged record at tile-local pixel centre (fx, fy); one definition for both phases
__device__ __forceinline__ float log2_alpha(const float4 g, const float4 c, float fx, float fy) {
  const float dx = fx - g.x, dy = fy - g.y;
  return fmaf(dx, fmaf(g.z, dx, g.w * dy), fmaf(c.x * dy, dy, c.y));
}

// One front-to-back step at a pixel (Sec. 2.1): alpha = min(0.999, 2^l2a), skipped below 1/255,
// the pixel stops before T (1 - alpha) < 1e-4, else C += alpha T c and T *= 1 - alpha.  Both blend
// kernels composite through this function, so their images are bit-identical.  Returns whether
// the record contributed.
__device__ __forceinline__ bool composite_step(float l2a, float r, float g, float b, float& T, float& cr, float& cg,
                                               float& cb, bool& done) {
  const float a = l2a < kLog2MinAlpha ? 0.f : fminf(0.999f, exp2f(l2a));
  if (a < 1.f / 255.f) return false;
  const float tn = T * (1.f - a);
  if (tn < 1e-4f) {
    done = true;
    return false;
  }
  const float wgt = a * T;
  cr = fmaf(wgt, r, cr);
  cg = fmaf(wgt, g, cg);
  cb = fmaf(wgt, b, cb);
  T = tn;
  return true;
}

// True when the box that a pair key carries (see kPairTileMask: rows y0..y1, column quads
// q0..q1) holds a pixel whose bit is set in `live` (one word per row pair: row 2w in bits
// 0..15, row 2w + 1 in 16..31).
__device__ __forceinline__ bool box_live(uint32_t key, const uint32_t* live) {
  const uint32_t y0 = (key >> 20) & 15u, y1 = (key >> 24) & 15u, q0 = (key >> 28) & 3u, q1 = key >> 30;
  const uint32_t cols = (0xFFFFu >> (12u - 4u * q1)) & (0xFFFFu << (4u * q0));
  for (uint32_t y = y0; y <= y1; ++y)
    if ((live[y >> 1] >> ((y & 1u) * 16u)) & cols) return true;
  return false;
}

// A record's pixel box (from its third float4) clipped to tile (tx, ty), tile-local.
__device__ __forceinline__ void box_in_tile(const float4 r2, int tx, int ty, int* x0, int* x1, int* y0, int* y1) {
  const uint32_t bx = __float_as_uint(r2.z), by = __float_as_uint(r2.w);
  *x0 = max(int(bx & 0xFFFFu) - 16 * tx, 0);
  *x1 = min(int(bx >> 16) - 16 * tx, 15);
  *y0 = max(int(by & 0xFFFFu) - 16 * ty, 0);
  *y1 = min(int(by >> 16) - 16 * ty, 15);
}

// The next batch of a work item: the records from list position *sp on whose box (carried by the
// pair key) holds an unfinished pixel, in list order, at most kBatch of them; kScan * 256
// consecutive keys per step.  Writes their slots to s_qslot and, when s_rows is given, the row
// pairs their box spans (bit w: rows 2w, 2w + 1) to s_rows; advances *sp past the last record
// taken and returns the batch size (uniform across the block; called by all threads).
template <int kBatch>
__device__ __forceinline__ uint32_t fill_batch(const uint32_t* __restrict__ tk, const uint32_t* __restrict__ pv,
                                               uint32_t end, uint32_t cap_slots, const uint32_t* s_live,
                                               uint32_t* s_qslot, uint8_t* s_rows, uint32_t* s_cnt,
                                               uint32_t* s_resume, uint32_t* s_total, uint32_t* sp_io) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t sp = *sp_io, q = 0;
  while (q < uint32_t(kBatch) && sp < end) {
    constexpr int kScan = 4;
    uint32_t key[kScan], ball[kScan], hits = 0;
#pragma unroll
    for (int k = 0; k < kScan; ++k) {
      const uint32_t pos = sp + k * kBlendThreads + threadIdx.x;
      key[k] = 0;
      if (pos < end) {
        key[k] = tk[pos];
        if (box_live(key[k], s_live)) hits |= 1u << k;
      }
      ball[k] = __ballot_sync(0xffffffffu, (hits >> k) & 1u);
      if (lane == 0) s_cnt[k * kBlendWarps + warp] = __popc(ball[k]);
    }
    __syncthreads();
    if (warp == 0) {   // exclusive scan over (step, warp) = list order
      const uint32_t v = s_cnt[lane];
      uint32_t incl = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
      }
      s_cnt[lane] = incl - v;
      if (lane == 31) *s_total = incl;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScan; ++k) {
      if ((hits >> k) & 1u) {
        const uint32_t pos = sp + k * kBlendThreads + threadIdx.x;
        const uint32_t idx = q + s_cnt[k * kBlendWarps + warp] + __popc(ball[k] & lanemask_lt());
        if (idx < uint32_t(kBatch)) {
          const uint32_t slot = pv[pos];
          s_qslot[idx] = slot;
          if (s_rows) {   // (a slot beyond the buffers never occurs in a valid frame: no warp reads it)
            const uint32_t w0 = ((key[k] >> 20) & 15u) >> 1, w1 = ((key[k] >> 24) & 15u) >> 1;
            s_rows[idx] = slot < cap_slots ? uint8_t((0xFFu >> (7u - w1)) & (0xFFu << w0)) : uint8_t(0);
          }
        } else if (idx == uint32_t(kBatch)) {
          *s_resume = pos;   // the first record left over
        }
      }
    }
    __syncthreads();
    const uint32_t total = *s_total;
    if (q + total > uint32_t(kBatch)) {
      sp = *s_resume;
      q = kBatch;
    } else {
      sp = min(sp + uint32_t(kBlendThreads * kScan), end);
      q += total;
    }
    static_assert(kScan * kBlendWarps == 32, "one scan lane per (step, warp)");
  }
  *sp_io = sp;
  return q;
}

// Resident blocks per SM: batches of 128 records keep shared memory (10 KB) and registers (40)
// small enough for 6 blocks, the larger ones run 4.
constexpr int blend_blocks_per_sm(int batch) { return batch == 128 ? 6 : 4; }

// kBatch: records staged per batch (128, 256 or 512; the image does not depend on it).
template <bool kCount, int kBatch>
__global__ void __launch_bounds__(kBlendThreads, blend_blocks_per_sm(kBatch))
k_blend(const uint2* __restrict__ ranges, const uint32_t* __restrict__ items, const uint32_t* __restrict__ n_items,
        uint32_t* __restrict__ tile_counter, const uint32_t* __restrict__ tk, const uint32_t* __restrict__ pv,
        const float4* __restrict__ rec, uint32_t cap_slots, int width,
        int height, int tiles_x, int tiles_per_view, float* __restrict__ rgb, float* __restrict__ t_out,
        unsigned long long* __restrict__ work, uint32_t* __restrict__ frame, uint32_t* __restrict__ sticky) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (frame[kOverflow]) atomicOr(sticky, 1u);
    if (frame[kTimeout]) atomicOr(sticky + 1, 1u);
  }
  constexpr int kPer = kBatch >= kBlendThreads ? kBatch / kBlendThreads : 1;   // records staged per thread
  constexpr int kMaskWords = kBatch / 32;                                       // per-pixel mask words
  static_assert(kBatch % 32 == 0 && (kBatch <= kBlendThreads || kBatch % kBlendThreads == 0), "batch size");
  __shared__ float4 s_g[kBatch];                    // (u, v, na, nb) in this tile's pixel frame
  __shared__ float4 s_c[kBatch];                    // (nc, log2 o, r, g)
  __shared__ float s_b[kBatch];                     // b
  __shared__ uint32_t s_mask[kBlendThreads][kMaskWords];  // [pixel][record word]: contributing records
  __shared__ uint32_t s_live[kBlendWarps];          // unfinished pixels of the item, one word per row pair
  __shared__ uint32_t s_qslot[kBatch];              // the batch: slots of its records, in list order
  __shared__ uint32_t s_cnt[32];
  __shared__ uint32_t s_next, s_resume, s_total;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = threadIdx.x & 15, ly = threadIdx.x >> 4;   // this thread's pixel in the tile
  const float fx = float(lx) + 0.5f, fy = float(ly) + 0.5f;
  uint32_t n_eval = 0, n_contrib = 0;
#pragma unroll
  for (int k = 0; k < kMaskWords; ++k) s_mask[threadIdx.x][k] = 0u;
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t next = s_next;
    __syncthreads();
    if (next >= *n_items) break;
    const uint32_t item = items[next];
    const int tile = int(item & 0xFFFFFFu), region = int(item >> 24);   // (view, tile) id
    const int view = tile / tiles_per_view, vt = tile - view * tiles_per_view;
    const int tx = vt % tiles_x, ty = vt / tiles_x;
    // the item's pixel rectangle within the tile: the whole tile or one 8x8 quadrant
    const int qx0 = region ? 8 * ((region - 1) & 1) : 0, qy0 = region ? 8 * ((region - 1) >> 1) : 0;
    const int qx1 = region ? qx0 + 7 : 15, qy1 = region ? qy0 + 7 : 15;
    const int px = tx * 16 + lx, py = ty * 16 + ly;
    const bool mine = lx >= qx0 && lx <= qx1 && ly >= qy0 && ly <= qy1;
    const bool inside = px < width && py < height && mine;
    const uint2 range = ranges[tile];
    float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f;
    bool done = !inside;
    uint32_t sp = range.x;   // next list position to look at (uniform across the block)
    for (;;) {
      // the item's unfinished pixels, one word per row pair (row 2w: bits 0..15, row 2w + 1: 16..31)
      const uint32_t dword = __ballot_sync(0xffffffffu, done);
      if (lane == 0) s_live[warp] = ~dword;
      __syncthreads();
      uint32_t any_live = 0;
#pragma unroll
      for (int w = 0; w < kBlendWarps; ++w) any_live |= s_live[w];
      if (any_live == 0 || sp >= range.y) break;
      // the batch: the next records of the list whose box (carried by the pair key) holds an
      // unfinished pixel, in list order; kScan * 256 consecutive keys per step
      const uint32_t q = fill_batch<kBatch>(tk, pv, range.y, cap_slots, s_live, s_qslot, nullptr, s_cnt, &s_resume, &s_total, &sp);
      if (q == 0) break;
      // stage the batch (kPer consecutive records per thread) for the compositing phase, and test
      // each of this thread's records at the pixels of its box that are still accumulating: a
      // pixel where alpha >= 1/255 gets the record's bit in its mask
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const uint32_t i = threadIdx.x * kPer + k;
        if (i >= q) continue;
        const uint32_t slot = s_qslot[i];
        if (slot >= cap_slots) continue;
        const float4* r = rec + 3 * size_t(slot);
        const float4 r0 = r[0], r1 = r[1], r2 = r[2];
        const uint32_t org = __float_as_uint(r2.y);
        const float ox = float(16 * (tx - int(org & 0xFFFFu))), oy = float(16 * (ty - int(org >> 16)));
        const float4 g = make_float4(r0.x - ox, r0.y - oy, r0.z, r0.w);
        s_g[i] = g;
        s_c[i] = r1;
        s_b[i] = r2.x;
        int x0, x1, y0, y1;
        box_in_tile(r2, tx, ty, &x0, &x1, &y0, &y1);
        x0 = max(x0, qx0); x1 = min(x1, qx1); y0 = max(y0, qy0); y1 = min(y1, qy1);
        if (x0 > x1) continue;
        const uint32_t cols = (0xFFFFu >> (15 - x1)) & (0xFFFFu << x0);
        const uint32_t bit = 1u << (i & 31);
        for (int yy = y0; yy <= y1; ++yy) {
          uint32_t m = (s_live[yy >> 1] >> ((yy & 1) * 16)) & cols;
          while (m) {
            const int xx = __ffs(m) - 1;
            m &= m - 1;
            const float l2a = log2_alpha(g, r1, float(xx) + 0.5f, float(yy) + 0.5f);
            if (kCount) ++n_eval;
            // alpha = min(0.999, 2^l2a) >= 1/255; well above the threshold it holds without exp2
            if (l2a >= kLog2MinAlpha + 1e-5f ||
                (l2a >= kLog2MinAlpha && fminf(0.999f, exp2f(l2a)) >= 1.f / 255.f))
              atomicOr(&s_mask[yy * 16 + xx][i >> 5], bit);
          }
        }
      }
      __syncthreads();
      // pixel-parallel blend of the contributing records, in depth order
#pragma unroll
      for (int wd = 0; wd < kMaskWords; ++wd) {
        uint32_t bits = s_mask[threadIdx.x][wd];
        if (!bits) continue;
        s_mask[threadIdx.x][wd] = 0u;
        while (bits && !done) {
          // two records at a time: their alphas are independent, only T is a chain
          constexpr int kAhead = 2;
          int jj[kAhead], n = 0;
#pragma unroll
          for (int q = 0; q < kAhead; ++q) {
            jj[q] = wd * 32 + __ffs(bits) - 1;   // bits == 0: a valid index, not used
            if (bits) {
              bits &= bits - 1;
              n = q + 1;
            }
          }
          float l2a[kAhead], r[kAhead], g[kAhead], b[kAhead];
#pragma unroll
          for (int q = 0; q < kAhead; ++q) {
            const int j = max(jj[q], wd * 32);
            const float4 c = s_c[j];
            l2a[q] = log2_alpha(s_g[j], c, fx, fy);
            r[q] = c.z;
            g[q] = c.w;
            b[q] = s_b[j];
          }
#pragma unroll
          for (int q = 0; q < kAhead; ++q) {
            if (q >= n || done) break;
            if (composite_step(l2a[q], r[q], g[q], b[q], T, cr, cg, cb, done) && kCount) ++n_contrib;
          }
        }
      }
      __syncthreads();
    }
    if (inside) {   // this item's pixels only
      const size_t p = (size_t(view) * height + py) * width + px;
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

// ---------------------------------------------------------------- bulk-copy staging
// One non-tensor cp.async.bulk per 48-byte record (16-byte aligned in global and shared memory)
// from this GPU's own memory into the CTA's shared memory, completing on an mbarrier.

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// One poll of the phase with the given parity; the thread may be suspended for up to about 1 us
// (the suspend-time hint) while the phase is incomplete.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the mbarrier phase of the given parity; false when it has not completed within about
// one second (and at most kSpinLimit polls).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 63u && global_ns() - t0 > 1000000000ull) break;
  }
  return false;
}

__device__ __forceinline__ void bulk_copy_to_shared(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Resident blocks per SM of the pixel-loop kernel (shared memory: 54 B per record of a batch; at
// six blocks the 40-register limit spills).
constexpr int blend_px_blocks_per_sm(int batch) { return batch == 512 ? 4 : 5; }

// Second blend variant (V3DG_OPT_BLEND_MODE 1): the same batches, staged by bulk copies, then
// composited pixel-parallel with no per-pixel masks.  Warp w owns rows 2w and 2w + 1 of the tile
// (lane = pixel) and walks, in list (= depth) order, only the batch records whose box spans one of
// its rows (known from the pair key at fill time), so a warp never visits a record that cannot
// reach it; each lane evaluates the record where its pixel lies in the record's box and is still
// accumulating, and composites at once (composite_step, the same arithmetic as the two-phase
// kernel, so the image is the same bit for bit).  A warp whose 32 pixels are all done skips the
// rest of the batch.  Quadrant work items are handled (the other rows' warps idle), though the
// launch keeps whole tiles for this variant.
template <bool kCount, int kBatch>
__global__ void __launch_bounds__(kBlendThreads, blend_px_blocks_per_sm(kBatch))
k_blend_px(const uint2* __restrict__ ranges, const uint32_t* __restrict__ items, const uint32_t* __restrict__ n_items,
           uint32_t* __restrict__ tile_counter, const uint32_t* __restrict__ tk, const uint32_t* __restrict__ pv,
           const float4* __restrict__ rec, uint32_t cap_slots, int width, int height, int tiles_x, int tiles_per_view,
           float* __restrict__ rgb, float* __restrict__ t_out, unsigned long long* __restrict__ work,
           uint32_t* __restrict__ frame, uint32_t* __restrict__ sticky) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (frame[kOverflow]) atomicOr(sticky, 1u);
    if (frame[kTimeout]) atomicOr(sticky + 1, 1u);
  }
  constexpr int kPer = kBatch >= kBlendThreads ? kBatch / kBlendThreads : 1;
  constexpr int kWords = kBatch / 32;
  static_assert(kBatch % 32 == 0 && kWords <= 32 && (kBatch <= kBlendThreads || kBatch % kBlendThreads == 0),
                "batch size");
  __shared__ __align__(16) float4 s_rec[3 * kBatch];   // the batch's records, as stored by the projection
  __shared__ uint32_t s_qslot[kBatch];
  __shared__ uint8_t s_rows[kBatch];                   // bit w: the record's box spans rows 2w or 2w + 1
  __shared__ uint32_t s_live[kBlendWarps];
  __shared__ uint32_t s_cnt[32];
  __shared__ uint32_t s_next, s_resume, s_total;
  __shared__ __align__(8) uint64_t s_bar;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = threadIdx.x & 15, ly = threadIdx.x >> 4;   // lane = 16 (ly & 1) + lx
  const float fx = float(lx) + 0.5f, fy = float(ly) + 0.5f;
  uint32_t n_eval = 0, n_contrib = 0, phase = 0;
  bool failed = false;
  if (threadIdx.x == 0) mbar_init(&s_bar, 1);
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t next = s_next;
    __syncthreads();
    if (next >= *n_items) break;
    const uint32_t item = items[next];
    const int tile = int(item & 0xFFFFFFu), region = int(item >> 24);
    const int view = tile / tiles_per_view, vt = tile - view * tiles_per_view;
    const int tx = vt % tiles_x, ty = vt / tiles_x;
    const int qx0 = region ? 8 * ((region - 1) & 1) : 0, qy0 = region ? 8 * ((region - 1) >> 1) : 0;
    const int qx1 = region ? qx0 + 7 : 15, qy1 = region ? qy0 + 7 : 15;
    const int px = tx * 16 + lx, py = ty * 16 + ly;
    const bool inside = px < width && py < height && lx >= qx0 && lx <= qx1 && ly >= qy0 && ly <= qy1;
    const uint2 range = ranges[tile];
    float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f;
    bool done = !inside;
    uint32_t sp = range.x;
    for (;;) {
      const uint32_t dword = __ballot_sync(0xffffffffu, done);
      if (lane == 0) s_live[warp] = ~dword;
      __syncthreads();
      uint32_t any_live = 0;
#pragma unroll
      for (int w = 0; w < kBlendWarps; ++w) any_live |= s_live[w];
      if (any_live == 0 || sp >= range.y) break;
      const uint32_t q = fill_batch<kBatch>(tk, pv, range.y, cap_slots, s_live, s_qslot, s_rows, s_cnt, &s_resume, &s_total, &sp);
      if (q == 0) break;
      // stage the batch: the previous batch's shared reads ended at the fill's barriers
      if (threadIdx.x == 0) mbar_arrive_expect_tx(&s_bar, q * 48u);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const uint32_t i = threadIdx.x + k * kBlendThreads;
        if (i >= q) continue;
        uint32_t slot = s_qslot[i];
        if (slot >= cap_slots) slot = 0;   // never for a valid frame; no warp reads the record (rows 0)
        bulk_copy_to_shared(&s_rec[3 * i], rec + 3 * size_t(slot), 48u, &s_bar);
      }
      // this warp's records: bit j of word k <=> record 32 k + j spans one of its rows
      uint32_t mine = 0;
#pragma unroll
      for (int k = 0; k < kWords; ++k) {
        __syncwarp();
        const uint32_t j = 32u * k + lane;
        const uint32_t b = __ballot_sync(0xffffffffu, j < q && ((s_rows[j] >> warp) & 1u));
        if (lane == k) mine = b;
      }
      if (!mbar_wait_bounded(&s_bar, phase)) failed = true;
      phase ^= 1u;
      if (__syncthreads_or(failed)) goto out;
      bool wdone = __all_sync(0xffffffffu, done);
      for (int k = 0; k < kWords && !wdone; ++k) {
        uint32_t bits = __shfl_sync(0xffffffffu, mine, k);
        while (bits) {
          const int j = 32 * k + __ffs(bits) - 1;
          bits &= bits - 1;
          const float4 r0 = s_rec[3 * j], r1 = s_rec[3 * j + 1], r2 = s_rec[3 * j + 2];
          const uint32_t bx = __float_as_uint(r2.z), by = __float_as_uint(r2.w);
          if (!done && px >= int(bx & 0xFFFFu) && px <= int(bx >> 16) && py >= int(by & 0xFFFFu) &&
              py <= int(by >> 16)) {
            const uint32_t org = __float_as_uint(r2.y);
            const float ox = float(16 * (tx - int(org & 0xFFFFu))), oy = float(16 * (ty - int(org >> 16)));
            const float l2a = log2_alpha(make_float4(r0.x - ox, r0.y - oy, r0.z, r0.w), r1, fx, fy);
            if (kCount) ++n_eval;
            if (composite_step(l2a, r1.z, r1.w, r2.x, T, cr, cg, cb, done) && kCount) ++n_contrib;
          }
          if (__all_sync(0xffffffffu, done)) {
            wdone = true;
            break;
          }
        }
      }
      __syncthreads();   // the batch's records are consumed before the next batch is staged
    }
    if (inside) {
      const size_t p = (size_t(view) * height + py) * width + px;
      rgb[3 * p + 0] = cr;
      rgb[3 * p + 1] = cg;
      rgb[3 * p + 2] = cb;
      if (t_out) t_out[p] = T;
    }
  }  // next tile
out:
  if (failed) {   // a bounded wait gave up: flag the frame, and let the copies in flight land first
    if (threadIdx.x == 0) {
      atomicOr(frame + kTimeout, 1u);
      atomicOr(sticky + 1, 1u);
    }
    mbar_wait_bounded(&s_bar, phase ^ 1u);
    return;
  }
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

// Work items, heaviest first.  A tile with at least split_pairs pairs becomes four items, one
// per 8x8 quadrant (each scans the tile's list by boxes but stages and evaluates only the
// records that reach its quadrant, so a long list is spread over four blocks); other tiles are
// one item.  Item = tile | region << 24 (region 0: whole tile, 1 + q: quadrant q).  One block
// buckets the items by floor(log2(pairs + 1)), descending.
__global__ void __launch_bounds__(1024) k_blend_items(const uint2* __restrict__ ranges, int n_tiles,
                                                      uint32_t split_pairs, uint32_t* __restrict__ items,
                                                      uint32_t* __restrict__ n_items) {
  __shared__ uint32_t s_hist[32];
  if (threadIdx.x < 32) s_hist[threadIdx.x] = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) {
    const uint32_t len = ranges[t].y - ranges[t].x;
    atomicAdd(&s_hist[__clz(len + 1u)], len >= split_pairs ? 4u : 1u);   // clz: 0 for the heaviest
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
    if (threadIdx.x == 31) *n_items = incl;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) {
    const uint32_t len = ranges[t].y - ranges[t].x;
    if (len >= split_pairs) {
      const uint32_t pos = atomicAdd(&s_hist[__clz(len + 1u)], 4u);
      for (uint32_t q = 0; q < 4; ++q) items[pos + q] = uint32_t(t) | ((q + 1u) << 24);
    } else {
      items[atomicAdd(&s_hist[__clz(len + 1u)], 1u)] = uint32_t(t);
    }
  }
}

}  // namespace

namespace {

template <int kMode, bool kCount, int kBatch>
void blend_launch_one(int grid, cudaStream_t st, const uint2* ranges, const uint32_t* items, const uint32_t* n_items,
                      uint32_t* tile_counter, const uint32_t* tk, const uint32_t* pv, const float4* rec,
                      uint32_t cap_slots, const CamConst& cam, float* rgb, float* t_out, unsigned long long* work,
                      uint32_t* frame, uint32_t* sticky) {
  if (kMode == 0)
    k_blend<kCount, kBatch><<<grid, kBlendThreads, 0, st>>>(ranges, items, n_items, tile_counter, tk, pv, rec, cap_slots,
                                                            cam.width, cam.height, cam.tiles_x,
                                                            cam.tiles_x * cam.tiles_y, rgb, t_out, work, frame, sticky);
  else
    k_blend_px<kCount, kBatch><<<grid, kBlendThreads, 0, st>>>(ranges, items, n_items, tile_counter, tk, pv, rec,
                                                               cap_slots, cam.width, cam.height, cam.tiles_x,
                                                               cam.tiles_x * cam.tiles_y, rgb, t_out, work, frame,
                                                               sticky);
}

template <int kMode, int kBatch>
void blend_launch(int grid, cudaStream_t st, const uint2* ranges, const uint32_t* items, const uint32_t* n_items,
                  uint32_t* tile_counter, const uint32_t* tk, const uint32_t* pv, const float4* rec, uint32_t cap_slots,
                  const CamConst& cam, float* rgb, float* t_out, unsigned long long* work, uint32_t* frame,
                  uint32_t* sticky) {
  if (work)
    blend_launch_one<kMode, true, kBatch>(grid, st, ranges, items, n_items, tile_counter, tk, pv, rec, cap_slots, cam,
                                          rgb, t_out, work, frame, sticky);
  else
    blend_launch_one<kMode, false, kBatch>(grid, st, ranges, items, n_items, tile_counter, tk, pv, rec, cap_slots, cam,
                                           rgb, t_out, nullptr, frame, sticky);
}

template <int kMode>
void blend_launch_batch(int batch, int grid, cudaStream_t st, const uint2* ranges, const uint32_t* items,
                        const uint32_t* n_items, uint32_t* tile_counter, const uint32_t* tk, const uint32_t* pv,
                        const float4* rec, uint32_t cap_slots, const CamConst& cam, float* rgb, float* t_out,
                        unsigned long long* work, uint32_t* frame, uint32_t* sticky) {
  if (batch == 128)
    blend_launch<kMode, 128>(grid, st, ranges, items, n_items, tile_counter, tk, pv, rec, cap_slots, cam, rgb, t_out,
                             work, frame, sticky);
  else if (batch == 256)
    blend_launch<kMode, 256>(grid, st, ranges, items, n_items, tile_counter, tk, pv, rec, cap_slots, cam, rgb, t_out,
                             work, frame, sticky);
  else
    blend_launch<kMode, 512>(grid, st, ranges, items, n_items, tile_counter, tk, pv, rec, cap_slots, cam, rgb, t_out,
                             work, frame, sticky);
}

}  // namespace

cudaError_t blend_set_attributes() {
  // several resident blocks of 11-43 KB shared memory per SM want the largest carveout
  const void* fns[] = {(const void*)k_blend<true, 128>,     (const void*)k_blend<false, 128>,
                       (const void*)k_blend<true, 256>,     (const void*)k_blend<false, 256>,
                       (const void*)k_blend<true, 512>,     (const void*)k_blend<false, 512>,
                       (const void*)k_blend_px<true, 128>,  (const void*)k_blend_px<false, 128>,
                       (const void*)k_blend_px<true, 256>,  (const void*)k_blend_px<false, 256>,
                       (const void*)k_blend_px<true, 512>,  (const void*)k_blend_px<false, 512>};
  for (const void* f : fns) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_blend(const uint2* ranges, uint32_t* items, uint32_t* tile_counter, const uint32_t* tk,
                         const uint32_t* pv, const float4* rec, uint32_t cap_slots, const CamConst& cam, float* rgb,
                         float* t_out, unsigned long long* work, uint32_t* frame, uint32_t* sticky,
                         uint32_t split_pairs, int batch, int mode, int n_views, int sm_count, cudaStream_t st) {
  const int n_tiles = cam.tiles_x * cam.tiles_y * n_views;
  if (n_tiles == 0) return cudaSuccess;
  if (batch != 128 && batch != 256 && batch != 512) return cudaErrorInvalidValue;
  if (mode != 0 && mode != 1) return cudaErrorInvalidValue;
  uint32_t* n_items = items + 4 * size_t(n_tiles);
  // the pixel-loop variant keeps whole tiles (a quadrant item would leave six of its warps idle)
  k_blend_items<<<1, 1024, 0, st>>>(ranges, n_tiles, mode == 1 ? 0xFFFFFFFFu : split_pairs, items, n_items);
  const int per_sm = mode == 1 ? blend_px_blocks_per_sm(batch) : blend_blocks_per_sm(batch);
  const int grid = std::min(4 * n_tiles, sm_count * per_sm);   // persistent: the resident blocks
  if (mode == 0)
    blend_launch_batch<0>(batch, grid, st, ranges, items, n_items, tile_counter, tk, pv, rec, cap_slots, cam, rgb, t_out,
                          work, frame, sticky);
  else
    blend_launch_batch<1>(batch, grid, st, ranges, items, n_items, tile_counter, tk, pv, rec, cap_slots, cam, rgb, t_out,
                          work, frame, sticky);
  return cudaGetLastError();
}

}  // namespace v3dg
