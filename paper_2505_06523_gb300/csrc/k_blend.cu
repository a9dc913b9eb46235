// Per-tile front-to-back alpha blending (Sec. 2.1): C = sum_i c_i a_i prod_{j<i} (1 - a_j).
//
// One 256-thread block per 16x16 tile, one pixel per thread.  The tile's depth-ordered records
// are staged through shared memory in batches of 256; a batch starts only while some pixel of the
// tile is still accumulating (block-wide early exit).  Per pixel and Gaussian:
//   log2 a = na dx^2 + nb dx dy + nc dy^2 + log2 o, a = min(0.999, 2^(log2 a)),
//   skip a < 1/255, stop before T (1 - a) < 1e-4.
// Each record's mean is stored relative to the pixel origin of its first tile, so the per-pixel
// offsets dx, dy are differences of small numbers.  Each record also carries the pixel box of its
// alpha >= 1/255 ellipse; staged as a row mask and a column mask for this tile, it lets a pixel
// outside the box skip the Gaussian with one AND (outside the box alpha < 1/255, so nothing
// changes).
#include "dev_common.cuh"

namespace v3dg {
namespace {

constexpr int kBlendThreads = 256;
constexpr float kLog2MinAlpha = -7.9943534f;  // log2(1/255)

template <bool kCount>
__global__ void __launch_bounds__(kBlendThreads)
k_blend(const uint2* __restrict__ ranges, const uint32_t* __restrict__ pv, const float4* __restrict__ rec,
        uint32_t cap_slots, int width, int height, int tiles_x, float* __restrict__ rgb, float* __restrict__ t_out,
        unsigned long long* __restrict__ work) {
  __shared__ float4 s_g[kBlendThreads];   // (u, v, na, nb) in this tile's pixel frame
  __shared__ float4 s_c[kBlendThreads];   // (nc, log2 o, r, g)
  __shared__ float2 s_b[kBlendThreads];   // (b, row mask << 16 | column mask)
  const int tile = blockIdx.x;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int lx = threadIdx.x & 15, ly = threadIdx.x >> 4;
  const int px = tx * 16 + lx, py = ty * 16 + ly;
  const bool inside = px < width && py < height;
  const float fx = float(lx) + 0.5f, fy = float(ly) + 0.5f;
  const uint32_t mybits = (1u << lx) | (1u << (16 + ly));
  const uint2 range = ranges[tile];
  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f;
  bool done = !inside;
  uint32_t n_eval = 0, n_contrib = 0;
  for (uint32_t b0 = range.x; b0 < range.y; b0 += kBlendThreads) {
    if (__syncthreads_count(done) == kBlendThreads) break;
    const uint32_t i = b0 + threadIdx.x;
    const uint32_t slot = i < range.y ? pv[i] : 0xFFFFFFFFu;
    if (slot < cap_slots) {
      const float4* r = rec + 3 * size_t(slot);
      const float4 r0 = r[0], r1 = r[1], r2 = r[2];
      const uint32_t org = __float_as_uint(r2.y);
      const float ox = float(16 * (tx - int(org & 0xFFFFu))), oy = float(16 * (ty - int(org >> 16)));
      s_g[threadIdx.x] = make_float4(r0.x - ox, r0.y - oy, r0.z, r0.w);
      s_c[threadIdx.x] = r1;
      // rows / columns of this tile inside the Gaussian's pixel box
      const uint32_t bx = __float_as_uint(r2.z), by = __float_as_uint(r2.w);
      const int cx0 = max(int(bx & 0xFFFFu) - 16 * tx, 0), cx1 = min(int(bx >> 16) - 16 * tx, 15);
      const int cy0 = max(int(by & 0xFFFFu) - 16 * ty, 0), cy1 = min(int(by >> 16) - 16 * ty, 15);
      const uint32_t cm = cx0 <= cx1 ? ((0xFFFFu >> (15 - cx1)) & (0xFFFFu << cx0)) : 0u;
      const uint32_t rm = cy0 <= cy1 ? ((0xFFFFu >> (15 - cy1)) & (0xFFFFu << cy0)) : 0u;
      s_b[threadIdx.x] = make_float2(r2.x, __uint_as_float(cm | (rm << 16)));
    } else {  // out of range (never for a valid frame): an empty record
      s_g[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
      s_c[threadIdx.x] = make_float4(0.f, -1e30f, 0.f, 0.f);
      s_b[threadIdx.x] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int nb = int(min(uint32_t(kBlendThreads), range.y - b0));
    for (int j = 0; j < nb && !done; ++j) {
      const float2 bm = s_b[j];
      if ((__float_as_uint(bm.y) & mybits) != mybits) continue;
      const float4 g = s_g[j];
      if (kCount) ++n_eval;
      const float dx = fx - g.x, dy = fy - g.y;
      const float4 c = s_c[j];
      const float l2a = fmaf(dx, fmaf(g.z, dx, g.w * dy), fmaf(c.x * dy, dy, c.y));
      if (l2a < kLog2MinAlpha) continue;
      const float alpha = fminf(0.999f, exp2f(l2a));
      if (alpha < 1.f / 255.f) continue;
      const float tn = T * (1.f - alpha);
      if (tn < 1e-4f) {
        done = true;
        break;
      }
      if (kCount) ++n_contrib;
      const float w = alpha * T;
      cr = fmaf(w, c.z, cr);
      cg = fmaf(w, c.w, cg);
      cb = fmaf(w, bm.x, cb);
      T = tn;
    }
  }
  if (inside) {
    const size_t p = size_t(py) * width + px;
    rgb[3 * p + 0] = cr;
    rgb[3 * p + 1] = cg;
    rgb[3 * p + 2] = cb;
    if (t_out) t_out[p] = T;
  }
  if (kCount) {
    unsigned long long e = n_eval, cnt = n_contrib;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, d);
      cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(work, e);
      atomicAdd(work + 1, cnt);
    }
  }
}

}  // namespace

cudaError_t launch_blend(const uint2* ranges, const uint32_t* pv, const float4* rec, uint32_t cap_slots,
                         const CamConst& cam, float* rgb, float* t_out, unsigned long long* work, cudaStream_t st) {
  const int n_tiles = cam.tiles_x * cam.tiles_y;
  if (n_tiles == 0) return cudaSuccess;
  if (work)
    k_blend<true><<<n_tiles, kBlendThreads, 0, st>>>(ranges, pv, rec, cap_slots, cam.width, cam.height, cam.tiles_x,
                                                     rgb, t_out, work);
  else
    k_blend<false><<<n_tiles, kBlendThreads, 0, st>>>(ranges, pv, rec, cap_slots, cam.width, cam.height, cam.tiles_x,
                                                      rgb, t_out, nullptr);
  return cudaGetLastError();
}

}  // namespace v3dg
