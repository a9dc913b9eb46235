// Selection: per-(instance, cluster) footprints and the cut predicate F_c <= tau < F_p
// (Sec. 3.3 Fig. 4, Sec. 3.4), with stable stream compaction of the cut in (instance, node) order.
//
// A block covers 2048 consecutive nodes of one instance, 8 per thread (node = base + i * 256 +
// thread).  Blocks take virtual tile ids from an atomic counter, compact their selected nodes in
// (item, warp, lane) order -- which is node order -- and find their output offset with a bounded
// decoupled look-back, so the cut is written in one pass.
#include "dev_common.cuh"

namespace v3dg {
namespace {

constexpr int kSelThreads = 256;
constexpr int kSelItems = 8;
constexpr int kSelWarps = kSelThreads / 32;
constexpr float kEps = 5.9604645e-08f;  // 2^-24

// F(sphere) <= tau for one asset-space sphere (c, r) under instance I, where
// F = pi fx fy (s r)^2 / z^2 and F = +inf when |z| <= s r.  The float32 evaluation carries a
// forward error bound; inside that band the value is recomputed in FP64 with the same operation
// order as the definition, so the decision agrees with an exact FP64 evaluation.
__device__ __forceinline__ bool footprint_le(const float4 c, const InstFrame& I, const CamConst& cam,
                                             float tau) {
  const float t0 = I.m[8] * c.x, t1 = I.m[9] * c.y, t2 = I.m[10] * c.z, t3 = I.m[11];
  const float z = ((t0 + t1) + t2) + t3;
  const float mag = fabsf(t0) + fabsf(t1) + fabsf(t2) + fabsf(t3);
  const float ez = mag * (8.f * kEps) + 1e-37f;
  const float r = I.s * c.w;
  const float er = r * (4.f * kEps);
  const float az = fabsf(z);
  if (az - ez > r + er) {
    const float lhs = cam.k_foot32 * r * r;  // pi fx fy r'^2
    const float rhs = tau * z * z;           // tau z^2
    const float el = lhs * (16.f * kEps);
    const float erh = rhs * (2.f * ez / az + 8.f * kEps);
    if (lhs + el < rhs - erh) return true;
    if (lhs - el > rhs + erh) return false;
  } else if (az + ez < r - er) {
    return false;  // the sphere surely reaches the camera plane: F = +inf
  }
  const double zd = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(I.m64[8], double(c.x)), __dmul_rn(I.m64[9], double(c.y))),
                                        __dmul_rn(I.m64[10], double(c.z))),
                              I.m64[11]);
  const double rd = I.s64 * double(c.w);
  if (!(fabs(zd) > rd)) return false;
  const double f = cam.k_foot * rd * rd / (zd * zd);
  return f <= double(tau);
}

// True when no Gaussian of the node can reach a pixel centre: every mean lies behind the near
// plane, or the node's means, widened by the largest alpha >= 1/255 half-width their 2D
// Gaussians can have, lie beyond one image edge.  Conservative by construction (1 px margin).
__device__ __forceinline__ bool cull_node(const float4 b, float sig, const InstFrame& I, const CamConst& cam) {
  const float px = fmaf(I.m[0], b.x, fmaf(I.m[1], b.y, fmaf(I.m[2], b.z, I.m[3])));
  const float py = fmaf(I.m[4], b.x, fmaf(I.m[5], b.y, fmaf(I.m[6], b.z, I.m[7])));
  const float pz = fmaf(I.m[8], b.x, fmaf(I.m[9], b.y, fmaf(I.m[10], b.z, I.m[11])));
  const float R = I.s * b.w;
  const float S = I.s * sig;
  const float slack = 1e-5f * (fabsf(px) + fabsf(py) + fabsf(pz) + R) + 1e-6f;
  if (pz + R + slack < cam.near_z) return true;
  const float m = 1.0f;
  {  // right edge: fx x - (W - 0.5 - cx + m) z > kx S fx over the ball
    const float nx = cam.fx, nz = -(float(cam.width) - 0.5f - cam.cx + m);
    const float nn = sqrtf(nx * nx + nz * nz);
    if (nx * px + nz * pz - nn * (R + slack) > cam.cull_kx * S * cam.fx) return true;
  }
  {  // left edge
    const float nx = -cam.fx, nz = 0.5f - cam.cx - m;
    const float nn = sqrtf(nx * nx + nz * nz);
    if (nx * px + nz * pz - nn * (R + slack) > cam.cull_kx * S * cam.fx) return true;
  }
  {  // bottom edge
    const float ny = cam.fy, nz = -(float(cam.height) - 0.5f - cam.cy + m);
    const float nn = sqrtf(ny * ny + nz * nz);
    if (ny * py + nz * pz - nn * (R + slack) > cam.cull_ky * S * cam.fy) return true;
  }
  {  // top edge
    const float ny = -cam.fy, nz = 0.5f - cam.cy - m;
    const float nn = sqrtf(ny * ny + nz * nz);
    if (ny * py + nz * pz - nn * (R + slack) > cam.cull_ky * S * cam.fy) return true;
  }
  return false;
}

__global__ void __launch_bounds__(kSelThreads)
k_select(const InstFrame* __restrict__ inst, int n_inst, const AssetDev* __restrict__ assets, int node_blocks,
         CamConst cam, int mode, uint2* __restrict__ out, uint32_t cap, uint32_t* __restrict__ frame,
         uint32_t tc_slot, uint64_t* __restrict__ status, uint32_t epoch) {
  __shared__ uint32_t s_tile, s_excl, s_total;
  __shared__ uint32_t s_cnt[kSelItems * kSelWarps];   // per (item, warp): selected count, then offset
  __shared__ uint32_t s_gauss[kSelWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(frame + kTileCounters + tc_slot, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t ntiles = uint32_t(n_inst) * uint32_t(node_blocks);
  if (tile >= ntiles) return;
  const uint32_t ii = tile / node_blocks, nb = tile % node_blocks;
  const InstFrame& I = inst[ii];
  const AssetDev& A = assets[I.asset];
  const float tau = I.tau_f;
  uint32_t keepmask = 0, gsum = 0;
#pragma unroll
  for (int i = 0; i < kSelItems; ++i) {
    const uint32_t node = nb * (kSelThreads * kSelItems) + i * kSelThreads + threadIdx.x;
    bool keep = false;
    if (node < A.n_nodes) {
      const uint8_t fl = A.flags[node];
      const bool own_ok = (fl & kLeaf) || footprint_le(A.own[node], I, cam, tau);
      const bool sel = own_ok && ((fl & kRoot) || !footprint_le(A.par[node], I, cam, tau));
      if (sel) {
        keep = (mode == 1) || !cull_node(A.bound[node], A.sigma_max[node], I, cam);
        if (mode == 1) gsum += A.count[node];
      }
    }
    const uint32_t b = __ballot_sync(0xffffffffu, keep);
    if (keep) keepmask |= 1u << i;
    if (lane == 0) s_cnt[i * kSelWarps + warp] = __popc(b);
  }
  if (mode == 1) {  // Gaussians in the cut, one atomic per block
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) gsum += __shfl_xor_sync(0xffffffffu, gsum, d);
    if (lane == 0) s_gauss[warp] = gsum;
  }
  __syncthreads();
  if (warp == 0) {  // exclusive scan of the 64 (item, warp) counts in that order
    const uint32_t a = s_cnt[2 * lane], b = s_cnt[2 * lane + 1];
    uint32_t incl = a + b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    const uint32_t ex = incl - a - b;
    s_cnt[2 * lane] = ex;
    s_cnt[2 * lane + 1] = ex + a;
    if (lane == 31) {
      s_total = incl;
      s_excl = chained_exclusive(status, 1, tile, incl, epoch, frame + kTimeout);
      if (mode == 1) {
        uint32_t g = 0;
        for (int w = 0; w < kSelWarps; ++w) g += s_gauss[w];
        if (g) atomicAdd(frame + kCutGauss, g);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kSelItems; ++i) {
    const bool keep = (keepmask >> i) & 1u;
    const uint32_t b = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const uint32_t pos = s_excl + s_cnt[i * kSelWarps + warp] + __popc(b & lanemask_lt());
      const uint32_t node = nb * (kSelThreads * kSelItems) + i * kSelThreads + threadIdx.x;
      if (pos < cap)
        out[pos] = make_uint2(ii, node);
      else
        atomicOr(frame + kOverflow, 1u);
    }
  }
  if (threadIdx.x == 0 && tile == ntiles - 1) frame[mode == 0 ? kRenderNodes : kCutNodes] = s_excl + s_total;
}

}  // namespace

cudaError_t launch_select(const InstFrame* inst, int n_inst, const AssetDev* assets, int node_blocks,
                          const CamConst& cam, int mode, uint2* out, uint32_t cap, uint32_t* frame,
                          uint32_t tile_counter_slot, uint64_t* status, uint32_t epoch, cudaStream_t st) {
  const uint32_t blocks = uint32_t(n_inst) * uint32_t(node_blocks);
  if (blocks == 0) return cudaSuccess;
  k_select<<<blocks, kSelThreads, 0, st>>>(inst, n_inst, assets, node_blocks, cam, mode, out, cap, frame,
                                           tile_counter_slot, status, epoch);
  return cudaGetLastError();
}

}  // namespace v3dg
