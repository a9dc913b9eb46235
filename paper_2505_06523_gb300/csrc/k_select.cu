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
// kSub: the sphere bounds a whole subtree; its rounding slack then also covers that of every
// sphere inside it (whose centre lies within R of this one), so that a culled subtree holds only
// nodes that the per-node test culls too.
template <bool kSub = false>
__device__ __forceinline__ bool cull_node(const float4 b, float sig, const InstFrame& I, const CamConst& cam) {
  const float px = fmaf(I.m[0], b.x, fmaf(I.m[1], b.y, fmaf(I.m[2], b.z, I.m[3])));
  const float py = fmaf(I.m[4], b.x, fmaf(I.m[5], b.y, fmaf(I.m[6], b.z, I.m[7])));
  const float pz = fmaf(I.m[8], b.x, fmaf(I.m[9], b.y, fmaf(I.m[10], b.z, I.m[11])));
  const float R = I.s * b.w;
  const float S = I.s * sig;
  const float slack = 1e-5f * (fabsf(px) + fabsf(py) + fabsf(pz) + (kSub ? 4.f : 1.f) * R) + (kSub ? 2e-6f : 1e-6f);
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
    const uint32_t block_total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t block_excl = chained_exclusive_warp(status, tile, block_total, epoch, frame + kTimeout);
    if (lane == 31) {
      s_total = incl;
      s_excl = block_excl;
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

// ---------------------------------------------------------------- top-down selection
// One level of the traversal.  Entry (i, n) of the frontier: if n is selected by the cut
// predicate (F_c(n) <= tau; F_p(n) = F_c(parent) > tau holds because the parent was expanded,
// and par[n] is a bit copy of own[parent], so footprint_le decides both alike), its bit is set
// in the instance's bitmap (mode 0: unless the visibility cull drops it); otherwise its children
// go to the next frontier.  n == n_nodes is the asset's virtual super-root, whose children are
// its roots.  in == nullptr: the implicit first frontier, one super-root per instance.
// mode 0 also drops every subtree whose bound the visibility cull rejects (no node in it could
// be kept).
__global__ void __launch_bounds__(kSelThreads)
k_td_step(const InstFrame* __restrict__ inst, int n_inst, const AssetDev* __restrict__ assets, CamConst cam,
          int mode, const uint2* __restrict__ in, const uint32_t* __restrict__ n_in, uint2* __restrict__ out,
          uint32_t* __restrict__ n_out, uint32_t cap_front, uint32_t* __restrict__ bitmap, uint32_t wpi,
          uint32_t* __restrict__ frame) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = in ? min(*n_in, cap_front) : uint32_t(n_inst);
  uint32_t gsum = 0, reached = 0;
  for (uint32_t e0 = blockIdx.x * blockDim.x; e0 < n; e0 += gridDim.x * blockDim.x) {   // uniform per warp
    const uint32_t e = e0 + threadIdx.x;
    uint32_t ii = 0, node = 0, c0 = 0, c1 = 0;
    const AssetDev* A = nullptr;
    if (e < n) {
      ++reached;
      if (in) {
        const uint2 en = in[e];
        ii = en.x;
        node = en.y;
      } else {
        ii = e;
        node = assets[inst[e].asset].n_nodes;
      }
      const InstFrame& I = inst[ii];
      A = &assets[I.asset];
      bool expand = node == A->n_nodes;
      if (!expand && !(mode == 0 && cull_node<true>(A->sub_bound[node], A->sub_sigma[node], I, cam))) {
        const uint8_t fl = A->flags[node];
        if ((fl & kLeaf) || footprint_le(A->own[node], I, cam, I.tau_f)) {
          if (mode == 1 || !cull_node(A->bound[node], A->sigma_max[node], I, cam)) {
            atomicOr(bitmap + size_t(ii) * wpi + (node >> 5), 1u << (node & 31u));
            if (mode == 1) gsum += A->count[node];
          }
        } else {
          expand = true;
        }
      }
      if (expand) {
        c0 = A->child_off[node];
        c1 = A->child_off[node + 1];
      }
    }
    // append the children, one atomic per warp
    const uint32_t k = c1 - c0;
    uint32_t incl = k;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= uint32_t(d)) incl += t;
    }
    const uint32_t wtotal = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t base = 0;
    if (lane == 31 && wtotal) base = atomicAdd(n_out, wtotal);
    base = __shfl_sync(0xffffffffu, base, 31) + incl - k;
    for (uint32_t j = 0; j < k; ++j) {
      if (base + j < cap_front)
        out[base + j] = make_uint2(ii, A->child_list[c0 + j]);
      else
        atomicOr(frame + kOverflow, 1u);
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    gsum += __shfl_xor_sync(0xffffffffu, gsum, d);
    reached += __shfl_xor_sync(0xffffffffu, reached, d);
  }
  if (lane == 0) {
    if (gsum) atomicAdd(frame + kCutGauss, gsum);
    if (reached) atomicAdd(frame + kTdReached, reached);
  }
}

// Ordered compaction of the selection bitmap into the (instance, node) list of k_select: one
// bitmap word per thread, words in (instance, node) order, offsets by a bounded look-back.
__global__ void __launch_bounds__(kSelThreads)
k_td_compact(const uint32_t* __restrict__ bitmap, uint32_t n_words, uint32_t wpi, int mode, uint2* __restrict__ out,
             uint32_t cap, uint32_t* __restrict__ frame, uint32_t tc_slot, uint64_t* __restrict__ status,
             uint32_t epoch) {
  __shared__ uint32_t s_tile, s_excl;
  __shared__ uint32_t s_scan[kSelWarps + 1];
  if (threadIdx.x == 0) s_tile = atomicAdd(frame + kTileCounters + tc_slot, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t ntiles = (n_words + kSelThreads - 1) / kSelThreads;
  if (tile >= ntiles) return;
  const uint32_t w = tile * kSelThreads + threadIdx.x;
  uint32_t word = w < n_words ? bitmap[w] : 0u;
  uint32_t total;
  const uint32_t ex = block_exclusive_scan<kSelWarps>(__popc(word), s_scan, &total);
  if (threadIdx.x < 32) {
    const uint32_t e = chained_exclusive_warp(status, tile, total, epoch, frame + kTimeout);
    if (threadIdx.x == 0) s_excl = e;
  }
  __syncthreads();
  uint32_t pos = s_excl + ex;
  const uint32_t ii = w / wpi, nb = (w % wpi) * 32u;
  while (word) {
    const uint32_t b = __ffs(word) - 1;
    word &= word - 1;
    if (pos < cap)
      out[pos] = make_uint2(ii, nb + b);
    else
      atomicOr(frame + kOverflow, 1u);
    ++pos;
  }
  if (threadIdx.x == 0 && tile == ntiles - 1) frame[mode == 0 ? kRenderNodes : kCutNodes] = s_excl + total;
}

}  // namespace

cudaError_t launch_select_topdown(const InstFrame* inst, int n_inst, const AssetDev* assets, const CamConst& cam,
                                  int mode, const TopDown& td, uint2* out, uint32_t cap, uint32_t* frame,
                                  uint32_t tile_counter_slot, uint64_t* status, uint32_t epoch, int sm_count,
                                  cudaStream_t st, int* launches) {
  if (n_inst <= 0) return cudaSuccess;
  const uint32_t n_words = uint32_t(n_inst) * td.wpi;
  cudaError_t e = cudaMemsetAsync(td.bitmap, 0, sizeof(uint32_t) * size_t(n_words), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(td.counts, 0, sizeof(uint32_t) * size_t(td.steps + 1), st);
  if (e != cudaSuccess) return e;
  for (int s = 0; s < td.steps; ++s) {
    const uint2* in = s == 0 ? nullptr : td.frontier[s & 1];
    k_td_step<<<sm_count * 8, kSelThreads, 0, st>>>(inst, n_inst, assets, cam, mode, in, td.counts + s,
                                                    td.frontier[(s + 1) & 1], td.counts + s + 1, td.cap_front,
                                                    td.bitmap, td.wpi, frame);
    ++*launches;
  }
  k_td_compact<<<(n_words + kSelThreads - 1) / kSelThreads, kSelThreads, 0, st>>>(
      td.bitmap, n_words, td.wpi, mode, out, cap, frame, tile_counter_slot, status, epoch);
  ++*launches;
  return cudaGetLastError();
}

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
