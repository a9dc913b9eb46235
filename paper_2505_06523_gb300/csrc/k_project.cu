// Projection of the selected Gaussians (Sec. 2.1; Sec. 5.1: EWA splatting without 2D dilation).
//
// k_noderef: one thread per render-list node computes, in FP64, the view-space position of the
//   node's mean centre and its pixel position, so that every Gaussian of the node can be placed
//   relative to it with small float32 offsets (the screen mean stays accurate to ~1e-7 of the
//   node's extent instead of 1 ulp of the whole view distance).
// k_project: a warp takes a chunk of consecutive render-list entries at a time (16 in list
//   order; 32 when, for scenes of many instances of few assets, the entries come grouped by
//   cluster through a radix sort of their global cluster ids), stages the chunk's per-entry
//   constants (instance matrix, camera centre, FP64 reference) in shared memory, and projects
//   each run of entries that draw the same cluster together, 2 Gaussians per lane: a Gaussian's
//   attributes -- mean, opacity, normalised quaternion, scales and all SH coefficients -- are
//   loaded into registers once per run and used for every entry of it, so a cluster drawn by k
//   instances is read once, not k times.  Loads are attribute-major (each cluster's attributes
//   are one contiguous block of planes of 64 values, so every warp load is one 128-byte line).
//   Writes a 48-byte blend record, the pixel box and the float32 depth key per Gaussian;
//   culled slots get the key 0xFFFFFFFF so that the depth sort moves them behind all visible ones.
#include <algorithm>

#include <cuda_fp16.h>

#include "dev_common.cuh"

namespace v3dg {
namespace {

constexpr int kProjThreads = 256;

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kMinOpacity = 0.0039215689f;  // smallest float >= 1/255 (0x3b808081)

// Real spherical harmonics l <= 3 (closed forms: 1/(2 sqrt(pi)), sqrt(3/(4 pi)), ...).
constexpr float kY0 = 0.28209479177387814f;   // 1/2 sqrt(1/pi)
constexpr float kY1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float kY2a = 1.0925484305920792f;   // 1/2 sqrt(15/pi)
constexpr float kY2b = 0.31539156525252005f;  // 1/4 sqrt(5/pi)
constexpr float kY2c = 0.5462742152960396f;   // 1/4 sqrt(15/pi)
constexpr float kY3a = 0.5900435899266435f;   // 1/4 sqrt(35/(2 pi))
constexpr float kY3b = 2.890611442640554f;    // 1/2 sqrt(105/pi)
constexpr float kY3c = 0.4570457994644658f;   // 1/4 sqrt(21/(2 pi))
constexpr float kY3d = 0.3731763325901154f;   // 1/4 sqrt(7/pi)
constexpr float kY3e = 1.445305721320277f;    // 1/4 sqrt(105/pi)

__global__ void __launch_bounds__(256)
k_noderef(const uint2* __restrict__ list, uint32_t cap, const InstFrame* __restrict__ inst,
          const AssetDev* __restrict__ assets, CamConst cam, float4* __restrict__ ref,
          const uint32_t* __restrict__ frame, uint32_t* __restrict__ order_keys, int key_shift) {
  const uint32_t n = min(frame[kRenderNodes], cap);
  for (uint32_t ci = blockIdx.x * blockDim.x + threadIdx.x; ci < n; ci += gridDim.x * blockDim.x) {
    const uint2 e = list[ci];
    const InstFrame& I = inst[e.x];
    const AssetDev& A = assets[I.asset];
    if (order_keys) order_keys[ci] = (A.node_base + e.y) >> key_shift;
    const float4 b = A.bound[e.y];
    const double bx = b.x, by = b.y, bz = b.z;
    const double X = ((I.m64[0] * bx + I.m64[1] * by) + I.m64[2] * bz) + I.m64[3];
    const double Y = ((I.m64[4] * bx + I.m64[5] * by) + I.m64[6] * bz) + I.m64[7];
    const double Z = ((I.m64[8] * bx + I.m64[9] * by) + I.m64[10] * bz) + I.m64[11];
    const double rho = I.s64 * double(b.w);
    float4 r0, r1;
    if (Z > 4.0 * rho && Z > 1e-6 && fabs(X) <= 4.0 * Z && fabs(Y) <= 4.0 * Z) {
      const double rx = X / Z, ry = Y / Z;
      const double U = double(cam.fx) * rx + double(cam.cx);
      const double V = double(cam.fy) * ry + double(cam.cy);
      const float uh = float(U), vh = float(V);
      r0 = make_float4(uh, float(U - double(uh)), vh, float(V - double(vh)));
      r1 = make_float4(float(rx), float(ry), float(Z), 1.f);
    } else {
      r0 = make_float4(cam.cx, 0.f, cam.cy, 0.f);
      r1 = make_float4(float(X), float(Y), float(Z), 0.f);
    }
    ref[2 * ci] = r0;
    ref[2 * ci + 1] = r1;
  }
}

__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__half x) { return __half2float(x); }

// Instance-independent values of one Gaussian: its mean and opacity, its normalised quaternion,
// its scales, the opacity terms of the record and the box, and its SH coefficients.  Computed
// once per (cluster run, Gaussian) and used for every instance of the run.
struct GaussPre {
  float mx, my, mz, op;
  float qw, qx, qy, qz;   // unit quaternion
  float s0, s1, s2;
  float kq;     // 2 ln(255 o): the alpha >= 1/255 ellipse is q <= kq
  float l2op;   // log2 o
  float sh[3 * kMaxShCoeffs];   // SH coefficients, coefficient-major (0 beyond the asset's degree)
};

template <typename TC>
__device__ __forceinline__ GaussPre gauss_pre(uint32_t j, int nsh, const float* __restrict__ at,
                                              const TC* __restrict__ col) {
  constexpr size_t st = kSlots;   // values between planes
  GaussPre G;
#pragma unroll
  for (int k = 0; k < 3 * kMaxShCoeffs; ++k) G.sh[k] = k < 3 * nsh ? to_f32(col[(kSh0 + k) * st + j]) : 0.f;
  G.mx = at[kX * st + j];
  G.my = at[kY * st + j];
  G.mz = at[kZ * st + j];
  G.op = to_f32(col[kOpacity * st + j]);
  float qw = at[kQw * st + j], qx = at[kQx * st + j], qy = at[kQy * st + j], qz = at[kQz * st + j];
  const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  G.qw = qw * qn; G.qx = qx * qn; G.qy = qy * qn; G.qz = qz * qn;
  G.s0 = expf(at[kLs0 * st + j]);
  G.s1 = expf(at[kLs1 * st + j]);
  G.s2 = expf(at[kLs2 * st + j]);
  G.kq = 2.f * logf(255.f * G.op);
  G.l2op = log2f(G.op);
  return G;
}

// Per-entry constants of a warp's chunk, staged in shared memory: the rows of the instance
// frame's float32 M, its camera centre in the asset frame (and scale), and the entry's FP64
// reference from k_noderef.
struct EntryConst {
  float4 m0, m1, m2;   // M[0..3], M[4..7], M[8..11]
  float4 cam;          // cam_a[0..2], s
  float4 r0, r1;
};
static_assert(offsetof(InstFrame, m) % 16 == 0 && offsetof(InstFrame, cam_a) % 16 == 0 &&
              offsetof(InstFrame, s) == offsetof(InstFrame, cam_a) + 12, "InstFrame float4 views");

// Projects a Gaussian of a cluster (its pre-computed values G) for one entry (its constants E)
// into slot `slot`; returns whether it is visible.  bc: the cluster's bound centre (asset frame).
__device__ __forceinline__ bool project_one(const GaussPre& G, size_t slot, const EntryConst& E,
                                            const CamConst& cam, const float4 bc, int nsh,
                                            float4* __restrict__ rec, uint2* __restrict__ rect,
                                            uint32_t* __restrict__ keys, uint32_t* __restrict__ frame) {
  const float4 M0 = E.m0, M1 = E.m1, M2 = E.m2, CA = E.cam, r0 = E.r0, r1 = E.r1;
  const struct { float m[12]; float cam_a[3]; } I = {{M0.x, M0.y, M0.z, M0.w, M1.x, M1.y, M1.z, M1.w, M2.x, M2.y, M2.z, M2.w},
                                                    {CA.x, CA.y, CA.z}};
  const bool comp = r1.w != 0.f;
  const float mx = G.mx, my = G.my, mz = G.mz;
  // float32 depth key: ((M20 x + M21 y) + M22 z) + M23, every step rounded (no fusion)
  const float z32 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(I.m[8], mx), __fmul_rn(I.m[9], my)),
                                        __fmul_rn(I.m[10], mz)), I.m[11]);
  bool vis = (z32 >= cam.near_z) && (G.op >= kMinOpacity);
  // offsets from the node centre in view space
  const float dx0 = mx - bc.x, dy0 = my - bc.y, dz0 = mz - bc.z;
  const float a = fmaf(I.m[0], dx0, fmaf(I.m[1], dy0, I.m[2] * dz0));
  const float b = fmaf(I.m[4], dx0, fmaf(I.m[5], dy0, I.m[6] * dz0));
  const float c = fmaf(I.m[8], dx0, fmaf(I.m[9], dy0, I.m[10] * dz0));
  const float z = r1.z + c;
  float corr_u, corr_v, xz, yz;
  if (comp) {
    const float eu = (a - r1.x * c) / z, ev = (b - r1.y * c) / z;
    corr_u = cam.fx * eu;
    corr_v = cam.fy * ev;
    xz = r1.x + eu;
    yz = r1.y + ev;
  } else {
    xz = (r1.x + a) / z;
    yz = (r1.y + b) / z;
    corr_u = cam.fx * xz;
    corr_v = cam.fy * yz;
  }
  // covariance factor A = M3 R(q) diag(exp(log-scale)): Sigma_v = A A^T
  const float qw = G.qw, qx = G.qx, qy = G.qy, qz = G.qz;
  const float R00 = 1.f - 2.f * (qy * qy + qz * qz), R01 = 2.f * (qx * qy - qw * qz), R02 = 2.f * (qx * qz + qw * qy);
  const float R10 = 2.f * (qx * qy + qw * qz), R11 = 1.f - 2.f * (qx * qx + qz * qz), R12 = 2.f * (qy * qz - qw * qx);
  const float R20 = 2.f * (qx * qz - qw * qy), R21 = 2.f * (qy * qz + qw * qx), R22 = 1.f - 2.f * (qx * qx + qy * qy);
  float Am[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float m0 = I.m[4 * r], m1 = I.m[4 * r + 1], m2 = I.m[4 * r + 2];
    Am[r][0] = fmaf(m0, R00, fmaf(m1, R10, m2 * R20)) * G.s0;
    Am[r][1] = fmaf(m0, R01, fmaf(m1, R11, m2 * R21)) * G.s1;
    Am[r][2] = fmaf(m0, R02, fmaf(m1, R12, m2 * R22)) * G.s2;
  }
  // EWA Jacobian at the mean, clamped to 1.3x the half field of view
  const float rz = 1.f / z;
  const float J00 = cam.fx * rz, J11 = cam.fy * rz;
  const float J02 = -cam.fx * fminf(fmaxf(xz, -cam.limx), cam.limx) * rz;
  const float J12 = -cam.fy * fminf(fmaxf(yz, -cam.limy), cam.limy) * rz;
  const float T00 = fmaf(J00, Am[0][0], J02 * Am[2][0]), T01 = fmaf(J00, Am[0][1], J02 * Am[2][1]),
              T02 = fmaf(J00, Am[0][2], J02 * Am[2][2]);
  const float T10 = fmaf(J11, Am[1][0], J12 * Am[2][0]), T11 = fmaf(J11, Am[1][1], J12 * Am[2][1]),
              T12 = fmaf(J11, Am[1][2], J12 * Am[2][2]);
  const float ca = fmaf(T00, T00, fmaf(T01, T01, T02 * T02));
  const float cb = fmaf(T00, T10, fmaf(T01, T11, T02 * T12));
  const float cc = fmaf(T10, T10, fmaf(T11, T11, T12 * T12));
  // det(T T^T) as the sum of squared 2x2 minors (Cauchy-Binet): never negative
  const float m01 = fmaf(T00, T11, -T01 * T10), m02 = fmaf(T00, T12, -T02 * T10), m12 = fmaf(T01, T12, -T02 * T11);
  const float det = fmaf(m01, m01, fmaf(m02, m02, m12 * m12));
  float ia, ib, ic;
  if (det >= 1e-12f) {
    const float id = 1.f / det;
    ia = cc * id;
    ib = -cb * id;
    ic = ca * id;
  } else {  // near-singular: form and invert Sigma_2D in FP64 (rare: counted)
    atomicAdd(frame + kConicFp64, 1u);
    const double d00 = double(T00), d01 = double(T01), d02 = double(T02);
    const double d10 = double(T10), d11 = double(T11), d12 = double(T12);
    const double e01 = d00 * d11 - d01 * d10, e02 = d00 * d12 - d02 * d10, e12 = d01 * d12 - d02 * d11;
    const double dd = e01 * e01 + e02 * e02 + e12 * e12;
    if (!(dd > 0.0)) vis = false;
    const double idd = 1.0 / dd;
    ia = float((d10 * d10 + d11 * d11 + d12 * d12) * idd);
    ib = float(-(d00 * d10 + d01 * d11 + d02 * d12) * idd);
    ic = float((d00 * d00 + d01 * d01 + d02 * d02) * idd);
  }
  // alpha >= 1/255 ellipse: q <= k = 2 ln(255 o); its box half-widths sqrt(k Sigma_xx), sqrt(k Sigma_yy)
  const float hx = sqrtf(fmaxf(G.kq * ca, 0.f)), hy = sqrtf(fmaxf(G.kq * cc, 0.f));
  const float u = r0.x + (r0.y + corr_u), v = r0.z + (r0.w + corr_v);
  float x0 = fmaxf(ceilf(u - hx - 0.5f), 0.f), x1 = fminf(floorf(u + hx - 0.5f), float(cam.width - 1));
  float y0 = fmaxf(ceilf(v - hy - 0.5f), 0.f), y1 = fminf(floorf(v + hy - 0.5f), float(cam.height - 1));
  vis = vis && (x0 <= x1) && (y0 <= y1) && isfinite(u) && isfinite(v);
  if (!vis) {
    keys[slot] = 0xFFFFFFFFu;
    return false;
  }
  const int tx0 = int(x0) >> 4, ty0 = int(y0) >> 4;
  // mean relative to the first tile's pixel origin (exact subtraction of the integer part)
  const float u_rel = (r0.x - float(16 * tx0)) + (r0.y + corr_u);
  const float v_rel = (r0.z - float(16 * ty0)) + (r0.w + corr_v);
  // colour: SH in the asset frame along the direction from the camera centre
  float dx = mx - I.cam_a[0], dy = my - I.cam_a[1], dz = mz - I.cam_a[2];
  const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
  dx *= dn; dy *= dn; dz *= dn;
  float Y[kMaxShCoeffs];
  Y[0] = kY0;
  if (nsh > 1) {
    Y[1] = -kY1 * dy; Y[2] = kY1 * dz; Y[3] = -kY1 * dx;
  }
  if (nsh > 4) {
    const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
    Y[4] = kY2a * dx * dy; Y[5] = -kY2a * dy * dz; Y[6] = kY2b * (2.f * zz - xx - yy);
    Y[7] = -kY2a * dx * dz; Y[8] = kY2c * (xx - yy);
    if (nsh > 9) {
      Y[9] = -kY3a * dy * (3.f * xx - yy); Y[10] = kY3b * dx * dy * dz;
      Y[11] = -kY3c * dy * (4.f * zz - xx - yy); Y[12] = kY3d * dz * (2.f * zz - 3.f * xx - 3.f * yy);
      Y[13] = -kY3c * dx * (4.f * zz - xx - yy); Y[14] = kY3e * dz * (xx - yy);
      Y[15] = -kY3a * dx * (xx - 3.f * yy);
    }
  }
  float rgb[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxShCoeffs; ++k)
      if (k < nsh) acc = fmaf(Y[k], G.sh[3 * k + ch], acc);
    rgb[ch] = fmaxf(acc + 0.5f, 0.f);
  }
  const uint32_t origin = uint32_t(tx0) | (uint32_t(ty0) << 16);
  float4* rp = rec + 3 * slot;
  rp[0] = make_float4(u_rel, v_rel, -0.5f * kLog2e * ia, -kLog2e * ib);
  rp[1] = make_float4(-0.5f * kLog2e * ic, G.l2op, rgb[0], rgb[1]);
  rp[2] = make_float4(rgb[2], __uint_as_float(origin), __uint_as_float(uint32_t(x0) | (uint32_t(x1) << 16)),
                      __uint_as_float(uint32_t(y0) | (uint32_t(y1) << 16)));
  rect[slot] = make_uint2(uint32_t(x0) | (uint32_t(x1) << 16), uint32_t(y0) | (uint32_t(y1) << 16));
  keys[slot] = __float_as_uint(z32);
  return true;
}

// One run of render-list entries that draw the same cluster (entries e = a .. b - 1 of the warp's
// chunk; their indices ci are in lanes e, their constants in ent[e]): each lane takes Gaussians
// lane and lane + 32 of the cluster, loads their attributes and computes their
// instance-independent values once, and projects them for every entry of the run.
template <typename TC>
__device__ __forceinline__ uint32_t project_run(int lane, int a, int b, uint32_t ci, uint32_t cnt,
                                                const EntryConst* ent, const CamConst& cam, const float4 bc, int nsh,
                                                const float* __restrict__ at, const TC* __restrict__ col,
                                                float4* __restrict__ rec, uint2* __restrict__ rect,
                                                uint32_t* __restrict__ keys, uint32_t* __restrict__ frame) {
  uint32_t nvis = 0;
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const uint32_t j = lane + 32 * h;
    GaussPre G;
    if (j < cnt) G = gauss_pre<TC>(j, nsh, at, col);
#pragma unroll 1
    for (int e = a; e < b; ++e) {
      const uint32_t ce = __shfl_sync(0xffffffffu, ci, e);
      const size_t slot = size_t(ce) * kSlots + j;
      if (j >= cnt) {
        keys[slot] = 0xFFFFFFFFu;
        continue;
      }
      nvis += project_one(G, slot, ent[e], cam, bc, nsh, rec, rect, keys, frame) ? 1u : 0u;
    }
  }
  return nvis;
}

// kFormats: bit 0 = float32 colour planes occur, bit 1 = float16 ones occur.  Each warp takes
// chunks of `chunk` (1..32) consecutive positions of the order (list order when `order` is NULL),
// stages their constants in shared memory and splits the chunk into runs of entries that draw the
// same (asset, cluster).
constexpr int kMaxChunk = 32;
// chunk sizes (measured on the crowd: 8 to 32 within 1% grouped; 16 best in list order)
constexpr int kProjChunkGrouped = 32, kProjChunkList = 16;
constexpr int kProjChunkCounter = 15;   // the frame's tile-counter word of the chunk queue
template <int kFormats>
__global__ void __launch_bounds__(kProjThreads, 2)
k_project(const uint2* __restrict__ list, uint32_t cap_nodes, const InstFrame* __restrict__ inst,
          const AssetDev* __restrict__ assets, CamConst cam, const float4* __restrict__ ref,
          float4* __restrict__ rec, uint2* __restrict__ rect, uint32_t* __restrict__ keys,
          uint32_t* __restrict__ frame, const uint32_t* __restrict__ order,
          const uint32_t* __restrict__ sorted_keys, int chunk) {
  __shared__ uint32_t s_vis[kProjThreads / 32], s_dist[kProjThreads / 32];
  __shared__ EntryConst s_ent[kProjThreads / 32][kMaxChunk];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t n_nodes = min(frame[kRenderNodes], cap_nodes);
  const uint32_t n_chunks = (n_nodes + chunk - 1) / chunk;
  EntryConst* ent = s_ent[warp];
  uint32_t nvis = 0, ndist = 0;
  for (;;) {   // persistent warps take the chunks in turn from a frame counter
    uint32_t ch = 0;
    if (lane == 0) ch = atomicAdd(frame + kTileCounters + kProjChunkCounter, 1u);
    ch = __shfl_sync(0xffffffffu, ch, 0);
    if (ch >= n_chunks) break;
    const uint32_t p = ch * chunk + lane;
    const bool okp = lane < chunk && p < n_nodes;
    uint32_t ci = 0, node = 0, asset = 0xFFFFFFFFu;
    __syncwarp();   // the previous chunk's constants are consumed
    if (okp) {
      ci = order ? order[p] : p;   // a permutation of [0, n_nodes)
      const uint2 e = list[ci];
      node = e.y;
      const InstFrame& I = inst[e.x];
      asset = I.asset;
      const float4* mi = reinterpret_cast<const float4*>(I.m);
      EntryConst& E = ent[lane];
      E.m0 = mi[0];
      E.m1 = mi[1];
      E.m2 = mi[2];
      E.cam = *reinterpret_cast<const float4*>(I.cam_a);
      E.r0 = ref[2 * ci];
      E.r1 = ref[2 * ci + 1];
      if (sorted_keys && (p == 0 || sorted_keys[p] != sorted_keys[p - 1])) ++ndist;
    }
    __syncwarp();
    // runs: maximal stretches of the chunk with the same (asset, node)
    const uint32_t pa = __shfl_up_sync(0xffffffffu, asset, 1), pn = __shfl_up_sync(0xffffffffu, node, 1);
    const uint32_t valid = __ballot_sync(0xffffffffu, okp);
    uint32_t heads = __ballot_sync(0xffffffffu, okp && (lane == 0 || pa != asset || pn != node));
    while (heads) {
      const int a = __ffs(heads) - 1;
      heads &= heads - 1;
      const int b = heads ? __ffs(heads) - 1 : __popc(valid);
      const uint32_t ra = __shfl_sync(0xffffffffu, asset, a), rn = __shfl_sync(0xffffffffu, node, a);
      const AssetDev& A = assets[ra];
      const uint32_t cnt = A.count[rn];
      const float4 bc = A.bound[rn];
      const unsigned char* blk = A.attr + size_t(rn) * A.stride;
      const float* at = reinterpret_cast<const float*>(blk);    // geometry planes
      const unsigned char* col = blk + size_t(kGeoPlanes) * kSlots * 4;   // colour planes
      if (kFormats == 2 || (kFormats == 3 && A.half_color))
        nvis += project_run<__half>(lane, a, b, ci, cnt, ent, cam, bc, int(A.sh_coeffs), at,
                                    reinterpret_cast<const __half*>(col), rec, rect, keys, frame);
      else
        nvis += project_run<float>(lane, a, b, ci, cnt, ent, cam, bc, int(A.sh_coeffs), at,
                                   reinterpret_cast<const float*>(col), rec, rect, keys, frame);
    }
  }
  // one atomic per block for the visible count (and the distinct clusters)
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    nvis += __shfl_xor_sync(0xffffffffu, nvis, d);
    ndist += __shfl_xor_sync(0xffffffffu, ndist, d);
  }
  if (lane == 0) {
    s_vis[threadIdx.x >> 5] = nvis;
    s_dist[threadIdx.x >> 5] = ndist;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0, u = 0;
    for (int w = 0; w < kProjThreads / 32; ++w) {
      t += s_vis[w];
      u += s_dist[w];
    }
    if (t) atomicAdd(frame + kVisible, t);
    if (u) atomicAdd(frame + kRenderClusters, u);
  }
}

}  // namespace

int g_project_blocks_per_sm[4] = {2, 2, 2, 2};   // resident k_project blocks per SM, per colour-format set

cudaError_t project_set_attributes() {
  int n1 = 0, n2 = 0, n3 = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, k_project<1>, kProjThreads, 0);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, k_project<2>, kProjThreads, 0);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n3, k_project<3>, kProjThreads, 0);
  if (e != cudaSuccess) return e;
  g_project_blocks_per_sm[1] = n1;
  g_project_blocks_per_sm[2] = n2;
  g_project_blocks_per_sm[3] = n3;
  return cudaSuccess;
}

cudaError_t launch_noderef(const uint2* list, uint32_t cap, const InstFrame* inst, const AssetDev* assets,
                           const CamConst& cam, float4* ref, const uint32_t* frame, uint32_t* order_keys,
                           int key_shift, int sm_count, cudaStream_t st) {
  k_noderef<<<sm_count * 4, 256, 0, st>>>(list, cap, inst, assets, cam, ref, frame, order_keys, key_shift);
  return cudaGetLastError();
}

cudaError_t launch_project(const uint2* list, uint32_t cap_nodes, const InstFrame* inst, const AssetDev* assets,
                           const CamConst& cam, const float4* ref, float4* rec, uint2* rect, uint32_t* keys,
                           uint32_t* frame, const uint32_t* order, const uint32_t* sorted_keys,
                           int color_formats, int sm_count, cudaStream_t st) {
  // persistent grid: the resident blocks of the specialisation
  const int f = color_formats == 2 ? 2 : color_formats == 3 ? 3 : 1;
  const int grid = sm_count * std::max(g_project_blocks_per_sm[f], 1);
  const int chunk = order ? kProjChunkGrouped : kProjChunkList;
  if (color_formats == 2)
    k_project<2><<<grid, kProjThreads, 0, st>>>(list, cap_nodes, inst, assets, cam, ref, rec, rect, keys, frame, order, sorted_keys, chunk);
  else if (color_formats == 3)
    k_project<3><<<grid, kProjThreads, 0, st>>>(list, cap_nodes, inst, assets, cam, ref, rec, rect, keys, frame, order, sorted_keys, chunk);
  else
    k_project<1><<<grid, kProjThreads, 0, st>>>(list, cap_nodes, inst, assets, cam, ref, rec, rect, keys, frame, order, sorted_keys, chunk);
  return cudaGetLastError();
}

}  // namespace v3dg
