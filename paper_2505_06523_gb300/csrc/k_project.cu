// Projection of the selected Gaussians (Sec. 2.1; Sec. 5.1: EWA splatting without 2D dilation).
//
// k_noderef: one thread per render-list node computes, in FP64, the view-space position of the
//   node's mean centre and its pixel position, so that every Gaussian of the node can be placed
//   relative to it with small float32 offsets (the screen mean stays accurate to ~1e-7 of the
//   node's extent instead of 1 ulp of the whole view distance).
// k_project: one warp per render-list node (<= 64 Gaussians, 2 per lane), attribute-major loads
//   (each cluster's attributes are one contiguous block of planes of 64 floats, so every warp load
//   is one 128-byte line and a cluster's data is one region of memory).
//   Writes a 48-byte blend record, the pixel box and the float32 depth key per Gaussian;
//   culled slots get the key 0xFFFFFFFF so that the depth sort moves them behind all visible ones.
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
          const uint32_t* __restrict__ frame) {
  const uint32_t n = min(frame[kRenderNodes], cap);
  for (uint32_t ci = blockIdx.x * blockDim.x + threadIdx.x; ci < n; ci += gridDim.x * blockDim.x) {
    const uint2 e = list[ci];
    const InstFrame& I = inst[e.x];
    const float4 b = assets[I.asset].bound[e.y];
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

// Projects the (<= 64) Gaussians of render-list entry ci, two per lane; returns how many of this
// lane's Gaussians are visible.  TC is the colour storage type (float or __half): the colour
// pointer is typed and restrict-qualified so that all of a Gaussian's loads can be in flight at
// once.
template <typename TC>
__device__ __forceinline__ uint32_t project_node(int lane, uint32_t ci, uint32_t cnt, const InstFrame& I,
                                                 const CamConst& cam, const float4 bc, const float4 r0,
                                                 const float4 r1, int nsh, const float* __restrict__ at,
                                                 const TC* __restrict__ col, float4* __restrict__ rec,
                                                 uint2* __restrict__ rect, uint32_t* __restrict__ keys,
                                                 uint32_t* __restrict__ frame) {
  const bool comp = r1.w != 0.f;
  constexpr size_t st = kSlots;   // values between planes
  uint32_t nvis = 0;
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const uint32_t j = lane + 32 * h;
    const size_t slot = size_t(ci) * kSlots + j;
    if (j >= cnt) {
      keys[slot] = 0xFFFFFFFFu;
      continue;
    }
    const float mx = at[kX * st + j], my = at[kY * st + j], mz = at[kZ * st + j];
    const float op = to_f32(col[kOpacity * st + j]);
    // float32 depth key: ((M20 x + M21 y) + M22 z) + M23, every step rounded (no fusion)
    const float z32 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(I.m[8], mx), __fmul_rn(I.m[9], my)),
                                          __fmul_rn(I.m[10], mz)), I.m[11]);
    bool vis = (z32 >= cam.near_z) && (op >= kMinOpacity);
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
    float qw = at[kQw * st + j], qx = at[kQx * st + j], qy = at[kQy * st + j], qz = at[kQz * st + j];
    const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= qn; qx *= qn; qy *= qn; qz *= qn;
    const float R00 = 1.f - 2.f * (qy * qy + qz * qz), R01 = 2.f * (qx * qy - qw * qz), R02 = 2.f * (qx * qz + qw * qy);
    const float R10 = 2.f * (qx * qy + qw * qz), R11 = 1.f - 2.f * (qx * qx + qz * qz), R12 = 2.f * (qy * qz - qw * qx);
    const float R20 = 2.f * (qx * qz - qw * qy), R21 = 2.f * (qy * qz + qw * qx), R22 = 1.f - 2.f * (qx * qx + qy * qy);
    const float s0 = expf(at[kLs0 * st + j]), s1 = expf(at[kLs1 * st + j]), s2 = expf(at[kLs2 * st + j]);
    float Am[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float m0 = I.m[4 * r], m1 = I.m[4 * r + 1], m2 = I.m[4 * r + 2];
      Am[r][0] = fmaf(m0, R00, fmaf(m1, R10, m2 * R20)) * s0;
      Am[r][1] = fmaf(m0, R01, fmaf(m1, R11, m2 * R21)) * s1;
      Am[r][2] = fmaf(m0, R02, fmaf(m1, R12, m2 * R22)) * s2;
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
    const float kq = 2.f * logf(255.f * op);
    const float hx = sqrtf(fmaxf(kq * ca, 0.f)), hy = sqrtf(fmaxf(kq * cc, 0.f));
    const float u = r0.x + (r0.y + corr_u), v = r0.z + (r0.w + corr_v);
    float x0 = fmaxf(ceilf(u - hx - 0.5f), 0.f), x1 = fminf(floorf(u + hx - 0.5f), float(cam.width - 1));
    float y0 = fmaxf(ceilf(v - hy - 0.5f), 0.f), y1 = fminf(floorf(v + hy - 0.5f), float(cam.height - 1));
    vis = vis && (x0 <= x1) && (y0 <= y1) && isfinite(u) && isfinite(v);
    if (!vis) {
      keys[slot] = 0xFFFFFFFFu;
      continue;
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
        if (k < nsh) acc = fmaf(Y[k], to_f32(col[(kSh0 + 3 * k + ch) * st + j]), acc);
      rgb[ch] = fmaxf(acc + 0.5f, 0.f);
    }
    const uint32_t origin = uint32_t(tx0) | (uint32_t(ty0) << 16);
    float4* rp = rec + 3 * slot;
    rp[0] = make_float4(u_rel, v_rel, -0.5f * kLog2e * ia, -kLog2e * ib);
    rp[1] = make_float4(-0.5f * kLog2e * ic, log2f(op), rgb[0], rgb[1]);
    rp[2] = make_float4(rgb[2], __uint_as_float(origin), __uint_as_float(uint32_t(x0) | (uint32_t(x1) << 16)),
                        __uint_as_float(uint32_t(y0) | (uint32_t(y1) << 16)));
    rect[slot] = make_uint2(uint32_t(x0) | (uint32_t(x1) << 16), uint32_t(y0) | (uint32_t(y1) << 16));
    keys[slot] = __float_as_uint(z32);
    ++nvis;
  }
  return nvis;
}

// kFormats: bit 0 = float32 colour planes occur, bit 1 = float16 ones occur.
template <int kFormats>
__global__ void __launch_bounds__(kProjThreads)
k_project(const uint2* __restrict__ list, uint32_t cap_nodes, const InstFrame* __restrict__ inst,
          const AssetDev* __restrict__ assets, CamConst cam, const float4* __restrict__ ref,
          float4* __restrict__ rec, uint2* __restrict__ rect, uint32_t* __restrict__ keys,
          uint32_t* __restrict__ frame) {
  __shared__ uint32_t s_vis[kProjThreads / 32];
  const int lane = threadIdx.x & 31;
  const uint32_t n_nodes = min(frame[kRenderNodes], cap_nodes);
  const uint32_t nwarps = (gridDim.x * kProjThreads) >> 5;
  uint32_t nvis = 0;
  for (uint32_t ci = (blockIdx.x * kProjThreads + threadIdx.x) >> 5; ci < n_nodes; ci += nwarps) {
    const uint2 e = list[ci];
    const InstFrame& I = inst[e.x];
    const AssetDev& A = assets[I.asset];
    const uint32_t node = e.y;
    const uint32_t cnt = A.count[node];
    const float4 bc = A.bound[node];
    const float4 r0 = ref[2 * ci], r1 = ref[2 * ci + 1];
    const unsigned char* blk = A.attr + size_t(node) * A.stride;
    const float* at = reinterpret_cast<const float*>(blk);    // geometry planes
    const unsigned char* col = blk + size_t(kGeoPlanes) * kSlots * 4;   // colour planes
    if (kFormats == 2 || (kFormats == 3 && A.half_color))
      nvis += project_node<__half>(lane, ci, cnt, I, cam, bc, r0, r1, A.sh_coeffs, at,
                                   reinterpret_cast<const __half*>(col), rec, rect, keys, frame);
    else
      nvis += project_node<float>(lane, ci, cnt, I, cam, bc, r0, r1, A.sh_coeffs, at,
                                  reinterpret_cast<const float*>(col), rec, rect, keys, frame);
  }
  // one atomic per block for the visible count
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) nvis += __shfl_xor_sync(0xffffffffu, nvis, d);
  if (lane == 0) s_vis[threadIdx.x >> 5] = nvis;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kProjThreads / 32; ++w) t += s_vis[w];
    if (t) atomicAdd(frame + kVisible, t);
  }
}

}  // namespace

cudaError_t launch_noderef(const uint2* list, uint32_t cap, const InstFrame* inst, const AssetDev* assets,
                           const CamConst& cam, float4* ref, const uint32_t* frame, int sm_count, cudaStream_t st) {
  k_noderef<<<sm_count * 4, 256, 0, st>>>(list, cap, inst, assets, cam, ref, frame);
  return cudaGetLastError();
}

cudaError_t launch_project(const uint2* list, uint32_t cap_nodes, const InstFrame* inst, const AssetDev* assets,
                           const CamConst& cam, const float4* ref, float4* rec, uint2* rect, uint32_t* keys,
                           uint32_t* frame, int color_formats, int sm_count, cudaStream_t st) {
  const int grid = sm_count * 8;
  if (color_formats == 2)
    k_project<2><<<grid, kProjThreads, 0, st>>>(list, cap_nodes, inst, assets, cam, ref, rec, rect, keys, frame);
  else if (color_formats == 3)
    k_project<3><<<grid, kProjThreads, 0, st>>>(list, cap_nodes, inst, assets, cam, ref, rec, rect, keys, frame);
  else
    k_project<1><<<grid, kProjThreads, 0, st>>>(list, cap_nodes, inst, assets, cam, ref, rec, rect, keys, frame);
  return cudaGetLastError();
}

}  // namespace v3dg
