// Host side of the C ABI declared in include/v3dg.h.
//
// Owns the device state of one context: the uploaded bundles (Sec. 3, Fig. 2), the instance table
// (Sec. 4.2), the per-frame FP64 set-up (camera V and instances composed into M = W [s R | t])
// and the work buffers of the splatting stages, whose capacities grow when a frame overflows.
// The per-frame state lives in a Pipe: the plain API drives the context's main pipe, and the
// request server (v3dg_server_start / v3dg_submit / v3dg_poll) runs one more pipe per slot, each
// on its own stream and host thread, over the same device-resident assets.
// Host code is compiled with -ffp-contract=off: M is composed in a fixed operation order.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <set>
#include <unordered_set>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "v3dg.h"
#include "v3dg_internal.h"

using namespace v3dg;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct AssetHost {
  uint32_t n_gauss = 0, n_nodes = 0, sh_coeffs = 0, gpg = 0;
  bool half_color = false;
  std::vector<uint32_t> node_first;
  uint32_t levels = 0;     // largest node level + 1
  DevBuf own, par, bound, sigma, flags, cnt, attr;
  DevBuf child_off, child_list, sub_bound, sub_sigma;   // top-down selection
};

constexpr uint32_t kInitNodes = 1u << 14;
constexpr uint32_t kInitPairs = 1u << 22;
constexpr uint32_t kMaxNodes = 1u << 25;               // render-list clusters: at most 2^31 slots
constexpr uint32_t kMaxPairs = 0xFFFFFFFFu - 4096u;    // pair indices are 32-bit (a sort tile of headroom)
enum { kStageSelect = 0, kStageProject, kStageDepthSort, kStageBin, kStageTileSort, kStageRanges, kStageBlend, kStages };

}  // namespace

struct Server;

// Per-frame state of one pipeline: the instance table and camera set-up of its frames, its work
// buffers and their capacities, frame counters and the stream its work goes to.  The context's
// plain API drives the main pipe; each serving slot owns one more.
struct Pipe {
  v3dg_ctx* ctx = nullptr;
  std::string err;
  cudaStream_t stream = nullptr;
  bool ctx_alloc = true;   // device memory from the context's allocator (else cudaMalloc)
  cudaMemPool_t pool = nullptr;   // serving slots: stream-ordered allocations from the server's pool

  std::vector<uint32_t> inst_asset;
  std::vector<double> inst_rot, inst_trans, inst_scale;
  std::vector<uint32_t> frame_asset;   // asset of each instance frame of the current selection

  bool selected = false, rendered = false;
  v3dg_camera cam{};
  float tau_px = 0.f;
  CamConst cc{};
  uint32_t n_inst_frame = 0;   // instance frames of the selection: n_views * instances
  uint32_t n_views = 1;        // cameras of the current frame (same intrinsics and image size)
  int color_formats = 1;       // colour storage formats of the current instances' assets (bit 0 FP32, bit 1 FP16)
  uint32_t distinct_assets = 0;   // assets drawn by the current instance frames
  int node_blocks = 0;

  DevBuf d_inst;
  InstFrame* h_inst = nullptr;
  size_t h_inst_cap = 0;
  cudaEvent_t ev_inst = nullptr;
  DevBuf d_frame, d_cutframe, d_misc;
  uint32_t* h_frame = nullptr;   // pinned copy of the frame words, written at the end of each frame
  uint32_t* h_tmp = nullptr;     // pinned scratch: [0, 48) frame words of read-backs, [48, 52) blend work

  uint32_t cap_nodes = 0, cap_slots = 0, cap_pairs = 0, status_words = 0, cap_cut = 0;
  DevBuf d_list, d_ref, d_keys0, d_keys1, d_vals0, d_vals1, d_rec, d_rect;
  DevBuf d_pk0, d_pk1, d_pv0, d_pv1, d_ranges, d_status, d_hist, d_cut;
  DevBuf d_img, d_timg, d_sort_k, d_sort_v, d_order;
  DevBuf d_front0, d_front1, d_tdcount, d_bitmap;   // top-down selection
  bool depth_in1 = false, tiles_in1 = false;
  uint32_t epoch = 1;
  cudaEvent_t ev[kStages + 1] = {};
  // CUDA-graph frames (V3DG_OPT_GRAPHS): the selection is enqueued with the render, and both are
  // captured once per configuration (gkey) on cap_stream, then replayed on `stream`
  bool select_pending = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<uint64_t> gkey;
  uint64_t glaunches = 0;   // kernel launches in the captured graph
};

struct v3dg_ctx {
  int device = 0;
  int sm_count = 0;
  v3dg_allocator alloc{};
  bool has_alloc = false;
  std::vector<AssetHost> assets;
  DevBuf d_assets;
  std::atomic<uint64_t> launches{0};
  bool sync_check = true, stage_timing = false, count_work = false;
  uint32_t split_pairs = 0xFFFFFFFFu;   // long-tile split threshold (none by default)
  bool attr_fp16 = false;   // store opacity and SH of the next loaded assets as float16
  int topdown = 2;          // 0 flat, 1 level by level from the roots (same cut), 2 top-down for large scenes
  int blend_batch = 512;    // records staged per blend batch: 128, 256 or 512
  int blend_mode = 0;       // 0: two-phase blend; 1: bulk-copy staging, warps composite row pairs
  int serve_merge = 1;      // server: most queued requests of one image geometry rendered together
  int project_order = 2;    // projection by cluster: 0 never, 1 always, 2 when instances repeat assets
  uint64_t total_nodes = 0; // nodes of all loaded assets (global cluster ids are below this)
  bool graphs = false;      // capture each frame's launches once and replay them as a CUDA graph
  Pipe main;
  Server* server = nullptr;
};

namespace {

v3dg_status fail(Pipe* c, v3dg_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CU(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(c, V3DG_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

#define ST(call)                                                                                   \
  do {                                                                                             \
    v3dg_status s_ = (call);                                                                       \
    if (s_ != V3DG_OK) return s_;                                                                  \
  } while (0)

void dfree(Pipe* c, DevBuf& b) {
  if (b.p) {
    if (c->pool)
      cudaFreeAsync(b.p, c->stream);   // back to the server's pool, in stream order
    else if (c->ctx->has_alloc && c->ctx_alloc)
      c->ctx->alloc.free(b.p, c->ctx->alloc.user);
    else
      cudaFree(b.p);
  }
  b.p = nullptr;
  b.bytes = 0;
}

v3dg_status dalloc(Pipe* c, DevBuf& b, size_t bytes, bool zero = false) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (c->pool) {
    const cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, c->pool, c->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, V3DG_ENOMEM, "pool allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
  } else if (c->ctx->has_alloc && c->ctx_alloc) {
    p = c->ctx->alloc.alloc(bytes, c->ctx->alloc.user);
    if (!p) return fail(c, V3DG_ENOMEM, "allocator returned NULL for %zu bytes", bytes);
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, V3DG_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
  }
  dfree(c, b);
  b.p = p;
  b.bytes = bytes;
  if (zero) CU(cudaMemsetAsync(p, 0, bytes, c->stream));
  return V3DG_OK;
}

v3dg_status ensure(Pipe* c, DevBuf& b, size_t bytes, bool zero = false) {
  if (b.p && b.bytes >= bytes) return V3DG_OK;
  return dalloc(c, b, bytes, zero);
}

template <class T>
T* P(const DevBuf& b) {
  return static_cast<T*>(b.p);
}

uint32_t next_epoch(Pipe* c) {
  c->epoch = (c->epoch + 1) & 0x3FFFFFFFu;
  if (c->epoch == 0) c->epoch = 1;
  return c->epoch;
}

float round_up_f(double x) {
  float f = float(x);
  if (double(f) < x) f = std::nextafter(f, INFINITY);
  return f;
}

v3dg_status ensure_status(Pipe* c, uint64_t words) {
  if (words <= c->status_words && c->d_status.p) return V3DG_OK;
  if (words > 0xFFFFFFFFull) return fail(c, V3DG_EOVERFLOW, "status array too large");
  ST(dalloc(c, c->d_status, 8 * words, true));
  c->status_words = uint32_t(words);
  return V3DG_OK;
}

// Work buffers sized by the current capacities.
v3dg_status ensure_work(Pipe* c) {
  if (c->cap_nodes == 0) c->cap_nodes = kInitNodes;
  if (c->cap_pairs == 0) c->cap_pairs = kInitPairs;
  c->cap_slots = c->cap_nodes * uint32_t(kSlots);
  const size_t S = c->cap_slots, PP = c->cap_pairs;
  ST(ensure(c, c->d_list, sizeof(uint2) * c->cap_nodes));
  ST(ensure(c, c->d_ref, sizeof(float4) * 2 * c->cap_nodes));
  ST(ensure(c, c->d_keys0, 4 * S));
  ST(ensure(c, c->d_keys1, 4 * S));
  ST(ensure(c, c->d_vals0, 4 * S));
  ST(ensure(c, c->d_vals1, 4 * S));
  ST(ensure(c, c->d_rec, sizeof(float4) * 3 * S));
  ST(ensure(c, c->d_rect, sizeof(uint2) * S));
  ST(ensure(c, c->d_pk0, 4 * PP));
  ST(ensure(c, c->d_pk1, 4 * PP));
  ST(ensure(c, c->d_pv0, 4 * PP));
  ST(ensure(c, c->d_pv1, 4 * PP));
  const uint64_t sort_tiles = (std::max<uint64_t>(S, PP) + kSortTile - 1) / kSortTile;
  uint64_t words = sort_tiles * 256;
  words = std::max<uint64_t>(words, uint64_t(c->n_inst_frame) * uint64_t(std::max(c->node_blocks, 1)));
  words = std::max<uint64_t>(words, (uint64_t(S) + 1023) / 1024);
  ST(ensure_status(c, words));
  ST(ensure(c, c->d_hist, 2 * 4 * 256 * 4));  // counts + exclusive offsets of up to 4 passes
  return V3DG_OK;
}

SortScratch sort_scratch(Pipe* c, uint32_t* tile_counters) {
  SortScratch sc;
  sc.hist = P<uint32_t>(c->d_hist);
  sc.status = P<uint64_t>(c->d_status);
  sc.max_tiles = c->status_words / 256;
  sc.tile_counters = tile_counters;
  return sc;
}

void stage_event(Pipe* c, int i) {
  if (c->ctx->stage_timing) cudaEventRecord(c->ev[i], c->stream);
}

// ------------------------------------------------------------------ per-frame set-up (FP64, host)

v3dg_status check_camera(Pipe* c, const v3dg_camera* cam) {
  if (!cam) return fail(c, V3DG_EINVAL, "camera is NULL");
  if (cam->width <= 0 || cam->height <= 0 || cam->width > 65535 * 16 || cam->height > 65535 * 16)
    return fail(c, V3DG_EINVAL, "bad image size %d x %d", cam->width, cam->height);
  if (!(cam->fx > 0.f) || !(cam->fy > 0.f) || !std::isfinite(cam->fx) || !std::isfinite(cam->fy) ||
      !std::isfinite(cam->cx) || !std::isfinite(cam->cy))
    return fail(c, V3DG_EINVAL, "bad intrinsics");
  for (double v : cam->world_to_cam)
    if (!std::isfinite(v)) return fail(c, V3DG_EINVAL, "non-finite world_to_cam");
  return V3DG_OK;
}

// One view of a frame: its camera, tolerance and instances (host arrays, FP64).
struct ViewSpec {
  const v3dg_camera* cam = nullptr;
  float tau_px = 0.f;
  uint32_t n = 0;
  const uint32_t* asset = nullptr;
  const double* rot = nullptr;
  const double* trans = nullptr;
  const double* scale = nullptr;
};

// Per-frame set-up of n_views views that share image size, intrinsics and near plane; each has
// its own camera, tolerance and instances.  The instance frames are the views' instances one view
// after the other, each carrying M = W_v [s R | t], its view id and its tau_F.
v3dg_status setup_views(Pipe* c, const ViewSpec* views, uint32_t n_views) {
  if (!views || n_views == 0) return fail(c, V3DG_EINVAL, "no camera");
  uint64_t nf64 = 0;
  for (uint32_t v = 0; v < n_views; ++v) {
    ST(check_camera(c, views[v].cam));
    const v3dg_camera& a = *views[0].cam;
    const v3dg_camera& b = *views[v].cam;
    if (b.width != a.width || b.height != a.height || b.fx != a.fx || b.fy != a.fy || b.cx != a.cx || b.cy != a.cy ||
        b.near_z != a.near_z)
      return fail(c, V3DG_EINVAL, "camera %u differs from camera 0 in image size, intrinsics or near plane", v);
    if (!(views[v].tau_px >= 0.f) || !std::isfinite(views[v].tau_px))
      return fail(c, V3DG_EINVAL, "tau_px must be finite and >= 0");
    nf64 += views[v].n;
  }
  const v3dg_camera* cam = views[0].cam;
  if (c->ctx->assets.empty()) return fail(c, V3DG_ENOTFOUND, "no hierarchy loaded");
  const uint64_t tiles = uint64_t((cam->width + kTile - 1) / kTile) * uint64_t((cam->height + kTile - 1) / kTile);
  if (tiles * n_views > uint64_t(kMaxTiles))
    return fail(c, V3DG_EINVAL, "image too large (%llu tiles of 16x16 over %u views, at most %d)",
                (unsigned long long)(tiles * n_views), n_views, kMaxTiles);
  if (nf64 > 0xFFFFFFFull) return fail(c, V3DG_EINVAL, "too many instance views");
  const uint32_t nf = uint32_t(nf64);

  c->cam = *cam;
  if (!(c->cam.near_z > 0.f)) c->cam.near_z = 0.01f;
  c->tau_px = views[0].tau_px;
  CamConst& k = c->cc;
  k.fx = cam->fx; k.fy = cam->fy; k.cx = cam->cx; k.cy = cam->cy;
  k.near_z = c->cam.near_z;
  k.width = cam->width; k.height = cam->height;
  k.tiles_x = (cam->width + kTile - 1) / kTile;
  k.tiles_y = (cam->height + kTile - 1) / kTile;
  k.limx = 1.3f * (0.5f * float(cam->width) / cam->fx);
  k.limy = 1.3f * (0.5f * float(cam->height) / cam->fy);
  k.k_foot = M_PI * double(cam->fx) * double(cam->fy);
  k.k_foot32 = float(k.k_foot);
  const double two_ln255 = 2.0 * std::log(255.0);
  k.cull_kx = float(std::sqrt(two_ln255 * (1.0 + double(k.limx) * double(k.limx))) * 1.01);
  k.cull_ky = float(std::sqrt(two_ln255 * (1.0 + double(k.limy) * double(k.limy))) * 1.01);

  uint32_t max_nodes = 0;
  for (auto& a : c->ctx->assets) max_nodes = std::max(max_nodes, a.n_nodes);
  c->node_blocks = int((max_nodes + 2047) / 2048);   // k_select covers 2048 nodes per block
  c->n_inst_frame = nf;
  c->n_views = n_views;
  c->frame_asset.resize(nf);
  // the projection is specialised for the colour formats of the assets this frame draws
  c->color_formats = 0;
  std::vector<uint8_t> drawn(c->ctx->assets.size(), 0);
  for (uint32_t v = 0; v < n_views; ++v)
    for (uint32_t i = 0; i < views[v].n; ++i) {
      c->color_formats |= c->ctx->assets[views[v].asset[i]].half_color ? 2 : 1;
      drawn[views[v].asset[i]] = 1;
    }
  if (!c->color_formats) c->color_formats = 1;
  c->distinct_assets = 0;
  for (uint8_t d : drawn) c->distinct_assets += d;

  // the pinned staging buffer is reused: wait until the previous upload out of it has completed
  if (c->ev_inst) CU(cudaEventSynchronize(c->ev_inst));
  if (c->h_inst_cap < std::max<uint32_t>(nf, 1)) {
    if (c->h_inst) cudaFreeHost(c->h_inst);
    c->h_inst = nullptr;
    c->h_inst_cap = 0;
    CU(cudaMallocHost(&c->h_inst, sizeof(InstFrame) * std::max<uint32_t>(nf, 1)));
    c->h_inst_cap = std::max<uint32_t>(nf, 1);
  }
  ST(ensure(c, c->d_inst, sizeof(InstFrame) * std::max<uint32_t>(nf, 1)));

  uint32_t fi = 0;
  for (uint32_t v = 0; v < n_views; ++v) {
    const ViewSpec& vs = views[v];
    const double* W = vs.cam->world_to_cam;
    double C[3];  // camera centre -R_w^T t_w
    for (int j = 0; j < 3; ++j) C[j] = -((W[0 * 4 + j] * W[3] + W[1 * 4 + j] * W[7]) + W[2 * 4 + j] * W[11]);
    for (uint32_t i = 0; i < vs.n; ++i, ++fi) {
      InstFrame& f = c->h_inst[fi];
      std::memset(&f, 0, sizeof f);
      const double* R = &vs.rot[9 * size_t(i)];
      const double* t = &vs.trans[3 * size_t(i)];
      const double s = vs.scale[i];
      double A[9];
      for (int q = 0; q < 9; ++q) A[q] = s * R[q];
      for (int r = 0; r < 3; ++r) {
        for (int col = 0; col < 3; ++col)
          f.m64[4 * r + col] = (W[4 * r + 0] * A[0 * 3 + col] + W[4 * r + 1] * A[1 * 3 + col]) + W[4 * r + 2] * A[2 * 3 + col];
        f.m64[4 * r + 3] = ((W[4 * r + 0] * t[0] + W[4 * r + 1] * t[1]) + W[4 * r + 2] * t[2]) + W[4 * r + 3];
      }
      for (int q = 0; q < 12; ++q) f.m[q] = float(f.m64[q]);
      for (int j = 0; j < 3; ++j) {
        const double d = (R[0 * 3 + j] * (C[0] - t[0]) + R[1 * 3 + j] * (C[1] - t[1])) + R[2 * 3 + j] * (C[2] - t[2]);
        f.cam_a[j] = float(d / s);
      }
      f.s = float(s);
      f.s64 = s;
      const uint32_t a = vs.asset[i];
      f.asset = a;
      f.view = v;
      f.tau_f = float(double(c->ctx->assets[a].gpg) * double(vs.tau_px) * double(vs.tau_px));
      c->frame_asset[fi] = a;
    }
  }
  if (nf) CU(cudaMemcpyAsync(c->d_inst.p, c->h_inst, sizeof(InstFrame) * nf, cudaMemcpyHostToDevice, c->stream));
  if (!c->ev_inst) CU(cudaEventCreateWithFlags(&c->ev_inst, cudaEventDisableTiming));
  CU(cudaEventRecord(c->ev_inst, c->stream));
  return V3DG_OK;
}

// Per-frame set-up of n_views cameras (same intrinsics, image size and near plane) over the
// pipe's instances: instance frame v * n + i holds M = W_v [s R | t] of instance i.
v3dg_status setup_frame(Pipe* c, const v3dg_camera* cams, uint32_t n_views, float tau_px) {
  if (!cams || n_views == 0) return fail(c, V3DG_EINVAL, "no camera");
  std::vector<ViewSpec> vs(n_views);
  for (uint32_t v = 0; v < n_views; ++v) {
    vs[v].cam = cams + v;
    vs[v].tau_px = tau_px;
    vs[v].n = uint32_t(c->inst_asset.size());
    vs[v].asset = c->inst_asset.data();
    vs[v].rot = c->inst_rot.data();
    vs[v].trans = c->inst_trans.data();
    vs[v].scale = c->inst_scale.data();
  }
  return setup_views(c, vs.data(), n_views);
}

// Buffers of the top-down selection for the current instances: two frontiers that can each hold
// every node of every instance, the per-level counts and the selection bitmap.
v3dg_status topdown_buffers(Pipe* c, TopDown* td) {
  uint32_t max_nodes = 0, levels = 0;
  for (const AssetHost& a : c->ctx->assets) {
    max_nodes = std::max(max_nodes, a.n_nodes);
    levels = std::max(levels, a.levels);
  }
  const uint64_t front = std::max<uint64_t>(uint64_t(c->n_inst_frame) * max_nodes, 1);
  if (front > 0xFFFFFFFFull) return fail(c, V3DG_EINVAL, "too many instance nodes for the top-down selection");
  td->cap_front = uint32_t(front);
  td->wpi = (max_nodes + 31) / 32;
  td->steps = int(levels) + 1;   // the super-root step, then one per level
  ST(ensure(c, c->d_front0, sizeof(uint2) * front));
  ST(ensure(c, c->d_front1, sizeof(uint2) * front));
  ST(ensure(c, c->d_tdcount, sizeof(uint32_t) * size_t(td->steps + 1)));
  ST(ensure(c, c->d_bitmap, sizeof(uint32_t) * std::max<size_t>(size_t(c->n_inst_frame) * td->wpi, 1)));
  td->frontier[0] = P<uint2>(c->d_front0);
  td->frontier[1] = P<uint2>(c->d_front1);
  td->counts = P<uint32_t>(c->d_tdcount);
  td->bitmap = P<uint32_t>(c->d_bitmap);
  return V3DG_OK;
}

// Whether this frame's selection walks the trees top-down: always (option 1), never (0), or when
// the flat kernel would test more than kTopDownTests (instance, node) pairs (2, the default; on
// small scenes the walk's one launch per level costs more than it saves).
constexpr uint64_t kTopDownTests = 8u << 20;
bool use_topdown(const Pipe* c) {
  if (c->ctx->topdown != 2) return c->ctx->topdown == 1;
  uint64_t max_nodes = 0;
  for (const AssetHost& a : c->ctx->assets) max_nodes = std::max<uint64_t>(max_nodes, a.n_nodes);
  return uint64_t(c->n_inst_frame) * max_nodes > kTopDownTests;
}

// Selection into `out` (mode 0: the render list, mode 1: the cut), flat or top-down.
v3dg_status launch_selection(Pipe* c, int mode, uint2* out, uint32_t cap, uint32_t* frame) {
  if (!c->n_inst_frame) return V3DG_OK;
  if (use_topdown(c)) {
    TopDown td{};
    ST(topdown_buffers(c, &td));
    int nl = 0;
    CU(launch_select_topdown(P<InstFrame>(c->d_inst), int(c->n_inst_frame), P<AssetDev>(c->ctx->d_assets), c->cc, mode,
                             td, out, cap, frame, 0, P<uint64_t>(c->d_status), next_epoch(c), c->ctx->sm_count,
                             c->stream, &nl));
    c->ctx->launches += nl;
  } else {
    CU(launch_select(P<InstFrame>(c->d_inst), int(c->n_inst_frame), P<AssetDev>(c->ctx->d_assets), c->node_blocks, c->cc,
                     mode, out, cap, frame, 0, P<uint64_t>(c->d_status), next_epoch(c), c->stream));
    ++c->ctx->launches;
  }
  return V3DG_OK;
}

v3dg_status enqueue_select(Pipe* c) {
  ST(ensure_work(c));
  CU(cudaMemsetAsync(c->d_frame.p, 0, sizeof(uint32_t) * kFrameWords, c->stream));
  stage_event(c, kStageSelect);
  ST(launch_selection(c, 0, P<uint2>(c->d_list), c->cap_nodes, P<uint32_t>(c->d_frame)));
  return V3DG_OK;
}

// Whether the projection takes the render list grouped by cluster: never (option 0), always (1),
// or (2, the default) when the frame's instance frames outnumber the assets they draw at least
// twice over, so that clusters are drawn by several instances and their attribute reads can be
// shared through L2.
bool use_project_order(const Pipe* c) {
  if (c->ctx->total_nodes > 0xFFFFFFFFull || c->ctx->project_order == 0) return false;
  if (c->ctx->project_order == 1) return true;
  return c->n_inst_frame >= 2 * uint64_t(std::max<uint32_t>(c->distinct_assets, 1)) && c->n_inst_frame >= 4;
}

// Start of a render: zero the render stages' counters (select's words stay, so that a render
// list overflow still invalidates the frame) and count the slots the depth sort covers.
__global__ void k_render_reset(uint32_t* frame, uint32_t cap_nodes) {
  const int i = threadIdx.x;
  if (i == kVisible || i == kPairs || i == kPairsEff || i == kConicFp64 || i == kRenderClusters || i == kPairs64 ||
      i == kPairs64 + 1 ||
      (i > kTileCounters && i < kFrameWords))
    frame[i] = 0;
  if (i == kSlotCount) frame[kSlotCount] = min(frame[kRenderNodes], cap_nodes) * uint32_t(kSlots);
}

__global__ void k_set_word(uint32_t* p, uint32_t v) { *p = v; }

v3dg_status enqueue_render(Pipe* c, float* rgb, float* t_out) {
  const CamConst& k = c->cc;
  uint32_t* frame = P<uint32_t>(c->d_frame);
  const int sm = c->ctx->sm_count;
  stage_event(c, kStageProject);
  k_render_reset<<<1, kFrameWords, 0, c->stream>>>(frame, c->cap_nodes);
  CU(cudaGetLastError());
  // projection order: grouped by cluster (the render list's global cluster ids, sorted on at most
  // 24 bits, keeping the high ones) when several instances draw the same assets.  The keys and
  // the order use d_keys1 (4 x cap_nodes words of its 4 x 64 x cap_nodes), which the depth sort
  // only writes after the projection.
  int key_bits = 1, key_shift = 0;
  while ((uint64_t(1) << key_bits) < c->ctx->total_nodes) ++key_bits;
  if (key_bits > 24) key_shift = key_bits - 24;
  uint32_t* okeys = nullptr;
  const uint32_t *order = nullptr, *sorted_keys = nullptr;
  if (use_project_order(c)) okeys = P<uint32_t>(c->d_keys1);
  CU(launch_noderef(P<uint2>(c->d_list), c->cap_nodes, P<InstFrame>(c->d_inst), P<AssetDev>(c->ctx->d_assets), k,
                    P<float4>(c->d_ref), frame, okeys, key_shift, sm, c->stream));
  c->ctx->launches += 2;
  if (okeys) {
    const size_t cn = c->cap_nodes;
    bool oin1 = false;
    int nl = 0;
    CU(launch_sort(okeys, okeys + cn, okeys + 2 * cn, okeys + 3 * cn, frame + kRenderNodes, c->cap_nodes, 0,
                   key_bits - key_shift, true, sort_scratch(c, frame + kTileCounters + 11), frame + kTimeout, c->epoch,
                   sm, c->stream, &oin1, &nl));
    next_epoch(c);
    c->ctx->launches += nl;
    order = oin1 ? okeys + 3 * cn : okeys + cn;
    if (key_shift == 0) sorted_keys = oin1 ? okeys + 2 * cn : okeys;   // (exact cluster ids: counted)
  }
  CU(launch_project(P<uint2>(c->d_list), c->cap_nodes, P<InstFrame>(c->d_inst), P<AssetDev>(c->ctx->d_assets), k,
                    P<float4>(c->d_ref), P<float4>(c->d_rec), P<uint2>(c->d_rect), P<uint32_t>(c->d_keys0), frame,
                    order, sorted_keys, c->color_formats, sm, c->stream));
  c->ctx->launches += 1;

  stage_event(c, kStageDepthSort);
  bool in1 = false;
  int nl = 0;
  CU(launch_sort(P<uint32_t>(c->d_keys0), P<uint32_t>(c->d_vals0), P<uint32_t>(c->d_keys1), P<uint32_t>(c->d_vals1),
                 frame + kSlotCount, c->cap_slots, 0, 32, true, sort_scratch(c, frame + kTileCounters + 2),
                 frame + kTimeout, c->epoch, sm, c->stream, &in1, &nl));
  next_epoch(c);
  c->ctx->launches += nl;
  c->depth_in1 = in1;
  const uint32_t* dslots = in1 ? P<uint32_t>(c->d_vals1) : P<uint32_t>(c->d_vals0);

  stage_event(c, kStageBin);
  const int tiles_view = k.tiles_x * k.tiles_y;
  CU(launch_expand(dslots, P<uint2>(c->d_rect), c->cap_slots, c->cap_pairs, k.tiles_x, P<uint2>(c->d_list),
                   c->n_views > 1 ? P<InstFrame>(c->d_inst) : nullptr, uint32_t(tiles_view), P<uint32_t>(c->d_pk0),
                   P<uint32_t>(c->d_pv0), frame, 1, P<uint64_t>(c->d_status), next_epoch(c), sm, c->stream));
  c->ctx->launches += 2;

  stage_event(c, kStageTileSort);
  const int n_tiles = tiles_view * int(c->n_views);   // (view, tile) ids
  int tile_bits = 1;
  while ((1 << tile_bits) < n_tiles) ++tile_bits;
  bool tin1 = false;
  nl = 0;
  CU(launch_sort(P<uint32_t>(c->d_pk0), P<uint32_t>(c->d_pv0), P<uint32_t>(c->d_pk1), P<uint32_t>(c->d_pv1),
                 frame + kPairsEff, c->cap_pairs, 0, tile_bits, false, sort_scratch(c, frame + kTileCounters + 6),
                 frame + kTimeout, c->epoch, sm, c->stream, &tin1, &nl));
  next_epoch(c);
  c->ctx->launches += nl;
  c->tiles_in1 = tin1;
  const uint32_t* tk = tin1 ? P<uint32_t>(c->d_pk1) : P<uint32_t>(c->d_pk0);
  const uint32_t* tv = tin1 ? P<uint32_t>(c->d_pv1) : P<uint32_t>(c->d_pv0);

  stage_event(c, kStageRanges);
  ST(ensure(c, c->d_ranges, sizeof(uint2) * size_t(n_tiles)));
  ST(ensure(c, c->d_order, sizeof(uint32_t) * (4 * size_t(n_tiles) + 1)));
  CU(launch_ranges(tk, c->cap_pairs, frame, P<uint2>(c->d_ranges), n_tiles, sm, c->stream));
  c->ctx->launches += 1;

  stage_event(c, kStageBlend);
  // d_misc: [0..7] the standalone sort's words, [8..11] two 64-bit blend work counters
  unsigned long long* work = c->ctx->count_work ? reinterpret_cast<unsigned long long*>(P<uint32_t>(c->d_misc) + 8) : nullptr;
  if (work) CU(cudaMemsetAsync(work, 0, 2 * sizeof(unsigned long long), c->stream));
  // d_misc[12], [13]: sticky overflow / timeout flags of all frames since the last v3dg_frame_stats
  CU(launch_blend(P<uint2>(c->d_ranges), P<uint32_t>(c->d_order), frame + kTileCounters + 10, tk, tv, P<float4>(c->d_rec),
                  c->cap_slots, k, rgb, t_out, work, frame, P<uint32_t>(c->d_misc) + 12, c->ctx->split_pairs,
                  c->ctx->blend_batch, c->ctx->blend_mode, int(c->n_views), sm, c->stream));
  c->ctx->launches += 2;
  if (work)
    CU(cudaMemcpyAsync(c->h_tmp + kFrameWords, work, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
  stage_event(c, kStages);
  CU(cudaMemcpyAsync(c->h_frame, c->d_frame.p, sizeof(uint32_t) * kFrameWords, cudaMemcpyDeviceToHost, c->stream));
  c->rendered = true;
  return V3DG_OK;
}

// Runs the frame; with sync checking, waits and re-runs it with larger buffers on overflow.
// After an overflowed frame (h_frame holds its words): grow the capacities it ran out of, clear
// the sticky flags (the frame is re-run) and enqueue its selection again.
v3dg_status grow_and_reselect(Pipe* c) {
  const uint32_t* f = c->h_frame;
  bool grew = false;
  if (f[kRenderNodes] > c->cap_nodes) {
    if (f[kRenderNodes] > kMaxNodes)
      return fail(c, V3DG_EOVERFLOW, "render list of %u nodes exceeds the limit", f[kRenderNodes]);
    c->cap_nodes = uint32_t(std::min<uint64_t>(uint64_t(f[kRenderNodes]) * 5 / 4 + 1024, kMaxNodes));
    grew = true;
  }
  if (f[kPairs] >= c->cap_pairs || !grew) {
    if (f[kPairs] > kMaxPairs || c->cap_pairs >= kMaxPairs)
      return fail(c, V3DG_EOVERFLOW, "%u pairs exceed the limit of %u", f[kPairs], kMaxPairs);
    const uint64_t want = std::max<uint64_t>(uint64_t(f[kPairs]) * 5 / 4, uint64_t(c->cap_pairs) * 2);
    c->cap_pairs = uint32_t(std::min<uint64_t>(want, kMaxPairs));
  }
  CU(cudaMemsetAsync(P<uint32_t>(c->d_misc) + 12, 0, 2 * sizeof(uint32_t), c->stream));
  ST(enqueue_select(c));
  return V3DG_OK;
}

v3dg_status run_frame(Pipe* c, float* rgb, float* t_out, bool sync) {
  for (int attempt = 0; attempt < 8; ++attempt) {
    ST(enqueue_render(c, rgb, t_out));
    if (!sync) return V3DG_OK;
    CU(cudaStreamSynchronize(c->stream));
    const uint32_t* f = c->h_frame;
    if (f[kTimeout]) return fail(c, V3DG_ETIMEOUT, "a bounded device-side wait gave up; frame invalid");
    if (!f[kOverflow]) return V3DG_OK;
    ST(grow_and_reselect(c));
  }
  return fail(c, V3DG_EOVERFLOW, "frame still overflows after growing the buffers");
}

void drop_graph(Pipe* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->gkey.clear();
}

// What a captured frame depends on besides the contents of the instance frames (uploaded before
// each replay): sizes, capacities, buffer addresses, camera constants, options and outputs.
std::vector<uint64_t> graph_key(Pipe* c, float* rgb, float* t_out) {
  const v3dg_ctx* ctx = c->ctx;
  std::vector<uint64_t> k = {c->n_inst_frame, c->n_views, uint64_t(c->node_blocks), c->cap_nodes, c->cap_pairs,
                             c->cap_slots, c->status_words, uint64_t(uintptr_t(rgb)), uint64_t(uintptr_t(t_out)),
                             uint64_t(use_topdown(c)), uint64_t(use_project_order(c)), uint64_t(ctx->blend_batch),
                             uint64_t(ctx->blend_mode),
                             ctx->split_pairs,
                             uint64_t(ctx->count_work), uint64_t(c->color_formats), ctx->assets.size(),
                             uint64_t(uintptr_t(ctx->d_assets.p))};
  const DevBuf* bufs[] = {&c->d_inst, &c->d_frame, &c->d_misc, &c->d_list, &c->d_ref, &c->d_keys0, &c->d_keys1,
                          &c->d_vals0, &c->d_vals1, &c->d_rec, &c->d_rect, &c->d_pk0, &c->d_pk1, &c->d_pv0,
                          &c->d_pv1, &c->d_ranges, &c->d_status, &c->d_hist, &c->d_order, &c->d_front0,
                          &c->d_front1, &c->d_tdcount, &c->d_bitmap};
  for (const DevBuf* b : bufs) k.push_back(uint64_t(uintptr_t(b->p)));
  uint64_t w[sizeof(CamConst) / 8 + 1] = {};
  std::memcpy(w, &c->cc, sizeof(CamConst));
  for (uint64_t v : w) k.push_back(v);
  return k;
}

// One frame as a CUDA graph: the selection and every render launch, captured on first use of a
// configuration and replayed after that.  The chained-scan status words are cleared by the graph
// itself, because a replay reuses the epochs that were baked in at capture.
v3dg_status run_graph_frame(Pipe* c, float* rgb, float* t_out, bool sync) {
  ST(ensure_work(c));
  const int n_tiles = c->cc.tiles_x * c->cc.tiles_y * int(c->n_views);
  ST(ensure(c, c->d_ranges, sizeof(uint2) * size_t(n_tiles)));
  ST(ensure(c, c->d_order, sizeof(uint32_t) * (4 * size_t(n_tiles) + 1)));
  if (use_topdown(c)) {
    TopDown td{};
    ST(topdown_buffers(c, &td));
  }
  std::vector<uint64_t> key = graph_key(c, rgb, t_out);
  if (!c->gexec || key != c->gkey) {
    drop_graph(c);
    if (!c->cap_stream) CU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    CU(cudaStreamSynchronize(c->stream));   // the capture stream must not run ahead of earlier work
    cudaStream_t saved = c->stream;
    c->stream = c->cap_stream;
    const uint64_t launches0 = c->ctx->launches;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    v3dg_status st = V3DG_OK;
    if (e == cudaSuccess) {
      e = cudaMemsetAsync(c->d_status.p, 0, sizeof(uint64_t) * size_t(c->status_words), c->cap_stream);
      if (e == cudaSuccess) st = enqueue_select(c);
      if (e == cudaSuccess && st == V3DG_OK) st = enqueue_render(c, rgb, t_out);
      const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
      if (e == cudaSuccess) e = e2;
    }
    c->stream = saved;
    if (e == cudaSuccess && st == V3DG_OK) e = cudaGraphInstantiate(&c->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (st != V3DG_OK) return st;
    if (e != cudaSuccess) {
      c->gexec = nullptr;
      return fail(c, V3DG_ECUDA, "frame capture failed: %s", cudaGetErrorString(e));
    }
    c->gkey = std::move(key);
    c->glaunches = c->ctx->launches - launches0;
    c->ctx->launches -= c->glaunches;   // counted when the graph runs
  }
  CU(cudaGraphLaunch(c->gexec, c->stream));
  c->ctx->launches += c->glaunches;
  c->rendered = true;
  if (!sync) return V3DG_OK;
  CU(cudaStreamSynchronize(c->stream));
  if (c->h_frame[kTimeout]) return fail(c, V3DG_ETIMEOUT, "a bounded device-side wait gave up; frame invalid");
  if (!c->h_frame[kOverflow]) return V3DG_OK;
  ST(grow_and_reselect(c));   // grown buffers: the next frame captures a new graph
  return run_frame(c, rgb, t_out, true);
}

// v3dg_select's launches: enqueued now, or -- for graph frames -- with the render.
v3dg_status select_or_defer(Pipe* c) {
  if (c->ctx->graphs && !c->ctx->stage_timing) {
    c->select_pending = true;
    return V3DG_OK;
  }
  c->select_pending = false;
  return enqueue_select(c);
}

// The render of the current selection, as a graph or launch by launch.
v3dg_status render_frame(Pipe* c, float* rgb, float* t_out, bool sync) {
  const bool graph = c->ctx->graphs && !c->ctx->stage_timing;
  if (graph) {
    c->select_pending = false;
    return run_graph_frame(c, rgb, t_out, sync);
  }
  if (c->select_pending) {
    ST(enqueue_select(c));
    c->select_pending = false;
  }
  return run_frame(c, rgb, t_out, sync);
}

v3dg_status sync_frame(Pipe* c) {
  CU(cudaStreamSynchronize(c->stream));
  if (!c->rendered) CU(cudaMemcpy(c->h_frame, c->d_frame.p, sizeof(uint32_t) * kFrameWords, cudaMemcpyDeviceToHost));
  return V3DG_OK;
}

// The cut itself (mode 1), into d_cut; returns its size.
v3dg_status run_cut(Pipe* c, uint32_t* n_cut, uint32_t* n_gauss) {
  if (!c->selected) return fail(c, V3DG_ENOTFOUND, "no frame selected");
  if (c->cap_cut == 0) c->cap_cut = 1u << 16;
  for (int attempt = 0; attempt < 8; ++attempt) {
    ST(ensure(c, c->d_cut, sizeof(uint2) * size_t(c->cap_cut)));
    CU(cudaMemsetAsync(c->d_cutframe.p, 0, sizeof(uint32_t) * kFrameWords, c->stream));
    ST(launch_selection(c, 1, P<uint2>(c->d_cut), c->cap_cut, P<uint32_t>(c->d_cutframe)));
    CU(cudaMemcpyAsync(c->h_tmp, c->d_cutframe.p, sizeof(uint32_t) * kFrameWords, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (c->h_tmp[kTimeout]) return fail(c, V3DG_ETIMEOUT, "a bounded device-side wait gave up");
    if (!c->h_tmp[kOverflow]) {
      *n_cut = c->h_tmp[kCutNodes];
      *n_gauss = c->h_tmp[kCutGauss];
      return V3DG_OK;
    }
    c->cap_cut = std::max(c->cap_cut * 2, c->h_tmp[kCutNodes] + 1024);
  }
  return fail(c, V3DG_EOVERFLOW, "cut read-back overflow");
}

v3dg_status validate_desc(Pipe* c, const v3dg_hierarchy_desc* d) {
  if (!d) return fail(c, V3DG_EINVAL, "descriptor is NULL");
  if (d->n_gauss == 0 || d->n_nodes == 0) return fail(c, V3DG_EINVAL, "empty hierarchy");
  if (d->n_nodes > (1u << 24)) return fail(c, V3DG_EINVAL, "too many nodes (%u)", d->n_nodes);
  if (d->sh_degree > 3) return fail(c, V3DG_EINVAL, "sh_degree %u > 3", d->sh_degree);
  if (!d->means || !d->log_scales || !d->quats || !d->opacity || !d->sh || !d->node_first || !d->node_count ||
      !d->node_level || !d->node_parent || !d->own_sphere)
    return fail(c, V3DG_EINVAL, "NULL array in descriptor");
  if (d->gaussians_per_group == 0) return fail(c, V3DG_EINVAL, "gaussians_per_group must be >= 1");
  int roots = 0;
  std::vector<uint32_t> children(d->n_nodes, 0);
  for (uint32_t n = 0; n < d->n_nodes; ++n) {
    const uint32_t cnt = d->node_count[n];
    if (cnt < 1 || cnt > uint32_t(kSlots)) return fail(c, V3DG_EINVAL, "node %u has %u Gaussians (1..64)", n, cnt);
    if (uint64_t(d->node_first[n]) + cnt > d->n_gauss) return fail(c, V3DG_EINVAL, "node %u range out of bounds", n);
    const int32_t p = d->node_parent[n];
    if (p < 0) {
      ++roots;
    } else {
      if (uint32_t(p) >= d->n_nodes) return fail(c, V3DG_EINVAL, "node %u parent %d out of range", n, p);
      if (d->node_level[p] != d->node_level[n] + 1) return fail(c, V3DG_EINVAL, "node %u: parent not one level up", n);
      ++children[p];
    }
    const float* s = d->own_sphere + 4 * size_t(n);
    for (int q = 0; q < 4; ++q)
      if (!std::isfinite(s[q])) return fail(c, V3DG_EINVAL, "node %u sphere not finite", n);
    if (s[3] < 0.f) return fail(c, V3DG_EINVAL, "node %u sphere radius < 0", n);
  }
  if (roots != 1) return fail(c, V3DG_EINVAL, "%d roots (need exactly 1)", roots);
  for (uint32_t n = 0; n < d->n_nodes; ++n)
    if (d->node_level[n] > 0 && children[n] == 0) return fail(c, V3DG_EINVAL, "interior node %u has no children", n);
  return V3DG_OK;
}

// Pinned words, frame counters and stage events of a pipe; `stream` NULL: the legacy stream (main
// pipe) -- serving slots pass their own.
v3dg_status pipe_init(v3dg_ctx* ctx, Pipe* c, cudaStream_t stream) {
  c->ctx = ctx;
  c->stream = stream;
  if (cudaMallocHost(&c->h_frame, sizeof(uint32_t) * kFrameWords) != cudaSuccess) return V3DG_ECUDA;
  if (cudaMallocHost(&c->h_tmp, sizeof(uint32_t) * (kFrameWords + 16)) != cudaSuccess) return V3DG_ECUDA;
  std::memset(c->h_frame, 0, sizeof(uint32_t) * kFrameWords);
  ST(dalloc(c, c->d_frame, sizeof(uint32_t) * kFrameWords, true));
  ST(dalloc(c, c->d_cutframe, sizeof(uint32_t) * kFrameWords, true));
  ST(dalloc(c, c->d_misc, sizeof(uint32_t) * 64, true));
  for (auto& e : c->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return V3DG_ECUDA;
  if (c->stream) CU(cudaStreamSynchronize(c->stream));
  return V3DG_OK;
}

void pipe_free(Pipe* c) {
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graph(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->cap_stream = nullptr;
  DevBuf* bs[] = {&c->d_inst, &c->d_frame, &c->d_cutframe, &c->d_misc, &c->d_list, &c->d_ref, &c->d_keys0,
                  &c->d_keys1, &c->d_vals0, &c->d_vals1, &c->d_rec, &c->d_rect, &c->d_pk0, &c->d_pk1,
                  &c->d_pv0, &c->d_pv1, &c->d_ranges, &c->d_status, &c->d_hist, &c->d_cut, &c->d_img,
                  &c->d_timg, &c->d_sort_k, &c->d_sort_v, &c->d_order, &c->d_front0, &c->d_front1,
                  &c->d_tdcount, &c->d_bitmap};
  for (DevBuf* b : bs) dfree(c, *b);
  if (c->h_inst) cudaFreeHost(c->h_inst);
  if (c->h_frame) cudaFreeHost(c->h_frame);
  if (c->h_tmp) cudaFreeHost(c->h_tmp);
  if (c->ev_inst) cudaEventDestroy(c->ev_inst);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  c->h_inst = nullptr;
  c->h_frame = c->h_tmp = nullptr;
  c->ev_inst = nullptr;
  for (auto& e : c->ev) e = nullptr;
}

// The frame buffers a pipe holds (they grow with the largest frame it has rendered).
DevBuf* const* frame_buffers(Pipe* c, size_t* n) {
  static thread_local DevBuf* bs[24];
  DevBuf* list[] = {&c->d_list, &c->d_ref, &c->d_keys0, &c->d_keys1, &c->d_vals0, &c->d_vals1, &c->d_rec,
                    &c->d_rect, &c->d_pk0, &c->d_pk1, &c->d_pv0, &c->d_pv1, &c->d_ranges, &c->d_status,
                    &c->d_cut, &c->d_img, &c->d_timg, &c->d_sort_k, &c->d_sort_v, &c->d_order, &c->d_front0,
                    &c->d_front1, &c->d_bitmap};
  *n = sizeof(list) / sizeof(list[0]);
  for (size_t i = 0; i < *n; ++i) bs[i] = list[i];
  return bs;
}

uint64_t pipe_bytes(Pipe* c) {
  size_t n = 0;
  DevBuf* const* bs = frame_buffers(c, &n);
  uint64_t t = 0;
  for (size_t i = 0; i < n; ++i) t += bs[i]->bytes;
  return t;
}

// Releases the frame buffers (after the pipe's stream has finished with them); capacities start
// over and grow again on demand.  A captured frame graph refers to them, so it is dropped.
void pipe_trim(Pipe* c) {
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graph(c);
  size_t n = 0;
  DevBuf* const* bs = frame_buffers(c, &n);
  for (size_t i = 0; i < n; ++i) dfree(c, *bs[i]);
  c->cap_nodes = c->cap_pairs = c->cap_slots = c->status_words = c->cap_cut = 0;
  c->selected = c->rendered = false;
}

// ------------------------------------------------------------------ serving

// One queued request: a copy of its scene and camera, where its image goes, and its admission
// estimate of device memory.
struct Request {
  uint64_t ticket = 0;
  std::vector<uint32_t> asset;
  std::vector<double> rot, trans, scale;
  v3dg_camera cam{};
  float tau_px = 0.f;
  float* rgb = nullptr;
  float* t = nullptr;
  bool out_device = false;
  uint64_t est_bytes = 0;
  double t_submit = 0.0;
  bool heavy = false;   // estimated above its share of the budget: never beside another heavy one
};

struct Finished {
  v3dg_status status = V3DG_OK;
  double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
  uint64_t visible = 0, pairs = 0;
  uint32_t batch_views = 1;
};

}  // namespace

// Continuous batching: each slot is a pipe with its own streams and host thread.  Requests wait in
// arrival order; a slot takes the next one as soon as it is free and the device-memory estimates
// of the requests in flight plus this one fit the budget (one request is always admitted), so
// requests that arrive while others run start at once and their kernels overlap on the GPU.  A
// request that starts while no other one is on the GPU runs on its slot's high-priority stream,
// the others on the low-priority one: a frame that has the GPU keeps it (its latency stays that of
// a frame alone), and the frames admitted beside it fill the SMs it leaves idle.  A request whose
// estimate is at most a quarter of every running one's also takes the high-priority stream, so a
// small frame does not wait behind a large one.
struct Server {
  v3dg_ctx* ctx = nullptr;
  uint64_t budget = 0;
  size_t merge = 1;   // most requests rendered together as the views of one frame
  cudaMemPool_t pool = nullptr;   // the slots' frame buffers: freed memory is reused by any slot
  uint64_t slot_keep = ~uint64_t(0);   // a slot holding more frame-buffer bytes than this releases them
  std::vector<std::unique_ptr<Pipe>> slots;
  std::vector<cudaStream_t> hi, lo;   // per slot: high- and low-priority streams
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::unordered_map<uint64_t, Finished> finished;
  std::unordered_set<uint64_t> pending;   // issued and not yet reported by v3dg_poll
  uint64_t next_ticket = 1, in_flight = 0, active = 0, waiting_alone = 0, heavy_active = 0;
  std::multiset<uint64_t> active_est;   // memory estimates (a proxy of the work) of the frames on the GPU
  bool alone_busy = false;   // a slot renders requests alone after running out of device memory
  bool stop = false;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Admission estimate of a request's device memory: image and per-pixel buffers plus a share per
// instance for its cut, records and pairs.
// Estimated frame size of a request, for admission and for sizing its buffers before the first
// frame (so that it rarely overflows and re-runs): about 1,000 render-list clusters per instance of
// a 1M-leaf crowd at tau 1 px (1.0M for the 1000-instance crowd at 1920x1080), growing with
// sqrt(1 / tau) (a finer cut) and 25% headroom; pairs 2.25 per visible slot at 1920x1080, growing
// with the square root of the pixel count (Gaussians span more tiles).  Bytes: per slot the depth
// keys and values, record and box (72 B), per pair keys and values (16 B), per pixel 64 B.
struct FrameEstimate {
  uint64_t nodes, pairs, bytes;
};

FrameEstimate estimate_frame(uint32_t n_inst, const v3dg_camera& cam, float tau_px) {
  const double px = double(cam.width) * double(cam.height);
  const double nodes = 1250.0 * double(n_inst) * std::sqrt(1.0 / std::max(double(tau_px), 0.25));
  const double pairs = nodes * 64.0 * 2.25 * std::sqrt(px / (1920.0 * 1080.0));
  FrameEstimate e;
  e.nodes = uint64_t(nodes);
  e.pairs = uint64_t(pairs);
  e.bytes = uint64_t(nodes * 64.0 * 72.0 + pairs * 16.0 + px * 64.0);
  return e;
}

uint64_t request_bytes(uint32_t n_inst, const v3dg_camera& cam, float tau_px) {
  return estimate_frame(n_inst, cam, tau_px).bytes;
}

constexpr uint64_t kMergePixels = 3840ull * 2160ull;   // pixels of a merged frame (all its views)
constexpr uint64_t kMergeFrames = 8192;                // instance frames of a merged frame

// Whether two requests can share one launch per stage: the same image size, intrinsics and near
// plane (each keeps its own camera pose, scene and tolerance).
bool same_geometry(const v3dg_camera& a, const v3dg_camera& b) {
  return a.width == b.width && a.height == b.height && a.fx == b.fx && a.fy == b.fy && a.cx == b.cx &&
         a.cy == b.cy && a.near_z == b.near_z;
}

// Renders the requests as the views of one frame (each view its own instances, camera and tau;
// every stage one launch for all of them) and writes each view's image to its request's output.
// Every view's image is the one its request gives alone, bit for bit.
v3dg_status run_requests(Pipe* c, std::vector<Request>& rqs, Finished* f) {
  const uint32_t nv = uint32_t(rqs.size());
  std::vector<ViewSpec> vs(nv);
  for (uint32_t v = 0; v < nv; ++v) {
    Request& rq = rqs[v];
    vs[v].cam = &rq.cam;
    vs[v].tau_px = rq.tau_px;
    vs[v].n = uint32_t(rq.asset.size());
    vs[v].asset = rq.asset.data();
    vs[v].rot = rq.rot.data();
    vs[v].trans = rq.trans.data();
    vs[v].scale = rq.scale.data();
  }
  ST(setup_views(c, vs.data(), nv));
  // buffers sized from the requests' estimates before the first frame (they still grow on overflow)
  uint64_t want_nodes = 0, want_pairs = 0;
  for (const Request& rq : rqs) {
    const FrameEstimate e = estimate_frame(uint32_t(rq.asset.size()), rq.cam, rq.tau_px);
    want_nodes += e.nodes;
    want_pairs += e.pairs;
  }
  c->cap_nodes = uint32_t(std::max<uint64_t>(c->cap_nodes, std::min<uint64_t>(want_nodes, kMaxNodes)));
  c->cap_pairs = uint32_t(std::max<uint64_t>(c->cap_pairs, std::min<uint64_t>(want_pairs, kMaxPairs)));
  ST(enqueue_select(c));
  c->selected = true;
  c->rendered = false;
  const v3dg_camera& cam = rqs[0].cam;
  const size_t px = size_t(cam.width) * size_t(cam.height);
  bool any_t = false;
  for (const Request& rq : rqs) any_t |= rq.t != nullptr;
  float* rgb = nullptr;
  float* t = nullptr;
  if (nv == 1 && rqs[0].out_device) {   // one device request renders in place
    rgb = rqs[0].rgb;
    t = rqs[0].t;
  } else {
    ST(ensure(c, c->d_img, sizeof(float) * 3 * px * nv));
    if (any_t) ST(ensure(c, c->d_timg, sizeof(float) * px * nv));
    rgb = P<float>(c->d_img);
    t = any_t ? P<float>(c->d_timg) : nullptr;
  }
  ST(run_frame(c, rgb, t, true));
  if (!(nv == 1 && rqs[0].out_device)) {
    for (uint32_t v = 0; v < nv; ++v) {
      const Request& rq = rqs[v];
      const cudaMemcpyKind kind = rq.out_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
      CU(cudaMemcpyAsync(rq.rgb, P<float>(c->d_img) + 3 * px * v, sizeof(float) * 3 * px, kind, c->stream));
      if (rq.t) CU(cudaMemcpyAsync(rq.t, P<float>(c->d_timg) + px * v, sizeof(float) * px, kind, c->stream));
    }
  }
  CU(cudaStreamSynchronize(c->stream));
  f->visible = c->h_frame[kVisible];
  f->pairs = c->h_frame[kPairs];
  f->batch_views = nv;
  return V3DG_OK;
}

// A slot takes the request at the head of the queue and, if more are waiting, up to merge - 1
// later ones with the same image geometry whose device-memory estimates still fit the budget;
// they run as the views of one frame.
void slot_main(Server* sv, Pipe* p, size_t slot) {
  cudaSetDevice(sv->ctx->device);
  for (;;) {
    std::vector<Request> rqs;
    uint64_t est = 0;
    bool heavy = false;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_work.wait(lk, [&] {
        if (sv->queue.empty()) return sv->stop;
        if (sv->waiting_alone || sv->alone_busy) return false;   // a slot waits for or has its turn alone
        const Request& next = sv->queue.front();
        if (sv->active == 0) return true;
        if (next.heavy && sv->heavy_active) return false;   // large frames saturate the GPU on their own
        // beside frames on the GPU, start another only under a backlog (two or more waiting):
        // the stages run on persistent grids that hold every SM until they finish, so frames
        // that share the GPU take turns kernel by kernel, and a frame started beside others
        // finishes later than it would queued, unless requests pile up
        if (sv->queue.size() < 2) return false;
        return sv->in_flight + next.est_bytes <= sv->budget;
      });
      if (sv->queue.empty()) return;   // stopping and nothing left
      rqs.push_back(std::move(sv->queue.front()));
      sv->queue.pop_front();
      est = rqs[0].est_bytes;
      // merge only when requests pile up (more waiting than slots): below that, every request
      // gets a slot of its own and merged frames would only lengthen latencies
      const bool backlog = sv->queue.size() >= sv->slots.size();
      const uint64_t tiles = uint64_t((rqs[0].cam.width + kTile - 1) / kTile) * uint64_t((rqs[0].cam.height + kTile - 1) / kTile);
      const uint64_t px = uint64_t(rqs[0].cam.width) * uint64_t(rqs[0].cam.height);
      uint64_t frames = rqs[0].asset.size();
      // a merged frame stays within about one 4K frame of pixels and 8192 instance frames, so that
      // its pairs and buffers stay within what one large request needs
      for (auto it = sv->queue.begin(); backlog && it != sv->queue.end() && rqs.size() < sv->merge;) {
        const bool fit = same_geometry(it->cam, rqs[0].cam) && !it->heavy && !rqs[0].heavy &&
                         sv->in_flight + est + it->est_bytes <= sv->budget &&
                         tiles * (rqs.size() + 1) <= uint64_t(kMaxTiles) && px * (rqs.size() + 1) <= kMergePixels &&
                         frames + it->asset.size() <= kMergeFrames;
        if (fit) {
          est += it->est_bytes;
          frames += it->asset.size();
          rqs.push_back(std::move(*it));
          it = sv->queue.erase(it);
        } else {
          ++it;
        }
      }
      sv->in_flight += est;
      for (const Request& rq : rqs) heavy |= rq.heavy;
      if (heavy) ++sv->heavy_active;
      // high priority for a frame that starts alone, or that is far smaller than every frame on
      // the GPU (it then shares the SMs with them instead of queueing behind them)
      const bool small = !sv->active_est.empty() && est * 4 <= *sv->active_est.begin();
      p->stream = sv->active == 0 || small ? sv->hi[slot] : sv->lo[slot];   // (this slot's previous frame has completed)
      ++sv->active;
      sv->active_est.insert(est);
    }
    Finished f;
    bool alone = false;
    f.t_start = sv->now_ms();
    f.status = run_requests(p, rqs, &f);
    if (f.status == V3DG_ENOMEM || (f.status == V3DG_EOVERFLOW && rqs.size() > 1)) {
      // out of device memory beside the other frames in flight (or a merged frame beyond the
      // buffer limits): release this slot's buffers, wait until no other request is on the GPU,
      // and render the requests again one at a time
      pipe_trim(p);
      cudaGetLastError();
      {   // every slot that holds requests is waiting, and none runs alone: take the turn
        std::unique_lock<std::mutex> lk(sv->mu);
        ++sv->waiting_alone;
        sv->cv_done.wait(lk, [&] { return !sv->alone_busy && sv->active == sv->waiting_alone; });
        --sv->waiting_alone;
        sv->alone_busy = true;
        alone = true;
      }
      f.status = V3DG_OK;
      for (size_t r = 0; r < rqs.size() && f.status == V3DG_OK; ++r) {
        std::vector<Request> one(1);
        one[0] = std::move(rqs[r]);
        f.status = run_requests(p, one, &f);
        rqs[r] = std::move(one[0]);
      }
      f.batch_views = uint32_t(rqs.size());
    }
    if (f.status != V3DG_OK || pipe_bytes(p) > sv->slot_keep) pipe_trim(p);
    f.t_done = sv->now_ms();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->in_flight -= est;
      --sv->active;
      sv->active_est.erase(sv->active_est.find(est));
      if (heavy) --sv->heavy_active;
      if (alone) sv->alone_busy = false;
      for (const Request& rq : rqs) {
        Finished g = f;
        g.t_submit = rq.t_submit;
        sv->finished[rq.ticket] = g;
      }
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
}

void server_stop(v3dg_ctx* ctx) {
  Server* sv = ctx->server;
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->threads) t.join();
  for (auto& p : sv->slots) pipe_free(p.get());
  for (cudaStream_t st : sv->hi)
    if (st) cudaStreamSynchronize(st);
  for (cudaStream_t st : sv->lo)
    if (st) cudaStreamSynchronize(st);
  if (sv->pool) cudaMemPoolDestroy(sv->pool);
  for (cudaStream_t st : sv->hi)
    if (st) cudaStreamDestroy(st);
  for (cudaStream_t st : sv->lo)
    if (st) cudaStreamDestroy(st);
  delete sv;
  ctx->server = nullptr;
}

}  // namespace

// ====================================================================== public ABI

extern "C" {

v3dg_status v3dg_create(int device, const v3dg_allocator* alloc, v3dg_ctx** out) {
  if (!out) return V3DG_EINVAL;
  *out = nullptr;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || n_dev == 0) {
    cudaGetLastError();
    return V3DG_ECUDA;
  }
  if (device < 0 || device >= n_dev) return V3DG_EINVAL;
  if (alloc && (!alloc->alloc || !alloc->free)) return V3DG_EINVAL;
  v3dg_ctx* ctx = new (std::nothrow) v3dg_ctx;
  if (!ctx) return V3DG_ENOMEM;
  ctx->device = device;
  if (alloc) {
    ctx->alloc = *alloc;
    ctx->has_alloc = true;
  }
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      sort_set_attributes() != cudaSuccess || blend_set_attributes() != cudaSuccess ||
      project_set_attributes() != cudaSuccess) {
    delete ctx;
    return V3DG_ECUDA;
  }
  const v3dg_status st = pipe_init(ctx, &ctx->main, nullptr);
  if (st != V3DG_OK) {
    v3dg_destroy(ctx);
    return st;
  }
  *out = ctx;
  return V3DG_OK;
}

void v3dg_destroy(v3dg_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  server_stop(ctx);
  Pipe* c = &ctx->main;
  if (c->stream) cudaStreamSynchronize(c->stream);
  cudaDeviceSynchronize();
  for (auto& a : ctx->assets) {
    DevBuf* bs[] = {&a.own, &a.par, &a.bound, &a.sigma, &a.flags, &a.cnt, &a.attr, &a.child_off, &a.child_list,
                    &a.sub_bound, &a.sub_sigma};
    for (DevBuf* b : bs) dfree(c, *b);
  }
  dfree(c, ctx->d_assets);
  pipe_free(c);
  delete ctx;
}

const char* v3dg_last_error(const v3dg_ctx* ctx) { return ctx ? ctx->main.err.c_str() : "NULL context"; }

v3dg_status v3dg_set_stream(v3dg_ctx* ctx, void* stream) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  c->stream = static_cast<cudaStream_t>(stream);
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_set_option(v3dg_ctx* ctx, int option, int64_t value) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  if (ctx->server) return fail(c, V3DG_EBUSY, "options cannot change while a server runs");
  switch (option) {
    case V3DG_OPT_SYNC_CHECK: ctx->sync_check = value != 0; break;
    case V3DG_OPT_STAGE_TIMING: ctx->stage_timing = value != 0; break;
    case V3DG_OPT_COUNT_WORK: ctx->count_work = value != 0; break;
    case V3DG_OPT_ATTR_FP16: ctx->attr_fp16 = value != 0; break;
    case V3DG_OPT_SELECT_TOPDOWN:
      if (value < 0 || value > 2) return fail(c, V3DG_EINVAL, "top-down selection: 0, 1 or 2");
      ctx->topdown = int(value);
      break;
    case V3DG_OPT_GRAPHS: ctx->graphs = value != 0; break;
    case V3DG_OPT_BLEND_BATCH:
      if (value != 128 && value != 256 && value != 512) return fail(c, V3DG_EINVAL, "blend batch must be 128, 256 or 512");
      ctx->blend_batch = int(value);
      break;
    case V3DG_OPT_SERVE_MERGE:
      if (value < 1 || value > 64) return fail(c, V3DG_EINVAL, "requests per launch must be in [1, 64]");
      ctx->serve_merge = int(value);
      break;
    case V3DG_OPT_PROJECT_ORDER:
      if (value < 0 || value > 2) return fail(c, V3DG_EINVAL, "projection order must be 0, 1 or 2");
      ctx->project_order = int(value);
      break;
    case V3DG_OPT_BLEND_MODE:
      if (value != 0 && value != 1) return fail(c, V3DG_EINVAL, "blend mode must be 0 or 1");
      ctx->blend_mode = int(value);
      break;
    case V3DG_OPT_SPLIT_PAIRS:
      if (value < 1 || value > 0xFFFFFFFFll) return fail(c, V3DG_EINVAL, "split threshold out of range");
      ctx->split_pairs = uint32_t(value);
      break;
    case V3DG_OPT_CAP_NODES:
      if (value < 64 || value > int64_t(kMaxNodes)) return fail(c, V3DG_EINVAL, "node capacity out of range");
      c->cap_nodes = uint32_t(value);
      break;
    case V3DG_OPT_CAP_PAIRS:
      if (value < 4096 || value > int64_t(kMaxPairs)) return fail(c, V3DG_EINVAL, "pair capacity out of range");
      c->cap_pairs = uint32_t(value);
      break;
    default: return fail(c, V3DG_EINVAL, "unknown option %d", option);
  }
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_load_hierarchy(v3dg_ctx* ctx, const v3dg_hierarchy_desc* d, uint32_t* asset_id) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  if (ctx->server) return fail(c, V3DG_EBUSY, "assets cannot be loaded while a server runs");
  ST(validate_desc(c, d));
  CU(cudaSetDevice(ctx->device));
  const uint32_t nn = d->n_nodes;
  const uint32_t coeffs = (d->sh_degree + 1) * (d->sh_degree + 1);
  const bool half = ctx->attr_fp16;
  const size_t block = cluster_block_bytes(int(coeffs), half);   // bytes per cluster block
  std::vector<float4> own(nn), par(nn), bound(nn);
  std::vector<float> sigma(nn);
  std::vector<uint8_t> flags(nn), cnt(nn);
  std::vector<unsigned char> attr(size_t(nn) * block, 0);
  for (uint32_t n = 0; n < nn; ++n) {
    const float* s = d->own_sphere + 4 * size_t(n);
    own[n] = make_float4(s[0], s[1], s[2], s[3]);
  }
  for (uint32_t n = 0; n < nn; ++n) {
    const int32_t p = d->node_parent[n];
    par[n] = own[p < 0 ? n : uint32_t(p)];
    flags[n] = uint8_t((d->node_level[n] == 0 ? kLeaf : 0) | (p < 0 ? kRoot : 0));
    const uint32_t f = d->node_first[n], k = d->node_count[n];
    cnt[n] = uint8_t(k);
    double mx = 0, my = 0, mz = 0, smax = 0;
    for (uint32_t j = 0; j < k; ++j) {
      const float* m = d->means + 3 * size_t(f + j);
      mx += m[0]; my += m[1]; mz += m[2];
    }
    const float cx = float(mx / k), cy = float(my / k), cz = float(mz / k);
    double rho = 0;
    for (uint32_t j = 0; j < k; ++j) {
      const size_t g = f + j;
      const float* m = d->means + 3 * g;
      const double dx = double(m[0]) - cx, dy = double(m[1]) - cy, dz = double(m[2]) - cz;
      rho = std::max(rho, std::sqrt(dx * dx + dy * dy + dz * dz));
      const float* ls = d->log_scales + 3 * g;
      smax = std::max(smax, std::exp(double(std::max(ls[0], std::max(ls[1], ls[2])))));
      unsigned char* cb = attr.data() + size_t(n) * block;
      float* geo = reinterpret_cast<float*>(cb) + j;   // geometry plane p of this Gaussian: geo[p * 64]
      geo[kX * kSlots] = m[0];
      geo[kY * kSlots] = m[1];
      geo[kZ * kSlots] = m[2];
      for (int q = 0; q < 3; ++q) geo[(kLs0 + q) * kSlots] = ls[q];
      for (int q = 0; q < 4; ++q) geo[(kQw + q) * kSlots] = d->quats[4 * g + q];
      unsigned char* col = cb + size_t(kGeoPlanes) * kSlots * 4;
      auto put = [&](int plane, float v) {
        if (half)
          reinterpret_cast<__half*>(col)[plane * kSlots + j] = __float2half_rn(v);
        else
          reinterpret_cast<float*>(col)[plane * kSlots + j] = v;
      };
      put(kOpacity, d->opacity[g]);
      const float* sh = d->sh + g * coeffs * 3;
      for (uint32_t q = 0; q < coeffs * 3; ++q) put(int(kSh0 + q), sh[q]);
    }
    bound[n] = make_float4(cx, cy, cz, round_up_f(rho * (1.0 + 1e-6)));
    sigma[n] = round_up_f(smax * (1.0 + 1e-6));
    for (uint32_t j = 0; j < k; ++j) {
      const size_t g = f + j;
      if (!std::isfinite(d->opacity[g]) || !std::isfinite(d->means[3 * g]) || !std::isfinite(d->means[3 * g + 1]) ||
          !std::isfinite(d->means[3 * g + 2]))
        return fail(c, V3DG_EINVAL, "non-finite Gaussian %zu", g);
    }
  }
  // top-down traversal tables: children of every node (CSR, in node order) plus a virtual
  // super-root (index nn) whose children are the roots; per node a sphere around the bound
  // spheres of its whole subtree and the largest sigma in it (children before parents: by level)
  std::vector<uint32_t> child_off(nn + 2, 0), child_list;
  uint32_t levels = 0;
  for (uint32_t n = 0; n < nn; ++n) {
    const int32_t p = d->node_parent[n];
    ++child_off[(p < 0 ? nn : uint32_t(p)) + 1];
    levels = std::max<uint32_t>(levels, uint32_t(d->node_level[n]) + 1u);
  }
  for (uint32_t n = 0; n <= nn; ++n) child_off[n + 1] += child_off[n];
  child_list.resize(child_off[nn + 1]);
  {
    std::vector<uint32_t> fill(child_off.begin(), child_off.end() - 1);
    for (uint32_t n = 0; n < nn; ++n) {
      const int32_t p = d->node_parent[n];
      child_list[fill[p < 0 ? nn : uint32_t(p)]++] = n;
    }
  }
  std::vector<float4> sub_bound(nn);
  std::vector<float> sub_sigma(nn);
  {
    std::vector<uint32_t> by_level(nn);
    for (uint32_t n = 0; n < nn; ++n) by_level[n] = n;
    std::stable_sort(by_level.begin(), by_level.end(),
                     [&](uint32_t x, uint32_t y) { return d->node_level[x] < d->node_level[y]; });
    for (uint32_t n : by_level) {
      const float4 b = bound[n];
      double r = b.w;
      float sg = sigma[n];
      for (uint32_t q = child_off[n]; q < child_off[n + 1]; ++q) {
        const float4 cb = sub_bound[child_list[q]];
        const double dx = double(cb.x) - b.x, dy = double(cb.y) - b.y, dz = double(cb.z) - b.z;
        r = std::max(r, std::sqrt(dx * dx + dy * dy + dz * dz) + double(cb.w));
        sg = std::max(sg, sub_sigma[child_list[q]]);
      }
      sub_bound[n] = make_float4(b.x, b.y, b.z, round_up_f(r * (1.0 + 1e-6)));
      sub_sigma[n] = sg;
    }
  }
  AssetHost a;
  a.levels = levels;
  a.n_gauss = d->n_gauss;
  a.n_nodes = nn;
  a.sh_coeffs = coeffs;
  a.gpg = d->gaussians_per_group;
  a.half_color = half;
  a.node_first.assign(d->node_first, d->node_first + nn);
  auto up = [&](DevBuf& b, const void* src, size_t bytes) -> v3dg_status {
    ST(dalloc(c, b, bytes));
    CU(cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice));
    return V3DG_OK;
  };
  v3dg_status s = V3DG_OK;
  if ((s = up(a.own, own.data(), sizeof(float4) * nn)) != V3DG_OK || (s = up(a.par, par.data(), sizeof(float4) * nn)) != V3DG_OK ||
      (s = up(a.bound, bound.data(), sizeof(float4) * nn)) != V3DG_OK ||
      (s = up(a.sigma, sigma.data(), sizeof(float) * nn)) != V3DG_OK ||
      (s = up(a.flags, flags.data(), nn)) != V3DG_OK || (s = up(a.cnt, cnt.data(), nn)) != V3DG_OK ||
      (s = up(a.attr, attr.data(), attr.size())) != V3DG_OK ||
      (s = up(a.child_off, child_off.data(), sizeof(uint32_t) * child_off.size())) != V3DG_OK ||
      (s = up(a.child_list, child_list.data(), sizeof(uint32_t) * std::max<size_t>(child_list.size(), 1))) != V3DG_OK ||
      (s = up(a.sub_bound, sub_bound.data(), sizeof(float4) * nn)) != V3DG_OK ||
      (s = up(a.sub_sigma, sub_sigma.data(), sizeof(float) * nn)) != V3DG_OK) {
    DevBuf* bs[] = {&a.own, &a.par, &a.bound, &a.sigma, &a.flags, &a.cnt, &a.attr, &a.child_off, &a.child_list,
                    &a.sub_bound, &a.sub_sigma};
    for (DevBuf* b : bs) dfree(c, *b);
    return s;
  }
  ctx->assets.push_back(std::move(a));
  std::vector<AssetDev> table(ctx->assets.size());
  ctx->total_nodes = 0;
  for (size_t i = 0; i < ctx->assets.size(); ++i) {
    const AssetHost& h = ctx->assets[i];
    AssetDev& t = table[i];
    t.node_base = uint32_t(ctx->total_nodes);   // (not used once the total passes 2^32)
    ctx->total_nodes += h.n_nodes;
    t.own = P<float4>(h.own);
    t.par = P<float4>(h.par);
    t.bound = P<float4>(h.bound);
    t.sigma_max = P<float>(h.sigma);
    t.flags = P<uint8_t>(h.flags);
    t.count = P<uint8_t>(h.cnt);
    t.attr = P<unsigned char>(h.attr);
    t.n_nodes = h.n_nodes;
    t.stride = uint32_t(cluster_block_bytes(int(h.sh_coeffs), h.half_color));
    t.sh_coeffs = h.sh_coeffs;
    t.half_color = h.half_color ? 1u : 0u;
    t.child_off = P<uint32_t>(h.child_off);
    t.child_list = P<uint32_t>(h.child_list);
    t.sub_bound = P<float4>(h.sub_bound);
    t.sub_sigma = P<float>(h.sub_sigma);
    t.root = h.n_nodes;
  }
  ST(ensure(c, ctx->d_assets, sizeof(AssetDev) * table.size()));
  CU(cudaMemcpy(ctx->d_assets.p, table.data(), sizeof(AssetDev) * table.size(), cudaMemcpyHostToDevice));
  if (asset_id) *asset_id = uint32_t(ctx->assets.size() - 1);
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_set_instances(v3dg_ctx* ctx, uint32_t n, const uint32_t* asset_id, const double* rot, const double* trans,
                               const double* scale) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  if (n && (!asset_id || !rot || !trans || !scale)) return fail(c, V3DG_EINVAL, "NULL instance array");
  for (uint32_t i = 0; i < n; ++i) {
    if (asset_id[i] >= ctx->assets.size()) return fail(c, V3DG_ENOTFOUND, "instance %u: unknown asset %u", i, asset_id[i]);
    if (!(scale[i] > 0.0) || !std::isfinite(scale[i])) return fail(c, V3DG_EINVAL, "instance %u: scale must be > 0", i);
    for (int q = 0; q < 9; ++q)
      if (!std::isfinite(rot[9 * size_t(i) + q])) return fail(c, V3DG_EINVAL, "instance %u: rotation not finite", i);
    for (int q = 0; q < 3; ++q)
      if (!std::isfinite(trans[3 * size_t(i) + q])) return fail(c, V3DG_EINVAL, "instance %u: translation not finite", i);
  }
  c->inst_asset.assign(asset_id, asset_id + n);
  c->inst_rot.assign(rot, rot + 9 * size_t(n));
  c->inst_trans.assign(trans, trans + 3 * size_t(n));
  c->inst_scale.assign(scale, scale + n);
  c->selected = false;
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_select(v3dg_ctx* ctx, const v3dg_camera* cam, float tau_px) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  CU(cudaSetDevice(ctx->device));
  ST(setup_frame(c, cam, 1, tau_px));
  ST(select_or_defer(c));
  c->selected = true;
  c->rendered = false;
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_select_views(v3dg_ctx* ctx, const v3dg_camera* cams, uint32_t n_views, float tau_px) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  CU(cudaSetDevice(ctx->device));
  ST(setup_frame(c, cams, n_views, tau_px));
  ST(select_or_defer(c));
  c->selected = true;
  c->rendered = false;
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_render(v3dg_ctx* ctx, float* rgb_out, float* t_out) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  if (!c->selected) return fail(c, V3DG_ENOTFOUND, "v3dg_render without a prior v3dg_select");
  if (!rgb_out) return fail(c, V3DG_EINVAL, "rgb_out is NULL");
  ST(render_frame(c, rgb_out, t_out, ctx->sync_check));
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_render_host(v3dg_ctx* ctx, float* rgb_host, float* t_host) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  if (!c->selected) return fail(c, V3DG_ENOTFOUND, "v3dg_render_host without a prior v3dg_select");
  if (!rgb_host) return fail(c, V3DG_EINVAL, "rgb_host is NULL");
  const size_t px = size_t(c->cam.width) * size_t(c->cam.height) * c->n_views;
  ST(ensure(c, c->d_img, sizeof(float) * 3 * px));
  if (t_host) ST(ensure(c, c->d_timg, sizeof(float) * px));
  ST(render_frame(c, P<float>(c->d_img), t_host ? P<float>(c->d_timg) : nullptr, ctx->sync_check));
  CU(cudaMemcpyAsync(rgb_host, c->d_img.p, sizeof(float) * 3 * px, cudaMemcpyDeviceToHost, c->stream));
  if (t_host) CU(cudaMemcpyAsync(t_host, c->d_timg.p, sizeof(float) * px, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (c->h_frame[kTimeout]) return fail(c, V3DG_ETIMEOUT, "a bounded device-side wait gave up; frame invalid");
  if (c->h_frame[kOverflow]) return fail(c, V3DG_EOVERFLOW, "frame overflowed its buffers");
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_frame_stats(v3dg_ctx* ctx, v3dg_stats* out) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c || !out) return V3DG_EINVAL;
  if (!c->selected) return fail(c, V3DG_ENOTFOUND, "no frame selected");
  if (c->select_pending) {   // a graph frame's selection not rendered yet: run it now for the counters
    ST(enqueue_select(c));
    c->select_pending = false;
  }
  ST(sync_frame(c));
  std::memset(out, 0, sizeof *out);
  const uint32_t* f = c->h_frame;
  out->render_nodes = f[kRenderNodes];
  out->visible = f[kVisible];
  out->pairs = f[kPairs];
  out->conic_fp64 = f[kConicFp64];
  out->render_clusters = f[kRenderClusters];
  uint32_t sticky[2] = {0, 0};
  CU(cudaMemcpy(sticky, P<uint32_t>(c->d_misc) + 12, sizeof sticky, cudaMemcpyDeviceToHost));
  CU(cudaMemset(P<uint32_t>(c->d_misc) + 12, 0, sizeof sticky));
  out->overflow = f[kOverflow] | sticky[0];
  out->timeout = f[kTimeout] | sticky[1];
  if (ctx->count_work) std::memcpy(&out->blend_evals, c->h_tmp + kFrameWords, 2 * sizeof(unsigned long long));
  uint32_t ncut = 0, ng = 0;
  ST(run_cut(c, &ncut, &ng));
  out->cut_nodes = ncut;
  out->cut_gaussians = ng;
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_get_cut(v3dg_ctx* ctx, uint32_t* inst_node, uint64_t cap, uint64_t* n) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c || !n) return V3DG_EINVAL;
  uint32_t ncut = 0, ng = 0;
  ST(run_cut(c, &ncut, &ng));
  *n = ncut;
  if (inst_node && cap) {
    const size_t m = size_t(std::min<uint64_t>(cap, ncut));
    CU(cudaMemcpy(inst_node, c->d_cut.p, sizeof(uint2) * m, cudaMemcpyDeviceToHost));
  }
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_get_projected(v3dg_ctx* ctx, uint64_t cap, uint64_t* n, uint32_t* inst, uint32_t* local, float* u,
                               float* conic, float* opacity, float* rgb, uint32_t* depth_key, int32_t* rect) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c || !n) return V3DG_EINVAL;
  if (!c->rendered) return fail(c, V3DG_ENOTFOUND, "no frame rendered");
  ST(sync_frame(c));
  const uint32_t nr = std::min(c->h_frame[kRenderNodes], c->cap_nodes);
  const uint32_t nv = c->h_frame[kVisible];
  const size_t S = size_t(nr) * kSlots;
  std::vector<uint2> list(nr);
  std::vector<uint32_t> keys(nv), slots(nv);
  std::vector<float4> rec(3 * S);
  std::vector<uint2> rc(S);
  if (nr) CU(cudaMemcpy(list.data(), c->d_list.p, sizeof(uint2) * nr, cudaMemcpyDeviceToHost));
  if (nv) {
    CU(cudaMemcpy(keys.data(), (c->depth_in1 ? c->d_keys1 : c->d_keys0).p, 4 * size_t(nv), cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(slots.data(), (c->depth_in1 ? c->d_vals1 : c->d_vals0).p, 4 * size_t(nv), cudaMemcpyDeviceToHost));
  }
  if (S) {
    CU(cudaMemcpy(rec.data(), c->d_rec.p, sizeof(float4) * 3 * S, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(rc.data(), c->d_rect.p, sizeof(uint2) * S, cudaMemcpyDeviceToHost));
  }
  std::vector<uint32_t> order(nv);
  for (uint32_t k = 0; k < nv; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return slots[a] < slots[b]; });
  *n = nv;
  const double log2e = 1.4426950408889634;
  const uint64_t m = std::min<uint64_t>(cap, nv);
  for (uint64_t q = 0; q < m; ++q) {
    const uint32_t k = order[q];
    const uint32_t slot = slots[k];
    const uint2 e = list[slot / kSlots];
    const uint32_t j = slot % kSlots;
    const float4 r0 = rec[3 * size_t(slot)], r1 = rec[3 * size_t(slot) + 1], r2 = rec[3 * size_t(slot) + 2];
    uint32_t org;
    std::memcpy(&org, &r2.y, 4);
    const uint2 rr = rc[slot];
    if (inst) inst[q] = e.x;
    if (local) local[q] = ctx->assets[c->frame_asset[e.x]].node_first[e.y] + j;
    if (u) {
      u[2 * q] = float(double(r0.x) + 16.0 * double(org & 0xFFFFu));
      u[2 * q + 1] = float(double(r0.y) + 16.0 * double(org >> 16));
    }
    if (conic) {
      conic[3 * q] = float(double(r0.z) / (-0.5 * log2e));
      conic[3 * q + 1] = float(double(r0.w) / (-log2e));
      conic[3 * q + 2] = float(double(r1.x) / (-0.5 * log2e));
    }
    if (opacity) opacity[q] = float(std::exp2(double(r1.y)));
    if (rgb) {
      rgb[3 * q] = r1.z;
      rgb[3 * q + 1] = r1.w;
      rgb[3 * q + 2] = r2.x;
    }
    if (depth_key) depth_key[q] = keys[k];
    if (rect) {
      rect[4 * q] = int32_t((rr.x & 0xFFFFu) >> 4);   // the pixel box's tiles
      rect[4 * q + 1] = int32_t((rr.x >> 16) >> 4);
      rect[4 * q + 2] = int32_t((rr.y & 0xFFFFu) >> 4);
      rect[4 * q + 3] = int32_t((rr.y >> 16) >> 4);
    }
  }
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_get_pairs(v3dg_ctx* ctx, uint64_t cap, uint64_t* n, uint32_t* tile, uint32_t* depth_key, uint32_t* inst,
                           uint32_t* local) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c || !n) return V3DG_EINVAL;
  if (!c->rendered) return fail(c, V3DG_ENOTFOUND, "no frame rendered");
  ST(sync_frame(c));
  const uint32_t np = std::min(c->h_frame[kPairsEff], c->cap_pairs);
  const uint32_t nr = std::min(c->h_frame[kRenderNodes], c->cap_nodes);
  const uint32_t nv = c->h_frame[kVisible];
  *n = np;
  const uint64_t m = std::min<uint64_t>(cap, np);
  if (m == 0) return V3DG_OK;
  std::vector<uint32_t> tk(m), tv(m), keys(nv), slots(nv);
  std::vector<uint2> list(nr);
  CU(cudaMemcpy(tk.data(), (c->tiles_in1 ? c->d_pk1 : c->d_pk0).p, 4 * m, cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(tv.data(), (c->tiles_in1 ? c->d_pv1 : c->d_pv0).p, 4 * m, cudaMemcpyDeviceToHost));
  if (nv) {
    CU(cudaMemcpy(keys.data(), (c->depth_in1 ? c->d_keys1 : c->d_keys0).p, 4 * size_t(nv), cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(slots.data(), (c->depth_in1 ? c->d_vals1 : c->d_vals0).p, 4 * size_t(nv), cudaMemcpyDeviceToHost));
  }
  if (nr) CU(cudaMemcpy(list.data(), c->d_list.p, sizeof(uint2) * nr, cudaMemcpyDeviceToHost));
  std::vector<uint32_t> key_of(size_t(nr) * kSlots, 0xFFFFFFFFu);
  for (uint32_t k = 0; k < nv; ++k)
    if (slots[k] < key_of.size()) key_of[slots[k]] = keys[k];
  for (uint64_t q = 0; q < m; ++q) {
    const uint32_t slot = tv[q];
    if (tile) tile[q] = tk[q] & kPairTileMask;
    if (slot / kSlots >= nr) return fail(c, V3DG_EINVAL, "pair %llu references slot %u beyond the render list",
                                         (unsigned long long)q, slot);
    const uint2 e = list[slot / kSlots];
    if (depth_key) depth_key[q] = key_of[slot];
    if (inst) inst[q] = e.x;
    if (local) local[q] = ctx->assets[c->frame_asset[e.x]].node_first[e.y] + slot % kSlots;
  }
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_get_tile_ranges(v3dg_ctx* ctx, uint32_t* range, uint64_t cap, uint64_t* n_tiles) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c || !n_tiles) return V3DG_EINVAL;
  if (!c->rendered) return fail(c, V3DG_ENOTFOUND, "no frame rendered");
  ST(sync_frame(c));
  const uint64_t nt = uint64_t(c->cc.tiles_x) * uint64_t(c->cc.tiles_y) * c->n_views;
  *n_tiles = nt;
  if (range && cap) CU(cudaMemcpy(range, c->d_ranges.p, sizeof(uint2) * std::min(cap, nt), cudaMemcpyDeviceToHost));
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_stage_times(v3dg_ctx* ctx, float* ms, int n, uint64_t* launches) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  if (launches) *launches = ctx->launches;
  if (ms && n > 0) {
    if (!ctx->stage_timing || !c->rendered) return fail(c, V3DG_ENOTFOUND, "stage timing is off or no frame rendered");
    CU(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < n && i < kStages; ++i) CU(cudaEventElapsedTime(ms + i, c->ev[i], c->ev[i + 1]));
  }
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_autotune_blend(v3dg_ctx* ctx, uint32_t* mode_out, uint32_t* batch_out, uint32_t* split_out,
                                float* ms_out) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  if (!c->rendered) return fail(c, V3DG_ENOTFOUND, "no frame rendered");
  ST(sync_frame(c));
  if (c->h_frame[kOverflow] || c->h_frame[kTimeout]) return fail(c, V3DG_EOVERFLOW, "the last frame was not valid");
  const CamConst& k = c->cc;
  const size_t px = size_t(k.width) * size_t(k.height) * c->n_views;
  ST(ensure(c, c->d_img, sizeof(float) * 3 * std::max<size_t>(px, 1)));
  const uint32_t* tk = P<uint32_t>(c->tiles_in1 ? c->d_pk1 : c->d_pk0);
  const uint32_t* tv = P<uint32_t>(c->tiles_in1 ? c->d_pv1 : c->d_pv0);
  uint32_t* frame = P<uint32_t>(c->d_frame);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(c, V3DG_ECUDA, "cudaEventCreate failed");
  }
  const int batches[] = {128, 256, 512};
  const uint32_t splits[] = {4096u, 16384u, 65536u, 0xFFFFFFFFu};
  float best = INFINITY;
  int best_b = ctx->blend_batch, best_m = ctx->blend_mode;
  uint32_t best_s = ctx->split_pairs;
  cudaError_t e = cudaSuccess;
  for (int mode = 0; mode < 2; ++mode)
  for (int b : batches) {
    for (uint32_t sp : splits) {
      if (mode == 1 && sp != 0xFFFFFFFFu) continue;   // that variant always blends whole tiles
      float t_min = INFINITY;
      for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first run warms up
        e = cudaMemsetAsync(frame + kTileCounters + 10, 0, sizeof(uint32_t), c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess)
          e = launch_blend(P<uint2>(c->d_ranges), P<uint32_t>(c->d_order), frame + kTileCounters + 10, tk, tv,
                           P<float4>(c->d_rec), c->cap_slots, k, P<float>(c->d_img), nullptr, nullptr, frame,
                           P<uint32_t>(c->d_misc) + 12, sp, b, mode, int(c->n_views), ctx->sm_count, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0) t_min = std::min(t_min, ms);
        ctx->launches += 2;
      }
      if (t_min < best) {
        best = t_min;
        best_b = b;
        best_s = sp;
        best_m = mode;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(c, V3DG_ECUDA, "CUDA error %s", cudaGetErrorString(e));
  ctx->blend_batch = best_b;
  ctx->split_pairs = best_s;
  ctx->blend_mode = best_m;
  if (mode_out) *mode_out = uint32_t(best_m);
  if (batch_out) *batch_out = uint32_t(best_b);
  if (split_out) *split_out = best_s;
  if (ms_out) *ms_out = best;
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_sort_pairs(v3dg_ctx* ctx, uint32_t* keys, uint32_t* vals, uint64_t n, int begin_bit, int end_bit) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  if (n == 0) return V3DG_OK;
  if (!keys || !vals) return fail(c, V3DG_EINVAL, "NULL keys or values");
  if (n > kMaxPairs) return fail(c, V3DG_EINVAL, "n = %llu exceeds %u", (unsigned long long)n, kMaxPairs);
  if (begin_bit < 0 || end_bit > 32 || begin_bit >= end_bit) return fail(c, V3DG_EINVAL, "bad bit range [%d, %d)", begin_bit, end_bit);
  CU(cudaSetDevice(ctx->device));
  ST(ensure(c, c->d_sort_k, 4 * n));
  ST(ensure(c, c->d_sort_v, 4 * n));
  ST(ensure_status(c, ((n + kSortTile - 1) / kSortTile) * 256));
  ST(ensure(c, c->d_hist, 2 * 4 * 256 * 4));  // counts + exclusive offsets of up to 4 passes
  uint32_t* misc = P<uint32_t>(c->d_misc);  // [0] n, [1..4] tile counters, [5] timeout flag
  CU(cudaMemsetAsync(misc, 0, sizeof(uint32_t) * 8, c->stream));
  k_set_word<<<1, 1, 0, c->stream>>>(misc, uint32_t(n));
  CU(cudaGetLastError());
  bool in1 = false;
  int nl = 0;
  CU(launch_sort(keys, vals, P<uint32_t>(c->d_sort_k), P<uint32_t>(c->d_sort_v), misc, uint32_t(n), begin_bit, end_bit,
                 false, sort_scratch(c, misc + 1), misc + 5, c->epoch, ctx->sm_count, c->stream, &in1, &nl));
  next_epoch(c);
  ctx->launches += nl + 1;
  if (in1) {
    CU(cudaMemcpyAsync(keys, c->d_sort_k.p, 4 * n, cudaMemcpyDeviceToDevice, c->stream));
    CU(cudaMemcpyAsync(vals, c->d_sort_v.p, 4 * n, cudaMemcpyDeviceToDevice, c->stream));
  }
  CU(cudaMemcpyAsync(c->h_tmp, misc + 5, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (c->h_tmp[0]) return fail(c, V3DG_ETIMEOUT, "a bounded device-side wait gave up; output invalid");
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_check_wait(v3dg_ctx* ctx, uint32_t spin_limit, int predecessor_publishes, uint32_t* prefix) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  if (spin_limit < 1 || spin_limit > kSpinLimit)
    return fail(c, V3DG_EINVAL, "spin_limit must be in [1, %u]", kSpinLimit);
  CU(cudaSetDevice(ctx->device));
  ST(ensure_status(c, std::max<uint64_t>(c->status_words, 4)));
  uint32_t* out = P<uint32_t>(c->d_misc) + 16;   // d_misc[16..18]: the two prefixes and the gave-up flag
  CU(cudaMemsetAsync(c->d_status.p, 0, 4 * sizeof(uint64_t), c->stream));   // epoch 0 is never a current epoch
  CU(cudaMemsetAsync(out, 0, 3 * sizeof(uint32_t), c->stream));
  CU(launch_check_wait(P<uint64_t>(c->d_status), next_epoch(c), spin_limit, predecessor_publishes, out, c->stream));
  ++ctx->launches;
  CU(cudaMemcpyAsync(c->h_tmp, out, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (prefix) *prefix = c->h_tmp[0];
  if (c->h_tmp[2]) return fail(c, V3DG_ETIMEOUT, "the look-back gave up after %u polls", spin_limit);
  if (c->h_tmp[0] != 1000u || c->h_tmp[1] != 1001u)
    return fail(c, V3DG_ECUDA, "look-back prefixes %u, %u (expected 1000, 1001)", c->h_tmp[0], c->h_tmp[1]);
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_release_buffers(v3dg_ctx* ctx, uint64_t* released) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  if (ctx->server) return fail(c, V3DG_EBUSY, "buffers cannot be released while a server runs");
  CU(cudaSetDevice(ctx->device));
  const uint64_t b = pipe_bytes(c);
  pipe_trim(c);
  if (released) *released = b;
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_server_start(v3dg_ctx* ctx, int slots, uint64_t hbm_budget) {
  Pipe* c = ctx ? &ctx->main : nullptr;
  if (!c) return V3DG_EINVAL;
  if (slots < 1 || slots > 64) return fail(c, V3DG_EINVAL, "slots must be in [1, 64]");
  if (ctx->server) return fail(c, V3DG_EBUSY, "the server is already running");
  if (ctx->assets.empty()) return fail(c, V3DG_ENOTFOUND, "no hierarchy loaded");
  CU(cudaSetDevice(ctx->device));
  Server* sv = new (std::nothrow) Server;
  if (!sv) return fail(c, V3DG_ENOMEM, "out of host memory");
  sv->ctx = ctx;
  sv->merge = size_t(ctx->serve_merge);
  {  // no budget given: 3/4 of the device memory free now; each slot keeps at most its share of
     // the budget between requests
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = 0;
    }
    sv->budget = hbm_budget ? hbm_budget : (free_b ? uint64_t(free_b) * 3 / 4 : ~uint64_t(0));
    // memory a slot releases returns to the shared pool and is reused without synchronising, so
    // a slot keeps between requests only buffers within half its share of the budget
    if (sv->budget != ~uint64_t(0)) sv->slot_keep = sv->budget / (2 * uint64_t(slots));
  }
  int least = 0, greatest = 0;
  CU(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  {  // one stream-ordered pool for every slot: no device-wide synchronisation on allocation or
     // release, and memory a slot releases is reused by the others
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->device;
    if (cudaMemPoolCreate(&sv->pool, &props) != cudaSuccess) {
      cudaGetLastError();
      delete sv;
      return fail(c, V3DG_ECUDA, "cudaMemPoolCreate failed");
    }
    uint64_t keep = ~uint64_t(0);
    cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  for (int i = 0; i < slots; ++i) {
    auto p = std::make_unique<Pipe>();
    p->ctx_alloc = false;   // workers allocate from the server's pool: the context's allocator is
                            // called from the owner's thread only
    p->pool = sv->pool;
    cudaStream_t hi = nullptr, lo = nullptr;
    const bool ok = cudaStreamCreateWithPriority(&hi, cudaStreamNonBlocking, greatest) == cudaSuccess &&
                    cudaStreamCreateWithPriority(&lo, cudaStreamNonBlocking, least) == cudaSuccess;
    sv->hi.push_back(hi);
    sv->lo.push_back(lo);
    if (!ok) {
      ctx->server = sv;
      server_stop(ctx);
      return fail(c, V3DG_ECUDA, "cudaStreamCreateWithPriority failed");
    }
    const v3dg_status s = pipe_init(ctx, p.get(), hi);
    sv->slots.push_back(std::move(p));
    if (s != V3DG_OK) {
      ctx->server = sv;
      server_stop(ctx);
      return fail(c, s, "slot set-up failed");
    }
  }
  ctx->server = sv;
  for (size_t i = 0; i < sv->slots.size(); ++i) sv->threads.emplace_back(slot_main, sv, sv->slots[i].get(), i);
  c->err.clear();
  return V3DG_OK;
}

v3dg_status v3dg_server_stop(v3dg_ctx* ctx) {
  if (!ctx) return V3DG_EINVAL;
  server_stop(ctx);
  return V3DG_OK;
}

v3dg_status v3dg_submit(v3dg_ctx* ctx, const v3dg_request* req, uint64_t* ticket) {
  if (!ctx || !req || !ticket) return V3DG_EINVAL;
  Server* sv = ctx->server;
  if (!sv) return V3DG_ENOTFOUND;
  const uint32_t n = req->n_instances;
  if (n && (!req->asset_id || !req->rot || !req->trans || !req->scale)) return V3DG_EINVAL;
  if (!req->rgb_out) return V3DG_EINVAL;
  const v3dg_camera& cam = req->camera;
  if (cam.width <= 0 || cam.height <= 0 || !(cam.fx > 0.f) || !(cam.fy > 0.f) || !(req->tau_px >= 0.f))
    return V3DG_EINVAL;
  if (uint64_t((cam.width + kTile - 1) / kTile) * uint64_t((cam.height + kTile - 1) / kTile) > uint64_t(kMaxTiles))
    return V3DG_EINVAL;
  for (uint32_t i = 0; i < n; ++i) {
    if (req->asset_id[i] >= ctx->assets.size()) return V3DG_ENOTFOUND;
    if (!(req->scale[i] > 0.0) || !std::isfinite(req->scale[i])) return V3DG_EINVAL;
  }
  Request rq;
  rq.asset.assign(req->asset_id, req->asset_id + n);
  rq.rot.assign(req->rot, req->rot + 9 * size_t(n));
  rq.trans.assign(req->trans, req->trans + 3 * size_t(n));
  rq.scale.assign(req->scale, req->scale + n);
  rq.cam = cam;
  rq.tau_px = req->tau_px;
  rq.rgb = req->rgb_out;
  rq.t = req->t_out;
  rq.out_device = req->out_on_device != 0;
  rq.est_bytes = request_bytes(n, cam, req->tau_px);
  rq.heavy = rq.est_bytes > sv->budget / (2 * uint64_t(sv->slots.size()));
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return V3DG_EBUSY;
    rq.ticket = sv->next_ticket++;
    rq.t_submit = sv->now_ms();
    *ticket = rq.ticket;
    sv->pending.insert(rq.ticket);
    sv->queue.push_back(std::move(rq));
  }
  sv->cv_work.notify_one();
  return V3DG_OK;
}

v3dg_status v3dg_poll(v3dg_ctx* ctx, uint64_t ticket, uint32_t timeout_us, v3dg_result* out) {
  if (!ctx || !out) return V3DG_EINVAL;
  Server* sv = ctx->server;
  if (!sv) return V3DG_ENOTFOUND;
  std::unique_lock<std::mutex> lk(sv->mu);
  if (!sv->pending.count(ticket)) return V3DG_ENOTFOUND;
  const bool ready = sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us),
                                          [&] { return sv->finished.count(ticket) != 0; });
  if (!ready) return V3DG_EBUSY;
  const Finished f = sv->finished[ticket];
  sv->finished.erase(ticket);
  sv->pending.erase(ticket);
  std::memset(out, 0, sizeof *out);
  out->status = f.status;
  out->submit_ms = f.t_submit;
  out->start_ms = f.t_start;
  out->done_ms = f.t_done;
  out->visible = f.visible;
  out->pairs = f.pairs;
  out->batch_views = f.batch_views;
  return V3DG_OK;
}

}  // extern "C"
