// Internal layouts shared by the host side (v3dg_api.cpp) and the kernels (*.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace v3dg {

constexpr int kTile = 16;              // 16x16 pixel tiles
constexpr int kSlots = 64;             // Gaussian slots per cluster block on the device
constexpr int kMaxShCoeffs = 16;       // degree 3

// Attributes of one asset, one contiguous block per cluster: planes of 64 values (j = 0..63 is
// the Gaussian within the cluster).  First the geometry planes, always float32, then the colour
// planes (opacity, then SH coefficient-major, channel-minor), float32 or -- for assets loaded with
// V3DG_OPT_ATTR_FP16 -- float16.
enum GeoPlane : int { kX = 0, kY, kZ, kLs0, kLs1, kLs2, kQw, kQx, kQy, kQz, kGeoPlanes };
enum ColorPlane : int { kOpacity = 0, kSh0 = 1 };   // SH: kSh0 + 3 * coeff + channel
constexpr int color_planes(int sh_coeffs) { return kSh0 + 3 * sh_coeffs; }
constexpr size_t cluster_block_bytes(int sh_coeffs, bool half) {
  return size_t(kGeoPlanes) * kSlots * 4 + size_t(color_planes(sh_coeffs)) * kSlots * (half ? 2 : 4);
}

// Node flags.
constexpr uint8_t kLeaf = 1, kRoot = 2;

struct AssetDev {
  const float4* own;       // own sphere (cluster group of the node), asset frame
  const float4* par;       // parent's own sphere (root: copy of own, unused)
  const float4* bound;     // sphere around the node's Gaussian means: centre = their mean
  const float* sigma_max;  // max over the node's Gaussians of exp(max log-scale)
  const uint8_t* flags;    // kLeaf | kRoot
  const uint8_t* count;    // Gaussians in the node, 1..64
  const unsigned char* attr;  // n_nodes cluster blocks of `stride` bytes
  uint32_t n_nodes;
  uint32_t stride;         // bytes per cluster block: cluster_block_bytes(sh_coeffs, half_color)
  uint32_t sh_coeffs;      // (degree + 1)^2
  uint32_t half_color;     // 1: opacity and SH stored as float16
  // top-down selection: children of node n are child_list[child_off[n] .. child_off[n + 1]);
  // sub_bound / sub_sigma bound the spheres and sigmas of every node of n's subtree
  const uint32_t* child_off;
  const uint32_t* child_list;
  const float4* sub_bound;
  const float* sub_sigma;
  uint32_t root;
  uint32_t node_base;      // global id of node 0: the node counts of the assets loaded before this one
};

// Per (frame, instance) constants, computed on the host in FP64 (128-byte aligned, 256 B).
struct alignas(16) InstFrame {
  double m64[12];          // M = W [s R | t], row-major 3x4
  float m[12];             // float32 rounding of m64
  float cam_a[3];          // camera centre in the asset frame, R^T (C - t) / s
  float s;                 // uniform scale
  double s64;
  float tau_f;             // area tolerance of this instance's asset
  uint32_t asset;
  uint32_t view;           // the camera (view) this instance frame belongs to
  uint32_t pad[19];
};
static_assert(sizeof(InstFrame) == 256, "InstFrame layout");

// Camera constants passed by value to the kernels.
struct CamConst {
  float fx, fy, cx, cy;
  float near_z;
  float limx, limy;        // Jacobian clamp: 1.3 * (w / 2) / fx
  int width, height;
  int tiles_x, tiles_y;
  double k_foot;           // pi * fx * fy (FP64) for the exact footprint re-test
  float k_foot32;
  float cull_kx, cull_ky;  // conservative pixel half-width factors of the visibility cull
};

// Frame counters (device, uint32 each).
enum Counter : int {
  kCutNodes = 0, kCutGauss, kRenderNodes, kVisible, kPairs, kOverflow, kTimeout,
  kSlotCount = 7,          // render nodes (clamped) * 64: the slots the depth sort covers
  kPairsEff = 8,           // pairs the tile sort / blend use: kPairs, or 0 when the frame overflowed
  kTdReached = 9,          // top-down selection: (instance, node) entries it tested
  kConicFp64 = 10,         // Gaussians whose 2D covariance had det < 1e-12 and was inverted in FP64
  kRenderClusters = 11,    // distinct clusters of the render list (projection grouped by cluster)
  kPairs64 = 12,           // [12, 14): the pair total as a 64-bit sum (detects totals beyond 2^32)
  kNumCounters = 16,
  kTileCounters = 16,      // [16, 48): atomic tile counters of the chained-scan kernels
  kFrameWords = 48,
};

// Status words of the chained (decoupled look-back) scans: epoch << 34 | flag << 32 | value.
constexpr uint64_t kFlagAgg = 1, kFlagPrefix = 2;
constexpr uint32_t kSpinLimit = 1u << 20;

// Diagnostic of the bounded waits: one look-back as tile 1 of a two-tile chain whose tile 0
// publishes (publish != 0) or never does, with at most spin_limit polls, by one thread and by a
// whole warp.  out[0], out[1]: the prefixes the two look-backs found; out[2]: nonzero if a wait
// gave up.  status: 2 * 2 words.
cudaError_t launch_check_wait(uint64_t* status, uint32_t epoch, uint32_t spin_limit, int publish, uint32_t* out,
                              cudaStream_t st);

// ---------------------------------------------------------------- launch functions (return cudaError)
// Selection (Sec. 3.3-3.4).  mode 0: render list (cut minus the visibility cull) + counters;
// mode 1: the cut itself (parity read-back).
cudaError_t launch_select(const InstFrame* inst, int n_inst, const AssetDev* assets, int node_blocks,
                          const CamConst& cam, int mode, uint2* out, uint32_t cap, uint32_t* frame,
                          uint32_t tile_counter_slot, uint64_t* status, uint32_t epoch, cudaStream_t st);

// Top-down selection (same result as launch_select on trees whose footprints never grow from a
// node to its parent, which the containment of the cluster-group spheres guarantees): level by
// level from each instance's root, a node whose own footprint exceeds tau_F hands its children
// to the next level; the others are selected.  mode 0 also skips every subtree whose bound
// proves the visibility cull of all its nodes.  Marks go to a bitmap of n_inst * wpi words
// (zeroed by the caller), which one ordered compaction turns into the list of launch_select.
// frontier: two buffers of cap_front entries; counts: steps + 1 words (zeroed by the caller).
struct TopDown {
  uint2* frontier[2];
  uint32_t cap_front;
  uint32_t* counts;
  uint32_t* bitmap;
  uint32_t wpi;            // bitmap words per instance: ceil(max nodes / 32)
  int steps;               // largest root level + 1
};
cudaError_t launch_select_topdown(const InstFrame* inst, int n_inst, const AssetDev* assets, const CamConst& cam,
                                  int mode, const TopDown& td, uint2* out, uint32_t cap, uint32_t* frame,
                                  uint32_t tile_counter_slot, uint64_t* status, uint32_t epoch, int sm_count,
                                  cudaStream_t st, int* launches);

// Per render-list node, FP64 reference for the projection (2 float4 per node):
//   [0] = (U0 hi, U0 lo, V0 hi, V0 lo): pixel position of the node's mean centre as float pairs
//   [1] = (rho_x, rho_y, Pz, mode): X/Z, Y/Z and Z of that centre in view space; mode 1 =
//         compensated (centre well in front), 0 = direct (rho_x, rho_y then hold X, Y).
// order_keys (may be NULL): also writes, per entry, its cluster's global id (node_base + node)
// shifted right by key_shift, the key that groups the render list by cluster for the projection.
cudaError_t launch_noderef(const uint2* render_list, uint32_t cap_nodes, const InstFrame* inst,
                           const AssetDev* assets, const CamConst& cam, float4* ref,
                           const uint32_t* frame, uint32_t* order_keys, int key_shift, int sm_count,
                           cudaStream_t st);

// Records (3 float4 per slot, slot = render index * 64 + j):
//   [0] = (u_rel, v_rel, na, nb), [1] = (nc, log2 o, r, g), [2] = (b, tile origin, x range, y range)
// with (u_rel, v_rel) the 2D mean relative to the pixel origin of the Gaussian's first tile
// (tx0, ty0), log2(alpha) = na dx^2 + nb dx dy + nc dy^2 + log2 o, and the inclusive pixel
// ranges x0 | x1 << 16, y0 | y1 << 16 of the alpha >= 1/255 ellipse's bounding box.
// color_formats: bit 0 set if some loaded asset stores its colour planes in float32, bit 1 if
// some asset stores them in float16 (the kernel is specialised for the formats present).
// order (may be NULL: list order): a permutation of the render-list indices that the warps take
// in turn.  Each entry's outputs stay at its own slots, so the order changes no result; ordered by
// cluster, the instances that draw one cluster read its attributes one after the other, and all
// but the first find them in L2.  sorted_keys (may be NULL): the global cluster id of each
// position of `order`; the distinct ones are counted into frame[kRenderClusters].
cudaError_t launch_project(const uint2* render_list, uint32_t cap_nodes, const InstFrame* inst,
                           const AssetDev* assets, const CamConst& cam, const float4* ref, float4* rec,
                           uint2* rect, uint32_t* keys, uint32_t* frame, const uint32_t* order,
                           const uint32_t* sorted_keys, int color_formats, int sm_count, cudaStream_t st);

// Radix sort of (key, value) pairs, n read from *n_dev (clamped to cap).  Ping-pongs between
// (k0, v0) and (k1, v1); the result lands in (k0, v0) when the pass count is even, else in
// (k1, v1) -- *result_in_1 tells which.  implicit_vals: the values of the first pass are the
// element indices (v0 is not read).
struct SortScratch {
  uint32_t* hist;          // 4 passes * 256 counts, then 4 passes * 256 exclusive offsets
  uint64_t* status;        // max_tiles * 256
  uint32_t max_tiles;
  uint32_t* tile_counters; // one per pass (zeroed by the caller's frame memset)
};
constexpr int kSortThreads = 256, kSortItems = 16, kSortTile = kSortThreads * kSortItems;
cudaError_t launch_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const uint32_t* n_dev,
                        uint32_t cap, int begin_bit, int end_bit, bool implicit_vals,
                        const SortScratch& sc, uint32_t* err_flag, uint32_t& epoch, int sm_count,
                        cudaStream_t st, bool* result_in_1, int* launches);

// Pair keys: tile id in bits 0..19 (at most 2^20 tiles), then the Gaussian's pixel box clipped
// to the tile, tile-local and inclusive: rows y0 in bits 20..23 and y1 in 24..27, columns rounded
// out to quads of 4, x0 / 4 in bits 28..29 and x1 / 4 in 30..31.
constexpr uint32_t kPairTileMask = 0xFFFFFu;
constexpr int kMaxTiles = 1 << 20;

// Per-device kernel attributes (shared-memory carveouts), set once per context before any launch
// (so that no attribute call happens during a stream capture).
cudaError_t sort_set_attributes();
cudaError_t blend_set_attributes();
cudaError_t project_set_attributes();

// Expansion of the depth-sorted visible Gaussians into (tile, slot) pairs in depth order; writes
// frame[kPairs] (the total) and frame[kPairsEff] (0 if the frame overflowed).  rect: per slot,
// the pixel box (x0 | x1 << 16, y0 | y1 << 16) of the alpha >= 1/255 ellipse, inclusive.
// Several views: the tile id of a pair is view * tiles_per_view + tile, with the view of the
// Gaussian's instance frame (inst_views[list[slot / 64].x].view; inst_views NULL: one view).
cudaError_t launch_expand(const uint32_t* sorted_slots, const uint2* rect, uint32_t cap_slots, uint32_t cap_pairs,
                          int tiles_x, const uint2* list, const InstFrame* inst_views, uint32_t tiles_per_view,
                          uint32_t* pair_keys, uint32_t* pair_vals, uint32_t* frame, uint32_t tile_counter_slot,
                          uint64_t* status, uint32_t epoch, int sm_count, cudaStream_t st);
cudaError_t launch_ranges(const uint32_t* tile_keys, uint32_t cap_pairs, const uint32_t* frame,
                          uint2* ranges, int n_tiles, int sm_count, cudaStream_t st);
// work != nullptr: also count (evaluations, contributions) into work[0], work[1].
// sticky[0] |= frame[kOverflow], sticky[1] |= frame[kTimeout] (the flags of every frame since the
// host last cleared them).
// items: 4 * n_tiles + 1 words of scratch (the heaviest-first work items and their count);
// tile_counter: a zeroed word.  batch: records staged per batch, 128, 256 or 512.  n_views
// images of cam's size, one after the other in rgb (and t_out); tile ids are (view, tile).
// tk, pair_vals: the sorted pair keys (tile id and in-tile box, see kPairTileMask) and values.
// mode 0: two-phase blend (record-parallel alpha test into per-pixel masks, then pixel-parallel
// compositing); mode 1: batches staged by bulk copies and composited by warps over row pairs.  The
// image is the same bit for bit.
cudaError_t launch_blend(const uint2* ranges, uint32_t* items, uint32_t* tile_counter, const uint32_t* tk,
                         const uint32_t* pair_vals, const float4* rec, uint32_t cap_slots, const CamConst& cam, float* rgb, float* t_out,
                         unsigned long long* work, uint32_t* frame, uint32_t* sticky, uint32_t split_pairs,
                         int batch, int mode, int n_views, int sm_count, cudaStream_t st);

}  // namespace v3dg
