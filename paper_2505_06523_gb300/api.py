"""Python front end of libv3dg.so: a context object that marshals arrays into the C ABI.

Device memory the library asks for is served by PyTorch's caching allocator, and work is enqueued
on PyTorch's current CUDA stream.  No computation of the path happens here.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as N


def camera_struct(cam) -> N.v3dg_camera:
    """C camera from an object with world_to_cam (3x4), fx, fy, cx, cy, width, height, near."""
    c = N.v3dg_camera()
    w = np.ascontiguousarray(np.asarray(cam.world_to_cam, np.float64).reshape(12))
    for i in range(12):
        c.world_to_cam[i] = float(w[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_z = float(getattr(cam, "near", 0.01))
    return c


def hierarchy_struct(asset):
    """C descriptor of an asset (numpy arrays as in the ABI); returns (desc, arrays kept alive)."""
    keep = {
        "means": np.ascontiguousarray(asset.means, np.float32),
        "log_scales": np.ascontiguousarray(asset.log_scales, np.float32),
        "quats": np.ascontiguousarray(asset.quats, np.float32),
        "opacity": np.ascontiguousarray(asset.opacity, np.float32),
        "sh": np.ascontiguousarray(asset.sh, np.float32),
        "node_first": np.ascontiguousarray(asset.node_first, np.uint32),
        "node_count": np.ascontiguousarray(asset.node_count, np.uint32),
        "node_level": np.ascontiguousarray(asset.node_level, np.uint8),
        "node_parent": np.ascontiguousarray(asset.node_parent, np.int32),
        "own_sphere": np.ascontiguousarray(asset.own_sphere, np.float32),
    }
    n = keep["means"].shape[0]
    coeffs = keep["sh"].reshape(n, -1, 3).shape[1]
    degree = int(round(coeffs ** 0.5)) - 1
    d = N.v3dg_hierarchy_desc()
    d.n_gauss, d.n_nodes, d.sh_degree = n, keep["node_first"].shape[0], degree
    for k, v in keep.items():
        setattr(d, k, v.ctypes.data)
    d.gaussians_per_group = int(getattr(asset, "gaussians_per_group", 256))
    return d, keep


class TorchAllocator:
    """Serves the library's device allocations from PyTorch's caching allocator."""

    def __init__(self, device):
        import torch
        self._torch = torch
        self.device = device
        self.blocks = {}
        self._alloc_cb = N.ALLOC_FN(self._alloc)
        self._free_cb = N.FREE_FN(self._free)
        self.struct = N.v3dg_allocator(self._alloc_cb, self._free_cb, None)

    def _alloc(self, nbytes, _user):
        try:
            t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device=self.device)
        except Exception:  # out of memory: the library reports V3DG_ENOMEM
            return None
        p = t.data_ptr()
        self.blocks[p] = t
        return p

    def _free(self, ptr, _user):
        self.blocks.pop(ptr, None)


class Context:
    """One library context on one GPU (v3dg_create ... v3dg_destroy)."""

    def __init__(self, device: int = 0, torch_memory: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available: the V3DG path has no CPU implementation")
        self._torch = torch
        self.device = torch.device("cuda", device)
        self._allocator = TorchAllocator(self.device) if torch_memory else None
        self.ctx = N.v3dg_create(device, self._allocator.struct if self._allocator else None)
        self.stream = torch.cuda.current_stream(self.device)
        N.v3dg_set_stream(self.ctx, self.stream.cuda_stream)
        self.cam = None
        self._requests = {}   # ticket -> output buffers kept alive until poll reports it

    # -- lifetime
    def close(self):
        if getattr(self, "ctx", None):
            N.v3dg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- scene
    def set_option(self, option: int, value: int):
        N.v3dg_set_option(self.ctx, option, int(value))

    def load_hierarchy(self, asset) -> int:
        desc, keep = hierarchy_struct(asset)
        aid = N.v3dg_load_hierarchy(self.ctx, desc)
        del keep
        return aid

    def set_instances(self, inst):
        n = int(len(inst.asset))
        a = np.ascontiguousarray(inst.asset, np.uint32)
        r = np.ascontiguousarray(np.asarray(inst.rot, np.float64).reshape(n, 9))
        t = np.ascontiguousarray(np.asarray(inst.trans, np.float64).reshape(n, 3))
        s = np.ascontiguousarray(inst.scale, np.float64)
        N.v3dg_set_instances(self.ctx, n, a.ctypes.data, r.ctypes.data, t.ctypes.data, s.ctypes.data)

    # -- frame
    def select(self, cam, tau_px: float):
        self.cam = cam
        self.n_views = 1
        N.v3dg_select(self.ctx, camera_struct(cam), float(tau_px))

    def select_views(self, cams, tau_px: float):
        """Several cameras (same image size and intrinsics) in one batch of launches; the next
        render returns (n_views, h, w, 3)."""
        self.cam = cams[0]
        self.n_views = len(cams)
        N.v3dg_select_views(self.ctx, [camera_struct(c) for c in cams], float(tau_px))

    def render(self, rgb=None, T=None, want_T: bool = False):
        """Render into torch tensors on the device; returns (rgb (h, w, 3), T (h, w) or None), or
        (n_views, h, w, 3) and (n_views, h, w) after select_views."""
        torch = self._torch
        h, w = int(self.cam.height), int(self.cam.width)
        lead = (self.n_views,) if getattr(self, "n_views", 1) > 1 else ()
        if rgb is None:
            rgb = torch.empty(lead + (h, w, 3), dtype=torch.float32, device=self.device)
        if T is None and want_T:
            T = torch.empty(lead + (h, w), dtype=torch.float32, device=self.device)
        N.v3dg_render(self.ctx, rgb.data_ptr(), T.data_ptr() if T is not None else None)
        return rgb, T

    def render_host(self, rgb: np.ndarray | None = None, T: np.ndarray | None = None, want_T: bool = False):
        h, w = int(self.cam.height), int(self.cam.width)
        lead = (self.n_views,) if getattr(self, "n_views", 1) > 1 else ()
        if rgb is None:
            rgb = np.empty(lead + (h, w, 3), np.float32)
        if T is None and want_T:
            T = np.empty(lead + (h, w), np.float32)
        N.v3dg_render_host(self.ctx, rgb.ctypes.data, T.ctypes.data if T is not None else None)
        return rgb, T

    def frame_stats(self) -> dict:
        return N.v3dg_frame_stats(self.ctx)

    def stage_times(self, n: int = 7):
        ms = (ctypes.c_float * n)()
        launches = N.v3dg_stage_times(self.ctx, ctypes.addressof(ms), n)
        return list(ms), launches

    def launches(self) -> int:
        return N.v3dg_stage_times(self.ctx, None, 0)

    # -- parity read-back
    def get_cut(self) -> np.ndarray:
        n = N.v3dg_get_cut(self.ctx, None, 0)
        out = np.empty((max(n, 1), 2), np.uint32)
        n = N.v3dg_get_cut(self.ctx, out.ctypes.data, n)
        return out[:n]

    def get_projected(self) -> dict:
        n = N.v3dg_get_projected(self.ctx, 0, {})
        out = {"inst": np.empty(n, np.uint32), "local": np.empty(n, np.uint32), "u": np.empty((n, 2), np.float32),
               "conic": np.empty((n, 3), np.float32), "opacity": np.empty(n, np.float32),
               "rgb": np.empty((n, 3), np.float32), "depth_key": np.empty(n, np.uint32),
               "rect": np.empty((n, 4), np.int32)}
        if n:
            N.v3dg_get_projected(self.ctx, n, {k: v.ctypes.data for k, v in out.items()})
        return out

    def get_pairs(self) -> dict:
        n = N.v3dg_get_pairs(self.ctx, 0, {})
        out = {k: np.empty(n, np.uint32) for k in ("tile", "depth_key", "inst", "local")}
        if n:
            N.v3dg_get_pairs(self.ctx, n, {k: v.ctypes.data for k, v in out.items()})
        return out

    def tile_ranges(self) -> np.ndarray:
        n = N.v3dg_get_tile_ranges(self.ctx, None, 0)
        out = np.empty((n, 2), np.uint32)
        if n:
            N.v3dg_get_tile_ranges(self.ctx, out.ctypes.data, n)
        return out

    def autotune_blend(self) -> dict:
        """Time the last frame's blend with every kernel variant, batch size and split threshold
        and keep the fastest (v3dg_autotune_blend)."""
        m, b, sp, ms = N.v3dg_autotune_blend(self.ctx)
        return {"mode": m, "batch": b, "split_pairs": sp, "ms": ms}

    def release_buffers(self) -> int:
        """Release the frame buffers (v3dg_release_buffers); returns the bytes released.  PyTorch's
        caching allocator keeps the blocks until torch.cuda.empty_cache()."""
        return N.v3dg_release_buffers(self.ctx)

    def check_wait(self, spin_limit: int, predecessor_publishes: bool) -> int:
        """The bounded-wait diagnostic (v3dg_check_wait); raises V3dgError(V3DG_ETIMEOUT) when the
        look-back gives up."""
        return N.v3dg_check_wait(self.ctx, spin_limit, predecessor_publishes)

    # -- serving
    def server_start(self, slots: int = 4, hbm_budget: int = 0):
        N.v3dg_server_start(self.ctx, int(slots), int(hbm_budget))
        self._requests = {}

    def server_stop(self):
        N.v3dg_server_stop(self.ctx)
        self._requests = {}

    def submit(self, inst, cam, tau_px: float, want_T: bool = False, pinned: bool = True) -> int:
        """Queue one frame (its own instances, camera and tolerance); returns its ticket.  The image
        is written into host memory that this object keeps until ``poll`` reports the request."""
        torch = self._torch
        n = int(len(inst.asset))
        a = np.ascontiguousarray(inst.asset, np.uint32)
        r = np.ascontiguousarray(np.asarray(inst.rot, np.float64).reshape(n, 9))
        t = np.ascontiguousarray(np.asarray(inst.trans, np.float64).reshape(n, 3))
        s = np.ascontiguousarray(inst.scale, np.float64)
        h, w = int(cam.height), int(cam.width)
        rgb = torch.empty((h, w, 3), dtype=torch.float32, pin_memory=pinned)
        T = torch.empty((h, w), dtype=torch.float32, pin_memory=pinned) if want_T else None
        req = N.v3dg_request(n_instances=n, out_on_device=0, asset_id=a.ctypes.data, rot=r.ctypes.data,
                             trans=t.ctypes.data, scale=s.ctypes.data, camera=camera_struct(cam),
                             tau_px=float(tau_px), rgb_out=rgb.data_ptr(),
                             t_out=T.data_ptr() if T is not None else None)
        ticket = N.v3dg_submit(self.ctx, req)
        self._requests[ticket] = (rgb, T)
        return ticket

    def poll(self, ticket: int, timeout_us: int = 0):
        """(record, rgb (h, w, 3) numpy, T or None) once request `ticket` is done, else None."""
        rec = N.v3dg_poll(self.ctx, int(ticket), int(timeout_us))
        if rec is None:
            return None
        rgb, T = self._requests.pop(ticket)
        if rec["status"] != N.V3DG_OK:
            raise N.V3dgError(rec["status"], f"request {ticket} failed")
        return rec, rgb.numpy(), (T.numpy() if T is not None else None)

    def sort_pairs(self, keys, vals, begin_bit: int = 0, end_bit: int = 32):
        """In-place stable radix sort of int32/uint32 CUDA tensors keys, vals (same length)."""
        assert keys.is_cuda and vals.is_cuda and keys.numel() == vals.numel()
        assert keys.element_size() == 4 and vals.element_size() == 4 and keys.is_contiguous() and vals.is_contiguous()
        N.v3dg_sort_pairs(self.ctx, keys.data_ptr(), vals.data_ptr(), keys.numel(), begin_bit, end_bit)
