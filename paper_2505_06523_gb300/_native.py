"""ctypes binding of libv3dg.so (declarations in include/v3dg.h).

Argument marshalling only: every step of the path runs in the library's CUDA kernels.  The
functions keep the C names; a non-zero status raises ``V3dgError`` with the library's message.
There is no fallback: if libv3dg.so is missing or no GPU is present, the calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libv3dg.so")

V3DG_OK, V3DG_EINVAL, V3DG_ENOMEM, V3DG_ECUDA, V3DG_EBUSY, V3DG_ETIMEOUT, V3DG_EOVERFLOW, V3DG_ENOTFOUND = range(8)
STATUS_NAMES = ["V3DG_OK", "V3DG_EINVAL", "V3DG_ENOMEM", "V3DG_ECUDA", "V3DG_EBUSY", "V3DG_ETIMEOUT",
                "V3DG_EOVERFLOW", "V3DG_ENOTFOUND"]
V3DG_OPT_SYNC_CHECK = 1
V3DG_OPT_STAGE_TIMING = 2
V3DG_OPT_CAP_NODES = 3
V3DG_OPT_CAP_PAIRS = 4
V3DG_OPT_COUNT_WORK = 5
V3DG_OPT_SPLIT_PAIRS = 6
V3DG_OPT_ATTR_FP16 = 7
V3DG_OPT_SELECT_TOPDOWN = 8
V3DG_OPT_BLEND_BATCH = 9
V3DG_OPT_GRAPHS = 10
V3DG_OPT_BLEND_MODE = 11
V3DG_OPT_SERVE_MERGE = 12
V3DG_OPT_PROJECT_ORDER = 13


class V3dgError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class v3dg_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


class v3dg_camera(ctypes.Structure):
    _fields_ = [("world_to_cam", ctypes.c_double * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("near_z", ctypes.c_float)]


class v3dg_hierarchy_desc(ctypes.Structure):
    _fields_ = [("n_gauss", ctypes.c_uint32), ("n_nodes", ctypes.c_uint32), ("sh_degree", ctypes.c_uint32),
                ("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("node_first", ctypes.c_void_p),
                ("node_count", ctypes.c_void_p), ("node_level", ctypes.c_void_p), ("node_parent", ctypes.c_void_p),
                ("own_sphere", ctypes.c_void_p), ("gaussians_per_group", ctypes.c_uint32)]


class v3dg_stats(ctypes.Structure):
    _fields_ = [("cut_nodes", ctypes.c_uint64), ("cut_gaussians", ctypes.c_uint64),
                ("render_nodes", ctypes.c_uint64), ("visible", ctypes.c_uint64), ("pairs", ctypes.c_uint64),
                ("overflow", ctypes.c_uint32), ("timeout", ctypes.c_uint32),
                ("blend_evals", ctypes.c_uint64), ("blend_contribs", ctypes.c_uint64),
                ("conic_fp64", ctypes.c_uint64), ("render_clusters", ctypes.c_uint64)]


class v3dg_request(ctypes.Structure):
    _fields_ = [("n_instances", ctypes.c_uint32), ("out_on_device", ctypes.c_int32), ("asset_id", ctypes.c_void_p),
                ("rot", ctypes.c_void_p), ("trans", ctypes.c_void_p), ("scale", ctypes.c_void_p),
                ("camera", v3dg_camera), ("tau_px", ctypes.c_float), ("rgb_out", ctypes.c_void_p),
                ("t_out", ctypes.c_void_p)]


class v3dg_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batch_views", ctypes.c_uint32), ("submit_ms", ctypes.c_double),
                ("start_ms", ctypes.c_double), ("done_ms", ctypes.c_double), ("visible", ctypes.c_uint64),
                ("pairs", ctypes.c_uint64)]


_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_I32 = ctypes.c_int
_F32 = ctypes.c_float

# name -> (restype, argtypes); every name here is declared in include/v3dg.h
SIGNATURES = {
    "v3dg_create": (_I32, [_I32, ctypes.POINTER(v3dg_allocator), ctypes.POINTER(_P)]),
    "v3dg_destroy": (None, [_P]),
    "v3dg_last_error": (ctypes.c_char_p, [_P]),
    "v3dg_set_stream": (_I32, [_P, _P]),
    "v3dg_set_option": (_I32, [_P, _I32, ctypes.c_int64]),
    "v3dg_load_hierarchy": (_I32, [_P, ctypes.POINTER(v3dg_hierarchy_desc), ctypes.POINTER(_U32)]),
    "v3dg_set_instances": (_I32, [_P, _U32, _P, _P, _P, _P]),
    "v3dg_select": (_I32, [_P, ctypes.POINTER(v3dg_camera), _F32]),
    "v3dg_select_views": (_I32, [_P, ctypes.POINTER(v3dg_camera), _U32, _F32]),
    "v3dg_render": (_I32, [_P, _P, _P]),
    "v3dg_render_host": (_I32, [_P, _P, _P]),
    "v3dg_frame_stats": (_I32, [_P, ctypes.POINTER(v3dg_stats)]),
    "v3dg_get_cut": (_I32, [_P, _P, _U64, ctypes.POINTER(_U64)]),
    "v3dg_get_projected": (_I32, [_P, _U64, ctypes.POINTER(_U64), _P, _P, _P, _P, _P, _P, _P, _P]),
    "v3dg_get_pairs": (_I32, [_P, _U64, ctypes.POINTER(_U64), _P, _P, _P, _P]),
    "v3dg_get_tile_ranges": (_I32, [_P, _P, _U64, ctypes.POINTER(_U64)]),
    "v3dg_stage_times": (_I32, [_P, _P, _I32, ctypes.POINTER(_U64)]),
    "v3dg_autotune_blend": (_I32, [_P, ctypes.POINTER(_U32), ctypes.POINTER(_U32), ctypes.POINTER(_U32),
                                   ctypes.POINTER(_F32)]),
    "v3dg_sort_pairs": (_I32, [_P, _P, _P, _U64, _I32, _I32]),
    "v3dg_sort_pairs_noalloc": (_I32, [_P, _P, _U64, _I32, _I32, _P]),
    "v3dg_check_wait": (_I32, [_P, _U32, _I32, ctypes.POINTER(_U32)]),
    "v3dg_release_buffers": (_I32, [_P, ctypes.POINTER(_U64)]),
    "v3dg_server_start": (_I32, [_P, _I32, _U64]),
    "v3dg_server_stop": (_I32, [_P]),
    "v3dg_submit": (_I32, [_P, ctypes.POINTER(v3dg_request), ctypes.POINTER(_U64)]),
    "v3dg_poll": (_I32, [_P, _U64, _U32, ctypes.POINTER(v3dg_result)]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libv3dg.so (built in-tree by ``paper_2505_06523_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_2505_06523_gb300.build.build() first")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _check(ctx, status: int) -> None:
    if status != V3DG_OK:
        msg = lib().v3dg_last_error(ctx)
        raise V3dgError(status, msg.decode() if msg else "")


# ----------------------------------------------------------------------------- C-named wrappers


def v3dg_create(device: int = 0, allocator: v3dg_allocator | None = None):
    out = _P()
    st = lib().v3dg_create(device, ctypes.byref(allocator) if allocator is not None else None, ctypes.byref(out))
    if st != V3DG_OK:
        raise V3dgError(st, f"v3dg_create(device={device}) failed")
    return out


def v3dg_destroy(ctx) -> None:
    lib().v3dg_destroy(ctx)


def v3dg_last_error(ctx) -> str:
    m = lib().v3dg_last_error(ctx)
    return m.decode() if m else ""


def v3dg_set_stream(ctx, stream_ptr: int) -> None:
    _check(ctx, lib().v3dg_set_stream(ctx, _P(stream_ptr)))


def v3dg_set_option(ctx, option: int, value: int) -> None:
    _check(ctx, lib().v3dg_set_option(ctx, option, value))


def v3dg_load_hierarchy(ctx, desc: v3dg_hierarchy_desc) -> int:
    aid = _U32()
    _check(ctx, lib().v3dg_load_hierarchy(ctx, ctypes.byref(desc), ctypes.byref(aid)))
    return aid.value


def v3dg_set_instances(ctx, n: int, asset_ptr: int, rot_ptr: int, trans_ptr: int, scale_ptr: int) -> None:
    _check(ctx, lib().v3dg_set_instances(ctx, n, _P(asset_ptr), _P(rot_ptr), _P(trans_ptr), _P(scale_ptr)))


def v3dg_select(ctx, cam: v3dg_camera, tau_px: float) -> None:
    _check(ctx, lib().v3dg_select(ctx, ctypes.byref(cam), float(tau_px)))


def v3dg_select_views(ctx, cams: list, tau_px: float) -> None:
    arr = (v3dg_camera * len(cams))(*cams)
    _check(ctx, lib().v3dg_select_views(ctx, arr, len(cams), float(tau_px)))


def v3dg_render(ctx, rgb_ptr: int, t_ptr: int | None) -> None:
    _check(ctx, lib().v3dg_render(ctx, _P(rgb_ptr), _P(t_ptr) if t_ptr else None))


def v3dg_render_host(ctx, rgb_ptr: int, t_ptr: int | None) -> None:
    _check(ctx, lib().v3dg_render_host(ctx, _P(rgb_ptr), _P(t_ptr) if t_ptr else None))


def v3dg_frame_stats(ctx) -> dict:
    s = v3dg_stats()
    _check(ctx, lib().v3dg_frame_stats(ctx, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in v3dg_stats._fields_}


def v3dg_get_cut(ctx, out_ptr: int | None, cap: int) -> int:
    n = _U64()
    _check(ctx, lib().v3dg_get_cut(ctx, _P(out_ptr) if out_ptr else None, cap, ctypes.byref(n)))
    return n.value


def v3dg_get_projected(ctx, cap: int, ptrs: dict) -> int:
    n = _U64()
    names = ["inst", "local", "u", "conic", "opacity", "rgb", "depth_key", "rect"]
    args = [_P(ptrs[k]) if ptrs.get(k) else None for k in names]
    _check(ctx, lib().v3dg_get_projected(ctx, cap, ctypes.byref(n), *args))
    return n.value


def v3dg_get_pairs(ctx, cap: int, ptrs: dict) -> int:
    n = _U64()
    names = ["tile", "depth_key", "inst", "local"]
    args = [_P(ptrs[k]) if ptrs.get(k) else None for k in names]
    _check(ctx, lib().v3dg_get_pairs(ctx, cap, ctypes.byref(n), *args))
    return n.value


def v3dg_get_tile_ranges(ctx, out_ptr: int | None, cap: int) -> int:
    n = _U64()
    _check(ctx, lib().v3dg_get_tile_ranges(ctx, _P(out_ptr) if out_ptr else None, cap, ctypes.byref(n)))
    return n.value


def v3dg_stage_times(ctx, ms_ptr: int | None, n: int) -> int:
    launches = _U64()
    _check(ctx, lib().v3dg_stage_times(ctx, _P(ms_ptr) if ms_ptr else None, n, ctypes.byref(launches)))
    return launches.value


def v3dg_autotune_blend(ctx) -> tuple[int, int, int, float]:
    m, b, sp, ms = _U32(), _U32(), _U32(), _F32()
    _check(ctx, lib().v3dg_autotune_blend(ctx, ctypes.byref(m), ctypes.byref(b), ctypes.byref(sp), ctypes.byref(ms)))
    return int(m.value), int(b.value), int(sp.value), float(ms.value)


def v3dg_sort_pairs(ctx, keys_ptr: int, vals_ptr: int, n: int, begin_bit: int, end_bit: int) -> None:
    _check(ctx, lib().v3dg_sort_pairs(ctx, _P(keys_ptr), _P(vals_ptr), n, begin_bit, end_bit))


def v3dg_sort_pairs_noalloc(keys_ptr: int, vals_ptr: int, n: int, begin_bit: int, end_bit: int,
                            stream_ptr: int | None = None) -> None:
    st = lib().v3dg_sort_pairs_noalloc(_P(keys_ptr), _P(vals_ptr), n, begin_bit, end_bit,
                                       _P(stream_ptr) if stream_ptr else None)
    if st != V3DG_OK:
        raise V3dgError(st, f"v3dg_sort_pairs_noalloc(n={n}, bits [{begin_bit}, {end_bit}))")


def v3dg_check_wait(ctx, spin_limit: int, predecessor_publishes: bool) -> int:
    p = _U32()
    _check(ctx, lib().v3dg_check_wait(ctx, spin_limit, 1 if predecessor_publishes else 0, ctypes.byref(p)))
    return p.value


def v3dg_release_buffers(ctx) -> int:
    b = _U64()
    _check(ctx, lib().v3dg_release_buffers(ctx, ctypes.byref(b)))
    return b.value


def v3dg_server_start(ctx, slots: int, hbm_budget: int = 0) -> None:
    _check(ctx, lib().v3dg_server_start(ctx, slots, hbm_budget))


def v3dg_server_stop(ctx) -> None:
    _check(ctx, lib().v3dg_server_stop(ctx))


def v3dg_submit(ctx, req: v3dg_request) -> int:
    t = _U64()
    _check(ctx, lib().v3dg_submit(ctx, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def v3dg_poll(ctx, ticket: int, timeout_us: int) -> dict | None:
    """The completion record of `ticket`, or None while it is not done (V3DG_EBUSY)."""
    r = v3dg_result()
    st = lib().v3dg_poll(ctx, ticket, timeout_us, ctypes.byref(r))
    if st == V3DG_EBUSY:
        return None
    _check(ctx, st)
    return {f: getattr(r, f) for f, _ in v3dg_result._fields_ if f != "reserved"}
