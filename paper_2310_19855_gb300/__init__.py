"""Python binding of libgi.so: the world-space radiance cache and screen-probe
stage of GI-1.0 on sm_103a.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  The functions keep the C names (gi_cache_create, gi_cache_update,
...); device buffers are passed as integers (device pointers) or as objects
with a data_ptr() method (torch tensors), streams as integers (cudaStream_t)
or objects with a cuda_stream attribute.  If the library is not built this
module raises on first use; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB_PATH, build  # noqa: F401

# ---------------------------------------------------------------- constants (gi.h)
GI_OK, GI_ERR_INVALID_ARG, GI_ERR_OOM, GI_ERR_CUDA, GI_ERR_TIMEOUT, GI_ERR_DEVICE_FAULT, GI_ERR_CAPACITY = range(7)
GI_WARN_DROPPED = 100
GI_SLOT_MISS = 0xFFFFFFFE
GI_SLOT_NONE = 0xFFFFFFFF
GI_SLOT_FAR = 0xFFFFFFFD
GI_PROBE_NONE = 0xFFFFFFFF
GI_INTERP_OK, GI_INTERP_RELAXED, GI_INTERP_NONE, GI_INTERP_SKY = 0, 1, 2, 3
GI_KEY_DIR_NORMAL, GI_KEY_DIR_RAY = 0, 1
GI_RESOLVED_F32, GI_RESOLVED_F16 = 0, 1
GI_FIRST_TOUCH_AUTO, GI_FIRST_TOUCH_LIST, GI_FIRST_TOUCH_BITMAP = 0, 1, 2
GI_MERGE_NONE, GI_MERGE_WARP = 0, 1
GI_MAX_MIPS = 16
GI_SH_STRIDE = 28
GI_NOALLOC_LOG2_SLOTS = 18
GI_NOALLOC_MAX_RECORDS = 131072

GI_NRC_LEVELS = 16
GI_NRC_FEATURES = 2
GI_NRC_HIDDEN = 64
GI_NRC_OUTPUTS = 3
GI_NRC_MAX_BATCH = 1 << 20

c_u32, c_u64, c_f32, c_f64, c_vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_float, ctypes.c_double, ctypes.c_void_p


class gi_cache_config(ctypes.Structure):
    _fields_ = [("log2_slots", c_u32), ("cell_size", c_f32), ("num_lods", c_u32), ("alpha", c_f32),
                ("evict_frames", c_u32), ("max_probe", c_u32), ("key_dir", c_u32), ("resolved_format", c_u32),
                ("rebuild_load", c_f32), ("first_touch", c_u32), ("tiles", c_u32), ("min_samples", c_u32),
                ("merge", c_u32)]


class gi_view(ctypes.Structure):
    _fields_ = [("frame", c_u32), ("width", c_u32), ("height", c_u32), ("cam_pos", c_f32 * 3),
                ("cam_fwd", c_f32 * 3), ("cam_right", c_f32 * 3), ("cam_up", c_f32 * 3), ("fov_y", c_f64)]


class gi_hits(ctypes.Structure):
    _fields_ = [("pos", c_vp * 3), ("nrm", c_vp * 3), ("rad", c_vp * 3), ("ray_len", c_vp), ("ray_dir", c_vp * 3),
                ("n", c_u64)]


class gi_gbuffer(ctypes.Structure):
    _fields_ = [("nd", c_vp), ("width", c_u32), ("height", c_u32)]


class gi_probe_layout(ctypes.Structure):
    _fields_ = [("tiles_x", c_u32), ("tiles_y", c_u32), ("num_probes", c_u32), ("mip_count", c_u32),
                ("mip_w", c_u32 * GI_MAX_MIPS), ("mip_h", c_u32 * GI_MAX_MIPS), ("mip_offset", c_u32 * GI_MAX_MIPS),
                ("mask_words", c_u32)]


class gi_probes(ctypes.Structure):
    _fields_ = [("layout", gi_probe_layout), ("mask", c_vp), ("pos", c_vp), ("nrm", c_vp), ("sh", c_vp)]


class gi_cache_stats_t(ctypes.Structure):
    _fields_ = [("slots", c_u64), ("occupied", c_u64), ("live", c_u64), ("touched", c_u64), ("dropped", c_u64),
                ("clamped", c_u64), ("rebuilds", c_u64), ("updates", c_u64), ("resolves", c_u64),
                ("max_probe_seen", c_u32), ("error_word", c_u32), ("last_resolved", ctypes.c_int64)]


class gi_cell(ctypes.Structure):
    _fields_ = [("identity", c_u64), ("sum", c_u64 * 3), ("count", c_u32), ("stamp", c_u32), ("value", c_f32 * 3),
                ("slot", c_u32)]


GI_TILE_VALUES = 85


class gi_tile(ctypes.Structure):
    _fields_ = [("identity", c_u64), ("slot", c_u32), ("live", c_u32), ("value", c_f32 * (3 * GI_TILE_VALUES)),
                ("samples", c_u32 * GI_TILE_VALUES)]


class gi_query(ctypes.Structure):
    _fields_ = [("slot_ids", c_vp), ("points", ctypes.POINTER(gi_hits)), ("view", ctypes.POINTER(gi_view)),
                ("n", c_u64), ("env", c_f32 * 3)]


class gi_batch_tuning(ctypes.Structure):
    _fields_ = [("update_records_per_block", c_u32), ("resolve_blocks_per_sm", c_u32), ("integrate_threads", c_u32)]


class gi_batch_view(ctypes.Structure):
    _fields_ = [("cache", c_vp), ("view", gi_view), ("resolve_frame", c_u32), ("hits", gi_hits), ("gbuf", gi_gbuffer),
                ("probes", gi_probes),
                ("slot_ids", c_vp), ("irradiance", c_vp), ("env", c_f32 * 3)]


class gi_nrc_config(ctypes.Structure):
    _fields_ = [("log2_table", c_u32), ("resolution", c_u32 * GI_NRC_LEVELS), ("aabb_lo", c_f32 * 3),
                ("aabb_hi", c_f32 * 3), ("lr", c_f32), ("beta1", c_f32), ("beta2", c_f32), ("adam_eps", c_f32),
                ("loss_eps", c_f32), ("batch", c_u32), ("train_steps", c_u32), ("max_records", c_u32),
                ("max_queries", c_u32),
                ("trust", c_f32), ("query_lod", c_u32), ("seed", c_u64)]


class gi_points(ctypes.Structure):
    _fields_ = [("pos", c_vp * 3), ("nrm", c_vp * 3), ("n", c_u32)]


class gi_nrc_stats_t(ctypes.Structure):
    _fields_ = [("steps", c_u64), ("loss", c_f32), ("judged_error", c_f32), ("trusted", c_u32), ("queries", c_u32)]


CELL_DTYPE = np.dtype([("identity", "<u8"), ("sum", "<u8", (3,)), ("count", "<u4"), ("stamp", "<u4"),
                       ("value", "<f4", (3,)), ("slot", "<u4")])
assert CELL_DTYPE.itemsize == ctypes.sizeof(gi_cell)
TILE_DTYPE = np.dtype([("identity", "<u8"), ("slot", "<u4"), ("live", "<u4"), ("value", "<f4", (GI_TILE_VALUES, 3)),
                       ("samples", "<u4", (GI_TILE_VALUES,))])
assert TILE_DTYPE.itemsize == ctypes.sizeof(gi_tile)

# ---------------------------------------------------------------- library
_LIB = None


class GiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


def lib() -> ctypes.CDLL:
    """The loaded libgi.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgi.so is not built ({LIB_PATH}); run paper_2310_19855_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "gi_last_error": (ctypes.c_char_p, []),
            "gi_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "gi_version": (c_u32, []),
            "gi_cache_create": (ctypes.c_int, [ctypes.POINTER(gi_cache_config), ctypes.POINTER(c_vp)]),
            "gi_cache_destroy": (ctypes.c_int, [c_vp]),
            "gi_cache_update": (ctypes.c_int, [c_vp, ctypes.POINTER(gi_hits), ctypes.POINTER(gi_view), c_vp, c_vp]),
            "gi_cache_resolve": (ctypes.c_int, [c_vp, c_u32, c_vp]),
            "gi_cache_query": (ctypes.c_int, [c_vp, ctypes.POINTER(gi_query), c_vp, c_vp]),
            "gi_cache_stats": (ctypes.c_int, [c_vp, ctypes.POINTER(gi_cache_stats_t), c_vp]),
            "gi_cache_export": (ctypes.c_int, [c_vp, c_vp, c_u64, ctypes.POINTER(c_u64), c_vp]),
            "gi_cache_export_tiles": (ctypes.c_int, [c_vp, c_vp, c_u64, ctypes.POINTER(c_u64), c_vp]),
            "gi_probes_layout": (ctypes.c_int, [c_u32, c_u32, ctypes.POINTER(gi_probe_layout)]),
            "gi_probes_spawn": (ctypes.c_int, [ctypes.POINTER(gi_gbuffer), ctypes.POINTER(gi_view),
                                               ctypes.POINTER(gi_probes), c_vp]),
            "gi_probes_integrate": (ctypes.c_int, [c_vp, ctypes.POINTER(gi_probes), c_vp, c_u32,
                                                   ctypes.POINTER(c_f32), c_vp]),
            "gi_probes_interpolate": (ctypes.c_int, [ctypes.POINTER(gi_gbuffer), ctypes.POINTER(gi_view),
                                                     ctypes.POINTER(gi_probes), c_vp, c_vp]),
            "gi_cell_moments": (ctypes.c_int, [ctypes.POINTER(c_f64)]),
            "gi_probes_gather": (ctypes.c_int, [c_vp, ctypes.POINTER(gi_probes), c_vp, c_vp, c_u32,
                                                ctypes.POINTER(c_f32), c_vp, c_vp]),
            "gi_probes_filter": (ctypes.c_int, [ctypes.POINTER(gi_probes), ctypes.POINTER(gi_view), c_vp, c_vp, c_u32,
                                                c_vp]),
            "gi_probes_project": (ctypes.c_int, [ctypes.POINTER(gi_probes), c_vp, c_vp]),
            "gi_probes_spawn_upscaled": (ctypes.c_int, [ctypes.POINTER(gi_gbuffer), ctypes.POINTER(gi_view), c_u32,
                                                        c_u32, ctypes.POINTER(gi_probes), c_vp]),
            "gi_probes_reproject": (ctypes.c_int, [ctypes.POINTER(gi_gbuffer), ctypes.POINTER(gi_view), c_vp,
                                                   ctypes.POINTER(gi_probes), ctypes.POINTER(gi_probes), c_vp, c_vp]),
            "gi_probes_gather_temporal": (ctypes.c_int, [c_vp, ctypes.POINTER(gi_gbuffer), ctypes.POINTER(gi_view),
                                                         c_u32, ctypes.POINTER(gi_probes), c_vp, c_vp, c_u32, c_vp,
                                                         c_vp, c_vp, ctypes.POINTER(c_f32), c_vp]),
            "gi_batch_create": (ctypes.c_int, [c_u32, c_u32, ctypes.POINTER(gi_batch_tuning), ctypes.POINTER(c_vp)]),
            "gi_batch_set_tuning": (ctypes.c_int, [c_vp, ctypes.POINTER(gi_batch_tuning)]),
            "gi_batch_frame": (ctypes.c_int, [c_vp, ctypes.POINTER(gi_batch_view), c_u32, c_vp]),
            "gi_batch_destroy": (ctypes.c_int, [c_vp]),
            "gi_batch_set_surrogate": (ctypes.c_int, [c_vp, c_vp]),
            "gi_batch_set_view_surrogates": (ctypes.c_int, [c_vp, ctypes.POINTER(c_vp)]),
            "gi_cell_means_noalloc": (ctypes.c_int, [ctypes.POINTER(gi_hits), ctypes.POINTER(gi_view), c_f32, c_u32,
                                                     c_u32, ctypes.POINTER(c_f32), c_vp, c_vp, c_vp]),
            "gi_nrc_config_defaults": (ctypes.c_int, [ctypes.POINTER(gi_nrc_config)]),
            "gi_cache_route_far": (ctypes.c_int, [c_vp, c_vp, c_u32]),
            "gi_nrc_create": (ctypes.c_int, [ctypes.POINTER(gi_nrc_config), ctypes.POINTER(c_vp)]),
            "gi_nrc_destroy": (ctypes.c_int, [c_vp]),
            "gi_nrc_set_params": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
            "gi_nrc_get_params": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
            "gi_nrc_set_gradients": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
            "gi_nrc_get_gradients": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
            "gi_nrc_infer": (ctypes.c_int, [c_vp, ctypes.POINTER(gi_points), c_vp, c_vp]),
            "gi_nrc_backward": (ctypes.c_int, [c_vp, ctypes.POINTER(gi_points), ctypes.POINTER(c_vp), c_vp, c_u32,
                                               c_vp]),
            "gi_nrc_adam": (ctypes.c_int, [c_vp, c_vp]),
            "gi_nrc_set_learning_rate": (ctypes.c_int, [c_vp, c_f32]),
            "gi_nrc_train_frame": (ctypes.c_int, [c_vp, c_vp, ctypes.POINTER(gi_hits), c_vp, c_u32, c_vp]),
            "gi_nrc_query_frame": (ctypes.c_int, [c_vp, c_vp, ctypes.POINTER(gi_hits), c_vp,
                                                  ctypes.POINTER(gi_view), c_vp]),
            "gi_nrc_answers": (ctypes.c_int, [c_vp, c_vp, c_vp, c_u32, ctypes.POINTER(c_u32), c_vp]),
            "gi_probes_integrate_nrc": (ctypes.c_int, [c_vp, c_vp, ctypes.POINTER(gi_probes), c_vp, c_u32,
                                                       ctypes.POINTER(c_f32), c_vp]),
            "gi_nrc_stats": (ctypes.c_int, [c_vp, ctypes.POINTER(gi_nrc_stats_t), c_vp]),
            "gi_diag_update_atomics": (ctypes.c_int, [c_vp, c_u64, c_u32, c_u32, c_vp, c_vp, c_vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"expected a device pointer or a tensor, got {type(x)}")


def _stream(s) -> int | None:
    if s is None or s == 0:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def check(status: int, what: str, allow=(GI_OK,)) -> int:
    if status in allow:
        return status
    L = lib()
    raise GiError(status, f"{what}: {L.gi_status_string(status).decode()}: {L.gi_last_error().decode()}")


# ---------------------------------------------------------------- marshalling helpers
def make_view(frame: int, width: int, height: int, cam_pos, cam_fwd, cam_right, cam_up, fov_y: float) -> gi_view:
    v = gi_view()
    v.frame, v.width, v.height = int(frame), int(width), int(height)
    for name, val in (("cam_pos", cam_pos), ("cam_fwd", cam_fwd), ("cam_right", cam_right), ("cam_up", cam_up)):
        arr = getattr(v, name)
        for k in range(3):
            arr[k] = float(np.float32(val[k]))
    v.fov_y = float(fov_y)
    return v


def hits_from_planes(planes, n: int) -> gi_hits:
    """gi_hits from a device float32 array of 13 contiguous planes of n records
    (pos xyz, nrm xyz, rad rgb, ray_len, ray_dir xyz) or from 13 plane pointers."""
    h = gi_hits()
    h._keep = planes  # the struct holds raw pointers: keep the arrays alive as long as it lives
    if isinstance(planes, (list, tuple)):
        ptrs = [_ptr(p) for p in planes]
    else:
        base = _ptr(planes)
        ptrs = [base + 4 * k * n for k in range(13)]
    for k in range(3):
        h.pos[k], h.nrm[k], h.rad[k] = ptrs[k], ptrs[3 + k], ptrs[6 + k]
        h.ray_dir[k] = ptrs[10 + k]
    h.ray_len = ptrs[9]
    h.n = int(n)
    return h


def gi_probes_layout(width: int, height: int) -> gi_probe_layout:
    out = gi_probe_layout()
    check(lib().gi_probes_layout(int(width), int(height), ctypes.byref(out)), "gi_probes_layout")
    return out


def make_probes(layout: gi_probe_layout, mask, pos, nrm, sh) -> gi_probes:
    p = gi_probes()
    p.layout = layout
    p.mask, p.pos, p.nrm, p.sh = _ptr(mask), _ptr(pos), _ptr(nrm), _ptr(sh)
    p._keep = (mask, pos, nrm, sh)
    return p


def gi_cell_moments() -> np.ndarray:
    out = (c_f64 * 640)()
    check(lib().gi_cell_moments(out), "gi_cell_moments")
    return np.frombuffer(out, np.float64).reshape(64, 10).copy()


# ---------------------------------------------------------------- entry points (same names as the C ABI)
def gi_cache_create(log2_slots: int, cell_size: float = 0.05, num_lods: int = 4, alpha: float = 0.1,
                    evict_frames: int = 8, max_probe: int = 128, key_dir: int = GI_KEY_DIR_NORMAL,
                    resolved_format: int = GI_RESOLVED_F32, rebuild_load: float = 0.8,
                    first_touch: int = GI_FIRST_TOUCH_AUTO, tiles: bool = False, min_samples: int = 16,
                    merge: int = GI_MERGE_NONE) -> int:
    """tiles=True: two-level cache (8 x 8 cell tiles with MIP levels); log2_slots then counts tiles.
    merge=GI_MERGE_WARP: same-cell hits of a warp merged before the probe and the accumulation."""
    cfg = gi_cache_config(log2_slots, cell_size, num_lods, alpha, evict_frames, max_probe, key_dir,
                          resolved_format, rebuild_load, first_touch, 1 if tiles else 0, min_samples, merge)
    h = c_vp()
    check(lib().gi_cache_create(ctypes.byref(cfg), ctypes.byref(h)), "gi_cache_create")
    return h.value


def gi_cache_destroy(cache: int) -> None:
    check(lib().gi_cache_destroy(cache), "gi_cache_destroy")


def gi_cache_update(cache: int, hits: gi_hits, view: gi_view, slot_ids, stream=None) -> None:
    check(lib().gi_cache_update(cache, ctypes.byref(hits), ctypes.byref(view), _ptr(slot_ids), _stream(stream)),
          "gi_cache_update")


def gi_cache_resolve(cache: int, frame: int, stream=None) -> None:
    check(lib().gi_cache_resolve(cache, int(frame), _stream(stream)), "gi_cache_resolve")


def gi_cache_query(cache: int, out, n: int, slot_ids=None, points: gi_hits | None = None,
                   view: gi_view | None = None, env=(0.0, 0.0, 0.0), stream=None) -> None:
    q = gi_query()
    q.slot_ids = _ptr(slot_ids)
    if points is not None:
        q.points = ctypes.pointer(points)
    if view is not None:
        q.view = ctypes.pointer(view)
    q.n = int(n)
    for k in range(3):
        q.env[k] = float(env[k])
    check(lib().gi_cache_query(cache, ctypes.byref(q), _ptr(out), _stream(stream)), "gi_cache_query")


def gi_cache_stats(cache: int, stream=None) -> dict:
    st = gi_cache_stats_t()
    status = check(lib().gi_cache_stats(cache, ctypes.byref(st), _stream(stream)), "gi_cache_stats",
                   allow=(GI_OK, GI_WARN_DROPPED))
    d = {name: getattr(st, name) for name, _ in gi_cache_stats_t._fields_}
    d["status"] = status
    return d


def gi_cache_export(cache: int, stream=None) -> np.ndarray:
    cnt = c_u64(0)
    check(lib().gi_cache_export(cache, None, 0, ctypes.byref(cnt), _stream(stream)), "gi_cache_export")
    out = np.zeros(cnt.value, CELL_DTYPE)
    if cnt.value:
        check(lib().gi_cache_export(cache, out.ctypes.data, cnt.value, ctypes.byref(cnt), _stream(stream)),
              "gi_cache_export")
    return out


def gi_cache_export_tiles(cache: int, stream=None) -> np.ndarray:
    cnt = c_u64(0)
    check(lib().gi_cache_export_tiles(cache, None, 0, ctypes.byref(cnt), _stream(stream)), "gi_cache_export_tiles")
    out = np.zeros(cnt.value, TILE_DTYPE)
    if cnt.value:
        check(lib().gi_cache_export_tiles(cache, out.ctypes.data, cnt.value, ctypes.byref(cnt), _stream(stream)),
              "gi_cache_export_tiles")
    return out


def gi_probes_spawn(gbuf: gi_gbuffer, view: gi_view, probes: gi_probes, stream=None) -> None:
    check(lib().gi_probes_spawn(ctypes.byref(gbuf), ctypes.byref(view), ctypes.byref(probes), _stream(stream)),
          "gi_probes_spawn")


def gi_probes_integrate(cache: int, probes: gi_probes, slot_ids, rays_per_probe: int, env=(0.0, 0.0, 0.0),
                        stream=None) -> None:
    e = (c_f32 * 3)(*[float(x) for x in env])
    check(lib().gi_probes_integrate(cache, ctypes.byref(probes), _ptr(slot_ids), int(rays_per_probe), e,
                                    _stream(stream)), "gi_probes_integrate")


def gi_probes_interpolate(gbuf: gi_gbuffer, view: gi_view, probes: gi_probes, out, stream=None) -> None:
    check(lib().gi_probes_interpolate(ctypes.byref(gbuf), ctypes.byref(view), ctypes.byref(probes), _ptr(out),
                                      _stream(stream)), "gi_probes_interpolate")


def gi_probes_gather(cache: int, probes: gi_probes, slot_ids, ray_len, rays_per_probe: int, atlas,
                     env=(0.0, 0.0, 0.0), stream=None) -> None:
    """Probe atlas (device float4 per probe and cell: radiance rgb, mean hit distance)."""
    e = (c_f32 * 3)(*[float(x) for x in env])
    check(lib().gi_probes_gather(cache, ctypes.byref(probes), _ptr(slot_ids), _ptr(ray_len), int(rays_per_probe), e,
                                 _ptr(atlas), _stream(stream)), "gi_probes_gather")


def gi_probes_filter(probes: gi_probes, view: gi_view, atlas_in, atlas_out, axis: int, stream=None) -> None:
    """One pass of the probe filter (Algorithm 5) along axis 0 (x) or 1 (y)."""
    check(lib().gi_probes_filter(ctypes.byref(probes), ctypes.byref(view), _ptr(atlas_in), _ptr(atlas_out), int(axis),
                                 _stream(stream)), "gi_probes_filter")


def gi_probes_project(probes: gi_probes, atlas, stream=None) -> None:
    check(lib().gi_probes_project(ctypes.byref(probes), _ptr(atlas), _stream(stream)), "gi_probes_project")


def gi_probes_spawn_upscaled(gbuf: gi_gbuffer, view: gi_view, upscale: int, keep: bool, probes: gi_probes,
                             stream=None) -> None:
    """Spawn with temporal upscale (one fresh probe per spawn tile of 8u x 8u pixels)."""
    check(lib().gi_probes_spawn_upscaled(ctypes.byref(gbuf), ctypes.byref(view), int(upscale), 1 if keep else 0,
                                         ctypes.byref(probes), _stream(stream)), "gi_probes_spawn_upscaled")


def gi_probes_reproject(gbuf: gi_gbuffer, view: gi_view, motion, prev: gi_probes, cur: gi_probes, src,
                        stream=None) -> None:
    """Screen-probe reprojection (Algorithm 1) of prev into cur; src[tile] = source probe index."""
    check(lib().gi_probes_reproject(ctypes.byref(gbuf), ctypes.byref(view), _ptr(motion), ctypes.byref(prev),
                                    ctypes.byref(cur), _ptr(src), _stream(stream)), "gi_probes_reproject")


def gi_probes_gather_temporal(cache: int, gbuf: gi_gbuffer, view: gi_view, upscale: int, probes: gi_probes,
                              slot_ids, ray_len, rays_per_probe: int, src, prev_atlas, atlas, env=(0.0, 0.0, 0.0),
                              stream=None) -> None:
    """The frame's probe atlas: fresh probes gathered and blended by Algorithm 4, reprojected ones carried."""
    e = (c_f32 * 3)(*[float(x) for x in env])
    check(lib().gi_probes_gather_temporal(cache, ctypes.byref(gbuf), ctypes.byref(view), int(upscale),
                                          ctypes.byref(probes), _ptr(slot_ids), _ptr(ray_len), int(rays_per_probe),
                                          _ptr(src), _ptr(prev_atlas), _ptr(atlas), e, _stream(stream)),
          "gi_probes_gather_temporal")


def make_gbuffer(nd, width: int, height: int) -> gi_gbuffer:
    g = gi_gbuffer()
    g.nd, g.width, g.height = _ptr(nd), int(width), int(height)
    g._keep = nd
    return g


def gi_cell_means_noalloc(hits: gi_hits, view: gi_view, out, cell_size: float = 0.05, num_lods: int = 4,
                          key_dir: int = GI_KEY_DIR_NORMAL, env=(0.0, 0.0, 0.0), stats_out=None,
                          stream=None) -> None:
    """Per-record cell means of one batch without any device allocation (see gi.h): for callers
    that cannot call cudaMalloc.  out: device float4[n]; stats_out: optional device int64[2] that
    receives the dropped and clamped hit counts."""
    e = (c_f32 * 3)(*[float(x) for x in env])
    check(lib().gi_cell_means_noalloc(ctypes.byref(hits), ctypes.byref(view), float(cell_size), int(num_lods),
                                      int(key_dir), e, _ptr(out), _ptr(stats_out) if stats_out is not None else None,
                                      _stream(stream)), "gi_cell_means_noalloc")


def gi_diag_update_atomics(slot_ids, n: int, log2_slots: int, scratch, first_touches=None,
                           first_touch: int = GI_FIRST_TOUCH_AUTO, stream=None) -> None:
    """Diagnostics (see gi.h): the update's accumulation alone, in the given form, for these slot
    ids, into the caller's zeroed scratch (2^log2_slots x 32 bytes of accumulators, then in the
    bitmap form 2^log2_slots / 8 bytes of bitmap); first_touches: device uint32 counter (list form)."""
    check(lib().gi_diag_update_atomics(_ptr(slot_ids), int(n), int(log2_slots), int(first_touch), _ptr(scratch),
                                       _ptr(first_touches), _stream(stream)), "gi_diag_update_atomics")


def gi_batch_create(n_views: int, rays_per_probe: int, tuning: gi_batch_tuning | None = None) -> int:
    h = c_vp()
    check(lib().gi_batch_create(int(n_views), int(rays_per_probe), ctypes.byref(tuning) if tuning else None,
                                ctypes.byref(h)), "gi_batch_create")
    return h.value


def gi_batch_set_tuning(batch: int, tuning: gi_batch_tuning) -> None:
    check(lib().gi_batch_set_tuning(batch, ctypes.byref(tuning)), "gi_batch_set_tuning")


def gi_batch_frame(batch: int, views, use_graph: bool = False, stream=None) -> None:
    """views: a ctypes array of gi_batch_view (one entry per view of the batch)."""
    check(lib().gi_batch_frame(batch, views, 1 if use_graph else 0, _stream(stream)), "gi_batch_frame")


def gi_batch_set_surrogate(batch: int, nrc: int | None) -> None:
    check(lib().gi_batch_set_surrogate(batch, nrc), "gi_batch_set_surrogate")


def gi_batch_set_view_surrogates(batch: int, nrcs) -> None:
    """nrcs: one handle (or None) per view of the batch, or None for the plain form."""
    arr = None if nrcs is None else (c_vp * len(nrcs))(*nrcs)
    check(lib().gi_batch_set_view_surrogates(batch, arr), "gi_batch_set_view_surrogates")


def gi_batch_destroy(batch: int) -> None:
    check(lib().gi_batch_destroy(batch), "gi_batch_destroy")


# ---------------------------------------------------------------- learned radiance surrogate
def default_resolutions() -> tuple:
    """The library's default level resolutions (gi_nrc_config_defaults)."""
    c = gi_nrc_config()
    check(lib().gi_nrc_config_defaults(ctypes.byref(c)), "gi_nrc_config_defaults")
    return tuple(int(r) for r in c.resolution)


def make_nrc_config(aabb_lo, aabb_hi, log2_table: int = 19, resolutions=None, lr: float = 1e-2, beta1: float = 0.9,
                    beta2: float = 0.99, adam_eps: float = 1e-15, loss_eps: float = 0.01, batch: int = 65536,
                    train_steps: int = 4, max_records: int = 1 << 22, max_queries: int = 1 << 20, trust: float = 0.05,
                    query_lod: int = 2, seed: int = 1) -> gi_nrc_config:
    """A surrogate configuration: the library's defaults (gi_nrc_config_defaults, which own the level
    resolutions unless `resolutions` is given) with the arguments written over them."""
    c = gi_nrc_config()
    check(lib().gi_nrc_config_defaults(ctypes.byref(c)), "gi_nrc_config_defaults")
    c.log2_table = int(log2_table)
    if resolutions is not None:
        for l in range(GI_NRC_LEVELS):
            c.resolution[l] = int(resolutions[l])
    for a in range(3):
        c.aabb_lo[a] = float(aabb_lo[a])
        c.aabb_hi[a] = float(aabb_hi[a])
    c.lr, c.beta1, c.beta2, c.adam_eps, c.loss_eps = float(lr), float(beta1), float(beta2), float(adam_eps), float(loss_eps)
    c.batch, c.train_steps = int(batch), int(train_steps)
    c.max_records, c.max_queries = int(max_records), int(max_queries)
    c.trust, c.query_lod, c.seed = float(trust), int(query_lod), int(seed)
    return c


def gi_cache_route_far(cache: int, nrc: int | None, far_lod: int) -> None:
    """While nrc is trusted, hits of LOD >= far_lod skip the table (slot id GI_SLOT_FAR) and are
    answered by the network (see gi.h); nrc None or far_lod >= 4 ends the routing."""
    check(lib().gi_cache_route_far(cache, nrc, int(far_lod)), "gi_cache_route_far")


def gi_nrc_create(cfg: gi_nrc_config) -> int:
    h = c_vp()
    check(lib().gi_nrc_create(ctypes.byref(cfg), ctypes.byref(h)), "gi_nrc_create")
    return h.value


def gi_nrc_destroy(nrc: int) -> None:
    check(lib().gi_nrc_destroy(nrc), "gi_nrc_destroy")


def _host_f32(a):
    if a is None:
        return None
    arr = np.ascontiguousarray(a, dtype=np.float32)
    return arr


def gi_nrc_set_params(nrc: int, table=None, w1=None, w2=None, w3=None) -> None:
    """Host float32 arrays: table (16, 2^log2_table, 2), w1 (64, 32), w2 (64, 64), w3 (3, 64); None keeps a part."""
    arrs = [_host_f32(x) for x in (table, w1, w2, w3)]
    check(lib().gi_nrc_set_params(nrc, *[a.ctypes.data if a is not None else None for a in arrs]), "gi_nrc_set_params")


def _get(fn, nrc: int, log2_table: int, what: str):
    table = np.empty((GI_NRC_LEVELS, 1 << log2_table, 2), np.float32)
    w1 = np.empty((GI_NRC_HIDDEN, 2 * GI_NRC_LEVELS), np.float32)
    w2 = np.empty((GI_NRC_HIDDEN, GI_NRC_HIDDEN), np.float32)
    w3 = np.empty((GI_NRC_OUTPUTS, GI_NRC_HIDDEN), np.float32)
    check(fn(nrc, table.ctypes.data, w1.ctypes.data, w2.ctypes.data, w3.ctypes.data), what)
    return table, w1, w2, w3


def gi_nrc_get_params(nrc: int, log2_table: int):
    """(table, w1, w2, w3) float32 master copies."""
    return _get(lib().gi_nrc_get_params, nrc, log2_table, "gi_nrc_get_params")


def gi_nrc_set_gradients(nrc: int, table=None, w1=None, w2=None, w3=None) -> None:
    arrs = [_host_f32(x) for x in (table, w1, w2, w3)]
    check(lib().gi_nrc_set_gradients(nrc, *[a.ctypes.data if a is not None else None for a in arrs]),
          "gi_nrc_set_gradients")


def gi_nrc_get_gradients(nrc: int, log2_table: int):
    return _get(lib().gi_nrc_get_gradients, nrc, log2_table, "gi_nrc_get_gradients")


def make_points(pos_planes, nrm_planes, n: int) -> gi_points:
    """gi_points from device tensors pos (3, n) and nrm (3, n) float32 (contiguous rows)."""
    p = gi_points()
    for a in range(3):
        p.pos[a] = _ptr(pos_planes[a])
        p.nrm[a] = _ptr(nrm_planes[a])
    p.n = int(n)
    p._keep = (pos_planes, nrm_planes)
    return p


def gi_nrc_infer(nrc: int, pts: gi_points, out, stream=None) -> None:
    check(lib().gi_nrc_infer(nrc, ctypes.byref(pts), _ptr(out), _stream(stream)), "gi_nrc_infer")


def gi_nrc_backward(nrc: int, pts: gi_points, target_planes, mask=None, batch_norm: int = 0, stream=None) -> None:
    tp = (c_vp * 3)(*[_ptr(target_planes[c]) for c in range(3)])
    check(lib().gi_nrc_backward(nrc, ctypes.byref(pts), tp, _ptr(mask), int(batch_norm), _stream(stream)),
          "gi_nrc_backward")


def gi_nrc_adam(nrc: int, stream=None) -> None:
    check(lib().gi_nrc_adam(nrc, _stream(stream)), "gi_nrc_adam")


def gi_nrc_set_learning_rate(nrc: int, lr: float) -> None:
    check(lib().gi_nrc_set_learning_rate(nrc, float(lr)), "gi_nrc_set_learning_rate")


def gi_nrc_train_frame(nrc: int, cache: int, hits: gi_hits, slot_ids, frame: int, stream=None) -> None:
    check(lib().gi_nrc_train_frame(nrc, cache, ctypes.byref(hits), _ptr(slot_ids), int(frame), _stream(stream)),
          "gi_nrc_train_frame")


def gi_nrc_query_frame(nrc: int, cache: int, hits: gi_hits, slot_ids, view: gi_view, stream=None) -> None:
    check(lib().gi_nrc_query_frame(nrc, cache, ctypes.byref(hits), _ptr(slot_ids), ctypes.byref(view),
                                   _stream(stream)), "gi_nrc_query_frame")


def gi_nrc_answers(nrc: int, records=None, rad=None, capacity: int = 0, stream=None) -> int:
    """Number of records answered by the latest query frame; with device buffers records (u32) and
    rad (float4) of `capacity` entries, also copies them."""
    c = c_u32()
    check(lib().gi_nrc_answers(nrc, _ptr(records), _ptr(rad), int(capacity), ctypes.byref(c), _stream(stream)),
          "gi_nrc_answers")
    return c.value


def gi_probes_integrate_nrc(cache: int, nrc: int, probes: gi_probes, slot_ids, rays_per_probe: int,
                            env=(0.0, 0.0, 0.0), stream=None) -> None:
    e = (c_f32 * 3)(*[float(x) for x in env])
    check(lib().gi_probes_integrate_nrc(cache, nrc, ctypes.byref(probes), _ptr(slot_ids), int(rays_per_probe), e,
                                        _stream(stream)), "gi_probes_integrate_nrc")


def gi_nrc_stats(nrc: int, stream=None) -> dict:
    st = gi_nrc_stats_t()
    check(lib().gi_nrc_stats(nrc, ctypes.byref(st), _stream(stream)), "gi_nrc_stats")
    return {k: getattr(st, k) for k, _ in gi_nrc_stats_t._fields_}
