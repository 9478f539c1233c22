"""Thin ctypes binding of libgazemap (include/gazemap.h): same names, argument marshalling only.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA); every computation
runs in the library's CUDA kernels. There is no CPU fallback: if the library is not built or
no sm_103a GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from .build import LIB

GM_OK, GM_ERR_INVALID_ARG, GM_ERR_CUDA, GM_ERR_OOM, GM_ERR_TIMEOUT = 0, 1, 2, 3, 4
GM_ERR_UNSUPPORTED, GM_ERR_INTERNAL, GM_WARN_EMPTY = 5, 6, 100
GM_F_TIMING, GM_F_DEBUG_PAIRS, GM_F_NO_REORDER, GM_F_NO_COMPACT, GM_F_WIDE_BVH = 1, 2, 4, 8, 16
GM_F_REGCAP64, GM_F_TILE_CONSECUTIVE, GM_F_STATIC_TILES, GM_F_NO_TILE_CULL, GM_F_BLOCK128 = 32, 64, 128, 256, 512
GM_F_EYE_GRID, GM_F_GRID64, GM_F_SPT1, GM_F_SPT2, GM_F_BLOCK512 = 1024, 2048, 4096, 8192, 16384
GM_F_FIX_L1 = 32768
GM_F_SPT4 = 65536
GM_Q_SAMPLE, GM_Q_PLAIN, GM_Q_FIELD = 0, 1, 2


class GazeMapError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[gm status {status}] {msg}")
        self.status = status


class gm_mesh_desc(C.Structure):
    _fields_ = [("vertices", C.c_void_p), ("indices", C.c_void_p), ("n_verts", C.c_uint32),
                ("n_tris", C.c_uint32), ("transform", C.c_double * 16), ("object_id", C.c_uint32)]


class gm_fixations(C.Structure):
    _fields_ = [("eye_xyz", C.c_void_p), ("gaze_xyz", C.c_void_p), ("duration_s", C.c_void_p),
                ("timestamp_s", C.c_void_p), ("n", C.c_uint32)]


class gm_session_desc(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("samples", C.c_void_p), ("fix", gm_fixations)]


class gm_params(C.Structure):
    _fields_ = [("theta_rad", C.c_float), ("cutoff_sigmas", C.c_float), ("eps_rel", C.c_float),
                ("t_begin", C.c_double), ("t_end", C.c_double), ("window_s", C.c_double),
                ("normalize", C.c_int32), ("flags", C.c_int32), ("debug_pair_cap", C.c_uint64)]


class gm_field_cfg(C.Structure):
    _fields_ = [("steps", C.c_uint32), ("batch", C.c_uint32), ("lr", C.c_float), ("lr_min", C.c_float),
                ("seed", C.c_uint64)]


GM_FIELD_N_PARAMS = 16705


class gm_build_opts(C.Structure):
    _fields_ = [("builder", C.c_int32), ("dynamic", C.c_int32), ("ploc_radius", C.c_int32)]


class gm_zbuffer_params(C.Structure):
    _fields_ = [("res", C.c_uint32), ("near_m", C.c_float), ("far_m", C.c_float), ("eps_m", C.c_float),
                ("compare", C.c_uint32), ("zbuffer_bytes", C.c_uint64)]


class gm_export_dst(C.Structure):
    _fields_ = [("value", C.c_void_p), ("object_id", C.c_void_p), ("triangle", C.c_void_p), ("bary3", C.c_void_p),
                ("local_xyz", C.c_void_p), ("world_xyz", C.c_void_p)]


class gm_map_stats(C.Structure):
    _fields_ = [("pairs", C.c_uint64), ("in_cone", C.c_uint64), ("visible", C.c_uint64),
                ("n_windows", C.c_uint32), ("n_fixations_used", C.c_uint32), ("prep_ms", C.c_float),
                ("accumulate_ms", C.c_float), ("normalize_ms", C.c_float), ("launches", C.c_uint32),
                ("nodes_visited", C.c_uint64), ("tris_tested", C.c_uint64), ("pairs_tested", C.c_uint64),
                ("grid_ms", C.c_float), ("grid_chunks", C.c_uint32), ("grid_launches", C.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_P = C.c_void_p

_SIGS = {
    "gm_create": (C.c_int, [C.c_int, C.POINTER(_P)]),
    "gm_destroy": (None, [_P]),
    "gm_last_error": (C.c_char_p, []),
    "gm_sync": (C.c_int, [_P, _P]),
    "gm_ctx_launches": (C.c_int, [_P, C.POINTER(C.c_uint64)]),
    "gm_build_scene": (C.c_int, [_P, C.POINTER(gm_mesh_desc), C.c_uint32, _P, C.POINTER(_P)]),
    "gm_build_scene_opts": (C.c_int, [_P, C.POINTER(gm_mesh_desc), C.c_uint32, C.POINTER(gm_build_opts), _P,
                                      C.POINTER(_P)]),
    "gm_scene_pose": (C.c_int, [_P, C.POINTER(C.c_double), _P]),
    "gm_samples_follow": (C.c_int, [_P, _P]),
    "gm_accumulate_dynamic": (C.c_int, [_P, _P, C.POINTER(gm_fixations), C.POINTER(gm_params), C.POINTER(C.c_double),
                                        _P, C.POINTER(_P)]),
    "gm_scene_info": (C.c_int, [_P, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    "gm_scene_triangles": (C.c_int, [_P, _P, _P]),
    "gm_scene_free": (None, [_P]),
    "gm_sample_surface": (C.c_int, [_P, _P, C.c_uint64, C.c_uint32, _P, C.POINTER(_P)]),
    "gm_samples_from_points": (C.c_int, [_P, _P, _P, C.c_uint64, _P, C.POINTER(_P)]),
    "gm_sample_surface_grid": (C.c_int, [_P, _P, _P, C.POINTER(_P)]),
    "gm_samples_info": (C.c_int, [_P, C.POINTER(C.c_uint64)]),
    "gm_samples_offsets": (C.c_int, [_P, _P, _P]),
    "gm_samples_copy": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "gm_samples_free": (None, [_P]),
    "gm_samples_export": (C.c_int, [_P, _P, C.c_uint32, C.POINTER(gm_export_dst), _P]),
    "gm_tri_offsets_noalloc": (C.c_int, [_P, _P, _P, C.c_uint32, _P, _P]),
    "gm_accumulate_fixations": (C.c_int, [_P, _P, C.POINTER(gm_fixations), C.POINTER(gm_params), _P,
                                          C.POINTER(_P)]),
    "gm_accumulate_zbuffer": (C.c_int, [_P, _P, C.POINTER(gm_fixations), _P, _P, C.POINTER(gm_params),
                                        C.POINTER(gm_zbuffer_params), _P, C.POINTER(_P)]),
    "gm_zbuffer_stats": (C.c_int, [_P] + [C.POINTER(C.c_uint64)] * 4),
    "gm_zbuffer_render": (C.c_int, [_P, _P, _P, _P, _P, C.c_uint32, C.c_float, C.c_float,
                                    C.POINTER(gm_zbuffer_params), _P, _P, _P]),
    "gm_map_info": (C.c_int, [_P, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64), C.POINTER(gm_map_stats)]),
    "gm_map_copy": (C.c_int, [_P, C.c_uint32, _P, C.POINTER(C.c_float), _P]),
    "gm_map_device_values": (_P, [_P]),
    "gm_map_debug_pairs": (C.c_int, [_P, _P, _P, _P, _P, C.c_uint64, C.POINTER(C.c_uint64)]),
    "gm_map_free": (None, [_P]),
    "gm_query_density": (C.c_int, [_P, _P, C.c_int, C.c_uint32, _P, _P, C.c_uint64, _P, _P]),
    "gm_batch_create": (C.c_int, [_P, C.POINTER(gm_session_desc), C.c_uint32, C.POINTER(gm_params), _P,
                                  C.POINTER(_P)]),
    "gm_batch_run": (C.c_int, [_P, _P]),
    "gm_batch_map": (C.c_int, [_P, C.c_uint32, C.POINTER(_P)]),
    "gm_batch_info": (C.c_int, [_P, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                C.POINTER(C.c_float), C.POINTER(C.c_int32)]),
    "gm_batch_autotune": (C.c_int, [_P, _P, C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
    "gm_batch_free": (None, [_P]),
    "gm_batch_buckets": (C.c_int, [_P, C.POINTER(C.c_uint32), _P, _P, _P, _P]),
    "gm_accumulate_batch": (C.c_int, [_P, C.POINTER(gm_session_desc), C.c_uint32, C.POINTER(gm_params), _P,
                                      C.POINTER(_P)]),
    "gm_autotune_accumulate": (C.c_int, [_P, _P, C.POINTER(gm_fixations), C.POINTER(gm_params), _P,
                                         C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
    "gm_field_create": (C.c_int, [_P, _P, _P, _P, _P, C.POINTER(_P)]),
    "gm_field_train": (C.c_int, [_P, _P, _P, C.c_uint32, C.POINTER(gm_field_cfg), _P, C.POINTER(C.c_float)]),
    "gm_field_step": (C.c_int, [_P, _P, _P, C.c_uint64, _P, C.c_uint32, C.c_float, _P]),
    "gm_field_loss_grad": (C.c_int, [_P, _P, _P, C.c_uint64, _P, C.c_uint32, _P, C.POINTER(C.c_float), _P]),
    "gm_field_query": (C.c_int, [_P, _P, C.c_uint64, _P, _P]),
    "gm_field_query_kernel": (C.c_int, [_P, C.c_int32]),
    "gm_field_train_kernel": (C.c_int, [_P, C.c_int32]),
    "gm_field_params": (C.c_int, [_P, _P, _P]),
    "gm_field_info": (C.c_int, [_P, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_float),
                                C.POINTER(C.c_float)]),
    "gm_field_free": (None, [_P]),
    "gm_field_get_state": (C.c_int, [_P, _P, _P, _P, C.POINTER(C.c_uint32), _P]),
    "gm_samples_slice": (C.c_int, [_P, C.c_uint64, C.c_uint64, _P, C.POINTER(_P)]),
    "gm_map_max": (C.c_int, [_P, _P, _P]),
    "gm_map_normalize": (C.c_int, [_P, _P, _P]),
    "gm_field_set_state": (C.c_int, [_P, _P, _P, _P, C.c_uint32, _P]),
    "gm_debug_wait_timeout": (C.c_int, [_P, C.c_uint32, _P]),
}


def lib():
    """Load libgazemap.so (built by paper_2601_07571_gb300.build.build()); raise if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"libgazemap.so is not built ({LIB}); run paper_2601_07571_gb300.build.build()")
        L = C.CDLL(LIB)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> Sequence[str]:
    L = lib()
    return [n for n in _SIGS if hasattr(L, n)]


def _check(st: int, allow_empty: bool = False) -> int:
    if st == GM_OK or (allow_empty and st == GM_WARN_EMPTY):
        return st
    raise GazeMapError(st, lib().gm_last_error().decode(errors="replace"))


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream or None
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream or None
    return int(stream) or None


# ---- context ---------------------------------------------------------------------------------
def gm_create(device: int = 0):
    h = _P()
    _check(lib().gm_create(device, C.byref(h)))
    return h


def gm_destroy(ctx) -> None:
    lib().gm_destroy(ctx)


def gm_sync(ctx, stream=None) -> None:
    _check(lib().gm_sync(ctx, _stream(stream)))


def gm_ctx_launches(ctx) -> int:
    n = C.c_uint64()
    _check(lib().gm_ctx_launches(ctx, C.byref(n)))
    return n.value


# ---- scene -----------------------------------------------------------------------------------
GM_BUILD_LBVH, GM_BUILD_PLOC = 0, 1


def gm_build_scene(ctx, meshes, stream=None, builder=None, dynamic=False, ploc_radius=0):
    """meshes: sequence of (vertices (nv,3) f32, indices (nt,3) u32, transform (4,4) f64, object_id).
    builder: None (library default), GM_BUILD_LBVH or GM_BUILD_PLOC. dynamic: keep the mesh-local
    triangles for gm_scene_pose."""
    descs = (gm_mesh_desc * len(meshes))()
    keep = []
    for d, (v, f, xf, obj) in zip(descs, meshes):
        keep += [v, f]
        d.vertices = _ptr(v)
        d.indices = _ptr(f)
        d.n_verts = int(v.shape[0])
        d.n_tris = int(f.shape[0])
        d.transform = (C.c_double * 16)(*np.asarray(xf, np.float64).reshape(16).tolist())
        d.object_id = int(obj)
    h = _P()
    if builder is None and not dynamic and not ploc_radius:
        _check(lib().gm_build_scene(ctx, descs, len(meshes), _stream(stream), C.byref(h)))
    else:
        opt = gm_build_opts(GM_BUILD_PLOC if builder is None else int(builder), 1 if dynamic else 0, int(ploc_radius))
        _check(lib().gm_build_scene_opts(ctx, descs, len(meshes), C.byref(opt), _stream(stream), C.byref(h)))
    return h


def _f64(a):
    a = np.ascontiguousarray(np.asarray(a, np.float64))
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def gm_scene_pose(scene, transforms, stream=None) -> None:
    """transforms: (n_meshes, 4, 4) FP64 row-major."""
    a, p = _f64(transforms)
    _check(lib().gm_scene_pose(scene, p, _stream(stream)))


def gm_samples_follow(samples, stream=None) -> None:
    _check(lib().gm_samples_follow(samples, _stream(stream)))


def gm_scene_info(scene):
    nt, depth = C.c_uint32(), C.c_uint32()
    _check(lib().gm_scene_info(scene, C.byref(nt), C.byref(depth)))
    return nt.value, depth.value


def gm_scene_triangles(scene, out, stream=None) -> None:
    _check(lib().gm_scene_triangles(scene, _ptr(out), _stream(stream)))


def gm_scene_free(scene) -> None:
    lib().gm_scene_free(scene)


# ---- samples ---------------------------------------------------------------------------------
def gm_sample_surface(scene, density_per_mesh, seed: int, session: int = 0, stream=None):
    dens = np.ascontiguousarray(density_per_mesh, np.float64)
    h = _P()
    _check(lib().gm_sample_surface(scene, _ptr(dens), C.c_uint64(seed), C.c_uint32(session), _stream(stream),
                                   C.byref(h)))
    return h


def gm_sample_surface_grid(scene, density_per_mesh, stream=None):
    dens = np.ascontiguousarray(density_per_mesh, np.float64)
    h = _P()
    _check(lib().gm_sample_surface_grid(scene, _ptr(dens), _stream(stream), C.byref(h)))
    return h


def gm_samples_from_points(scene, xyz, tri, stream=None):
    h = _P()
    _check(lib().gm_samples_from_points(scene, _ptr(xyz), _ptr(tri), C.c_uint64(int(xyz.shape[0])),
                                        _stream(stream), C.byref(h)))
    return h


def gm_samples_info(samples) -> int:
    n = C.c_uint64()
    _check(lib().gm_samples_info(samples, C.byref(n)))
    return n.value


def gm_samples_offsets(samples, out, stream=None) -> None:
    _check(lib().gm_samples_offsets(samples, _ptr(out), _stream(stream)))


def gm_samples_copy(samples, xyz=None, tri=None, bary2=None, obj=None, stream=None) -> None:
    _check(lib().gm_samples_copy(samples, _ptr(xyz), _ptr(tri), _ptr(bary2), _ptr(obj), _stream(stream)))


def gm_samples_export(samples, m, window: int, value=None, object_id=None, triangle=None, bary3=None,
                      local_xyz=None, world_xyz=None, stream=None) -> None:
    dst = gm_export_dst(_ptr(value), _ptr(object_id), _ptr(triangle), _ptr(bary3), _ptr(local_xyz), _ptr(world_xyz))
    _check(lib().gm_samples_export(samples, m, int(window), C.byref(dst), _stream(stream)))


def gm_samples_free(samples) -> None:
    lib().gm_samples_free(samples)


def gm_tri_offsets_noalloc(ctx, tri_xyz, density_per_tri, n_tris: int, offsets, stream=None) -> None:
    """Per-triangle offsets from caller-owned device buffers, allocating nothing (see the header).

    The C entry point cannot see buffer sizes, so they are checked here: tri_xyz float32 with at
    least 9 * n_tris elements, density_per_tri float64 with at least n_tris, offsets int64 with at
    least n_tris + 1, all on a CUDA device. Sizes beyond the fixed scratch are left to the library,
    which refuses them before launching anything."""
    import torch
    n = int(n_tris)
    if n < 0 or n > 0xFFFFFFFF:
        raise ValueError("gm_tri_offsets_noalloc: n_tris must fit in uint32")
    need = n if n <= 65536 * 2048 else 0   # oversized requests reach the library's own refusal
    for name, t, dt, cnt in (("tri_xyz", tri_xyz, torch.float32, 9 * need),
                             ("density_per_tri", density_per_tri, torch.float64, need),
                             ("offsets", offsets, torch.int64, need + 1)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"gm_tri_offsets_noalloc: {name} must be a CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"gm_tri_offsets_noalloc: {name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous() or t.numel() < cnt:
            raise ValueError(f"gm_tri_offsets_noalloc: {name} must be contiguous with at least {cnt} elements")
    _check(lib().gm_tri_offsets_noalloc(ctx, _ptr(tri_xyz), _ptr(density_per_tri), C.c_uint32(n),
                                        _ptr(offsets), _stream(stream)))


# ---- accumulation ----------------------------------------------------------------------------
def make_params(theta_rad, cutoff_sigmas=4.0, eps_rel=1e-5, t_begin=-np.inf, t_end=np.inf, window_s=0.0,
                normalize=True, flags=0, debug_pair_cap=0) -> gm_params:
    return gm_params(float(theta_rad), float(cutoff_sigmas), float(eps_rel), float(t_begin), float(t_end),
                     float(window_s), int(bool(normalize)), int(flags), int(debug_pair_cap))


def gm_accumulate_fixations(scene, samples, eye, gaze, duration_s, timestamp_s, params: gm_params, stream=None):
    fx = gm_fixations(_ptr(eye), _ptr(gaze), _ptr(duration_s), _ptr(timestamp_s), int(eye.shape[0]))
    h = _P()
    _check(lib().gm_accumulate_fixations(scene, samples, C.byref(fx), C.byref(params), _stream(stream), C.byref(h)))
    return h


def gm_accumulate_dynamic(scene, samples, eye, gaze, duration_s, timestamp_s, params: gm_params, window_transforms,
                          stream=None):
    """window_transforms: (n_windows, n_meshes, 4, 4) FP64 row-major."""
    fx = gm_fixations(_ptr(eye), _ptr(gaze), _ptr(duration_s), _ptr(timestamp_s), int(eye.shape[0]))
    a, p = _f64(window_transforms)
    h = _P()
    _check(lib().gm_accumulate_dynamic(scene, samples, C.byref(fx), C.byref(params), p, _stream(stream), C.byref(h)))
    return h


def zbuffer_params(res=256, near=0.05, far=100.0, eps=0.005, compare=False, zbuffer_bytes=0):
    return gm_zbuffer_params(int(res), float(near), float(far), float(eps), 1 if compare else 0, int(zbuffer_bytes))


def gm_accumulate_zbuffer(scene, samples, eye, gaze, duration_s, timestamp_s, params: gm_params,
                          zb: gm_zbuffer_params, cam_forward=None, cam_up=None, stream=None):
    fx = gm_fixations(_ptr(eye), _ptr(gaze), _ptr(duration_s), _ptr(timestamp_s), int(eye.shape[0]))
    h = _P()
    _check(lib().gm_accumulate_zbuffer(scene, samples, C.byref(fx), _ptr(cam_forward), _ptr(cam_up), C.byref(params),
                                       C.byref(zb), _stream(stream), C.byref(h)))
    return h


def gm_zbuffer_stats(m) -> dict:
    v = [C.c_uint64() for _ in range(4)]
    _check(lib().gm_zbuffer_stats(m, *[C.byref(x) for x in v]))
    return dict(skipped_fixations=v[0].value, flips_to_visible=v[1].value, flips_to_hidden=v[2].value,
                raster_pairs=v[3].value)


def gm_zbuffer_render(scene, eye, gaze, theta_rad, cutoff_sigmas, zb: gm_zbuffer_params, cam_forward=None,
                      cam_up=None, stream=None):
    """Returns (zbuf (n, res, res) float32, crop (n, 4) float64)."""
    n = int(np.asarray(eye).shape[0])
    z = np.empty((n, zb.res, zb.res), np.float32)
    crop = np.empty((n, 4), np.float64)
    _check(lib().gm_zbuffer_render(scene, _ptr(eye), _ptr(gaze), _ptr(cam_forward), _ptr(cam_up), n, float(theta_rad),
                                   float(cutoff_sigmas), C.byref(zb), _ptr(z), _ptr(crop), _stream(stream)))
    return z, crop


def gm_map_info(m):
    W, ns, st = C.c_uint32(), C.c_uint64(), gm_map_stats()
    status = _check(lib().gm_map_info(m, C.byref(W), C.byref(ns), C.byref(st)), allow_empty=True)
    return W.value, ns.value, st.as_dict(), status


def gm_map_copy(m, window: int, out, stream=None) -> float:
    mx = C.c_float()
    _check(lib().gm_map_copy(m, int(window), _ptr(out), C.byref(mx), _stream(stream)))
    return mx.value


def gm_map_device_values(m) -> int:
    return lib().gm_map_device_values(m)


def gm_map_debug_pairs(m, cap: int):
    s = np.empty(cap, np.uint32)
    f = np.empty(cap, np.uint32)
    v = np.empty(cap, np.uint8)
    g = np.empty(cap, np.float32)
    n = C.c_uint64()
    _check(lib().gm_map_debug_pairs(m, _ptr(s), _ptr(f), _ptr(v), _ptr(g), C.c_uint64(cap), C.byref(n)))
    k = min(n.value, cap)
    return dict(sample=s[:k], fix=f[:k], visible=v[:k], g=g[:k], n=n.value)


def gm_map_free(m) -> None:
    lib().gm_map_free(m)


def gm_query_density(m, field, mode: int, window: int, sample_idx, xyz, n: int, out, stream=None) -> None:
    _check(lib().gm_query_density(m, field, int(mode), int(window), _ptr(sample_idx), _ptr(xyz), C.c_uint64(n),
                                  _ptr(out), _stream(stream)))


# ---- batched sessions -------------------------------------------------------------------------
def _session_descs(sessions):
    """sessions: sequence of (scene, samples, eye, gaze, duration_s, timestamp_s)."""
    arr = (gm_session_desc * len(sessions))()
    for d, (sc, sm, eye, gaze, dur, ts) in zip(arr, sessions):
        d.scene = sc.value if isinstance(sc, C.c_void_p) else sc
        d.samples = sm.value if isinstance(sm, C.c_void_p) else sm
        d.fix = gm_fixations(_ptr(eye), _ptr(gaze), _ptr(dur), _ptr(ts), int(eye.shape[0]))
    return arr


def gm_batch_create(ctx, sessions, params: gm_params, stream=None):
    arr = _session_descs(sessions)
    h = _P()
    _check(lib().gm_batch_create(ctx, arr, len(sessions), C.byref(params), _stream(stream), C.byref(h)))
    return h


def gm_batch_run(batch, stream=None) -> None:
    _check(lib().gm_batch_run(batch, _stream(stream)))


def gm_batch_map(batch, i: int):
    h = _P()
    _check(lib().gm_batch_map(batch, int(i), C.byref(h)))
    return h


def gm_batch_info(batch):
    n, items, pairs, ms, fl = C.c_uint32(), C.c_uint64(), C.c_uint64(), C.c_float(), C.c_int32()
    _check(lib().gm_batch_info(batch, C.byref(n), C.byref(items), C.byref(pairs), C.byref(ms), C.byref(fl)))
    return dict(n_sessions=n.value, n_work_items=items.value, pairs=pairs.value, last_ms=ms.value,
                variant_flags=fl.value)


def gm_batch_autotune(batch, stream=None):
    fl, ms = C.c_int32(), C.c_float()
    _check(lib().gm_batch_autotune(batch, _stream(stream), C.byref(fl), C.byref(ms)))
    return fl.value, ms.value


def gm_batch_free(batch) -> None:
    lib().gm_batch_free(batch)


def gm_accumulate_batch(ctx, sessions, params: gm_params, stream=None):
    arr = _session_descs(sessions)
    outs = (_P * len(sessions))()
    _check(lib().gm_accumulate_batch(ctx, arr, len(sessions), C.byref(params), _stream(stream), outs))
    return [_P(o) for o in outs]


def gm_autotune_accumulate(scene, samples, eye, gaze, duration_s, timestamp_s, params: gm_params, stream=None):
    fx = gm_fixations(_ptr(eye), _ptr(gaze), _ptr(duration_s), _ptr(timestamp_s), int(eye.shape[0]))
    fl, ms = C.c_int32(), C.c_float()
    _check(lib().gm_autotune_accumulate(scene, samples, C.byref(fx), C.byref(params), _stream(stream),
                                        C.byref(fl), C.byref(ms)))
    return fl.value, ms.value


# ---- neural density field ---------------------------------------------------------------------
def gm_field_create(ctx, box_lo, box_hi, init_params, stream=None):
    lo = np.ascontiguousarray(box_lo, np.float32)
    hi = np.ascontiguousarray(box_hi, np.float32)
    h = _P()
    _check(lib().gm_field_create(ctx, _ptr(lo), _ptr(hi), _ptr(init_params), _stream(stream), C.byref(h)))
    return h


def gm_field_train(field, samples, m, window: int, steps: int, batch: int, lr: float, lr_min: float, seed: int,
                   stream=None) -> float:
    cfg = gm_field_cfg(int(steps), int(batch), float(lr), float(lr_min), int(seed))
    loss = C.c_float()
    _check(lib().gm_field_train(field, samples, m, int(window), C.byref(cfg), _stream(stream), C.byref(loss)))
    return loss.value


def gm_field_step(field, xyz, target, n: int, batch_idx, batch: int, lr: float, stream=None) -> None:
    _check(lib().gm_field_step(field, _ptr(xyz), _ptr(target), C.c_uint64(n), _ptr(batch_idx), int(batch),
                               float(lr), _stream(stream)))


def gm_field_loss_grad(field, xyz, target, n: int, batch_idx, batch: int, grad_out, stream=None) -> float:
    loss = C.c_float()
    _check(lib().gm_field_loss_grad(field, _ptr(xyz), _ptr(target), C.c_uint64(n), _ptr(batch_idx), int(batch),
                                    _ptr(grad_out), C.byref(loss), _stream(stream)))
    return loss.value


GM_FIELD_QUERY_TCGEN05, GM_FIELD_QUERY_MMA_SYNC = 0, 1


def gm_field_query_kernel(field, kernel: int) -> None:
    _check(lib().gm_field_query_kernel(field, int(kernel)))


def gm_field_train_kernel(field, kernel: int) -> None:
    _check(lib().gm_field_train_kernel(field, int(kernel)))


def gm_field_query(field, xyz, n: int, out, stream=None) -> None:
    _check(lib().gm_field_query(field, _ptr(xyz), C.c_uint64(n), _ptr(out), _stream(stream)))


def gm_field_params(field, out, stream=None) -> None:
    _check(lib().gm_field_params(field, _ptr(out), _stream(stream)))


def gm_field_get_state(field, theta=None, m=None, v=None, stream=None) -> int:
    """Copy parameters and Adam moments out (any of them may be None); returns the steps taken."""
    t = C.c_uint32()
    _check(lib().gm_field_get_state(field, _ptr(theta), _ptr(m), _ptr(v), C.byref(t), _stream(stream)))
    return t.value


def gm_field_set_state(field, theta, m, v, steps: int, stream=None) -> None:
    _check(lib().gm_field_set_state(field, _ptr(theta), _ptr(m), _ptr(v), C.c_uint32(int(steps)), _stream(stream)))


def gm_debug_wait_timeout(ctx, iterations: int, stream=None) -> None:
    _check(lib().gm_debug_wait_timeout(ctx, C.c_uint32(int(iterations)), _stream(stream)))


def gm_field_info(field):
    n, t, loss, ms = C.c_uint32(), C.c_uint32(), C.c_float(), C.c_float()
    _check(lib().gm_field_info(field, C.byref(n), C.byref(t), C.byref(loss), C.byref(ms)))
    return dict(n_params=n.value, steps=t.value, last_loss=loss.value, train_ms=ms.value)


def gm_field_free(field) -> None:
    lib().gm_field_free(field)


def gm_samples_slice(samples, begin: int, end: int, stream=None):
    h = _P()
    _check(lib().gm_samples_slice(samples, C.c_uint64(int(begin)), C.c_uint64(int(end)), _stream(stream), C.byref(h)))
    return h


def gm_map_max(m, out, stream=None) -> None:
    _check(lib().gm_map_max(m, _ptr(out), _stream(stream)))


def gm_map_normalize(m, maxima=None, stream=None) -> None:
    _check(lib().gm_map_normalize(m, _ptr(maxima), _stream(stream)))


def gm_batch_buckets(b):
    """Per size bucket: variant flags, sessions, work items and the last replay's launch time (ms)."""
    n = C.c_uint32()
    fl = np.zeros(3, np.int32)
    se = np.zeros(3, np.uint32)
    it = np.zeros(3, np.uint32)
    ms = np.zeros(3, np.float32)
    _check(lib().gm_batch_buckets(b, C.byref(n), _ptr(fl), _ptr(se), _ptr(it), _ptr(ms)))
    return [dict(flags=int(fl[k]), sessions=int(se[k]), work_items=int(it[k]), ms=float(ms[k])) for k in range(n.value)]
