"""FP64 CPU oracle for surface-based gaze mapping -- TEST INFRASTRUCTURE.

Plain, slow, obviously-correct reference for every step of the hot path: world transform,
triangle areas, per-triangle sample counts, Philox sample positions, the cone test, brute-force
occlusion against every triangle, the duration-weighted Gaussian, per-window sums and
max-normalisation. The arithmetic lives in `gm_oracle.c` (built with gcc, FP contraction off);
this module only loads it and marshals numpy arrays.

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg use this
package. The CUDA library never imports, links or calls it, and it shares no code with it.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgm_oracle.so")
_lib = None

PF_IN_CONE, PF_VISIBLE, PF_VIS_AMBIG, PF_CONE_EDGE = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FP contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(C.Structure):
    _fields_ = [("theta", C.c_double), ("cutoff", C.c_double), ("eps_rel", C.c_double),
                ("t_begin", C.c_double), ("t_end", C.c_double), ("window_s", C.c_double),
                ("delta_abs", C.c_double), ("cone_band", C.c_double),
                ("n_windows", C.c_int32), ("nthreads", C.c_int32)]


class _Stats(C.Structure):
    _fields_ = [("pairs", C.c_int64), ("in_cone", C.c_int64), ("rays", C.c_int64),
                ("visible", C.c_int64), ("ambiguous", C.c_int64), ("cone_edge", C.c_int64)]


class _Frustum(C.Structure):
    _fields_ = [("e", C.c_double * 3), ("right", C.c_double * 3), ("up", C.c_double * 3), ("fwd", C.c_double * 3),
                ("n", C.c_double), ("f", C.c_double), ("l", C.c_double), ("r", C.c_double), ("b", C.c_double),
                ("t", C.c_double), ("ok", C.c_int32)]


class _ZbParams(C.Structure):
    _fields_ = [("res", C.c_int32), ("n", C.c_double), ("f", C.c_double), ("eps", C.c_double),
                ("delta_px", C.c_double), ("delta_w_rel", C.c_double)]


class _ZbStats(C.Structure):
    _fields_ = [("in_cone", C.c_int64), ("visible", C.c_int64), ("ambiguous", C.c_int64),
                ("skipped_fixations", C.c_int64)]


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB_PATH)
        _lib.ora_tri_offsets.restype = C.c_int
        _lib.ora_samples.restype = C.c_int
        _lib.ora_accumulate.restype = C.c_int
        _lib.ora_world_triangles.restype = C.c_int
        _lib.ora_pair_weight.restype = C.c_int
        _lib.ora_normalize.restype = C.c_double
        _lib.ora_grid_samples.restype = C.c_int
        for fn in ("ora_camera_basis", "ora_crop_paper", "ora_crop_exact", "ora_zb_frustum", "ora_zb_render",
                   "ora_zb_accumulate", "ora_zb_pairs"):
            getattr(_lib, fn).restype = C.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def world_vertices(v: np.ndarray, m: np.ndarray) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.float32)
    m = np.ascontiguousarray(m, dtype=np.float64)
    out = np.empty_like(v)
    lib().ora_world_vertices(_p(v), C.c_int64(len(v)), _p(m), _p(out))
    return out


def world_triangles(workload) -> np.ndarray:
    """(n_tris, 9) float32 world-space triangles, meshes concatenated in order."""
    verts = np.ascontiguousarray(np.concatenate([m.vertices for m in workload.meshes]), np.float32)
    idx = np.ascontiguousarray(np.concatenate([m.indices for m in workload.meshes]), np.uint32)
    xf = np.ascontiguousarray(np.stack([m.transform for m in workload.meshes]), np.float64)
    nv = np.array([len(m.vertices) for m in workload.meshes], np.int64)
    nt = np.array([m.n_tris for m in workload.meshes], np.int64)
    out = np.empty((int(nt.sum()), 9), np.float32)
    rc = lib().ora_world_triangles(_p(verts), _p(idx), _p(xf), _p(nv), _p(nt),
                                   C.c_int32(len(nt)), _p(out))
    if rc != 0:
        raise ValueError(f"ora_world_triangles failed ({rc})")
    return out


def tri_density(workload) -> np.ndarray:
    return np.concatenate([np.full(m.n_tris, m.density, np.float64) for m in workload.meshes])


def tri_object(workload) -> np.ndarray:
    return np.concatenate([np.full(m.n_tris, m.object_id, np.uint32) for m in workload.meshes])


def areas(tri: np.ndarray) -> np.ndarray:
    tri = np.ascontiguousarray(tri, np.float32)
    out = np.empty(len(tri), np.float64)
    lib().ora_tri_areas(_p(tri), C.c_int64(len(tri)), _p(out))
    return out


def areas_heron(tri: np.ndarray) -> np.ndarray:
    tri = np.ascontiguousarray(tri, np.float32)
    out = np.empty(len(tri), np.float64)
    lib().ora_tri_areas_heron(_p(tri), C.c_int64(len(tri)), _p(out))
    return out


def tri_offsets(area: np.ndarray, density: np.ndarray) -> np.ndarray:
    area = np.ascontiguousarray(area, np.float64)
    density = np.ascontiguousarray(np.broadcast_to(density, area.shape), np.float64)
    out = np.empty(len(area) + 1, np.int64)
    rc = lib().ora_tri_offsets(_p(area), _p(density), C.c_int64(len(area)), _p(out))
    if rc != 0:
        raise ValueError("sample count overflow")
    return out


def philox(ctr: np.ndarray, key) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(np.asarray(key, np.uint32).reshape(2))
    out = np.empty_like(ctr)
    lib().ora_philox_batch(_p(ctr), C.c_int64(len(ctr)), _p(k), _p(out))
    return out


@dataclass
class Samples:
    index: np.ndarray       # (n,) int64 global sample index
    tri: np.ndarray         # (n,) int64 global triangle index
    words: np.ndarray       # (n, 2) uint32 the two Philox words used
    bary: np.ndarray        # (n, 3) float64
    xyz: np.ndarray         # (n, 3) float64 world position


def samples(tri: np.ndarray, offsets: np.ndarray, seed: int, session: int,
            which: Optional[np.ndarray] = None) -> Samples:
    tri = np.ascontiguousarray(tri, np.float32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    if which is None:
        which = np.arange(int(offsets[-1]), dtype=np.int64)
    which = np.ascontiguousarray(which, np.int64)
    n = len(which)
    t = np.empty(n, np.int64)
    w = np.empty((n, 2), np.uint32)
    b = np.empty((n, 3), np.float64)
    x = np.empty((n, 3), np.float64)
    rc = lib().ora_samples(_p(tri), _p(offsets), C.c_int64(len(tri)), C.c_uint64(seed),
                           C.c_uint32(session), _p(which), C.c_int64(n), _p(t), _p(w), _p(b), _p(x))
    if rc != 0:
        raise ValueError("sample index out of range")
    return Samples(which, t, w, b, x)


def pair_weight(s, e, r, t, theta, cutoff=4.0):
    g = C.c_double()
    s, e, r = (np.ascontiguousarray(a, np.float64) for a in (s, e, r))
    inside = lib().ora_pair_weight(_p(s), _p(e), _p(r), C.c_double(t), C.c_double(theta),
                                   C.c_double(cutoff), C.byref(g))
    return bool(inside), g.value


def n_windows(params) -> int:
    if params.window_s <= 0:
        return 1
    return int(math.ceil((params.t_end - params.t_begin) / params.window_s))


def accumulate(tri, sxyz, stri, fixations, params, delta_abs=0.0, cone_band=0.0,
               record=False, nthreads=0, rec_cap=10_000_000):
    """Density of every given sample for every fixation window (brute force, FP64).

    Returns a dict with density/amb/sens arrays of shape (n_windows, n_samples), the pair
    statistics, and (record=True) the in-cone or cone-edge pairs in sample-major order."""
    tri = np.ascontiguousarray(tri, np.float32)
    sxyz = np.ascontiguousarray(sxyz, np.float64).reshape(-1, 3)
    stri = np.ascontiguousarray(stri, np.int64)
    fx = fixations
    eye = np.ascontiguousarray(fx.eye, np.float32)
    gaze = np.ascontiguousarray(fx.gaze, np.float32)
    dur = np.ascontiguousarray(fx.duration_s, np.float32)
    ts = np.ascontiguousarray(fx.timestamp_s, np.float64)
    W = n_windows(params)
    P = _Params(params.theta_rad, params.cutoff_sigmas, params.eps_rel, params.t_begin,
                params.t_end, params.window_s, delta_abs, cone_band, W, nthreads)
    ns = len(sxyz)
    dens = np.empty((W, ns), np.float64)
    amb = np.empty((W, ns), np.float64)
    sens = np.empty((W, ns), np.float64)
    st = _Stats()
    cap = rec_cap if record else -1
    m = max(cap, 0)
    rs, rf = np.empty(m, np.int64), np.empty(m, np.int32)
    rfl, rg = np.empty(m, np.uint8), np.empty(m, np.float64)
    nrec = C.c_int64(0)
    rc = lib().ora_accumulate(_p(tri), C.c_int64(len(tri)), _p(sxyz), _p(stri), C.c_int64(ns),
                              _p(eye), _p(gaze), _p(dur), _p(ts), C.c_int64(fx.n), C.byref(P),
                              _p(dens), _p(amb), _p(sens), C.byref(st), C.c_int64(cap),
                              _p(rs), _p(rf), _p(rfl), _p(rg), C.byref(nrec))
    if rc != 0:
        raise RuntimeError(f"ora_accumulate failed ({rc})")
    out = dict(density=dens, amb=amb, sens=sens,
               stats=dict(pairs=st.pairs, in_cone=st.in_cone, rays=st.rays, visible=st.visible,
                          ambiguous=st.ambiguous, cone_edge=st.cone_edge))
    if record:
        k = min(nrec.value, m)
        if nrec.value > m:
            raise RuntimeError("pair record capacity exceeded")
        out["pairs"] = dict(sample=rs[:k], fix=rf[:k], flag=rfl[:k], g=rg[:k])
    return out


def normalize(v: np.ndarray):
    v = np.ascontiguousarray(v, np.float64)
    out = np.empty_like(v)
    m = lib().ora_normalize(_p(v), C.c_int64(v.size), _p(out))
    return out, m


def fixation_windows(ts, params) -> np.ndarray:
    ts = np.ascontiguousarray(ts, np.float64)
    out = np.empty(len(ts), np.int32)
    lib().ora_fixation_windows(_p(ts), C.c_int64(len(ts)), C.c_double(params.t_begin),
                               C.c_double(params.t_end), C.c_double(params.window_s),
                               C.c_int32(n_windows(params)), _p(out))
    return out


def grid_resolution(area, density):
    """Per-triangle integer resolution of the paper's grid sampler (and the real root)."""
    area = np.ascontiguousarray(area, np.float64)
    density = np.ascontiguousarray(np.broadcast_to(density, area.shape), np.float64)
    r = np.empty(len(area), np.int64)
    rr = np.empty(len(area), np.float64)
    lib().ora_grid_resolution(_p(area), _p(density), C.c_int64(len(area)), _p(r), _p(rr))
    return r, rr


def grid_offsets(r):
    r = np.ascontiguousarray(r, np.int64)
    out = np.empty(len(r) + 1, np.int64)
    lib().ora_grid_offsets(_p(r), C.c_int64(len(r)), _p(out))
    return out


def grid_index(idx):
    row, col = C.c_int64(), C.c_int64()
    lib().ora_grid_index(C.c_int64(int(idx)), C.byref(row), C.byref(col))
    return row.value, col.value


def grid_samples(tri, offsets, r, which=None):
    tri = np.ascontiguousarray(tri, np.float32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    r = np.ascontiguousarray(r, np.int64)
    if which is None:
        which = np.arange(int(offsets[-1]), dtype=np.int64)
    which = np.ascontiguousarray(which, np.int64)
    n = len(which)
    t = np.empty(n, np.int64)
    rc = np.empty((n, 2), np.int64)
    b = np.empty((n, 3), np.float64)
    x = np.empty((n, 3), np.float64)
    st = lib().ora_grid_samples(_p(tri), _p(offsets), _p(r), C.c_int64(len(tri)), _p(which), C.c_int64(n),
                                _p(t), _p(rc), _p(b), _p(x))
    if st != 0:
        raise ValueError("sample index out of range")
    return dict(index=which, tri=t, rowcol=rc, bary=b, xyz=x)


def export_record(workload, smp: Samples, values=None) -> dict:
    """The per-sample export record of Section 3.3.3 for the oracle's samples: value, object id,
    triangle id, barycentrics (w0, w1, w2), mesh-local position and world position. The local
    position solves M x_local + t = x_world with the mesh's own FP64 transform (np.linalg.solve;
    the inverse is not formed)."""
    tri_mesh = np.repeat(np.arange(len(workload.meshes)), [m.n_tris for m in workload.meshes])
    mesh = tri_mesh[smp.tri]
    local = np.empty_like(smp.xyz)
    for mi, m in enumerate(workload.meshes):
        sel = mesh == mi
        if sel.any():
            T = np.asarray(m.transform, np.float64)
            local[sel] = np.linalg.solve(T[:3, :3], (smp.xyz[sel] - T[:3, 3]).T).T
    return dict(value=None if values is None else np.asarray(values, np.float64),
                object_id=tri_object(workload)[smp.tri], triangle=smp.tri.copy(), bary3=smp.bary.copy(),
                local_xyz=local, world_xyz=smp.xyz.copy())


def run_dynamic(workload, window_transforms, which=None, delta_abs=0.0, cone_band=0.0, nthreads=0):
    """Densities of a scene whose meshes move from window to window. Surface-bound values belong
    to the objects, not to world space (Section 2 holds this against volumetric maps, whose cells
    stay behind when an object moves), so every sample keeps its triangle and barycentrics: the
    counts are those of the workload's own (rest) transforms, and in window k the samples sit on
    the triangles posed by window_transforms[k] (n_meshes x 4 x 4 each). Window k accumulates the
    fixations of window k only (the windows of Section 3.2's time interval), against the scene in
    that pose. Returns density/amb/sens of shape (n_windows, n_samples) and the normalised maps."""
    import copy
    p = workload.params
    W = n_windows(p)
    wins = fixation_windows(workload.fixations.timestamp_s, p)
    off = tri_offsets(areas(world_triangles(workload)), tri_density(workload))
    n = int(off[-1]) if which is None else len(which)
    dens, amb, sens = (np.zeros((W, n)) for _ in range(3))
    for k in range(W):
        wk = copy.copy(workload)
        wk.meshes = [copy.copy(m) for m in workload.meshes]
        for m, T in zip(wk.meshes, window_transforms[k]):
            m.transform = np.asarray(T, np.float64)
        tri = world_triangles(wk)
        smp = samples(tri, off, workload.seed, workload.session, which)
        sel = np.nonzero(wins == k)[0]
        acc = accumulate(tri, smp.xyz, smp.tri, workload.fixations.subset(sel), p, delta_abs, cone_band,
                         nthreads=nthreads)
        dens[k], amb[k], sens[k] = acc["density"][k], acc["amb"][k], acc["sens"][k]
    norm = np.stack([normalize(d)[0] for d in dens])
    return dict(offsets=off, density=dens, amb=amb, sens=sens, normalized=norm)


def run(workload, which=None, delta_abs=0.0, cone_band=0.0, record=False, nthreads=0):
    """Whole method for one workload: world triangles, counts, the chosen samples (all by
    default), their densities per window and the normalised maps."""
    tri = world_triangles(workload)
    A = areas(tri)
    off = tri_offsets(A, tri_density(workload))
    smp = samples(tri, off, workload.seed, workload.session, which)
    acc = accumulate(tri, smp.xyz, smp.tri, workload.fixations, workload.params, delta_abs,
                     cone_band, record, nthreads)
    return dict(tri=tri, area=A, offsets=off, samples=smp, **acc)


# ---- the paper's z-buffer occlusion path (Sections 3.2.2, 3.3.2, Appendix A) ----------------
@dataclass
class ZBuffer:
    """Parameters of the z-buffer form: resolution (pixels per side of the crop window), clip
    planes and the +-eps depth tolerance (metres)."""
    res: int = 256
    near: float = 0.05
    far: float = 100.0
    eps: float = 0.005


def _d3(a):
    return np.ascontiguousarray(np.asarray(a, np.float64).reshape(3))


def camera_basis(fwd, up):
    r, u, f = (np.empty(3) for _ in range(3))
    rc = lib().ora_camera_basis(_p(_d3(fwd)), _p(_d3(up)), _p(r), _p(u), _p(f))
    if rc != 0:
        raise ValueError("zero forward vector")
    return r, u, f


def crop_paper(rc, phi, n):
    """Appendix A's crop window for the unit camera-space gaze rc: dict l, r, b, t, E, a, b_, alpha."""
    out = np.empty(9)
    if lib().ora_crop_paper(_p(_d3(rc)), C.c_double(phi), C.c_double(n), _p(out)) != 0:
        return None
    return dict(l=out[0], r=out[1], b=out[2], t=out[3], E=out[4:6].copy(), a=out[6], b_=out[7], alpha=out[8])


def crop_exact(rc, phi, n):
    out = np.empty(4)
    if lib().ora_crop_exact(_p(_d3(rc)), C.c_double(phi), C.c_double(n), _p(out)) != 0:
        return None
    return out


def _frustum_dict(F):
    return dict(e=np.array(F.e), right=np.array(F.right), up=np.array(F.up), fwd=np.array(F.fwd), n=F.n, f=F.f,
                l=F.l, r=F.r, b=F.b, t=F.t, ok=bool(F.ok))


def zb_frustum(eye, gaze, cam_fwd, cam_up, theta, cutoff, near, far):
    F = _Frustum()
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, np.float32).reshape(3))
    rc = lib().ora_zb_frustum(_p(f32(eye)), _p(f32(gaze)), _p(f32(cam_fwd)), _p(f32(cam_up)), C.c_double(theta),
                              C.c_double(cutoff), C.c_double(near), C.c_double(far), C.byref(F))
    return _frustum_dict(F) if rc == 0 else None


def zb_render(tri, frustum, res, delta_px=1e-3):
    F = _Frustum()
    for k in ("e", "right", "up", "fwd"):
        getattr(F, k)[:] = list(np.asarray(frustum[k], np.float64))
    for k in ("n", "f", "l", "r", "b", "t"):
        setattr(F, k, float(frustum[k]))
    F.ok = 1
    tri = np.ascontiguousarray(tri, np.float32)
    z = np.empty((res, res))
    a = np.empty((res, res), np.uint8)
    if lib().ora_zb_render(_p(tri), C.c_int64(len(tri)), C.byref(F), C.c_int32(res), C.c_double(delta_px), _p(z),
                           _p(a)) != 0:
        raise ValueError("bad frustum")
    return z, a.astype(bool)


def zb_accumulate(tri, sxyz, fixations, cam_fwd, cam_up, params, zb: ZBuffer, delta_px=1e-3, delta_w_rel=1e-5,
                  cone_band=0.0, record=False, keep_buffers=False, nthreads=0, rec_cap=10_000_000):
    """Densities of the z-buffer form for the given samples (FP64). Returns density/amb/sens
    (n_windows, n_samples), stats, the frusta and (keep_buffers) every fixation's z-buffer."""
    tri = np.ascontiguousarray(tri, np.float32)
    sxyz = np.ascontiguousarray(sxyz, np.float64).reshape(-1, 3)
    fx = fixations
    eye = np.ascontiguousarray(fx.eye, np.float32)
    gaze = np.ascontiguousarray(fx.gaze, np.float32)
    dur = np.ascontiguousarray(fx.duration_s, np.float32)
    ts = np.ascontiguousarray(fx.timestamp_s, np.float64)
    cf = np.ascontiguousarray(cam_fwd, np.float32).reshape(-1, 3)
    cu = np.ascontiguousarray(cam_up, np.float32).reshape(-1, 3)
    W = n_windows(params)
    P = _Params(params.theta_rad, params.cutoff_sigmas, params.eps_rel, params.t_begin, params.t_end,
                params.window_s, 0.0, cone_band, W, nthreads)
    Z = _ZbParams(int(zb.res), zb.near, zb.far, zb.eps, delta_px, delta_w_rel)
    ns, nf = len(sxyz), fx.n
    dens, amb, sens = (np.empty((W, ns)) for _ in range(3))
    st = _ZbStats()
    cap = rec_cap if record else -1
    m = max(cap, 0)
    rs, rf = np.empty(m, np.int64), np.empty(m, np.int32)
    rfl, rg = np.empty(m, np.uint8), np.empty(m, np.float64)
    nrec = C.c_int64(0)
    frusta = (_Frustum * max(nf, 1))()
    zbuf = np.empty((nf, zb.res, zb.res)) if keep_buffers else None
    zamb = np.empty((nf, zb.res, zb.res), np.uint8) if keep_buffers else None
    rc = lib().ora_zb_accumulate(_p(tri), C.c_int64(len(tri)), _p(sxyz), C.c_int64(ns), _p(eye), _p(gaze), _p(dur),
                                 _p(ts), _p(cf), _p(cu), C.c_int64(nf), C.byref(P), C.byref(Z), _p(dens), _p(amb),
                                 _p(sens), C.byref(st), C.c_int64(cap), _p(rs), _p(rf), _p(rfl), _p(rg),
                                 C.byref(nrec), frusta, _p(zbuf) if keep_buffers else None,
                                 _p(zamb) if keep_buffers else None)
    if rc != 0:
        raise RuntimeError(f"ora_zb_accumulate failed ({rc})")
    out = dict(density=dens, amb=amb, sens=sens, frusta=[_frustum_dict(frusta[i]) for i in range(nf)],
               stats=dict(in_cone=st.in_cone, visible=st.visible, ambiguous=st.ambiguous,
                          skipped_fixations=st.skipped_fixations))
    if keep_buffers:
        out["zbuf"], out["zamb"] = zbuf, zamb.astype(bool)
    if record:
        k = min(nrec.value, m)
        if nrec.value > m:
            raise RuntimeError("pair record capacity exceeded")
        out["pairs"] = dict(sample=rs[:k], fix=rf[:k], flag=rfl[:k], g=rg[:k])
    return out


def zb_pairs(tri, sxyz, eye, gaze, cam_fwd, cam_up, theta, cutoff, zb: ZBuffer, delta_px=1e-3, delta_w_rel=1e-5,
             nthreads=0):
    """z-buffer visibility of individual (sample, fixation) pairs (one row per pair in every array),
    casting only the pixels each decision reads: the full-size form of zb_accumulate's test.
    Returns (vis, amb, frustum_ok) as bool arrays."""
    tri = np.ascontiguousarray(tri, np.float32)
    sxyz = np.ascontiguousarray(sxyz, np.float64).reshape(-1, 3)
    n = len(sxyz)
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, np.float32).reshape(n, 3))
    e, g, fw, up = f32(eye), f32(gaze), f32(cam_fwd), f32(cam_up)
    Z = _ZbParams(int(zb.res), zb.near, zb.far, zb.eps, delta_px, delta_w_rel)
    vis, amb, ok = (np.zeros(n, np.int8) for _ in range(3))
    rc = lib().ora_zb_pairs(_p(tri), C.c_int64(len(tri)), C.c_int64(n), _p(sxyz), _p(e), _p(g), _p(fw), _p(up),
                            C.c_double(theta), C.c_double(cutoff), C.byref(Z), _p(vis), _p(amb), _p(ok),
                            C.c_int32(nthreads))
    if rc != 0:
        raise RuntimeError(f"ora_zb_pairs failed ({rc})")
    return vis.astype(bool), amb.astype(bool), ok.astype(bool)
