"""Seeded synthetic workloads shaped like the paper's experiments.

The paper's recorded fixations and scenes (Fig. 1: 800k triangles, 6000 fixations, four
meshes with difficult properties; Section 4 stress test: 10M triangles) are not available.
These builders produce inputs with the same shapes, sizes and structure. Both the CPU
oracle and the CUDA path read the same arrays; this module computes nothing the method
computes (the one area evaluation below only picks a scale factor for one workload and is
never passed to either side).

Workloads (all seeded, all synthetic):
  tiny_sphere()      icosphere r=1 (320 tris) + 0.4 m occluder cube, 500 samples/m^2,
                     100 fixations from a 2-4 m shell                       (seed 0)
  paper_scene()      four procedural meshes totalling ~800k tris, 50 m^2, 40 000/m^2
                     -> ~2M samples, 6000 fixations at 1.7 m eye height      (seed 1)
  batched_sessions() 64 independent sessions, 5k-300k tris, 500-20k fixations,
                     1e3-5e4 samples/m^2, all log-uniform                   (seed = session)
  city_block()       ~5M-tri city block, ~20M samples, 100k fixations in 600 1-s windows
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import meshes as M


@dataclass
class Mesh:
    vertices: np.ndarray            # (nv, 3) float32, mesh-local space
    indices: np.ndarray             # (nt, 3) uint32
    transform: np.ndarray           # (4, 4) float64, row-major, local -> world (metres)
    object_id: int
    density: float                  # samples per square metre for this mesh

    @property
    def n_tris(self) -> int:
        return int(self.indices.shape[0])


@dataclass
class Fixations:
    eye: np.ndarray                 # (n, 3) float32, world space
    gaze: np.ndarray                # (n, 3) float32, gaze direction (any length > 0)
    duration_s: np.ndarray          # (n,) float32, seconds
    timestamp_s: np.ndarray         # (n,) float64, seconds

    @property
    def n(self) -> int:
        return int(self.eye.shape[0])

    def subset(self, idx) -> "Fixations":
        return Fixations(self.eye[idx], self.gaze[idx], self.duration_s[idx], self.timestamp_s[idx])


@dataclass
class Params:
    theta_rad: float = math.radians(1.0)   # angular deviation = one standard deviation
    cutoff_sigmas: float = 4.0             # propagate up to 4 sigma
    eps_rel: float = 1e-5                  # occlusion segment stops (1 - eps_rel) of the way
    t_begin: float = -math.inf
    t_end: float = math.inf
    window_s: float = 0.0                  # <= 0: one map over [t_begin, t_end)
    normalize: bool = True


@dataclass
class Workload:
    name: str
    meshes: List[Mesh]
    fixations: Fixations
    params: Params = field(default_factory=Params)
    seed: int = 0                   # sampler seed (Philox key)
    session: int = 0                # sampler stream id (Philox counter word 2)

    @property
    def n_tris(self) -> int:
        return sum(m.n_tris for m in self.meshes)

    def n_windows(self) -> int:
        p = self.params
        if p.window_s <= 0:
            return 1
        return int(math.ceil((p.t_end - p.t_begin) / p.window_s))


def identity() -> np.ndarray:
    return np.eye(4, dtype=np.float64)


def scale_translate(s: float, t) -> np.ndarray:
    """world = s * (local + t)."""
    m = np.eye(4, dtype=np.float64) * s
    m[3, 3] = 1.0
    m[:3, 3] = s * np.asarray(t, dtype=np.float64)
    return m


def _world(mesh: Mesh) -> np.ndarray:
    v = mesh.vertices.astype(np.float64)
    return v @ mesh.transform[:3, :3].T + mesh.transform[:3, 3]


def _surface_area_for_sizing(meshes: List[Mesh]) -> float:
    tot = 0.0
    for m in meshes:
        w = _world(m)
        a, b, c = (w[m.indices[:, k].astype(np.int64)] for k in range(3))
        tot += 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum()
    return float(tot)


def _jitter(rng: np.random.Generator, d: np.ndarray, sigma_rad: float) -> np.ndarray:
    """Perturb unit directions by an isotropic 2-D Gaussian angle in the tangent plane."""
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    helper = np.where(np.abs(d[:, :1]) < 0.9, [[1.0, 0.0, 0.0]], [[0.0, 1.0, 0.0]])
    u = np.cross(d, helper)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = np.cross(d, u)
    a = rng.normal(0.0, sigma_rad, size=(len(d), 2))
    out = d + np.tan(a[:, :1]) * u + np.tan(a[:, 1:]) * v
    return out / np.linalg.norm(out, axis=1, keepdims=True)


def _random_surface_points(rng: np.random.Generator, mesh: Mesh, n: int) -> np.ndarray:
    """Points on uniformly chosen triangles (by index) at uniform barycentric positions."""
    w = _world(mesh)
    t = rng.integers(0, mesh.n_tris, size=n)
    f = mesh.indices[t].astype(np.int64)
    r1, r2 = rng.random(n), rng.random(n)
    s = np.sqrt(r1)
    b = np.stack([1 - s, s * (1 - r2), s * r2], axis=1)
    return (b[:, :1] * w[f[:, 0]] + b[:, 1:2] * w[f[:, 1]] + b[:, 2:] * w[f[:, 2]])


def _durations(rng: np.random.Generator, n: int):
    dur = rng.uniform(0.1, 0.6, size=n)
    ts = np.concatenate([[0.0], np.cumsum(dur)[:-1]])
    return dur.astype(np.float32), ts.astype(np.float64)


def tiny_sphere(seed: int = 0, n_fix: int = 100, density: float = 500.0) -> Workload:
    """Icosphere r = 1 m (2 subdivisions, 320 tris) with an axis-aligned occluder cube of
    half-side 0.2 m at (1.5, 0, 0); eyes uniform in the volume of the 2-4 m shell, gaze at a
    uniform point of the unit sphere plus 1 degree Gaussian jitter; durations U(100, 600) ms."""
    rng = np.random.default_rng(seed)
    sv, sf = M.icosphere(2, 1.0)
    cv, cf = M.box((1.5, 0.0, 0.0), 0.2)
    meshes = [Mesh(sv, sf, identity(), 0, density), Mesh(cv, cf, identity(), 1, density)]
    rad = np.cbrt(rng.uniform(8.0, 64.0, size=n_fix))
    d = rng.normal(size=(n_fix, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    eye = d * rad[:, None]
    tgt = rng.normal(size=(n_fix, 3))
    tgt /= np.linalg.norm(tgt, axis=1, keepdims=True)
    gaze = _jitter(rng, tgt - eye, math.radians(1.0))
    dur, ts = _durations(rng, n_fix)
    fx = Fixations(eye.astype(np.float32), gaze.astype(np.float32), dur, ts)
    return Workload("tiny_sphere_320tri_100fix", meshes, fx, Params(), seed=seed, session=0)


def paper_scene(seed: int = 1, n_fix: int = 6000, density: float = 40_000.0,
                total_area: float = 50.0) -> Workload:
    """Four procedural meshes shaped like the paper's challenging scene (Fig. 1):
    a noise-displaced sphere (399 424 tris), a (2,3) torus knot (250 000 tris), a 1 m cube
    (12 tris) and a two-density blob (~150k tris: ~1 cm edges on one half, ~1 mm on the other).
    Uniformly rescaled so the world area is `total_area` m^2 (50 m^2 at 40 000/m^2 -> ~2M
    samples). 6000 fixations at 1.7 m eye height among the objects, gaze at a point of a mesh
    plus 1 degree jitter, durations U(100, 600) ms."""
    rng = np.random.default_rng(seed)
    parts = [
        (M.uv_sphere(317, 632, radius=1.2, noise_amp=0.05, noise_freq=3.0, seed=seed), (-2.4, 1.3, -2.4)),
        (M.torus_knot(2500, 50, scale=1.5, tube=0.5), (2.4, 1.6, -2.4)),
        (M.box((0.0, 0.0, 0.0), 0.5), (2.4, 0.5, 2.4)),
        (M.mixed_density_blob(seed + 7), (-2.4, 0.65, 2.4)),
    ]
    meshes = [Mesh(v, f, scale_translate(1.0, t), i, density) for i, ((v, f), t) in enumerate(parts)]
    s = math.sqrt(total_area / _surface_area_for_sizing(meshes))
    for m, (_, t) in zip(meshes, parts):
        m.transform = scale_translate(s, t)
    centers = np.array([[t[0], t[2]] for _, t in parts]) * s
    radii = np.array([1.35, 1.75, 0.75, 0.7]) * s
    eyes = []
    while len(eyes) < n_fix:
        p = rng.uniform(-6.5, 6.5, size=(4 * n_fix, 2))
        ok = (np.linalg.norm(p, axis=1) < 6.5)
        for c, r in zip(centers, radii):
            ok &= np.linalg.norm(p - c, axis=1) > r + 0.4
        eyes.extend(p[ok].tolist())
    e2 = np.asarray(eyes[:n_fix])
    eye = np.stack([e2[:, 0], np.full(n_fix, 1.7), e2[:, 1]], axis=1)
    which = rng.choice(4, size=n_fix, p=[0.35, 0.3, 0.1, 0.25])
    tgt = np.zeros((n_fix, 3))
    for i, m in enumerate(meshes):
        sel = np.nonzero(which == i)[0]
        if len(sel):
            tgt[sel] = _random_surface_points(rng, m, len(sel))
    gaze = _jitter(rng, tgt - eye, math.radians(1.0))
    dur, ts = _durations(rng, n_fix)
    fx = Fixations(eye.astype(np.float32), gaze.astype(np.float32), dur, ts)
    return Workload("paper_scene_800ktri_2Msample_6000fix", meshes, fx, Params(), seed=seed, session=0)


def _loguniform(rng, lo, hi):
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


def session(sid: int, tri_range=(5_000, 300_000), fix_range=(500, 20_000),
            density_range=(1e3, 5e4)) -> Workload:
    """One session of the batched workload: a displaced sphere or a torus knot with a
    log-uniform triangle count, bounding radius U(0.5, 2) m, log-uniform fixation count and
    density; eyes 1.5-4 bounding radii from the centre, gaze at mesh points + 1 degree."""
    rng = np.random.default_rng(1000 + sid)
    nt = _loguniform(rng, *tri_range)
    R = rng.uniform(0.5, 2.0)
    if rng.random() < 0.5:
        n_lat = max(4, int(round(math.sqrt(nt / 4.0))))
        v, f = M.uv_sphere(n_lat, 2 * n_lat, radius=R / 1.06, noise_amp=0.05,
                           noise_freq=3.0, seed=sid)
    else:
        n_ring = 24
        n_seg = max(8, int(round(nt / (2 * n_ring))))
        v, f = M.torus_knot(n_seg, n_ring, scale=R, tube=0.45)
    k = _loguniform(rng, *density_range)
    mesh = Mesh(v, f, identity(), 0, k)
    nf = int(round(_loguniform(rng, *fix_range)))
    d = rng.normal(size=(nf, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    eye = d * (R * rng.uniform(1.5, 4.0, size=nf))[:, None]
    tgt = _random_surface_points(rng, mesh, nf)
    gaze = _jitter(rng, tgt - eye, math.radians(1.0))
    dur, ts = _durations(rng, nf)
    fx = Fixations(eye.astype(np.float32), gaze.astype(np.float32), dur, ts)
    return Workload(f"session{sid}", [mesh], fx, Params(), seed=sid, session=sid)


def batched_sessions(n: int = 64, **kw) -> List[Workload]:
    return [session(i, **kw) for i in range(n)]


def city_block(seed: int = 4, n_fix: int = 100_000, n_samples: float = 20e6,
               grid: int = 20, boxes_per_block: int = 10, n_spheres: int = 25,
               sphere_lat: int = 223, duration_s: float = 600.0, window_s: float = 1.0) -> Workload:
    """Procedural city block: `grid` x `grid` blocks of `boxes_per_block` boxes (12 tris each)
    on a 12 m street pitch, plus `n_spheres` noise-displaced spheres of ~198k tris each
    (~5M tris in total, flattened, no instancing). Density is set so the scene holds
    ~`n_samples` samples. Fixations follow a seeded random walk at 1.7 m eye height with
    timestamps uniform over [0, duration_s), sorted; one map per `window_s` window."""
    rng = np.random.default_rng(seed)
    pitch = 12.0
    meshes: List[Mesh] = []
    parts = []
    centers = []
    for bx in range(grid):
        for bz in range(grid):
            cx, cz = (bx - grid / 2 + 0.5) * pitch, (bz - grid / 2 + 0.5) * pitch
            for _ in range(boxes_per_block):
                hx, hz = rng.uniform(0.5, 1.5, size=2)
                hy = rng.uniform(1.0, 4.0)
                px, pz = cx + rng.uniform(-3.5, 3.5), cz + rng.uniform(-3.5, 3.5)
                parts.append(M.box((px, hy, pz), (hx, hy, hz)))
                centers.append((px, hy, pz))
    boxes = M.merge(parts)
    meshes.append(Mesh(boxes[0], boxes[1], identity(), 0, 1.0))
    for i in range(n_spheres):
        r = rng.uniform(2.0, 4.0)
        v, f = M.uv_sphere(sphere_lat, 2 * sphere_lat, radius=r, noise_amp=0.05,
                           noise_freq=2.0, seed=seed * 100 + i)
        gx, gz = rng.integers(0, grid, size=2)
        c = ((gx - grid / 2) * pitch, r, (gz - grid / 2) * pitch)   # on street crossings
        meshes.append(Mesh(v, f, scale_translate(1.0, c), 1 + i, 1.0))
        centers.append(c)
    area = _surface_area_for_sizing(meshes)
    for m in meshes:
        m.density = n_samples / area
    centers = np.asarray(centers)
    # object extents for gaze targets: boxes (half sizes) first, then spheres (radius)
    n_box = len(parts)
    ext = np.zeros((len(centers), 3))
    rad = np.zeros(len(centers))
    box_half = np.array([(pp[0].max(0) - pp[0].min(0)) / 2 for pp in parts])
    ext[:n_box] = box_half
    for i in range(n_spheres):
        rad[n_box + i] = centers[n_box + i][1]
    # the viewer walks the 2 m streets between blocks (x or z a multiple of the pitch), one step
    # of 0.3 m per fixation, turning at crossings, and steps around the spheres on the crossings
    pos = np.zeros((n_fix, 3))
    half = grid * pitch / 2
    lines = np.arange(-grid // 2 + 1, grid // 2) * pitch          # interior streets
    along = 0                                                      # 0: moving along x, 1: along z
    line = rng.choice(lines)
    coord = rng.uniform(-half + pitch, half - pitch)
    sign = 1.0
    sph_c = centers[n_box:, [0, 2]]
    sph_r = rad[n_box:]
    for i in range(n_fix):
        coord += sign * 0.3
        if abs(coord) > half - pitch:
            sign = -sign
            coord = np.clip(coord, -half + pitch, half - pitch)
        # at a crossing, turn onto the cross street half of the time
        near_cross = np.abs(coord - np.round(coord / pitch) * pitch) < 0.15
        if near_cross and rng.random() < 0.5:
            c = np.round(coord / pitch) * pitch
            if abs(c) < half - pitch / 2:
                along, line, coord = 1 - along, c, line
                sign = rng.choice([-1.0, 1.0])
        off = rng.uniform(-0.6, 0.6)
        xz = np.array([coord, line + off]) if along == 0 else np.array([line + off, coord])
        # outside every sphere (in plan, with half a metre to spare)
        d = xz[None, :] - sph_c
        dist = np.sqrt((d ** 2).sum(1))
        j = np.argmin(dist - sph_r)
        if dist[j] < sph_r[j] + 0.5:
            xz = sph_c[j] + d[j] / max(dist[j], 1e-6) * (sph_r[j] + 0.5)
        pos[i] = (xz[0], 1.7, xz[1])
    # gaze at a point on the surface of one of the 8 nearest objects
    tgt = np.zeros((n_fix, 3))
    for i0 in range(0, n_fix, 2000):
        sl = slice(i0, min(n_fix, i0 + 2000))
        m = sl.stop - sl.start
        dd = ((pos[sl, None, :] - centers[None, :, :]) ** 2).sum(-1)
        near = np.argsort(dd, axis=1)[:, :8]
        pick = near[np.arange(m), rng.integers(0, 8, size=m)]
        u = rng.normal(size=(m, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        is_box = pick < n_box
        h = np.where(is_box[:, None], ext[pick], 1.0)
        scale = np.where(is_box, 1.0 / np.max(np.abs(u) / np.maximum(h, 1e-9), axis=1), rad[pick])
        tgt[sl] = centers[pick] + u * scale[:, None]
    gaze = _jitter(rng, tgt - pos, math.radians(1.0))
    ts = np.sort(rng.uniform(0.0, duration_s, size=n_fix))
    dur = rng.uniform(0.1, 0.6, size=n_fix).astype(np.float32)
    fx = Fixations(pos.astype(np.float32), gaze.astype(np.float32), dur, ts.astype(np.float64))
    prm = Params(t_begin=0.0, t_end=duration_s, window_s=window_s)
    return Workload("city_block_5Mtri_20Msample_100kfix_600win", meshes, fx, prm, seed=seed, session=0)


def flatten(w: Workload):
    """Concatenate the meshes of a workload: (vertices, indices, transforms, per-mesh tri counts,
    per-mesh vertex counts, per-mesh density) as flat arrays for the C interfaces."""
    verts = np.concatenate([m.vertices for m in w.meshes]).astype(np.float32)
    idx = np.concatenate([m.indices for m in w.meshes]).astype(np.uint32)
    xf = np.stack([m.transform for m in w.meshes]).astype(np.float64)
    nt = np.array([m.n_tris for m in w.meshes], dtype=np.int64)
    nv = np.array([len(m.vertices) for m in w.meshes], dtype=np.int64)
    dens = np.array([m.density for m in w.meshes], dtype=np.float64)
    return verts, idx, xf, nt, nv, dens


def head_frames(fixations: Fixations, seed: int = 9, max_dev_deg: float = 15.0):
    """Head pose per fixation for the z-buffer form: the head's forward vector is the gaze turned
    by a uniform angle in [0, max_dev_deg] about a random axis perpendicular to it (the eyes look
    up to that far from straight ahead), its up hint is +y. Returns (forward, up), (n, 3) float32."""
    rng = np.random.default_rng(seed)
    g = fixations.gaze.astype(np.float64)
    g = g / np.linalg.norm(g, axis=1, keepdims=True)
    a = rng.normal(size=g.shape)
    a -= (a * g).sum(1, keepdims=True) * g
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    ang = np.radians(rng.uniform(0.0, max_dev_deg, size=len(g)))[:, None]
    fwd = g * np.cos(ang) + np.cross(a, g) * np.sin(ang)
    up = np.tile(np.array([0.0, 1.0, 0.0]), (len(g), 1))
    return fwd.astype(np.float32), up.astype(np.float32)
