"""Seeded procedural meshes used as synthetic stand-ins for the paper's scenes.

The paper measures on recorded scenes (an angel statue, a cube, a bunny with two
very different mesh densities; Fig. 1 and Section 4) that are not available, so
every workload here is built from procedural meshes with the same traits:
many triangles, curved closed surfaces, and regions whose triangle sizes differ
by an order of magnitude.

This module builds geometry only (vertex and index arrays). It holds none of
the gaze-mapping arithmetic: no areas, no sampling, no cone or ray tests.
"""
from __future__ import annotations

import numpy as np


def icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
    ], dtype=np.float64)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def icosphere(subdiv: int, radius: float = 1.0):
    """Icosahedron with `subdiv` midpoint subdivisions, re-projected to the sphere.

    20 * 4**subdiv triangles, counter-clockwise seen from outside.
    """
    v, f = icosahedron()
    verts = [tuple(x) for x in v]
    for _ in range(subdiv):
        cache = {}
        nf = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key in cache:
                return cache[key]
            p = (np.asarray(verts[a]) + np.asarray(verts[b])) * 0.5
            p /= np.linalg.norm(p)
            verts.append(tuple(p))
            cache[key] = len(verts) - 1
            return cache[key]

        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        f = np.asarray(nf, dtype=np.int64)
    v = np.asarray(verts, dtype=np.float64) * radius
    return v.astype(np.float32), f.astype(np.uint32)


def box(center, half):
    """Axis-aligned box with half-extents `half` (scalar or 3-vector): 8 vertices, 12 triangles,
    counter-clockwise seen from outside."""
    c = np.asarray(center, dtype=np.float64)
    h = np.broadcast_to(np.asarray(half, dtype=np.float64), (3,))
    s = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], dtype=np.float64)
    v = c + s * h
    # vertex id = 4*ix + 2*iy + iz
    f = np.array([
        [0, 1, 3], [0, 3, 2],      # x = -1
        [4, 6, 7], [4, 7, 5],      # x = +1
        [0, 4, 5], [0, 5, 1],      # y = -1
        [2, 3, 7], [2, 7, 6],      # y = +1
        [0, 2, 6], [0, 6, 4],      # z = -1
        [1, 5, 7], [1, 7, 3],      # z = +1
    ], dtype=np.uint32)
    return v.astype(np.float32), f


def _value_noise(rng: np.random.Generator, pts: np.ndarray, freq: float) -> np.ndarray:
    """Smooth 3-D value noise in [-1, 1]: a random lattice, trilinear blend with smoothstep."""
    n = 64
    lattice = rng.uniform(-1.0, 1.0, size=(n, n, n))
    q = pts * freq + n / 2.0
    i0 = np.floor(q).astype(np.int64)
    fr = q - i0
    w = fr * fr * (3.0 - 2.0 * fr)
    out = np.zeros(len(pts))
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                ix = (i0[:, 0] + dx) % n
                iy = (i0[:, 1] + dy) % n
                iz = (i0[:, 2] + dz) % n
                wx = w[:, 0] if dx else 1.0 - w[:, 0]
                wy = w[:, 1] if dy else 1.0 - w[:, 1]
                wz = w[:, 2] if dz else 1.0 - w[:, 2]
                out += wx * wy * wz * lattice[ix, iy, iz]
    return out


def uv_sphere(n_lat: int, n_lon: int, radius: float = 1.0, noise_amp: float = 0.0,
              noise_freq: float = 3.0, seed: int = 0):
    """Latitude/longitude sphere, optionally displaced radially by value noise.

    n_lat bands (n_lat - 1 vertex rings plus two poles), n_lon segments:
    2 * n_lon * (n_lat - 1) triangles, counter-clockwise seen from outside.
    """
    rng = np.random.default_rng(seed)
    th = np.pi * np.arange(1, n_lat) / n_lat                  # polar angle of each ring
    ph = 2.0 * np.pi * np.arange(n_lon) / n_lon
    st, ct = np.sin(th)[:, None], np.cos(th)[:, None]
    ring = np.stack([st * np.cos(ph)[None, :], ct * np.ones_like(ph)[None, :],
                     st * np.sin(ph)[None, :]], axis=-1).reshape(-1, 3)
    dirs = np.concatenate([[[0.0, 1.0, 0.0]], ring, [[0.0, -1.0, 0.0]]], axis=0)
    r = np.full(len(dirs), float(radius))
    if noise_amp > 0:
        r = radius * (1.0 + noise_amp * _value_noise(rng, dirs, noise_freq))
    v = dirs * r[:, None]
    top, bot = 0, len(dirs) - 1

    def vid(i, j):  # ring i in [0, n_lat-2], segment j
        return 1 + i * n_lon + (j % n_lon)

    j = np.arange(n_lon)
    faces = [np.stack([np.full(n_lon, top), vid(0, j + 1), vid(0, j)], axis=1)]
    for i in range(n_lat - 2):
        a, b = vid(i, j), vid(i, j + 1)
        c, d = vid(i + 1, j), vid(i + 1, j + 1)
        faces.append(np.stack([a, b, d], axis=1))
        faces.append(np.stack([a, d, c], axis=1))
    faces.append(np.stack([vid(n_lat - 2, j), vid(n_lat - 2, j + 1), np.full(n_lon, bot)], axis=1))
    f = np.concatenate(faces, axis=0)
    return v.astype(np.float32), f.astype(np.uint32)


def torus_knot(n_seg: int, n_ring: int, p: int = 2, q: int = 3, scale: float = 1.0,
               tube: float = 0.25):
    """(p, q) torus knot swept by a circular tube: 2 * n_seg * n_ring triangles."""
    t = 2.0 * np.pi * np.arange(n_seg) / n_seg

    def curve(tt):
        rr = 2.0 + np.cos(q * tt)
        return np.stack([rr * np.cos(p * tt), -np.sin(q * tt), rr * np.sin(p * tt)], axis=-1)

    c = curve(t)
    tan = curve(t + 1e-4) - curve(t - 1e-4)
    tan /= np.linalg.norm(tan, axis=1, keepdims=True)
    # a normal from the curvature direction (the knot has no inflection points for these p, q)
    nrm = curve(t + 1e-3) + curve(t - 1e-3) - 2.0 * c
    nrm -= (nrm * tan).sum(1, keepdims=True) * tan
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    bin_ = np.cross(tan, nrm)
    a = 2.0 * np.pi * np.arange(n_ring) / n_ring
    v = (c[:, None, :] + tube * (np.cos(a)[None, :, None] * nrm[:, None, :]
                                 + np.sin(a)[None, :, None] * bin_[:, None, :]))
    v = (v * scale / 3.25).reshape(-1, 3)
    i = np.arange(n_seg)[:, None]
    j = np.arange(n_ring)[None, :]
    a0 = i * n_ring + j
    a1 = ((i + 1) % n_seg) * n_ring + j
    b0 = i * n_ring + (j + 1) % n_ring
    b1 = ((i + 1) % n_seg) * n_ring + (j + 1) % n_ring
    f = np.concatenate([np.stack([a0, a1, b1], -1).reshape(-1, 3),
                        np.stack([a0, b1, b0], -1).reshape(-1, 3)], axis=0)
    return v.astype(np.float32), f.astype(np.uint32)


def merge(parts):
    """Concatenate (vertices, faces) pairs into one mesh."""
    vs, fs, off = [], [], 0
    for v, f in parts:
        vs.append(np.asarray(v, dtype=np.float32))
        fs.append(np.asarray(f, dtype=np.int64) + off)
        off += len(v)
    return np.concatenate(vs).astype(np.float32), np.concatenate(fs).astype(np.uint32)


def translate(v, t):
    return (np.asarray(v, dtype=np.float64) + np.asarray(t, dtype=np.float64)).astype(np.float32)


def mixed_density_blob(seed: int, n_coarse: int = 75_000, n_fine: int = 75_000):
    """Two-density blob: a coarse displaced body whose triangles have edges near 1 cm and a
    small dense cap whose triangles have edges near 1 mm, in one mesh (like the bunny of Fig. 1
    with two very different mesh densities)."""
    def grid(n):
        # 2 * n_lon * (n_lat - 1) ~ n with n_lon = 2 * n_lat
        n_lat = max(3, int(round((n / 4.0) ** 0.5)))
        return n_lat, 2 * n_lat
    lat_c, lon_c = grid(n_coarse)
    lat_f, lon_f = grid(n_fine)
    body = uv_sphere(lat_c, lon_c, radius=0.55, noise_amp=0.06, noise_freq=4.0, seed=seed)
    cap = uv_sphere(lat_f, lon_f, radius=0.055, noise_amp=0.05, noise_freq=30.0, seed=seed + 1)
    cap = (translate(cap[0], (0.0, 0.58, 0.0)), cap[1])
    return merge([body, cap])
