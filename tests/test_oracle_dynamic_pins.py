"""Pins of the oracle's dynamic-scene densities (meshes posed per window, samples attached to
their triangles) to facts outside its triangle arithmetic: a box that moves between windows
casts its shadow where an FP64 slab test puts it; moving the whole scene and the eyes by one
rigid motion leaves the densities unchanged; a scene that does not move gives the static
densities exactly."""
import math

import numpy as np

import oracle
import synth
from synth import meshes as M
from tests.parity_utils import ulp32
from tests.test_oracle_pins import _fix, _slab_hits


def _plane(g=24, half=1.0):
    xs = np.linspace(-half, half, g + 1)
    v = np.array([(x, y, 0.0) for x in xs for y in xs], np.float32)
    f = []
    for i in range(g):
        for j in range(g):
            a, b, c, d = i * (g + 1) + j, (i + 1) * (g + 1) + j, (i + 1) * (g + 1) + j + 1, i * (g + 1) + j + 1
            f += [(a, b, c), (a, c, d)]
    return v, np.array(f, np.uint32)


def _translate(t):
    T = np.eye(4)
    T[:3, 3] = t
    return T


def moving_box_workload():
    """A plane (fixed) and a box (half sizes 0.11 x 0.12 x 0.125, centre (-0.01, 0.02, 0.475) at
    rest) seen from one eye in each of three one-second windows; the box moves by +0.45 m in x in
    window 1 and leaves the view in window 2."""
    pv, pf = _plane()
    half = np.array([0.11, 0.12, 0.125])
    centre = np.array([-0.01, 0.02, 0.475])
    bv, bf = M.box((0.0, 0.0, 0.0), half)
    meshes = [synth.Mesh(pv, pf, synth.identity(), 0, 20000.0),
              synth.Mesh(np.asarray(bv, np.float32), np.asarray(bf, np.uint32), _translate(centre), 1, 20000.0)]
    eye = np.array([[0.05, -0.05, 2.0]] * 3)
    gaze = np.array([[0.02, 0.03, -2.0]] * 3)
    fx = _fix(eye, gaze, ts=[0.5, 1.5, 2.5])
    params = synth.Params(theta_rad=math.radians(6.0), t_begin=0.0, t_end=3.0, window_s=1.0)
    w = synth.Workload("moving_box", meshes, fx, params, seed=11)
    shifts = [np.zeros(3), np.array([0.45, 0.0, 0.0]), np.array([0.0, 0.0, 50.0])]
    xf = np.stack([[synth.identity(), _translate(centre + d)] for d in shifts])
    boxes = [(centre + d - half, centre + d + half) for d in shifts]
    return w, xf, boxes


def test_moving_box_shadow_follows_the_box():
    w, xf, boxes = moving_box_workload()
    r = oracle.run_dynamic(w, xf, delta_abs=1e-9)
    tri = oracle.world_triangles(w)
    off = r["offsets"]
    smp = oracle.samples(tri, off, w.seed, w.session)
    on_plane = smp.tri < 2 * 24 * 24
    e = w.fixations.eye[0].astype(np.float64)
    d = smp.xyz - e
    tmax = 1 - w.params.eps_rel
    lit = r["density"] > 0
    shadow_counts = []
    for k, (lo, hi) in enumerate(boxes):
        occ = _slab_hits(e, d, lo, hi, tmax)
        sure = _slab_hits(e, d, lo - 1e-7, hi + 1e-7, tmax) == _slab_hits(e, d, lo + 1e-7, hi - 1e-7, tmax)
        sel = on_plane & sure & (r["amb"][k] == 0)
        assert not np.any(lit[k][sel & occ])                  # the shadow of this window's box is dark
        shadow_counts.append(int((on_plane & occ).sum()))
    assert shadow_counts[0] > 200 and shadow_counts[1] > 200 and shadow_counts[2] == 0
    # the shadow moved: samples dark in window 0 are lit in window 1 and all lit in window 2
    occ0 = _slab_hits(e, d, *boxes[0], tmax)
    occ1 = _slab_hits(e, d, *boxes[1], tmax)
    moved = on_plane & occ0 & ~occ1 & lit[2]
    assert moved.sum() > 100 and np.all(lit[1][moved])
    assert np.array_equal(lit[2][on_plane], (r["density"][2] > 0)[on_plane])
    assert (lit[2][on_plane]).sum() > (lit[0][on_plane]).sum()


def test_rigid_motion_of_scene_and_eyes_leaves_densities_unchanged():
    w = synth.tiny_sphere(n_fix=40)
    n = w.fixations.n
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])   # exact quarter turn about z
    t = np.array([2.0, -1.0, 0.5])
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = R, t
    fx = w.fixations
    eye = np.concatenate([fx.eye, (fx.eye.astype(np.float64) @ R.T + t).astype(np.float32)])
    gaze = np.concatenate([fx.gaze, (fx.gaze.astype(np.float64) @ R.T).astype(np.float32)])
    ts = np.concatenate([np.full(n, 0.25), np.full(n, 1.25)])
    w.fixations = synth.Fixations(eye, gaze, np.concatenate([fx.duration_s, fx.duration_s]), ts)
    w.params = synth.Params(t_begin=0.0, t_end=2.0, window_s=1.0)
    rest = [m.transform for m in w.meshes]
    xf = np.stack([rest, [T @ m for m in rest]])
    r = oracle.run_dynamic(w, xf, delta_abs=2e-5, cone_band=1e-4)
    d0, d1 = r["density"]
    assert (d0 > 0).sum() > 300
    tol = 1e-9 * d0 + r["amb"][0] + r["amb"][1] + (r["sens"][0] + r["sens"][1]) * 16 * ulp32(6.0) + 1e-300
    assert np.all(np.abs(d1 - d0) <= tol)


def test_scene_at_rest_gives_the_static_densities():
    w = synth.tiny_sphere(n_fix=60)
    w.params = synth.Params(t_begin=0.0, t_end=24.0, window_s=6.0)
    rest = np.stack([m.transform for m in w.meshes])
    r = oracle.run_dynamic(w, np.stack([rest] * 4))
    s = oracle.run(w)
    assert np.array_equal(r["density"], s["density"])
    assert (s["density"] > 0).sum(1).min() > 50
