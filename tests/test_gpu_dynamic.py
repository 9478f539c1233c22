"""Dynamic scenes on the GPU (gm_scene_pose, gm_samples_follow, gm_accumulate_dynamic) against the
oracle: posed triangles bit-exact, followed samples within FP32 rounding, per-window densities
within the accumulation tolerance, and a pose equal to the build's transforms changes nothing."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.parity_utils import tri_max_coord, ulp32
from tests.test_oracle_dynamic_pins import moving_box_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_07571_gb300 import build
    build.build()
    import paper_2601_07571_gb300 as G
    from paper_2601_07571_gb300 import pipeline
    ctx = G.gm_create(0)
    yield G, pipeline, ctx
    G.gm_destroy(ctx)


def _rot(axis, a):
    c, s = math.cos(a), math.sin(a)
    i, j = [(1, 2), (2, 0), (0, 1)][axis]
    R = np.eye(4)
    R[i, i], R[i, j], R[j, i], R[j, j] = c, -s, s, c
    return R


def spinning_workload():
    """tiny_sphere over four 8-second windows: the sphere turns and stretches, the cube orbits."""
    w = synth.tiny_sphere(n_fix=100)
    w.params = synth.Params(t_begin=0.0, t_end=32.0, window_s=8.0)
    xf = []
    for k in range(4):
        S = np.diag([1.0 + 0.1 * k, 1.0, 1.0 - 0.05 * k, 1.0])
        cube = _rot(2, 0.6 * k) @ np.eye(4)
        xf.append([_rot(1, 0.4 * k) @ S, cube])
    return w, np.array(xf)


def _scene_tris(G, sc, n):
    t = np.empty((n, 9), np.float32)
    G.gm_scene_triangles(sc, t)
    return t


def test_pose_triangles_bit_exact_and_rest_pose_is_identity(env):
    G, pipe, ctx = env
    w, xf = spinning_workload()
    sc = G.gm_build_scene(ctx, pipe.mesh_args(w), dynamic=True)
    nt = w.n_tris
    built = _scene_tris(G, sc, nt)
    G.gm_scene_pose(sc, xf[2])
    posed = w.meshes
    wk = synth.Workload(w.name, [synth.Mesh(m.vertices, m.indices, T, m.object_id, m.density)
                                 for m, T in zip(posed, xf[2])], w.fixations, w.params)
    assert np.array_equal(_scene_tris(G, sc, nt).view(np.uint32), oracle.world_triangles(wk).view(np.uint32))
    G.gm_scene_pose(sc, np.stack([m.transform for m in w.meshes]))
    assert np.array_equal(_scene_tris(G, sc, nt).view(np.uint32), built.view(np.uint32))
    G.gm_scene_free(sc)


def test_rest_pose_maps_equal_static_maps(env):
    G, pipe, ctx = env
    w = synth.tiny_sphere()
    h = pipe.run(ctx, w, normalize=False)
    static = pipe.map_array(h)[0]
    h.free()
    sc = G.gm_build_scene(ctx, pipe.mesh_args(w), dynamic=True)
    sm = G.gm_sample_surface(sc, [m.density for m in w.meshes], w.seed, w.session)
    eye, gaze, dur, ts = pipe.fixation_args(w.fixations)
    rest = np.stack([m.transform for m in w.meshes])[None]
    m = G.gm_accumulate_dynamic(sc, sm, eye, gaze, dur, ts, pipe.params_of(w, normalize=False), rest)
    v = np.empty(G.gm_samples_info(sm), np.float32)
    G.gm_map_copy(m, 0, v)
    assert np.array_equal(v.view(np.uint32), static.view(np.uint32))
    G.gm_map_free(m)
    G.gm_samples_free(sm)
    G.gm_scene_free(sc)


@pytest.mark.parametrize("case", ["spinning", "moving_box"])
def test_dynamic_accumulation_against_oracle(env, case):
    G, pipe, ctx = env
    w, xf = spinning_workload() if case == "spinning" else moving_box_workload()[:2]
    r = oracle.run_dynamic(w, xf, delta_abs=2e-5, cone_band=1e-4)
    sc = G.gm_build_scene(ctx, pipe.mesh_args(w), dynamic=True)
    sm = G.gm_sample_surface(sc, [m.density for m in w.meshes], w.seed, w.session)
    n = G.gm_samples_info(sm)
    assert n == r["offsets"][-1]
    eye, gaze, dur, ts = pipe.fixation_args(w.fixations)
    m = G.gm_accumulate_dynamic(sc, sm, eye, gaze, dur, ts, pipe.params_of(w, normalize=False), xf)
    W, ns, stats, _ = G.gm_map_info(m)
    assert W == len(xf) and ns == n
    assert stats["n_fixations_used"] == int((oracle.fixation_windows(w.fixations.timestamp_s, w.params) >= 0).sum())
    # the samples are left in the last window's pose
    wl = synth.Workload(w.name, [synth.Mesh(mm.vertices, mm.indices, T, mm.object_id, mm.density)
                                 for mm, T in zip(w.meshes, xf[-1])], w.fixations, w.params)
    tri_l = oracle.world_triangles(wl)
    smp_l = oracle.samples(tri_l, r["offsets"], w.seed, w.session)
    xyz = np.empty((n, 3), np.float32)
    st = np.empty(n, np.uint32)
    G.gm_samples_copy(sm, xyz, st, None, None)
    assert np.array_equal(st.astype(np.int64), smp_l.tri)
    Ml = tri_max_coord(tri_l, smp_l.tri)
    assert np.all(np.abs(xyz.astype(np.float64) - smp_l.xyz) <= 8 * ulp32(Ml)[:, None])
    for k in range(W):
        v = np.empty(n, np.float32)
        G.gm_map_copy(m, k, v)
        d = r["density"][k]
        wk = synth.Workload(w.name, [synth.Mesh(mm.vertices, mm.indices, T, mm.object_id, mm.density)
                                     for mm, T in zip(w.meshes, xf[k])], w.fixations, w.params)
        tri_k = oracle.world_triangles(wk)
        M = tri_max_coord(tri_k, smp_l.tri)
        tol = 1e-4 * (d + r["amb"][k]) + r["amb"][k] + r["sens"][k] * 8 * ulp32(M) + 1e-30
        assert (d > 0).sum() > 20
        assert np.all(np.abs(v.astype(np.float64) - d) <= tol), k
    G.gm_map_free(m)
    # normalised: every window divided by its own maximum
    m = G.gm_accumulate_dynamic(sc, sm, eye, gaze, dur, ts, pipe.params_of(w, normalize=True), xf)
    for k in range(W):
        v = np.empty(n, np.float32)
        G.gm_map_copy(m, k, v)
        assert abs(float(v.max()) - 1.0) <= 1e-6
    G.gm_map_free(m)
    G.gm_samples_free(sm)
    G.gm_scene_free(sc)


def test_dynamic_argument_errors(env):
    G, pipe, ctx = env
    w = synth.tiny_sphere()
    rest = np.stack([m.transform for m in w.meshes])
    sc = G.gm_build_scene(ctx, pipe.mesh_args(w))
    with pytest.raises(RuntimeError, match="dynamic"):
        G.gm_scene_pose(sc, rest)
    G.gm_scene_free(sc)
    sc = G.gm_build_scene(ctx, pipe.mesh_args(w), dynamic=True)
    pts = G.gm_samples_from_points(sc, np.zeros((4, 3), np.float32), np.zeros(4, np.uint32))
    with pytest.raises(RuntimeError, match="explicit points"):
        G.gm_samples_follow(pts)
    bad = rest.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(RuntimeError, match="non-finite"):
        G.gm_scene_pose(sc, bad)
    G.gm_samples_free(pts)
    G.gm_scene_free(sc)
