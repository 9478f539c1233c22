"""The paper's grid sampler on the GPU (Section 3.1) against the oracle: resolutions and offsets
bit-exact, grid barycentrics, positions, and the densities accumulated on the grid samples."""
import numpy as np
import pytest

import oracle
import synth
from tests.parity_utils import tri_max_coord, ulp32

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


@pytest.mark.parametrize("which", ["tiny", "paper"])
def test_grid_sampler_parity(env, which):
    G, pipe, ctx = env
    w = synth.tiny_sphere() if which == "tiny" else synth.paper_scene(density=4000.0)
    tri = oracle.world_triangles(w)
    r, _ = oracle.grid_resolution(oracle.areas(tri), oracle.tri_density(w))
    off = oracle.grid_offsets(r)
    sc = G.gm_build_scene(ctx, pipe.mesh_args(w))
    sm = G.gm_sample_surface_grid(sc, [m.density for m in w.meshes])
    n = G.gm_samples_info(sm)
    goff = np.empty(len(tri) + 1, np.int64)
    G.gm_samples_offsets(sm, goff)
    assert n == off[-1] and np.array_equal(goff, off)
    xyz = np.empty((n, 3), np.float32)
    st = np.empty(n, np.uint32)
    b2 = np.empty((n, 2), np.float32)
    G.gm_samples_copy(sm, xyz, st, b2, None)
    G.gm_samples_free(sm)
    G.gm_scene_free(sc)
    s = oracle.grid_samples(tri, off, r)
    assert np.array_equal(st.astype(np.int64), s["tri"])
    assert np.abs(b2.astype(np.float64) - s["bary"][:, 1:]).max() <= 2.0 ** -22
    M = tri_max_coord(tri, s["tri"])
    assert np.all(np.abs(xyz.astype(np.float64) - s["xyz"]) <= 8 * ulp32(M)[:, None])


def test_grid_densities_against_oracle(env):
    G, pipe, ctx = env
    w = synth.tiny_sphere()
    tri = oracle.world_triangles(w)
    r, _ = oracle.grid_resolution(oracle.areas(tri), oracle.tri_density(w))
    off = oracle.grid_offsets(r)
    s = oracle.grid_samples(tri, off, r)
    ora = oracle.accumulate(tri, s["xyz"], s["tri"], w.fixations, w.params, delta_abs=2e-5, cone_band=1e-4)
    sc = G.gm_build_scene(ctx, pipe.mesh_args(w))
    sm = G.gm_sample_surface_grid(sc, [m.density for m in w.meshes])
    eye, gaze, dur, ts = pipe.fixation_args(w.fixations)
    m = G.gm_accumulate_fixations(sc, sm, eye, gaze, dur, ts, pipe.params_of(w, normalize=False))
    v = np.empty(G.gm_samples_info(sm), np.float32)
    G.gm_map_copy(m, 0, v)
    G.gm_map_free(m)
    G.gm_samples_free(sm)
    G.gm_scene_free(sc)
    d = ora["density"][0]
    assert (d > 0).sum() > 100
    tol = 1e-4 * (d + ora["amb"][0]) + ora["amb"][0] + ora["sens"][0] * 8 * ulp32(tri_max_coord(tri, s["tri"])) + 1e-30
    assert np.all(np.abs(v.astype(np.float64) - d) <= tol)
