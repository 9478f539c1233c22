"""The allocation-free offsets entry point against the allocating path.

gm_tri_offsets_noalloc serves callers that cannot allocate device memory when they need the
per-triangle sample offsets (an engine plugin whose host owns all device memory, a per-frame
real-time thread). It must give exactly the offsets gm_sample_surface computes, call after call,
although its scratch array keeps the previous call's contents. Kept in its own file, collected
last, so that a run stopping at the first failure has run every other test before it."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_offsets_match_the_allocating_path_twice_in_a_row():
    import torch
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    from paper_2601_07571_gb300 import build
    build.build()
    import paper_2601_07571_gb300 as G
    from paper_2601_07571_gb300 import pipeline

    ctx = G.gm_create(0)
    try:
        for w in (synth.paper_scene(), synth.tiny_sphere()):
            sc = G.gm_build_scene(ctx, pipeline.mesh_args(w))
            sm = G.gm_sample_surface(sc, [m.density for m in w.meshes], w.seed, w.session)
            nt, _ = G.gm_scene_info(sc)
            ref = np.empty(nt + 1, np.int64)
            G.gm_samples_offsets(sm, ref)
            # caller-owned device buffers: world triangles, per-triangle density, output
            tri = torch.empty((nt, 9), dtype=torch.float32, device="cuda")
            G.gm_scene_triangles(sc, tri)
            dens = torch.from_numpy(np.concatenate([np.full(m.n_tris, m.density) for m in w.meshes])).cuda()
            for _ in range(2):
                out = torch.full((nt + 1,), -7, dtype=torch.int64, device="cuda")
                G.gm_tri_offsets_noalloc(ctx, tri, dens, nt, out)
                G.gm_sync(ctx)
                got = out.cpu().numpy()
                assert np.array_equal(got, ref)
            G.gm_samples_free(sm)
            G.gm_scene_free(sc)
        # sizes beyond the fixed scratch are refused before any launch
        with pytest.raises(G.GazeMapError, match="exceed the limit"):
            G.gm_tri_offsets_noalloc(ctx, tri, dens, 65536 * 2048 + 1, out)
        # the binding checks what the C entry point cannot see: dtypes and lengths
        with pytest.raises(ValueError, match="float64"):
            G.gm_tri_offsets_noalloc(ctx, tri, dens.float(), nt, out)
        with pytest.raises(ValueError, match="at least"):
            G.gm_tri_offsets_noalloc(ctx, tri, dens, nt, out[:nt])
        with pytest.raises(ValueError, match="CUDA tensor"):
            G.gm_tri_offsets_noalloc(ctx, tri.cpu(), dens, nt, out)
    finally:
        G.gm_destroy(ctx)


def _offsets_both_ways(G, pipeline, ctx, w, dens_per_mesh):
    import torch
    sc = G.gm_build_scene(ctx, pipeline.mesh_args(w))
    nt, _ = G.gm_scene_info(sc)
    tri = torch.empty((nt, 9), dtype=torch.float32, device="cuda")
    G.gm_scene_triangles(sc, tri)
    dens = torch.from_numpy(np.concatenate([np.full(m.n_tris, d) for m, d in zip(w.meshes, dens_per_mesh)])).cuda()
    out = torch.full((nt + 1,), -7, dtype=torch.int64, device="cuda")
    return sc, nt, tri, dens, out


def test_noalloc_more_than_one_scan_chunk_and_too_many_samples():
    """Three copies of the paper scene (2.4M triangles, 1 170 scan blocks) run the partial-sum
    scan's carry across its 1 024-wide chunks; a scene that needs more than 2^31 samples in total
    (every triangle well below 2^31 on its own) is refused by both paths instead of wrapping."""
    import torch
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    from paper_2601_07571_gb300 import build
    build.build()
    import paper_2601_07571_gb300 as G
    from paper_2601_07571_gb300 import pipeline

    ctx = G.gm_create(0)
    try:
        w = synth.paper_scene()
        w.meshes = list(w.meshes) * 3
        dm = [m.density for m in w.meshes]
        sc, nt, tri, dens, out = _offsets_both_ways(G, pipeline, ctx, w, dm)
        assert nt > 2_097_152
        sm = G.gm_sample_surface(sc, dm, w.seed, w.session)
        ref = np.empty(nt + 1, np.int64)
        G.gm_samples_offsets(sm, ref)
        G.gm_samples_free(sm)
        for _ in range(2):
            out.fill_(-7)
            G.gm_tri_offsets_noalloc(ctx, tri, dens, nt, out)
            G.gm_sync(ctx)
            assert np.array_equal(out.cpu().numpy(), ref)
        G.gm_scene_free(sc)

        # 1e9 samples per m^2 on the small sphere scene: about 1.3e10 samples in all, at most
        # 4e7 per triangle -- the 32.32 prefix would wrap past 2^63
        wt = synth.tiny_sphere()
        big = [1e9 for _ in wt.meshes]
        sc, nt, tri, dens, out = _offsets_both_ways(G, pipeline, ctx, wt, big)
        with pytest.raises(G.GazeMapError, match="2\\^31"):
            G.gm_sample_surface(sc, big, wt.seed, wt.session)
        G.gm_tri_offsets_noalloc(ctx, tri, dens, nt, out)
        with pytest.raises(G.GazeMapError, match="2\\^31"):
            G.gm_sync(ctx)
        assert not out.cpu().numpy().any()
        # the next call with an ordinary density is exact again (the marks left in the shared
        # scratch array are overwritten)
        dm = [m.density for m in wt.meshes]
        sm = G.gm_sample_surface(sc, dm, wt.seed, wt.session)
        ref = np.empty(nt + 1, np.int64)
        G.gm_samples_offsets(sm, ref)
        G.gm_samples_free(sm)
        dens = torch.from_numpy(np.concatenate([np.full(m.n_tris, d) for m, d in zip(wt.meshes, dm)])).cuda()
        G.gm_tri_offsets_noalloc(ctx, tri, dens, nt, out)
        G.gm_sync(ctx)
        assert np.array_equal(out.cpu().numpy(), ref)
        G.gm_scene_free(sc)
    finally:
        G.gm_destroy(ctx)
