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
    finally:
        G.gm_destroy(ctx)
