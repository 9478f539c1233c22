"""The sample-sharded path on one GPU: the ranks of a 2- and 3-way split run one after another in
this process (each its slice of the samples through gm_samples_slice and gm_accumulate_fixations),
the per-window maxima are combined on the host as the all-reduce would, and every slice is
normalised by them with gm_map_normalize. Concatenated, the slices equal the single-call map bit
for bit, raw and normalised. (No kernel waits for another rank: nothing here needs several GPUs.)"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_07571_gb300 import build
    build.build()
    import paper_2601_07571_gb300 as G
    from paper_2601_07571_gb300 import pipeline, shard
    ctx = G.gm_create(0)
    yield G, pipeline, shard, ctx
    G.gm_destroy(ctx)


def _windows(G, pipeline, m, W, n):
    return np.stack([_copy(G, m, k, n) for k in range(W)])


def _copy(G, m, k, n):
    v = np.empty(n, np.float32)
    G.gm_map_copy(m, k, v)
    return v


@pytest.mark.parametrize("which", ["tiny_windows", "session", "paper"])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_slices_equal_the_single_map(env, which, world):
    G, pipeline, shard, ctx = env
    if which == "tiny_windows":
        w = synth.tiny_sphere(n_fix=200)
        ts = w.fixations.timestamp_s
        w.params = synth.Params(t_begin=0.0, t_end=float(ts.max()) + 1.0, window_s=10.0)
    elif which == "session":
        w = synth.session(9)
        w.fixations = w.fixations.subset(slice(0, 400))
    else:
        w = synth.paper_scene()
        w.fixations = w.fixations.subset(slice(0, 600))
    W = pipeline.n_windows(w)
    h = pipeline.run(ctx, w, normalize=False)
    n = h.n_samples
    raw = _windows(G, pipeline, h.map, W, n)
    mx_single = np.empty(W, np.float32)
    G.gm_map_max(h.map, mx_single)
    G.gm_map_normalize(h.map)
    norm = _windows(G, pipeline, h.map, W, n)
    h.free()
    parts = [shard.accumulate_shard(ctx, w, r, world) for r in range(world)]
    gmax = np.max(np.stack([p[4] for p in parts]), axis=0)   # what the all-reduce computes
    assert np.array_equal(gmax, mx_single)
    raw_parts, norm_parts = [], []
    for sc, part, m, (b, e), _ in parts:
        raw_parts.append(_windows(G, pipeline, m, W, e - b))
        shard.normalize_shard(m, gmax)
        norm_parts.append(_windows(G, pipeline, m, W, e - b))
        back = np.empty(W, np.float32)
        G.gm_map_max(m, back)
        assert np.array_equal(back, gmax)
        G.gm_map_free(m)
        G.gm_samples_free(part)
        G.gm_scene_free(sc)
    assert parts[0][3][0] == 0 and parts[-1][3][1] == n
    assert np.array_equal(np.concatenate(raw_parts, axis=1).view(np.uint32), raw.view(np.uint32))
    assert np.array_equal(np.concatenate(norm_parts, axis=1).view(np.uint32), norm.view(np.uint32))
    assert (raw > 0).sum() > 100


def test_slice_and_normalize_refuse_bad_arguments(env):
    G, pipeline, shard, ctx = env
    w = synth.tiny_sphere(n_fix=10)
    h = pipeline.run(ctx, w, normalize=False)
    with pytest.raises(G.GazeMapError):
        G.gm_samples_slice(h.samples, 10, 5)
    with pytest.raises(G.GazeMapError):
        G.gm_samples_slice(h.samples, 0, h.n_samples + 1)
    empty = G.gm_samples_slice(h.samples, 3, 3)
    assert G.gm_samples_info(empty) == 0
    G.gm_samples_free(empty)
    with pytest.raises(G.GazeMapError):
        G.gm_map_normalize(h.map, np.array([np.nan], np.float32))
    h.free()
