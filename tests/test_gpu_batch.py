"""Batched sessions in one persistent, graph-captured launch, and the autotuner (GPU).

Each session's map from the batch must be bit-identical to the plain single-session call (the
batch runs the same warp-tile code on the same inputs, in the same fixation order), and one
session is also checked against the oracle on a sample of its samples."""
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


def _small_sessions(n=6):
    out = []
    for i in range(n):
        w = synth.session(i, tri_range=(2_000, 20_000), fix_range=(50, 400), density_range=(500, 4000))
        out.append(w)
    return out


def _prepare(G, pipe, ctx, ws):
    handles = []
    for w in ws:
        sc = G.gm_build_scene(ctx, pipe.mesh_args(w))
        sm = G.gm_sample_surface(sc, [m.density for m in w.meshes], w.seed, w.session)
        handles.append((sc, sm, *pipe.fixation_args(w.fixations)))
    return handles


@pytest.mark.parametrize("windows", [False, True])
def test_batch_equals_plain_per_session(env, windows):
    G, pipe, ctx = env
    ws = _small_sessions()
    if windows:
        for w in ws:
            w.params = synth.Params(t_begin=0.0, t_end=float(w.fixations.timestamp_s.max()) + 1.0, window_s=20.0)
    tmax = max(float(w.fixations.timestamp_s.max()) for w in ws) + 1.0
    prm_w = synth.Params(t_begin=0.0, t_end=tmax, window_s=20.0) if windows else synth.Params()
    for w in ws:
        w.params = prm_w
    hs = _prepare(G, pipe, ctx, ws)
    prm = pipe.params_of(ws[0], normalize=True)
    b = G.gm_batch_create(ctx, hs, prm)
    info = G.gm_batch_info(b)
    assert info["n_sessions"] == len(ws) and info["n_work_items"] > 0
    for rep in range(2):                       # replaying the graph gives the same maps
        G.gm_batch_run(b)
        for i, (w, h) in enumerate(zip(ws, hs)):
            mb = G.gm_batch_map(b, i)
            W, ns, st, status = G.gm_map_info(mb)
            assert st["n_fixations_used"] <= w.fixations.n
            ref = G.gm_accumulate_fixations(h[0], h[1], *h[2:], prm)
            W2, ns2, st2, _ = G.gm_map_info(ref)
            assert (W, ns, st["in_cone"], st["visible"]) == (W2, ns2, st2["in_cone"], st2["visible"])
            for k in range(W):
                a = np.empty(ns, np.float32)
                c = np.empty(ns, np.float32)
                ma = G.gm_map_copy(mb, k, a)
                mc = G.gm_map_copy(ref, k, c)
                assert ma == mc
                assert np.array_equal(a.view(np.uint32), c.view(np.uint32))
            G.gm_map_free(ref)
    G.gm_batch_free(b)
    for sc, sm, *_ in hs:
        G.gm_samples_free(sm)
        G.gm_scene_free(sc)


def test_batch_session_against_oracle(env):
    G, pipe, ctx = env
    ws = _small_sessions(4)
    hs = _prepare(G, pipe, ctx, ws)
    prm = pipe.params_of(ws[0], normalize=False)
    maps = G.gm_accumulate_batch(ctx, hs, prm)
    w = ws[2]
    r_tri = oracle.world_triangles(w)
    off = oracle.tri_offsets(oracle.areas(r_tri), oracle.tri_density(w))
    rng = np.random.default_rng(5)
    which = np.sort(rng.choice(int(off[-1]), 300, replace=False)).astype(np.int64)
    s = oracle.samples(r_tri, off, w.seed, w.session, which)
    ora = oracle.accumulate(r_tri, s.xyz, s.tri, w.fixations, w.params, delta_abs=2e-5, cone_band=1e-4)
    v = np.empty(int(off[-1]), np.float32)
    G.gm_map_copy(maps[2], 0, v)
    d = ora["density"][0]
    tol = 1e-4 * (d + ora["amb"][0]) + ora["amb"][0] + ora["sens"][0] * 8 * ulp32(tri_max_coord(r_tri, s.tri)) + 1e-30
    assert np.all(np.abs(v[which].astype(np.float64) - d) <= tol)
    for m in maps:
        G.gm_map_free(m)
    for sc, sm, *_ in hs:
        G.gm_samples_free(sm)
        G.gm_scene_free(sc)


def _batch_variant_flags(G):
    """The batched kernel variants: ray queue or in-place tracing, binary or 4-wide tree, 80- or
    64-register cap; the ray-queue binary tree with 4, 2 or 1 samples per thread."""
    out = []
    for code in range(8):
        f = ((0 if code & 1 else G.GM_F_NO_COMPACT) | (G.GM_F_WIDE_BVH if code & 2 else 0)
             | (G.GM_F_REGCAP64 if code & 4 else 0))
        if code & 3 == 1:
            out += [f | G.GM_F_SPT4, f | G.GM_F_SPT2] + ([f] if code == 1 else [])
        else:
            out.append(f)
    return out


def test_batched_variants_agree_bit_for_bit(env):
    """Every batched kernel variant gives the same maps: the same additions per sample in the
    same order, each weight rounded on its own before it enters the compensated sum."""
    G, pipe, ctx = env
    ws = _small_sessions(3)
    hs = _prepare(G, pipe, ctx, ws)
    ref = None
    for code, f in enumerate(_batch_variant_flags(G)):
        b = G.gm_batch_create(ctx, hs, pipe.params_of(ws[0], normalize=False, flags=f))
        G.gm_batch_run(b)
        maps = []
        for i in range(len(ws)):
            a = np.empty(G.gm_samples_info(hs[i][1]), np.float32)
            G.gm_map_copy(G.gm_batch_map(b, i), 0, a)
            maps.append(a.view(np.uint32))
        G.gm_batch_free(b)
        if ref is None:
            ref = maps
        for a, r in zip(maps, ref):
            assert np.array_equal(a, r), code


def test_autotune_picks_a_variant_and_keeps_results(env, tmp_path, monkeypatch):
    G, pipe, ctx = env
    ws = _small_sessions(3)
    hs = _prepare(G, pipe, ctx, ws)
    prm = pipe.params_of(ws[0], normalize=False)
    b = G.gm_batch_create(ctx, hs, prm)
    G.gm_batch_run(b)
    before = []
    for i in range(len(ws)):
        a = np.empty(G.gm_samples_info(hs[i][1]), np.float32)
        G.gm_map_copy(G.gm_batch_map(b, i), 0, a)
        before.append(a)
    flags, ms = G.gm_batch_autotune(b)
    assert flags in _batch_variant_flags(G) and ms > 0
    assert G.gm_batch_info(b)["variant_flags"] == flags
    G.gm_batch_run(b)
    G.gm_sync(ctx)
    bk = G.gm_batch_buckets(b)
    # every session in the bucket of its triangle count (< 2^14, < 2^17, more); each bucket's
    # launch is timed
    nts = [G.gm_scene_info(h[0])[0] for h in hs]
    want = [sum(1 for nt in nts if (nt < 2 ** 14 if k == 0 else 2 ** 14 <= nt < 2 ** 17 if k == 1 else nt >= 2 ** 17))
            for k in range(3)]
    assert [x["sessions"] for x in bk] == want
    assert sum(x["work_items"] for x in bk) == G.gm_batch_info(b)["n_work_items"]
    for x in bk:
        assert x["flags"] in _batch_variant_flags(G)
        assert (x["ms"] > 0) == (x["work_items"] > 0)
    for i in range(len(ws)):
        a = np.empty_like(before[i])
        G.gm_map_copy(G.gm_batch_map(b, i), 0, a)
        assert np.array_equal(a.view(np.uint32), before[i].view(np.uint32))
    G.gm_batch_free(b)
    fl2, _ = G.gm_autotune_accumulate(hs[0][0], hs[0][1], *hs[0][2:], prm)
    shape = (G.GM_F_NO_COMPACT | G.GM_F_WIDE_BVH | G.GM_F_REGCAP64 | G.GM_F_TILE_CONSECUTIVE | G.GM_F_STATIC_TILES
             | G.GM_F_BLOCK128 | G.GM_F_EYE_GRID | G.GM_F_GRID64 | G.GM_F_SPT1 | G.GM_F_SPT2 | G.GM_F_SPT4
             | G.GM_F_BLOCK512)
    assert fl2 & ~shape == 0
    if not fl2 & G.GM_F_EYE_GRID:
        assert not fl2 & G.GM_F_GRID64
        if fl2 & G.GM_F_SPT1:        # only as the in-place one-sample form (the ray-queue default needs no flag)
            assert fl2 & G.GM_F_NO_COMPACT and not fl2 & (G.GM_F_WIDE_BVH | G.GM_F_BLOCK128 | G.GM_F_BLOCK512)
        if fl2 & (G.GM_F_BLOCK128 | G.GM_F_BLOCK512 | G.GM_F_SPT2 | G.GM_F_SPT4):
            # only offered for the ray-queue binary-tree kernels
            assert not fl2 & (G.GM_F_NO_COMPACT | G.GM_F_WIDE_BVH)
        if fl2 & G.GM_F_BLOCK512:   # one sample per thread
            assert not fl2 & (G.GM_F_SPT2 | G.GM_F_SPT4 | G.GM_F_BLOCK128)
    else:                            # eye-grid shapes only
        assert not fl2 & (G.GM_F_NO_COMPACT | G.GM_F_WIDE_BVH | G.GM_F_REGCAP64 | G.GM_F_STATIC_TILES | G.GM_F_SPT4)
    # the tuned variant gives the same map as the default one
    ref = G.gm_accumulate_fixations(hs[0][0], hs[0][1], *hs[0][2:], prm)
    p2 = pipe.params_of(ws[0], normalize=False, flags=fl2)
    tuned = G.gm_accumulate_fixations(hs[0][0], hs[0][1], *hs[0][2:], p2)
    a0 = np.empty(G.gm_samples_info(hs[0][1]), np.float32)
    a1 = np.empty_like(a0)
    G.gm_map_copy(ref, 0, a0)
    G.gm_map_copy(tuned, 0, a1)
    G.gm_map_free(ref)
    G.gm_map_free(tuned)
    assert np.array_equal(a0.view(np.uint32), a1.view(np.uint32))
    for sc, sm, *_ in hs:
        G.gm_samples_free(sm)
        G.gm_scene_free(sc)
