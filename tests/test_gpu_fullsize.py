"""Parity at the full sizes of the batched and the city workloads, in the launch forms the
benchmark times, against the FP64 oracle on sampled samples (one by one, brute force over every
triangle).

Identical inputs: the oracle's sample positions rounded to FP32 go to both sides
(gm_samples_from_points), so the strict bar 1e-4 (oracle + amb) + amb holds with no position
term; amb is the oracle's weight of the pairs whose cone or visibility decision lies within its
bookkeeping margins (grazing margin: 16 ulp of the scene's coordinates)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

REL = 1e-4


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


def _pick(s_all, fx, rng, n_uniform, n_fix, per_fix, pool=None, front=0.0):
    """Uniform samples plus, for a few fixations, the samples nearest to the gaze ray or (front
    > 0: within that angle of the ray) the ones nearest to the eye -- the surface the gaze meets,
    seen from the eye. Chosen from the oracle's positions alone."""
    n = len(s_all.tri)
    pick = set(rng.choice(n, min(n, n_uniform), replace=False).tolist())
    cand = np.arange(n) if pool is None or pool >= n else np.sort(rng.choice(n, pool, replace=False))
    xyz = s_all.xyz[cand]
    for f in rng.choice(fx.n, min(fx.n, n_fix), replace=False):
        p = xyz - fx.eye[f].astype(np.float64)
        r = fx.gaze[f].astype(np.float64) / np.linalg.norm(fx.gaze[f])
        d1 = p @ r
        ang = np.linalg.norm(np.cross(p, r), axis=1) / np.maximum(d1, 1e-9)
        ang[d1 <= 0] = np.inf
        if front > 0:
            near = np.nonzero(ang <= front)[0]
            if len(near):
                pick.update(cand[near[np.argsort(d1[near])[:per_fix]]].tolist())
                continue
        pick.update(cand[np.argsort(ang)[:per_fix]].tolist())
    return np.array(sorted(pick), np.int64)


def _check(gpu, d, amb, what):
    tol = REL * (d + amb) + amb + 1e-30
    err = np.abs(gpu.astype(np.float64) - d)
    bad = err > tol
    assert not bad.any(), f"{what}: {bad.sum()} samples off, worst rel {(err / np.maximum(d, 1e-30))[bad].max():.3e}"


def test_64_sessions_full_size_batched_against_oracle(env):
    """All 64 sessions of the batched workload (5k-300k triangles, 500-20k fixations,
    1e3-5e4 samples per m^2) in one graph-captured batched launch; every session checked on
    eight of its samples over all its fixations."""
    G, pipe, ctx = env
    ws = synth.batched_sessions(64)
    hs, ref = [], []
    for i, w in enumerate(ws):
        tri = oracle.world_triangles(w)
        off = oracle.tri_offsets(oracle.areas(tri), oracle.tri_density(w))
        s_all = oracle.samples(tri, off, w.seed, w.session)
        pts = s_all.xyz.astype(np.float32)
        which = _pick(s_all, w.fixations, np.random.default_rng(300 + i), 4, 2, 2)
        # 16 ulp of the largest coordinate of the session's scene
        delta = 16 * float(np.spacing(np.float32(np.abs(tri).max() + np.abs(w.fixations.eye).max())))
        ora = oracle.accumulate(tri, pts[which].astype(np.float64), s_all.tri[which], w.fixations, w.params,
                                delta_abs=delta, cone_band=1e-4)
        sc = G.gm_build_scene(ctx, pipe.mesh_args(w))
        sm = G.gm_samples_from_points(sc, pts, s_all.tri.astype(np.uint32))
        hs.append((sc, sm, *pipe.fixation_args(w.fixations)))
        ref.append((which, ora))
    prm = pipe.params_of(ws[0], normalize=False)
    b = G.gm_batch_create(ctx, hs, prm)
    G.gm_batch_run(b)
    nonzero = 0
    for i, (which, ora) in enumerate(ref):
        out = np.empty(len(which), np.float32)
        G.gm_query_density(G.gm_batch_map(b, i), None, G.GM_Q_SAMPLE, 0, which.astype(np.uint32), None, len(which),
                           out)
        d = ora["density"][0]
        nonzero += int((d > 0).sum())
        _check(out, d, ora["amb"][0], f"session {i}")
    G.gm_batch_free(b)
    for sc, sm, *_ in hs:
        G.gm_samples_free(sm)
        G.gm_scene_free(sc)
    print(f"PARITY 64 sessions: {sum(len(r[0]) for r in ref)} samples, {nonzero} non-zero")
    assert nonzero >= 150


def test_city_block_full_size_all_windows_against_oracle(env):
    """The full city block (5M triangles, 20M samples, 100k fixations, 600 one-second windows,
    48 GB of maps) in one call; 46 samples checked in every window."""
    G, pipe, ctx = env
    w = synth.city_block()
    tri = oracle.world_triangles(w)
    off = oracle.tri_offsets(oracle.areas(tri), oracle.tri_density(w))
    s_all = oracle.samples(tri, off, w.seed, w.session)
    fx = w.fixations
    which = _pick(s_all, fx, np.random.default_rng(44), 6, 40, 1, pool=2_000_000, front=np.tan(w.params.theta_rad))
    pts = s_all.xyz.astype(np.float32)
    delta = 16 * float(np.spacing(np.float32(np.abs(tri).max())))
    ora = oracle.accumulate(tri, pts[which].astype(np.float64), s_all.tri[which], fx, w.params, delta_abs=delta,
                            cone_band=1e-4)
    W = ora["density"].shape[0]
    h = pipe.run(ctx, w, normalize=False, points=(pts, s_all.tri.astype(np.uint32)))
    W2, ns, stats, _ = G.gm_map_info(h.map)
    assert W2 == W == 600 and ns == int(off[-1])
    out = np.empty(len(which), np.float32)
    nonzero = 0
    for k in range(W):
        G.gm_query_density(h.map, None, G.GM_Q_SAMPLE, k, which.astype(np.uint32), None, len(which), out)
        d = ora["density"][k]
        nonzero += int((d > 0).sum())
        _check(out, d, ora["amb"][k], f"window {k}")
    h.free()
    st = ora["stats"]
    print(f"PARITY city: {len(which)} samples x {W} windows, {nonzero} non-zero values, in-cone pairs "
          f"{st['in_cone']}, ambiguous {st['ambiguous']}")
    assert nonzero >= 20
