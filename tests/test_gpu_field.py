"""The neural density field on the GPU against the FP64 field oracle (which emulates the bf16
rounding the definition fixes): queries, the loss gradient, one Adam step, and a short training
run on the tiny sphere's map.

Element-wise bars: the definition fixes every bf16 rounding but neither the order of the FP32
additions of a layer (or of a batch sum) nor the evaluation of the features' sines and cosines;
where a value to be rounded lies near a bf16 boundary, two correct implementations round it
apart and the later layers carry the difference on. The oracle's enclosures (forward_bounds,
loss_and_grad_bounds: interval arithmetic through every rounding, FP32 sums as chains with one
unit of error per addition, features within 1e-5) bound every value such an implementation can
produce; each GPU value must lie inside its own. The median agreement checks beside them are
empirical (typical values agree far better than the worst case)."""
import numpy as np
import pytest

import synth
from oracle import field as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_07571_gb300 import build
    build.build()
    import paper_2601_07571_gb300 as G
    ctx = G.gm_create(0)
    yield G, torch, ctx
    G.gm_destroy(ctx)


BOX_LO, BOX_HI = np.array([-2.0, -1.0, -1.5], np.float32), np.array([2.0, 1.5, 1.0], np.float32)


def _points(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(BOX_LO, BOX_HI, size=(n, 3)).astype(np.float32)


def _xt(x):
    return F.normalise32(x, BOX_LO, BOX_HI)


def _inside(v, lo, hi, rel=2e-6, what=""):
    """v within [lo, hi], widened by the FP32 evaluation of the final softplus / sigmoid."""
    v = np.asarray(v, np.float64)
    slack = rel * np.maximum(np.abs(lo), np.abs(hi)) + 1e-12
    bad = (v < lo - slack) | (v > hi + slack)
    assert not bad.any(), f"{what}: {bad.sum()} of {v.size} outside their enclosures"


def _chain_tc(batch):
    """Longest FP32 addition chain of a batch sum in the tensor-core training kernel: the tiles of
    one block accumulate in tensor memory, then the blocks' sums are added in block order."""
    import torch
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    tiles = -(-batch // 128)
    nblk = min(n_sm, tiles)
    return -(-tiles // nblk) * 128 + nblk + 1


def _chain_mma(batch):
    """The warp-level kernel: 128 points a block, the blocks' sums added by atomics."""
    return 128 + -(-batch // 128) + 1


def test_field_query_matches_oracle(env):
    G, torch, ctx = env
    theta = synth.field_init(11)
    theta[64 * 64:64 * 64 + 64] = np.random.default_rng(1).normal(0, 0.2, 64)   # some non-zero biases
    f = G.gm_field_create(ctx, BOX_LO, BOX_HI, theta)
    x = _points(5000, 2)
    out = np.empty(len(x), np.float32)
    G.gm_field_query(f, x, len(x), out)
    feats = F.features(_xt(x))
    ref, _ = F.forward(theta.astype(np.float64), feats, emulate_bf16=True)
    lo, hi, _ = F.forward_bounds(theta.astype(np.float64), _xt(x))
    _inside(out, lo, hi, what="tcgen05 queries")
    err = np.abs(out - ref)
    assert np.median(err / np.maximum(np.abs(ref), 1e-6)) < 2e-3
    # the same through gm_query_density
    out2 = np.empty(len(x), np.float32)
    G.gm_query_density(None, f, G.GM_Q_FIELD, 0, None, x, len(x), out2)
    assert np.array_equal(out, out2)
    # the warp-level mma.sync kernel: same bar, and close to the tensor-memory kernel (the two
    # accumulate in different orders, so a bf16 rounding of an activation can differ)
    G.gm_field_query_kernel(f, G.GM_FIELD_QUERY_MMA_SYNC)
    out3 = np.empty(len(x), np.float32)
    G.gm_field_query(f, x, len(x), out3)
    _inside(out3, lo, hi, what="mma.sync queries")
    assert np.median(np.abs(out3 - out) / np.maximum(np.abs(ref), 1e-6)) < 1e-3
    G.gm_field_query_kernel(f, G.GM_FIELD_QUERY_TCGEN05)
    G.gm_sync(ctx)
    G.gm_field_free(f)


@pytest.mark.parametrize("n, offset", [(1, 0), (127, 0), (128, 0), (129, 0), (1000, 1), (70001, 0), (70001, 3)])
def test_field_query_tiles_tails_and_alignment(env, n, offset):
    """Ragged tails, single points, several tiles per block, and inputs that are not 16-byte aligned
    (plain loads instead of bulk copies) give the mma.sync kernel's values to within a bf16 step."""
    import torch
    G, torch, ctx = env
    theta = synth.field_init(12)
    f = G.gm_field_create(ctx, BOX_LO, BOX_HI, theta)
    x = _points(n, 3)
    buf = torch.zeros(3 * n + 3, dtype=torch.float32, device="cuda")
    dx = buf[offset:offset + 3 * n]
    dx.copy_(torch.from_numpy(x.reshape(-1)))
    out_tc = torch.empty(n, dtype=torch.float32, device="cuda")
    G.gm_field_query(f, dx, n, out_tc)
    G.gm_field_query_kernel(f, G.GM_FIELD_QUERY_MMA_SYNC)
    out_ms = torch.empty(n, dtype=torch.float32, device="cuda")
    G.gm_field_query(f, dx, n, out_ms)
    G.gm_sync(ctx)
    a, b = out_tc.cpu().numpy(), out_ms.cpu().numpy()
    lo, hi, _ = F.forward_bounds(theta.astype(np.float64), _xt(x))
    assert np.all(np.isfinite(a))
    _inside(a, lo, hi, what="tcgen05 queries")
    _inside(b, lo, hi, what="mma.sync queries")
    G.gm_field_free(f)


@pytest.mark.parametrize("kernel", ["TCGEN05", "MMA_SYNC"])
def test_field_gradient_and_adam_step_match_oracle(env, kernel):
    G, torch, ctx = env
    theta = synth.field_init(12)
    f = G.gm_field_create(ctx, BOX_LO, BOX_HI, theta)
    G.gm_field_train_kernel(f, getattr(G, "GM_FIELD_QUERY_" + kernel))
    n = 4000
    x = _points(n, 3)
    y = np.random.default_rng(4).uniform(0, 1, n).astype(np.float32)
    idx = np.random.default_rng(5).choice(n, 300, replace=False).astype(np.uint32)
    dx, dy, di = (torch.from_numpy(a).cuda() for a in (x, y, idx.view(np.int32)))
    g = np.empty(G.GM_FIELD_N_PARAMS, np.float32)
    loss = G.gm_field_loss_grad(f, dx, dy, n, di, len(idx), g)
    feats = F.features(_xt(x[idx]))
    l_ref, g_ref = F.loss_and_grad(theta.astype(np.float64), feats, y[idx].astype(np.float64), emulate_bf16=True)
    chain = _chain_tc(len(idx)) if kernel == "TCGEN05" else _chain_mma(len(idx))
    (llo, lhi), glo, ghi = F.loss_and_grad_bounds(theta.astype(np.float64), _xt(x[idx]), y[idx].astype(np.float64),
                                                  chain)
    _inside([loss], [llo], [lhi], rel=1e-5, what="loss")
    _inside(g, glo, ghi, rel=1e-5, what="gradient")
    assert F.relative_l2(g, g_ref) < 2e-2
    # one Adam step from zero moments: theta - lr g / (|g| + eps) (bias-corrected), increasing in g,
    # so the enclosure of g gives the enclosure of the step; plus the FP32 update's own rounding
    lr = 1e-3
    G.gm_field_step(f, dx, dy, n, di, len(idx), lr)
    after = np.empty(G.GM_FIELD_N_PARAMS, np.float32)
    G.gm_field_params(f, after)
    t64 = theta.astype(np.float64)
    step = lambda gg: gg / (np.abs(gg) + 1e-8)
    a_lo, a_hi = t64 - lr * step(ghi), t64 - lr * step(glo)
    rnd = 4 * 2.0 ** -24 * (np.abs(t64) + lr)
    assert np.all((after >= a_lo - rnd) & (after <= a_hi + rnd))
    th_ref, _, _ = F.adam_step(t64, 0.0, 0.0, g_ref, 1, lr)
    sure = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()
    assert sure.sum() > 1000
    assert np.allclose(after[sure], th_ref[sure], rtol=0, atol=1e-6)
    G.gm_field_free(f)


def test_field_tensor_core_gradient_over_many_tiles(env):
    """70 001 batch points: 547 full tiles and a ragged one, several tiles per block, so the weight
    and bias gradients accumulate in tensor memory across tiles. The gradient matches the oracle to
    the bf16 rounding, is bit-identical when repeated (fixed-order reduction of the blocks' sums),
    and agrees with the warp-level kernel's."""
    G, torch, ctx = env
    theta = synth.field_init(21)
    f = G.gm_field_create(ctx, BOX_LO, BOX_HI, theta)
    n, batch = 90_000, 70_001
    x = _points(n, 7)
    y = np.random.default_rng(8).uniform(0, 1, n).astype(np.float32)
    idx = np.random.default_rng(9).integers(0, n, batch).astype(np.uint32)
    dx, dy, di = (torch.from_numpy(a).cuda() for a in (x, y, idx.view(np.int32)))
    g1, g2, g3 = (np.empty(G.GM_FIELD_N_PARAMS, np.float32) for _ in range(3))
    l1 = G.gm_field_loss_grad(f, dx, dy, n, di, batch, g1)
    l2 = G.gm_field_loss_grad(f, dx, dy, n, di, batch, g2)
    G.gm_field_train_kernel(f, G.GM_FIELD_QUERY_MMA_SYNC)
    l3 = G.gm_field_loss_grad(f, dx, dy, n, di, batch, g3)
    G.gm_field_free(f)
    feats = F.features(_xt(x[idx]))
    l_ref, g_ref = F.loss_and_grad(theta.astype(np.float64), feats, y[idx].astype(np.float64), emulate_bf16=True)
    assert np.array_equal(g1, g2) and l1 == l2
    for g, l, chain, what in ((g1, l1, _chain_tc(batch), "tcgen05"), (g3, l3, _chain_mma(batch), "mma.sync")):
        (llo, lhi), glo, ghi = F.loss_and_grad_bounds(theta.astype(np.float64), _xt(x[idx]),
                                                      y[idx].astype(np.float64), chain)
        _inside([l], [llo], [lhi], rel=1e-5, what=what + " loss")
        _inside(g, glo, ghi, rel=1e-5, what=what + " gradient")
    assert abs(l1 - l_ref) <= 2e-3 * l_ref and abs(l3 - l_ref) <= 2e-3 * l_ref
    assert F.relative_l2(g1, g_ref) < 2e-2
    assert F.relative_l2(g1, g3) < 2e-2


@pytest.mark.parametrize("batch", [1, 127, 129])
def test_field_tensor_core_gradient_small_batches(env, batch):
    """One point, one ragged tile and one full tile plus a single point: the padding rows of a
    tile add nothing and the mean uses the true batch size."""
    G, torch, ctx = env
    theta = synth.field_init(17)
    f = G.gm_field_create(ctx, BOX_LO, BOX_HI, theta)
    n = 500
    x = _points(n, 11)
    y = np.random.default_rng(12).uniform(0, 1, n).astype(np.float32)
    idx = np.random.default_rng(13).integers(0, n, batch).astype(np.uint32)
    dx, dy, di = (torch.from_numpy(a).cuda() for a in (x, y, idx.view(np.int32)))
    g = np.empty(G.GM_FIELD_N_PARAMS, np.float32)
    loss = G.gm_field_loss_grad(f, dx, dy, n, di, batch, g)
    G.gm_field_free(f)
    feats = F.features(_xt(x[idx]))
    l_ref, g_ref = F.loss_and_grad(theta.astype(np.float64), feats, y[idx].astype(np.float64), emulate_bf16=True)
    (llo, lhi), glo, ghi = F.loss_and_grad_bounds(theta.astype(np.float64), _xt(x[idx]), y[idx].astype(np.float64),
                                                  _chain_tc(batch))
    _inside([loss], [llo], [lhi], rel=1e-5, what="loss")
    _inside(g, glo, ghi, rel=1e-5, what="gradient")
    assert abs(loss - l_ref) <= 2e-3 * l_ref
    assert F.relative_l2(g, g_ref) < 2e-2


def test_field_kernel_selectors_refuse_unknown_kernels(env):
    G, torch, ctx = env
    f = G.gm_field_create(ctx, BOX_LO, BOX_HI, synth.field_init(2))
    with pytest.raises(RuntimeError, match="unknown kernel"):
        G.gm_field_train_kernel(f, 7)
    with pytest.raises(RuntimeError, match="unknown kernel"):
        G.gm_field_query_kernel(f, -1)
    G.gm_field_train_kernel(f, G.GM_FIELD_QUERY_MMA_SYNC)
    G.gm_field_train_kernel(f, G.GM_FIELD_QUERY_TCGEN05)
    G.gm_field_free(f)


def test_field_trains_on_the_tiny_sphere_map(env):
    G, torch, ctx = env
    from paper_2601_07571_gb300 import pipeline
    w = synth.tiny_sphere()
    h = pipeline.run(ctx, w, normalize=True)
    xyz, tri, b2, obj = pipeline.samples_arrays(h)
    target, _ = pipeline.map_array(h)
    lo, hi = xyz.min(0), xyz.max(0)
    f = G.gm_field_create(ctx, lo, hi, synth.field_init(3))
    pred0 = np.empty(len(xyz), np.float32)
    G.gm_field_query(f, xyz, len(xyz), pred0)
    e0 = F.relative_l2(pred0, target)
    loss = G.gm_field_train(f, h.samples, h.map, 0, steps=1500, batch=4096, lr=3e-3, lr_min=1e-4, seed=9)
    pred = np.empty(len(xyz), np.float32)
    G.gm_field_query(f, xyz, len(xyz), pred)
    e1 = F.relative_l2(pred, target)
    info = G.gm_field_info(f)
    G.gm_field_free(f)
    h.free()
    assert info["steps"] == 1500 and np.isfinite(loss)
    assert e1 < 0.5 * e0 and e1 < 0.6, (e0, e1)


def test_field_checkpoint_resumes_training_exactly(env):
    """Parameters, both Adam moments and the step count saved after one training call and
    restored into a fresh field: the next call continues bit for bit as on the original."""
    G, torch, ctx = env
    from paper_2601_07571_gb300 import pipeline
    w = synth.tiny_sphere()
    h = pipeline.run(ctx, w, normalize=True)
    xyz, _, _, _ = pipeline.samples_arrays(h)
    lo, hi = xyz.min(0), xyz.max(0)
    n = G.GM_FIELD_N_PARAMS
    a = G.gm_field_create(ctx, lo, hi, synth.field_init(3))
    G.gm_field_train(a, h.samples, h.map, 0, steps=300, batch=4096, lr=3e-3, lr_min=1e-3, seed=9)
    th, m, v = (np.empty(n, np.float32) for _ in range(3))
    steps = G.gm_field_get_state(a, th, m, v)
    assert steps == 300 and np.abs(m).max() > 0 and v.min() >= 0 and v.max() > 0
    b = G.gm_field_create(ctx, lo, hi, synth.field_init(4))   # other initial parameters, zero moments
    G.gm_field_set_state(b, th, m, v, steps)
    for f in (a, b):
        G.gm_field_train(f, h.samples, h.map, 0, steps=200, batch=4096, lr=1e-3, lr_min=1e-4, seed=9)
    ta, ma, va = (np.empty(n, np.float32) for _ in range(3))
    tb, mb, vb = (np.empty(n, np.float32) for _ in range(3))
    sa = G.gm_field_get_state(a, ta, ma, va)
    sb = G.gm_field_get_state(b, tb, mb, vb)
    qa, qb = np.empty(len(xyz), np.float32), np.empty(len(xyz), np.float32)
    G.gm_field_query(a, xyz, len(xyz), qa)
    G.gm_field_query(b, xyz, len(xyz), qb)
    G.gm_field_free(a)
    G.gm_field_free(b)
    h.free()
    assert sa == sb == 500
    for x, y in ((ta, tb), (ma, mb), (va, vb), (qa, qb)):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    # device buffers work too, and set_state refuses missing parts
    dth = torch.from_numpy(th).cuda()
    c = G.gm_field_create(ctx, lo, hi, synth.field_init(3))
    G.gm_field_set_state(c, dth, torch.from_numpy(m).cuda(), torch.from_numpy(v).cuda(), 300)
    back = np.empty(n, np.float32)
    assert G.gm_field_get_state(c, back) == 300 and np.array_equal(back, th)
    with pytest.raises(G.GazeMapError):
        G.gm_field_set_state(c, th, None, v, 1)
    G.gm_field_free(c)


def test_bounded_wait_runs_out_and_the_context_stays_usable(env):
    """A wait on an mbarrier that nothing completes gives up after its poll budget; gm_sync
    reports GM_ERR_TIMEOUT once, and the context keeps working."""
    G, torch, ctx = env
    G.gm_debug_wait_timeout(ctx, 2000)
    with pytest.raises(G.GazeMapError) as ei:
        G.gm_sync(ctx)
    assert ei.value.status == G.GM_ERR_TIMEOUT
    G.gm_sync(ctx)   # cleared
    f = G.gm_field_create(ctx, BOX_LO, BOX_HI, synth.field_init(11))
    x = _points(1000, 5)
    out = np.empty(len(x), np.float32)
    G.gm_field_query(f, x, len(x), out)
    G.gm_sync(ctx)
    G.gm_field_free(f)
    lo, hi, _ = F.forward_bounds(synth.field_init(11).astype(np.float64), _xt(x))
    assert np.all(np.isfinite(out))
    _inside(out, lo, hi, what="queries after the timeout")
    with pytest.raises(G.GazeMapError):
        G.gm_debug_wait_timeout(ctx, 0)
