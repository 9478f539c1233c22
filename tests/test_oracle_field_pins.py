"""Pins for the FP64 field oracle: closed forms, an independent bf16 conversion, finite
differences for the backward pass and a library Adam for the update rule."""
import math

import numpy as np
import pytest

from oracle import field as F
import synth


def test_features_closed_forms():
    f = F.features(np.array([[0.0, 0.5, -0.25]]))[0]
    assert f.shape == (64,) and f[63] == 0.0
    assert np.allclose(f[:3], [0.0, 0.5, -0.25])
    for k in range(F.OCTAVES):
        s, c = f[3 + 6 * k:6 + 6 * k], f[6 + 6 * k:9 + 6 * k]
        assert abs(s[0]) < 1e-15 and abs(c[0] - 1) < 1e-15          # x = 0
        assert np.allclose(s ** 2 + c ** 2, 1.0, atol=1e-14)
    assert abs(f[3 + 1] - 1.0) < 1e-15                                # sin(pi / 2)
    assert abs(f[3 + 6 + 1] - 0.0) < 1e-15 and abs(f[6 + 6 + 1] + 1.0) < 1e-15   # sin, cos of pi
    assert abs(f[3 + 2] + math.sin(math.pi / 4)) < 1e-15             # sin(-pi / 4)


def test_normalise_maps_the_box_into_unit_cube():
    lo, hi = np.array([-1.0, 0.0, 2.0]), np.array([3.0, 1.0, 2.5])
    x = np.array([lo, hi, 0.5 * (lo + hi)])
    t = F.normalise(x, lo, hi)
    assert np.allclose(t[2], 0.0) and np.abs(t).max() <= 1.0 + 1e-15 and abs(t[1, 0] - 1.0) < 1e-15


def test_bf16_rounding_against_torch():
    torch = pytest.importorskip("torch")
    assert F.bf16(np.float32(1.0 + 2 ** -8)) == 1.0                    # tie to even
    assert F.bf16(np.float32(1.0 + 3 * 2 ** -8)) == 1.0 + 2 ** -6      # tie to even (up)
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(F.bf16(x), ref)


def test_softplus_and_sigmoid():
    assert abs(F.softplus(0.0) - math.log(2.0)) < 1e-15
    assert F.softplus(50.0) == 50.0
    assert abs(F.softplus(-40.0) - math.exp(-40.0)) < 1e-25
    assert abs(F.sigmoid(0.0) - 0.5) < 1e-15


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = synth.field_init(7).astype(np.float64)
    theta[F.DEPTH * (64 * 64 + 64) - 64:F.DEPTH * (64 * 64 + 64)] = rng.normal(0, 0.1, 64)   # b4
    x = rng.uniform(-1, 1, size=(24, 3))
    feats = F.features(x)
    y = rng.uniform(0, 1, size=24)
    loss, g = F.loss_and_grad(theta, feats, y, emulate_bf16=False)
    idx = np.concatenate([rng.choice(len(theta), 300, replace=False), [len(theta) - 1, len(theta) - 2]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp = F.loss_and_grad(tp, feats, y, emulate_bf16=False)[0]
        lm = F.loss_and_grad(tm, feats, y, emulate_bf16=False)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, i


def test_adam_matches_closed_form_and_torch():
    th, m, v = F.adam_step(np.array([1.0]), np.zeros(1), np.zeros(1), np.array([2.5]), t=1, lr=0.01)
    assert abs(th[0] - (1.0 - 0.01 * 2.5 / (2.5 + 1e-8))) < 1e-15
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    p0 = rng.normal(size=50)
    grads = rng.normal(size=(4, 50))
    p = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    th, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t, gr in enumerate(grads, start=1):
        opt.zero_grad()
        p.grad = torch.tensor(gr)
        opt.step()
        th, m, v = F.adam_step(th, m, v, gr, t, 3e-3)
    assert np.allclose(th, p.detach().numpy(), rtol=0, atol=1e-12)


def test_cosine_schedule_endpoints():
    assert F.cosine_lr(0, 100, 1e-3, 1e-5) == 1e-3
    assert abs(F.cosine_lr(99, 100, 1e-3, 1e-5) - 1e-5) < 1e-18
    assert abs(F.cosine_lr(49.5, 100, 1e-3, 1e-5) - 0.5 * (1e-3 + 1e-5)) < 1e-15


def test_bf16_emulated_forward_stays_close_to_exact():
    rng = np.random.default_rng(3)
    theta = synth.field_init(3).astype(np.float64)
    feats = F.features(rng.uniform(-1, 1, size=(2000, 3)))
    a, _ = F.forward(theta, feats, emulate_bf16=True)
    b, _ = F.forward(theta, feats, emulate_bf16=False)
    assert F.relative_l2(a, b) < 2e-2


# ---- enclosures of admissible implementations (element-wise bars of the GPU field tests) ----
def _emulate_fp32(theta, xt, rng, feat_eps):
    """One admissible implementation: features perturbed within feat_eps (FP32), every layer's
    products (exact in FP32) added to the bias in a random order in FP32, the output layer's FP32
    products added in a random order, softplus in FP32."""
    Ws, bs, w5, b5 = F.unpack(theta)
    f = F.features(xt)
    noise = rng.uniform(-feat_eps, feat_eps, f.shape)
    noise[:, :3] = 0.0
    noise[:, 63] = 0.0
    h = F.bf16((f + noise).astype(np.float32))
    for W, b in zip(Ws, bs):
        Wq = F.bf16(W)
        prod = (h[:, None, :] * Wq[None, :, :]).astype(np.float32)        # exact: bf16 x bf16
        acc = np.broadcast_to(np.float32(b), (len(h), F.WIDTH)).astype(np.float32).copy()
        for j in rng.permutation(F.WIDTH):
            acc = (acc + prod[:, :, j]).astype(np.float32)
        h = F.bf16(np.maximum(acc, np.float32(0)))
    p5 = (h.astype(np.float32) * np.float32(w5)).astype(np.float32)
    acc = np.full(len(h), np.float32(b5), np.float32)
    for j in rng.permutation(F.WIDTH):
        acc = (acc + p5[:, j]).astype(np.float32)
    z = acc.astype(np.float32)
    return np.where(z > 30, z, np.log1p(np.exp(np.minimum(z, 30)).astype(np.float32))).astype(np.float64)


def test_forward_bounds_enclose_admissible_implementations():
    theta = synth.field_init(12).astype(np.float64)
    lo_box, hi_box = np.array([-2.0, -1.0, -1.5], np.float32), np.array([2.0, 1.5, 1.0], np.float32)
    x = np.random.default_rng(2).uniform(lo_box, hi_box, size=(600, 3)).astype(np.float32)
    xt = F.normalise32(x, lo_box, hi_box)
    lo, hi, _ = F.forward_bounds(theta, xt)
    exact, _ = F.forward(theta, F.features(xt))
    assert np.all((lo <= exact) & (exact <= hi))
    rng = np.random.default_rng(7)
    for _ in range(4):
        e = _emulate_fp32(theta, xt, rng, F.FEAT_EPS)
        slack = 2e-6 * np.abs(e) + 1e-12          # the FP32 softplus itself
        assert np.all((e >= lo - slack) & (e <= hi + slack))
    # each term is needed: with exact features, FP32 sums in random orders leave the bounds that
    # omit the accumulation term, and stay inside the ones that keep it
    lo_a, hi_a, _ = F.forward_bounds(theta, xt, feat_eps=0.0)
    lo_0, hi_0, _ = F.forward_bounds(theta, xt, feat_eps=0.0, acc_u=0.0)
    outside = 0
    for _ in range(4):
        e = _emulate_fp32(theta, xt, rng, 0.0)
        slack = 2e-6 * np.abs(e) + 1e-12
        assert np.all((e >= lo_a - slack) & (e <= hi_a + slack))
        outside += int(((e < lo_0 - slack) | (e > hi_0 + slack)).sum())
    assert outside > 0
    # and feature errors alone move outputs beyond the bounds that omit them
    lo_f, hi_f, _ = F.forward_bounds(theta, xt, feat_eps=0.0, acc_u=0.0)
    e_f = [F.forward(theta, np.where(np.arange(64) < 3, F.features(xt), F.features(xt) + d))[0]
           for d in (3e-5, -3e-5)]
    assert any(((v < lo_f - 1e-12) | (v > hi_f + 1e-12)).any() for v in e_f)


def test_normalise32_is_the_fp32_definition():
    lo_box, hi_box = np.array([-2.0, -1.0, -1.5], np.float32), np.array([2.0, 1.5, 1.0], np.float32)
    x = np.random.default_rng(3).uniform(lo_box, hi_box, size=(1000, 3)).astype(np.float32)
    a = F.normalise32(x, lo_box, hi_box)
    b = F.normalise(x, lo_box, hi_box)
    # the FP32 evaluation is within a few FP32 roundings of the exact value, and inside [-1, 1]
    assert np.abs(a - b).max() <= 4 * 2.0 ** -24 * 2 and np.abs(a).max() <= 1.0 + 1e-6
    assert np.array_equal(a, a.astype(np.float32).astype(np.float64))


def test_grad_bounds_enclose_the_exact_sums():
    theta = synth.field_init(12).astype(np.float64)
    lo_box, hi_box = np.array([-2.0, -1.0, -1.5], np.float32), np.array([2.0, 1.5, 1.0], np.float32)
    x = np.random.default_rng(2).uniform(lo_box, hi_box, size=(256, 3)).astype(np.float32)
    xt = F.normalise32(x, lo_box, hi_box)
    y = np.random.default_rng(4).uniform(0, 1, 256)
    l, g = F.loss_and_grad(theta, F.features(xt), y)
    (llo, lhi), glo, ghi = F.loss_and_grad_bounds(theta, xt, y, chain=256 + 2)
    assert llo <= l <= lhi
    assert np.all((glo <= g) & (g <= ghi))
    # and they are not vacuous: most weight gradients are pinned to within their own size
    w = (ghi - glo) / np.maximum(np.abs(g), 1e-30)
    assert np.median(w) < 10
