"""FP64 oracle of the neural density field -- TEST INFRASTRUCTURE.

The field is not in the paper: it is a learned, resolution-free stand-in for the per-sample map
of Section 3.2, trained on maps the plain method produces. Its definition (fixed here, mirrored
by the CUDA kernels, checked against this module):

  x~ = (x - c) * (1/h), with c the centre and h half the largest side of the scene box
      (|x~| <= 1), evaluated in FP32 as the kernels do: c = 0.5 (lo + hi), 1/h = 2 / side,
      each operation rounded to FP32 (normalise32; `normalise` is the exact value);
  features f (64): f[a] = x~_a (a = 0..2); for octave k = 0..9:
      f[3 + 6k + a] = sin(2^k pi x~_a), f[6 + 6k + a] = cos(2^k pi x~_a); f[63] = 0
  h0 = bf16(f); for l = 1..4: z_l = h_{l-1} bf16(W_l)^T + b_l, h_l = bf16(relu(z_l))
  (64 x 64 weights, FP32 biases, FP32 accumulation); z5 = h4 . w5 + b5 (FP32); out = softplus(z5).
  Loss: mean squared error over the batch. Backward as the chain rule dictates, with the
  operands that enter tensor-core products rounded to bf16 (dz_l and the activations h).
  Adam (Kingma & Ba 2015) with bias correction on FP32 master parameters.

The parameter vector packs, in order: W1 (64x64, row = output), b1, W2, b2, W3, b3, W4, b4,
w5 (64), b5 (1): 16 705 FP32 values.

Only the tests and the benchmark's baseline leg use this module.
"""
from __future__ import annotations

import math

import numpy as np

WIDTH = 64
DEPTH = 4
OCTAVES = 10
N_FEAT = 3 + 6 * OCTAVES          # 63, padded to 64
N_PARAMS = DEPTH * (WIDTH * WIDTH + WIDTH) + WIDTH + 1


def bf16(x):
    """Round FP32 values to bfloat16 (round to nearest, ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    nan = np.isnan(a)
    if nan.any():
        out[nan] = np.nan
    return out


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    Ws, bs, o = [], [], 0
    for _ in range(DEPTH):
        Ws.append(theta[o:o + WIDTH * WIDTH].reshape(WIDTH, WIDTH))
        o += WIDTH * WIDTH
        bs.append(theta[o:o + WIDTH])
        o += WIDTH
    w5 = theta[o:o + WIDTH]
    b5 = theta[o + WIDTH]
    return Ws, bs, w5, b5


def pack(Ws, bs, w5, b5):
    parts = []
    for W, b in zip(Ws, bs):
        parts += [np.asarray(W, np.float64).reshape(-1), np.asarray(b, np.float64)]
    parts += [np.asarray(w5, np.float64), np.atleast_1d(np.float64(b5))]
    return np.concatenate(parts)


def normalise(x, box_lo, box_hi):
    lo, hi = np.asarray(box_lo, np.float64), np.asarray(box_hi, np.float64)
    c = 0.5 * (lo + hi)
    h = 0.5 * float(np.max(hi - lo))
    return (np.asarray(x, np.float64) - c) / h


def normalise32(x, box_lo, box_hi):
    """x~ as the definition fixes it for the kernels, in FP32 arithmetic: c = 0.5 (lo + hi),
    1/h = 2 / (largest side of the box), x~ = (x - c) * (1/h), each operation rounded to FP32
    (numpy's float32 operations are IEEE round-to-nearest). Returned as float64 values."""
    lo, hi = np.asarray(box_lo, np.float32), np.asarray(box_hi, np.float32)
    c = np.float32(0.5) * (lo + hi)
    inv_h = np.float32(2.0) / np.max(hi - lo)
    x = np.asarray(x, np.float32)
    return ((x - c) * inv_h).astype(np.float32).astype(np.float64)


def features(xt):
    """Fourier features of normalised positions (n, 3) -> (n, 64)."""
    xt = np.asarray(xt, np.float64)
    n = len(xt)
    f = np.zeros((n, 64))
    f[:, 0:3] = xt
    for k in range(OCTAVES):
        f[:, 3 + 6 * k:6 + 6 * k] = np.sin((2.0 ** k) * math.pi * xt)
        f[:, 6 + 6 * k:9 + 6 * k] = np.cos((2.0 ** k) * math.pi * xt)
    return f


def softplus(z):
    z = np.asarray(z, np.float64)
    return np.where(z > 30.0, z, np.log1p(np.exp(np.minimum(z, 30.0))))


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-np.asarray(z, np.float64)))


def forward(theta, feats, emulate_bf16=True):
    """Returns (out, cache). emulate_bf16=False gives the exact FP64 function (for gradient
    checks); True rounds the tensor-core operands as the definition says."""
    Ws, bs, w5, b5 = unpack(theta)
    q = bf16 if emulate_bf16 else (lambda v: np.asarray(v, np.float64))
    h = q(feats)
    hs, zs = [h], []
    for W, b in zip(Ws, bs):
        z = h @ q(W).T + b
        zs.append(z)
        h = q(np.maximum(z, 0.0))
        hs.append(h)
    z5 = h @ w5 + b5
    return softplus(z5), dict(hs=hs, zs=zs, z5=z5)


def loss_and_grad(theta, feats, target, emulate_bf16=True):
    """Mean squared error and its gradient with respect to the packed parameters."""
    Ws, bs, w5, b5 = unpack(theta)
    q = bf16 if emulate_bf16 else (lambda v: np.asarray(v, np.float64))
    out, c = forward(theta, feats, emulate_bf16)
    B = len(feats)
    r = out - np.asarray(target, np.float64)
    loss = float(np.mean(r * r))
    dz5 = 2.0 * r / B * sigmoid(c["z5"])
    h4 = c["hs"][DEPTH]
    gw5 = h4.T @ dz5
    gb5 = dz5.sum()
    dh = np.outer(dz5, w5)
    gWs, gbs = [None] * DEPTH, [None] * DEPTH
    for l in range(DEPTH - 1, -1, -1):
        dz = q(dh * (c["zs"][l] > 0.0))
        gWs[l] = dz.T @ c["hs"][l]
        gbs[l] = dz.sum(axis=0)
        if l > 0:
            dh = dz @ q(Ws[l])
    return loss, pack(gWs, gbs, gw5, gb5)


def adam_step(theta, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step t >= 1), FP64. Returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def cosine_lr(step, steps, lr0, lr_min):
    """Cosine decay from lr0 at step 0 to lr_min at the last step."""
    if steps <= 1:
        return lr0
    return lr_min + 0.5 * (lr0 - lr_min) * (1.0 + math.cos(math.pi * step / (steps - 1)))


def relative_l2(pred, ref):
    pred, ref = np.asarray(pred, np.float64), np.asarray(ref, np.float64)
    return float(np.linalg.norm(pred - ref) / max(np.linalg.norm(ref), 1e-300))


# ---------------------------------------------------------------------------------------------
# Enclosures of what any implementation of the definition may compute
# ---------------------------------------------------------------------------------------------
# The definition fixes every bf16 rounding but not (a) how the sines and cosines of the features
# are evaluated nor (b) the order in which a layer's FP32 products are added. Two implementations
# can therefore differ when a value that is rounded to bf16 lies near a rounding boundary: one
# rounding step apart, which the later layers carry on. The functions below propagate intervals
# (midpoint and radius, in FP64) through the network so that the result encloses the output (and
# the loss gradient) of every implementation whose features are within feat_eps of the exact
# values and whose sums carry at most acc_u relative error per addition in a chain of n
# additions (the classical bound |error| <= n acc_u sum |terms| of recursive summation).

FEAT_EPS = 1e-5     # hardware sine/cosine (<= 2^-21.4 on [-pi, pi]) and two double-angle steps
ACC_U = 2.0 ** -23  # one FP32 unit in the last place per addition (covers truncating adders)


def _mr_mul_sum(am, ar, bm, br):
    """Midpoint and radius of sum_j a_j b_j (matrix product over the last axis of a and the first
    of b) for a in am +- ar, b in bm +- br."""
    c = am @ bm
    r = np.abs(am) @ br + ar @ np.abs(bm) + ar @ br
    return c, r


def forward_bounds(theta, xt, feat_eps=FEAT_EPS, acc_u=ACC_U):
    """[lo, hi] of the softplus output at normalised positions xt (n, 3; the FP32 values of
    normalise32), and the per-layer intervals for loss_and_grad_bounds."""
    Ws, bs, w5, b5 = unpack(theta)
    f = features(xt)
    eps = np.full(64, float(feat_eps))
    eps[:3] = 0.0     # the coordinates themselves are exact
    eps[63] = 0.0     # padding
    h_lo, h_hi = bf16(f - eps), bf16(f + eps)
    hs, zs = [(h_lo, h_hi)], []
    for W, b in zip(Ws, bs):
        Wq = bf16(W)
        hm, hr = 0.5 * (h_lo + h_hi), 0.5 * (h_hi - h_lo)
        zc, zr = _mr_mul_sum(hm, hr, Wq.T, np.zeros_like(Wq.T))
        zc = zc + b
        # 64 products (exact in FP32: bf16 x bf16) and the bias, added in some order
        mag = np.maximum(np.abs(h_lo), np.abs(h_hi)) @ np.abs(Wq).T + np.abs(b)
        zr = zr + (WIDTH + 1) * acc_u * mag
        z_lo, z_hi = zc - zr, zc + zr
        zs.append((z_lo, z_hi))
        h_lo, h_hi = bf16(np.maximum(z_lo, 0.0)), bf16(np.maximum(z_hi, 0.0))
        hs.append((h_lo, h_hi))
    hm, hr = 0.5 * (h_lo + h_hi), 0.5 * (h_hi - h_lo)
    z5c = hm @ w5 + b5
    # w5 enters as three exact bf16 parts (or FP32 products): at most 3 x 64 products and the bias
    z5r = hr @ np.abs(w5) + (3 * WIDTH + 1) * acc_u * (np.maximum(np.abs(h_lo), np.abs(h_hi)) @ np.abs(w5) + abs(b5))
    z5_lo, z5_hi = z5c - z5r, z5c + z5r
    return softplus(z5_lo), softplus(z5_hi), dict(hs=hs, zs=zs, z5=(z5_lo, z5_hi))


def _bf16_iv(lo, hi):
    return bf16(lo), bf16(hi)


def loss_and_grad_bounds(theta, xt, target, chain, feat_eps=FEAT_EPS, acc_u=ACC_U):
    """Enclosures of the batch loss (mean squared error) and of its gradient with respect to the
    packed parameters, for implementations as in forward_bounds whose batch sums (over the B
    points of the batch) are chains of at most `chain` additions. Returns
    ((loss_lo, loss_hi), g_lo, g_hi)."""
    Ws, bs, w5, b5 = unpack(theta)
    o_lo, o_hi, c = forward_bounds(theta, xt, feat_eps, acc_u)
    y = np.asarray(target, np.float64)
    B = len(y)
    r_lo, r_hi = o_lo - y, o_hi - y
    # loss = sum r^2 / B
    r2_lo = np.where((r_lo <= 0) & (r_hi >= 0), 0.0, np.minimum(r_lo * r_lo, r_hi * r_hi))
    r2_hi = np.maximum(r_lo * r_lo, r_hi * r_hi)
    lerr = chain * acc_u * r2_hi.sum() / B
    loss = (r2_lo.sum() / B - lerr, r2_hi.sum() / B + lerr)
    # dz5 = 2 r sigmoid(z5) / B, sigmoid > 0; a few FP32 roundings (4 units, relative)
    s_lo, s_hi = sigmoid(c["z5"][0]), sigmoid(c["z5"][1])
    cand = np.stack([r_lo * s_lo, r_lo * s_hi, r_hi * s_lo, r_hi * s_hi])
    d_lo, d_hi = 2.0 * cand.min(0) / B, 2.0 * cand.max(0) / B
    d_lo, d_hi = d_lo - 4 * acc_u * np.abs(d_lo), d_hi + 4 * acc_u * np.abs(d_hi)
    dm, dr = 0.5 * (d_lo + d_hi), 0.5 * (d_hi - d_lo)

    def batch_sum(am, ar, bm, br):
        # sum over the batch of the products a_b b_b^T (a: (B,), or (B, m); b: (B, k))
        cc, rr = _mr_mul_sum(am.T, ar.T, bm, br)
        mag = (np.abs(am) + ar).T @ (np.abs(bm) + br)
        return cc - rr - chain * acc_u * mag, cc + rr + chain * acc_u * mag

    h4_lo, h4_hi = c["hs"][DEPTH]
    h4m, h4r = 0.5 * (h4_lo + h4_hi), 0.5 * (h4_hi - h4_lo)
    gw5 = batch_sum(dm[:, None], dr[:, None], h4m, h4r)
    gw5 = (gw5[0][0], gw5[1][0])
    gb5 = batch_sum(dm[:, None], dr[:, None], np.ones((B, 1)), np.zeros((B, 1)))
    gb5 = (gb5[0][0, 0], gb5[1][0, 0])
    # dh4 = dz5 w5 (one FP32 product per element)
    dh_m = dm[:, None] * w5[None, :]
    dh_r = dr[:, None] * np.abs(w5)[None, :]
    dh_r = dh_r + acc_u * (np.abs(dh_m) + dh_r)
    gW, gb = [None] * DEPTH, [None] * DEPTH
    for l in range(DEPTH - 1, -1, -1):
        z_lo, z_hi = c["zs"][l]
        a_lo, a_hi = dh_m - dh_r, dh_m + dh_r
        # dz = bf16(dh * [z > 0]); where the sign of z is uncertain both 0 and dh are possible
        on = z_lo > 0.0
        off = z_hi <= 0.0
        lo = np.where(on, a_lo, np.where(off, 0.0, np.minimum(a_lo, 0.0)))
        hi = np.where(on, a_hi, np.where(off, 0.0, np.maximum(a_hi, 0.0)))
        dz_lo, dz_hi = _bf16_iv(lo, hi)
        zm, zr = 0.5 * (dz_lo + dz_hi), 0.5 * (dz_hi - dz_lo)
        hl, hh = c["hs"][l]
        gW[l] = batch_sum(zm, zr, 0.5 * (hl + hh), 0.5 * (hh - hl))
        gbl = batch_sum(zm, zr, np.ones((B, 1)), np.zeros((B, 1)))
        gb[l] = (gbl[0][:, 0], gbl[1][:, 0])
        if l > 0:
            Wq = bf16(Ws[l])
            cc, rr = _mr_mul_sum(zm, zr, Wq, np.zeros_like(Wq))
            rr = rr + (WIDTH + 1) * acc_u * ((np.abs(zm) + zr) @ np.abs(Wq))
            dh_m, dh_r = cc, rr
    g_lo = pack([g[0] for g in gW], [g[0] for g in gb], gw5[0], gb5[0])
    g_hi = pack([g[1] for g in gW], [g[1] for g in gb], gw5[1], gb5[1])
    return loss, g_lo, g_hi
