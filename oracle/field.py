"""FP64 oracle of the neural density field -- TEST INFRASTRUCTURE.

The field is not in the paper: it is a learned, resolution-free stand-in for the per-sample map
of Section 3.2, trained on maps the plain method produces. Its definition (fixed here, mirrored
by the CUDA kernels, checked against this module):

  x~ = (x - c) / h, with c the centre and h half the largest side of the scene box (|x~| <= 1);
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
