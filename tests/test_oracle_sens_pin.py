"""Pin of the oracle's position-sensitivity term `sens` against finite differences.

`sens[s]` is the oracle's first-order bound of how far a sample's density moves when the sample
moves by one metre: the sum, over its visible in-cone pairs, of g * (|d ln g / d d2| +
|d ln g / d d1|) with ln g = -(d2 / d1)^2 / (2 tan^2 theta) (the Gaussian of Section 3.2.1,
d1 the distance along the gaze, d2 the distance from the gaze axis). The GPU parity tests widen
their end-to-end density bar by `sens` times the FP32 position error, so a `sens` that is too
large would hide real disagreements. Two properties pin it, both exact consequences of the
definition and checked here with central differences of the oracle's own densities:

  * upper bound: along any direction u, |D(s + h u) - D(s - h u)| / 2h <= sens (the triangle
    inequality over pairs and over the two partial derivatives);
  * tightness for one pair: the gradient of d1 is the gaze direction and the gradient of d2 is
    perpendicular to it, so |grad g| = g sqrt(a^2 + b^2) >= g (a + b) / sqrt(2) = sens / sqrt(2).

A dropped factor (1 + d2/d1), a wrong power of d1 or of tan(theta), or a missing pair breaks one
of the two bounds at these geometries (d1 between 1 and 5 m, d2/d1 up to 4 tan 1 deg).
"""
import math

import numpy as np
import pytest

import oracle
import synth

H = 1e-6          # finite-difference step (metres): far inside the ambiguity margins below
DELTA = 2e-5      # grazing margin of the oracle's visibility bookkeeping (metres)
BAND = 1e-4       # relative band around the cone cut-off of the bookkeeping


@pytest.fixture(scope="module")
def scene():
    oracle.build()
    w = synth.tiny_sphere()
    tri = oracle.world_triangles(w)
    off = oracle.tri_offsets(oracle.areas(tri), oracle.tri_density(w))
    s = oracle.samples(tri, off, w.seed, w.session)
    return w, tri, s


def _acc(w, tri, xyz, stri, fix=None):
    return oracle.accumulate(tri, xyz, stri, fix if fix is not None else w.fixations, w.params,
                             delta_abs=DELTA, cone_band=BAND)


def _clean_lit_samples(w, tri, s, fix, n_max, rng):
    """Samples with a non-zero density and no pair near a cone edge or a grazing ray: their
    density is a smooth function of position within +-H."""
    base = _acc(w, tri, s.xyz, s.tri, fix)
    d, amb, sens = base["density"][0], base["amb"][0], base["sens"][0]
    ok = np.nonzero((d > 0) & (amb == 0) & (sens > 0))[0]
    assert len(ok) >= 10
    pick = np.sort(rng.choice(ok, min(n_max, len(ok)), replace=False))
    return pick, d[pick], sens[pick]


def test_sens_bounds_every_directional_derivative(scene):
    w, tri, s = scene
    rng = np.random.default_rng(11)
    pick, d0, sens = _clean_lit_samples(w, tri, s, None, 60, rng)
    xyz, stri = s.xyz[pick], s.tri[pick]
    worst = 0.0
    for _ in range(6):
        u = rng.normal(size=(len(pick), 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        dp = _acc(w, tri, xyz + H * u, stri)
        dm = _acc(w, tri, xyz - H * u, stri)
        assert not dp["amb"][0].any() and not dm["amb"][0].any()
        slope = np.abs(dp["density"][0] - dm["density"][0]) / (2 * H)
        # FD error: second-order truncation and rounding, far below 1e-6 of the density per metre
        assert np.all(slope <= sens * (1 + 1e-4) + 1e-6 * d0), "sens is below an observed slope"
        worst = max(worst, float((slope / sens).max()))
    # over 360 random directions some derivative comes close to the bound
    assert worst > 0.3


@pytest.mark.parametrize("f", [3, 17, 42, 77])
def test_sens_is_tight_for_a_single_pair(scene, f):
    w, tri, s = scene
    fix = w.fixations.subset(slice(f, f + 1))
    rng = np.random.default_rng(100 + f)
    try:
        pick, d0, sens = _clean_lit_samples(w, tri, s, fix, 40, rng)
    except AssertionError:
        pytest.skip(f"fixation {f} lights fewer than 10 clean samples")
    xyz, stri = s.xyz[pick], s.tri[pick]
    grad = np.empty((len(pick), 3))
    for c in range(3):
        e = np.zeros(3)
        e[c] = H
        dp = _acc(w, tri, xyz + e, stri, fix)["density"][0]
        dm = _acc(w, tri, xyz - e, stri, fix)["density"][0]
        grad[:, c] = (dp - dm) / (2 * H)
    gn = np.linalg.norm(grad, axis=1)
    tol = 1e-6 * d0
    assert np.all(gn <= sens * (1 + 1e-4) + tol), "gradient above sens"
    assert np.all(gn >= sens / math.sqrt(2) * (1 - 1e-4) - tol), "sens more than sqrt(2) above the gradient"


def test_sens_is_zero_where_nothing_is_seen(scene):
    """Samples with no visible in-cone pair have density 0 and sens 0 (sens only sums what is
    added to the density)."""
    w, tri, s = scene
    r = _acc(w, tri, s.xyz, s.tri)
    d, sens = r["density"][0], r["sens"][0]
    assert np.all(sens[d == 0] == 0)
    assert np.all(sens[d > 0] >= 0)
