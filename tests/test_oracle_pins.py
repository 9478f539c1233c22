"""Pins for the FP64 oracle: each check ties it to something other than itself.

- Philox4x32-10 against Triton's independent implementation (run on the CPU interpreter);
- areas against Heron's formula (Section 3.1.2) and exact closed forms;
- per-triangle counts against the invariants count ~ k*A within one sample (Section 3.1.2);
- sample positions: barycentric sums, in-plane/inside checks and a chi-square uniformity test;
- the Gaussian of Section 3.2.1 against its closed forms (peak, one sigma, the 4 sigma edge);
- occlusion against the convex-polyhedron facet rule, a box's shadow by an FP64 slab test, and
  an independent pure-Python plane-crossing test on a random triangle soup;
- a plane seen head-on against g(atan(rho/D)) and its integral;
- per-window sums and max-normalisation (Section 3.2.3).
All run on the CPU in a few seconds each.
"""
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
import synth
from synth import meshes as M

TH1 = math.radians(1.0)


def _one_mesh_workload(v, f, density, fixations, params=None, seed=5, session=0):
    mesh = synth.Mesh(np.asarray(v, np.float32), np.asarray(f, np.uint32), synth.identity(), 0, density)
    return synth.Workload("t", [mesh], fixations, params or synth.Params(), seed=seed, session=session)


def _fix(eye, gaze, dur=None, ts=None):
    eye = np.atleast_2d(np.asarray(eye, np.float32))
    gaze = np.atleast_2d(np.asarray(gaze, np.float32))
    n = len(eye)
    dur = np.full(n, 0.25, np.float32) if dur is None else np.asarray(dur, np.float32)
    ts = np.arange(n, dtype=np.float64) if ts is None else np.asarray(ts, np.float64)
    return synth.Fixations(eye, gaze, dur, ts)


# --------------------------------------------------------------------------------------
# Philox4x32-10
# --------------------------------------------------------------------------------------
_TRITON_SCRIPT = textwrap.dedent(r'''
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(out, cp, seed, N: tl.constexpr):
        i = tl.arange(0, N)
        c0 = tl.load(cp + 4 * i + 0)
        c1 = tl.load(cp + 4 * i + 1)
        c2 = tl.load(cp + 4 * i + 2)
        c3 = tl.load(cp + 4 * i + 3)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out + 4 * i + 0, a)
        tl.store(out + 4 * i + 1, b)
        tl.store(out + 4 * i + 2, c)
        tl.store(out + 4 * i + 3, d)

    req = json.loads(sys.stdin.read())
    res = []
    for seed, ctr in req:
        c = torch.tensor(np.array(ctr, dtype=np.uint32).view(np.int32))
        o = torch.zeros_like(c)
        k[(1,)](o, c, seed, N=len(ctr))
        res.append((o.numpy().view(np.uint32).reshape(-1, 4)).tolist())
    print(json.dumps(res))
''')


def test_philox_matches_triton_interpreter():
    pytest.importorskip("triton")
    rng = np.random.default_rng(11)
    cases = []
    for seed in (0, 1, 12345, 0xDEADBEEFCAFEF00D, (1 << 64) - 1):
        ctr = rng.integers(0, 2 ** 32, size=(16, 4), dtype=np.uint64).astype(np.uint32)
        ctr[0] = 0
        ctr[1] = [0xFFFFFFFF] * 4
        ctr[2] = [7, 0, 3, 0]           # (j lo, j hi, session, 0) as the sampler uses it
        cases.append((seed, ctr))
    import json
    env = dict(os.environ, TRITON_INTERPRET="1")
    out = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], env=env, check=True,
                         input=json.dumps([(s if s < (1 << 63) else s - (1 << 64), c.tolist()) for s, c in cases]),
                         capture_output=True, text=True, timeout=600)
    ref = json.loads(out.stdout.strip().splitlines()[-1])
    for (seed, ctr), r in zip(cases, ref):
        key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
        mine = oracle.philox(ctr, key)
        assert np.array_equal(mine, np.asarray(r, np.uint32)), f"seed {seed}"


def test_philox_depends_on_every_input_word():
    base = np.zeros((1, 4), np.uint32)
    ref = oracle.philox(base, (0, 0))
    for w in range(4):
        c = base.copy()
        c[0, w] = 1
        assert not np.array_equal(oracle.philox(c, (0, 0)), ref)
    assert not np.array_equal(oracle.philox(base, (1, 0)), ref)
    assert not np.array_equal(oracle.philox(base, (0, 1)), ref)


# --------------------------------------------------------------------------------------
# World transform and areas
# --------------------------------------------------------------------------------------
def test_world_transform_exact_and_against_matmul():
    rng = np.random.default_rng(0)
    v = rng.uniform(-3, 3, size=(1000, 3)).astype(np.float32)
    m = np.eye(4)
    m[:3, :3] *= 2.0
    m[:3, 3] = (0.5, -0.25, 4.0)
    out = oracle.world_vertices(v, m)
    assert np.array_equal(out, (v.astype(np.float64) * 2.0 + m[:3, 3]).astype(np.float32))
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    m[:3, :3] = q * 1.37
    out = oracle.world_vertices(v, m)
    ref = (v.astype(np.float64) @ m[:3, :3].T + m[:3, 3]).astype(np.float32)
    ulp = np.spacing(np.abs(ref).astype(np.float32))
    assert np.all(np.abs(out.astype(np.float64) - ref) <= ulp)


def test_area_closed_forms():
    tri = np.array([[0, 0, 0, 3, 0, 0, 0, 4, 0],           # right triangle 3-4-5 -> 6
                    [1, 1, 1, 1, 1, 1, 2, 2, 2],           # degenerate -> 0
                    [0, 0, 0, 1, 0, 0, 2, 0, 0],           # collinear -> 0
                    [0, 0, 0, 0.5, 0, 0, 0, 0, 0.25]],     # 1/16
                   np.float32)
    a = oracle.areas(tri)
    assert a[0] == 6.0 and a[1] == 0.0 and a[2] == 0.0 and a[3] == 0.0625
    v, f = M.box((1.5, 0.0, 0.0), 0.2)
    w = _one_mesh_workload(v, f, 1.0, _fix([0, 0, 5], [0, 0, -1]))
    assert abs(oracle.areas(oracle.world_triangles(w)).sum() - 0.96) < 1e-6


def test_area_cross_product_equals_heron():
    rng = np.random.default_rng(1)
    tri = rng.normal(size=(20000, 9)).astype(np.float32) * rng.uniform(1e-3, 10, size=(20000, 1)).astype(np.float32)
    a = oracle.areas(tri)
    h = oracle.areas_heron(tri)
    t = tri.astype(np.float64).reshape(-1, 3, 3)
    e = [t[:, 1] - t[:, 0], t[:, 2] - t[:, 1], t[:, 0] - t[:, 2]]
    L = np.stack([np.linalg.norm(x, axis=1) for x in e], 1)
    # skip slivers, where Heron loses digits: smallest altitude over longest edge above 1e-2
    ok = (2 * a / L.max(1)) / L.max(1) > 1e-2
    assert ok.sum() > 15000
    assert np.all(np.abs(a[ok] - h[ok]) <= 1e-9 * a[ok])


def test_icosphere_area_converges_to_sphere():
    prev = None
    for sd in (1, 2, 3, 4):
        v, f = M.icosphere(sd, 1.0)
        w = _one_mesh_workload(v, f, 1.0, _fix([0, 0, 5], [0, 0, -1]))
        a = oracle.areas(oracle.world_triangles(w)).sum()
        assert a < 4 * math.pi
        if prev is not None:
            assert a > prev
        prev = a
    assert abs(prev - 4 * math.pi) / (4 * math.pi) < 5e-3


# --------------------------------------------------------------------------------------
# Counts (area-weighted, within one sample of k*A per triangle)
# --------------------------------------------------------------------------------------
def test_counts_invariants():
    rng = np.random.default_rng(2)
    n = 50000
    area = np.exp(rng.uniform(math.log(1e-9), math.log(1e-1), size=n))
    area[rng.integers(0, n, 500)] = 0.0
    k = np.exp(rng.uniform(math.log(10), math.log(1e6), size=n))
    off = oracle.tri_offsets(area, k)
    cnt = np.diff(off)
    assert off[0] == 0 and np.all(cnt >= 0)
    c = k * area
    assert np.all(np.abs(cnt - c) <= 1.0 + 1e-9)
    assert np.all(cnt[area == 0] == 0)
    assert abs(off[-1] - c.sum()) <= 0.5 + n * 2.0 ** -32
    # exact integers stay exact
    off = oracle.tri_offsets(np.full(10, 0.5), np.full(10, 4.0))
    assert np.array_equal(off, np.arange(11) * 2)


def test_tiny_sphere_total_count():
    w = synth.tiny_sphere()
    tri = oracle.world_triangles(w)
    a = oracle.areas(tri)
    off = oracle.tri_offsets(a, oracle.tri_density(w))
    assert abs(off[-1] - 500 * a.sum()) <= 0.5 + 1e-6
    assert off[-1] == 6645


# --------------------------------------------------------------------------------------
# Sample positions
# --------------------------------------------------------------------------------------
def test_samples_lie_in_their_triangle():
    rng = np.random.default_rng(3)
    tri = rng.normal(size=(300, 9)).astype(np.float32)
    off = oracle.tri_offsets(oracle.areas(tri), 2000.0)
    s = oracle.samples(tri, off, seed=77, session=3)
    n = off[-1]
    assert len(s.tri) == n
    assert np.all(off[s.tri] <= s.index) and np.all(s.index < off[s.tri + 1])
    assert np.all(s.bary >= 0) and np.allclose(s.bary.sum(1), 1.0, atol=1e-15)
    t = tri.astype(np.float64).reshape(-1, 3, 3)[s.tri]
    # recover barycentrics from the position by least squares: they must match and be >= 0
    A = np.stack([t[:, 1] - t[:, 0], t[:, 2] - t[:, 0]], axis=2)
    sol = np.linalg.lstsq(A[0], (s.xyz[0] - t[0, 0]), rcond=None)[0]
    assert np.allclose(sol, s.bary[0, 1:], atol=1e-9)
    rhs = s.xyz - t[:, 0]
    ata = np.einsum("nki,nkj->nij", A, A)
    atb = np.einsum("nki,nk->ni", A, rhs)
    b12 = np.linalg.solve(ata, atb[..., None])[..., 0]
    assert np.allclose(b12, s.bary[:, 1:], atol=1e-7)
    resid = rhs - np.einsum("nij,nj->ni", A, b12)
    assert np.abs(resid).max() < 1e-9


def test_sample_words_are_philox_of_index():
    rng = np.random.default_rng(4)
    tri = rng.normal(size=(50, 9)).astype(np.float32)
    off = oracle.tri_offsets(oracle.areas(tri), 500.0)
    seed, session = 0x0123456789ABCDEF, 9
    s = oracle.samples(tri, off, seed, session)
    ctr = np.stack([s.index & 0xFFFFFFFF, s.index >> 32, np.full(len(s.index), session),
                    np.zeros(len(s.index))], 1).astype(np.uint32)
    w = oracle.philox(ctr, (seed & 0xFFFFFFFF, seed >> 32))
    assert np.array_equal(s.words, w[:, :2])
    u1 = ((w[:, 0] >> 9).astype(np.float64) + 0.5) / 2 ** 23
    assert np.allclose(s.bary[:, 0], 1 - np.sqrt(u1), rtol=0, atol=1e-15)
    u2 = ((w[:, 1] >> 9).astype(np.float64) + 0.5) / 2 ** 23
    assert np.allclose(s.bary[:, 2] / (s.bary[:, 1] + s.bary[:, 2]), u2, rtol=1e-12, atol=0)


def test_samples_uniform_in_triangle_chi_square():
    stats = pytest.importorskip("scipy.stats")
    tri = np.array([[0, 0, 0, 1, 0, 0, 0, 1, 0]], np.float32)
    off = oracle.tri_offsets(oracle.areas(tri), 2_000_000.0)     # 1e6 samples
    s = oracle.samples(tri, off, seed=2024, session=0)
    b = s.bary
    # 16 congruent sub-triangles of the level-2 midpoint subdivision, each 1/16 of the area
    g1, g2 = b[:, 1] * 4, b[:, 2] * 4
    i, j = np.floor(g1).astype(int), np.floor(g2).astype(int)
    up = (g1 - i) + (g2 - j) < 1
    cell = np.where(up, 0, 1) + 2 * (i * 4 + j)
    valid = i + j <= 3
    counts = np.bincount(cell[valid], minlength=32)
    used = np.array([c for c in range(32) if ((c // 2) // 4 + (c // 2) % 4 + (c % 2)) <= 3])
    obs = counts[used]
    assert len(used) == 16 and obs.sum() == len(b)
    chi2 = ((obs - len(b) / 16) ** 2 / (len(b) / 16)).sum()
    assert stats.chi2.sf(chi2, 15) > 1e-4


# --------------------------------------------------------------------------------------
# The Gaussian projection (Section 3.2.1)
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("theta_deg", [0.5, 1.0, 2.0])
def test_gaussian_closed_forms(theta_deg):
    th = math.radians(theta_deg)
    s_ = math.tan(th)
    t = 0.37
    D = 2.5
    peak = t / (s_ * math.sqrt(2 * math.pi))
    inside, g = oracle.pair_weight([0, 0, D], [0, 0, 0], [0, 0, 1], t, th)
    assert inside and abs(g - peak) <= 1e-15 * peak
    inside, g = oracle.pair_weight([D * s_, 0, D], [0, 0, 0], [0, 0, 1], t, th)
    assert inside and abs(g / peak - math.exp(-0.5)) < 1e-12
    inside, g = oracle.pair_weight([0, 2 * D * s_, D], [0, 0, 0], [0, 0, 3.0], t, th)
    assert inside and abs(g / peak - math.exp(-2.0)) < 1e-12
    inside, g = oracle.pair_weight([D * 4 * s_ * (1 - 1e-12), 0, D], [0, 0, 0], [0, 0, 1], t, th)
    assert inside and abs(g / peak - math.exp(-8.0)) < 1e-9
    inside, _ = oracle.pair_weight([D * 4 * s_ * (1 + 1e-9), 0, D], [0, 0, 0], [0, 0, 1], t, th)
    assert not inside
    assert not oracle.pair_weight([0, 0, -D], [0, 0, 0], [0, 0, 1], t, th)[0]
    assert not oracle.pair_weight([1, 0, 0], [0, 0, 0], [0, 0, 1], t, th)[0]


def test_gaussian_invariant_under_rigid_motion_and_gaze_length():
    rng = np.random.default_rng(5)
    for _ in range(200):
        q, _r = np.linalg.qr(rng.normal(size=(3, 3)))
        tr = rng.normal(size=3) * 3
        D = rng.uniform(0.3, 8)
        psi = rng.uniform(0, 4.2 * TH1)
        phi = rng.uniform(0, 2 * math.pi)
        s = np.array([D * math.tan(psi) * math.cos(phi), D * math.tan(psi) * math.sin(phi), D])
        r = np.array([0, 0, rng.uniform(0.1, 10)])
        t = rng.uniform(0.1, 0.6)
        ins, g = oracle.pair_weight(q @ s + tr, tr, q @ r, t, TH1)
        expect = t / (math.tan(TH1) * math.sqrt(2 * math.pi)) * math.exp(-(math.tan(psi) ** 2) / (2 * math.tan(TH1) ** 2))
        if abs(math.tan(psi) - 4 * math.tan(TH1)) > 1e-9:
            assert ins == (math.tan(psi) <= 4 * math.tan(TH1))
        assert abs(g - expect) <= 1e-11 * expect


# --------------------------------------------------------------------------------------
# Occlusion
# --------------------------------------------------------------------------------------
def _outward_normals(tri):
    t = tri.astype(np.float64).reshape(-1, 3, 3)
    n = np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0])
    c = t.mean(1)
    return np.where(((n * c).sum(1) < 0)[:, None], -n, n), t


def test_convex_icosphere_facet_rule():
    """On a convex polyhedron a point of facet F is visible from an outside eye e exactly when
    e is strictly on the outer side of F's plane."""
    rng = np.random.default_rng(6)
    v, f = M.icosphere(3, 1.0)
    nfx = 24
    d = rng.normal(size=(nfx, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    eye = d * rng.uniform(1.3, 3.0, size=(nfx, 1))
    tgt = rng.normal(size=(nfx, 3))
    tgt /= np.linalg.norm(tgt, axis=1, keepdims=True)
    # half the gazes graze the limb: aim at points near the silhouette
    w = _one_mesh_workload(v, f, 3000.0, _fix(eye, tgt - eye))
    r = oracle.run(w, delta_abs=1e-9, cone_band=0.0, record=True)
    n, t = _outward_normals(r["tri"])
    P = r["pairs"]
    s_tri = r["samples"].tri[P["sample"]]
    e = eye[P["fix"]]
    rule = ((n[s_tri] * (e - t[s_tri, 0])).sum(1)) > 0
    inc = (P["flag"] & oracle.PF_IN_CONE) > 0
    amb = (P["flag"] & oracle.PF_VIS_AMBIG) > 0
    vis = (P["flag"] & oracle.PF_VISIBLE) > 0
    sel = inc & ~amb
    assert sel.sum() > 10000 and rule[sel].sum() > 3000 and (~rule[sel]).sum() > 3000
    assert np.array_equal(vis[sel], rule[sel])
    assert amb.sum() <= 1e-3 * inc.sum()
    expect = np.zeros(len(r["samples"].tri))
    np.add.at(expect, P["sample"][inc & rule], P["g"][inc & rule])
    dens = r["density"][0]
    assert np.all(np.abs(dens - expect) <= 1e-12 * expect + r["amb"][0] + 1e-300)


def _slab_hits(o, d, lo, hi, tmax):
    """FP64 slab test: does o + t d, 0 < t < tmax, meet the closed box [lo, hi]?"""
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t0 = (lo - o) * inv
        t1 = (hi - o) * inv
    tn = np.nanmax(np.minimum(t0, t1), axis=-1)
    tf = np.nanmin(np.maximum(t0, t1), axis=-1)
    return (tn <= tf) & (tf > 0) & (tn < tmax)


def test_box_shadow_on_plane():
    """A box hovering over a plane: a plane sample is occluded exactly when the segment from
    the eye meets the box (FP64 slab test, no triangles involved)."""
    rng = np.random.default_rng(7)
    pv, pf = [], []
    g = 24
    xs = np.linspace(-1, 1, g + 1)
    for i in range(g + 1):
        for j in range(g + 1):
            pv.append((xs[i], xs[j], 0.0))
    for i in range(g):
        for j in range(g):
            a, b, c, d = i * (g + 1) + j, (i + 1) * (g + 1) + j, (i + 1) * (g + 1) + j + 1, i * (g + 1) + j + 1
            pf += [(a, b, c), (a, c, d)]
    lo, hi = np.array([-0.12, -0.1, 0.35]), np.array([0.1, 0.14, 0.6])
    bv, bf = M.box((lo + hi) / 2, (hi - lo) / 2)
    v, f = M.merge([(np.array(pv, np.float32), np.array(pf)), (bv, bf)])
    nfx = 12
    eye = np.stack([rng.uniform(-0.3, 0.3, nfx), rng.uniform(-0.3, 0.3, nfx), rng.uniform(1.5, 2.5, nfx)], 1)
    tgt = np.stack([rng.uniform(-0.3, 0.3, nfx), rng.uniform(-0.3, 0.3, nfx), np.zeros(nfx)], 1)
    w = _one_mesh_workload(v, f, 20000.0, _fix(eye, tgt - eye))
    r = oracle.run(w, delta_abs=1e-9, record=True)
    P = r["pairs"]
    on_plane = r["samples"].tri[P["sample"]] < 2 * g * g
    inc = (P["flag"] & oracle.PF_IN_CONE) > 0
    sel = inc & on_plane
    s = r["samples"].xyz[P["sample"][sel]]
    e = eye[P["fix"][sel]]
    d = s - e
    tmax = 1 - w.params.eps_rel
    occl = _slab_hits(e, d, lo, hi, tmax)
    grown = _slab_hits(e, d, lo - 1e-7, hi + 1e-7, tmax)
    shrunk = _slab_hits(e, d, lo + 1e-7, hi - 1e-7, tmax)
    sure = grown == shrunk
    vis = (P["flag"][sel] & oracle.PF_VISIBLE) > 0
    assert occl.sum() > 1000 and (~occl).sum() > 1000
    assert np.array_equal(vis[sure], ~occl[sure])
    # single fixation: the shadowed samples are exactly zero
    w1 = _one_mesh_workload(v, f, 20000.0, _fix(eye[:1], (tgt - eye)[:1]))
    r1 = oracle.run(w1, delta_abs=1e-9)
    sx = r1["samples"].xyz
    plane = r1["samples"].tri < 2 * g * g
    occ1 = _slab_hits(np.broadcast_to(eye[0], sx.shape), sx - eye[0], lo, hi, tmax)
    assert occ1[plane].sum() > 100
    assert np.all(r1["density"][0][plane & occ1] == 0.0)
    assert np.all(r1["density"][0][plane & ~occ1 & (r1["density"][0] > 0)] > 0)


def _py_segment_blocked(e, s, tris, own, eps):
    """Independent test: plane crossing + same-side point-in-triangle, plain Python floats."""
    end = [e[k] + (1 - eps) * (s[k] - e[k]) for k in range(3)]
    sub = lambda a, b: [a[0] - b[0], a[1] - b[1], a[2] - b[2]]
    dot = lambda a, b: a[0] * b[0] + a[1] * b[1] + a[2] * b[2]
    crs = lambda a, b: [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]
    for j, T in enumerate(tris):
        if j == own:
            continue
        a, b, c = T[0:3], T[3:6], T[6:9]
        n = crs(sub(b, a), sub(c, a))
        de, ds = dot(n, sub(e, a)), dot(n, sub(end, a))
        if de * ds >= 0:
            continue
        lam = de / (de - ds)
        X = [e[k] + lam * (end[k] - e[k]) for k in range(3)]
        s1 = dot(crs(sub(b, a), sub(X, a)), n)
        s2 = dot(crs(sub(c, b), sub(X, b)), n)
        s3 = dot(crs(sub(a, c), sub(X, c)), n)
        if (s1 >= 0 and s2 >= 0 and s3 >= 0) or (s1 <= 0 and s2 <= 0 and s3 <= 0):
            return True
    return False


def test_visibility_against_independent_python_on_triangle_soup():
    rng = np.random.default_rng(8)
    nt = 30
    c = rng.uniform(-1, 1, size=(nt, 1, 3))
    tri = (c + rng.normal(scale=0.35, size=(nt, 3, 3))).reshape(nt, 9).astype(np.float32)
    v = tri.reshape(-1, 3)
    f = np.arange(3 * nt).reshape(nt, 3)
    nfx = 10
    d = rng.normal(size=(nfx, 3))
    eye = d / np.linalg.norm(d, axis=1, keepdims=True) * 3.0
    prm = synth.Params(theta_rad=math.radians(9.0))
    w = _one_mesh_workload(v, f, 300.0, _fix(eye, -eye), params=prm)
    r = oracle.run(w, delta_abs=1e-9, record=True)
    P = r["pairs"]
    inc = (P["flag"] & oracle.PF_IN_CONE) > 0
    amb = (P["flag"] & oracle.PF_VIS_AMBIG) > 0
    sx, st = r["samples"].xyz, r["samples"].tri
    tl = r["tri"].astype(np.float64).tolist()
    n_checked = n_blocked = 0
    for k in np.nonzero(inc & ~amb)[0]:
        s = int(P["sample"][k])
        fi = int(P["fix"][k])
        blocked = _py_segment_blocked(eye[fi].tolist(), sx[s].tolist(), tl, int(st[s]), prm.eps_rel)
        assert blocked == (not (P["flag"][k] & oracle.PF_VISIBLE)), (s, fi)
        n_checked += 1
        n_blocked += blocked
    assert n_checked > 500 and 0.1 < n_blocked / n_checked < 0.9


def test_own_triangle_never_occludes_its_samples():
    """With eps_rel = 0 the segment ends on the sample's own triangle; only the exclusion of
    that triangle keeps rounding from hiding the sample."""
    v = np.array([[-1, -1, 0], [1.3, -0.9, 0.2], [-0.7, 1.1, -0.1]], np.float32)
    f = np.array([[0, 1, 2]])
    prm = synth.Params(theta_rad=math.radians(10.0), eps_rel=0.0)
    w = _one_mesh_workload(v, f, 20000.0, _fix([[0.1, 0.2, 3.0], [0.3, -0.2, -2.5]], [[0, 0, -1], [0, 0, 1]]), params=prm)
    r = oracle.run(w, record=True)
    P = r["pairs"]
    inc = (P["flag"] & oracle.PF_IN_CONE) > 0
    assert inc.sum() > 5000
    assert np.all((P["flag"][inc] & oracle.PF_VISIBLE) > 0)


def test_plane_head_on_closed_form():
    """Quad at distance D, gaze along its normal: d1 = D and d2 = rho, so each sample's value
    is t/(sigma sqrt(2 pi)) exp(-(rho/D)^2 / (2 sigma^2)) out to rho = 4 sigma D, and the sum
    over samples approaches k times the integral 2 pi sigma^2 D^2 (1 - e^-8) t/(sigma sqrt(2 pi))."""
    D, t, k = 2.0, float(np.float32(0.3)), 200_000.0
    v = np.array([[-0.5, -0.5, 0], [0.5, -0.5, 0], [0.5, 0.5, 0], [-0.5, 0.5, 0]], np.float32)
    f = np.array([[0, 1, 2], [0, 2, 3]])
    w = _one_mesh_workload(v, f, k, _fix([0, 0, D], [0, 0, -1], dur=[t]))
    r = oracle.run(w)
    x = r["samples"].xyz
    rho = np.hypot(x[:, 0], x[:, 1])
    sg = math.tan(TH1)
    expect = t / (sg * math.sqrt(2 * math.pi)) * np.exp(-((rho / D) ** 2) / (2 * sg * sg))
    expect[rho / D > 4 * sg] = 0.0
    dens = r["density"][0]
    edge = np.abs(rho / D - 4 * sg) < 1e-9
    assert np.all(np.abs(dens[~edge] - expect[~edge]) <= 1e-12 * expect[~edge])
    integral = t / (sg * math.sqrt(2 * math.pi)) * 2 * math.pi * sg * sg * D * D * (1 - math.exp(-8))
    assert abs(dens.sum() / k - integral) / integral < 0.02
    # 4 sigma holds 1 - e^-8 of the radial Gaussian, nearly all of it (Fig. 4 caption)
    assert 1 - math.exp(-8) > 0.9996


# --------------------------------------------------------------------------------------
# Windows and normalisation
# --------------------------------------------------------------------------------------
def test_windows_partition_the_sum():
    w = synth.tiny_sphere()
    base = oracle.run(w)
    ts = w.fixations.timestamp_s
    w.params = synth.Params(t_begin=0.0, t_end=float(ts.max()) + 1e-6, window_s=4.0)
    r = oracle.run(w)
    W = oracle.n_windows(w.params)
    assert r["density"].shape[0] == W > 3
    assert np.allclose(r["density"].sum(0), base["density"][0], rtol=1e-13, atol=0)
    win = oracle.fixation_windows(ts, w.params)
    assert np.array_equal(win, np.floor(ts / 4.0).astype(np.int32))
    # a time interval drops the fixations outside it
    w.params = synth.Params(t_begin=5.0, t_end=20.0)
    r2 = oracle.run(w)
    keep = (ts >= 5.0) & (ts < 20.0)
    assert r2["stats"]["pairs"] == keep.sum() * base["density"].shape[1]


def test_normalisation():
    v = np.array([0.0, 2.0, 8.0, 1.5])
    n, m = oracle.normalize(v)
    assert m == 8.0 and n.max() == 1.0 and np.all((n >= 0) & (n <= 1))
    n, m = oracle.normalize(np.zeros(5))
    assert m == 0.0 and np.all(n == 0.0)
    r = oracle.run(synth.tiny_sphere())
    n, m = oracle.normalize(r["density"][0])
    assert n.max() == 1.0 and m == r["density"][0].max()


def test_recorded_pairs_sum_to_density():
    r = oracle.run(synth.tiny_sphere(), record=True)
    P = r["pairs"]
    ok = ((P["flag"] & oracle.PF_IN_CONE) > 0) & ((P["flag"] & oracle.PF_VISIBLE) > 0)
    d = np.zeros(r["density"].shape[1])
    np.add.at(d, P["sample"][ok], P["g"][ok])
    assert np.allclose(d, r["density"][0], rtol=1e-13, atol=0)
    assert r["stats"]["visible"] == ok.sum()
