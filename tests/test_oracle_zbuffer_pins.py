"""Pins of the oracle's z-buffer path (Sections 3.2.2 and 3.3.2, Appendix A) to facts outside its
own arithmetic: the crop window against a brute-force bounding box of the cone's rim; the
printed Appendix-A construction against closed forms of a conic section; z-buffer depths of a
square and a tilted plane against ray/plane closed forms; z-buffer visibility against the convex
facet rule and an FP64 slab-test shadow."""
import math

import numpy as np
import pytest

import oracle
import synth
from synth import meshes as M
from tests.test_oracle_pins import _fix, _one_mesh_workload, _outward_normals, _slab_hits


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def _rim_bbox(rc, phi, n, m=20000):
    """Bounding box on the plane z = -n of m directions at angle phi from rc (brute force)."""
    rc = _unit(rc)
    a = _unit(np.cross(rc, [0.3, 0.7, 0.1]))
    b = np.cross(rc, a)
    t = np.linspace(0, 2 * np.pi, m, endpoint=False)
    d = math.cos(phi) * rc + math.sin(phi) * (np.cos(t)[:, None] * a + np.sin(t)[:, None] * b)
    x = -n * d[:, 0] / d[:, 2]
    y = -n * d[:, 1] / d[:, 2]
    return np.array([x.min(), x.max(), y.min(), y.max()])


@pytest.mark.parametrize("theta_deg", [0.5, 1.0, 3.0])
def test_exact_crop_window_is_the_rim_bounding_box(theta_deg):
    rng = np.random.default_rng(21)
    phi = math.atan(4 * math.tan(math.radians(theta_deg)))
    for _ in range(30):
        ang = math.radians(rng.uniform(0, 40))
        az = rng.uniform(0, 2 * np.pi)
        rc = np.array([math.sin(ang) * math.cos(az), math.sin(ang) * math.sin(az), -math.cos(ang)])
        n = rng.uniform(0.01, 0.5)
        ex = oracle.crop_exact(rc, phi, n)
        bf = _rim_bbox(rc, phi, n)
        width = ex[1] - ex[0]
        # the sampled rim lies inside the exact box and reaches it to O((2 pi / m)^2)
        assert np.all(np.abs(ex - bf) <= 1e-6 * width)
        assert bf[0] >= ex[0] - 1e-12 and bf[1] <= ex[1] + 1e-12 and bf[2] >= ex[2] - 1e-12 and bf[3] <= ex[3] + 1e-12
    # a cone reaching behind the camera has no crop window
    assert oracle.crop_exact([1.0, 0.0, -0.01], phi, 0.1) is None


def test_appendix_crop_construction_closed_forms():
    phi = math.atan(4 * math.tan(math.radians(1.0)))
    n = 0.05
    # gaze along the forward axis: a circle of radius n tan(phi) centred on M
    c = oracle.crop_paper([0, 0, -1], phi, n)
    assert c["a"] == pytest.approx(n * math.tan(phi), rel=1e-14) and c["alpha"] == 0.0
    assert np.allclose([c["l"], c["r"], c["b"], c["t"]], [-c["a"], c["a"], -c["a"], c["a"]], rtol=0, atol=1e-15)
    rng = np.random.default_rng(22)
    for _ in range(20):
        beta = math.radians(rng.uniform(2, 35))
        az = rng.uniform(0, 2 * np.pi)
        rc = np.array([math.sin(beta) * math.cos(az), math.sin(beta) * math.sin(az), -math.cos(beta)])
        c = oracle.crop_paper(rc, phi, n)
        # A0, A1 are the vertices of the section on its major axis: a = n (tan(beta+phi) - tan(beta-phi)) / 2
        assert c["a"] == pytest.approx(0.5 * n * (math.tan(beta + phi) - math.tan(beta - phi)), rel=1e-9)
        # the major axis points away from M: alpha is the azimuth of E (up to sign)
        assert math.cos(c["alpha"]) == pytest.approx(abs(math.cos(az)) * np.sign(math.cos(az)), abs=1e-9)
        assert np.allclose(c["E"], n * math.tan(beta) * np.array([math.cos(az), math.sin(az)]), rtol=1e-12, atol=0)
        # the printed window is E-centred; the section's centre is not E, so the window is off by a small shift
        ex = oracle.crop_exact(rc, phi, n)
        width = ex[1] - ex[0]
        assert np.all(np.abs(np.array([c["l"], c["r"], c["b"], c["t"]]) - ex) <= 0.03 * width)


def _square(D, half, cx=0.0, cy=0.0):
    v = np.array([[cx - half, cy - half, -D], [cx + half, cy - half, -D], [cx + half, cy + half, -D],
                  [cx - half, cy + half, -D]], np.float32)
    return v[[0, 1, 2, 0, 2, 3]].reshape(2, 9)


def test_render_square_depth_and_coverage_closed_form():
    n, res = 0.05, 48
    F = oracle.zb_frustum([0, 0, 0], [0, 0, -1], [0, 0, -1], [0, 1, 0], math.radians(2.0), 4.0, n, 100.0)
    D, half = 2.0, 0.11
    tri = _square(D, half, cx=0.03)
    z, amb = oracle.zb_render(tri, F, res)
    xs = F["l"] + (np.arange(res) + 0.5) * (F["r"] - F["l"]) / res
    ys = F["b"] + (np.arange(res) + 0.5) * (F["t"] - F["b"]) / res
    X, Y = np.meshgrid(xs * D / n, ys * D / n)
    inside = (np.abs(X - 0.03) < half) & (np.abs(Y) < half)
    assert inside.sum() > 100 and (~inside).sum() > 100
    sure = ~amb
    assert np.all(z[inside & sure] == pytest.approx(D, rel=1e-12))
    assert np.all(np.isinf(z[~inside & sure]))


def test_render_tilted_plane_depth_closed_form():
    n, res = 0.05, 32
    F = oracle.zb_frustum([0.1, 0.2, 0.3], [0.05, 0.02, -1], [0, 0, -1], [0, 1, 0], math.radians(2.0), 4.0, n, 100.0)
    # plane z = 0.3 - 1.5 + 0.4 (x - 0.1) through a large quad (the camera looks down -z)
    quad = np.array([[-2, -2, 0], [2, -2, 0], [2, 2, 0], [-2, 2, 0]], np.float64)
    quad[:, 2] = -1.2 + 0.4 * (quad[:, 0] - 0.1)
    tri = quad[[0, 1, 2, 0, 2, 3]].reshape(2, 9).astype(np.float32)
    z, amb = oracle.zb_render(tri, F, res)
    e = F["e"]
    xs = F["l"] + (np.arange(res) + 0.5) * (F["r"] - F["l"]) / res
    ys = F["b"] + (np.arange(res) + 0.5) * (F["t"] - F["b"]) / res
    v0 = tri[0, :3].astype(np.float64)
    nrm = np.cross(tri[0, 3:6].astype(np.float64) - v0, tri[0, 6:9].astype(np.float64) - v0)
    for j, y in enumerate(ys):
        for i, x in enumerate(xs):
            d = x * F["right"] + y * F["up"] + n * F["fwd"]
            t = np.dot(v0 - e, nrm) / np.dot(d, nrm)
            if not amb[j, i]:
                assert z[j, i] == pytest.approx(t * n, rel=1e-12)


def _ray_and_zb(w, cam_fwd, cam_up, zb, delta_px=1e-3):
    tri = oracle.world_triangles(w)
    off = oracle.tri_offsets(oracle.areas(tri), oracle.tri_density(w))
    smp = oracle.samples(tri, off, w.seed, w.session)
    zr = oracle.zb_accumulate(tri, smp.xyz, w.fixations, cam_fwd, cam_up, w.params, zb, delta_px=delta_px,
                              record=True)
    return tri, smp, zr


def test_zbuffer_visibility_on_convex_sphere_is_the_facet_rule():
    rng = np.random.default_rng(23)
    v, f = M.icosphere(3, 1.0)
    nfx = 8
    d = rng.normal(size=(nfx, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    eye = d * rng.uniform(2.0, 3.0, size=(nfx, 1))
    tgt = rng.normal(size=(nfx, 3)) * 0.3
    gaze = tgt - eye
    w = _one_mesh_workload(v, f, 4000.0, _fix(eye, gaze), params=synth.Params(theta_rad=math.radians(3.0)))
    cam_fwd = -eye                      # the head faces the sphere's centre, the gaze wanders off it
    cam_up = np.tile([0.0, 1.0, 0.0], (nfx, 1))
    tri, smp, zr = _ray_and_zb(w, cam_fwd, cam_up, oracle.ZBuffer(res=256, eps=0.01))
    P = zr["pairs"]
    nrm, t = _outward_normals(tri)
    st = smp.tri[P["sample"]]
    e = eye[P["fix"]]
    s = smp.xyz[P["sample"]]
    facing = ((nrm[st] * (e - t[st, 0])).sum(1)) / np.linalg.norm(nrm[st], axis=1) / np.linalg.norm(e - s, axis=1)
    inc = (P["flag"] & oracle.PF_IN_CONE) > 0
    amb = (P["flag"] & oracle.PF_VIS_AMBIG) > 0
    vis = (P["flag"] & oracle.PF_VISIBLE) > 0
    clear = inc & ~amb & (np.abs(facing) > 0.35)     # away from the silhouette (slope x pixel < eps)
    assert clear.sum() > 2000 and (facing[clear] > 0).sum() > 1000 and (facing[clear] < 0).sum() > 500
    assert np.array_equal(vis[clear], facing[clear] > 0)
    assert zr["stats"]["skipped_fixations"] == 0


def test_zbuffer_shadow_of_a_box_on_a_plane():
    rng = np.random.default_rng(24)
    g = 24
    xs = np.linspace(-1, 1, g + 1)
    pv = np.array([(x, y, 0.0) for x in xs for y in xs])
    pf = []
    for i in range(g):
        for j in range(g):
            a, b, c, d = i * (g + 1) + j, (i + 1) * (g + 1) + j, (i + 1) * (g + 1) + j + 1, i * (g + 1) + j + 1
            pf += [(a, b, c), (a, c, d)]
    lo, hi = np.array([-0.12, -0.1, 0.35]), np.array([0.1, 0.14, 0.6])
    bv, bf = M.box((lo + hi) / 2, (hi - lo) / 2)
    v, f = M.merge([(pv.astype(np.float32), np.array(pf)), (bv, bf)])
    nfx = 6
    eye = np.stack([rng.uniform(-0.2, 0.2, nfx), rng.uniform(-0.2, 0.2, nfx), rng.uniform(1.6, 2.2, nfx)], 1)
    tgt = np.stack([rng.uniform(-0.1, 0.1, nfx), rng.uniform(-0.1, 0.1, nfx), np.zeros(nfx)], 1)
    w = _one_mesh_workload(v, f, 30000.0, _fix(eye, tgt - eye), params=synth.Params(theta_rad=math.radians(4.0)))
    tri, smp, zr = _ray_and_zb(w, tgt - eye, np.tile([0.0, 1.0, 0.0], (nfx, 1)), oracle.ZBuffer(res=192, eps=0.004))
    P = zr["pairs"]
    on_plane = smp.tri[P["sample"]] < 2 * g * g
    inc = (P["flag"] & oracle.PF_IN_CONE) > 0
    amb = (P["flag"] & oracle.PF_VIS_AMBIG) > 0
    vis = (P["flag"] & oracle.PF_VISIBLE) > 0
    s = smp.xyz[P["sample"]]
    e = eye[P["fix"]]
    tmax = 1 - 1e-5
    grow, shrink = 0.01, 0.01       # a margin of a few pixels around the shadow's edge
    deep = _slab_hits(e, s - e, lo + shrink, hi - shrink, tmax)
    clear = ~_slab_hits(e, s - e, lo - grow, hi + grow, tmax)
    sel = inc & on_plane & ~amb
    assert (sel & deep).sum() > 300 and (sel & clear).sum() > 1000
    assert not vis[sel & deep].any()
    assert vis[sel & clear].all()


def test_sampled_pair_form_agrees_with_the_full_form():
    """zb_pairs (pixels cast on demand, for full-size scenes) reproduces zb_accumulate's recorded
    decisions pair by pair."""
    w = synth.tiny_sphere(n_fix=30)
    w.params = synth.Params(theta_rad=math.radians(3.0))
    fwd, up = synth.head_frames(w.fixations)
    zb = oracle.ZBuffer(res=64, eps=0.005)
    tri = oracle.world_triangles(w)
    off = oracle.tri_offsets(oracle.areas(tri), oracle.tri_density(w))
    smp = oracle.samples(tri, off, w.seed, w.session)
    full = oracle.zb_accumulate(tri, smp.xyz, w.fixations, fwd, up, w.params, zb, record=True)
    P = full["pairs"]
    inc = (P["flag"] & oracle.PF_IN_CONE) > 0
    s_i, f_i = P["sample"][inc], P["fix"][inc]
    pick = np.random.default_rng(25).choice(len(s_i), size=min(1500, len(s_i)), replace=False)
    s_i, f_i, flags = s_i[pick], f_i[pick], P["flag"][inc][pick]
    fx = w.fixations
    vis, amb, ok = oracle.zb_pairs(tri, smp.xyz[s_i], fx.eye[f_i], fx.gaze[f_i], fwd[f_i], up[f_i],
                                   w.params.theta_rad, w.params.cutoff_sigmas, zb)
    assert ok.all()
    assert np.array_equal(vis, (flags & oracle.PF_VISIBLE) > 0)
    assert np.array_equal(amb, (flags & oracle.PF_VIS_AMBIG) > 0)
    assert vis.sum() > 100 and (~vis).sum() > 100


def test_fp32_camera_depth_error_bound():
    """The clip-plane ambiguity band of the oracle's z-buffer bookkeeping is twice a bound on the
    error of a camera depth w = (p - e).fwd evaluated in FP32 from FP32 inputs (subtraction, then a
    chain of multiply-adds with an FP32 copy of the unit axis): six units of 2^-24 of ||p - e||_1.
    Checked against FP32 evaluations of random points up to 200 m from random eyes."""
    rng = np.random.default_rng(12)
    n = 200_000
    e = rng.uniform(-100, 100, (n, 3)).astype(np.float32)
    p = (e.astype(np.float64) + rng.normal(0, 60, (n, 3))).astype(np.float32)
    f64 = rng.normal(size=(n, 3))
    f64 /= np.linalg.norm(f64, axis=1, keepdims=True)
    f32 = f64.astype(np.float32)

    def fma32(a, b, c):   # a*b is exact in FP64 for FP32 a, b; one rounding of the sum to FP32
        return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)

    d = (p - e).astype(np.float32)
    w32 = fma32(d[:, 0], f32[:, 0], fma32(d[:, 1], f32[:, 1], (d[:, 2] * f32[:, 2]).astype(np.float32)))
    dx = p.astype(np.float64) - e.astype(np.float64)
    w64 = (dx * f64).sum(1)
    bound = 6 * 2.0 ** -24 * np.abs(dx).sum(1)
    err = np.abs(w32.astype(np.float64) - w64)
    assert np.all(err <= bound)
    assert err.max() > 0.1 * bound.max() / 6    # the bound is not vacuous: errors of a unit occur
