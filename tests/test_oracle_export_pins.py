"""Pins of the oracle's export record (Section 3.3.3) to facts outside its own arithmetic:
the mesh-local position is the barycentric combination of the mesh's own local vertices; an
identity transform leaves positions unchanged; object ids follow the meshes' triangle ranges."""
import math

import numpy as np

import oracle
import synth


def rotated_workload():
    """tiny_sphere with each mesh under a rotation, a non-uniform scale and a translation."""
    w = synth.tiny_sphere()
    for k, m in enumerate(w.meshes):
        a, b = 0.7 + k, -0.4 + 0.3 * k
        Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
        Rx = np.array([[1, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
        T = np.eye(4)
        T[:3, :3] = Rz @ Rx @ np.diag([1.3, 0.8, 1.1 + 0.2 * k])
        T[:3, 3] = (0.5 * k, -0.25, 0.1 * k)
        m.transform = T
    return w


def _samples(w):
    tri = oracle.world_triangles(w)
    off = oracle.tri_offsets(oracle.areas(tri), oracle.tri_density(w))
    return oracle.samples(tri, off, w.seed, w.session)


def test_local_position_is_barycentric_combination_of_local_vertices():
    w = rotated_workload()
    smp = _samples(w)
    rec = oracle.export_record(w, smp)
    base = np.cumsum([0] + [m.n_tris for m in w.meshes])
    exp = np.empty_like(rec["local_xyz"])
    for mi, m in enumerate(w.meshes):
        sel = (smp.tri >= base[mi]) & (smp.tri < base[mi + 1])
        v = m.vertices.astype(np.float64)[m.indices[smp.tri[sel] - base[mi]]]   # (k, 3, 3)
        exp[sel] = np.einsum("kc,kcd->kd", smp.bary[sel], v)
    # world vertices are rounded to FP32 before sampling: a few FP32 ulps of the scene size
    assert np.abs(rec["local_xyz"] - exp).max() < 2e-6
    assert np.all(rec["bary3"] >= 0) and np.allclose(rec["bary3"].sum(1), 1.0, atol=1e-12)


def test_identity_transform_leaves_positions_unchanged():
    w = synth.tiny_sphere()
    smp = _samples(w)
    rec = oracle.export_record(w, smp, values=np.arange(len(smp.tri)))
    assert np.array_equal(rec["local_xyz"], smp.xyz)
    assert np.array_equal(rec["value"], np.arange(len(smp.tri)))


def test_object_ids_follow_mesh_ranges():
    w = rotated_workload()
    w.meshes[0].object_id, w.meshes[1].object_id = 17, 4
    smp = _samples(w)
    rec = oracle.export_record(w, smp)
    n0 = w.meshes[0].n_tris
    assert np.array_equal(rec["object_id"], np.where(smp.tri < n0, 17, 4))
    assert np.array_equal(rec["triangle"], smp.tri)
