"""The export record of Section 3.3.3 assembled on the GPU (gm_samples_export) against the
oracle's: triangle and object ids bit-exact, barycentrics and positions within FP32 rounding,
values identical to the map's, host and device destinations alike."""
import numpy as np
import pytest

import oracle
from tests.parity_utils import tri_max_coord, ulp32
from tests.test_oracle_export_pins import rotated_workload

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


def test_export_record_parity(env, tmp_path):
    import torch
    G, pipe, ctx = env
    w = rotated_workload()
    w.meshes[1].object_id = 9
    tri = oracle.world_triangles(w)
    off = oracle.tri_offsets(oracle.areas(tri), oracle.tri_density(w))
    smp = oracle.samples(tri, off, w.seed, w.session)
    ref = oracle.export_record(w, smp)
    h = pipe.run(ctx, w)
    n = G.gm_samples_info(h.samples)
    assert n == len(smp.tri)
    rec = dict(value=np.empty(n, np.float32), object_id=np.empty(n, np.uint32), triangle=np.empty(n, np.uint32),
               bary3=np.empty((n, 3), np.float32), local_xyz=np.empty((n, 3), np.float32),
               world_xyz=np.empty((n, 3), np.float32))
    G.gm_samples_export(h.samples, h.map, 0, **rec)
    v = np.empty(n, np.float32)
    G.gm_map_copy(h.map, 0, v)
    assert np.array_equal(rec["value"], v)
    assert np.array_equal(rec["triangle"].astype(np.int64), ref["triangle"])
    assert np.array_equal(rec["object_id"], ref["object_id"].astype(np.uint32))
    assert np.abs(rec["bary3"].astype(np.float64) - ref["bary3"]).max() <= 2.0 ** -21
    M = tri_max_coord(tri, smp.tri)
    assert np.all(np.abs(rec["world_xyz"].astype(np.float64) - ref["world_xyz"]) <= 8 * ulp32(M)[:, None])
    # local = A^-1 (x - t): the world error grows by at most ||A^-1||_2 (< 1/0.8 here), plus FP32 rounding
    L = np.abs(ref["local_xyz"]).max(1)
    tol = 8 * ulp32(M) / 0.8 + 2 * ulp32(L) + 1e-12
    assert np.all(np.abs(rec["local_xyz"].astype(np.float64) - ref["local_xyz"]) <= tol[:, None])
    # device destinations and a subset of fields give the same bytes
    dl = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    dt = torch.empty(n, dtype=torch.int32, device="cuda")
    G.gm_samples_export(h.samples, h.map, 0, local_xyz=dl, triangle=dt)
    G.gm_sync(ctx)
    assert np.array_equal(dl.cpu().numpy(), rec["local_xyz"])
    assert np.array_equal(dt.cpu().numpy().view(np.uint32), rec["triangle"])
    from paper_2601_07571_gb300 import export
    export.write_npz(str(tmp_path / "rec.npz"), h.samples, h.map)
    z = np.load(tmp_path / "rec.npz")
    assert np.array_equal(z["value_w0"], v) and np.array_equal(z["local_xyz"], rec["local_xyz"])
    h.free()


def test_export_rejects_singular_transform_for_local_positions(env):
    G, pipe, ctx = env
    w = rotated_workload()
    w.meshes[1].transform = np.diag([1.0, 0.0, 1.0, 1.0])   # flattens the cube: no local frame
    h = pipe.run(ctx, w)
    n = G.gm_samples_info(h.samples)
    with pytest.raises(RuntimeError, match="singular"):
        G.gm_samples_export(h.samples, h.map, 0, local_xyz=np.empty((n, 3), np.float32))
    G.gm_samples_export(h.samples, h.map, 0, world_xyz=np.empty((n, 3), np.float32))   # other fields still fine
    with pytest.raises(RuntimeError):
        G.gm_samples_export(h.samples, h.map, 1, value=np.empty(n, np.float32))           # one window only
    h.free()
