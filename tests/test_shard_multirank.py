"""The sample-sharded path's host logic on the CPU, with two and three gloo ranks.

Each rank takes its slice of the stored sample order (`shard.sample_shard`), computes its slice's
raw per-window values -- here with the FP64 oracle, rounded to FP32 like the GPU map, since this
box has no GPU -- exchanges its per-window maxima (`shard.allreduce_max`) and divides its slice by
the maximum over all ranks. Gathered, the slices must equal the single-process normalised map
bit for bit: every sample once, in order, divided by the same maximum. The same sharding on the
GPU (the library's slice, accumulation and normalisation calls) is checked in test_gpu_shard.py."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    import synth
    w = synth.tiny_sphere(n_fix=120)
    ts = w.fixations.timestamp_s
    w.params = synth.Params(t_begin=0.0, t_end=float(ts.max()) + 1.0, window_s=9.0)
    return w


def _raw_values(w, which):
    """Raw per-window values of the stored samples `which`, FP32 (the oracle stands in for a GPU)."""
    import oracle
    tri = oracle.world_triangles(w)
    off = oracle.tri_offsets(oracle.areas(tri), oracle.tri_density(w))
    s = oracle.samples(tri, off, w.seed, w.session, which)
    r = oracle.accumulate(tri, s.xyz, s.tri, w.fixations, w.params, nthreads=2)
    return r["density"].astype(np.float32)


def _n_samples(w):
    import oracle
    tri = oracle.world_triangles(w)
    return int(oracle.tri_offsets(oracle.areas(tri), oracle.tri_density(w))[-1])


def _normalise(v, m):
    out = np.zeros_like(v)
    for k in range(v.shape[0]):
        if m[k] > 0:
            out[k] = v[k] / np.float32(m[k])
    return out


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2601_07571_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        w = _workload()
        b, e = shard.sample_shard(_n_samples(w), rank, world)
        raw = _raw_values(w, np.arange(b, e, dtype=np.int64))
        local = raw.max(axis=1) if raw.shape[1] else np.zeros(raw.shape[0], np.float32)
        gmax = shard.allreduce_max(local, dist, "cpu")
        got = [None] * world
        dist.all_gather_object(got, (b, e, _normalise(raw, gmax), gmax))
        if rank == 0:
            out["parts"] = got
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_maps_equal_the_single_process_map(world):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    oracle.build()
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    parts = out["parts"]
    w = _workload()
    n = _n_samples(w)
    # the slices are contiguous, disjoint and cover every sample
    assert parts[0][0] == 0 and parts[-1][1] == n
    assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
    whole = _raw_values(w, np.arange(n, dtype=np.int64))
    ref = _normalise(whole, whole.max(axis=1))
    got = np.concatenate([p[2] for p in parts], axis=1)
    assert whole.shape[0] > 3 and np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    for p in parts:
        assert np.array_equal(p[3], whole.max(axis=1))


def test_shard_bounds():
    from paper_2601_07571_gb300 import shard
    for n in (0, 1, 7, 1000, 2_000_003):
        for world in (1, 2, 3, 8):
            b = [shard.sample_shard(n, r, world) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
            sizes = [e - s for s, e in b]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.sample_shard(10, 2, 2)
    assert np.array_equal(shard.allreduce_max(np.array([1.0, 3.0])), np.array([1.0, 3.0], np.float32))
