"""The sample-sharded form of the path on several GPUs (one process per GPU).

Every rank holds the whole scene and every fixation and takes one contiguous slice of the stored
sample order. A sample's value depends on no other sample, so each slice's raw map is exactly
that part of the whole map. Normalisation (Section 3.2.3) divides by the maximum over all
samples: the ranks exchange one float per window (an all-reduce of the maximum) and divide their
slices by it. That maximum is the only data the ranks exchange.

Argument marshalling and orchestration only: the slice, the accumulation and the division run in
the library's kernels.
"""
from __future__ import annotations

from typing import Optional

import numpy as np


def sample_shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """[begin, end) of the stored sample order that `rank` of `world` takes (contiguous, disjoint,
    covering 0 .. n; sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("sample_shard: need 0 <= rank < world")
    return n * rank // world, n * (rank + 1) // world


def allreduce_max(x: np.ndarray, dist=None, device: str = "cpu") -> np.ndarray:
    """Element-wise maximum of `x` over all ranks (identity without torch.distributed)."""
    x = np.ascontiguousarray(x, np.float32)
    if dist is None:
        return x.copy()
    import torch
    t = torch.from_numpy(x.copy()).to(device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.cpu().numpy()


def accumulate_shard(ctx, w, rank: int, world: int, stream=None, flags: int = 0, meshes=None, fixations=None):
    """This rank's part of one map: the scene, the samples, this rank's slice of them and its raw
    (unnormalised) map. Returns (scene, slice, map, (begin, end), per-window raw maxima)."""
    from . import gazemap as G
    from . import pipeline
    scene = G.gm_build_scene(ctx, meshes if meshes is not None else pipeline.mesh_args(w), stream)
    full = G.gm_sample_surface(scene, [m.density for m in w.meshes], w.seed, w.session, stream)
    b, e = sample_shard(G.gm_samples_info(full), rank, world)
    part = G.gm_samples_slice(full, b, e, stream)
    G.gm_samples_free(full)
    fix = fixations if fixations is not None else pipeline.fixation_args(w.fixations)
    m = G.gm_accumulate_fixations(scene, part, *fix, pipeline.params_of(w, flags=flags, normalize=False), stream)
    W = pipeline.n_windows(w)
    mx = np.empty(W, np.float32)
    G.gm_map_max(m, mx, stream)
    return scene, part, m, (b, e), mx


def normalize_shard(m, global_max: np.ndarray, stream=None) -> None:
    """Divide this rank's slice by the maximum over all ranks."""
    from . import gazemap as G
    G.gm_map_normalize(m, np.ascontiguousarray(global_max, np.float32), stream)


def run_sharded(ctx, w, rank: int, world: int, dist=None, stream=None, flags: int = 0, device: str = "cpu",
                meshes=None, fixations=None):
    """The whole sharded step on this rank: its slice, the maximum exchange, the normalisation.
    Returns (scene, slice, map, (begin, end), global maxima); the caller frees the handles."""
    scene, part, m, rng, mx = accumulate_shard(ctx, w, rank, world, stream, flags, meshes, fixations)
    gmax = allreduce_max(mx, dist, device)
    normalize_shard(m, gmax, stream)
    return scene, part, m, rng, gmax
