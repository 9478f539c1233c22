"""Write the per-sample export record of Section 3.3.3 (value, object, triangle, barycentrics,
mesh-local and world positions) to a .npz file. The record is assembled on the GPU by
gm_samples_export; this module only allocates the host arrays and writes the file."""
from __future__ import annotations

import numpy as np

from . import gazemap as G


def export_arrays(samples, m, window: int = 0):
    n = G.gm_samples_info(samples)
    rec = dict(value=np.empty(n, np.float32), object_id=np.empty(n, np.uint32), triangle=np.empty(n, np.uint32),
               bary3=np.empty((n, 3), np.float32), local_xyz=np.empty((n, 3), np.float32),
               world_xyz=np.empty((n, 3), np.float32))
    G.gm_samples_export(samples, m, window, **rec)
    return rec


def write_npz(path: str, samples, m, windows=None) -> None:
    """One record set per window (all windows by default), compressed .npz."""
    W, ns, _, _ = G.gm_map_info(m)
    wins = range(W) if windows is None else windows
    out = {}
    for k in wins:
        rec = export_arrays(samples, m, k)
        if not out:
            out.update({f: rec[f] for f in ("object_id", "triangle", "bary3", "local_xyz", "world_xyz")})
        out[f"value_w{k}"] = rec["value"]
    np.savez_compressed(path, **out)
