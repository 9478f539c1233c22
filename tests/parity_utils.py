"""Helpers shared by the GPU parity tests (comparison logic only; no method arithmetic)."""
import numpy as np

import oracle

# flipped visibilities allowed, as a fraction of the in-cone pairs
FLIP_BUDGET = 1e-4


def ulp32(x):
    return np.spacing(np.abs(np.asarray(x, np.float32))).astype(np.float64)


def tri_max_coord(tri, tri_idx):
    t = np.abs(tri[np.asarray(tri_idx, np.int64)].astype(np.float64))
    return t.max(axis=1)


def compare_pairs(gpu_pairs, ora_pairs, n_fix):
    """GPU in-cone pairs vs the oracle's record (in-cone or cone-edge pairs).

    Returns a dict of counts; raises AssertionError on any disagreement that the oracle does
    not mark as ambiguous."""
    gk = gpu_pairs["sample"].astype(np.int64) * n_fix + gpu_pairs["fix"].astype(np.int64)
    ok = ora_pairs["sample"].astype(np.int64) * n_fix + ora_pairs["fix"].astype(np.int64)
    assert len(np.unique(gk)) == len(gk), "GPU recorded a pair twice"
    fl = ora_pairs["flag"]
    o_in = (fl & oracle.PF_IN_CONE) > 0
    o_edge = (fl & oracle.PF_CONE_EDGE) > 0
    o_amb = (fl & oracle.PF_VIS_AMBIG) > 0
    o_vis = (fl & oracle.PF_VISIBLE) > 0
    # every GPU pair is known to the oracle (in cone, or at the cone edge)
    pos = np.searchsorted(ok, gk)
    pos = np.minimum(pos, len(ok) - 1)
    known = ok[pos] == gk
    assert known.all(), f"{(~known).sum()} GPU pairs are neither in the cone nor at its edge"
    # every oracle in-cone pair away from the edge was found by the GPU
    found = np.isin(ok, gk)
    must = o_in & ~o_edge
    assert found[must].all(), f"{(~found[must]).sum()} in-cone pairs missing on the GPU"
    # decisions that differ are at the cone edge only
    gin_here = found
    assert np.all((gin_here == o_in) | o_edge)
    # visibility equal where both saw the pair and the oracle calls it unambiguous
    gv = gpu_pairs["visible"][np.argsort(gk)]
    gks = np.sort(gk)
    both = np.nonzero(found)[0]
    gvis = gv[np.searchsorted(gks, ok[both])] > 0
    sure = ~o_amb[both]
    flips = (gvis != o_vis[both])
    assert not flips[sure].any(), f"{flips[sure].sum()} visibility flips on unambiguous pairs"
    # the flip budget: visibility decisions that differ (all of them on grazing pairs, by the
    # assertion above) stay within 1e-4 of the in-cone pairs
    n_in = int(o_in.sum())
    n_flip = int(flips[~sure].sum())
    assert n_flip <= FLIP_BUDGET * n_in, f"{n_flip} visibility flips among {n_in} in-cone pairs (budget {FLIP_BUDGET})"
    rep = dict(gpu=len(gk), oracle_in=n_in, edge=int(o_edge.sum()), ambiguous=int(o_amb.sum()),
               flips_ambiguous=n_flip, ambiguous_frac=float(o_amb.sum()) / max(1, n_in),
               flip_frac=n_flip / max(1, n_in))
    print("PARITY pairs " + " ".join(f"{k}={v:.3g}" if isinstance(v, float) else f"{k}={v}" for k, v in rep.items()))
    return rep
