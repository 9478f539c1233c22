"""Run a whole workload through the C ABI: scene build -> sampling -> accumulation.

A workload is any object with `meshes` (each with vertices, indices, transform, object_id,
density), `fixations` (eye, gaze, duration_s, timestamp_s), `params` (theta_rad,
cutoff_sigmas, eps_rel, t_begin, t_end, window_s, normalize), `seed` and `session`.
Arrays are passed as they are: numpy arrays are host inputs, CUDA tensors device inputs.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Any, Optional

import numpy as np

from . import gazemap as G


@dataclass
class Handles:
    scene: Any
    samples: Any
    map: Any
    n_samples: int

    def free(self):
        if self.map:
            G.gm_map_free(self.map)
        if self.samples:
            G.gm_samples_free(self.samples)
        if self.scene:
            G.gm_scene_free(self.scene)
        self.map = self.samples = self.scene = None


def mesh_args(workload, to_device: bool = False):
    out = []
    for m in workload.meshes:
        v, f = np.ascontiguousarray(m.vertices, np.float32), np.ascontiguousarray(m.indices, np.uint32)
        if to_device:
            import torch
            v = torch.from_numpy(v).cuda()
            f = torch.from_numpy(f.view(np.int32)).cuda()
        out.append((v, f, m.transform, m.object_id))
    return out


def fixation_args(fixations, to_device: bool = False):
    arrs = [np.ascontiguousarray(fixations.eye, np.float32), np.ascontiguousarray(fixations.gaze, np.float32),
            np.ascontiguousarray(fixations.duration_s, np.float32),
            np.ascontiguousarray(fixations.timestamp_s, np.float64)]
    if to_device:
        import torch
        arrs = [torch.from_numpy(a).cuda() for a in arrs]
    return arrs


def n_windows(workload) -> int:
    """Maps a call makes: ceil((t_end - t_begin) / window_s) windows when window_s > 0, else one."""
    import math
    p = workload.params
    if p.window_s > 0:
        return max(1, int(math.ceil((p.t_end - p.t_begin) / p.window_s)))
    return 1


def params_of(workload, flags: int = 0, normalize: Optional[bool] = None, debug_pair_cap: int = 0):
    p = workload.params
    return G.make_params(p.theta_rad, p.cutoff_sigmas, p.eps_rel, p.t_begin, p.t_end, p.window_s,
                         p.normalize if normalize is None else normalize, flags, debug_pair_cap)


def run(ctx, workload, stream=None, flags: int = 0, normalize: Optional[bool] = None, debug_pair_cap: int = 0,
        device_inputs: bool = False, points=None, builder=None) -> Handles:
    """Build, sample (or take explicit `points` = (xyz f32, tri u32)) and accumulate."""
    scene = G.gm_build_scene(ctx, mesh_args(workload, device_inputs), stream, builder=builder)
    if points is None:
        samples = G.gm_sample_surface(scene, [m.density for m in workload.meshes], workload.seed, workload.session,
                                      stream)
    else:
        samples = G.gm_samples_from_points(scene, points[0], points[1], stream)
    eye, gaze, dur, ts = fixation_args(workload.fixations, device_inputs)
    prm = params_of(workload, flags, normalize, debug_pair_cap)
    m = G.gm_accumulate_fixations(scene, samples, eye, gaze, dur, ts, prm, stream)
    return Handles(scene, samples, m, G.gm_samples_info(samples))


def map_array(h: Handles, window: int = 0):
    out = np.empty(h.n_samples, np.float32)
    mx = G.gm_map_copy(h.map, window, out)
    return out, mx


def samples_arrays(h: Handles):
    n = h.n_samples
    xyz = np.empty((n, 3), np.float32)
    tri = np.empty(n, np.uint32)
    b2 = np.empty((n, 2), np.float32)
    obj = np.empty(n, np.uint32)
    G.gm_samples_copy(h.samples, xyz, tri, b2, obj)
    return xyz, tri, b2, obj
