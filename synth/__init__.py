"""Seeded synthetic inputs (meshes and fixations) shared by the oracle tests, the GPU tests and
the benchmark. Data only: nothing here performs the gaze-mapping computation."""
from .field_init import field_init
from .workloads import (Mesh, Fixations, Params, Workload, tiny_sphere, paper_scene, session, head_frames,
                        batched_sessions, city_block, flatten, identity, scale_translate)
