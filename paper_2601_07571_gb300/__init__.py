"""GB300 (sm_103a) surface-based gaze mapping: CUDA kernels behind the C ABI of
include/gazemap.h, with a thin ctypes binding (`gazemap`) and the in-tree build (`build`)."""
from . import build
from .gazemap import *  # noqa: F401,F403
from .gazemap import GazeMapError, lib
