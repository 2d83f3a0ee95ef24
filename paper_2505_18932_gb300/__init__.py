"""GB300 (sm_103a) geometry core of arXiv 2505.18932: temporal depth
refinement, image-based TSDF fusion and per-view forward splatting, as a
C-ABI CUDA library (libgvs.so) with a thin Python binding (`gvs`)."""
from . import gvs  # noqa: F401
from .gvs import (forward_splat, fuse_depth, gauss_splat, refine_depth, GvsError)  # noqa: F401
