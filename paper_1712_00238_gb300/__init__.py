"""GB300-native skeletal-density shape-complementarity scoring (sm_103a).

The compute path is libsdfdock.so (CUDA kernels behind the C ABI of
include/sdfdock.h); this package builds it in-tree and binds it with ctypes.
"""
from .sdfdock import (Context, Grid, SdError, Shape, SdfScore, decode_cands, load,  # noqa: F401
                      merge_top_k, refine_poses, sdf_score, shard_range)
