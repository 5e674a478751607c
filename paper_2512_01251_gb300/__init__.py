"""GB300-native embedding of closed triangle meshes into forest-of-octrees grids.

The compute path is libemb.so (hand-written CUDA for sm_103a behind the C ABI in
include/emb.h); this package only marshals arguments to it.
"""
from .emb import (  # noqa: F401
    EMB_ERR_BAD_INPUT,
    EMB_ERR_CAPACITY,
    EMB_ERR_CUDA,
    EMB_ERR_NOT_WATERTIGHT,
    EMB_ERR_RANGE,
    EMB_ERR_STATE,
    EMB_ERR_TIMEOUT,
    EMB_OK,
    Embedding,
    EmbError,
    embed,
    emb_bin,
    emb_bins_copy,
    emb_bins_stats,
    emb_cutlinks,
    emb_cutlinks_backward,
    emb_cutlinks_count,
    emb_directions,
    emb_launch_count,
    emb_forest_blocks,
    emb_forest_masks,
    emb_forest_neighbors,
    emb_forest_num_blocks,
    emb_forest_refine,
    emb_forest_root,
    emb_mesh_create,
    emb_mex_force,
    emb_mex_force_backward,
    emb_mex_force_noalloc,
    emb_refine_flags,
    emb_status_get,
    emb_voxelize,
)
