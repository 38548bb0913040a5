"""FP64 CPU oracle of BDIS (arXiv 2106.07136).

TEST INFRASTRUCTURE ONLY: the plain restatement of the method that the CUDA
path is checked against. Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import it. It shares no code with the CUDA
library and never imports it.
"""
from .oracle import (  # noqa: F401
    OracleParams,
    build,
    load,
    level_dim,
    grid_stride,
    grid_count,
    grid_origin,
    grid_origins,
    downsample,
    sobel_x,
    search_patch,
    patch_init,
    search_level,
    densify_level,
    upsample,
    match,
    match_seeded,
    match_stages,
    select_start,
    warm_map,
    FLAG_FLAT,
    FLAG_DIVERGED,
    FLAG_SADDLE,
    FLAG_GAMMA,
    FLAG_EMPTY,
    FLAG_UNCONVERGED,
    DISCARD_FLAGS,
    FUSION_BDIS,
    FUSION_DIS,
)
