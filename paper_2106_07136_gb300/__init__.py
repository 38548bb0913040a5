"""BDIS (Bayesian Dense Inverse Search, arXiv 2106.07136) on GB300 / sm_103a.

The method runs in hand-written CUDA kernels behind the C ABI of
include/bdis.h (libbdis.so, built in-tree by `build.build()`); this package
only marshals arguments. There is no CPU fallback: without the CUDA library
every call raises.
"""
from .api import (  # noqa: F401
    Matcher,
    Plan,
    ProposalNet,
    net_init_weights,
    net_weight_count,
    load_net_weights,
    save_net_weights,
    default_params,
    densify_level,
    grid,
    image_desc,
    inject_alloc_failures,
    level_dims,
    match_static,
    pack_right,
    patch_count,
    probe_fp32_tflops,
    proposal_level,
    set_search_variant,
    get_search_variant,
    set_search_tiling,
    get_search_tiling,
    set_densify_variant,
    get_densify_variant,
    set_pyramid_variant,
    get_pyramid_variant,
    set_net_variant,
    get_net_variant,
    set_launch_overlap,
    get_launch_overlap,
    check_status,
    checked_build,
    prepare_level0,
    pyramid_level,
    search_level,
    select_start,
    upsample,
    warm_map,
)
from ._lib import ASYNC_SLOTS, BdisError, BdisParams, library_path, load  # noqa: F401
