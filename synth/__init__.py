"""Seeded synthetic stereo pairs with analytic ground truth.

This package builds inputs only. It holds none of the matcher's arithmetic, so
both the FP64 oracle and the CUDA path can be fed from it without sharing any
of the method's code.
"""
from .stereo import (  # noqa: F401
    StereoPair,
    make_pair,
    make_cfg1,
    make_cfg2,
    make_batch,
    make_linear_texture_pair,
    make_integer_shift_pair,
    make_flat_pair,
    SEED_BASE,
    VideoStream,
)
from .evaluate import error_stats  # noqa: F401
