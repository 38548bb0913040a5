"""Conditioning of the end-to-end test inputs at float32 scale (R13).

Coarse-to-fine inverse search is discontinuous at float32 resolution (basin
boundaries, the saddle and gamma tests, the convergence thresholds), so how
far a float32 implementation may land from the FP64 oracle depends on the
input. The measure used here is how far the oracle lands from itself when the
coarse-level disparity that seeds each finer level carries one float32
rounding (relative 1e-6, several draws).

Every GPU end-to-end test explains each of its differences from the oracle
level by level (tests/attribution.py). Most inputs are also held to the
method's 99.9% bar (pixels within 0.01 px). That bar is only meaningful where
the oracle itself stays well inside it, so each such input is pinned here as
well-conditioned: in every draw, within the bar (99.9% within 0.01 px, at most
0.1% beyond 0.05 px or with a different mask). One ill-conditioned input is
pinned as such; its GPU test is held to the attribution alone.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import (CFG1_KW, CFG2_KW, E2E_FRAC, E2E_MASK, ILL_CONDITIONED_PAIR,
                         PLAN_KW, SEEDED_PAIR, WARM_STREAM, e2e_report, oracle_perturbed_match)

DRAWS = (1, 2, 3, 4)


def spread(orc, left, right, op, draws=DRAWS, prev=None):
    base = oracle_perturbed_match(orc, left, right, op, prev=prev)
    return [e2e_report(oracle_perturbed_match(orc, left, right, op, seed=d, prev=prev), base)
            for d in draws]


def assert_well_conditioned(reports, label):
    for r in reports:
        cap = E2E_MASK * r["pixels"]
        assert r["frac_within_fine"] >= E2E_FRAC, (label, r)
        assert r["n_over_max"] <= cap and r["mask_diff"] <= cap, (label, r)


def test_perturbed_match_reproduces_the_oracle(orc):
    """Unperturbed, the stage-by-stage helper is the oracle (cold and warm)."""
    pair = synth.make_cfg1()
    op = orc.OracleParams.make(**CFG1_KW)
    for prev in (None, orc.match(pair.left, pair.right, op)):
        a = oracle_perturbed_match(orc, pair.left, pair.right, op, prev=prev)
        b = orc.match(pair.left, pair.right, op, prev=prev)
        assert np.array_equal(np.isnan(a), np.isnan(b))
        assert np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)])


@pytest.mark.parametrize("name,pair,kw", [
    ("cfg1", lambda: synth.make_cfg1(), CFG1_KW),
    ("cfg2 ps8", lambda: synth.make_pair(*SEEDED_PAIR), CFG2_KW),
    ("cfg2 ps12", lambda: synth.make_pair(*SEEDED_PAIR), dict(CFG2_KW, patch_size=12)),
    ("cfg2 pair 5", lambda: synth.make_pair(2, 5), CFG2_KW),
    ("plan group 0", lambda: synth.make_cfg2(seed=synth.stereo.pair_seed(3, 0), h=120, w=160),
     PLAN_KW),
    ("plan group 1", lambda: synth.make_cfg2(seed=synth.stereo.pair_seed(3, 2), h=61, w=97),
     PLAN_KW),
    ("plan group 2", lambda: synth.make_cfg2(seed=synth.stereo.pair_seed(3, 5), h=240, w=320),
     PLAN_KW),
])
def test_end_to_end_inputs_are_well_conditioned(orc, name, pair, kw):
    p = pair()
    assert_well_conditioned(spread(orc, p.left, p.right, orc.OracleParams.make(**kw)), name)


def test_full_hd_input_is_well_conditioned(orc):
    p = synth.make_cfg2(seed=synth.stereo.pair_seed(3, 0), h=1080, w=1920)
    op = orc.OracleParams.make(**dict(CFG2_KW, coarsest_scale=5))
    assert_well_conditioned(spread(orc, p.left, p.right, op, draws=(1, 2)), "1920x1080")


def test_warm_start_stream_is_well_conditioned(orc):
    """Both frames of the warm-start test: frame 0 cold, frame 1 warm started
    from the oracle's frame-0 map."""
    op = orc.OracleParams.make(**PLAN_KW)
    v = synth.VideoStream(seed=synth.stereo.pair_seed(*WARM_STREAM), h=240, w=320)
    f0, f1 = v.next(), v.next()
    assert_well_conditioned(spread(orc, f0.left, f0.right, op), "frame 0")
    prev = orc.match(f0.left, f0.right, op)
    assert_well_conditioned(spread(orc, f1.left, f1.right, op, prev=prev), "frame 1 warm")


def test_ill_conditioned_pair_exceeds_the_fixed_bar(orc):
    """The pair whose GPU test is held to the attribution alone: one float32
    rounding of the oracle's own coarse maps already moves it past the fixed
    bar in some draw."""
    p = synth.make_pair(*ILL_CONDITIONED_PAIR)
    reps = spread(orc, p.left, p.right, orc.OracleParams.make(**CFG2_KW), draws=(0, 3, 5))
    worst = min(r["frac_within_fine"] for r in reps)
    assert worst < E2E_FRAC or max(r["n_over_max"] for r in reps) > E2E_MASK * reps[0]["pixels"]
