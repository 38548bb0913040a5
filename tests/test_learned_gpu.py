"""Seeded and learned starts of the coarsest level (R16), GPU against the
oracle and against the plain path."""
import numpy as np
import pytest
import torch

import paper_2106_07136_gb300 as bd
import synth
from gpu_helpers import SEEDED_PAIR, assert_explained, dev, host

pytestmark = pytest.mark.gpu

CFG2 = dict(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=4, finest_scale=0,
            gamma=0.75)


@pytest.fixture(scope="module")
def pair():
    return synth.make_pair(*SEEDED_PAIR)  # well-conditioned; the seed changes its result


@pytest.fixture(scope="module")
def matcher():
    m = bd.Matcher()
    yield m
    m.close()


def level3_proposal(orc, pair):
    """A plausible level-3 proposal: the plain oracle's level-3 map, roughened."""
    op = orc.OracleParams.make(**CFG2)
    st = orc.match_stages(pair.left, pair.right, op)
    d3 = st["levels"][3]["dense"]
    rng = np.random.default_rng(0)
    return d3 + rng.normal(0, 0.3, d3.shape)


@pytest.mark.parametrize("fallback", [True, False])
def test_seeded_matches_oracle(orc, pair, matcher, fallback):
    gp, op = bd.default_params(**CFG2), orc.OracleParams.make(**CFG2)
    seed = level3_proposal(orc, pair)
    out = host(matcher.match_seeded(dev(pair.left, torch.uint8), dev(pair.right, torch.uint8),
                                    dev(seed), 3, gp, fallback=fallback))
    assert_explained(orc, out, pair.left, pair.right, gp, op, f"seeded fallback={fallback}",
                     seed=seed, seed_level=3, fallback=fallback)


def test_rejected_proposal_gives_the_plain_result(pair, matcher):
    gp = bd.default_params(**CFG2)
    L, R = dev(pair.left, torch.uint8), dev(pair.right, torch.uint8)
    plain = host(matcher.match(L, R, gp))
    seed = torch.full((1, 60, 80), 5000.0, device="cuda")
    out = host(matcher.match_seeded(L, R, seed, 3, gp, fallback=True))
    assert np.array_equal(np.isnan(out), np.isnan(plain))
    assert np.array_equal(out[np.isfinite(out)], plain[np.isfinite(plain)])


def test_missing_proposal_gives_the_plain_result(pair, matcher):
    """A proposal that is NaN everywhere (what the network's timeout path
    leaves in its bands) is missing, not wrong: the seed map is 0 there, the
    coarsest level starts as the plain method does, and the result is
    exactly the plain one, with or without the fallback search."""
    gp = bd.default_params(**CFG2)
    L, R = dev(pair.left, torch.uint8), dev(pair.right, torch.uint8)
    plain = host(matcher.match(L, R, gp))
    seed = torch.full((1, 60, 80), float("nan"), device="cuda")
    for fallback in (False, True):
        out = host(matcher.match_seeded(L, R, seed, 3, gp, fallback=fallback))
        assert np.array_equal(np.isnan(out), np.isnan(plain)), fallback
        assert np.array_equal(out[np.isfinite(out)], plain[np.isfinite(plain)]), fallback


def test_learned_start_equals_seeding_with_the_net_output(orc, pair, matcher):
    gp, op = bd.default_params(**CFG2), orc.OracleParams.make(**CFG2)
    net = bd.ProposalNet(bd.net_init_weights(seed=11))
    L, R = dev(pair.left, torch.uint8), dev(pair.right, torch.uint8)
    level = bd.proposal_level(gp.coarsest_scale)
    Lp, Rp, _ = bd.prepare_level0(L, R)
    for _ in range(level):
        Lp, Rp, _ = bd.pyramid_level(Lp, Rp)
    prop = net.forward(Lp, Rp)
    a = host(matcher.match_learned(net, L, R, gp, fallback=True))
    b = host(matcher.match_seeded(L, R, prop, level, gp, fallback=True))
    assert np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(a[np.isfinite(a)],
                                                                       b[np.isfinite(b)])
    assert_explained(orc, a, pair.left, pair.right, gp, op,
                     "learned vs oracle seeded with the same proposal", net=net, fallback=True)
    net.close()
