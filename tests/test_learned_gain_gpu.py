"""What the trained proposal network gains over the method without it.

On held-out surgical-like 640x480 pairs (seeds the training never saw), the
learned start (committed weights, fallback on) must not be worse than the
plain start at the paper's 12 iterations (bad-1 within 0.1 point), and with
fewer iterations (5) it must keep clearly more pixels within 1 px than the
plain start run with the same iterations, with a lower mean error: the
better coarse start is what lets the refinement stop earlier.
"""
import os

import numpy as np
import pytest
import torch

import paper_2106_07136_gb300 as bd
import synth

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(bd.__file__), "weights", "proposal.bdisnet")


@pytest.fixture(scope="module")
def held_out():
    L, R, D = synth.make_batch(2, 8, first_index=200)
    return torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), D


def test_weights_file_is_valid():
    w, note = bd.load_net_weights(WEIGHTS)
    assert w.size == bd.net_weight_count() and np.all(np.isfinite(w))
    assert "50000" in note
    level = bd.proposal_level(bd.default_params().coarsest_scale)
    assert f"level-{level} ground truth" in note  # trained on the level it runs on


def test_learned_start_gains_over_plain(held_out):
    L, R, D = held_out
    w, _ = bd.load_net_weights(WEIGHTS)
    net = bd.ProposalNet(w)
    m = bd.Matcher()
    stats = {}
    for it in (12, 5):
        p = bd.default_params(iterations=it)
        plain = synth.error_stats(m.match(L, R, p).cpu().numpy(), D)
        learned = synth.error_stats(m.match_learned(net, L, R, p, fallback=True).cpu().numpy(), D)
        stats[it] = (plain, learned)
    p12, l12 = stats[12]
    assert l12["bad1"] <= p12["bad1"] + 0.001, stats
    p5, l5 = stats[5]
    assert l5["bad1"] < p5["bad1"] - 0.003, stats
    assert l5["mean_abs"] < p5["mean_abs"], stats
    # and at 5 iterations the learned start is as good as the plain start at 12
    assert l5["bad1"] <= p12["bad1"] + 0.001, stats
    m.close()
    net.close()
