"""Mixed-resolution batches in one CUDA graph (bdis_plan_*), GPU.

The plan must reproduce, for every pair of every group, exactly what the
library's step entry points compute with the lane layout the autotuner chose
for each level (other layouts change float rounding only), the oracle on a
sampled pair of each size with every difference explained, and identical
results on a second graph launch; refilled inputs must be picked up because
the graph binds buffers by address.
"""
import numpy as np
import pytest
import torch

import paper_2106_07136_gb300 as bd
import synth
from gpu_helpers import assert_explained, dev, gpu_stages, host, same_map

pytestmark = pytest.mark.gpu

KW = dict(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=3, finest_scale=0,
          gamma=0.5)
SIZES = [(2, 120, 160), (3, 61, 97), (1, 240, 320)]


def make_group(b, h, w, first):
    pairs = [synth.make_cfg2(seed=synth.stereo.pair_seed(3, first + i), h=h, w=w)
             for i in range(b)]
    L = dev(np.stack([p.left for p in pairs]), torch.uint8)
    R = dev(np.stack([p.right for p in pairs]), torch.uint8)
    return pairs, L, R, torch.empty((b, h, w), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("autotune", [True, False])
def test_plan_matches_per_group_calls_and_oracle(orc, autotune):
    params = bd.default_params(**KW)
    op = orc.OracleParams.make(**KW)
    groups, pairs = [], []
    first = 0
    for (b, h, w) in SIZES:
        pp, L, R, out = make_group(b, h, w, first)
        first += b
        groups.append((L, R, out))
        pairs.append(pp)
    plan = bd.Plan(groups, params, autotune=autotune)
    plan.run()
    torch.cuda.synchronize()
    first_run = [host(g[2]).copy() for g in groups]
    variants = []
    for gi, (L, R, out) in enumerate(groups):
        var = {lvl: plan.choice(gi, lvl)["search_columns_per_lane"] for lvl in plan.levels}
        variants.append(var)
        for b in range(L.shape[0]):
            _, g_out = gpu_stages(pairs[gi][b].left, pairs[gi][b].right, params, variants=var)
            assert same_map(first_run[gi][b], g_out), (gi, b)
        assert_explained(orc, first_run[gi][0], pairs[gi][0].left, pairs[gi][0].right, params,
                         op, f"group {gi} vs oracle", variants=var)
        if autotune:
            for lvl in plan.levels:
                ch = plan.choice(gi, lvl)
                assert ch["search_columns_per_lane"] in (1, 2, 4)
                assert ch["search_tiling"] in (0, 1)
                assert ch["search_block_threads"] in (64, 128)
                assert ch["densify_tile_height"] in (0, 8, 16, 32)  # 0: strip kernel
                assert ch["coarsest_scale"] == KW["coarsest_scale"]
    # second launch: identical
    plan.run()
    torch.cuda.synchronize()
    for gi, g in enumerate(groups):
        a, b = first_run[gi], host(g[2])
        assert np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(a[~np.isnan(a)],
                                                                           b[~np.isnan(b)])
    # refill the first group's inputs in place with another pair: the graph reads them
    pp, L2, R2, _ = make_group(*SIZES[0], first=50)
    groups[0][0].copy_(L2)
    groups[0][1].copy_(R2)
    plan.run()
    torch.cuda.synchronize()
    new = host(groups[0][2])
    assert_explained(orc, new[0], pp[0].left, pp[0].right, params, op, "refilled group",
                     variants=variants[0])
    plan.close()


def test_plan_scale_to_width():
    """BDIS_PLAN_SCALE_TO_WIDTH: a group's coarsest scale becomes the smallest
    c >= the plan's with 2^c >= width / 40, lowered while the coarsest level
    would be smaller than a patch; each group then computes exactly what
    bdis_match computes with that scale (no autotuning: the same kernels)."""
    params = bd.default_params(**KW)
    sizes = [(1, 160, 640), (2, 120, 160), (1, 140, 1300)]
    # 640: 2^4 * 40 >= 640 -> 4. 160: 2^2 * 40 >= 160 -> stays 3. 1300: 6, but
    # 140 rows are 3 at scale 6 and 5 at scale 5, 9 at scale 4 -> 4.
    expect = [4, 3, 4]
    groups = [make_group(b, h, w, 50 + 10 * i)[1:] for i, (b, h, w) in enumerate(sizes)]
    plan = bd.Plan(groups, params, autotune=False, scale_to_width=True)
    plan.run()
    torch.cuda.synchronize()
    m = bd.Matcher()
    for gi, (L, R, out) in enumerate(groups):
        c = plan.choice(gi, 0)["coarsest_scale"]
        assert c == expect[gi]
        ref = host(m.match(L, R, bd.default_params(**dict(KW, coarsest_scale=c))))
        got = host(out)
        assert np.array_equal(np.isnan(got), np.isnan(ref))
        assert np.array_equal(got[~np.isnan(got)], ref[~np.isnan(ref)])
    plan.close()


def test_plan_on_the_mixed_size_batch_sizes(orc):
    """One autotuned plan over one pair of each size of the mixed-size batch
    (320x240, 640x480, 1280x720, 1920x1080; disparity range a tenth of the
    width, 5 scales): each group is exactly the step entry points' result
    with the lane layouts the autotuner chose, and against the oracle every
    difference is explained (tests/attribution.py)."""
    kw = dict(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=4, finest_scale=0,
              gamma=0.75)
    params = bd.default_params(**kw)
    op = orc.OracleParams.make(**kw)
    sizes = [(240, 320), (480, 640), (720, 1280), (1080, 1920)]
    pairs = [synth.make_cfg2(seed=synth.stereo.pair_seed(3, 400 + i), h=h, w=w)
             for i, (h, w) in enumerate(sizes)]
    groups = [(dev(p.left, torch.uint8).unsqueeze(0), dev(p.right, torch.uint8).unsqueeze(0),
               torch.empty((1, h, w), dtype=torch.float32, device="cuda"))
              for p, (h, w) in zip(pairs, sizes)]
    plan = bd.Plan(groups, params, autotune=True)
    plan.run()
    torch.cuda.synchronize()
    for gi, (p, g) in enumerate(zip(pairs, groups)):
        var = {lvl: plan.choice(gi, lvl)["search_columns_per_lane"] for lvl in plan.levels}
        got = host(g[2])[0]
        _, g_out = gpu_stages(p.left, p.right, params, variants=var)
        assert same_map(got, g_out), gi
        assert_explained(orc, got, p.left, p.right, params, op, f"{sizes[gi]}", variants=var,
                         budget=False)
    plan.close()
