"""Shared helpers of the GPU parity tests: tolerances and comparisons.

Tolerances (float32 kernels against the float64 oracle):
  - pyramid planes and gradients: 2e-4 gray levels (values <= 255 after at
    most a few dozen float32 roundings);
  - per-patch D*: 1e-3 px; posterior and weight: 2e-4 absolute;
  - dense maps fed the same patches: 1e-4 px;
  - end to end (assert_explained): the map equals the step entry points'
    composition bit for bit, and every difference from the oracle is
    explained level by level (tests/attribution.py): a per-patch decision
    (saddle, gamma, divergence, convergence) may differ only where the
    oracle's own margin to the threshold is below what float32 resolves, or
    where the oracle's own result moves under one float32 rounding of its
    inputs; every other patch agrees to the bars above, and the dense maps
    along the same trajectory agree to 2e-3 px away from such patches. On
    inputs pinned well-conditioned (test_conditioning) at least 99.9% of the
    pixels also lie within 0.01 px of the oracle (the method's stated bar).
    Coarse-to-fine inverse search is discontinuous at float32 resolution
    (basin boundaries, the saddle and convergence thresholds): the FP64
    oracle itself moves pixels by more than 0.05 px when only its
    coarse-level disparities are rounded to float32 precision
    (test_oracle_pins: test_float32_scale_sensitivity_is_bounded), so "every
    pixel within 0.05 px" cannot hold for any float32 implementation; the
    attribution shows instead that each such pixel comes from a decision
    float32 cannot resolve.
"""
import numpy as np
import torch

import attribution as at

PYR_ATOL = 2e-4
DSTAR_ATOL = 1e-3
POST_ATOL = 2e-4
DENSE_ATOL = 1e-4
E2E_FINE, E2E_FRAC, E2E_MAX, E2E_MASK = 0.01, 0.999, 0.05, 0.001

# Parameters and inputs of the end-to-end tests. Inputs held to the 99.9% bar
# are pinned as well-conditioned at float32 scale in test_conditioning;
# ILL_CONDITIONED_PAIR is pinned as not, and its GPU test is held to the
# attribution alone.
CFG1_KW = dict(patch_size=8, overlap=0.5, iterations=8, coarsest_scale=2, finest_scale=0,
               gamma=0.25)
CFG2_KW = dict(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=4, finest_scale=0,
               gamma=0.75)
PLAN_KW = dict(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=3, finest_scale=0,
               gamma=0.5)
SEEDED_PAIR = (2, 0)        # synth.make_pair arguments
WARM_STREAM = (5, 1)        # synth.stereo.pair_seed arguments of a VideoStream
ILL_CONDITIONED_PAIR = (2, 3)

SADDLE_TAU = at.SADDLE_TAU
DROP = at.DROP
decision_margins = at.decision_margins
oracle_unstable = at.oracle_unstable
explained_flag_mismatch = at.explained_flag_mismatch


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def e2e_report(gpu, ref):
    g_nan, r_nan = np.isnan(gpu), np.isnan(ref)
    both = ~g_nan & ~r_nan
    err = np.abs(gpu[both] - ref[both])
    n = gpu.size
    mask_diff = int((g_nan != r_nan).sum())
    within = int((err <= E2E_FINE).sum()) + int((g_nan & r_nan).sum())
    return {
        "pixels": n,
        "frac_within_fine": within / n,
        "max_err": float(err.max()) if err.size else 0.0,
        "mask_diff": mask_diff,
        "n_over_max": int((err > E2E_MAX).sum()),
    }


def oracle_perturbed_match(orc, left, right, op, seed=None, rel=1e-6, prev=None):
    """The oracle's stages with the coarse-level disparity that seeds each finer
    level multiplied by (1 + u), u uniform in [-rel, rel] (one float32 rounding
    at rel = 1e-6); seed None = unperturbed. prev: a previous disparity to warm
    start from (R15), as at orc.match(prev=). Returns the finest dense map."""
    rng = None if seed is None else np.random.default_rng(seed)
    Ls, Rs = [np.asarray(left, np.float64)], [np.asarray(right, np.float64)]
    for _ in range(op.coarsest_scale):
        Ls.append(orc.downsample(Ls[-1]))
        Rs.append(orc.downsample(Rs[-1]))
    coarse = None if prev is None else orc.warm_map(prev, op.coarsest_scale + 1)
    for lvl in range(op.coarsest_scale, op.finest_scale - 1, -1):
        c = coarse
        if rng is not None and c is not None:
            c = c * (1 + rng.uniform(-1, 1, c.shape) * rel)
        s = orc.search_level(Ls[lvl], Rs[lvl], orc.sobel_x(Ls[lvl]), c, op)
        coarse = orc.densify_level(Ls[lvl].shape, op, s["d_star"], s["weight"], c,
                                   lvl == op.finest_scale, Ls[lvl], Rs[lvl])
    return coarse


def gpu_stages(left, right, gp, prev=None, seed=None, seed_level=0, fallback=False, net=None,
               variants=None):
    """The method on one pair through the library's step entry points (the
    kernels bdis_match and its variants launch), keeping every level's
    intermediates as host arrays: planes L, R (the value part of the packed
    plane), G; the coarse map the level started from; the map its uncovered
    pixels carry; the search outputs with the debug ones; the dense map. A
    start from prev (R15), a seed map (R16, with or without the fallback
    search) or the proposal network `net` (on level bd.proposal_level(top))
    seeds the coarsest
    level. variants: {level: columns per lane} (the search lane layout of each
    level; None = the process-wide choice). Returns (levels, final map)."""
    import paper_2106_07136_gb300 as bd
    top, fin = gp.coarsest_scale, gp.finest_scale
    dt = torch.uint8 if left.dtype == np.uint8 else torch.float32
    L, R, G = bd.prepare_level0(dev(left, dt), dev(right, dt))
    planes = [(L, R, G)]
    for _ in range(top):
        L, R, G = bd.pyramid_level(L, R)
        planes.append((L, R, G))
    coarse = None
    if prev is not None:
        coarse = bd.warm_map(dev(prev), top + 1)
    elif seed is not None:
        coarse = bd.warm_map(dev(seed), top + 1 - seed_level)
    levels = {}
    if net is not None:
        seed_level = bd.proposal_level(top)
        Ln, Rn, _ = planes[seed_level]
        prop = net.forward(Ln, Rn)
        levels["proposal"] = host(prop)[0]  # the network's map (not a level of the method)
        coarse = bd.warm_map(prop, top + 1 - seed_level)
    seeded = seed is not None or net is not None
    old = bd.get_search_variant()
    try:
        for lvl in range(top, fin - 1, -1):
            L, R, G = planes[lvl]
            if variants and variants.get(lvl):
                bd.set_search_variant(variants[lvl])
            s = bd.search_level(L, R, G, coarse, gp)
            bd.set_search_variant(old)
            carry = coarse
            extra = {}
            if seeded and fallback and lvl == top:
                plain = bd.search_level(L, R, G, None, gp)
                d, w = bd.select_start(s, plain)
                sh, ph = {k: host(v)[0] for k, v in s.items()}, \
                    {k: host(v)[0] for k, v in plain.items()}
                # where the choice kept the seeded result (equal results need no choice)
                use = ~((host(d)[0] == ph["d_star"]) & (host(w)[0] == ph["weight"])) | \
                    ((sh["d_star"] == ph["d_star"]) & (sh["weight"] == ph["weight"]))
                extra = dict(seeded=sh, plain=ph, use_seed=use)
                s = dict(s, d_star=d, weight=w)
                carry = None
            dense = bd.densify_level(tuple(L.shape[1:]), gp, s["d_star"], s["weight"], carry,
                                     lvl == fin, L, R)
            lv = {k: host(v)[0] for k, v in s.items()}
            lv.update(L=host(L)[0], R=host(R)[0][..., 0], G=host(G)[0],
                      coarse=None if coarse is None else host(coarse)[0],
                      carry=None if carry is None else host(carry)[0], dense=host(dense)[0],
                      **extra)
            levels[lvl] = lv
            coarse = dense
    finally:
        bd.set_search_variant(old)
    out = coarse if fin == 0 else bd.upsample(coarse, fin, tuple(planes[0][0].shape[1:]))
    return levels, host(out)[0]


def same_map(a, b):
    """Bit-identical maps, NaN masks included."""
    return np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(a[~np.isnan(a)],
                                                                       b[~np.isnan(b)])


def assert_explained(orc, out, left, right, gp, op, label="", budget=True, prev=None, seed=None,
                     seed_level=0, fallback=False, net=None, variants=None):
    """End-to-end parity of one pair's map `out` against the FP64 oracle.

    The map must be exactly what the library's step entry points compute for
    the same pair and start (gpu_stages), and every difference from the
    oracle's own end-to-end map must be explained level by level
    (attribution.explain_e2e): each patch difference by the oracle's own
    decision margin or its instability under one float32 rounding of its
    inputs, each dense difference by such a patch. With `budget`, also at
    least 99.9% of the pixels within 0.01 px of the oracle (the method's
    stated bar; inputs held to it are pinned well-conditioned in
    test_conditioning). Returns the attribution report."""
    levels, g_out = gpu_stages(left, right, gp, prev=prev, seed=seed, seed_level=seed_level,
                               fallback=fallback, net=net, variants=variants)
    assert same_map(np.asarray(out), g_out), (label, "entry point and step entry points differ")
    o_seed = seed
    if net is not None:
        import paper_2106_07136_gb300 as bd
        o_seed, seed_level = levels["proposal"], bd.proposal_level(gp.coarsest_scale)
    o_st = orc.match_stages(left, right, op, prev=prev, seed=o_seed, seed_level=seed_level,
                            fallback=fallback)
    rep = at.explain_e2e(orc, op, o_st, levels, g_out, label)
    if budget:
        assert rep["e2e"]["frac_within_fine"] >= E2E_FRAC, (label, rep)
    return rep
