"""Shared helpers of the GPU parity tests: tolerances and comparisons.

Tolerances (float32 kernels against the float64 oracle):
  - pyramid planes and gradients: 2e-4 gray levels (values <= 255 after at
    most a few dozen float32 roundings);
  - per-patch D*: 1e-3 px; posterior and weight: 2e-4 absolute;
  - dense maps fed the same patches: 1e-4 px;
  - end to end: at least 99.9% of pixels within 0.01 px of the oracle (the
    method's stated bar); pixels off by more than 0.05 px, and pixels
    estimated by one side only, at most 0.1% each. Coarse-to-fine inverse
    search is discontinuous at float32 resolution (basin boundaries, the
    saddle and convergence thresholds): the FP64 oracle itself moves up to
    ~0.04% of pixels by more than 0.05 px when only its coarse-level
    disparities are rounded to float32 precision (test_oracle_pins:
    test_float32_scale_sensitivity_is_bounded), so "every pixel within
    0.05 px" cannot hold for any float32 implementation.
A per-patch decision (saddle, gamma, divergence) may differ only where the
oracle's own margin to the threshold is below what float32 can resolve.
"""
import numpy as np
import torch

PYR_ATOL = 2e-4
DSTAR_ATOL = 1e-3
POST_ATOL = 2e-4
DENSE_ATOL = 1e-4
E2E_FINE, E2E_FRAC, E2E_MAX, E2E_MASK = 0.01, 0.999, 0.05, 0.001

# Parameters and inputs of the end-to-end tests. Inputs held to the fixed bar
# above are pinned as well-conditioned at float32 scale in test_conditioning;
# ILL_CONDITIONED_PAIR is pinned as not, and its GPU test uses the oracle's
# own spread (assert_e2e_within_self_sensitivity) as the bar.
CFG1_KW = dict(patch_size=8, overlap=0.5, iterations=8, coarsest_scale=2, finest_scale=0,
               gamma=0.25)
CFG2_KW = dict(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=4, finest_scale=0,
               gamma=0.75)
PLAN_KW = dict(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=3, finest_scale=0,
               gamma=0.5)
SEEDED_PAIR = (2, 0)        # synth.make_pair arguments
WARM_STREAM = (5, 1)        # synth.stereo.pair_seed arguments of a VideoStream
ILL_CONDITIONED_PAIR = (2, 3)

SADDLE_TAU = 1e-6
DROP = 2 | 4 | 8 | 16 | 32


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def decision_margins(o, ps):
    """Oracle margins of each patch decision, relative to the quantity compared."""
    E = o["energies"]
    s = E.shape[-1]
    c = (s - 1) // 2
    Ec = E[..., c]
    others = np.delete(E, c, axis=-1)
    Eo = others.min(axis=-1) if others.shape[-1] else np.full(Ec.shape, np.inf)
    scale = np.maximum(Ec, 1.0)
    saddle = np.abs(Eo - (Ec - SADDLE_TAU * scale)) / scale
    div = np.abs(np.abs(o["d_star"] - o["u_init"]) - ps)
    frac = o["d_star"] - np.floor(o["d_star"])
    edge = np.minimum(frac, 1.0 - frac)  # distance of D* to a column boundary
    return saddle, div, edge


def oracle_unstable(orc, o, params, eps=1e-6, runs=2, with_steps=False):
    """Patches whose oracle result is itself ill-conditioned: the keep/drop
    decision changes, or D* moves by more than 1e-4 px, when the level's
    planes get eps gray levels of noise and its coarse disparities a relative
    perturbation of 1e-6 (one float32 rounding).

    with_steps: also return the patches whose update count (R12) moves by more
    than one under the same perturbation. Where the updates hover at the
    1e-4 px stop for several steps, when the patch stops is not fixed at
    float32 resolution even though D* is."""
    dropped = (o["flags"] & DROP) != 0
    bad = np.zeros(dropped.shape, dtype=bool)
    step_bad = np.zeros(dropped.shape, dtype=bool)
    for seed in range(runs):
        rng = np.random.default_rng(100 + seed)
        L = o["L"] + rng.normal(0, eps, o["L"].shape)
        R = o["R"] + rng.normal(0, eps, o["R"].shape)
        c = o["coarse"]
        if c is not None:
            c = c * (1 + rng.uniform(-1, 1, c.shape) * 1e-6)
        p2 = orc.search_level(L, R, orc.sobel_x(L), c, params)
        d2 = (p2["flags"] & DROP) != 0
        bad |= d2 != dropped
        bad |= ~dropped & ~d2 & (np.abs(p2["d_star"] - o["d_star"]) > 1e-4)
        step_bad |= np.abs(p2["steps"].astype(np.int64) - o["steps"]) > 1
    return (bad, step_bad) if with_steps else bad


def explained_flag_mismatch(o, g_flags, ps, unstable, tol=1e-4):
    """Patches kept by one side and dropped by the other; and whether each is
    explained by a near-zero oracle margin or an ill-conditioned oracle result."""
    od = (o["flags"] & DROP) != 0
    gd = (g_flags.astype(np.int64) & DROP) != 0
    diff = od != gd
    saddle, div, edge = decision_margins(o, ps)
    ok = unstable | (saddle < tol) | (div < 1e-3) | (edge < 1e-3)
    return diff, ok | ~diff


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


def assert_e2e(gpu, ref, label=""):
    r = e2e_report(gpu, ref)
    assert r["frac_within_fine"] >= E2E_FRAC, (label, r)
    assert r["mask_diff"] <= E2E_MASK * r["pixels"], (label, r)
    assert r["n_over_max"] <= E2E_MASK * r["pixels"], (label, r)
    return r


def assert_e2e_within_self_sensitivity(gpu, ref, orc, left, right, op, label=""):
    """For a method that is ill-conditioned at float32 resolution (DIS fusion
    keeps every patch, runaway and oscillating ones included): the kernels may
    differ from the FP64 oracle by no more than the oracle differs from itself
    when its coarse-level disparities carry one float32 rounding (the worse
    of two draws), with 1 point of margin on the 0.01 px share and 2x on the
    count of pixels beyond 0.05 px."""
    r = e2e_report(gpu, ref)
    selfs = [e2e_report(oracle_perturbed_match(orc, left, right, op, seed), ref)
             for seed in (1, 2)]
    frac_floor = min(x["frac_within_fine"] for x in selfs) - 0.01
    over_cap = 2 * max(x["n_over_max"] for x in selfs) + E2E_MASK * r["pixels"]
    mask_cap = 2 * max(x["mask_diff"] for x in selfs) + E2E_MASK * r["pixels"]
    assert r["frac_within_fine"] >= frac_floor, (label, r, selfs)
    assert r["n_over_max"] <= over_cap, (label, r, selfs)
    assert r["mask_diff"] <= mask_cap, (label, r, selfs)
    return r, selfs
