"""Explaining an implementation's end-to-end disparity against the FP64 oracle.

Test infrastructure (no GPU needed here): the GPU tests pass the kernels'
per-level intermediates, the CPU tests pass an oracle run with float32-rounded
intermediates, and, to show the checks bite, one with a planted mistake.

Coarse-to-fine inverse search is discontinuous at float32 resolution: at
basin boundaries, at the saddle-test ties and at the convergence thresholds
(Sec. 2.1-2.2), a change of an input in its last float32 bit can flip a
patch's keep/drop decision or send it to another basin, and the flip then
moves the finer levels' starts. So the two end-to-end maps are compared as
follows.

1. The oracle is run along the implementation's own trajectory: at every
   level it searches and densifies from the implementation's coarse map
   (the next coarser dense map, or the seed map at the coarsest level).
2. Stage check, every level: each patch of the implementation agrees with
   the oracle's patch on those same inputs (keep/drop decision equal, D*
   within 1e-3 px, weight within 2e-4), except where the difference is
   explained: the oracle's own decision margin is below what float32
   resolves, or the oracle's own result moves when its inputs get one
   float32 rounding of noise (`oracle_unstable`). The densification of the
   implementation's own patches agrees with the oracle's densification of
   the same patches to 1e-4 px, with the same NaN mask.
3. Dense check, every level: the implementation's dense map agrees with the
   oracle's map along the same trajectory within A_TOL, with the same NaN
   mask, at every pixel that no explained patch covers.
4. Trace (reported): every finest-level pixel that differs from the
   oracle's own end-to-end map by more than E2E_MAX px, or is estimated by
   one side only, is followed through the levels. Either a patch covering it
   is an explained stage difference ("stage"), or the oracle's own map moves
   there when its start changes by at most U_TOL px, float32-scale
   ("oracle sensitivity"), or its start moved by more and the covering
   patches' coarse support is followed to the next level ("inherited").

By induction over the levels, the implementation's map is then the oracle's
method applied with explained perturbations only; no pixel may stay
unexplained.
"""
from __future__ import annotations

import numpy as np

DROP = 2 | 4 | 8 | 16 | 32
FLAG_DIVERGED = 2
SADDLE_TAU = 1e-6
SAME_SOLUTION = 0.1  # px, R16

DSTAR_ATOL = 1e-3  # px, per-patch D* on the same inputs
POST_ATOL = 2e-4   # posterior and weight, on the same inputs
DENSE_ATOL = 1e-4  # px, densification of the same patches
# DIS fusion weighs each pixel by 1 / max(r^2, 1) with r = R(x - D*) - L(x):
# float32 rounding of the interpolated R (values up to 255, ulp 1.5e-5) moves
# r, hence the weights, by about 1e-5 relative where r is near 1, and a weight
# change moves the pixel by that times the spread of its patches' D* (a few
# px at a depth edge)
DENSE_ATOL_DIS = 5e-4
A_TOL = 2e-3       # px, dense maps along the same trajectory away from explained patches
U_TOL = 2e-3       # px, start difference below which a moved result is the oracle's own
E2E_FINE, E2E_MAX = 0.01, 0.05

FUSION_BDIS, FUSION_DIS = 0, 1


# ------------------------------------------------------------------ geometry

def covering_ranges(orc, n, ps, overlap):
    """Per pixel of an axis of n pixels, the first and last index of the
    patches whose extent [origin, origin + ps - 1] contains it."""
    o = np.asarray(orc.grid_origins(n, ps, overlap))
    p = np.arange(n)
    lo = np.searchsorted(o + ps - 1, p, side="left")
    hi = np.searchsorted(o, p, side="right") - 1
    return lo, hi


def covered_by(mask, ry, rx):
    """Per pixel: does any patch in `mask` (ny, nx) cover it."""
    ny, nx = mask.shape
    S = np.zeros((ny + 1, nx + 1), dtype=np.int64)
    S[1:, 1:] = np.cumsum(np.cumsum(mask.astype(np.int64), axis=0), axis=1)
    (ly, hy), (lx, hx) = ry, rx
    ok_y, ok_x = ly <= hy, lx <= hx
    ly, hy = np.clip(ly, 0, ny - 1), np.clip(hy, 0, ny - 1)
    lx, hx = np.clip(lx, 0, nx - 1), np.clip(hx, 0, nx - 1)
    cnt = (S[hy[:, None] + 1, hx[None, :] + 1] - S[ly[:, None], hx[None, :] + 1]
           - S[hy[:, None] + 1, lx[None, :]] + S[ly[:, None], lx[None, :]])
    return (cnt > 0) & ok_y[:, None] & ok_x[None, :]


def nan_aware_diff(a, b):
    """|a - b|, inf where exactly one is NaN, 0 where both are."""
    an, bn = np.isnan(a), np.isnan(b)
    d = np.abs(np.where(an | bn, 0.0, a - b))
    d[an != bn] = np.inf
    return d


# ------------------------------------------------ per-patch decisions

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


def oracle_unstable(orc, o, params, rel=1e-6, runs=2, with_steps=False):
    """Patches whose oracle result is itself ill-conditioned at float32 scale:
    when every value of the level's planes and of its coarse map is scaled by
    (1 + u), u uniform in [-rel, rel] (rel = 1e-6: about the rounding a
    float32 sum over a patch accumulates, 8 to 16 ulp), the keep/drop decision
    changes or D* moves by more than 1e-4 px. D* counts for dropped patches
    too: a patch whose trajectory moves at float32 scale (a wandering search
    in a textureless region) ends wherever rounding takes it, so its
    convergence and saddle decisions are not fixed by its inputs either. With
    DIS fusion the leave-the-range decision is the one that counts.

    with_steps: also return the patches whose update count (R12) moves by more
    than one under the same perturbation."""
    dis = params.fusion == FUSION_DIS
    dropped = ((o["flags"] & FLAG_DIVERGED) if dis else (o["flags"] & DROP)) != 0
    bad = np.zeros(dropped.shape, dtype=bool)
    step_bad = np.zeros(dropped.shape, dtype=bool)
    for seed in range(runs):
        rng = np.random.default_rng(100 + seed)
        L = o["L"] * (1 + rng.uniform(-rel, rel, o["L"].shape))
        R = o["R"] * (1 + rng.uniform(-rel, rel, o["R"].shape))
        c = o["coarse"]
        if c is not None:
            c = c * (1 + rng.uniform(-rel, rel, c.shape))
        p2 = orc.search_level(L, R, orc.sobel_x(L), c, params)
        d2 = ((p2["flags"] & FLAG_DIVERGED) if dis else (p2["flags"] & DROP)) != 0
        bad |= d2 != dropped
        fin2, fin = np.isfinite(p2["d_star"]), np.isfinite(o["d_star"])
        bad |= fin2 != fin
        bad |= fin2 & fin & (np.abs(np.where(fin2 & fin, p2["d_star"] - o["d_star"], 0.0))
                             > 1e-4)
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


def describe(o, g, bad, ps, n=4):
    """A few unexplained patches, with both sides' results and the oracle's
    decision margins, for the failure message."""
    out = []
    saddle, div, edge = decision_margins(o, ps) if "energies" in o else (None,) * 3
    for j, i in np.argwhere(bad)[:n]:
        d = {"patch": (int(j), int(i)), "flags": (int(o["flags"][j, i]), int(g["flags"][j, i])),
             "d_star": (float(o["d_star"][j, i]), float(g["d_star"][j, i])),
             "u_init": (float(o["u_init"][j, i]), float(g["u_init"][j, i])),
             "steps": (int(o["steps"][j, i]), int(g["steps"][j, i])),
             "weight": (float(o["weight"][j, i]), float(g["weight"][j, i]))}
        if saddle is not None:
            d["margins"] = (float(saddle[j, i]), float(div[j, i]), float(edge[j, i]))
        out.append(d)
    return out


def posterior_slope(o, params):
    """|dP/dD*| of each patch's posterior, to first order from its window
    energies: moving D* by e moves every window sample by e, so E_i changes
    by e E_i', with E_i' the slope of E along the window (finite differences
    of neighbouring samples), and P = exp(-E_c / kappa) / sum_i exp(-E_i /
    kappa) changes by (P / kappa) |E_c' - sum_i p_i E_i'|, p_i the softmax
    weights. Used where D* itself legitimately differs (within its bar)."""
    E = o["energies"]
    s = E.shape[-1]
    if s < 3:
        return np.zeros(E.shape[:-1])
    step = params.window_step if params.window_step > 0 else 1.0
    dE = np.gradient(E, step, axis=-1, edge_order=2)  # exact on quadratic E
    kappa = 2.0 * params.sigma_r ** 2 * s ** 2
    z = -(E - E.min(axis=-1, keepdims=True)) / kappa
    p = np.exp(z)
    p /= p.sum(axis=-1, keepdims=True)
    c = (s - 1) // 2
    return p[..., c] / kappa * np.abs(dE[..., c] - (p * dE).sum(axis=-1))


def explain_stage(orc, params, o, g, unstable=None):
    """One level's search, implementation `g` against the oracle's `o` on the
    same inputs (o carries L, R and coarse). Returns (explained, bad, info):
    explained marks the patches allowed to differ, bad the differences that
    nothing explains."""
    ps = params.patch_size
    if unstable is None:
        unstable = oracle_unstable(orc, o, params)
    gf = g["flags"].astype(np.int64)
    if params.fusion == FUSION_DIS:
        od, gd = (o["flags"] & FLAG_DIVERGED) != 0, (gf & FLAG_DIVERGED) != 0
        diff = od != gd
        _, div, _ = decision_margins(o, ps)
        ok = unstable | (div < 1e-3)
        same = ~diff & ~unstable
        dbad = same & (np.abs(g["d_star"] - o["d_star"]) > DSTAR_ATOL)
        explained = (diff & ok) | unstable
        bad = (diff & ~ok) | dbad
        return explained, bad, {"flag_diff": int(diff.sum()), "unstable": int(unstable.sum()),
                                "dstar_bad": int(dbad.sum()),
                                "unexplained": describe(o, g, bad, ps)}
    diff, ok = explained_flag_mismatch(o, gf, ps, unstable)
    kept = ~diff & ((o["flags"] & DROP) == 0) & ~unstable
    dd = np.abs(g["d_star"] - o["d_star"])
    dbad = kept & (dd > DSTAR_ATOL)
    # the posterior follows D*: where D* differs within its bar (e.g. one side
    # took one more update below the 1e-4 px stop), the weight may move by
    # twice its first-order slope times that difference
    wtol = POST_ATOL + 2.0 * posterior_slope(o, params) * np.where(kept, dd, 0.0)
    wbad = kept & (np.abs(g["weight"] - o["weight"]) > wtol)
    dropped = ~diff & ((o["flags"] & DROP) != 0)
    zbad = dropped & (g["weight"] != 0.0)
    # patches dropped on both sides reach no dense map: only the others count
    reach = ((o["flags"] & DROP) == 0) | ((gf & DROP) == 0)
    explained = (diff & ok) | (unstable & reach)
    bad = (diff & ~ok) | dbad | wbad | zbad
    return explained, bad, {"flag_diff": int(diff.sum()), "unstable": int(unstable.sum()),
                            "dstar_bad": int(dbad.sum()), "weight_bad": int(wbad.sum()),
                            "unexplained": describe(o, g, bad, ps)}


def explain_select(orc, params, og, g):
    """The coarsest level searched twice (R16): both searches as at
    explain_stage, then the per-patch choice. A choice that differs is
    explained where either search's result is, or where the oracle's choice
    sits within float32 resolution of its own thresholds (posteriors within
    2e-4, or |D*_a - D*_b| within 2e-3 px of the 0.1 px rule)."""
    oa = dict(og["seeded"], L=og["L"], R=og["R"], G=og["G"], coarse=og["coarse"])
    ob = dict(og["plain"], L=og["L"], R=og["R"], G=og["G"], coarse=None)
    ea, ba, ia = explain_stage(orc, params, oa, g["seeded"])
    eb, bb, ib = explain_stage(orc, params, ob, g["plain"])
    g_use = g["use_seed"]
    o_use = og["use_seed"]
    cdiff = g_use != o_use
    pmargin = np.abs(oa["posterior"] - ob["posterior"]) < POST_ATOL
    smargin = np.abs(np.abs(oa["d_star"] - ob["d_star"]) - SAME_SOLUTION) < 2 * DSTAR_ATOL
    cok = ea | eb | pmargin | smargin
    explained = ea | eb | (cdiff & cok)
    bad = ba | bb | (cdiff & ~cok)
    return explained, bad, {"seeded": ia, "plain": ib, "choice_diff": int(cdiff.sum())}


# ------------------------------------------------------------ end to end

def oracle_along(orc, params, g_levels):
    """The oracle's steps on the implementation's own inputs, level by level:
    its pyramid planes (L, R, G) and its coarse map (the next coarser dense
    map, or the seed map at the coarsest level). A level the implementation
    searched twice (it holds "use_seed") is searched twice here too, from the
    same seed map and from the plain start, then the R16 choice is made."""
    top, fin = params.coarsest_scale, params.finest_scale
    levels = {}
    for lvl in range(top, fin - 1, -1):
        g = g_levels[lvl]
        L, R, G = (np.asarray(g[k], dtype=np.float64) for k in ("L", "R", "G"))
        coarse = None if g["coarse"] is None else np.asarray(g["coarse"], dtype=np.float64)
        s = orc.search_level(L, R, G, coarse, params)
        carry = coarse
        extra = {}
        if "use_seed" in g:
            plain = orc.search_level(L, R, G, None, params)
            d, wt, use = orc.select_start(s, plain)
            extra = dict(seeded=dict(s), plain=plain, use_seed=use)
            s = dict(s, d_star=d, weight=wt)
            carry = None
        dense = orc.densify_level(L.shape, params, s["d_star"], s["weight"], carry, lvl == fin,
                                  L, R)
        levels[lvl] = dict(L=L, R=R, G=G, coarse=coarse, carry=carry, dense=dense, **s, **extra)
    return {"levels": levels}


def explain_e2e(orc, params, o_st, g_levels, g_out, label=""):
    """Stage and dense checks at every level plus the trace of the finest
    level's differences (module docstring). o_st: the oracle's own staged run
    (orc.match_stages); g_levels: the implementation's per-level
    intermediates (planes L, R, G; coarse; carry; search outputs with the
    debug ones; dense; at a level searched twice also seeded, plain and
    use_seed); g_out: its final map. Raises AssertionError on anything
    unexplained; returns the report."""
    ps, ov = params.patch_size, params.overlap
    top, fin = params.coarsest_scale, params.finest_scale
    og_st = oracle_along(orc, params, g_levels)
    rep = {"label": label, "levels": {}}
    ranges, explained_px = {}, {}
    problems = []
    for lvl in range(top, fin - 1, -1):
        og, g = og_st["levels"][lvl], g_levels[lvl]
        h, w = og["L"].shape
        ry = covering_ranges(orc, h, ps, ov)
        rx = covering_ranges(orc, w, ps, ov)
        ranges[lvl] = (ry, rx)
        if "use_seed" in og:
            ex, bad, info = explain_select(orc, params, og, g)
        else:
            ex, bad, info = explain_stage(orc, params, og, g)
        if bad.any():
            problems.append(f"level {lvl}: {int(bad.sum())} patch differences not explained "
                            f"{info} first at {np.argwhere(bad)[:4].tolist()}")
        # densification of the implementation's own patches, same inputs
        ref = orc.densify_level((h, w), params, g["d_star"], g["weight"], g["carry"],
                                lvl == fin, og["L"], og["R"])
        dd = nan_aware_diff(g["dense"], ref)
        tol = DENSE_ATOL_DIS if params.fusion == FUSION_DIS else DENSE_ATOL
        if (dd > tol).any():
            problems.append(f"level {lvl}: densify differs from the oracle's densify of the "
                            f"same patches at {int((dd > tol).sum())} pixels "
                            f"(max {float(dd[np.isfinite(dd)].max(initial=0))}, "
                            f"{int(np.isinf(dd).sum())} NaN flips)")
        # dense maps along the same trajectory. With DIS fusion the per-pixel
        # residual weight turns a within-tolerance D* difference into a larger
        # dense one where the image gradient is steep (its derivative is the
        # gradient over r^3), so there the patches and the densification of the
        # same patches, both checked above, are the whole check.
        cov = covered_by(ex, ry, rx)
        a = nan_aware_diff(g["dense"], og["dense"])
        un = (a > A_TOL) & ~cov
        if params.fusion == FUSION_DIS:
            un &= np.isinf(a)  # a pixel estimated by one side only still needs a patch
        if un.any():
            problems.append(f"level {lvl}: {int(un.sum())} pixels differ from the oracle on the "
                            f"same inputs beyond {A_TOL} px with no explained patch covering "
                            f"them, first at {np.argwhere(un)[:4].tolist()}")
        explained_px[lvl] = cov
        rep["levels"][lvl] = dict(info, explained_patches=int(ex.sum()),
                                  pixels_covered_by_explained=int(cov.sum()),
                                  max_dense_diff_unexplained=float(
                                      a[~cov & np.isfinite(a)].max(initial=0.0)))
    # final output (an upsample when the finest scale is above 0)
    if fin > 0:
        up = orc.upsample(g_levels[fin]["dense"], fin, g_out.shape)
        du = nan_aware_diff(g_out, up)
        if (du > DENSE_ATOL).any():
            problems.append(f"upsample differs at {int((du > DENSE_ATOL).sum())} pixels")
    if problems:
        raise AssertionError(f"{label}: " + "; ".join(problems))
    rep["trace"] = trace(orc, params, o_st, og_st, g_levels, ranges, explained_px)
    rep["e2e"] = e2e_report(g_out, o_st["out"])
    return rep


def trace(orc, params, o_st, og_st, g_levels, ranges, explained_px):
    """Classify each finest-level pixel beyond E2E_MAX (or with a NaN flip)
    against the oracle's own run, level by level (module docstring, 4)."""
    top, fin = params.coarsest_scale, params.finest_scale
    X = nan_aware_diff(g_levels[fin]["dense"], o_st["levels"][fin]["dense"]) > E2E_MAX
    out = {"pixels": int(X.sum()), "by_level": {}}
    for lvl in range(fin, top + 1):
        if not X.any():
            break
        g, og, o = g_levels[lvl], og_st["levels"][lvl], o_st["levels"][lvl]
        ry, rx = ranges[lvl]
        a = nan_aware_diff(g["dense"], og["dense"])
        b = nan_aware_diff(og["dense"], o["dense"])
        stage = X & (a > A_TOL)
        assert not (stage & ~explained_px[lvl]).any()  # the dense check holds everywhere
        # start differences of the patches: the two runs' coarse maps differ
        du = np.abs(og["u_init"] - o["u_init"])
        if "use_seed" in og:
            du = np.maximum(du, np.abs(og["seeded"]["u_init"] - o["seeded"]["u_init"]))
        big = du > U_TOL
        moved_start = covered_by(big, ry, rx)
        # carried pixels (no kept covering patch on one side) read the coarse map at x / 2
        carried = np.zeros_like(X)
        if lvl > fin and og["carry"] is not None and o["carry"] is not None:
            kept_o = covered_by(o["weight"] > 0, ry, rx)
            kept_og = covered_by(og["weight"] > 0, ry, rx)
            carried = ~(kept_o & kept_og)
        traj = X & (b > A_TOL) & ~stage
        inherited = traj & (moved_start | carried)
        sensitivity = traj & ~inherited
        small = X & ~stage & ~traj
        out["by_level"][lvl] = {"pixels": int(X.sum()), "stage": int(stage.sum()),
                                "oracle_sensitivity": int(sensitivity.sum()),
                                "inherited": int(inherited.sum()),
                                "within_tolerance": int(small.sum())}
        if lvl == top:
            # the coarsest level starts from identical (or seed) maps; a moved
            # start there can only come from the seed maps' own rounding
            out["by_level"][lvl]["seed_start_max_diff"] = float(du.max(initial=0.0))
            assert not inherited.any() or du.max(initial=0.0) <= 1e-3, out
            break
        # follow the inherited pixels to the coarse support at the next level
        nxt_shape = g_levels[lvl + 1]["dense"].shape
        ys, xs = np.nonzero(inherited)
        Xn = np.zeros(nxt_shape, dtype=bool)
        r = params.patch_size // 4 + 2
        for y, x in zip(ys // 2, xs // 2):
            Xn[max(0, y - r):y + r + 1, max(0, x - r):x + r + 1] = True
        gn, on = g_levels[lvl + 1]["dense"], o_st["levels"][lvl + 1]["dense"]
        X = Xn & (nan_aware_diff(gn, on) > U_TOL / 2)
    return out


def e2e_report(out, ref):
    g_nan, r_nan = np.isnan(out), np.isnan(ref)
    both = ~g_nan & ~r_nan
    err = np.abs(out[both] - ref[both])
    n = out.size
    within = int((err <= E2E_FINE).sum()) + int((g_nan & r_nan).sum())
    return {"pixels": n, "frac_within_fine": within / n,
            "max_err": float(err.max()) if err.size else 0.0,
            "mask_diff": int((g_nan != r_nan).sum()), "n_over_max": int((err > E2E_MAX).sum())}
