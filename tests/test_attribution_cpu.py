"""The end-to-end attribution (tests/attribution.py) on the CPU.

A stand-in for a float32 implementation is built from the oracle's own steps:
every plane and map is rounded to float32, and each level's search reads its
planes with one float32 rounding of noise, so its decisions differ from the
oracle's where, and only where, float32 resolution decides them. The
attribution must explain all of its differences; and when a mistake is
planted in it (a wrong D*, a dropped patch that should be kept, a wrong dense
value), the attribution must fail.
"""
import numpy as np
import pytest

import attribution as at
import synth

CFG1_KW = dict(patch_size=8, overlap=0.5, iterations=8, coarsest_scale=2, finest_scale=0,
               gamma=0.25)
SMALL_CFG2_KW = dict(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=3,
                     finest_scale=0, gamma=0.5)


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def stand_in(orc, left, right, op, plant=None, seed=7):
    """Per-level intermediates of the float32 stand-in (module docstring),
    optionally with a planted mistake."""
    rng = np.random.default_rng(seed)
    top, fin = op.coarsest_scale, op.finest_scale
    Ls, Rs = [f32(left)], [f32(right)]
    for _ in range(top):
        Ls.append(f32(orc.downsample(Ls[-1])))
        Rs.append(f32(orc.downsample(Rs[-1])))
    levels, coarse = {}, None
    for lvl in range(top, fin - 1, -1):
        L, R = Ls[lvl], Rs[lvl]
        G = f32(orc.sobel_x(L))
        Ln = L * (1 + rng.uniform(-6e-8, 6e-8, L.shape))
        Rn = R * (1 + rng.uniform(-6e-8, 6e-8, R.shape))
        s = orc.search_level(Ln, Rn, G, coarse, op)
        s = {k: (f32(v) if v.dtype == np.float64 else v) for k, v in s.items()}
        if plant is not None and plant[0] == lvl:
            s = plant[1](s)
        dense = f32(orc.densify_level(L.shape, op, s["d_star"], s["weight"], coarse, lvl == fin,
                                      L, R))
        if plant is not None and plant[0] == lvl and len(plant) > 2:
            dense = plant[2](dense)
        levels[lvl] = dict(L=L, R=R, G=G, coarse=coarse, carry=coarse, dense=dense, **s)
        coarse = dense
    return levels, coarse


def firmly_kept(s, n):
    """n patches kept far from every threshold (saddle margin large, D* not
    near a column boundary, well inside the search range)."""
    ok = ((s["flags"] & at.DROP) == 0) & (s["weight"] > 0.05)
    frac = s["d_star"] - np.floor(s["d_star"])
    ok &= (np.minimum(frac, 1 - frac) > 0.1) & (np.abs(s["d_star"] - s["u_init"]) < 4)
    idx = np.argwhere(ok)
    return [tuple(i) for i in idx[len(idx) // 3:len(idx) // 3 + n]]


@pytest.mark.parametrize("which", ["cfg1", "cfg2_small"])
def test_float32_stand_in_is_fully_explained(orc, which):
    if which == "cfg1":
        pair, kw = synth.make_cfg1(), CFG1_KW
    else:
        pair, kw = synth.make_cfg2(seed=synth.stereo.pair_seed(2, 1), h=240, w=320), \
            SMALL_CFG2_KW
    op = orc.OracleParams.make(**kw)
    levels, out = stand_in(orc, pair.left, pair.right, op)
    o_st = orc.match_stages(pair.left, pair.right, op)
    rep = at.explain_e2e(orc, op, o_st, levels, out, which)
    tr = rep["trace"]
    for lvl, c in tr["by_level"].items():
        assert c["pixels"] == (c["stage"] + c["oracle_sensitivity"] + c["inherited"]
                               + c["within_tolerance"]), (lvl, c)
    assert rep["e2e"]["frac_within_fine"] >= 0.999, rep


def test_planted_wrong_dstar_is_not_explained(orc):
    pair = synth.make_cfg1()
    op = orc.OracleParams.make(**CFG1_KW)

    def plant(s):
        s = {k: v.copy() for k, v in s.items()}
        for j, i in firmly_kept(s, 3):
            s["d_star"][j, i] += 0.05
        return s

    levels, out = stand_in(orc, pair.left, pair.right, op, plant=(0, plant))
    o_st = orc.match_stages(pair.left, pair.right, op)
    with pytest.raises(AssertionError, match="patch differences not explained"):
        at.explain_e2e(orc, op, o_st, levels, out, "planted D*")


def test_planted_dropped_patch_is_not_explained(orc):
    pair = synth.make_cfg1()
    op = orc.OracleParams.make(**CFG1_KW)

    def plant(s):
        s = {k: v.copy() for k, v in s.items()}
        for j, i in firmly_kept(s, 2):
            s["flags"][j, i] |= 4  # a saddle the energies do not show
            s["weight"][j, i] = 0.0
        return s

    levels, out = stand_in(orc, pair.left, pair.right, op, plant=(1, plant))
    o_st = orc.match_stages(pair.left, pair.right, op)
    with pytest.raises(AssertionError, match="patch differences not explained"):
        at.explain_e2e(orc, op, o_st, levels, out, "planted drop")


def test_planted_wrong_dense_value_is_not_explained(orc):
    pair = synth.make_cfg1()
    op = orc.OracleParams.make(**CFG1_KW)

    def dense_bug(d):
        d = d.copy()
        d[30, 40] += 0.01
        return d

    levels, out = stand_in(orc, pair.left, pair.right, op, plant=(1, lambda s: s, dense_bug))
    o_st = orc.match_stages(pair.left, pair.right, op)
    with pytest.raises(AssertionError, match="densify differs"):
        at.explain_e2e(orc, op, o_st, levels, out, "planted dense")


def test_planted_search_bias_is_not_explained(orc):
    """A systematic error in every level-0 patch (D* off by 2e-3 px, twice the
    per-patch bar), too small to move many pixels beyond 0.05 px, still fails."""
    pair = synth.make_cfg1()
    op = orc.OracleParams.make(**CFG1_KW)

    def plant(s):
        s = {k: v.copy() for k, v in s.items()}
        s["d_star"] = s["d_star"] + 2e-3
        return s

    levels, out = stand_in(orc, pair.left, pair.right, op, plant=(0, plant))
    o_st = orc.match_stages(pair.left, pair.right, op)
    with pytest.raises(AssertionError):
        at.explain_e2e(orc, op, o_st, levels, out, "planted bias")


def test_covered_by_matches_brute_force(orc):
    rng = np.random.default_rng(3)
    for (h, w, ps, ov) in [(30, 41, 8, 0.75), (17, 23, 5, 0.4), (40, 40, 8, 0.5)]:
        ry = at.covering_ranges(orc, h, ps, ov)
        rx = at.covering_ranges(orc, w, ps, ov)
        oy, ox = orc.grid_origins(h, ps, ov), orc.grid_origins(w, ps, ov)
        mask = rng.uniform(size=(len(oy), len(ox))) < 0.1
        got = at.covered_by(mask, ry, rx)
        want = np.zeros((h, w), dtype=bool)
        for j, y0 in enumerate(oy):
            for i, x0 in enumerate(ox):
                if mask[j, i]:
                    want[y0:y0 + ps, x0:x0 + ps] = True
        assert np.array_equal(got, want)


def test_posterior_slope_matches_the_closed_form(orc):
    """On the exactly quadratic energies of a linear texture, E_i = C (d_i +
    e)^2 around a patch whose D* is off by e, the first-order slope of the
    posterior equals the derivative of its closed form."""
    op = orc.OracleParams.make()
    kappa = 2 * op.sigma_r ** 2 * op.window_samples ** 2
    offs = np.array([-1.0, -0.5, 0.0, 0.5, 1.0])

    def post(C, e):
        E = C * (offs + e) ** 2
        z = np.exp(-(E - E.min()) / kappa)
        return z[2] / z.sum()

    for C, e in [(50.0, 0.2), (400.0, -0.1), (2000.0, 0.05)]:
        o = {"energies": (C * (offs + e) ** 2)[None, None, :]}
        got = at.posterior_slope(o, op)[0, 0]
        h = 1e-6
        want = abs(post(C, e + h) - post(C, e - h)) / (2 * h)
        assert abs(got - want) <= 1e-6 + 1e-6 * want, (C, e, got, want)
