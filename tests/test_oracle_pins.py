"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Every test here checks the oracle against something other than itself: a
value printed in the paper, a closed form, a library routine that computes a
special case, brute force on a tiny input, or an invariant the paper states.
None needs a GPU.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import ndimage

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_params(orc, **kw):
    d = dict(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=2, finest_scale=0,
             gamma=0.25)
    d.update(kw)
    return orc.OracleParams.make(**d)


# ----------------------------------------------------------- paper values

def test_paper_parameters_are_the_defaults(orc):
    """Sec. 3 fixes sigma_r = sigma_s = 4, 5 window samples at 0.5 and 1 px,
    gamma 0.75 at 640x480."""
    g = json.load(open(os.path.join(GOLDEN, "paper_params.json")))
    p = orc.OracleParams.make()
    assert p.sigma_r == g["sigma_r"] and p.sigma_s == g["sigma_s"]
    assert p.window_samples == g["window_samples"]
    offs = sorted({abs((i - (p.window_samples - 1) // 2) * p.window_step)
                   for i in range(p.window_samples)} - {0.0})
    assert offs == g["window_offsets_px"]
    assert p.gamma == g["gamma"]["640x480"]


# --------------------------------------------------------------- geometry

def test_grid_counts_match_hand_worked_values(orc):
    g = json.load(open(os.path.join(GOLDEN, "grid_counts.json")))
    for case in g["cases"]:
        total = 0
        for lvl in range(case["levels"]):
            w = orc.level_dim(case["width"], lvl)
            h = orc.level_dim(case["height"], lvl)
            assert [w, h] == case["level_dims"][lvl]
            s = orc.grid_stride(case["patch"], case["overlap"])
            n = orc.grid_count(w, case["patch"], s) * orc.grid_count(h, case["patch"], s)
            assert n == case["patches"][lvl]
            total += n
        assert total == case["total"]


@pytest.mark.parametrize("n,ps,ov", [(40, 8, 0.75), (41, 8, 0.5), (33, 12, 0.75), (12, 12, 0.9),
                                     (17, 5, 0.0), (100, 7, 0.3)])
def test_grid_covers_every_pixel_with_regular_stride(orc, n, ps, ov):
    o = orc.grid_origins(n, ps, ov)
    s = orc.grid_stride(ps, ov)
    assert o[0] == 0 and o[-1] == n - ps
    assert np.all(np.diff(o) > 0) and np.all(np.diff(o) <= s)
    assert np.all(np.diff(o)[:-1] == s)
    cover = np.zeros(n, dtype=int)
    for x0 in o:
        cover[x0:x0 + ps] += 1
    assert cover.min() >= 1
    # one fewer origin would leave a gap: the count is minimal
    assert len(o) == 1 or (len(o) - 2) * s + ps < n


# ---------------------------------------------------------------- pyramid

def test_downsample_equals_separable_library_filter(orc):
    rng = np.random.default_rng(1)
    img = rng.uniform(0, 255, (37, 50))
    k = np.array([1, 4, 6, 4, 1]) / 16.0
    ref = ndimage.correlate1d(ndimage.correlate1d(img, k, axis=0, mode="mirror"), k, axis=1,
                              mode="mirror")[::2, ::2]
    np.testing.assert_allclose(orc.downsample(img), ref, rtol=0, atol=1e-10)


def test_downsample_polynomial_closed_forms(orc):
    h, w = 30, 41
    yy, xx = np.mgrid[0:h, 0:w].astype(float)
    lin = 0.7 * xx - 1.3 * yy + 5.0
    d = orc.downsample(lin)
    Y, X = np.mgrid[0:d.shape[0], 0:d.shape[1]].astype(float)
    inner = (slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(d[inner], (1.4 * X - 2.6 * Y + 5.0)[inner], atol=1e-12)
    # x^2 is even about x = 0, so reflect-101 keeps it exact at the left border:
    # the binomial adds its second moment (1) -> 4 X^2 + 1.
    q = orc.downsample(xx ** 2)
    np.testing.assert_allclose(q[:, :-2], (4 * X ** 2 + 1)[:, :-2], atol=1e-9)
    c = orc.downsample(np.full((h, w), 77.0))
    assert np.all(c == 77.0)


def test_sobel_equals_library_and_closed_forms(orc):
    rng = np.random.default_rng(2)
    img = rng.uniform(0, 255, (23, 31))
    ref = ndimage.sobel(img, axis=1, mode="mirror") / 8.0
    np.testing.assert_allclose(orc.sobel_x(img), ref, atol=1e-10)
    yy, xx = np.mgrid[0:20, 0:25].astype(float)
    g = orc.sobel_x(xx ** 2 + 3 * yy)
    np.testing.assert_allclose(g[:, :-1], 2 * xx[:, :-1], atol=1e-12)
    assert np.all(orc.sobel_x(yy ** 2) == 0.0)


# ------------------------------------------------------ inverse search, Eq. 1

@pytest.mark.parametrize("k", [1, 3, 5])
def test_integer_shift_recovered_exactly(orc, k):
    """R(x) = L(x + k) exactly: the true disparity zeroes every residual."""
    pair = synth.make_integer_shift_pair(48, 64, k)
    p = small_params(orc)
    st = orc.match_stages(pair.left, pair.right, p)
    out = st["out"]
    known = np.isfinite(pair.disp)
    est = np.isfinite(out) & known
    assert est.sum() > 0.95 * known.sum()
    assert np.max(np.abs(out[est] - k)) < 1e-3
    lv0 = st["levels"][0]
    kept = lv0["weight"] > 0
    e = lv0["energies"][kept]
    # E(D*) vanishes at the exact shift, up to the last step below the
    # convergence stop (1e-4 px): E(D*) / E(D* +- 1) ~ |D* - k|^2 < 1e-6
    assert np.all(e[:, 2] < 1e-6 * e.max(axis=1))
    assert np.all(e[:, 2] <= e.min(axis=1))


LIN_A0, LIN_A1 = 0.5, 2.0


@pytest.mark.parametrize("d", [0.25, 0.5, 2.37])
def test_linear_texture_subpixel_and_posterior_closed_form(orc, d):
    """L = a(y) x + b(y), R = L(x + d): linear interpolation is exact, so D* = d,
    E(D* + delta) = C delta^2 with C = sum over pixels of (a(y) - mean a)^2, and
    Eq. 3 with Eq. 4 gives P = 1 / sum_delta exp(-C delta^2 / (2 sigma_r^2 s^2))."""
    h, w = 48, 64
    pair = synth.make_linear_texture_pair(h, w, d, a0=LIN_A0, a1=LIN_A1, dtype=np.float64)
    left, right = pair.left, pair.right
    p = small_params(orc, iterations=20)
    st = orc.match_stages(left, right, p)
    out = st["out"]
    # pixels covered only by patches clear of the one-pixel border where the
    # reflected Sobel differs from a(y): there one Gauss-Newton step is exact
    inner = out[8:-8, 8:-8]
    assert np.all(np.isfinite(inner))
    assert np.max(np.abs(inner - d)) < 1e-3
    assert np.nanmax(np.abs(out - d)) < 0.25  # border patches converge more slowly

    lv0 = st["levels"][0]
    ps = p.patch_size
    xo = orc.grid_origins(w, ps, p.overlap)
    yo = orc.grid_origins(h, ps, p.overlap)
    kappa = 2 * p.sigma_r ** 2 * p.window_samples ** 2
    deltas = np.array([-1.0, -0.5, 0.0, 0.5, 1.0])
    checked = 0
    for j, y0 in enumerate(yo):
        for i, x0 in enumerate(xo):
            if x0 - d - 1 < 0 or x0 + ps - 1 - d + 1 > w - 1:
                continue  # not every pixel valid at every window sample
            if x0 < 1 or y0 < 1 or x0 + ps > w - 1 or y0 + ps > h - 1:
                continue  # touches the border row/column where g differs from a(y)
            a = LIN_A0 + LIN_A1 * (y0 + np.arange(ps))
            C = ps * np.sum((a - a.mean()) ** 2)
            ds = lv0["d_star"][j, i]
            np.testing.assert_allclose(ds, d, atol=1e-9)
            Ecl = C * (ds + deltas - d) ** 2  # closed form at the reached D*
            np.testing.assert_allclose(lv0["energies"][j, i], Ecl, rtol=1e-9, atol=1e-7)
            q = np.exp(-(Ecl - Ecl.min()) / kappa)
            P = q[2] / q.sum()
            np.testing.assert_allclose(P, 1.0 / np.sum(np.exp(-C * deltas ** 2 / kappa)),
                                       rtol=1e-5)
            np.testing.assert_allclose(lv0["posterior"][j, i], P, rtol=1e-9)
            np.testing.assert_allclose(lv0["weight"][j, i], P, rtol=1e-9)  # all 64 px valid
            checked += 1
    assert checked > 20


def test_fixed_point_matches_bisection_root(orc):
    """On a sub-pixel warp of smoothed noise the inverse search converges to
    the root of F(D) = sum g_n (R~_n(D) - T_n), found here by bisection."""
    pair = synth.make_cfg1()
    L = pair.left.astype(float)
    R = pair.right.astype(float)
    G = ndimage.sobel(L, axis=1, mode="mirror") / 8.0
    p = small_params(orc, iterations=50)
    ps = p.patch_size
    rng = np.random.default_rng(3)
    xs = np.arange(ps)

    def F(x0, y0, D):
        T = L[y0:y0 + ps, x0:x0 + ps]
        g = G[y0:y0 + ps, x0:x0 + ps]
        Rt = np.stack([np.interp(x0 + xs - D, np.arange(L.shape[1]), R[y0 + r])
                       for r in range(ps)])
        gn = g - g.mean()
        return np.sum(gn * ((Rt - Rt.mean()) - (T - T.mean())))

    done = 0
    for _ in range(60):
        x0 = int(rng.integers(20, L.shape[1] - ps - 2))
        y0 = int(rng.integers(2, L.shape[0] - ps - 2))
        d0 = pair.disp[y0 + ps // 2, x0 + ps // 2]
        if not np.isfinite(d0):
            continue
        res = orc.search_patch(L, R, G, x0, y0, d0 + 0.3, p)
        D = res.d_star
        lo, hi = D - 0.05, D + 0.05
        flo, fhi = F(x0, y0, lo), F(x0, y0, hi)
        if np.sign(flo) == np.sign(fhi):
            continue
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            fm = F(x0, y0, mid)
            if np.sign(fm) == np.sign(flo):
                lo, flo = mid, fm
            else:
                hi = mid
        assert abs(0.5 * (lo + hi) - D) < 1e-3
        done += 1
        if done >= 20:
            break
    assert done >= 10


def test_agrees_with_brute_force_integer_ssd(orc):
    """Tiny pair with a constant sub-pixel shift: each kept patch's D* lies
    within half a pixel of the integer minimiser of the normalised SSD."""
    rng = np.random.Generator(np.random.PCG64(11))
    h, w, d = 24, 40, 2.3
    tex = ndimage.gaussian_filter(rng.uniform(0, 255, (h, w + 8)), 1.5) * 3
    left = tex[:, :w]
    xg = np.arange(w)
    right = np.stack([np.interp(xg + d, np.arange(w + 8), tex[r]) for r in range(h)])
    p = small_params(orc, coarsest_scale=1, overlap=0.5)
    st = orc.match_stages(left, right, p)
    lv0 = st["levels"][0]
    ps = p.patch_size
    xo = orc.grid_origins(w, ps, p.overlap)
    yo = orc.grid_origins(h, ps, p.overlap)
    n = 0
    for j, y0 in enumerate(yo):
        for i, x0 in enumerate(xo):
            if x0 < 6 or lv0["weight"][j, i] <= 0:
                continue
            T = left[y0:y0 + ps, x0:x0 + ps]
            ssd = []
            for k in range(0, 6):
                Rk = right[y0:y0 + ps, x0 - k:x0 - k + ps]
                ssd.append(np.sum(((Rk - Rk.mean()) - (T - T.mean())) ** 2))
            kb = int(np.argmin(ssd))
            assert abs(lv0["d_star"][j, i] - kb) <= 0.5 + 1e-9
            assert abs(lv0["d_star"][j, i] - d) < 0.15
            n += 1
    assert n >= 4


def test_flat_texture_gives_uninformative_posterior(orc):
    """Fig. 2 / Sec. 2.2: on a textureless surface every candidate explains the
    pair equally, so the posterior over the 5-sample window is exactly 1/5."""
    pair = synth.make_flat_pair(48, 64)
    p = small_params(orc)
    st = orc.match_stages(pair.left, pair.right, p)
    for lvl, v in st["levels"].items():
        assert np.all(v["flags"] == orc.FLAG_FLAT)
        assert np.all(v["posterior"] == 0.2)
        assert np.all(v["d_star"] == 0.0)
    assert np.all(st["out"] == 0.0)


def test_patch_decisions_closed_form(orc):
    """Saddle, gamma and divergence rules on the linear texture, where every
    energy and every step is known in closed form."""
    h, w, d = 48, 64, 2.37
    yy, xx = np.mgrid[0:h, 0:w].astype(float)
    a = 0.5 + 2.0 * yy
    L = a * xx
    R = a * (xx + d)
    G = orc.sobel_x(L)
    # saddle: start 0.75 px off, no iteration -> E(D* - 0.5) < E(D*)
    p0 = small_params(orc, iterations=0)
    r = orc.search_patch(L, R, G, 20, 10, d + 0.75, p0)
    assert r.flags & orc.FLAG_SADDLE and r.weight == 0.0
    r = orc.search_patch(L, R, G, 20, 10, d + 0.2, p0)
    assert r.flags == 0 and r.weight > 0
    # gamma: a patch at the left border has columns x < d invalid at D* = d
    p1 = small_params(orc, iterations=3, gamma=0.75)
    r = orc.search_patch(L, R, G, 0, 10, d, p1)
    assert r.n_valid == 8 * 5 and (r.flags & orc.FLAG_GAMMA) and r.weight == 0.0
    p2 = small_params(orc, iterations=3, gamma=0.5)
    r = orc.search_patch(L, R, G, 0, 10, d, p2)
    assert not (r.flags & orc.FLAG_GAMMA)
    np.testing.assert_allclose(r.weight, r.posterior * 40 / 64, rtol=1e-12)
    # convergence: one exact Gauss-Newton step from 3 px off lands on d, but a
    # 3 px last step is not convergence; a second (zero) step is
    r = orc.search_patch(L, R, G, 20, 10, d + 3.0, small_params(orc, iterations=1))
    assert abs(r.d_star - d) < 1e-9 and (r.flags & orc.FLAG_UNCONVERGED) and r.weight == 0.0
    r = orc.search_patch(L, R, G, 20, 10, d + 3.0, small_params(orc, iterations=2))
    assert abs(r.d_star - d) < 1e-9 and r.flags == 0 and r.weight > 0
    # divergence: an exact Gauss-Newton step jumps 20 px, beyond the patch size
    R20 = a * (xx + 20.0)
    r = orc.search_patch(L, R20, G, 30, 10, 0.0, small_params(orc, iterations=1))
    assert abs(r.d_star - 20.0) < 1e-9 and (r.flags & orc.FLAG_DIVERGED)


# -------------------------------------------------------- densification

def _coverage(shape, ps, ov, weight, orc):
    h, w = shape
    xo = orc.grid_origins(w, ps, ov)
    yo = orc.grid_origins(h, ps, ov)
    cov = np.zeros(shape, dtype=bool)
    for j, y0 in enumerate(yo):
        for i, x0 in enumerate(xo):
            if weight[j, i] > 0:
                cov[y0:y0 + ps, x0:x0 + ps] = True
    return cov


def test_constant_field_is_preserved(orc):
    """Normalised weights (Eq. 2 form, Sec. 2.3): patches that all carry c give c."""
    h, w = 30, 44
    p = small_params(orc)
    xo = orc.grid_origins(w, 8, p.overlap)
    yo = orc.grid_origins(h, 8, p.overlap)
    rng = np.random.default_rng(5)
    weight = rng.uniform(0.05, 1.0, (len(yo), len(xo)))
    weight[rng.uniform(size=weight.shape) < 0.4] = 0.0
    dstar = np.full(weight.shape, 3.7)
    out = orc.densify_level((h, w), p, dstar, weight, None, True)
    cov = _coverage((h, w), 8, p.overlap, weight, orc)
    np.testing.assert_allclose(out[cov], 3.7, rtol=0, atol=1e-12)
    assert np.all(np.isnan(out[~cov]))
    coarse = np.full(((h + 1) // 2, (w + 1) // 2), 1.5)
    out2 = orc.densify_level((h, w), p, dstar, weight, coarse, False)
    np.testing.assert_allclose(out2[~cov], 3.0, atol=1e-12)  # carried from 2 x coarse


def test_two_patch_gaussian_mixture_closed_form(orc):
    """Two overlapping patches with D = 0 and 1: the fused value is a logistic
    of the difference of squared distances to the centres (Eq. 5), and does not
    depend on y because the centres share a row."""
    h, w = 8, 16
    p = small_params(orc, overlap=0.5)  # stride 4: origins 0, 4, 8
    weight = np.array([[0.6, 0.3, 0.0]])
    dstar = np.array([[0.0, 1.0, 5.0]])
    out = orc.densify_level((h, w), p, dstar, weight, None, True)
    s2 = 2 * p.sigma_s ** 2
    for x in range(4, 8):
        expect = 1.0 / (1.0 + (0.6 / 0.3) * math.exp(-(8 * x - 44) / s2))
        np.testing.assert_allclose(out[:, x], expect, rtol=1e-12)
    assert np.all(out[:, :4] == 0.0)
    np.testing.assert_allclose(out[:, 8:12], 1.0, atol=0)
    assert np.all(np.isnan(out[:, 12:]))


def test_patch_init_and_upsample_closed_forms(orc):
    yy, xx = np.mgrid[0:20, 0:30].astype(float)
    M = 0.3 * xx + 0.1 * yy
    # twice the coarse map at half the centre: alpha * cx + beta * cy
    for x0, y0 in [(4, 6), (10, 2), (20, 20)]:
        cx, cy = x0 + 3.5, y0 + 3.5
        assert abs(orc.patch_init(M, x0, y0, 8) - (0.3 * cx + 0.1 * cy)) < 1e-12
    assert orc.patch_init(None, 3, 3, 8) == 0.0
    up = orc.upsample(M, 1, (40, 60))
    Y, X = np.mgrid[0:40, 0:60].astype(float)
    np.testing.assert_allclose(up[:-2, :-2], (0.3 * X + 0.1 * Y)[:-2, :-2], atol=1e-12)
    Mn = M.copy()
    Mn[5, 7] = np.nan
    up = orc.upsample(Mn, 1, (40, 60))
    assert np.isnan(up[10, 14]) and np.isfinite(up[10, 15])


# ------------------------------------------------------------- end to end

def test_stagewise_equals_match(orc):
    pair = synth.make_cfg1()
    p = small_params(orc, overlap=0.5, iterations=8)
    a = orc.match(pair.left, pair.right, p)
    b = orc.match_stages(pair.left, pair.right, p)["out"]
    assert np.array_equal(np.isnan(a), np.isnan(b))
    assert np.array_equal(a[np.isfinite(a)], b[np.isfinite(b)])


def test_cfg1_accuracy_against_ground_truth(orc):
    """Not a pin of the arithmetic: a sanity bound that the restated method
    recovers the generator's field on the small textured pair."""
    pair = synth.make_cfg1()
    p = small_params(orc, overlap=0.5, iterations=8)
    st = synth.error_stats(orc.match(pair.left, pair.right, p), pair.disp)
    assert st["median_abs"] < 0.1 and st["bad1"] < 0.01


def test_well_posed_under_float32_sized_perturbations(orc):
    """The restated method must be a well-posed function of its inputs for a
    float32 implementation to be checkable against it: perturbing both views by
    1e-6 gray levels moves no pixel by more than 1e-3 px and flips no
    estimated/not-estimated decision (surgical-like 640x480 pair)."""
    pair = synth.make_cfg2()
    p = orc.OracleParams.make()
    a = orc.match(pair.left.astype(float), pair.right.astype(float), p)
    rng = np.random.default_rng(1)
    b = orc.match(pair.left + rng.normal(0, 1e-6, pair.shape),
                  pair.right + rng.normal(0, 1e-6, pair.shape), p)
    assert np.array_equal(np.isnan(a), np.isnan(b))
    assert np.nanmax(np.abs(a - b)) < 1e-3


def test_float32_scale_sensitivity_is_bounded(orc):
    """Coarse-to-fine inverse search is discontinuous at float32 resolution:
    rounding the coarse-level disparities that seed each finer level by one
    float32 ulp (relative 1e-6) moves some pixels of the FP64 result by more
    than 0.05 px (basin boundaries, saddle and convergence thresholds), but
    no more than 0.1% of them. This is why the float32 kernels are held to
    99.9% of pixels within 0.01 px and at most 0.1% beyond 0.05 px."""
    from gpu_helpers import oracle_perturbed_match
    pair = synth.make_cfg2()
    p = orc.OracleParams.make()
    a = oracle_perturbed_match(orc, pair.left, pair.right, p)
    assert np.array_equal(np.isnan(a), np.isnan(orc.match(pair.left, pair.right, p)))
    b = oracle_perturbed_match(orc, pair.left, pair.right, p, seed=1)
    both = np.isfinite(a) & np.isfinite(b)
    over = int((np.abs(a - b)[both] > 0.05).sum())
    flips = int((np.isnan(a) != np.isnan(b)).sum())
    assert 0 < over <= 1e-3 * a.size
    assert flips <= 1e-3 * a.size
    assert (np.abs(a - b)[both] <= 0.01).mean() >= 0.999


def test_bayesian_weighting_is_better_conditioned_than_dis(orc):
    """Sec. 2.2's point in numerical terms: with the posterior and the patch
    tests the estimate barely moves under float32-sized perturbations of the
    coarse levels; DIS fusion (Eq. 2), which keeps every patch, moves tens of
    times more pixels by more than 0.05 px."""
    from gpu_helpers import oracle_perturbed_match
    pair = synth.make_cfg2()
    over = {}
    for fusion in (orc.FUSION_BDIS, orc.FUSION_DIS):
        p = orc.OracleParams.make(fusion=fusion)
        a = oracle_perturbed_match(orc, pair.left, pair.right, p)
        b = oracle_perturbed_match(orc, pair.left, pair.right, p, seed=1)
        both = np.isfinite(a) & np.isfinite(b)
        over[fusion] = int((np.abs(a - b)[both] > 0.05).sum())
    assert over[orc.FUSION_DIS] > 10 * max(over[orc.FUSION_BDIS], 1)


def test_rejects_bad_arguments(orc):
    pair = synth.make_cfg1()
    for kw in [dict(window_samples=4), dict(overlap=1.0), dict(coarsest_scale=6),
               dict(finest_scale=3, coarsest_scale=2), dict(iterations=-1)]:
        with pytest.raises(ValueError):
            orc.match(pair.left, pair.right, small_params(orc, **kw))


# ------------------------------------------------------------ DIS mode, Eq. 2

def test_dis_fusion_closed_form_on_linear_texture(orc):
    """Eq. 2: each covering patch is weighted by 1 / max(r^2, 1) with r the
    photometric residual of its disparity at the pixel. On L = a(y) x + b(y),
    R = L(x + d), a patch at D = d + e has r = -a(y) e exactly."""
    h, w, d, e = 8, 16, 1.5, 0.3
    pair = synth.make_linear_texture_pair(h, w, d, a0=0.5, a1=2.0, dtype=np.float64)
    p = small_params(orc, overlap=0.5, fusion=orc.FUSION_DIS)  # origins 0, 4, 8
    weight = np.array([[1.0, 1.0, 0.0]])
    dstar = np.array([[d, d + e, 0.0]])
    out = orc.densify_level((h, w), p, dstar, weight, None, True, pair.left, pair.right)
    for y in range(h):
        a = 0.5 + 2.0 * y
        wb = 1.0 / max(a * a * e * e, 1.0)
        for x in range(4, 8):
            np.testing.assert_allclose(out[y, x], (d + wb * (d + e)) / (1.0 + wb), rtol=1e-12)
        assert np.all(np.isnan(out[y, :2]))  # x - d < 0: no valid sample, not estimated
        np.testing.assert_allclose(out[y, 2:4], d, rtol=1e-12)  # only the exact patch
        np.testing.assert_allclose(out[y, 8:12], d + e, rtol=1e-12)  # only the offset patch


@pytest.mark.parametrize("k", [1, 3])
def test_dis_integer_shift_recovered_exactly(orc, k):
    pair = synth.make_integer_shift_pair(48, 64, k)
    out = orc.match(pair.left, pair.right, small_params(orc, fusion=orc.FUSION_DIS))
    est = np.isfinite(out) & np.isfinite(pair.disp)
    assert est.sum() > 0.95 * np.isfinite(pair.disp).sum()
    assert np.max(np.abs(out[est] - k)) < 1e-3


def test_bdis_beats_dis_on_surgical_like_pair(orc):
    """The paper's comparison (Table 1): the Bayesian weighting lowers the
    error against DIS's residual fusion. On the surgical-like synthetic pair
    BDIS must have a lower mean absolute error and fewer bad-1 pixels among
    those it estimates."""
    pair = synth.make_cfg2()
    b = synth.error_stats(orc.match(pair.left, pair.right, orc.OracleParams.make()), pair.disp)
    dis = synth.error_stats(orc.match(pair.left, pair.right,
                                      orc.OracleParams.make(fusion=orc.FUSION_DIS)), pair.disp)
    assert b["mean_abs"] < dis["mean_abs"]
    assert b["median_abs"] < dis["median_abs"]
    assert dis["valid"] >= b["valid"]  # DIS estimates more pixels (Table 1's valid counts)


# ------------------------------------------------------- warm start (serving)

def test_warm_map_closed_forms(orc):
    """R15: block means of the finite previous disparities, divided by 2^level."""
    h, w = 50, 70
    yy, xx = np.mgrid[0:h, 0:w].astype(float)
    c = np.full((h, w), 6.4)
    m = orc.warm_map(c, 2)
    np.testing.assert_allclose(m, 6.4 / 4, rtol=1e-14)
    # a ramp in x: centred block means of x are the block centres (s X - 1/2)
    # away from the border, so the map is (4 X - 0.5) / 4 there
    m = orc.warm_map(xx, 2)
    X = np.arange(m.shape[1], dtype=float)
    expect = np.broadcast_to(((4 * X - 0.5) / 4)[1:-2], m[1:-1, 1:-2].shape)
    np.testing.assert_allclose(m[1:-1, 1:-2], expect, rtol=1e-12)
    nanblock = c.copy()
    nanblock[:, :] = np.nan
    assert np.all(orc.warm_map(nanblock, 3) == 0.0)  # nothing finite: cold start


def test_warm_start_from_truth_keeps_the_result(orc):
    """Seeding the coarsest level with the true previous disparity of an exact
    shift gives the same exact answer as the cold start."""
    k = 3
    pair = synth.make_integer_shift_pair(48, 64, k)
    p = small_params(orc)
    prev = np.full(pair.shape, float(k))
    out = orc.match(pair.left, pair.right, p, prev=prev)
    est = np.isfinite(out) & np.isfinite(pair.disp)
    assert est.sum() > 0.95 * np.isfinite(pair.disp).sum()
    assert np.max(np.abs(out[est] - k)) < 1e-3


def test_warm_start_reaches_beyond_the_cold_basin(orc):
    """A shift too large for the coarse-to-fine start from 0 (20 px with two
    scales: 5 px at the coarsest level, beyond its 8 px patches' reach after
    the divergence rule) is recovered when the previous frame seeds it."""
    k = 20
    pair = synth.make_integer_shift_pair(48, 96, k)
    p = small_params(orc, coarsest_scale=1, gamma=0.25)
    warm = orc.match(pair.left, pair.right, p, prev=np.full(pair.shape, k - 0.7))
    est = np.isfinite(warm) & np.isfinite(pair.disp)
    assert est.sum() > 0.9 * np.isfinite(pair.disp).sum()
    assert np.median(np.abs(warm[est] - k)) < 1e-3
    cold = orc.match(pair.left, pair.right, p)
    good_cold = np.isfinite(cold) & (np.abs(cold - k) < 1e-3)
    assert good_cold.sum() < 0.5 * est.sum()


# ----------------------------------------------------- early stop (R12)

def test_update_count_and_early_stop(orc):
    """R12: a patch takes at most `iterations` updates and stops after the
    first one below 1e-4 px. For a patch that took k < iterations updates:
    capping the search at k updates changes nothing, its k-th update is below
    1e-4 px and its (k-1)-th is not."""
    pair = synth.make_cfg1()
    p = small_params(orc)
    st = orc.match_stages(pair.left, pair.right, p)
    o = st["levels"][0]
    assert o["steps"].min() >= 0 and o["steps"].max() <= p.iterations
    assert np.all(o["steps"][(o["flags"] & 1) != 0] == 0)  # flat: no update
    early = np.argwhere((o["steps"] >= 2) & (o["steps"] < p.iterations) & (o["flags"] == 0))
    assert len(early) > 0.5 * o["steps"].size  # most patches converge before the cap
    h, w = o["L"].shape
    xs, ys = orc.grid_origins(w, p.patch_size, p.overlap), orc.grid_origins(h, p.patch_size,
                                                                           p.overlap)
    rng = np.random.default_rng(0)
    for j, i in early[rng.choice(len(early), 40, replace=False)]:
        k = int(o["steps"][j, i])
        u0 = o["u_init"][j, i]

        def run(n):
            q = small_params(orc, iterations=n)
            return orc.search_patch(o["L"], o["R"], o["G"], xs[i], ys[j], u0, q)
        full, at_k, at_k1, at_k2 = run(p.iterations), run(k), run(k - 1), run(k - 2)
        assert full.d_star == o["d_star"][j, i] and full.steps == k
        assert at_k.d_star == full.d_star and at_k.steps == k
        assert abs(at_k.d_star - at_k1.d_star) < 1e-4
        assert abs(at_k1.d_star - at_k2.d_star) >= 1e-4


def test_diverged_patch_reads_no_window(orc):
    """R8: a patch that leaves its search range (|D - u0| > patch size) is
    dropped as diverged; its window is not evaluated, so its posterior is 0
    and it carries no saddle or empty bit. A start 12 px off the true shift
    on a pair whose patches cannot lock on sends most patches away."""
    pair = synth.make_integer_shift_pair(48, 96, 20)
    p = small_params(orc, coarsest_scale=1, gamma=0.25)
    L, R = np.asarray(pair.left, np.float64), np.asarray(pair.right, np.float64)
    G = orc.sobel_x(L)
    res = orc.search_level(L, R, G, np.full((24, 48), 16.0), p)
    div = (res["flags"] & 2) != 0
    assert div.sum() > 0
    assert np.all(res["posterior"][div] == 0.0) and np.all(res["weight"][div] == 0.0)
    assert np.all((res["flags"][div] & (4 | 16)) == 0)
    assert np.all(res["energies"][div] == 0.0)


def test_zero_iterations_take_no_update(orc):
    pair = synth.make_cfg1()
    p = small_params(orc, iterations=0)
    o = orc.match_stages(pair.left, pair.right, p)["levels"][0]
    assert np.all(o["steps"] == 0) and np.array_equal(o["d_star"], o["u_init"])


# ------------------------------------------- proposal start with fallback (R16)

def test_seeded_without_fallback_is_the_warm_start(orc):
    pair = synth.make_cfg1()
    p = small_params(orc, overlap=0.5, iterations=8)
    prev = orc.match(pair.left, pair.right, p)
    a = orc.match(pair.left, pair.right, p, prev=prev)
    b = orc.match_seeded(pair.left, pair.right, p, prev, 0, fallback=False)
    assert np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(a[np.isfinite(a)],
                                                                       b[np.isfinite(b)])


def test_rejected_proposal_falls_back_to_the_plain_method(orc):
    """A proposal far outside the image (every seeded coarsest patch has no
    valid pixel and is dropped) gives exactly the plain result."""
    pair = synth.make_cfg1()
    p = small_params(orc, overlap=0.5, iterations=8)
    plain = orc.match(pair.left, pair.right, p)
    seed = np.full((orc.level_dim(120, 1), orc.level_dim(160, 1)), 500.0)
    out = orc.match_seeded(pair.left, pair.right, p, seed, 1, fallback=True)
    assert np.array_equal(np.isnan(out), np.isnan(plain))
    assert np.array_equal(out[np.isfinite(out)], plain[np.isfinite(plain)])


def test_proposal_that_reaches_the_plain_solution_gives_the_plain_result(orc):
    """A proposal near the plain method's own solution (its level-3 map plus
    0.3 px noise, 640x480) leads each coarsest patch to the solution the plain search
    finds. The seeded and plain results of such a patch agree to the 1e-4 px
    convergence stop and their posteriors to rounding, so the choice between
    them must not depend on the posteriors: the plain one stands, and the
    output equals the plain method's up to rounding. (Choosing by posterior
    there, the coarse D moves by up to ~1e-3 px and the output with it.)"""
    pair = synth.make_pair(2, 3)
    p = orc.OracleParams.make(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=4,
                              finest_scale=0, gamma=0.75)
    plain = orc.match(pair.left, pair.right, p)
    d = orc.match_stages(pair.left, pair.right, p)["levels"][3]["dense"]
    seed = d + np.random.default_rng(0).normal(0, 0.3, d.shape)
    out = orc.match_seeded(pair.left, pair.right, p, seed, 3, fallback=True)
    assert np.array_equal(np.isnan(out), np.isnan(plain))
    assert np.nanmax(np.abs(out - plain)) < 1e-5


def test_good_proposal_is_kept_where_the_plain_start_fails(orc):
    """A shift beyond the cold start's reach (as in the warm-start pin) is
    recovered from a proposal given at level 1, and the fallback keeps it."""
    k = 20
    pair = synth.make_integer_shift_pair(48, 96, k)
    p = small_params(orc, coarsest_scale=1, gamma=0.25)
    seed = np.full((orc.level_dim(48, 1), orc.level_dim(96, 1)), (k - 0.7) / 2.0)
    out = orc.match_seeded(pair.left, pair.right, p, seed, 1, fallback=True)
    est = np.isfinite(out) & np.isfinite(pair.disp)
    assert est.sum() > 0.9 * np.isfinite(pair.disp).sum()
    assert np.median(np.abs(out[est] - k)) < 1e-3


def test_stagewise_warm_and_seeded_equal_match(orc):
    """The staged run with a warm start (R15) or a seed map with and without
    the fallback search (R16) is exactly the oracle's whole-method entry."""
    pair = synth.make_cfg2(seed=synth.stereo.pair_seed(2, 9), h=120, w=160)
    p = orc.OracleParams.make(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=2,
                              gamma=0.5)
    prev = orc.match(pair.left, pair.right, p)
    a = orc.match_stages(pair.left, pair.right, p, prev=prev)["out"]
    b = orc.match(pair.left, pair.right, p, prev=prev)
    assert np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(a[~np.isnan(a)],
                                                                       b[~np.isnan(b)])
    seed = orc.match_stages(pair.left, pair.right, p)["levels"][1]["dense"] + 0.7
    for fb in (False, True):
        st = orc.match_stages(pair.left, pair.right, p, seed=seed, seed_level=1, fallback=fb)
        b = orc.match_seeded(pair.left, pair.right, p, seed, 1, fallback=fb)
        a = st["out"]
        assert np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(a[~np.isnan(a)],
                                                                           b[~np.isnan(b)])
        assert ("use_seed" in st["levels"][2]) == fb


def test_select_start_truth_table(orc):
    """R16's per-patch choice on hand-built cases: the seeded result a stands
    only if it is kept, is not within 0.1 px of a kept plain result b, and b
    is dropped or has no higher posterior."""
    # (a kept, b kept, d_a, d_b, p_a, p_b) -> keep a?
    cases = [
        (True, True, 3.0, 1.0, 0.5, 0.4, True),    # both kept, a more probable
        (True, True, 3.0, 1.0, 0.4, 0.4, True),    # tie keeps a
        (True, True, 3.0, 1.0, 0.3, 0.4, False),   # b more probable
        (True, False, 3.0, 1.0, 0.1, 0.9, True),   # b dropped
        (False, True, 3.0, 1.0, 0.9, 0.1, False),  # a dropped
        (False, False, 3.0, 1.0, 0.9, 0.1, False),  # both dropped: b's (zero) weight
        (True, True, 1.05, 1.0, 0.9, 0.1, False),  # one solution: the plain one
        (True, True, 1.09375, 1.0, 0.9, 0.1, False),  # within 0.1 px: one solution
        (True, True, 1.2, 1.0, 0.9, 0.1, True),
        (True, False, 1.05, 1.0, 0.9, 0.1, True),  # b dropped: no same-solution rule
    ]
    a = {k: np.array(v, dtype=np.float64) for k, v in
         {"d_star": [c[2] for c in cases], "posterior": [c[4] for c in cases],
          "weight": [10.0 + i for i in range(len(cases))]}.items()}
    a["flags"] = np.array([0 if c[0] else 4 for c in cases], dtype=np.int32)
    b = {k: np.array(v, dtype=np.float64) for k, v in
         {"d_star": [c[3] for c in cases], "posterior": [c[5] for c in cases],
          "weight": [20.0 + i for i in range(len(cases))]}.items()}
    b["flags"] = np.array([0 if c[1] else 8 for c in cases], dtype=np.int32)
    d, w, use = orc.select_start(a, b)
    want = np.array([c[6] for c in cases])
    assert np.array_equal(use, want)
    assert np.array_equal(d, np.where(want, a["d_star"], b["d_star"]))
    assert np.array_equal(w, np.where(want, a["weight"], b["weight"]))
