"""ctypes binding of the FP64 C oracle (bdis_oracle.c).

TEST INFRASTRUCTURE ONLY. Argument marshalling: every number is computed by
the C file. `build()` compiles it with the host gcc; `load()` builds on first
use if the library is missing or older than its source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bdis_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")

FLAG_FLAT = 1
FLAG_DIVERGED = 2
FLAG_SADDLE = 4
FLAG_GAMMA = 8
FLAG_EMPTY = 16
FLAG_UNCONVERGED = 32
FUSION_BDIS, FUSION_DIS = 0, 1
DISCARD_FLAGS = FLAG_DIVERGED | FLAG_SADDLE | FLAG_GAMMA | FLAG_EMPTY | FLAG_UNCONVERGED


class OracleParams(ctypes.Structure):
    """Mirror of orc_params. Defaults are the paper's settings (Sec. 3):
    sigma_r = sigma_s = 4, a window of 5 samples at 0.5 and 1 px, gamma 0.75
    at 640x480; patch 8 with overlap 0.75, 12 iterations, 5 scales."""

    _fields_ = [
        ("patch_size", ctypes.c_int),
        ("overlap", ctypes.c_double),
        ("iterations", ctypes.c_int),
        ("coarsest_scale", ctypes.c_int),
        ("finest_scale", ctypes.c_int),
        ("sigma_r", ctypes.c_double),
        ("sigma_s", ctypes.c_double),
        ("window_samples", ctypes.c_int),
        ("window_step", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("normalize", ctypes.c_int),
        ("fusion", ctypes.c_int),
    ]

    @classmethod
    def make(cls, **kw):
        d = dict(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=4, finest_scale=0,
                 sigma_r=4.0, sigma_s=4.0, window_samples=5, window_step=0.5, gamma=0.75,
                 normalize=1, fusion=FUSION_BDIS)
        d.update(kw)
        return cls(**d)

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile bdis_oracle.c into liborc.so next to it (plain -O2, no fast-math)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC,
           "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        pp = ctypes.POINTER(OracleParams)
        i = ctypes.c_int
        lib.orc_level_dim.argtypes = [i, i]
        lib.orc_grid_stride.argtypes = [i, ctypes.c_double]
        lib.orc_grid_count.argtypes = [i, i, i]
        lib.orc_grid_origin.argtypes = [i, i, i, i, i]
        lib.orc_downsample.argtypes = [dp, i, i, dp]
        lib.orc_sobel_x.argtypes = [dp, i, i, dp]
        lib.orc_patch_init.argtypes = [dp, i, i, i, i, i]
        lib.orc_patch_init.restype = ctypes.c_double
        lib.orc_search_patch.argtypes = [dp, dp, dp, i, i, i, i, ctypes.c_double, pp,
                                         ctypes.c_void_p, dp]
        lib.orc_search_level.argtypes = [dp, dp, dp, i, i, dp, i, i, pp, dp, dp, dp, dp, ip, ip,
                                         dp, ip]
        lib.orc_densify_level.argtypes = [i, i, pp, dp, dp, dp, i, i, i, dp, dp, dp]
        lib.orc_upsample.argtypes = [dp, i, i, i, i, i, dp]
        lib.orc_match.argtypes = [dp, dp, i, i, pp, dp]
        lib.orc_match_u8.argtypes = [ctypes.c_void_p, ctypes.c_void_p, i, i, pp, dp]
        lib.orc_match_warm.argtypes = [dp, dp, i, i, pp, dp, dp]
        lib.orc_warm_map.argtypes = [dp, i, i, i, dp]
        lib.orc_match_seeded.argtypes = [dp, dp, i, i, pp, dp, i, i, dp]
        lib.orc_select_start.argtypes = [i, dp, dp, dp, ip, dp, dp, dp, ip, ip]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def level_dim(n, level):
    return load().orc_level_dim(int(n), int(level))


def grid_stride(ps, overlap):
    return load().orc_grid_stride(int(ps), float(overlap))


def grid_count(n, ps, stride):
    return load().orc_grid_count(int(n), int(ps), int(stride))


def grid_origin(i, count, n, ps, stride):
    return load().orc_grid_origin(int(i), int(count), int(n), int(ps), int(stride))


def grid_origins(n, ps, overlap):
    s = grid_stride(ps, overlap)
    c = grid_count(n, ps, s)
    return np.array([grid_origin(i, c, n, ps, s) for i in range(c)], dtype=np.int64)


def downsample(img):
    img = _f64(img)
    h, w = img.shape
    out = np.empty(((h + 1) // 2, (w + 1) // 2))
    load().orc_downsample(_dp(img), w, h, _dp(out))
    return out


def sobel_x(img):
    img = _f64(img)
    h, w = img.shape
    out = np.empty_like(img)
    load().orc_sobel_x(_dp(img), w, h, _dp(out))
    return out


def patch_init(coarse, x0, y0, ps):
    if coarse is None:
        return load().orc_patch_init(None, 0, 0, int(x0), int(y0), int(ps))
    coarse = _f64(coarse)
    return load().orc_patch_init(_dp(coarse), coarse.shape[1], coarse.shape[0], int(x0), int(y0),
                                 int(ps))


class _PatchResult(ctypes.Structure):
    _fields_ = [("u_init", ctypes.c_double), ("d_star", ctypes.c_double),
                ("posterior", ctypes.c_double), ("weight", ctypes.c_double),
                ("flags", ctypes.c_int), ("n_valid", ctypes.c_int), ("steps", ctypes.c_int)]


@dataclass
class PatchResult:
    u_init: float
    d_star: float
    posterior: float
    weight: float
    flags: int
    n_valid: int
    energies: np.ndarray
    steps: int = 0  # updates applied to D (R12: at most `iterations`)


def search_patch(L, R, G, x0, y0, u_init, params: OracleParams) -> PatchResult:
    L, R, G = _f64(L), _f64(R), _f64(G)
    h, w = L.shape
    res = _PatchResult()
    e = np.zeros(params.window_samples)
    load().orc_search_patch(_dp(L), _dp(R), _dp(G), w, h, int(x0), int(y0), float(u_init),
                            ctypes.byref(params), ctypes.byref(res), _dp(e))
    return PatchResult(res.u_init, res.d_star, res.posterior, res.weight, res.flags, res.n_valid, e,
                       res.steps)


def search_level(L, R, G, coarse, params: OracleParams) -> dict:
    """All patches of one level; arrays shaped (ny, nx) (energies: (ny, nx, s))."""
    L, R, G = _f64(L), _f64(R), _f64(G)
    h, w = L.shape
    s = grid_stride(params.patch_size, params.overlap)
    nx, ny = grid_count(w, params.patch_size, s), grid_count(h, params.patch_size, s)
    out = {k: np.empty((ny, nx)) for k in ("u_init", "d_star", "posterior", "weight")}
    out["flags"] = np.empty((ny, nx), dtype=np.int32)
    out["n_valid"] = np.empty((ny, nx), dtype=np.int32)
    out["steps"] = np.empty((ny, nx), dtype=np.int32)
    out["energies"] = np.empty((ny, nx, params.window_samples))
    if coarse is None:
        cp, cw, ch = None, 0, 0
    else:
        coarse = _f64(coarse)
        cp, cw, ch = _dp(coarse), coarse.shape[1], coarse.shape[0]
    load().orc_search_level(_dp(L), _dp(R), _dp(G), w, h, cp, cw, ch, ctypes.byref(params),
                            _dp(out["u_init"]), _dp(out["d_star"]), _dp(out["posterior"]),
                            _dp(out["weight"]), _ip(out["flags"]), _ip(out["n_valid"]),
                            _dp(out["energies"]), _ip(out["steps"]))
    return out


def densify_level(shape, params: OracleParams, d_star, weight, coarse, is_finest, L=None,
                  R=None):
    """Dense map of one level; L and R (the level's planes) are needed for DIS fusion."""
    h, w = shape
    d_star, weight = _f64(d_star), _f64(weight)
    out = np.empty((h, w))
    if params.fusion == FUSION_DIS and (L is None or R is None):
        raise ValueError("DIS fusion needs the level's L and R planes")
    if coarse is None:
        cp, cw, ch = None, 0, 0
    else:
        coarse = _f64(coarse)
        cp, cw, ch = _dp(coarse), coarse.shape[1], coarse.shape[0]
    Lc = None if L is None else _f64(L)
    Rc = None if R is None else _f64(R)
    load().orc_densify_level(w, h, ctypes.byref(params), _dp(d_star), _dp(weight), cp, cw, ch,
                             int(bool(is_finest)), None if Lc is None else _dp(Lc),
                             None if Rc is None else _dp(Rc), _dp(out))
    return out


def upsample(M, f, shape):
    M = _f64(M)
    h, w = shape
    out = np.empty((h, w))
    load().orc_upsample(_dp(M), M.shape[1], M.shape[0], int(f), w, h, _dp(out))
    return out


def warm_map(prev, level):
    """R15: the level-`level` seed map made from a previous full-size disparity."""
    prev = _f64(prev)
    h, w = prev.shape
    out = np.empty((level_dim(h, level), level_dim(w, level)))
    load().orc_warm_map(_dp(prev), w, h, int(level), _dp(out))
    return out


def match(left, right, params: OracleParams, prev=None) -> np.ndarray:
    """Full method on one pair (uint8 or float images). Returns (H, W) float64, NaN = not
    estimated. `prev`: a previous disparity of the same scene to warm-start from (R15)."""
    h, w = left.shape
    out = np.empty((h, w))
    if prev is not None:
        lf, rf, pf = _f64(left), _f64(right), _f64(prev)
        rc_ = load().orc_match_warm(_dp(lf), _dp(rf), w, h, ctypes.byref(params), _dp(pf),
                                    _dp(out))
        if rc_ != 0:
            raise ValueError(f"oracle rejected the arguments (code {rc_})")
        return out
    if left.dtype == np.uint8 and right.dtype == np.uint8:
        lc = np.ascontiguousarray(left)
        rc = np.ascontiguousarray(right)
        rc_ = load().orc_match_u8(lc.ctypes.data, rc.ctypes.data, w, h, ctypes.byref(params),
                                  _dp(out))
    else:
        lf, rf = _f64(left), _f64(right)
        rc_ = load().orc_match(_dp(lf), _dp(rf), w, h, ctypes.byref(params), _dp(out))
    if rc_ != 0:
        raise ValueError(f"oracle rejected the arguments (code {rc_})")
    return out


def match_seeded(left, right, params: OracleParams, seed, seed_level, fallback=True):
    """R16: the method with the coarsest level seeded from `seed`, a disparity
    map at pyramid level `seed_level`, with (or without) the per-patch
    fallback to the plain start."""
    h, w = left.shape
    out = np.empty((h, w))
    lf, rf, sf = _f64(left), _f64(right), _f64(seed)
    rc_ = load().orc_match_seeded(_dp(lf), _dp(rf), w, h, ctypes.byref(params), _dp(sf),
                                  int(seed_level), int(bool(fallback)), _dp(out))
    if rc_ != 0:
        raise ValueError(f"oracle rejected the arguments (code {rc_})")
    return out


def select_start(a: dict, b: dict):
    """R16 per-patch choice between search_level results a (from the seed) and
    b (from the plain start): returns (d_star, weight, use_a) after the choice."""
    d = np.array(a["d_star"], dtype=np.float64, order="C")
    wt = np.array(a["weight"], dtype=np.float64, order="C")
    fa = np.ascontiguousarray(a["flags"], dtype=np.int32)
    fb = np.ascontiguousarray(b["flags"], dtype=np.int32)
    pa, pb = _f64(a["posterior"]), _f64(b["posterior"])
    db, wb = _f64(b["d_star"]), _f64(b["weight"])
    use = np.empty(d.shape, dtype=np.int32)
    load().orc_select_start(int(d.size), _dp(d), _dp(wt), _dp(pa), _ip(fa), _dp(db), _dp(wb),
                            _dp(pb), _ip(fb), _ip(use))
    return d, wt, use.astype(bool)


def match_stages(left, right, params: OracleParams, prev=None, seed=None, seed_level=0,
                 fallback=False) -> dict:
    """The method step by step through the per-stage C functions, keeping
    every intermediate: levels[l] = {L, R, G, coarse, search outputs, dense}.

    prev: warm start from a previous full-size disparity (R15); seed /
    seed_level / fallback: proposal start (R16); with fallback the coarsest
    level also holds the plain search ("plain") and the choice ("use_seed")."""
    top, fin = params.coarsest_scale, params.finest_scale
    Ls, Rs = [_f64(left)], [_f64(right)]
    for _ in range(top):
        Ls.append(downsample(Ls[-1]))
        Rs.append(downsample(Rs[-1]))
    levels = {}
    coarse = None
    if prev is not None:
        coarse = warm_map(prev, top + 1)
    elif seed is not None:
        coarse = warm_map(seed, top + 1 - seed_level)
    for lvl in range(top, fin - 1, -1):
        G = sobel_x(Ls[lvl])
        srch = search_level(Ls[lvl], Rs[lvl], G, coarse, params)
        carry = coarse
        extra = {}
        if seed is not None and fallback and lvl == top:
            plain = search_level(Ls[lvl], Rs[lvl], G, None, params)
            d, wt, use = select_start(srch, plain)
            extra = dict(seeded=dict(srch), plain=plain, use_seed=use)
            srch = dict(srch, d_star=d, weight=wt)
            carry = None  # carried pixels keep the plain start
        dense = densify_level(Ls[lvl].shape, params, srch["d_star"], srch["weight"], carry,
                              lvl == fin, Ls[lvl], Rs[lvl])
        levels[lvl] = dict(L=Ls[lvl], R=Rs[lvl], G=G, coarse=coarse, carry=carry, dense=dense,
                           **srch, **extra)
        coarse = dense
    out = coarse if fin == 0 else upsample(coarse, fin, left.shape)
    return {"levels": levels, "out": out, "pyramid_L": Ls, "pyramid_R": Rs}
