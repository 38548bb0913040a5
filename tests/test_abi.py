"""The C-ABI library loads, exports every declared symbol, and its host-side
geometry and argument checks agree with the oracle. No GPU needed."""
import ctypes
import os
import re
import subprocess

import pytest
import torch

import paper_2106_07136_gb300 as bd
from paper_2106_07136_gb300 import _lib

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "bdis.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bdis_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_list_the_same_entry_points():
    assert declared_symbols() == sorted(_lib.EXPORTED)


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (bdis_[a-z0-9_]+)", out))
    assert set(declared_symbols()) <= exported


def test_default_params_are_the_papers(orc):
    p = bd.default_params()
    o = orc.OracleParams.make()
    for k, v in p.as_dict().items():
        assert abs(getattr(o, k) - v) < 1e-12, k


@pytest.mark.parametrize("n", [4, 5, 7, 8, 12, 13, 31, 40, 97, 160, 321, 480, 640, 719, 1080,
                               1920])
@pytest.mark.parametrize("ps,ov", [(8, 0.75), (8, 0.5), (12, 0.75), (4, 0.0), (16, 0.9),
                                   (32, 0.3), (5, 0.25)])
def test_geometry_bit_exact_against_oracle(orc, n, ps, ov):
    for lvl in range(6):
        assert bd.level_dims(n, n + 1, lvl) == (orc.level_dim(n, lvl), orc.level_dim(n + 1, lvl))
    ov32 = float(torch.tensor(ov, dtype=torch.float32))
    s, c = bd.grid(n, ps, ov32)
    assert s == orc.grid_stride(ps, ov32)
    assert c == orc.grid_count(n, ps, s)


def test_patch_count_of_the_paper_workloads():
    assert bd.patch_count(160, 120, bd.default_params(overlap=0.5, coarsest_scale=2)) == 1460
    assert bd.patch_count(640, 480, bd.default_params()) == 99090
    assert bd.patch_count(640, 480, bd.default_params(patch_size=12)) == 43507


@pytest.mark.parametrize("kw,status", [
    (dict(window_samples=4), _lib.BDIS_E_INVALID_ARG),
    (dict(overlap=1.0), _lib.BDIS_E_INVALID_ARG),
    (dict(iterations=-1), _lib.BDIS_E_INVALID_ARG),
    (dict(finest_scale=3, coarsest_scale=2), _lib.BDIS_E_INVALID_ARG),
    (dict(sigma_r=0.0), _lib.BDIS_E_INVALID_ARG),
    (dict(gamma=1.5), _lib.BDIS_E_INVALID_ARG),
    (dict(coarsest_scale=7), _lib.BDIS_E_INVALID_ARG),  # 640 / 2^7 < patch
    (dict(patch_size=40, coarsest_scale=2), _lib.BDIS_E_UNSUPPORTED),
    (dict(window_samples=17), _lib.BDIS_E_UNSUPPORTED),
])
def test_parameter_checks(kw, status):
    t = ctypes.c_int64()
    p = bd.default_params(**kw)
    assert _lib.load().bdis_patch_count(640, 480, ctypes.byref(p), ctypes.byref(t)) == status


def test_status_strings_and_version():
    lib = _lib.load()
    for s in range(6):
        assert lib.bdis_status_string(s)
    assert lib.bdis_version() >> 16 == 1


def test_proposal_level():
    """The learned start's network runs on the coarsest level, at most level
    4 (the level its weights are trained on); a host-only call."""
    assert [bd.proposal_level(c) for c in (0, 1, 2, 3, 4, 5, 6)] == [0, 1, 2, 3, 4, 4, 4]
    assert bd.proposal_level(-1) == -1


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU error path")
def test_create_without_gpu_reports_cuda_error():
    lib = _lib.load()
    h = ctypes.c_void_p()
    assert lib.bdis_create(ctypes.byref(h), 0, None) == _lib.BDIS_E_CUDA
    assert not h.value
    assert lib.bdis_last_error_string()
