"""bdis_match_static, the entry point that allocates nothing, against bdis_match.

Callers that cannot allocate GPU memory (a real-time loop with a frozen memory
map, a plug-in inside a process that owns the allocator) call
bdis_match_static: the same kernels, with their scratch in a fixed array
inside libbdis.so instead of a handle's workspace. Through the C ABI, two
calls in a row must each return what bdis_match returns for the same input;
the second call is smaller and different, so anything the first left in the
shared array would show. Work larger than the array must be refused.

This file is collected last on purpose: the array is held by the process
once the library's module is loaded.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2106_07136_gb300 as bd
import synth
from gpu_helpers import dev, host
from paper_2106_07136_gb300 import _lib

pytestmark = pytest.mark.gpu

CFG1 = dict(patch_size=8, overlap=0.5, iterations=8, coarsest_scale=2, finest_scale=0,
            gamma=0.25)


def call_static(left, right, params):
    """bdis_match_static through ctypes; returns (status, output tensor)."""
    lb = left if left.dim() == 3 else left.unsqueeze(0)
    rb = right if right.dim() == 3 else right.unsqueeze(0)
    out = torch.full(lb.shape, -7.0, dtype=torch.float32, device="cuda")
    li, ri = bd.image_desc(lb), bd.image_desc(rb)
    st = _lib.load().bdis_match_static(ctypes.byref(li), ctypes.byref(ri), ctypes.byref(params),
                                       out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st, out


def test_static_entry_equals_handle_entry_on_two_calls():
    m = bd.Matcher()
    cases = [(synth.make_cfg2(), bd.default_params()),
             (synth.make_cfg1(), bd.default_params(**CFG1))]
    for call, (pair, params) in enumerate(cases):
        left, right = dev(pair.left, torch.uint8), dev(pair.right, torch.uint8)
        st, out = call_static(left, right, params)
        assert st == _lib.BDIS_OK, (call, _lib.load().bdis_last_error_string())
        ref = m.match(left, right, params)
        torch.cuda.synchronize()
        a, b = host(out)[0], host(ref)
        assert np.array_equal(np.isnan(a), np.isnan(b))
        assert np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)])
    m.close()


def test_static_entry_allocates_nothing_after_warm_up():
    """After one warm-up call (the first call on a device loads the array),
    further calls leave the device's free memory and torch's pool unchanged:
    the library asks the driver for nothing."""
    pair = synth.make_cfg2(seed=synth.stereo.pair_seed(2, 4))
    params = bd.default_params()
    left, right = dev(pair.left, torch.uint8), dev(pair.right, torch.uint8)
    out = torch.empty(left.shape, dtype=torch.float32, device="cuda")
    li, ri = bd.image_desc(left.unsqueeze(0)), bd.image_desc(right.unsqueeze(0))
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        st = lib.bdis_match_static(ctypes.byref(li), ctypes.byref(ri), ctypes.byref(params),
                                   out.data_ptr(), stream)
        assert st == _lib.BDIS_OK, lib.bdis_last_error_string()
        torch.cuda.synchronize()

    call()  # warm-up
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_static_entry_refuses_work_beyond_its_array():
    pair = synth.make_cfg2(seed=synth.stereo.pair_seed(3, 1), h=1080, w=1920)
    params = bd.default_params(coarsest_scale=5)
    left, right = dev(pair.left, torch.uint8), dev(pair.right, torch.uint8)
    st, out = call_static(left, right, params)
    assert st == _lib.BDIS_E_UNSUPPORTED
    assert b"scratch" in _lib.load().bdis_last_error_string()
    torch.cuda.synchronize()
    assert torch.all(out == -7.0)  # nothing was launched
