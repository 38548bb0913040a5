"""The bounds-checked build (GPU): the memory-sanitizer substitute.

libbdis_checked.so is the library compiled with -DBDIS_CHECKED: every
data-dependent global access of the pyramid, search and densify kernels
checks its element index against the buffer's extent and records the access
site when it is out of bounds (skipping the access). A child process loads it
(BDIS_LIBRARY) and runs the method over small, ragged and full-size inputs in
every kernel variant; no access may be caught, and every map must equal the
normal build's bit for bit (an access in bounds reads what the normal build
reads).
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import paper_2106_07136_gb300 as bd
from paper_2106_07136_gb300 import build as cuda_build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Run in both processes: the maps of every case, keyed by name.
CASES = r'''
import numpy as np
import torch
import paper_2106_07136_gb300 as bd
import synth


def cases():
    out = {}
    m = bd.Matcher()
    small = dict(patch_size=8, overlap=0.75, iterations=12, finest_scale=0, gamma=0.5)
    shapes = [(16, 24, 1), (61, 97, 2), (35, 47, 2), (120, 160, 2)]
    for h, w, top in shapes:
        pairs = [synth.make_cfg2(seed=synth.stereo.pair_seed(6, i), h=h, w=w) for i in range(3)]
        L = torch.from_numpy(np.stack([p.left for p in pairs])).cuda()
        R = torch.from_numpy(np.stack([p.right for p in pairs])).cuda()
        p = bd.default_params(**dict(small, coarsest_scale=top))
        for cpl in (1, 2, 4):
            bd.set_search_variant(cpl)
            for tiled in (False, True):
                bd.set_search_tiling(tiled)
                out[f"{h}x{w} cpl{cpl} tiled{int(tiled)}"] = m.match(L, R, p).cpu().numpy()
        bd.set_search_variant(2)
        bd.set_search_tiling(False)
        for dv in (8, 16, 32):
            bd.set_densify_variant(dv)
            out[f"{h}x{w} densify{dv}"] = m.match(L, R, p).cpu().numpy()
        bd.set_densify_variant(0)
        for pv in (1, 0):
            bd.set_pyramid_variant(pv)
            out[f"{h}x{w} pyramid{pv}"] = m.match(L, R, p).cpu().numpy()
        bd.set_pyramid_variant(2)
        for ps in (12, 16):
            q = bd.default_params(**dict(small, coarsest_scale=top, patch_size=ps))
            if min(h, w) >> top >= ps:
                out[f"{h}x{w} ps{ps}"] = m.match(L, R, q).cpu().numpy()
        pd = bd.default_params(**dict(small, coarsest_scale=top, fusion=1))
        out[f"{h}x{w} dis"] = m.match(L, R, pd).cpu().numpy()
    # full size: the bench's pair, the learned start and a warm start
    L, R, _ = synth.make_batch(2, 2)
    L, R = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
    p = bd.default_params()
    d = m.match(L, R, p)
    out["640x480"] = d.cpu().numpy()
    out["640x480 warm"] = m.match_warm(L, R, d, p).cpu().numpy()
    net = bd.ProposalNet(bd.net_init_weights(seed=5))
    out["640x480 learned"] = m.match_learned(net, L, R, p, fallback=True).cpu().numpy()
    net.close()
    m.close()
    return out
'''


def run_cases():
    ns = {}
    exec(CASES, ns)
    return ns["cases"]()


CHILD = CASES + r'''
import sys
assert bd.checked_build(), "the child must load the checked build"
res = cases()
res["__sites__"] = np.array([bd.check_status()], dtype=np.int64)
np.savez(sys.argv[1], **res)
'''


def test_checked_build_catches_nothing_and_changes_nothing(tmp_path):
    lib = cuda_build.build(checked=True)
    script = tmp_path / "child.py"
    script.write_text(CHILD)
    out = tmp_path / "maps.npz"
    env = dict(os.environ, BDIS_LIBRARY=lib, PYTHONPATH=ROOT + os.pathsep +
               os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, str(script), str(out)], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    got = dict(np.load(out))
    assert int(got.pop("__sites__")[0]) == 0, "an access out of bounds was caught"
    assert not bd.checked_build()
    ref = run_cases()
    assert set(got) == set(ref)
    for k in ref:
        a, b = got[k], ref[k]
        assert np.array_equal(np.isnan(a), np.isnan(b)), k
        assert np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)]), k
    assert bd.check_status() == 0  # the normal build records nothing
