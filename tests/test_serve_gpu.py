"""Serving loop (continuous batching, warm start, admission), GPU.

Each served result must equal the same frame matched alone with the same
warm start (the stream's previous served result), whatever batch it shared;
frames of a stream must complete in order; streams beyond the memory budget
must be refused.
"""
import numpy as np
import pytest
import torch

import paper_2106_07136_gb300 as bd
import synth
from gpu_helpers import WARM_STREAM, assert_explained, dev, host
from paper_2106_07136_gb300 import serve

pytestmark = pytest.mark.gpu

KW = dict(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=3, finest_scale=0,
          gamma=0.5)
SHAPES = [(120, 160), (240, 320)]


def make_frames(n_streams, n_frames):
    frames = {}
    for sid in range(n_streams):
        h, w = SHAPES[sid % 2]
        v = synth.VideoStream(seed=synth.stereo.pair_seed(5, sid), h=h, w=w)
        frames[sid] = [(f.left, f.right) for f in (v.next() for _ in range(n_frames))]
    return frames


def test_served_results_equal_alone_results():
    params = bd.default_params(**KW)
    frames = make_frames(6, 4)
    server = serve.StereoServer(SHAPES, params, max_batch=4, inflight=2)
    for sid in frames:
        assert server.admit(sid, SHAPES[sid % 2])
    order = [sid for _ in range(4) for sid in frames]  # frames interleave across streams
    # bursty arrivals (20k/s) so requests wait while both workers are busy
    arrivals = serve.poisson_arrivals(20000.0, len(order), seed=7)
    reqs, _ = serve.simulate(server, frames, arrivals, order)
    server.close()
    assert len(reqs) == 24 and all(r.done > 0 for r in reqs)
    assert max(r.batch_size for r in reqs) > 1  # requests shared launches
    m = bd.Matcher()
    by_stream = {}
    for r in reqs:
        by_stream.setdefault(r.stream_id, []).append(r)
    for sid, rs in by_stream.items():
        rs.sort(key=lambda r: r.frame)
        assert [r.frame for r in rs] == list(range(len(rs)))
        assert all(a.done <= b.launched for a, b in zip(rs, rs[1:]))  # in order, one at a time
        prev = None
        for r in rs:
            left, right = dev(r.left, torch.uint8), dev(r.right, torch.uint8)
            alone = host(m.match_warm(left, right, None if prev is None else dev(prev), params))
            a, b = r.disparity, alone
            assert np.array_equal(np.isnan(a), np.isnan(b))
            assert np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)]), (sid, r.frame)
            assert r.warm == (prev is not None)
            prev = r.disparity
    m.close()


def test_results_equal_alone_under_heavy_batching():
    """At a load where requests pile up (32 streams, arrivals at 200k/s, up to
    16 per launch), launches carry several requests each (mean batch above 4)
    and every result is still exactly what its frame gives alone with the
    same warm start."""
    params = bd.default_params(**KW)
    shape = SHAPES[0]
    frames = {}
    for sid in range(32):
        v = synth.VideoStream(seed=synth.stereo.pair_seed(9, sid), h=shape[0], w=shape[1])
        frames[sid] = [(f.left, f.right) for f in (v.next() for _ in range(3))]
    server = serve.StereoServer([shape], params, max_batch=16, inflight=2)
    for sid in frames:
        assert server.admit(sid, shape)
    order = [sid for _ in range(3) for sid in frames]
    arrivals = serve.poisson_arrivals(200000.0, len(order), seed=11)
    reqs, _ = serve.simulate(server, frames, arrivals, order)
    server.close()
    stats = serve.StereoServer.latency_stats(reqs)
    assert len(reqs) == 96 and stats["mean_batch"] > 4, stats
    m = bd.Matcher()
    by_stream = {}
    for r in reqs:
        by_stream.setdefault(r.stream_id, []).append(r)
    for sid, rs in by_stream.items():
        prev = None
        for r in sorted(rs, key=lambda r: r.frame):
            alone = host(m.match_warm(dev(r.left, torch.uint8), dev(r.right, torch.uint8),
                                      None if prev is None else dev(prev), params))
            a = r.disparity
            assert np.array_equal(np.isnan(a), np.isnan(alone))
            assert np.array_equal(a[~np.isnan(a)], alone[~np.isnan(alone)]), (sid, r.frame)
            prev = r.disparity
    m.close()


def test_warm_start_gpu_matches_oracle(orc):
    """bdis_match_warm against the oracle's warm start on consecutive frames."""
    params = bd.default_params(**KW)
    op = orc.OracleParams.make(**KW)
    v = synth.VideoStream(seed=synth.stereo.pair_seed(*WARM_STREAM), h=240, w=320)
    f0, f1 = v.next(), v.next()
    m = bd.Matcher()
    d0 = host(m.match(dev(f0.left, torch.uint8), dev(f0.right, torch.uint8), params))
    ref0 = orc.match(f0.left, f0.right, op)
    assert_explained(orc, d0, f0.left, f0.right, params, op, "frame 0")
    # both sides warm-start frame 1 from the same previous map (the oracle's)
    out = host(m.match_warm(dev(f1.left, torch.uint8), dev(f1.right, torch.uint8), dev(ref0),
                            params))
    assert_explained(orc, out, f1.left, f1.right, params, op, "frame 1 warm", prev=ref0)
    wm = host(bd.warm_map(dev(ref0), KW["coarsest_scale"] + 1))[0]
    np.testing.assert_allclose(wm, orc.warm_map(ref0, KW["coarsest_scale"] + 1), atol=1e-4)
    # in place: prev aliases the output
    buf = dev(ref0).clone()
    m.match_warm(dev(f1.left, torch.uint8), dev(f1.right, torch.uint8), buf, params, out=buf)
    b = host(buf)
    assert np.array_equal(np.isnan(b), np.isnan(out)) and np.array_equal(b[~np.isnan(b)],
                                                                         out[~np.isnan(out)])
    m.close()


def test_admission_by_device_memory():
    params = bd.default_params(**KW)
    probe = serve.StereoServer(SHAPES, params, max_batch=2, inflight=1)
    fixed = probe.fixed_bytes
    probe.close()
    per = 240 * 320 * 4
    server = serve.StereoServer(SHAPES, params, max_batch=2, inflight=1,
                                memory_budget_bytes=fixed + 3 * per + 10)
    admitted = [server.admit(sid, (240, 320)) for sid in range(5)]
    assert admitted == [True, True, True, False, False]
    server.close_stream(1)
    assert server.admit(7, (240, 320))  # room again once a stream closes
    assert server.refused == [3, 4]
    server.close()
