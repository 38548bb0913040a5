"""Failure handling, with every fault made on the host (GPU).

- A device allocation that fails (injected on the host: the library's next
  allocations report out of memory without asking the driver) returns
  BDIS_E_NOMEM and leaves the handle, plan or network usable.
- A forward pass of the proposal network whose bounded wait ran out is
  reported by bdis_net_status as BDIS_E_TIMEOUT; the record is written from
  the host exactly where the kernel's timeout path writes it (making the
  device wait run out for real could leave MMAs in flight, so it is not
  done on a GPU).
- A bounded host wait on an asynchronous call returns BDIS_E_TIMEOUT while
  the call is still running, and the call then completes normally.
- The serving loop refuses malformed frames and drops closed streams while
  every other stream's results stay exactly what they are alone.
"""
import numpy as np
import pytest
import torch

import paper_2106_07136_gb300 as bd
import synth
from gpu_helpers import dev, host, same_map
from paper_2106_07136_gb300 import _lib, serve

pytestmark = pytest.mark.gpu

KW = dict(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=3, finest_scale=0,
          gamma=0.5)


@pytest.fixture(autouse=True)
def clear_injection():
    bd.inject_alloc_failures(0)
    yield
    bd.inject_alloc_failures(0)


def small_pair(i=0):
    p = synth.make_cfg2(seed=synth.stereo.pair_seed(7, i), h=120, w=160)
    return dev(p.left, torch.uint8), dev(p.right, torch.uint8)


def test_failed_workspace_grow_leaves_the_handle_usable():
    params = bd.default_params(**KW)
    L, R = small_pair()
    ref_m = bd.Matcher()
    ref = host(ref_m.match(L, R, params))
    ref_m.close()
    m = bd.Matcher()
    bd.inject_alloc_failures(1)
    with pytest.raises(bd.BdisError) as ei:
        m.match(L, R, params)
    assert ei.value.status == _lib.BDIS_E_NOMEM
    assert m.workspace_bytes == 0
    out = host(m.match(L, R, params))  # the next call grows the workspace
    assert same_map(out, ref)
    # a grow beyond a workspace in use: the failure leaves the handle usable again
    L2 = torch.cat([L.unsqueeze(0)] * 3)
    R2 = torch.cat([R.unsqueeze(0)] * 3)
    bd.inject_alloc_failures(1)
    with pytest.raises(bd.BdisError) as ei:
        m.match(L2, R2, params)
    assert ei.value.status == _lib.BDIS_E_NOMEM
    out3 = host(m.match(L2, R2, params))
    for b in range(3):
        assert same_map(out3[b], ref)
    m.close()


def test_failed_plan_and_network_allocations():
    params = bd.default_params(**KW)
    L, R = small_pair(1)
    out = torch.empty(L.shape, dtype=torch.float32, device="cuda")
    bd.inject_alloc_failures(1)
    with pytest.raises(bd.BdisError) as ei:
        bd.Plan([(L, R, out)], params, autotune=False)
    assert ei.value.status == _lib.BDIS_E_NOMEM
    plan = bd.Plan([(L, R, out)], params, autotune=False)
    plan.run()
    torch.cuda.synchronize()
    m = bd.Matcher()
    assert same_map(host(out), host(m.match(L, R, params)))
    plan.close()
    bd.inject_alloc_failures(1)  # the network's first buffer
    with pytest.raises(bd.BdisError) as ei:
        bd.ProposalNet(bd.net_init_weights(seed=1))
    assert ei.value.status == _lib.BDIS_E_NOMEM
    net = bd.ProposalNet(bd.net_init_weights(seed=1))
    # activations grow on first use: that allocation fails, then works
    Ln = torch.rand((1, 60, 80), device="cuda") * 255
    Rn = torch.rand((1, 60, 80), device="cuda") * 255
    bd.inject_alloc_failures(1)
    with pytest.raises(bd.BdisError) as ei:
        net.forward(Ln, Rn)
    assert ei.value.status == _lib.BDIS_E_NOMEM
    a = host(net.forward(Ln, Rn))
    assert np.all(np.isfinite(a))
    net.close()
    m.close()


def test_network_timeout_is_reported_and_cleared():
    net = bd.ProposalNet(bd.net_init_weights(seed=2))
    Ln = torch.rand((2, 60, 80), device="cuda") * 255
    Rn = torch.rand((2, 60, 80), device="cuda") * 255
    a = host(net.forward(Ln, Rn))
    net.status()  # a normal forward pass records nothing
    net.inject_timeout()
    with pytest.raises(bd.BdisError) as ei:
        net.status()
    assert ei.value.status == _lib.BDIS_E_TIMEOUT
    net.status()  # reported once, then clear
    assert np.array_equal(host(net.forward(Ln, Rn)), a)
    net.status()
    net.close()


def test_bounded_host_wait_times_out_then_completes():
    params = bd.default_params(**dict(KW, coarsest_scale=4, gamma=0.75))
    L, R, _ = synth.make_batch(2, 8)
    Lb = torch.from_numpy(np.concatenate([L] * 8)).pin_memory()
    Rb = torch.from_numpy(np.concatenate([R] * 8)).pin_memory()
    m = bd.Matcher()
    ref = host(m.match(Lb.cuda(), Rb.cuda(), params))
    torch.cuda.synchronize()
    t, out = m.match_host_async(Lb, Rb, params)
    with pytest.raises(bd.BdisError) as ei:  # 64 pairs of 640x480 take milliseconds
        m.host_wait(t, timeout_s=0.0)
    assert ei.value.status == _lib.BDIS_E_TIMEOUT
    m.host_wait(t, timeout_s=60.0)
    assert same_map(out.numpy(), ref)
    m.close()


def test_serving_refuses_malformed_frames_and_drops_closed_streams():
    params = bd.default_params(**KW)
    shape = (120, 160)
    frames = {}
    for sid in range(4):
        v = synth.VideoStream(seed=synth.stereo.pair_seed(8, sid), h=shape[0], w=shape[1])
        frames[sid] = [(f.left, f.right) for f in (v.next() for _ in range(3))]
    server = serve.StereoServer([shape], params, max_batch=4, inflight=2)
    for sid in frames:
        assert server.admit(sid, shape)
    reqs = []
    for k in range(3):
        for sid in range(4):
            reqs.append(serve.Request(sid, k, *frames[sid][k]))
            server.submit(reqs[-1])
        server.poll()
    bad = [serve.Request(1, 9, frames[1][0][0][:, :100], frames[1][0][1][:, :100]),
           serve.Request(1, 10, frames[1][0][0].astype(np.float32), frames[1][0][1]),
           serve.Request(77, 0, *frames[0][0])]
    for r in bad:
        with pytest.raises(ValueError, match="malformed"):
            server.submit(r)
    assert len(server.rejected) == 3
    server.close_stream(3)  # stream 3 goes away with frames queued (and maybe one running)
    server.drain()
    server.close()
    done = [r for r in reqs if r.stream_id != 3]
    assert all(r.done > 0 and r.disparity is not None and not r.dropped for r in done)
    s3 = [r for r in reqs if r.stream_id == 3]
    assert all(r.dropped or r.disparity is not None for r in s3)
    assert any(r.dropped for r in s3)
    assert {id(r) for r in server.dropped} <= {id(r) for r in s3}
    # every other stream: each result exactly what it is alone with the same warm start
    m = bd.Matcher()
    for sid in range(3):
        prev = None
        for r in sorted((r for r in done if r.stream_id == sid), key=lambda r: r.frame):
            alone = host(m.match_warm(dev(r.left, torch.uint8), dev(r.right, torch.uint8),
                                      None if prev is None else dev(prev), params))
            assert same_map(r.disparity, alone), (sid, r.frame)
            prev = r.disparity
    m.close()
