"""Serving loop for stereo video streams: continuous batching on the GPU.

Every step of the method runs in libbdis.so (bdis_match_warm); this module
schedules. Design:

- Admission by device memory: a stream is admitted only if its on-device
  state (the previous frame's disparity, kept as the warm start) fits the
  server's memory budget next to the workers' fixed workspaces; otherwise it
  is refused until another stream closes.
- Continuous batching: requests wait per frame size; whenever one of
  `inflight` workers (each a CUDA stream with its own matcher handle and
  pinned staging buffers) is free, it takes up to `max_batch` waiting
  requests of the size whose oldest request has waited longest, so requests
  that arrive while others run join the next launch, and batches on
  different workers overlap on the device (copies and kernels).
- Warm start: each stream's frame is matched with its previous frame's
  disparity as the seed of the coarsest level. A stream has at most one
  frame in flight; its next frame waits for it, so the seed is always the
  immediately preceding result.
- Per request the server records arrival, launch and completion times
  (completion = its disparity is back in host memory).
- Faults stay with the request or stream they belong to: a malformed frame
  (wrong size or type, unknown stream) is refused at submit with ValueError
  and recorded in `rejected`; a stream closed while its frames wait or run
  is dropped (queued frames removed, a running frame's result discarded and
  recorded in `dropped`), and every other stream carries on. Waits on the
  device are polled against host deadlines.

The result of a request does not depend on which other requests share its
batch: each pair's kernels read only that pair's data.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .api import Matcher, default_params


@dataclass
class Request:
    stream_id: int
    frame: int
    left: object        # (H, W) uint8: numpy array, or a pinned CPU tensor (copied directly)
    right: object
    arrival: float = 0.0
    launched: float = 0.0
    done: float = 0.0
    disparity: np.ndarray | None = None  # (H, W) float32 when done
    batch_size: int = 0
    warm: bool = False
    dropped: bool = False  # its stream was closed before the result arrived

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Stream:
    stream_id: int
    shape: tuple
    state: torch.Tensor          # previous disparity on the device, (H, W) float32
    has_state: bool = False
    busy: bool = False
    frames: collections.deque = field(default_factory=collections.deque)


class _Worker:
    """One CUDA stream with its matcher handle and staging buffers."""

    def __init__(self, device, shapes, max_batch, params):
        self.cuda_stream = torch.cuda.Stream(device=device)
        self.matcher = Matcher(device, self.cuda_stream)
        self.buffers = {}
        for (h, w) in shapes:
            with torch.cuda.device(device):
                self.matcher.reserve(w, h, max_batch, params)
            pin = dict(dtype=torch.uint8, pin_memory=True)
            self.buffers[(h, w)] = dict(
                hl=torch.empty((max_batch, h, w), **pin), hr=torch.empty((max_batch, h, w), **pin),
                ho=torch.empty((max_batch, h, w), dtype=torch.float32, pin_memory=True),
                dl=torch.empty((max_batch, h, w), dtype=torch.uint8, device=device),
                dr=torch.empty((max_batch, h, w), dtype=torch.uint8, device=device),
                prev=torch.empty((max_batch, h, w), dtype=torch.float32, device=device),
                out=torch.empty((max_batch, h, w), dtype=torch.float32, device=device))
        self.event = torch.cuda.Event()
        self.batch = None  # (shape, [requests], [stream states]) in flight

    def close(self):
        self.matcher.close()


class StereoServer:
    def __init__(self, shapes, params=None, device=None, max_batch=16, inflight=3,
                 memory_budget_bytes=None, warm_start=True, keep_results=True):
        """shapes: the (H, W) frame sizes this server handles. keep_results: copy
        each disparity out of the pinned staging buffer into the request."""
        self.keep_results = keep_results
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.params = params if params is not None else default_params()
        self.max_batch = max_batch
        self.warm_start = warm_start
        self.shapes = [tuple(s) for s in shapes]
        self.workers = [_Worker(self.device, self.shapes, max_batch, self.params)
                        for _ in range(inflight)]
        self.fixed_bytes = sum(w.matcher.workspace_bytes for w in self.workers)
        for w in self.workers:
            for b in w.buffers.values():
                self.fixed_bytes += sum(t.numel() * t.element_size() for k, t in b.items()
                                        if t.device.type == "cuda")
        if memory_budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            memory_budget_bytes = self.fixed_bytes + int(0.5 * free)
        self.budget = memory_budget_bytes
        self.state_bytes = 0
        self.streams: dict[int, _Stream] = {}
        self.waiting = {s: collections.deque() for s in self.shapes}
        self.completed: list[Request] = []
        self.refused: list[int] = []
        self.rejected: list[tuple] = []   # (stream_id, frame, reason) of malformed frames
        self.dropped: list[Request] = []  # frames of streams closed before they finished

    # --------------------------------------------------------- admission
    def stream_bytes(self, shape) -> int:
        h, w = shape
        return h * w * 4

    def admit(self, stream_id: int, shape) -> bool:
        shape = tuple(shape)
        if shape not in self.waiting:
            raise ValueError(f"server has no worker buffers for frames of {shape}")
        need = self.stream_bytes(shape)
        if self.fixed_bytes + self.state_bytes + need > self.budget:
            self.refused.append(stream_id)
            return False
        state = torch.full(shape, float("nan"), dtype=torch.float32, device=self.device)
        self.streams[stream_id] = _Stream(stream_id, shape, state)
        self.state_bytes += need
        return True

    def close_stream(self, stream_id: int):
        """Drop a stream: its waiting frames are removed; a frame of it already
        on the GPU finishes there but its result is discarded (`dropped`)."""
        st = self.streams.pop(stream_id)
        self.state_bytes -= self.stream_bytes(st.shape)
        for r in list(st.frames):
            r.dropped = True
            self.dropped.append(r)
        st.frames.clear()
        q = self.waiting[st.shape]
        keep = [r for r in q if r.stream_id != stream_id]
        for r in q:
            if r.stream_id == stream_id:
                r.dropped = True
                self.dropped.append(r)
        q.clear()
        q.extend(keep)

    # --------------------------------------------------------- requests
    def _check_frame(self, req: Request):
        st = self.streams.get(req.stream_id)
        if st is None:
            return "unknown or closed stream"
        for img in (req.left, req.right):
            shape = tuple(img.shape) if hasattr(img, "shape") else None
            dtype = getattr(img, "dtype", None)
            if shape != st.shape:
                return f"frame of shape {shape}, stream is {st.shape}"
            if dtype not in (np.uint8, torch.uint8):
                return f"frame of type {dtype}, need uint8"
            if isinstance(img, torch.Tensor) and (img.device.type != "cpu"
                                                  or not img.is_contiguous()):
                return "frame tensors must be dense host tensors"
        return None

    def submit(self, req: Request, now: float | None = None):
        """Queue a frame. A malformed one is refused with ValueError (and
        recorded in `rejected`); the server and every stream carry on."""
        why = self._check_frame(req)
        if why is not None:
            self.rejected.append((req.stream_id, req.frame, why))
            raise ValueError(f"malformed frame {req.frame} of stream {req.stream_id}: {why}")
        st = self.streams[req.stream_id]
        req.arrival = time.perf_counter() if now is None else now
        st.frames.append(req)
        self._release(st)

    def _release(self, st: _Stream):
        # a stream's next frame becomes schedulable only when none is in flight
        if not st.busy and st.frames:
            self.waiting[st.shape].append(st.frames.popleft())
            st.busy = True

    def _pick_shape(self):
        best, t = None, None
        for shape, q in self.waiting.items():
            if q and (t is None or q[0].arrival < t):
                best, t = shape, q[0].arrival
        return best

    def _launch(self, worker: _Worker, shape):
        q = self.waiting[shape]
        batch = [q.popleft() for _ in range(min(self.max_batch, len(q)))]
        n = len(batch)
        b = worker.buffers[shape]
        now = time.perf_counter()
        for i, r in enumerate(batch):
            if isinstance(r.left, torch.Tensor):
                continue  # pinned: copied straight to the device below
            b["hl"][i].numpy()[...] = r.left
            b["hr"][i].numpy()[...] = r.right
        for r in batch:
            r.launched = now
            r.batch_size = n
        states = [self.streams[r.stream_id].state for r in batch]
        with torch.cuda.stream(worker.cuda_stream):
            for i, r in enumerate(batch):
                src_l = r.left if isinstance(r.left, torch.Tensor) else b["hl"][i]
                src_r = r.right if isinstance(r.right, torch.Tensor) else b["hr"][i]
                b["dl"][i].copy_(src_l, non_blocking=True)
                b["dr"][i].copy_(src_r, non_blocking=True)
            warm = self.warm_start and any(self.streams[r.stream_id].has_state for r in batch)
            if warm:
                for i, r in enumerate(batch):
                    b["prev"][i].copy_(self.streams[r.stream_id].state, non_blocking=True)
                    r.warm = self.streams[r.stream_id].has_state
            worker.matcher.match_warm(b["dl"][:n], b["dr"][:n], b["prev"][:n] if warm else None,
                                      self.params, out=b["out"][:n])
            for i, r in enumerate(batch):
                states[i].copy_(b["out"][i], non_blocking=True)
            b["ho"][:n].copy_(b["out"][:n], non_blocking=True)
            worker.event.record(worker.cuda_stream)
        # the stream states stay referenced until the batch is done (a stream
        # closed meanwhile must not hand its tensor back while a copy is pending)
        worker.batch = (shape, batch, states)

    def _finish(self, worker: _Worker):
        shape, batch, _ = worker.batch
        now = time.perf_counter()
        ho = worker.buffers[shape]["ho"]
        for i, r in enumerate(batch):
            r.done = now
            st = self.streams.get(r.stream_id)
            if st is None:  # the stream was closed while this frame ran
                r.dropped = True
                self.dropped.append(r)
                continue
            if self.keep_results:
                r.disparity = ho[i].numpy().copy()
            st.has_state = True
            st.busy = False
            self._release(st)
            self.completed.append(r)
        worker.batch = None

    def poll(self):
        """Retire finished batches and launch waiting work on free workers.
        Returns the number of requests completed by this call."""
        n0 = len(self.completed)
        for w in self.workers:
            if w.batch is not None and w.event.query():
                self._finish(w)
        for w in self.workers:
            if w.batch is None:
                shape = self._pick_shape()
                if shape is None:
                    break
                self._launch(w, shape)
        return len(self.completed) - n0

    def busy(self) -> bool:
        return any(w.batch is not None for w in self.workers) or \
            any(q for q in self.waiting.values()) or \
            any(st.frames for st in self.streams.values())

    def drain(self, timeout_s: float = 60.0):
        t_end = time.perf_counter() + timeout_s
        while self.busy():
            if time.perf_counter() > t_end:
                raise TimeoutError("serving queue did not drain")
            if self.poll() == 0:
                time.sleep(5e-5)

    def close(self, timeout_s: float = 30.0):
        """Wait (polling, against a host deadline) for the batches on the GPU,
        then release the workers. TimeoutError if they do not finish."""
        t_end = time.perf_counter() + timeout_s
        for w in self.workers:
            while w.batch is not None and not w.event.query():
                if time.perf_counter() > t_end:
                    raise TimeoutError("a batch did not finish on the GPU")
                time.sleep(1e-4)
            w.close()

    # --------------------------------------------------------- reporting
    @staticmethod
    def latency_stats(reqs) -> dict:
        lat = np.array([r.latency for r in reqs]) * 1e3
        if lat.size == 0:
            return {}
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "n": int(lat.size),
                "mean_batch": float(np.mean([r.batch_size for r in reqs]))}


def poisson_arrivals(rate_per_s: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (s from 0) of a Poisson process."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


def simulate(server: StereoServer, frames: dict, arrivals: np.ndarray, order: list,
             time_scale: float = 1.0):
    """Replay an arrival schedule in real time.

    frames: stream_id -> list of (left, right) frames (cycled);
    order: the stream id of each arrival. Returns the list of requests."""
    t0 = time.perf_counter()
    next_frame = collections.Counter()
    reqs = []
    i = 0
    while i < len(arrivals) or server.busy():
        now = time.perf_counter() - t0
        while i < len(arrivals) and arrivals[i] * time_scale <= now:
            sid = order[i]
            fr = frames[sid]
            k = next_frame[sid]
            left, right = fr[k % len(fr)]
            next_frame[sid] += 1
            r = Request(sid, k, left, right)
            server.submit(r, now=t0 + arrivals[i] * time_scale)
            reqs.append(r)
            i += 1
        if server.poll() == 0:
            time.sleep(2e-5)
    return reqs, time.perf_counter() - t0
