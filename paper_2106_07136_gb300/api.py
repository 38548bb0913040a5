"""Python face of the BDIS CUDA library: argument marshalling over the C ABI.

Every step of the method runs in libbdis.so's kernels. PyTorch provides the
device memory (tensors) and the CUDA stream; nothing here computes.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import BdisImage, BdisParams, BdisPatchDebug, check


def default_params(**overrides) -> BdisParams:
    """The paper's settings (Sec. 3) with optional overrides."""
    p = BdisParams()
    _lib.load().bdis_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def level_dims(width: int, height: int, level: int):
    w, h = ctypes.c_int(), ctypes.c_int()
    check(_lib.load().bdis_level_dims(width, height, level, ctypes.byref(w), ctypes.byref(h)),
          "bdis_level_dims")
    return w.value, h.value


def grid(n: int, patch_size: int, overlap: float):
    s, c = ctypes.c_int(), ctypes.c_int()
    check(_lib.load().bdis_grid(n, patch_size, overlap, ctypes.byref(s), ctypes.byref(c)),
          "bdis_grid")
    return s.value, c.value


def patch_count(width: int, height: int, params: BdisParams) -> int:
    t = ctypes.c_int64()
    check(_lib.load().bdis_patch_count(width, height, ctypes.byref(params), ctypes.byref(t)),
          "bdis_patch_count")
    return t.value


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _as_batch(t: torch.Tensor) -> torch.Tensor:
    if t.dim() == 2:
        return t.unsqueeze(0)
    if t.dim() != 3:
        raise ValueError("images must be (H, W) or (B, H, W)")
    return t


def image_desc(t: torch.Tensor) -> BdisImage:
    """Describe a (B, H, W) or (H, W) CUDA tensor (uint8 or float32, unit column stride)."""
    t = _as_batch(t)
    if t.dtype == torch.uint8:
        fmt, es = _lib.BDIS_U8, 1
    elif t.dtype == torch.float32:
        fmt, es = _lib.BDIS_F32, 4
    else:
        raise TypeError("images must be uint8 or float32")
    if t.stride(2) != 1:
        raise ValueError("image rows must be contiguous")
    b, h, w = t.shape
    return BdisImage(t.data_ptr(), w, h, t.stride(1) * es, t.stride(0) * es, b, fmt)


class Matcher:
    """A BDIS matcher bound to one CUDA device and stream (bdis_create)."""

    def __init__(self, device=None, stream=None):
        self._lib = _lib.load()
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else \
            torch.device(device)
        self.device = dev
        with torch.cuda.device(dev):
            self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        h = ctypes.c_void_p()
        check(self._lib.bdis_create(ctypes.byref(h), dev.index or 0,
                                    ctypes.c_void_p(int(self.stream.cuda_stream))), "bdis_create")
        self._h = h
        self._inflight = {}  # ticket -> host buffers of bdis_match_host_async calls

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.bdis_destroy(self._h)  # waits for all work, asynchronous calls included
            self._h = None
            self._inflight = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, width, height, count, params: BdisParams):
        check(self._lib.bdis_reserve(self._h, width, height, count, ctypes.byref(params)),
              "bdis_reserve")

    @property
    def workspace_bytes(self) -> int:
        return int(self._lib.bdis_workspace_bytes(self._h))

    def enable_timing(self, on: bool = True):
        """Bracket every kernel launch of this handle with CUDA events."""
        check(self._lib.bdis_enable_timing(self._h, int(bool(on))), "bdis_enable_timing")

    def read_timing(self) -> dict:
        """Per kernel class: (total ms, launches) since the last read; waits for them."""
        t = _lib.BdisTiming()
        check(self._lib.bdis_read_timing(self._h, ctypes.byref(t)), "bdis_read_timing")
        return {name: (t.ms[i], int(t.launches[i]))
                for i, name in enumerate(_lib.TIMING_CLASSES)}

    def match(self, left: torch.Tensor, right: torch.Tensor, params: BdisParams = None,
              out: torch.Tensor = None) -> torch.Tensor:
        """Disparity of device images (H, W) or (B, H, W); NaN = not estimated."""
        params = params if params is not None else default_params()
        squeeze = left.dim() == 2
        lb, rb = _as_batch(left), _as_batch(right)
        b, h, w = lb.shape
        if out is None:
            out = torch.empty((b, h, w), dtype=torch.float32, device=left.device)
        if not (out.is_contiguous() and out.dtype == torch.float32 and out.numel() == b * h * w):
            raise ValueError("out must be a dense float32 tensor of B*H*W elements")
        li, ri = image_desc(lb), image_desc(rb)
        check(self._lib.bdis_match(self._h, ctypes.byref(li), ctypes.byref(ri),
                                   ctypes.byref(params), out.data_ptr()), "bdis_match")
        return out[0] if squeeze else out

    def match_warm(self, left: torch.Tensor, right: torch.Tensor, prev: torch.Tensor,
                   params: BdisParams = None, out: torch.Tensor = None) -> torch.Tensor:
        """bdis_match with the coarsest level seeded from `prev` (same shape as the
        output; may be `out` itself). prev None = match."""
        params = params if params is not None else default_params()
        squeeze = left.dim() == 2
        lb, rb = _as_batch(left), _as_batch(right)
        b, h, w = lb.shape
        if out is None:
            out = torch.empty((b, h, w), dtype=torch.float32, device=left.device)
        if not (out.is_contiguous() and out.dtype == torch.float32 and out.numel() == b * h * w):
            raise ValueError("out must be a dense float32 tensor of B*H*W elements")
        pp = None
        if prev is not None:
            if not (prev.is_contiguous() and prev.dtype == torch.float32
                    and prev.numel() == b * h * w):
                raise ValueError("prev must be a dense float32 tensor of B*H*W elements")
            pp = prev.data_ptr()
        li, ri = image_desc(lb), image_desc(rb)
        check(self._lib.bdis_match_warm(self._h, ctypes.byref(li), ctypes.byref(ri),
                                        ctypes.byref(params), pp, out.data_ptr()),
              "bdis_match_warm")
        return out.view(b, h, w)[0] if squeeze else out

    def _out(self, lb, out):
        b, h, w = lb.shape
        if out is None:
            out = torch.empty((b, h, w), dtype=torch.float32, device=lb.device)
        if not (out.is_contiguous() and out.dtype == torch.float32 and out.numel() == b * h * w):
            raise ValueError("out must be a dense float32 tensor of B*H*W elements")
        return out

    def match_seeded(self, left, right, seed, seed_level, params: BdisParams = None,
                     fallback: bool = True, out=None):
        """Coarsest level seeded from `seed` (B, h_l, w_l) at pyramid level seed_level."""
        params = params if params is not None else default_params()
        squeeze = left.dim() == 2
        lb, rb = _as_batch(left), _as_batch(right)
        out = self._out(lb, out)
        seed = _as_batch(seed).contiguous()
        li, ri = image_desc(lb), image_desc(rb)
        check(self._lib.bdis_match_seeded(self._h, ctypes.byref(li), ctypes.byref(ri),
                                          ctypes.byref(params), seed.data_ptr(), int(seed_level),
                                          int(bool(fallback)), out.data_ptr()),
              "bdis_match_seeded")
        return out.view(lb.shape)[0] if squeeze else out

    def match_learned(self, net, left, right, params: BdisParams = None, fallback: bool = True,
                      out=None):
        """Coarsest level seeded by the proposal network (ProposalNet) run on
        pyramid level proposal_level(params.coarsest_scale)."""
        params = params if params is not None else default_params()
        squeeze = left.dim() == 2
        lb, rb = _as_batch(left), _as_batch(right)
        out = self._out(lb, out)
        li, ri = image_desc(lb), image_desc(rb)
        check(self._lib.bdis_match_learned(self._h, net._h, ctypes.byref(li), ctypes.byref(ri),
                                           ctypes.byref(params), int(bool(fallback)),
                                           out.data_ptr()), "bdis_match_learned")
        return out.view(lb.shape)[0] if squeeze else out

    def match_host(self, left, right, params: BdisParams = None, out=None):
        """Host buffers in and out (numpy arrays or CPU tensors, pinned for DMA).

        left/right: uint8 (H, W) or (B, H, W) dense; returns float32 of the
        same shape. The call blocks until the result is in `out`."""
        params = params if params is not None else default_params()
        lt = torch.as_tensor(left)
        rt = torch.as_tensor(right)
        if lt.dtype != torch.uint8 or rt.dtype != torch.uint8 or lt.device.type != "cpu":
            raise TypeError("match_host takes uint8 host images")
        lt, rt = lt.contiguous(), rt.contiguous()
        shape = lt.shape
        b = 1 if lt.dim() == 2 else lt.shape[0]
        h, w = lt.shape[-2], lt.shape[-1]
        if out is None:
            out = torch.empty(shape, dtype=torch.float32)
        ot = torch.as_tensor(out)
        if not (ot.is_contiguous() and ot.dtype == torch.float32 and ot.numel() == b * h * w):
            raise ValueError("out must be a dense float32 host buffer of B*H*W elements")
        check(self._lib.bdis_match_host(self._h, lt.data_ptr(), rt.data_ptr(), w, h, b,
                                        ctypes.byref(params), ot.data_ptr()), "bdis_match_host")
        return out

    def match_host_async(self, left, right, params: BdisParams = None, out=None):
        """bdis_match_host_async: enqueue one batch with host buffers and return
        (ticket, out) at once. `left`, `right` and `out` must be left alone
        until host_wait(ticket); they are kept referenced until then. Pinned
        buffers make the call asynchronous."""
        params = params if params is not None else default_params()
        lt, rt = torch.as_tensor(left), torch.as_tensor(right)
        if lt.dtype != torch.uint8 or rt.dtype != torch.uint8 or lt.device.type != "cpu":
            raise TypeError("match_host_async takes uint8 host images")
        if not (lt.is_contiguous() and rt.is_contiguous()):
            raise ValueError("match_host_async takes dense host images")
        b = 1 if lt.dim() == 2 else lt.shape[0]
        h, w = lt.shape[-2], lt.shape[-1]
        if out is None:
            out = torch.empty(lt.shape, dtype=torch.float32).pin_memory() if lt.is_pinned() \
                else torch.empty(lt.shape, dtype=torch.float32)
        ot = torch.as_tensor(out)
        if not (ot.is_contiguous() and ot.dtype == torch.float32 and ot.numel() == b * h * w):
            raise ValueError("out must be a dense float32 host buffer of B*H*W elements")
        ticket = ctypes.c_uint64(0)
        check(self._lib.bdis_match_host_async(self._h, lt.data_ptr(), rt.data_ptr(), w, h, b,
                                              ctypes.byref(params), ot.data_ptr(),
                                              ctypes.byref(ticket)), "bdis_match_host_async")
        self._inflight[ticket.value] = (lt, rt, ot)
        return ticket.value, out

    def host_wait(self, ticket: int, timeout_s: float | None = None):
        """bdis_host_wait: return once call `ticket` (and all before it) is done.
        With timeout_s, bdis_host_wait_timeout: raise BdisError (status
        BDIS_E_TIMEOUT) if it is not done by then; the call stays in flight."""
        if timeout_s is None:
            check(self._lib.bdis_host_wait(self._h, ticket), "bdis_host_wait")
        else:
            check(self._lib.bdis_host_wait_timeout(self._h, ticket, 1e3 * float(timeout_s)),
                  "bdis_host_wait_timeout")
        for t in [t for t in self._inflight if t <= ticket]:
            del self._inflight[t]


def match_static(left: torch.Tensor, right: torch.Tensor, params: BdisParams = None,
                 out: torch.Tensor = None, stream=None) -> torch.Tensor:
    """bdis_match_static: the method without any device allocation inside the
    library, for callers that cannot allocate GPU memory on this path (the
    scratch is a fixed array in libbdis.so; work larger than it is refused).
    Runs on the current device; `out` should be preallocated by such callers."""
    params = params if params is not None else default_params()
    squeeze = left.dim() == 2
    lb, rb = _as_batch(left), _as_batch(right)
    b, h, w = lb.shape
    if out is None:
        out = torch.empty((b, h, w), dtype=torch.float32, device=left.device)
    if not (out.is_contiguous() and out.dtype == torch.float32 and out.numel() == b * h * w):
        raise ValueError("out must be a dense float32 tensor of B*H*W elements")
    li, ri = image_desc(lb), image_desc(rb)
    check(_lib.load().bdis_match_static(ctypes.byref(li), ctypes.byref(ri), ctypes.byref(params),
                                        out.data_ptr(), _stream_ptr(stream)), "bdis_match_static")
    return out.view(b, h, w)[0] if squeeze else out


def inject_alloc_failures(count: int):
    """Host-side fault injection: the library's next `count` device allocations
    fail as out of memory (bdis_inject_alloc_failures); 0 clears it."""
    _lib.load().bdis_inject_alloc_failures(int(count))


def set_search_variant(columns_per_lane: int):
    """Lane layout of the fixed-size search kernel: 1, 2 (default) or 4 columns per lane."""
    check(_lib.load().bdis_set_search_variant(int(columns_per_lane)), "bdis_set_search_variant")


def get_search_variant() -> int:
    return int(_lib.load().bdis_get_search_variant())


def set_search_tiling(on: bool):
    """Warp-tiled shared-memory sampling in the fixed-size search kernel (default off)."""
    _lib.load().bdis_set_search_tiling(1 if on else 0)


def get_search_tiling() -> bool:
    return bool(_lib.load().bdis_get_search_tiling())


def set_densify_variant(tile_height: int):
    """Densify kernel: 0 = strips where they apply (default), 8/16/32 = tiles of that height."""
    check(_lib.load().bdis_set_densify_variant(int(tile_height)), "bdis_set_densify_variant")


def get_densify_variant() -> int:
    return int(_lib.load().bdis_get_densify_variant())


def set_pyramid_variant(variant: int):
    """Pyramid: 2 (default) level 0 and the first step in one kernel, later steps
    fused; 1 every step one fused kernel; 0 downsample, then gradient, per step.
    A bool selects 1 (True) or 0 (False)."""
    _lib.load().bdis_set_pyramid_variant(int(variant))


def get_pyramid_variant() -> int:
    return int(_lib.load().bdis_get_pyramid_variant())


def checked_build() -> bool:
    """Whether the loaded library is the bounds-checked build."""
    return bool(_lib.load().bdis_checked_build())


def check_status() -> int:
    """Bit mask of the access sites the bounds-checked build caught out of
    bounds since the last call (0 in the normal build); waits for the device."""
    v = ctypes.c_uint32(0)
    check(_lib.load().bdis_check_status(ctypes.byref(v)), "bdis_check_status")
    return int(v.value)


def set_launch_overlap(on: bool):
    """Launch the default pyramid, search and densify kernels as programmatic
    dependents of the kernel before them (default on); results are identical."""
    _lib.load().bdis_set_launch_overlap(int(bool(on)))


def get_launch_overlap() -> bool:
    return bool(_lib.load().bdis_get_launch_overlap())


def set_net_variant(tensor_path: int):
    """Proposal network forward convolutions: 1 = banded tcgen05 kernel (default),
    2 = per-tile tcgen05 kernel, 0 = mma.sync kernel."""
    _lib.load().bdis_set_net_variant(int(tensor_path))


def get_net_variant() -> int:
    return int(_lib.load().bdis_get_net_variant())


def probe_fp32_tflops(iterations: int = 1 << 16, stream=None) -> float:
    """Measured FP32 FMA throughput of the current GPU (TFLOP/s)."""
    t = ctypes.c_double()
    check(_lib.load().bdis_probe_fp32_tflops(int(iterations), ctypes.byref(t), _stream_ptr(stream)),
          "bdis_probe_fp32_tflops")
    return t.value


class Plan:
    """Mixed-resolution batch as one CUDA graph (bdis_plan_create / run).

    groups: list of (left, right, out) CUDA tensors, each (B, H, W) with one
    size per group; the plan binds their addresses, so refill them in place
    between runs. scale_to_width: raise each group's coarsest scale to keep a
    disparity range of a tenth of its width within 4 px there
    (BDIS_PLAN_SCALE_TO_WIDTH)."""

    def __init__(self, groups, params: BdisParams = None, autotune: bool = True, device=None,
                 stream=None, scale_to_width: bool = False):
        self._lib = _lib.load()
        params = params if params is not None else default_params()
        self._keep = []
        arr = (_lib.BdisGroup * len(groups))()
        for i, (left, right, out) in enumerate(groups):
            lb, rb = _as_batch(left), _as_batch(right)
            if not (out.is_contiguous() and out.dtype == torch.float32
                    and out.numel() == lb.numel()):
                raise ValueError("each output must be a dense float32 tensor like its images")
            arr[i].left = image_desc(lb)
            arr[i].right = image_desc(rb)
            arr[i].disparity_out = out.data_ptr()
            self._keep += [lb, rb, out]
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else \
            torch.device(device)
        h = ctypes.c_void_p()
        check(self._lib.bdis_plan_create(dev.index or 0, arr, len(groups), ctypes.byref(params),
                                         (_lib.BDIS_PLAN_AUTOTUNE if autotune else 0)
                                         | (_lib.BDIS_PLAN_SCALE_TO_WIDTH if scale_to_width
                                            else 0),
                                         _stream_ptr(stream), ctypes.byref(h)),
              "bdis_plan_create")
        self._h = h
        self.n_groups = len(groups)
        self.levels = range(params.finest_scale, params.coarsest_scale + 1)

    def run(self, stream=None):
        check(self._lib.bdis_plan_run(self._h, _stream_ptr(stream)), "bdis_plan_run")

    def choice(self, group: int, level: int) -> dict:
        c = _lib.BdisPlanChoice()
        check(self._lib.bdis_plan_info(self._h, group, level, ctypes.byref(c)), "bdis_plan_info")
        return {"search_columns_per_lane": c.search_columns_per_lane,
                "search_block_threads": c.search_block_threads,
                "densify_tile_height": c.densify_tile_height,
                "workspace_bytes": int(c.workspace_bytes),
                "coarsest_scale": c.coarsest_scale,
                "search_tiling": c.search_tiling}

    @property
    def workspace_bytes(self) -> int:
        return int(self._lib.bdis_plan_workspace_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.bdis_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NET_DILATIONS = (1, 2, 4, 4, 2, 1)
NET_CHANNELS = ((2, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 1))


def net_weight_count() -> int:
    return int(_lib.load().bdis_net_weight_count())


def proposal_level(coarsest_scale: int) -> int:
    """The pyramid level the learned start runs the proposal network on."""
    return int(_lib.load().bdis_proposal_level(int(coarsest_scale)))


def net_init_weights(seed: int = 0) -> np.ndarray:
    """He-initialised master weights (host float32), layer by layer W[co][tap][ci], b[co]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for (ci, co) in NET_CHANNELS:
        std = np.sqrt(2.0 / (9 * ci))
        parts.append(rng.normal(0.0, std, size=co * 9 * ci))
        parts.append(np.zeros(co))
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == net_weight_count()
    return w


WEIGHTS_MAGIC = b"BDISNET1"


def save_net_weights(path, weights, note: str = ""):
    """Versioned weights file: magic, version, count, note length, sha256 of the
    float32 payload, note (utf-8), payload (little-endian float32)."""
    import hashlib
    import struct
    w = np.ascontiguousarray(weights, dtype="<f4")
    payload = w.tobytes()
    nb = note.encode()
    with open(path, "wb") as f:
        f.write(WEIGHTS_MAGIC)
        f.write(struct.pack("<III", 1, w.size, len(nb)))
        f.write(hashlib.sha256(payload).digest())
        f.write(nb)
        f.write(payload)


def load_net_weights(path):
    """Read save_net_weights' format; checks magic, count and hash."""
    import hashlib
    import struct
    data = open(path, "rb").read()
    if data[:8] != WEIGHTS_MAGIC:
        raise ValueError(f"{path}: not a proposal-network weights file")
    version, count, nlen = struct.unpack("<III", data[8:20])
    if version != 1 or count != net_weight_count():
        raise ValueError(f"{path}: version {version}, {count} weights (need {net_weight_count()})")
    digest = data[20:52]
    note = data[52:52 + nlen].decode()
    payload = data[52 + nlen:]
    if len(payload) != 4 * count or hashlib.sha256(payload).digest() != digest:
        raise ValueError(f"{path}: weights payload is corrupt")
    return np.frombuffer(payload, dtype="<f4").astype(np.float32), note


class ProposalNet:
    """The learned coarse proposal (bdis_net_*): forward, gradient, Adam steps."""

    def __init__(self, weights=None, device=None):
        self._lib = _lib.load()
        w = net_init_weights() if weights is None else np.ascontiguousarray(weights, np.float32)
        if w.size != net_weight_count():
            raise ValueError("wrong number of weights")
        dev = torch.cuda.current_device() if device is None else torch.device(device).index or 0
        h = ctypes.c_void_p()
        check(self._lib.bdis_net_create(dev, w.ctypes.data, ctypes.byref(h)), "bdis_net_create")
        self._h = h

    @staticmethod
    def _planes(L, R):
        L = _as_batch(L).contiguous()
        if R.dim() >= 3 and R.shape[-1] == 2 and R.dim() == L.dim() + 1:
            return L, _packed(R), 2
        return L, _as_batch(R).contiguous(), 1

    def forward(self, L, R, stream=None) -> torch.Tensor:
        L, Rp, rs = self._planes(L, R)
        b, h, w = L.shape
        out = torch.empty((b, h, w), dtype=torch.float32, device=L.device)
        check(self._lib.bdis_net_forward(self._h, L.data_ptr(), Rp.data_ptr(), rs, w, h, b,
                                         out.data_ptr(), _stream_ptr(stream)), "bdis_net_forward")
        return out

    def gradient(self, L, R, label, stream=None):
        L, Rp, rs = self._planes(L, R)
        b, h, w = L.shape
        label = _as_batch(label).contiguous()
        loss = ctypes.c_float()
        grad = np.empty(net_weight_count(), dtype=np.float32)
        check(self._lib.bdis_net_gradient(self._h, L.data_ptr(), Rp.data_ptr(), rs, w, h, b,
                                          label.data_ptr(), ctypes.byref(loss), grad.ctypes.data,
                                          _stream_ptr(stream)), "bdis_net_gradient")
        return loss.value, grad

    def train_step(self, L, R, label, lr, stream=None) -> float:
        L, Rp, rs = self._planes(L, R)
        b, h, w = L.shape
        label = _as_batch(label).contiguous()
        loss = ctypes.c_float()
        check(self._lib.bdis_net_train_step(self._h, L.data_ptr(), Rp.data_ptr(), rs, w, h, b,
                                            label.data_ptr(), float(lr), ctypes.byref(loss),
                                            _stream_ptr(stream)), "bdis_net_train_step")
        return loss.value

    def status(self, stream=None):
        """bdis_net_status: raise BdisError (BDIS_E_TIMEOUT) if a forward pass's
        bounded wait ran out since the last check; waits for the stream."""
        check(self._lib.bdis_net_status(self._h, _stream_ptr(stream)), "bdis_net_status")

    def inject_timeout(self):
        """Host-side fault injection: record a forward-pass timeout."""
        check(self._lib.bdis_net_inject_timeout(self._h), "bdis_net_inject_timeout")

    def weights(self) -> np.ndarray:
        w = np.empty(net_weight_count(), dtype=np.float32)
        check(self._lib.bdis_net_get_weights(self._h, w.ctypes.data), "bdis_net_get_weights")
        return w

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.bdis_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ steps

def prepare_level0(left: torch.Tensor, right: torch.Tensor, stream=None):
    """Level 0: (L0, R0 packed (B, H, W, 2), G0)."""
    lb, rb = _as_batch(left), _as_batch(right)
    b, h, w = lb.shape
    L0, G0 = (torch.empty((b, h, w), dtype=torch.float32, device=left.device) for _ in range(2))
    R0 = torch.empty((b, h, w, 2), dtype=torch.float32, device=left.device)
    li, ri = image_desc(lb), image_desc(rb)
    check(_lib.load().bdis_prepare_level0(ctypes.byref(li), ctypes.byref(ri), L0.data_ptr(),
                                          R0.data_ptr(), G0.data_ptr(), _stream_ptr(stream)),
          "bdis_prepare_level0")
    return L0, R0, G0


def _packed(R):
    if R.dim() == 3:
        R = R.unsqueeze(0)
    if R.dim() != 4 or R.shape[-1] != 2:
        raise ValueError("packed right planes are (B, H, W, 2)")
    return R.contiguous()


def pack_right(R: torch.Tensor, stream=None) -> torch.Tensor:
    """(B, H, W) float32 right plane -> packed (B, H, W, 2)."""
    R = _as_batch(R).contiguous()
    b, h, w = R.shape
    out = torch.empty((b, h, w, 2), dtype=torch.float32, device=R.device)
    check(_lib.load().bdis_pack_right(R.data_ptr(), w, h, b, out.data_ptr(), _stream_ptr(stream)),
          "bdis_pack_right")
    return out


def pyramid_level(L: torch.Tensor, R: torch.Tensor, stream=None):
    """One pyramid step: (L, packed R) -> (L1, packed R1, G1)."""
    L, R = _as_batch(L).contiguous(), _packed(R)
    b, h, w = L.shape
    dh, dw = (h + 1) // 2, (w + 1) // 2
    L1, G1 = (torch.empty((b, dh, dw), dtype=torch.float32, device=L.device) for _ in range(2))
    R1 = torch.empty((b, dh, dw, 2), dtype=torch.float32, device=L.device)
    check(_lib.load().bdis_pyramid_level(L.data_ptr(), R.data_ptr(), w, h, b, L1.data_ptr(),
                                         R1.data_ptr(), G1.data_ptr(), _stream_ptr(stream)),
          "bdis_pyramid_level")
    return L1, R1, G1


def search_level(L, R, G, coarse, params: BdisParams, debug: bool = True, stream=None) -> dict:
    """Inverse search + posterior of every patch of one level (R packed).

    Returns tensors shaped (B, ny, nx): d_star, weight and, with debug, u_init,
    posterior, flags, n_valid, steps (updates applied to D, uint8) and energies
    (B, ny, nx, s)."""
    L, G = (_as_batch(t).contiguous() for t in (L, G))
    R = _packed(R)
    b, h, w = L.shape
    s, nx = grid(w, params.patch_size, params.overlap)
    _, ny = grid(h, params.patch_size, params.overlap)
    dev = L.device
    f32 = dict(dtype=torch.float32, device=dev)
    out = {"d_star": torch.empty((b, ny, nx), **f32), "weight": torch.empty((b, ny, nx), **f32)}
    dbg = None
    if debug:
        out.update(u_init=torch.empty((b, ny, nx), **f32),
                   posterior=torch.empty((b, ny, nx), **f32),
                   energies=torch.empty((b, ny, nx, params.window_samples), **f32),
                   flags=torch.empty((b, ny, nx), dtype=torch.uint8, device=dev),
                   n_valid=torch.empty((b, ny, nx), dtype=torch.int32, device=dev),
                   steps=torch.empty((b, ny, nx), dtype=torch.uint8, device=dev))
        dbg = BdisPatchDebug(out["u_init"].data_ptr(), out["posterior"].data_ptr(),
                             out["energies"].data_ptr(), out["flags"].data_ptr(),
                             out["n_valid"].data_ptr(), out["steps"].data_ptr())
    if coarse is not None:
        coarse = _as_batch(coarse).contiguous()
        cp, cw, ch = coarse.data_ptr(), coarse.shape[2], coarse.shape[1]
    else:
        cp, cw, ch = None, 0, 0
    check(_lib.load().bdis_search_level(L.data_ptr(), R.data_ptr(), G.data_ptr(), w, h, b, cp, cw,
                                        ch, ctypes.byref(params), out["d_star"].data_ptr(),
                                        out["weight"].data_ptr(),
                                        ctypes.byref(dbg) if dbg is not None else None,
                                        _stream_ptr(stream)), "bdis_search_level")
    return out


def densify_level(shape, params: BdisParams, d_star, weight, coarse, is_finest, L=None, R=None,
                  stream=None):
    """Dense map of one level; L and packed R of the level are needed for DIS fusion."""
    d_star, weight = _as_batch(d_star).contiguous(), _as_batch(weight).contiguous()
    b = d_star.shape[0]
    h, w = shape
    out = torch.empty((b, h, w), dtype=torch.float32, device=d_star.device)
    if coarse is not None:
        coarse = _as_batch(coarse).contiguous()
        cp, cw, ch = coarse.data_ptr(), coarse.shape[2], coarse.shape[1]
    else:
        cp, cw, ch = None, 0, 0
    Lp = None if L is None else _as_batch(L).contiguous()
    Rp = None if R is None else _packed(R)
    check(_lib.load().bdis_densify_level(w, h, b, ctypes.byref(params), d_star.data_ptr(),
                                         weight.data_ptr(), cp, cw, ch, int(bool(is_finest)),
                                         None if Lp is None else Lp.data_ptr(),
                                         None if Rp is None else Rp.data_ptr(),
                                         out.data_ptr(), _stream_ptr(stream)),
          "bdis_densify_level")
    return out


def select_start(a: dict, b: dict, stream=None):
    """R16 choice on a level searched twice: search_level results a (from a
    seed) and b (from the plain start), both with debug outputs. Returns the
    chosen (d_star, weight) as new tensors; a and b are left unchanged."""
    d, w = a["d_star"].clone(), a["weight"].clone()
    pa, fa = a["posterior"].contiguous(), a["flags"].contiguous()
    db, wb = b["d_star"].contiguous(), b["weight"].contiguous()
    pb, fb = b["posterior"].contiguous(), b["flags"].contiguous()
    check(_lib.load().bdis_select_start(d.data_ptr(), w.data_ptr(), pa.data_ptr(), fa.data_ptr(),
                                        db.data_ptr(), wb.data_ptr(), pb.data_ptr(),
                                        fb.data_ptr(), d.numel(), _stream_ptr(stream)),
          "bdis_select_start")
    return d, w


def warm_map(prev: torch.Tensor, level: int, stream=None) -> torch.Tensor:
    """Warm-start seed map of `level` from a (B, H, W) previous disparity."""
    prev = _as_batch(prev).contiguous()
    b, h, w = prev.shape
    out = torch.empty((b, (h + (1 << level) - 1) >> level, (w + (1 << level) - 1) >> level),
                      dtype=torch.float32, device=prev.device)
    check(_lib.load().bdis_warm_map(prev.data_ptr(), w, h, level, b, out.data_ptr(),
                                    _stream_ptr(stream)), "bdis_warm_map")
    return out


def upsample(M, level, shape, stream=None):
    M = _as_batch(M).contiguous()
    b, mh, mw = M.shape
    h, w = shape
    out = torch.empty((b, h, w), dtype=torch.float32, device=M.device)
    check(_lib.load().bdis_upsample(M.data_ptr(), mw, mh, level, w, h, b, out.data_ptr(),
                                    _stream_ptr(stream)), "bdis_upsample")
    return out
