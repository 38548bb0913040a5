"""FP64 CPU oracle of the learned coarse-proposal network.

TEST INFRASTRUCTURE ONLY: plain PyTorch CPU operations in float64 (conv2d as
the library primitive, autograd for the gradient), written from the
architecture the CUDA library declares: six 3x3 convolutions with dilations
1, 2, 4, 4, 2, 1 and zero padding, channels 2 -> 32 x5 -> 1, ReLU between
layers, input [(L - 128) / 64, (R - 128) / 64], Huber loss (delta 1) averaged
over all pixels with unlabelled (NaN) pixels counting 0. The network is not
part of the paper; it proposes the coarsest start that BDIS refines.
Master weight order, layer by layer: W[co][ky*3+kx][ci], then b[co].
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

DILATIONS = (1, 2, 4, 4, 2, 1)
CHANNELS = ((2, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 1))


def weight_count() -> int:
    return sum(co * 9 * ci + co for ci, co in CHANNELS)


def unpack(w):
    """Flat master weights -> [(W (co, ci, 3, 3), b (co,))] as float64 tensors."""
    w = torch.as_tensor(np.asarray(w, dtype=np.float64))
    layers, off = [], 0
    for ci, co in CHANNELS:
        n = co * 9 * ci
        W = w[off:off + n].reshape(co, 3, 3, ci).permute(0, 3, 1, 2)
        off += n
        b = w[off:off + co]
        off += co
        layers.append((W, b))
    assert off == w.numel()
    return layers


def _input(L, R):
    L = torch.as_tensor(np.asarray(L, dtype=np.float64))
    R = torch.as_tensor(np.asarray(R, dtype=np.float64))
    if L.dim() == 2:
        L, R = L[None], R[None]
    return torch.stack([(L - 128.0) / 64.0, (R - 128.0) / 64.0], dim=1)


def _net(x, layers):
    for i, ((W, b), d) in enumerate(zip(layers, DILATIONS)):
        x = F.conv2d(x, W, b, padding=d, dilation=d)
        if i < len(layers) - 1:
            x = torch.relu(x)
    return x[:, 0]


def forward(L, R, w) -> np.ndarray:
    with torch.no_grad():
        return _net(_input(L, R), unpack(w)).numpy()


def huber(e):
    a = e.abs()
    return torch.where(a <= 1.0, 0.5 * e * e, a - 0.5)


def loss_and_grad(L, R, label, w):
    """Loss and its gradient with respect to the flat master weights (float64)."""
    wt = torch.as_tensor(np.asarray(w, dtype=np.float64)).clone().requires_grad_(True)
    out = _net(_input(L, R), unpack_tensor(wt))
    lab = torch.as_tensor(np.asarray(label, dtype=np.float64))
    if lab.dim() == 2:
        lab = lab[None]
    valid = torch.isfinite(lab)
    e = torch.where(valid, out - torch.nan_to_num(lab), torch.zeros_like(out))
    loss = torch.where(valid, huber(e), torch.zeros_like(e)).sum() / out.numel()
    loss.backward()
    return float(loss.detach()), wt.grad.numpy().copy()


def unpack_tensor(wt):
    layers, off = [], 0
    for ci, co in CHANNELS:
        n = co * 9 * ci
        W = wt[off:off + n].reshape(co, 3, 3, ci).permute(0, 3, 1, 2)
        off += n
        layers.append((W, wt[off:off + co]))
        off += co
    return layers


def conv_loops(x, W, b, dil):
    """One layer written as loops (for pinning the library convolution)."""
    x = np.asarray(x, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    B, C, H, Wd = x.shape
    co_n = W.shape[0]
    out = np.zeros((B, co_n, H, Wd))
    for n in range(B):
        for co in range(co_n):
            for y in range(H):
                for xx in range(Wd):
                    s = float(b[co])
                    for ci in range(C):
                        for ky in range(3):
                            for kx in range(3):
                                yy, xs = y + (ky - 1) * dil, xx + (kx - 1) * dil
                                if 0 <= yy < H and 0 <= xs < Wd:
                                    s += W[co, ci, ky, kx] * x[n, ci, yy, xs]
                    out[n, co, y, xx] = s
    return out
