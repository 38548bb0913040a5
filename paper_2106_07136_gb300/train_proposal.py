"""Train the learned coarse proposal on the GPU with the library's kernels.

  python -m paper_2106_07136_gb300.train_proposal [--pairs 50000] [--batch 64] [--epochs 4]
         [--out paper_2106_07136_gb300/weights/proposal.bdisnet]

Each step draws a batch of seeded surgical-like 640x480 pairs on the device
(synth.stereo_torch), builds their pyramid with the library's kernels, and
takes one Adam step of the network on the proposal level (the level the
learned start runs it on, `proposal_level(coarsest_scale)`: level 4 at the
paper's 5 scales). The labels come from the generator and the plain method:
the ground-truth disparity at that level (every 2^l-th pixel, divided by
2^l) where it exists, and where it does not (pixels occluded in the right
view) the plain method's own map of that level, searched from the coarsest
level down with the paper's settings by the same kernels (`--labels gt`
keeps the ground truth alone). The forward pass, backward pass and optimiser
all run in libbdis.so.
"""
from __future__ import annotations

import argparse
import math
import os
import sys
import time

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_2106_07136_gb300 as bd  # noqa: E402
from synth.stereo_torch import TorchCfg2Generator  # noqa: E402

DEFAULT_OUT = os.path.join(HERE, "weights", "proposal.bdisnet")
TRAIN_SEED = 7_000_000  # disjoint from the evaluation seeds (2106_07136 + ...)


def level_planes(L, R, level):
    Lp, Rp, _ = bd.prepare_level0(L, R)
    for _ in range(level):
        Lp, Rp, _ = bd.pyramid_level(Lp, Rp)
    return Lp, Rp


def plain_level(L, R, params, level):
    """The plain method's dense map at `level` (coarse to fine from the
    coarsest level), with every pixel estimated or carried (not the finest
    level), by the library's step kernels."""
    Lp, Rp, Gp = bd.prepare_level0(L, R)
    planes = {0: (Lp, Rp, Gp)}
    for lvl in range(1, params.coarsest_scale + 1):
        Lp, Rp, Gp = bd.pyramid_level(Lp, Rp)
        planes[lvl] = (Lp, Rp, Gp)
    coarse = None
    for lvl in range(params.coarsest_scale, level - 1, -1):
        Lp, Rp, Gp = planes[lvl]
        s = bd.search_level(Lp, Rp, Gp, coarse, params, debug=False)
        coarse = bd.densify_level(tuple(Lp.shape[1:]), params, s["d_star"], s["weight"], coarse,
                                  False, Lp, Rp)
    return coarse


def train(pairs=50000, batch=64, lr=2e-3, lr_end=1e-4, seed=0, log_every=100, device="cuda",
          epochs=1, labels="gt+plain"):
    """`epochs` passes over the same `pairs` seeded pairs, one cosine schedule.
    labels: "gt+plain" (ground truth, the plain method where it has none) or "gt"."""
    gen = TorchCfg2Generator(device=device)
    net = bd.ProposalNet(bd.net_init_weights(seed=seed))
    params = bd.default_params()
    level = bd.proposal_level(params.coarsest_scale)
    f = 1 << level
    per_epoch = max(1, pairs // batch)
    steps = per_epoch * max(1, epochs)
    hist = []
    t0 = time.perf_counter()
    for s in range(steps):
        L, R, gt = gen.batch(TRAIN_SEED + s % per_epoch, batch)
        Ll, Rl = level_planes(L, R, level)
        label = (gt[:, ::f, ::f] / float(f)).contiguous()
        if labels == "gt+plain":
            label = torch.where(torch.isfinite(label), label, plain_level(L, R, params, level))
        frac = s / max(steps - 1, 1)
        rate = lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * frac))
        loss = net.train_step(Ll, Rl, label, rate)
        hist.append(loss)
        if log_every and (s % log_every == 0 or s == steps - 1):
            print(f"step {s:5d}/{steps} loss {loss:.4f} lr {rate:.2e} "
                  f"{time.perf_counter() - t0:.1f}s", flush=True)
    w = net.weights()
    net.close()
    return w, hist, time.perf_counter() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=50000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--labels", choices=["gt+plain", "gt"], default="gt+plain")
    a = ap.parse_args()
    w, hist, secs = train(a.pairs, a.batch, a.lr, epochs=a.epochs, labels=a.labels)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    lv = bd.proposal_level(bd.default_params().coarsest_scale)
    what = (f"level-{lv} ground truth, the plain method's level-{lv} map where the ground truth "
            "has none" if a.labels == "gt+plain" else f"level-{lv} ground truth")
    note = (f"trained on {a.pairs} seeded 640x480 surgical-like pairs (seeds from {TRAIN_SEED}), "
            f"{a.epochs} epoch(s), batch {a.batch}, Adam lr {a.lr} cosine to 1e-4, Huber loss on "
            f"{what}; final loss {hist[-1]:.4f}, {secs:.1f}s")
    bd.save_net_weights(a.out, w, note)
    print(note)


if __name__ == "__main__":
    main()
