"""Where the search kernel's time goes: one level's search at several iteration caps.

    python -m paper_2106_07136_gb300.search_sweep [--batch 32] [--caps 0,1,2,3,12] [--no-time]

Builds the level-0 inputs of `batch` seeded 640x480 surgical-like pairs with
the library's own stages (pyramid, then search and densify from the coarsest
level down to level 1), then launches the level-0 search once per cap, in
order, with debug outputs off. With timing on it then times each cap (20
launches after 3 warm-up ones, CUDA events, warm L2) and prints the mean
update count per patch at the full cap.

Under a profiler, the launches to capture are the `len(caps)` search
launches after the first (coarsest_scale - finest_scale) ones: the cap 0
launch is the fixed part (set-up, window, tests), and each further cap adds
one update per patch still moving.
"""
import argparse

import numpy as np
import torch

import synth
from . import api as bd


def level0_inputs(batch, params, device):
    left, right, _ = synth.make_batch(2, batch)
    to = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(device)
    L0, R0, G0 = bd.prepare_level0(to(left), to(right))
    levels = [(L0, R0, G0)]
    for _ in range(params.coarsest_scale):
        levels.append(bd.pyramid_level(levels[-1][0], levels[-1][1]))
    coarse = None
    for lvl in range(params.coarsest_scale, 0, -1):
        L, R, G = levels[lvl]
        s = bd.search_level(L, R, G, coarse, params, debug=False)
        coarse = bd.densify_level(L.shape[1:], params, s["d_star"], s["weight"], coarse, False)
    torch.cuda.synchronize(device)
    return levels[0], coarse


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--caps", default="0,1,2,3,12")
    ap.add_argument("--no-time", action="store_true", help="launch each cap once, no timing")
    args = ap.parse_args(argv)
    device = torch.device("cuda", torch.cuda.current_device())
    kw = dict(patch_size=8, overlap=0.75, iterations=12, coarsest_scale=4, finest_scale=0,
              gamma=0.75)
    (L, R, G), coarse = level0_inputs(args.batch, bd.default_params(**kw), device)
    caps = [int(c) for c in args.caps.split(",")]
    per_cap = [bd.default_params(**dict(kw, iterations=c)) for c in caps]
    for p in per_cap:
        bd.search_level(L, R, G, coarse, p, debug=False)
    torch.cuda.synchronize(device)
    if args.no_time:
        return 0
    for cap, p in zip(caps, per_cap):
        for _ in range(3):
            bd.search_level(L, R, G, coarse, p, debug=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            bd.search_level(L, R, G, coarse, p, debug=False)
        e1.record()
        torch.cuda.synchronize(device)
        print(f"cap {cap}: {e0.elapsed_time(e1) / 20 * 1e3:.1f} us per launch (warm L2)")
    steps = bd.search_level(L, R, G, coarse, bd.default_params(**kw), debug=True)["steps"]
    print(f"mean updates per patch at {kw['iterations']}: {float(steps.float().mean()):.3f}")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
