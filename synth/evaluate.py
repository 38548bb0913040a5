"""Error statistics of a disparity map against ground truth.

The statistics mirror the columns of the paper's Table 1 (median and mean
absolute error over valid pixels, number of valid pixels) and add the bad-1
rate: the fraction of pixels with known ground truth whose estimate is
missing or off by more than 1 px.
"""
from __future__ import annotations

import numpy as np


def error_stats(est: np.ndarray, gt: np.ndarray, bad_px: float = 1.0) -> dict:
    est = np.asarray(est, dtype=np.float64)
    gt = np.asarray(gt, dtype=np.float64)
    known = np.isfinite(gt)
    valid = known & np.isfinite(est)
    err = np.abs(est[valid] - gt[valid])
    n_known = int(known.sum())
    bad = int((~np.isfinite(est[known])).sum() + (err > bad_px).sum())
    return {
        "median_abs": float(np.median(err)) if err.size else float("nan"),
        "mean_abs": float(err.mean()) if err.size else float("nan"),
        "valid": int(valid.sum()),
        "known": n_known,
        "bad1": bad / max(n_known, 1),
    }
