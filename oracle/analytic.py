"""Closed forms used to pin the oracle (TEST INFRASTRUCTURE ONLY).

The parallel-beam projection of a uniform disk of value v, radius r and
centre (cx, cy) at angle theta and detector coordinate t is the chord length
times v:  p(theta, t) = 2 v sqrt(r^2 - (t - cx cos theta - cy sin theta)^2)
for |t - cx cos theta - cy sin theta| < r, else 0.  With the detector
convention of the oracle (bin s at t = s - Ns/2, pixel pitch 1, X = q - N/2,
Y = p - N/2, theta from +x towards +y) this is what Radon{x} approaches for a
finely sampled disk (section "fast radon transform"; the object model of
section "Introduction": blocks of uniform material).
"""
from __future__ import annotations

import numpy as np


def disk_projection(angles, n_det, disks):
    """Sum over disks (cx, cy, r, v) of the chord-length projection."""
    t = np.arange(n_det, dtype=np.float64) - n_det // 2
    out = np.zeros((len(angles), n_det))
    for (cx, cy, r, v) in disks:
        c = cx * np.cos(angles)[:, None] + cy * np.sin(angles)[:, None]
        d2 = r * r - (t[None, :] - c) ** 2
        out += 2.0 * v * np.sqrt(np.maximum(d2, 0.0))
    return out
