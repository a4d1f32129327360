"""Preprocessing front end, FP64 reference (oracle).

TEST INFRASTRUCTURE ONLY -- never imported by the product path.

Section "Introduction" and Fig. 1: the radiographs of each projection angle
are background normalized, the image taken with the detector at a short
distance from the sample and the one taken 1 m downstream are subtracted
(the difference shows the propagation-based phase contrast, an image of the
Laplacian of the projected phase), and the rows of those difference images
over all angles form the sinograms, one per detector row (slice).

Background normalization (reading; the paper names the step only): the
standard flat-field correction
    n = (I - D) / (F - D)
with I the camera frame, F the open-beam (flat) frame at the same detector
distance and D the dark frame; a reference pixel with F - D <= 0 (dead or
saturated) gives 0.  The phase-contrast sinogram of detector row z:
    sino_z[j, s] = n_near[j, z, s] - n_far[j, z, s].
For a weakly absorbing object the transport-of-intensity equation makes the
downstream image I_far = I_near (1 - (dz / k) lap(phi)) to first order, so
the difference is (dz / k) lap(phi) times the transmission: a sinogram of
the Laplacian of the object's phase (the solver's x).

Parity pins (tests/test_oracle_preprocess.py): the difference vanishes for
equal frames, the normalization maps a frame equal to its flat to 1 and is
invariant to a common gain of frame and flat above the dark level, dead
reference pixels give 0, and the output is the transpose (angle, row) ->
(row, angle) of the per-frame differences.
"""
from __future__ import annotations

import numpy as np


def normalize(frame, flat, dark):
    """(I - D) / (F - D) in FP64, 0 where F - D <= 0."""
    frame = np.asarray(frame, dtype=np.float64)
    den = np.asarray(flat, dtype=np.float64) - np.asarray(dark, dtype=np.float64)
    num = frame - np.asarray(dark, dtype=np.float64)
    out = np.zeros(np.broadcast(num, den).shape)
    ok = np.broadcast_to(den > 0, out.shape)
    q = num / np.where(den > 0, den, 1.0)
    out[ok] = np.broadcast_to(q, out.shape)[ok]
    return out


def phase_contrast_sinograms(near, far, flat_near, flat_far, dark):
    """near, far: (M, rows, Ns) camera frames; flats and dark: (rows, Ns).
    Returns (rows, M, Ns): sino[z, j, s] = n_near[j, z, s] - n_far[j, z, s]."""
    d = normalize(near, flat_near[None], dark[None]) - normalize(far, flat_far[None], dark[None])
    return np.ascontiguousarray(d.transpose(1, 0, 2))
