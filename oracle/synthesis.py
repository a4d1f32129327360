"""FP64 reference of the finite-difference synthesis operator (the
analysis-l1 variant of the solve).

Test infrastructure only (like the rest of ``oracle/``): the product path
never imports it.

The paper minimises the l1 norm of the phase-contrast image itself, which is
sparse because it is a Laplacian of the object (section "Introduction"); the
l1 problem is solved by SPGL1 with the Radon operator and its adjoint.  Its
Conclusions point to total-variation regularisation, l1 of the object's
gradient.  The variant here puts the l1 norm on the horizontal finite
differences of a piecewise-constant image u instead, through an invertible
synthesis operator:

    z = D_h u:   z[p, 0] = u[p, 0],   z[p, q] = u[p, q] - u[p, q - 1]
    u = C z:     u[p, q] = sum_{q' <= q} z[p, q']          (C = D_h^{-1})
    C^T w:       (C^T w)[p, q] = sum_{q' >= q} w[p, q']

(p = row, q = column of the N x N image, row-major).  The solve is
min ||z||_1 subject to ||F(R C z) - F b||_2 <= sigma, and u = C z.
"""
from __future__ import annotations

import numpy as np


def synth_dh(z: np.ndarray) -> np.ndarray:
    """u = C z: cumulative sum along every row."""
    return np.cumsum(np.asarray(z, dtype=np.float64), axis=-1)


def synth_dh_adj(w: np.ndarray) -> np.ndarray:
    """C^T w: cumulative sum from the end of every row."""
    w = np.asarray(w, dtype=np.float64)
    return np.cumsum(w[..., ::-1], axis=-1)[..., ::-1]


def diff_h(u: np.ndarray) -> np.ndarray:
    """z = D_h u: first column kept, then differences along every row."""
    u = np.asarray(u, dtype=np.float64)
    z = u.copy()
    z[..., 1:] = u[..., 1:] - u[..., :-1]
    return z
