"""Ring-artifact filter ("polynomial subtraction"), FP64 reference (oracle).

TEST INFRASTRUCTURE ONLY -- never imported by the product path.

Section "Introduction": defective or miscalibrated detector elements give a
per-detector-column error that is constant over the rotation and shows up as
rings; a 3rd-order polynomial fit is used to smooth the sinogram, and the
constraint of the L1 problem measures the misfit after this filter.  Reading
used here: the filter removes, from every detector column s, the part of the
column mean over angles that a least-squares cubic in s does not explain,

    F y = y - 1_M (m - Pi_3 m),   m[s] = (1/M) sum_j y[j, s],

with Pi_3 the orthogonal projection of a length-Ns vector onto cubics in s.
F is an orthogonal projector (F = F^T = F^2) of rank M Ns - (Ns - 4).

Parity pins (tests/test_oracle_ring.py): F^2 = F and F^T = F to round-off,
F annihilates column-constant sinograms orthogonal to cubics, leaves
sinograms whose column means are cubic unchanged, and its rank matches.
"""
from __future__ import annotations

import numpy as np


def cubic_basis(n_det: int) -> np.ndarray:
    """Orthonormal basis (Ns x 4) of cubics in s on s = 0..Ns-1 (via QR of the
    monomials in the centred, scaled variable t = (s - (Ns-1)/2) / (Ns/2))."""
    s = np.arange(n_det, dtype=np.float64)
    t = (s - (n_det - 1) / 2.0) / (n_det / 2.0)
    V = np.stack([t ** d for d in range(4)], axis=1)
    Q, _ = np.linalg.qr(V)
    return Q


def column_means(y: np.ndarray) -> np.ndarray:
    """m[s] = (1/M) sum_j y[j, s]."""
    return y.mean(axis=0)


def cubic_fit(m: np.ndarray) -> np.ndarray:
    """Pi_3 m: least-squares cubic fit of m over s."""
    Q = cubic_basis(m.shape[0])
    return Q @ (Q.T @ m)


def ring_filter(y: np.ndarray) -> np.ndarray:
    """F y = y - 1_M (m - Pi_3 m)."""
    y = np.asarray(y, dtype=np.float64)
    m = column_means(y)
    return y - (m - cubic_fit(m))[None, :]


def ring_filter_matrix(n_views: int, n_det: int) -> np.ndarray:
    """Dense matrix of F acting on row-major flattened sinograms (tiny sizes)."""
    n = n_views * n_det
    E = np.eye(n)
    return np.stack([ring_filter(E[i].reshape(n_views, n_det)).ravel() for i in range(n)], axis=1)
