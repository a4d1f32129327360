"""Pins of the ring filter (cubic column-mean residual projector)."""
import numpy as np

from oracle import ring


def test_projector_properties():
    M, Ns = 5, 12
    F = ring.ring_filter_matrix(M, Ns)
    np.testing.assert_allclose(F @ F, F, atol=1e-13)
    np.testing.assert_allclose(F, F.T, atol=1e-13)
    # rank M*Ns - (Ns - 4): the removed subspace is {1_M (x) c : c orthogonal to cubics}
    assert int(round(np.trace(F))) == M * Ns - (Ns - 4)
    assert np.linalg.matrix_rank(F, tol=1e-9) == M * Ns - (Ns - 4)


def test_annihilates_non_cubic_column_offsets():
    rng = np.random.default_rng(0)
    M, Ns = 7, 32
    c = rng.standard_normal(Ns)
    s = np.arange(Ns, dtype=np.float64)
    # remove the cubic part by an independent least-squares fit (lstsq on raw monomials)
    V = np.stack([s ** d for d in range(4)], axis=1)
    c_perp = c - V @ np.linalg.lstsq(V, c, rcond=None)[0]
    y = np.tile(c_perp, (M, 1))
    assert np.abs(ring.ring_filter(y)).max() < 1e-10


def test_keeps_sinograms_with_cubic_column_means():
    rng = np.random.default_rng(1)
    M, Ns = 9, 40
    s = np.arange(Ns, dtype=np.float64)
    cubic = 0.3 - 0.01 * s + 2e-4 * s ** 2 - 3e-6 * s ** 3
    z = rng.standard_normal((M, Ns))
    z -= z.mean(axis=0, keepdims=True)  # zero column means
    y = z + cubic[None, :]
    np.testing.assert_allclose(ring.ring_filter(y), y, atol=1e-12)


def test_removes_stuck_column_offset_exactly():
    # a stuck column (constant offset over angles) on top of a column-mean-free
    # sinogram is removed up to the cubic trend of that single spike
    M, Ns = 16, 64
    rng = np.random.default_rng(2)
    z = rng.standard_normal((M, Ns))
    z -= z.mean(axis=0, keepdims=True)
    spike = np.zeros(Ns)
    spike[20] = 5.0
    out = ring.ring_filter(z + spike[None, :])
    s = np.arange(Ns, dtype=np.float64)
    V = np.stack([s ** d for d in range(4)], axis=1)
    trend = V @ np.linalg.lstsq(V, spike, rcond=None)[0]
    np.testing.assert_allclose(out, z + trend[None, :], atol=1e-12)


def _pins_hold():
    """The checks of the tests above, as one predicate."""
    try:
        test_projector_properties()
        test_annihilates_non_cubic_column_offsets()
        test_keeps_sinograms_with_cubic_column_means()
        test_removes_stuck_column_offset_exactly()
    except AssertionError:
        return False
    return True


def test_planted_mistakes_fail_the_pins(monkeypatch):
    """Plausible mistakes planted in the filter (on the CPU) each fail at
    least one pin: a quadratic instead of a cubic trend, column sums instead
    of means, the trend removed instead of kept, means over the detector
    instead of over the angles."""
    assert _pins_hold()
    basis, means = ring.cubic_basis, ring.column_means
    mistakes = {
        "quadratic": ("cubic_basis", lambda n: basis(n)[:, :3]),
        "sums": ("column_means", lambda y: y.sum(axis=0)),
        "trend_removed": ("cubic_fit", lambda m: m - basis(m.shape[0]) @ (basis(m.shape[0]).T @ m)),
        "row_means": ("column_means", lambda y: np.resize(y.mean(axis=1), y.shape[1])),
    }
    for name, (attr, fn) in mistakes.items():
        with monkeypatch.context() as mp:
            mp.setattr(ring, attr, fn)
            assert not _pins_hold(), name
    assert ring.column_means is means and _pins_hold()
