"""Pins of the FP64 finite-difference synthesis operator (oracle/synthesis.py)
against things other than itself:

* D_h inverts C exactly on integers (and to round-off on reals), and C
  inverts D_h;
* C and C^T are adjoint: <C z, w> = <z, C^T w>;
* impulse responses in closed form: C of a unit impulse at (p, q0) is the
  step 1[q >= q0] in row p; C^T of it is 1[q <= q0] in row p;
* a planted mistake (C^T taken as the forward cumulative sum) fails the
  adjoint pin.
"""
import numpy as np

from oracle import synthesis as sy


def test_inverse_pairs():
    rng = np.random.default_rng(1)
    zi = rng.integers(-50, 50, size=(7, 33)).astype(np.float64)
    np.testing.assert_array_equal(sy.diff_h(sy.synth_dh(zi)), zi)
    np.testing.assert_array_equal(sy.synth_dh(sy.diff_h(zi)), zi)
    z = rng.standard_normal((5, 64))
    np.testing.assert_allclose(sy.diff_h(sy.synth_dh(z)), z, rtol=0, atol=1e-12)


def test_adjoint_identity():
    rng = np.random.default_rng(2)
    z = rng.standard_normal((16, 16))
    w = rng.standard_normal((16, 16))
    lhs = float(np.sum(sy.synth_dh(z) * w))
    rhs = float(np.sum(z * sy.synth_dh_adj(w)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_impulse_responses():
    n, p, q0 = 12, 4, 5
    e = np.zeros((n, n))
    e[p, q0] = 1.0
    step = np.zeros((n, n))
    step[p, q0:] = 1.0
    np.testing.assert_array_equal(sy.synth_dh(e), step)
    back = np.zeros((n, n))
    back[p, :q0 + 1] = 1.0
    np.testing.assert_array_equal(sy.synth_dh_adj(e), back)


def test_planted_mistake_is_caught():
    rng = np.random.default_rng(3)
    z = rng.standard_normal((8, 8))
    w = rng.standard_normal((8, 8))
    lhs = float(np.sum(sy.synth_dh(z) * w))
    wrong = float(np.sum(z * sy.synth_dh(w)))  # C instead of C^T
    assert abs(lhs - wrong) > 1e-3 * abs(lhs)
