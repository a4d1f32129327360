"""Pins of the preprocessing oracle (background normalization and the
near/far phase-contrast difference, section "Introduction", Fig. 1)."""
import numpy as np

from oracle import preprocess as pp
from paper_1009_1380_gb300 import synth


def _frames(seed=0, m=5, rows=3, ns=16):
    rng = np.random.default_rng(seed)
    dark = rng.uniform(90, 110, (rows, ns))
    flat_n = dark + rng.uniform(2000, 3000, (rows, ns))
    flat_f = dark + rng.uniform(2000, 3000, (rows, ns))
    near = dark[None] + (flat_n - dark)[None] * rng.uniform(0.3, 1.0, (m, rows, ns))
    far = dark[None] + (flat_f - dark)[None] * rng.uniform(0.3, 1.0, (m, rows, ns))
    return near, far, flat_n, flat_f, dark


def test_normalization_identities():
    near, far, flat_n, flat_f, dark = _frames()
    # a frame equal to its flat normalizes to 1, the dark frame to 0
    np.testing.assert_allclose(pp.normalize(flat_n, flat_n, dark), 1.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(pp.normalize(dark, flat_n, dark), 0.0, atol=0)
    # a common gain of frame and flat above the dark level cancels
    g = 1.7
    a = pp.normalize(near[0], flat_n, dark)
    b = pp.normalize(dark + g * (near[0] - dark), dark + g * (flat_n - dark), dark)
    np.testing.assert_allclose(a, b, rtol=1e-14)


def test_dead_reference_pixels_give_zero():
    near, far, flat_n, flat_f, dark = _frames(1)
    flat_n[1, 4] = dark[1, 4]          # dead: no open-beam signal
    flat_f[2, 7] = dark[2, 7] - 5.0    # below the dark level
    s = pp.phase_contrast_sinograms(near, far, flat_n, flat_f, dark)
    assert np.all(np.isfinite(s))
    n_far = pp.normalize(far[:, 1, 4], flat_f[1, 4], dark[1, 4])
    np.testing.assert_allclose(s[1, :, 4], -n_far, rtol=1e-14)
    n_near = pp.normalize(near[:, 2, 7], flat_n[2, 7], dark[2, 7])
    np.testing.assert_allclose(s[2, :, 7], n_near, rtol=1e-14)


def test_equal_frames_and_transpose():
    near, far, flat_n, flat_f, dark = _frames(2)
    s = pp.phase_contrast_sinograms(near, near, flat_n, flat_n, dark)
    assert not s.any()
    s = pp.phase_contrast_sinograms(near, far, flat_n, flat_f, dark)
    assert s.shape == (3, 5, 16)
    for j in range(5):
        for z in range(3):
            ref = (near[j, z] - dark[z]) / (flat_n[z] - dark[z]) - (far[j, z] - dark[z]) / (flat_f[z] - dark[z])
            np.testing.assert_allclose(s[z, j], ref, rtol=1e-13, atol=1e-15)


def test_noise_free_difference_is_the_phase_laplacian():
    """On noise-free synthetic radiographs of spheres the difference of the
    normalized images equals (dz / k) lap(phi) times the transmission, the
    first-order transport-of-intensity term the generator puts in."""
    r = synth.pc_radiographs(n_views=6, n_rows=8, n_det=64, rng=np.random.default_rng(3), noise=False,
                             counts=False)
    s = pp.phase_contrast_sinograms(r["near"], r["far"], r["flat_near"], r["flat_far"], r["dark"])
    np.testing.assert_allclose(s, r["pc_term"].transpose(1, 0, 2), rtol=1e-10, atol=1e-12)


def _pins_hold():
    try:
        test_normalization_identities()
        test_dead_reference_pixels_give_zero()
        test_equal_frames_and_transpose()
        test_noise_free_difference_is_the_phase_laplacian()
    except (AssertionError, FloatingPointError, ValueError):
        return False
    return True


def test_planted_mistakes_fail_the_pins(monkeypatch):
    """Plausible mistakes planted in the preprocessing oracle (on the CPU)
    each fail at least one pin: the dark frame not subtracted from the flat,
    the dark frame not subtracted from the image, far minus near, the
    (angle, row) axes left untransposed."""
    assert _pins_hold()
    norm, pcs = pp.normalize, pp.phase_contrast_sinograms

    def flat_raw(frame, flat, dark):
        f = np.asarray(frame, np.float64)
        return (f - dark) / np.asarray(flat, np.float64)

    def frame_raw(frame, flat, dark):
        den = np.asarray(flat, np.float64) - dark
        return np.where(den > 0, np.asarray(frame, np.float64) / np.where(den > 0, den, 1.0), 0.0)

    def swapped(near, far, flat_near, flat_far, dark):
        return pcs(far, near, flat_far, flat_near, dark)

    def untransposed(near, far, flat_near, flat_far, dark):
        return np.ascontiguousarray(pcs(near, far, flat_near, flat_far, dark).transpose(1, 0, 2))

    for name, attr, fn in [("flat_raw", "normalize", flat_raw), ("frame_raw", "normalize", frame_raw),
                           ("swapped", "phase_contrast_sinograms", swapped),
                           ("untransposed", "phase_contrast_sinograms", untransposed)]:
        with monkeypatch.context() as mp:
            mp.setattr(pp, attr, fn)
            with np.errstate(all="ignore"):
                assert not _pins_hold(), name
    assert pp.normalize is norm and _pins_hold()
