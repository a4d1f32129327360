"""The seeded synthetic input generators (shared by the GPU path and the
oracle; they hold none of the method's arithmetic): determinism, support
inside the reconstruction circle, the Laplacian phantom of the phase-contrast
image, the corruption model (1% Gaussian noise, stuck detector columns) and
the view-count mix of the batched workload."""
import numpy as np

from paper_1009_1380_gb300 import synth


def test_seeds_and_phantoms_are_deterministic():
    assert synth.seed_for(2) == synth.SEED_BASE + 2
    assert synth.seed_for(2, 5) == (synth.SEED_BASE + 2) * 10007 + 5
    a = synth.phantom("c1_128")
    b = synth.phantom("c1_128")
    np.testing.assert_array_equal(a, b)
    assert a.shape == (128, 128) and a.dtype == np.float32 and np.isfinite(a).all()
    # different slices of a batched configuration differ
    s0 = synth.phantom("c5_warm512", slice_index=0)
    s1 = synth.phantom("c5_warm512", slice_index=1)
    assert not np.array_equal(s0, s1)


def test_support_inside_the_inscribed_circle():
    rng = np.random.default_rng(3)
    n = 128
    for img in (synth.disk_phantom(n, 5, rng)[0], synth.ellipse_phantom(n, 10, rng)[0]):
        yy, xx = np.mgrid[0:n, 0:n]
        r = np.hypot(yy + 0.5 - n / 2, xx + 0.5 - n / 2)
        assert np.abs(img[r > n / 2 + 1]).max() == 0.0
        assert img.max() > 0.0


def test_laplacian_phantom():
    # the 5-point Laplacian vanishes on constants and on linear ramps away
    # from the border; on a single pixel it is the stencil itself
    c = np.full((9, 9), 3.0)
    assert np.abs(synth.laplacian5(c)[1:-1, 1:-1]).max() == 0.0
    ramp = np.add.outer(np.arange(9.0), 2.0 * np.arange(9.0))
    assert np.abs(synth.laplacian5(ramp)[1:-1, 1:-1]).max() < 1e-12
    e = np.zeros((5, 5))
    e[2, 2] = 1.0
    L = synth.laplacian5(e)
    assert L[2, 2] == -4.0 and L[1, 2] == L[3, 2] == L[2, 1] == L[2, 3] == 1.0 and L.sum() == 0.0
    # the phase-contrast images of the SPGL1 workloads are such Laplacians
    u, _ = synth.ellipse_phantom(64, 6, np.random.default_rng(4))
    assert np.abs(synth.laplacian5(u)).sum() > 0.0


def test_corruption_model():
    rng = np.random.default_rng(5)
    y = np.outer(np.ones(400), np.linspace(0.0, 10.0, 64))
    b, std, cols = synth.corrupt_sinogram(y, rng)
    assert std == 0.01 * 10.0
    assert len(cols) == 8 and len(set(cols.tolist())) == 8
    d = b - y
    others = np.setdiff1d(np.arange(64), cols)
    # Gaussian noise of the stated std on the clean columns
    assert abs(d[:, others].std() / std - 1.0) < 0.05
    assert abs(d[:, others].mean()) < 0.05 * std
    # each stuck column carries one constant offset within +-0.2 max
    for c in cols:
        off = d[:, c].mean()
        assert abs(off) <= 0.2 * 10.0 + 5 * std / np.sqrt(400)
        assert abs((d[:, c] - off).std() / std - 1.0) < 0.2


def test_batch_view_mix():
    v = synth.views_for_batch("c3_batch1024")
    assert len(v) == 256
    assert set(np.unique(v).tolist()) <= {64, 128, 256, 512}
    assert len(np.unique(v)) == 4
    np.testing.assert_array_equal(v, synth.views_for_batch("c3_batch1024"))
