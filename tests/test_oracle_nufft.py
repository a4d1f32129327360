"""Pins of the FP64 Radon/NUFFT oracle against facts fixed by the mathematics.

Each test pins a different part of the oracle so that a plausible mistake (a
dropped term, a wrong sign, a transposed operand, a wrong centre) fails one:

* brute-force pixel loop          -> the exact operator's matrix algebra
* explicit ray DFT sum            -> the centred FFT index maps
* theta = 0 / pi/2 sums           -> orientation, centre, sign convention
* DC invariant                    -> ray normalisation 1/Ns
* closed-form disk projection     -> scale (1 px = 1 unit) and geometry
* adjoint identity (1e-12)        -> every adjoint
* quadrature of the kernel        -> the Kaiser-Bessel Fourier transform
* exact vs gridding (1e-4)        -> deapodization, taps, oversampled FFT
* planted mistakes                -> that pin fails for each of them
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import analytic, nufft
from paper_1009_1380_gb300 import synth


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def test_exact_matches_bruteforce_loop():
    rng = np.random.default_rng(1)
    n, ns, m = 8, 8, 6
    x = rng.standard_normal((n, n))
    th = nufft.default_angles(m)
    y1 = nufft.radon_exact_c(x, ns, th)
    y2 = nufft.radon_bruteforce_c(x, ns, th)
    assert _rel(y1, y2) < 1e-12
    # detector longer than the image, irregular angles
    th2 = np.array([0.1, 0.7, 1.3, 2.9])
    assert _rel(nufft.radon_exact_c(x, 12, th2), nufft.radon_bruteforce_c(x, 12, th2)) < 1e-12


def test_ray_idft_index_maps():
    rng = np.random.default_rng(2)
    P = rng.standard_normal((3, 16)) + 1j * rng.standard_normal((3, 16))
    assert _rel(nufft.ray_idft(P), nufft.ray_idft_explicit(P)) < 1e-13
    y = rng.standard_normal((3, 16)) + 1j * rng.standard_normal((3, 16))
    # adjoint of the explicit matrix
    lhs = np.vdot(nufft.ray_idft_explicit(P), y)
    rhs = np.vdot(P, nufft.ray_idft_adj(y))
    assert abs(lhs - rhs) / abs(lhs) < 1e-13


def test_special_angles_give_column_and_row_sums():
    rng = np.random.default_rng(3)
    n = 32
    x = rng.standard_normal((n, n))
    th = nufft.default_angles(8)  # contains 0 and pi/2 (j = 4)
    y = nufft.radon_exact_c(x, n, th)
    np.testing.assert_allclose(y[0].real, x.sum(axis=0), rtol=0, atol=1e-11)
    np.testing.assert_allclose(y[4].real, x.sum(axis=1), rtol=0, atol=1e-11)
    assert np.abs(y[0].imag).max() < 1e-11
    # theta = pi/4 pins the sign of the sin term: a single pixel at (X, Y) =
    # (3, 5) projects to t = (3 + 5)/sqrt(2) ~ 5.66, i.e. the band-limited
    # profile peaks at bin Ns/2 + 6 (the pixel at (3, -5) would peak at -1)
    e = np.zeros((n, n))
    e[n // 2 + 5, n // 2 + 3] = 1.0
    yp = nufft.radon_exact(e, n, np.array([math.pi / 4]))
    assert int(np.argmax(yp[0])) == n // 2 + 6


def test_dc_invariant():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((16, 16))
    th = nufft.default_angles(10)
    y = nufft.radon_exact(x, 16, th)
    np.testing.assert_allclose(y.sum(axis=1), np.full(10, x.sum()), rtol=1e-12)


def test_disk_closed_form_projection():
    n = 128
    th = nufft.default_angles(180)
    rng = synth.rng_for(0)
    img, disks = synth.disk_phantom(n, 1, rng)
    cx, cy, r, v = disks[0]
    y = nufft.radon_exact(img, n, th)
    ya = analytic.disk_projection(th, n, disks)
    t = np.arange(n) - n // 2
    c = cx * np.cos(th)[:, None] + cy * np.sin(th)[:, None]
    interior = np.abs(t[None, :] - c) < r - 1.5
    err = np.linalg.norm((y - ya)[interior]) / np.linalg.norm(ya[interior])
    assert err < 0.03, err
    # centre of each profile (first moment above half maximum) sits at the
    # projected disk centre: pins the orientation of both axes
    hm = y > 0.5 * y.max(axis=1, keepdims=True)
    centre = (np.where(hm, y, 0) * t[None, :]).sum(1) / np.where(hm, y, 0).sum(1)
    assert np.all(np.abs(centre - c[:, 0]) <= 0.5)
    # the full five-disk phantom of the 128 x 128 workload
    img5, disks5 = synth.disk_phantom(n, 5, synth.rng_for(0))
    y5 = nufft.radon_exact(img5, n, th)
    ya5 = analytic.disk_projection(th, n, disks5)
    assert _rel(y5, ya5) < 0.03


@pytest.mark.parametrize("which", ["exact", "grid"])
def test_adjoint_identity(which):
    rng = np.random.default_rng(5)
    n, ns, m = 24, 24, 14
    th = nufft.default_angles(m)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    y = rng.standard_normal((m, ns)) + 1j * rng.standard_normal((m, ns))
    if which == "exact":
        Ax = nufft.radon_exact_c(x, ns, th)
        Ahy = nufft.radon_exact_adj_c(y, n, th)
    else:
        geo = nufft.GridGeometry(n, ns, th)
        Ax = nufft.radon_grid_c(x, geo)
        Ahy = nufft.radon_grid_adj_c(y, geo)
    lhs, rhs = np.vdot(y, Ax), np.vdot(Ahy, x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12
    # real operator pair
    xr, wr = x.real, y.real
    if which == "exact":
        Rx, Rtw = nufft.radon_exact(xr, ns, th), nufft.radon_exact_adj(wr, n, th)
    else:
        Rx, Rtw = nufft.radon_grid(xr, geo), nufft.radon_grid_adj(wr, geo)
    l2, r2 = float(np.sum(Rx * wr)), float(np.sum(xr * Rtw))
    assert abs(l2 - r2) / abs(l2) < 1e-12


def test_kb_fourier_transform_by_quadrature():
    W = 6
    beta = nufft.kb_beta(W, 2.0)
    assert nufft.kb_kernel(0.0, W, beta) == pytest.approx(1.0)
    assert nufft.kb_kernel(3.0, W, beta) == 0.0  # support edge
    assert nufft.kb_kernel(3.0 - 1e-9, W, beta) < 1e-11  # continuous there (no pedestal)
    for xi in [0.0, 0.05, 0.125, 0.2, 0.25, 0.4]:
        val, _ = integrate.quad(lambda t: float(nufft.kb_kernel(t, W, beta)) * math.cos(2 * math.pi * xi * t),
                                -3, 3, limit=200, epsabs=1e-14, epsrel=1e-13)
        assert float(nufft.kb_ft(xi, W, beta)) == pytest.approx(val, rel=1e-9, abs=1e-13)


def test_taps_cover_open_support():
    geo = nufft.GridGeometry(16, 16, nufft.default_angles(4))
    coords = np.array([0.0, 0.5, -2.999, 7.25, -8.0, 3.0 - 1e-12])
    a, w = geo.taps(coords)
    for c, aa, ww in zip(coords, a, w):
        need = [k for k in range(int(math.floor(c)) - 4, int(math.floor(c)) + 5) if abs(c - k) < 3]
        got = [int(k) for k, wk in zip(aa, ww) if wk > 0]
        assert got == need


@pytest.mark.parametrize("n,m", [(32, 45), (128, 180)])
def test_grid_matches_exact(n, m):
    th = nufft.default_angles(m)
    if n == 128:
        img, _ = synth.disk_phantom(n, 5, synth.rng_for(0))
    else:
        img = np.random.default_rng(6).standard_normal((n, n))
    geo = nufft.GridGeometry(n, n, th)
    ye = nufft.radon_exact_c(img, n, th)
    yg = nufft.radon_grid_c(img, geo)
    err = _rel(yg, ye)
    # Kaiser-Bessel W = 6, sigma = 2 aliasing error is ~1e-6..1e-5
    assert err < 1e-4, err
    w = np.random.default_rng(7).standard_normal((m, n))
    ae = nufft.radon_exact_adj(w, n, th)
    ag = nufft.radon_grid_adj(w, geo)
    assert _rel(ag, ae) < 1e-4


def test_grid_rays_subset_matches_full():
    n, m = 32, 12
    geo = nufft.GridGeometry(n, n, nufft.default_angles(m))
    x = np.random.default_rng(8).standard_normal((n, n))
    full = nufft.radon_grid(x, geo)
    rays = np.array([0, 5, 11])
    np.testing.assert_allclose(nufft.radon_grid(x, geo, rays), full[rays], rtol=0, atol=1e-12)


def test_fbp_recovers_disk_value():
    n, m = 128, 180
    th = nufft.default_angles(m)
    img, disks = synth.disk_phantom(n, 3, synth.rng_for(0))
    geo = nufft.GridGeometry(n, n, th)
    rec = nufft.fbp_grid(nufft.radon_grid(img, geo), geo)
    X = np.arange(n) - n // 2
    for (cx, cy, r, v) in disks:
        mask = (X[None, :] - cx) ** 2 + (X[:, None] - cy) ** 2 < (r - 3) ** 2
        assert abs(rec[mask].mean() - v) / v < 0.05


@pytest.mark.parametrize("mistake", ["no_deapod", "swapped_axes", "tap_shift", "fft_sign", "spread_one_axis"])
def test_planted_mistakes_fail_the_gridding_pin(monkeypatch, mistake):
    """A plausible mistake planted in the gridding oracle (on the CPU) makes
    it miss the exact operator by far more than the 1e-4 the pin allows:
    the deapodization left out, the u and v axes swapped, the taps shifted by
    one grid point, the forward 2D FFT of the wrong sign, the spread weighting
    by one axis only (adjoint)."""
    n, m = 32, 45
    th = nufft.default_angles(m)
    img = np.random.default_rng(6).standard_normal((n, n))
    w = np.random.default_rng(7).standard_normal((m, n))
    geo = nufft.GridGeometry(n, n, th)
    if mistake == "no_deapod":
        geo.cx = np.ones_like(geo.cx)
    elif mistake == "swapped_axes":
        geo.u, geo.v = geo.v.copy(), geo.u.copy()
    elif mistake == "tap_shift":
        taps = geo.taps
        monkeypatch.setattr(geo, "taps", lambda c: (lambda a, wt: (a + 1, wt))(*taps(c)))
    elif mistake == "fft_sign":
        G = geo.grid
        monkeypatch.setattr(nufft, "fft2", lambda a: nufft.ifft2(a) * (G * G))
    elif mistake == "spread_one_axis":
        def spread(Pt, g, rays=None):
            G = g.grid
            a, wa = g.taps(g.u)
            b, _ = g.taps(g.v)
            out = np.zeros(G * G, dtype=np.complex128)
            for ib in range(b.shape[-1]):
                for ia in range(a.shape[-1]):
                    np.add.at(out, ((b[..., ib] % G) * G + (a[..., ia] % G)).ravel(), (wa[..., ia] * Pt).ravel())
            return out.reshape(G, G)
        monkeypatch.setattr(nufft, "grid_spread", spread)
    if mistake == "spread_one_axis":
        err = _rel(nufft.radon_grid_adj(w, geo), nufft.radon_exact_adj(w, n, th))
    else:
        err = _rel(nufft.radon_grid_c(img, geo), nufft.radon_exact_c(img, n, th))
    print(mistake, err)
    assert err > 1e-2, (mistake, err)
