"""Fourier-slice Radon transform and its adjoint, FP64 reference (oracle).

TEST INFRASTRUCTURE ONLY -- never imported by the product path.

The paper (section "fast radon transform") computes Radon{x} in three steps:
a 2D FFT of the image on a regular grid, interpolation of that transform onto
a polar grid (lines through the origin at the projection angles), and a 1D
inverse FFT along every radial line.  The interpolation between the Cartesian
and the polar grid is a "gridding" convolution with a kernel (the paper cites
Jackson et al.), i.e. a non-uniform FFT; the adjoint runs the same steps in
reverse.  This module states that operator twice:

* ``radon_exact_c`` / ``radon_exact_adj_c``: the exact discrete definition --
  the polar spectrum is the direct non-uniform DFT of the image, followed by
  the centred inverse DFT along each ray.  Gridding approximates this.
* ``radon_grid_c`` / ``radon_grid_adj_c``: the gridding approximation, step by
  step in the paper's order: deapodize and zero-pad, oversampled 2D FFT,
  Kaiser-Bessel interpolation onto the polar samples, ray inverse FFT.

Conventions (the paper states none; these are the readings used here and on the GPU):

* image ``x[p, q]``: row ``p`` is the y axis, column ``q`` the x axis; pixel
  coordinates ``X = q - N/2``, ``Y = p - N/2``;
* projection angles ``theta_j = pi j / M`` (uniform on [0, pi), endpoint
  excluded), measured from +x towards +y;
* detector frequencies ``k = -Ns/2 .. Ns/2-1`` (cycles per detector length);
  detector bin ``s = 0 .. Ns-1`` with the centre at ``s = Ns/2``; detector
  pitch = pixel pitch;
* polar spectrum ``P[j,k] = sum_{p,q} x[p,q] exp(-2 pi i (k/Ns)(X cos + Y sin))``;
* ray inverse DFT ``y[j,s] = (1/Ns) sum_k P[j,k] exp(+2 pi i k (s - Ns/2)/Ns)``;
* the real Radon transform is ``Re y``; its adjoint is ``Re(A^H w)``;
* Kaiser-Bessel kernel of width ``W`` (support ``|t| < W/2``) on a grid
  oversampled by ``sigma``, with its edge pedestal removed so that it is
  continuous at the support edge:
  ``g(t) = (I0(beta sqrt(1-(2t/W)^2)) - 1) / (I0(beta) - 1)``,
  ``beta = pi sqrt((W/sigma)^2 (sigma-1/2)^2 - 0.8)`` (Beatty, Nishimura and
  Pauly 2005); deapodization divides by its continuous Fourier transform
  ``ghat(X/G)``; the kernel footprint wraps periodically on the ``G x G`` grid
  (``G = sigma N``).

Parity pins (tests/test_oracle_nufft.py): the exact operator is pinned to
exact column/row sums at theta = 0 and pi/2, to the DC invariant, to the
closed-form projection of disks and to a brute-force pixel loop; the gridding
operator is pinned to the exact one within the kernel's aliasing error and
both satisfy the adjoint identity to 1e-12.
"""
from __future__ import annotations

import math
import os

import numpy as np
import scipy.fft
from scipy import special

# the 2D transforms of the oversampled grid run on every host core (a library
# FFT in FP64; the gridding loops below are plain NumPy)
FFT_WORKERS = os.cpu_count() or 1


def fft2(a):
    """Unnormalised forward 2D DFT (scipy.fft, FP64, all host cores)."""
    return scipy.fft.fft2(a, workers=FFT_WORKERS)


def ifft2(a):
    """Inverse 2D DFT with scipy's 1/(G*G) normalisation (all host cores)."""
    return scipy.fft.ifft2(a, workers=FFT_WORKERS)


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------
def default_angles(n_views: int) -> np.ndarray:
    """theta_j = pi j / M, j = 0..M-1 (uniform on [0, pi), endpoint excluded)."""
    return np.pi * np.arange(n_views, dtype=np.float64) / n_views


def detector_freqs(n_det: int) -> np.ndarray:
    """k = -Ns/2 .. Ns/2 - 1 (Ns even)."""
    return np.arange(-(n_det // 2), n_det - n_det // 2, dtype=np.float64)


def pixel_coords(n: int) -> np.ndarray:
    """X (or Y) = index - N/2 for index 0..N-1."""
    return np.arange(n, dtype=np.float64) - n // 2


# ---------------------------------------------------------------------------
# ray DFTs (the "1D inverse Fourier transforms ... along the same radial
# lines" of section "fast radon transform") -- explicit centred definitions
# ---------------------------------------------------------------------------
def ray_idft(P: np.ndarray) -> np.ndarray:
    """y[j,s] = (1/Ns) sum_k P[j,k] exp(+2 pi i k (s - Ns/2)/Ns).

    ``P[:, kk]`` holds frequency ``k = kk - Ns/2``.  Uses the library FFT as a
    step: with the centred index maps, ifftshift/ifft/fftshift is exactly the
    sum above (pinned against the explicit sum in the tests).
    """
    return np.fft.fftshift(np.fft.ifft(np.fft.ifftshift(P, axes=-1), axis=-1), axes=-1)


def ray_idft_adj(y: np.ndarray) -> np.ndarray:
    """Adjoint of ``ray_idft``: P~[j,k] = (1/Ns) sum_s y[j,s] exp(-2 pi i k (s-Ns/2)/Ns)."""
    ns = y.shape[-1]
    return np.fft.fftshift(np.fft.fft(np.fft.ifftshift(y, axes=-1), axis=-1), axes=-1) / ns


def ray_idft_explicit(P: np.ndarray) -> np.ndarray:
    """The same sum written out as a dense matrix (small Ns only; used as a pin)."""
    ns = P.shape[-1]
    k = detector_freqs(ns)
    s = np.arange(ns, dtype=np.float64)
    E = np.exp(2j * np.pi * np.outer(s - ns // 2, k) / ns) / ns
    return P @ E.T


# ---------------------------------------------------------------------------
# exact operator: direct non-uniform DFT onto the polar grid
# ---------------------------------------------------------------------------
def polar_spectrum_exact(x: np.ndarray, n_det: int, angles: np.ndarray) -> np.ndarray:
    """P[j,k] = sum_{p,q} x[p,q] exp(-2 pi i (k/Ns)(X cos th_j + Y sin th_j)).

    Evaluated per angle as a matrix product; the exponential of a sum is split
    into the product of its X and Y factors (exact).
    """
    n = x.shape[0]
    assert x.shape == (n, n)
    k = detector_freqs(n_det)
    X = pixel_coords(n)
    out = np.empty((len(angles), n_det), dtype=np.complex128)
    xc = x.astype(np.complex128)
    for j, th in enumerate(angles):
        ex = np.exp(-2j * np.pi * np.outer(k, X) * (math.cos(th) / n_det))  # [k, q]
        ey = np.exp(-2j * np.pi * np.outer(k, X) * (math.sin(th) / n_det))  # [k, p]
        out[j] = np.einsum("kq,kq->k", ey @ xc, ex)
    return out


def polar_spectrum_exact_adj(Pt: np.ndarray, n: int, angles: np.ndarray) -> np.ndarray:
    """Adjoint of ``polar_spectrum_exact``:
    z[p,q] = sum_{j,k} Pt[j,k] exp(+2 pi i (k/Ns)(X cos th_j + Y sin th_j))."""
    n_det = Pt.shape[1]
    k = detector_freqs(n_det)
    X = pixel_coords(n)
    z = np.zeros((n, n), dtype=np.complex128)
    for j, th in enumerate(angles):
        ex = np.exp(2j * np.pi * np.outer(k, X) * (math.cos(th) / n_det))  # [k, q]
        ey = np.exp(2j * np.pi * np.outer(k, X) * (math.sin(th) / n_det))  # [k, p]
        z += ey.T @ (Pt[j][:, None] * ex)
    return z


def radon_exact_c(x: np.ndarray, n_det: int, angles: np.ndarray) -> np.ndarray:
    """Complex Fourier-slice Radon transform y = A x (direct NUDFT, exact)."""
    return ray_idft(polar_spectrum_exact(x, n_det, angles))


def radon_exact_adj_c(y: np.ndarray, n: int, angles: np.ndarray) -> np.ndarray:
    """A^H y (exact)."""
    return polar_spectrum_exact_adj(ray_idft_adj(y), n, angles)


def radon_exact(x, n_det, angles):
    """Real Radon transform R x = Re(A x) (exact)."""
    return radon_exact_c(np.asarray(x, np.float64), n_det, angles).real


def radon_exact_adj(w, n, angles):
    """R^T w = Re(A^H w) for real w (exact)."""
    return radon_exact_adj_c(np.asarray(w, np.float64), n, angles).real


def radon_bruteforce_c(x, n_det, angles):
    """Pixel-by-pixel quadruple loop of the same definition (tiny inputs only).

    Used as an independent pin of ``radon_exact_c``: no matrix algebra, no FFT.
    """
    n = x.shape[0]
    ks = detector_freqs(n_det)
    y = np.zeros((len(angles), n_det), dtype=np.complex128)
    for j, th in enumerate(angles):
        c, s_ = math.cos(th), math.sin(th)
        P = np.zeros(n_det, dtype=np.complex128)
        for kk, k in enumerate(ks):
            acc = 0j
            for p in range(n):
                for q in range(n):
                    if x[p, q] != 0:
                        ph = -2 * math.pi * (k / n_det) * ((q - n // 2) * c + (p - n // 2) * s_)
                        acc += x[p, q] * complex(math.cos(ph), math.sin(ph))
            P[kk] = acc
        for s in range(n_det):
            acc = 0j
            for kk, k in enumerate(ks):
                ph = 2 * math.pi * k * (s - n_det // 2) / n_det
                acc += P[kk] * complex(math.cos(ph), math.sin(ph))
            y[j, s] = acc / n_det
    return y


# ---------------------------------------------------------------------------
# Kaiser-Bessel kernel and deapodization (gridding, section "fast radon
# transform"; kernel family of the cited gridding method)
# ---------------------------------------------------------------------------
def kb_beta(width: int = 6, oversamp: float = 2.0) -> float:
    """beta = pi sqrt((W/sigma)^2 (sigma - 1/2)^2 - 0.8)  (Beatty et al. 2005)."""
    return math.pi * math.sqrt((width / oversamp) ** 2 * (oversamp - 0.5) ** 2 - 0.8)


def kb_kernel(t, width: int = 6, beta: float | None = None):
    """g(t) = (I0(beta sqrt(1 - (2t/W)^2)) - 1) / (I0(beta) - 1) on |t| < W/2, else 0.

    The Kaiser-Bessel window with its edge pedestal I0(0) = 1 removed, so that
    g vanishes continuously at |t| = W/2 (reading: the paper names no kernel).
    """
    if beta is None:
        beta = kb_beta(width)
    t = np.asarray(t, dtype=np.float64)
    inside = np.abs(t) < width / 2.0
    arg = np.where(inside, 1.0 - (2.0 * t / width) ** 2, 0.0)
    return np.where(inside, (special.i0(beta * np.sqrt(arg)) - 1.0) / (special.i0(beta) - 1.0), 0.0)


def kb_ft(xi, width: int = 6, beta: float | None = None):
    """Continuous Fourier transform of ``kb_kernel``:
    ghat(xi) = W [sinh(z)/z - sin(pi W xi)/(pi W xi)] / (I0(beta) - 1),
    z = sqrt(beta^2 - (pi W xi)^2) (sin(|z|)/|z| when z^2 < 0); the first term
    transforms the Kaiser-Bessel window, the second the removed pedestal."""
    if beta is None:
        beta = kb_beta(width)
    xi = np.asarray(xi, dtype=np.float64)
    z2 = beta ** 2 - (np.pi * width * xi) ** 2
    out = np.empty_like(xi)
    pos = z2 > 0
    z = np.sqrt(np.abs(z2))
    out[pos] = np.sinh(z[pos]) / z[pos]
    neg = z2 < 0
    out[neg] = np.sin(z[neg]) / z[neg]
    out[z2 == 0] = 1.0
    return width * (out - np.sinc(width * xi)) / (special.i0(beta) - 1.0)


def deapod(n: int, grid: int, width: int = 6, beta: float | None = None) -> np.ndarray:
    """c(X) = 1 / ghat(X / G) for X = -N/2 .. N/2 - 1 (indexed by X + N/2)."""
    return 1.0 / kb_ft(pixel_coords(n) / grid, width, beta)


# ---------------------------------------------------------------------------
# gridding operator, step by step
# ---------------------------------------------------------------------------
class GridGeometry:
    """Sample coordinates of the polar grid on the oversampled Cartesian grid.

    For ray j and frequency k the sample sits at grid coordinates
    ``u = (G/Ns) k cos(theta_j)`` (x frequency) and ``v = (G/Ns) k sin(theta_j)``.
    """

    def __init__(self, n, n_det, angles, width=6, oversamp=2.0):
        self.n, self.n_det, self.width, self.oversamp = n, n_det, width, oversamp
        self.grid = int(round(oversamp * n))
        self.angles = np.asarray(angles, dtype=np.float64)
        self.beta = kb_beta(width, oversamp)
        k = detector_freqs(n_det)
        scale = self.grid / n_det
        cos = np.array([math.cos(t) for t in self.angles])
        sin = np.array([math.sin(t) for t in self.angles])
        self.u = (scale * k)[None, :] * cos[:, None]  # [j, kk]
        self.v = (scale * k)[None, :] * sin[:, None]
        self.cx = deapod(n, self.grid, width, self.beta)

    def taps(self, coord):
        """All integer grid points a with |coord - a| < W/2 and their weights.

        Returns (a, w) of shape coord.shape + (W+1,): the W+1 integers
        floor(coord) - W/2 .. floor(coord) + W/2 contain every point of the open
        support; the kernel gives zero weight to those outside it.
        """
        half = self.width // 2
        base = np.floor(coord)
        offs = np.arange(-half, half + 1, dtype=np.float64)
        a = base[..., None] + offs
        w = kb_kernel(coord[..., None] - a, self.width, self.beta)
        return a.astype(np.int64), w


def grid_deapod_pad(x: np.ndarray, geo: GridGeometry) -> np.ndarray:
    """Step 1: x~[Y, X] = x[p,q] c(X) c(Y), placed at (Y mod G, X mod G)."""
    n, G = geo.n, geo.grid
    xt = np.zeros((G, G), dtype=np.complex128)
    idx = (pixel_coords(n).astype(np.int64)) % G
    xt[np.ix_(idx, idx)] = x * geo.cx[:, None] * geo.cx[None, :]
    return xt


def grid_interp(F: np.ndarray, geo: GridGeometry, rays=None) -> np.ndarray:
    """Step 3: P[j,k] = sum_{a,b} g(u - a) g(v - b) F[b mod G, a mod G]."""
    G = geo.grid
    u = geo.u if rays is None else geo.u[rays]
    v = geo.v if rays is None else geo.v[rays]
    a, wa = geo.taps(u)
    b, wb = geo.taps(v)
    out = np.zeros(u.shape, dtype=np.complex128)
    for ib in range(b.shape[-1]):
        rowsum = np.zeros(u.shape, dtype=np.complex128)
        for ia in range(a.shape[-1]):
            rowsum += wa[..., ia] * F[b[..., ib] % G, a[..., ia] % G]
        out += wb[..., ib] * rowsum
    return out


def grid_spread(Pt: np.ndarray, geo: GridGeometry, rays=None) -> np.ndarray:
    """Adjoint of step 3: Yh[b mod G, a mod G] += g(u - a) g(v - b) Pt[j,k].

    With ``rays`` only those rays' samples are spread (Pt holds just them).
    """
    G = geo.grid
    a, wa = geo.taps(geo.u if rays is None else geo.u[rays])
    b, wb = geo.taps(geo.v if rays is None else geo.v[rays])
    acc_re = np.zeros(G * G)
    acc_im = np.zeros(G * G)
    for ib in range(b.shape[-1]):
        for ia in range(a.shape[-1]):
            w = wb[..., ib] * wa[..., ia]
            flat = ((b[..., ib] % G) * G + (a[..., ia] % G)).ravel()
            val = (w * Pt).ravel()
            acc_re += np.bincount(flat, weights=val.real, minlength=G * G)
            acc_im += np.bincount(flat, weights=val.imag, minlength=G * G)
    return (acc_re + 1j * acc_im).reshape(G, G)


def grid_crop_deapod(z: np.ndarray, geo: GridGeometry) -> np.ndarray:
    """Adjoint of step 1: crop (Y, X) in [-N/2, N/2)^2 and multiply c(X) c(Y)."""
    n, G = geo.n, geo.grid
    idx = (pixel_coords(n).astype(np.int64)) % G
    return z[np.ix_(idx, idx)] * geo.cx[:, None] * geo.cx[None, :]


def polar_spectrum_grid(x: np.ndarray, geo: GridGeometry, rays=None) -> np.ndarray:
    """Steps 1-3: deapodize/pad, unnormalized forward 2D FFT, interpolate."""
    F = fft2(grid_deapod_pad(x, geo))
    return grid_interp(F, geo, rays)


def radon_grid_c(x: np.ndarray, geo: GridGeometry, rays=None) -> np.ndarray:
    """Complex Fourier-slice Radon transform by gridding (steps 1-4)."""
    return ray_idft(polar_spectrum_grid(x, geo, rays))


def radon_grid_adj_c(y: np.ndarray, geo: GridGeometry) -> np.ndarray:
    """A^H y by gridding: ray DFT^H, spread, unnormalized inverse 2D FFT, crop."""
    G = geo.grid
    Yh = grid_spread(ray_idft_adj(y), geo)
    z = ifft2(Yh) * (G * G)
    return grid_crop_deapod(z, geo)


def radon_grid(x, geo, rays=None):
    """Real Radon transform Re(A x) by gridding."""
    return radon_grid_c(np.asarray(x, np.float64), geo, rays).real


def radon_grid_adj(w, geo):
    """Re(A^H w) by gridding, for real w."""
    return radon_grid_adj_c(np.asarray(w, np.float64), geo).real


# ---------------------------------------------------------------------------
# filtered backprojection (baseline reconstruction "using a filter")
# ---------------------------------------------------------------------------
def ramp_weights(n_det: int, n_views: int) -> np.ndarray:
    """Fourier-slice inversion weights h[k] = (pi/M) |k| / Ns, with the DC bin
    given the mean of |k| over its width (1/4 of a bin)."""
    k = np.abs(detector_freqs(n_det))
    k[k == 0] = 0.25
    return (np.pi / n_views) * k / n_det


def ramp_filter(y: np.ndarray, n_views: int) -> np.ndarray:
    """w = ray_idft(h * P) where P = ray DFT of the real sinogram y."""
    ns = y.shape[-1]
    P = ray_idft_adj(y) * ns
    return ray_idft(P * ramp_weights(ns, n_views)[None, :]).real


def fbp_grid(y, geo: GridGeometry):
    """x_fbp = R^T(ramp * y): the polar Fourier inversion integral discretised
    with d(theta) = pi/M and d(rho) = 1/Ns."""
    return radon_grid_adj(ramp_filter(np.asarray(y, np.float64), len(geo.angles)), geo)
