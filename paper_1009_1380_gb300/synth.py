"""Seeded synthetic inputs shaped like the beamline data of the paper.

This module holds only input generation (random shapes, noise, detector
defects); none of the method's arithmetic lives here.  Both the CUDA path's
tests/benchmarks and the CPU oracle take their inputs from it.

The paper's data (60 micron glass spheres at 1.8 micron voxels, section
"Introduction") are not available; piecewise-constant disk and ellipse
phantoms stand in for them:

* disks:    radii 8-20 px, values U[0.5, 1], non-overlapping, inside the
            inscribed circle, pixel value = covered area fraction (4x4
            super-sampling);
* ellipses: semi-axes U[20, 200] px (scaled with N), orientation U[0, pi),
            values U[0.5, 1], overlaps summed, inside the inscribed circle;
* phase-contrast image: 5-point discrete Laplacian of such a phantom (the
            measured quantity is the Laplacian of the phase, section
            "Introduction"), which is sparse;
* sinogram defects: Gaussian noise of standard deviation 1% of the clean
            sinogram's maximum plus 8 "stuck" detector columns carrying a
            constant offset U[-0.2, 0.2] x max over all angles (ring artifacts).

Seeds: configuration c uses seed 1009 + c; slice i of a batch uses
(1009 + c) * 10007 + i.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 1009


def seed_for(config_index: int, slice_index: int | None = None) -> int:
    s = SEED_BASE + config_index
    return s if slice_index is None else s * 10007 + slice_index


def rng_for(config_index: int, slice_index: int | None = None) -> np.random.Generator:
    return np.random.default_rng(seed_for(config_index, slice_index))


# named workloads (sizes of the five benchmark configurations)
CONFIGS = {
    "c1_128": dict(index=0, n=128, n_det=128, n_views=180, kind="disks", n_shapes=5),
    "c2_2048": dict(index=1, n=2048, n_det=2048, n_views=1024, kind="ellipses", n_shapes=40),
    "c3_batch1024": dict(index=2, n=1024, n_det=1024, views_choices=(64, 128, 256, 512),
                         batch=256, kind="ellipses", n_shapes=20),
    "c4_spgl1_1024": dict(index=3, n=1024, n_det=1024, n_views=128, batch=64,
                          kind="laplacian", n_shapes=20, iterations=300),
    "c5_warm512": dict(index=4, n=512, n_det=512, n_views=90, kind="laplacian", n_shapes=12),
    # the size of the paper's own timing (1024 x 1024 grid, 180 angles x 1024
    # pixels per angle, section "fast radon transform")
    "paper_1024": dict(index=5, n=1024, n_det=1024, n_views=180, kind="ellipses", n_shapes=20),
}


def _coverage(n, inside_fn, ss=4, bbox=None):
    """Fraction of each pixel covered by a shape (ss x ss sub-samples).

    ``bbox`` = (xmin, xmax, ymin, ymax) in pixel coordinates limits the work
    to the pixels that can be covered.
    """
    off = (np.arange(ss) + 0.5) / ss - 0.5
    img = np.zeros((n, n))
    q0, q1, p0, p1 = 0, n, 0, n
    if bbox is not None:
        q0 = max(0, int(math.floor(bbox[0])) + n // 2 - 1)
        q1 = min(n, int(math.ceil(bbox[1])) + n // 2 + 2)
        p0 = max(0, int(math.floor(bbox[2])) + n // 2 - 1)
        p1 = min(n, int(math.ceil(bbox[3])) + n // 2 + 2)
    Xq = np.arange(q0, q1, dtype=np.float64) - n // 2
    Yp = np.arange(p0, p1, dtype=np.float64) - n // 2
    acc = np.zeros((p1 - p0, q1 - q0))
    for dy in off:
        for dx in off:
            acc += inside_fn(Xq[None, :] + dx, Yp[:, None] + dy)
    img[p0:p1, q0:q1] = acc / (ss * ss)
    return img


def disk_phantom(n: int, n_disks: int, rng: np.random.Generator,
                 r_range=(8.0, 20.0), v_range=(0.5, 1.0), max_tries=10000):
    """Non-overlapping disks; returns (image float64, [(cx, cy, r, v), ...])."""
    R_in = n / 2 - 2.0
    disks = []
    tries = 0
    while len(disks) < n_disks and tries < max_tries:
        tries += 1
        r = rng.uniform(*r_range)
        rho = (R_in - r) * math.sqrt(rng.uniform())
        phi = rng.uniform(0, 2 * math.pi)
        cx, cy = rho * math.cos(phi), rho * math.sin(phi)
        if all((cx - d[0]) ** 2 + (cy - d[1]) ** 2 > (r + d[2] + 1.0) ** 2 for d in disks):
            disks.append((cx, cy, r, rng.uniform(*v_range)))
    img = np.zeros((n, n))
    for (cx, cy, r, v) in disks:
        box = _coverage(n, lambda X, Y, cx=cx, cy=cy, r=r: ((X - cx) ** 2 + (Y - cy) ** 2 < r * r),
                        bbox=(cx - r, cx + r, cy - r, cy + r))
        img += v * box
    return img, disks


def ellipse_phantom(n: int, n_shapes: int, rng: np.random.Generator,
                    axes_range=(20.0, 200.0), v_range=(0.5, 1.0), ss=2):
    """Random ellipses (overlaps summed) inside the inscribed circle.

    Semi-axes are drawn from ``axes_range`` scaled by n / 2048.
    """
    scale = n / 2048.0
    R_in = n / 2 - 2.0
    img = np.zeros((n, n))
    shapes = []
    for _ in range(n_shapes):
        a = max(2.0, rng.uniform(*axes_range) * scale)
        b = max(2.0, rng.uniform(*axes_range) * scale)
        a, b = min(a, 0.45 * R_in), min(b, 0.45 * R_in)
        ang = rng.uniform(0, math.pi)
        rho = (R_in - max(a, b)) * math.sqrt(rng.uniform())
        phi = rng.uniform(0, 2 * math.pi)
        cx, cy = rho * math.cos(phi), rho * math.sin(phi)
        v = rng.uniform(*v_range)
        ca, sa = math.cos(ang), math.sin(ang)

        def inside(X, Y, cx=cx, cy=cy, a=a, b=b, ca=ca, sa=sa):
            xr = (X - cx) * ca + (Y - cy) * sa
            yr = -(X - cx) * sa + (Y - cy) * ca
            return (xr / a) ** 2 + (yr / b) ** 2 < 1.0

        ext = max(a, b)
        img += v * _coverage(n, inside, ss, bbox=(cx - ext, cx + ext, cy - ext, cy + ext))
        shapes.append((cx, cy, a, b, ang, v))
    return img, shapes


def laplacian5(u: np.ndarray) -> np.ndarray:
    """5-point discrete Laplacian with zero outside the image."""
    p = np.pad(u, 1)
    return p[:-2, 1:-1] + p[2:, 1:-1] + p[1:-1, :-2] + p[1:-1, 2:] - 4.0 * u


def phantom(config: str, slice_index: int | None = None, dtype=np.float32):
    """Image of a named configuration (one slice)."""
    c = CONFIGS[config]
    rng = rng_for(c["index"], slice_index)
    n = c["n"]
    if c["kind"] == "disks":
        img, _ = disk_phantom(n, c["n_shapes"], rng)
    elif c["kind"] == "ellipses":
        img, _ = ellipse_phantom(n, c["n_shapes"], rng)
    else:
        u, _ = ellipse_phantom(n, c["n_shapes"], rng)
        img = laplacian5(u)
    return img.astype(dtype)


def views_for_batch(config: str = "c3_batch1024") -> np.ndarray:
    """Per-slice view counts, uniform over the configuration's choices."""
    c = CONFIGS[config]
    rng = rng_for(c["index"])
    return rng.choice(np.asarray(c["views_choices"]), size=c["batch"])


def corrupt_sinogram(y_clean: np.ndarray, rng: np.random.Generator,
                     noise_frac=0.01, n_stuck=8, stuck_frac=0.2):
    """Add Gaussian noise (std = noise_frac * max) and stuck-column offsets.

    Returns (y_noisy, noise_std, stuck_columns).
    """
    y = np.asarray(y_clean, dtype=np.float64)
    ymax = float(np.abs(y).max())
    std = noise_frac * ymax
    out = y + rng.normal(0.0, std, size=y.shape)
    cols = rng.choice(y.shape[1], size=n_stuck, replace=False)
    offs = rng.uniform(-stuck_frac, stuck_frac, size=n_stuck) * ymax
    out[:, cols] += offs[None, :]
    return out, std, np.sort(cols)


def random_sinogram(n_views: int, n_det: int, rng: np.random.Generator, dtype=np.float32):
    """Dense random test vector in sinogram space (for adjoint tests)."""
    return rng.standard_normal((n_views, n_det)).astype(dtype)


def pc_radiographs(n_views: int, n_rows: int, n_det: int, rng: np.random.Generator, n_spheres: int = 6,
                   noise: bool = True, counts: bool = True, contrast: float = 0.05, i0: float = 20000.0):
    """Synthetic near/far radiographs of a stack of spheres (input generation
    for the preprocessing front end; the paper's Fig. 1 shows such frames of
    two glass balls).

    Spheres (radius R, centre (cx, cy, cz) in pixels, x/y about the rotation
    axis at detector column n_det/2) project to chords
    t = 2 sqrt(R^2 - (u - cx cos th - cy sin th)^2 - (z - cz)^2).  With the
    projected phase phi = -sum a_phi t and absorption A = sum a_mu t
    (a_mu << a_phi), the near (contact) frame is F T with transmission
    T = exp(-A) and the far frame F' T (1 - c lap(phi)), the first-order
    transport-of-intensity term of a propagation distance c = dz / k;
    lap is the 5-point detector Laplacian over (row, column).  Flats F, F'
    carry a per-pixel gain, dark D an offset; with ``noise`` the frames get
    beam fluctuations per frame (0.3%), shot noise and (detectors of 8 or
    more columns) 3 dead columns (gain 0 in both flats); with ``counts``
    they are rounded to uint16.

    Returns dict(near, far (M, rows, Ns), flat_near, flat_far, dark
    (rows, Ns), pc_term (M, rows, Ns) = T c lap(phi) (noise-free value of
    the normalized near - far difference), spheres)."""
    th = np.pi * np.arange(n_views) / n_views
    u = np.arange(-1, n_det + 1, dtype=np.float64) - n_det / 2.0
    z = np.arange(-1, n_rows + 1, dtype=np.float64)
    sph = []
    for _ in range(n_spheres):
        R = rng.uniform(0.08, 0.2) * n_det
        rho = rng.uniform(0.0, 0.45 * n_det - R)
        ang = rng.uniform(0.0, 2 * np.pi)
        sph.append((R, rho * np.cos(ang), rho * np.sin(ang), rng.uniform(-0.3, 1.3) * n_rows,
                    rng.uniform(0.5, 1.0), rng.uniform(0.002, 0.01)))
    phi = np.zeros((n_views, n_rows + 2, n_det + 2))
    A = np.zeros_like(phi)
    for R, cx, cy, cz, a_phi, a_mu in sph:
        sc = cx * np.cos(th) + cy * np.sin(th)
        q = R * R - (u[None, None, :] - sc[:, None, None]) ** 2 - (z[None, :, None] - cz) ** 2
        t = 2.0 * np.sqrt(np.maximum(q, 0.0))
        phi -= a_phi * t
        A += a_mu * t
    lap = (phi[:, :-2, 1:-1] + phi[:, 2:, 1:-1] + phi[:, 1:-1, :-2] + phi[:, 1:-1, 2:] - 4 * phi[:, 1:-1, 1:-1])
    T = np.exp(-A[:, 1:-1, 1:-1])
    c = contrast / max(float(np.abs(lap).max()), 1e-30)
    dark = rng.uniform(95.0, 105.0, (n_rows, n_det))
    gain_n = rng.uniform(0.8, 1.2, (n_rows, n_det))
    gain_f = rng.uniform(0.8, 1.2, (n_rows, n_det))
    if noise and n_det >= 8:
        dead = rng.choice(n_det, size=3, replace=False)
        gain_n[:, dead] = 0.0
        gain_f[:, dead] = 0.0
    flat_n = dark + i0 * gain_n
    flat_f = dark + i0 * gain_f
    beam = 1.0 + (0.003 * rng.standard_normal(n_views) if noise else 0.0)
    near = dark[None] + i0 * gain_n[None] * T * np.reshape(beam, (-1, 1, 1))
    far = dark[None] + i0 * gain_f[None] * T * (1.0 - c * lap) * np.reshape(beam, (-1, 1, 1))
    if noise:
        near = near + np.sqrt(np.maximum(near, 0.0)) * rng.standard_normal(near.shape)
        far = far + np.sqrt(np.maximum(far, 0.0)) * rng.standard_normal(far.shape)
    if counts:
        near = np.clip(np.rint(near), 0, 65535).astype(np.uint16)
        far = np.clip(np.rint(far), 0, 65535).astype(np.uint16)
    return {"near": near, "far": far, "flat_near": flat_n, "flat_far": flat_f, "dark": dark,
            "pc_term": T * c * lap, "spheres": sph}
