"""Thin ctypes binding of libcpct (include/cpct.h).

Argument marshalling only: every step of the operators and of the solver runs
in the CUDA library.  PyTorch provides device memory and the current stream.
There is no CPU fallback: if the library is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
LIB_PATH = os.path.join(_PKG, "_lib", "libcpct.so")
HEADER = os.path.join(_ROOT, "include", "cpct.h")

_lib = None

STATUS = {
    0: "CPCT_OK", -1: "CPCT_EINVAL", -2: "CPCT_ENOMEM", -3: "CPCT_ECUDA", -4: "CPCT_ETIMEOUT",
    -5: "CPCT_ENONFINITE", -6: "CPCT_ENOTCONV", -7: "CPCT_EUNSUPPORTED",
}

PLAN_FAIL_ALLOC = 0x1000
NUM_KERNELS = 9


def kernel_name(kid):
    return lib().cpct_kernel_name(int(kid)).decode()


class CpctError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


class Geom(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int), ("n_det", ctypes.c_int), ("n_views", ctypes.c_int),
        ("angles", ctypes.POINTER(ctypes.c_double)), ("kb_width", ctypes.c_int),
        ("oversamp", ctypes.c_double), ("flags", ctypes.c_int),
    ]


def lib():
    """Load libcpct.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        L.cpct_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Geom), vp]
        L.cpct_plan_destroy.argtypes = [vp]
        L.cpct_plan_sync.argtypes = [vp, vp]
        L.cpct_plan_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                     ctypes.POINTER(i), ctypes.POINTER(ctypes.c_size_t)]
        for name in ("radon_fwd", "radon_adj", "radon_fbp", "radon_fwd_host", "radon_adj_host", "radon_adj_noalloc"):
            getattr(L, name).argtypes = [vp, vp, vp, vp]
        for name in ("radon_fwd_c", "radon_adj_c"):
            getattr(L, name).argtypes = [vp, vp, vp, vp]
        L.cpct_plan_set_caps.argtypes = [vp, i, i, vp]
        L.cpct_plan_auto_caps.argtypes = [vp, i, vp]
        L.cpct_plan_set_bins.argtypes = [vp, i, i, i, vp]
        L.cpct_plan_set_rounds.argtypes = [vp, i, vp]
        L.cpct_plan_rounds.argtypes = [vp]
        L.cpct_plan_set_graphs.argtypes = [vp, i]
        L.cpct_plan_graphs.argtypes = [vp]
        L.cpct_plan_bins.argtypes = [vp] + [ctypes.POINTER(i)] * 4 + [vp, vp]
        L.cpct_debug_binplan.argtypes = [ctypes.POINTER(Geom), i, i, i, ctypes.POINTER(i), ctypes.POINTER(i), vp,
                                         ctypes.POINTER(i), ctypes.POINTER(i)]
        L.cpct_plan_work.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
        L.cpct_debug_adj_items.argtypes = [ctypes.POINTER(Geom), i, ctypes.POINTER(i), ctypes.POINTER(i),
                                           ctypes.POINTER(i)]
        L.radon_pair_host_stream.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), i, vp]
        L.cpct_strerror.restype = ctypes.c_char_p
        L.cpct_strerror.argtypes = [i]
        L.cpct_debug_bins.argtypes = [ctypes.POINTER(Geom), i, ctypes.POINTER(i), ctypes.POINTER(i),
                                      ctypes.POINTER(ctypes.c_int64)]
        L.cpct_debug_bin_tile.argtypes = [ctypes.POINTER(Geom), i, i, vp, i]
        L.cpct_debug_split.argtypes = [f, f, f, ctypes.POINTER(i), ctypes.POINTER(f)]
        L.cpct_debug_tables.argtypes = [vp, vp, vp]
        L.cpct_profile_enable.argtypes = [vp, ctypes.c_uint]
        L.cpct_profile_read.argtypes = [vp, vp, vp]
        L.cpct_kernel_name.restype = ctypes.c_char_p
        L.cpct_kernel_name.argtypes = [i]
        L.cpct_launch_count.restype = ctypes.c_longlong
        L.cpct_launch_count.argtypes = [vp, i]
        _lib = L
    return _lib


def header_functions():
    """Names of the functions declared in include/cpct.h."""
    with open(HEADER) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)))


def check(status, what):
    if status != 0:
        raise CpctError(status, what)


def make_geom(n, n_det, n_views, angles=None, flags=0):
    g = Geom()
    g.n, g.n_det, g.n_views = int(n), int(n_det), int(n_views)
    g.kb_width, g.oversamp, g.flags = 6, 2.0, int(flags)
    keep = None
    if angles is not None:
        keep = np.ascontiguousarray(angles, dtype=np.float64)
        g.angles = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return g, keep


def _stream(torch, stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, shape, torch):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _dev_ptr_c(t, shape, torch):
    if not (t.is_cuda and t.dtype == torch.complex64 and t.is_contiguous()):
        raise ValueError("expected a contiguous complex64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """Geometry plan of one slice: N x N image, M views x Ns detector bins."""

    def __init__(self, n, n_det=None, n_views=180, angles=None, flags=0, stream=None):
        import torch
        self._torch = torch
        n_det = n if n_det is None else n_det
        g, self._angles = make_geom(n, n_det, n_views, angles, flags)
        h = ctypes.c_void_p()
        check(lib().cpct_plan_create(ctypes.byref(h), ctypes.byref(g), _stream(torch, stream)), "cpct_plan_create")
        self._h = h
        self.n, self.n_det, self.n_views = n, n_det, n_views

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().cpct_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        n, ns, m, G = (ctypes.c_int() for _ in range(4))
        b = ctypes.c_size_t()
        check(lib().cpct_plan_info(self._h, ctypes.byref(n), ctypes.byref(ns), ctypes.byref(m), ctypes.byref(G),
                                   ctypes.byref(b)), "cpct_plan_info")
        return dict(n=n.value, n_det=ns.value, n_views=m.value, grid=G.value, device_bytes=b.value)

    def sync(self, stream=None):
        check(lib().cpct_plan_sync(self._h, _stream(self._torch, stream)), "cpct_plan_sync")

    def fwd(self, img, out=None, stream=None):
        torch = self._torch
        if out is None:
            out = torch.empty((self.n_views, self.n_det), device=img.device, dtype=torch.float32)
        check(lib().radon_fwd(self._h, _dev_ptr(img, (self.n, self.n), torch),
                              _dev_ptr(out, (self.n_views, self.n_det), torch), _stream(torch, stream)), "radon_fwd")
        return out

    def adj(self, sino, out=None, stream=None):
        torch = self._torch
        if out is None:
            out = torch.empty((self.n, self.n), device=sino.device, dtype=torch.float32)
        check(lib().radon_adj(self._h, _dev_ptr(sino, (self.n_views, self.n_det), torch),
                              _dev_ptr(out, (self.n, self.n), torch), _stream(torch, stream)), "radon_adj")
        return out

    def fwd_c(self, img, out=None, stream=None):
        """Complex sinogram A x (complex64, M x Ns) of a real image."""
        torch = self._torch
        if out is None:
            out = torch.empty((self.n_views, self.n_det), device=img.device, dtype=torch.complex64)
        check(lib().radon_fwd_c(self._h, _dev_ptr(img, (self.n, self.n), torch),
                                _dev_ptr_c(out, (self.n_views, self.n_det), torch), _stream(torch, stream)),
              "radon_fwd_c")
        return out

    def adj_c(self, sino_c, out=None, stream=None):
        """Re(A^H w) of a complex sinogram (complex64, M x Ns)."""
        torch = self._torch
        if out is None:
            out = torch.empty((self.n, self.n), device=sino_c.device, dtype=torch.float32)
        check(lib().radon_adj_c(self._h, _dev_ptr_c(sino_c, (self.n_views, self.n_det), torch),
                                _dev_ptr(out, (self.n, self.n), torch), _stream(torch, stream)), "radon_adj_c")
        return out

    def adj_noalloc(self, sino, out=None, stream=None):
        """radon_adj_noalloc: the adjoint with the library's static scratch."""
        torch = self._torch
        if out is None:
            out = torch.empty((self.n, self.n), device=sino.device, dtype=torch.float32)
        check(lib().radon_adj_noalloc(self._h, _dev_ptr(sino, (self.n_views, self.n_det), torch),
                                      _dev_ptr(out, (self.n, self.n), torch), _stream(torch, stream)),
              "radon_adj_noalloc")
        return out

    def set_caps(self, fwd_cap=0, adj_cap=0, stream=None):
        check(lib().cpct_plan_set_caps(self._h, int(fwd_cap), int(adj_cap), _stream(self._torch, stream)),
              "cpct_plan_set_caps")

    def auto_caps(self, concurrent=1, stream=None):
        """Automatic work-item caps for `concurrent` slices at once
        (cpct_plan_auto_caps)."""
        check(lib().cpct_plan_auto_caps(self._h, int(concurrent), _stream(self._torch, stream)), "cpct_plan_auto_caps")

    def set_bins(self, which, kind, tile=0, stream=None):
        """Bin plan of one operator (which 'fwd' or 'adj'): kind 'uniform'
        with tile 16 / 32 / 64, or 'quadtree' (cpct_plan_set_bins)."""
        w = {"fwd": 0, "adj": 1}[which]
        k = {"uniform": BINS_UNIFORM, "quadtree": BINS_QUADTREE}[kind]
        check(lib().cpct_plan_set_bins(self._h, w, k, int(tile), _stream(self._torch, stream)), "cpct_plan_set_bins")

    def set_rounds(self, lanes, stream=None):
        """Width of the adjoint's conflict-free rounds: 16, 32 or 64 (two
        warps per work item), or ROUNDS_COLUMNS (column groups of five
        samples)."""
        check(lib().cpct_plan_set_rounds(self._h, int(lanes), _stream(self._torch, stream)), "cpct_plan_set_rounds")

    def rounds(self):
        return int(lib().cpct_plan_rounds(self._h))

    def set_graphs(self, enable=True):
        """Graph replay of the operators (cpct_plan_set_graphs)."""
        check(lib().cpct_plan_set_graphs(self._h, 1 if enable else 0), "cpct_plan_set_graphs")

    def graphs(self):
        """Number of captured operator graphs held by the plan."""
        return int(lib().cpct_plan_graphs(self._h))

    def bins(self):
        """Installed bin plans: {'fwd': (kind, tile, bins per class), 'adj': ...}."""
        v = [ctypes.c_int() for _ in range(4)]
        fc = np.zeros(3, dtype=np.int32)
        ac = np.zeros(3, dtype=np.int32)
        check(lib().cpct_plan_bins(self._h, *[ctypes.byref(x) for x in v], fc.ctypes.data_as(ctypes.c_void_p),
                                   ac.ctypes.data_as(ctypes.c_void_p)), "cpct_plan_bins")
        name = {BINS_UNIFORM: "uniform", BINS_QUADTREE: "quadtree"}
        return {"fwd": (name[v[0].value], v[1].value, fc.tolist()), "adj": (name[v[2].value], v[3].value, ac.tolist())}

    def work(self):
        v = [ctypes.c_int() for _ in range(4)]
        check(lib().cpct_plan_work(self._h, *[ctypes.byref(x) for x in v]), "cpct_plan_work")
        return dict(fwd_items=v[0].value, adj_items=v[1].value, n_split=v[2].value, n_slots=v[3].value)

    def fbp(self, sino, out=None, stream=None):
        """Filtered back-projection R^T(ramp * sino)."""
        torch = self._torch
        if out is None:
            out = torch.empty((self.n, self.n), device=sino.device, dtype=torch.float32)
        check(lib().radon_fbp(self._h, _dev_ptr(sino, (self.n_views, self.n_det), torch),
                              _dev_ptr(out, (self.n, self.n), torch), _stream(torch, stream)), "radon_fbp")
        return out

    def fwd_host(self, img: np.ndarray, out: np.ndarray | None = None, stream=None):
        img = np.ascontiguousarray(img, dtype=np.float32)
        if out is None:
            out = np.empty((self.n_views, self.n_det), dtype=np.float32)
        check(lib().radon_fwd_host(self._h, img.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                                   _stream(self._torch, stream)), "radon_fwd_host")
        return out

    def adj_host(self, sino: np.ndarray, out: np.ndarray | None = None, stream=None):
        sino = np.ascontiguousarray(sino, dtype=np.float32)
        if out is None:
            out = np.empty((self.n, self.n), dtype=np.float32)
        check(lib().radon_adj_host(self._h, sino.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                                   _stream(self._torch, stream)), "radon_adj_host")
        return out

    def pair_host_stream(self, imgs, sinos=None, outs=None, stream=None):
        """Forward and adjoint of every image in `imgs` (host float32 arrays,
        N x N), pipelined with the host<->device copies (radon_pair_host_stream);
        returns (sinos, outs), host arrays (given or new).  Pinned buffers let
        the copies overlap the kernels."""
        count = len(imgs)
        imgs = [np.ascontiguousarray(a, dtype=np.float32) for a in imgs]
        for a in imgs:
            if a.shape != (self.n, self.n):
                raise ValueError(f"image shape {a.shape}, expected {(self.n, self.n)}")
        if sinos is None:
            sinos = [np.empty((self.n_views, self.n_det), dtype=np.float32) for _ in range(count)]
        if outs is None:
            outs = [np.empty((self.n, self.n), dtype=np.float32) for _ in range(count)]
        for a, shape in [(x, (self.n_views, self.n_det)) for x in sinos] + [(x, (self.n, self.n)) for x in outs]:
            if a.shape != shape or a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("output arrays must be C-contiguous float32 of the operator's shapes")
        vp = ctypes.c_void_p
        P = (vp * count)(*[a.ctypes.data for a in imgs])
        S = (vp * count)(*[a.ctypes.data for a in sinos])
        O = (vp * count)(*[a.ctypes.data for a in outs])
        check(lib().radon_pair_host_stream(self._h, P, S, O, count, _stream(self._torch, stream)),
              "radon_pair_host_stream")
        return sinos, outs

    def profile_enable(self, mask=0x1FF):
        check(lib().cpct_profile_enable(self._h, ctypes.c_uint(mask)), "cpct_profile_enable")

    def profile_read(self):
        ms = np.zeros(NUM_KERNELS, dtype=np.float64)
        cnt = np.zeros(NUM_KERNELS, dtype=np.int64)
        check(lib().cpct_profile_read(self._h, ms.ctypes.data_as(ctypes.c_void_p), cnt.ctypes.data_as(ctypes.c_void_p)),
              "cpct_profile_read")
        return {kernel_name(k): (float(ms[k]), int(cnt[k])) for k in range(NUM_KERNELS) if cnt[k] > 0}

    def launch_count(self, reset=False):
        return int(lib().cpct_launch_count(self._h, 1 if reset else 0))

    def debug_tables(self):
        poly = np.zeros((6, 10), dtype=np.float64)
        dp = np.zeros(self.n, dtype=np.float32)
        check(lib().cpct_debug_tables(self._h, poly.ctypes.data_as(ctypes.c_void_p), dp.ctypes.data_as(ctypes.c_void_p)),
              "cpct_debug_tables")
        return poly, dp


def debug_bins(n, n_det, n_views, which, angles=None):
    """Host-side bin statistics (no GPU needed): (tiles, entries, checksum)."""
    g, _keep = make_geom(n, n_det, n_views, angles)
    t, e, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    check(lib().cpct_debug_bins(ctypes.byref(g), int(which), ctypes.byref(t), ctypes.byref(e), ctypes.byref(c)),
          "cpct_debug_bins")
    return t.value, e.value, c.value


# ---------------------------------------------------------------------------
# per-slice statistics and scaling (learned warm start)
# ---------------------------------------------------------------------------
def _slices_setup():
    L = lib()
    vp, ll = ctypes.c_void_p, ctypes.c_longlong
    L.cpct_slice_moments.argtypes = [vp, ctypes.c_int, ll, vp, vp, vp]
    L.cpct_slice_soft_l1.argtypes = [vp, ctypes.c_int, ll, vp, vp, vp]
    L.cpct_slice_scale.argtypes = [vp, vp, ctypes.c_int, ll, vp, vp]
    return L


def _slices_ptr(x):
    import torch
    if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous() and x.dim() >= 2):
        raise ValueError("expected a contiguous float32 CUDA tensor of slices (batch, ...)")
    return ctypes.c_void_p(x.data_ptr()), x.shape[0], x[0].numel()


def slice_moments(x, stream=None):
    """Per-slice (mean, sample standard deviation) of a batch of slices,
    host float64 arrays (cpct_slice_moments)."""
    import torch
    p, b, n = _slices_ptr(x)
    mean, std = np.zeros(b), np.zeros(b)
    check(_slices_setup().cpct_slice_moments(p, b, n, mean.ctypes.data_as(ctypes.c_void_p),
                                             std.ctypes.data_as(ctypes.c_void_p), _stream(torch, stream)),
          "cpct_slice_moments")
    return mean, std


def slice_soft_l1(x, thresh, stream=None):
    """Per-slice sum max(|x| - thresh_i, 0) (cpct_slice_soft_l1)."""
    import torch
    p, b, n = _slices_ptr(x)
    th = np.ascontiguousarray(np.broadcast_to(np.asarray(thresh, dtype=np.float64), (b,)))
    out = np.zeros(b)
    check(_slices_setup().cpct_slice_soft_l1(p, b, n, th.ctypes.data_as(ctypes.c_void_p),
                                             out.ctypes.data_as(ctypes.c_void_p), _stream(torch, stream)),
          "cpct_slice_soft_l1")
    return out


def slice_scale(x, factor, out=None, stream=None):
    """out slice i = factor_i * x slice i (cpct_slice_scale); new tensor
    unless `out` is given (may be x itself)."""
    import torch
    p, b, n = _slices_ptr(x)
    if out is None:
        out = torch.empty_like(x)
    q, _, _ = _slices_ptr(out)
    f = np.ascontiguousarray(np.broadcast_to(np.asarray(factor, dtype=np.float64), (b,)))
    check(_slices_setup().cpct_slice_scale(p, q, b, n, f.ctypes.data_as(ctypes.c_void_p), _stream(torch, stream)),
          "cpct_slice_scale")
    return out


def preprocess_pc(near, far, flat_near, flat_far, dark, out=None, stream=None):
    """Phase-contrast sinograms from near/far camera frames (uint16 CUDA
    tensors (M, rows, Ns); int16 tensors holding the same bits are accepted)
    and float32 flats and dark (rows, Ns): (rows, M, Ns) float32
    (cpct_preprocess_pc)."""
    import torch
    L = lib()
    vp = ctypes.c_void_p
    L.cpct_preprocess_pc.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    M, rows, ns = near.shape
    raw = (getattr(torch, "uint16", torch.int16), torch.int16)
    for t, dt, shape in ((near, raw, (M, rows, ns)), (far, raw, (M, rows, ns)),
                         (flat_near, (torch.float32,), (rows, ns)), (flat_far, (torch.float32,), (rows, ns)),
                         (dark, (torch.float32,), (rows, ns))):
        if not (t.is_cuda and t.dtype in dt and t.is_contiguous() and tuple(t.shape) == shape):
            raise ValueError(f"expected a contiguous {dt} CUDA tensor of shape {shape}")
    if out is None:
        out = torch.empty((rows, M, ns), device=near.device, dtype=torch.float32)
    check(L.cpct_preprocess_pc(vp(near.data_ptr()), vp(far.data_ptr()), vp(flat_near.data_ptr()),
                               vp(flat_far.data_ptr()), vp(dark.data_ptr()), M, rows, ns,
                               _dev_ptr(out, (rows, M, ns), torch), _stream(torch, stream)), "cpct_preprocess_pc")
    return out


BINS_UNIFORM = 0
BINS_QUADTREE = 1
ROUNDS_COLUMNS = 5  # round width of column groups (CPCT_ROUNDS_COLUMNS)


def debug_binplan(n, n_det, n_views, kind, tile=0, angles=None, lanes=0):
    """Host-side bin plan of a geometry (no GPU needed): kind 'uniform' (tile
    16/32/64) or 'quadtree', adjoint rounds of `lanes` samples (16/32/64, 0:
    default); dict(fwd_bins, adj_bins, adj_class_bins, rounds, valid)."""
    g, _keep = make_geom(n, n_det, n_views, angles)
    k = {"uniform": BINS_UNIFORM, "quadtree": BINS_QUADTREE}[kind]
    nf, na, nr, ok = (ctypes.c_int() for _ in range(4))
    cls = np.zeros(3, dtype=np.int32)
    check(lib().cpct_debug_binplan(ctypes.byref(g), k, int(tile), int(lanes), ctypes.byref(nf), ctypes.byref(na),
                                   cls.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nr), ctypes.byref(ok)),
          "cpct_debug_binplan")
    return dict(fwd_bins=nf.value, adj_bins=na.value, adj_class_bins=cls.tolist(), rounds=nr.value, valid=ok.value)


def debug_adj_items(n, n_det, n_views, cap=0, angles=None):
    """Host-side adjoint work items of a geometry with `cap` rounds per item
    (no GPU needed): dict(items, n_split, n_slots)."""
    g, _keep = make_geom(n, n_det, n_views, angles)
    v = [ctypes.c_int() for _ in range(3)]
    check(lib().cpct_debug_adj_items(ctypes.byref(g), int(cap), *[ctypes.byref(x) for x in v]),
          "cpct_debug_adj_items")
    return dict(items=v[0].value, n_split=v[1].value, n_slots=v[2].value)


def debug_bin_tile(n, n_det, n_views, which, tile, cap=1 << 20, angles=None):
    g, _keep = make_geom(n, n_det, n_views, angles)
    buf = np.zeros(cap, dtype=np.uint32)
    cnt = lib().cpct_debug_bin_tile(ctypes.byref(g), int(which), int(tile), buf.ctypes.data_as(ctypes.c_void_p), cap)
    if cnt < 0:
        raise CpctError(cnt, "cpct_debug_bin_tile")
    return buf[:min(cnt, cap)].copy()


def debug_split(k, hi, lo):
    fl, z = ctypes.c_int(), ctypes.c_float()
    lib().cpct_debug_split(ctypes.c_float(k), ctypes.c_float(hi), ctypes.c_float(lo), ctypes.byref(fl), ctypes.byref(z))
    return fl.value, z.value


def debug_rounds(n, n_det, n_views, angles=None):
    """Host-side round packing of the adjoint bins: (rounds, packed samples, valid)."""
    g, _keep = make_geom(n, n_det, n_views, angles)
    r, pk, ok = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    L = lib()
    L.cpct_debug_rounds.argtypes = [ctypes.POINTER(Geom), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    check(L.cpct_debug_rounds(ctypes.byref(g), ctypes.byref(r), ctypes.byref(pk), ctypes.byref(ok)),
          "cpct_debug_rounds")
    return r.value, pk.value, bool(ok.value)


# ---------------------------------------------------------------------------
# ring filter and SPGL1
# ---------------------------------------------------------------------------
SPGL1_TAU0 = 0x1
SPGL1_NO_FILTER = 0x2
SPGL1_SYNTH_DH = 0x4
SPGL1_LASSO = 0x8
SPGL1_STATUS = {1: "root found", 2: "basis pursuit solution", 3: "iteration cap", 4: "line search failure",
                5: "non-finite"}


class Spgl1Opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("memory", ctypes.c_int), ("max_line", ctypes.c_int),
                ("flags", ctypes.c_int), ("opt_tol", ctypes.c_double), ("bp_tol", ctypes.c_double),
                ("gamma", ctypes.c_double), ("step_min", ctypes.c_double), ("step_max", ctypes.c_double),
                ("tau0", ctypes.c_double), ("ls_tol", ctypes.c_double), ("dec_tol", ctypes.c_double),
                ("max_line_errors", ctypes.c_int), ("pad_", ctypes.c_int)]


class Spgl1Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("ticks", ctypes.c_int),
                ("trials", ctypes.c_int), ("tau", ctypes.c_double), ("rnorm", ctypes.c_double),
                ("xnorm1", ctypes.c_double), ("rel_gap", ctypes.c_double), ("newton", ctypes.c_int),
                ("line_errors", ctypes.c_int), ("safeguards", ctypes.c_int), ("stationary", ctypes.c_int),
                ("gstep", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


def _spgl1_setup():
    L = lib()
    vp = ctypes.c_void_p
    L.cpct_ring_filter.argtypes = [vp, vp, vp, vp]
    L.spgl1_solve.argtypes = [vp, vp, ctypes.c_double, vp, ctypes.POINTER(Spgl1Opts), ctypes.POINTER(Spgl1Info), vp]
    L.spgl1_solve_batched.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(vp),
                                      ctypes.POINTER(Spgl1Opts), ctypes.POINTER(Spgl1Info), vp]
    L.cpct_project_l1.argtypes = [vp, ctypes.c_longlong, ctypes.c_double, vp, ctypes.POINTER(ctypes.c_double), vp]
    L.cpct_project_l1_batched.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_longlong,
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(vp),
                                          ctypes.POINTER(ctypes.c_double), vp]
    return L


def project_l1_batched(vs, taus, outs=None, stream=None):
    """Projections of equally sized float32 CUDA tensors onto l1 balls of the
    given radii; returns (outs, thetas)."""
    import torch
    L = _spgl1_setup()
    B = len(vs)
    if outs is None:
        outs = [torch.empty_like(v) for v in vs]
    n = vs[0].numel()
    for v, o in zip(vs, outs):
        _dev_ptr(v, tuple(vs[0].shape), torch)
        _dev_ptr(o, tuple(vs[0].shape), torch)
    V = (ctypes.c_void_p * B)(*[v.data_ptr() for v in vs])
    O = (ctypes.c_void_p * B)(*[o.data_ptr() for o in outs])
    T = (ctypes.c_double * B)(*[float(t) for t in taus])
    th = (ctypes.c_double * B)()
    check(L.cpct_project_l1_batched(V, B, n, T, O, th, _stream(torch, stream)), "cpct_project_l1_batched")
    return outs, list(th)


def project_l1(v, tau, out=None, stream=None):
    """Projection of the float32 CUDA tensor ``v`` onto {||x||_1 <= tau}.

    Returns (out, theta) with out_i = sign(v_i) max(|v_i| - theta, 0).
    """
    import torch
    L = _spgl1_setup()
    if out is None:
        out = torch.empty_like(v)
    th = ctypes.c_double()
    check(L.cpct_project_l1(_dev_ptr(v, tuple(v.shape), torch), v.numel(), float(tau),
                            _dev_ptr(out, tuple(v.shape), torch), ctypes.byref(th), _stream(torch, stream)),
          "cpct_project_l1")
    return out, th.value


def make_opts(max_iter=0, opt_tol=0.0, bp_tol=0.0, memory=0, max_line=0, tau0=None, ring_filter=True,
              synth_dh=False, lasso_tau=None, step_min=0.0, step_max=0.0):
    """SPGL1 options (0 = default).  synth_dh: the analysis-l1 variant, the
    solution is z with the image u = synth_dh(z).  lasso_tau: solve the LASSO
    problem with that fixed radius instead (sigma ignored)."""
    o = Spgl1Opts()
    o.max_iter, o.opt_tol, o.bp_tol, o.memory, o.max_line = max_iter, opt_tol, bp_tol, memory, max_line
    o.step_min, o.step_max = step_min, step_max
    o.flags = ((0 if ring_filter else SPGL1_NO_FILTER) | (SPGL1_TAU0 if tau0 is not None else 0)
               | (SPGL1_SYNTH_DH if synth_dh else 0) | (SPGL1_LASSO if lasso_tau is not None else 0))
    o.tau0 = float(lasso_tau) if lasso_tau is not None else (0.0 if tau0 is None else float(tau0))
    return o


def synth_dh(x, adjoint=False, out=None, stream=None):
    """u = C x (row prefix sums) or C^T x (row suffix sums) of an N x N float32
    CUDA tensor (cpct_synth_dh)."""
    import torch
    L = lib()
    L.cpct_synth_dh.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    n = x.shape[0]
    if out is None:
        out = torch.empty_like(x)
    check(L.cpct_synth_dh(_dev_ptr(x, (n, n), torch), _dev_ptr(out, (n, n), torch), n, 1 if adjoint else 0,
                          _stream(torch, stream)), "cpct_synth_dh")
    return out


def ring_filter(plan, sino, out=None, stream=None):
    """F y on the device (same shape as the sinogram)."""
    torch = plan._torch
    L = _spgl1_setup()
    if out is None:
        out = torch.empty_like(sino)
    check(L.cpct_ring_filter(plan.handle, _dev_ptr(sino, (plan.n_views, plan.n_det), torch),
                             _dev_ptr(out, (plan.n_views, plan.n_det), torch), _stream(torch, stream)),
          "cpct_ring_filter")
    return out


def spgl1(plan, b, sigma, x0=None, opts=None, stream=None, allow_notconv=True):
    """Solve min ||x||_1 s.t. ||F(R x - b)||_2 <= sigma on the device.

    Returns (x, info dict).  ``x0`` (N x N CUDA tensor) warm-starts the solve
    (tau starts at ||x0||_1); otherwise the solve starts cold from x = 0.
    """
    torch = plan._torch
    L = _spgl1_setup()
    x = torch.zeros((plan.n, plan.n), device=b.device, dtype=torch.float32) if x0 is None else x0.clone()
    info = Spgl1Info()
    o = opts if opts is not None else make_opts()
    rc = L.spgl1_solve(plan.handle, _dev_ptr(b, (plan.n_views, plan.n_det), torch), float(sigma),
                       _dev_ptr(x, (plan.n, plan.n), torch), ctypes.byref(o), ctypes.byref(info),
                       _stream(torch, stream))
    if rc != 0 and not (allow_notconv and rc == -6):
        raise CpctError(rc, "spgl1_solve")
    return x, info.as_dict()


def spgl1_batched(plans, bs, sigmas, x0s=None, opts=None, stream=None, allow_notconv=True):
    """Solve len(plans) independent slices together (one plan per slice)."""
    torch = plans[0]._torch
    L = _spgl1_setup()
    B = len(plans)
    xs = [torch.zeros((p.n, p.n), device=b.device, dtype=torch.float32) if x0s is None else x0s[i].clone()
          for i, (p, b) in enumerate(zip(plans, bs))]
    H = (ctypes.c_void_p * B)(*[p.handle.value for p in plans])
    Bp = (ctypes.c_void_p * B)(*[_dev_ptr(b, (p.n_views, p.n_det), torch).value for p, b in zip(plans, bs)])
    Xp = (ctypes.c_void_p * B)(*[_dev_ptr(x, (p.n, p.n), torch).value for p, x in zip(plans, xs)])
    S = (ctypes.c_double * B)(*[float(s) for s in sigmas])
    infos = (Spgl1Info * B)()
    o = opts if opts is not None else make_opts()
    rc = L.spgl1_solve_batched(H, B, Bp, S, Xp, ctypes.byref(o), infos, _stream(torch, stream))
    if rc != 0 and not (allow_notconv and rc == -6):
        raise CpctError(rc, "spgl1_solve_batched")
    return xs, [i.as_dict() for i in infos]


# ---------------------------------------------------------------------------
# clones, autotuner, batches
# ---------------------------------------------------------------------------
BATCH_FWD, BATCH_ADJ, BATCH_PAIR = 0, 1, 2


def _batch_setup():
    L = lib()
    vp = ctypes.c_void_p
    L.cpct_plan_clone.argtypes = [vp, ctypes.POINTER(vp), vp]
    L.cpct_plan_tune.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), vp]
    L.cpct_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp),
                                    ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, vp]
    L.cpct_batch_run.argtypes = [vp, vp]
    L.cpct_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong),
                                  ctypes.POINTER(ctypes.c_int)]
    L.cpct_batch_destroy.argtypes = [vp]
    return L


def clone(plan, stream=None):
    """A plan of the same geometry sharing tables and bins, with own workspaces."""
    L = _batch_setup()
    h = ctypes.c_void_p()
    check(L.cpct_plan_clone(plan.handle, ctypes.byref(h), _stream(plan._torch, stream)), "cpct_plan_clone")
    c = Plan.__new__(Plan)
    c._torch, c._h, c._angles = plan._torch, h, plan._angles
    c.n, c.n_det, c.n_views = plan.n, plan.n_det, plan.n_views
    return c


def tune(plan, reps=5, stream=None):
    """Time candidate work-item caps and keep the fastest: (fwd_cap, adj_cap)."""
    L = _batch_setup()
    f, a = ctypes.c_int(), ctypes.c_int()
    check(L.cpct_plan_tune(plan.handle, int(reps), ctypes.byref(f), ctypes.byref(a), _stream(plan._torch, stream)),
          "cpct_plan_tune")
    return f.value, a.value


class Batch:
    """The operator over many slices as one CUDA graph (one plan per slice)."""

    def __init__(self, plans, ins, outs, mode=BATCH_PAIR, branches=0, stream=None):
        torch = plans[0]._torch
        L = _batch_setup()
        B = len(plans)
        vp = ctypes.c_void_p
        self._keep = (list(plans), list(ins), list(outs))
        H = (vp * B)(*[p.handle.value for p in plans])
        I = (vp * B)(*[t.data_ptr() for t in ins])
        O = (vp * B)(*[t.data_ptr() for t in outs])
        h = vp()
        check(L.cpct_batch_create(ctypes.byref(h), H, B, I, O, int(mode), int(branches), _stream(torch, stream)),
              "cpct_batch_create")
        self._h, self._torch = h, torch

    def run(self, stream=None):
        check(_batch_setup().cpct_batch_run(self._h, _stream(self._torch, stream)), "cpct_batch_run")

    def info(self):
        n, s, b = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_int()
        check(_batch_setup().cpct_batch_info(self._h, ctypes.byref(n), ctypes.byref(s), ctypes.byref(b)),
              "cpct_batch_info")
        return dict(slices=n.value, samples=s.value, branches=b.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _batch_setup().cpct_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# learned warm start: the convolutional denoiser
# ---------------------------------------------------------------------------
def _unet_setup():
    L = lib()
    vp = ctypes.c_void_p
    L.cpct_unet_param_count.argtypes = [ctypes.c_int, ctypes.c_int]
    L.cpct_unet_param_count.restype = ctypes.c_longlong
    L.cpct_unet_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, vp]
    L.cpct_unet_destroy.argtypes = [vp]
    for name in ("cpct_unet_set_params", "cpct_unet_get_params", "cpct_unet_get_grads"):
        getattr(L, name).argtypes = [vp, vp, vp]
    L.cpct_unet_forward.argtypes = [vp, vp, vp, ctypes.c_int, vp]
    L.cpct_unet_sync.argtypes = [vp, vp]
    L.cpct_unet_backward.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), vp]
    L.cpct_unet_adam_step.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.POINTER(ctypes.c_double), vp]
    return L


def unet_param_count(levels, base):
    """Length of the parameter vector of cpct_unet (-1: unsupported shape)."""
    return int(_unet_setup().cpct_unet_param_count(int(levels), int(base)))


class UNet:
    """The denoiser of the learned warm start (device weights and buffers)."""

    def __init__(self, levels, base, max_batch, height, width, stream=None):
        import torch
        self._torch = torch
        self.levels, self.base, self.max_batch, self.height, self.width = levels, base, max_batch, height, width
        L = _unet_setup()
        h = ctypes.c_void_p()
        check(L.cpct_unet_create(ctypes.byref(h), levels, base, max_batch, height, width, _stream(torch, stream)),
              "cpct_unet_create")
        self.handle = h
        self.n_params = unet_param_count(levels, base)

    def close(self):
        if self.handle is not None and self.handle.value:
            _unet_setup().cpct_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params, stream=None):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {p.size}")
        check(_unet_setup().cpct_unet_set_params(self.handle, p.ctypes.data_as(ctypes.c_void_p),
                                                 _stream(self._torch, stream)), "cpct_unet_set_params")

    def _host_vec(self, fn, stream):
        import numpy as np
        out = np.empty(self.n_params, dtype=np.float32)
        check(getattr(_unet_setup(), fn)(self.handle, out.ctypes.data_as(ctypes.c_void_p),
                                         _stream(self._torch, stream)), fn)
        return out

    def get_params(self, stream=None):
        return self._host_vec("cpct_unet_get_params", stream)

    def get_grads(self, stream=None):
        return self._host_vec("cpct_unet_get_grads", stream)

    def forward(self, x, out=None, stream=None):
        torch = self._torch
        B = x.shape[0]
        shape = (B, self.height, self.width)
        if out is None:
            out = torch.empty_like(x)
        check(_unet_setup().cpct_unet_forward(self.handle, _dev_ptr(x, shape, torch), _dev_ptr(out, shape, torch), B,
                                              _stream(torch, stream)), "cpct_unet_forward")
        return out

    def sync(self, stream=None):
        """Synchronize and raise if a bounded device wait of a forward pass
        expired since the last call."""
        check(_unet_setup().cpct_unet_sync(self.handle, _stream(self._torch, stream)), "cpct_unet_sync")

    def backward(self, x, target, stream=None):
        """Forward + loss + parameter gradients; returns the loss."""
        torch = self._torch
        B = x.shape[0]
        shape = (B, self.height, self.width)
        loss = ctypes.c_double()
        check(_unet_setup().cpct_unet_backward(self.handle, _dev_ptr(x, shape, torch), _dev_ptr(target, shape, torch),
                                               B, ctypes.byref(loss), _stream(torch, stream)), "cpct_unet_backward")
        return loss.value

    def adam_step(self, lr, max_grad_norm=0.0, return_norm=False, stream=None):
        """One Adam step; gradients clipped to max_grad_norm (0: none).
        Returns the gradient norm before clipping when return_norm is set."""
        nrm = ctypes.c_double()
        check(_unet_setup().cpct_unet_adam_step(self.handle, float(lr), float(max_grad_norm),
                                                ctypes.byref(nrm) if return_norm else None,
                                                _stream(self._torch, stream)), "cpct_unet_adam_step")
        return nrm.value if return_norm else None


def unet_debug_op(op, a, b, out_shape, w=None, C1=None, C2=0, Cout=0, stream=None):
    """Run one denoiser operation (cpct_unet_debug_op) on NHWC CUDA tensors."""
    import numpy as np
    import torch
    L = _unet_setup()
    vp = ctypes.c_void_p
    L.cpct_unet_debug_op.argtypes = [ctypes.c_int, vp, vp, vp, vp] + [ctypes.c_int] * 6 + [vp]
    B, H, W = a.shape[0], a.shape[1], a.shape[2]
    if op in (3, 4):
        B, H, W = out_shape[0], out_shape[1], out_shape[2]
    C1 = a.shape[3] if C1 is None else C1
    y = torch.empty(out_shape, device=a.device, dtype=torch.float32)
    for t in (a, b, y):
        if t is not None and not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("expected contiguous float32 CUDA tensors")
    hw = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    check(L.cpct_unet_debug_op(op, vp(a.data_ptr()), vp(b.data_ptr()) if b is not None else None,
                               vp(y.data_ptr()), hw.ctypes.data_as(vp) if hw is not None else None,
                               B, H, W, C1, C2, Cout, _stream(torch, stream)), "cpct_unet_debug_op")
    return y


def debug_tc_gemm(a_bf16, b_bf16):
    """D = A * B^T on the tensor cores (tcgen05), A 128 x K, B N x K (bfloat16
    CUDA tensors); returns D (float32)."""
    import torch
    L = lib()
    vp = ctypes.c_void_p
    L.cpct_debug_tc_gemm.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    n, k = b_bf16.shape
    d = torch.empty((128, n), device=a_bf16.device, dtype=torch.float32)
    check(L.cpct_debug_tc_gemm(vp(a_bf16.data_ptr()), vp(b_bf16.data_ptr()), vp(d.data_ptr()), n, k,
                               _stream(torch, None)), "cpct_debug_tc_gemm")
    return d
