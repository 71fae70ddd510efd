"""Thin Python binding of libtopot.so (C ABI in include/topot.h).

Argument marshalling only: every step of the computation runs in the CUDA library.
Tensors are PyTorch CUDA tensors (PyTorch provides device memory and streams); the
library is loaded on first use and a missing library raises -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtopot.so")

U8, I32 = 0, 1
VERTEX, TOP = 0, 1
KERNELS = {"laplace": 0, "fourier": 1, "bessel": 2, "sine": 3}
TABLE = 4
PRECISIONS = {"fp32c": 0, "fp64": 1}
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "OOM", 4: "CUDA", 5: "OVERFLOW", 6: "TIMEOUT"}

API_SYMBOLS = (
    "build_critical_tables", "tables_create", "tables_build", "tables_sync", "tables_info",
    "tables_copy_to_host", "tables_set_tuning", "free_tables", "ect", "radon", "hybrid_transform",
    "hybrid_transform_grad", "hybrid_transform_noalloc", "exact_representation", "ect_exact_eval",
    "radon_exact_eval", "topot_selftest_wait", "topot_last_error", "kernel_table_create", "kernel_table_free",
    "hybrid_transform_table", "hybrid_transform_table_grad", "tables_create_slab", "slab_sum_i32", "slab_sum_f64",
)


class TopotError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"topot {STATUS.get(status, status)}: {msg}")
        self.status = status


class Tuning(ctypes.Structure):
    _fields_ = [("ect_dirs_per_warp", ctypes.c_int), ("ect_chunk", ctypes.c_int), ("ect_ctas_per_sm", ctypes.c_int),
                ("ht_dirs_per_lane", ctypes.c_int), ("ht_chunk", ctypes.c_int), ("ht_ctas_per_sm", ctypes.c_int),
                ("ht_warp_split", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load libtopot.so and declare the C signatures (no CUDA call is made)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtopot.so not found at {path}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    vp, i32, i64p, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_double
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "build_critical_tables": [vp, i32, i32, i64p, i64p, i32, i32, vp, pp],
        "tables_create": [i32, i32, i64p, i64p, i32, i32, pp],
        "tables_build": [vp, vp, vp],
        "tables_sync": [vp, vp],
        "tables_info": [vp, i32, i32, i64p, i64p, i64p],
        "tables_copy_to_host": [vp, i32, i32, i32, vp, vp],
        "tables_set_tuning": [vp, ctypes.POINTER(Tuning)],
        "ect": [vp, vp, i32, i32, dp, dp, i32, vp, vp],
        "radon": [vp, vp, i32, i32, dp, dp, i32, vp, vp],
        "hybrid_transform": [vp, i32, i32, vp, i32, i32, vp, vp],
        "hybrid_transform_grad": [vp, i32, i32, vp, i32, i32, vp, vp, vp],
        "hybrid_transform_noalloc": [vp, i32, i32, vp, i32, i32, vp, vp],
        "exact_representation": [vp, i32, vp, i32, i32, ctypes.c_int64, vp, vp, vp, vp],
        "ect_exact_eval": [i32, ctypes.c_int64, vp, vp, vp, vp, i32, vp, vp],
        "radon_exact_eval": [i32, ctypes.c_int64, vp, vp, vp, ctypes.c_int64, vp, vp, vp, vp, i32, vp, vp],
        "topot_selftest_wait": [i32, i32, vp],
        "kernel_table_create": [vp, i32, dp, dp, pp],
        "hybrid_transform_table": [vp, vp, i32, vp, i32, i32, vp, vp],
        "hybrid_transform_table_grad": [vp, vp, i32, vp, i32, i32, vp, vp, vp],
        "tables_create_slab": [i32, i32, i64p, i64p, i64p, i32, pp],
        "slab_sum_i32": [vp, i32, ctypes.c_int64, vp, vp, vp],
        "slab_sum_f64": [vp, i32, ctypes.c_int64, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.free_tables.argtypes = [vp]
    L.free_tables.restype = None
    L.kernel_table_free.argtypes = [vp]
    L.kernel_table_free.restype = None
    L.topot_last_error.argtypes = []
    L.topot_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise TopotError(status, load().topot_last_error().decode(errors="replace"))


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _i64(a) -> ctypes.Array:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int64).reshape(-1))
    return (ctypes.c_int64 * len(a))(*a.tolist())


def _dirs(dirs: torch.Tensor, n: int, B: int):
    if dirs.dtype != torch.float64 or not dirs.is_cuda:
        raise ValueError("directions must be a CUDA float64 tensor")
    dirs = dirs.contiguous()
    if dirs.dim() == 2 and dirs.shape[1] == n:
        return dirs, dirs.shape[0], 0
    if dirs.dim() == 3 and dirs.shape[0] == B and dirs.shape[2] == n:
        return dirs, dirs.shape[1], 1
    raise ValueError(f"directions must be [D, {n}] or [{B}, D, {n}]")


@dataclass
class ImageBatch:
    """Images packed in one device buffer: pixels (flat), shapes [B][n] (m_0 fastest), offsets."""
    pixels: torch.Tensor
    shapes: np.ndarray
    offsets: np.ndarray

    @property
    def n(self) -> int:
        return self.shapes.shape[1]

    @property
    def B(self) -> int:
        return self.shapes.shape[0]


def pack_images(images, device="cuda", align: int = 16) -> ImageBatch:
    """Pack numpy images (C order, last axis = coordinate 0) into one device buffer.

    Each image starts at a multiple of ``align`` elements so that row copies can use
    16-byte aligned bulk transfers when the row length allows it.
    """
    images = [np.ascontiguousarray(im) for im in images]
    dt = images[0].dtype
    if dt not in (np.uint8, np.int32):
        raise ValueError("images must be uint8 or int32")
    n = images[0].ndim
    shapes, offsets, pos = [], [], 0
    for im in images:
        if im.ndim != n or im.dtype != dt:
            raise ValueError("all images need the same rank and dtype")
        shapes.append(list(reversed(im.shape)))
        offsets.append(pos)
        pos += -(-im.size // align) * align
    host = np.zeros(pos, dtype=dt)
    for im, off in zip(images, offsets):
        host[off:off + im.size] = im.reshape(-1)
    pix = torch.from_numpy(host).to(device)
    return ImageBatch(pix, np.array(shapes, dtype=np.int64), np.array(offsets, dtype=np.int64))


class Tables:
    """Critical-point tables of a batch of images (owns the device tables)."""

    def __init__(self, handle, n: int, B: int, dtype: int, shapes, offsets):
        self._h = handle
        self.n, self.B, self.dtype = n, B, dtype
        self.shapes = np.asarray(shapes)
        self.offsets = np.asarray(offsets)

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("tables already freed")
        return self._h

    def free(self):
        if self._h is not None:
            load().free_tables(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def build(self, pixels: torch.Tensor, stream=None):
        """Re-extract the tables from new pixels of the same shapes (asynchronous)."""
        _check(load().tables_build(self.handle, _ptr(pixels), _stream(stream)))

    def sync(self, stream=None):
        _check(load().tables_sync(self.handle, _stream(stream)))

    def info(self, image: int, orthant: int):
        nl, nd, chi = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().tables_info(self.handle, image, orthant, ctypes.byref(nl), ctypes.byref(nd),
                                  ctypes.byref(chi)))
        return nl.value, nd.value, chi.value

    def table(self, image: int, orthant: int, kind: int):
        """(idx, val) of one table as int64 numpy arrays (kind 0: Delta^-, 1: Delta)."""
        nl, nd, _ = self.info(image, orthant)
        cnt = nl if kind == 0 else nd
        idx = np.zeros(max(cnt, 1), dtype=np.int32)
        val = np.zeros(max(cnt, 1), dtype=np.int32)
        _check(load().tables_copy_to_host(self.handle, image, orthant, kind,
                                          idx.ctypes.data_as(ctypes.c_void_p),
                                          val.ctypes.data_as(ctypes.c_void_p)))
        return idx[:cnt].astype(np.int64), val[:cnt].astype(np.int64)

    def set_tuning(self, **kw):
        """Tile shapes per operation (fields of Tuning; omitted fields keep their value)."""
        cur = getattr(self, "_tuning", Tuning())
        tu = Tuning(**{**cur.as_dict(), **kw})
        _check(load().tables_set_tuning(self.handle, ctypes.byref(tu)))
        self._tuning = tu

    @property
    def tuning(self) -> dict:
        return getattr(self, "_tuning", Tuning()).as_dict()


CONSTRUCTIONS = {"vertex": VERTEX, "top": TOP}


def build_critical_tables(batch: ImageBatch, construction: str = "vertex", stream=None) -> Tables:
    """Tables of every image: construction "vertex" (pixels are vertices) or "top" (pixels
    are top-dimensional cells; the tables live on the m_k + 1 pixel corners per axis)."""
    L = load()
    dtype = U8 if batch.pixels.dtype == torch.uint8 else I32
    h = ctypes.c_void_p()
    _check(L.build_critical_tables(_ptr(batch.pixels), dtype, batch.n, _i64(batch.shapes), _i64(batch.offsets),
                                   batch.B, CONSTRUCTIONS[construction], _stream(stream), ctypes.byref(h)))
    return Tables(h, batch.n, batch.B, dtype, batch.shapes, batch.offsets)


def tables_create(shapes, offsets, dtype=U8, construction: str = "vertex") -> Tables:
    shapes = np.asarray(shapes, dtype=np.int64)
    h = ctypes.c_void_p()
    _check(load().tables_create(dtype, shapes.shape[1], _i64(shapes), _i64(offsets), shapes.shape[0],
                                CONSTRUCTIONS[construction], ctypes.byref(h)))
    return Tables(h, shapes.shape[1], shapes.shape[0], dtype, shapes, offsets)


def tables_create_slab(shapes, offsets, zrange, dtype=U8) -> Tables:
    """A handle for slabs of volumes: image b is planes [zrange[b][0], zrange[b][1]) of a
    volume of shape shapes[b] (axis 0 fastest); its pixels hold the slab plus the
    neighbouring plane on each side that exists (paper_2405_02256_gb300.slabs packs them)."""
    shapes = np.asarray(shapes, dtype=np.int64)
    h = ctypes.c_void_p()
    _check(load().tables_create_slab(dtype, shapes.shape[1], _i64(shapes), _i64(offsets), _i64(zrange),
                                     shapes.shape[0], ctypes.byref(h)))
    return Tables(h, shapes.shape[1], shapes.shape[0], dtype, shapes, offsets)


def slab_sum(parts: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    """Sum of P slab parts [P, ...] in slab order: exact for int32 (TopotError OVERFLOW if a
    sum leaves the int32 range), compensated for float64.  Returns [...]."""
    parts = parts.contiguous()
    P = parts.shape[0]
    n = parts[0].numel()
    if out is None:
        out = torch.empty(parts.shape[1:], dtype=parts.dtype, device=parts.device)
    L = load()
    if parts.dtype == torch.int32:
        flag = torch.zeros(1, dtype=torch.int32, device=parts.device)
        _check(L.slab_sum_i32(_ptr(parts), P, n, _ptr(out), _ptr(flag), _stream(stream)))
        if int(flag.item()) != 0:
            raise TopotError(5, "slab_sum: a sum leaves the int32 range")
    elif parts.dtype == torch.float64:
        _check(L.slab_sum_f64(_ptr(parts), P, n, _ptr(out), _stream(stream)))
    else:
        raise ValueError("slab parts must be int32 or float64")
    return out


def ect(tables: Tables, dirs: torch.Tensor, t_min: float, t_max: float, T: int, out=None, stream=None):
    """ECT(xi_d, t_j) for every image: int32 [B, D, T]."""
    L = load()
    dirs, D, per = _dirs(dirs, tables.n, tables.B)
    if out is None:
        out = torch.empty((tables.B, D, T), dtype=torch.int32, device=dirs.device)
    _check(L.ect(tables.handle, _ptr(dirs), D, per, float(t_min), float(t_max), int(T), _ptr(out), _stream(stream)))
    return out


def radon(tables: Tables, dirs: torch.Tensor, t_min: float, t_max: float, T: int, out=None, stream=None):
    """Radon transform R(xi_d, t_j) for every image: int32 [B, D, T]."""
    L = load()
    dirs, D, per = _dirs(dirs, tables.n, tables.B)
    if out is None:
        out = torch.empty((tables.B, D, T), dtype=torch.int32, device=dirs.device)
    _check(L.radon(tables.handle, _ptr(dirs), D, per, float(t_min), float(t_max), int(T), _ptr(out),
                   _stream(stream)))
    return out


class ExactRep:
    """Exact representations of one kind for every image and direction (device tensors):
    T float64 [B, D, cap], E int32 [B, D, cap], length int64 [B, D]; entries past the
    length of a segment are unspecified."""

    def __init__(self, kind: int, T: torch.Tensor, E: torch.Tensor, length: torch.Tensor):
        self.kind, self.T, self.E, self.length = kind, T, E, length

    @property
    def cap(self) -> int:
        return self.T.shape[-1]

    def segment(self, b: int, d: int):
        """(T, E) of image b and direction d as numpy arrays."""
        n = int(self.length[b, d])
        return self.T[b, d, :n].cpu().numpy(), self.E[b, d, :n].cpu().numpy()


def exact_representation(tables: Tables, kind: int, dirs: torch.Tensor, cap: int = None, stream=None) -> ExactRep:
    """Kind 0: (T, E) of t -> ECT(xi_d, t); kind 1: (T', E') of the Radon transform between
    critical values, for every image and direction (Section 4.3, Appendix A.2)."""
    L = load()
    dirs, D, per = _dirs(dirs, tables.n, tables.B)
    if cap is None:
        cap = 1
        for b in range(tables.B):
            for o in range(1 << tables.n):
                nl, nd, _ = tables.info(b, o)
                cap = max(cap, nl if kind == 0 else nd)
    T = torch.empty((tables.B, D, cap), dtype=torch.float64, device=dirs.device)
    E = torch.empty((tables.B, D, cap), dtype=torch.int32, device=dirs.device)
    n = torch.empty((tables.B, D), dtype=torch.int64, device=dirs.device)
    _check(L.exact_representation(tables.handle, int(kind), _ptr(dirs), D, per, int(cap), _ptr(T), _ptr(E),
                                  _ptr(n), _stream(stream)))
    return ExactRep(kind, T, E, n)


def _queries(t, device):
    t = torch.as_tensor(t, dtype=torch.float64, device=device).reshape(-1).contiguous()
    if t.numel() < 1:
        raise ValueError("need at least one threshold")
    return t


def ect_exact_eval(rep: ExactRep, t, stream=None) -> torch.Tensor:
    """ECT(xi_d, t_q) from kind-0 representations (Appendix A.3): int32 [B, D, Q]."""
    if rep.kind != 0:
        raise ValueError("ect_exact_eval needs a kind-0 representation")
    B, D, cap = rep.T.shape
    t = _queries(t, rep.T.device)
    out = torch.empty((B, D, t.numel()), dtype=torch.int32, device=rep.T.device)
    _check(load().ect_exact_eval(B * D, cap, _ptr(rep.T), _ptr(rep.E), _ptr(rep.length), _ptr(t), t.numel(),
                                 _ptr(out), _stream(stream)))
    return out


def radon_exact_eval(rep_lower: ExactRep, rep_ord: ExactRep, t, stream=None) -> torch.Tensor:
    """R(xi_d, t_q) at arbitrary t_q from a kind-0 and a kind-1 representation of the same
    images and directions: int32 [B, D, Q]."""
    if rep_lower.kind != 0 or rep_ord.kind != 1 or rep_lower.T.shape[:2] != rep_ord.T.shape[:2]:
        raise ValueError("radon_exact_eval needs kind-0 and kind-1 representations of the same directions")
    B, D, cap = rep_lower.T.shape
    t = _queries(t, rep_lower.T.device)
    out = torch.empty((B, D, t.numel()), dtype=torch.int32, device=rep_lower.T.device)
    _check(load().radon_exact_eval(B * D, cap, _ptr(rep_lower.T), _ptr(rep_lower.E), _ptr(rep_lower.length),
                                   rep_ord.cap, _ptr(rep_ord.T), _ptr(rep_ord.E), _ptr(rep_ord.length), _ptr(t),
                                   t.numel(), _ptr(out), _stream(stream)))
    return out


class KernelTable:
    """A kernel given by K samples of its primitive, kbar(s_min + i h), h = (s_max - s_min) / (K - 1):
    piecewise-linear in between, constant outside (include/topot.h, kernel_table_create).
    Pass it as the ``kernel`` of hybrid_transform / hybrid_transform_grad / HybridTransform."""

    def __init__(self, values, s_min: float, s_max: float):
        L = load()
        y = np.ascontiguousarray(np.asarray(values, dtype=np.float64).ravel())
        h = ctypes.c_void_p()
        _check(L.kernel_table_create(y.ctypes.data_as(ctypes.c_void_p), int(y.size), float(s_min), float(s_max),
                                     ctypes.byref(h)))
        self._h = h
        self.K, self.s_min, self.s_max = int(y.size), float(s_min), float(s_max)

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("kernel table already freed")
        return self._h

    def free(self):
        if self._h is not None:
            torch.cuda.synchronize()
            load().kernel_table_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hybrid_transform(tables: Tables, kernel, dirs: torch.Tensor, precision: str = "fp32c", out=None,
                     stream=None):
    """HT(xi_d) per image: float64 [B, D] (Fourier: [B, D, 2] = (re, im)).  ``kernel`` is a
    name of KERNELS or a KernelTable."""
    L = load()
    dirs, D, per = _dirs(dirs, tables.n, tables.B)
    shape = (tables.B, D, 2) if kernel == "fourier" else (tables.B, D)
    if out is None:
        out = torch.empty(shape, dtype=torch.float64, device=dirs.device)
    if isinstance(kernel, KernelTable):
        _check(L.hybrid_transform_table(tables.handle, kernel.handle, PRECISIONS[precision], _ptr(dirs), D, per,
                                        _ptr(out), _stream(stream)))
        return out
    _check(L.hybrid_transform(tables.handle, KERNELS[kernel], PRECISIONS[precision], _ptr(dirs), D, per,
                              _ptr(out), _stream(stream)))
    return out


def hybrid_transform_grad(tables: Tables, kernel, dirs: torch.Tensor, gout: torch.Tensor,
                          precision: str = "fp32c", out=None, stream=None):
    """sum over outputs of gout * dHT/dxi, shaped like dirs (float64)."""
    L = load()
    dirs, D, per = _dirs(dirs, tables.n, tables.B)
    gout = gout.contiguous().to(torch.float64)
    if out is None:
        out = torch.empty_like(dirs)
    if isinstance(kernel, KernelTable):
        _check(L.hybrid_transform_table_grad(tables.handle, kernel.handle, PRECISIONS[precision], _ptr(dirs), D,
                                             per, _ptr(gout), _ptr(out), _stream(stream)))
        return out
    _check(L.hybrid_transform_grad(tables.handle, KERNELS[kernel], PRECISIONS[precision], _ptr(dirs), D, per,
                                   _ptr(gout), _ptr(out), _stream(stream)))
    return out


class HybridTransform(torch.autograd.Function):
    """HT as a differentiable function of the directions (adjoint kernel in backward)."""

    @staticmethod
    def forward(ctx, dirs, tables, kernel, precision):
        ctx.tables, ctx.kernel, ctx.precision = tables, kernel, precision
        ctx.save_for_backward(dirs)
        return hybrid_transform(tables, kernel, dirs.detach(), precision)

    @staticmethod
    def backward(ctx, gout):
        (dirs,) = ctx.saved_tensors
        g = hybrid_transform_grad(ctx.tables, ctx.kernel, dirs.detach(), gout, ctx.precision)
        return g, None, None, None


class Pipeline:
    """Extraction + ECT (+ Radon) + hybrid transforms of a fixed batch layout, replayed as
    one CUDA graph.

    The tables handle, the pixel buffer and every output are allocated once; ``run``
    copies new pixels into the captured input buffer and replays the graph (no host
    synchronisation, no allocation, every kernel of the path in one graph launch).  In
    the graph the grid transforms (ECT, Radon) run on a second stream beside the hybrid
    transforms: the handle gives each family of calls its own workspace.  With
    ``tune=True``, ``capture`` first picks the tile shapes of every operation with the
    autotuner (cached per GPU and size, see autotune.py).
    """

    def __init__(self, shapes, offsets, n_pixels: int, dtype=U8, ect=None, radon=None, hybrid=(),
                 device="cuda", tune: bool = False):
        """ect / radon: (dirs, t_min, t_max, T) or None; hybrid: list of (kernel, dirs, precision)."""
        self.tables = tables_create(shapes, offsets, dtype)
        tdt = torch.uint8 if dtype == U8 else torch.int32
        self.pixels = torch.zeros(n_pixels, dtype=tdt, device=device)
        self.ect_args, self.radon_args, self.hybrid_args = ect, radon, list(hybrid)
        B = self.tables.B
        self.ect_out = None if ect is None else torch.empty(
            (B, ect[0].shape[-2], ect[3]), dtype=torch.int32, device=device)
        self.radon_out = None if radon is None else torch.empty(
            (B, radon[0].shape[-2], radon[3]), dtype=torch.int32, device=device)
        self.hybrid_out = []
        for kernel, dirs, _prec in self.hybrid_args:
            D = dirs.shape[-2]
            shape = (B, D, 2) if kernel == "fourier" else (B, D)
            self.hybrid_out.append(torch.empty(shape, dtype=torch.float64, device=device))
        self.graph = None
        self.tune = tune
        self.tuned = {}
        self.side = torch.cuda.Stream(device=device)

    def _grid(self):
        if self.ect_args is not None:
            d, a, b, T = self.ect_args
            ect(self.tables, d, a, b, T, out=self.ect_out)
        if self.radon_args is not None:
            d, a, b, T = self.radon_args
            radon(self.tables, d, a, b, T, out=self.radon_out)

    def _hybrid(self):
        for (kernel, d, prec), out in zip(self.hybrid_args, self.hybrid_out):
            hybrid_transform(self.tables, kernel, d, prec, out=out)

    def _launch(self):
        self.tables.build(self.pixels)
        if (self.ect_args is not None or self.radon_args is not None) and self.hybrid_args:
            main = torch.cuda.current_stream()
            self.side.wait_stream(main)
            with torch.cuda.stream(self.side):
                self._grid()
            self._hybrid()
            main.wait_stream(self.side)
        else:
            self._grid()
            self._hybrid()

    def _autotune(self):
        from . import autotune
        if self.ect_args is not None:
            d, a, b, T = self.ect_args
            self.tuned["ect"] = autotune.tune(self.tables, "ect", d, t_min=a, t_max=b, T=T)["tuning"]
        if self.radon_args is not None:
            d, a, b, T = self.radon_args
            self.tuned["radon"] = autotune.tune(self.tables, "radon", d, t_min=a, t_max=b, T=T)["tuning"]
        for kernel, d, prec in self.hybrid_args:   # one tiling per handle: the last kernel's wins
            self.tuned[kernel] = autotune.tune(self.tables, "hybrid", d, kernel=kernel, precision=prec)["tuning"]

    def capture(self):
        """Run once eagerly (sizes every workspace; tunes the tiles when asked), then capture
        the launch sequence."""
        self._launch()
        torch.cuda.synchronize()
        self.tables.sync()
        if self.tune:
            self._autotune()
            self._launch()   # the workspaces of the chosen tiles
            torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._launch()
        torch.cuda.synchronize()
        return self

    def run(self, pixels=None):
        if pixels is not None:
            self.pixels.copy_(pixels, non_blocking=True)
        if self.graph is None:
            self._launch()
        else:
            self.graph.replay()
        return self
