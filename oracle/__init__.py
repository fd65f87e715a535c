"""CPU FP64 oracle for the product-to-sum element-matrix fill -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs
of ``bench.py`` may import this package.  The product path (the CUDA library in
``paper_1703_09619_gb300``) never imports, links or executes anything here, and
this package imports nothing from the product.

The numerical work lives in ``oracle.c`` (plain C, FP64, Neumaier summation,
pthread pool over matrix rows); this module compiles it with gcc on first use
and exposes it through ctypes.  Each function cites the passage of
Khodapanah, arXiv:1703.09619, that it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ALPHA_SCALAR = 0
ALPHA_METRIC_EPS = 1
ALPHA_POLY = 2
POLY_DEG = 8

TYPES = ("vv", "dv", "vd", "dd")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
               "-fno-fast-math", "-pthread", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d, i32, i64, u32 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
            P = ctypes.c_void_p
            lib.or_legendre.argtypes = [ctypes.c_int, d, P, P]
            lib.or_legendre.restype = None
            lib.or_gauss_legendre.argtypes = [ctypes.c_int, P, P]
            lib.or_gauss_legendre.restype = ctypes.c_int
            lib.or_map.argtypes = [P, P, d, d, d, P, P]
            lib.or_map.restype = None
            lib.or_alpha.argtypes = [ctypes.c_int, P, P, P, d, d, d, P]
            lib.or_alpha.restype = d
            lib.or_alpha_nparams.argtypes = [ctypes.c_int]
            lib.or_alpha_nparams.restype = ctypes.c_int
            lib.or_output_offsets.argtypes = [i64, ctypes.c_int, P, u32, P]
            lib.or_output_offsets.restype = i64
            lib.or_fill.argtypes = [i64, ctypes.c_int, P, ctypes.c_int, P, P, P, P, u32, P, ctypes.c_int]
            lib.or_fill_terms.restype = ctypes.c_int
            lib.or_fill_terms.argtypes = [i64, ctypes.c_int, P, ctypes.c_int, P, P, P, P, ctypes.c_int, P, P, P,
                                          ctypes.c_int]
            lib.or_fill.restype = ctypes.c_int
            lib.or_linearisation.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, P]
            lib.or_linearisation.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def legendre(n: int, x: float):
    """P_j(x), P'_j(x) for j < n: three-term recurrence (values) and
    (1-x^2) P'_j = j (P_{j-1} - x P_j) (derivatives).  Basis of Eq. (1)."""
    P = np.zeros(n)
    dP = np.zeros(n)
    _load().or_legendre(n, float(x), _ptr(P), _ptr(dP))
    return P, dP


def gauss_legendre(G: int):
    """G-point Gauss-Legendre rule on [-1, 1] (Newton on P_G); the quadrature of Eq. (2)."""
    x = np.zeros(G)
    w = np.zeros(G)
    rc = _load().or_gauss_legendre(G, _ptr(x), _ptr(w))
    if rc:
        raise ValueError("bad G")
    return x, w


def geometry_map(nodes, bulge, u, v, w):
    """Trilinear-plus-bulge map x(u,v,w) and J = dx/d(u,v,w) of one element."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(8, 3)
    b = None if bulge is None else np.ascontiguousarray(bulge, dtype=np.float64).reshape(4)
    x = np.zeros(3)
    J = np.zeros(9)
    _load().or_map(_ptr(nodes), _ptr(b), float(u), float(v), float(w), _ptr(x), _ptr(J))
    return x, J.reshape(3, 3)


def alpha_point(kind, params, nodes, bulge, u, v, w):
    """Coupling factors alpha_{gi gj}(u,v,w) of Eq. (2) at one point; returns (alpha, detJ)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    nd = None if nodes is None else np.ascontiguousarray(nodes, dtype=np.float64).reshape(8, 3)
    b = None if bulge is None else np.ascontiguousarray(bulge, dtype=np.float64).reshape(4)
    out = np.zeros(9)
    det = _load().or_alpha(int(kind), _ptr(p), _ptr(nd), _ptr(b), float(u), float(v), float(w), _ptr(out))
    nc = 3 if kind == ALPHA_METRIC_EPS else 1
    return out[: nc * nc].reshape(nc, nc), det


def output_offsets(orders, types_mask=0xF):
    """Per-element entry offsets (E+1) of the concatenated output."""
    orders = np.ascontiguousarray(orders, dtype=np.int32)
    E, nc = orders.shape[0], orders.shape[1]
    off = np.zeros(E + 1, dtype=np.int64)
    _load().or_output_offsets(E, nc, _ptr(orders), types_mask, _ptr(off))
    return off


def fill(orders, kind, params, nodes, bulge, npts, types_mask=0xF, nthreads=None):
    """Direct triple Gauss-Legendre fill of Eq. (2) for every entry (FP64, Neumaier).

    orders: int32 [E, n_comp, 3]; params: float64 [E, nparams(kind)];
    nodes: float64 [E, 8, 3]; bulge: float64 [E, 4] or None; npts: int32 [E] or int.
    Returns (flat float64 output, int64 offsets[E+1], status)."""
    lib = _load()
    orders = np.ascontiguousarray(orders, dtype=np.int32)
    E, nc = orders.shape[0], orders.shape[1]
    params = np.ascontiguousarray(params, dtype=np.float64).reshape(E, -1)
    if params.shape[1] != lib.or_alpha_nparams(int(kind)):
        raise ValueError("params has %d columns, kind %d wants %d" % (params.shape[1], kind,
                                                                       lib.or_alpha_nparams(int(kind))))
    if nodes is None:
        nodes = np.zeros((E, 8, 3))
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(E, 8, 3)
    if bulge is not None:
        bulge = np.ascontiguousarray(bulge, dtype=np.float64).reshape(E, 4)
    if np.isscalar(npts):
        npts = np.full(E, int(npts), dtype=np.int32)
    npts = np.ascontiguousarray(npts, dtype=np.int32).reshape(E)
    off = output_offsets(orders, types_mask)
    out = np.zeros(int(off[-1]), dtype=np.float64)
    rc = lib.or_fill(E, nc, _ptr(orders), int(kind), _ptr(params), _ptr(nodes), _ptr(bulge), _ptr(npts),
                     types_mask, _ptr(out), int(nthreads or default_threads()))
    if rc not in (0, -3):
        raise RuntimeError("oracle fill failed: %d" % rc)
    return out, off, rc


def fill_terms(orders, kind, params, nodes, bulge, npts, terms, scales, nthreads=None):
    """Direct triple Gauss-Legendre fill of an operator given as a term list (Eq. (2) with
    the value/derivative choice per axis and several coupling-factor entries summed).

    terms: int [T, 10] rows (gi, gj, sa, sb, du, dv, dw, eu, ev, ew): block (gi, gj),
    coupling entry alpha[sa][sb], derivative orders of the test (d*) and trial (e*)
    functions per axis; scales: float [T].  Returns (flat output: one n x n matrix per
    element, offsets[E+1], status)."""
    lib = _load()
    orders = np.ascontiguousarray(orders, dtype=np.int32)
    E, nc = orders.shape[0], orders.shape[1]
    params = np.ascontiguousarray(params, dtype=np.float64).reshape(E, -1)
    if nodes is None:
        nodes = np.zeros((E, 8, 3))
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(E, 8, 3)
    if bulge is not None:
        bulge = np.ascontiguousarray(bulge, dtype=np.float64).reshape(E, 4)
    if np.isscalar(npts):
        npts = np.full(E, int(npts), dtype=np.int32)
    npts = np.ascontiguousarray(npts, dtype=np.int32).reshape(E)
    terms = np.ascontiguousarray(terms, dtype=np.int32).reshape(-1, 10)
    scales = np.ascontiguousarray(scales, dtype=np.float64).reshape(-1)
    if terms.shape[0] != scales.shape[0]:
        raise ValueError("terms and scales differ in length")
    off = output_offsets(orders, 1)
    out = np.zeros(int(off[-1]), dtype=np.float64)
    rc = lib.or_fill_terms(E, nc, _ptr(orders), int(kind), _ptr(params), _ptr(nodes), _ptr(bulge), _ptr(npts),
                           int(terms.shape[0]), _ptr(terms), _ptr(scales), _ptr(out), int(nthreads or default_threads()))
    if rc not in (0, -3):
        raise RuntimeError("oracle term fill failed: %d" % rc)
    return out, off, rc


def element_matrices(out, off, orders, e, types_mask=0xF):
    """Split element e's slice of a flat output into {type: n x n matrix}."""
    orders = np.asarray(orders)
    n = int(sum(int(np.prod(orders[e, g])) for g in range(orders.shape[1])))
    res = {}
    slot = 0
    for t in range(4):
        if types_mask & (1 << t):
            s = int(off[e]) + slot * n * n
            res[TYPES[t]] = out[s:s + n * n].reshape(n, n)
            slot += 1
    return res


def linearisation(d1, d2, m1, m2, kmax):
    """Coefficients C_k of Eq. (3), P^{(d1)}_{m1} P^{(d2)}_{m2} = sum_k C_k P_k, by
    exact Gauss-Legendre projection onto P_k (Legendre orthogonality)."""
    C = np.zeros(kmax + 1)
    rc = _load().or_linearisation(int(d1), int(d2), int(m1), int(m2), int(kmax), _ptr(C))
    if rc:
        raise ValueError("bad linearisation arguments")
    return C


class use_library:
    """Context manager that points this module at another build of oracle.c.

    Only the mutation tests use it: they compile copies of oracle.c with a
    planted mistake and check that the pins catch it."""

    def __init__(self, path):
        self.path = path
        self.saved = None

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        lib = ctypes.CDLL(self.path)
        for name in ("or_legendre", "or_gauss_legendre", "or_map", "or_alpha", "or_alpha_nparams",
                     "or_output_offsets", "or_fill", "or_linearisation"):
            f, g = getattr(lib, name), getattr(self.saved, name)
            f.argtypes, f.restype = g.argtypes, g.restype
        _lib = lib
        return lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def build_variant(source_text: str, out_path: str) -> str:
    """Compile an edited copy of oracle.c (used by the mutation tests only)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                    "-fno-fast-math", "-pthread", "-o", out_path, src, "-lm"], check=True)
    return out_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()
