"""Thin Python binding of libp2s (the C ABI in include/p2s.h).

Argument marshalling only: torch tensors become raw device pointers, the current
torch stream becomes the cudaStream_t, host arrays become host pointers.  Every
step of the fill runs in the library's CUDA kernels.  Importing this module does
not need a GPU; using it does, and it raises if libp2s.so has not been built.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libp2s.so")

OK, ERR_ARG, ERR_ORDER, ERR_JACOBIAN, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_BUFFER = 0, -1, -2, -3, -4, -5, -6, -7
MAX_ORDER, MAX_NPTS = 12, 64
ALPHA_SCALAR, ALPHA_METRIC_EPS = 0, 1
FP64, MIXED = 0, 1
TYPES_ALL = 0xF
TYPES = ("vv", "dv", "vd", "dd")


class P2SError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = error_string(code) if _lib is not None else str(code)
        detail = _lib.p2s_last_error().decode() if _lib is not None else ""
        self.detail = detail
        text = "%s: %s (%d)" % (what, msg, code) if what else "%s (%d)" % (msg, code)
        super().__init__(text + ("; " + detail if detail else ""))


class Geometry(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int64), ("nodes", ctypes.c_void_p), ("bulge", ctypes.c_void_p)]


class Material(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("params", ctypes.c_void_p)]


class Orders(ctypes.Structure):
    _fields_ = [("n_comp", ctypes.c_int), ("orders", ctypes.c_void_p)]


class Quadrature(ctypes.Structure):
    _fields_ = [("npts_uniform", ctypes.c_int), ("npts", ctypes.c_void_p)]


class FillOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("types_mask", ctypes.c_uint32)]


class Term(ctypes.Structure):
    """p2s_term: one term of an operator (block, coupling entry, per-axis derivatives, scale)."""
    _fields_ = [("gi", ctypes.c_int32), ("gj", ctypes.c_int32), ("sa", ctypes.c_int32), ("sb", ctypes.c_int32),
                ("d_test", ctypes.c_int32 * 3), ("d_trial", ctypes.c_int32 * 3), ("scale", ctypes.c_double)]


class TileConfig(ctypes.Structure):
    """p2s_tile_config: contraction work-unit shape (zero fields: library default)."""
    _fields_ = [("combo_target", ctypes.c_int), ("unit_kbytes", ctypes.c_int), ("threads", ctypes.c_int),
                ("kernel", ctypes.c_int)]

    def as_dict(self):
        return {"combo_target": self.combo_target, "unit_kbytes": self.unit_kbytes, "threads": self.threads,
                "kernel": self.kernel}


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes); every symbol include/p2s.h declares
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
SIGNATURES = {
    "p2s_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]),
    "p2s_destroy": (None, [_P]),
    "p2s_output_entries": (_I64, [_I64, ctypes.POINTER(Orders), ctypes.c_uint32, _P]),
    "p2s_moment_entries": (_I64, [_I64, ctypes.POINTER(Orders), _P]),
    "p2s_plan_create": (ctypes.c_int, [_P, _I64, ctypes.POINTER(Orders), ctypes.POINTER(Quadrature),
                                       ctypes.POINTER(FillOpts), ctypes.POINTER(ctypes.c_void_p)]),
    "p2s_plan_create_tuned": (ctypes.c_int, [_P, _I64, ctypes.POINTER(Orders), ctypes.POINTER(Quadrature),
                                             ctypes.POINTER(FillOpts), _P, ctypes.POINTER(ctypes.c_void_p)]),
    "p2s_plan_tile_config": (ctypes.c_int, [_P, ctypes.POINTER(TileConfig)]),
    "p2s_operator_plan_create": (ctypes.c_int, [_P, _I64, ctypes.POINTER(Orders), ctypes.POINTER(Quadrature),
                                                ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P,
                                                ctypes.POINTER(ctypes.c_void_p)]),
    "p2s_autotune_tiles": (ctypes.c_int, [_P, ctypes.POINTER(Geometry), ctypes.POINTER(Material),
                                          ctypes.POINTER(Orders), ctypes.POINTER(Quadrature),
                                          ctypes.POINTER(FillOpts), _I64, ctypes.c_int, ctypes.POINTER(TileConfig),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), _P]),
    "p2s_plan_use_graph": (ctypes.c_int, [_P, ctypes.c_int]),
    "p2s_plan_destroy": (None, [_P]),
    "p2s_plan_output_entries": (_I64, [_P]),
    "p2s_plan_moment_entries": (_I64, [_P]),
    "p2s_plan_moments": (ctypes.c_int, [_P, ctypes.POINTER(Geometry), ctypes.POINTER(Material), _P, _P, _P]),
    "p2s_plan_contract": (ctypes.c_int, [_P, _P, _P, _P]),
    "p2s_plan_fill": (ctypes.c_int, [_P, ctypes.POINTER(Geometry), ctypes.POINTER(Material), _P, _P, _P]),
    "p2s_fill_elements": (ctypes.c_int, [_P, ctypes.POINTER(Geometry), ctypes.POINTER(Material),
                                         ctypes.POINTER(Orders), ctypes.POINTER(Quadrature),
                                         ctypes.POINTER(FillOpts), _P, _P, _P]),
    "p2s_fill_elements_noalloc": (ctypes.c_int, [_P, ctypes.POINTER(Geometry), ctypes.POINTER(Material),
                                                 ctypes.POINTER(Orders), ctypes.POINTER(Quadrature),
                                                 ctypes.POINTER(FillOpts), _P, _P, _P]),
    "p2s_assembly_structure_host": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   _P, _P, _P, _P]),
    "p2s_assembly_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, _P, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "p2s_assembly_destroy": (None, [_P]),
    "p2s_assembly_rows": (_I64, [_P]),
    "p2s_assembly_nnz": (_I64, [_P]),
    "p2s_assembly_use_graph": (ctypes.c_int, [_P, ctypes.c_int]),
    "p2s_assembly_fused": (ctypes.c_int, [_P]),
    "p2s_assembly_fill": (ctypes.c_int, [_P, ctypes.POINTER(Geometry), ctypes.POINTER(Material), _P, _P]),
    "p2s_assembly_add": (ctypes.c_int, [_P, _P, _P, _P]),
    "p2s_assembly_reassemble": (ctypes.c_int, [_P, _P, _P]),
    "p2s_cheb2d_dofs": (_I64, [ctypes.c_int, ctypes.c_int]),
    "p2s_cheb2d_fill": (ctypes.c_int, [_P, _I64, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, _P, _P, _P]),
    "p2s_sync_status": (ctypes.c_int, [_P, _P]),
    "p2s_linearisation": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "p2s_gauss_legendre": (ctypes.c_int, [ctypes.c_int, _P, _P]),
    "p2s_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "p2s_last_error": (ctypes.c_char_p, []),
    "p2s_learned_npts": (ctypes.c_int, [ctypes.c_int]),
    "p2s_coarse_features": (ctypes.c_int, [_P, ctypes.POINTER(Geometry), ctypes.POINTER(Material), _P, _P]),
    "p2s_mlp_predict": (ctypes.c_int, [_P, _P, _P, _I64, ctypes.c_int, ctypes.c_float, _P, _P, _P]),
    "p2s_mlp_predict_ensemble": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _I64, ctypes.c_int, ctypes.c_float, _P, _P,
                                                _P]),
    "p2s_mlp_grad": (ctypes.c_int, [_P, _P, _P, _P, _I64, _P, _P, _P, _P]),
    "p2s_mlp_adam": (ctypes.c_int, [_P, _P, _P, _P, _I64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, ctypes.c_int, _P]),
    "p2s_element_errors": (ctypes.c_int, [_P, _P, _P, _P, _P, _I64, ctypes.c_int, _P, _P]),
    "p2s_judge_select": (ctypes.c_int, [_I64, ctypes.c_double, ctypes.c_uint64, _P]),
    "p2s_learned_plan_create": (ctypes.c_int, [_P, _I64, ctypes.POINTER(Orders), _P, ctypes.POINTER(ctypes.c_void_p)]),
    "p2s_learned_plan_destroy": (None, [_P]),
    "p2s_learned_plan_output_entries": (_I64, [_P]),
    "p2s_learned_fill": (ctypes.c_int, [_P, ctypes.POINTER(Geometry), ctypes.POINTER(Material), _P, _P, _P, _P]),
    "p2s_learned_report_get": (ctypes.c_int, [_P, _P, _P, _P]),
    "p2s_measure_peaks": (ctypes.c_int, [_P, _I64, _P, _P]),
    "p2s_mode1_product": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _I64, _I64, _P, _P]),
}
MODE1_SIMT, MODE1_TC = 0, 1

MLP_IN, MLP_HIDDEN, MLP_CLASSES, MLP_PARAMS = 576, 64, 6, 41478
MLP_MAX_NETS = 8  # P2S_MLP_MAX_NETS: networks of one ensemble
CLASS_NPTS = (8, 12, 16, 24, 32, 48)


class Peaks(ctypes.Structure):
    _fields_ = [("fp64_fma_tflops", ctypes.c_double), ("fp32_fma_tflops", ctypes.c_double),
                ("hbm_write_gbs", ctypes.c_double), ("fp64_ms", ctypes.c_double), ("fp32_ms", ctypes.c_double),
                ("write_ms", ctypes.c_double), ("write_bytes", ctypes.c_int64)]


class LearnedOpts(ctypes.Structure):
    _fields_ = [("margin", ctypes.c_int), ("risk", ctypes.c_double), ("precision", ctypes.c_int),
                ("judge_frac", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("judge_tol", ctypes.c_double), ("n_nets", ctypes.c_int)]


class LearnedReport(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int64), ("judged", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("per_class", ctypes.c_int64 * 6), ("max_judged_err", ctypes.c_double)]


def load():
    """Load libp2s.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libp2s.so is not built (run __graft_entry__.build() or "
                                   "python paper_1703_09619_gb300/build.py)")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def error_string(code: int) -> str:
    return load().p2s_error_string(int(code)).decode()


def _check(rc, what):
    if rc != OK:
        raise P2SError(rc, what)


def _hptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _dptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _orders_struct(orders):
    orders = np.ascontiguousarray(orders, dtype=np.int32)
    return Orders(int(orders.shape[1]), ctypes.c_void_p(orders.ctypes.data)), orders


def output_entries(orders, types_mask=TYPES_ALL, offsets=False):
    """Total FP64 entries (and optionally the per-element offsets) of a fill."""
    o, keep = _orders_struct(orders)
    E = keep.shape[0]
    off = np.zeros(E + 1, dtype=np.int64) if offsets else None
    n = load().p2s_output_entries(E, ctypes.byref(o), types_mask, _hptr(off))
    if n < 0:
        raise P2SError(int(n), "p2s_output_entries")
    return (n, off) if offsets else n


def moment_entries(orders, offsets=False):
    o, keep = _orders_struct(orders)
    E = keep.shape[0]
    off = np.zeros(E + 1, dtype=np.int64) if offsets else None
    n = load().p2s_moment_entries(E, ctypes.byref(o), _hptr(off))
    if n < 0:
        raise P2SError(int(n), "p2s_moment_entries")
    return (n, off) if offsets else n


def linearisation(t, m1, m2, kmax):
    C = np.zeros(kmax + 1)
    _check(load().p2s_linearisation(int(t), int(m1), int(m2), int(kmax), _hptr(C)), "p2s_linearisation")
    return C


def gauss_legendre(G):
    x = np.zeros(G)
    w = np.zeros(G)
    _check(load().p2s_gauss_legendre(int(G), _hptr(x), _hptr(w)), "p2s_gauss_legendre")
    return x, w


class Context:
    """A p2s_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.p2s_create(ctypes.byref(h), int(device)), "p2s_create")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            load().p2s_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync_status(self, stream=None) -> int:
        return int(load().p2s_sync_status(self.handle, _stream(stream)))


class Plan:
    """A p2s_plan: descriptors, work list and launch shapes for one batch shape."""

    def __init__(self, ctx: Context, orders, npts, precision=FP64, types_mask=TYPES_ALL, tile=None, graph=False):
        """tile: a TileConfig or dict (combo_target, unit_kbytes, threads, kernel) for
        p2s_plan_create_tuned; graph: replay fills from a CUDA graph (p2s_plan_use_graph)."""
        lib = load()
        self.ctx = ctx
        o, self._orders = _orders_struct(orders)
        E = self._orders.shape[0]
        q, self._npts = _quadrature_struct(npts, E)
        opts = FillOpts(int(precision), int(types_mask))
        h = ctypes.c_void_p()
        if tile is None:
            _check(lib.p2s_plan_create(ctx.handle, E, ctypes.byref(o), ctypes.byref(q), ctypes.byref(opts),
                                       ctypes.byref(h)), "p2s_plan_create")
        else:
            t = tile if isinstance(tile, TileConfig) else TileConfig(**tile)
            _check(lib.p2s_plan_create_tuned(ctx.handle, E, ctypes.byref(o), ctypes.byref(q), ctypes.byref(opts),
                                             ctypes.byref(t), ctypes.byref(h)), "p2s_plan_create_tuned")
        self.handle = h
        self.n_elem = E
        self.n_comp = int(self._orders.shape[1])
        self.types_mask = types_mask
        self.precision = precision
        self.output_entries = int(lib.p2s_plan_output_entries(h))
        self.moment_entries = int(lib.p2s_plan_moment_entries(h))
        if graph:
            self.use_graph(True)

    def tile_config(self) -> dict:
        t = TileConfig()
        _check(load().p2s_plan_tile_config(self.handle, ctypes.byref(t)), "p2s_plan_tile_config")
        return t.as_dict()

    def use_graph(self, enable=True):
        _check(load().p2s_plan_use_graph(self.handle, int(bool(enable))), "p2s_plan_use_graph")

    def close(self):
        if getattr(self, "handle", None):
            load().p2s_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _inputs(kind, params, nodes, bulge):
        g = Geometry(int(params.shape[0]), _dptr(nodes), _dptr(bulge))
        m = Material(int(kind), _dptr(params))
        return g, m

    def moments(self, kind, params, nodes, bulge, moments, elem_status=None, stream=None):
        g, m = self._inputs(kind, params, nodes, bulge)
        _check(load().p2s_plan_moments(self.handle, ctypes.byref(g), ctypes.byref(m), _dptr(moments),
                                       _dptr(elem_status), _stream(stream)), "p2s_plan_moments")

    def contract(self, moments, out, stream=None):
        _check(load().p2s_plan_contract(self.handle, _dptr(moments), _dptr(out), _stream(stream)),
               "p2s_plan_contract")

    def fill(self, kind, params, nodes, bulge, out, elem_status=None, stream=None):
        g, m = self._inputs(kind, params, nodes, bulge)
        _check(load().p2s_plan_fill(self.handle, ctypes.byref(g), ctypes.byref(m), _dptr(out),
                                    _dptr(elem_status), _stream(stream)), "p2s_plan_fill")


def _quadrature_struct(npts, E):
    if np.isscalar(npts):
        return Quadrature(int(npts), None), None
    keep = np.ascontiguousarray(npts, dtype=np.int32).reshape(E)
    return Quadrature(0, ctypes.c_void_p(keep.ctypes.data)), keep


def autotune_tiles(ctx: Context, orders, npts, kind, params, nodes, bulge, precision=FP64, types_mask=TYPES_ALL,
                   sample=0, reps=3, stream=None):
    """p2s_autotune_tiles: the fastest contraction tile configuration on the leading
    `sample` elements (0: all).  Returns (config dict, best ms, candidates tried)."""
    lib = load()
    o, keep = _orders_struct(orders)
    E = keep.shape[0]
    q, npk = _quadrature_struct(npts, E)
    g = Geometry(E, _dptr(nodes), _dptr(bulge))
    m = Material(int(kind), _dptr(params))
    opts = FillOpts(int(precision), int(types_mask))
    best = TileConfig()
    ms = ctypes.c_double()
    tried = ctypes.c_int()
    _check(lib.p2s_autotune_tiles(ctx.handle, ctypes.byref(g), ctypes.byref(m), ctypes.byref(o), ctypes.byref(q),
                                  ctypes.byref(opts), int(sample), int(reps), ctypes.byref(best), ctypes.byref(ms),
                                  ctypes.byref(tried), _stream(stream)), "p2s_autotune_tiles")
    return best.as_dict(), ms.value, tried.value


def terms_struct(terms, scales):
    """A p2s_term array from rows (gi, gj, sa, sb, du, dv, dw, eu, ev, ew) and scales."""
    terms = np.asarray(terms, dtype=np.int64).reshape(-1, 10)
    scales = np.asarray(scales, dtype=np.float64).reshape(-1)
    if terms.shape[0] != scales.shape[0]:
        raise ValueError("terms and scales differ in length")
    arr = (Term * max(1, terms.shape[0]))()
    for k, (row, sc) in enumerate(zip(terms, scales)):
        arr[k].gi, arr[k].gj, arr[k].sa, arr[k].sb = (int(x) for x in row[:4])
        for x in range(3):
            arr[k].d_test[x] = int(row[4 + x])
            arr[k].d_trial[x] = int(row[7 + x])
        arr[k].scale = float(sc)
    return arr, terms.shape[0]


class OperatorPlan(Plan):
    """A p2s_plan of an operator given as a term list (p2s_operator_plan_create): one n x n
    matrix per element, the sum of its terms.  terms: rows (gi, gj, sa, sb, du, dv, dw, eu, ev,
    ew) -- block, coupling entry alpha[sa][sb], derivative orders of the test (d*) and trial
    (e*) functions per axis; scales alongside."""

    def __init__(self, ctx: Context, orders, npts, terms, scales, kind, precision=FP64, tile=None, graph=False):
        lib = load()
        self.ctx = ctx
        o, self._orders = _orders_struct(orders)
        E = self._orders.shape[0]
        q, self._npts = _quadrature_struct(npts, E)
        self._terms, nt = terms_struct(terms, scales)
        t = None if tile is None else (tile if isinstance(tile, TileConfig) else TileConfig(**tile))
        h = ctypes.c_void_p()
        _check(lib.p2s_operator_plan_create(ctx.handle, E, ctypes.byref(o), ctypes.byref(q), int(precision), int(kind),
                                            ctypes.cast(self._terms, ctypes.c_void_p), nt,
                                            ctypes.byref(t) if t is not None else None, ctypes.byref(h)),
               "p2s_operator_plan_create")
        self.handle = h
        self.n_elem = E
        self.n_comp = int(self._orders.shape[1])
        self.types_mask = 1
        self.precision = precision
        self.kind = kind
        self.output_entries = int(lib.p2s_plan_output_entries(h))
        self.moment_entries = int(lib.p2s_plan_moment_entries(h))
        if graph:
            self.use_graph(True)


def assembly_structure(nx, ny, nz, order):
    """CSR structure (row_ptr int64 [rows + 1], col_idx int32 [nnz]) of the global matrix of an
    nx x ny x nz structured mesh with `order` per axis (p2s_assembly_structure_host, host only)."""
    lib = load()
    rows, nnz = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.p2s_assembly_structure_host(nx, ny, nz, order, ctypes.byref(rows), ctypes.byref(nnz), None, None),
           "p2s_assembly_structure_host")
    row_ptr = np.zeros(rows.value + 1, dtype=np.int64)
    col_idx = np.zeros(nnz.value, dtype=np.int32)
    _check(lib.p2s_assembly_structure_host(nx, ny, nz, order, None, None, _hptr(row_ptr), _hptr(col_idx)),
           "p2s_assembly_structure_host")
    return row_ptr, col_idx


class Assembly:
    """A p2s_assembly: operator fill of a structured mesh's elements plus the deterministic
    scatter into one global CSR matrix in the hierarchic C0 basis."""

    def __init__(self, ctx: Context, nx, ny, nz, order, npts, terms, scales, kind, precision=FP64, graph=False):
        lib = load()
        self.ctx = ctx
        self._terms, nt = terms_struct(terms, scales)
        h = ctypes.c_void_p()
        _check(lib.p2s_assembly_create(ctx.handle, nx, ny, nz, order, int(npts), int(precision), int(kind),
                                       ctypes.cast(self._terms, ctypes.c_void_p), nt, ctypes.byref(h)),
               "p2s_assembly_create")
        self.handle = h
        self.shape = (nx, ny, nz)
        self.order = order
        self.n_elem = nx * ny * nz
        self.rows = int(lib.p2s_assembly_rows(h))
        self.nnz = int(lib.p2s_assembly_nnz(h))
        self.fused = bool(lib.p2s_assembly_fused(h))
        if graph:
            _check(lib.p2s_assembly_use_graph(h, 1), "p2s_assembly_use_graph")

    def structure(self):
        return assembly_structure(*self.shape, self.order)

    def fill(self, kind, params, nodes, bulge, values, stream=None):
        g, m = Plan._inputs(kind, params, nodes, bulge)
        _check(load().p2s_assembly_fill(self.handle, ctypes.byref(g), ctypes.byref(m), _dptr(values),
                                        _stream(stream)), "p2s_assembly_fill")

    def reassemble(self, values, stream=None):
        """Assemble the element matrices of the last fill again into `values` (overwritten)."""
        _check(load().p2s_assembly_reassemble(self.handle, _dptr(values), _stream(stream)),
               "p2s_assembly_reassemble")

    def add(self, emat, values, stream=None):
        """Add Legendre-basis element matrices (device [E][n][n]) to `values` (not zeroed)."""
        _check(load().p2s_assembly_add(self.handle, _dptr(emat), _dptr(values), _stream(stream)),
               "p2s_assembly_add")

    def close(self):
        if getattr(self, "handle", None):
            load().p2s_assembly_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


CHEB2D_P2S, CHEB2D_DIRECT = 0, 1


def cheb2d_dofs(M, N):
    n = load().p2s_cheb2d_dofs(int(M), int(N))
    if n < 0:
        raise P2SError(int(n), "p2s_cheb2d_dofs")
    return int(n)


def cheb2d_fill(ctx: Context, params, M, N, npts, S, Mass, method=CHEB2D_P2S, precision=FP64, stream=None):
    """p2s_cheb2d_fill: stiffness and mass matrices of the 2-D curl-curl example (device params
    [E][5], outputs [E][n][n] float64 each)."""
    _check(load().p2s_cheb2d_fill(ctx.handle, int(params.shape[0]), _dptr(params), int(M), int(N), int(npts),
                                  int(method), int(precision), _dptr(S), _dptr(Mass), _stream(stream)),
           "p2s_cheb2d_fill")


def fill_elements(ctx: Context, orders, npts, kind, params, nodes, bulge, out, elem_status=None,
                  precision=FP64, types_mask=TYPES_ALL, stream=None):
    """One-shot fill through p2s_fill_elements (synchronises the stream)."""
    lib = load()
    o, keep = _orders_struct(orders)
    E = keep.shape[0]
    if np.isscalar(npts):
        q = Quadrature(int(npts), None)
        npk = None
    else:
        npk = np.ascontiguousarray(npts, dtype=np.int32).reshape(E)
        q = Quadrature(0, ctypes.c_void_p(npk.ctypes.data))
    g = Geometry(E, _dptr(nodes), _dptr(bulge))
    m = Material(int(kind), _dptr(params))
    opts = FillOpts(int(precision), int(types_mask))
    _check(lib.p2s_fill_elements(ctx.handle, ctypes.byref(g), ctypes.byref(m), ctypes.byref(o), ctypes.byref(q),
                                 ctypes.byref(opts), _dptr(out), _dptr(elem_status), _stream(stream)),
           "p2s_fill_elements")


def fill_elements_noalloc(ctx: Context, orders, npts, kind, params, nodes, bulge, out, elem_status=None,
                          precision=FP64, types_mask=TYPES_ALL, stream=None):
    """Fill through p2s_fill_elements_noalloc: the library's fixed device scratch instead of
    any allocation, for callers that must not allocate device memory.  Asynchronous."""
    lib = load()
    o, keep = _orders_struct(orders)
    E = keep.shape[0]
    if np.isscalar(npts):
        q = Quadrature(int(npts), None)
        npk = None
    else:
        npk = np.ascontiguousarray(npts, dtype=np.int32).reshape(E)
        q = Quadrature(0, ctypes.c_void_p(npk.ctypes.data))
    g = Geometry(E, _dptr(nodes), _dptr(bulge))
    m = Material(int(kind), _dptr(params))
    opts = FillOpts(int(precision), int(types_mask))
    _check(lib.p2s_fill_elements_noalloc(ctx.handle, ctypes.byref(g), ctypes.byref(m), ctypes.byref(o),
                                         ctypes.byref(q), ctypes.byref(opts), _dptr(out), _dptr(elem_status),
                                         _stream(stream)), "p2s_fill_elements_noalloc")


def device_inputs(workload, device="cuda"):
    """Copy a workloads.Workload's geometry/material arrays to the device (torch tensors)."""
    import torch
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)
    return t(workload.params), t(workload.nodes), t(workload.bulge)


# ------------------------------------------------------------------ learned quadrature order
def coarse_features(ctx: Context, kind, params, nodes, bulge, features, stream=None):
    g = Geometry(int(params.shape[0]), _dptr(nodes), _dptr(bulge))
    m = Material(int(kind), _dptr(params))
    _check(load().p2s_coarse_features(ctx.handle, ctypes.byref(g), ctypes.byref(m), _dptr(features),
                                      _stream(stream)), "p2s_coarse_features")


def mlp_predict(ctx: Context, mlp_params, features, npts, margin=0, logits=None, risk=0.0, stream=None, n_nets=1):
    """p2s_mlp_predict, or p2s_mlp_predict_ensemble for n_nets > 1 (mlp_params then holds n_nets
    parameter sets one after another, and logits [n][6] is required)."""
    n = int(features.shape[0])
    if int(n_nets) == 1:
        _check(load().p2s_mlp_predict(ctx.handle, _dptr(mlp_params), _dptr(features), n, int(margin), float(risk),
                                      _dptr(npts), _dptr(logits), _stream(stream)), "p2s_mlp_predict")
    else:
        _check(load().p2s_mlp_predict_ensemble(ctx.handle, _dptr(mlp_params), int(n_nets), _dptr(features), n,
                                               int(margin), float(risk), _dptr(npts), _dptr(logits),
                                               _stream(stream)), "p2s_mlp_predict_ensemble")


def mlp_grad(ctx: Context, mlp_params, features, labels, grad, loss, class_weight=None, stream=None):
    n = int(features.shape[0])
    _check(load().p2s_mlp_grad(ctx.handle, _dptr(mlp_params), _dptr(features), _dptr(labels), n,
                               _dptr(class_weight), _dptr(grad), _dptr(loss), _stream(stream)), "p2s_mlp_grad")


def mlp_adam(mlp_params, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
    _check(load().p2s_mlp_adam(_dptr(mlp_params), _dptr(grad), _dptr(m), _dptr(v), int(mlp_params.numel()),
                               float(lr), float(beta1), float(beta2), float(eps), float(weight_decay), int(step),
                               _stream(stream)), "p2s_mlp_adam")


def element_errors(ctx: Context, a, offsets_a, b, offsets_b, n_types, err, stream=None):
    n = int(err.shape[0])
    _check(load().p2s_element_errors(ctx.handle, _dptr(a), _dptr(offsets_a), _dptr(b), _dptr(offsets_b), n,
                                     int(n_types), _dptr(err), _stream(stream)), "p2s_element_errors")


def judge_select(n_elem, frac, seed):
    out = np.zeros(max(int(n_elem), 1), dtype=np.int8)
    _check(load().p2s_judge_select(int(n_elem), float(frac), ctypes.c_uint64(int(seed)), _hptr(out)),
           "p2s_judge_select")
    return out[: int(n_elem)].astype(bool)


class LearnedPlan:
    """A p2s_learned_plan: learned-order fill with its seeded 48-point FP64 judge."""

    def __init__(self, ctx: Context, orders, margin=0, precision=MIXED, judge_frac=0.02, seed=1, judge_tol=1e-9,
                 risk=0.0, n_nets=1):
        lib = load()
        self.ctx = ctx
        o, self._orders = _orders_struct(orders)
        self.n_elem = int(self._orders.shape[0])
        opts = LearnedOpts(int(margin), float(risk), int(precision), float(judge_frac), int(seed), float(judge_tol),
                           int(n_nets))
        h = ctypes.c_void_p()
        _check(lib.p2s_learned_plan_create(ctx.handle, self.n_elem, ctypes.byref(o), ctypes.byref(opts),
                                           ctypes.byref(h)), "p2s_learned_plan_create")
        self.handle = h
        self.output_entries = int(lib.p2s_learned_plan_output_entries(h))

    def close(self):
        if getattr(self, "handle", None):
            load().p2s_learned_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fill(self, kind, params, nodes, bulge, mlp_params, out, npts_out=None, stream=None):
        g = Geometry(int(params.shape[0]), _dptr(nodes), _dptr(bulge))
        m = Material(int(kind), _dptr(params))
        _check(load().p2s_learned_fill(self.handle, ctypes.byref(g), ctypes.byref(m), _dptr(mlp_params), _dptr(out),
                                       _dptr(npts_out), _stream(stream)), "p2s_learned_fill")

    def report(self, stream=None, judge_state=False):
        rep = LearnedReport()
        js = np.zeros(max(self.n_elem, 1), dtype=np.int8) if judge_state else None
        _check(load().p2s_learned_report_get(self.handle, ctypes.byref(rep), _hptr(js), _stream(stream)),
               "p2s_learned_report_get")
        d = {"n_elem": rep.n_elem, "judged": rep.judged, "failed": rep.failed,
             "per_class": list(rep.per_class), "max_judged_err": rep.max_judged_err}
        if judge_state:
            d["judge_state"] = js[: self.n_elem]
        return d


def measure_peaks(ctx: Context, write_bytes=4 << 30, stream=None):
    """p2s_measure_peaks: FP64 and FP32 FMA rates (TFLOP/s) and the store-only HBM rate (GB/s)
    measured by the library's probe kernels on the context's device."""
    pk = Peaks()
    _check(load().p2s_measure_peaks(ctx.handle, int(write_bytes), ctypes.byref(pk), _stream(stream)),
           "p2s_measure_peaks")
    return {f: getattr(pk, f) for f, _ in Peaks._fields_}


def mode1_product(ctx: Context, method, G, x, n_rows, out, slices=4, stream=None):
    """p2s_mode1_product: T[r][k] = sum_a B[k][a] x[r mod n_src][a] for k < 7 on the G-point
    rule; x: float32 device tensor [n_src][G][2] (hi, lo), out: float32 [n_rows][8][2]."""
    n_src = int(x.shape[0])
    _check(load().p2s_mode1_product(ctx.handle, int(method), int(G), int(slices), _dptr(x), n_src, int(n_rows),
                                    _dptr(out), _stream(stream)), "p2s_mode1_product")
