"""CPU checks of the C ABI: the library loads, exports every declared symbol, and its
host-built tables agree with the oracle's independent ones.  No GPU compute."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1703_09619_gb300 import build as B
from paper_1703_09619_gb300 import p2s
from paper_1703_09619_gb300 import workloads as W
from tests import p2s_math as pm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    if not os.path.exists(p2s.LIB_PATH):
        B.build()
    return p2s.load()


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            with open(os.path.join(inc, f)) as fh:
                text = fh.read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(p2s_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 16
    lib = ctypes.CDLL(p2s.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    # and the binding declares a signature for each
    assert set(names) <= set(p2s.SIGNATURES), set(names) - set(p2s.SIGNATURES)


def test_gauss_legendre_table_matches_oracle_and_numpy():
    for G in range(1, p2s.MAX_NPTS + 1):
        x, w = p2s.gauss_legendre(G)
        xo, wo = oracle.gauss_legendre(G)
        assert np.max(np.abs(x - xo)) < 3e-15
        assert np.max(np.abs(w - wo)) < 3e-15 * max(1, wo.max())


@pytest.mark.parametrize("t", range(4))
def test_linearisation_table_matches_oracle_projection(t):
    """The library's Adams-Neumann tables (Eq. (3)) against the oracle's projection."""
    d1, d2 = t & 1, t >> 1
    for m1 in range(p2s.MAX_ORDER):
        for m2 in range(p2s.MAX_ORDER):
            K = m1 + m2 + 1
            C = p2s.linearisation(t, m1, m2, K)
            Co = oracle.linearisation(d1, d2, m1, m2, K)
            assert np.max(np.abs(C - Co)) < 2e-13 * max(1.0, np.abs(Co).max()), (t, m1, m2)


def test_linearisation_table_exact_rationals_small():
    for t, name in enumerate(("vv", "dv", "vd", "dd")):
        d1, d2 = t & 1, t >> 1
        for m1 in range(6):
            for m2 in range(6):
                C = p2s.linearisation(t, m1, m2, 12)
                ref = pm.product_dense(d1, d2, m1, m2, 13)
                assert np.max(np.abs(C - ref)) < 1e-14 * max(1, np.abs(ref).max())


@pytest.mark.parametrize("name", ["c1", "c3", "c4"])
def test_output_and_moment_entries(name):
    wl = W.make(name, 64)
    n, off = p2s.output_entries(wl.orders, 0xF, offsets=True)
    assert np.array_equal(off, oracle.output_offsets(wl.orders, 0xF))
    assert n == wl.entries()
    n2, off2 = p2s.output_entries(wl.orders, 0x6, offsets=True)
    assert np.array_equal(off2, oracle.output_offsets(wl.orders, 0x6))
    m, moff = p2s.moment_entries(wl.orders, offsets=True)
    nc = wl.n_comp
    pairs = [(0, 0)] if nc == 1 else [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    ref = [sum(int(np.prod(wl.orders[e, i] + wl.orders[e, j] - 1)) for i, j in pairs) for e in range(wl.n_elem)]
    assert np.array_equal(np.diff(moff), ref)


def test_argument_errors_on_host():
    bad = np.zeros((1, 1, 3), np.int32)
    with pytest.raises(p2s.P2SError) as ei:
        p2s.output_entries(bad)
    assert ei.value.code == p2s.ERR_ORDER
    with pytest.raises(p2s.P2SError) as ei:
        p2s.output_entries(np.full((1, 1, 3), 13, np.int32))
    assert ei.value.code == p2s.ERR_ORDER
    with pytest.raises(p2s.P2SError) as ei:
        p2s.output_entries(np.full((1, 1, 3), 2, np.int32), types_mask=0)
    assert ei.value.code == p2s.ERR_ARG
    with pytest.raises(p2s.P2SError):
        p2s.linearisation(4, 0, 0, 3)
    assert p2s.error_string(p2s.ERR_JACOBIAN).startswith("detJ")


def test_linearisation_tables_mirror_bit_for_bit():
    """P^(d1)_m1 P^(d2)_m2 = P^(d2)_m2 P^(d1)_m1: the table of (vv, m1, m2) equals that of
    (vv, m2, m1), dv that of vd mirrored, dd its mirror, bit for bit (the kernels that
    compute a block in its own orientation rely on it to match the transposed write-out)."""
    n = p2s.MAX_ORDER
    for a in range(n):
        for b in range(n):
            for t, tm in ((0, 0), (1, 2), (3, 3)):
                assert np.array_equal(p2s.linearisation(t, a, b, 2 * n), p2s.linearisation(tm, b, a, 2 * n)), (t, a, b)
