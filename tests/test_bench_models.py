"""CPU checks of the work models behind bench.py's roofline fractions.

The bench divides algorithmic work by kernel time; these tests pin that work to counts made
independently of the library:
  * the nonzero linearisation coefficients of Eq. (3) are recomputed with numpy's Legendre
    series (products, derivatives, projection), and the sparse three-stage contraction of
    Eq. (4) is counted by walking its loops;
  * the sum-factorised moment MACs (Eq. (4)) are counted by walking the three mode products."""
import itertools

import numpy as np
import numpy.polynomial.legendre as npl
import pytest

import bench
from paper_1703_09619_gb300 import workloads as W


def nnz_runs(d1, d2, a, b):
    """Nonzero Legendre coefficients of P_a^(d1) P_b^(d2), from numpy's series arithmetic."""
    ca = np.zeros(a + 1)
    ca[a] = 1.0
    cb = np.zeros(b + 1)
    cb[b] = 1.0
    if d1:
        ca = npl.legder(ca) if a > 0 else np.zeros(1)
    if d2:
        cb = npl.legder(cb) if b > 0 else np.zeros(1)
    prod = npl.legmul(ca, cb)
    return int(np.count_nonzero(np.abs(prod) > 1e-12))


def walk_operator(orders_e, terms):
    """MACs of the three sparse stages for one element, by walking them (blocks gi <= gj)."""
    macs = 0
    for tm in terms:
        gi, gj = int(tm[0]), int(tm[1])
        if gi > gj:
            continue
        du, dv, dw = (int(tm[4 + x]) for x in range(3))
        eu, ev, ew = (int(tm[7 + x]) for x in range(3))
        Ni, Nj = orders_e[gi], orders_e[gj]
        Kv, Kw = Ni[1] + Nj[1] - 1, Ni[2] + Nj[2] - 1
        for m1, m2 in itertools.product(range(Ni[0]), range(Nj[0])):   # stage 1: contract k
            macs += nnz_runs(du, eu, m1, m2) * Kv * Kw
        for m1, m2 in itertools.product(range(Ni[0]), range(Nj[0])):   # stage 2: contract l
            for n1, n2 in itertools.product(range(Ni[1]), range(Nj[1])):
                macs += nnz_runs(dv, ev, n1, n2) * Kw
        for m1, n1, m2, n2 in itertools.product(range(Ni[0]), range(Ni[1]), range(Nj[0]), range(Nj[1])):
            for p1, p2 in itertools.product(range(Ni[2]), range(Nj[2])):  # stage 3: contract q
                macs += nnz_runs(dw, ew, p1, p2)
    return macs


@pytest.mark.parametrize("N", [2, 3, 4])
def test_operator_fma_count_matches_walk(N):
    T, _ = W.diffusion_terms()
    orders = np.full((3, 1, 3), N, dtype=np.int32)
    assert bench.operator_fma_count(orders, T, symmetric=True) == 3 * walk_operator(orders[0], T)


def test_operator_fma_count_uneven_two_components():
    rng = np.random.default_rng(3)
    terms = [[int(rng.integers(0, 2)), int(rng.integers(0, 2)), 0, 0] + [int(x) for x in rng.integers(0, 2, 6)]
             for _ in range(6)]
    orders = np.array([[[2, 3, 4], [3, 2, 2]], [[4, 2, 3], [2, 2, 2]]], dtype=np.int32)
    want = sum(walk_operator(o, terms) for o in orders)
    assert bench.operator_fma_count(orders, terms, symmetric=True) == want


def walk_moments(K, G, npairs, folded):
    """MACs of the three mode products of Eq. (4) for one element (the first one folded over
    ceil(G/2) points when the rule is symmetric)."""
    ga = (G + 1) // 2 if folded else G
    macs = 0
    for _ in range(npairs):
        macs += sum(ga for _k in range(K[0]) for _b in range(G) for _c in range(G))      # T1[k][b][c]
        macs += sum(G for _k in range(K[0]) for _l in range(K[1]) for _c in range(G))     # T2[k][l][c]
        macs += sum(G for _k in range(K[0]) for _l in range(K[1]) for _q in range(K[2]))  # I[k][l][q]
    return macs


@pytest.mark.parametrize("folded", [False, True])
def test_moment_mac_count_matches_walk(folded):
    orders = np.array([[[4, 4, 4], [4, 4, 4], [4, 4, 4]], [[3, 5, 2], [2, 2, 2], [4, 3, 3]]], dtype=np.int32)
    npts = np.array([8, 5])
    macs, pts, npairs = bench.moment_mac_points(orders, npts, folded=folded)
    want = 0
    for e in range(2):
        K = [int(2 * orders[e, :, x].max() - 1) for x in range(3)]
        want += walk_moments(K, int(npts[e]), 6, folded)
    assert macs == want and pts == 8 ** 3 + 5 ** 3 and npairs == 6


def test_library_run_counts_match_numpy():
    """The library's Eq. (3) run lengths, which the models read, equal numpy's nonzero counts."""
    cnt = bench._runs()
    for t in range(4):
        d1, d2 = t & 1, (t >> 1) & 1
        for a in range(8):
            for b in range(8):
                assert cnt[t, a, b] == nnz_runs(d1, d2, a, b), (t, a, b)


def test_bench_names_the_kernel_the_library_picks():
    """The bench labels its roofline with the contraction kernel the plan runs: mixed, the
    per-order kernel for uniform orders 2..8 and the bounded-order kernel for uneven orders
    <= 8; FP64, the bounded-order kernel for orders <= 8; the general kernel above 8 or when
    the tile names it."""
    k = bench.contract_kernel
    assert k(np.full((3, 3, 3), 4)) == "k_contract_ffn<4>"
    assert k(np.full((3, 1, 3), 8)) == "k_contract_ffn<8>"
    assert k(np.full((3, 1, 3), 8), kernel=2) == "k_contract_ffb<ArithFF>"
    assert k(np.full((3, 3, 3), 4), kernel=1) == "k_contract<ArithFF>"
    assert k(np.full((3, 3, 3), 6), mixed=False) == "k_contract_ffb<ArithF64>"
    assert k(np.full((3, 3, 3), 6), mixed=False, kernel=1) == "k_contract<ArithF64>"
    uneven = np.array([[[2, 3, 8], [8, 8, 8], [1, 2, 3]]])
    assert k(uneven) == "k_contract_ffb<ArithFF>"
    assert k(np.full((2, 1, 3), 1)) == "k_contract_ffb<ArithFF>"
    uneven[0, 1, 2] = 9
    assert k(uneven) == "k_contract<ArithFF>"
    assert k(uneven, mixed=False) == "k_contract<ArithF64>"
