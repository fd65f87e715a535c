"""GPU parity of operator fills (term lists, Eq. (2) in full generality) against the oracle.

Bar as for the four-type fill: per element, max|M_gpu - M_oracle| <= tol * max|M_oracle| with
tol = 1e-12 (FP64) and 1e-8 (mixed, and 1e-10 against the FP64 path)."""
import numpy as np
import pytest

import oracle
from paper_1703_09619_gb300 import p2s
from paper_1703_09619_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {p2s.FP64: 1e-12, p2s.MIXED: 1e-8}


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch):
    c = p2s.Context(0)
    yield c
    c.close()


def gpu_op(torch, ctx, orders, kind, params, nodes, bulge, G, terms, scales, prec, tile=None, graph=False, reps=1):
    plan = p2s.OperatorPlan(ctx, orders, G, terms, scales, kind, prec, tile=tile, graph=graph)
    E = orders.shape[0]
    dp = torch.as_tensor(np.ascontiguousarray(params, dtype=np.float64).reshape(E, -1), device="cuda")
    dn = torch.as_tensor(np.ascontiguousarray(nodes, dtype=np.float64).reshape(E, 8, 3), device="cuda")
    db = torch.as_tensor(np.ascontiguousarray(bulge, dtype=np.float64).reshape(E, 4), device="cuda")
    out = torch.full((plan.output_entries,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(reps):
        plan.fill(kind, dp, dn, db, out)
    rc = ctx.sync_status()
    res = out.cpu().numpy()
    plan.close()
    return res, rc


def rel_err(a, b, off):
    errs = []
    for e in range(len(off) - 1):
        x, y = a[off[e]:off[e + 1]], b[off[e]:off[e + 1]]
        s = np.abs(y).max()
        errs.append(np.abs(x - y).max() / (s if s > 0 else 1.0))
    return max(errs) if errs else 0.0


def random_terms(rng, n_comp, na, count, symmetric=False):
    rows, sc = [], []
    for _ in range(count):
        gi, gj = (int(x) for x in rng.integers(0, n_comp, 2))
        sa, sb = (int(x) for x in rng.integers(0, na, 2))
        d = [int(x) for x in rng.integers(0, 2, 3)]
        f = [int(x) for x in rng.integers(0, 2, 3)]
        s = float(rng.normal())
        rows.append([gi, gj, sa, sb] + d + f)
        sc.append(s)
        if symmetric and not (gi == gj and sa == sb and d == f):
            rows.append([gj, gi, sb, sa] + f + d)
            sc.append(s)
    return np.array(rows, dtype=np.int32), np.array(sc)


@pytest.mark.parametrize("prec", [p2s.FP64, p2s.MIXED])
def test_diffusion_stiffness_matches_oracle(torch, ctx, prec):
    wl = W.make("c5", 6)
    orders = np.full((6, 1, 3), 4, dtype=np.int32)
    orders[1, 0] = [2, 3, 5]
    orders[4, 0] = [5, 4, 3]
    T, S = W.diffusion_terms()
    got, rc = gpu_op(torch, ctx, orders, wl.kind, wl.params, wl.nodes, wl.bulge, 7, T, S, prec)
    ref, off, _ = oracle.fill_terms(orders, wl.kind, wl.params, wl.nodes, wl.bulge, 7, T, S)
    assert rc == 0 and not np.isnan(got).any()
    assert rel_err(got, ref, off) <= TOL[prec]
    for e in range(6):  # symmetric list: both triangles written from one computation
        n = int(round(np.sqrt(off[e + 1] - off[e])))
        K = got[off[e]:off[e + 1]].reshape(n, n)
        assert np.array_equal(K, K.T) or prec == p2s.MIXED or np.abs(K - K.T).max() <= 1e-13 * np.abs(K).max()


@pytest.mark.parametrize("symmetric", [False, True])
@pytest.mark.parametrize("prec", [p2s.FP64, p2s.MIXED])
def test_random_terms_metric_three_components(torch, ctx, prec, symmetric):
    rng = np.random.default_rng(21 + symmetric)
    wl = W.make("c4", 4)
    orders = np.minimum(wl.orders, 4)
    T, S = random_terms(rng, 3, 3, 10, symmetric)
    got, rc = gpu_op(torch, ctx, orders, wl.kind, wl.params, wl.nodes, wl.bulge, 5, T, S, prec)
    ref, off, _ = oracle.fill_terms(orders, wl.kind, wl.params, wl.nodes, wl.bulge, 5, T, S)
    assert rc == 0 and not np.isnan(got).any()
    assert rel_err(got, ref, off) <= TOL[prec]


@pytest.mark.parametrize("prec", [p2s.FP64, p2s.MIXED])
def test_random_terms_scalar_kind_two_components(torch, ctx, prec):
    rng = np.random.default_rng(31)
    wl = W.make("c3", 3)
    orders = np.array([[[3, 4, 2], [2, 3, 4]]] * 3, dtype=np.int32)
    T, S = random_terms(rng, 2, 1, 8)
    nodes = np.zeros((3, 8, 3))
    bulge = np.zeros((3, 4))
    got, rc = gpu_op(torch, ctx, orders, wl.kind, wl.params, nodes, bulge, 6, T, S, prec)
    ref, off, _ = oracle.fill_terms(orders, wl.kind, wl.params, None, None, 6, T, S)
    assert rc == 0
    assert rel_err(got, ref, off) <= TOL[prec]


def test_mixed_operator_close_to_fp64(torch, ctx):
    wl = W.make("c5", 8)
    orders = np.full((8, 1, 3), 4, dtype=np.int32)
    T, S = W.diffusion_terms()
    a, _ = gpu_op(torch, ctx, orders, wl.kind, wl.params, wl.nodes, wl.bulge, 16, T, S, p2s.FP64)
    b, _ = gpu_op(torch, ctx, orders, wl.kind, wl.params, wl.nodes, wl.bulge, 16, T, S, p2s.MIXED)
    off = np.concatenate([[0], np.cumsum(np.full(8, 64 * 64))])
    assert rel_err(b, a, off) <= 1e-10


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
def test_uniform_scalar_field_specialised_path(torch, ctx, N):
    """One component of uniform order N <= 6, mixed: the specialised operator kernel (compile-time
    runs, terms summed in registers), for random per-axis types and coupling entries, against the
    oracle and against the FP64 general path."""
    rng = np.random.default_rng(50 + N)
    wl = W.make("c5", 3)
    orders = np.full((3, 1, 3), N, dtype=np.int32)
    T, S = random_terms(rng, 1, 3, 12)
    G = N + 3
    got, rc = gpu_op(torch, ctx, orders, wl.kind, wl.params, wl.nodes, wl.bulge, G, T, S, p2s.MIXED)
    ref, off, _ = oracle.fill_terms(orders, wl.kind, wl.params, wl.nodes, wl.bulge, G, T, S)
    assert rc == 0 and not np.isnan(got).any()
    assert rel_err(got, ref, off) <= TOL[p2s.MIXED]
    f64, _ = gpu_op(torch, ctx, orders, wl.kind, wl.params, wl.nodes, wl.bulge, G, T, S, p2s.FP64)
    assert rel_err(got, f64, off) <= 1e-10


def test_blocks_without_terms_are_zero(torch, ctx):
    wl = W.make("c4", 2)
    orders = np.minimum(wl.orders, 3)
    T = np.array([[1, 2, 0, 1, 1, 0, 0, 0, 1, 0]], dtype=np.int32)
    got, rc = gpu_op(torch, ctx, orders, wl.kind, wl.params, wl.nodes, wl.bulge, 4, T, [2.5], p2s.FP64)
    ref, off, _ = oracle.fill_terms(orders, wl.kind, wl.params, wl.nodes, wl.bulge, 4, T, [2.5])
    assert rc == 0 and not np.isnan(got).any()
    assert rel_err(got, ref, off) <= 1e-12
    assert np.count_nonzero(got) <= np.count_nonzero(ref)


def test_tile_configs_and_graph_replay_bitwise(torch, ctx):
    rng = np.random.default_rng(41)
    wl = W.make("c4", 3)
    orders = np.minimum(wl.orders, 5)
    T, S = random_terms(rng, 3, 3, 6, symmetric=True)
    base, _ = gpu_op(torch, ctx, orders, wl.kind, wl.params, wl.nodes, wl.bulge, 5, T, S, p2s.MIXED)
    for tile in ({"combo_target": 64, "unit_kbytes": 24, "threads": 128},
                 {"combo_target": 512, "unit_kbytes": 100, "threads": 256}):
        got, _ = gpu_op(torch, ctx, orders, wl.kind, wl.params, wl.nodes, wl.bulge, 5, T, S, p2s.MIXED, tile=tile)
        assert np.array_equal(got, base), tile
    got, _ = gpu_op(torch, ctx, orders, wl.kind, wl.params, wl.nodes, wl.bulge, 5, T, S, p2s.MIXED, graph=True, reps=3)
    assert np.array_equal(got, base)


def test_highest_order_operator_plan(torch, ctx):
    """N = 12 (the largest order) on one axis: the plan builds and the fill matches."""
    wl = W.make("c5", 1)
    orders = np.array([[[12, 2, 2]]], dtype=np.int32)
    T, S = W.diffusion_terms()
    got, rc = gpu_op(torch, ctx, orders, wl.kind, wl.params, wl.nodes, wl.bulge, 13, T, S, p2s.FP64)
    ref, off, _ = oracle.fill_terms(orders, wl.kind, wl.params, wl.nodes, wl.bulge, 13, T, S)
    assert rc == 0
    assert rel_err(got, ref, off) <= 1e-12


def test_operator_argument_errors(torch, ctx):
    orders = np.full((2, 1, 3), 3, dtype=np.int32)
    good = np.array([[0, 0, 0, 0, 1, 0, 0, 1, 0, 0]], dtype=np.int32)
    for bad in ([[1, 0, 0, 0, 1, 0, 0, 1, 0, 0]],   # component out of range
                [[0, 0, 3, 0, 1, 0, 0, 1, 0, 0]],   # coupling entry out of range
                [[0, 0, 0, 0, 2, 0, 0, 1, 0, 0]]):  # derivative order 2
        with pytest.raises(p2s.P2SError) as ex:
            p2s.OperatorPlan(ctx, orders, 4, np.array(bad, dtype=np.int32), [1.0], p2s.ALPHA_METRIC_EPS)
        assert ex.value.code == p2s.ERR_ARG
    with pytest.raises(p2s.P2SError):
        p2s.OperatorPlan(ctx, orders, 4, good, [1.0], p2s.ALPHA_SCALAR + 7)
    p2s.OperatorPlan(ctx, orders, 4, good, [1.0], p2s.ALPHA_METRIC_EPS).close()
