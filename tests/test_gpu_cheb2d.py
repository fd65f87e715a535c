"""GPU parity of the 2-D curl-curl example (Sec. III): the product-to-sum fill and the direct
fill against the oracle (oracle/cheb2d.py) and against each other.

Bar: per element and matrix, max |X_gpu - X_oracle| <= 1e-12 max |X_oracle| (both methods use the
same Gauss-Legendre rule, so they agree with the direct sums to rounding)."""
import numpy as np
import pytest

from oracle import cheb2d as C
from paper_1703_09619_gb300 import p2s
from paper_1703_09619_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


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


def gpu_fill(torch, ctx, params, M, N, G, method, precision=p2s.FP64):
    n = p2s.cheb2d_dofs(M, N)
    E = params.shape[0]
    dp = torch.as_tensor(np.ascontiguousarray(params), device="cuda")
    S = torch.full((E, n, n), float("nan"), dtype=torch.float64, device="cuda")
    Mm = torch.full((E, n, n), float("nan"), dtype=torch.float64, device="cuda")
    p2s.cheb2d_fill(ctx, dp, M, N, G, S, Mm, method, precision)
    rc = ctx.sync_status()
    return S.cpu().numpy(), Mm.cpu().numpy(), rc


def rel(a, b):
    return max(np.abs(x - y).max() / max(np.abs(y).max(), 1e-300) for x, y in zip(a, b))


@pytest.mark.parametrize("method", [p2s.CHEB2D_P2S, p2s.CHEB2D_DIRECT])
@pytest.mark.parametrize("M,N,G", [(3, 3, 7), (4, 3, 8), (2, 5, 9), (1, 1, 3), (8, 8, 14)])
def test_matches_oracle(torch, ctx, method, M, N, G):
    mesh = W.make_mesh2d(3, 2, M, G)
    S, Mm, rc = gpu_fill(torch, ctx, mesh.params, M, N, G, method)
    assert rc == 0 and not np.isnan(S).any() and not np.isnan(Mm).any()
    ref = [C.element_matrices(p, M, N, G) for p in mesh.params]
    assert rel(S, [r[0] for r in ref]) <= TOL
    assert rel(Mm, [r[1] for r in ref]) <= TOL


@pytest.mark.parametrize("M,N,G", [(3, 3, 7), (5, 2, 9), (8, 8, 14)])
def test_mixed_p2s_matches_oracle(torch, ctx, M, N, G):
    """Mixed product-to-sum: entries formed in double-word FP32 from FP64 v-axis sums."""
    mesh = W.make_mesh2d(3, 2, M, G)
    S, Mm, rc = gpu_fill(torch, ctx, mesh.params, M, N, G, p2s.CHEB2D_P2S, p2s.MIXED)
    assert rc == 0 and not np.isnan(S).any()
    ref = [C.element_matrices(p, M, N, G) for p in mesh.params]
    assert rel(S, [r[0] for r in ref]) <= 1e-11
    assert rel(Mm, [r[1] for r in ref]) <= 1e-11


def test_mixed_high_order_close_to_fp64(torch, ctx):
    M = N = 18
    G = W.cheb2d_npts(M)
    mesh = W.make_mesh2d(4, 2, M, G)
    S1, M1, _ = gpu_fill(torch, ctx, mesh.params, M, N, G, p2s.CHEB2D_P2S, p2s.FP64)
    S2, M2, rc = gpu_fill(torch, ctx, mesh.params, M, N, G, p2s.CHEB2D_P2S, p2s.MIXED)
    assert rc == 0
    assert rel(S2, S1) <= 1e-11 and rel(M2, M1) <= 1e-11


def test_high_order_p2s_equals_direct_and_properties(torch, ctx):
    """Order 18 (Table I's largest) on a 4 x 4 mesh: the two methods agree, S annihilates gradients,
    both matrices are symmetric."""
    M = N = 18
    G = W.cheb2d_npts(M)
    mesh = W.make_mesh2d(4, 4, M, G)
    S1, M1, rc1 = gpu_fill(torch, ctx, mesh.params, M, N, G, p2s.CHEB2D_P2S)
    S2, M2, rc2 = gpu_fill(torch, ctx, mesh.params, M, N, G, p2s.CHEB2D_DIRECT)
    assert rc1 == 0 and rc2 == 0
    assert rel(S1, S2) <= 1e-11 and rel(M1, M2) <= 1e-11
    for e in (0, 7, 15):
        S, Mm = S1[e], M1[e]
        assert np.abs(S - S.T).max() <= 1e-12 * np.abs(S).max()
        assert np.abs(Mm - Mm.T).max() <= 1e-12 * np.abs(Mm).max()
        for a, b in ((0, 1), (3, 5), (18, 18), (17, 2)):
            c = np.zeros(S.shape[0])
            if a >= 1:
                c[(a - 1) * (N + 1) + b] = a
            if b >= 1:
                c[M * (N + 1) + a * N + (b - 1)] = b
            assert np.abs(S @ c).max() <= 1e-10 * np.abs(S).max() * np.abs(c).max()


def test_sampled_elements_of_the_benchmark_mesh(torch, ctx):
    """The 32 x 32 mesh at M = N = 6: sampled elements against the oracle."""
    M = N = 6
    G = W.cheb2d_npts(M)
    mesh = W.make_mesh2d(32, 32, M, G)
    S, Mm, rc = gpu_fill(torch, ctx, mesh.params, M, N, G, p2s.CHEB2D_P2S)
    assert rc == 0
    for e in (0, 31, 500, 1023, 527):
        Sr, Mr = C.element_matrices(mesh.params[e], M, N, G)
        assert np.abs(S[e] - Sr).max() <= TOL * np.abs(Sr).max()
        assert np.abs(Mm[e] - Mr).max() <= TOL * np.abs(Mr).max()


def test_empty_batch_and_errors(torch, ctx):
    import torch as T
    S = T.zeros((0, 4, 4), dtype=T.float64, device="cuda")
    p2s.cheb2d_fill(ctx, T.zeros((0, 5), dtype=T.float64, device="cuda"), 1, 1, 3, S, S)
    dp = T.zeros((1, 5), dtype=T.float64, device="cuda")
    S = T.zeros((1, 4, 4), dtype=T.float64, device="cuda")
    for M, N, G, code in ((0, 3, 5, p2s.ERR_ORDER), (25, 3, 5, p2s.ERR_ORDER), (3, 3, 49, p2s.ERR_ORDER)):
        with pytest.raises(p2s.P2SError) as ex:
            p2s.cheb2d_fill(ctx, dp, M, N, G, S, S)
        assert ex.value.code == code
    with pytest.raises(p2s.P2SError) as ex:
        p2s.cheb2d_fill(ctx, dp, 3, 3, 5, S, S, method=7)
    assert ex.value.code == p2s.ERR_ARG
    with pytest.raises(p2s.P2SError) as ex:  # mixed precision is a product-to-sum option only
        p2s.cheb2d_fill(ctx, dp, 3, 3, 5, S, S, method=p2s.CHEB2D_DIRECT, precision=p2s.MIXED)
    assert ex.value.code == p2s.ERR_ARG
