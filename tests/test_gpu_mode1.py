"""The first mode product of the moments (Eq. (4), the a-axis sum) in its two forms:
double-word SIMT and split-precision tensor-core products (tcgen05), against an FP64
reference built from numpy's Gauss-Legendre rule and Legendre series."""
import numpy as np
import pytest

from paper_1703_09619_gb300 import p2s

pytestmark = pytest.mark.gpu
GS = [8, 12, 16, 24, 32, 48]


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


def b_table(G):
    """B[k][a] = w_a P_k(u_a), k < 7, on the G-point rule (numpy's routines)."""
    u, w = np.polynomial.legendre.leggauss(G)
    return np.array([w * np.polynomial.legendre.legval(u, np.eye(7)[k]) for k in range(7)])


def sample_rows(G, n, seed):
    """Signed, oscillating rows whose magnitudes span six decades, as (hi, lo) FP32 pairs,
    with the exact FP64 value they represent; the last row is zero."""
    rng = np.random.default_rng(seed)
    u = np.linspace(-1.0, 1.0, G)
    amp = rng.normal(size=(n, 1)) * 10.0 ** rng.uniform(-3, 3, size=(n, 1))
    x = amp * (1 + 0.8 * np.sin(rng.uniform(1, 40, (n, 1)) * u + rng.uniform(0, 6, (n, 1))))
    x += amp * 1e-3 * rng.normal(size=(n, G))
    x[-1] = 0.0
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return np.stack([hi, lo], axis=-1), hi.astype(np.float64) + lo.astype(np.float64)


def run(torch, ctx, method, G, xs, n_rows, slices=4):
    xd = torch.as_tensor(np.ascontiguousarray(xs), device="cuda")
    out = torch.full((n_rows, 8, 2), float("nan"), dtype=torch.float32, device="cuda")
    p2s.mode1_product(ctx, method, G, xd, n_rows, out, slices=slices)
    assert ctx.sync_status() == 0
    o = out.cpu().numpy().astype(np.float64)
    return o[..., 0] + o[..., 1]


@pytest.mark.parametrize("G", GS)
def test_mode1_forms_against_fp64(torch, ctx, G):
    n_src, n_rows = 300, 1000  # rows wrap around the source; a ragged last tile of 128
    xs, x = sample_rows(G, n_src, G)
    B = b_table(G)
    ref = x @ B.T                                          # [n_src][7]
    norm = np.abs(x).max(axis=1, keepdims=True) * np.abs(B).sum(axis=1)[None, :]
    norm[norm == 0] = 1.0
    src = np.arange(n_rows) % n_src
    for method, slices, tol in ((p2s.MODE1_SIMT, 4, 1e-13), (p2s.MODE1_TC, 4, 4e-9), (p2s.MODE1_TC, 5, 2e-11)):
        T = run(torch, ctx, method, G, xs, n_rows, slices)
        assert not np.isnan(T).any()
        assert np.all(T[:, 7] == 0.0)
        err = np.abs(T[:, :7] - ref[src]) / norm[src]
        assert err.max() <= tol, (method, slices, G, err.max())
        assert np.all(T[src == n_src - 1, :7] == 0.0)  # the zero row


def test_mode1_argument_errors(torch, ctx):
    xs, _ = sample_rows(16, 4, 1)
    xd = torch.as_tensor(xs, device="cuda")
    out = torch.empty((4, 8, 2), dtype=torch.float32, device="cuda")
    for bad in (dict(method=p2s.MODE1_TC, G=20, slices=4), dict(method=p2s.MODE1_TC, G=16, slices=3),
                dict(method=7, G=16, slices=4)):
        with pytest.raises(p2s.P2SError):
            p2s.mode1_product(ctx, bad["method"], bad["G"], xd, 4, out, slices=bad["slices"])
