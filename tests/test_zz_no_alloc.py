"""The allocation-free fill (p2s_fill_elements_noalloc) against the ordinary one.

Callers that may not allocate device memory while they run (a solver whose memory
pool already holds the free device memory, a service under a fixed budget) use this
entry point; it keeps its scratch in a fixed array inside the library.  This file
runs last so that a failure here leaves every other test already run; it passes alone
in a fresh process as well as after the others."""
import numpy as np
import pytest

import oracle
from paper_1703_09619_gb300 import p2s
from paper_1703_09619_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {p2s.FP64: 1e-12, p2s.MIXED: 1e-8}


def rel_errors(a, b, off, orders):
    errs = []
    for e in range(orders.shape[0]):
        ma = oracle.element_matrices(a, off, orders, e)
        mb = oracle.element_matrices(b, off, orders, e)
        for t in mb:
            s = np.abs(mb[t]).max()
            errs.append(np.abs(ma[t] - mb[t]).max() / s if s > 0 else np.abs(ma[t]).max())
    return np.array(errs)


def test_noalloc_fill_matches_fill_elements_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = p2s.Context(0)
    # two calls in a row with different shapes, so the second one starts from the first
    # one's leftover scratch contents
    cases = [("c2", 40, 6, p2s.FP64), ("c4", 23, 5, p2s.MIXED)]
    for name, n, G, prec in cases:
        wl = W.make(name, n).with_npts(G)
        params, nodes, bulge = p2s.device_inputs(wl)
        total, off = p2s.output_entries(wl.orders, offsets=True)
        ref = torch.empty(total, dtype=torch.float64, device="cuda")
        p2s.fill_elements(ctx, wl.orders, G, wl.kind, params, nodes, bulge, ref, precision=prec)
        got = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
        status = torch.full((wl.n_elem,), 99, dtype=torch.int32, device="cuda")
        p2s.fill_elements_noalloc(ctx, wl.orders, G, wl.kind, params, nodes, bulge, got, status, precision=prec)
        assert ctx.sync_status() == 0
        g = got.cpu().numpy()
        assert not np.isnan(g).any()
        assert (status.cpu().numpy() == 0).all()
        err = rel_errors(g, ref.cpu().numpy(), off, wl.orders)
        assert err.max() <= TOL[prec], (name, err.max())
    # requests beyond the fixed capacity are refused before anything is launched
    big = W.make("c4", 2049)
    params, nodes, bulge = p2s.device_inputs(big)
    dummy = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(p2s.P2SError) as ei:
        p2s.fill_elements_noalloc(ctx, big.orders, 4, big.kind, params, nodes, bulge, dummy)
    assert ei.value.code == p2s.ERR_BUFFER
    ctx.close()
