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
    # Three calls in a row with different shapes (uniform rules in both precisions, then a
    # per-element rule), so each call starts from the previous one's leftover scratch.
    per_elem = np.array([8, 12, 16, 24, 5, 16, 12, 8, 24, 16] * 3, dtype=np.int32)
    cases = [("c2", 40, 6, p2s.FP64), ("c4", 23, 5, p2s.MIXED), ("c5", 30, per_elem, p2s.MIXED)]
    inputs = []
    for name, n, G, prec in cases:  # every input and output buffer exists before the first call
        wl = W.make(name, n).with_npts(G)
        params, nodes, bulge = p2s.device_inputs(wl)
        total, off = p2s.output_entries(wl.orders, offsets=True)
        got = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
        status = torch.full((wl.n_elem,), 99, dtype=torch.int32, device="cuda")
        inputs.append((wl, G, prec, params, nodes, bulge, total, off, got, status))
    ctx = p2s.Context(0)  # p2s_create: allocates its tables and looks up the fixed scratch
    torch.cuda.synchronize()
    free = [torch.cuda.mem_get_info()[0]]
    for wl, G, prec, params, nodes, bulge, total, off, got, status in inputs:
        p2s.fill_elements_noalloc(ctx, wl.orders, G, wl.kind, params, nodes, bulge, got, status, precision=prec)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    # no call, the first one after p2s_create included, changed the device's free memory
    assert len(set(free)) == 1, free
    for wl, G, prec, params, nodes, bulge, total, off, got, status in inputs:
        assert ctx.sync_status() == 0
        ref = torch.empty(total, dtype=torch.float64, device="cuda")
        p2s.fill_elements(ctx, wl.orders, G, wl.kind, params, nodes, bulge, ref, precision=prec)
        g = got.cpu().numpy()
        assert not np.isnan(g).any()
        assert (status.cpu().numpy() == 0).all()
        err = rel_errors(g, ref.cpu().numpy(), off, wl.orders)
        assert err.max() <= TOL[prec], (wl.name, err.max())
    # requests beyond the fixed capacity are refused before anything is launched
    big = W.make("c4", 2049)
    params, nodes, bulge = p2s.device_inputs(big)
    dummy = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(p2s.P2SError) as ei:
        p2s.fill_elements_noalloc(ctx, big.orders, 4, big.kind, params, nodes, bulge, dummy)
    assert ei.value.code == p2s.ERR_BUFFER
    ctx.close()
