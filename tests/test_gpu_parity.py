"""GPU parity of the fill against the CPU oracle (element by element).

Bar (Eq. (2) vs Eq. (4) with the same quadrature rule): per element and product type,
max|M_gpu - M_oracle| <= tol * max|M_oracle|, tol = 1e-12 for the FP64 path and 1e-8
for the mixed-precision path.  The two paths share only the seeded input generators."""
import numpy as np
import pytest

import oracle
from paper_1703_09619_gb300 import p2s
from paper_1703_09619_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL_FP64 = 1e-12
TOL_MIXED = 1e-8
TOL = {p2s.FP64: TOL_FP64, p2s.MIXED: TOL_MIXED}
PRECS = [p2s.FP64, p2s.MIXED]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    c = p2s.Context(0)
    yield c
    c.close()


def gpu_fill(torch, ctx, wl, precision=p2s.FP64, types_mask=0xF, split=False):
    params, nodes, bulge = p2s.device_inputs(wl)
    npts = wl.npts if len(set(wl.npts.tolist())) > 1 else int(wl.npts[0])
    plan = p2s.Plan(ctx, wl.orders, npts, precision, types_mask)
    out = torch.full((max(plan.output_entries, 1),), float("nan"), dtype=torch.float64, device="cuda")
    status = torch.full((max(wl.n_elem, 1),), 99, dtype=torch.int32, device="cuda")
    if split:
        mom = torch.empty(max(plan.moment_entries, 1), dtype=torch.float64, device="cuda")
        plan.moments(wl.kind, params, nodes, bulge, mom, status)
        plan.contract(mom, out)
    else:
        plan.fill(wl.kind, params, nodes, bulge, out, status)
    rc = ctx.sync_status()
    res = out.cpu().numpy()[: plan.output_entries], status.cpu().numpy()[: wl.n_elem], rc
    plan.close()
    return res


def oracle_fill(wl, types_mask=0xF):
    out, off, rc = oracle.fill(wl.orders, wl.kind, wl.params, wl.nodes, wl.bulge, wl.npts, types_mask)
    return out, off


def per_type_errors(gpu, ref, off, orders, types_mask=0xF):
    errs = []
    for e in range(orders.shape[0]):
        mg = oracle.element_matrices(gpu, off, orders, e, types_mask)
        mr = oracle.element_matrices(ref, off, orders, e, types_mask)
        for t in mr:
            scale = np.abs(mr[t]).max()
            d = np.abs(mg[t] - mr[t]).max()
            errs.append(d / scale if scale > 0 else d)
    return np.array(errs)


def check(torch, ctx, wl, types_mask=0xF, precision=p2s.FP64, split=False):
    tol = TOL[precision]
    g, status, rc = gpu_fill(torch, ctx, wl, precision=precision, types_mask=types_mask, split=split)
    r, off = oracle_fill(wl, types_mask)
    assert g.shape == r.shape
    assert not np.isnan(g).any()
    err = per_type_errors(g, r, off, wl.orders, types_mask)
    assert err.max() <= tol, (wl.name, precision, err.max())
    assert (status == 0).all() and rc == 0
    return err


@pytest.mark.parametrize("prec", PRECS)
def test_c1_whole(torch_cuda, ctx, prec):
    err = check(torch_cuda, ctx, W.make("c1"), precision=prec)
    assert err.size == 4


@pytest.mark.parametrize("prec", PRECS)
def test_c2_shape_small_orders_many_elements(torch_cuda, ctx, prec):
    """3 components, curved elements, several CTAs/warps and a ragged last wave."""
    wl = W.make("c2", 37)
    wl.orders[:] = 3
    wl = wl.with_npts(5)
    check(torch_cuda, ctx, wl, precision=prec)


@pytest.mark.parametrize("prec", PRECS)
def test_c2_full_order_two_elements(torch_cuda, ctx, prec):
    check(torch_cuda, ctx, W.make("c2", 2), precision=prec)


@pytest.mark.parametrize("prec", PRECS)
def test_c4_uneven_orders(torch_cuda, ctx, prec):
    check(torch_cuda, ctx, W.make("c4", 6), precision=prec)


@pytest.mark.parametrize("prec", PRECS)
def test_c3_order8(torch_cuda, ctx, prec):
    wl = W.make("c3", 2).with_npts(12)
    check(torch_cuda, ctx, wl, precision=prec)


@pytest.mark.parametrize("prec", PRECS)
def test_moments_then_contract_equals_fill(torch_cuda, ctx, prec):
    wl = W.make("c4", 5)
    a, _, _ = gpu_fill(torch_cuda, ctx, wl, precision=prec)
    b, _, _ = gpu_fill(torch_cuda, ctx, wl, precision=prec, split=True)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", PRECS)
def test_repeatable_bitwise(torch_cuda, ctx, prec):
    wl = W.make("c2", 3)
    a, _, _ = gpu_fill(torch_cuda, ctx, wl, precision=prec)
    b, _, _ = gpu_fill(torch_cuda, ctx, wl, precision=prec)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mask", [0x1, 0x2, 0x4, 0x8, 0x6, 0x9, 0x3, 0xC, 0xB])
def test_type_subsets(torch_cuda, ctx, mask, prec):
    """Every subset keeps the transpose partners consistent (dv alone, vd alone, both)."""
    wl = W.make("c4", 3)
    wl = wl.with_npts(6)
    check(torch_cuda, ctx, wl, types_mask=mask, precision=prec)


@pytest.mark.parametrize("prec", PRECS)
def test_degenerate_orders_and_points(torch_cuda, ctx, prec):
    """N = 1 on some axes, anisotropic orders, G = 1 and G = 2 quadrature."""
    wl = W.make("c4", 4)
    wl.orders[0] = [[1, 1, 1], [1, 2, 3], [3, 1, 2]]
    wl.orders[1] = [[2, 1, 1], [1, 1, 1], [1, 1, 4]]
    wl.orders[2] = [[1, 1, 1], [1, 1, 1], [1, 1, 1]]
    wl.orders[3] = [[8, 1, 2], [2, 8, 1], [1, 2, 8]]
    for G in (1, 2, 7):
        check(torch_cuda, ctx, wl.with_npts(G), precision=prec)


@pytest.mark.parametrize("prec", PRECS)
def test_per_element_quadrature(torch_cuda, ctx, prec):
    wl = W.make("c5", 6)
    wl = wl.with_npts(np.array([4, 9, 16, 3, 24, 7]))
    check(torch_cuda, ctx, wl, precision=prec)


@pytest.mark.parametrize("prec", PRECS)
def test_large_G_scalar(torch_cuda, ctx, prec):
    wl = W.make("c3", 1)
    wl.orders[:] = 3
    check(torch_cuda, ctx, wl.with_npts(64), precision=prec)


@pytest.mark.parametrize("name,G", [("c5", 8), ("c5", 12), ("c5", 16), ("c5", 24), ("c5", 32), ("c5", 48),
                                    ("c2", 24), ("c3", 12)])
def test_mixed_close_to_fp64(torch_cuda, ctx, name, G):
    """The double-word coupling factor, moments and contraction stay within 1e-10 of the
    FP64 path (the learned fill's judge compares at 1e-9); c5 includes |k| up to 40, so the
    double-word sine sees phases up to about 70 rad."""
    wl = W.make(name, 48).with_npts(G)
    a, _, _ = gpu_fill(torch_cuda, ctx, wl, precision=p2s.FP64)
    b, _, _ = gpu_fill(torch_cuda, ctx, wl, precision=p2s.MIXED)
    off = oracle.output_offsets(wl.orders)
    err = per_type_errors(b, a, off, wl.orders)
    assert err.max() <= 1e-10, err.max()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("G", [32, 48])
def test_c5_specialised_moment_bodies_against_oracle(torch_cuda, ctx, prec, G):
    """Three-component N = 4 elements at G = 32 and 48 run the moment kernels' compile-time
    bodies for those rules (the learned fill's G = 32 class and its judge / fallback rule);
    two c5 elements each, entry by entry against the oracle's direct triple sums."""
    wl = W.make("c5", 2).with_npts(G)
    check(torch_cuda, ctx, wl, precision=prec)


def test_plan_beyond_device_memory_is_oom(torch_cuda, ctx):
    """A plan whose moment scratch exceeds the device's memory is refused at creation with
    P2S_ERR_OOM (nothing is launched), and the context fills correctly afterwards."""
    _, total = torch_cuda.cuda.mem_get_info()
    per_elem = 6 * 15 ** 3 * 8  # three components at N = 8: six pairs of 15^3 FP64 moments
    E = int(1.05 * total) // per_elem + 1
    orders = np.full((E, 3, 3), 8, dtype=np.int32)
    # bounded-order kernel, two m1 rows per unit (the largest unit that fits shared memory at N = 8)
    tile = {"combo_target": 1024, "unit_kbytes": 0, "threads": 512, "kernel": 2}
    with pytest.raises(p2s.P2SError) as ei:
        p2s.Plan(ctx, orders, 2, p2s.FP64, types_mask=0x1, tile=tile)
    assert ei.value.code == p2s.ERR_OOM
    check(torch_cuda, ctx, W.make("c1"))


def test_empty_batch(torch_cuda, ctx):
    wl = W.make("c4", 1).subset([])
    plan = p2s.Plan(ctx, wl.orders, 4)
    assert plan.output_entries == 0
    out = torch_cuda.empty(1, dtype=torch_cuda.float64, device="cuda")
    params, nodes, bulge = p2s.device_inputs(W.make("c4", 1))
    plan.fill(wl.kind, params[:0], nodes[:0], bulge[:0], out)
    assert ctx.sync_status() == 0


def test_inverted_element_is_flagged(torch_cuda, ctx):
    """detJ <= 0 (mirrored element) sets the element's status and the context flag."""
    wl = W.make("c2", 3)
    wl.orders[:] = 2
    wl = wl.with_npts(3)
    wl.nodes[1, :, 0] = -wl.nodes[1, :, 0]
    g, status, rc = gpu_fill(torch_cuda, ctx, wl)
    assert status.tolist() == [0, p2s.ERR_JACOBIAN, 0]
    assert rc == p2s.ERR_JACOBIAN
    assert ctx.sync_status() == 0  # flag cleared by the read


def test_argument_errors(torch_cuda, ctx):
    wl = W.make("c2", 2)
    params, nodes, bulge = p2s.device_inputs(wl)
    plan = p2s.Plan(ctx, wl.orders, 4)
    out = torch_cuda.empty(plan.output_entries, dtype=torch_cuda.float64, device="cuda")
    with pytest.raises(p2s.P2SError) as ei:
        plan.fill(p2s.ALPHA_SCALAR, params, nodes, bulge, out)  # scalar kind with 3 components
    assert ei.value.code == p2s.ERR_ARG
    with pytest.raises(p2s.P2SError) as ei:
        plan.fill(wl.kind, params, None, bulge, out)  # metric kind needs nodes
    assert ei.value.code == p2s.ERR_ARG
    with pytest.raises(p2s.P2SError) as ei:
        p2s.Plan(ctx, wl.orders, 65)
    assert ei.value.code == p2s.ERR_ORDER
    with pytest.raises(p2s.P2SError) as ei:
        p2s.Plan(ctx, wl.orders, 4, precision=7)
    assert ei.value.code == p2s.ERR_ARG


def test_one_shot_entry_point(torch_cuda, ctx):
    wl = W.make("c1")
    params, nodes, bulge = p2s.device_inputs(wl)
    n = p2s.output_entries(wl.orders)
    out = torch_cuda.empty(n, dtype=torch_cuda.float64, device="cuda")
    p2s.fill_elements(ctx, wl.orders, 12, wl.kind, params, nodes, bulge, out)
    r, off = oracle_fill(wl)
    err = per_type_errors(out.cpu().numpy(), r, off, wl.orders)
    assert err.max() <= TOL_FP64


def test_full_size_c5_mixed_sampled(torch_cuda, ctx):
    """The full 32768-element three-component N=4 workload through the mixed path at a
    fixed 12-point rule; three seeded elements checked entry by entry (<= 1e-8)."""
    torch = torch_cuda
    wl = W.make("c5").with_npts(12)
    params, nodes, bulge = p2s.device_inputs(wl)
    plan = p2s.Plan(ctx, wl.orders, 12, p2s.MIXED)
    out = torch.empty(plan.output_entries, dtype=torch.float64, device="cuda")
    plan.fill(wl.kind, params, nodes, bulge, out)
    assert ctx.sync_status() == 0
    off = oracle.output_offsets(wl.orders)
    rng = np.random.default_rng(12)
    for e in sorted(rng.choice(wl.n_elem, 3, replace=False)):
        sub = wl.subset([e])
        r, roff = oracle_fill(sub)
        g = out[int(off[e]):int(off[e + 1])].cpu().numpy()
        err = per_type_errors(g, r, roff, sub.orders)
        assert err.max() <= TOL_MIXED, (e, err.max())
    del out
    plan.close()


def test_full_size_c2_sampled(torch_cuda, ctx):
    """The full 4096-element workload in the benchmark's launch shape; two seeded elements
    checked entry by entry against the oracle."""
    torch = torch_cuda
    wl = W.make("c2")
    params, nodes, bulge = p2s.device_inputs(wl)
    plan = p2s.Plan(ctx, wl.orders, 16)
    out = torch.empty(plan.output_entries, dtype=torch.float64, device="cuda")
    plan.fill(wl.kind, params, nodes, bulge, out)
    assert ctx.sync_status() == 0
    off = oracle.output_offsets(wl.orders)
    rng = np.random.default_rng(11)
    for e in sorted(rng.choice(wl.n_elem, 2, replace=False)):
        sub = wl.subset([e])
        r, roff = oracle_fill(sub)
        g = out[int(off[e]):int(off[e + 1])].cpu().numpy()
        err = per_type_errors(g, r, roff, sub.orders)
        assert err.max() <= TOL_FP64, (e, err.max())
    del out
    plan.close()
