"""GPU checks of the contraction's tile configurations, the autotuner and graph replay.

Every work-unit shape computes each entry of Eq. (4) with the same operations in the same
order, so any tile configuration must give the default plan's output bit for bit; the
same holds for a fill replayed from a CUDA graph."""
import numpy as np
import pytest

import oracle
from paper_1703_09619_gb300 import p2s
from paper_1703_09619_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


def uneven(n=24, G=6):
    """c4 elements: orders U{2..8} per component and axis."""
    return W.make("c4", n).with_npts(G)


def fill(torch, ctx, wl, prec, tile=None, graph=False, types_mask=p2s.TYPES_ALL):
    params, nodes, bulge = p2s.device_inputs(wl)
    plan = p2s.Plan(ctx, wl.orders, int(wl.npts[0]), prec, types_mask=types_mask, tile=tile, graph=graph)
    out = torch.full((plan.output_entries,), float("nan"), dtype=torch.float64, device="cuda")
    plan.fill(wl.kind, params, nodes, bulge, out)
    assert ctx.sync_status() == 0
    res = out.cpu().numpy()
    cfg = plan.tile_config()
    plan.close()
    return res, cfg


@pytest.mark.parametrize("prec", [p2s.FP64, p2s.MIXED])
def test_tile_configs_bitwise_equal(torch, ctx, prec):
    wl = uneven()
    ref, cfg0 = fill(torch, ctx, wl, prec)
    assert cfg0["combo_target"] == 256 and cfg0["unit_kbytes"] == 100
    for tile in ({"combo_target": 64, "unit_kbytes": 24, "threads": 0},
                 {"combo_target": 128, "unit_kbytes": 48, "threads": 128},
                 {"combo_target": 512, "unit_kbytes": 100, "threads": 256},
                 {"combo_target": 1, "unit_kbytes": 0, "threads": 64}):
        got, cfg = fill(torch, ctx, wl, prec, tile=tile)
        assert np.array_equal(got, ref), tile
        if tile["threads"]:
            assert cfg["threads"] == tile["threads"]


def test_tuned_plan_matches_oracle(torch, ctx):
    wl = uneven(6, 5)
    got, _ = fill(torch, ctx, wl, p2s.FP64, tile={"combo_target": 64, "unit_kbytes": 48, "threads": 128})
    ref, off, _ = oracle.fill(wl.orders, wl.kind, wl.params, wl.nodes, wl.bulge, wl.npts)
    for e in range(wl.n_elem):
        for t in range(4):
            n = int(np.sqrt((off[e + 1] - off[e]) // 4))
            a = got[off[e] + t * n * n: off[e] + (t + 1) * n * n]
            b = ref[off[e] + t * n * n: off[e] + (t + 1) * n * n]
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_spec_kernel_tile_configs_bitwise_equal(torch, ctx):
    """Uniform N = 4 mixed plans use the specialised contraction; its slab follows combo_target."""
    wl = W.make("c5", 16).with_npts(8)
    ref, _ = fill(torch, ctx, wl, p2s.MIXED)
    for tile in ({"combo_target": 64}, {"combo_target": 128, "threads": 64}, {"combo_target": 512, "threads": 512}):
        got, _ = fill(torch, ctx, wl, p2s.MIXED, tile=dict({"unit_kbytes": 0, "threads": 0}, **tile))
        assert np.array_equal(got, ref), tile


def test_spec_kernel_default_cta(torch, ctx):
    """The uniform-order kernel's default CTA holds at most 128 threads (two stage-3
    combinations per thread at N = 4); it gives the one-thread-per-combination CTA's bits."""
    wl = W.make("c5", 40).with_npts(12)
    ref, cfg = fill(torch, ctx, wl, p2s.MIXED)
    assert cfg["threads"] == 128
    got, cfg2 = fill(torch, ctx, wl, p2s.MIXED, tile={"combo_target": 0, "unit_kbytes": 0, "threads": 256})
    assert cfg2["threads"] == 256 and np.array_equal(got, ref)


def with_orders(wl, lo, hi, seed):
    """The workload with per-component per-axis orders redrawn from U{lo..hi}."""
    import dataclasses
    rng = np.random.default_rng(seed)
    return dataclasses.replace(wl, orders=rng.integers(lo, hi + 1, size=wl.orders.shape).astype(np.int32))


@pytest.mark.parametrize("prec", [p2s.FP64, p2s.MIXED])
@pytest.mark.parametrize("mask", [0xF, 0x1, 0x2, 0x4, 0x8, 0x6, 0x9])
def test_bounded_order_kernel_matches_general_bitwise(torch, ctx, mask, prec):
    """Uneven orders 1..8: the bounded-order kernel (default) and the general kernel compute
    every entry with the same operations in the same order -- identical bits, in either
    precision and for every product-type subset (vd alone is computed directly, not as a
    transpose)."""
    wl = with_orders(uneven(20, 5), 1, 8, 17)
    ref, cfg = fill(torch, ctx, wl, prec, tile={"kernel": 1}, types_mask=mask)
    assert cfg["kernel"] == 1
    for tile in (None, {"combo_target": 1, "threads": 64}, {"combo_target": 512, "threads": 256, "kernel": 2}):
        got, cfg = fill(torch, ctx, wl, prec, tile=tile, types_mask=mask)
        assert cfg["kernel"] == (tile or {}).get("kernel", 0)
        assert np.array_equal(got, ref), (mask, tile)


@pytest.mark.parametrize("prec", [p2s.FP64, p2s.MIXED])
@pytest.mark.parametrize("name,N", [("c5", 4), ("c3", 8), ("c2", 6)])
def test_uniform_orders_all_kernels_bitwise(torch, ctx, name, N, prec):
    """Uniform orders: the library's kernel (mixed: per-order; FP64: bounded-order), the
    bounded-order kernel and the general kernel give identical bits."""
    wl = W.make(name, 3).with_npts(5)
    assert (wl.orders == N).all()
    ref, _ = fill(torch, ctx, wl, prec, tile={"kernel": 1})
    for tile in (None, {"kernel": 2}, {"kernel": 2, "combo_target": 64, "threads": 128}):
        got, _ = fill(torch, ctx, wl, prec, tile=tile)
        assert np.array_equal(got, ref), (name, tile)


@pytest.mark.parametrize("prec", [p2s.FP64, p2s.MIXED])
def test_bounded_order_kernel_refuses_orders_above_its_bound(torch, ctx, prec):
    wl = with_orders(uneven(4, 5), 2, 8, 31)
    p2s.Plan(ctx, wl.orders, 5, prec, tile={"kernel": 2}).close()
    wl.orders[0, 0, 0] = 9
    with pytest.raises(p2s.P2SError) as ex:
        p2s.Plan(ctx, wl.orders, 5, prec, tile={"kernel": 2})
    assert ex.value.code == p2s.ERR_ORDER


def test_bounded_order_kernel_against_oracle(torch, ctx):
    """Orders 1..8 with every order-1 edge: element-wise parity with the oracle at the mixed
    tolerance (1e-8 of max|M| per element and type)."""
    wl = with_orders(uneven(6, 5), 1, 8, 23)
    wl.orders[0, 0] = (1, 8, 1)
    wl.orders[1, 2] = (8, 1, 8)
    wl.orders[2] = 1
    got, _ = fill(torch, ctx, wl, p2s.MIXED)
    ref, off, _ = oracle.fill(wl.orders, wl.kind, wl.params, wl.nodes, wl.bulge, wl.npts)
    assert not np.isnan(got).any()
    for e in range(wl.n_elem):
        n = int(np.sqrt((off[e + 1] - off[e]) // 4))
        for t in range(4):
            a = got[off[e] + t * n * n: off[e] + (t + 1) * n * n]
            b = ref[off[e] + t * n * n: off[e] + (t + 1) * n * n]
            assert np.abs(a - b).max() <= 1e-8 * np.abs(b).max(), (e, t)


@pytest.mark.parametrize("prec", [p2s.FP64, p2s.MIXED])
def test_order_above_bound_takes_general_kernel(torch, ctx, prec):
    """An order above 8 anywhere in the batch: the general kernel for the whole batch, same bits."""
    wl = with_orders(uneven(8, 5), 2, 8, 29)
    wl.orders[3, 1, 2] = 9
    ref, _ = fill(torch, ctx, wl, prec, tile={"kernel": 1})
    got, _ = fill(torch, ctx, wl, prec)
    assert np.array_equal(got, ref)


def test_bad_tile_config(torch, ctx):
    wl = uneven(2)
    for tile in ({"combo_target": -1, "unit_kbytes": 0, "threads": 0},
                 {"combo_target": 0, "unit_kbytes": 0, "threads": 100},
                 {"combo_target": 0, "unit_kbytes": 300, "threads": 0},
                 {"combo_target": 0, "unit_kbytes": 0, "threads": 0, "kernel": 3}):
        with pytest.raises(p2s.P2SError) as ex:
            p2s.Plan(ctx, wl.orders, 4, p2s.FP64, tile=tile)
        assert ex.value.code == p2s.ERR_ARG


@pytest.mark.parametrize("prec", [p2s.FP64, p2s.MIXED])
def test_autotune_picks_a_fitting_config(torch, ctx, prec):
    """The tuner's pick (shape and kernel) fits and gives the default plan's bits."""
    wl = uneven(96, 8)
    params, nodes, bulge = p2s.device_inputs(wl)
    best, ms, tried = p2s.autotune_tiles(ctx, wl.orders, 8, wl.kind, params, nodes, bulge, prec,
                                         sample=48, reps=2)
    assert tried >= 1 and ms > 0
    assert 1 <= best["combo_target"] <= 4096 and 64 <= best["threads"] <= 512 and best["kernel"] in (0, 2)
    got, cfg = fill(torch, ctx, wl, prec, tile=best)
    ref, _ = fill(torch, ctx, wl, prec)
    assert np.array_equal(got, ref)
    assert cfg["threads"] == best["threads"]


@pytest.mark.parametrize("prec", [p2s.FP64, p2s.MIXED])
def test_graph_replay(torch, ctx, prec):
    """Replayed fills equal direct ones; new output pointers re-capture; new values behind
    the same pointers are read at replay."""
    wl = uneven(12, 6)
    ref, _ = fill(torch, ctx, wl, prec)
    params, nodes, bulge = p2s.device_inputs(wl)
    plan = p2s.Plan(ctx, wl.orders, 6, prec, graph=True)
    outs = [torch.full((plan.output_entries,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    for i in (0, 0, 1, 0):
        outs[i].fill_(float("nan"))
        plan.fill(wl.kind, params, nodes, bulge, outs[i])
        assert np.array_equal(outs[i].cpu().numpy(), ref)
    # same pointers, other values: element 0 takes element 1's inputs
    wl2 = wl.subset(np.r_[1, np.arange(1, wl.n_elem)])
    wl2.orders[:] = wl.orders
    p2, n2, b2 = p2s.device_inputs(wl2)
    params.copy_(p2)
    nodes.copy_(n2)
    bulge.copy_(b2)
    plan.fill(wl.kind, params, nodes, bulge, outs[0])
    ref2, _ = fill(torch, ctx, wl2, prec)
    assert np.array_equal(outs[0].cpu().numpy(), ref2)
    assert ctx.sync_status() == 0
    plan.close()
