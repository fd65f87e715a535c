"""The seeded input generators follow their stated recipes (CPU).

Every configuration's element count, component count, orders, quadrature size and coupling-factor
parameters, the geometry's jitter and bulge, the wavenumber distributions, and the generators'
determinism; and every curved element keeps detJ > 0 over the reference cube (the fill flags an
element otherwise).  The recipes are those of the workload module's docstring."""
import numpy as np
import pytest

import oracle
from paper_1703_09619_gb300 import workloads as W

CORNERS = np.array([[(i >> 0) & 1, (i >> 1) & 1, (i >> 2) & 1] for i in range(8)], dtype=np.float64)


@pytest.fixture(scope="module")
def batches():
    return {name: W.make(name) for name in ("c1", "c2", "c3", "c4", "c5")}


def test_sizes_orders_and_rules(batches):
    expect = {  # elements, components, orders (None: uneven), points, kind
        "c1": (1, 1, 4, 12, W.KIND_SCALAR),
        "c2": (4096, 3, 6, 16, W.KIND_METRIC_EPS),
        "c3": (512, 1, 8, 24, W.KIND_SCALAR),
        "c4": (8192, 3, None, 16, W.KIND_METRIC_EPS),
        "c5": (32768, 3, 4, 48, W.KIND_METRIC_EPS),
    }
    for name, (E, nc, N, G, kind) in expect.items():
        w = batches[name]
        assert (w.n_elem, w.n_comp, w.kind) == (E, nc, kind), name
        assert w.orders.shape == (E, nc, 3) and w.orders.dtype == np.int32
        assert w.params.shape == (E, 4) and w.nodes.shape == (E, 8, 3) and w.bulge.shape == (E, 4)
        assert (w.npts == G).all(), name
        if N is not None:
            assert (w.orders == N).all(), name
    o = batches["c4"].orders  # U{2..8}, drawn independently per element, component and axis
    assert o.min() == 2 and o.max() == 8
    counts = np.bincount(o.ravel(), minlength=9)[2:]
    assert abs(counts / counts.sum() - 1 / 7).max() < 0.01
    assert len(np.unique(o.reshape(o.shape[0], -1), axis=0)) > 8000  # order triples vary by element


def test_scalar_recipes(batches):
    c1 = batches["c1"]
    assert np.array_equal(c1.params[0], [0.5, 0.0, 0.0, 0.5])  # 1 + 0.5 sin(pi u) cos(pi v) exp(w/2)
    c3 = batches["c3"]
    assert (c3.params[:, 0] == 0.5).all() and (c3.params[:, 3] == 0.5).all()
    for col in (1, 2):  # phi_e, psi_e ~ U[0, 1)
        x = c3.params[:, col]
        assert x.min() >= 0.0 and x.max() < 1.0
        assert abs(x.mean() - 0.5) < 0.05 and abs(x.std() - np.sqrt(1 / 12)) < 0.03
    assert abs(np.corrcoef(c3.params[:, 1], c3.params[:, 2])[0, 1]) < 0.15
    for w in (c1, c3):  # the undistorted reference cube, no bulge
        assert np.array_equal(w.nodes, np.broadcast_to(CORNERS, w.nodes.shape))
        assert not w.bulge.any()


def test_curved_geometry(batches):
    for name in ("c2", "c4", "c5"):
        w = batches[name]
        jit = (w.nodes - CORNERS).ravel()  # i.i.d. U(-0.15, 0.15) per node and coordinate
        assert jit.min() > -0.15 and jit.max() < 0.15
        assert abs(jit.mean()) < 0.005 and abs(jit.std() - 0.15 / np.sqrt(3)) < 0.005
        assert (w.bulge[:, 0] == 0.1).all()
        b = w.bulge[:, 1:]
        assert np.allclose(np.linalg.norm(b, axis=1), 1.0, atol=1e-12)
        assert abs(b.mean(axis=0)).max() < 0.05  # directions spread over the sphere


def test_material_recipes(batches):
    c2 = batches["c2"]  # eps = 1 + 0.5 sin(2 pi x.d), one unit d for the batch
    assert (c2.params[:, 0] == 0.5).all()
    k = c2.params[:, 1:]
    assert (k == k[0]).all()
    assert np.isclose(np.linalg.norm(k[0]), 2 * np.pi, rtol=1e-13)
    c4 = batches["c4"]  # eps = 1 + 0.5 sin(2 pi |k| x.d_e), |k| log-uniform on [1, 8]
    assert (c4.params[:, 0] == 0.5).all()
    km = np.linalg.norm(c4.params[:, 1:], axis=1) / (2 * np.pi)
    assert km.min() >= 1.0 - 1e-12 and km.max() <= 8.0 + 1e-12
    lk = np.log(km) / np.log(8.0)  # uniform on [0, 1]
    assert abs(lk.mean() - 0.5) < 0.02 and abs(lk.std() - np.sqrt(1 / 12)) < 0.02
    c5 = batches["c5"]  # eps = 1 + 0.8 sin(k_e . x), |k_e| log-uniform on [1, 40]
    assert (c5.params[:, 0] == 0.8).all()
    km = np.linalg.norm(c5.params[:, 1:], axis=1)
    assert km.min() >= 1.0 - 1e-12 and km.max() <= 40.0 + 1e-12
    lk = np.log(km) / np.log(40.0)
    assert abs(lk.mean() - 0.5) < 0.01 and abs(lk.std() - np.sqrt(1 / 12)) < 0.01
    d = c5.params[:, 1:] / km[:, None]
    assert abs(d.mean(axis=0)).max() < 0.03


def test_seeded_prefixes_and_shards():
    for name in ("c2", "c4", "c5"):
        a, b = W.make(name), W.make(name)
        for f in ("orders", "params", "nodes", "bulge", "npts"):
            assert np.array_equal(getattr(a, f), getattr(b, f)), (name, f)
        p = W.make(name, 100)  # element e does not depend on how many are taken
        for f in ("orders", "params", "nodes", "bulge", "npts"):
            assert np.array_equal(getattr(p, f), getattr(a, f)[:100]), (name, f)
        s = W.make(name, 100, shard=1)  # another batch of the same recipe
        assert not np.array_equal(s.nodes, p.nodes) and not np.array_equal(s.params, p.params)
        assert (s.params[:, 0] == p.params[0, 0]).all() and (s.bulge[:, 0] == 0.1).all()
    with pytest.raises(ValueError):
        W.make("c2", 1, shard=-1)


def _jacobians(nodes, bulge, u, v, w):
    """dx/d(u,v,w) of the trilinear-plus-bulge map at points (u, v, w), every element at once:
    [E, P, 3 (x), 3 (u, v, w)]."""
    s = 2 * CORNERS - 1  # corner signs, node index iu + 2 iv + 4 iw
    fu, fv, fw = (1 + s[:, 0][None] * u[:, None]), (1 + s[:, 1][None] * v[:, None]), (1 + s[:, 2][None] * w[:, None])
    dN = np.stack([s[:, 0][None] * fv * fw, fu * s[:, 1][None] * fw, fu * fv * s[:, 2][None]], axis=-1) / 8  # [P, 8, 3]
    J = np.einsum("enx,pnd->epxd", nodes, dN)
    h = np.pi / 2
    cu, cv, cw = np.cos(h * u), np.cos(h * v), np.cos(h * w)
    db = np.stack([-h * np.sin(h * u) * cv * cw, -h * cu * np.sin(h * v) * cw, -h * cu * cv * np.sin(h * w)], -1)
    return J + np.einsum("e,ex,pd->epxd", bulge[:, 0], bulge[:, 1:], db)


def test_curved_elements_keep_positive_jacobian(batches):
    g = np.linspace(-1.0, 1.0, 6)
    u, v, w = (a.ravel() for a in np.meshgrid(g, g, g, indexing="ij"))
    # the map above is the one the fill integrates over: the oracle's J at sample points
    c5 = batches["c5"]
    J = _jacobians(c5.nodes[:3], c5.bulge[:3], u, v, w)
    for e in range(3):
        for p in (0, 17, 100, 215):
            _, Jo = oracle.geometry_map(c5.nodes[e], c5.bulge[e], u[p], v[p], w[p])
            assert np.allclose(J[e, p], Jo, rtol=0, atol=1e-14)
    for name in ("c2", "c4", "c5"):
        wl = batches[name]
        dets = np.concatenate([np.linalg.det(_jacobians(wl.nodes[i:i + 4096], wl.bulge[i:i + 4096], u, v, w)).ravel()
                               for i in range(0, wl.n_elem, 4096)])
        assert dets.min() > 0.02, (name, dets.min())  # the unit cube's map has detJ = 1/8
