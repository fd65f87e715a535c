"""Pins of the oracle's term-list fill (Eq. (2) with per-axis value/derivative choices and
several coupling-factor entries summed into one operator).

Each check fixes the oracle against something other than itself:
  * the undistorted unit cube with eps = 1 has alpha = I/2 exactly, so the diffusion
    stiffness is (S x M x M + M x S x M + M x M x S) / 2 with the 1-D closed forms
    int P_m P_n = 2/(2m+1) delta_mn and int P'_m P'_n = min(m,n)(min(m,n)+1) for m+n even;
  * on a curved element, a brute-force numpy evaluation of the definition (numpy's Legendre
    routines, alpha from the pinned coupling-factor routine) for random term lists;
  * one term with the same choice on every axis equals the uniform product type of the
    four-type fill (a second code path, pinned by test_oracle_pins);
  * invariants: a symmetric term list gives a symmetric matrix; the constant function lies
    in the null space of the diffusion stiffness."""
import numpy as np
import numpy.polynomial.legendre as npl

import oracle
from paper_1703_09619_gb300 import workloads as W


def mass_1d(n):
    return np.diag([2.0 / (2 * m + 1) for m in range(n)])


def stiff_1d(n):
    S = np.zeros((n, n))
    for m in range(n):
        for k in range(n):
            if (m + k) % 2 == 0:
                s = min(m, k)
                S[m, k] = s * (s + 1)
    return S


def cube_element(A=0.0):
    wl = W.make("c2", 1)
    nodes = W.cube_nodes(1)
    params = np.array([[A, 0.3, -0.2, 0.5]])
    return nodes, np.zeros((1, 4)), params


def test_diffusion_on_unit_cube_closed_form():
    nodes, bulge, params = cube_element()
    orders = np.array([[[4, 3, 5]]], dtype=np.int32)
    T, S = W.diffusion_terms()
    out, off, rc = oracle.fill_terms(orders, oracle.ALPHA_METRIC_EPS, params, nodes, bulge, 6, T, S)
    assert rc == 0
    Nu, Nv, Nw = orders[0, 0]
    Mu, Mv, Mw = mass_1d(Nu), mass_1d(Nv), mass_1d(Nw)
    Su, Sv, Sw = stiff_1d(Nu), stiff_1d(Nv), stiff_1d(Nw)
    ref = 0.5 * (np.kron(np.kron(Su, Mv), Mw) + np.kron(np.kron(Mu, Sv), Mw) + np.kron(np.kron(Mu, Mv), Sw))
    got = out.reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def legendre_tables(N, x):
    """P_m(x) and P'_m(x) for m < N by numpy."""
    P = np.zeros((N, x.size))
    dP = np.zeros((N, x.size))
    for m in range(N):
        c = np.zeros(m + 1)
        c[m] = 1.0
        P[m] = npl.legval(x, c)
        dP[m] = npl.legval(x, npl.legder(c)) if m > 0 else 0.0
    return P, dP


def brute_force(orders, kind, params, nodes, bulge, G, terms, scales):
    """The definition of a term-list operator evaluated with numpy (one element)."""
    x, w = npl.leggauss(G)
    nmax = int(orders.max())
    P, dP = legendre_tables(nmax, x)
    tab = (P, dP)
    na = 3 if kind == oracle.ALPHA_METRIC_EPS else 1
    al = np.zeros((G, G, G, na, na))  # [a, b, c]
    for a in range(G):
        for b in range(G):
            for c in range(G):
                A_, _ = oracle.alpha_point(kind, params, nodes, bulge, x[a], x[b], x[c])
                al[a, b, c] = A_[:na, :na]
    ndofs = [int(np.prod(o)) for o in orders]
    n = sum(ndofs)
    start = np.concatenate([[0], np.cumsum(ndofs)])
    M = np.zeros((n, n))
    for (gi, gj, sa, sb, du, dv, dw, eu, ev, ew), sc in zip(terms, scales):
        Ni, Nj = orders[gi], orders[gj]
        fu = np.einsum("ia,ja,a->ija", tab[du][: Ni[0]], tab[eu][: Nj[0]], w)
        fv = np.einsum("ia,ja,a->ija", tab[dv][: Ni[1]], tab[ev][: Nj[1]], w)
        fw = np.einsum("ia,ja,a->ija", tab[dw][: Ni[2]], tab[ew][: Nj[2]], w)
        blk = np.einsum("mqa,nrb,psc,abc->mnpqrs", fu, fv, fw, al[:, :, :, sa, sb])
        blk = blk.reshape(Ni[0] * Ni[1] * Ni[2], Nj[0] * Nj[1] * Nj[2])
        M[start[gi]:start[gi + 1], start[gj]:start[gj + 1]] += sc * blk
    return M


def random_terms(rng, n_comp, na, count):
    terms = []
    for _ in range(count):
        gi, gj = rng.integers(0, n_comp, 2)
        sa, sb = rng.integers(0, na, 2)
        terms.append([gi, gj, sa, sb] + list(rng.integers(0, 2, 6)))
    return np.array(terms, dtype=np.int32), rng.normal(size=count)


def test_random_terms_match_brute_force_metric():
    rng = np.random.default_rng(11)
    wl = W.make("c4", 3)
    for e in range(2):
        orders = np.array([[2, 3, 2], [3, 2, 2]], dtype=np.int32)
        T, S = random_terms(rng, 2, 3, 7)
        out, off, rc = oracle.fill_terms(orders[None], wl.kind, wl.params[e:e + 1], wl.nodes[e:e + 1],
                                         wl.bulge[e:e + 1], 4, T, S)
        assert rc == 0
        ref = brute_force(orders, wl.kind, wl.params[e], wl.nodes[e], wl.bulge[e], 4, T, S)
        got = out.reshape(ref.shape)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_random_terms_match_brute_force_scalar():
    rng = np.random.default_rng(12)
    wl = W.make("c3", 1)
    orders = np.array([[3, 2, 3]], dtype=np.int32)
    T, S = random_terms(rng, 1, 1, 5)
    out, off, rc = oracle.fill_terms(orders[None], wl.kind, wl.params, None, None, 5, T, S)
    assert rc == 0
    ref = brute_force(orders, wl.kind, wl.params[0], np.zeros((8, 3)), None, 5, T, S)
    assert np.abs(out.reshape(ref.shape) - ref).max() <= 1e-13 * np.abs(ref).max()


def test_uniform_term_equals_product_type():
    wl = W.make("c4", 2).with_npts(4)
    wl.orders[:] = np.minimum(wl.orders, 3)
    ref, off4, _ = oracle.fill(wl.orders, wl.kind, wl.params, wl.nodes, wl.bulge, 4)
    for t, (d1, d2) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
        for gi, gj in ((0, 0), (1, 2), (2, 0)):
            T = np.array([[gi, gj, gi, gj, d1, d1, d1, d2, d2, d2]], dtype=np.int32)
            out, off, rc = oracle.fill_terms(wl.orders, wl.kind, wl.params, wl.nodes, wl.bulge, 4, T, [1.0])
            for e in range(wl.n_elem):
                n = int(round(np.sqrt(off[e + 1] - off[e])))
                got = out[off[e]:off[e + 1]].reshape(n, n)
                full = oracle.element_matrices(ref, off4, wl.orders, e)[oracle.TYPES[t]]
                ndofs = [int(np.prod(o)) for o in wl.orders[e]]
                st = np.concatenate([[0], np.cumsum(ndofs)])
                blk = full[st[gi]:st[gi + 1], st[gj]:st[gj + 1]]
                assert np.array_equal(got[st[gi]:st[gi + 1], st[gj]:st[gj + 1]], blk)
                mask = np.ones_like(got, dtype=bool)
                mask[st[gi]:st[gi + 1], st[gj]:st[gj + 1]] = False
                assert not got[mask].any()


def test_diffusion_invariants_on_curved_element():
    wl = W.make("c5", 2)
    orders = np.full((2, 1, 3), 3, dtype=np.int32)
    T, S = W.diffusion_terms()
    out, off, rc = oracle.fill_terms(orders, wl.kind, wl.params, wl.nodes, wl.bulge, 6, T, S)
    assert rc == 0
    for e in range(2):
        K = out[off[e]:off[e + 1]].reshape(27, 27)
        scale = np.abs(K).max()
        assert np.abs(K - K.T).max() <= 1e-13 * scale
        # constant function (dof 0) has zero gradient: its row and column vanish
        assert not K[0].any() and not K[:, 0].any()
        # positive semi-definite with the constant as the only null direction
        ev = np.linalg.eigvalsh(0.5 * (K + K.T))
        assert ev[0] > -1e-12 * scale and ev[1] > 1e-8 * scale
