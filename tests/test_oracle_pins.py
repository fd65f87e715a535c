"""Pins of the CPU oracle to things other than itself (CPU only).

Each test names what fixes the expected value: a library routine, a closed
form, an exact integral, a defining identity or a brute-force restatement of
the product-to-sum identity of Eq. (3)-(4) of arXiv:1703.09619.
"""
import warnings

import numpy as np
import pytest
from numpy.polynomial import legendre as L
from scipy import integrate

import oracle
from paper_1703_09619_gb300 import workloads as W
from tests import p2s_math as pm

TYPES = ("vv", "dv", "vd", "dd")


def unit_cube():
    return W.cube_nodes(1)[0]


# ---------------------------------------------------------------- 1-D pieces
@pytest.mark.parametrize("G", [1, 2, 3, 5, 8, 12, 16, 24, 33, 48, 64])
def test_gauss_legendre_matches_numpy(G):
    """Pin: Gauss-Legendre nodes/weights equal numpy's leggauss (library routine)."""
    x, w = oracle.gauss_legendre(G)
    xr, wr = L.leggauss(G)
    assert np.max(np.abs(x - xr)) < 2e-15
    assert np.max(np.abs(w - wr)) < 2e-14 * max(1.0, wr.max())
    assert abs(w.sum() - 2.0) < 1e-13


def test_legendre_values_and_derivatives_match_numpy():
    """Pin: P_j and P'_j equal numpy's legval / legder (library routines), interior and ends."""
    for x in [-1.0, -0.999, -0.7, -0.1, 0.0, 0.33, 0.9, 1.0]:
        P, dP = oracle.legendre(20, x)
        for j in range(20):
            c = np.zeros(j + 1)
            c[j] = 1
            assert abs(P[j] - L.legval(x, c)) < 1e-13
            ref = L.legval(x, L.legder(c)) if j > 0 else 0.0
            assert abs(dP[j] - ref) < 1e-11 * max(1.0, abs(ref))


@pytest.mark.parametrize("t", TYPES)
def test_linearisation_projection_matches_adams_neumann(t):
    """Pin: projection coefficients of Eq. (3) equal the Adams-Neumann formula
    (plus P'_m = sum (2j+1) P_j for the derivative types)."""
    d1, d2 = pm.TYPE_D[t]
    for m1 in range(12):
        for m2 in range(12):
            K = m1 + m2 + 1
            C = oracle.linearisation(d1, d2, m1, m2, K)
            ref = pm.product_dense(d1, d2, m1, m2, K + 1)
            scale = max(1.0, np.abs(ref).max())
            assert np.max(np.abs(C - ref)) < 1e-13 * scale, (t, m1, m2)


# ------------------------------------------------------------- closed forms
@pytest.mark.parametrize("N,G", [(1, 1), (2, 3), (3, 3), (4, 5), (5, 8)])
def test_unit_alpha_scalar_closed_form(N, G):
    """Pin: with alpha = 1 each entry is the product of the three 1-D closed forms
    (orthogonality, int P'_m P_n = 2 for n<m, m+n odd; int P'_m P'_n = min(min+1))."""
    orders = np.full((1, 1, 3), N, np.int32)
    params = np.array([[0.0, 0.0, 0.0, 0.0]])
    out, off, rc = oracle.fill(orders, oracle.ALPHA_SCALAR, params, unit_cube()[None], None, G)
    assert rc == 0
    mats = oracle.element_matrices(out, off, orders, 0)
    dofs = pm.dof_list(orders[0])
    for t in TYPES:
        ref = np.array([[pm.closed_form_1d(t, a[1], b[1]) * pm.closed_form_1d(t, a[2], b[2]) *
                         pm.closed_form_1d(t, a[3], b[3]) for b in dofs] for a in dofs])
        assert np.max(np.abs(mats[t] - ref)) < 1e-13 * max(1.0, np.abs(ref).max()), t


def test_unit_cube_metric_is_half_identity():
    """Pin: undistorted cube, eps = 1: J = I/2, detJ J^-1 J^-T = I/2, so diagonal
    blocks are 1/2 x closed form and off-diagonal blocks vanish."""
    N = 3
    orders = np.full((1, 3, 3), N, np.int32)
    params = np.array([[0.0, 1.0, 2.0, 3.0]])
    bulge = np.zeros((1, 4))
    out, off, rc = oracle.fill(orders, oracle.ALPHA_METRIC_EPS, params, unit_cube()[None], bulge, 4)
    assert rc == 0
    mats = oracle.element_matrices(out, off, orders, 0)
    dofs = pm.dof_list(orders[0])
    for t in TYPES:
        ref = np.array([[(0.5 if a[0] == b[0] else 0.0) * pm.closed_form_1d(t, a[1], b[1]) *
                         pm.closed_form_1d(t, a[2], b[2]) * pm.closed_form_1d(t, a[3], b[3])
                         for b in dofs] for a in dofs])
        assert np.max(np.abs(mats[t] - ref)) < 1e-13, t


def _exact_poly_alpha_matrix(t, N, coef, deg):
    """int f_u f_v f_w alpha for polynomial alpha from monomial moments (no quadrature)."""
    d1, d2 = pm.TYPE_D[t]

    def axis_table(deg_alpha):
        # T[m1, m2, i] = int P^(d1)_m1 P^(d2)_m2 x^i
        T = np.zeros((N, N, deg_alpha))
        for m1 in range(N):
            a = pm.legendre_power_coeffs(m1, d1)
            for m2 in range(N):
                b = pm.legendre_power_coeffs(m2, d2)
                prod = np.convolve(a, b)
                for i in range(deg_alpha):
                    T[m1, m2, i] = sum(prod[j] * pm.monomial_integral(j + i) for j in range(len(prod)))
        return T

    T = axis_table(deg)
    dofs = pm.dof_list([(N, N, N)])
    M = np.zeros((len(dofs), len(dofs)))
    for r, (_, m1, n1, p1) in enumerate(dofs):
        for c, (_, m2, n2, p2) in enumerate(dofs):
            M[r, c] = np.einsum("ijk,i,j,k->", coef, T[m1, m2], T[n1, n2], T[p1, p2])
    return M


@pytest.mark.parametrize("deg", [1, 3, 5])
def test_polynomial_alpha_is_integrated_exactly(deg):
    """Pin: for polynomial alpha of per-axis degree < deg the G-point rule is exact when
    2(N-1) + deg - 1 <= 2G - 1; compare with exact monomial moments int x^j = 2/(j+1)."""
    N = 3
    rng = np.random.default_rng(7 + deg)
    coef = rng.uniform(-1, 1, size=(deg, deg, deg))
    coef[0, 0, 0] += 3.0
    full = np.zeros((oracle.POLY_DEG,) * 3)
    full[:deg, :deg, :deg] = coef
    G = (2 * (N - 1) + deg - 1) // 2 + 1
    orders = np.full((1, 1, 3), N, np.int32)
    out, off, rc = oracle.fill(orders, oracle.ALPHA_POLY, full.reshape(1, -1), unit_cube()[None], None, G)
    mats = oracle.element_matrices(out, off, orders, 0)
    for t in TYPES:
        ref = _exact_poly_alpha_matrix(t, N, coef, deg)
        assert np.max(np.abs(mats[t] - ref)) < 1e-13 * np.abs(ref).max(), t
    # one point fewer must no longer be exact for the top-degree case
    if deg == 5:
        out2, off2, _ = oracle.fill(orders, oracle.ALPHA_POLY, full.reshape(1, -1), unit_cube()[None], None, G - 1)
        m2 = oracle.element_matrices(out2, off2, orders, 0)
        ref = _exact_poly_alpha_matrix("vv", N, coef, deg)
        assert np.max(np.abs(m2["vv"] - ref)) > 1e-10


def test_scalar_alpha_axes_against_adaptive_quadrature():
    """Pin: alpha - 1 = A sin(pi(u+phi)) cos(pi(v+psi)) exp(c w) is separable, so each entry
    is closed_form + A * product of three 1-D integrals, here from scipy's adaptive quad.
    The G = 30 rule is converged to ~1e-15 for these smooth factors."""
    A, phi, psi, cc = 0.5, 0.3, 0.8, 0.5
    N, G = 3, 30
    orders = np.full((1, 1, 3), N, np.int32)
    out, off, _ = oracle.fill(orders, oracle.ALPHA_SCALAR, np.array([[A, phi, psi, cc]]),
                              unit_cube()[None], None, G)
    mats = oracle.element_matrices(out, off, orders, 0)
    fu = lambda u: np.sin(np.pi * (u + phi))
    fv = lambda v: np.cos(np.pi * (v + psi))
    fw = lambda w: np.exp(cc * w)

    def one_d(t, m1, m2, f):
        d1, d2 = pm.TYPE_D[t]
        c1 = np.zeros(m1 + 1); c1[m1] = 1
        c2 = np.zeros(m2 + 1); c2[m2] = 1
        g1 = L.legder(c1) if d1 else c1
        g2 = L.legder(c2) if d2 else c2
        # integrals that vanish (parity) reach only roundoff, below epsabs: quad says so, harmlessly
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", integrate.IntegrationWarning)
            val, _ = integrate.quad(lambda x: L.legval(x, g1) * L.legval(x, g2) * f(x), -1, 1,
                                    epsabs=1e-15, epsrel=1e-14, limit=200)
        return val

    dofs = pm.dof_list(orders[0])
    for t in TYPES:
        ref = np.array([[pm.closed_form_1d(t, a[1], b[1]) * pm.closed_form_1d(t, a[2], b[2]) *
                         pm.closed_form_1d(t, a[3], b[3]) +
                         A * one_d(t, a[1], b[1], fu) * one_d(t, a[2], b[2], fv) * one_d(t, a[3], b[3], fw)
                         for b in dofs] for a in dofs])
        assert np.max(np.abs(mats[t] - ref)) < 1e-12 * np.abs(ref).max(), t


# ----------------------------------------------------------------- geometry
def test_geometry_map_corners_centre_and_jacobian():
    """Pin: the map hits the 8 nodes at the corners (bulge vanishes on faces), the centre
    is the node mean plus the bulge vector, and J equals central finite differences."""
    wl = W.make("c2", 8)
    for e in range(8):
        nodes, bulge = wl.nodes[e], wl.bulge[e]
        for i in range(8):
            u, v, w = [(-1.0 if ((i >> k) & 1) == 0 else 1.0) for k in range(3)]
            x, _ = oracle.geometry_map(nodes, bulge, u, v, w)
            assert np.max(np.abs(x - nodes[i])) < 1e-14
        x0, _ = oracle.geometry_map(nodes, bulge, 0, 0, 0)
        assert np.max(np.abs(x0 - (nodes.mean(axis=0) + bulge[0] * bulge[1:]))) < 1e-14
        rng = np.random.default_rng(e)
        for _ in range(5):
            p = rng.uniform(-0.95, 0.95, 3)
            _, J = oracle.geometry_map(nodes, bulge, *p)
            h = 1e-6
            Jfd = np.zeros((3, 3))
            for j in range(3):
                dp = np.zeros(3); dp[j] = h
                xp, _ = oracle.geometry_map(nodes, bulge, *(p + dp))
                xm, _ = oracle.geometry_map(nodes, bulge, *(p - dp))
                Jfd[:, j] = (xp - xm) / (2 * h)
            assert np.max(np.abs(J - Jfd)) < 1e-8


def test_metric_coupling_defining_identity():
    """Pin: alpha = eps detJ J^-1 J^-T satisfies J alpha J^T = eps detJ I, with J and detJ
    taken from finite differences of the map (independent of the oracle's cofactors),
    and eps = 1 + A sin(k . x) at the mapped point."""
    wl = W.make("c5", 16)
    rng = np.random.default_rng(3)
    for e in range(16):
        nodes, bulge, prm = wl.nodes[e], wl.bulge[e], wl.params[e]
        for _ in range(4):
            p = rng.uniform(-0.9, 0.9, 3)
            al, det = oracle.alpha_point(oracle.ALPHA_METRIC_EPS, prm, nodes, bulge, *p)
            h = 1e-6
            Jfd = np.zeros((3, 3))
            for j in range(3):
                dp = np.zeros(3); dp[j] = h
                xp, _ = oracle.geometry_map(nodes, bulge, *(p + dp))
                xm, _ = oracle.geometry_map(nodes, bulge, *(p - dp))
                Jfd[:, j] = (xp - xm) / (2 * h)
            x, _ = oracle.geometry_map(nodes, bulge, *p)
            eps = 1 + prm[0] * np.sin(prm[1:] @ x)
            dfd = np.linalg.det(Jfd)
            assert abs(det - dfd) < 1e-8
            lhs = Jfd @ al @ Jfd.T
            assert np.max(np.abs(lhs - eps * dfd * np.eye(3))) < 1e-7
            assert np.max(np.abs(al - al.T)) < 1e-15


# ---------------------------------------------------- brute-force P2S pin
@pytest.mark.parametrize("kind", ["scalar", "metric"])
def test_direct_equals_product_to_sum_small_orders(kind):
    """Pin (Eq. (3)-(4)): with the same G the direct sum equals sum_klq C^u C^v C^w I_klq,
    I_klq = sum w w w P_k P_l P_q alpha, C from Adams-Neumann -- written here in numpy."""
    G = 7
    if kind == "scalar":
        wl = W.make("c3", 2)
        orders = np.array([[[3, 2, 3]], [[2, 3, 1]]], np.int32)
        okind = oracle.ALPHA_SCALAR
    else:
        wl = W.make("c4", 2)
        orders = np.array([[[3, 2, 1], [1, 3, 2], [2, 2, 3]], [[2, 1, 3], [3, 3, 1], [1, 2, 2]]], np.int32)
        okind = oracle.ALPHA_METRIC_EPS
    out, off, _ = oracle.fill(orders, okind, wl.params, wl.nodes, wl.bulge, G)
    x, w = L.leggauss(G)
    Kmax = 6
    Pk = np.array([L.legval(x, np.eye(Kmax)[k]) for k in range(Kmax)])  # [k, a]
    B = Pk * w[None, :]
    for e in range(2):
        nc = orders.shape[1]
        alpha = np.zeros((G, G, G, nc, nc))  # a, b, c
        for a in range(G):
            for b in range(G):
                for c in range(G):
                    al, _ = oracle.alpha_point(okind, wl.params[e], wl.nodes[e], wl.bulge[e], x[a], x[b], x[c])
                    alpha[a, b, c] = al
        I = np.einsum("ka,lb,qc,abcij->ijklq", B, B, B, alpha)
        mats = oracle.element_matrices(out, off, orders, e)
        dofs = pm.dof_list(orders[e])
        for t in TYPES:
            d1, d2 = pm.TYPE_D[t]
            ref = np.zeros((len(dofs), len(dofs)))
            for r, (gi, m1, n1, p1) in enumerate(dofs):
                for c_, (gj, m2, n2, p2) in enumerate(dofs):
                    cu = pm.product_dense(d1, d2, m1, m2, Kmax)
                    cv = pm.product_dense(d1, d2, n1, n2, Kmax)
                    cw = pm.product_dense(d1, d2, p1, p2, Kmax)
                    ref[r, c_] = np.einsum("k,l,q,klq->", cu, cv, cw, I[gi, gj])
            scale = max(np.abs(ref).max(), 1e-300)
            assert np.max(np.abs(mats[t] - ref)) < 1e-14 * scale * 10, (kind, e, t)


# ---------------------------------------------------------------- invariants
def test_invariants_on_curved_metric_element():
    """Invariants of Eq. (2): vv diagonal blocks symmetric positive definite (alpha_ii > 0),
    vd(gi,gj) = dv(gj,gi)^T (alpha symmetric), dv rows with a zero test index on any axis
    vanish exactly (P'_0 = 0), dd symmetric."""
    wl = W.make("c2", 1)
    orders = np.full((1, 3, 3), 3, np.int32)
    out, off, rc = oracle.fill(orders, oracle.ALPHA_METRIC_EPS, wl.params, wl.nodes, wl.bulge, 6)
    assert rc == 0
    m = oracle.element_matrices(out, off, orders, 0)
    n1 = 27
    for g in range(3):
        blk = m["vv"][g * n1:(g + 1) * n1, g * n1:(g + 1) * n1]
        assert np.allclose(blk, blk.T, rtol=0, atol=1e-15 * np.abs(blk).max())
        assert np.linalg.eigvalsh(blk).min() > 0
    assert np.max(np.abs(m["vd"] - m["dv"].T)) < 1e-15 * np.abs(m["dv"]).max()
    assert np.max(np.abs(m["dd"] - m["dd"].T)) < 1e-15 * np.abs(m["dd"]).max()
    dofs = pm.dof_list(orders[0])
    for r, (_, a, b, c) in enumerate(dofs):
        if a == 0 or b == 0 or c == 0:
            assert np.all(m["dv"][r] == 0.0)
            assert np.all(m["dd"][r] == 0.0)


def test_output_offsets_count_four_n_squared():
    orders = np.array([[[2, 3, 4], [1, 1, 1], [5, 2, 2]], [[1, 1, 1], [1, 1, 1], [1, 1, 1]]], np.int32)
    off = oracle.output_offsets(orders, 0xF)
    n0 = 24 + 1 + 20
    assert off.tolist() == [0, 4 * n0 * n0, 4 * n0 * n0 + 4 * 9]
    off2 = oracle.output_offsets(orders, 0x5)
    assert off2[-1] == 2 * n0 * n0 + 2 * 9


def test_config1_shape_and_sanity():
    """Config c1 is one element of 4 x 64 x 64 entries; vv is SPD since alpha > 0 there."""
    wl = W.make("c1")
    out, off, rc = oracle.fill(wl.orders, wl.kind, wl.params, wl.nodes, None, wl.npts)
    assert out.size == 4 * 4096 and rc == 0
    m = oracle.element_matrices(out, off, wl.orders, 0)
    assert np.linalg.eigvalsh(m["vv"]).min() > 0
