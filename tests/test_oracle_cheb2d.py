"""Pins of the 2-D curl-curl oracle (oracle/cheb2d.py; arXiv:1703.09619, Sec. III, Eq. (6)-(17)).

Each check fixes the oracle against something other than itself:
  * T_n and U_n against numpy's Chebyshev series (U_n = T'_{n+1} / (n+1));
  * the product-to-sum identities of Eq. (16) with the readings that the T.T and U.T lines carry a
    1/2 (U_{-1} = 0, U_{-j} = -U_{j-2}), T^ns of Eq. (17), and the form T^ns_n = -sum U_{n-2-2k}
    used by the GPU path, at random points;
  * an axis-aligned rectangle with eps = mu = 1: every block is a product of 1-D integrals, computed
    here exactly by numpy's Chebyshev multiplication and integration;
  * the curl of a gradient vanishes: S c = 0 for the coefficients of grad(T_a(u) T_b(v)), on curved
    elements with and without material;
  * S and M recomputed in physical space (E = E_u grad u + E_v grad v, curl = (d_u E_v - d_v E_u)/J,
    derivatives by numpy's chebder), a different code path for the metric terms and signs;
  * the element maps against the boundary curves of Fig. 1 and central differences;
  * symmetry, and M positive definite.
A last test plants mistakes in copies of the oracle and checks that a pin fails for each."""
import inspect
import types

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

from oracle import cheb2d
from paper_1703_09619_gb300 import workloads as W


def T_ref(n, x):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return npc.chebval(x, c)


def U_ref(n, x):
    if n < 0:
        return np.zeros_like(x)
    c = np.zeros(n + 2)
    c[n + 1] = 1.0
    return npc.chebval(x, npc.chebder(c)) / (n + 1)


def Tns_def(n, x):
    """Eq. (17) as printed."""
    base = 1.0 if n % 2 == 0 else x
    return (T_ref(n, x) - base) / (2.0 * (1.0 - x * x))


def pin_chebyshev_values(C=cheb2d):
    x = np.linspace(-0.97, 0.97, 41)
    for n in range(0, 20):
        assert np.allclose(C.cheb_T(n, x), T_ref(n, x), atol=1e-13)
        assert np.allclose(C.cheb_U(n, x), U_ref(n, x), atol=1e-12 * (n + 1) ** 2)


def test_chebyshev_values():
    pin_chebyshev_values()


def U_ext(j, x):
    """U_j with U_{-1} = 0 and U_{-j} = -U_{j-2} (reading of Eq. (16))."""
    if j >= 0:
        return U_ref(j, x)
    if j == -1:
        return np.zeros_like(x)
    return -U_ref(-j - 2, x)


def test_product_to_sum_identities():
    rng = np.random.default_rng(3)
    x = rng.uniform(-0.95, 0.95, 64)
    for a in range(0, 12):
        for b in range(0, 12):
            uu = U_ref(a, x) * U_ref(b, x)
            assert np.allclose(uu, Tns_def(abs(a - b), x) - Tns_def(a + b + 2, x), atol=1e-9 * (a + b + 2) ** 2)
            tt = T_ref(a, x) * T_ref(b, x)
            assert np.allclose(tt, 0.5 * (T_ref(abs(a - b), x) + T_ref(a + b, x)), atol=1e-12)
            ut = U_ref(a, x) * T_ref(b, x)
            assert np.allclose(ut, 0.5 * (U_ext(a + b, x) + U_ext(a - b, x)), atol=1e-11 * (a + b + 1))
    for n in range(0, 24):  # T^ns_n = -(U_{n-2} + U_{n-4} + ...), n < 2: 0
        s = sum(U_ref(j, x) for j in range(n - 2, -1, -2)) if n >= 2 else np.zeros_like(x)
        assert np.allclose(Tns_def(n, x), -s, atol=1e-9 * (n + 1) ** 2)


def rectangle(C, a, b):
    """The oracle's element_matrices (and couplings) rebound to the map x = a u, y = b v
    (J = a b) with eps = 1: its own code on an element with constant metric."""
    g = dict(C.__dict__)

    def geometry(p, u, v):
        z = np.zeros_like(u)
        return a * u, b * v, a + z, z, z, b + z

    g["geometry"] = geometry
    g["eps_r"] = lambda p, x, y: np.ones_like(x)
    g["couplings"] = types.FunctionType(C.couplings.__code__, g, "couplings", C.couplings.__defaults__)
    return types.FunctionType(C.element_matrices.__code__, g, "element_matrices")


def cheb_int(kind1, i, kind2, j):
    """Exact int_{-1}^{1} of the product of two Chebyshev polynomials (kind 'T' or 'U', index < 0: 0)."""
    def series(kind, n):
        if n < 0:
            return np.zeros(1)
        c = np.zeros(n + 2)
        if kind == "T":
            c[n] = 1.0
            return c
        c[n + 1] = 1.0
        return npc.chebder(c) / (n + 1)
    prod = npc.chebmul(series(kind1, i), series(kind2, j))
    F = npc.chebint(prod)
    return npc.chebval(1.0, F) - npc.chebval(-1.0, F)


def pin_rectangle_closed_form(C=cheb2d, M=3, N=4, a=0.7, b=1.3):
    S, Ms = rectangle(C, a, b)(np.zeros(5), M, N, max(M, N) + 3)
    iu = [(m, k) for m in range(M) for k in range(N + 1)]
    iv = [(m, k) for m in range(M + 1) for k in range(N)]
    ov = M * (N + 1)
    Sref, Mref = np.zeros_like(S), np.zeros_like(Ms)
    cS, cuu, cvv = 1.0 / (a * b), b / a, a / b
    for r, (m1, n1) in enumerate(iu):
        for c, (m2, n2) in enumerate(iu):
            Sref[r, c] = n1 * n2 * cS * cheb_int("U", m1, "U", m2) * cheb_int("U", n1 - 1, "U", n2 - 1)
            Mref[r, c] = cuu * cheb_int("U", m1, "U", m2) * cheb_int("T", n1, "T", n2)
        for c, (m2, n2) in enumerate(iv):
            Sref[r, ov + c] = -n1 * m2 * cS * cheb_int("U", m1, "U", m2 - 1) * cheb_int("U", n1 - 1, "U", n2)
    for r, (m1, n1) in enumerate(iv):
        for c, (m2, n2) in enumerate(iu):
            Sref[ov + r, c] = -m1 * n2 * cS * cheb_int("U", m1 - 1, "U", m2) * cheb_int("U", n1, "U", n2 - 1)
        for c, (m2, n2) in enumerate(iv):
            Sref[ov + r, ov + c] = m1 * m2 * cS * cheb_int("U", m1 - 1, "U", m2 - 1) * cheb_int("U", n1, "U", n2)
            Mref[ov + r, ov + c] = cvv * cheb_int("T", m1, "T", m2) * cheb_int("U", n1, "U", n2)
    assert np.abs(S - Sref).max() <= 1e-12 * np.abs(Sref).max()
    assert np.abs(Ms - Mref).max() <= 1e-12 * np.abs(Mref).max()


def test_rectangle_closed_form():
    pin_rectangle_closed_form()
    pin_rectangle_closed_form(M=5, N=2, a=1.1, b=0.4)


def gradient_coefficients(M, N, a, b):
    """Coefficients of grad(T_a(u) T_b(v)) = a U_{a-1}(u) T_b(v) grad u + b T_a(u) U_{b-1}(v) grad v."""
    c = np.zeros(cheb2d.dofs(M, N))
    if a >= 1:
        c[(a - 1) * (N + 1) + b] = a
    if b >= 1:
        c[M * (N + 1) + a * N + (b - 1)] = b
    return c


def pin_curl_of_gradient(C=cheb2d, M=4, N=3):
    mesh = W.make_mesh2d(3, 4, M, 0)
    for e in (0, 5, 11):  # filled (t < 0) and empty elements, corner and interior
        S, _ = C.element_matrices(mesh.params[e], M, N, M + 4)
        for a in range(M + 1):
            for b in range(N + 1):
                c = gradient_coefficients(M, N, a, b)
                assert np.abs(S @ c).max() <= 1e-12 * np.abs(S).max() * np.abs(c).max()


def test_curl_of_gradient_vanishes():
    pin_curl_of_gradient()
    pin_curl_of_gradient(M=2, N=5)


def pin_physical_space(C=cheb2d, M=3, N=3, G=7):
    """S and M from physical vectors at the points: grad u = (y_v, -x_v)/J, grad v = (-y_u, x_u)/J."""
    mesh = W.make_mesh2d(2, 2, M, G)
    x, w = np.polynomial.legendre.leggauss(G)
    for e in (0, 3):
        p = mesh.params[e]
        S, Ms = C.element_matrices(p, M, N, G)
        U, V = np.meshgrid(x, x, indexing="ij")
        Wt = np.outer(w, w)
        X, Y, xu, xv, yu, yv = C.geometry(p, U, V)
        J = xu * yv - xv * yu
        eps = 2.0 * np.exp(X + Y + 2.0) if p[4] else np.ones_like(X)
        gu = np.stack([yv / J, -xv / J])
        gv = np.stack([-yu / J, xu / J])
        fields, curls = [], []
        for m in range(M):
            for k in range(N + 1):  # E_u = U_m(u) T_k(v)
                Eu = U_ref(m, U) * T_ref(k, V)
                dEu_dv = U_ref(m, U) * (npc.chebval(V, npc.chebder(np.eye(k + 1)[k])) if k else 0 * V)
                fields.append(Eu * gu)
                curls.append(-dEu_dv / J)
        for m in range(M + 1):
            for k in range(N):  # E_v = T_m(u) U_k(v)
                Ev = T_ref(m, U) * U_ref(k, V)
                dEv_du = (npc.chebval(U, npc.chebder(np.eye(m + 1)[m])) if m else 0 * U) * U_ref(k, V)
                fields.append(Ev * gv)
                curls.append(dEv_du / J)
        n = len(fields)
        Sp, Mp = np.zeros((n, n)), np.zeros((n, n))
        for i in range(n):
            for j in range(n):
                Sp[i, j] = np.sum(Wt * J * curls[i] * curls[j])
                Mp[i, j] = np.sum(Wt * J * eps * (fields[i] * fields[j]).sum(axis=0))
        assert np.abs(S - Sp).max() <= 1e-11 * np.abs(Sp).max()
        assert np.abs(Ms - Mp).max() <= 1e-11 * np.abs(Mp).max()


def test_physical_space_recomputation():
    pin_physical_space()


def pin_geometry(C=cheb2d):
    """The element maps tile the domain bounded by x = +-g(y), y = +-f(x) (f, g of Fig. 1, written
    here), and their Jacobian entries match central differences of the map."""
    f = lambda x: -0.2 * (x * x - 1.0) ** 2 + 1.0
    g = lambda y: 0.2 * (y * y - 1.0) ** 2 + 1.0
    mesh = W.make_mesh2d(3, 4, 3, 5)
    r = np.linspace(-1.0, 1.0, 9)
    for e, p in enumerate(mesh.params):
        i, j = e % 3, e // 3
        if i == 2:  # right boundary u = 1
            x, y = C.geometry(p, np.ones_like(r), r)[:2]
            assert np.allclose(x, g(y), atol=1e-14)
        if j == 0:  # bottom boundary v = -1
            x, y = C.geometry(p, r, -np.ones_like(r))[:2]
            assert np.allclose(y, -f(x), atol=1e-14)
        u, v = np.meshgrid(np.linspace(-0.9, 0.9, 5), np.linspace(-0.8, 0.8, 5))
        h = 1e-6
        x, y, xu, xv, yu, yv = C.geometry(p, u, v)
        xp, yp = C.geometry(p, u + h, v)[:2]
        xm, ym = C.geometry(p, u - h, v)[:2]
        assert np.allclose(xu, (xp - xm) / (2 * h), atol=1e-8) and np.allclose(yu, (yp - ym) / (2 * h), atol=1e-8)
        xp, yp = C.geometry(p, u, v + h)[:2]
        xm, ym = C.geometry(p, u, v - h)[:2]
        assert np.allclose(xv, (xp - xm) / (2 * h), atol=1e-8) and np.allclose(yv, (yp - ym) / (2 * h), atol=1e-8)
    # neighbouring elements share their edge points
    a, b = mesh.params[0], mesh.params[1]
    assert np.allclose(np.array(C.geometry(a, np.ones_like(r), r)[:2]), np.array(C.geometry(b, -np.ones_like(r), r)[:2]))


def test_geometry():
    pin_geometry()


def pin_symmetry_and_definiteness(C=cheb2d):
    mesh = W.make_mesh2d(2, 2, 4, 8)
    for p in mesh.params:
        S, Ms = C.element_matrices(p, 4, 4, 8)
        assert np.abs(S - S.T).max() <= 1e-13 * np.abs(S).max()
        assert np.abs(Ms - Ms.T).max() <= 1e-13 * np.abs(Ms).max()
        assert np.linalg.eigvalsh(Ms)[0] > 0


def test_symmetry_and_definiteness():
    pin_symmetry_and_definiteness()


MUTATIONS = {
    "uv_sign": ("S[ou + r, ov + c] = -n1 * m2", "S[ou + r, ov + c] = n1 * m2"),
    "uv_index": ("integral(Uu[m1], Um1(m2), Um1(n1), Uu[n2], cS)", "integral(Uu[m1], Uu[m2], Um1(n1), Uu[n2], cS)"),
    "mass_uu_metric": ("e * (xv * xv + yv * yv) / J", "e * (xu * xu + yv * yv) / J"),
    "mass_uv_sign": ("-e * (xu * xv + yu * yv) / J", "e * (xu * xv + yu * yv) / J"),
    "uu_T_for_U": ("Ms[ou + r, ou + c] = integral(Uu[m1], Uu[m2], Tu[n1], Tu[n2], cuu)",
                   "Ms[ou + r, ou + c] = integral(Tu[m1], Uu[m2], Tu[n1], Tu[n2], cuu)"),
    "jacobian_sign": ("J = xu * yv - xv * yu", "J = xu * yv + xv * yu"),
    "side_derivative": ("xv = hs * g_side(t), ht * s * dg_side(t)", "xv = hs * g_side(t), ht * dg_side(t)"),
    "top_curve": ("return 1.0 - 0.2 * (x * x - 1.0) ** 2", "return 1.0 - 0.2 * (x * x - 1.0)"),
    "eps_exponent": ("2.0 * np.exp(x + y + 2.0)", "2.0 * np.exp(x - y + 2.0)"),
    "u_chebyshev": ("np.sin((n + 1) * th) / np.sin(th)", "np.sin(n * th) / np.sin(th)"),
    "vv_scale": ("S[ov + r, ov + c] = m1 * m2", "S[ov + r, ov + c] = m1 * m1"),
}
PINS = [pin_chebyshev_values, pin_rectangle_closed_form, pin_curl_of_gradient, pin_physical_space,
        pin_geometry, pin_symmetry_and_definiteness]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name):
    old, new = MUTATIONS[name]
    src = inspect.getsource(cheb2d)
    assert src.count(old) == 1, "mutation anchor not found exactly once: %s" % name
    mod = types.ModuleType("cheb2d_mutant")
    exec(compile(src.replace(old, new), "cheb2d_mutant", "exec"), mod.__dict__)
    caught = 0
    for pin in PINS:
        try:
            with np.errstate(all="ignore"):
                pin(mod)
        except (AssertionError, ValueError, IndexError, ZeroDivisionError):
            caught += 1
    assert caught > 0, "no pin caught the planted mistake %s" % name
