"""Element matrices of the 2-D curl-curl example (arXiv:1703.09619, Sec. III) -- TEST INFRASTRUCTURE ONLY.

Plain numpy in FP64, by the definitions: the curl-conforming basis of Eq. (6)
    E_u = U_m(u) T_n(v)  (m < M, n <= N),     E_v = T_m(u) U_n(v)  (m <= M, n < N),
and the stiffness and mass submatrices of Eq. (8)-(15) as direct 2-D Gauss-Legendre sums over the
G x G points of the reference square, with the coupling factors
    S: 1 / (mu_r J),   M_uu: eps_r (x_v^2 + y_v^2) / J,   M_uv = M_vu: -eps_r (x_u x_v + y_u y_v) / J,
    M_vv: eps_r (x_u^2 + y_u^2) / J.
T_n and U_n are evaluated from their trigonometric definitions (cos(n theta), sin((n+1) theta) /
sin(theta), x = cos(theta)); the geometry is the exact map of the mesh (paper_1703_09619_gb300.
workloads.Mesh2D).  Dof order per element: the E_u functions (m, n) at m (N+1) + n, then the E_v
functions at M (N+1) + m N + n; S and M are n x n with rows = testing and columns = basis functions.
The product path never imports this module.
"""
from __future__ import annotations

import numpy as np


def cheb_T(n, x):
    return np.cos(n * np.arccos(x))


def cheb_U(n, x):
    th = np.arccos(x)
    return np.sin((n + 1) * th) / np.sin(th)


def f_top(x):
    return 1.0 - 0.2 * (x * x - 1.0) ** 2


def g_side(y):
    return 1.0 + 0.2 * (y * y - 1.0) ** 2


def df_top(x):
    return -0.8 * x * (x * x - 1.0)


def dg_side(y):
    return 0.8 * y * (y * y - 1.0)


def geometry(p, u, v):
    """x, y and the Jacobian entries (x_u, x_v, y_u, y_v) of element p = (s_lo, s_hi, t_lo, t_hi, .)
    at reference points (u, v): X(s, t) = (s g(t), t f(s)), s and t affine in u and v."""
    hs, ht = 0.5 * (p[1] - p[0]), 0.5 * (p[3] - p[2])
    s = p[0] + (u + 1.0) * hs
    t = p[2] + (v + 1.0) * ht
    x, y = s * g_side(t), t * f_top(s)
    xu, xv = hs * g_side(t), ht * s * dg_side(t)
    yu, yv = hs * t * df_top(s), ht * f_top(s)
    return x, y, xu, xv, yu, yv


def eps_r(p, x, y):
    return 2.0 * np.exp(x + y + 2.0) if p[4] else np.ones_like(x)


def couplings(p, u, v, mu_r=1.0):
    """(c_S, c_uu, c_uv, c_vv) at the points (u, v)."""
    x, y, xu, xv, yu, yv = geometry(p, u, v)
    J = xu * yv - xv * yu
    e = eps_r(p, x, y)
    return 1.0 / (mu_r * J), e * (xv * xv + yv * yv) / J, -e * (xu * xv + yu * yv) / J, e * (xu * xu + yu * yu) / J


def dofs(M, N):
    return M * (N + 1) + (M + 1) * N


def element_matrices(p, M, N, G):
    """(S, Mass) of one element by direct 2-D Gauss-Legendre sums (Eq. (8)-(15))."""
    x, w = np.polynomial.legendre.leggauss(G)
    U, V = np.meshgrid(x, x, indexing="ij")        # [a][b]: u = x_a, v = x_b
    W = np.outer(w, w)
    cS, cuu, cuv, cvv = couplings(p, U, V)
    K = max(M, N) + 1
    Tu = np.array([cheb_T(k, x) for k in range(K)])  # [k][point]
    Uu = np.array([cheb_U(k, x) for k in range(K)])
    n = dofs(M, N)
    S = np.zeros((n, n))
    Ms = np.zeros((n, n))
    iu = [(m, k) for m in range(M) for k in range(N + 1)]   # E_u: U_m(u) T_k(v)
    iv = [(m, k) for m in range(M + 1) for k in range(N)]   # E_v: T_m(u) U_k(v)
    ou = 0
    ov = M * (N + 1)

    def integral(fu1, fu2, fv1, fv2, c):
        return np.sum(W * np.outer(fu1 * fu2, fv1 * fv2) * c)

    def Um1(k):  # U_{k-1}, with U_{-1} = 0
        return Uu[k - 1] if k >= 1 else np.zeros(G)

    for r, (m1, n1) in enumerate(iu):
        for c, (m2, n2) in enumerate(iu):       # Eq. (8), (12)
            S[ou + r, ou + c] = n1 * n2 * integral(Uu[m1], Uu[m2], Um1(n1), Um1(n2), cS)
            Ms[ou + r, ou + c] = integral(Uu[m1], Uu[m2], Tu[n1], Tu[n2], cuu)
        for c, (m2, n2) in enumerate(iv):       # Eq. (9), (13)
            S[ou + r, ov + c] = -n1 * m2 * integral(Uu[m1], Um1(m2), Um1(n1), Uu[n2], cS)
            Ms[ou + r, ov + c] = integral(Uu[m1], Tu[m2], Tu[n1], Uu[n2], cuv)
    for r, (m1, n1) in enumerate(iv):
        for c, (m2, n2) in enumerate(iu):       # Eq. (10), (14)
            S[ov + r, ou + c] = -m1 * n2 * integral(Um1(m1), Uu[m2], Uu[n1], Um1(n2), cS)
            Ms[ov + r, ou + c] = integral(Tu[m1], Uu[m2], Uu[n1], Tu[n2], cuv)
        for c, (m2, n2) in enumerate(iv):       # Eq. (11), (15)
            S[ov + r, ov + c] = m1 * m2 * integral(Um1(m1), Um1(m2), Uu[n1], Uu[n2], cS)
            Ms[ov + r, ov + c] = integral(Tu[m1], Tu[m2], Uu[n1], Uu[n2], cvv)
    return S, Ms


def fill(params, M, N, G):
    """Element matrices of a batch: (S [E][n][n], Mass [E][n][n])."""
    out = [element_matrices(p, M, N, G) for p in np.asarray(params)]
    return np.array([o[0] for o in out]), np.array([o[1] for o in out])
