"""Global assembly of element matrices on a conforming structured mesh -- TEST INFRASTRUCTURE ONLY.

Plain numpy, for small meshes: the element matrices of an operator (from ``oracle.fill_terms``,
Legendre basis P_m per axis) are transformed to the hierarchic C0 basis

    l_0 = (P_0 - P_1) / 2,   l_1 = (P_0 + P_1) / 2,   l_k = (P_k - P_{k-2}) / sqrt(2 (2k - 1))  (k >= 2)

(vertex functions of u = -1 and u = +1, then the normalised integrated Legendre bubbles), and
added into one dense global matrix.  On a structured mesh with aligned elements the global
space is the tensor product of 1-D C0 spaces, so a global dof is (gu, gv, gw) with 1-D indices

    vertex i (i = 0..n_el), then bubble k of interval i at n_el + 1 + i (N - 2) + (k - 2),

and global index (gu Ngv + gv) Ngw + gw (the local dof (m, n, p) has p fastest, likewise).
This is the "total" assembly step after the fill (arXiv:1703.09619, Sec. V); the product path
never imports this module.
"""
from __future__ import annotations

import numpy as np


def hierarchic_transform(N: int) -> np.ndarray:
    """T [N][N] (N >= 2): row k holds the Legendre coefficients of l_k."""
    if N < 2:
        raise ValueError("a C0 basis needs N >= 2 per axis")
    T = np.zeros((N, N))
    T[0, 0], T[0, 1] = 0.5, -0.5
    T[1, 0], T[1, 1] = 0.5, 0.5
    for k in range(2, N):
        c = 1.0 / np.sqrt(2.0 * (2 * k - 1))
        T[k, k], T[k, k - 2] = c, -c
    return T


def global_size_1d(n_el: int, N: int) -> int:
    return n_el + 1 + n_el * max(N - 2, 0)


def global_dof_1d(n_el: int, N: int, i: int, m: int) -> int:
    if m == 0:
        return i
    if m == 1:
        return i + 1
    return n_el + 1 + i * (N - 2) + (m - 2)


def assemble(nx, ny, nz, N, elem_mats):
    """Dense global matrix from Legendre-basis element matrices [E][n][n] (n = N^3), element
    (i, j, k) at (k ny + j) nx + i."""
    T = hierarchic_transform(N)
    Tk = np.kron(np.kron(T, T), T)
    gu, gv, gw = global_size_1d(nx, N), global_size_1d(ny, N), global_size_1d(nz, N)
    K = np.zeros((gu * gv * gw, gu * gv * gw))
    loc = np.array([(m, n, p) for m in range(N) for n in range(N) for p in range(N)])
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                e = (k * ny + j) * nx + i
                Ml = Tk @ elem_mats[e] @ Tk.T
                g = np.array([(global_dof_1d(nx, N, i, m) * gv + global_dof_1d(ny, N, j, n)) * gw
                              + global_dof_1d(nz, N, k, p) for m, n, p in loc])
                K[np.ix_(g, g)] += Ml
    return K


def vertex_indicator(nx, ny, nz, N):
    """Coefficients of the constant function 1 in the global hierarchic basis (1 on every
    vertex dof: the vertex functions form a partition of unity on each element)."""
    gu, gv, gw = global_size_1d(nx, N), global_size_1d(ny, N), global_size_1d(nz, N)
    c = np.zeros((gu, gv, gw))
    c[: nx + 1, : ny + 1, : nz + 1] = 1.0
    return c.reshape(-1)
