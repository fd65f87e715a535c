"""Pins of the assembly oracle (oracle/assembly.py): hierarchic basis, global numbering, scatter.

  * the basis: l_0, l_1 are the vertex functions (1 at their own end, 0 at the other) and the
    bubbles vanish at both ends, checked by numpy's Legendre evaluation;
  * the undistorted mesh with eps = 1 has alpha = I/2 on every element, so the global diffusion
    stiffness is (S x M x M + M x S x M + M x M x S)/2 with S, M the 1-D global matrices assembled
    here from the 1-D closed forms int P_m P_n = 2/(2m+1) delta, int P'_m P'_n = min(m,n)(min+1);
  * on a curved mesh the constant function lies in the null space, and the matrix is symmetric
    and positive semi-definite with a one-dimensional null space."""
import numpy as np
import numpy.polynomial.legendre as npl
import pytest

import oracle
from oracle import assembly as A
from paper_1703_09619_gb300 import workloads as W


def test_hierarchic_basis_end_values():
    for N in (2, 3, 5, 8):
        T = A.hierarchic_transform(N)
        for k in range(N):
            lo, hi = npl.legval(-1.0, T[k]), npl.legval(1.0, T[k])
            want = (1.0, 0.0) if k == 0 else ((0.0, 1.0) if k == 1 else (0.0, 0.0))
            assert abs(lo - want[0]) < 1e-15 and abs(hi - want[1]) < 1e-15
        # bubbles are the normalised integrals of P_{k-1}: l_k' = sqrt((2k-1)/2) P_{k-1}
        for k in range(2, N):
            d = npl.legder(T[k])
            ref = np.zeros(N - 1)
            ref[k - 1] = np.sqrt((2 * k - 1) / 2.0)
            assert np.allclose(np.pad(d, (0, N - 1 - d.size)), ref, atol=1e-15)
    with pytest.raises(ValueError):
        A.hierarchic_transform(1)


def element_mats(mesh, N, G):
    wl = mesh.workload
    T, S = W.diffusion_terms()
    out, off, rc = oracle.fill_terms(wl.orders, wl.kind, wl.params, wl.nodes, wl.bulge, G, T, S)
    assert rc == 0
    n = N ** 3
    return out.reshape(wl.n_elem, n, n)


def global_1d(n_el, N, Mloc):
    g = A.global_size_1d(n_el, N)
    M = np.zeros((g, g))
    for i in range(n_el):
        idx = [A.global_dof_1d(n_el, N, i, m) for m in range(N)]
        M[np.ix_(idx, idx)] += Mloc
    return M


def test_undistorted_mesh_closed_form():
    nx, ny, nz, N = 3, 2, 2, 4
    mesh = W.make_mesh(nx, ny, nz, N, 5, jitter=0.0, bulge_amp=0.0, eps_amp=0.0)
    K = A.assemble(nx, ny, nz, N, element_mats(mesh, N, 5))
    T = A.hierarchic_transform(N)
    Mp = np.diag([2.0 / (2 * m + 1) for m in range(N)])
    Sp = np.array([[min(a, b) * (min(a, b) + 1) if (a + b) % 2 == 0 else 0.0 for b in range(N)] for a in range(N)])
    Ml, Sl = T @ Mp @ T.T, T @ Sp @ T.T
    Mu, Mv, Mw = global_1d(nx, N, Ml), global_1d(ny, N, Ml), global_1d(nz, N, Ml)
    Su, Sv, Sw = global_1d(nx, N, Sl), global_1d(ny, N, Sl), global_1d(nz, N, Sl)
    ref = 0.5 * (np.kron(np.kron(Su, Mv), Mw) + np.kron(np.kron(Mu, Sv), Mw) + np.kron(np.kron(Mu, Mv), Sw))
    assert np.abs(K - ref).max() <= 1e-13 * np.abs(ref).max()


def test_curved_mesh_null_space_symmetry_definiteness():
    nx, ny, nz, N = 2, 2, 1, 3
    mesh = W.make_mesh(nx, ny, nz, N, 6)
    K = A.assemble(nx, ny, nz, N, element_mats(mesh, N, 6))
    scale = np.abs(K).max()
    assert np.abs(K - K.T).max() <= 1e-13 * scale
    c = A.vertex_indicator(nx, ny, nz, N)
    assert np.abs(K @ c).max() <= 1e-12 * scale
    ev = np.linalg.eigvalsh(0.5 * (K + K.T))
    assert ev[0] > -1e-12 * scale and ev[1] > 1e-9 * scale
