"""CPU checks of the assembly's CSR structure (p2s_assembly_structure_host) against brute force:
the set of (row, column) pairs that some element couples, built here from the oracle's 1-D dof
numbering, must be exactly the CSR pattern, each row sorted and without repeats."""
import numpy as np
import pytest

from oracle import assembly as A
from paper_1703_09619_gb300 import p2s


def brute_pattern(nx, ny, nz, N):
    gv, gw = A.global_size_1d(ny, N), A.global_size_1d(nz, N)
    pairs = set()
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                g = [(A.global_dof_1d(nx, N, i, m) * gv + A.global_dof_1d(ny, N, j, n)) * gw
                     + A.global_dof_1d(nz, N, k, p) for m in range(N) for n in range(N) for p in range(N)]
                pairs.update((a, b) for a in g for b in g)
    return pairs


@pytest.mark.parametrize("nx,ny,nz,N", [(1, 1, 1, 2), (2, 1, 1, 3), (3, 2, 2, 2), (2, 3, 1, 4), (1, 2, 2, 5)])
def test_structure_is_the_coupling_pattern(nx, ny, nz, N):
    row_ptr, col_idx = p2s.assembly_structure(nx, ny, nz, N)
    rows = A.global_size_1d(nx, N) * A.global_size_1d(ny, N) * A.global_size_1d(nz, N)
    assert row_ptr.shape == (rows + 1,) and row_ptr[0] == 0
    assert np.all(np.diff(row_ptr) > 0)
    got = set()
    for r in range(rows):
        cols = col_idx[row_ptr[r]:row_ptr[r + 1]]
        assert np.all(np.diff(cols) > 0)  # sorted, no repeats
        got.update((r, int(c)) for c in cols)
    assert got == brute_pattern(nx, ny, nz, N)


def test_structure_argument_errors():
    for args in ((0, 1, 1, 3), (1, 1, 1, 1), (1, 1, 1, 13), (1, -2, 1, 4)):
        with pytest.raises(p2s.P2SError) as ex:
            p2s.assembly_structure(*args)
        assert ex.value.code == p2s.ERR_ARG
