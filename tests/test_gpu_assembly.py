"""GPU parity of the global assembly (p2s_assembly_fill) against the oracle.

Small meshes: the CSR values against the oracle's dense global matrix (oracle.fill_terms element
matrices, oracle.assembly.assemble), max |K_gpu - K_oracle| <= tol max |K_oracle| with tol = 1e-12
(FP64 fill) and 1e-8 (mixed fill).  A larger mesh: sampled rows rebuilt by the oracle from the
(at most 8) elements around the row's dof, plus symmetry and the constant function in the null
space of the diffusion stiffness over the whole matrix."""
import numpy as np
import pytest

import oracle
from oracle import assembly as A
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


def gpu_assemble(torch, ctx, mesh, N, G, prec, reps=1, graph=False):
    wl = mesh.workload
    T, S = W.diffusion_terms()
    asm = p2s.Assembly(ctx, mesh.nx, mesh.ny, mesh.nz, N, G, T, S, wl.kind, prec, graph=graph)
    dp, dn, db = (torch.as_tensor(np.ascontiguousarray(a), device="cuda") for a in (wl.params, wl.nodes, wl.bulge))
    vals = torch.full((asm.nnz,), float("nan"), dtype=torch.float64, device="cuda")
    outs = []
    for _ in range(reps):
        asm.fill(wl.kind, dp, dn, db, vals)
        outs.append(vals.cpu().numpy().copy())
    rc = ctx.sync_status()
    row_ptr, col_idx = asm.structure()
    asm.close()
    return outs, row_ptr, col_idx, rc


def dense(row_ptr, col_idx, vals):
    rows = row_ptr.size - 1
    K = np.zeros((rows, rows))
    r = np.repeat(np.arange(rows), np.diff(row_ptr))
    K[r, col_idx] = vals
    return K


def oracle_global(mesh, N, G):
    wl = mesh.workload
    T, S = W.diffusion_terms()
    out, off, rc = oracle.fill_terms(wl.orders, wl.kind, wl.params, wl.nodes, wl.bulge, G, T, S)
    assert rc == 0
    n = N ** 3
    return A.assemble(mesh.nx, mesh.ny, mesh.nz, N, out.reshape(wl.n_elem, n, n))


@pytest.mark.parametrize("nx,ny,nz,N,G", [(1, 1, 1, 2, 3), (2, 2, 2, 3, 5), (3, 2, 1, 4, 6), (1, 2, 3, 5, 6),
                                          (2, 1, 1, 6, 7)])
def test_assembly_matches_oracle_fp64(torch, ctx, nx, ny, nz, N, G):
    mesh = W.make_mesh(nx, ny, nz, N, G, seed=nx + 3 * ny + 7 * nz + N)
    (vals,), row_ptr, col_idx, rc = gpu_assemble(torch, ctx, mesh, N, G, p2s.FP64)
    assert rc == 0 and not np.isnan(vals).any()
    K = dense(row_ptr, col_idx, vals)
    ref = oracle_global(mesh, N, G)
    assert np.abs(K - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("nx,ny,nz,N,G", [(2, 2, 2, 4, 8), (3, 1, 2, 2, 4), (2, 2, 1, 3, 5), (1, 2, 2, 5, 7),
                                          (2, 1, 1, 6, 7)])
def test_assembly_matches_oracle_mixed(torch, ctx, nx, ny, nz, N, G):
    """Mixed fills: N <= 5 keep float-float through the basis change, N = 6 converts first."""
    mesh = W.make_mesh(nx, ny, nz, N, G, seed=3 + N)
    (vals,), row_ptr, col_idx, rc = gpu_assemble(torch, ctx, mesh, N, G, p2s.MIXED)
    assert rc == 0 and not np.isnan(vals).any()
    ref = oracle_global(mesh, N, G)
    assert np.abs(dense(row_ptr, col_idx, vals) - ref).max() <= 1e-8 * np.abs(ref).max()


def test_mixed_assembly_close_to_fp64(torch, ctx):
    mesh = W.make_mesh(4, 3, 3, 4, 12, seed=9)
    (a,), _, _, _ = gpu_assemble(torch, ctx, mesh, 4, 12, p2s.FP64)
    (b,), _, _, _ = gpu_assemble(torch, ctx, mesh, 4, 12, p2s.MIXED)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()


def test_assembly_deterministic_and_graph_replay(torch, ctx):
    mesh = W.make_mesh(3, 3, 2, 4, 6, seed=5)
    outs, _, _, rc = gpu_assemble(torch, ctx, mesh, 4, 6, p2s.MIXED, reps=3)
    assert rc == 0
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    outs_g, _, _, _ = gpu_assemble(torch, ctx, mesh, 4, 6, p2s.MIXED, reps=2, graph=True)
    assert all(np.array_equal(outs[0], o) for o in outs_g)


@pytest.mark.parametrize("prec", [p2s.FP64, p2s.MIXED])
def test_reassemble_equals_fill(torch, ctx, prec):
    mesh = W.make_mesh(2, 3, 2, 4, 6, seed=13)
    wl = mesh.workload
    T, S = W.diffusion_terms()
    asm = p2s.Assembly(ctx, 2, 3, 2, 4, 6, T, S, wl.kind, prec)
    dp, dn, db = (torch.as_tensor(np.ascontiguousarray(a), device="cuda") for a in (wl.params, wl.nodes, wl.bulge))
    a = torch.empty(asm.nnz, dtype=torch.float64, device="cuda")
    b = torch.full((asm.nnz,), 7.0, dtype=torch.float64, device="cuda")
    asm.fill(wl.kind, dp, dn, db, a)
    asm.reassemble(b)
    assert ctx.sync_status() == 0
    assert torch.equal(a, b)
    asm.close()


def oracle_row(mesh, N, G, r):
    """Row r of the global matrix from the oracle, built from the elements that hold dof r."""
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    gv, gw = A.global_size_1d(ny, N), A.global_size_1d(nz, N)
    Tk = np.kron(np.kron(A.hierarchic_transform(N), A.hierarchic_transform(N)), A.hierarchic_transform(N))
    wl = mesh.workload
    Tm, Sc = W.diffusion_terms()
    row = {}
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                g = [(A.global_dof_1d(nx, N, i, m) * gv + A.global_dof_1d(ny, N, j, n)) * gw
                     + A.global_dof_1d(nz, N, k, p) for m in range(N) for n in range(N) for p in range(N)]
                if r not in g:
                    continue
                e = (k * ny + j) * nx + i
                out, _, rc = oracle.fill_terms(wl.orders[e:e + 1], wl.kind, wl.params[e:e + 1], wl.nodes[e:e + 1],
                                               wl.bulge[e:e + 1], G, Tm, Sc, nthreads=1)
                assert rc == 0
                n = N ** 3
                Ml = Tk @ out.reshape(n, n) @ Tk.T
                a = g.index(r)
                for b, c in enumerate(g):
                    row[c] = row.get(c, 0.0) + Ml[a, b]
    return row


def test_assembly_larger_mesh_sampled_rows_and_properties(torch, ctx):
    nx, ny, nz, N, G = 10, 9, 8, 4, 6
    mesh = W.make_mesh(nx, ny, nz, N, G, seed=11)
    (vals,), row_ptr, col_idx, rc = gpu_assemble(torch, ctx, mesh, N, G, p2s.FP64)
    assert rc == 0 and not np.isnan(vals).any()
    rows = row_ptr.size - 1
    rng = np.random.default_rng(5)
    gu, gv, gw = (A.global_size_1d(x, N) for x in (nx, ny, nz))
    vertex = (4 * gv + 5) * gw + 3                      # interior vertex: 8 elements
    bubble = ((nx + 1 + 3) * gv + 2) * gw + nz + 1 + 4  # bubble x vertex x bubble
    for r in [0, vertex, bubble, rows - 1] + [int(x) for x in rng.integers(0, rows, 4)]:
        ref = oracle_row(mesh, N, G, r)
        cols = col_idx[row_ptr[r]:row_ptr[r + 1]]
        got = dict(zip(cols.tolist(), vals[row_ptr[r]:row_ptr[r + 1]].tolist()))
        assert set(got) == set(ref)
        scale = max(abs(v) for v in ref.values())
        assert max(abs(got[c] - ref[c]) for c in ref) <= 1e-12 * scale
    # symmetric, and the constant function (1 on every vertex dof) is in the null space
    rr = np.repeat(np.arange(rows), np.diff(row_ptr))
    key = rr.astype(np.int64) * rows + col_idx
    keyT = col_idx.astype(np.int64) * rows + rr
    order, orderT = np.argsort(key), np.argsort(keyT)
    scale = np.abs(vals).max()
    assert np.abs(vals[order] - vals[orderT]).max() <= 1e-13 * scale
    one = A.vertex_indicator(nx, ny, nz, N)
    Kone = np.bincount(rr, weights=vals * one[col_idx], minlength=rows)
    assert np.abs(Kone).max() <= 1e-11 * scale


def test_assembly_argument_errors(torch, ctx):
    T, S = W.diffusion_terms()
    for args in ((0, 1, 1, 4), (1, 1, 1, 1), (2, 2, 2, 13)):
        with pytest.raises(p2s.P2SError) as ex:
            p2s.Assembly(ctx, *args, 5, T, S, p2s.ALPHA_METRIC_EPS)
        assert ex.value.code in (p2s.ERR_ARG, p2s.ERR_ORDER)
    T2 = np.array(T).copy()
    T2[0, 0] = 1  # a second field component
    with pytest.raises(p2s.P2SError) as ex:
        p2s.Assembly(ctx, 2, 2, 2, 3, 4, T2, S, p2s.ALPHA_METRIC_EPS)
    assert ex.value.code == p2s.ERR_ARG


def test_assembly_add_of_oracle_element_matrices(torch, ctx):
    """p2s_assembly_add alone (transform + scatter) on the oracle's own element matrices, twice
    into the same values: 2 K to rounding, independent of the GPU fill."""
    for (nx, ny, nz, N, G) in ((3, 1, 2, 4, 5), (2, 2, 1, 6, 7)):
        mesh = W.make_mesh(nx, ny, nz, N, G, seed=19)
        wl = mesh.workload
        T, S = W.diffusion_terms()
        out, off, rc = oracle.fill_terms(wl.orders, wl.kind, wl.params, wl.nodes, wl.bulge, G, T, S)
        assert rc == 0
        asm = p2s.Assembly(ctx, nx, ny, nz, N, G, T, S, wl.kind, p2s.FP64)
        emat = torch.as_tensor(out, device="cuda")
        vals = torch.zeros(asm.nnz, dtype=torch.float64, device="cuda")
        asm.add(emat, vals)
        asm.add(emat, vals)
        assert ctx.sync_status() == 0
        assert torch.equal(emat.cpu(), torch.as_tensor(out))  # the input is left as it was
        row_ptr, col_idx = asm.structure()
        asm.close()
        ref = A.assemble(nx, ny, nz, N, out.reshape(wl.n_elem, N ** 3, N ** 3))
        K = dense(row_ptr, col_idx, vals.cpu().numpy())
        assert np.abs(K - 2 * ref).max() <= 1e-13 * np.abs(ref).max()
