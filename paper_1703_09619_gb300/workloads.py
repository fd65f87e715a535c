"""Seeded synthetic inputs for the element-matrix fill.

This module only draws random inputs (geometry nodes, bulge, material
parameters, per-axis orders, quadrature sizes).  It contains none of the
fill's arithmetic, so both the CUDA path and the CPU oracle can be fed from
it.  It imports nothing else from this package.

Workload recipes (all on the reference element [-1,1]^3, Eq. (2) of
arXiv:1703.09619; the paper's own tests are 2-D Chebyshev problems, so these
3-D Legendre batches are synthetic stand-ins with the shape of the method's
inputs):

* ``c1``  1 element, 1 component, N = 4 on every axis, scalar coupling factor
  alpha = 1 + 0.5 sin(pi u) cos(pi v) exp(w/2), 12-point rule.
* ``c2``  4096 curved hexahedra, 3 components, N = 6, metric coupling
  eps * detJ * J^-1 J^-T with eps = 1 + 0.5 sin(2 pi x.d), d one seeded unit
  vector for the batch; 16-point rule.
* ``c3``  512 elements, 1 component, N = 8, per-element scalar factor
  alpha_e = 1 + 0.5 sin(pi (u + phi_e)) cos(pi (v + psi_e)) exp(w/2),
  phi_e, psi_e ~ U[0,1); 24-point rule.
* ``c4``  8192 elements, 3 components, per-component per-axis orders drawn
  uniformly from {2..8}; eps = 1 + 0.5 sin(2 pi |k| x.d_e), |k| log-uniform
  in [1, 8]; 16-point rule.
* ``c5``  32768 elements, 3 components, N = 4, eps = 1 + 0.8 sin(k_e . x),
  |k_e| log-uniform in [1, 40]; quadrature chosen per element (learned) or
  48 points (plain).

Geometry of every curved element: the 8 corners of the physical unit cube
[0,1]^3 (node index iu + 2 iv + 4 iw) each moved by i.i.d. U(-0.15, 0.15)
per coordinate, plus a bulge a * b_e * cos(pi u/2) cos(pi v/2) cos(pi w/2)
with a = 0.1 and b_e a seeded unit vector (the bulge vanishes on the faces).
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED_BASE = 0x170309619

KIND_SCALAR = 0
KIND_METRIC_EPS = 1

TYPES_ALL = 0xF


@dataclasses.dataclass
class Workload:
    name: str
    n_elem: int
    n_comp: int
    orders: np.ndarray  # int32 [E, n_comp, 3]
    kind: int
    params: np.ndarray  # float64 [E, 4]
    nodes: np.ndarray  # float64 [E, 8, 3]
    bulge: np.ndarray  # float64 [E, 4]
    npts: np.ndarray  # int32 [E]
    types_mask: int = TYPES_ALL
    description: str = ""

    def subset(self, idx) -> "Workload":
        idx = np.asarray(idx, dtype=np.int64).reshape(-1)
        return dataclasses.replace(
            self,
            name="%s[%d]" % (self.name, idx.size),
            n_elem=int(idx.size),
            orders=np.ascontiguousarray(self.orders[idx]),
            params=np.ascontiguousarray(self.params[idx]),
            nodes=np.ascontiguousarray(self.nodes[idx]),
            bulge=np.ascontiguousarray(self.bulge[idx]),
            npts=np.ascontiguousarray(self.npts[idx]),
        )

    def with_npts(self, npts) -> "Workload":
        npts = np.broadcast_to(np.asarray(npts, dtype=np.int32), (self.n_elem,))
        return dataclasses.replace(self, npts=np.ascontiguousarray(npts))

    def ndof(self) -> np.ndarray:
        return np.prod(self.orders, axis=2).sum(axis=1).astype(np.int64)

    def entries(self) -> int:
        nt = bin(self.types_mask & 0xF).count("1")
        n = self.ndof()
        return int(nt * (n * n).sum())


def unit_vectors(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def cube_nodes(n):
    """Corners of [0,1]^3, node index iu + 2 iv + 4 iw."""
    c = np.array([[(i >> 0) & 1, (i >> 1) & 1, (i >> 2) & 1] for i in range(8)], dtype=np.float64)
    return np.broadcast_to(c, (n, 8, 3)).copy()


def curved_geometry(rng, n, jitter=0.15, bulge_amp=0.1):
    nodes = cube_nodes(n) + rng.uniform(-jitter, jitter, size=(n, 8, 3))
    b = unit_vectors(rng, n)
    bulge = np.concatenate([np.full((n, 1), bulge_amp), b], axis=1)
    return nodes, bulge


def _scalar_params(n, A, phi, psi, c):
    p = np.zeros((n, 4))
    p[:, 0] = A
    p[:, 1] = phi
    p[:, 2] = psi
    p[:, 3] = c
    return p


SHARD_SEED_STRIDE = 1000


def make(name: str, n_elem: int | None = None, shard: int = 0) -> Workload:
    """Build one of the named workloads (``c1`` .. ``c5``), optionally with fewer elements.

    Elements are always drawn for the full workload size and then truncated,
    so element e is the same whatever ``n_elem`` is.  ``shard`` s > 0 draws another
    batch of the same recipe from its own seed (the batch of rank s when every rank
    of a multi-GPU run fills a batch of its own); shard 0 is the canonical batch."""
    cid = {"c1": 1, "c2": 2, "c3": 3, "c4": 4, "c5": 5, "c5train": 50}[name]
    if shard < 0:
        raise ValueError("shard must be >= 0")
    rng = np.random.default_rng(SEED_BASE + cid + SHARD_SEED_STRIDE * shard)
    if cid == 50:  # training elements for the learned order: the c5 recipe, its own seed
        E = 65536
        nodes, bulge = curved_geometry(rng, E)
        kmag = np.exp(rng.uniform(np.log(1.0), np.log(40.0), E))
        d = unit_vectors(rng, E)
        params = np.zeros((E, 4))
        params[:, 0] = 0.8
        params[:, 1:] = kmag[:, None] * d
        orders = np.full((E, 3, 3), 4, dtype=np.int32)
        w = Workload(name, E, 3, orders, KIND_METRIC_EPS, params, nodes, bulge, np.full(E, 48, np.int32),
                     description="65536 training hexahedra, the c5 recipe with its own seed")
        if n_elem is not None and n_elem < w.n_elem:
            w = w.subset(np.arange(n_elem))
            w.name = name
        return w
    if cid == 1:
        E = 1
        orders = np.full((E, 1, 3), 4, dtype=np.int32)
        params = _scalar_params(E, 0.5, 0.0, 0.0, 0.5)
        nodes, bulge = cube_nodes(E), np.zeros((E, 4))
        w = Workload(name, E, 1, orders, KIND_SCALAR, params, nodes, bulge, np.full(E, 12, np.int32),
                     description="1 element, N=4, scalar alpha, G=12")
    elif cid == 2:
        E = 4096
        nodes, bulge = curved_geometry(rng, E)
        d = unit_vectors(rng, 1)[0]
        params = np.zeros((E, 4))
        params[:, 0] = 0.5
        params[:, 1:] = 2.0 * np.pi * d
        orders = np.full((E, 3, 3), 6, dtype=np.int32)
        w = Workload(name, E, 3, orders, KIND_METRIC_EPS, params, nodes, bulge, np.full(E, 16, np.int32),
                     description="4096 curved hexahedra, 3 comp, N=6, metric*eps, G=16")
    elif cid == 3:
        E = 512
        phi = rng.uniform(0.0, 1.0, E)
        psi = rng.uniform(0.0, 1.0, E)
        params = _scalar_params(E, 0.5, phi, psi, 0.5)
        orders = np.full((E, 1, 3), 8, dtype=np.int32)
        nodes, bulge = cube_nodes(E), np.zeros((E, 4))
        w = Workload(name, E, 1, orders, KIND_SCALAR, params, nodes, bulge, np.full(E, 24, np.int32),
                     description="512 elements, 1 comp, N=8, per-element scalar alpha, G=24")
    elif cid == 4:
        E = 8192
        nodes, bulge = curved_geometry(rng, E)
        kmag = np.exp(rng.uniform(np.log(1.0), np.log(8.0), E))
        d = unit_vectors(rng, E)
        params = np.zeros((E, 4))
        params[:, 0] = 0.5
        params[:, 1:] = 2.0 * np.pi * kmag[:, None] * d
        orders = rng.integers(2, 9, size=(E, 3, 3)).astype(np.int32)
        w = Workload(name, E, 3, orders, KIND_METRIC_EPS, params, nodes, bulge, np.full(E, 16, np.int32),
                     description="8192 curved hexahedra, 3 comp, orders U{2..8} per comp/axis, G=16")
    else:
        E = 32768
        nodes, bulge = curved_geometry(rng, E)
        kmag = np.exp(rng.uniform(np.log(1.0), np.log(40.0), E))
        d = unit_vectors(rng, E)
        params = np.zeros((E, 4))
        params[:, 0] = 0.8
        params[:, 1:] = kmag[:, None] * d
        orders = np.full((E, 3, 3), 4, dtype=np.int32)
        w = Workload(name, E, 3, orders, KIND_METRIC_EPS, params, nodes, bulge, np.full(E, 48, np.int32),
                     description="32768 curved hexahedra, 3 comp, N=4, eps=1+0.8 sin(k.x), |k| in [1,40]")
    if n_elem is not None and n_elem < w.n_elem:
        w = w.subset(np.arange(n_elem))
        w.name = name
    if shard:
        w.name = "%s/shard%d" % (w.name, shard)
    return w


@dataclasses.dataclass
class Mesh:
    """A conforming structured mesh of curved hexahedra: element (i, j, k) (index
    (k ny + j) nx + i) has the 8 lattice vertices around it, node index iu + 2 iv + 4 iw."""
    nx: int
    ny: int
    nz: int
    vertices: np.ndarray  # float64 [(nz+1)(ny+1)(nx+1), 3], vertex (i, j, k) at ((k (ny+1) + j)(nx+1) + i)
    workload: Workload    # the elements (nodes from the shared vertices), one scalar field component


def make_mesh(nx: int, ny: int, nz: int, order: int, npts: int, seed: int = 7, jitter: float = 0.15,
              bulge_amp: float = 0.1, eps_amp: float = 0.5, kmag: float = 2.0) -> Mesh:
    """Seeded conforming mesh: lattice vertices (i, j, k) moved by i.i.d. U(-jitter, jitter) per
    coordinate (shared by the elements around them), a per-element bulge that vanishes on the
    faces, one material eps = 1 + eps_amp sin(k . x) for the whole mesh (|k| = kmag); one scalar
    field with `order` per axis and `npts` Gauss-Legendre points."""
    rng = np.random.default_rng(SEED_BASE + 60 + SHARD_SEED_STRIDE * seed)
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    lattice = np.stack([ii, jj, kk], axis=-1).astype(np.float64)          # [nx+1][ny+1][nz+1][3]
    verts = lattice.transpose(2, 1, 0, 3).reshape(-1, 3).copy()          # ((k (ny+1) + j)(nx+1) + i)
    verts += rng.uniform(-jitter, jitter, size=verts.shape)
    E = nx * ny * nz
    nodes = np.zeros((E, 8, 3))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                e = (k * ny + j) * nx + i
                for nd in range(8):
                    a, b, c = nd & 1, (nd >> 1) & 1, (nd >> 2) & 1
                    nodes[e, nd] = verts[((k + c) * (ny + 1) + (j + b)) * (nx + 1) + (i + a)]
    bulge = np.concatenate([np.full((E, 1), bulge_amp), unit_vectors(rng, E)], axis=1)
    d = unit_vectors(rng, 1)[0]
    params = np.zeros((E, 4))
    params[:, 0] = eps_amp
    params[:, 1:] = kmag * d
    orders = np.full((E, 1, 3), order, dtype=np.int32)
    w = Workload("mesh%dx%dx%d" % (nx, ny, nz), E, 1, orders, KIND_METRIC_EPS, params, nodes, bulge,
                 np.full(E, npts, np.int32),
                 description="%dx%dx%d conforming curved hexahedra, 1 scalar field, N=%d, G=%d" % (nx, ny, nz, order, npts))
    return Mesh(nx, ny, nz, verts, w)


def diffusion_terms(component: int = 0, scale: float = 1.0):
    """Term list of the diffusion stiffness sum_ab alpha_ab d_a(test) d_b(trial) on one
    field component, with alpha the metric coupling factor eps detJ J^-1 J^-T: nine
    terms (a, b), derivative on axis a of the test and on axis b of the trial function.
    Rows (gi, gj, sa, sb, du, dv, dw, eu, ev, ew) and scales; input data only."""
    terms, scales = [], []
    for a in range(3):
        for b in range(3):
            d = [0, 0, 0]
            f = [0, 0, 0]
            d[a] = 1
            f[b] = 1
            terms.append([component, component, a, b] + d + f)
            scales.append(scale)
    return np.array(terms, dtype=np.int32), np.array(scales, dtype=np.float64)


def judge_elements(n_elem: int, frac: float, seed: int) -> np.ndarray:
    """Seeded, sorted sample of element indices re-filled by the full-order judge."""
    k = int(np.ceil(frac * n_elem)) if frac > 0 else 0
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_elem, size=min(k, n_elem), replace=False)).astype(np.int32)


# ----------------------------------------------------------------------------- 2-D curl-curl example
@dataclasses.dataclass
class Mesh2D:
    """Structured mesh of the curved quadrilateral domain of the paper's Sec. III example: the image
    of [-1,1]^2 under X(s, t) = (s g(t), t f(s)) with f(x) = 1 - 0.2 (x^2-1)^2 and g(y) = 1 + 0.2
    (y^2-1)^2, so the boundary is x = +-g(y), y = +-f(x).  Element (i, j) (index j nx + i) is the
    image of the cell [s_i, s_i+1] x [t_j, t_j+1] of a uniform nx x ny grid; params[e] = (s_lo, s_hi,
    t_lo, t_hi, filled): the material eps_r = 2 exp(x + y + 2) fills the lower half (t < 0), eps_r = 1
    elsewhere, mu_r = 1.  M = N = order; G Gauss-Legendre points per axis."""
    nx: int
    ny: int
    order: int
    npts: int
    params: np.ndarray  # float64 [E][5]

    @property
    def n_elem(self):
        return self.nx * self.ny


def make_mesh2d(nx: int, ny: int, order: int, npts: int) -> Mesh2D:
    if ny % 2:
        raise ValueError("ny must be even (the material interface t = 0 lies on element edges)")
    s = np.linspace(-1.0, 1.0, nx + 1)
    t = np.linspace(-1.0, 1.0, ny + 1)
    params = np.zeros((nx * ny, 5))
    for j in range(ny):
        for i in range(nx):
            e = j * nx + i
            params[e] = (s[i], s[i + 1], t[j], t[j + 1], 1.0 if t[j + 1] <= 0.0 else 0.0)
    return Mesh2D(nx, ny, order, npts, params)


def cheb2d_npts(order: int) -> int:
    """Quadrature points per axis for the 2-D example: 1.5 M + 2 (the paper assumes about 2 D =
    2 M N points per element for the direct integration, i.e. sqrt(2) M per axis)."""
    return (3 * order + 1) // 2 + 2
