"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module builds problem *inputs* only: sparse matrices in CSR form and
right-hand sides.  It contains none of the Krylov method's arithmetic, so both
the CPU oracle and the CUDA path can consume the same bytes without sharing any
part of the method.

Matrices stand in for the PDE/FEM operators of the paper's experiments
(Sec. 5.1 convection-diffusion, Sec. 5.2 membrane): the paper's own meshes are
not available, so structured-grid operators of the same shape class (5 to 15
nonzeros per row, n of 10^4 to 10^7, non-symmetric convection) are generated.

Conventions
-----------
* Grids are interior grids of the unit square/cube with Dirichlet nodes
  eliminated, spacing h = 1/(N+1), lexicographic ordering with x fastest.
* Convection uses first-order upwinding: for a velocity component beta_d > 0
  the lower neighbour in direction d carries -1/h^2 - beta_d/h, the upper one
  -1/h^2, and the diagonal 2*dim/h^2 + sum_d |beta_d|/h.
* CSR arrays: int32 row_ptr (n+1), int32 col_idx (sorted within a row),
  float64 values.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Csr",
    "stencil_matrix",
    "poisson2d",
    "convdiff3d",
    "fem_p1_kuhn",
    "rhs_normal",
    "rhs_uniform",
    "sine_mode_mixture_2d",
    "batched_instances",
    "rmat_laplacian",
    "rhs_probability",
    "CONFIGS",
]


@dataclass(frozen=True)
class Csr:
    """Square sparse matrix in compressed-sparse-row form."""

    n: int
    row_ptr: np.ndarray  # int32, n+1
    col_idx: np.ndarray  # int32, nnz
    val: np.ndarray  # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def transpose(self) -> "Csr":
        """CSR of the transposed matrix (host-side helper for test inputs)."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))
        order = np.lexsort((rows, self.col_idx))
        counts = np.bincount(self.col_idx, minlength=self.n)
        rp = np.zeros(self.n + 1, dtype=np.int64)
        np.cumsum(counts, out=rp[1:])
        return Csr(self.n, rp.astype(np.int32), rows[order].astype(np.int32),
                   self.val[order].copy())

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        np.add.at(d, (rows, self.col_idx), self.val)
        return d


def _grid_index(shape):
    """Linear index of every grid point, x fastest (shape given as (Nz, Ny, Nx))."""
    return np.arange(int(np.prod(shape)), dtype=np.int64).reshape(shape)


def stencil_matrix(shape, offsets, coeffs) -> Csr:
    """Assemble a CSR matrix from a constant-coefficient grid stencil.

    shape   : grid extent per axis, slowest first (e.g. (Nz, Ny, Nx)).
    offsets : list of integer offset tuples (same axis order as ``shape``).
    coeffs  : matching list of coefficients.
    Neighbours outside the grid are dropped (homogeneous Dirichlet).
    Entries of a row are emitted in increasing column order.
    """
    shape = tuple(int(s) for s in shape)
    dim = len(shape)
    n = int(np.prod(shape))
    strides = [int(np.prod(shape[a + 1:])) for a in range(dim)]
    lin = [sum(o[a] * strides[a] for a in range(dim)) for o in offsets]
    order = np.argsort(lin, kind="stable")
    offsets = [offsets[i] for i in order]
    coeffs = [coeffs[i] for i in order]
    lin = [lin[i] for i in order]

    coords = np.indices(shape).reshape(dim, -1)
    cols = np.empty((n, len(offsets)), dtype=np.int64)
    vals = np.empty((n, len(offsets)), dtype=np.float64)
    mask = np.empty((n, len(offsets)), dtype=bool)
    base = np.arange(n, dtype=np.int64)
    for q, (o, c) in enumerate(zip(offsets, coeffs)):
        ok = np.ones(n, dtype=bool)
        for a in range(dim):
            ca = coords[a] + o[a]
            ok &= (ca >= 0) & (ca < shape[a])
        mask[:, q] = ok
        cols[:, q] = base + lin[q]
        vals[:, q] = c
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col_idx = cols[mask].astype(np.int32)
    val = vals[mask]
    return Csr(n, row_ptr.astype(np.int32), col_idx, val)


def poisson2d(N: int) -> Csr:
    """5-point -Laplacian on an N x N interior grid, h = 1/(N+1)."""
    return convdiff(N, dim=2, beta=(0.0, 0.0))


def convdiff(N: int, dim: int, beta) -> Csr:
    """Upwind convection-diffusion -Lap u + beta . grad u on an N^dim interior grid."""
    inv_h = float(N + 1)  # 1/h, exact
    inv_h2 = inv_h * inv_h
    beta = [float(b) for b in beta]
    assert len(beta) == dim
    # beta is given in (x, y, z) order; grid axes are slowest first.
    offsets, coeffs = [], []
    diag = 2.0 * dim * inv_h2 + sum(abs(b) for b in beta) * inv_h
    offsets.append((0,) * dim)
    coeffs.append(diag)
    for d in range(dim):
        axis = dim - 1 - d  # x is the fastest (last) axis
        lo = -inv_h2
        hi = -inv_h2
        if beta[d] >= 0:
            lo -= beta[d] * inv_h
        else:
            hi -= -beta[d] * inv_h
        o_lo = [0] * dim
        o_lo[axis] = -1
        o_hi = [0] * dim
        o_hi[axis] = 1
        offsets += [tuple(o_lo), tuple(o_hi)]
        coeffs += [lo, hi]
    return stencil_matrix((N,) * dim, offsets, coeffs)


def convdiff3d(N: int, beta=(50.0, 50.0, 50.0)) -> Csr:
    """7-point upwind convection-diffusion on an N^3 interior grid."""
    return convdiff(N, dim=3, beta=beta)


def fem_p1_kuhn(cells: int, sigma: float, seed: int) -> Csr:
    """P1 stiffness matrix of -div(kappa grad u) on the unit cube.

    The cube is cut into cells^3 cubes of side h = 1/cells, each split into the
    six Kuhn tetrahedra that share the main diagonal (0,0,0)-(1,1,1).  kappa is
    constant per cube, kappa = exp(sigma * g) with g ~ N(0,1) i.i.d. from
    ``seed`` and shared by the cube's six tetrahedra.  Dirichlet boundary nodes
    are eliminated, leaving (cells-1)^3 unknowns; interior rows couple along
    the seven edge directions e_x, e_y, e_z, e_x+e_y, e_x+e_z, e_y+e_z,
    e_x+e_y+e_z (15 entries per interior row).
    """
    import itertools

    h = 1.0 / cells
    rng = np.random.default_rng(seed)
    kappa = np.exp(sigma * rng.standard_normal((cells, cells, cells)))  # (z, y, x)

    # Element stiffness of the unit cube split into its six Kuhn tetrahedra.
    corners = np.array(list(itertools.product((0, 1), repeat=3)))[:, ::-1]  # (x,y,z), x fastest
    corner_id = {tuple(c): i for i, c in enumerate(corners)}
    kcube = np.zeros((8, 8))
    for perm in itertools.permutations(range(3)):
        path = [np.zeros(3, dtype=int)]
        for ax in perm:
            nxt = path[-1].copy()
            nxt[ax] = 1
            path.append(nxt)
        verts = np.array(path, dtype=float)
        M = np.hstack([np.ones((4, 1)), verts])
        grads = np.linalg.inv(M)[1:, :].T  # gradient of each barycentric fn, unit cell
        vol = abs(np.linalg.det(M)) / 6.0
        ke = vol * grads @ grads.T  # for side h: multiply by h^3 / h^2 = h
        ids = [corner_id[tuple(v.astype(int))] for v in verts]
        for a in range(4):
            for b in range(4):
                kcube[ids[a], ids[b]] += ke[a, b]
    kcube *= h

    # Round-off of the inverse above leaves ~1e-17 where the exact entry is 0
    # (couplings across face and body diagonals: their gradients are orthogonal).
    kcube[np.abs(kcube) < 1e-12 * np.abs(kcube).max()] = 0.0

    # The sparsity pattern is structural: every pair of nodes joined by an edge
    # of some tetrahedron (offsets with all components in {0, 1} or all in
    # {0, -1}: 7 directions, both signs, plus the diagonal) is stored, also
    # where the stiffness entry is exactly zero.
    Nn = cells + 1
    diag_arrays = {}
    for a in range(8):
        ca = corners[a]
        for b in range(8):
            cb = corners[b]
            d = cb - ca
            if not (np.all(d >= 0) or np.all(d <= 0)):
                continue
            off = tuple(int(x) for x in d)  # (dx, dy, dz)
            arr = diag_arrays.setdefault(off, np.zeros((Nn, Nn, Nn)))
            # node of corner a in cell (k, j, i) is (k+az, j+ay, i+ax)
            arr[ca[2]:ca[2] + cells, ca[1]:ca[1] + cells, ca[0]:ca[0] + cells] += kappa * kcube[a, b]
    # Interior nodes only.
    N = cells - 1
    offsets, coeff_arrays = [], []
    for (dx, dy, dz), arr in diag_arrays.items():
        offsets.append((dz, dy, dx))
        coeff_arrays.append(arr[1:cells, 1:cells, 1:cells].reshape(-1))
    return _stencil_matrix_varcoef((N, N, N), offsets, coeff_arrays)


def _stencil_matrix_varcoef(shape, offsets, coeff_arrays) -> Csr:
    dim = len(shape)
    n = int(np.prod(shape))
    strides = [int(np.prod(shape[a + 1:])) for a in range(dim)]
    lin = [sum(o[a] * strides[a] for a in range(dim)) for o in offsets]
    order = np.argsort(lin, kind="stable")
    coords = np.indices(shape).reshape(dim, -1)
    base = np.arange(n, dtype=np.int64)
    cols = np.empty((n, len(offsets)), dtype=np.int64)
    vals = np.empty((n, len(offsets)), dtype=np.float64)
    mask = np.empty((n, len(offsets)), dtype=bool)
    for q, i in enumerate(order):
        o = offsets[i]
        ok = np.ones(n, dtype=bool)
        for a in range(dim):
            ca = coords[a] + o[a]
            ok &= (ca >= 0) & (ca < shape[a])
        mask[:, q] = ok
        cols[:, q] = base + lin[i]
        vals[:, q] = coeff_arrays[i]
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Csr(n, row_ptr.astype(np.int32), cols[mask].astype(np.int32), vals[mask])


def rhs_normal(n: int, seed: int, normalize: bool = False) -> np.ndarray:
    """b ~ N(0, 1) i.i.d. (numpy PCG64 stream of ``seed``)."""
    b = np.random.default_rng(seed).standard_normal(n)
    if normalize:
        b /= np.linalg.norm(b)
    return b


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """b ~ U[0, 1) i.i.d. (numpy PCG64 stream of ``seed``)."""
    return np.random.default_rng(seed).random(n)


def sine_mode_mixture_2d(N: int, n_modes: int, seed: int):
    """b = sum_l c_l phi_{p_l q_l} of discrete sine modes on an N x N grid.

    phi_{pq}(i, j) = sin(p pi (i+1) h) sin(q pi (j+1) h) with h = 1/(N+1) are
    eigenvectors of the 5-point Laplacian.  Returns (b, c, p, q) so that a test
    can form the closed-form exp(-tA) b without any Krylov code.
    """
    rng = np.random.default_rng(seed)
    pairs = set()
    while len(pairs) < n_modes:
        pairs.add((int(rng.integers(1, N + 1)), int(rng.integers(1, N + 1))))
    pairs = sorted(pairs)
    p = np.array([a for a, _ in pairs])
    q = np.array([b for _, b in pairs])
    c = rng.standard_normal(n_modes)
    h = 1.0 / (N + 1)
    ii = np.arange(1, N + 1)
    b = np.zeros((N, N))  # (y, x)
    for cl, pl, ql in zip(c, p, q):
        b += cl * np.outer(np.sin(ql * np.pi * ii * h), np.sin(pl * np.pi * ii * h))
    return b.reshape(-1), c, p, q


def batched_instances(count: int, seed: int, n_lo: float = 1e4, n_hi: float = 1e6):
    """Uneven batch of matrices for the batched form (2D Laplacians, 3D conv-diff).

    The type is chosen 50/50, the target size is log-uniform in [n_lo, n_hi]
    and rounded to N^2 or N^3, t is log-uniform in [1e-4, 1e-1].
    Returns a list of dicts {kind, N, n, t, beta}.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        kind = "2d" if rng.random() < 0.5 else "3d"
        n_target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        t = math.exp(rng.uniform(math.log(1e-4), math.log(1e-1)))
        if kind == "2d":
            N = max(2, int(round(n_target ** 0.5)))
            out.append(dict(kind=kind, N=N, n=N * N, t=t, beta=(0.0, 0.0)))
        else:
            N = max(2, int(round(n_target ** (1.0 / 3.0))))
            out.append(dict(kind=kind, N=N, n=N ** 3, t=t, beta=(50.0, 50.0, 50.0)))
    return out


def batched_matrix(inst) -> Csr:
    if inst["kind"] == "2d":
        return poisson2d(inst["N"])
    return convdiff3d(inst["N"], inst["beta"])


# The five workloads (inputs only).  Seeds are fixed so every consumer reads the
# same bytes.
SEED = 20250331
def rmat_laplacian(scale: int, edge_factor: int, seed: int, abc=(0.57, 0.19, 0.19), directed=False) -> Csr:
    """Out-degree Laplacian of an R-MAT graph (the Graph500 Kronecker
    generator's recursive quadrant choice; a stand-in for the paper's graph
    networks, Sec. 5): L[i, i] = out-degree of i, L[i, j] = -1 per edge i -> j,
    2^scale nodes, edge_factor 2^scale drawn edges before self loops and
    duplicates are dropped; undirected (the default) symmetrizes the edge set.
    Every row stores its diagonal (0 for a node without out-edges).  Power-law
    degrees: undirected at scale 20 the largest row has ~65,000 entries and rows
    longer than 256 entries hold ~60 % of them.
    """
    n = 1 << scale
    m = edge_factor * n
    a, b, c = abc
    rng = np.random.default_rng(seed)
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    for lvl in range(scale):  # one bit of both endpoints per level
        r = rng.random(m, dtype=np.float32)
        src |= (r >= a + b).astype(np.int64) << lvl
        dst |= (((r >= a) & (r < a + b)) | (r >= a + b + c)).astype(np.int64) << lvl
    keep = src != dst
    if directed:
        key = src[keep] * n + dst[keep]
    else:
        key = np.concatenate([src[keep] * n + dst[keep], dst[keep] * n + src[keep]])
    key.sort()
    first = np.ones(key.size, dtype=bool)
    first[1:] = key[1:] != key[:-1]
    key = key[first]
    rows = key // n
    cols = key % n
    deg = np.bincount(rows, minlength=n)
    # insert the diagonal of every row at its sorted position
    diag_key = np.arange(n, dtype=np.int64) * n + np.arange(n, dtype=np.int64)
    allk = np.concatenate([key, diag_key])
    order = np.argsort(allk, kind="stable")
    allk = allk[order]
    vals = np.concatenate([-np.ones(key.size), deg.astype(np.float64)])[order]
    rows = allk // n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(rows, minlength=n))
    return Csr(n, row_ptr.astype(np.int32), (allk % n).astype(np.int32), vals)


def rhs_probability(n: int, seed: int) -> np.ndarray:
    """x_0 = y / ||y||_1 with y ~ U(0, 1) i.i.d. (the paper's initial
    distribution on a graph, Sec. 5)."""
    y = np.random.default_rng(seed).random(n)
    return y / y.sum()


CONFIGS = {
    "poisson2d_64": dict(matrix=lambda: poisson2d(64), t=1e-3, m=30, k=2, s=60, zeta=8,
                         rhs=lambda n: rhs_normal(n, SEED, normalize=True), tol=1e-10),
    "convdiff3d_128": dict(matrix=lambda: convdiff3d(128, (50.0, 50.0, 50.0)), t=1e-2, m=40,
                           k=2, s=160, zeta=8, rhs=lambda n: rhs_uniform(n, SEED), tol=1e-8),
    "fem_kuhn_160": dict(matrix=lambda: fem_p1_kuhn(160, 1.0, SEED), t=None, m=50, k=4,
                         s=200, zeta=8, rhs=lambda n: rhs_normal(n, SEED), tol=1e-8),
    "convdiff3d_96_adjoint": dict(matrix=lambda: convdiff3d(96, (20.0, 0.0, 0.0)), t=5e-3,
                                  m=40, k=2, s=160, zeta=8,
                                  rhs=lambda n: rhs_normal(n, SEED), tol=1e-8),
}
