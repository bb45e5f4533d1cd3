"""Finite-difference building blocks (oracle; test infrastructure only).

Follows Appendix A of the paper literally:
* Theorem A.1: 1D Dirichlet, T = h^-2 tridiag(-1, 2, -1) on the interior
  nodes x_1..x_q.
* Theorem A.2: 1D absorbing, unknowns x_0..x_{q+1}; T has 1/h^2 in both
  corners; D_1 = h^-1 diag(k_0, 0, ..., 0, k_{q+1});
  D_2 = diag(k_0^2/2, k_1^2, ..., k_{q+1}^2/2); F_0 = [f_0/2, f_1, ...,
  f_{q+1}/2].  The one-sided closure row is derived in App. A.1 from a
  Taylor expansion at the end point.
* Theorem A.5: 2D Dirichlet, L = I (x) T + T (x) I on the q x q interior.
* Theorem A.6: 2D absorbing, (q+2)^2 nodes ordered x fastest,
  L = D (x) T + T (x) D with D = diag(1/2, 1, ..., 1, 1/2); D_1 = h^-1 times
  the node value on every boundary node (corners included, once);
  D_2 = diag(d_i d_j k_ij^2); b_0 = d_i d_j f_ij.
* App. A.3: a point source delta(x - a) becomes 1/h^d at the grid node
  t = ceil(q/2) (per axis).
* Sec. 6: mesh rule lev = max(ceil(log2(15 maxk / (2 pi))), 1), q = 2^lev - 1.

One reading beyond the paper (the paper treats both ends alike): a 1D
problem may be Dirichlet at one end and absorbing at the other.  Each end
then takes its own row from Theorem A.1 or Theorem A.2 respectively.

Pins: tests/test_oracle_fd.py (consistency with the 1D closed-form solution
at O(h^2), symmetric positive semidefiniteness and the kernel of T stated in
Theorem A.2, and the nnz column of Table 2 via tests/test_oracle_sg.py).
"""
from __future__ import annotations

from dataclasses import dataclass
from math import ceil, log2, pi

import numpy as np
import scipy.sparse as sp

DIRICHLET = 0
ABSORBING = 1


def mesh_rule(maxk: float) -> int:
    """q from the mesh rule of Sec. 6 (h = 1/(q+1))."""
    lev = max(ceil(log2((15.0 * maxk) / (2.0 * pi))), 1)
    return 2 ** lev - 1


def point_source_index(q: int) -> int:
    """t = ceil(q/2) = floor((q+1)/2), App. A.3."""
    return (q + 1) // 2


def nearest_node(a: float, h: float, nnodes: int) -> int:
    """Index j of the grid point x_j = j h closest to a; of two equally close
    points the smaller one (App. A.3: for a = 1/2 on x_0..x_{q+1} this is
    t = ceil(q/2)).  The 1e-9 guard keeps exact ties from being split by the
    rounding of a / h."""
    j = ceil(a / h - 0.5 - 1e-9)
    return min(max(j, 0), nnodes - 1)


def point_source(dim: int, nx: int, ny: int, h: float, point) -> np.ndarray:
    """Node values of a unit point source f = delta(x - a) (App. A.3): 1/h in
    1D, 1/h^2 in 2D at the grid point closest to a, zero elsewhere; nodes
    x fastest, boundary nodes included."""
    f = np.zeros(nx * ny)
    tx = nearest_node(point[0], h, nx)
    ty = nearest_node(point[1], h, ny) if dim == 2 else 0
    f[tx + nx * ty] = 1.0 / h ** dim
    return f


@dataclass
class Axis:
    """One grid direction: nodes x_0..x_{q+1}, the unknown nodes among them,
    the 1D matrix T on the unknowns (Theorems A.1/A.2), the end-weight vector
    d (1/2 on an absorbing end, else 1) and the absorbing-end indicator e."""

    nodes: np.ndarray      # indices (into 0..q+1) of the unknown nodes
    T: sp.csr_matrix       # h^-2 * tridiagonal, on the unknowns
    d: np.ndarray          # D weights on the unknowns
    e: np.ndarray          # 1 on absorbing end nodes, 0 elsewhere


def axis_1d(nnodes: int, h: float, left: int, right: int) -> Axis:
    """1D matrix T for a grid of `nnodes` = q+2 nodes with the given end
    conditions.  Interior rows: (-u_{j-1} + 2u_j - u_{j+1}) / h^2.  A
    Dirichlet end drops its node (u = 0), leaving the 2 on the first interior
    row (Theorem A.1).  An absorbing end keeps its node with the row
    (u_0 - u_1)/h^2 (Theorem A.2)."""
    lo = 0 if left == ABSORBING else 1
    hi = nnodes - 1 if right == ABSORBING else nnodes - 2
    nodes = np.arange(lo, hi + 1)
    n = len(nodes)
    main = np.full(n, 2.0)
    if left == ABSORBING:
        main[0] = 1.0
    if right == ABSORBING:
        main[-1] = 1.0
    off = np.full(n - 1, -1.0)
    T = sp.diags([off, main, off], [-1, 0, 1], shape=(n, n), format="csr") / (h * h)
    d = np.ones(n)
    e = np.zeros(n)
    if left == ABSORBING:
        d[0] = 0.5
        e[0] = 1.0
    if right == ABSORBING:
        d[-1] = 0.5
        e[-1] = 1.0
    return Axis(nodes=nodes, T=T.tocsr(), d=d, e=e)


@dataclass
class Grid:
    """Spatial discretisation: the unknown-node index list (into the full
    node array, x fastest), the FD Laplacian L on the unknowns, the node
    weights w2 (diagonal of D_2 / k^2) and w1 (diagonal of D_1 / k, which
    already includes the 1/h factor)."""

    dim: int
    nx: int
    ny: int
    h: float
    unknowns: np.ndarray
    L: sp.csr_matrix
    w1: np.ndarray
    w2: np.ndarray


def make_grid(dim: int, nx: int, ny: int, h: float, bc) -> Grid:
    """bc = (left, right, bottom, top), each DIRICHLET or ABSORBING.

    dim 1: Theorem A.1 / A.2 (ends may differ).
    dim 2: Theorem A.5 (all Dirichlet) or Theorem A.6 (all absorbing)."""
    if dim == 1:
        ax = axis_1d(nx, h, bc[0], bc[1])
        return Grid(1, nx, 1, h, ax.nodes.copy(), ax.T, ax.e / h, ax.d.copy())
    if dim != 2:
        raise ValueError("dim must be 1 or 2")
    if all(b == ABSORBING for b in bc):
        axx = axis_1d(nx, h, ABSORBING, ABSORBING)
        axy = axis_1d(ny, h, ABSORBING, ABSORBING)
        Dx = sp.diags(axx.d)
        Dy = sp.diags(axy.d)
        # x fastest: kron(Y-operator, X-operator)   (Theorem A.6: D (x) T + T (x) D)
        L = (sp.kron(Dy, axx.T) + sp.kron(axy.T, Dx)).tocsr()
        w2 = np.kron(axy.d, axx.d)
        bnd = np.zeros((ny, nx))
        bnd[0, :] = bnd[-1, :] = 1.0
        bnd[:, 0] = bnd[:, -1] = 1.0
        w1 = bnd.reshape(-1) / h
        jj, ii = np.meshgrid(axy.nodes, axx.nodes, indexing="ij")
        unk = (ii + nx * jj).reshape(-1)
        return Grid(2, nx, ny, h, unk, L, w1, w2)
    if all(b == DIRICHLET for b in bc):
        axx = axis_1d(nx, h, DIRICHLET, DIRICHLET)
        axy = axis_1d(ny, h, DIRICHLET, DIRICHLET)
        Ix = sp.identity(len(axx.nodes))
        Iy = sp.identity(len(axy.nodes))
        L = (sp.kron(Iy, axx.T) + sp.kron(axy.T, Ix)).tocsr()   # Theorem A.5
        n = L.shape[0]
        jj, ii = np.meshgrid(axy.nodes, axx.nodes, indexing="ij")
        unk = (ii + nx * jj).reshape(-1)
        return Grid(2, nx, ny, h, unk, L, np.zeros(n), np.ones(n))
    raise ValueError("2D grids are all-Dirichlet or all-absorbing (Theorems A.5/A.6)")


def rhs_block(grid: Grid, f_nodes: np.ndarray) -> np.ndarray:
    """b_0 = D_2-weights * f on the unknowns (F_0 of Theorem A.2, b_0 of
    Theorem A.6; weight 1 in the Dirichlet theorems)."""
    return grid.w2 * np.asarray(f_nodes, dtype=float).reshape(-1)[grid.unknowns]


def deterministic_matrix(grid: Grid, k_nodes: np.ndarray) -> sp.csr_matrix:
    """S = L - i D_1(k) - D_2(k^2) for one realisation k of the wavenumber on
    the nodes (Theorems A.1, A.2, A.5, A.6)."""
    k = np.asarray(k_nodes, dtype=float).reshape(-1)[grid.unknowns]
    return (grid.L - 1j * sp.diags(grid.w1 * k) - sp.diags(grid.w2 * k * k)).tocsr()
