"""Explicit stochastic Galerkin system (oracle; test infrastructure only).

The SG matrix is assembled as the paper writes it: a Kronecker sum

    A = I_P (x) L  -  i [B_ij]  -  [C_ij]                 (Theorem 3.4)
    B_ij = <D_1(xi) phi_i, phi_j>,  C_ij = <D_2(xi) phi_i, phi_j>
                                                    (Theorems A.2, A.6)

with the random wavenumber k(x, xi) = k_0(x) + sum_l xi_l k_l(x) (Sec. 2.2).
Because D_1 is linear and D_2 quadratic in k, with the moments of
oracle.pc:

    [B_ij] = I (x) diag(w1 k_0) + sum_l G_l (x) diag(w1 k_l)
    [C_ij] = I (x) diag(w2 k_0^2) + sum_l G_l (x) diag(2 w2 k_0 k_l)
             + sum_{l <= l'} G_{l,l'} (x) diag(c_{l l'} w2 k_l k_l'),
             c = 1 if l = l' else 2.

Unknowns are ordered V = [V_0; ...; V_{P-1}] (Sec. 3.1), each V_i over the
grid unknowns with x fastest (Theorems A.5/A.6).  b = e_0 (x) b_0.

Also defined here:
* S(xi) for one realisation (Sec. 3.1), for quadrature pins;
* the mean-value block S(xi_bar) with xi_bar = 0 for uniform variables
  (Sec. 5; Remark 6.1: A_0 = I (x) S(0));
* the CSL matrix M(beta) = A - i beta K with K = [C_ij] (Sec. 4) and its
  mean-value form M_0 = I (x) (S(0) - i beta D_2(k_0^2)) (Sec. 6.3).

Pins: tests/test_oracle_sg.py (size and nnz of Table 2 for r = 0..8,
complex symmetry A^T = A and the semidefiniteness statements of Theorem 3.4,
the theta = 0 collapse of Remark 6.1, the spectrum inclusion of Theorem 4.1,
the condition numbers printed in Sec. 6.2 and 6.3, the inf-norm ordering of
Sec. 6.3, SG mean against quadrature of deterministic solves);
tests/test_oracle_galerkin_quadrature.py (every Galerkin block against the
Gauss-Legendre mean of phi_i phi_j S(xi) built one realisation at a time,
the Frobenius bound of Theorem 5.1 and the O(theta) rate of Theorem 5.2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import fd, pc


@dataclass
class SGSystem:
    grid: fd.Grid
    s: int
    r: int
    P: int
    A: sp.csr_matrix          # full SG matrix
    Lbig: sp.csr_matrix       # I (x) L
    Bbig: sp.csr_matrix       # [B_ij]
    Cbig: sp.csr_matrix       # [C_ij] (= K of Sec. 4)
    b: np.ndarray             # e_0 (x) b_0
    S0: sp.csr_matrix         # S(xi_bar) on the grid unknowns
    K0: sp.csr_matrix         # D_2(k_0^2): the k^2 part of S(xi_bar)


def assemble(dim, nx, ny, h, bc, s, r, k0, kl, f) -> SGSystem:
    """Assemble the explicit SG system.

    k0: node values of k_0 (nx*ny, x fastest); kl: (s, nx*ny) node values of
    k_1..k_s; f: node values of the source."""
    grid = fd.make_grid(dim, nx, ny, h, bc)
    P = pc.num_modes(s, r)
    unk = grid.unknowns
    k0u = np.asarray(k0, dtype=float).reshape(-1)[unk]
    klu = np.asarray(kl, dtype=float).reshape(s, -1)[:, unk] if s > 0 else np.zeros((0, len(unk)))
    G1, G2 = pc.expectation_matrices(s, r)
    I = sp.identity(P, format="csr")
    w1, w2 = grid.w1, grid.w2

    Lbig = sp.kron(I, grid.L, format="csr")
    B = sp.kron(I, sp.diags(w1 * k0u), format="csr")
    C = sp.kron(I, sp.diags(w2 * k0u * k0u), format="csr")
    for l in range(s):
        Gl = sp.csr_matrix(G1[l])
        B = B + sp.kron(Gl, sp.diags(w1 * klu[l]), format="csr")
        C = C + sp.kron(Gl, sp.diags(2.0 * w2 * k0u * klu[l]), format="csr")
    for (l, lp), G in G2.items():
        c = 1.0 if l == lp else 2.0
        C = C + sp.kron(sp.csr_matrix(G), sp.diags(c * w2 * klu[l] * klu[lp]), format="csr")
    A = (Lbig - 1j * B - C).tocsr()
    A.eliminate_zeros()
    b0 = fd.rhs_block(grid, f)
    b = np.zeros(P * len(unk), dtype=complex)
    b[: len(unk)] = b0
    S0 = fd.deterministic_matrix(grid, k0)
    K0 = sp.diags(w2 * k0u * k0u).tocsr()
    return SGSystem(grid, s, r, P, A, Lbig.tocsr(), B.tocsr(), C.tocsr(), b, S0, K0)


def assemble_problem(prob) -> SGSystem:
    """Assemble from an input record with the fields dim, nx, ny, h, bc, s,
    r, k0, kl, f (the seeded workload generators produce such records)."""
    return assemble(prob.dim, prob.nx, prob.ny, prob.h, prob.bc, prob.s, prob.r,
                    prob.k0, prob.kl, source_nodes(prob))


def source_nodes(prob) -> np.ndarray:
    """The record's source f at the nodes, plus its unit point source
    (``prob.point``, if any) discretised as App. A.3 states."""
    f = np.asarray(prob.f, dtype=float).reshape(-1).copy()
    if getattr(prob, "point", None) is not None:
        f = f + fd.point_source(prob.dim, prob.nx, prob.ny, prob.h, prob.point)
    return f


def csl_matrix(sys: SGSystem, beta: float) -> sp.csr_matrix:
    """M(beta) = L - iB - (1 + i beta) K = A - i beta K   (Sec. 4)."""
    return (sys.A - 1j * beta * sys.Cbig).tocsr()


def mean_value_matrix(sys: SGSystem) -> sp.csr_matrix:
    """A_0 = I_P (x) S(xi_bar)   (Sec. 5, Remark 6.1)."""
    return sp.kron(sp.identity(sys.P), sys.S0, format="csr")


def csl_mean_block(sys: SGSystem, beta: float) -> sp.csr_matrix:
    """Block of M_0 = I (x) (S(0) - i beta D_2(k_0^2))   (Sec. 6.3)."""
    return (sys.S0 - 1j * beta * sys.K0).tocsr()


def realisation_matrix(sys: SGSystem, k0, kl, xi) -> sp.csr_matrix:
    """S(xi) for one sample xi (Sec. 3.1), k(x, xi) = k_0 + sum_l xi_l k_l."""
    k = np.asarray(k0, dtype=float).reshape(-1).copy()
    kl = np.asarray(kl, dtype=float).reshape(len(xi), -1) if len(xi) else kl
    for l, x in enumerate(xi):
        k = k + x * kl[l]
    return fd.deterministic_matrix(sys.grid, k)


def apply_rows(prob, x, rows, absolute: bool = False) -> np.ndarray:
    """Selected entries (A x)[rows] without assembling A, for sizes where the
    explicit matrix does not fit: row (a, u) of A is the row u of the FD
    Laplacian L applied to V_a plus row a of the per-node coupling
    -i w1(u) <k phi phi> - w2(u) <k^2 phi phi> applied to (V_0(u), ..., V_{P-1}(u))
    (Theorem 3.4; Sec. 3.2, c_ij and b_ij).  With absolute=True returns the
    sum of |term| over the Laplacian part and the coupling part taken
    separately (>= (|A| |x|)[rows]), the scale of the rounding error of a
    row computed as those two parts.

    Pinned by tests/test_oracle_sg.py against the explicit assembly."""
    grid = fd.make_grid(prob.dim, prob.nx, prob.ny, prob.h, prob.bc)
    n = len(grid.unknowns)
    s, r = prob.s, prob.r
    P = pc.num_modes(s, r)
    X = np.asarray(x).reshape(P, n)
    if absolute:
        X = np.abs(X)
    k0 = np.asarray(prob.k0, dtype=float).reshape(-1)[grid.unknowns]
    kl = np.asarray(prob.kl, dtype=float).reshape(s, -1)[:, grid.unknowns] if s else np.zeros((0, n))
    G1, G2 = pc.expectation_matrices(s, r)
    L = grid.L.tocsr()
    if absolute:
        L = abs(L)
    out = np.zeros(len(rows), dtype=complex if not absolute else float)
    for t, row in enumerate(np.asarray(rows)):
        a, u = divmod(int(row), n)
        lap = (L.getrow(u) @ X[a])[0]
        K1 = k0[u] * np.eye(P) + sum(kl[l, u] * G1[l] for l in range(s))
        K2 = k0[u] ** 2 * np.eye(P) + sum(2 * k0[u] * kl[l, u] * G1[l] for l in range(s))
        for (l, lp), G in G2.items():
            K2 = K2 + (1.0 if l == lp else 2.0) * kl[l, u] * kl[lp, u] * G
        M = -1j * grid.w1[u] * K1 - grid.w2[u] * K2
        if absolute:
            out[t] = abs(lap) + np.abs(M[a]) @ X[:, u]
        else:
            out[t] = lap + M[a] @ X[:, u]
    return out


def modes(sys: SGSystem, x: np.ndarray) -> np.ndarray:
    """Reshape an SG vector into (P, n): row i is V_i (Sec. 3.1)."""
    return np.asarray(x).reshape(sys.P, -1)
