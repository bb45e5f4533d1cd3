"""Solvers for the SG system (oracle; test infrastructure only).

* ``direct``: SuperLU of the explicit SG matrix, the analogue of the
  paper's x = A\\b (Sec. 6.3, Sec. 7).
* ``BlockPrecond``: a block-diagonal preconditioner I_P (x) S_blk applied
  with ONE sparse LU of the n x n block to all P modes at once, by viewing
  the SG vector as an n x P matrix (the reshape of Sec. 6.3).  With
  S_blk = S(xi_bar) this is the mean-value preconditioner A_0 (Sec. 5),
  with S_blk = S(xi_bar) - i beta D_2(k_0^2) the mean-value CSL M_0.
* ``FullPrecond``: LU of a full SG-sized matrix (the CSL M of Sec. 4).
* ``gmres``: restarted GMRES (Saad & Schultz) as used in Sec. 6.3/7:
  right preconditioning A M^-1 y = b, x = M^-1 y (stopping on
  ||b - A x|| / ||b||), or left preconditioning M^-1 A x = M^-1 b (stopping
  on the preconditioned residual).  Arnoldi with classical Gram-Schmidt
  applied twice, complex Givens rotations, Hermitian inner product.  The
  paper names MATLAB's gmres without its orthogonalisation; CGS2 is this
  build's reading (exact-arithmetic equivalent).
* ``stationary``: A_0 x^(i+1) = b - (A - A_0) x^(i), x^(0) = A_0^-1 b
  (Sec. 5 and Sec. 7).

Pins: tests/test_oracle_krylov.py (GMRES iteration counts of Sec. 6.3 for
none / M / M_0 / A_0 at kbar = 50, agreement with the direct solution to the
1.7e-14 printed there, convergence at theta = 0.1 and divergence at
theta = 0.2 of the stationary iteration, and its slower convergence for a
larger degree, Sec. 7).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl


def direct(A: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    return spl.splu(sp.csc_matrix(A)).solve(np.asarray(b, dtype=complex))


class BlockPrecond:
    """z = (I_P (x) S_blk)^-1 r with one LU of S_blk for all P modes."""

    def __init__(self, S_blk: sp.spmatrix, P: int):
        self.lu = spl.splu(sp.csc_matrix(S_blk, dtype=complex))
        self.n = S_blk.shape[0]
        self.P = P

    def __call__(self, r: np.ndarray) -> np.ndarray:
        R = np.asarray(r, dtype=complex).reshape(self.P, self.n).T   # n x P
        Z = self.lu.solve(np.ascontiguousarray(R))
        return Z.T.reshape(-1)


class FullPrecond:
    def __init__(self, M: sp.spmatrix):
        self.lu = spl.splu(sp.csc_matrix(M, dtype=complex))

    def __call__(self, r: np.ndarray) -> np.ndarray:
        return self.lu.solve(np.asarray(r, dtype=complex))


def _identity(v):
    return v


@dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    relres: float              # final true ||b - A x|| / ||b||
    converged: bool
    history: list = field(default_factory=list)   # residual estimate per iteration


def _givens(a: complex, b: complex):
    """c real, s complex with [c s; -conj(s) c] [a; b] = [rho; 0]."""
    aa = abs(a)
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if aa == 0.0:
        return 0.0, np.conj(b) / abs(b) + 0.0j
    rr = np.hypot(aa, abs(b))
    return aa / rr, (a / aa) * np.conj(b) / rr


def gmres(A, b, M=None, restart=None, tol=1e-8, maxit=None, x0=None,
          side="right") -> GmresResult:
    """Restarted GMRES(restart) for A x = b.

    A: matrix or callable; M: callable applying M^-1 (None = identity).
    restart None = full GMRES (restart = n).  maxit = max total Arnoldi
    steps (default n).  Relative residual for right preconditioning and no
    preconditioning is ||b - A x|| / ||b|| (Sec. 6.3); for side='left' it is
    ||M^-1 (b - A x)|| / ||M^-1 b||."""
    Aop = A if callable(A) else (lambda v, A=A: A @ v)
    Mop = M if M is not None else _identity
    b = np.asarray(b, dtype=complex)
    n = b.size
    restart = n if restart is None else min(restart, n)
    maxit = n if maxit is None else maxit
    x = np.zeros(n, dtype=complex) if x0 is None else np.array(x0, dtype=complex)

    if side == "left":
        Mb = Mop(b)
        bnorm = np.linalg.norm(Mb)

        def resid(xx):
            return Mop(b - Aop(xx))

        def op(v):
            return Mop(Aop(v))
    else:
        bnorm = np.linalg.norm(b)

        def resid(xx):
            return b - Aop(xx)

        def op(v):
            return Aop(Mop(v))

    if bnorm == 0.0:
        return GmresResult(np.zeros(n, dtype=complex), 0, 0.0, True)
    hist = []
    iters = 0
    r = resid(x)
    beta = np.linalg.norm(r)
    if beta / bnorm <= tol:
        return GmresResult(x, 0, beta / bnorm, True, hist)
    while iters < maxit:
        m = restart
        V = np.zeros((m + 1, n), dtype=complex)
        H = np.zeros((m + 1, m), dtype=complex)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=complex)
        g = np.zeros(m + 1, dtype=complex)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = op(V[j])
            # classical Gram-Schmidt, twice (Hermitian inner product)
            h1 = V[: j + 1].conj() @ w
            w = w - V[: j + 1].T @ h1
            h2 = V[: j + 1].conj() @ w
            w = w - V[: j + 1].T @ h2
            H[: j + 1, j] = h1 + h2
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            k = j + 1
            est = abs(g[j + 1]) / bnorm
            hist.append(est)
            if est <= tol or hn == 0.0 or iters >= maxit:
                break
            V[j + 1] = w / hn
        y = np.zeros(k, dtype=complex)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1: k] @ y[i + 1: k]) / H[i, i]
        upd = V[:k].T @ y
        x = x + (Mop(upd) if side != "left" else upd)
        r = resid(x)
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol:
            return GmresResult(x, iters, beta / bnorm, True, hist)
        if beta == 0.0:
            break
    return GmresResult(x, iters, beta / bnorm, beta / bnorm <= tol, hist)


def stationary(A, A0_solve, b, iters: int, x_ref=None):
    """Stationary iteration of Sec. 5 with B = A_0 (Sec. 7):
    A_0 x^(i+1) = b - (A - A_0) x^(i), i.e. x^(i+1) = x^(i) + A_0^-1 (b - A x^(i)),
    starting from x^(0) = A_0^-1 b.  Returns the iterates' relative errors in
    the max-norm against x_ref (if given) and the final iterate."""
    b = np.asarray(b, dtype=complex)
    x = A0_solve(b)
    errs = []
    for _ in range(iters):
        if x_ref is not None:
            errs.append(np.abs(x - x_ref).max() / np.abs(x_ref).max())
        x = x + A0_solve(b - A @ x)
    if x_ref is not None:
        errs.append(np.abs(x - x_ref).max() / np.abs(x_ref).max())
    return x, errs
