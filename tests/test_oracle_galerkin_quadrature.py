"""Pins for oracle.sg from the definition of the Galerkin blocks and from the
mean-value preconditioner theorems (CPU, no GPU).

1. Sec. 3 / Theorem 3.4: block (i, j) of the SG matrix is E[phi_i phi_j
   S(xi)], the expectation over xi uniform on [-1, 1]^s of the deterministic
   FD matrix of one realisation.  The reference here builds S(xi) one sample
   at a time and integrates by tensor Gauss-Legendre quadrature (exact: the
   integrand has degree <= 2r + 2 in each variable) with the orthonormal
   basis taken from numpy's Legendre module, so it shares neither the
   three-term-recurrence tables nor the Kronecker-sum formula with the
   oracle's assembly.  A dropped factor 2 in the cross terms, a wrong sign
   of the boundary term or a transposed block fails it.
2. Theorem 5.1: ||Abar^-1 A - I||_F <= C_m ||S(xi_bar)^-1||_F
   || ||Delta S(xi)||_F ||_{L2}, C_m = sqrt(m+1) (sum_ij ||phi_i phi_j||^2)^(1/2),
   and the same bound for A Abar^-1 - I (the remark after it).
3. Theorem 5.2: with S(xi) = S_0 + O(theta), ||A_0^-1 A - I||_F = O(theta):
   halving theta halves it to first order.
"""
import itertools

import numpy as np
import pytest
from numpy.polynomial import legendre

from oracle import pc, sg
from paper_2209_14740_gb300 import inputs


def basis_values(multi, xi):
    """phi_alpha(xi) = prod_l sqrt(2 a_l + 1) P_{a_l}(xi_l) (orthonormal for the
    uniform density 1/2 on [-1, 1] in each variable)."""
    out = np.empty(len(multi))
    for i, a in enumerate(multi):
        v = 1.0
        for l, n in enumerate(a):
            c = np.zeros(n + 1)
            c[n] = 1.0
            v *= np.sqrt(2 * n + 1) * legendre.legval(xi[l], c)
        out[i] = v
    return out


def tensor_rule(s, npts):
    x, w = legendre.leggauss(npts)
    w = w / 2.0                                   # density 1/2 per variable
    for idx in itertools.product(range(npts), repeat=s):
        yield np.array([x[i] for i in idx]), float(np.prod([w[i] for i in idx]))


def realisation(S, prob, xi):
    return sg.realisation_matrix(S, prob.k0, prob.kl, list(xi)).toarray()


@pytest.mark.parametrize("dim,g,s,r,seed", [(1, 24, 2, 3, 1), (1, 16, 1, 5, 2), (2, 8, 3, 2, 3),
                                            (2, 7, 2, 3, 4)])
def test_galerkin_blocks_are_quadrature_means(dim, g, s, r, seed):
    prob = inputs.random_problem(seed, dim=dim, g=g, s=s, r=r)
    S = sg.assemble_problem(prob)
    multi = pc.multi_indices(s, r)
    P = len(multi)
    n = S.S0.shape[0]
    Aq = np.zeros((P * n, P * n), dtype=complex)
    for xi, wq in tensor_rule(s, r + 2):
        phi = basis_values(multi, xi)
        Aq += wq * np.kron(np.outer(phi, phi), realisation(S, prob, xi))
    A = S.A.toarray()
    scale = np.abs(A).max()
    assert np.abs(A - Aq).max() <= 1e-12 * scale
    # the right-hand side: E[phi_i f] = delta_i0 f for a deterministic source
    bq = np.zeros(P * n, dtype=complex)
    b0 = S.b[:n]
    for xi, wq in tensor_rule(s, r + 1):
        bq += wq * np.kron(basis_values(multi, xi), b0)
    assert np.abs(S.b - bq).max() <= 1e-13 * np.abs(b0).max()


def _mean_value_quantities(prob):
    S = sg.assemble_problem(prob)
    multi = pc.multi_indices(prob.s, prob.r)
    P = len(multi)
    n = S.S0.shape[0]
    S0 = S.S0.toarray()
    # S(xi_bar) with xi_bar = 0 (uniform variables) is the realisation at 0
    assert np.abs(S0 - realisation(S, prob, np.zeros(prob.s))).max() <= 1e-14 * np.abs(S0).max()
    S0inv = np.linalg.inv(S0)
    A = S.A.toarray()
    Abar_inv = np.kron(np.eye(P), S0inv)
    I = np.eye(P * n)
    left = np.linalg.norm(Abar_inv @ A - I, "fro")
    right = np.linalg.norm(A @ Abar_inv - I, "fro")
    # E ||Delta S(xi)||_F^2: degree 4 in each variable
    eds2 = sum(wq * np.linalg.norm(realisation(S, prob, xi) - S0, "fro") ** 2
               for xi, wq in tensor_rule(prob.s, 4))
    # sum_ij E[phi_i^2 phi_j^2]: degree 4r in each variable
    sphi = 0.0
    for xi, wq in tensor_rule(prob.s, 2 * prob.r + 1):
        phi = basis_values(multi, xi)
        sphi += wq * np.sum(np.outer(phi * phi, phi * phi))
    Cm = np.sqrt(P) * np.sqrt(sphi)
    bound = Cm * np.linalg.norm(S0inv, "fro") * np.sqrt(eds2)
    return left, right, bound


@pytest.mark.parametrize("dim,g,s,r,seed", [(1, 20, 2, 2, 7), (2, 6, 2, 2, 8), (1, 30, 1, 4, 9)])
def test_theorem_5_1_frobenius_bound(dim, g, s, r, seed):
    prob = inputs.random_problem(seed, dim=dim, g=g, s=s, r=r)
    left, right, bound = _mean_value_quantities(prob)
    assert 0.0 < left <= bound
    assert 0.0 < right <= bound
    # A and Abar are complex symmetric, so (Abar^-1 A)^T = A Abar^-1
    assert abs(left - right) <= 1e-10 * left


def test_theorem_5_2_order_theta():
    vals = []
    for theta in (0.005, 0.01, 0.02):
        prob = inputs.paper_1d(20.0, theta, 2, q=31)
        left, right, bound = _mean_value_quantities(prob)
        vals.append(left)
        assert left <= bound
    # first order in theta: doubling theta doubles the distance, up to a
    # deviation that itself grows with theta
    r1, r2 = vals[1] / vals[0], vals[2] / vals[1]
    assert abs(r1 - 2.0) <= 1e-3 and abs(r2 - 2.0) <= 1e-3, (r1, r2)
    assert abs(r2 - 2.0) > abs(r1 - 2.0)
