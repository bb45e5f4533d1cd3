"""Pins for oracle.pc: chaos basis size and Galerkin triple products.

The triple products are checked against Gauss-Legendre quadrature of
Legendre polynomials that numpy evaluates from its own coefficient series
(numpy.polynomial.legendre), a route independent of the three-term
recurrence the oracle uses.  Quadrature with n nodes is exact for
polynomials of degree <= 2n - 1, so the check is exact up to rounding."""
import itertools
from math import comb

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import pc

GOLDEN_NBASIS = {0: 1, 1: 4, 2: 10, 3: 20, 4: 35, 5: 56, 6: 84, 7: 120, 8: 165}   # Table 2, s = 3


def phi_1d(n, x):
    """Orthonormal Legendre p_n = sqrt(2n+1) P_n w.r.t. density 1/2 on [-1, 1]."""
    c = np.zeros(n + 1)
    c[n] = 1.0
    return np.sqrt(2 * n + 1) * npleg.legval(x, c)


def quad_tensor(s, npts):
    x, w = npleg.leggauss(npts)
    w = w / 2.0                                  # density 1/2 per variable
    nodes = np.array(list(itertools.product(x, repeat=s)))
    weights = np.prod(np.array(list(itertools.product(w, repeat=s))), axis=1)
    return nodes, weights


def phi_multi(alpha, nodes):
    v = np.ones(len(nodes))
    for t, a in enumerate(alpha):
        v *= phi_1d(int(a), nodes[:, t])
    return v


@pytest.mark.parametrize("s,r", [(1, 5), (2, 3), (3, 2), (3, 3), (6, 1)])
def test_basis_size_closed_form(s, r):
    al = pc.multi_indices(s, r)
    assert len(al) == comb(s + r, s) == pc.num_modes(s, r)
    # all distinct, total degree <= r, graded order, phi_0 first
    assert len({tuple(a) for a in al}) == len(al)
    deg = al.sum(axis=1)
    assert deg.max() == r and deg[0] == 0 and np.all(np.diff(deg) >= 0)


def test_table2_nbasis():
    for r, nb in GOLDEN_NBASIS.items():
        assert pc.num_modes(3, r) == nb


@pytest.mark.parametrize("s,r", [(1, 5), (2, 3), (3, 2), (2, 4)])
def test_triple_products_against_quadrature(s, r):
    al = pc.multi_indices(s, r)
    P = len(al)
    nodes, w = quad_tensor(s, r + 3)                  # exact for degree 2r + 2
    Phi = np.array([phi_multi(a, nodes) for a in al])  # P x nq
    # orthonormality (Sec. 2.3)
    np.testing.assert_allclose((Phi * w) @ Phi.T, np.eye(P), atol=1e-12)
    G1 = pc.galerkin_first(s, r)
    G2 = pc.galerkin_second(s, r)
    for l in range(s):
        ref = (Phi * (w * nodes[:, l])) @ Phi.T
        np.testing.assert_allclose(G1[l], ref, atol=1e-12)
        for lp in range(l, s):
            ref2 = (Phi * (w * nodes[:, l] * nodes[:, lp])) @ Phi.T
            np.testing.assert_allclose(G2[(l, lp)], ref2, atol=1e-12)


@pytest.mark.parametrize("s,r", [(1, 6), (3, 3)])
def test_bandwidth_lemma(s, r):
    """Lemma A.3: a degree-d coefficient couples only modes whose total
    degrees differ by at most d; with one variable the matrices of k and k^2
    are tridiagonal and pentadiagonal (Sec. 6)."""
    al = pc.multi_indices(s, r)
    deg = al.sum(axis=1)
    G1 = pc.galerkin_first(s, r)
    G2 = pc.galerkin_second(s, r)
    dd = np.abs(deg[:, None] - deg[None, :])
    for G in G1:
        assert np.all(G[dd > 1] == 0.0)
        np.testing.assert_array_equal(G, G.T)          # Lemma 3.2 symmetry
    for G in G2.values():
        assert np.all(G[dd > 2] == 0.0)
        np.testing.assert_array_equal(G, G.T)
    if s == 1:
        idx = np.arange(len(al))
        band = np.abs(idx[:, None] - idx[None, :])
        assert np.all(G1[0][band > 1] == 0) and np.any(G1[0][band == 1] != 0)
        assert np.all(G2[(0, 0)][band > 2] == 0) and np.any(G2[(0, 0)][band == 2] != 0)


def test_known_values():
    """Closed forms: E[xi p_0 p_1] = 1/sqrt(3); E[xi^2] = 1/3;
    E[xi^2 p_0 p_2] = 2/(3 sqrt 5); E[xi^2 p_1 p_1] = 3/5."""
    G1 = pc.galerkin_first(1, 3)[0]
    G2 = pc.galerkin_second(1, 3)[(0, 0)]
    assert G1[0, 1] == pytest.approx(1 / np.sqrt(3), abs=1e-15)
    assert G2[0, 0] == pytest.approx(1 / 3, abs=1e-15)
    assert G2[0, 2] == pytest.approx(2 / (3 * np.sqrt(5)), abs=1e-15)
    assert G2[1, 1] == pytest.approx(3 / 5, abs=1e-15)
