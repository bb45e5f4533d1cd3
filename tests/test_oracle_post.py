"""Pins of the oracle's post-processing (oracle/post.py, Sec. 7 of the paper).

The closed forms (E = V_0, Var = sum_{i>=1} |.|^2) rest on the orthonormality
of the chaos basis.  They are checked here against a route that does not use
it: the SG polynomial u~(x, xi) = sum_i V_i(x) phi_i(xi) is evaluated at the
nodes of a tensor Gauss-Legendre rule (numpy's Legendre module, normalised
Legendre polynomials built from it, not the oracle's recurrence), and its
mean and variance are taken by quadrature, which is exact for these
polynomial degrees.  A dropped mode, a mode-0 term left in the variance, or a
real/imaginary mix-up fails it.
"""
import itertools

import numpy as np
import pytest
from numpy.polynomial import legendre as npl

from oracle import krylov, pc, post, sg
from paper_2209_14740_gb300 import inputs


def _phi(alpha, xi):
    """Product of orthonormal Legendre polynomials sqrt(2a+1) P_a(xi_l)."""
    v = 1.0
    for a, x in zip(alpha, xi):
        c = np.zeros(a + 1)
        c[a] = 1.0
        v = v * np.sqrt(2 * a + 1) * npl.legval(x, c)
    return v


def _quadrature_stats(V, s, r):
    alpha = pc.multi_indices(s, r)
    x, w = npl.leggauss(r + 2)
    w = w / 2.0                                    # density 1/2 per variable
    m1 = np.zeros(V.shape[1], dtype=complex)
    m2r = np.zeros(V.shape[1])
    m2i = np.zeros(V.shape[1])
    for idx in itertools.product(range(len(x)), repeat=s):
        xi = x[list(idx)]
        wt = np.prod(w[list(idx)])
        u = sum(V[i] * _phi(alpha[i], xi) for i in range(len(alpha)))
        m1 += wt * u
        m2r += wt * u.real ** 2
        m2i += wt * u.imag ** 2
    return m1, m2r - m1.real ** 2, m2i - m1.imag ** 2


@pytest.mark.parametrize("s,r", [(1, 4), (2, 3), (3, 2)])
def test_mean_and_variance_against_quadrature(s, r):
    rng = np.random.default_rng(10 * s + r)
    P = pc.num_modes(s, r)
    V = rng.standard_normal((P, 7)) + 1j * rng.standard_normal((P, 7))
    qm, qvr, qvi = _quadrature_stats(V, s, r)
    np.testing.assert_allclose(post.mean(V), qm, rtol=0, atol=1e-12)
    vr, vi = post.variances(V)
    np.testing.assert_allclose(vr, qvr, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(vi, qvi, rtol=1e-11, atol=1e-12)


def test_theta_zero_has_no_variance():
    """theta = 0 (Remark 6.1): A = I (x) S(0), so every mode i >= 1 of the SG
    solution is zero: the variance and gamma_j (j >= 1) vanish and gamma_0 is
    the max-norm of the deterministic solution."""
    pr = inputs.paper_1d(20.0, 0.0, 3, q=31)
    S = sg.assemble_problem(pr)
    V = sg.modes(S, krylov.direct(S.A, S.b))
    vr, vi = post.variances(V)
    assert vr.max() == 0.0 and vi.max() == 0.0
    g = post.gamma(V, pr.s, pr.r)
    assert np.all(g[1:] == 0.0)
    u = krylov.direct(S.S0, S.b[: S.S0.shape[0]])
    assert abs(g[0] - np.abs(u).max()) <= 1e-12 * np.abs(u).max()


def test_gamma_by_brute_force():
    s, r = 3, 3
    rng = np.random.default_rng(4)
    P = pc.num_modes(s, r)
    V = rng.standard_normal((P, 5)) + 1j * rng.standard_normal((P, 5))
    g = post.gamma(V, s, r)
    for j in range(r + 1):
        best = 0.0
        for i, a in enumerate(pc.multi_indices(s, r)):
            if sum(a) == j:
                best = max(best, max(abs(v) for v in V[i]))
        assert abs(g[j] - best) <= 4e-16 * best   # |z| by Python and numpy may differ in the last bit
