"""Pins for oracle.fd: the finite-difference matrices of Appendix A."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle import fd


def exact_c1(x, k):
    """-u'' - k^2 u = 1 on (0, 1), u(0) = 0, u'(1) - i k u(1) = 0.  Solved
    by hand: u = k^-2 [cos kx - 1 + i (1 - e^{ik}) sin kx]."""
    return (np.cos(k * x) - 1.0 + 1j * (1.0 - np.exp(1j * k)) * np.sin(k * x)) / k ** 2


def test_exact_solution_satisfies_bvp():
    k = 20.0
    x = np.linspace(0, 1, 2001)
    u = exact_c1(x, k)
    dx = x[1] - x[0]
    upp = (u[2:] - 2 * u[1:-1] + u[:-2]) / dx ** 2
    res = -upp - k * k * u[1:-1] - 1.0
    assert np.abs(res).max() < 1e-3 * np.abs(k * k * u).max()
    assert abs(u[0]) == 0.0
    up1 = (3 * u[-1] - 4 * u[-2] + u[-3]) / (2 * dx)
    assert abs(up1 - 1j * k * u[-1]) < 1e-3 * abs(k * u[-1])


def test_second_order_convergence_1d():
    """Theorem A.1 interior rows + Theorem A.2 closure: the scheme is second
    order (App. A.1); the max error against the closed form drops ~4x per
    halving of h."""
    k = 20.0
    errs = []
    for n in (200, 400, 800):
        g = fd.make_grid(1, n + 1, 1, 1.0 / n, (fd.DIRICHLET, fd.ABSORBING, 0, 0))
        S = fd.deterministic_matrix(g, np.full(n + 1, k))
        b = fd.rhs_block(g, np.ones(n + 1))
        u = spl.spsolve(S.tocsc(), b.astype(complex))
        xs = g.unknowns / n
        errs.append(np.abs(u - exact_c1(xs, k)).max())
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert errs[0] < 1e-2 * np.abs(exact_c1(np.linspace(0, 1, 201), k)).max()
    for q in ratios:
        assert 3.7 < q < 4.3


def test_absorbing_T_kernel_and_semidefinite():
    """Theorem A.2: T symmetric positive semidefinite with ker T = span{1};
    D_2 weights (1/2 at ends) positive."""
    h = 1.0 / 17
    ax = fd.axis_1d(18, h, fd.ABSORBING, fd.ABSORBING)
    T = ax.T.toarray()
    np.testing.assert_allclose(T, T.T)
    ev = np.linalg.eigvalsh(T)
    assert abs(ev[0]) < 1e-9 * ev[-1] and ev[1] > 1e-6
    np.testing.assert_allclose(T @ np.ones(18), 0.0, atol=1e-9)
    assert ax.d[0] == ax.d[-1] == 0.5 and np.all(ax.d[1:-1] == 1.0)


def test_dirichlet_T_spd():
    """Theorem A.1: T = h^-2 tridiag(-1, 2, -1) is SPD with the known
    eigenvalues (2 - 2 cos(j pi h)) / h^2."""
    q = 15
    h = 1.0 / (q + 1)
    ax = fd.axis_1d(q + 2, h, fd.DIRICHLET, fd.DIRICHLET)
    ev = np.sort(np.linalg.eigvalsh(ax.T.toarray()))
    ref = np.sort((2 - 2 * np.cos(np.arange(1, q + 1) * np.pi * h)) / h ** 2)
    np.testing.assert_allclose(ev, ref, rtol=1e-12)


def test_2d_absorbing_structure():
    """Theorem A.6: L = D (x) T + T (x) D symmetric PSD with constants in its
    kernel; D_1 / h puts 1/h on every boundary node, corners once; D_2 and
    b_0 weights are d_i d_j (1/4 at corners, 1/2 on edges)."""
    g = 9
    h = 1.0 / (g - 1)
    G = fd.make_grid(2, g, g, h, (fd.ABSORBING,) * 4)
    L = G.L.toarray()
    np.testing.assert_allclose(L, L.T)
    assert np.linalg.eigvalsh(L)[0] > -1e-9
    np.testing.assert_allclose(L @ np.ones(g * g), 0.0, atol=1e-8)
    W2 = G.w2.reshape(g, g)
    assert W2[0, 0] == 0.25 and W2[0, 3] == 0.5 and W2[3, 3] == 1.0
    W1 = G.w1.reshape(g, g) * h
    assert W1[0, 0] == 1.0 and W1[0, 4] == 1.0 and W1[4, 0] == 1.0 and W1[4, 4] == 0.0
    # 5-point row in the interior: (4u - sum of 4 neighbours)/h^2
    c = 4 + g * 4
    row = L[c]
    assert row[c] == pytest.approx(4 / h ** 2)
    assert sorted(row[row != 0])[:4] == pytest.approx([-1 / h ** 2] * 4)


def test_mesh_rule_and_source():
    """Sec. 6: kbar = 50 gives q = 127, kbar = 150 and 200 give q = 511,
    kbar = 10 gives q = 31.  App. A.3: t = ceil(q/2)."""
    assert fd.mesh_rule(50) == 127 and fd.mesh_rule(150) == 511
    assert fd.mesh_rule(200) == 511 and fd.mesh_rule(10) == 31
    assert fd.point_source_index(127) == 64 and fd.point_source_index(6) == 3
