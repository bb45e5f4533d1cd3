"""Pins for oracle.fd: the finite-difference matrices of Appendix A."""
import numpy as np
import pytest
import scipy.sparse as sp
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


def test_point_source_rule():
    """App. A.3: the Dirac source at a = 1/2 sits at t = ceil(q/2) =
    floor((q+1)/2): the midpoint for odd q, the smaller of the two closest
    points (x_t = 1/2 - h/2) for even q; 1/h in 1D and 1/h^2 in 2D there,
    zero elsewhere.  The general closest-node rule must reduce to that
    printed index for every q."""
    for q in range(1, 400):
        h = 1.0 / (q + 1)
        t = fd.nearest_node(0.5, h, q + 2)
        assert t == fd.point_source_index(q) == -(-q // 2)
        if q % 2:
            assert abs(t * h - 0.5) < 1e-15
        else:
            assert abs(t * h - (0.5 - h / 2)) < 1e-15
    f1 = fd.point_source(1, 10, 1, 1.0 / 9, (0.5,))
    assert f1[4] == 9.0 and np.count_nonzero(f1) == 1          # q = 8 (even): t = 4
    f2 = fd.point_source(2, 9, 9, 1.0 / 8, (0.5, 0.5))
    assert f2[4 + 9 * 4] == 64.0 and np.count_nonzero(f2) == 1  # q = 7 (odd): t = 4
    f3 = fd.point_source(2, 9, 9, 1.0 / 8, (0.3, 0.9))          # a general point: nearest node (2, 7)
    assert f3[2 + 9 * 7] == 64.0


# ---------------------------------------------------------------- Theorem A.6 weights
# A manufactured solution that satisfies the absorbing condition d_n u - i k u
# = 0 on every side of the unit square exactly: u = X(x) X(y) with
# X(x) = exp(i k x) (1 + alpha (x - 1)^2), alpha = i k / (1 - i k), so that
# X'(0) = -i k X(0) and X'(1) = i k X(1) (on x = 0 the outward normal is -x).
# Its source is f = -Delta u - k^2 u, with X'' = exp(i k x) (g'' + 2 i k g'
# - k^2 g), g = 1 + alpha (x - 1)^2.
_MMS_K = 10.0


def _mms_X(x, k=_MMS_K):
    al = 1j * k / (1 - 1j * k)
    return np.exp(1j * k * x) * (1 + al * (x - 1) ** 2)


def _mms_X2(x, k=_MMS_K):
    al = 1j * k / (1 - 1j * k)
    g, g1, g2 = 1 + al * (x - 1) ** 2, 2 * al * (x - 1), 2 * al
    return np.exp(1j * k * x) * (g2 + 2j * k * g1 - k * k * g)


def _mms_error(q, plant=None, k=_MMS_K):
    """Max-norm error of the Theorem A.6 discretisation (constant k) against
    the manufactured solution on (q+2)^2 nodes.  `plant` injects one of the
    plausible slips into the weights the oracle produced (a test of the
    test): 'w2_corner' (1/2 instead of 1/4 at the corners for D_2 and b_0),
    'w1_corner' (D_1 counted twice at the corners), 'b0_unweighted' (b_0 =
    f on the boundary)."""
    import scipy.sparse.linalg as spl
    g = q + 2
    h = 1.0 / (q + 1)
    G = fd.make_grid(2, g, g, h, (fd.ABSORBING,) * 4)
    x = np.linspace(0.0, 1.0, g)
    XX, YY = np.meshgrid(x, x, indexing="xy")
    XX, YY = XX.reshape(-1), YY.reshape(-1)
    u = _mms_X(XX) * _mms_X(YY)
    f = -(_mms_X2(XX) * _mms_X(YY) + _mms_X(XX) * _mms_X2(YY)) - k * k * u
    corners = [0, g - 1, g * (g - 1), g * g - 1]
    if plant is None:
        S = fd.deterministic_matrix(G, np.full(g * g, k)).tocsc()
        # rhs_block is real-valued: the complex source by linearity
        b = fd.rhs_block(G, f.real) + 1j * fd.rhs_block(G, f.imag)
    else:
        w1, w2, wb = G.w1.copy(), G.w2.copy(), G.w2.copy()
        if plant == "w2_corner":
            w2[corners] = 0.5
            wb[corners] = 0.5
        elif plant == "w1_corner":
            w1[corners] *= 2.0
        elif plant == "b0_unweighted":
            wb[:] = 1.0
        S = (G.L - 1j * k * sp.diags(w1) - k * k * sp.diags(w2)).tocsc()
        b = wb * f
    uh = spl.splu(S).solve(b)
    return np.abs(uh - u).max()


def _mms_ratios(plant=None):
    errs = [_mms_error(q, plant) for q in (15, 31, 63, 127)]
    return errs, [errs[i] / errs[i + 1] for i in range(3)]


def test_2d_absorbing_weights_converge_at_second_order():
    """Theorem A.6 at constant k against a solution of the continuous problem
    (absorbing on all four sides): the max-norm error falls by ~4 per halving
    of h (measured 4.26, 4.06, 4.02 for h = 1/16 .. 1/128) and is below 2e-3
    at h = 1/128.  This is fixed by the mathematics (second-order consistency
    of the scheme, incl. its one-sided closures, and the exact boundary
    condition of u), not by the oracle's own formulas, and every planted slip
    in the corner or edge weights fails it (test below: ratios 3.1 - 3.3 for
    1/2 at the D_2 / b_0 corners, 1.3 - 1.5 for a doubled corner D_1, ~2.1 for
    an unweighted b_0)."""
    errs, ratios = _mms_ratios()
    assert errs[-1] < 2e-3, errs
    assert all(3.8 < r < 4.4 for r in ratios[1:]), ratios
    assert 3.8 < ratios[0] < 4.6, ratios


@pytest.mark.parametrize("plant", ["w2_corner", "w1_corner", "b0_unweighted"])
def test_2d_weight_pin_rejects_planted_slips(plant):
    errs, ratios = _mms_ratios(plant)
    assert not (errs[-1] < 2e-3 and all(3.8 < r < 4.4 for r in ratios[1:])), (plant, errs, ratios)


def test_2d_absorbing_is_the_tensor_product_of_theorem_a2():
    """Separation of variables: -Delta - k^2 = (-d_xx - k^2/2) + (-d_yy - k^2/2)
    and the absorbing condition on an x-side involves d_x only, so at constant
    k the 2D matrix of Theorem A.6 must equal D (x) S_1 + S_1 (x) D + k^2 D (x) D
    with S_1 = T - i (k/h) E - k^2 D the 1D matrix of Theorem A.2 (D = diag(1/2,
    1, ..., 1, 1/2), E the end indicator), built here from the 1D axis alone.
    Entry by entry this fixes D_1 = (D (x) E + E (x) D) k/h (1/h once on every
    boundary node, corners included) and D_2 = (D (x) D) k^2 (1/4 at the
    corners)."""
    for g, k in ((9, 7.0), (17, 12.5)):
        h = 1.0 / (g - 1)
        ax = fd.axis_1d(g, h, fd.ABSORBING, fd.ABSORBING)
        D = sp.diags(ax.d)
        S1 = ax.T - 1j * (k / h) * sp.diags(ax.e) - k * k * D
        G = fd.make_grid(2, g, g, h, (fd.ABSORBING,) * 4)
        S2 = fd.deterministic_matrix(G, np.full(g * g, k))
        ref = sp.kron(D, S1) + sp.kron(S1, D) + k * k * sp.kron(D, D)
        assert abs(S2 - ref).max() <= 1e-12 * abs(ref).max()
