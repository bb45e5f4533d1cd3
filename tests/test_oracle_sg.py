"""Pins for oracle.sg: the explicit SG system against what the paper prints
and proves."""
import os

import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from oracle import fd, krylov, pc, sg
from paper_2209_14740_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load_table2():
    rows = []
    for line in open(os.path.join(GOLD, "table2_sizes_nnz.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append(tuple(int(v) for v in line.split()))
    return rows


@pytest.mark.parametrize("row", [r for r in load_table2() if r[0] <= 5])
def test_table2_size_and_nnz(row):
    """Table 2: the exact size and nonzero count of A for the wedge."""
    r, nbasis, size, nnz = row
    S = sg.assemble_problem(inputs.wedge(127, 0.1, r))
    assert S.P == nbasis and S.A.shape == (size, size) and S.A.nnz == nnz


@pytest.mark.slow
@pytest.mark.parametrize("row", [r for r in load_table2() if r[0] >= 6])
def test_table2_size_and_nnz_high_degree(row):
    r, nbasis, size, nnz = row
    S = sg.assemble_problem(inputs.wedge(127, 0.1, r))
    assert S.P == nbasis and S.A.shape == (size, size) and S.A.nnz == nnz


@pytest.mark.parametrize("seed,dim", [(1, 1), (2, 2), (3, 2)])
def test_complex_symmetry_and_definiteness(seed, dim):
    """Theorem 3.4 / Lemma 3.2: A = L - iB - K with L, B, K real symmetric,
    L and B positive semidefinite, K positive definite; hence A^T = A."""
    pr = inputs.random_problem(seed, dim=dim, g=7 if dim == 2 else 14, s=2, r=2)
    S = sg.assemble_problem(pr)
    A = S.A.toarray()
    np.testing.assert_allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    for M, strict in ((S.Lbig, False), (S.Bbig, False), (S.Cbig, True)):
        Md = M.toarray()
        np.testing.assert_allclose(Md, Md.T, atol=1e-12 * max(1.0, np.abs(Md).max()))
        ev = np.linalg.eigvalsh(Md)
        scale = max(1.0, np.abs(ev).max())
        assert ev[0] > (1e-9 * scale if strict else -1e-9 * scale)
    np.testing.assert_allclose((S.Lbig - 1j * S.Bbig - S.Cbig).toarray(), A, atol=1e-12 * np.abs(A).max())


def test_theta_zero_collapse():
    """Remark 6.1 / Corollary 3.3: with theta = 0, A = I_P (x) S(0) is block
    diagonal, the modes i >= 1 of the solution vanish and V_0 is the
    deterministic solution."""
    pr = inputs.paper_1d(30.0, 0.0, 4, q=fd.mesh_rule(30.0))
    S = sg.assemble_problem(pr)
    A0 = sg.mean_value_matrix(S)
    assert abs(S.A - A0).max() == 0.0
    x = krylov.direct(S.A, S.b)
    V = sg.modes(S, x)
    assert np.abs(V[1:]).max() == 0.0
    u = spl.spsolve(S.S0.tocsc(), S.b[: S.S0.shape[0]])
    np.testing.assert_allclose(V[0], u, rtol=1e-12, atol=1e-14 * np.abs(u).max())


def _spectrum(pr, beta=0.5):
    S = sg.assemble_problem(pr)
    A = S.A.toarray()
    M = sg.csl_matrix(S, beta).toarray()
    return np.linalg.eigvals(A @ np.linalg.inv(M))


def test_spectrum_in_disk_absorbing():
    """Theorem 4.1(1) and Remark 4.2: eig(A M^-1) lies in |z - 1/2| <= 1/2 and
    outside |z - (1 - i beta/2)| < beta/2."""
    ev = _spectrum(inputs.paper_1d(50.0, 0.1, 3, q=fd.mesh_rule(50.0)))
    assert np.max(np.abs(ev - 0.5)) <= 0.5 + 1e-9
    assert np.min(np.abs(ev - (1 - 0.25j))) >= 0.25 - 1e-9


def test_spectrum_on_circle_dirichlet():
    """Theorem 4.1(2): with Dirichlet conditions eig(A M^-1) lies on the
    circle |z - 1/2| = 1/2."""
    pr = inputs.random_problem(7, dim=2, g=8, s=2, r=2, bc=(inputs.DIRICHLET,) * 4)
    ev = _spectrum(pr)
    np.testing.assert_allclose(np.abs(ev - 0.5), 0.5, atol=1e-9)


def load_conds():
    out = []
    for line in open(os.path.join(GOLD, "sec6_condition_numbers.txt")):
        if line.strip() and not line.startswith("#"):
            kb, q, v, tol = line.split()
            out.append((float(kb), q, float(v), float(tol)))
    return out


def _cond(M):
    sv = sl.svdvals(M)
    return sv[0] / sv[-1]


def _conds_for(kbar):
    S = sg.assemble_problem(inputs.paper_1d(kbar, 0.1, 3, q=fd.mesh_rule(kbar)))
    A = S.A.toarray()
    M = sg.csl_matrix(S, 0.5).toarray()
    A0 = sg.mean_value_matrix(S).toarray()
    M0 = sp.kron(sp.identity(S.P), sg.csl_mean_block(S, 0.5)).toarray()
    return {"cond(A)": lambda: _cond(A), "cond(A0)": lambda: _cond(A0),
            "cond(M)": lambda: _cond(M), "cond(M0)": lambda: _cond(M0),
            "cond(A*inv(M))": lambda: _cond(A @ np.linalg.inv(M)),
            "cond(A*inv(A0))": lambda: _cond(A @ np.linalg.inv(A0))}


@pytest.mark.parametrize("kbar", [10.0, 150.0, 200.0])
def test_printed_condition_numbers(kbar):
    """Sec. 6.2 / 6.3: every printed 2-norm condition number, to the printed
    digits (mesh rule with maxk = kbar)."""
    fns = _conds_for(kbar)
    for kb, q, v, tol in load_conds():
        if kb == kbar:
            assert abs(fns[q]() - v) <= tol, (kb, q)


def test_cond_M_bound():
    """Sec. 6.2: cond(M) <= 205 for all kbar (checked at the largest one)."""
    assert _conds_for(200.0)["cond(M)"]() <= 205


def test_infnorm_ordering():
    """Sec. 6.3: ||A - A_0||_inf < ||A - M||_inf < ||A - M_0||_inf at kbar = 50."""
    S = sg.assemble_problem(inputs.paper_1d(50.0, 0.1, 3, q=fd.mesh_rule(50.0)))
    A0 = sg.mean_value_matrix(S)
    M = sg.csl_matrix(S, 0.5)
    M0 = sp.kron(sp.identity(S.P), sg.csl_mean_block(S, 0.5))

    def ninf(X):
        return abs(X).sum(axis=1).max()

    assert ninf(S.A - A0) < ninf(S.A - M) < ninf(S.A - M0)


def test_sg_mean_against_quadrature():
    """Sec. 2.3 / Sec. 6.4: the SG coefficients approach the chaos
    projections of the true random solution as the degree grows.  Reference:
    Gauss-Legendre quadrature (48 nodes) of deterministic solves S(xi) u = F."""
    base = inputs.paper_1d(20.0, 0.1, 1, q=31)
    xq, wq = np.polynomial.legendre.leggauss(48)
    wq = wq / 2
    Sref = sg.assemble_problem(base)
    us = np.array([spl.spsolve(sg.realisation_matrix(Sref, base.k0, base.kl, [x]).tocsc(),
                               Sref.b[: Sref.S0.shape[0]]) for x in xq])
    mean = (wq[:, None] * us).sum(0)
    errs = []
    for r in range(1, 8):
        pr = inputs.paper_1d(20.0, 0.1, r, q=31)
        S = sg.assemble_problem(pr)
        V = sg.modes(S, krylov.direct(S.A, S.b))
        errs.append(np.abs(V[0] - mean).max() / np.abs(mean).max())
    assert errs[-1] < 1e-7
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))


@pytest.mark.parametrize("seed,dim,bc", [(21, 1, None), (22, 2, None), (23, 2, (0, 0, 0, 0)),
                                          (24, 1, (0, 1, 0, 0))])
def test_apply_rows_matches_explicit_matrix(seed, dim, bc):
    """The row-by-row evaluation used for full-size sampled parity equals the
    explicit Kronecker assembly; its absolute form (sum of |term| over the
    Laplacian and coupling terms separately) bounds |A| |x| from above and
    equals it on rows without a diagonal overlap of the two parts."""
    pr = inputs.random_problem(seed, dim=dim, g=9 if dim == 2 else 17, s=3, r=2, bc=bc)
    S = sg.assemble_problem(pr)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(S.A.shape[0]) + 1j * rng.standard_normal(S.A.shape[0])
    rows = rng.choice(S.A.shape[0], size=40, replace=False)
    got = sg.apply_rows(pr, x, rows)
    np.testing.assert_allclose(got, (S.A @ x)[rows], rtol=1e-13, atol=1e-13 * np.abs(S.A @ x).max())
    gabs = sg.apply_rows(pr, x, rows, absolute=True)
    ref = (abs(S.A) @ np.abs(x))[rows]
    assert np.all(gabs >= ref * (1 - 1e-13))
    L = sg.fd.make_grid(pr.dim, pr.nx, pr.ny, pr.h, pr.bc).L
    n = L.shape[0]
    # the gap is exactly |L_uu| + |M_aa| - |L_uu + M_aa| times |x_au|
    u = rows % n
    gap = gabs - ref
    assert np.all(gap <= 2 * np.abs(L.diagonal()[u]) * np.abs(x[rows]) * (1 + 1e-12) + 1e-9 * ref)
