"""Pins for oracle.krylov: GMRES and the stationary iteration."""
import os

import numpy as np
import pytest

from oracle import fd, krylov, sg
from paper_2209_14740_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load_counts():
    out = {}
    for line in open(os.path.join(GOLD, "sec6_gmres_kbar50.txt")):
        if line.strip() and not line.startswith("#"):
            name, v, lo, hi = line.split()
            out[name] = (int(v), int(lo), int(hi))
    return out


@pytest.fixture(scope="module")
def kbar50():
    S = sg.assemble_problem(inputs.paper_1d(50.0, 0.1, 3, q=fd.mesh_rule(50.0)))
    return S, krylov.direct(S.A, S.b)


def test_gmres_counts_kbar50(kbar50):
    """Sec. 6.3: full GMRES to tol 1e-12 takes about 250 / 50 / 50 / 25 steps
    without preconditioner / with M / M_0 / A_0, and every GMRES solution is
    within 1.7e-14 (max-norm) of the direct solution."""
    S, xd = kbar50
    precs = {"none": None, "M": krylov.FullPrecond(sg.csl_matrix(S, 0.5)),
             "M0": krylov.BlockPrecond(sg.csl_mean_block(S, 0.5), S.P),
             "A0": krylov.BlockPrecond(S.S0, S.P)}
    counts = load_counts()
    got = {}
    for name, M in precs.items():
        res = krylov.gmres(S.A, S.b, M, tol=1e-12)
        assert res.converged and res.relres <= 1e-12
        got[name] = res.iters
        lo, hi = counts[name][1:]
        assert lo <= res.iters <= hi, (name, res.iters)
        assert np.abs(res.x - xd).max() <= 1.7e-14
    assert got["A0"] < got["M"] <= got["M0"] < got["none"]


def test_left_preconditioning_matches(kbar50):
    """Sec. 6.3: left and right preconditioning give very similar counts."""
    S, xd = kbar50
    M = krylov.BlockPrecond(S.S0, S.P)
    rl = krylov.gmres(S.A, S.b, M, tol=1e-12, side="left")
    rr = krylov.gmres(S.A, S.b, M, tol=1e-12, side="right")
    assert abs(rl.iters - rr.iters) <= 3
    assert np.abs(rl.x - xd).max() <= 1e-13


@pytest.mark.parametrize("restart", [5, 20])
def test_restarted_gmres_reaches_direct(restart):
    pr = inputs.random_problem(11, dim=2, g=10, s=2, r=2)
    S = sg.assemble_problem(pr)
    xd = krylov.direct(S.A, S.b)
    res = krylov.gmres(S.A, S.b, krylov.BlockPrecond(S.S0, S.P), restart=restart, tol=1e-11, maxit=2000)
    assert res.converged
    assert np.linalg.norm(S.b - S.A @ res.x) / np.linalg.norm(S.b) <= 1e-11
    assert np.linalg.norm(res.x - xd) / np.linalg.norm(xd) < 1e-8


def test_gmres_nonzero_initial_guess_and_exact_start():
    pr = inputs.random_problem(12, dim=1, g=30, s=1, r=3)
    S = sg.assemble_problem(pr)
    xd = krylov.direct(S.A, S.b)
    res = krylov.gmres(S.A, S.b, None, tol=1e-10, x0=xd)
    assert res.iters == 0 and res.converged
    res2 = krylov.gmres(S.A, S.b, None, tol=1e-10, x0=0.5 * xd)
    assert res2.converged and np.linalg.norm(res2.x - xd) / np.linalg.norm(xd) < 1e-7


def test_stationary_iteration_converges_and_diverges():
    """Sec. 7: the stationary iteration with B = A_0 converges for theta =
    0.1 and diverges for theta = 0.2 (wedge, degree 2; q reduced to 63 to
    keep the test short)."""
    out = {}
    for theta in (0.1, 0.2):
        S = sg.assemble_problem(inputs.wedge(63, theta, 2))
        xd = krylov.direct(S.A, S.b)
        pre = krylov.BlockPrecond(S.S0, S.P)
        _, errs = krylov.stationary(S.A, pre, S.b, 25, x_ref=xd)
        out[theta] = errs
    assert out[0.1][-1] < 1e-3 * out[0.1][0]
    assert out[0.2][-1] > out[0.2][0]


def test_stationary_iteration_slower_for_larger_degree():
    """Sec. 7: at theta = 0.1 the stationary iteration with B = A_0 converges,
    more slowly for a larger degree r (the SG matrix grows with r).  Wedge
    with q = 63 (the paper uses 127; at q = 31 the iteration already diverges
    for r >= 4): contraction rate over iterations 10..30 at r = 2 and r = 4."""
    rates = {}
    for r in (2, 4):
        S = sg.assemble_problem(inputs.wedge(63, 0.1, r))
        xd = krylov.direct(S.A, S.b)
        pre = krylov.BlockPrecond(S.S0, S.P)
        _, errs = krylov.stationary(S.A, pre, S.b, 30, x_ref=xd)
        assert errs[-1] < 1e-3 * errs[0]
        rates[r] = (errs[-1] / errs[10]) ** (1.0 / 20)
    assert rates[2] < rates[4] < 1.0, rates
