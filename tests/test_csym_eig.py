"""CPU test of the host eigen-solver of the 2D preconditioner set-up
(paper_2209_14740_gb300/csrc/csym_eig.h): implicit QR with complex
orthogonal rotations for the eigenvalues, inverse iteration for the
eigenvectors, of the complex symmetric 1D pencils
G = D^-1/2 (T - i (k/h) E - (k^2/2) D) D^-1/2 of Theorem A.6's separable
mean-value block.

The header is plain C++; it is compiled here with g++ into a small shared
library (no CUDA, no GPU) and compared with numpy's dense eigen-solver
(LAPACK zgeev: an independent algorithm).  Checked: every eigenvalue
(matched one to one), the residual ||G Q - Q diag(lam)||, the bilinear
orthogonality Q^T Q = I that the preconditioner relies on (it applies Q^T as
Q^-1), and the reported condition number ||Q||_2^2 (a power-iteration
estimate from below) against numpy's cond(Q).
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2209_14740_gb300", "csrc")

HARNESS = r"""
#include "csym_eig.h"
extern "C" int eig(int n, const double* dre, const double* dim_, const double* ore, const double* oim,
                   double* lre, double* lim, double* qre, double* qim, double* orth, double* kappa) {
  using sgi::csym::cd;
  std::vector<cd> d(n), o(n > 1 ? n - 1 : 0), lam, Q;
  for (int i = 0; i < n; ++i) d[i] = cd(dre[i], dim_[i]);
  for (int i = 0; i + 1 < n; ++i) o[i] = cd(ore[i], oim[i]);
  if (!sgi::csym::tridiag_eig(n, d, o, lam, Q, orth, kappa)) return 0;
  for (int i = 0; i < n; ++i) { lre[i] = lam[i].real(); lim[i] = lam[i].imag(); }
  for (size_t i = 0; i < (size_t)n * n; ++i) { qre[i] = Q[i].real(); qim[i] = Q[i].imag(); }
  return 1;
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("csym")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    so = d / "libh.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    L.eig.restype = ctypes.c_int
    return L


def run(lib, diag, off):
    n = len(diag)
    P = ctypes.POINTER(ctypes.c_double)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in
            (diag.real, diag.imag, off.real if n > 1 else np.zeros(1), off.imag if n > 1 else np.zeros(1))]
    lre, lim = np.zeros(n), np.zeros(n)
    qre, qim = np.zeros(n * n), np.zeros(n * n)
    orth, kappa = ctypes.c_double(0), ctypes.c_double(0)
    ok = lib.eig(n, *[a.ctypes.data_as(P) for a in arrs], lre.ctypes.data_as(P), lim.ctypes.data_as(P),
                 qre.ctypes.data_as(P), qim.ctypes.data_as(P), ctypes.byref(orth), ctypes.byref(kappa))
    assert ok == 1
    return lre + 1j * lim, (qre + 1j * qim).reshape(n, n), orth.value, kappa.value


def pencil(m, h, kbar):
    """The 1D pencil of one grid direction with absorbing ends (as the
    preconditioner set-up forms it)."""
    tdiag = np.full(m, 2.0 / h ** 2)
    tdiag[0] = tdiag[-1] = 1.0 / h ** 2
    d = np.ones(m)
    d[0] = d[-1] = 0.5
    e = np.zeros(m)
    e[0] = e[-1] = 1.0
    gd = (tdiag - 0.5 * kbar ** 2 * d - 1j * (kbar / h) * e) / d
    go = (-1.0 / h ** 2) / np.sqrt(d[:-1] * d[1:]) + 0j
    return gd.astype(complex), go.astype(complex)


def check(lib, gd, go, orth_tol):
    n = len(gd)
    lam, Q, orth, kappa = run(lib, gd, go)
    G = np.diag(gd) + np.diag(go, 1) + np.diag(go, -1)
    ref = np.linalg.eigvals(G)
    scale = np.abs(ref).max()
    # one-to-one matching of the eigenvalues
    used = np.zeros(n, dtype=bool)
    for z in lam:
        dist = np.where(used, np.inf, np.abs(ref - z))
        k = int(np.argmin(dist))
        assert dist[k] <= 1e-11 * scale, (z, ref[k], dist[k] / scale)
        used[k] = True
    assert np.all(np.diff(lam.real) >= -1e-12 * scale)
    res = np.abs(G @ Q - Q * lam[None, :]).max()
    assert res <= 1e-10 * scale, res / scale
    qtq = np.abs(Q.T @ Q - np.eye(n)).max()
    assert qtq <= orth_tol and abs(orth - qtq) <= 1e-12 + 1e-3 * qtq, (orth, qtq)
    cond = np.linalg.cond(Q)
    assert 0.97 * cond <= kappa <= cond * (1 + 1e-9), (kappa, cond)
    return orth, kappa


@pytest.mark.parametrize("g,kbar", [(13, 9.0), (21, 12.0), (127, 30.0), (255, 40.0), (331, 30.0), (511, 60.0)])
def test_preconditioner_pencils(lib, g, kbar):
    h = 1.0 / (g - 1)
    gd, go = pencil(g, h, kbar)
    orth, kappa = check(lib, gd, go, 1e-11)
    assert kappa < 100.0


def test_random_complex_symmetric(lib):
    rng = np.random.default_rng(5)
    for n in (1, 2, 3, 8, 40):
        gd = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        go = rng.standard_normal(max(n - 1, 0)) + 0.3j * rng.standard_normal(max(n - 1, 0))
        if n == 1:
            lam, Q, orth, kappa = run(lib, gd, np.zeros(0, complex))
            assert abs(lam[0] - gd[0]) == 0.0 and abs(Q[0, 0] ** 2 - 1) < 1e-15
            continue
        check(lib, gd, go, 1e-8)


def test_real_symmetric_limit(lib):
    """A real symmetric tridiagonal matrix (no absorbing term): the rotations
    are real, eigenvalues real (to rounding: inverse iteration takes a
    slightly complex shift) and equal to the closed form of the Dirichlet
    second-difference matrix, 2 - 2 cos(j pi / (n+1))."""
    n = 30
    gd = np.full(n, 2.0) + 0j
    go = np.full(n - 1, -1.0) + 0j
    lam, Q, orth, kappa = run(lib, gd, go)
    exact = 2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    np.testing.assert_allclose(lam.real, exact, rtol=0, atol=1e-13)
    assert np.abs(lam.imag).max() <= 1e-14
    assert abs(kappa - 1.0) < 1e-10
