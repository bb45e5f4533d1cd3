"""CPU test of the banded LU phases (paper_2209_14740_gb300/csrc/band_core.h).

The device factorisation and solves run these per-thread phases between
barriers.  Here the same header is compiled as plain C++ and driven the way
the kernels drive it (phases in order, every thread of a phase run before the
next phase, a sliding window of rows in a scratch array, several groups of
right-hand sides), on random complex banded matrices, against SciPy (LU of
the dense matrix; the pivots may differ, the solution may not).  Checked:
factors and solutions, rows and columns at the band's edges, right-hand-side
groups that do not fill the last group, in-place use (R = Y = Z), a
diagonally dominant matrix (no row swaps) and one that needs many.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg as sl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2209_14740_gb300", "csrc")

HARNESS = r"""
#include <vector>
#include <cstring>
#include <algorithm>
struct d2 { double x, y; };
#include "band_core.h"
using namespace sgi::band;

// factor: emulates k_band_factor with nt threads
extern "C" int factor(int n, int kl, int ku, d2* ab, int* piv, int nt) {
  const int kv = kl + ku, ldab = 2 * kl + ku + 1;
  std::vector<d2> lcol(kl + 1), urow(kl + ku + 1);
  int bad = 0;
  for (int j = 0; j < n; ++j) {
    const int last = std::min(n - 1, j + kl), clast = std::min(n - 1, j + kv);
    double best = -1; int row = j;
    for (int t = 0; t < nt; ++t) {
      double b; int r;
      pivot_candidates(ab, kv, ldab, j, last, t, nt, &b, &r);
      if (b > best || (b == best && r < row)) { best = b; row = r; }
    }
    piv[j] = row;
    if (!(best > 0)) bad = 1;
    for (int t = 0; t < nt; ++t) swap_rows(ab, kv, ldab, j, row, clast, t, nt);
    d2 d = ab[at(kv, ldab, j, j)];
    double den = d.x * d.x + d.y * d.y;
    if (!(den > 0)) { bad = 1; den = 1e-300; }
    d2 rinv{d.x / den, -d.y / den};
    for (int t = 0; t < nt; ++t) multipliers(ab, kv, ldab, j, last, clast, rinv, lcol.data(), urow.data(), t, nt);
    for (int t = 0; t < nt; ++t) rank1_update(ab, kv, ldab, j, last, clast, lcol.data(), urow.data(), t, nt);
  }
  return bad;
}

// solve: emulates k_band_solve (forward then backward sweep) for nrhs
// right-hand sides in groups of pc, nt threads; R, Y, Z may alias.
extern "C" void solve(int n, int kl, int ku, const d2* ab, const int* piv, int nrhs, int pc, const d2* R, d2* Y,
                      d2* Z, long long ld, int nt) {
  const int kv = kl + ku, ldab = 2 * kl + ku + 1;
  for (int q0 = 0; q0 < nrhs; q0 += pc) {
    const int pcb = std::min(pc, nrhs - q0);
    std::vector<d2> win((size_t)(kv + 1) * pcb);
    const int W1 = kl + 1;
    const int first = std::min(kl, n - 1);
    for (int r = 0; r <= first; ++r)
      for (int q = 0; q < pcb; ++q) win[(size_t)(r % W1) * pcb + q] = R[(long long)(q0 + q) * ld + r];
    std::vector<d2> fcol(kv + 1);
    for (int j = 0; j < n; ++j) {
      for (int t = 0; t < nt; ++t) fwd_swap(win.data(), W1, pcb, j, piv[j], t);
      for (int ii = 0; ii < kl; ++ii) fcol[ii] = (j + 1 + ii < n) ? ab[at(kv, ldab, j + 1 + ii, j)] : d2{0, 0};
      for (int t = 0; t < nt; ++t) fwd_update(win.data(), W1, pcb, fcol.data(), j, n, kl, t, nt, Y, ld, q0);
      if (j + kl + 1 < n)
        for (int q = 0; q < pcb; ++q) win[(size_t)(j % W1) * pcb + q] = R[(long long)(q0 + q) * ld + j + kl + 1];
    }
    const int W2 = kv + 1;
    for (int r = n - 1; r >= std::max(0, n - 1 - kv); --r)
      for (int q = 0; q < pcb; ++q) win[(size_t)(r % W2) * pcb + q] = Y[(long long)(q0 + q) * ld + r];
    for (int j = n - 1; j >= 0; --j) {
      const d2* col = ab + (long long)j * ldab;      // band column j as stored
      d2 d = col[kv];
      double den = d.x * d.x + d.y * d.y;
      d2 dinv{d.x / den, -d.y / den};
      for (int t = 0; t < nt; ++t) bwd_update(win.data(), W2, pcb, col, dinv, j, kv, t, nt, Z, ld, q0);
      if (j - kv - 1 >= 0)
        for (int q = 0; q < pcb; ++q) win[(size_t)(j % W2) * pcb + q] = Y[(long long)(q0 + q) * ld + j - kv - 1];
    }
  }
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("band")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    so = d / "libh.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    L.factor.restype = ctypes.c_int
    return L


def to_band(A, kl, ku):
    n = A.shape[0]
    kv = kl + ku
    ldab = 2 * kl + ku + 1
    ab = np.zeros((n, ldab), dtype=complex)          # column-major: ab[c, kv + i - c]
    for c in range(n):
        for i in range(max(0, c - ku), min(n, c + kl + 1)):
            ab[c, kv + i - c] = A[i, c]
    return ab


def run(lib, A, kl, ku, R, pc, nt, inplace=False):
    n = A.shape[0]
    ab = np.ascontiguousarray(to_band(A, kl, ku))
    piv = np.zeros(n, dtype=np.int32)
    P = ctypes.c_void_p
    bad = lib.factor(n, kl, ku, P(ab.ctypes.data), P(piv.ctypes.data), nt)
    nrhs = R.shape[1]
    Rm = np.ascontiguousarray(R.T)                    # rhs q at q * n
    if inplace:
        Y = Z = Rm
    else:
        Y = np.zeros_like(Rm)
        Z = np.zeros_like(Rm)
    lib.solve(n, kl, ku, P(ab.ctypes.data), P(piv.ctypes.data), nrhs, pc, P(Rm.ctypes.data), P(Y.ctypes.data),
              P(Z.ctypes.data), ctypes.c_longlong(n), nt)
    return bad, piv, Z.T.copy()


def rand_band(rng, n, kl, ku, dominant=False):
    A = np.zeros((n, n), dtype=complex)
    for d in range(-kl, ku + 1):
        m = n - abs(d)
        v = rng.standard_normal(m) + 1j * rng.standard_normal(m)
        A += np.diag(v, d)
    if dominant:
        A += np.diag(np.full(n, 4.0 * (kl + ku + 1)))
    return A


@pytest.mark.parametrize("n,kl,ku,nrhs,pc,nt", [(40, 3, 2, 5, 2, 8), (57, 7, 7, 9, 4, 32), (33, 1, 1, 3, 3, 4),
                                                (64, 12, 5, 1, 1, 64), (20, 19, 19, 4, 3, 16), (80, 9, 9, 11, 4, 64)])
def test_factor_and_solve_against_scipy(lib, n, kl, ku, nrhs, pc, nt):
    rng = np.random.default_rng(n + 100 * kl + ku)
    A = rand_band(rng, n, kl, ku)
    R = rng.standard_normal((n, nrhs)) + 1j * rng.standard_normal((n, nrhs))
    bad, piv, X = run(lib, A, kl, ku, R, pc, nt)
    assert bad == 0
    assert np.all(piv >= np.arange(n)) and np.all(piv <= np.arange(n) + kl)
    ref = np.linalg.solve(A, R)
    err = np.linalg.norm(X - ref) / np.linalg.norm(ref)
    assert err < 1e-11 * np.linalg.cond(A), (err, np.linalg.cond(A))
    # in place (R = Y = Z) gives the same bits
    _, _, Xi = run(lib, A, kl, ku, R, pc, nt, inplace=True)
    np.testing.assert_array_equal(Xi, X)


def test_no_swaps_on_a_diagonally_dominant_matrix(lib):
    rng = np.random.default_rng(1)
    A = rand_band(rng, 50, 4, 4, dominant=True)
    R = rng.standard_normal((50, 2)) + 0j
    bad, piv, X = run(lib, A, 4, 4, R, 2, 16)
    assert np.all(piv == np.arange(50))
    np.testing.assert_allclose(X, np.linalg.solve(A, R), rtol=0, atol=1e-13)


def test_swaps_on_a_matrix_that_needs_them(lib):
    """Zero diagonal: every step must pivot (SciPy's LU agrees on the
    solution)."""
    rng = np.random.default_rng(2)
    n, kl, ku = 30, 2, 2
    A = rand_band(rng, n, kl, ku)
    np.fill_diagonal(A, 0.0)
    R = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
    bad, piv, X = run(lib, A, kl, ku, R, 2, 8)
    assert bad == 0 and np.count_nonzero(piv != np.arange(n)) > n // 2
    lu, p = sl.lu_factor(A)
    ref = sl.lu_solve((lu, p), R)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) < 1e-10


def test_singular_matrix_is_flagged(lib):
    n = 12
    A = rand_band(np.random.default_rng(3), n, 2, 2)
    A[:, 5] = 0.0
    bad, _, _ = run(lib, A, 2, 2, np.ones((n, 1), dtype=complex), 1, 4)
    assert bad == 1
