"""Polynomial chaos basis and Galerkin triple products (oracle; test
infrastructure only).

Paper sections followed:
* Sec. 2.2: independent xi_l ~ U[-1, 1], joint density rho = 2^-s.
* Sec. 2.3: orthonormal multivariate Legendre basis, phi_0 = 1, all
  multi-indices of total degree <= r, count P = (s+r)! / (s! r!).
* Lemma 3.2: Galerkin entries <a phi_i, phi_j> are symmetric in i, j.
* Lemma A.3: a coefficient of degree d in xi couples only modes whose
  degrees differ by at most d.

Basis order (the paper does not fix one): graded, and within one total
degree the multi-indices (alpha_1, ..., alpha_s) are sorted in DESCENDING
lexicographic order, so for s = 3, degree 1 reads e_1, e_2, e_3.

Triple products use the three-term recurrence of the orthonormal Legendre
polynomials p_n = sqrt(2n+1) P_n under the density 1/2 on [-1, 1]:
    xi p_n = b_{n+1} p_{n+1} + b_n p_{n-1},   b_n = n / sqrt(4 n^2 - 1),
so that E[xi p_a p_b] = b_{max(a,b)} when |a - b| = 1 and 0 otherwise, and
E[xi^2 p_a p_b] = (xi p_a, xi p_b) expanded with the same recurrence.

Pins (tests/test_oracle_pc.py): basis size against the closed form and the
n.basis column of Table 2; every triple product against Gauss-Legendre
quadrature of Legendre polynomials evaluated by numpy (an independent
evaluation route); the bandwidth statement of Lemma A.3; symmetry.
"""
from __future__ import annotations

from math import comb, sqrt

import numpy as np


def num_modes(s: int, r: int) -> int:
    """P = (s+r)! / (s! r!)  (Sec. 2.3, count of basis polynomials)."""
    return comb(s + r, s)


def multi_indices(s: int, r: int) -> np.ndarray:
    """All alpha in N_0^s with |alpha| <= r, graded, descending lex within a
    degree.  Row 0 is the zero multi-index (phi_0 = 1, Sec. 2.3)."""
    out = []
    for d in range(r + 1):
        level = []

        def rec(prefix, left, slots):
            if slots == 1:
                level.append(prefix + [left])
                return
            for a in range(left, -1, -1):
                rec(prefix + [a], left - a, slots - 1)

        if s == 0:
            if d == 0:
                level.append([])
        else:
            rec([], d, s)
        out.extend(level)
    return np.array(out, dtype=np.int64).reshape(len(out), s)


def legendre_b(n: int) -> float:
    """Recurrence coefficient b_n = n / sqrt(4n^2 - 1) of the orthonormal
    Legendre polynomials (b_0 = 0)."""
    if n <= 0:
        return 0.0
    return n / sqrt(4.0 * n * n - 1.0)


def e_xi(a: int, b: int) -> float:
    """E[xi p_a(xi) p_b(xi)] for one uniform variable."""
    if abs(a - b) != 1:
        return 0.0
    return legendre_b(max(a, b))


def e_xi2(a: int, b: int) -> float:
    """E[xi^2 p_a p_b] = sum_c E[xi p_a p_c] E[xi p_c p_b] (Parseval over
    the complete basis; only c = a +- 1 contribute)."""
    tot = 0.0
    for c in (a - 1, a + 1):
        if c >= 0:
            tot += e_xi(a, c) * e_xi(c, b)
    return tot


def delta(a: int, b: int) -> float:
    return 1.0 if a == b else 0.0


def galerkin_first(s: int, r: int) -> list[np.ndarray]:
    """G_l[i, j] = <xi_l phi_i, phi_j>, l = 1..s (returned 0-based), dense
    P x P.  Product over variables of the 1D moments (independence,
    Sec. 2.2)."""
    al = multi_indices(s, r)
    P = len(al)
    mats = []
    for l in range(s):
        G = np.zeros((P, P))
        for i in range(P):
            for j in range(P):
                v = 1.0
                for t in range(s):
                    if t == l:
                        v *= e_xi(al[i, t], al[j, t])
                    else:
                        v *= delta(al[i, t], al[j, t])
                    if v == 0.0:
                        break
                G[i, j] = v
        mats.append(G)
    return mats


def galerkin_second(s: int, r: int) -> dict[tuple[int, int], np.ndarray]:
    """G_{l,l'}[i, j] = <xi_l xi_l' phi_i, phi_j> for 0 <= l <= l' < s."""
    al = multi_indices(s, r)
    P = len(al)
    out = {}
    for l in range(s):
        for lp in range(l, s):
            G = np.zeros((P, P))
            for i in range(P):
                for j in range(P):
                    v = 1.0
                    for t in range(s):
                        a, b = al[i, t], al[j, t]
                        if t == l and t == lp:
                            v *= e_xi2(a, b)
                        elif t == l or t == lp:
                            v *= e_xi(a, b)
                        else:
                            v *= delta(a, b)
                        if v == 0.0:
                            break
                    G[i, j] = v
            out[(l, lp)] = G
    return out


def expectation_matrices(s: int, r: int):
    """The Galerkin matrices of the wavenumber model k = k_0 + sum_l xi_l k_l
    (Sec. 2.2):

        <k phi_i, phi_j>   = k_0 I + sum_l k_l G_l
        <k^2 phi_i, phi_j> = k_0^2 I + 2 k_0 sum_l k_l G_l
                             + sum_{l, l'} k_l k_l' G_{l,l'}

    Returned as (G_first list, G_second dict) so callers combine them with
    their node fields."""
    return galerkin_first(s, r), galerkin_second(s, r)
