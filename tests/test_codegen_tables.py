"""CPU checks of the tables the generated operator kernels are emitted from
(paper_2209_14740_gb300/codegen_matvec.py) against the oracle's Galerkin
matrices (oracle/pc.py, closed-form Legendre moments, Lemma 3.2 products).

The kernels apply the coupling as W = T_k X over degree <= r + 1 followed by
T_k^T W; for the model k = k_0 + sum_l xi_l k_l this must give
<k phi_a phi_b> = (T_k)_ab (a, b of degree <= r) and <k^2 phi_a phi_b> =
(T_k^T T_k)_ab.  Both sides are built here from random k_0, k_l and compared
entry by entry, for every (s, r) with a generated kernel."""
import numpy as np
import pytest

from oracle import pc
from paper_2209_14740_gb300 import codegen_matvec as cg


def _tk_matrix(s, r, k0, kl):
    idx, rows = cg._tk_rows(s, r)
    coef = {"k0": k0}
    for l in range(s):
        for n in range(1, r + 2):
            coef["kb%d_%d" % (l + 1, n)] = kl[l] * cg._b(n)
    T = np.zeros((len(rows), len(idx)))
    gms = []
    for gi, (gm, terms) in enumerate(rows):
        gms.append(gm)
        for name, b in terms:
            T[gi, b] += coef[name]
    return idx, gms, T


@pytest.mark.parametrize("s,r", cg.SPECIALISED)
def test_factorised_coupling_matches_galerkin_tables(s, r):
    # the generator's mode order is the oracle's (graded, descending lex)
    al = [tuple(int(v) for v in row) for row in pc.multi_indices(s, r)]
    assert cg._multi_indices(s, r) == al
    rng = np.random.default_rng(10 * s + r)
    k0 = 2.0 + rng.random()
    kl = 0.3 * (2 * rng.random(s) - 1)
    idx, gms, T = _tk_matrix(s, r, k0, kl)
    P = len(idx)
    G1, G2 = pc.expectation_matrices(s, r)
    ref1 = k0 * np.eye(P) + sum(kl[l] * G1[l] for l in range(s))
    ref2 = k0 * k0 * np.eye(P) + 2 * k0 * sum(kl[l] * G1[l] for l in range(s))
    for l in range(s):
        for lp in range(s):
            ref2 = ref2 + kl[l] * kl[lp] * G2[(min(l, lp), max(l, lp))]
    # rows of degree <= r, in the generator's order, are the first P rows
    rows_low = [gi for gi, gm in enumerate(gms) if gm in idx]
    T_low = np.zeros((P, P))
    for gi in rows_low:
        T_low[idx[gms[gi]]] = T[gi]
    np.testing.assert_allclose(T_low, ref1, rtol=0, atol=1e-14)
    np.testing.assert_allclose(T.T @ T, ref2, rtol=0, atol=1e-13)


def test_every_row_of_degree_r_plus_1_feeds_degree_r_only():
    """Rows of degree r + 1 read and scatter only degree-r modes (their lower
    neighbours): the property the persistent kernel relies on when it issues
    the next tile's copies before those rows."""
    for s, r in cg.SPECIALISED:
        idx, rows = cg._tk_rows(s, r)
        inv = {i: a for a, i in idx.items()}
        for gm, terms in rows:
            if sum(gm) == r + 1:
                assert all(sum(inv[b]) == r for _, b in terms)
