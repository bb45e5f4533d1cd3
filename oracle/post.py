"""Post-processing of a stochastic Galerkin solution (oracle; test
infrastructure only).

With the orthonormal chaos basis (E[phi_i phi_j] = delta_ij, phi_0 = 1,
Sec. 2.3), the SG approximation u~(x, xi) = sum_i V_i(x) phi_i(xi) has
* expected value E[u~](x) = V_0(x);
* variances of its real and imaginary parts
  Var[Re u~](x) = sum_{i >= 1} (Re V_i(x))^2,
  Var[Im u~](x) = sum_{i >= 1} (Im V_i(x))^2
  (the two quantities the paper plots in Sec. 7);
* per total degree j the largest maximum norm of a coefficient vector,
  gamma_j = max { ||V_i||_inf : deg(phi_i) = j }   (Sec. 7).

Pins: tests/test_oracle_post.py (mean and variances against tensor
Gauss-Legendre quadrature of the polynomial u~(x, xi) itself, evaluated with
numpy's Legendre module; theta = 0 makes every mode i >= 1 vanish, so the
variance and gamma_j, j >= 1, are zero; gamma_j by brute force over the
multi-indices).
"""
from __future__ import annotations

import numpy as np

from . import pc


def mean(V: np.ndarray) -> np.ndarray:
    """E[u~] = V_0 for V of shape (P, n)."""
    return np.asarray(V)[0].copy()


def variances(V: np.ndarray):
    """(Var[Re u~], Var[Im u~]) at every grid unknown."""
    V = np.asarray(V)
    return (V[1:].real ** 2).sum(axis=0), (V[1:].imag ** 2).sum(axis=0)


def gamma(V: np.ndarray, s: int, r: int) -> np.ndarray:
    """gamma_j, j = 0..r: the largest ||V_i||_inf over the modes of total degree j."""
    V = np.asarray(V)
    deg = pc.multi_indices(s, r).sum(axis=1) if s > 0 else np.zeros(1, dtype=int)
    out = np.zeros(r + 1)
    for i in range(V.shape[0]):
        out[deg[i]] = max(out[deg[i]], np.abs(V[i]).max())
    return out
