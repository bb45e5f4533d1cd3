"""Seeded synthetic inputs for the stochastic Helmholtz workloads.

This module only DESCRIBES problems: grid sizes, boundary conditions, the
wavenumber model k(x, xi) = k_0(x) + sum_l xi_l k_l(x) sampled at the grid
nodes (Sec. 2.2 of Pulch & Sete), the source f at the nodes, the chaos
degree.  It contains none of the method's arithmetic (no finite-difference
weights, no Galerkin products, no solves), so both the CUDA path and the
CPU oracle consume its records.

Workload recipes (all deterministic; the random ones draw from
numpy.random.default_rng(seed)):

* ``helmholtz_1d_c1``: [0, 1], 201 nodes (h = 1/200, 200 unknowns after the
  Dirichlet node x = 0 is removed), Dirichlet at x = 0, absorbing at x = 1,
  k = kbar (1 + sigma xi), kbar = 20, sigma = 0.1, one variable, degree 5
  (P = 6), f = 1.  System size 1200.
* ``helmholtz_2d``: unit square, g x g nodes including the boundary
  (h = 1/(g-1)), absorbing on all sides, s cosine modes
  k = kbar (1 + sigma sum_l sqrt(lam_l) psi_l(x) xi_l),
  psi_l = cos(l pi x) cos(l pi y), lam_l = l^-2 (or the correlation-length
  law 1 / (1 + (pi lc l)^2)), Gaussian source of width 0.02 and unit mass
  centred at (x_s, y_s).
  - 127 x 127, s = 3, kbar = 30, sigma = 0.15, degree 3 (P = 20): 322,580
    unknowns.
  - 511 x 511, s = 6, kbar = 60, sigma = 0.1, degree 3 (P = 84): 21,934,164
    unknowns.
* ``batch_64``: 64 problems with g ~ U{63..255}, kbar ~ U[10, 40],
  sigma ~ U[0.05, 0.2], s ~ U{2, 3, 4}, degree ~ U{2, 3}.
* ``paper_1d``: the 1D experiment of Sec. 6 (absorbing at both ends, unit
  point source at x = 1/2, k = (1 + theta xi) kbar) on q interior nodes; the
  caller picks q (Sec. 6 takes it from its mesh rule with maxk = kbar, e.g.
  q = 127 for kbar = 50).
* ``wedge``: the 2D experiment of Sec. 7 (three layers with k_1 = 30,
  k_2 = 15, k_3 = 20, theta = 0.1, unit point source at the centre).

Point sources are described by their location only (``Problem.point``); each
consumer discretises the Dirac distribution itself (App. A.3).
* ``random_problem``: small random positive fields for parity tests.

The paper measures on analytic workloads only (no dataset); these recipes
stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import pi

import numpy as np

DIRICHLET = 0
ABSORBING = 1


@dataclass
class Problem:
    name: str
    dim: int
    nx: int
    ny: int
    h: float
    bc: tuple            # (left, right, bottom, top)
    s: int
    r: int
    k0: np.ndarray       # (nx*ny,) float64, x fastest
    kl: np.ndarray       # (s, nx*ny) float64
    f: np.ndarray        # (nx*ny,) float64
    beta: float = 0.5
    meta: dict = field(default_factory=dict)
    point: tuple | None = None   # location of a unit point source delta(x - a), added to f

    @property
    def nodes(self) -> int:
        return self.nx * self.ny


def _grid_xy(g: int):
    x = np.linspace(0.0, 1.0, g)
    X, Y = np.meshgrid(x, x, indexing="xy")     # row = y, column = x -> x fastest
    return X.reshape(-1), Y.reshape(-1)


def gaussian_source(g: int, xs: float = 0.5, ys: float = 0.5, w: float = 0.02) -> np.ndarray:
    X, Y = _grid_xy(g)
    return np.exp(-((X - xs) ** 2 + (Y - ys) ** 2) / (2 * w * w)) / (2 * pi * w * w)


def helmholtz_1d_c1(n_unknowns: int = 200, kbar: float = 20.0, sigma: float = 0.1, r: int = 5) -> Problem:
    nx = n_unknowns + 1
    h = 1.0 / n_unknowns
    k0 = np.full(nx, kbar)
    kl = np.full((1, nx), kbar * sigma)
    f = np.ones(nx)
    return Problem("helmholtz_1d_n%d_P%d" % (n_unknowns, r + 1), 1, nx, 1, h,
                   (DIRICHLET, ABSORBING, DIRICHLET, DIRICHLET), 1, r, k0, kl, f,
                   meta=dict(kbar=kbar, sigma=sigma))


def helmholtz_2d(g: int = 127, s: int = 3, r: int = 3, kbar: float = 30.0, sigma: float = 0.15,
                 lc: float | None = None, xs: float = 0.5, ys: float = 0.5, width: float = 0.02,
                 beta: float = 0.5) -> Problem:
    X, Y = _grid_xy(g)
    k0 = np.full(g * g, kbar)
    kl = np.zeros((s, g * g))
    for l in range(1, s + 1):
        lam = l ** -2.0 if lc is None else 1.0 / (1.0 + (pi * lc * l) ** 2)
        kl[l - 1] = kbar * sigma * np.sqrt(lam) * np.cos(l * pi * X) * np.cos(l * pi * Y)
    f = gaussian_source(g, xs, ys, width)
    return Problem("helmholtz_2d_g%d_s%d_r%d" % (g, s, r), 2, g, g, 1.0 / (g - 1),
                   (ABSORBING,) * 4, s, r, k0, kl, f, beta=beta,
                   meta=dict(kbar=kbar, sigma=sigma, lc=lc, xs=xs, ys=ys))


def config_2d_127() -> Problem:
    return helmholtz_2d(127, 3, 3, 30.0, 0.15)


def config_2d_511() -> Problem:
    return helmholtz_2d(511, 6, 3, 60.0, 0.1)


def batch_64(seed: int = 20220932, count: int = 64, gmin: int = 63, gmax: int = 255) -> list[Problem]:
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        g = int(rng.integers(gmin, gmax + 1))
        kbar = float(rng.uniform(10.0, 40.0))
        sigma = float(rng.uniform(0.05, 0.2))
        s = int(rng.integers(2, 5))
        r = int(rng.integers(2, 4))
        out.append(helmholtz_2d(g, s, r, kbar, sigma))
    return out


def warmstart_params(seed: int, count: int) -> np.ndarray:
    """(kbar, sigma, lc, x_s, y_s) uniform in [10,40] x [0.05,0.2] x [0.1,0.5]
    x [0.2,0.8]^2."""
    rng = np.random.default_rng(seed)
    lo = np.array([10.0, 0.05, 0.1, 0.2, 0.2])
    hi = np.array([40.0, 0.2, 0.5, 0.8, 0.8])
    return lo + (hi - lo) * rng.random((count, 5))


def warmstart_problem(p, g: int = 127, s: int = 3, r: int = 3) -> Problem:
    kbar, sigma, lc, xs, ys = (float(v) for v in p)
    return helmholtz_2d(g, s, r, kbar, sigma, lc=lc, xs=xs, ys=ys)


def paper_1d(kbar: float, theta: float, m: int, q: int, beta: float = 0.5) -> Problem:
    nx = q + 2
    h = 1.0 / (q + 1)
    k0 = np.full(nx, kbar)
    kl = np.full((1, nx), theta * kbar)
    return Problem("paper_1d_k%g_t%g_m%d_q%d" % (kbar, theta, m, q), 1, nx, 1, h,
                   (ABSORBING, ABSORBING, DIRICHLET, DIRICHLET), 1, m, k0, kl, np.zeros(nx), beta=beta,
                   meta=dict(kbar=kbar, theta=theta, q=q), point=(0.5,))


def wedge(q: int = 127, theta: float = 0.1, r: int = 3, k=(30.0, 15.0, 20.0), beta: float = 0.5) -> Problem:
    g = q + 2
    X, Y = _grid_xy(g)
    reg1 = Y <= 0.2 + 0.1 * X
    reg3 = Y >= 0.6 - 0.2 * X
    reg2 = ~reg1 & ~reg3
    regs = [reg1, reg2, reg3]
    k0 = np.zeros(g * g)
    kl = np.zeros((3, g * g))
    for l in range(3):
        k0[regs[l]] = k[l]
        kl[l, regs[l]] = theta * k[l]
    return Problem("wedge_q%d_t%g_r%d" % (q, theta, r), 2, g, g, 1.0 / (q + 1),
                   (ABSORBING,) * 4, 3, r, k0, kl, np.zeros(g * g), beta=beta, meta=dict(theta=theta),
                   point=(0.5, 0.5))


def random_problem(seed: int, dim: int = 2, g: int = 12, s: int = 2, r: int = 2,
                   bc=None, kbar: float = 8.0, spread: float = 0.25) -> Problem:
    """Random smooth-ish positive fields: k_0 in kbar*[1, 1.3], each k_l with
    |k_l| <= spread*kbar/s so that k > 0 for all xi in [-1, 1]^s."""
    rng = np.random.default_rng(seed)
    nx = g
    ny = g if dim == 2 else 1
    n = nx * ny
    if bc is None:
        bc = (ABSORBING,) * 4 if dim == 2 else (ABSORBING, ABSORBING, DIRICHLET, DIRICHLET)
    k0 = kbar * (1.0 + 0.3 * rng.random(n))
    kl = (spread * kbar / max(s, 1)) * (2.0 * rng.random((s, n)) - 1.0)
    f = rng.standard_normal(n)
    return Problem("random_d%d_g%d_s%d_r%d_%d" % (dim, g, s, r, seed), dim, nx, ny,
                   1.0 / (g - 1), tuple(bc), s, r, k0, kl, f, beta=0.5)
