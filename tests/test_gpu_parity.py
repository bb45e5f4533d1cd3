"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (derived from the arithmetic):
* matvec FP64: each output sums <= ~25 terms, so the rounding error is at
  most ~25 u64 (|terms|) -> 1e-13 relative to the row's absolute scale.
* matvec FP32: same count with u32 = 6e-8 -> 3e-6 relative to the row scale
  (inputs rounded to complex64 first, so only arithmetic error is measured).
* preconditioner FP64: <= 1e-10 relative to SuperLU's block solve (the
  bound set for a diagonalisation variant of the block factorisation; the
  pivoted tridiagonal 1D solve and the eigenvector route, whose factors have
  |Q^T Q - I| <= 1e-10 and cond(Q) <= 100 by construction, both land near
  1e-13).
* GMRES FP64 at tol 1e-13: ||x - x*|| <= kappa(A) * relres; kappa(A) <= 6e3
  on these problems, so both the device GMRES and the oracle's CGS2 GMRES at
  the same restart and tolerance land within ~1e-12 of SuperLU (measured on
  the oracle: 3e-15 .. 1.2e-12); the bound asserted is 1e-10 against both,
  in the 2-norm and element by element (max-norm).  The true relres is
  re-computed by the oracle (FP64) and must be below 1e-12 (rounding of the
  residual itself is ~ u64 |A||x| / |b|).
* mixed: relres <= 1e-8 computed by the oracle in FP64 (the target of the
  mixed-precision path); the error against the direct solution is reported.
"""
import numpy as np
import pytest

from oracle import krylov, sg
from paper_2209_14740_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def B():
    from paper_2209_14740_gb300 import binding
    binding.load()
    return binding


def problems():
    D, A = inputs.DIRICHLET, inputs.ABSORBING
    return [
        inputs.helmholtz_1d_c1(n_unknowns=37, r=5),
        inputs.paper_1d(10.0, 0.1, 3, q=31),          # q from the Sec. 6 mesh rule at kbar = 10
        inputs.random_problem(31, dim=1, g=150, s=1, r=8, bc=(A, A, D, D)),
        inputs.random_problem(32, dim=2, g=13, s=2, r=2),
        inputs.random_problem(33, dim=2, g=11, s=3, r=3, bc=(D, D, D, D)),
        inputs.random_problem(34, dim=2, g=9, s=6, r=2),
        inputs.random_problem(35, dim=2, g=17, s=0, r=0),
        inputs.helmholtz_2d(21, 3, 3, 12.0, 0.15),
        inputs.helmholtz_2d(19, 2, 4, 8.0, 0.2),
        _dirichlet_2d(),
        _rect_2d(),
        inputs.helmholtz_2d(13, 6, 3, 10.0, 0.1),     # P = 84: the largest generated kernels (FP32 and FP64)
        inputs.helmholtz_1d_c1(),                     # the 1D workload at its size: 200 unknowns, P = 6, N = 1200
    ]


def _dirichlet_2d():
    p = inputs.helmholtz_2d(15, 2, 2, 9.0, 0.1)
    p.bc = (inputs.DIRICHLET,) * 4
    return p


def _rect_2d():
    """Non-square absorbing grid (13 x 9 nodes) with constant k_0: mx != my."""
    rng = np.random.default_rng(77)
    nx, ny, s = 13, 9, 2
    k0 = np.full(nx * ny, 7.0)
    kl = 0.8 * (2 * rng.random((s, nx * ny)) - 1)
    f = rng.standard_normal(nx * ny)
    return inputs.Problem("rect_13x9", 2, nx, ny, 1.0 / 12, (inputs.ABSORBING,) * 4, s, 3, k0, kl, f, beta=0.5)


def rand_vec(N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(N) + 1j * rng.standard_normal(N)


@pytest.mark.parametrize("idx", range(len(problems())))
def test_matvec_fp64_fp32(B, idx):
    pr = problems()[idx]
    ref = sg.assemble_problem(pr)
    op = B.SG(pr)
    N = op.N
    assert N == ref.A.shape[0]
    x = rand_vec(N, idx)
    X = torch.from_numpy(x).to(DEV)
    Y = torch.empty_like(X)
    op.matvec(X, Y, B.FP64)
    y = Y.cpu().numpy()
    yr = ref.A @ x
    scale = abs(ref.A) @ np.abs(x) + abs(ref.Lbig) @ np.abs(x)
    assert np.all(np.abs(y - yr) <= 1e-13 * scale + 1e-300), np.max(np.abs(y - yr) / scale)
    x32 = x.astype(np.complex64)
    X32 = torch.from_numpy(x32).to(DEV)
    Y32 = torch.empty_like(X32)
    op.matvec(X32, Y32, B.FP32)
    y32 = Y32.cpu().numpy().astype(np.complex128)
    yr32 = ref.A @ x32.astype(np.complex128)
    assert np.all(np.abs(y32 - yr32) <= 3e-6 * scale), np.max(np.abs(y32 - yr32) / scale)
    op.close()


def test_rhs(B):
    pr = inputs.helmholtz_2d(21, 3, 3, 12.0, 0.15)
    ref = sg.assemble_problem(pr)
    op = B.SG(pr)
    b = torch.empty(op.N, dtype=torch.complex128, device=DEV)
    op.rhs(b, B.FP64)
    np.testing.assert_array_equal(b.cpu().numpy(), ref.b)
    b32 = torch.empty(op.N, dtype=torch.complex64, device=DEV)
    op.rhs(b32, B.FP32)
    np.testing.assert_array_equal(b32.cpu().numpy(), ref.b.astype(np.complex64))


def test_rhs_point_source(B):
    """Point sources (App. A.3) are discretised by the library (sg_desc's
    point fields) and by the oracle (oracle.fd.point_source) independently;
    the two right-hand sides must agree bit for bit: odd and even q (the
    midpoint and the tie broken towards the smaller node), 1D and 2D, a
    general location, a source on an absorbing edge (weight 1/2), a
    distributed f added to it, and a source on an eliminated Dirichlet node."""
    cases = [inputs.paper_1d(50.0, 0.1, 3, q=127), inputs.paper_1d(20.0, 0.1, 2, q=30),
             inputs.wedge(63, 0.1, 2), inputs.wedge(62, 0.1, 2)]
    p = inputs.random_problem(50, dim=2, g=14, s=2, r=2)
    p.point = (0.31, 0.77)
    cases.append(p)
    p = inputs.random_problem(51, dim=2, g=14, s=2, r=2)
    p.point = (0.0, 0.42)                 # on the absorbing edge x = 0
    cases.append(p)
    p = inputs.random_problem(52, dim=2, g=12, s=1, r=2, bc=(inputs.DIRICHLET,) * 4)
    p.point = (1.0, 0.5)                  # on an eliminated Dirichlet node: no contribution
    cases.append(p)
    for pr in cases:
        ref = sg.assemble_problem(pr)
        op = B.SG(pr)
        b = torch.empty(op.N, dtype=torch.complex128, device=DEV)
        op.rhs(b, B.FP64)
        np.testing.assert_array_equal(b.cpu().numpy(), ref.b, err_msg=pr.name)
        op.close()


PREC_CASES = [0, 1, 2, 3, 7, 8, 9, 10, 12]   # 1D, 2D with constant k_0, and index 3 (k_0 varies: band LU)


@pytest.mark.parametrize("idx", PREC_CASES)
@pytest.mark.parametrize("kind", [1, 2])
def test_precond(B, idx, kind):
    pr = problems()[idx]
    ref = sg.assemble_problem(pr)
    blk = ref.S0 if kind == 1 else sg.csl_mean_block(ref, pr.beta)
    M = krylov.BlockPrecond(blk, ref.P)
    op = B.SG(pr)
    x = rand_vec(op.N, 100 + idx)
    zr = M(x)
    X = torch.from_numpy(x).to(DEV)
    Z = torch.empty_like(X)
    op.precond(X, Z, kind, B.FP64)
    z = Z.cpu().numpy()
    e64 = np.linalg.norm(z - zr) / np.linalg.norm(zr)
    print("precond case %d kind %d: FP64 error vs SuperLU %.2e" % (idx, kind, e64))
    assert e64 <= 1e-10, e64
    # in place
    op.precond(X, X, kind, B.FP64)
    assert np.linalg.norm(X.cpu().numpy() - zr) / np.linalg.norm(zr) <= 1e-10
    # FP32: forward error of a stable solve ~ kappa * u32
    x32 = x.astype(np.complex64)
    zr32 = M(x32.astype(np.complex128))
    X32 = torch.from_numpy(x32).to(DEV)
    Z32 = torch.empty_like(X32)
    op.precond(X32, Z32, kind, B.FP32)
    e32 = np.linalg.norm(Z32.cpu().numpy() - zr32) / np.linalg.norm(zr32)
    assert e32 < 2e-4, e32
    op.close()


@pytest.mark.parametrize("n_unknowns", [3000, 6000])
def test_precond_1d_long_lines(B, n_unknowns):
    """1D lines too long for the shared-memory sweep (FP64 above ~2,500
    unknowns, FP32 above ~5,000): the pivoted tridiagonal solve runs from
    global memory, out of place through the scratch vector when R = Z.
    Against SuperLU's block solve, both blocks, in and out of place.  The
    blocks grow ill-conditioned with n (kappa_1 = 1.7e6 and 7e6 for the mean
    block at 3,000 and 6,000 unknowns), so the FP32 forward error is held to
    kappa_1 u32 (measured 1.8e-3 and 5.7e-3 against bounds 0.10 and 0.42) and
    its normwise backward error ||S z - r|| / (|| |S| |z| || + ||r||) to 1e-6."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    pr = inputs.helmholtz_1d_c1(n_unknowns=n_unknowns, kbar=20.0, sigma=0.1, r=3)
    ref = sg.assemble_problem(pr)
    op = B.SG(pr)
    for kind in (1, 2):
        blk = ref.S0 if kind == 1 else sg.csl_mean_block(ref, pr.beta)
        M = krylov.BlockPrecond(blk, ref.P)
        lu = spl.splu(sp.csc_matrix(blk))
        n = blk.shape[0]
        inv = spl.LinearOperator((n, n), matvec=lambda v: lu.solve(np.asarray(v, complex).ravel()),
                                 rmatvec=lambda v: lu.solve(np.asarray(v, complex).ravel(), trans="H"), dtype=complex)
        kappa1 = spl.norm(blk, 1) * spl.onenormest(inv)
        x = rand_vec(op.N, 300 + kind)
        zr = M(x)
        X = torch.from_numpy(x).to(DEV)
        Z = torch.empty_like(X)
        op.precond(X, Z, kind, B.FP64)
        e64 = np.linalg.norm(Z.cpu().numpy() - zr) / np.linalg.norm(zr)
        op.precond(X, X, kind, B.FP64)
        e64i = np.linalg.norm(X.cpu().numpy() - zr) / np.linalg.norm(zr)
        assert e64 <= 1e-10 and e64i <= 1e-10, (e64, e64i)
        x32 = x.astype(np.complex64)
        zr32 = M(x32.astype(np.complex128))
        X32 = torch.from_numpy(x32).to(DEV)
        Z32 = torch.empty_like(X32)
        op.precond(X32, Z32, kind, B.FP32)
        e32 = np.linalg.norm(Z32.cpu().numpy() - zr32) / np.linalg.norm(zr32)
        z32 = Z32.cpu().numpy().astype(np.complex128)
        op.precond(X32, X32, kind, B.FP32)
        e32i = np.linalg.norm(X32.cpu().numpy() - zr32) / np.linalg.norm(zr32)
        bound = kappa1 * 2.0 ** -24
        print("1D n=%d kind %d: FP64 %.2e, FP32 %.2e (kappa_1 u32 = %.2e)" % (n_unknowns, kind, e64, e32, bound))
        assert e32 <= bound and e32i <= bound, (e32, e32i, bound)
        Zm = z32.reshape(ref.P, n).T
        Rm = x32.astype(np.complex128).reshape(ref.P, n).T
        back = np.linalg.norm(blk @ Zm - Rm) / (np.linalg.norm(abs(blk) @ np.abs(Zm)) + np.linalg.norm(Rm))
        assert back <= 1e-6, back
    op.close()


@pytest.mark.parametrize("idx", [7, 8, 9, 10])
@pytest.mark.parametrize("kind", [1, 2])
def test_precond_tf32(B, idx, kind):
    """The plain-TF32 apply (the preconditioner of the complex64 GMRES
    cycles): TF32 inputs carry a relative rounding of 2^-11 (the factors,
    rounded) to 2^-10 (the data, truncated by the tensor core), through four
    transforms whose eigenvector factors have condition numbers below 10, so
    the apply is within ~2e-3 of the exact block solve; 5e-3 is the bound."""
    pr = problems()[idx]
    ref = sg.assemble_problem(pr)
    blk = ref.S0 if kind == 1 else sg.csl_mean_block(ref, pr.beta)
    M = krylov.BlockPrecond(blk, ref.P)
    op = B.SG(pr)
    x32 = rand_vec(op.N, 200 + idx).astype(np.complex64)
    zr = M(x32.astype(np.complex128))
    X = torch.from_numpy(x32).to(DEV)
    Z = torch.empty_like(X)
    op.precond(X, Z, kind, B.TF32)
    e = np.linalg.norm(Z.cpu().numpy() - zr) / np.linalg.norm(zr)
    assert e < 5e-3, e
    # in place, and a second call gives the same result (a fixed operator)
    Xi = X.clone()
    op.precond(Xi, Xi, kind, B.TF32)
    assert torch.equal(Xi, Z)
    op.close()


@pytest.mark.parametrize("g", [63, 127])
def test_precond_tf32_larger_grids(B, g):
    """The plain-TF32 apply on grids with 4 and 8 K stages per transform
    (ragged last stage at 63) against the FP64 apply (a separate code path,
    checked against the oracle above), within the 5e-3 bound; a second call
    gives the same bits."""
    pr = inputs.helmholtz_2d(g, 3, 3, 30.0, 0.15)
    op = B.SG(pr)
    gen = torch.Generator(device=DEV).manual_seed(g)
    X = torch.randn(op.N, dtype=torch.complex64, device=DEV, generator=gen)
    for kind in (B.PREC_MEAN, B.PREC_CSL_MEAN):
        Zr = torch.empty(op.N, dtype=torch.complex128, device=DEV)
        op.precond(X.to(torch.complex128), Zr, kind, B.FP64)
        Zt = torch.empty_like(X)
        op.precond(X, Zt, kind, B.TF32)
        err = float(torch.linalg.vector_norm(Zt.to(torch.complex128) - Zr) / torch.linalg.vector_norm(Zr))
        assert err < 5e-3, (kind, err)
        Zt2 = torch.empty_like(X)
        op.precond(X, Zt2, kind, B.TF32)
        assert torch.equal(Zt, Zt2)
    op.close()


def test_precond_tf32_needs_the_2d_route(B):
    op = B.SG(problems()[0])     # 1D
    X = torch.zeros(op.N, dtype=torch.complex64, device=DEV)
    with pytest.raises(B.SgError) as ei:
        op.precond(X, X, B.PREC_MEAN, B.TF32)
    assert ei.value.status == B.SG_EUNSUPPORTED
    op.close()


def test_tf32_unsupported_for_varying_k0(B):
    """A 2D problem whose k_0 varies has the banded block solve (FP64, FP32),
    not the fast-diagonalisation route: SG_TF32 is refused."""
    pr = problems()[3]
    assert np.ptp(pr.k0) > 0
    op = B.SG(pr)
    assert not op.info["separable"] and not op.info["tf32_route"]
    X = torch.zeros(op.N, dtype=torch.complex64, device=DEV)
    with pytest.raises(B.SgError) as ei:
        op.precond(X, X, B.PREC_MEAN, B.TF32)
    assert ei.value.status == B.SG_EUNSUPPORTED
    op.close()


GMRES_CASES = [(0, 0, 1), (0, 0, 2), (0, 0, 0), (1, 0, 1), (7, 20, 1), (7, 20, 2), (8, 10, 1), (4, 15, 0),
               (3, 15, 1), (3, 15, 2),
               (12, 0, 1), (12, 0, 2)]


@pytest.mark.parametrize("idx,restart,prec", GMRES_CASES)
def test_gmres_fp64_against_oracle(B, idx, restart, prec):
    """FP64 GMRES to tol 1e-13 against SuperLU and against the oracle's GMRES
    with the same restart, preconditioner and tolerance: within 1e-10
    relative (2-norm and max-norm)."""
    pr = problems()[idx]
    ref = sg.assemble_problem(pr)
    xd = krylov.direct(ref.A, ref.b)
    Mo = None
    if prec:
        blk = ref.S0 if prec == 1 else sg.csl_mean_block(ref, pr.beta)
        Mo = krylov.BlockPrecond(blk, ref.P)
    tol = 1e-13
    ro = krylov.gmres(ref.A, ref.b, Mo, restart=restart or None, tol=tol, maxit=6000)
    assert ro.converged
    op = B.SG(pr)
    b = torch.from_numpy(ref.b).to(DEV)
    x = torch.zeros_like(b)
    info = op.gmres(b, x, restart=restart, tol=tol, prec=prec, mode=B.FP64, maxit=6000)
    xg = x.cpu().numpy()
    relres = np.linalg.norm(ref.b - ref.A @ xg) / np.linalg.norm(ref.b)
    rscale = np.linalg.norm(abs(ref.A) @ np.abs(xg) + np.abs(ref.b)) / np.linalg.norm(ref.b)
    e_direct = np.linalg.norm(xg - xd) / np.linalg.norm(xd)
    e_oracle = np.linalg.norm(xg - ro.x) / np.linalg.norm(ro.x)
    e_max = np.abs(xg - ro.x).max() / np.abs(ro.x).max()
    print("fp64 gmres case %d restart %d prec %d: iters %d (oracle %d) relres %.2e err vs direct %.2e "
          "vs oracle %.2e (max-norm %.2e)" % (idx, restart, prec, info["iters"], ro.iters, relres, e_direct,
                                             e_oracle, e_max))
    assert info["status"] == B.SG_OK, info
    assert info["relres"] <= tol
    assert relres <= 1e-12, relres
    assert abs(info["relres"] - relres) <= 1e-3 * relres + 1e-15 * rscale
    assert e_direct <= 1e-10 and e_oracle <= 1e-10 and e_max <= 1e-10, (e_direct, e_oracle, e_max)
    assert abs(info["iters"] - ro.iters) <= max(2, ro.iters // 20), (info["iters"], ro.iters)
    op.close()


@pytest.mark.parametrize("idx,restart,prec", [(0, 0, 1), (7, 20, 1), (7, 20, 2), (8, 10, 1), (2, 40, 1), (4, 0, 0)])
def test_gmres_mixed_reaches_1e8(B, idx, restart, prec):
    pr = problems()[idx]
    ref = sg.assemble_problem(pr)
    xd = krylov.direct(ref.A, ref.b)
    op = B.SG(pr)
    b = torch.from_numpy(ref.b).to(DEV)
    x = torch.zeros_like(b)
    info = op.gmres(b, x, restart=restart, tol=1e-8, prec=prec, mode=B.MIXED, maxit=20000)
    xg = x.cpu().numpy()
    relres = np.linalg.norm(ref.b - ref.A @ xg) / np.linalg.norm(ref.b)
    err = np.linalg.norm(xg - xd) / np.linalg.norm(xd)
    print("mixed case %d: relres %.3e err vs direct %.3e iters %d outer %d" % (idx, relres, err, info["iters"],
                                                                             info["outer"]))
    assert info["status"] == B.SG_OK, info
    assert relres <= 1e-8
    assert abs(info["relres"] - relres) <= 1e-3 * relres + 1e-14
    op.close()


def test_gmres_fp32_mode(B):
    pr = problems()[7]
    ref = sg.assemble_problem(pr)
    op = B.SG(pr)
    b = torch.from_numpy(ref.b.astype(np.complex64)).to(DEV)
    x = torch.zeros_like(b)
    info = op.gmres(b, x, restart=20, tol=1e-5, prec=B.PREC_MEAN, mode=B.FP32)
    xg = x.cpu().numpy().astype(np.complex128)
    relres = np.linalg.norm(ref.b - ref.A @ xg) / np.linalg.norm(ref.b)
    assert info["status"] == B.SG_OK and relres < 2e-5, (info, relres)
    op.close()


def test_gmres_edge_cases(B):
    pr = problems()[7]
    ref = sg.assemble_problem(pr)
    xd = krylov.direct(ref.A, ref.b)
    op = B.SG(pr)
    b = torch.from_numpy(ref.b).to(DEV)
    # exact initial guess: zero iterations
    x0 = torch.from_numpy(xd).to(DEV)
    x = torch.zeros_like(b)
    info = op.gmres(b, x, restart=20, tol=1e-8, prec=B.PREC_MEAN, mode=B.FP64, x0=x0)
    assert info["iters"] == 0 and info["status"] == B.SG_OK
    # zero right-hand side: x = 0
    z = torch.zeros_like(b)
    x.fill_(1.0)
    info = op.gmres(z, x, restart=20, tol=1e-8, prec=B.PREC_MEAN, mode=B.FP64)
    assert info["status"] == B.SG_OK and float(x.abs().max()) == 0.0
    # maxit too small: not converged, best iterate returned
    x = torch.zeros_like(b)
    info = op.gmres(b, x, restart=20, tol=1e-12, prec=B.PREC_NONE, mode=B.FP64, maxit=3)
    assert info["status"] == B.SG_ENOTCONV and info["iters"] == 3
    # restart 1 still converges (slowly) with the mean-value preconditioner
    x = torch.zeros_like(b)
    info = op.gmres(b, x, restart=1, tol=1e-6, prec=B.PREC_MEAN, mode=B.FP64, maxit=5000)
    assert info["status"] == B.SG_OK
    # NaN right-hand side is rejected
    bn = b.clone()
    bn[3] = float("nan")
    with pytest.raises(B.SgError) as ei:
        op.gmres(bn, x, restart=20, tol=1e-8, prec=B.PREC_MEAN, mode=B.FP64)
    assert ei.value.status == B.SG_EINVAL
    # host buffers (host_io) give the same answer as device buffers
    bh = ref.b.copy()
    xh = np.zeros_like(bh)
    info_h = op.gmres(bh, xh, restart=20, tol=1e-10, prec=B.PREC_MEAN, mode=B.FP64, host_io=True)
    xdev = torch.zeros_like(b)
    info_d = op.gmres(b, xdev, restart=20, tol=1e-10, prec=B.PREC_MEAN, mode=B.FP64)
    assert info_h["iters"] == info_d["iters"]
    np.testing.assert_array_equal(xh, xdev.cpu().numpy())
    op.close()


def test_assemble_rejects_bad_input(B):
    pr = inputs.random_problem(40, dim=2, g=9, s=2, r=2)
    pr.kl = pr.kl * 50.0          # k(x, xi) < 0 for some xi
    with pytest.raises(B.SgError) as ei:
        B.SG(pr)
    assert ei.value.status == B.SG_EINVAL
    pr = inputs.random_problem(41, dim=2, g=9, s=2, r=2)
    pr.k0[5] = float("nan")
    with pytest.raises(B.SgError):
        B.SG(pr)
    pr = inputs.random_problem(42, dim=2, g=9, s=2, r=2, bc=(1, 0, 1, 1))
    with pytest.raises(B.SgError):
        B.SG(pr)


def test_complex_symmetry_property_fp64(B):
    """A^T = A (Theorem 3.4): x^T (A y) = y^T (A x) for random x, y."""
    pr = inputs.helmholtz_2d(61, 4, 3, 20.0, 0.15)
    op = B.SG(pr)
    x = torch.from_numpy(rand_vec(op.N, 1)).to(DEV)
    y = torch.from_numpy(rand_vec(op.N, 2)).to(DEV)
    Ax = torch.empty_like(x)
    Ay = torch.empty_like(y)
    op.matvec(x, Ax, B.FP64)
    op.matvec(y, Ay, B.FP64)
    lhs = complex((x * Ay).sum())
    rhs = complex((y * Ax).sum())
    assert abs(lhs - rhs) <= 1e-12 * float((x.abs() * Ay.abs()).sum())
    op.close()
