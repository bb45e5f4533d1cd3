"""Parity at the full workload sizes, in the configuration bench.py times.

* 127 x 127, s = 3, degree 3 (322,580 unknowns): the oracle assembles the
  explicit SG matrix, so matvec and preconditioner are compared element by
  element, and the GMRES solutions are checked by the oracle's FP64 residual.
* 511 x 511, s = 6, degree 3 (21.9 M unknowns): the explicit matrix does not
  fit the oracle, so matvec outputs are compared on sampled rows the oracle
  evaluates one by one (oracle.sg.apply_rows), the preconditioner by the
  residual of the n x n block S(xi_bar) on sampled modes, and the solve by
  its FP64 residual (properties that hold at any size).
"""
import numpy as np
import pytest

from oracle import fd, krylov, sg
from paper_2209_14740_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def B():
    from paper_2209_14740_gb300 import binding
    binding.load()
    return binding


@pytest.fixture(scope="module")
def cfg127():
    pr = inputs.config_2d_127()
    return pr, sg.assemble_problem(pr)


def test_127_matvec_and_precond(B, cfg127):
    pr, ref = cfg127
    op = B.SG(pr)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)
    X = torch.from_numpy(x).to(DEV)
    Y = torch.empty_like(X)
    op.matvec(X, Y, B.FP64)
    scale = abs(ref.A) @ np.abs(x) + abs(ref.Lbig) @ np.abs(x)
    assert np.all(np.abs(Y.cpu().numpy() - ref.A @ x) <= 1e-13 * scale)
    x32 = x.astype(np.complex64)
    X32 = torch.from_numpy(x32).to(DEV)
    Y32 = torch.empty_like(X32)
    op.matvec(X32, Y32, B.FP32)
    d32 = np.abs(Y32.cpu().numpy().astype(np.complex128) - ref.A @ x32.astype(np.complex128))
    assert np.all(d32 <= 3e-6 * scale)
    for kind, blk in ((B.PREC_MEAN, ref.S0), (B.PREC_CSL_MEAN, sg.csl_mean_block(ref, pr.beta))):
        zr = krylov.BlockPrecond(blk, ref.P)(x)
        Z = torch.empty_like(X)
        op.precond(X, Z, kind, B.FP64)
        e64 = np.linalg.norm(Z.cpu().numpy() - zr) / np.linalg.norm(zr)
        print("127x127 precond kind %d: FP64 error vs SuperLU %.2e" % (kind, e64))
        assert e64 <= 1e-10, e64
    op.close()


def test_127_fp64_gmres_1e13(B, cfg127):
    """FP64 GMRES(50), mean-value preconditioner, to tol 1e-13 on the 127 x 127
    workload, against the oracle's CGS2 GMRES(50) with the same preconditioner
    and tolerance (which agrees with SuperLU's direct solve of the full SG
    system to 4e-14; the direct solve itself takes minutes, so it is not
    re-run here): within 1e-10 relative, 2-norm and max-norm."""
    pr, ref = cfg127
    ro = krylov.gmres(ref.A, ref.b, krylov.BlockPrecond(ref.S0, ref.P), restart=50, tol=1e-13, maxit=2000)
    assert ro.converged
    op = B.SG(pr)
    b = torch.empty(op.N, dtype=torch.complex128, device=DEV)
    op.rhs(b, B.FP64)
    x = torch.zeros_like(b)
    info = op.gmres(b, x, restart=50, tol=1e-13, prec=B.PREC_MEAN, mode=B.FP64, maxit=2000)
    xg = x.cpu().numpy()
    relres = np.linalg.norm(ref.b - ref.A @ xg) / np.linalg.norm(ref.b)
    err = np.linalg.norm(xg - ro.x) / np.linalg.norm(ro.x)
    emax = np.abs(xg - ro.x).max() / np.abs(ro.x).max()
    print("127x127 fp64 1e-13: iters %d (oracle %d) relres %.2e err vs oracle %.2e (max-norm %.2e)"
          % (info["iters"], ro.iters, relres, err, emax))
    assert info["status"] == B.SG_OK
    assert relres <= 1e-12
    assert err <= 1e-10 and emax <= 1e-10, (err, emax)
    assert abs(info["iters"] - ro.iters) <= max(2, ro.iters // 20)
    op.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_127_gmres_bench_configuration(B, cfg127, mode):
    """The exact solve bench.py times: GMRES(50), mean-value preconditioner,
    tol 1e-8, zero initial guess."""
    pr, ref = cfg127
    op = B.SG(pr)
    b = torch.empty(op.N, dtype=torch.complex128, device=DEV)
    op.rhs(b, B.FP64)
    x = torch.zeros_like(b)
    info = op.gmres(b, x, restart=50, tol=1e-8, prec=B.PREC_MEAN, mode=B.FP64 if mode == "fp64" else B.MIXED)
    xg = x.cpu().numpy()
    relres = np.linalg.norm(ref.b - ref.A @ xg) / np.linalg.norm(ref.b)
    ro = krylov.gmres(ref.A, ref.b, krylov.BlockPrecond(ref.S0, ref.P), restart=50, tol=1e-11, maxit=500)
    err = np.linalg.norm(xg - ro.x) / np.linalg.norm(ro.x)
    print("127x127 %s: iters %d outer %d relres(oracle) %.3e err vs oracle(1e-11) %.3e"
          % (mode, info["iters"], info["outer"], relres, err))
    assert info["status"] == B.SG_OK
    assert relres <= 1e-8
    assert err < 1e-5
    op.close()


@pytest.fixture(scope="module")
def cfg511(B):
    pr = inputs.config_2d_511()
    op = B.SG(pr)
    yield pr, op
    op.close()


def test_511_matvec_sampled_rows(B, cfg511):
    pr, op = cfg511
    N = op.N
    g = torch.Generator(device=DEV).manual_seed(11)
    X32 = torch.randn(N, dtype=torch.complex64, device=DEV, generator=g)
    Y32 = torch.empty_like(X32)
    op.matvec(X32, Y32, B.FP32)
    X64 = X32.to(torch.complex128)
    Y64 = torch.empty_like(X64)
    op.matvec(X64, Y64, B.FP64)
    rng = np.random.default_rng(3)
    n = op.n
    # rows near the boundary, the corners and the interior, every mode range
    u = np.concatenate([rng.integers(0, n, 300), [0, 510, n - 1, n - 511, 511, 1022, 5 * 511 + 510]])
    a = rng.integers(0, op.P, len(u))
    a[:7] = [0, 83, 5, 40, 0, 83, 1]
    rows = a * n + u
    x = X64.cpu().numpy()
    ref = sg.apply_rows(pr, x, rows)
    scale = sg.apply_rows(pr, x, rows, absolute=True)
    y64 = Y64.cpu().numpy()[rows]
    y32 = Y32.cpu().numpy()[rows].astype(np.complex128)
    assert np.all(np.abs(y64 - ref) <= 1e-13 * scale)
    assert np.all(np.abs(y32 - ref) <= 3e-6 * scale)


def test_511_precond_block_residual(B, cfg511):
    pr, op = cfg511
    N, n, P = op.N, op.n, op.P
    grid = fd.make_grid(pr.dim, pr.nx, pr.ny, pr.h, pr.bc)
    S0 = fd.deterministic_matrix(grid, pr.k0)
    g = torch.Generator(device=DEV).manual_seed(12)
    R = torch.randn(N, dtype=torch.complex128, device=DEV, generator=g)
    Z = torch.empty_like(R)
    op.precond(R, Z, B.PREC_MEAN, B.FP64)
    R32 = R.to(torch.complex64)
    Z32 = torch.empty_like(R32)
    op.precond(R32, Z32, B.PREC_MEAN, B.FP32)
    for mode in (0, 17, 83):
        r = R[mode * n:(mode + 1) * n].cpu().numpy()
        z = Z[mode * n:(mode + 1) * n].cpu().numpy()
        res = np.linalg.norm(S0 @ z - r) / (abs(S0) @ np.abs(z) + np.abs(r)).max() / np.sqrt(n)
        assert res < 1e-12, res
        z32 = Z32[mode * n:(mode + 1) * n].cpu().numpy().astype(np.complex128)
        r32 = R32[mode * n:(mode + 1) * n].cpu().numpy().astype(np.complex128)
        res32 = np.linalg.norm(S0 @ z32 - r32) / (abs(S0) @ np.abs(z32) + np.abs(r32)).max() / np.sqrt(n)
        assert res32 < 1e-5, res32


def test_255_precond_wide_tiles(B):
    """255 x 255, s = 3, degree 3 (1.3 M unknowns): the FP32 apply takes the
    fast-diagonalisation route with 128-column tensor-core tiles in all four
    transforms (ragged in rows and columns) and odd lines, so the
    intermediates have padded even-length rows.  Checked by the residual of
    the n x n block on sampled modes and against the FP64 apply (sweeps on
    the CUDA cores, a separate code path), on two calls in a row; the
    plain-TF32 apply against the same, within its 5e-3 bound."""
    pr = inputs.helmholtz_2d(255, 3, 3, 30.0, 0.15)
    op = B.SG(pr)
    assert op.info["fast_diag"]
    N, n = op.N, op.n
    grid = fd.make_grid(pr.dim, pr.nx, pr.ny, pr.h, pr.bc)
    S0 = fd.deterministic_matrix(grid, pr.k0)
    g = torch.Generator(device=DEV).manual_seed(21)
    for call in range(2):
        R = torch.randn(N, dtype=torch.complex128, device=DEV, generator=g)
        R32 = R.to(torch.complex64)
        for kind in (B.PREC_MEAN, B.PREC_CSL_MEAN):
            Z = torch.empty_like(R)
            op.precond(R32.to(torch.complex128), Z, kind, B.FP64)
            Z32 = torch.empty_like(R32)
            op.precond(R32, Z32, kind, B.FP32)
            err = float(torch.linalg.vector_norm(Z32.to(torch.complex128) - Z) / torch.linalg.vector_norm(Z))
            assert err < 2e-4, (call, kind, err)
            Zt = torch.empty_like(R32)
            op.precond(R32, Zt, kind, B.TF32)
            errt = float(torch.linalg.vector_norm(Zt.to(torch.complex128) - Z) / torch.linalg.vector_norm(Z))
            assert errt < 5e-3, (call, kind, errt)
            if kind == B.PREC_MEAN:
                for mode in (0, 7, 19):
                    z32 = Z32[mode * n:(mode + 1) * n].cpu().numpy().astype(np.complex128)
                    r32 = R32[mode * n:(mode + 1) * n].cpu().numpy().astype(np.complex128)
                    res = np.linalg.norm(S0 @ z32 - r32) / (abs(S0) @ np.abs(z32) + np.abs(r32)).max() / np.sqrt(n)
                    assert res < 1e-5, (call, mode, res)
    op.close()


def test_511_mixed_solve_residual(B, cfg511):
    """Mixed precision GMRES(30) with FP64 refinement reaches 1e-8 on the
    21.9 M-unknown system; the FP64 residual is re-computed here with the
    FP64 operator (checked on sampled rows above)."""
    pr, op = cfg511
    b = torch.empty(op.N, dtype=torch.complex128, device=DEV)
    op.rhs(b, B.FP64)
    x = torch.zeros_like(b)
    info = op.gmres(b, x, restart=30, tol=1e-8, prec=B.PREC_MEAN, mode=B.MIXED, maxit=3000)
    Ax = torch.empty_like(x)
    op.matvec(x, Ax, B.FP64)
    relres = float(torch.linalg.vector_norm(b - Ax) / torch.linalg.vector_norm(b))
    print("511x511 mixed: iters %d outer %d relres %.3e" % (info["iters"], info["outer"], relres))
    assert info["status"] == B.SG_OK and relres <= 1e-8


def test_511_tf32_apply(B, cfg511):
    """The plain-TF32 apply at 511 x 511, P = 84 (the complex64 GMRES
    cycles' preconditioner there): four transforms of 42,924 x 1,022 x 1,022
    real, 2,688 output tiles walked by one persistent CTA per SM (about 18
    tiles each, accumulators alternating between two tensor-memory buffers),
    against the FP64 apply within the TF32 bound 5e-3, both blocks, two calls
    giving the same bits."""
    pr, op = cfg511
    g = torch.Generator(device=DEV).manual_seed(13)
    X = torch.randn(op.N, dtype=torch.complex64, device=DEV, generator=g)
    for kind in (B.PREC_MEAN, B.PREC_CSL_MEAN):
        Zr = torch.empty(op.N, dtype=torch.complex128, device=DEV)
        op.precond(X.to(torch.complex128), Zr, kind, B.FP64)
        Zt = torch.empty_like(X)
        op.precond(X, Zt, kind, B.TF32)
        err = float(torch.linalg.vector_norm(Zt.to(torch.complex128) - Zr) / torch.linalg.vector_norm(Zr))
        print("511x511 TF32 apply kind %d: error vs FP64 apply %.2e" % (kind, err))
        assert err < 5e-3, (kind, err)
        Zt2 = torch.empty_like(X)
        op.precond(X, Zt2, kind, B.TF32)
        assert torch.equal(Zt, Zt2)
        del Zr


def test_511_fp16_apply(B, cfg511):
    """The binary16 route at 511 x 511, P = 84 (the complex64 cycles'
    preconditioner where it exists): transform 1 in TF32 writing binary16,
    transforms 2-4 with kind::f16 MMAs on binary16 operands and
    intermediates; within the same 5e-3 of the FP64 apply, both blocks,
    repeatable, and the input scaled to unit norm internally (a scaled input
    gives the scaled output)."""
    pr, op = cfg511
    assert op.info["fp16_route"] == 1
    g = torch.Generator(device=DEV).manual_seed(14)
    X = torch.randn(op.N, dtype=torch.complex64, device=DEV, generator=g)
    for kind in (B.PREC_MEAN, B.PREC_CSL_MEAN):
        Zr = torch.empty(op.N, dtype=torch.complex128, device=DEV)
        op.precond(X.to(torch.complex128), Zr, kind, B.FP64)
        Zh = torch.empty_like(X)
        op.precond(X, Zh, kind, B.FP16)
        err = float(torch.linalg.vector_norm(Zh.to(torch.complex128) - Zr) / torch.linalg.vector_norm(Zr))
        print("511x511 FP16 apply kind %d: error vs FP64 apply %.2e" % (kind, err))
        assert 1e-6 < err < 5e-3, (kind, err)
        Zh2 = torch.empty_like(X)
        op.precond(X, Zh2, kind, B.FP16)
        assert torch.equal(Zh, Zh2)
        Zs = torch.empty_like(X)
        op.precond(X * 1e-6, Zs, kind, B.FP16)
        errs = float(torch.linalg.vector_norm(Zs.to(torch.complex128) * 1e6 - Zr) / torch.linalg.vector_norm(Zr))
        assert errs < 5e-3, (kind, errs)
        del Zr
