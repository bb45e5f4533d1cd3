"""The binary16 route of the 2D fast-diagonalisation preconditioner (SG_FP16;
transforms 2-4 with kind::f16 tensor-core MMAs and binary16 intermediates,
transform 1 in TF32 writing binary16), on the GPU: the apply against the
FP64 apply within the same 5e-3 as the TF32 form, the four transforms
through sg_fd_transform, and mixed-precision GMRES with the binary16
preconditioner in its flexible cycles against the TF32 one (same tolerance
reached, steps within +-2, the oracle's residual)."""
import numpy as np
import pytest

from oracle import sg
from paper_2209_14740_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def B():
    from paper_2209_14740_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("g,s,r", [(63, 3, 2), (64, 2, 3), (127, 3, 3)])
def test_fp16_apply_against_fp64(B, g, s, r):
    op = B.SG(inputs.helmholtz_2d(g, s, r, 20.0, 0.1), tuned=False)
    assert op.info["fp16_route"] == 1 and op.info["tf32_route"] == 1
    rng = np.random.default_rng(g + s)
    x = (rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)).astype(np.complex64)
    X = torch.from_numpy(x).to(DEV)
    for kind in (B.PREC_MEAN, B.PREC_CSL_MEAN):
        Zr = torch.empty(op.N, dtype=torch.complex128, device=DEV)
        op.precond(X.to(torch.complex128), Zr, kind, B.FP64)
        Zh = torch.empty_like(X)
        op.precond(X, Zh, kind, B.FP16)
        Zt = torch.empty_like(X)
        op.precond(X, Zt, kind, B.TF32)
        eh = float(torch.linalg.vector_norm(Zh.to(torch.complex128) - Zr) / torch.linalg.vector_norm(Zr))
        et = float(torch.linalg.vector_norm(Zt.to(torch.complex128) - Zr) / torch.linalg.vector_norm(Zr))
        assert 1e-6 < eh < 5e-3 and et < 5e-3, (kind, eh, et)
        Xi = X.clone()
        op.precond(Xi, Xi, kind, B.FP16)         # in place
        assert torch.equal(Xi, Zh)
    op.close()


def test_fp16_transforms_compose(B):
    """sg_fd_transform in its SG_FP16 form, t = 0 .. 3 on a unit-norm input,
    gives the FP64 apply within 5e-3."""
    op = B.SG(inputs.helmholtz_2d(127, 3, 2, 25.0, 0.1), tuned=False)
    mx, my, P = op.info["mx"], op.info["my"], op.P
    mx4, my4 = (mx + 3) // 4 * 4, (my + 3) // 4 * 4
    rng = np.random.default_rng(5)
    x = rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)
    x /= np.linalg.norm(x)
    X = torch.from_numpy(x.astype(np.complex64)).to(DEV)
    # binary16 pairs are 4 bytes: float32 storage of the same size
    T1 = torch.zeros(P * max(mx, my) * max(mx4, my4), dtype=torch.float32, device=DEV)
    T2 = torch.zeros_like(T1)
    Y = torch.empty_like(X)
    op.fd_transform(0, X, T1, B.PREC_MEAN, B.FP16)
    op.fd_transform(1, T1, T2, B.PREC_MEAN, B.FP16)
    op.fd_transform(2, T2, T1, B.PREC_MEAN, B.FP16)
    op.fd_transform(3, T1, Y, B.PREC_MEAN, B.FP16)
    Zr = torch.empty(op.N, dtype=torch.complex128, device=DEV)
    op.precond(torch.from_numpy(x).to(DEV), Zr, B.PREC_MEAN, B.FP64)
    err = float(torch.linalg.vector_norm(Y.to(torch.complex128) - Zr) / torch.linalg.vector_norm(Zr))
    assert err < 5e-3, err
    op.close()


@pytest.mark.parametrize("g", [96, 127])
def test_fp16_route_in_mixed_gmres(B, g):
    pr = inputs.helmholtz_2d(g, 3, 3, 30.0, 0.15)
    S = sg.assemble_problem(pr)
    b = torch.from_numpy(S.b).to(DEV)
    its = {}
    for tf32 in (0, 1):
        op = B.SG(pr, tuned=False)
        op.tune_set({"tf32_transforms": tf32})
        x = torch.zeros_like(b)
        # (the complex64 basis in both, so that only the transforms differ)
        info = op.gmres(b, x, restart=50, tol=1e-9, prec=B.PREC_MEAN, mode=B.MIXED, maxit=4000, basis16=-1)
        assert info["status"] == B.SG_OK
        relres = np.linalg.norm(S.b - S.A @ x.cpu().numpy()) / np.linalg.norm(S.b)
        assert relres <= 1e-9, (tf32, relres)
        its[tf32] = info["iters"]
        op.close()
    assert abs(its[0] - its[1]) <= 2, its


def test_fp16_route_absent_on_small_grids(B):
    op = B.SG(inputs.helmholtz_2d(15, 2, 2, 9.0, 0.1), tuned=False)
    assert op.info["fp16_route"] == 0
    X = torch.zeros(op.N, dtype=torch.complex64, device=DEV)
    with pytest.raises(B.SgError) as ei:
        op.precond(X, torch.empty_like(X), B.PREC_MEAN, B.FP16)
    assert ei.value.status == B.SG_EUNSUPPORTED
    op.close()


@pytest.mark.parametrize("g,kind,basis16", [(96, "csl", -1), (129, "mean", -1), (96, "csl", 0), (129, "mean", 0)])
def test_fp16_copy_route_scale_invariant(B, g, kind, basis16):
    """The binary16 values of the flexible cycles take their scales from the
    vectors' norms: the copy of each new basis vector that the second CGS2
    pass writes beside the complex64 basis (basis16 = -1), and the binary16
    basis itself (basis16 = 0, slot 0 scaled from the residual's norm).  A
    right-hand side scaled by 2^-40 or 2^40 converges in the same number of
    steps (within 1) to the same tolerance, and the result is the scaled
    solution."""
    pr = inputs.helmholtz_2d(g, 3, 2, 25.0, 0.1)
    S = sg.assemble_problem(pr)
    prec = B.PREC_CSL_MEAN if kind == "csl" else B.PREC_MEAN
    op = B.SG(pr, tuned=False)
    assert op.info["fp16_route"] == 1
    its = {}
    for e in (0, -40, 40):
        f = 2.0 ** e
        b = torch.from_numpy(S.b * f).to(DEV)
        x = torch.zeros_like(b)
        info = op.gmres(b, x, restart=40, tol=1e-9, prec=prec, mode=B.MIXED, maxit=4000, basis16=basis16)
        assert info["status"] == B.SG_OK, (e, info)
        xs = x.cpu().numpy() / f
        relres = np.linalg.norm(S.b - S.A @ xs) / np.linalg.norm(S.b)
        assert relres <= 1e-9, (e, relres)
        its[e] = info["iters"]
    assert max(its.values()) - min(its.values()) <= 1, its
    op.close()


@pytest.mark.parametrize("g,s,r", [(63, 3, 2), (127, 3, 3), (200, 2, 3)])
def test_paired_256_form_apply(B, g, s, r):
    """The binary16 transforms in the paired 256-column form (tc_tile_n 256:
    clusters of two CTAs on adjacent row tiles, each B stage shared by
    multicast copies) give the 128-column form's apply to FP32 rounding and
    the FP64 apply within 5e-3; 63^2 with P = 10 has an odd number of row
    tiles (the last pair's second CTA works on rows past the end) and a
    single, mostly empty column tile."""
    op = B.SG(inputs.helmholtz_2d(g, s, r, 20.0, 0.1), tuned=False)
    assert op.info["fp16_route"] == 1
    rng = np.random.default_rng(g * 7 + r)
    x = (rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)).astype(np.complex64)
    X = torch.from_numpy(x).to(DEV)
    for kind in (B.PREC_MEAN, B.PREC_CSL_MEAN):
        Zr = torch.empty(op.N, dtype=torch.complex128, device=DEV)
        op.precond(X.to(torch.complex128), Zr, kind, B.FP64)
        out = {}
        for tn in (128, 256):
            op.tune_set({"tc_tile_n": tn})
            assert op.tune_get()["tc_tile_n"] == tn
            Z = torch.empty_like(X)
            op.precond(X, Z, kind, B.FP16)
            out[tn] = Z
        d = float(torch.linalg.vector_norm(out[256] - out[128]) / torch.linalg.vector_norm(out[128]))
        assert d <= 1e-6, (kind, d)
        e = float(torch.linalg.vector_norm(out[256].to(torch.complex128) - Zr) / torch.linalg.vector_norm(Zr))
        assert e < 5e-3, (kind, e)
    op.close()


def test_paired_256_form_in_mixed_gmres(B):
    """Mixed GMRES with the paired form in its flexible cycles (transform 1
    from the binary16 copy of each new basis vector included) reaches the
    tolerance in the 128-column form's number of steps (within 1), with the
    oracle's residual."""
    pr = inputs.helmholtz_2d(127, 3, 3, 30.0, 0.15)
    S = sg.assemble_problem(pr)
    b = torch.from_numpy(S.b).to(DEV)
    its = {}
    for tn in (128, 256):
        op = B.SG(pr, tuned=False)
        op.tune_set({"tc_tile_n": tn, "tf32_transforms": 0})
        x = torch.zeros_like(b)
        info = op.gmres(b, x, restart=50, tol=1e-9, prec=B.PREC_MEAN, mode=B.MIXED, maxit=4000)
        assert info["status"] == B.SG_OK
        relres = np.linalg.norm(S.b - S.A @ x.cpu().numpy()) / np.linalg.norm(S.b)
        assert relres <= 1e-9, (tn, relres)
        its[tn] = info["iters"]
        op.close()
    assert abs(its[256] - its[128]) <= 1, its


def test_paired_256_form_refused_without_fp16_route(B):
    op = B.SG(inputs.helmholtz_2d(15, 2, 2, 9.0, 0.1), tuned=False)
    assert op.info["fp16_route"] == 0
    with pytest.raises(B.SgError) as ei:
        op.tune_set({"tc_tile_n": 256})
    assert ei.value.status == B.SG_EUNSUPPORTED
    op.close()


@pytest.mark.parametrize("sigma,basis16", [(0.25, 0), (0.35, 0), (0.35, -1), (0.45, 0)])
def test_flexible_long_cycles(B, sigma, basis16):
    """Flexible cycles longer than 64 steps (the CGS2 passes then read the
    basis factor R from device memory instead of staging it in shared
    memory), on the binary16 and the complex64 basis: a strongly varying
    wavenumber and a tight inner reduction make the cycles long; the solve
    still reaches the tolerance with the oracle's residual."""
    pr = inputs.helmholtz_2d(63, 3, 3, 25.0, sigma)
    S = sg.assemble_problem(pr)
    b = torch.from_numpy(S.b).to(DEV)
    op = B.SG(pr, tuned=False)
    x = torch.zeros_like(b)
    info = op.gmres(b, x, restart=120, tol=1e-10, prec=B.PREC_MEAN, mode=B.MIXED, maxit=4000, inner_tol=1e-9,
                    basis16=basis16)
    assert info["status"] == B.SG_OK, info
    relres = np.linalg.norm(S.b - S.A @ x.cpu().numpy()) / np.linalg.norm(S.b)
    assert relres <= 1e-10, relres
    print("long cycles: sigma %.2f basis16 %d iters %d outer %d cycles %d" %
          (sigma, basis16, info["iters"], info["outer"], info["cycles"]))
    op.close()


@pytest.mark.parametrize("g,kind", [(96, "mean"), (127, "csl"), (160, "mean")])
def test_binary16_basis_against_complex64(B, g, kind):
    """SG_MIXED with the flexible cycles' Krylov basis stored as binary16
    (basis16 = 0, the default on the binary16 route) against the complex64
    basis (basis16 = -1): both reach the tolerance with the oracle's
    residual; the binary16 basis limits a cycle's reduction to about 1e-3, so
    it may take up to two more refinement steps, but no more than a third
    more Arnoldi steps (plus 3)."""
    pr = inputs.helmholtz_2d(g, 4, 3, 30.0, 0.15)
    S = sg.assemble_problem(pr)
    prec = B.PREC_CSL_MEAN if kind == "csl" else B.PREC_MEAN
    b = torch.from_numpy(S.b).to(DEV)
    res = {}
    for basis16 in (-1, 0):
        op = B.SG(pr, tuned=False)
        assert op.info["fp16_route"] == 1
        x = torch.zeros_like(b)
        info = op.gmres(b, x, restart=40, tol=1e-9, prec=prec, mode=B.MIXED, maxit=4000, basis16=basis16)
        assert info["status"] == B.SG_OK, (basis16, info)
        relres = np.linalg.norm(S.b - S.A @ x.cpu().numpy()) / np.linalg.norm(S.b)
        assert relres <= 1e-9, (basis16, relres)
        assert abs(info["relres"] - relres) <= 1e-3 * relres + 1e-15
        res[basis16] = info
        op.close()
    print("basis16: complex64 %d steps / %d refinements, binary16 %d / %d" %
          (res[-1]["iters"], res[-1]["outer"], res[0]["iters"], res[0]["outer"]))
    assert res[0]["iters"] <= (4 * res[-1]["iters"]) // 3 + 3, res
    assert res[0]["outer"] <= res[-1]["outer"] + 2, res


def test_binary16_basis_option_checked(B):
    op = B.SG(inputs.helmholtz_2d(63, 2, 2, 15.0, 0.1), tuned=False)
    b = torch.zeros(op.N, dtype=torch.complex128, device=DEV)
    op.rhs(b, B.FP64)
    with pytest.raises(B.SgError) as ei:
        op.gmres(b, torch.zeros_like(b), restart=20, tol=1e-8, prec=B.PREC_MEAN, mode=B.MIXED, basis16=3)
    assert ei.value.status == B.SG_EINVAL
    op.close()

