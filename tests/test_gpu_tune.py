"""Launch-shape tuning on the GPU (sg_autotune / sg_tune_get / sg_tune_set).

The shapes change no result beyond rounding order: the complex64 operator
gives the same bits for every CTA count, the plain-TF32 preconditioner the
same values for both tile widths (to FP32 rounding), and a GMRES solve with
tuned shapes meets the oracle's residual in the same number of steps (+-1)."""
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


@pytest.mark.parametrize("case", ["2d_sep", "1d", "2d_s6"])
def test_autotune_choices_and_invariance(B, case):
    pr = {"2d_sep": inputs.helmholtz_2d(63, 3, 3, 20.0, 0.1), "1d": inputs.helmholtz_1d_c1(),
          "2d_s6": inputs.helmholtz_2d(47, 6, 3, 15.0, 0.1)}[case]
    base = B.SG(pr, tuned=False)
    op = B.SG(pr, tuned=False)
    t = op.autotune(restart=20)
    assert t == op.tune_get()
    assert t["cgs_blocks_per_sm"] in (2, 3, 4, 6, 8) and t["cgs_us"] > 0 and t["op_us"] > 0
    assert 0 <= t["op_ctas_per_sm"] <= 16
    if op.info["tf32_route"]:
        assert t["tc_tile_n"] in (64, 128) and t["apply_us"] > 0
    else:
        assert t["tc_tile_n"] == 0 and t["apply_us"] == 0
    rng = np.random.default_rng(3)
    x = rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)
    X = torch.from_numpy(x.astype(np.complex64)).to(DEV)
    Y0, Y1 = torch.empty_like(X), torch.empty_like(X)
    base.matvec(X, Y0, B.FP32)
    op.matvec(X, Y1, B.FP32)
    assert torch.equal(Y0, Y1)
    if op.info["tf32_route"]:
        base.precond(X, Y0, B.PREC_MEAN, B.TF32)
        op.precond(X, Y1, B.PREC_MEAN, B.TF32)
        assert (torch.linalg.vector_norm(Y0 - Y1) / torch.linalg.vector_norm(Y0)).item() <= 1e-6
    S = sg.assemble_problem(pr)
    b = torch.from_numpy(S.b).to(DEV)
    kw = dict(restart=20, tol=1e-9, prec=B.PREC_MEAN, mode=B.MIXED, maxit=4000)
    x0, x1 = torch.zeros_like(b), torch.zeros_like(b)
    i0 = base.gmres(b, x0, **kw)
    i1 = op.gmres(b, x1, **kw)
    assert i0["status"] == i1["status"] == B.SG_OK
    assert abs(i0["iters"] - i1["iters"]) <= 1
    relres = np.linalg.norm(S.b - S.A @ x1.cpu().numpy()) / np.linalg.norm(S.b)
    assert relres <= 1e-9
    base.close()
    op.close()


def test_tune_set_validates_and_round_trips(B):
    op = B.SG(inputs.helmholtz_2d(31, 2, 2, 9.0, 0.1), tuned=False)
    for bad in ({"cgs_blocks_per_sm": 9}, {"op_ctas_per_sm": 17}, {"tc_tile_n": 32}):
        with pytest.raises(B.SgError) as ei:
            op.tune_set(bad)
        assert ei.value.status == B.SG_EINVAL
    op.tune_set({"cgs_blocks_per_sm": 3, "op_ctas_per_sm": 1, "tc_tile_n": 64})
    t = op.tune_get()
    assert (t["cgs_blocks_per_sm"], t["op_ctas_per_sm"]) == (3, 1)
    assert t["tc_tile_n"] == (64 if op.info["fast_diag"] else 0)
    # a solve after a change of the CGS2 grid (workspace rebuilt) still converges
    S = sg.assemble_problem(inputs.helmholtz_2d(31, 2, 2, 9.0, 0.1))
    b = torch.from_numpy(S.b).to(DEV)
    x = torch.zeros_like(b)
    assert op.gmres(b, x, restart=20, tol=1e-9, prec=B.PREC_MEAN, mode=B.MIXED)["status"] == B.SG_OK
    op.tune_set({"cgs_blocks_per_sm": 6})
    x2 = torch.zeros_like(b)
    assert op.gmres(b, x2, restart=20, tol=1e-9, prec=B.PREC_MEAN, mode=B.MIXED)["status"] == B.SG_OK
    assert (torch.linalg.vector_norm(x - x2) / torch.linalg.vector_norm(x)).item() < 1e-6
    op.close()


def test_table_entries_are_applied(B):
    """SG(...) applies the committed table's entry for its size."""
    from paper_2209_14740_gb300 import tune_table
    pr = inputs.config_2d_127()
    entry = tune_table.lookup(2, 127, 127, 3, 3)
    op = B.SG(pr)
    t = op.tune_get()
    for k in B.TUNE_KEYS:
        want = entry[k] if k != "tc_tile_n" or op.info["fast_diag"] else 0
        assert t[k] == want, (k, t, entry)
    op.close()


@pytest.mark.parametrize("g,kind", [(63, "mean"), (64, "csl_mean"), (127, "mean")])
def test_fd_transforms_compose_to_the_tf32_apply(B, g, kind):
    """sg_fd_transform t = 0 .. 3 in turn gives the SG_TF32 preconditioner
    apply bit for bit (odd and even grid widths: padded intermediates)."""
    pr = inputs.helmholtz_2d(g, 3, 2, 20.0, 0.1)
    op = B.SG(pr)
    pk = B.PREC_MEAN if kind == "mean" else B.PREC_CSL_MEAN
    mx, my, P = op.info["mx"], op.info["my"], op.P
    mxp, myp = mx + (mx & 1), my + (my & 1)
    rng = np.random.default_rng(g)
    x = (rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)).astype(np.complex64)
    X = torch.from_numpy(x).to(DEV)
    Z = torch.empty_like(X)
    op.precond(X, Z, pk, B.TF32)
    size = P * max(mx, my) * max(mxp, myp)
    T1 = torch.full((size,), float("nan"), dtype=torch.complex64, device=DEV)
    T2 = torch.full((size,), float("nan"), dtype=torch.complex64, device=DEV)
    Y = torch.full_like(X, float("nan"))
    op.fd_transform(0, X, T1, pk)
    op.fd_transform(1, T1, T2, pk)
    op.fd_transform(2, T2, T1, pk)
    op.fd_transform(3, T1, Y, pk)
    torch.cuda.synchronize()
    assert torch.equal(Y, Z)
    with pytest.raises(B.SgError) as ei:
        op.fd_transform(4, X, T1, pk)
    assert ei.value.status == B.SG_EINVAL
    op.close()


def test_retuning_after_solves_drops_captured_graphs(B):
    """Solves capture their Arnoldi-step chunks as graphs (on the second
    use).  Changing the transform precision or tile width afterwards must
    reach the next solve: the route change shows in the result's bits, and a
    rebuilt operand (tile width) is never read through a stale graph; every
    solve meets the oracle's residual."""
    pr = inputs.helmholtz_2d(127, 3, 2, 25.0, 0.1)
    S = sg.assemble_problem(pr)
    op = B.SG(pr, tuned=False)
    assert op.info["fp16_route"] == 1
    b = torch.from_numpy(S.b).to(DEV)
    kw = dict(restart=30, tol=1e-9, prec=B.PREC_MEAN, mode=B.MIXED, maxit=4000)

    def solve():
        x = torch.zeros_like(b)
        for _ in range(3):                      # captured on the second use, replayed on the third
            x.zero_()
            info = op.gmres(b, x, **kw)
        assert info["status"] == B.SG_OK
        rr = np.linalg.norm(S.b - S.A @ x.cpu().numpy()) / np.linalg.norm(S.b)
        assert rr <= 1e-9, rr
        return x

    x16 = solve()
    op.tune_set({"tf32_transforms": 1})
    x32 = solve()
    assert not torch.equal(x16, x32)            # the TF32 transforms really ran
    for width in (64, 128, 64):
        op.tune_set({"tf32_transforms": 1, "tc_tile_n": width})
        solve()
    op.tune_set({"tf32_transforms": 0})
    assert torch.equal(solve(), x16)            # back to the binary16 route, same bits
    op.close()


def test_cgs2_pass_entry_point(B):
    """sg_cgs2_pass: prepares the workspace, runs either pass of a flexible
    step without error (graph-free, on the caller's stream), rejects steps
    outside the workspace and problems without the two-pass form, and leaves
    the handle usable for a solve."""
    from oracle import sg
    pr = inputs.helmholtz_2d(63, 2, 2, 15.0, 0.1)
    op = B.SG(pr, tuned=False)
    op.cgs2_pass(5, 0, restart=20)
    for _ in range(2):
        op.cgs2_pass(5, 1)
        op.cgs2_pass(5, 2)
    torch.cuda.synchronize()
    with pytest.raises(B.SgError) as ei:
        op.cgs2_pass(20, 1)
    assert ei.value.status == B.SG_EINVAL
    with pytest.raises(B.SgError) as ei:
        op.cgs2_pass(5, 3)
    assert ei.value.status == B.SG_EINVAL
    S = sg.assemble_problem(pr)
    b = torch.from_numpy(S.b).to(DEV)
    x = torch.zeros_like(b)
    info = op.gmres(b, x, restart=20, tol=1e-9, prec=B.PREC_MEAN, mode=B.MIXED, maxit=2000)
    assert info["status"] == B.SG_OK
    assert np.linalg.norm(S.b - S.A @ x.cpu().numpy()) / np.linalg.norm(S.b) <= 1e-9
    op.close()
    op1 = B.SG(inputs.helmholtz_1d_c1(), tuned=False)
    with pytest.raises(B.SgError) as ei:
        op1.cgs2_pass(3, 0)
    assert ei.value.status == B.SG_EUNSUPPORTED
    op1.close()
