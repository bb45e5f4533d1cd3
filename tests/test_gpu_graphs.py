"""Arnoldi chunks replayed from CUDA graphs give the same bits as direct launches.

The first solve on a handle launches every kernel directly, the second
captures each chunk of steps into a graph, later solves replay the graphs; all
must produce identical iterates."""
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


@pytest.mark.parametrize("mode,prec", [("mixed", "mean"), ("fp64", "mean"), ("fp32", "csl"), ("mixed", "none")])
def test_replayed_solves_are_identical(B, mode, prec):
    p = inputs.helmholtz_2d(23, 3, 2, 12.0, 0.1)
    ref = sg.assemble_problem(p)
    op = B.SG(p)
    m = {"mixed": B.MIXED, "fp64": B.FP64, "fp32": B.FP32}[mode]
    pk = {"mean": B.PREC_MEAN, "csl": B.PREC_CSL_MEAN, "none": B.PREC_NONE}[prec]
    dt = torch.complex64 if m == B.FP32 else torch.complex128
    b = torch.from_numpy(ref.b).to(DEV).to(dt)
    tol = 1e-5 if m == B.FP32 else 1e-8
    xs, infos = [], []
    maxit = 3000 if pk != B.PREC_NONE else 60   # unpreconditioned: a fixed number of steps
    for _ in range(4):
        x = torch.zeros_like(b)
        infos.append(op.gmres(b, x, restart=12, tol=tol, prec=pk, mode=m, maxit=maxit, check_every=4))
        xs.append(x)
    assert len({(i["status"], i["iters"], i["relres"]) for i in infos}) == 1
    for x in xs[1:]:
        assert torch.equal(x, xs[0])
    if pk != B.PREC_NONE:
        assert infos[0]["status"] == B.SG_OK
        xh = xs[0].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(ref.b - ref.A @ xh) <= 1.01 * tol * np.linalg.norm(ref.b) + (2e-5 if m == B.FP32 else 0)
    op.close()


def test_solve_on_the_default_stream_orders_with_caller_work(B):
    """Work queued on the caller's stream before sg_gmres is seen by the solve,
    and the caller's stream sees the solution after it."""
    p = inputs.helmholtz_2d(19, 2, 2, 9.0, 0.1)
    op = B.SG(p)
    b = torch.empty(op.N, dtype=torch.complex128, device=DEV)
    op.rhs(b, B.FP64)
    b2 = torch.zeros_like(b)
    b2.copy_(b)                       # queued on the default stream
    x = torch.zeros_like(b)
    info = op.gmres(b2, x, restart=20, tol=1e-9, prec=B.PREC_MEAN, mode=B.FP64)
    y = x * 1.0                       # queued after the solve on the default stream
    assert info["status"] == B.SG_OK
    assert torch.equal(y, x)
    r = torch.empty_like(b)
    op.matvec(x, r, B.FP64)
    assert float(torch.linalg.norm(b - r) / torch.linalg.norm(b)) <= 1.01e-9
    op.close()
