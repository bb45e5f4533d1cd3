"""sg_gmres_batched: concurrent solves of heterogeneous SG systems.

Each system's result must equal, bit for bit, the result of solving it alone
with sg_gmres (the same kernels run in the same order on its own stream), and
the oracle's FP64 residual of every solution must meet the tolerance."""
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


def batch_problems():
    return [inputs.helmholtz_2d(15, 2, 2, 9.0, 0.1), inputs.helmholtz_2d(19, 3, 3, 12.0, 0.15),
            inputs.helmholtz_2d(23, 4, 2, 14.0, 0.2), inputs.helmholtz_2d(17, 2, 3, 10.0, 0.05),
            inputs.helmholtz_2d(21, 3, 2, 11.0, 0.12), inputs.helmholtz_1d_c1(n_unknowns=60, r=5)]


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_batched_equals_sequential(B, mode):
    m = B.MIXED if mode == "mixed" else B.FP64
    probs = batch_problems()
    ops = [B.SG(p) for p in probs]
    refs = [sg.assemble_problem(p) for p in probs]
    bs = [torch.from_numpy(r.b).to(DEV) for r in refs]
    kw = dict(restart=20, tol=1e-8, prec=B.PREC_MEAN, mode=m, maxit=5000)
    xs_seq = []
    infos_seq = []
    for op, b in zip(ops, bs):
        x = torch.zeros_like(b)
        infos_seq.append(op.gmres(b, x, **kw))
        xs_seq.append(x)
    xs = [torch.zeros_like(b) for b in bs]
    st, infos = B.gmres_batched(ops, bs, xs, concurrency=3, **kw)
    assert st == B.SG_OK
    for k, (ref, x, xsq, i1, i2) in enumerate(zip(refs, xs, xs_seq, infos, infos_seq)):
        assert i1["iters"] == i2["iters"] and i1["outer"] == i2["outer"], (k, i1, i2)
        assert torch.equal(x, xsq), k
        xg = x.cpu().numpy()
        relres = np.linalg.norm(ref.b - ref.A @ xg) / np.linalg.norm(ref.b)
        assert relres <= 1e-8, (k, relres)
    for op in ops:
        op.close()


def test_batched_argument_errors(B):
    p = inputs.helmholtz_2d(15, 2, 2, 9.0, 0.1)
    op = B.SG(p)
    b = torch.zeros(op.N, dtype=torch.complex128, device=DEV)
    x = torch.zeros_like(b)
    with pytest.raises(B.SgError) as ei:
        B.gmres_batched([op, op], [b, b], [x, x], tol=1e-8)
    assert ei.value.status == B.SG_EINVAL
    st, infos = B.gmres_batched([], [], [], tol=1e-8)
    assert st == B.SG_OK and infos == []
    op.close()
