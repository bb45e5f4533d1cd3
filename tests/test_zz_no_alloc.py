"""sg_precond_noalloc: the allocation-free preconditioner apply.

It exists for callers that cannot allocate device memory when they run the
preconditioner (allocation forbidden or too slow where they are, or device
memory owned by another allocator's pool); it takes its scratch from a fixed
array inside the library.  This file is collected last on purpose: if it
fails, a run that stops at the first failure has run everything else.

Each case calls the new entry point twice in a row (the shared static
scratch keeps the previous call's contents) and compares every result with
sg_precond, within the tolerances the preconditioner tests use."""
import numpy as np
import pytest

from paper_2209_14740_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def B():
    from paper_2209_14740_gb300 import binding
    binding.load()
    return binding


def _cases():
    return [inputs.helmholtz_2d(21, 3, 3, 12.0, 0.15),      # 2D separable: GEMM + tridiagonal + GEMM
            inputs.helmholtz_1d_c1(n_unknowns=37, r=5),      # 1D tridiagonal from shared memory
            inputs.config_2d_127(),                           # the bench workload, N = 322,580
            # lines of 331 nodes: FP32 takes the tensor-core x transforms with the
            # intermediates at row stride mx plus the y sweeps (N = 438,244)
            inputs.helmholtz_2d(331, 1, 3, 30.0, 0.15),
            # 1D lines too long for shared memory: the global-memory sweep, in place
            # through the first scratch vector (N = 24,000)
            inputs.helmholtz_1d_c1(n_unknowns=6000, r=3)]


@pytest.mark.parametrize("case", range(5))
@pytest.mark.parametrize("kind", [1, 2])
def test_noalloc_matches_precond_twice(B, case, kind):
    pr = _cases()[case]
    op = B.SG(pr)
    assert op.N <= B.NOALLOC_MAX_N
    if case == 3:
        assert not op.info["fast_diag"]
    rng = np.random.default_rng(1000 + case)
    for call in range(2):
        x = rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N)
        for prec, dt, tol in ((B.FP64, torch.complex128, 1e-10), (B.FP32, torch.complex64, 2e-4)):
            X = torch.from_numpy(x).to(DEV).to(dt)
            Zr = torch.empty_like(X)
            op.precond(X, Zr, kind, prec)
            Zn = torch.full_like(X, float("nan"))
            op.precond_noalloc(X, Zn, kind, prec)
            torch.cuda.synchronize()
            err = float(torch.linalg.vector_norm(Zn - Zr) / torch.linalg.vector_norm(Zr))
            assert err <= tol, (call, prec, err)
            # in place, as sg_precond allows
            Xi = X.clone()
            op.precond_noalloc(Xi, Xi, kind, prec)
            err2 = float(torch.linalg.vector_norm(Xi - Zr) / torch.linalg.vector_norm(Zr))
            assert err2 <= tol, (call, prec, err2)
    op.close()


def test_noalloc_rejects_too_large(B):
    pr = inputs.helmholtz_2d(171, 3, 3, 30.0, 0.15)          # N = 171^2 * 20 = 584,820 > limit
    op = B.SG(pr)
    assert op.N > B.NOALLOC_MAX_N
    X = torch.zeros(op.N, dtype=torch.complex128, device=DEV)
    with pytest.raises(B.SgError) as ei:
        op.precond_noalloc(X, X, B.PREC_MEAN, B.FP64)
    assert ei.value.status == B.SG_EINVAL
    assert "SG_NOALLOC_MAX_N" in str(ei.value)
    op.close()
