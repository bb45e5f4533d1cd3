"""Learned initial guess: the native MLP (forward, gradients, Adam) against the
FP64 oracle, the complex low-rank products against numpy, and the warm start
against the zero initial guess."""
import numpy as np
import pytest

from oracle import krylov
from oracle import mlp as omlp
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


def bf16_round(a):
    """Round FP32 values to the nearest bf16 (ties to even), kept as FP32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def xavier(dims, seed):
    from paper_2209_14740_gb300 import warmstart
    p = warmstart.xavier_params(dims, seed)
    # nonzero biases so the bias paths are exercised
    rng = np.random.default_rng(seed + 1)
    off = 0
    for l in range(len(dims) - 1):
        off += dims[l + 1] * dims[l]
        p[off:off + dims[l + 1]] = rng.uniform(-0.2, 0.2, dims[l + 1])
        off += dims[l + 1]
    return bf16_round(p)


SHAPES = [(5, 512, 3, 128, 128),    # the warm-start network, full size
          (5, 37, 2, 13, 70),       # ragged: no dimension a multiple of the 64 x 64 tile
          (3, 64, 0, 9, 1)]         # no hidden layer, batch of one


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_and_gradient_match_oracle(B, shape):
    din, width, hidden, dout, batch = shape
    dims = omlp.layer_dims(din, width, hidden, dout)
    p = xavier(dims, 11)
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (batch, din)).astype(np.float32)
    T = rng.standard_normal((batch, dout)).astype(np.float32)
    net = B.MLP(din, width, hidden, dout)
    assert net.nparams == p.size
    net.set_params(torch.from_numpy(p).to(DEV))
    Xd, Td = torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV)
    Y = torch.empty((batch, dout), dtype=torch.float32, device=DEV)
    net.forward(Xd, Y)
    g = torch.empty(p.size, dtype=torch.float32, device=DEV)
    loss = net.loss_grad(Xd, Td, g)
    # weights are bf16-representable, so the bf16 copy equals the FP32 masters
    # and the FP64 oracle sees the same network
    acts = omlp.forward(p, dims, X)
    lref, gref = omlp.loss_and_grad(p, dims, X, T)
    Yg = Y.cpu().numpy()
    assert np.max(np.abs(Yg - acts[-1])) <= 2e-5 * max(1.0, np.max(np.abs(acts[-1])))
    assert abs(loss - lref) <= 2e-5 * lref
    gg = g.cpu().numpy().astype(np.float64)
    off = 0
    for l in range(len(dims) - 1):
        for n in (dims[l + 1] * dims[l], dims[l + 1]):
            a, r = gg[off:off + n], gref[off:off + n]
            off += n
            assert np.linalg.norm(a - r) <= 1e-4 * np.linalg.norm(r) + 1e-12, (l, n)


def test_first_adam_step_matches_oracle(B):
    dims = omlp.layer_dims(5, 96, 2, 20)
    p = xavier(dims, 3)
    rng = np.random.default_rng(9)
    X = rng.uniform(-1, 1, (64, 5)).astype(np.float32)
    T = rng.standard_normal((64, 20)).astype(np.float32)
    net = B.MLP(5, 96, 2, 20)
    net.set_params(torch.from_numpy(p).to(DEV))
    lr = 1e-3
    hist = net.train(torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV), 64, 1, lr)
    lref, gref = omlp.loss_and_grad(p, dims, X, T)
    assert abs(hist[0] - lref) <= 2e-5 * lref
    z = np.zeros(p.size)
    pref, _, _ = omlp.adam_step(p.astype(np.float64), gref, z, z, 1, lr)
    p1 = torch.empty(p.size, dtype=torch.float32, device=DEV)
    net.get_params(p1)
    p1 = p1.cpu().numpy().astype(np.float64)
    # the first step is lr * g / (|g| + eps): its sign is only decided where
    # |g| is well above the FP32 gradient error
    sure = np.abs(gref) > 1e-3 * np.max(np.abs(gref))
    assert sure.mean() > 0.5
    np.testing.assert_allclose(p1[sure], pref[sure], rtol=0, atol=1e-5 * lr + 1e-7)
    assert np.all(np.abs(p1 - p) <= lr * (1 + 1e-4) + 1e-7)


def test_training_reduces_loss(B):
    from paper_2209_14740_gb300 import warmstart
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, (512, 5)).astype(np.float32)
    W = rng.standard_normal((5, 24))
    T = np.sin(X @ W).astype(np.float32)
    dims = omlp.layer_dims(5, 256, 3, 24)
    net = B.MLP(5, 256, 3, 24)
    net.set_params(torch.from_numpy(warmstart.xavier_params(dims, 0)).to(DEV))
    hist = net.train(torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV), 64, 150, 1e-3)
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 0.05 * hist[0]


def test_mlp_rejects_bad_arguments(B):
    with pytest.raises(B.SgError):
        B.MLP(0, 8, 1, 2)
    net = B.MLP(2, 8, 1, 2)
    X = torch.zeros((4, 2), dtype=torch.float32, device=DEV)
    with pytest.raises(B.SgError):
        net.train(X, X, 4, 1, -1.0)


@pytest.mark.parametrize("m,n,k", [(7, 9, 1000), (37, 45, 70001), (64, 200, 4096), (1, 1, 1)])
def test_cgemm_hn_matches_numpy(B, m, n, k):
    rng = np.random.default_rng(m * 1000 + n)
    A = (rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))).astype(np.complex64)
    Bm = (rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))).astype(np.complex64)
    C = torch.empty((m, n), dtype=torch.complex64, device=DEV)
    work = torch.empty(m * n, dtype=torch.complex128, device=DEV)
    B.cgemm_hn(torch.from_numpy(A).to(DEV), k, torch.from_numpy(Bm).to(DEV), k, m, n, k, C, work)
    ref = A.astype(np.complex128).conj() @ Bm.astype(np.complex128).T
    err = np.abs(C.cpu().numpy() - ref)
    # FP32 sums over slices of at most 1024 terms, slices added in FP64, result
    # rounded to complex64
    assert np.linalg.norm(err) <= 5e-6 * np.linalg.norm(ref) + 1e-6
    assert np.max(err) <= 2e-5 * np.max(np.abs(ref)) + 1e-6


@pytest.mark.parametrize("m,n,k,c128", [(5, 1000, 16, True), (64, 4099, 64, False), (33, 77, 200, True)])
def test_cgemm_nn_matches_numpy(B, m, n, k, c128):
    rng = np.random.default_rng(n)
    A = (rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))).astype(np.complex64)
    Bm = (rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))).astype(np.complex64)
    C = torch.empty((m, n), dtype=torch.complex128 if c128 else torch.complex64, device=DEV)
    B.cgemm_nn(torch.from_numpy(A).to(DEV), torch.from_numpy(Bm).to(DEV), m, n, k, C, out_c128=c128)
    ref = A.astype(np.complex128) @ Bm.astype(np.complex128)
    assert np.max(np.abs(C.cpu().numpy() - ref)) <= 1e-6 * np.sqrt(k) * 4


# a narrow box of the warm-start workload on a small mesh
LO = np.array([14.0, 0.05, 0.2, 0.4, 0.4])
HI = np.array([18.0, 0.1, 0.3, 0.6, 0.6])
G, S_, R_ = 31, 2, 2


def box_params(seed, count):
    rng = np.random.default_rng(seed)
    return LO + (HI - LO) * rng.random((count, 5))


@pytest.fixture(scope="module")
def trained(B):
    from paper_2209_14740_gb300 import warmstart
    ptrain = box_params(100, 192)
    S, _ = warmstart.solve_batch(ptrain, torch, DEV, g=G, s=S_, r=R_, tol=1e-10, restart=40)
    ws = warmstart.build(ptrain, S, torch, DEV, rank=16, n_snapshots=192, width=256, hidden=3, epochs=400,
                         batch=64, lr=1e-3, seed=3, lo=LO, hi=HI)
    return ws, S


def test_pod_basis_is_orthonormal(B, trained):
    ws, S = trained
    r = ws.rank
    Gm = torch.empty((r, r), dtype=torch.complex64, device=DEV)
    work = torch.empty(r * r, dtype=torch.complex128, device=DEV)
    B.cgemm_hn(ws.U, ws.U.shape[1], ws.U, ws.U.shape[1], r, r, ws.U.shape[1], Gm, work)
    assert np.max(np.abs(Gm.cpu().numpy() - np.eye(r))) < 1e-3
    assert ws.energy_captured > 0.9


def test_predict_matches_the_composition(B, trained):
    """sg_warmstart_predict (normalisation kernel, network, complex view,
    expansion, all in the library) against the same steps composed from the
    separate entry points: normalisation in numpy, sg_mlp_forward, the
    complex view of its output, sg_cgemm_nn.  Bit for bit: the normalisation
    formula is the same in FP64, and the products are the same kernels."""
    from paper_2209_14740_gb300 import warmstart
    ws, _ = trained
    ptest = box_params(300, 7)
    X = torch.from_numpy(warmstart.normalise(ptest, ws.lo, ws.hi)).to(DEV)
    Y = torch.empty((X.shape[0], 2 * ws.rank), dtype=torch.float32, device=DEV)
    ws.mlp.forward(X, Y)
    c = torch.view_as_complex(Y.view(X.shape[0], ws.rank, 2)).contiguous()
    N = ws.U.shape[1]
    xc = torch.empty((X.shape[0], N), dtype=torch.complex128, device=DEV)
    B.cgemm_nn(c, ws.Udec, X.shape[0], N, ws.rank, xc, out_c128=True)
    xp = ws.predict(ptest, torch, DEV)
    assert torch.equal(xp, xc)


def test_predict_one_parameter_set_through_ctypes(B, trained):
    """The C ABI called directly with one parameter set (5 doubles) and a
    device buffer, as a C caller would: the same row as a batched call."""
    import ctypes as C
    ws, _ = trained
    ptest = box_params(301, 3)
    xb = ws.predict(ptest, torch, DEV)
    lib = B.load()
    N = ws.U.shape[1]
    for k in range(3):
        p = (C.c_double * 5)(*ptest[k])
        x0 = torch.empty(N, dtype=torch.complex128, device=DEV)
        st = lib.sg_warmstart_predict(ws.model.h, p, 1, C.c_void_p(x0.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == B.SG_OK
        assert torch.equal(x0, xb[k])
    # a bad count is rejected
    p = (C.c_double * 5)(*ptest[0])
    assert lib.sg_warmstart_predict(ws.model.h, p, 0, C.c_void_p(xb.data_ptr()), None) == B.SG_EINVAL


def test_warm_start_beats_zero_guess(B, trained):
    ws, _ = trained
    ptest = box_params(200, 12)
    x0 = ws.predict(ptest, torch, DEV)
    ops = [B.SG(inputs.warmstart_problem(p, G, S_, R_)) for p in ptest]
    kw = dict(restart=40, tol=1e-8, prec=B.PREC_MEAN, mode=B.MIXED, maxit=5000)
    bs = []
    for op in ops:
        b = torch.empty(op.N, dtype=torch.complex128, device=DEV)
        op.rhs(b, B.FP64)
        bs.append(b)
    xz = [torch.zeros_like(b) for b in bs]
    xw = [torch.zeros_like(b) for b in bs]
    stz, infz = B.gmres_batched(ops, bs, xz, **kw)
    stw, infw = B.gmres_batched(ops, bs, xw, x0s=[x0[k] for k in range(len(ops))], x0_policy=B.X0_SCALED,
                                **kw)
    assert stz == B.SG_OK and stw == B.SG_OK
    itz = np.array([f["iters"] for f in infz])
    itw = np.array([f["iters"] for f in infw])
    assert all(f["relres"] <= 1e-8 for f in infw)
    # the guess is close to the solution, and the solves start from it
    rel = [float(torch.linalg.norm(x0[k] - xz[k]) / torch.linalg.norm(xz[k])) for k in range(len(ops))]
    assert np.median(rel) < 0.3, rel
    # fewer Arnoldi steps in total; the floor is set by the guess error (a
    # relative residual near 0.1 saves about one of ~9 steps per solve)
    assert itw.sum() <= 0.92 * itz.sum(), (itw, itz, rel)
    # the warm-started solution satisfies the FP64 system (oracle residual)
    for k in (0, 5):
        ref = sg.assemble_problem(inputs.warmstart_problem(ptest[k], G, S_, R_))
        x = xw[k].cpu().numpy()
        assert np.linalg.norm(ref.b - ref.A @ x) <= 1.5e-8 * np.linalg.norm(ref.b)
    for op in ops:
        op.close()


def test_fallback_to_zero_guess_on_bad_guess(B):
    """A guess with residual above ||b|| is dropped for the zero guess."""
    p = inputs.helmholtz_2d(15, 2, 2, 9.0, 0.1)
    op = B.SG(p)
    b = torch.empty(op.N, dtype=torch.complex128, device=DEV)
    op.rhs(b, B.FP64)
    kw = dict(restart=20, tol=1e-8, prec=B.PREC_MEAN, mode=B.FP64, maxit=5000)
    xz = torch.zeros_like(b)
    iz = op.gmres(b, xz, **kw)
    bad = 1e3 * torch.ones_like(b)
    xf = torch.zeros_like(b)
    inf = op.gmres(b, xf, x0=bad, x0_policy=B.X0_FALLBACK, **kw)
    assert inf["status"] == B.SG_OK and inf["iters"] == iz["iters"]
    assert torch.equal(xf, xz)
    op.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_scaled_guess_recovers_any_multiple_of_the_solution(B, mode):
    """zeta x0 with zeta = (A x0)^H b / ||A x0||^2 is the exact solution when
    x0 is any nonzero multiple of it: the solve ends at its first residual
    check."""
    m = B.FP64 if mode == "fp64" else B.MIXED
    p = inputs.helmholtz_2d(19, 3, 2, 11.0, 0.12)
    ref = sg.assemble_problem(p)
    xs = krylov.direct(ref.A, ref.b)
    op = B.SG(p)
    b = torch.from_numpy(ref.b).to(DEV)
    x0 = torch.from_numpy((3.7 - 2.1j) * xs).to(DEV)
    x = torch.zeros_like(b)
    inf = op.gmres(b, x, x0=x0, x0_policy=B.X0_SCALED, restart=20, tol=1e-8, prec=B.PREC_MEAN, mode=m, maxit=500)
    assert inf["status"] == B.SG_OK and inf["iters"] == 0
    assert np.linalg.norm(x.cpu().numpy() - xs) <= 1e-10 * np.linalg.norm(xs)
    op.close()


def test_scaled_guess_never_starts_above_zero_guess(B):
    """For a guess unrelated to the solution the scaled start has residual
    at most ||b||, and the solve meets the tolerance."""
    p = inputs.helmholtz_2d(19, 3, 2, 11.0, 0.12)
    ref = sg.assemble_problem(p)
    op = B.SG(p)
    b = torch.from_numpy(ref.b).to(DEV)
    rng = np.random.default_rng(4)
    g = 1e4 * (rng.standard_normal(op.N) + 1j * rng.standard_normal(op.N))
    x = torch.zeros_like(b)
    inf = op.gmres(b, x, x0=torch.from_numpy(g).to(DEV), x0_policy=B.X0_SCALED, restart=20, tol=1e-8,
                   prec=B.PREC_MEAN, mode=B.FP64, maxit=2000, max_outer=0)
    assert inf["status"] == B.SG_OK
    xh = x.cpu().numpy()
    assert np.linalg.norm(ref.b - ref.A @ xh) <= 1.01e-8 * np.linalg.norm(ref.b)
    # the scaled start itself: residual of zeta g against the oracle
    Ag = ref.A @ g
    zeta = np.vdot(Ag, ref.b) / np.vdot(Ag, Ag).real
    assert np.linalg.norm(ref.b - zeta * Ag) <= np.linalg.norm(ref.b)
    op.close()


def test_pod_ceiling_against_numpy(B):
    """pod_basis / pod_errors (the decoder's best-approximation floor) on
    random low-rank-plus-noise snapshots: the basis rows are orthonormal, span
    the leading left singular space of the snapshots (numpy SVD), and the
    reported errors equal numpy's projection errors."""
    from paper_2209_14740_gb300 import warmstart
    rng = np.random.default_rng(11)
    n, N, r = 96, 2000, 12
    A = (rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r))) @ \
        (rng.standard_normal((r, N)) + 1j * rng.standard_normal((r, N)))
    A += 0.3 * (rng.standard_normal((n, N)) + 1j * rng.standard_normal((n, N)))
    S = torch.from_numpy(A.astype(np.complex64)).to(DEV)
    U, lam = warmstart.pod_basis(S, 16, 80, torch, DEV)
    Uh = U.cpu().numpy().astype(np.complex128)
    assert np.abs(Uh.conj() @ Uh.T - np.eye(16)).max() < 2e-4
    sv = np.linalg.svd(A[:80].astype(np.complex64).astype(np.complex128), compute_uv=False)
    np.testing.assert_allclose(lam[:16], sv[:16] ** 2, rtol=1e-3)
    X = rng.standard_normal((5, N)) + 0j
    X[:3] = (rng.standard_normal((3, n)) @ A) / n          # inside the snapshot span (mostly)
    Xd = torch.from_numpy(X.astype(np.complex64)).to(DEV)
    errs = warmstart.pod_errors(U, Xd, (4, 12, 16), torch, DEV)
    Xc = X.astype(np.complex64).astype(np.complex128)
    for R, e in errs.items():
        Q = Uh[:R].conj()                                   # coefficients c = conj(U) x
        proj = (Q @ Xc.T).T @ Uh[:R]
        ref = np.linalg.norm(Xc - proj, axis=1) / np.linalg.norm(Xc, axis=1)
        np.testing.assert_allclose(e, ref, rtol=5e-3, atol=2e-3)
    assert errs[12][:3].max() < 0.2 and np.all(errs[4][:3] > errs[12][:3]) and errs[16][3:].min() > 0.9
