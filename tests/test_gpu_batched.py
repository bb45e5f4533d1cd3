"""sg_gmres_batched: solves of heterogeneous SG systems in one call.

Each system's result must equal, bit for bit, the result of solving it alone
with sg_gmres (the same kernels run in the same order), on both routes: the
one-graph launch (SG_MIXED, device-decided refinement steps and Arnoldi
chunks through conditional graph nodes) and the per-system streams
(concurrency < 0, or SG_FP64); the oracle's FP64 residual of every solution
must meet the tolerance."""
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
        assert i1["graph_outer"] == (i1["outer"] if mode == "mixed" else 0), (k, i1)
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


def _solve_both(B, probs, kw, concurrency=3):
    """Per system alone (sg_gmres), then batched on the graph route, then
    batched on the per-system route; returns the three (xs, infos)."""
    ops = [B.SG(p) for p in probs]
    refs = [sg.assemble_problem(p) for p in probs]
    bs = [torch.from_numpy(r.b).to(DEV) for r in refs]
    seq = []
    for op, b in zip(ops, bs):
        x = torch.zeros_like(b)
        try:
            inf = op.gmres(b, x, **kw)
        except B.SgError as e:
            inf = dict(status=e.status)
        seq.append((x, inf))
    xg = [torch.full_like(b, float("nan")) for b in bs]
    stg, infg = B.gmres_batched(ops, bs, xg, concurrency=concurrency, **kw)
    xp = [torch.full_like(b, float("nan")) for b in bs]
    stp, infp = B.gmres_batched(ops, bs, xp, concurrency=-1, **kw)
    return ops, refs, bs, seq, (stg, xg, infg), (stp, xp, infp)


@pytest.mark.parametrize("restart,prec", [(20, "mean"), (8, "mean"), (13, "csl_mean"), (24, "none")])
def test_graph_route_equals_per_system_route(B, restart, prec):
    """Chunks of 8 steps with a ragged last chunk (20, 13), a single chunk
    (8), the CSL mean block and no preconditioner (more refinement steps than
    the graph unrolls: those systems continue on the per-system route)."""
    pc = dict(mean=B.PREC_MEAN, csl_mean=B.PREC_CSL_MEAN, none=B.PREC_NONE)[prec]
    kw = dict(restart=restart, tol=1e-8, prec=pc, mode=B.MIXED, maxit=3000, max_outer=40)
    ops, refs, bs, seq, (stg, xg, infg), (stp, xp, infp) = _solve_both(B, batch_problems(), kw)
    assert stg == stp
    for k in range(len(ops)):
        xs, i0 = seq[k]
        assert torch.equal(xg[k], xs) and torch.equal(xp[k], xs), k
        for key in ("iters", "outer", "status"):
            assert infg[k][key] == i0[key] == infp[k][key], (k, key, infg[k], i0, infp[k])
        assert infp[k]["graph_outer"] == 0 and 1 <= infg[k]["graph_outer"] <= min(4, i0["outer"]), infg[k]
        if i0["status"] == B.SG_OK:
            r = refs[k]
            relres = np.linalg.norm(r.b - r.A @ xg[k].cpu().numpy()) / np.linalg.norm(r.b)
            assert relres <= 1e-8, (k, relres)
    if prec == "none":
        assert any(i["outer"] > 4 for i in infg)      # continued after the graph
    for op in ops:
        op.close()


def test_graph_route_continues_after_unrolled_steps(B):
    """tol 1e-12 with inner_tol 1e-2 needs about six refinement steps: the
    graph runs four, the rest continue from the graph's iterate; the result
    is still the one-at-a-time solve's, bit for bit."""
    kw = dict(restart=30, tol=1e-12, inner_tol=1e-2, prec=B.PREC_MEAN, mode=B.MIXED, maxit=5000)
    ops, refs, bs, seq, (stg, xg, infg), (stp, xp, infp) = _solve_both(B, batch_problems(), kw)
    assert stg == B.SG_OK
    cont = 0
    for k in range(len(ops)):
        xs, i0 = seq[k]
        assert torch.equal(xg[k], xs), k
        assert infg[k]["iters"] == i0["iters"] and infg[k]["outer"] == i0["outer"], (k, infg[k], i0)
        assert infg[k]["graph_outer"] == min(4, i0["outer"])
        cont += i0["outer"] > 4
        r = refs[k]
        relres = np.linalg.norm(r.b - r.A @ xg[k].cpu().numpy()) / np.linalg.norm(r.b)
        assert relres <= 1e-11, (k, relres)
    assert cont >= 1
    for op in ops:
        op.close()


def test_graph_relaunch_and_caps(B):
    """The cached graph relaunched (same handles and vectors) gives the same
    bits; a zero right-hand side gives x = 0 at once; the step cap and the
    refinement cap end systems with SG_ENOTCONV, as sg_gmres does."""
    probs = batch_problems()[:3]
    ops = [B.SG(p) for p in probs]
    refs = [sg.assemble_problem(p) for p in probs]
    bs = [torch.from_numpy(r.b).to(DEV) for r in refs]
    bs[1].zero_()
    kw = dict(restart=16, tol=1e-9, prec=B.PREC_MEAN, mode=B.MIXED, maxit=4000)
    xs = [torch.zeros_like(b) for b in bs]
    st1, i1 = B.gmres_batched(ops, bs, xs, **kw)
    first = [x.clone() for x in xs]
    for x in xs:
        x.fill_(3.0)
    st2, i2 = B.gmres_batched(ops, bs, xs, **kw)
    assert st1 == st2 == B.SG_OK and i1 == i2
    assert all(torch.equal(a, b) for a, b in zip(first, xs))
    assert i1[1]["iters"] == 0 and i1[1]["outer"] == 0 and i1[1]["relres"] == 0.0 and not xs[1].any()
    for kw2 in (dict(kw, maxit=5), dict(kw, max_outer=1, inner_tol=0.3)):
        xs2 = [torch.zeros_like(b) for b in bs]
        st, inf = B.gmres_batched(ops, bs, xs2, **kw2)
        assert st == B.SG_ENOTCONV
        for k, op in enumerate(ops):
            x1 = torch.zeros_like(bs[k])
            try:
                ref = op.gmres(bs[k], x1, **kw2)
            except B.SgError as e:
                ref = dict(status=e.status)
            assert inf[k]["status"] == ref["status"], (k, inf[k], ref)
            assert torch.equal(xs2[k], x1), k
    for op in ops:
        op.close()


def test_graph_route_64_heterogeneous_systems(B):
    """The 64-system workload (g 63 ... 255, P 6 ... 35): many chains in
    flight at once, transforms large enough for X by tensor copies.  Both
    routes converge every system with equal bits and counts; the FP64
    residual, formed on the device, meets tol."""
    probs = inputs.batch_64()
    ops = [B.SG(p) for p in probs]
    bs = []
    for op in ops:
        b = torch.empty(op.N, dtype=torch.complex128, device=DEV)
        op.rhs(b, B.FP64)
        bs.append(b)
    kw = dict(restart=30, tol=1e-8, prec=B.PREC_MEAN, mode=B.MIXED, maxit=20000)
    xg = [torch.zeros_like(b) for b in bs]
    stg, infg = B.gmres_batched(ops, bs, xg, **kw)
    xp = [torch.zeros_like(b) for b in bs]
    stp, infp = B.gmres_batched(ops, bs, xp, concurrency=-1, **kw)
    assert stg == stp == B.SG_OK
    for k, op in enumerate(ops):
        assert infg[k]["status"] == B.SG_OK and infg[k]["graph_outer"] >= 1, (k, infg[k])
        assert infg[k]["iters"] == infp[k]["iters"] and infg[k]["outer"] == infp[k]["outer"], (k, infg[k], infp[k])
        assert torch.equal(xg[k], xp[k]), k
        ax = torch.empty_like(xg[k])
        op.matvec(xg[k], ax, B.FP64)
        relres = (torch.linalg.vector_norm(bs[k] - ax) / torch.linalg.vector_norm(bs[k])).item()
        assert relres <= 1e-8, (k, relres)
    # the oracle's residual and direct solution for the three smallest systems
    small = sorted(range(len(ops)), key=lambda k: ops[k].N)[:3]
    for k in small:
        ref = sg.assemble_problem(probs[k])
        assert np.array_equal(bs[k].cpu().numpy(), ref.b)
        xk = xg[k].cpu().numpy()
        rr = np.linalg.norm(ref.b - ref.A @ xk) / np.linalg.norm(ref.b)
        assert rr <= 1e-8, (k, rr)
        from oracle import krylov
        xd = krylov.direct(ref.A, ref.b)
        assert np.linalg.norm(xk - xd) / np.linalg.norm(xd) <= 1e-5, k
    for op in ops:
        op.close()


@pytest.mark.parametrize("policy", ["scaled", "fallback", "as_given"])
def test_graph_route_with_initial_guesses(B, policy):
    """Per-system guesses on the graph route: good guesses (the solution
    perturbed), one guess worse than zero (restarted from zero by sg_gmres:
    the graph hands that system back under SG_X0_FALLBACK; scaled, it is
    never worse than zero; as given, it is kept), one
    system without a guess and one with b = 0; every system equals the
    one-at-a-time sg_gmres with the same guess, bit for bit."""
    pol = {"scaled": B.X0_SCALED, "fallback": B.X0_FALLBACK, "as_given": B.X0_AS_GIVEN}[policy]
    probs = batch_problems()[:5]
    ops = [B.SG(p) for p in probs]
    refs = [sg.assemble_problem(p) for p in probs]
    bs = [torch.from_numpy(r.b).to(DEV) for r in refs]
    bs[4].zero_()
    rng = np.random.default_rng(9)
    x0s = []
    for k, r in enumerate(refs):
        xd = np.linalg.solve(r.A.toarray(), r.b) if r.A.shape[0] <= 4000 else None
        if k == 2:
            x0s.append(None)
            continue
        if k == 1 or xd is None:
            g = 1e3 * (rng.standard_normal(r.A.shape[0]) + 1j * rng.standard_normal(r.A.shape[0]))
        else:
            g = xd * (1 + 0.05 * rng.standard_normal(xd.shape))
        x0s.append(torch.from_numpy(g).to(DEV))
    kw = dict(restart=20, tol=1e-9, prec=B.PREC_MEAN, mode=B.MIXED, maxit=5000, x0_policy=pol)
    seq = []
    for op, b, g in zip(ops, bs, x0s):
        x = torch.zeros_like(b)
        inf = op.gmres(b, x, x0=g, **kw)
        seq.append((x, inf))
    xs = [torch.full_like(b, float("nan")) for b in bs]
    st, infos = B.gmres_batched(ops, bs, xs, x0s=x0s, **kw)
    statuses = [i0["status"] for _, i0 in seq]
    assert st == (B.SG_OK if all(s == B.SG_OK for s in statuses) else B.SG_ENOTCONV)
    for k in range(len(ops)):
        x1, i0 = seq[k]
        assert infos[k]["status"] == i0["status"], (k, infos[k], i0)
        assert infos[k]["iters"] == i0["iters"] and infos[k]["outer"] == i0["outer"], (k, infos[k], i0)
        assert torch.equal(xs[k], x1), k
    assert not xs[4].any() and infos[4]["relres"] == 0.0
    if pol == B.X0_FALLBACK:
        assert infos[1]["graph_outer"] == 0          # handed back: its guess is worse than zero
    assert infos[0]["graph_outer"] >= 1 and infos[2]["graph_outer"] >= 1
    for op in ops:
        op.close()
