"""Learned initial guess for the SG-GMRES solve (a throughput aid; the paper
has no learned component).

Pipeline, all device work in the library's kernels (this module only moves
arguments around):

1. training data: SG solutions of the parametrised 2D workload (mean
   wavenumber, sigma, correlation length, source position), solved by the
   batched GPU GMRES (`sg_gmres_batched`, mixed precision with FP64
   refinement) to a tolerance well below the one the warm start serves;
2. decoder: rank-R POD of the solutions — Gram matrix of a snapshot subset
   (`sg_cgemm_hn`), its Hermitian eigen-decomposition (a small dense
   problem of size n_snapshots, done on the host once), modes
   U = Lambda^-1/2 V^T S (`sg_cgemm_nn`), V the eigenvectors;
3. targets: coefficients of every training solution on U (`sg_cgemm_hn`),
   scaled to unit RMS;
4. network: 5 -> 512 -> 512 -> 512 -> 2R, tanh, bf16 weights with FP32
   accumulation, trained with Adam by `sg_mlp_train`;
5. inference: x0 = (net(params) as R complex) * scale @ U (`sg_warmstart_predict`:
   normalisation, network and expansion on the device), then `sg_gmres` from x0
   with the zero-guess fallback on.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import binding as B
from . import inputs

PARAM_LO = np.array([10.0, 0.05, 0.1, 0.2, 0.2])
PARAM_HI = np.array([40.0, 0.2, 0.5, 0.8, 0.8])


def normalise(params: np.ndarray, lo=PARAM_LO, hi=PARAM_HI) -> np.ndarray:
    """Map the parameter box [lo, hi] to [-1, 1]^5 (network input)."""
    p = np.atleast_2d(np.asarray(params, dtype=np.float64))
    return (2.0 * (p - lo) / (hi - lo) - 1.0).astype(np.float32)


def xavier_params(dims, seed: int) -> np.ndarray:
    """Flat FP32 parameters in the C ABI layout, Xavier-uniform weights, zero
    biases (random numbers drawn here and passed to the library)."""
    rng = np.random.default_rng(seed)
    out = []
    for l in range(len(dims) - 1):
        a = np.sqrt(6.0 / (dims[l] + dims[l + 1]))
        out.append(rng.uniform(-a, a, dims[l + 1] * dims[l]))
        out.append(np.zeros(dims[l + 1]))
    return np.concatenate(out).astype(np.float32)


def solve_batch(params, torch, dev, g=127, s=3, r=3, tol=1e-10, restart=50, chunk=64, mode=None):
    """SG solutions for every parameter row, solved `chunk` systems at a time
    by the batched solver; returns (S complex64 n_samples x N on the device,
    iteration counts)."""
    mode = B.MIXED if mode is None else mode
    S = None
    iters = []
    for c0 in range(0, len(params), chunk):
        ops = [B.SG(inputs.warmstart_problem(p, g, s, r)) for p in params[c0:c0 + chunk]]
        if S is None:
            S = torch.empty((len(params), ops[0].N), dtype=torch.complex64, device=dev)
        bs, xs = [], []
        for op in ops:
            b = torch.empty(op.N, dtype=torch.complex128, device=dev)
            op.rhs(b, B.FP64)
            bs.append(b)
            xs.append(torch.zeros_like(b))
        st, infos = B.gmres_batched(ops, bs, xs, restart=restart, tol=tol, prec=B.PREC_MEAN, mode=mode,
                                    maxit=20000)
        if st != B.SG_OK:
            raise B.SgError(st, "training solve did not converge")
        for k, x in enumerate(xs):
            S[c0 + k].copy_(x)
        iters += [f["iters"] for f in infos]
        for op in ops:
            op.close()
    return S, iters


@dataclass
class WarmStart:
    U: object          # rank x N complex64 (device), rows orthonormal
    Udec: object       # scale * U
    mlp: B.MLP
    scale: float
    rank: int
    loss_history: list
    energy_captured: float
    lo: np.ndarray
    hi: np.ndarray
    timings: dict
    model: B.WarmStartModel = None   # sg_warmstart: normalisation, network, expansion on the device

    def predict(self, params, torch, dev):
        """x0 (k x N complex128, device) for k parameter rows, by
        sg_warmstart_predict."""
        p = np.atleast_2d(np.asarray(params, dtype=np.float64))
        x0 = torch.empty((p.shape[0], self.U.shape[1]), dtype=torch.complex128, device=dev)
        self.model.predict(p, x0)
        return x0


def pod_basis(S, rank, n_snapshots, torch, dev):
    """Rank-`rank` POD basis of the first n_snapshots rows of S (n x N
    complex64, device): rows u_i = lambda_i^-1/2 sum_k V_ki s_k from the
    eigenpairs (lambda_i, V_i) of the snapshot Gram matrix, in decreasing
    lambda, orthonormal.  Returns U (rank x N complex64, device) and all
    eigenvalues in decreasing order (host)."""
    n, N = S.shape
    ns = min(n_snapshots, n)
    G = torch.empty((ns, ns), dtype=torch.complex64, device=dev)
    work = torch.empty(ns * ns, dtype=torch.complex128, device=dev)
    B.cgemm_hn(S, N, S, N, ns, ns, N, G, work)
    Gh = G.cpu().numpy().astype(np.complex128)
    Gh = 0.5 * (Gh + Gh.conj().T)
    lam, V = np.linalg.eigh(Gh)
    order = np.argsort(lam)[::-1]
    rank = min(rank, ns)
    lam_top = np.maximum(lam[order[:rank]], 1e-30)
    W = (V[:, order[:rank]] / np.sqrt(lam_top)).T.astype(np.complex64)
    U = torch.empty((rank, N), dtype=torch.complex64, device=dev)
    B.cgemm_nn(torch.from_numpy(np.ascontiguousarray(W)).to(dev), S[:ns].contiguous(), rank, N, ns, U)
    return U, lam[order]


def pod_errors(U, X, ranks, torch, dev):
    """Best-approximation errors of the rows x_j of X (m x N complex64,
    device) in the spans of the first R rows of U (orthonormal), for each R
    in ranks: ||x - P_R x|| / ||x|| = sqrt(1 - sum_{i<R} |<u_i, x>|^2 /
    ||x||^2).  Returns {R: per-row errors (host)} -- the floor that any
    decoder x0 = U_R c reaches with the best coefficients c."""
    r, N = U.shape
    m = X.shape[0]
    Cm = torch.empty((r, m), dtype=torch.complex64, device=dev)
    work = torch.empty(r * m, dtype=torch.complex128, device=dev)
    B.cgemm_hn(U, N, X, N, r, m, N, Cm, work)
    c2 = (Cm.abs().double() ** 2).cpu().numpy()               # r x m
    x2 = (X.abs().double() ** 2).sum(dim=1).cpu().numpy()     # m
    csum = np.cumsum(c2, axis=0)
    return {R: np.sqrt(np.clip(1.0 - csum[min(R, r) - 1] / x2, 0.0, None)) for R in ranks}


def build(params, S, torch, dev, rank=64, n_snapshots=512, width=512, hidden=3, epochs=300, batch=128, lr=1e-3,
          seed=7, lo=PARAM_LO, hi=PARAM_HI):
    """POD decoder + trained network from training parameters (n x 5, host)
    and their solutions S (n x N complex64, device)."""
    import time
    n, N = S.shape
    ns = min(n_snapshots, n)
    timings = {}
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    # POD of the first ns snapshots
    G = torch.empty((ns, ns), dtype=torch.complex64, device=dev)
    work = torch.empty(ns * ns, dtype=torch.complex128, device=dev)
    B.cgemm_hn(S, N, S, N, ns, ns, N, G, work)
    Gh = G.cpu().numpy().astype(np.complex128)
    timings["gram_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    Gh = 0.5 * (Gh + Gh.conj().T)
    lam, V = np.linalg.eigh(Gh)
    order = np.argsort(lam)[::-1][:rank]
    lam_top = np.maximum(lam[order], 1e-30)
    W = (V[:, order] / np.sqrt(lam_top)).T.astype(np.complex64)           # rank x ns
    energy = float(lam_top.sum() / max(lam.clip(min=0).sum(), 1e-300))
    timings["eig_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    Wd = torch.from_numpy(np.ascontiguousarray(W)).to(dev)
    U = torch.empty((rank, N), dtype=torch.complex64, device=dev)
    B.cgemm_nn(Wd, S[:ns].contiguous(), rank, N, ns, U)
    # coefficients of every solution on U
    Cm = torch.empty((rank, n), dtype=torch.complex64, device=dev)
    work2 = torch.empty(rank * n, dtype=torch.complex128, device=dev)
    B.cgemm_hn(U, N, S, N, rank, n, N, Cm, work2)
    T = torch.view_as_real(Cm.t().contiguous()).reshape(n, 2 * rank).contiguous()
    scale = float(T.pow(2).mean().sqrt().item()) or 1.0
    T = (T / scale).contiguous()
    X = torch.from_numpy(normalise(params, lo, hi)).to(dev)
    perm = torch.from_numpy(np.random.default_rng(seed).permutation(n)).to(dev)
    X, T = X[perm].contiguous(), T[perm].contiguous()
    torch.cuda.synchronize(dev)
    timings["basis_targets_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    mlp = B.MLP(5, width, hidden, 2 * rank)
    dims = [5] + [width] * hidden + [2 * rank]
    mlp.set_params(torch.from_numpy(xavier_params(dims, seed)).to(dev))
    hist = mlp.train(X, T, batch, epochs, lr)
    timings["train_s"] = time.perf_counter() - t0
    Udec = (U * scale).contiguous()
    model = B.WarmStartModel(mlp, Udec, rank, lo, hi)
    return WarmStart(U, Udec, mlp, scale, rank, hist, energy, np.asarray(lo, float), np.asarray(hi, float),
                     timings, model)
