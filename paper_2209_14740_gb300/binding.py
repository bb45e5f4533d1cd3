"""Thin Python binding of the C ABI in include/sg.h (argument marshalling only).

Every computation runs in libsg_gb300.so.  Device buffers are passed as raw
pointers taken from torch tensors (torch supplies device memory and streams,
nothing else).  If the shared library is missing this module raises at once:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libsg_gb300.so")

SG_OK, SG_EINVAL, SG_ENOMEM, SG_ECUDA, SG_ENOTCONV, SG_EBREAKDOWN, SG_ESINGULAR, SG_ETIMEOUT, SG_EUNSUPPORTED = range(9)
STATUS_NAMES = ["SG_OK", "SG_EINVAL", "SG_ENOMEM", "SG_ECUDA", "SG_ENOTCONV", "SG_EBREAKDOWN",
                "SG_ESINGULAR", "SG_ETIMEOUT", "SG_EUNSUPPORTED"]
BC_DIRICHLET, BC_ABSORBING = 0, 1
PREC_NONE, PREC_MEAN, PREC_CSL_MEAN, PREC_CSL = 0, 1, 2, 3
FP64, FP32, MIXED, TF32, FP16 = 0, 1, 2, 3, 4
X0_AS_GIVEN, X0_FALLBACK, X0_SCALED = 0, 1, 2

# every symbol include/sg.h declares
EXPORTED = ["sg_assemble", "sg_destroy", "sg_get_info", "sg_rhs", "sg_matvec", "sg_precond", "sg_gmres",
            "sg_last_error", "sg_version", "sg_kernel_launches", "sg_precond_noalloc", "sg_gmres_batched",
            "sg_mlp_create", "sg_mlp_destroy", "sg_mlp_num_params", "sg_mlp_set_params", "sg_mlp_get_params",
            "sg_mlp_forward", "sg_mlp_loss_grad", "sg_mlp_train", "sg_cgemm_hn", "sg_cgemm_nn",
            "sg_selftest_wait_timeout", "sg_alu_peak", "sg_stationary", "sg_statistics",
            "sg_warmstart_create", "sg_warmstart_destroy", "sg_warmstart_predict", "sg_autotune", "sg_tune_get",
            "sg_tune_set", "sg_fd_transform", "sg_cgs2_pass"]
NOALLOC_MAX_N = 524288   # SG_NOALLOC_MAX_N in include/sg.h


class SgDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("h", C.c_double),
                ("bc", C.c_int * 4), ("s", C.c_int), ("r", C.c_int),
                ("k0", C.POINTER(C.c_double)), ("kl", C.POINTER(C.c_double)), ("f", C.POINTER(C.c_double)),
                ("beta", C.c_double), ("point_source", C.c_int), ("point_x", C.c_double), ("point_y", C.c_double)]


class SgInfo(C.Structure):
    _fields_ = [("dim", C.c_int), ("mx", C.c_int), ("my", C.c_int), ("n", C.c_int), ("P", C.c_int),
                ("N", C.c_longlong), ("s", C.c_int), ("r", C.c_int), ("terms", C.c_int),
                ("coupling_nnz", C.c_int), ("separable", C.c_int), ("specialised", C.c_int),
                ("fast_diag", C.c_int), ("eig_orth_err", C.c_double), ("eig_kappa", C.c_double),
                ("tf32_route", C.c_int), ("fp16_route", C.c_int)]


class SgGmresOpts(C.Structure):
    _fields_ = [("restart", C.c_int), ("maxit", C.c_int), ("max_outer", C.c_int), ("tol", C.c_double),
                ("inner_tol", C.c_double), ("prec", C.c_int), ("mode", C.c_int), ("x0", C.c_void_p),
                ("host_io", C.c_int), ("check_every", C.c_int), ("x0_policy", C.c_int), ("side", C.c_int),
                ("basis16", C.c_int)]


class SgGmresInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer", C.c_int), ("cycles", C.c_int), ("relres", C.c_double),
                ("status", C.c_int), ("relres_prec", C.c_double), ("graph_outer", C.c_int)]


class SgTune(C.Structure):
    _fields_ = [("cgs_blocks_per_sm", C.c_int), ("op_ctas_per_sm", C.c_int), ("tc_tile_n", C.c_int),
                ("tf32_transforms", C.c_int), ("cgs_us", C.c_double), ("op_us", C.c_double), ("apply_us", C.c_double)]


TUNE_KEYS = ("cgs_blocks_per_sm", "op_ctas_per_sm", "tc_tile_n", "tf32_transforms")


class SgStationaryOpts(C.Structure):
    _fields_ = [("prec", C.c_int), ("mode", C.c_int), ("maxit", C.c_int), ("tol", C.c_double),
                ("x0_given", C.c_int)]


class SgStationaryInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("relres", C.c_double), ("diverged", C.c_int), ("status", C.c_int)]


class SgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load the shared library (raises OSError if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libsg_gb300.so not built (run __graft_entry__.build()): %s" % path)
    lib = C.CDLL(path)
    vp, i = C.c_void_p, C.c_int
    lib.sg_assemble.argtypes = [C.POINTER(SgDesc), vp, C.POINTER(vp)]
    lib.sg_assemble.restype = i
    lib.sg_destroy.argtypes = [vp]
    lib.sg_destroy.restype = None
    lib.sg_get_info.argtypes = [vp, C.POINTER(SgInfo)]
    lib.sg_get_info.restype = i
    lib.sg_rhs.argtypes = [vp, i, vp, vp]
    lib.sg_rhs.restype = i
    lib.sg_matvec.argtypes = [vp, i, vp, vp, vp]
    lib.sg_matvec.restype = i
    lib.sg_precond.argtypes = [vp, i, i, vp, vp, vp]
    lib.sg_precond.restype = i
    lib.sg_gmres.argtypes = [vp, C.POINTER(SgGmresOpts), vp, vp, C.POINTER(SgGmresInfo), vp]
    lib.sg_gmres.restype = i
    lib.sg_last_error.argtypes = []
    lib.sg_last_error.restype = C.c_char_p
    lib.sg_version.argtypes = []
    lib.sg_version.restype = i
    lib.sg_kernel_launches.argtypes = []
    lib.sg_kernel_launches.restype = C.c_longlong
    lib.sg_precond_noalloc.argtypes = [vp, i, i, vp, vp, vp]
    lib.sg_precond_noalloc.restype = i
    lib.sg_gmres_batched.argtypes = [C.POINTER(vp), i, C.POINTER(SgGmresOpts), C.POINTER(vp), C.POINTER(vp),
                                     C.POINTER(vp), C.POINTER(SgGmresInfo), i, vp]
    lib.sg_gmres_batched.restype = i
    fp, dp = C.POINTER(C.c_float), C.POINTER(C.c_double)
    lib.sg_mlp_create.argtypes = [i, i, i, i, C.POINTER(vp)]
    lib.sg_mlp_create.restype = i
    lib.sg_mlp_destroy.argtypes = [vp]
    lib.sg_mlp_destroy.restype = None
    lib.sg_mlp_num_params.argtypes = [vp]
    lib.sg_mlp_num_params.restype = C.c_longlong
    lib.sg_mlp_set_params.argtypes = [vp, vp, vp]
    lib.sg_mlp_set_params.restype = i
    lib.sg_mlp_get_params.argtypes = [vp, vp, vp]
    lib.sg_mlp_get_params.restype = i
    lib.sg_mlp_forward.argtypes = [vp, vp, i, vp, vp]
    lib.sg_mlp_forward.restype = i
    lib.sg_mlp_loss_grad.argtypes = [vp, vp, vp, i, dp, vp, vp]
    lib.sg_mlp_loss_grad.restype = i
    lib.sg_mlp_train.argtypes = [vp, vp, vp, i, i, i, C.c_float, dp, vp]
    lib.sg_mlp_train.restype = i
    lib.sg_cgemm_hn.argtypes = [vp, C.c_longlong, vp, C.c_longlong, i, i, C.c_longlong, vp, vp, vp]
    lib.sg_cgemm_hn.restype = i
    lib.sg_cgemm_nn.argtypes = [vp, vp, i, i, i, vp, i, vp]
    lib.sg_cgemm_nn.restype = i
    lib.sg_selftest_wait_timeout.argtypes = [vp, C.POINTER(i), dp]
    lib.sg_selftest_wait_timeout.restype = i
    lib.sg_alu_peak.argtypes = [i, dp, vp]
    lib.sg_alu_peak.restype = i
    lib.sg_fd_transform.argtypes = [vp, i, i, i, vp, vp, vp]
    lib.sg_fd_transform.restype = i
    lib.sg_cgs2_pass.argtypes = [vp, i, i, i, vp]
    lib.sg_cgs2_pass.restype = i
    lib.sg_autotune.argtypes = [vp, i, C.POINTER(SgTune), vp]
    lib.sg_autotune.restype = i
    lib.sg_tune_get.argtypes = [vp, C.POINTER(SgTune)]
    lib.sg_tune_get.restype = i
    lib.sg_tune_set.argtypes = [vp, C.POINTER(SgTune)]
    lib.sg_tune_set.restype = i
    lib.sg_stationary.argtypes = [vp, C.POINTER(SgStationaryOpts), vp, vp, C.POINTER(SgStationaryInfo), dp, vp]
    lib.sg_stationary.restype = i
    lib.sg_statistics.argtypes = [vp, i, vp, vp, vp, vp, dp, vp]
    lib.sg_statistics.restype = i
    lib.sg_warmstart_create.argtypes = [vp, vp, i, C.c_longlong, dp, dp, C.POINTER(vp)]
    lib.sg_warmstart_create.restype = i
    lib.sg_warmstart_destroy.argtypes = [vp]
    lib.sg_warmstart_destroy.restype = None
    lib.sg_warmstart_predict.argtypes = [vp, dp, i, vp, vp]
    lib.sg_warmstart_predict.restype = i
    del fp
    _lib = lib
    return lib


def alu_peak(fp64: bool, stream=None) -> float:
    """sg_alu_peak: measured FMA rate of the CUDA cores in TFLOP/s."""
    v = C.c_double(0.0)
    _check(load().sg_alu_peak(1 if fp64 else 0, C.byref(v), _stream(stream)))
    return v.value


def kernel_launches() -> int:
    return int(load().sg_kernel_launches())


def selftest_wait_timeout(stream=None):
    """sg_selftest_wait_timeout: (status, timed_out, seconds)."""
    lib = load()
    t = C.c_int(0)
    sec = C.c_double(0.0)
    st = lib.sg_selftest_wait_timeout(_stream(stream), C.byref(t), C.byref(sec))
    return st, t.value, sec.value


class MLP:
    """sg_mlp: the warm-start network (device parameters, native kernels)."""

    def __init__(self, in_dim, width, hidden, out_dim):
        h = C.c_void_p()
        _check(load().sg_mlp_create(in_dim, width, hidden, out_dim, C.byref(h)))
        self.h = h
        self.nparams = int(load().sg_mlp_num_params(h))
        self.in_dim, self.out_dim = in_dim, out_dim

    def close(self):
        if getattr(self, "h", None):
            load().sg_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p, stream=None):
        _check(load().sg_mlp_set_params(self.h, _ptr(p), _stream(stream)))

    def get_params(self, p, stream=None):
        _check(load().sg_mlp_get_params(self.h, _ptr(p), _stream(stream)))

    def forward(self, X, Y, stream=None):
        _check(load().sg_mlp_forward(self.h, _ptr(X), X.shape[0], _ptr(Y), _stream(stream)))

    def loss_grad(self, X, T, grad=None, stream=None):
        loss = C.c_double()
        _check(load().sg_mlp_loss_grad(self.h, _ptr(X), _ptr(T), X.shape[0], C.byref(loss),
                                       _ptr(grad) if grad is not None else None, _stream(stream)))
        return loss.value

    def train(self, X, T, batch, epochs, lr, stream=None):
        hist = (C.c_double * max(epochs, 1))()
        _check(load().sg_mlp_train(self.h, _ptr(X), _ptr(T), X.shape[0], batch, epochs, C.c_float(lr), hist,
                                   _stream(stream)))
        return list(hist)[:epochs]


class WarmStartModel:
    """sg_warmstart: a trained network plus its decoder, predicting initial
    guesses on the device."""

    def __init__(self, mlp, D, rank, lo, hi):
        self._lo = np.ascontiguousarray(lo, dtype=np.float64)
        self._hi = np.ascontiguousarray(hi, dtype=np.float64)
        self.mlp = mlp                       # the model borrows the network
        self.rank, self.N = rank, int(D.shape[-1])
        h = C.c_void_p()
        dp = C.POINTER(C.c_double)
        _check(load().sg_warmstart_create(mlp.h, _ptr(D), rank, self.N, self._lo.ctypes.data_as(dp),
                                          self._hi.ctypes.data_as(dp), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().sg_warmstart_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def predict(self, params, x0, stream=None):
        """x0 (device, count x N complex128) for the parameter rows (host)."""
        p = np.ascontiguousarray(np.atleast_2d(params), dtype=np.float64)
        _check(load().sg_warmstart_predict(self.h, p.ctypes.data_as(C.POINTER(C.c_double)), p.shape[0], _ptr(x0),
                                           _stream(stream)))


def cgemm_hn(A, lda, B, ldb, m, n, k, Cout, work, stream=None):
    _check(load().sg_cgemm_hn(_ptr(A), lda, _ptr(B), ldb, m, n, k, _ptr(Cout), _ptr(work), _stream(stream)))


def cgemm_nn(A, B, m, n, k, Cout, out_c128=False, stream=None):
    _check(load().sg_cgemm_nn(_ptr(A), _ptr(B), m, n, k, _ptr(Cout), 1 if out_c128 else 0, _stream(stream)))


def _check(st):
    if st != SG_OK:
        raise SgError(st, load().sg_last_error().decode())


def _ptr(t) -> int:
    """Raw data pointer of a torch tensor or a numpy array."""
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream)


class SG:
    """One assembled SG Helmholtz system (owns an sg_handle)."""

    def __init__(self, prob, stream=None, tuned=True):
        """tuned: apply the launch shapes of the committed tuning table
        (tune_table.json) when it has this problem size."""
        lib = load()
        self._keep = []
        k0 = np.ascontiguousarray(prob.k0, dtype=np.float64)
        kl = np.ascontiguousarray(np.asarray(prob.kl, dtype=np.float64).reshape(-1))
        f = np.ascontiguousarray(prob.f, dtype=np.float64)
        self._keep += [k0, kl, f]
        d = SgDesc()
        d.dim, d.nx, d.ny, d.h = prob.dim, prob.nx, prob.ny, prob.h
        for k in range(4):
            d.bc[k] = int(prob.bc[k])
        d.s, d.r = prob.s, prob.r
        dp = C.POINTER(C.c_double)
        d.k0 = k0.ctypes.data_as(dp)
        d.kl = kl.ctypes.data_as(dp) if kl.size else None
        d.f = f.ctypes.data_as(dp)
        d.beta = float(getattr(prob, "beta", 0.5))
        pt = getattr(prob, "point", None)
        if pt is not None:
            d.point_source = 1
            d.point_x = float(pt[0])
            d.point_y = float(pt[1]) if len(pt) > 1 else 0.0
        h = C.c_void_p()
        _check(lib.sg_assemble(C.byref(d), _stream(stream), C.byref(h)))
        self.h = h
        inf = SgInfo()
        _check(lib.sg_get_info(h, C.byref(inf)))
        self.info = {k: getattr(inf, k) for k, _ in SgInfo._fields_}
        self.n, self.P, self.N = inf.n, inf.P, inf.N
        if tuned:
            from . import tune_table
            entry = tune_table.lookup(prob.dim, inf.mx, inf.my, prob.s, prob.r)
            if entry is not None:
                self.tune_set(entry)

    def fd_transform(self, t, X, Y, kind=PREC_MEAN, prec=TF32, stream=None):
        """sg_fd_transform: transform t (0 .. 3) of the fast diagonalisation
        (SG_TF32 or SG_FP16 form), X -> Y (device tensors, layouts in sg.h)."""
        _check(load().sg_fd_transform(self.h, kind, prec, t, _ptr(X), _ptr(Y), _stream(stream)))

    def cgs2_pass(self, j, pass_, restart=30, stream=None):
        """sg_cgs2_pass: pass 0 prepares the workspace, 1 / 2 launch that CGS2
        pass of Arnoldi step j of the flexible complex64 cycles."""
        _check(load().sg_cgs2_pass(self.h, restart, j, pass_, _stream(stream)))

    def autotune(self, restart=30, stream=None) -> dict:
        """sg_autotune: time the candidate launch shapes on this problem and
        keep the fastest; returns the choices and their times."""
        t = SgTune()
        _check(load().sg_autotune(self.h, restart, C.byref(t), _stream(stream)))
        return {k: getattr(t, k) for k, _ in SgTune._fields_}

    def tune_get(self) -> dict:
        t = SgTune()
        _check(load().sg_tune_get(self.h, C.byref(t)))
        return {k: getattr(t, k) for k, _ in SgTune._fields_}

    def tune_set(self, shapes: dict):
        """sg_tune_set with the keys of TUNE_KEYS (missing keys: 0 = rule)."""
        t = SgTune()
        for k in TUNE_KEYS:
            setattr(t, k, int(shapes.get(k, 0)))
        _check(load().sg_tune_set(self.h, C.byref(t)))

    def close(self):
        if getattr(self, "h", None):
            load().sg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rhs(self, b, prec=FP64, stream=None):
        _check(load().sg_rhs(self.h, prec, _ptr(b), _stream(stream)))

    def matvec(self, X, Y, prec=FP64, stream=None):
        _check(load().sg_matvec(self.h, prec, _ptr(X), _ptr(Y), _stream(stream)))

    def precond(self, R, Z, kind=PREC_MEAN, prec=FP64, stream=None):
        _check(load().sg_precond(self.h, kind, prec, _ptr(R), _ptr(Z), _stream(stream)))

    def precond_noalloc(self, R, Z, kind=PREC_MEAN, prec=FP64, stream=None):
        """sg_precond_noalloc: the same apply with the library's static scratch
        (no device memory is allocated by the call)."""
        _check(load().sg_precond_noalloc(self.h, kind, prec, _ptr(R), _ptr(Z), _stream(stream)))

    def stationary(self, b, x, *, prec=PREC_MEAN, mode=FP64, maxit=50, tol=1e-8, x0_given=False, stream=None):
        """sg_stationary: returns (info dict, relres history list)."""
        o = SgStationaryOpts()
        o.prec, o.mode, o.maxit, o.tol, o.x0_given = prec, mode, maxit, tol, 1 if x0_given else 0
        inf = SgStationaryInfo()
        hist = (C.c_double * (maxit + 1))()
        st = load().sg_stationary(self.h, C.byref(o), _ptr(b), _ptr(x), C.byref(inf), hist, _stream(stream))
        if st not in (SG_OK, SG_ENOTCONV, SG_EBREAKDOWN):
            _check(st)
        return (dict(iters=inf.iters, relres=inf.relres, diverged=inf.diverged, status=st),
                list(hist)[: inf.iters + 1])

    def statistics(self, V, mean=None, var_re=None, var_im=None, gamma=True, prec=FP64, stream=None):
        """sg_statistics: fills the given device outputs; returns gamma_0..r (or None)."""
        g = (C.c_double * (self.info["r"] + 1))() if gamma else None
        _check(load().sg_statistics(self.h, prec, _ptr(V), _ptr(mean) if mean is not None else None,
                                    _ptr(var_re) if var_re is not None else None,
                                    _ptr(var_im) if var_im is not None else None, g, _stream(stream)))
        return list(g) if gamma else None

    def gmres(self, b, x, *, restart=0, maxit=0, tol=1e-8, prec=PREC_MEAN, mode=FP64, x0=None, max_outer=0,
              inner_tol=0.0, host_io=False, check_every=0, stream=None, raise_on_notconv=False,
              x0_policy=0, side=0, basis16=0):
        o = SgGmresOpts()
        o.x0_policy = x0_policy
        o.side = side
        o.basis16 = basis16
        o.restart, o.maxit, o.max_outer, o.tol, o.inner_tol = restart, maxit, max_outer, tol, inner_tol
        o.prec, o.mode = prec, mode
        o.x0 = _ptr(x0) if x0 is not None else None
        o.host_io = 1 if host_io else 0
        o.check_every = check_every
        inf = SgGmresInfo()
        st = load().sg_gmres(self.h, C.byref(o), _ptr(b), _ptr(x), C.byref(inf),
                             None if host_io and stream is None else _stream(stream))
        if st not in (SG_OK, SG_ENOTCONV) or (raise_on_notconv and st == SG_ENOTCONV):
            _check(st)
        return dict(iters=inf.iters, outer=inf.outer, cycles=inf.cycles, relres=inf.relres, status=st,
                    relres_prec=inf.relres_prec)


def _opts(restart=0, maxit=0, tol=1e-8, prec=PREC_MEAN, mode=FP64, max_outer=0, inner_tol=0.0, host_io=False,
          check_every=0, x0_policy=0, side=0, basis16=0):
    o = SgGmresOpts()
    o.side = side
    o.basis16 = basis16
    o.restart, o.maxit, o.max_outer, o.tol, o.inner_tol = restart, maxit, max_outer, tol, inner_tol
    o.prec, o.mode = prec, mode
    o.x0 = None
    o.host_io = 1 if host_io else 0
    o.check_every = check_every
    o.x0_policy = x0_policy
    return o


def gmres_batched(ops, bs, xs, *, x0s=None, concurrency=0, stream=None, **kw):
    """sg_gmres_batched over SG objects `ops` with right-hand sides `bs`,
    solutions `xs` (torch tensors, or numpy arrays with host_io=True) and
    optional per-system initial guesses `x0s`."""
    n = len(ops)
    hs = (C.c_void_p * n)(*[op.h.value for op in ops])
    bp = (C.c_void_p * n)(*[_ptr(v) for v in bs])
    xp = (C.c_void_p * n)(*[_ptr(v) for v in xs])
    x0p = (C.c_void_p * n)(*[_ptr(v) if v is not None else None for v in x0s]) if x0s is not None else None
    infos = (SgGmresInfo * n)()
    o = _opts(**kw)
    st = load().sg_gmres_batched(hs, n, C.byref(o), bp, xp, x0p, infos, concurrency,
                                 None if kw.get("host_io") and stream is None else _stream(stream))
    if st not in (SG_OK, SG_ENOTCONV):
        _check(st)
    return st, [dict(iters=f.iters, outer=f.outer, cycles=f.cycles, relres=f.relres, status=f.status,
                     graph_outer=f.graph_outer) for f in infos]
