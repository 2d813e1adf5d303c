"""Thin ctypes binding of libplanc.so (include/planc.h).

Argument marshalling only: every step of the NNCP hot path runs in the CUDA
library.  PyTorch supplies device memory and the CUDA stream.  If the
library has not been built, importing this module raises ImportError; there
is no CPU fallback.

Layouts (see include/planc.h): X is a contiguous 1-D device tensor holding
the I_1 x ... x I_N tensor with mode 1 fastest; factors and MTTKRP results
are contiguous I_n x R row-major device tensors; Grams are R x R float64.
"""

from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libplanc.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "planc.h")

F64, F32, BF16, F16 = 0, 1, 2, 3
ALGS = {"mu": 0, "hals": 1, "bpp": 2, "admm": 3, "pgd": 4, "ucp": 5, "nes": 6}
_DT = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}


class PlancError(RuntimeError):
    """A libplanc call returned a non-OK status."""

    def __init__(self, status: int, msg: str):
        super().__init__(f"libplanc status {status}: {msg}")
        self.status = status


class NlsOpts(C.Structure):
    _fields_ = [("mu_eps", C.c_double), ("admm_max_inner", C.c_int),
                ("admm_tol", C.c_double), ("bpp_max_iter", C.c_int),
                ("pgd_steps", C.c_int), ("nes_max_inner", C.c_int),
                ("nes_tol", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("alg", C.c_int), ("iters", C.c_int), ("tol", C.c_double),
                ("nls", NlsOpts), ("use_graph", C.c_int), ("profile", C.c_int),
                ("nes_accel", C.c_int), ("batch_persistent", C.c_int)]


class Report(C.Structure):
    _fields_ = [("iters_done", C.c_int), ("rel_err", C.c_double), ("fit", C.c_double),
                ("rel_err_hist", C.POINTER(C.c_double)),
                ("inner_hist", C.POINTER(C.c_int32)),
                ("bpp_unconverged", C.c_int), ("pm_ms", C.c_float),
                ("pm_launches", C.c_int), ("launches", C.c_longlong),
                ("pm_tensor_cores", C.c_int), ("accel_hist", C.POINTER(C.c_int32)),
                ("accel_accepted", C.c_int)]


class BatchInstance(C.Structure):
    _fields_ = [("dims", C.c_int64 * 3), ("R", C.c_int), ("x_dtype", C.c_int),
                ("X", C.c_void_p), ("H", C.c_void_p * 3), ("lambda_", C.POINTER(C.c_double)),
                ("rel_err_hist", C.POINTER(C.c_double)), ("rel_err", C.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libplanc.so is not built ({LIB_PATH}); run "
            "`python -m paper_1909_01149_gb300.build` (nvcc, sm_103a)")
    lib = C.CDLL(LIB_PATH)
    P, I, I64, D = C.c_void_p, C.c_int, C.c_int64, C.c_double
    PP = C.POINTER(C.c_void_p)
    sig = {
        "planc_status_str": (C.c_char_p, [I]),
        "planc_last_error": (C.c_char_p, [P]),
        "planc_nls_opts_default": (NlsOpts, []),
        "planc_solve_opts_default": (SolveOpts, []),
        "planc_plan_split": (I, [I, C.POINTER(I64), C.POINTER(I)]),
        "planc_init": (I, [C.POINTER(P), I, C.POINTER(I64), I, I, P, I, P, I]),
        "planc_destroy": (I, [P]),
        "planc_get_split": (I, [P]),
        "planc_pm_tensor_cores": (I, [P]),
        "planc_describe": (I, [I, C.POINTER(I64), I, C.c_char_p, C.c_size_t]),
        "planc_sqnorm": (I, [P, P]),
        "planc_mttkrp": (I, [P, PP, I, P]),
        "planc_partial_mttkrp": (I, [P, PP, I, P]),
        "planc_mttkrp_all": (I, [P, PP, PP]),
        "planc_gram_hadamard": (I, [P, P, I, P]),
        "planc_gram": (I, [P, I64, P, P]),
        "planc_nls_update": (I, [P, I, C.POINTER(NlsOpts), I64, P, P, P, P, P]),
        "planc_normalize": (I, [P, I64, P, P, P]),
        "planc_fit": (I, [P, PP, P, C.POINTER(D), C.POINTER(D)]),
        "planc_nncp_solve": (I, [P, C.POINTER(SolveOpts), PP, C.POINTER(D), C.POINTER(Report)]),
        "planc_cp_grad": (I, [P, PP, PP, C.POINTER(D)]),
        "planc_sqnorm_noalloc": (I, [I, P, I64, P, P]),
        "planc_batch_solve": (I, [C.POINTER(BatchInstance), I, C.POINTER(SolveOpts), P,
                                  C.POINTER(Report)]),
        "planc_batch_schedule": (I, [C.POINTER(I)]),
        "planc_batch_plan": (I, [C.POINTER(BatchInstance), I, I, C.POINTER(I), C.POINTER(I),
                                 C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def header_functions():
    """Names of the functions include/planc.h declares."""
    import re
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*[\w\s\*]+?\b(planc_\w+)\s*\(", txt, re.M)))


def plan_split(dims) -> int:
    arr = (C.c_int64 * len(dims))(*dims)
    out = C.c_int()
    st = lib.planc_plan_split(len(dims), arr, C.byref(out))
    if st != 0:
        raise PlancError(st, lib.planc_last_error(None).decode())
    return out.value


def describe(dims, split: int = -1) -> str:
    """The dimension-tree schedule (host-only, no GPU needed)."""
    arr = (C.c_int64 * len(dims))(*dims)
    buf = C.create_string_buffer(16384)
    st = lib.planc_describe(len(dims), arr, int(split), buf, 16384)
    if st != 0:
        raise PlancError(st, lib.planc_last_error(None).decode())
    return buf.value.decode()


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _ptrs(ts):
    return (C.c_void_p * len(ts))(*[None if t is None else t.data_ptr() for t in ts])


def _check_mat(t, rows, cols, dtype, what):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and
            t.dtype == dtype and tuple(t.shape) == (rows, cols)):
        got = (tuple(t.shape), t.dtype, t.device) if isinstance(t, torch.Tensor) else type(t)
        raise ValueError(f"{what} must be a contiguous CUDA {dtype} tensor of shape "
                         f"({rows}, {cols}), got {got}")


def _check_buf(t, numel, dtype, what):
    """The library reads and writes through raw pointers: a buffer must be a
    contiguous CUDA tensor of the expected dtype with room for `numel` entries.
    Raises ValueError naming the first property that fails."""
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{what} must be a torch tensor, got {type(t)}")
    if t.dtype != dtype:
        raise ValueError(f"{what} must have dtype {dtype}, got {t.dtype}")
    if t.numel() < numel:
        raise ValueError(f"{what} needs at least {numel} entries, got {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor, got {t.device}")


def _rows_of(H, R, dtype, what):
    if not (isinstance(H, torch.Tensor) and H.dim() == 2):
        raise ValueError(f"{what} must be a 2-D (rows, {R}) tensor")
    _check_mat(H, H.shape[0], R, dtype, what)
    return H.shape[0]


class Context:
    """One planc_t: the tensor X (borrowed), its rank, split and workspace."""

    def __init__(self, X: torch.Tensor, dims, R: int, split: int = -1, stream=None):
        if not X.is_cuda or not X.is_contiguous():
            raise ValueError("X must be a contiguous CUDA tensor (mode-1-fastest flat buffer)")
        if X.dtype not in _DT:
            raise ValueError(f"unsupported X dtype {X.dtype}")
        n = 1
        for d in dims:
            n *= int(d)
        if n != X.numel():
            raise ValueError(f"X has {X.numel()} entries, dims {tuple(dims)} need {n}")
        self.X = X  # keep the borrowed buffer alive
        self.dims = tuple(int(d) for d in dims)
        self.N = len(self.dims)
        self.R = int(R)
        self.fdtype = torch.float64 if X.dtype == torch.float64 else torch.float32
        self.device = X.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(X.device)
        arr = (C.c_int64 * self.N)(*self.dims)
        h = C.c_void_p()
        st = lib.planc_init(C.byref(h), self.N, arr, self.R, _DT[X.dtype], _ptr(X),
                            _DT[self.fdtype], self.stream.cuda_stream, int(split))
        if st != 0:
            raise PlancError(st, lib.planc_last_error(None).decode())
        self.h = h

    # -- helpers
    def _check(self, st):
        if st != 0:
            raise PlancError(st, lib.planc_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib.planc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def split(self) -> int:
        return lib.planc_get_split(self.h)

    def describe(self) -> str:
        return describe(self.dims, self.split)

    @property
    def tc_mask(self) -> int:
        """bit 0 / bit 1: left / right partial MTTKRP on the tensor cores."""
        return lib.planc_pm_tensor_cores(self.h)

    def _empty(self, rows, cols=None):
        cols = self.R if cols is None else cols
        return torch.empty((rows, cols), dtype=self.fdtype, device=self.device)

    # -- steps of Alg. 1
    def sqnorm(self) -> torch.Tensor:
        out = torch.empty(1, dtype=torch.float64, device=self.device)
        self._check(lib.planc_sqnorm(self.h, _ptr(out)))
        return out

    def _check_H(self, H, skip=None):
        if len(H) != self.N:
            raise ValueError(f"need {self.N} factors")
        for k, h in enumerate(H):
            if k != skip:
                _check_mat(h, self.dims[k], self.R, self.fdtype, f"H[{k}]")

    def mttkrp(self, H, n: int, M: torch.Tensor | None = None) -> torch.Tensor:
        if 0 <= n < self.N:
            self._check_H(H, skip=n)
        M = self._empty(self.dims[n] if 0 <= n < self.N else 1) if M is None else M
        if 0 <= n < self.N:
            _check_buf(M, self.dims[n] * self.R, self.fdtype, "M")
        self._check(lib.planc_mttkrp(self.h, _ptrs(H), int(n), _ptr(M)))
        return M

    def mttkrp_all(self, H, M=None):
        """M^(n) for every mode through one dimension-tree pass."""
        self._check_H(H)
        M = [torch.empty_like(h) for h in H] if M is None else M
        self._check_H(M)
        self._check(lib.planc_mttkrp_all(self.h, _ptrs(H), _ptrs(M)))
        return M

    def partial_mttkrp(self, H, side: int, T: torch.Tensor | None = None) -> torch.Tensor:
        S = self.split
        rows = 1
        for d in (self.dims[:S] if side == 0 else self.dims[S:]):
            rows *= d
        self._check_H(H)
        if T is None:
            T = torch.empty(self.R * rows, dtype=self.fdtype, device=self.device)
        _check_buf(T, self.R * rows, self.fdtype, "T")
        self._check(lib.planc_partial_mttkrp(self.h, _ptrs(H), int(side), _ptr(T)))
        return T

    def gram_hadamard(self, G: torch.Tensor, n: int, S: torch.Tensor | None = None):
        S = torch.empty((self.R, self.R), dtype=torch.float64, device=self.device) if S is None else S
        _check_buf(G, self.N * self.R * self.R, torch.float64, "G")
        _check_buf(S, self.R * self.R, torch.float64, "S")
        self._check(lib.planc_gram_hadamard(self.h, _ptr(G), int(n), _ptr(S)))
        return S

    def gram(self, H: torch.Tensor, G: torch.Tensor | None = None) -> torch.Tensor:
        rows = _rows_of(H, self.R, self.fdtype, "H")
        G = torch.empty((self.R, self.R), dtype=torch.float64, device=self.device) if G is None else G
        _check_buf(G, self.R * self.R, torch.float64, "G")
        self._check(lib.planc_gram(self.h, rows, _ptr(H), _ptr(G)))
        return G

    def nls_update(self, alg: str, S, M, H, aux=None, opts: NlsOpts | None = None,
                   inner: torch.Tensor | None = None):
        o = lib.planc_nls_opts_default() if opts is None else opts
        rows = _rows_of(H, self.R, self.fdtype, "H")
        _check_buf(S, self.R * self.R, torch.float64, "S")
        _check_buf(M, rows * self.R, self.fdtype, "M")
        if aux is not None:
            _check_buf(aux, rows * self.R, self.fdtype, "aux")
        if inner is not None:
            _check_buf(inner, 1, torch.int32, "inner")
        self._check(lib.planc_nls_update(
            self.h, ALGS[alg], C.byref(o), rows, _ptr(S), _ptr(M), _ptr(H),
            None if aux is None else _ptr(aux), None if inner is None else _ptr(inner)))
        return H

    def normalize(self, H, lam: torch.Tensor | None = None, G: torch.Tensor | None = None):
        rows = _rows_of(H, self.R, self.fdtype, "H")
        lam = torch.empty(self.R, dtype=torch.float64, device=self.device) if lam is None else lam
        _check_buf(lam, self.R, torch.float64, "lam")
        if G is not None:
            _check_buf(G, self.R * self.R, torch.float64, "G")
        self._check(lib.planc_normalize(self.h, rows, _ptr(H), _ptr(lam),
                                        None if G is None else _ptr(G)))
        return H, lam

    def fit(self, H, lam: torch.Tensor):
        self._check_H(H)
        _check_buf(lam, self.R, torch.float64, "lam")
        e = C.c_double()
        f = C.c_double()
        self._check(lib.planc_fit(self.h, _ptrs(H), _ptr(lam), C.byref(e), C.byref(f)))
        return e.value, f.value

    def solve(self, H, alg: str = "hals", iters: int = 10, tol: float = 0.0,
              use_graph: bool = True, profile: bool = False, nls: NlsOpts | None = None,
              nes_accel: bool = True):
        o = lib.planc_solve_opts_default()
        o.nes_accel = 1 if nes_accel else 0
        o.alg = ALGS[alg]
        o.iters = int(iters)
        o.tol = float(tol)
        if nls is not None:
            o.nls = nls
        o.use_graph = 1 if use_graph else 0
        o.profile = 1 if profile else 0
        self._check_H(H)
        lam = (C.c_double * self.R)()
        hist = (C.c_double * max(1, iters))()
        inner = (C.c_int32 * max(1, iters * self.N))()
        rep = Report()
        rep.rel_err_hist = C.cast(hist, C.POINTER(C.c_double))
        rep.inner_hist = C.cast(inner, C.POINTER(C.c_int32))
        accel = (C.c_int32 * max(1, iters))()
        rep.accel_hist = C.cast(accel, C.POINTER(C.c_int32))
        self._check(lib.planc_nncp_solve(self.h, C.byref(o), _ptrs(H), lam, C.byref(rep)))
        n = rep.iters_done
        return dict(lam=list(lam), rel_err=list(hist[:n]), inner=list(inner[:n * self.N]),
                    iters=n, fit=rep.fit, bpp_unconverged=rep.bpp_unconverged,
                    pm_ms=rep.pm_ms, pm_launches=rep.pm_launches, launches=rep.launches,
                    use_tc=rep.pm_tensor_cores != 0, tc_mask=rep.pm_tensor_cores,
                    accepted=[bool(a) for a in accel[:n]], accel_accepted=rep.accel_accepted)

    def cp_grad(self, H, dH=None):
        """Loss ||X - [[H]]||^2 (host float) and its gradients dH (device)."""
        self._check_H(H)
        dH = [torch.empty_like(h) for h in H] if dH is None else dH
        self._check_H(dH)
        loss = C.c_double()
        self._check(lib.planc_cp_grad(self.h, _ptrs(H), _ptrs(dH), C.byref(loss)))
        return loss.value, dH


class CPLoss(torch.autograd.Function):
    """f(H^(1..N)) = ||X - [[H^(1), ..., H^(N)]]||^2 as an autograd node.

    forward runs planc_cp_grad (one call yields the loss and every factor
    gradient 2 (H^(n) S^(n) - M^(n)), the adjoint of the CP reconstruction);
    backward returns those gradients scaled by the incoming gradient.  Usage:
    ``loss = CPLoss.apply(context, *H)`` with H the context's factor tensors.
    """

    @staticmethod
    def forward(fctx, context, *H):
        loss, dH = context.cp_grad([h.detach() for h in H])
        fctx.save_for_backward(*dH)
        return torch.tensor(loss, dtype=torch.float64, device=H[0].device)

    @staticmethod
    def backward(fctx, g):
        dH = fctx.saved_tensors
        if float(g) == 1.0:
            return (None,) + tuple(dH)
        return (None,) + tuple(d * g.to(d.dtype) for d in dH)


def batch_plan(shapes, nclusters: int):
    """planc_batch_plan (host-only): how the persistent batched launch deals
    instances, given as ((I1, I2, I3), R) pairs, to `nclusters` clusters.
    Returns (lists, loads): each cluster's instance indices in the order it
    solves them, and its summed estimated cost."""
    count = len(shapes)
    if count < 1:
        raise ValueError("need at least one instance")
    arr = (BatchInstance * count)()
    for b, (dims, R) in enumerate(shapes):
        for k in range(3):
            arr[b].dims[k] = int(dims[k])
        arr[b].R = int(R)
    clist = (C.c_int * count)()
    coff = (C.c_int * (nclusters + 1))()
    load = (C.c_double * nclusters)()
    st = lib.planc_batch_plan(arr, count, int(nclusters), clist, coff, load)
    if st != 0:
        raise PlancError(st, lib.planc_last_error(None).decode())
    lists = [list(clist[coff[q]:coff[q + 1]]) for q in range(nclusters)]
    return lists, list(load)


def batch_solve(Xs, Hs, alg: str = "hals", iters: int = 25, use_graph: bool = True,
                nls: NlsOpts | None = None, stream=None, persistent: bool = True):
    """planc_batch_solve over instances (X_b, [H1, H2, H3]_b): X_b a flat device
    tensor (mode 1 fastest, float32 or bfloat16) whose dims come from the
    factors, H_b three float32 device tensors I_n x R updated in place.
    persistent: one persistent launch for the whole solve (else one launch
    per phase).  Returns one dict per instance (lam, rel_err history) and the
    report."""
    if len(Xs) != len(Hs) or not Xs:
        raise ValueError("need one factor triple per tensor")
    arr = (BatchInstance * len(Xs))()
    keep = []
    for b, (X, H) in enumerate(zip(Xs, Hs)):
        if len(H) != 3:
            raise ValueError("batched solve is 3-way")
        dims = [int(h.shape[0]) for h in H]
        R = int(H[0].shape[1])
        if X.numel() != dims[0] * dims[1] * dims[2] or X.dtype not in (torch.float32, torch.bfloat16):
            raise ValueError(f"X[{b}] does not match its factors")
        for k, h in enumerate(H):
            _check_mat(h, dims[k], R, torch.float32, f"H[{b}][{k}]")
        if not (X.is_cuda and X.is_contiguous()):
            raise ValueError(f"X[{b}] must be a contiguous CUDA tensor")
        lam = (C.c_double * R)()
        hist = (C.c_double * iters)()
        keep.append((lam, hist))
        inst = arr[b]
        for k in range(3):
            inst.dims[k] = dims[k]
            inst.H[k] = _ptr(H[k])
        inst.R = R
        inst.x_dtype = _DT[X.dtype]
        inst.X = _ptr(X)
        inst.lambda_ = C.cast(lam, C.POINTER(C.c_double))
        inst.rel_err_hist = C.cast(hist, C.POINTER(C.c_double))
    o = lib.planc_solve_opts_default()
    o.alg = ALGS[alg]
    o.iters = int(iters)
    o.use_graph = 1 if use_graph else 0
    o.batch_persistent = 1 if persistent else 0
    if nls is not None:
        o.nls = nls
    rep = Report()
    st = lib.planc_batch_solve(arr, len(Xs), C.byref(o),
                               None if stream is None else C.c_void_p(stream.cuda_stream),
                               C.byref(rep))
    if st != 0:
        raise PlancError(st, lib.planc_last_error(None).decode())
    out = [dict(lam=list(lam), rel_err=list(hist), final=arr[b].rel_err)
           for b, (lam, hist) in enumerate(keep)]
    sched = (C.c_int * 4)()
    lib.planc_batch_schedule(sched)
    return out, dict(launches=rep.launches, rel_err=rep.rel_err,
                     schedule=dict(left_rows=sched[0], right_threads=sched[1],
                                   left_rank_blocking=sched[2], right_rank_blocking=sched[3]))
