"""Thin ctypes binding of the liblyap C ABI (include/liblyap.h).

Argument marshalling only: torch supplies device memory and the current CUDA
stream, every arithmetic step runs in liblyap's kernels.  Matrices cross the
boundary column-major FP64 (a torch tensor ``x`` of logical shape (rows, cols) is
passed through ``_cm(x)``, a column-major copy or view of it).
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build_lib

FP64, FP32, FP16, BF16 = 0, 1, 2, 3
PREC = {"fp64": FP64, "fp32": FP32, "fp16": FP16, "bf16": BF16}
INNER_SIGN, INNER_ADI, INNER_EKSM = 0, 1, 2
INNER = {"sign": INNER_SIGN, "adi": INNER_ADI, "eksm": INNER_EKSM}
SCALE_FROB, SCALE_DET, SCALE_NONE, SCALE_NORM2, SCALE_SPECTRAL = 0, 1, 2, 3, 4
SCALING = {"frob": SCALE_FROB, "det": SCALE_DET, "none": SCALE_NONE, "norm2": SCALE_NORM2,
           "spectral": SCALE_SPECTRAL}

PHASES = ["invert", "newton", "factor", "compress", "resfac", "eig", "solupt", "other", "eig_refine", "spare9",
          "spare10", "spare11"]
NUM_PHASES = 12

OK = 0
ERR_ARG, ERR_NONFINITE, ERR_SINGULAR, ERR_NOCONV, ERR_CAPACITY, ERR_TIMEOUT, ERR_CUDA, ERR_NOMEM = (
    -1, -2, -3, -4, -5, -6, -7, -8)
WARN_STAGNATED, WARN_MAXIT = 1, 2


class LyapOpts(C.Structure):
    _fields_ = [
        ("u_s", C.c_int), ("scaling", C.c_int), ("tau_newton", C.c_double), ("newton_norm_fro", C.c_int),
        ("stop_after", C.c_int), ("delta_rule", C.c_int), ("scale_off", C.c_double), ("rank_tol", C.c_double),
        ("rho", C.c_double), ("kmax", C.c_int), ("imax", C.c_int), ("tau_ir", C.c_double), ("eta_r", C.c_double),
        ("eta_s", C.c_double), ("stag_theta", C.c_double), ("stag_count", C.c_int), ("project_psd", C.c_int),
        ("profile", C.c_int), ("ckpt_every", C.c_int), ("mem_budget", C.c_int64), ("fp64_products", C.c_int),
        ("u", C.c_int), ("u_r", C.c_int), ("u_c", C.c_int), ("inner", C.c_int), ("adi_shifts", C.c_int),
        ("adi_maxit", C.c_int), ("adi_tol", C.c_double), ("eksm_maxit", C.c_int), ("reserved2", C.c_int),
    ]


class LyapInfo(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("rank", C.c_int), ("ir_steps", C.c_int), ("newton_calls", C.c_int),
        ("newton_total", C.c_int), ("newton_max", C.c_int), ("n_inversions", C.c_int), ("stagnated", C.c_int),
        ("converged", C.c_int), ("n_res", C.c_int), ("res_final", C.c_double), ("res_hist", C.c_double * 64),
        ("mu", C.c_double * 64), ("kernel_launches", C.c_int64), ("device_ms", C.c_double),
        ("phase_ms", C.c_double * 12), ("phase_calls", C.c_int64 * 12), ("phase_flops", C.c_double * 12),
    ]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_
             if f not in ("res_hist", "mu", "phase_ms", "phase_calls", "phase_flops")}
        used = [i for i, p in enumerate(PHASES) if not p.startswith("spare")]
        d["phase_ms"] = {PHASES[i]: self.phase_ms[i] for i in used}
        d["phase_calls"] = {PHASES[i]: self.phase_calls[i] for i in used}
        d["phase_flops"] = {PHASES[i]: self.phase_flops[i] for i in used}
        d["res_hist"] = list(self.res_hist[: self.n_res])
        d["mu"] = [m for m in self.mu[: max(self.newton_max, 0)]]
        return d


class LyapError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"liblyap status {status}: {msg}")
        self.status = status


_lib = None

_P = C.c_void_p
_I64 = C.c_int64
_D = C.c_double
SIGNATURES = {
    "lyap_opts_default": (C.c_int, [C.POINTER(LyapOpts)]),
    "lyap_ctx_create": (C.c_int, [C.POINTER(_P), _P]),
    "lyap_ctx_destroy": (C.c_int, [_P]),
    "lyap_ctx_set_stream": (C.c_int, [_P, _P]),
    "lyap_sign_solve": (C.c_int, [_P, _P, _I64, _I64, _P, _I64, _I64, _P, _I64, C.POINTER(LyapOpts), _P, _I64,
                                  _I64, _P, C.POINTER(_I64), C.POINTER(LyapInfo)]),
    "lyap_solve_ir": (C.c_int, [_P, _P, _I64, _I64, _P, _I64, _I64, _P, _I64, C.POINTER(LyapOpts), _P, _I64,
                                _I64, _P, C.POINTER(_I64), C.POINTER(LyapInfo)]),
    "lyap_residual": (C.c_int, [_P, _P, _I64, _I64, _P, _I64, _I64, _P, _I64, _P, _I64, _I64, _P,
                                C.POINTER(_D)]),
    "lyap_invert": (C.c_int, [_P, _P, _I64, _I64, C.c_int, _P, _I64, _P, C.POINTER(_D)]),
    "lyap_invert_noalloc": (C.c_int, [_P, _I64, _I64, C.c_int, _P, _I64, _P, C.POINTER(_D), _P]),
    "lyap_solve_ir_batched": (C.c_int, [_P, C.c_int, C.POINTER(_P), C.POINTER(_I64), C.POINTER(_P), C.POINTER(_I64),
                                        C.POINTER(LyapOpts), C.POINTER(_P), C.POINTER(_I64), C.POINTER(_I64),
                                        C.POINTER(LyapInfo), C.c_int]),
    "lyap_adjoint": (C.c_int, [_P, _P, _I64, _I64, _P, _I64, _I64, _P, _I64, _P, _I64, _I64, _P, _P, _I64, _I64,
                               C.POINTER(LyapOpts), _P, _I64, _P, _I64, _P, _I64, _P, _I64, _I64, C.POINTER(_I64),
                               C.POINTER(LyapInfo)]),
    "lyap_dgemm": (C.c_int, [_P, C.c_char, C.c_char, _I64, _I64, _I64, _D, _P, _I64, _P, _I64, _D, _P, _I64, C.c_int]),
    "lyap_trace_loss": (C.c_int, [_P, _P, _I64, _I64, _I64, _P, _P, _I64, _I64, C.POINTER(_D), _P, _I64]),
    "lyap_kappa_sign": (C.c_int, [_P, _P, _I64, _I64, _P, _I64, _I64, _P, _I64, C.c_int, C.POINTER(_D),
                                  C.POINTER(_D), C.POINTER(C.c_int)]),
    "lyap_rank_trunc": (C.c_int, [_P, _P, _I64, _I64, _I64, _D, C.POINTER(_I64)]),
    "lyap_sym_eig": (C.c_int, [_P, _P, _I64, _I64, _P, _P, _I64, C.c_int]),
    "lyap_last_error": (C.c_char_p, []),
    "lyap_status_string": (C.c_char_p, [C.c_int]),
    "lyap_version": (C.c_char_p, []),
}


def lib_path() -> str:
    return build_lib.LIB_PATH


def load(build_if_missing: bool = True):
    """Load liblyap.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not build_lib.up_to_date():
        build_lib.build()
    if not os.path.exists(build_lib.LIB_PATH):
        raise RuntimeError("liblyap.so is not built; run __graft_entry__.build()")
    lib = C.CDLL(build_lib.LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int, allow_warn: bool = True) -> int:
    if status < 0 or (status > 0 and not allow_warn):
        lib = load()
        raise LyapError(status, f"{lib.lyap_status_string(status).decode()}: {lib.lyap_last_error().decode()}")
    return status


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _cm(x: torch.Tensor) -> torch.Tensor:
    """Column-major FP64 CUDA view/copy of a 2-D tensor (ld = rows)."""
    if x.dtype != torch.float64 or not x.is_cuda:
        raise TypeError("liblyap takes FP64 CUDA tensors")
    if x.dim() == 1:
        x = x[:, None]
    r, c = x.shape
    if x.stride() == (1, r) or (c == 1 and x.stride(0) == 1):
        return x
    return x.t().contiguous().t()


def cm_empty(rows: int, cols: int, device) -> torch.Tensor:
    return torch.empty((cols, rows), dtype=torch.float64, device=device).t()


def cm_copy(x: torch.Tensor) -> torch.Tensor:
    y = cm_empty(x.shape[0], x.shape[1], x.device)
    y.copy_(x)
    return y


class Context:
    """A liblyap context bound to the current torch stream (one per thread)."""

    def __init__(self):
        lib = load()
        h = _P()
        _check(lib.lyap_ctx_create(C.byref(h), _P(_stream())))
        self.h = h
        self.lib = lib

    def close(self):
        if self.h:
            self.lib.lyap_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _bind(self):
        self.lib.lyap_ctx_set_stream(self.h, _P(_stream()))


_ctx: Context | None = None


def context() -> Context:
    global _ctx
    if _ctx is None:
        _ctx = Context()
    _ctx._bind()
    return _ctx


def make_opts(u_s="fp16", **kw) -> LyapOpts:
    o = LyapOpts()
    load().lyap_opts_default(C.byref(o))
    o.u_s = PREC[u_s] if isinstance(u_s, str) else int(u_s)
    for k, v in kw.items():
        if k == "scaling" and isinstance(v, str):
            v = SCALING[v]
        if k == "inner" and isinstance(v, str):
            v = INNER[v]
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _solve(fn_name: str, A, L, S=None, z_cap=None, opts: LyapOpts | None = None, raise_on_warn=False):
    ctx = context()
    A = _cm(A)
    L = _cm(L)
    n, m = L.shape
    if A.shape != (n, n):
        raise ValueError("A must be n x n")
    Sd = _cm(S) if S is not None else None
    cap = int(z_cap) if z_cap is not None else n
    Z = cm_empty(n, cap, A.device)
    D = torch.empty(cap, dtype=torch.float64, device=A.device) if S is not None else None
    rank = _I64(0)
    info = LyapInfo()
    o = opts if opts is not None else make_opts()
    st = getattr(ctx.lib, fn_name)(ctx.h, _P(A.data_ptr()), n, n, _P(L.data_ptr()), n, m,
                                   _P(Sd.data_ptr()) if Sd is not None else None, m, C.byref(o),
                                   _P(Z.data_ptr()), n, cap, _P(D.data_ptr()) if D is not None else None,
                                   C.byref(rank), C.byref(info))
    _check(st, allow_warn=not raise_on_warn)
    r = rank.value
    return Z[:, :r], (D[:r] if D is not None else None), info


def solve_ir(A, L, S=None, z_cap=None, opts=None, **kw):
    """Mixed-precision IR (Algorithms IR-Chol / IR-LDLT): returns (Z, D, info)."""
    return _solve("lyap_solve_ir", A, L, S, z_cap, opts if opts is not None else make_opts(**kw))


def solve_ir_batched(As, Ls, opts=None, workers=8, z_caps=None, raise_on_error=True, **kw):
    """Independent Cholesky-type IR solves in one call (lyap_solve_ir_batched).
    Returns (list of Z_e, list of LyapInfo, status)."""
    ctx = context()
    nb = len(As)
    As = [_cm(a) for a in As]
    Ls = [_cm(l) for l in Ls]
    ns = [a.shape[0] for a in As]
    caps = [int(c) for c in z_caps] if z_caps is not None else list(ns)
    Zs = [cm_empty(n, c, a.device) for n, c, a in zip(ns, caps, As)]
    PA = (_P * nb)(*[a.data_ptr() for a in As])
    PL = (_P * nb)(*[l.data_ptr() for l in Ls])
    PZ = (_P * nb)(*[z.data_ptr() for z in Zs])
    N = (_I64 * nb)(*ns)
    M = (_I64 * nb)(*[l.shape[1] for l in Ls])
    CAP = (_I64 * nb)(*caps)
    R = (_I64 * nb)()
    infos = (LyapInfo * nb)()
    o = opts if opts is not None else make_opts(**kw)
    st = ctx.lib.lyap_solve_ir_batched(ctx.h, nb, PA, N, PL, M, C.byref(o), PZ, CAP, R, infos, int(workers))
    if raise_on_error:
        _check(st)
    return [z[:, : R[e]] for e, z in enumerate(Zs)], list(infos), st


def sign_solve(A, L, S=None, z_cap=None, opts=None, **kw):
    """One sign-function Newton solve at u_s (Algorithms Newton-Chol / Newton-LDLT)."""
    return _solve("lyap_sign_solve", A, L, S, z_cap, opts if opts is not None else make_opts(**kw))


def adjoint(A, L, Z, Cm, S=None, D=None, opts=None, want=("dA", "dL", "dS"), factor=False, **kw):
    """Gradients of l = trace(C X C^T), X = Z diag(D) Z^T solving A X + X A^T + L S L^T = 0,
    through lyap_adjoint (adjoint equation A^T Y + Y A + C^T C = 0 solved by the refinement,
    replaying the context's stored inverse sequence transposed when it belongs to this A).
    Returns dict(dA, dL, dS, Zy, info) (entries not requested are None)."""
    ctx = context()
    A, L, Z, Cm = _cm(A), _cm(L), _cm(Z), _cm(Cm)
    n, m = L.shape
    r = Z.shape[1]
    q = Cm.shape[0]
    Sd = _cm(S) if S is not None else None
    Dd = D.contiguous() if D is not None else None
    dev = A.device
    dA = cm_empty(n, n, dev) if "dA" in want else None
    dL = cm_empty(n, m, dev) if "dL" in want else None
    dS = cm_empty(m, m, dev) if ("dS" in want and S is not None) else None
    cap = n + 8
    Zy = cm_empty(n, cap, dev) if factor else None
    ry = _I64(0)
    info = LyapInfo()
    o = opts if opts is not None else make_opts(**kw)
    ptr = lambda t: _P(t.data_ptr()) if t is not None else None  # noqa: E731
    st = ctx.lib.lyap_adjoint(ctx.h, ptr(A), n, n, ptr(L), n, m, ptr(Sd), m, ptr(Z), n, r, ptr(Dd), ptr(Cm), q, q,
                              C.byref(o), ptr(dA), n, ptr(dL), n, ptr(dS), m, ptr(Zy), n, cap, C.byref(ry),
                              C.byref(info))
    _check(st)
    return {"dA": dA, "dL": dL, "dS": dS, "Zy": Zy[:, : ry.value] if Zy is not None else None, "info": info}


def kappa_sign(A, L, S=None, power_steps=8):
    """kappa_sign(B) in the Frobenius norm for B = [[A, L S L^T], [0, -A^T]] (lyap_kappa_sign):
    returns {"kappa", "lnorm", "newton_steps"}."""
    ctx = context()
    A, L = _cm(A), _cm(L)
    n, m = L.shape
    Sc = _cm(S) if S is not None else None
    kap, ln, ks = _D(0.0), _D(0.0), C.c_int(0)
    _check(ctx.lib.lyap_kappa_sign(ctx.h, _P(A.data_ptr()), n, n, _P(L.data_ptr()), n, m,
                                   _P(Sc.data_ptr()) if Sc is not None else None, m, int(power_steps),
                                   C.byref(kap), C.byref(ln), C.byref(ks)), allow_warn=False)
    return {"kappa": kap.value, "lnorm": ln.value, "newton_steps": ks.value}


def trace_loss_value(Z, Cm, D=None, want_grad=False):
    """l = trace(C X C^T) for X = Z diag(D) Z^T, and dl/dC = 2 C X when want_grad
    (lyap_trace_loss).  Returns (loss, dC or None)."""
    ctx = context()
    Z, Cm = _cm(Z), _cm(Cm)
    n, r = Z.shape
    q = Cm.shape[0]
    Dd = D.contiguous() if D is not None else None
    dC = cm_empty(q, n, Z.device) if want_grad else None
    out = _D(0.0)
    _check(ctx.lib.lyap_trace_loss(ctx.h, _P(Z.data_ptr()), n, n, r, _P(Dd.data_ptr()) if Dd is not None else None,
                                   _P(Cm.data_ptr()), q, q, C.byref(out), _P(dC.data_ptr()) if dC is not None else None,
                                   q), allow_warn=False)
    return out.value, dC


class LyapTraceLoss(torch.autograd.Function):
    """l = trace(C X C^T) for the solution X = Z diag(D) Z^T of A X + X A^T + L S L^T = 0
    (lyap_solve_ir forward; S = None: W = L L^T; the loss itself by lyap_trace_loss).
    backward: dA, dL, dS from lyap_adjoint (which replays the forward inverse sequence
    transposed) and dC = 2 C X from lyap_trace_loss."""

    @staticmethod
    def forward(fctx, A, L, Cm, S=None, opts=None):
        Z, D, info = solve_ir(A, L, S, opts=opts)
        loss, _ = trace_loss_value(Z, Cm, D)
        fctx.opts = opts
        fctx.info = info
        fctx.save_for_backward(A, L, Cm, S if S is not None else torch.empty(0, device=A.device), Z,
                               D if D is not None else torch.empty(0, device=A.device))
        return torch.tensor(loss, dtype=torch.float64, device=A.device)

    @staticmethod
    def backward(fctx, g):
        A, L, Cm, S, Z, D = fctx.saved_tensors
        S = S if S.numel() else None
        D = D if D.numel() else None
        out = adjoint(A, L, Z, Cm, S=S, D=D, opts=fctx.opts)
        _, dC = trace_loss_value(Z, Cm, D, want_grad=True)
        dS = g * out["dS"] if S is not None else None
        return g * out["dA"], g * out["dL"], g * dC, dS, None


def trace_loss(A, L, Cm, S=None, opts=None, **kw):
    """Differentiable l = trace(C X C^T) (LyapTraceLoss)."""
    return LyapTraceLoss.apply(A, L, Cm, S, opts if opts is not None else make_opts(**kw))


def residual(A, L, Z, S=None, D=None) -> float:
    """Relative residual of Eq. (4.1) computed in FP64 on the GPU from the factors."""
    ctx = context()
    A, L, Z = _cm(A), _cm(L), _cm(Z)
    n, m = L.shape
    r = Z.shape[1]
    Sd = _cm(S) if S is not None else None
    Dd = D.contiguous() if D is not None else None
    out = _D(0.0)
    _check(ctx.lib.lyap_residual(ctx.h, _P(A.data_ptr()), n, n, _P(L.data_ptr()), n, m,
                                 _P(Sd.data_ptr()) if Sd is not None else None, m, _P(Z.data_ptr()), n, r,
                                 _P(Dd.data_ptr()) if Dd is not None else None, C.byref(out)))
    return out.value


DGEMM = {"auto": 0, "simt": 1, "tensor": 2}


def dgemm(A, B, ta="N", tb="N", alpha=1.0, beta=0.0, C=None, method="auto"):
    """C = alpha op(A) op(B) + beta C in FP64 (lyap_dgemm): method "simt", "tensor" (FP64
    emulated on the FP16 tensor cores) or "auto"."""
    ctx = context()
    A, B = _cm(A), _cm(B)
    m = A.shape[1] if ta == "T" else A.shape[0]
    k = A.shape[0] if ta == "T" else A.shape[1]
    n = B.shape[0] if tb == "T" else B.shape[1]
    if C is None:
        C = cm_empty(m, n, A.device)
    else:
        C = _cm(C)
    _check(ctx.lib.lyap_dgemm(ctx.h, ta.encode(), tb.encode(), m, n, k, float(alpha), _P(A.data_ptr()), A.shape[0],
                              _P(B.data_ptr()), B.shape[0], float(beta), _P(C.data_ptr()), C.shape[0],
                              DGEMM[method] if isinstance(method, str) else int(method)), allow_warn=False)
    return C


def invert(A, prec="fp64"):
    """Blocked Gauss-Jordan inverse with partial pivoting: returns (Ainv, ipiv, logabsdet)."""
    ctx = context()
    A = _cm(A)
    n = A.shape[0]
    Ai = cm_empty(n, n, A.device)
    ipiv = torch.empty(n, dtype=torch.int32, device=A.device)
    ld = _D(0.0)
    _check(ctx.lib.lyap_invert(ctx.h, _P(A.data_ptr()), n, n, PREC[prec] if isinstance(prec, str) else prec,
                               _P(Ai.data_ptr()), n, _P(ipiv.data_ptr()), C.byref(ld)), allow_warn=False)
    return Ai, ipiv, ld.value


NOALLOC_MAX_N = 512  # LYAP_NOALLOC_MAX_N


def invert_noalloc(A, prec="fp64", out=None, ipiv=None):
    """lyap_invert through the entry point that allocates no device memory (FP64/FP32,
    n <= NOALLOC_MAX_N).  `out` / `ipiv` may be preallocated (column-major n x n FP64,
    int32[n]); returns (Ainv, ipiv, logabsdet)."""
    lib = load()
    A = _cm(A)
    n = A.shape[0]
    Ai = cm_empty(n, n, A.device) if out is None else out
    if ipiv is None:
        ipiv = torch.empty(n, dtype=torch.int32, device=A.device)
    ld = _D(0.0)
    _check(lib.lyap_invert_noalloc(_P(A.data_ptr()), n, n, PREC[prec] if isinstance(prec, str) else prec,
                                   _P(Ai.data_ptr()), n, _P(ipiv.data_ptr()), C.byref(ld), _P(_stream())),
           allow_warn=False)
    return Ai, ipiv, ld.value


def rank_trunc(Z, tol: float):
    """RankTruncChol: QR with column pivoting of Z^T; returns Pi [T C]^T (n x r)."""
    ctx = context()
    Zc = cm_copy(Z)
    n, c = Zc.shape
    r = _I64(0)
    _check(ctx.lib.lyap_rank_trunc(ctx.h, _P(Zc.data_ptr()), n, c, n, float(tol), C.byref(r)), allow_warn=False)
    return Zc[:, : r.value]


def sym_eig(H, refine: bool = True):
    """Symmetric eigendecomposition H = Q diag(w) Q^T (ascending w)."""
    ctx = context()
    Hc = cm_copy(H)
    q = Hc.shape[0]
    w = torch.empty(q, dtype=torch.float64, device=H.device)
    Q = cm_empty(q, q, H.device)
    _check(ctx.lib.lyap_sym_eig(ctx.h, _P(Hc.data_ptr()), q, q, _P(w.data_ptr()), _P(Q.data_ptr()), q,
                                1 if refine else 0), allow_warn=False)
    return w, Q


def exported_symbols() -> list[str]:
    return list(SIGNATURES)


# The C entry points under their own names (same arguments as the wrappers above).
lyap_solve_ir = solve_ir
lyap_sign_solve = sign_solve
lyap_residual = residual
lyap_invert = invert
lyap_invert_noalloc = invert_noalloc
lyap_adjoint = adjoint
lyap_solve_ir_batched = solve_ir_batched
lyap_rank_trunc = rank_trunc
lyap_trace_loss = trace_loss_value
lyap_dgemm = dgemm
lyap_kappa_sign = kappa_sign
lyap_sym_eig = sym_eig
