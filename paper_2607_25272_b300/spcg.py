"""Python binding of the SPCG C ABI (include/spcg.h): argument marshalling only.

Every step of the solver runs in the CUDA library ``libspcg.so`` that sits
next to this file; this module converts torch CUDA tensors (device memory
and streams) and Python values to the C calls and back.  There is no CPU
fallback: if the library is missing or fails to load, every call raises.

The functions keep the C names (``spcg_create``, ``spcg_sketch``,
``spcg_pcg_stage``, ``spcg_refine``, ``spcg_solve``, ...); ``Solver`` is a
thin owner of one context.
"""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspcg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "spcg.h")

MAX_STAGES = 40
MAX_D = 1024

STATUS = {
    0: "SPCG_OK",
    1: "SPCG_E_INVALID_ARG",
    2: "SPCG_E_OOM",
    3: "SPCG_E_CUDA",
    4: "SPCG_E_BREAKDOWN",
    5: "SPCG_E_NOT_CONVERGED",
    6: "SPCG_E_TIMEOUT",
    7: "SPCG_E_STATE",
}
SPCG_OK = 0
SPCG_E_INVALID_ARG = 1
SPCG_E_OOM = 2
SPCG_E_CUDA = 3
SPCG_E_BREAKDOWN = 4
SPCG_E_NOT_CONVERGED = 5
SPCG_E_TIMEOUT = 6
SPCG_E_STATE = 7

PREC_FP64 = 0
PREC_MIXED = 1
INNER_AUTO = 0
INNER_F32 = 1
INNER_DF = 2
GRAD_AUTO = 0
GRAD_F64 = 1
GRAD_DF = 2
SKETCH_SRHT = 0
SKETCH_COUNT = 1
DTYPE_CODE = {"float64": 0, "float32": 1, "bfloat16": 2}
OP_NAMES = ("float64", "float32", "bfloat16", "pair")   # spcg_info.*_by_op order


class SpcgError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class Schedule(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int32),
        ("m", ctypes.c_int64 * MAX_STAGES),
        ("a", ctypes.c_int32 * MAX_STAGES),
        ("r", ctypes.c_int64),
        ("tol", ctypes.c_double),
        ("max_iters", ctypes.c_int32),
        ("max_restarts", ctypes.c_int32),
        ("sketch", ctypes.c_int32),
    ]

    def as_dict(self):
        return {"m": list(self.m[: self.K]), "a": list(self.a[: self.K]), "r": self.r,
                "tol": self.tol, "max_iters": self.max_iters, "max_restarts": self.max_restarts,
                "sketch": self.sketch}


class Opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("grid_ctas", ctypes.c_int32),
        ("spin_budget", ctypes.c_int64),
        ("inject_stall", ctypes.c_int32),
        ("profile", ctypes.c_int32),
        ("inner_prec", ctypes.c_int32),
        ("grad_prec", ctypes.c_int32),
        ("max_workspace_bytes", ctypes.c_int64),
        ("qr_by_column", ctypes.c_int32),
        ("fwht_tile", ctypes.c_int32),
        ("fwht_first_levels", ctypes.c_int32),
        ("qr_panel_ctas", ctypes.c_int32),
        ("dspace_ctas", ctypes.c_int32),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int32),
        ("stage_iters", ctypes.c_int32 * MAX_STAGES),
        ("refine_iters", ctypes.c_int32),
        ("restarts", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("sqrt_gamma", ctypes.c_double),
        ("norm_R_beta", ctypes.c_double),
        ("ms_sketch", ctypes.c_double),
        ("ms_stages", ctypes.c_double),
        ("ms_refine", ctypes.c_double),
        ("bytes_pass", ctypes.c_uint64),
        ("pass_launches", ctypes.c_int32),
        ("launches", ctypes.c_int32),
        ("pass_ms", ctypes.c_double),
        ("cond_est", ctypes.c_double),
        ("inner_prec", ctypes.c_int32),
        ("grad_prec", ctypes.c_int32),
        ("pass_ms_by_op", ctypes.c_double * 4),
        ("bytes_by_op", ctypes.c_uint64 * 4),
        ("launches_by_op", ctypes.c_int32 * 4),
    ]


class ProblemF32(ctypes.Structure):
    _fields_ = [
        ("X", ctypes.c_void_p),
        ("Y", ctypes.c_void_p),
        ("N", ctypes.c_int64),
        ("d", ctypes.c_int32),
        ("ldx", ctypes.c_int64),
        ("beta", ctypes.c_void_p),
    ]


_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "spcg_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "spcg_default_schedule": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Schedule)]),
    "spcg_tuned_schedule": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Schedule)]),
    "spcg_create": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _P,
                                   ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "spcg_destroy": (None, [_P]),
    "spcg_sketch": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(Schedule)]),
    "spcg_pcg_stage": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P]),
    "spcg_refine": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int32, _P,
                                   ctypes.POINTER(ctypes.c_int32)]),
    "spcg_solve": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(Schedule), _P,
                                  ctypes.POINTER(Info)]),
    "spcg_philox": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int64, _P, _P]),
    "spcg_feistel": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                    ctypes.c_int32, _P, _P]),
    "spcg_signs": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int64, _P, _P]),
    "spcg_export_sketch": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P]),
    "spcg_export_precond": (ctypes.c_int, [_P, _P, _P, _P]),
    "spcg_gram_apply": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int64, _P, _P]),
    "spcg_gram_apply_typed": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                             _P, _P]),
    "spcg_split_f32": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _P, _P,
                                      ctypes.c_int64, _P]),
    "spcg_resid_apply_typed": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int64,
                                              ctypes.c_int64, _P, _P, _P]),
    "spcg_batch_create": (ctypes.c_int, [ctypes.POINTER(ProblemF32), ctypes.c_int32, _P,
                                         ctypes.POINTER(_P)]),
    "spcg_batch_destroy": (None, [_P]),
    "spcg_batch_solve": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_double)]),
    "spcg_batch_set_tiles": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "spcg_batch_phase_cycles": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "spcg_solve_batched": (ctypes.c_int, [ctypes.POINTER(ProblemF32), ctypes.c_int32,
                                          ctypes.c_uint64, ctypes.c_double, _P,
                                          ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "spcg_batch_autotune": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_int32)]),
    "spcg_num_candidates": (ctypes.c_int32, []),
    "spcg_candidate_schedule": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.POINTER(Schedule)]),
    "spcg_features": (ctypes.c_int, [_P, _P, _P]),
    "spcg_solve_learned": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.c_int32, _P,
                                          ctypes.c_double, _P, ctypes.POINTER(Info),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "spcg_solve_candidate": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double,
                                            ctypes.c_int32, _P, ctypes.POINTER(Info)]),
    "spcg_mlp_params": (ctypes.c_int64, [ctypes.c_int32]),
    "spcg_mlp_workspace_floats": (ctypes.c_int64, [ctypes.c_int32, ctypes.c_int64]),
    "spcg_mlp_forward": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, _P]),
    "spcg_mlp_grad": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int64, _P, _P, _P, _P]),
    "spcg_mlp_adam": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_float,
                                     ctypes.c_int32, _P, _P]),
    "spcg_mlp_to_bf16": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P]),
    "spcg_gram_apply_noalloc": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                               _P, _P, _P]),
    "spcg_probe_fma_tflops": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_double), _P]),
    "spcg_host_pool_trim": (ctypes.c_int, []),
    "spcg_solve_enqueue": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32]),
    "spcg_solve_result": (ctypes.c_int, [_P, ctypes.POINTER(Info)]),
    "spcg_solve_host": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                       ctypes.c_uint64, ctypes.POINTER(Schedule),
                                       ctypes.POINTER(Opts), _P, _P, ctypes.POINTER(Info)]),
}


def declared_symbols():
    """Names of the functions include/spcg.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spcg_[a-z_0-9]+)\s*\(", text)))


def lib():
    """Load libspcg.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"SPCG CUDA library not built: {LIB_PATH} is missing "
                               "(run python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st, where):
    if st != SPCG_OK:
        raise SpcgError(st, where)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def status_str(st):
    return lib().spcg_status_str(st).decode()


def spcg_default_schedule(N, d):
    s = Schedule()
    _check(lib().spcg_default_schedule(N, d, ctypes.byref(s)), "spcg_default_schedule")
    return s


def spcg_tuned_schedule(N, d):
    s = Schedule()
    _check(lib().spcg_tuned_schedule(N, d, ctypes.byref(s)), "spcg_tuned_schedule")
    return s


def make_schedule(m, a, r, tol=1e-6, max_iters=100, max_restarts=5, sketch=0):
    s = Schedule()
    s.sketch = int(sketch)
    s.K = len(m)
    for i, (mi, ai) in enumerate(zip(m, a)):
        s.m[i] = int(mi)
        s.a[i] = int(ai)
    s.r = int(r)
    s.tol = float(tol)
    s.max_iters = int(max_iters)
    s.max_restarts = int(max_restarts)
    return s


def spcg_philox(ctr, seed, out=None, stream=None):
    """ctr: CUDA uint32 tensor of shape (n, 4) (or int32 view); returns (n, 4)."""
    import torch
    n = ctr.shape[0]
    if out is None:
        out = torch.empty_like(ctr)
    _check(lib().spcg_philox(_ptr(ctr), seed, n, _ptr(out), _stream_ptr(stream)), "spcg_philox")
    return out


def spcg_feistel(seed, nbits, tag, count, inverse=False, stream=None):
    import torch
    out = torch.empty(max(count, 1), dtype=torch.int64, device="cuda")
    _check(lib().spcg_feistel(seed, nbits, tag, count, int(inverse), _ptr(out), _stream_ptr(stream)),
           "spcg_feistel")
    return out[:count]


def spcg_signs(seed, n, stream=None):
    import torch
    out = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    _check(lib().spcg_signs(seed, n, _ptr(out), _stream_ptr(stream)), "spcg_signs")
    return out[:n]


class Solver:
    """Owner of one spcg_ctx over device-resident (X, Y)."""

    def __init__(self, X, Y, opts=None, stream=None):
        import torch
        if X.dtype != torch.float64 or Y.dtype != torch.float64:
            raise ValueError("X and Y must be float64")
        if X.dim() != 2 or X.stride(1) != 1:
            raise ValueError("X must be a row-major 2-D tensor")
        self.N, self.d = X.shape
        self.X, self.Y = X, Y   # keep the borrowed buffers alive
        self.stream = stream
        ctx = ctypes.c_void_p()
        o = ctypes.byref(opts) if opts is not None else None
        _check(lib().spcg_create(_ptr(X), _ptr(Y), self.N, self.d, X.stride(0),
                                 _stream_ptr(stream), o, ctypes.byref(ctx)), "spcg_create")
        self.ctx = ctx

    def close(self):
        if self.ctx:
            lib().spcg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sketch(self, seed, sched=None):
        _check(lib().spcg_sketch(self.ctx, seed, ctypes.byref(sched) if sched else None),
               "spcg_sketch")

    def pcg_stage(self, i, a_i, beta):
        _check(lib().spcg_pcg_stage(self.ctx, i, a_i, _ptr(beta)), "spcg_pcg_stage")
        return beta

    def refine(self, tol, max_iters, beta, raise_on_error=True):
        it = ctypes.c_int32(0)
        st = lib().spcg_refine(self.ctx, tol, max_iters, _ptr(beta), ctypes.byref(it))
        if raise_on_error:
            _check(st, "spcg_refine")
        return st, it.value

    def solve(self, seed, sched=None, beta=None, raise_on_error=True):
        import torch
        if beta is None:
            beta = torch.empty(self.d, dtype=torch.float64, device=self.X.device)
        info = Info()
        st = lib().spcg_solve(self.ctx, seed, ctypes.byref(sched) if sched else None,
                              _ptr(beta), ctypes.byref(info))
        if raise_on_error:
            _check(st, "spcg_solve")
        return beta, info, st

    def solve_enqueue(self, beta, rounds=6, iters_per_round=20):
        """Enqueue the stages and a fixed Stage II schedule without any host
        read (capture-safe; needs a prior sketch)."""
        _check(lib().spcg_solve_enqueue(self.ctx, _ptr(beta), rounds, iters_per_round),
               "spcg_solve_enqueue")

    def solve_result(self, raise_on_error=True):
        info = Info()
        st = lib().spcg_solve_result(self.ctx, ctypes.byref(info))
        if raise_on_error:
            _check(st, "spcg_solve_result")
        return info, st

    def features(self, beta):
        out = (ctypes.c_float * 4)()
        _check(lib().spcg_features(self.ctx, _ptr(beta), out), "spcg_features")
        return list(out)

    def solve_learned(self, seed, Wb, norm, tol=1e-6, beta=None, raise_on_error=True):
        """Algorithm 1 with the model's schedule (Wb None: the paper's schedule)."""
        import torch
        if beta is None:
            beta = torch.empty(self.d, dtype=torch.float64, device=self.X.device)
        info = Info()
        choice = ctypes.c_int32(-1)
        normc = (ctypes.c_float * 8)(*[float(v) for v in norm]) if norm is not None else None
        st = lib().spcg_solve_learned(self.ctx, seed, _ptr(Wb) if Wb is not None else None, 25,
                                      normc, tol, _ptr(beta), ctypes.byref(info),
                                      ctypes.byref(choice))
        if raise_on_error:
            _check(st, "spcg_solve_learned")
        return beta, info, choice.value, st

    def solve_candidate(self, seed, idx, tol=1e-6, reuse_sketch=False, beta=None,
                        raise_on_error=True):
        import torch
        if beta is None:
            beta = torch.empty(self.d, dtype=torch.float64, device=self.X.device)
        info = Info()
        st = lib().spcg_solve_candidate(self.ctx, seed, idx, tol, int(reuse_sketch), _ptr(beta),
                                        ctypes.byref(info))
        if raise_on_error:
            _check(st, "spcg_solve_candidate")
        return beta, info, st

    def export_sketch(self, row0, nrows):
        import torch
        A = torch.empty((max(nrows, 1), self.d), dtype=torch.float64, device=self.X.device)
        b = torch.empty(max(nrows, 1), dtype=torch.float64, device=self.X.device)
        _check(lib().spcg_export_sketch(self.ctx, row0, nrows, _ptr(A), _ptr(b)),
               "spcg_export_sketch")
        return A[:nrows], b[:nrows]

    def export_precond(self, r=None):
        import torch
        d = self.d
        R = torch.empty((d, d), dtype=torch.float64, device=self.X.device)
        Rinv = torch.empty((d, d), dtype=torch.float64, device=self.X.device)
        Ahat = None
        if r is not None:
            Ahat = torch.empty((r, d), dtype=torch.float64, device=self.X.device)
        _check(lib().spcg_export_precond(self.ctx, _ptr(R), _ptr(Rinv), _ptr(Ahat)),
               "spcg_export_precond")
        return R, Rinv, Ahat

    def gram_apply_typed(self, A, p, w=None):
        """w = A^T (A p) for an FP64, FP32 or BF16 operand A (row-major CUDA tensor)."""
        import torch
        if w is None:
            w = torch.empty(self.d, dtype=torch.float64, device=p.device)
        code = DTYPE_CODE[str(A.dtype).replace("torch.", "")]
        m = A.shape[0]
        lda = A.stride(0) if m > 0 else self.d
        st = lib().spcg_gram_apply_typed(self.ctx, _ptr(A) if m > 0 else None, code, m, lda,
                                         _ptr(p), _ptr(w))
        _check(st, "spcg_gram_apply_typed")
        return w

    def gram_apply_pair(self, AhAl, m, lda, p, w=None):
        """w = A^T (A p) for the double-FP32 pair A = Ah + Al.

        AhAl: CUDA float32 tensor holding Ah (m x lda) and then Al (m x lda)
        contiguously; the first d columns of each row are used."""
        import torch
        if w is None:
            w = torch.empty(self.d, dtype=torch.float64, device=p.device)
        st = lib().spcg_gram_apply_typed(self.ctx, _ptr(AhAl) if m > 0 else None, 3, m, lda,
                                         _ptr(p), _ptr(w))
        _check(st, "spcg_gram_apply_typed")
        return w

    def resid_apply(self, A, b, x, g=None, dtype=None, m=None, lda=None):
        """g = A^T (b - A x); A a row-major CUDA tensor (FP64/FP32/BF16), or
        with dtype=3 the hi-then-lo FP32 pair buffer of gram_apply_pair."""
        import torch
        if g is None:
            g = torch.empty(self.d, dtype=torch.float64, device=x.device)
        if dtype is None:
            dtype = DTYPE_CODE[str(A.dtype).replace("torch.", "")]
            m = A.shape[0]
            lda = A.stride(0) if m > 0 else self.d
        st = lib().spcg_resid_apply_typed(self.ctx, _ptr(A) if m > 0 else None, dtype, m, lda,
                                          _ptr(b) if m > 0 else None, _ptr(x), _ptr(g))
        _check(st, "spcg_resid_apply_typed")
        return g

    def gram_apply(self, A, p, w=None):
        import torch
        if w is None:
            w = torch.empty(self.d, dtype=torch.float64, device=p.device)
        m = A.shape[0]
        lda = A.stride(0) if m > 0 else self.d
        st = lib().spcg_gram_apply(self.ctx, _ptr(A) if m > 0 else None, m, lda, _ptr(p), _ptr(w))
        _check(st, "spcg_gram_apply")
        return w


def spcg_split_f32(X, Xh=None, Xl=None, stream=None):
    """(Xh, Xl) = the double-FP32 split of a row-major CUDA FP64 matrix X
    (its rows 16-byte aligned), as FP32 tensors of X's shape."""
    import torch
    N, d = X.shape
    ldx = X.stride(0) if N > 0 else d
    if Xh is None:
        ld = (d + 1) // 2 * 2
        Xh = torch.zeros((N, ld), dtype=torch.float32, device=X.device)[:, :d]
        Xl = torch.zeros((N, ld), dtype=torch.float32, device=X.device)[:, :d]
    ldxf = Xh.stride(0) if N > 0 else d
    st = lib().spcg_split_f32(_ptr(X) if N > 0 else None, N, d, ldx,
                              _ptr(Xh) if N > 0 else None, _ptr(Xl) if N > 0 else None, ldxf,
                              stream)
    _check(st, "spcg_split_f32")
    return Xh, Xl


def spcg_candidate_schedule(N, d, idx):
    s = Schedule()
    _check(lib().spcg_candidate_schedule(N, d, idx, ctypes.byref(s)), "spcg_candidate_schedule")
    return s


def spcg_mlp_params(n_out):
    return int(lib().spcg_mlp_params(n_out))


def spcg_mlp_forward(Wb, n_out, x, y=None, stream=None):
    """y = MLP(x); Wb: CUDA int16/uint16 tensor of BF16 bits, x: (B, 4) float32."""
    import torch
    B = x.shape[0]
    if y is None:
        y = torch.empty((B, n_out), dtype=torch.float32, device=x.device)
    _check(lib().spcg_mlp_forward(_ptr(Wb), n_out, _ptr(x), B, _ptr(y), _stream_ptr(stream)),
           "spcg_mlp_forward")
    return y


def spcg_mlp_grad(Wb, n_out, x, t, grad, loss, workspace, stream=None):
    _check(lib().spcg_mlp_grad(_ptr(Wb), n_out, _ptr(x), _ptr(t), x.shape[0], _ptr(grad),
                               _ptr(loss), _ptr(workspace), _stream_ptr(stream)), "spcg_mlp_grad")


def spcg_mlp_adam(theta, grad, m, v, lr, step, Wb, stream=None):
    _check(lib().spcg_mlp_adam(_ptr(theta), _ptr(grad), _ptr(m), _ptr(v), theta.numel(),
                               ctypes.c_float(lr), step, _ptr(Wb), _stream_ptr(stream)),
           "spcg_mlp_adam")


def spcg_mlp_to_bf16(theta, Wb, stream=None):
    _check(lib().spcg_mlp_to_bf16(_ptr(theta), theta.numel(), _ptr(Wb), _stream_ptr(stream)),
           "spcg_mlp_to_bf16")


def spcg_gram_apply_noalloc(A, p, w=None, stream=None):
    """w = A^T (A p) through the allocation-free entry point.

    For callers that may not allocate device memory: the library uses its own
    fixed device scratch array (shared by all calls; calls that overlap on the
    GPU race).  The output w may be supplied so that nothing is allocated here
    either.  A: row-major float64 CUDA matrix (stride(1) == 1); p, w: float64
    CUDA vectors of d entries on A's device.  The call runs with A's device
    current, since the C side works on the current device."""
    import torch
    if A.dim() != 2 or A.dtype != torch.float64 or (A.shape[0] > 0 and A.stride(1) != 1):
        raise ValueError("A must be a row-major 2-D float64 tensor")
    m, d = A.shape
    if p.dtype != torch.float64 or p.numel() != d or p.device != A.device:
        raise ValueError("p must be a float64 vector of d entries on A's device")
    if w is None:
        with torch.cuda.device(A.device):
            w = torch.empty(d, dtype=torch.float64, device=A.device)
    if w.dtype != torch.float64 or w.numel() != d or w.device != A.device:
        raise ValueError("w must be a float64 vector of d entries on A's device")
    lda = A.stride(0) if m > 0 else d
    with torch.cuda.device(A.device):
        st = lib().spcg_gram_apply_noalloc(_ptr(A) if m > 0 else None, m, d, lda, _ptr(p),
                                           _ptr(w), _stream_ptr(stream))
    _check(st, "spcg_gram_apply_noalloc")
    return w


def spcg_probe_fma_tflops(dtype="float64", iters=1 << 16, stream=None):
    """Measured FMA rate of the current GPU in TFLOP/s (2 flops per FMA) for
    float64 or float32: the roofline denominator of an FMA-bound kernel."""
    out = ctypes.c_double(0.0)
    code = {"float64": 0, "float32": 1}[dtype]
    _check(lib().spcg_probe_fma_tflops(code, int(iters), ctypes.byref(out), _stream_ptr(stream)),
           "spcg_probe_fma_tflops")
    return out.value


def spcg_solve_host(X_host, Y_host, seed, sched=None, opts=None, stream=None):
    """End to end from host memory through the C ABI (spcg_solve_host): the
    library copies X and Y to the device, solves, and copies beta back.
    X_host: row-major float64 CPU tensor (pinned memory copies fastest),
    Y_host: float64 CPU vector.  Returns (beta as a CPU tensor, info, status)."""
    import torch
    if X_host.is_cuda or Y_host.is_cuda:
        raise ValueError("X_host and Y_host must be CPU tensors")
    if X_host.dtype != torch.float64 or Y_host.dtype != torch.float64 or X_host.stride(1) != 1:
        raise ValueError("X_host must be a row-major float64 matrix and Y_host float64")
    N, d = X_host.shape
    beta = torch.empty(d, dtype=torch.float64)
    info = Info()
    st = lib().spcg_solve_host(ctypes.c_void_p(X_host.data_ptr()), ctypes.c_void_p(Y_host.data_ptr()),
                               N, d, X_host.stride(0), seed,
                               ctypes.byref(sched) if sched else None,
                               ctypes.byref(opts) if opts is not None else None,
                               _stream_ptr(stream), ctypes.c_void_p(beta.data_ptr()),
                               ctypes.byref(info))
    return beta, info, st


def spcg_host_pool_trim():
    """Hand the memory spcg_solve_host keeps between calls back to the devices."""
    _check(lib().spcg_host_pool_trim(), "spcg_host_pool_trim")


def spcg_solve_batched(Xs, Ys, seed, tol=1e-6, stream=None):
    """Solve a batch in one call (create, solve, destroy).  Returns
    (betas, statuses, Stage II iterations, first non-zero status)."""
    import torch
    n = len(Xs)
    betas = [torch.zeros(X.shape[1], dtype=torch.float64, device=X.device) for X in Xs]
    arr = (ProblemF32 * n)()
    for i, (X, Y, b) in enumerate(zip(Xs, Ys, betas)):
        if X.dtype != torch.float32 or Y.dtype != torch.float32 or X.stride(1) != 1:
            raise ValueError("batched problems take row-major float32 X and float32 Y")
        arr[i].X, arr[i].Y = X.data_ptr(), Y.data_ptr()
        arr[i].N, arr[i].d, arr[i].ldx = X.shape[0], X.shape[1], X.stride(0)
        arr[i].beta = b.data_ptr()
    st = (ctypes.c_int32 * n)()
    it = (ctypes.c_int32 * n)()
    rc = lib().spcg_solve_batched(arr, n, seed, tol, _stream_ptr(stream), st, it)
    return betas, list(st), list(it), rc


class Batch:
    """Owner of an spcg_batch over lists of FP32 CUDA tensors X_i (N_i x d_i), Y_i."""

    def __init__(self, Xs, Ys, stream=None):
        import torch
        self.Xs, self.Ys = list(Xs), list(Ys)
        self.n = len(self.Xs)
        self.betas = [torch.zeros(X.shape[1], dtype=torch.float64, device=X.device)
                      for X in self.Xs]
        arr = (ProblemF32 * self.n)()
        for i, (X, Y, b) in enumerate(zip(self.Xs, self.Ys, self.betas)):
            if X.dtype != torch.float32 or Y.dtype != torch.float32 or X.stride(1) != 1:
                raise ValueError("batched problems take row-major float32 X and float32 Y")
            arr[i].X = X.data_ptr()
            arr[i].Y = Y.data_ptr()
            arr[i].N = X.shape[0]
            arr[i].d = X.shape[1]
            arr[i].ldx = X.stride(0)
            arr[i].beta = b.data_ptr()
        h = ctypes.c_void_p()
        _check(lib().spcg_batch_create(arr, self.n, _stream_ptr(stream), ctypes.byref(h)),
               "spcg_batch_create")
        self.h = h

    def solve(self, seed, tol=1e-6, raise_on_error=False):
        st = (ctypes.c_int32 * self.n)()
        it = (ctypes.c_int32 * self.n)()
        ms = ctypes.c_double(0.0)
        rc = lib().spcg_batch_solve(self.h, seed, tol, st, it, ctypes.byref(ms))
        if raise_on_error:
            _check(rc, "spcg_batch_solve")
        return rc, list(st), list(it), ms.value

    def autotune(self, seed, tol=1e-6):
        ch = (ctypes.c_int32 * 4)()
        _check(lib().spcg_batch_autotune(self.h, seed, tol, ch), "spcg_batch_autotune")
        return list(ch)

    def phase_cycles(self):
        """Per problem, the SM clock cycles of each phase of the last solve
        (column maxima, CountSketch row maps, CountSketch sums, stage
        matrices, QR, Stage I, Stage II)."""
        arr = (ctypes.c_int64 * (8 * self.n))()
        _check(lib().spcg_batch_phase_cycles(self.h, arr), "spcg_batch_phase_cycles")
        return [list(arr[8 * i: 8 * i + 7]) for i in range(self.n)]

    def set_tiles(self, chunk_bytes4):
        arr = (ctypes.c_int32 * 4)(*chunk_bytes4)
        _check(lib().spcg_batch_set_tiles(self.h, arr), "spcg_batch_set_tiles")

    def close(self):
        if getattr(self, "h", None):
            lib().spcg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
