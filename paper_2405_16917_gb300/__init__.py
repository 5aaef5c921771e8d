"""Python binding of the LRAMM CUDA library (liblramm.so, C ABI in include/lramm.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  PyTorch supplies device memory and streams.  The
binding refuses to run when the library is missing; there is no fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblramm.so")

F32, BF16 = 0, 1
P_F32, P_INT8, P_INT4, P_E4M3, P_MXFP4 = 0, 1, 2, 3, 4
S_ROWCOL, S_TENSOR = 0, 1
SKETCH_F32, SKETCH_TF32, SKETCH_BF16, SKETCH_E4M3 = 0, 1, 2, 3

STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported", 3: "workspace", 4: "cuda error",
          5: "numeric (Cholesky breakdown)", 6: "timeout", 7: "Jacobi not converged"}

_lib = None


class LrammError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: LRAMM status %d (%s)" % (where, code, STATUS.get(code, "?")))


class Desc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("ldb", ctypes.c_int64), ("ldc", ctypes.c_int64),
                ("a_type", ctypes.c_int32), ("b_type", ctypes.c_int32),
                ("r", ctypes.c_int32), ("p", ctypes.c_int32), ("q", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("prec", ctypes.c_int32 * 3),
                ("scale", ctypes.c_int32), ("sketch", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("max_sweeps", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("lead", ctypes.c_int32), ("lead_prec", ctypes.c_int32), ("lead_split", ctypes.c_int32)]


_VP, _I64, _I32, _U64, _U32, _F = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                   ctypes.c_uint32, ctypes.c_float)
_SIGS = {
    "lramm_plan_create": (_I32, [ctypes.POINTER(Desc), ctypes.POINTER(_VP)]),
    "lramm_plan_destroy": (_I32, [_VP]),
    "lramm_workspace_size": (_I32, [_VP, ctypes.POINTER(ctypes.c_size_t)]),
    "lramm_rsvd": (_I32, [_VP, _I32, _VP, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "lramm_matmul": (_I32, [_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "lramm_chain": (_I32, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "lramm_status_read": (_I32, [_VP, _VP]),
    "lramm_info_read": (_I32, [_VP, ctypes.POINTER(ctypes.c_int32), _I32, _VP]),
    "lramm_status_str": (ctypes.c_char_p, [_I32]),
    "lramm_last_cuda_error": (ctypes.c_char_p, []),
    "lramm_philox_words": (_I32, [_U64, _U32, _I64, _VP, _VP]),
    "lramm_gaussian": (_I32, [_U64, _U32, _I64, _I64, _VP, _VP]),
    "lramm_quantize": (_I32, [_VP, _I64, _I64, _I64, _I32, _I32, _VP, _I64, _VP, _VP, _VP]),
    "lramm_qgemm": (_I32, [_VP, _VP, _I64, _I64, _I64, _I64, _I64, _I32, _I32, _VP, _VP, _F, _F,
                           _VP, _I64, _VP, _I64, _I32, _VP]),
    "lramm_rf_forward": (_I32, [_VP, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "lramm_rf_backward": (_I32, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "lramm_qgemm_tc": (_I32, [_I32, _VP, _VP, _I64, _I64, _I64, _I64, _I64, _I32, _VP, _VP, _F, _F, _VP, _I64, _VP,
                              _I64, _VP, ctypes.c_size_t, _VP]),
    "lramm_qgemm_tc_ws_bytes": (ctypes.c_size_t, [_I32, _I64, _I64, _I64]),
    "lramm_tgemm_tc": (_I32, [_I64, _I64, _I64, _F, _VP, _I64, _VP, _I64, _F, _VP, _I64, _VP, ctypes.c_size_t, _VP]),
    "lramm_tgemm_tc_ws_bytes": (ctypes.c_size_t, [_I64, _I64, _I64]),
    "lramm_launch_count": (ctypes.c_uint64, []),
    "lramm_dq_matmul": (_I32, [_I32, _I32, _I64, _I64, _I64, _F, _VP, _I64, _VP, _I64, _F, _VP, _I64, _VP, _I64, _VP,
                               ctypes.c_size_t, _VP]),
    "lramm_dq_ws_bytes": (ctypes.c_size_t, [_I32, _I64, _I64, _I64]),
    "lramm_qsvd": (_I32, [_VP, _I32, _VP, _I32, _I32, _VP, _VP, _VP, _VP, _I64, _VP, _VP, _VP, _I64, _VP,
                          ctypes.c_size_t, _VP]),
    "lramm_qsvd_ws_bytes": (ctypes.c_size_t, [_VP, _I32, _I32, _I32]),
    "lramm_quantize_cols": (_I32, [_VP, _I64, _I64, _I64, _I32, _VP, _I64, _VP, _VP, _VP]),
    "lramm_quantize_mx": (_I32, [_VP, _I64, _I64, _I64, _VP, _I64, _VP, _VP]),
    "lramm_qgemm_mx": (_I32, [_VP, _VP, _VP, _VP, _I64, _I64, _I64, _I64, _I64, _F, _F, _VP, _I64, _VP, _I64, _VP]),
    "lramm_quant_ws_bytes": (ctypes.c_size_t, []),
    "lramm_sketch_product": (_I32, [_VP, _I64, _I64, _I64, _I32, _I32, _VP, _I64, _VP, _I32, _VP, ctypes.c_size_t,
                                    _VP]),
    "lramm_sketch_ws_bytes": (ctypes.c_size_t, [_I64, _I64, _I64]),
    "lramm_quantize_noalloc": (_I32, [_VP, _I64, _I64, _I64, _I32, _I32, _VP, _I64, _VP, _VP]),
    "lramm_noalloc_scratch_bytes": (ctypes.c_size_t, []),
    "lramm_timing_read": (_I32, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)]),
    "lramm_kernel_kind_name": (ctypes.c_char_p, [_I32]),
}

FLAG_TIMING = 1
FLAG_GRAPH = 2
FLAG_SHORT_WAITS = 4       # failure-path tests: bounded waits of ~2^20 SM cycles
FLAG_TEST_DROP_MOVE = 8    # failure-path tests: one cluster-Jacobi CTA skips its first block move
K_COUNT = 17


def load(path=LIB_PATH):
    """Load liblramm.so (built in-tree by paper_2405_16917_gb300._build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("LRAMM CUDA library not found at %s; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st, where):
    if st != 0:
        if st == 4 and _lib is not None:
            where = "%s [%s]" % (where, _lib.lramm_last_cuda_error().decode())
        raise LrammError(st, where)


def _torch():
    import torch
    return torch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError("operands must be float32 or bfloat16, got %s" % t.dtype)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("LRAMM operands must be CUDA tensors")


class Plan:
    """An LRAMM problem: sizes, rank parameters, precisions, seed."""

    def __init__(self, m, n, k, r, p, q, seed=7, prec=(P_INT8, P_INT8, P_INT8), scale=S_ROWCOL,
                 sketch=SKETCH_F32, alpha=1.0, beta=0.0, a_type=F32, b_type=F32, lda=None, ldb=None,
                 ldc=None, max_sweeps=0, timing=False, lead=0, lead_prec=P_INT8, lead_split=0, graph=False,
                 test_flags=0):
        lib = load()
        d = Desc()
        d.m, d.n, d.k = m, n, k
        d.lda = lda if lda is not None else k
        d.ldb = ldb if ldb is not None else n
        d.ldc = ldc if ldc is not None else n
        d.a_type, d.b_type = a_type, b_type
        d.r, d.p, d.q = r, p, q
        d.seed = seed
        d.prec[0], d.prec[1], d.prec[2] = prec
        d.scale, d.sketch = scale, sketch
        d.alpha, d.beta = alpha, beta
        d.max_sweeps = max_sweeps
        d.flags = (FLAG_TIMING if timing else 0) | (FLAG_GRAPH if graph else 0) | test_flags
        d.lead, d.lead_prec, d.lead_split = lead, lead_prec, lead_split
        self.desc = d
        h = ctypes.c_void_p()
        _check(lib.lramm_plan_create(ctypes.byref(d), ctypes.byref(h)), "lramm_plan_create")
        self.handle = h
        sz = ctypes.c_size_t()
        _check(lib.lramm_workspace_size(h, ctypes.byref(sz)), "lramm_workspace_size")
        self.ws_bytes = sz.value

    def timing(self):
        """{kind name: (total ms, launches)} of the last call (plan made with timing=True)."""
        lib = load()
        ms = (ctypes.c_float * K_COUNT)()
        n = (ctypes.c_int32 * K_COUNT)()
        _check(lib.lramm_timing_read(self.handle, ms, n), "lramm_timing_read")
        return {lib.lramm_kernel_kind_name(k).decode(): (ms[k], n[k]) for k in range(K_COUNT) if n[k]}

    def workspace(self, device="cuda"):
        torch = _torch()
        return torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.lramm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def matmul(plan, A, B, C=None, out=None, ws=None, stream=None):
    """D = alpha * E3 + beta * C (Algorithm 3); returns D (m x n FP32)."""
    torch = _torch()
    _need_cuda(A, B, C)
    d = plan.desc
    if out is None:
        out = torch.empty((d.m, d.ldc), dtype=torch.float32, device=A.device)[:, : d.n]
    if ws is None:
        ws = plan.workspace(A.device)
    _check(load().lramm_matmul(plan.handle, _ptr(A), _ptr(B), _ptr(C), _ptr(out), _ptr(ws),
                               ws.numel(), _stream(stream)), "lramm_matmul")
    return out


def rf_forward(plan, X, W, C=None, ws=None, stream=None):
    """Range-finder form: C = alpha * QM((X Q)(Q^T W)) + beta * C; returns C (m x n FP32)."""
    torch = _torch()
    _need_cuda(X, W, C)
    d = plan.desc
    if C is None:
        C = torch.zeros((d.m, d.ldc), dtype=torch.float32, device=X.device)[:, : d.n]
    if ws is None:
        ws = plan.workspace(X.device)
    _check(load().lramm_rf_forward(plan.handle, _ptr(X), _ptr(W), _ptr(C), _ptr(ws), ws.numel(), _stream(stream)),
           "lramm_rf_forward")
    return C


def rf_backward(plan, X, W, G, ws=None, stream=None):
    """Gradients (dX, dW) of <G, C> for the range-finder form (straight-through quantisers)."""
    torch = _torch()
    _need_cuda(X, W, G)
    d = plan.desc
    dX = torch.empty((d.m, d.k), dtype=torch.float32, device=X.device)
    dW = torch.empty((d.k, d.n), dtype=torch.float32, device=X.device)
    if ws is None:
        ws = plan.workspace(X.device)
    _check(load().lramm_rf_backward(plan.handle, _ptr(X), _ptr(W), _ptr(G), _ptr(dX), _ptr(dW), _ptr(ws),
                                    ws.numel(), _stream(stream)), "lramm_rf_backward")
    return dX, dW


def _rf_function():
    """torch.autograd.Function of the range-finder form: forward and the
    hand-written backward both run in the library."""
    torch = _torch()

    class RangeFinderMatmul(torch.autograd.Function):
        @staticmethod
        def forward(ctx, X, W, plan):
            ctx.plan = plan
            ctx.save_for_backward(X, W)
            return rf_forward(plan, X.contiguous(), W.contiguous())

        @staticmethod
        def backward(ctx, G):
            X, W = ctx.saved_tensors
            dX, dW = rf_backward(ctx.plan, X.contiguous(), W.contiguous(), G.contiguous().float())
            return dX.to(X.dtype), dW.to(W.dtype), None

    return RangeFinderMatmul


def rf_matmul(X, W, plan):
    """Differentiable C ~ X W in the range-finder form (autograd through the library's backward)."""
    return _rf_function().apply(X, W, plan)


def rsvd(plan, which, X, ws=None, stream=None):
    """Rank-r randomized SVD of A (which=0) or B (which=1): (U, S, V)."""
    torch = _torch()
    _need_cuda(X)
    d = plan.desc
    rows, cols = (d.m, d.k) if which == 0 else (d.k, d.n)
    U = torch.empty((rows, d.r), dtype=torch.float32, device=X.device)
    S = torch.empty((d.r,), dtype=torch.float32, device=X.device)
    V = torch.empty((cols, d.r), dtype=torch.float32, device=X.device)
    if ws is None:
        ws = plan.workspace(X.device)
    _check(load().lramm_rsvd(plan.handle, which, _ptr(X), _ptr(U), _ptr(S), _ptr(V), _ptr(ws),
                             ws.numel(), _stream(stream)), "lramm_rsvd")
    return U, S, V


def qsvd(plan, which, X, prec_u=P_INT8, prec_v=P_INT8, ldq=None, factors=False, reconstruct=True,
         ws=None, stream=None):
    """Algorithm 4 on A (which=0) or B (which=1): the rank-r RSVD, U~ = U_r Sigma_r
    quantised with prec_u and V_r with prec_v (rows along the rank index).

    Returns a dict: Uc, Us, Vc, Vs (codes and scales as `quantize` lays them
    out, ldq columns), Uf, Vf (the FP32 factors, when factors=True) and Xr
    (the approximation deq(U~') deq(V')^T, when reconstruct=True)."""
    torch = _torch()
    _need_cuda(X)
    d = plan.desc
    rows, cols = (d.m, d.k) if which == 0 else (d.k, d.n)
    ldq = ldq or -(-d.r // 32) * 32
    dev = X.device
    per_row = d.scale == S_ROWCOL
    out = dict(Uc=torch.empty((rows, ldq), dtype=code_dtype(prec_u), device=dev),
               Us=torch.empty((rows if per_row else 1,), dtype=torch.float32, device=dev),
               Vc=torch.empty((cols, ldq), dtype=code_dtype(prec_v), device=dev),
               Vs=torch.empty((cols if per_row else 1,), dtype=torch.float32, device=dev))
    if factors:
        out["Uf"] = torch.empty((rows, d.r), dtype=torch.float32, device=dev)
        out["Vf"] = torch.empty((cols, d.r), dtype=torch.float32, device=dev)
    if reconstruct:
        out["Xr"] = torch.empty((rows, cols), dtype=torch.float32, device=dev)
    lib = load()
    need = lib.lramm_qsvd_ws_bytes(plan.handle, which, prec_u, prec_v)
    if need == 0:
        raise LrammError(1, "lramm_qsvd_ws_bytes")
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    _check(lib.lramm_qsvd(plan.handle, which, _ptr(X), prec_u, prec_v, _ptr(out["Uc"]), _ptr(out["Us"]),
                          _ptr(out["Vc"]), _ptr(out["Vs"]), ldq, _ptr(out.get("Uf")), _ptr(out.get("Vf")),
                          _ptr(out.get("Xr")), cols, _ptr(ws), ws.numel(), _stream(stream)), "lramm_qsvd")
    return out


def chain(plan, Ut, Vt, Wt, Zt, C=None, out=None, ws=None, stream=None):
    """Quantised factor chain of Algorithm 3 on given FP32 factors."""
    torch = _torch()
    _need_cuda(Ut, Vt, Wt, Zt, C)
    d = plan.desc
    for t in (Ut, Vt, Wt, Zt):
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("factors must be contiguous float32")
    if out is None:
        out = torch.empty((d.m, d.ldc), dtype=torch.float32, device=Ut.device)[:, : d.n]
    if ws is None:
        ws = plan.workspace(Ut.device)
    _check(load().lramm_chain(plan.handle, _ptr(Ut), _ptr(Vt), _ptr(Wt), _ptr(Zt), _ptr(C), _ptr(out),
                              _ptr(ws), ws.numel(), _stream(stream)), "lramm_chain")
    return out


def info_read(ws, n=3, stream=None):
    """[status word, Jacobi sweeps A side, Jacobi sweeps B side, ...] of the last call."""
    buf = (ctypes.c_int32 * n)()
    _check(load().lramm_info_read(_ptr(ws), buf, n, _stream(stream)), "lramm_info_read")
    return list(buf)


def dq_matmul(A, B, prec=P_INT8, per_row=True, alpha=1.0, beta=0.0, C=None, out=None, ws=None, stream=None):
    """Direct quantised product alpha QM(A B, prec) + beta C (the DQ8 / DQ4 comparators)."""
    torch = _torch()
    _need_cuda(A, B, C)
    m, k = A.shape
    n = B.shape[1]
    if out is None:
        out = torch.empty((m, n), dtype=torch.float32, device=A.device)
    need = load().lramm_dq_ws_bytes(prec, m, n, k)
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=A.device)
    _check(load().lramm_dq_matmul(prec, S_ROWCOL if per_row else S_TENSOR, m, n, k, alpha, _ptr(A), A.stride(0), _ptr(B),
                                  B.stride(0), beta, _ptr(C), C.stride(0) if C is not None else 0, _ptr(out),
                                  out.stride(0), _ptr(ws), ws.numel(), _stream(stream)), "lramm_dq_matmul")
    return out


def launch_count():
    """Kernels the library has launched in this process so far."""
    return load().lramm_launch_count()


def status_read(ws, stream=None):
    """Synchronise and return (and clear) the workspace's device status code."""
    return load().lramm_status_read(_ptr(ws), _stream(stream))


def philox_words(seed, stream_id, n_blocks, device="cuda"):
    torch = _torch()
    out = torch.empty((n_blocks, 4), dtype=torch.int32, device=device)
    _check(load().lramm_philox_words(seed, stream_id, n_blocks, _ptr(out), _stream()), "lramm_philox_words")
    return out


def gaussian(seed, stream_id, rows, cols, device="cuda"):
    torch = _torch()
    out = torch.empty((rows, cols), dtype=torch.float32, device=device)
    _check(load().lramm_gaussian(seed, stream_id, rows, cols, _ptr(out), _stream()), "lramm_gaussian")
    return out


def sketch_product(X, B, transpose=False, sketch=SKETCH_TF32):
    """X B or X^T B (the range finder's products) through lramm_sketch_product."""
    torch = _torch()
    _need_cuda(X, B)
    rows, cols = X.shape
    l = B.shape[1]
    out = torch.empty((cols if transpose else rows, l), dtype=torch.float32, device=X.device)
    lib = load()
    ws = torch.zeros(lib.lramm_sketch_ws_bytes(rows, cols, l), dtype=torch.uint8, device=X.device)
    _check(lib.lramm_sketch_product(_ptr(X), rows, cols, X.stride(0), _dtype_code(X), int(transpose), _ptr(B), l,
                                    _ptr(out), sketch, _ptr(ws), ws.numel(), _stream()), "lramm_sketch_product")
    st = int(ws[:4].view(torch.int32).item())
    if st != 0:
        raise LrammError(st, "lramm_sketch_product (device)")
    return out


def code_dtype(prec):
    torch = _torch()
    return torch.bfloat16 if prec == P_INT8 else torch.float8_e4m3fn


def quantize(X, prec, per_row=True, ldcodes=None):
    """Codes (rows x ldcodes, bf16 for INT8, e4m3 for INT4/E4M3) and FP32 scales."""
    torch = _torch()
    _need_cuda(X)
    rows, cols = X.shape
    ldc = ldcodes or cols
    codes = torch.empty((rows, ldc), dtype=code_dtype(prec), device=X.device)
    scales = torch.empty((rows if per_row else 1,), dtype=torch.float32, device=X.device)
    lib = load()
    ws = torch.empty(lib.lramm_quant_ws_bytes(), dtype=torch.uint8, device=X.device)
    _check(lib.lramm_quantize(_ptr(X), rows, cols, X.stride(0), prec, int(per_row), _ptr(codes), ldc,
                              _ptr(scales), _ptr(ws), _stream()), "lramm_quantize")
    return codes, scales


def quantize_cols(X, prec, ldcodes=None):
    """Per-column codes of X as the rows of a K-major matrix (cols x ldcodes) and FP32 scales."""
    torch = _torch()
    _need_cuda(X)
    rows, cols = X.shape
    ldc = ldcodes or rows
    codes = torch.empty((cols, ldc), dtype=code_dtype(prec), device=X.device)
    scales = torch.empty((cols,), dtype=torch.float32, device=X.device)
    ws = torch.empty(4 * cols, dtype=torch.uint8, device=X.device)
    _check(load().lramm_quantize_cols(_ptr(X), rows, cols, X.stride(0), prec, _ptr(codes), ldc, _ptr(scales),
                                      _ptr(ws), _stream()), "lramm_quantize_cols")
    return codes, scales


def quantize_noalloc(X, prec, per_row=False, ldcodes=None, codes=None, scales=None):
    """lramm_quantize_noalloc: the quantiser without a caller workspace.

    For callers that cannot allocate device memory: the per-tensor a_max
    accumulator lives in the library's own device array.  Output buffers
    may be passed in (codes, scales) so the call itself allocates nothing.
    """
    torch = _torch()
    _need_cuda(X, codes, scales)
    rows, cols = X.shape
    cdt = code_dtype(prec)
    if codes is not None:
        # caller-supplied codes: the library writes rows x ldc codes through it
        ldc = ldcodes or codes.stride(0)
        if codes.dtype != cdt or codes.dim() != 2 or codes.shape[0] != rows or codes.stride(1) != 1 \
                or codes.stride(0) != ldc or ldc < cols or codes.device != X.device:
            raise ValueError("quantize_noalloc: codes must be a %s tensor of shape (%d, >= %d) with row stride "
                             "ldcodes on %s" % (cdt, rows, cols, X.device))
    else:
        ldc = ldcodes or cols
        codes = torch.empty((rows, ldc), dtype=cdt, device=X.device)
    need = rows if per_row else 1
    if scales is not None:
        if scales.dtype != torch.float32 or scales.numel() < need or not scales.is_contiguous() \
                or scales.device != X.device:
            raise ValueError("quantize_noalloc: scales must be a contiguous float32 tensor of at least %d "
                             "elements on %s" % (need, X.device))
    else:
        scales = torch.empty((need,), dtype=torch.float32, device=X.device)
    _check(load().lramm_quantize_noalloc(_ptr(X), rows, cols, X.stride(0), prec, int(per_row), _ptr(codes),
                                         ldc, _ptr(scales), _stream()), "lramm_quantize_noalloc")
    return codes, scales


def qgemm_tc(Lc, Rc, sL, sR, per_row=True, alpha=1.0, beta=0.0, C=None, ws=None, prec=None):
    """QM product on the tensor cores (codes as lramm_quantize writes them,
    K-major): INT8 codes (bfloat16) by default for bfloat16 codes, E4M3 for
    byte codes unless prec says INT4."""
    torch = _torch()
    _need_cuda(Lc, Rc, C)
    if prec is None:
        prec = P_INT8 if Lc.dtype == torch.bfloat16 else P_E4M3
    M, K = Lc.shape
    N = Rc.shape[0]
    out = torch.empty((M, N), dtype=torch.float32, device=Lc.device)
    need = load().lramm_qgemm_tc_ws_bytes(prec, M, N, K)
    if ws is None or ws.numel() < need:
        ws = torch.zeros(need, dtype=torch.uint8, device=Lc.device)
    _check(load().lramm_qgemm_tc(prec, _ptr(Lc), _ptr(Rc), M, N, K, Lc.stride(0), Rc.stride(0), int(per_row),
                                 _ptr(sL), _ptr(sR), alpha, beta, _ptr(C), C.stride(0) if C is not None else 0,
                                 _ptr(out), N, _ptr(ws), ws.numel(), _stream()), "lramm_qgemm_tc")
    return out


def quantize_mx(X, ldcodes=None):
    """MXFP4 codes (int8, twice the e2m1 value) and block exponents (int8) of the rows of X."""
    torch = _torch()
    _need_cuda(X)
    rows, cols = X.shape
    ldc = ldcodes if ldcodes is not None else -(-cols // 32) * 32
    codes = torch.empty((rows, ldc), dtype=torch.int8, device=X.device)
    exps = torch.empty((rows, ldc // 32), dtype=torch.int8, device=X.device)
    _check(load().lramm_quantize_mx(_ptr(X), rows, cols, X.stride(0), _ptr(codes), ldc, _ptr(exps), _stream()),
           "lramm_quantize_mx")
    return codes, exps


def qgemm_mx(Lc, Le, Rc, Re, alpha=1.0, beta=0.0, C=None):
    """Block-scaled QM on MXFP4 codes (K-major, K a multiple of 32)."""
    torch = _torch()
    _need_cuda(Lc, Rc, C)
    M, K = Lc.shape
    N = Rc.shape[0]
    out = torch.empty((M, N), dtype=torch.float32, device=Lc.device)
    _check(load().lramm_qgemm_mx(_ptr(Lc), _ptr(Le), _ptr(Rc), _ptr(Re), M, N, K, Lc.stride(0), Rc.stride(0), alpha,
                                 beta, _ptr(C), C.stride(0) if C is not None else 0, _ptr(out), N, _stream()),
           "lramm_qgemm_mx")
    return out


def tgemm_tc(A, B, alpha=1.0, beta=0.0, C=None, ws=None):
    """C = alpha A B^T + beta C on the tensor cores (FP32 operands as TF32); returns C."""
    torch = _torch()
    _need_cuda(A, B, C)
    M, K = A.shape
    N = B.shape[0]
    if C is None:
        C = torch.zeros((M, N), dtype=torch.float32, device=A.device)
    need = load().lramm_tgemm_tc_ws_bytes(M, N, K)
    if ws is None or ws.numel() < need:
        ws = torch.zeros(need, dtype=torch.uint8, device=A.device)
    _check(load().lramm_tgemm_tc(M, N, K, alpha, _ptr(A), A.stride(0), _ptr(B), B.stride(0), beta, _ptr(C),
                                 C.stride(0), _ptr(ws), ws.numel(), _stream()), "lramm_tgemm_tc")
    return C


def qgemm(Lc, Rc, prec, sL=None, sR=None, per_row=True, alpha=1.0, beta=0.0, C=None, raw=False):
    """QM product of K-major code matrices; raw=True returns the accumulator."""
    torch = _torch()
    _need_cuda(Lc, Rc, C)
    M, K = Lc.shape
    N = Rc.shape[0]
    if raw:
        out = torch.empty((M, N), dtype=torch.int32 if prec != P_E4M3 else torch.float32, device=Lc.device)
    else:
        out = torch.empty((M, N), dtype=torch.float32, device=Lc.device)
    _check(load().lramm_qgemm(_ptr(Lc), _ptr(Rc), M, N, K, Lc.stride(0), Rc.stride(0), prec, int(per_row),
                              _ptr(sL), _ptr(sR), alpha, beta, _ptr(C), C.stride(0) if C is not None else 0,
                              _ptr(out), N, 1 if raw else 0, _stream()), "lramm_qgemm")
    return out
