"""Thin Python binding of libspm (C ABI in include/spm.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Device buffers are torch CUDA tensors; the current torch stream is passed to
each call.  There is no CPU fallback: if libspm.so is missing or no sm_103
device is present, calls raise.
"""
import ctypes
import os

import torch

from . import _build

F32, F64 = 0, 1
SPARSE_SIGN, IDENTITY, DENSE_SIGN, SRHT = 0, 1, 2, 3
EUNSUPPORTED = 7  # SPM_EUNSUPPORTED
PREC_FP64, PREC_MIXED, PREC_FP32 = 0, 1, 2
EINVAL = 1  # SPM_EINVAL
STAGES = ("sketch", "apply", "power", "orth", "project", "small", "finish", "other")

_STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
           4: "Cholesky breakdown", 5: "non-finite value", 6: "device wait timed out",
           7: "unsupported"}


class SpmError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {_STATUS.get(code, code)} (status {code})")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("reorth", ctypes.c_int32),
                ("final_passes", ctypes.c_int32), ("small_fp64", ctypes.c_int32),
                ("power_passes", ctypes.c_int32), ("eig_refine", ctypes.c_int32),
                ("omega", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("want_timing", ctypes.c_int32), ("eig_sweeps", ctypes.c_int32),
                ("device_status", ctypes.c_int32), ("cholqr_passes", ctypes.c_int32),
                ("resid_est", ctypes.c_double), ("fro_a", ctypes.c_double),
                ("stage_ms", ctypes.c_float * 8), ("auto_q", ctypes.c_int32),
                ("auto_fp32", ctypes.c_int32), ("a_split", ctypes.c_int32)]

    def as_dict(self):
        return {"device_status": self.device_status, "cholqr_passes": self.cholqr_passes,
                "eig_sweeps": self.eig_sweeps,
                "resid_est": self.resid_est, "fro_a": self.fro_a,
                "stage_ms": {k: float(v) for k, v in zip(STAGES, self.stage_ms)},
                "auto_q": self.auto_q, "auto_fp32": self.auto_fp32, "a_split": self.a_split}


_LIB = None
I64, I32, U64, VP = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p

_SIGS = {
    "spm_version": ([], I32),
    "spm_status_string": ([I32], ctypes.c_char_p),
    "spm_device_ok": ([], I32),
    "spm_launch_count": ([], U64),
    "spm_sketch_create": ([ctypes.POINTER(VP), I64, I64, I32, U64, I32, VP], I32),
    "spm_sketch_destroy": ([VP], I32),
    "spm_sketch_shape": ([VP, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I32),
                          ctypes.POINTER(I32)], I32),
    "spm_sketch_tables": ([VP, VP, VP, VP, VP, VP, VP], I32),
    "spm_gaussian": ([VP, I32, I64, I64, I64, U64, VP], I32),
    "spm_sketch_apply": ([VP, VP, I32, I64, I64, VP, I64, VP], I32),
    "spm_sketch_apply_t": ([VP, VP, I32, I64, I64, VP, I64, VP], I32),
    "spm_range_finder": ([VP, VP, I32, I64, I64, I64, I32, U64, ctypes.POINTER(Opts), VP, I64,
                          ctypes.POINTER(Info), VP], I32),
    "spm_rsvd": ([VP, VP, I32, I64, I64, I64, I32, U64, I64, ctypes.POINTER(Opts), VP, I64, VP,
                  VP, I64, ctypes.POINTER(Info), VP], I32),
    "spm_trim_memory": ([], I32),
    "spm_sketch_apply_csr": ([VP, VP, I32, VP, I64, VP], I32),
    "spm_rsvd_csr": ([VP, VP, I32, I64, I32, U64, I64, ctypes.POINTER(Opts), VP, I64, VP, VP, I64,
                      ctypes.POINTER(Info), VP], I32),
    "spm_rsvd_host": ([VP, VP, I32, I64, I64, I64, I32, U64, I64, ctypes.POINTER(Opts), VP, I64,
                       VP, VP, I64, ctypes.POINTER(Info), VP], I32),
    "spm_lowrank": ([VP, VP, VP, I32, I64, I64, I64, I32, U64, ctypes.POINTER(Opts), VP, I64, VP,
                     I64, ctypes.POINTER(Info), VP], I32),
    "spm_gemm_bf16": ([I64, I64, I64, I32, ctypes.POINTER(VP), I64, I32, ctypes.POINTER(VP), I64,
                       I32, VP, I64, I32, VP], I32),
    "spm_nystrom": ([VP, VP, I32, I64, I64, I64, I32, U64, ctypes.POINTER(Opts), VP, I64, VP, I64,
                     ctypes.POINTER(Info), VP], I32),
}


def lib_path():
    return _build.LIB


def lib():
    """Load libspm.so (built in-tree by ``__graft_entry__.build()``)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libspm.so not built at {path}; run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = L
    return _LIB


def _check(rc, where):
    if rc != 0:
        raise SpmError(rc, where)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dt(t):
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError("only float32 / float64 matrices")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _require_cuda(*ts):
    for t in ts:
        if not t.is_cuda:
            raise ValueError("device (CUDA) tensors required")
        if t.dim() == 2 and t.stride(1) != 1:
            raise ValueError("row-major (last-dim contiguous) matrices required")


class Sketch:
    """Device tables of one sketch S in R^{n x r1}: sparse sign (default), identity,
    dense sign or SRHT (``kind``; s is not used by the two dense kinds)."""

    def __init__(self, n, r1, s=8, seed=42, kind=SPARSE_SIGN):
        h = ctypes.c_void_p()
        _check(lib().spm_sketch_create(ctypes.byref(h), int(n), int(r1), int(s), int(seed),
                                       int(kind), _stream()), "spm_sketch_create")
        self.handle = h
        self.n, self.r1, self.s, self.seed, self.kind = int(n), int(r1), int(s), int(seed), kind

    def close(self):
        if self.handle:
            lib().spm_sketch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tables(self):
        """Draw-order (cols, signs) and column buckets (ptr, rows, signs) as device tensors."""
        dev = torch.device("cuda")
        nnz = self.n * (self.s if self.kind == SPARSE_SIGN else 1)
        cols = torch.empty(nnz, dtype=torch.int32, device=dev)
        signs = torch.empty(nnz, dtype=torch.int8, device=dev)
        bptr = torch.empty(self.r1 + 1, dtype=torch.int64, device=dev)
        brows = torch.empty(nnz, dtype=torch.int32, device=dev)
        bsg = torch.empty(nnz, dtype=torch.int8, device=dev)
        _check(lib().spm_sketch_tables(self.handle, _ptr(cols), _ptr(signs), _ptr(bptr),
                                       _ptr(brows), _ptr(bsg), _stream()), "spm_sketch_tables")
        return cols, signs, bptr, brows, bsg


def gaussian(rows, cols, seed, dtype=torch.float64):
    out = torch.empty(rows, cols, dtype=dtype, device="cuda")
    _check(lib().spm_gaussian(_ptr(out), _dt(out), rows, cols, cols, int(seed), _stream()),
           "spm_gaussian")
    return out


def sketch_apply(S, A):
    _require_cuda(A)
    out = torch.empty(A.shape[0], S.r1, dtype=A.dtype, device=A.device)
    _check(lib().spm_sketch_apply(S.handle, _ptr(A), _dt(A), A.shape[0], A.stride(0), _ptr(out),
                                  out.stride(0), _stream()), "spm_sketch_apply")
    return out


def sketch_apply_t(S, X):
    _require_cuda(X)
    out = torch.empty(S.r1, X.shape[1], dtype=X.dtype, device=X.device)
    _check(lib().spm_sketch_apply_t(S.handle, _ptr(X), _dt(X), X.shape[1], X.stride(0), _ptr(out),
                                    out.stride(0), _stream()), "spm_sketch_apply_t")
    return out


def make_opts(precision=PREC_FP64, reorth=True, final_passes=3, small_fp64=False, omega=None,
              power_passes=3, eig_refine=0):
    o = Opts(int(precision), int(reorth), int(final_passes), int(bool(small_fp64)),
             int(power_passes), int(eig_refine), None)
    if omega is not None:
        o.omega = omega.data_ptr()
    return o


def _info(timing):
    """timing: False, True (stage times and |A|_F), or 2 (stage times only: the
    sketch pass then skips the |A|_F sum, as calls without info do)."""
    inf = Info()
    inf.want_timing = 2 if timing == 2 else (1 if timing else 0)
    return inf


def range_finder(S, A, r2, q, omega_seed=43, precision=PREC_FP64, timing=False, **kw):
    _require_cuda(A)
    o = make_opts(precision, **kw)
    Q = torch.empty(A.shape[0], r2, dtype=A.dtype, device=A.device)
    inf = _info(timing)
    _check(lib().spm_range_finder(S.handle, _ptr(A), _dt(A), A.shape[0], A.stride(0), r2, q,
                                  int(omega_seed), ctypes.byref(o), _ptr(Q), Q.stride(0),
                                  ctypes.byref(inf), _stream()), "spm_range_finder")
    return Q, inf.as_dict()


def rsvd(S, A, r2, q, k, omega_seed=43, precision=PREC_FP64, timing=False, out=None, info=True,
         **kw):
    """Randomized SVD on the sketch-powered range finder: (U, sigma, Vt, info)."""
    _require_cuda(A)
    o = make_opts(precision, **kw)
    m, n = A.shape
    if out is None:
        U = torch.empty(m, k, dtype=A.dtype, device=A.device)
        sig = torch.empty(k, dtype=A.dtype, device=A.device)
        Vt = torch.empty(k, n, dtype=A.dtype, device=A.device)
    else:
        U, sig, Vt = out
    inf = _info(timing) if info else None
    rc = lib().spm_rsvd(S.handle, _ptr(A), _dt(A), m, A.stride(0), r2, q, int(omega_seed), k,
                        ctypes.byref(o), _ptr(U), U.stride(0), _ptr(sig), _ptr(Vt), Vt.stride(0),
                        ctypes.byref(inf) if inf is not None else None, _stream())
    _check(rc, "spm_rsvd")
    return U, sig, Vt, (inf.as_dict() if inf is not None else None)


class CsrStruct(ctypes.Structure):
    _fields_ = [("rowptr", VP), ("colind", VP), ("vals", VP), ("m", I64), ("n", I64), ("nnz", I64),
                ("U", VP), ("ldu", I64), ("sig", VP), ("V", VP), ("ldv", I64), ("p", I64)]


class CsrMatrix:
    """A = A_csr + U diag(sig) V^T on the device (spm_csr); the tensors stay
    referenced while the object lives.  rowptr int64 (m + 1), colind int32
    (nnz), vals / U / sig / V float32 or float64 on one CUDA device."""

    def __init__(self, rowptr, colind, vals, n, U=None, sig=None, V=None):
        _require_cuda(rowptr, colind, vals)
        if rowptr.dtype != torch.int64 or colind.dtype != torch.int32:
            raise TypeError("rowptr int64, colind int32")
        self.rowptr, self.colind, self.vals = rowptr, colind, vals
        self.m, self.n, self.nnz = rowptr.numel() - 1, int(n), colind.numel()
        self.U, self.sig, self.V = U, sig, V
        self.dtype = vals.dtype
        s = CsrStruct(_ptr(rowptr), _ptr(colind), _ptr(vals), self.m, self.n, self.nnz, None, 0,
                      None, None, 0, 0)
        if U is not None:
            _require_cuda(U, sig, V)
            s.U, s.ldu, s.sig, s.V, s.ldv, s.p = (_ptr(U), U.stride(0), _ptr(sig), _ptr(V),
                                                   V.stride(0), U.shape[1])
        self.struct = s


def sketch_apply_csr(S, A, out=None):
    """A~ = A S for a CsrMatrix A (m x r1, A's dtype)."""
    if out is None:
        out = torch.empty(A.m, S.r1, dtype=A.dtype, device=A.vals.device)
    dt = F64 if A.dtype == torch.float64 else F32
    _check(lib().spm_sketch_apply_csr(S.handle, ctypes.byref(A.struct), dt, _ptr(out), out.stride(0),
                                      _stream()), "spm_sketch_apply_csr")
    return out


def rsvd_csr(S, A, r2, q, k, omega_seed=43, precision=PREC_FP64, timing=False, **kw):
    """RandSVD of a CsrMatrix A: (U, sigma, Vt, info)."""
    o = make_opts(precision, **kw)
    dev = A.vals.device
    U = torch.empty(A.m, k, dtype=A.dtype, device=dev)
    sig = torch.empty(k, dtype=A.dtype, device=dev)
    Vt = torch.empty(k, A.n, dtype=A.dtype, device=dev)
    inf = _info(timing)
    dt = F64 if A.dtype == torch.float64 else F32
    _check(lib().spm_rsvd_csr(S.handle, ctypes.byref(A.struct), dt, r2, q, int(omega_seed), k,
                              ctypes.byref(o), _ptr(U), U.stride(0), _ptr(sig), _ptr(Vt),
                              Vt.stride(0), ctypes.byref(inf), _stream()), "spm_rsvd_csr")
    return U, sig, Vt, inf.as_dict()


def trim_memory():
    """Hand the library pool's unused device memory back to the device."""
    _check(lib().spm_trim_memory(), "spm_trim_memory")


def rsvd_host(S, A, r2, q, k, omega_seed=43, precision=PREC_FP64, timing=False, out=None,
              info=True, **kw):
    """spm_rsvd_host: RandSVD of a host (CPU) matrix, results in host tensors.

    A and ``out`` should be page-locked (``tensor.pin_memory()``) for the copies
    to overlap; the library stages A into device memory in row chunks and
    starts the sketch product of each chunk on arrival.  Returns (U, sigma, Vt,
    info) once the current stream has been synchronised."""
    if A.is_cuda or A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("a row-major host (CPU) matrix is required")
    o = make_opts(precision, **kw)
    m, n = A.shape
    if out is None:
        U = torch.empty(m, k, dtype=A.dtype).pin_memory()
        sig = torch.empty(k, dtype=A.dtype).pin_memory()
        Vt = torch.empty(k, n, dtype=A.dtype).pin_memory()
    else:
        U, sig, Vt = out
        if U.is_cuda or sig.is_cuda or Vt.is_cuda:
            raise ValueError("host (CPU) output tensors are required")
    inf = _info(timing) if info else None
    rc = lib().spm_rsvd_host(S.handle, _ptr(A), _dt(A), m, A.stride(0), r2, q, int(omega_seed), k,
                             ctypes.byref(o), _ptr(U), U.stride(0), _ptr(sig), _ptr(Vt),
                             Vt.stride(0), ctypes.byref(inf) if inf is not None else None,
                             _stream())
    _check(rc, "spm_rsvd_host")
    if inf is None:
        torch.cuda.current_stream().synchronize()
    return U, sig, Vt, (inf.as_dict() if inf is not None else None)


def lowrank(S1, S2, A, r2, q, omega_seed=43, precision=PREC_FP64, timing=False, **kw):
    _require_cuda(A)
    o = make_opts(precision, **kw)
    m, n = A.shape
    Y = torch.empty(m, r2, dtype=A.dtype, device=A.device)
    X = torch.empty(r2, n, dtype=A.dtype, device=A.device)
    inf = _info(timing)
    _check(lib().spm_lowrank(S1.handle, S2.handle, _ptr(A), _dt(A), m, A.stride(0), r2, q,
                             int(omega_seed), ctypes.byref(o), _ptr(Y), Y.stride(0), _ptr(X),
                             X.stride(0), ctypes.byref(inf), _stream()), "spm_lowrank")
    return Y, X, inf.as_dict()


def nystrom(S, A, r2, q, omega_seed=43, precision=PREC_FP64, timing=False, **kw):
    _require_cuda(A)
    o = make_opts(precision, **kw)
    n = A.shape[0]
    Cm = torch.empty(n, r2, dtype=A.dtype, device=A.device)
    W = torch.empty(r2, r2, dtype=A.dtype, device=A.device)
    inf = _info(timing)
    _check(lib().spm_nystrom(S.handle, _ptr(A), _dt(A), n, A.stride(0), r2, q, int(omega_seed),
                             ctypes.byref(o), _ptr(Cm), Cm.stride(0), _ptr(W), W.stride(0),
                             ctypes.byref(inf), _stream()), "spm_nystrom")
    return Cm, W, inf.as_dict()


def nystrom_eig(S, A, r2, q, omega_seed=43, precision=PREC_FP64, timing=False, **kw):
    """Algorithm 3 in factored form (spm_nystrom_eig): (U, lam, info) with
    A_hat = U diag(lam) U^T."""
    _require_cuda(A)
    o = make_opts(precision, **kw)
    n = A.shape[0]
    U = torch.empty(n, r2, dtype=A.dtype, device=A.device)
    lam = torch.empty(r2, dtype=A.dtype, device=A.device)
    inf = _info(timing)
    fn = _fn("spm_nystrom_eig", [VP, VP, I32, I64, I64, I64, I32, U64, ctypes.POINTER(Opts), VP, I64,
                                 VP, ctypes.POINTER(Info), VP])
    _check(fn(S.handle, _ptr(A), _dt(A), n, A.stride(0), r2, q, int(omega_seed), ctypes.byref(o),
              _ptr(U), U.stride(0), _ptr(lam), ctypes.byref(inf), _stream()), "spm_nystrom_eig")
    return U, lam, inf.as_dict()


def set_autotune(mode):
    """spm_set_autotune: 1 = time the split-K candidates of each product shape on
    first use and cache the fastest; 0 = the cost model (default)."""
    _check(lib().spm_set_autotune(int(mode)), "spm_set_autotune")


def autotune_entries(clear=False):
    """Number of product shape classes tuned so far (spm_autotune_entries)."""
    return int(lib().spm_autotune_entries(int(bool(clear))))


def gauss_sketch(S, X, h):
    """K S for the Gaussian kernel of the rows of X (spm_gauss_sketch): K never formed."""
    _require_cuda(X)
    n, d = X.shape
    out = torch.empty(n, S.r1, dtype=X.dtype, device=X.device)
    fn = _fn("spm_gauss_sketch", [VP, VP, I32, I64, I64, I64, ctypes.c_double, VP, I64, VP])
    _check(fn(S.handle, _ptr(X), _dt(X), n, d, X.stride(0), float(h), _ptr(out), out.stride(0),
              _stream()), "spm_gauss_sketch")
    return out


def nystrom_gauss(S, X, h, r2, q, omega_seed=43, precision=PREC_FP64, timing=False, **kw):
    """Factored Nystrom of the Gaussian kernel of the rows of X (spm_nystrom_gauss):
    (U, lam, info) with K_hat = U diag(lam) U^T."""
    _require_cuda(X)
    o = make_opts(precision, **kw)
    n, d = X.shape
    U = torch.empty(n, r2, dtype=X.dtype, device=X.device)
    lam = torch.empty(r2, dtype=X.dtype, device=X.device)
    inf = _info(timing)
    fn = _fn("spm_nystrom_gauss", [VP, VP, I32, I64, I64, I64, ctypes.c_double, I64, I32, U64,
                                   ctypes.POINTER(Opts), VP, I64, VP, ctypes.POINTER(Info), VP])
    _check(fn(S.handle, _ptr(X), _dt(X), n, d, X.stride(0), float(h), r2, q, int(omega_seed),
              ctypes.byref(o), _ptr(U), U.stride(0), _ptr(lam), ctypes.byref(inf), _stream()),
           "spm_nystrom_gauss")
    return U, lam, inf.as_dict()


def gemm_bf16(A_list, B_list, M, N, K, a_mn=False, b_mn=False, splitk=1):
    """D (M x N, fp32) = sum_q A_q B_q^T with bf16 operand tensors (see spm.h)."""
    npass = len(A_list)
    D = torch.empty(M, N, dtype=torch.float32, device="cuda")
    Ap = (VP * npass)(*[a.data_ptr() for a in A_list])
    Bp = (VP * npass)(*[b.data_ptr() for b in B_list])
    _check(lib().spm_gemm_bf16(M, N, K, npass, Ap, A_list[0].stride(0), int(a_mn), Bp,
                               B_list[0].stride(0), int(b_mn), _ptr(D), D.stride(0), int(splitk),
                               _stream()), "spm_gemm_bf16")
    return D


def gemm_bf16_noalloc(A_list, B_list, M, N, K, D, a_mn=False, b_mn=False, splitk=1):
    """Same product as gemm_bf16 into a caller-provided fp32 D, with no device allocation.

    For callers that may not allocate device memory (see spm_gemm_bf16_noalloc in spm.h):
    split-K partial sums use a fixed library-owned device array instead of workspace.
    """
    L = lib()
    fn = L.spm_gemm_bf16_noalloc
    fn.argtypes = [I64, I64, I64, I32, ctypes.POINTER(VP), I64, I32, ctypes.POINTER(VP), I64, I32,
                   VP, I64, I32, VP]
    fn.restype = I32
    npass = len(A_list)
    Ap = (VP * npass)(*[a.data_ptr() for a in A_list])
    Bp = (VP * npass)(*[b.data_ptr() for b in B_list])
    _check(fn(M, N, K, npass, Ap, A_list[0].stride(0), int(a_mn), Bp, B_list[0].stride(0),
              int(b_mn), _ptr(D), D.stride(0), int(splitk), _stream()), "spm_gemm_bf16_noalloc")
    return D


def sketch_set_plan(S, mode):
    """spm_sketch_set_plan: 0 (or False) keeps this sketch on the general kernels,
    1 (or True) plans at its first eligible product, 2 plans only for large products."""
    fn = _fn("spm_sketch_set_plan", [VP, I32])
    _check(fn(S.handle, int(mode)), "spm_sketch_set_plan")


def sketch_plan(S):
    """(state, steps_per_row, groups) of the sketch's scheduled product (spm_sketch_plan):
    state 0 = not planned yet, 1 = ready, -1 = does not fit."""
    st, steps, g = I32(), I64(), I32()
    fn = _fn("spm_sketch_plan", [VP, ctypes.POINTER(I32), ctypes.POINTER(I64), ctypes.POINTER(I32)])
    _check(fn(S.handle, ctypes.byref(st), ctypes.byref(steps), ctypes.byref(g)), "spm_sketch_plan")
    return int(st.value), int(steps.value), int(g.value)


SCHED_TT, SCHED_LANES, SCHED_PAD = 96, 1024, 32


def sched_plan_host(n, r1, col_ptr, col_ent, search=300000):
    """Host-side plan of the scheduled product for a sparse sign matrix given by its
    columns (spm_sched_plan_host; no GPU needed).  col_ptr (r1 + 1, int64) and col_ent
    (uint32: j | 0x80000000 for a -1 entry) are numpy arrays.  Returns a dict with the
    group count, steps per row and the per-warp tables, or raises SpmError."""
    import numpy as np
    col_ptr = np.ascontiguousarray(col_ptr, dtype=np.int64)
    col_ent = np.ascontiguousarray(col_ent, dtype=np.uint32)
    fn = _fn("spm_sched_plan_host", [I64, I64, VP, VP, I64, ctypes.POINTER(I32),
                                     ctypes.POINTER(I64), VP, VP, VP, VP])
    g, steps = I32(), I64()
    _check(fn(n, r1, col_ptr.ctypes.data, col_ent.ctypes.data, search, ctypes.byref(g),
              ctypes.byref(steps), None, None, None, None), "spm_sched_plan_host")
    G = int(g.value)
    cw = -(-r1 // G)
    words = np.zeros(G * 32 * (SCHED_TT // 2) * 32, dtype=np.uint32)
    wsteps = np.zeros(G * 32 * 2, dtype=np.int32)
    slots = np.zeros(G * SCHED_LANES, dtype=np.int32)
    partner = np.zeros(G * cw, dtype=np.int32)
    _check(fn(n, r1, col_ptr.ctypes.data, col_ent.ctypes.data, search, ctypes.byref(g),
              ctypes.byref(steps), words.ctypes.data, wsteps.ctypes.data, slots.ctypes.data,
              partner.ctypes.data), "spm_sched_plan_host")
    return {"groups": G, "cw": cw, "steps": int(steps.value),
            "words": words.reshape(G, 32, SCHED_TT // 2, 32), "wsteps": wsteps.reshape(G, 32, 2),
            "slots": slots.reshape(G, SCHED_LANES), "partner": partner.reshape(G, cw)}


def gemm_bf16_status(clear=True):
    """Device status of the public product entry points on the current device
    (spm_gemm_bf16_status): 0, or SPM_ETIMEOUT if one of their bounded waits expired."""
    fn = _fn("spm_gemm_bf16_status", [I32, VP])
    return int(fn(int(bool(clear)), _stream()))


# ---------------------------------------------------------------- learned selector
MLP_IN, MLP_OUT, MLP_PARAMS = 8, 15, 9871
CANDIDATES = [(q, c) for q in range(5) for c in (2, 4, 8)]   # output index 3 q + c_idx


def _fn(name, args, res=I32):
    f = getattr(lib(), name)
    f.argtypes = args
    f.restype = res
    return f


def mlp_forward(params, X):
    Y = torch.empty(X.shape[0], MLP_OUT, device="cuda", dtype=torch.float32)
    f = _fn("spm_mlp_forward", [VP, VP, I64, VP, VP])
    _check(f(_ptr(params), _ptr(X), X.shape[0], _ptr(Y), _stream()), "spm_mlp_forward")
    return Y


def mlp_loss_grad(params, X, T, M):
    grad = torch.empty(MLP_PARAMS, device="cuda", dtype=torch.float32)
    loss = torch.empty(1, device="cuda", dtype=torch.float32)
    f = _fn("spm_mlp_loss_grad", [VP, VP, VP, VP, I64, VP, VP, VP])
    _check(f(_ptr(params), _ptr(X), _ptr(T), _ptr(M), X.shape[0], _ptr(grad), _ptr(loss), _stream()),
           "spm_mlp_loss_grad")
    return loss, grad


def mlp_adam(params, m, v, grad, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    f = _fn("spm_mlp_adam", [VP, VP, VP, VP, I32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, VP])
    _check(f(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), int(step), lr, b1, b2, eps, _stream()),
           "spm_mlp_adam")


def selector_features(S, A, r2, omega_seed=43):
    _require_cuda(A)
    feat = torch.empty(MLP_IN, device="cuda", dtype=torch.float32)
    f = _fn("spm_selector_features", [VP, VP, I32, I64, I64, I64, U64, VP, VP])
    _check(f(S.handle, _ptr(A), _dt(A), A.shape[0], A.stride(0), r2, int(omega_seed), _ptr(feat),
             _stream()), "spm_selector_features")
    return feat


def rsvd_auto(A, k, target_ratio, params, seed=42, precision=PREC_MIXED, **kw):
    """RandSVD with (q, r1) picked by the selector network; returns U, sigma, Vt, (q, c), info."""
    _require_cuda(A)
    m, n = A.shape
    o = make_opts(precision, **kw)
    U = torch.empty(m, k, dtype=A.dtype, device=A.device)
    sg = torch.empty(k, dtype=A.dtype, device=A.device)
    Vt = torch.empty(k, n, dtype=A.dtype, device=A.device)
    choice = (ctypes.c_int32 * 2)()
    inf = _info(False)
    f = _fn("spm_rsvd_auto", [VP, I32, I64, I64, I64, I64, ctypes.c_double, VP, U64,
                              ctypes.POINTER(Opts), VP, I64, VP, VP, I64, ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(Info), VP])
    _check(f(_ptr(A), _dt(A), m, n, A.stride(0), k, float(target_ratio), _ptr(params), int(seed),
             ctypes.byref(o), _ptr(U), U.stride(0), _ptr(sg), _ptr(Vt), Vt.stride(0), choice,
             ctypes.byref(inf), _stream()), "spm_rsvd_auto")
    return U, sg, Vt, (int(choice[0]), int(choice[1])), inf.as_dict()


# ---------------------------------------------------------------- batched RandSVD
class BatchItem(ctypes.Structure):
    _fields_ = [("A", VP), ("m", I64), ("n", I64), ("lda", I64), ("k", I64), ("r1", I64),
                ("s", I32), ("q", I32), ("seed", U64), ("U", VP), ("ldu", I64), ("sigma", VP),
                ("Vt", VP), ("ldvt", I64)]


class Batch:
    """A prepared batch of RandSVD problems with preallocated outputs.

    problems: list of dicts {A (cuda m x n), k, r1, q, s=8, seed=42}.  run()
    issues one spm_rsvd_batched call on the current stream; it may be captured
    with torch.cuda.graph and replayed.  outputs[i] = (U, sigma, Vt), status =
    device int32 per problem.
    """

    def __init__(self, problems, precision=PREC_MIXED, nstreams=0, **kw):
        self.items = (BatchItem * len(problems))()
        self.outputs = []
        self.inputs = []
        dt = None
        dev = None
        for i, p in enumerate(problems):
            A = p["A"]
            _require_cuda(A)
            if A.stride(1) != 1:
                raise ValueError("A must be row-major")
            d = _dt(A)
            if dt is not None and d != dt:
                raise ValueError("all problems of a batch share one dtype")
            dt, dev = d, A.device
            m, n = A.shape
            k = p["k"]
            U = torch.empty(m, k, dtype=A.dtype, device=A.device)
            sg = torch.empty(k, dtype=A.dtype, device=A.device)
            Vt = torch.empty(k, n, dtype=A.dtype, device=A.device)
            self.items[i] = BatchItem(A.data_ptr(), m, n, A.stride(0), k, p.get("r1", min(2 * k, n)),
                                      p.get("s", 8), p.get("q", 2), p.get("seed", 42), U.data_ptr(), U.stride(0),
                                      sg.data_ptr(), Vt.data_ptr(), Vt.stride(0))
            self.inputs.append(A)
            self.outputs.append((U, sg, Vt))
        self.dtype = dt if dt is not None else F32
        self.status = torch.zeros(max(len(problems), 1), dtype=torch.int32,
                                  device=dev if dev is not None else "cuda")
        self.opts = make_opts(precision, **kw)
        self.nstreams = nstreams
        self._f = _fn("spm_rsvd_batched", [I32, ctypes.POINTER(BatchItem), I32,
                                           ctypes.POINTER(Opts), I32, VP, VP])

    def run(self):
        _check(self._f(len(self.outputs), self.items, self.dtype, ctypes.byref(self.opts),
                       self.nstreams, self.status.data_ptr(), _stream()), "spm_rsvd_batched")
        return self.outputs

    def run_auto(self, target_ratio, params):
        """spm_rsvd_batched_auto: pick (q, r1) per problem with the selector network, run
        the batch and judge every result by its residual estimate (more power steps,
        a doubled sketch, FP32 at the precision limit; see spm.h).  Returns the network's
        (q, c) picks (r1 = c k); the (q, r1, s) of each kept result stay in the items,
        so run() replays them."""
        count = len(self.outputs)
        ch = (ctypes.c_int32 * max(2 * count, 2))()
        f = _fn("spm_rsvd_batched_auto", [I32, ctypes.POINTER(BatchItem), I32, ctypes.c_double, VP,
                                          ctypes.POINTER(Opts), I32, VP, ctypes.POINTER(ctypes.c_int32),
                                          VP])
        _check(f(count, self.items, self.dtype, float(target_ratio), _ptr(params),
                 ctypes.byref(self.opts), self.nstreams, self.status.data_ptr(), ch, _stream()),
               "spm_rsvd_batched_auto")
        return [(int(ch[2 * i]), int(ch[2 * i + 1])) for i in range(count)]

    def item_params(self):
        """The (q, r1, s) each item runs with (after run_auto: those of the kept result)."""
        return [(int(self.items[i].q), int(self.items[i].r1), int(self.items[i].s))
                for i in range(len(self.outputs))]

    def check_status(self):
        st = self.status.cpu()
        bad = [(i, int(v)) for i, v in enumerate(st.tolist()[:len(self.outputs)]) if v != 0]
        if bad:
            raise RuntimeError(f"spm_rsvd_batched: device status {bad[:5]}")


def rsvd_batched(problems, precision=PREC_MIXED, nstreams=0, **kw):
    """One eager batched call; returns [(U, sigma, Vt)] after checking device status."""
    b = Batch(problems, precision, nstreams, **kw)
    out = b.run()
    b.check_status()
    return out
