"""The library's error codes through the C ABI, each made on purpose without
faulting or hanging the GPU.

  * SPM_ENONFINITE: a NaN in A reaches the Cholesky factorisation of the
    CholeskyQR Gram matrix, which records it (FP64, mixed and FP32 modes).
  * SPM_EBREAKDOWN: Algorithm 2's least-squares step X = (S2^T Y)^+ (S2^T A)
    factors the Gram matrix of S2^T Q; a row sketch S2 with empty column buckets
    makes S2^T Q rank deficient, and a singular factor is reported rather than
    deflated (deflation is only for orthonormalisation).
  * SPM_ETIMEOUT: spm_selftest_bounded_wait makes a device wait run out on
    purpose (it waits for one more CTA than it launches, with a clock limit);
    the kernel returns, the status reports it, and the context stays usable.
"""
import numpy as np
import pytest
import torch

from oracle import sketch as osk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spm():
    from paper_2605_09755_gb300 import _build, spm as _spm
    _build.build()
    _spm.lib()
    assert torch.cuda.is_available()
    return _spm


@pytest.mark.parametrize("prec,dtype", [("fp64", torch.float64), ("mixed", torch.float32),
                                        ("fp32", torch.float32)])
def test_nan_input_reports_nonfinite(spm, prec, dtype):
    p = {"fp64": spm.PREC_FP64, "mixed": spm.PREC_MIXED, "fp32": spm.PREC_FP32}[prec]
    m, n = 300, 200
    A = torch.randn(m, n, dtype=dtype, device="cuda")
    A[17, 33] = float("nan")
    S = spm.Sketch(n, 60, 8, 42)
    with pytest.raises(spm.SpmError) as e:
        spm.rsvd(S, A, 20, 1, 20, precision=p)
    assert e.value.code == 5            # SPM_ENONFINITE


def test_singular_least_squares_factor_reports_breakdown(spm):
    m, n, r2, seed = 40, 120, 20, 7
    cols, _ = osk.sketch_entries(m, r2, 1, seed)
    assert len(np.unique(cols)) < r2    # some bucket of S2 is empty: S2^T Q has rank < r2
    rng = np.random.default_rng(1)
    A = torch.tensor(rng.standard_normal((m, n)), device="cuda")
    S1 = spm.Sketch(n, 60, 8, 42)
    S2 = spm.Sketch(m, r2, 1, seed)
    with pytest.raises(spm.SpmError) as e:
        spm.lowrank(S1, S2, A, r2, 1, precision=spm.PREC_FP64)
    assert e.value.code == 4            # SPM_EBREAKDOWN
    # with a full-rank S2^T Q the same call succeeds
    S2ok = spm.Sketch(m, 2 * r2, 8, 11)
    Y, X, info = spm.lowrank(S1, S2ok, A, r2, 1, precision=spm.PREC_FP64)
    assert info["device_status"] == 0


def test_bounded_wait_runs_out_and_context_stays_usable(spm):
    L = spm.lib()
    st = torch.cuda.current_stream().cuda_stream
    fn = L.spm_selftest_bounded_wait
    import ctypes
    fn.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    assert fn(8, 0, 1 << 24, st) == 0             # everyone arrives: no timeout
    assert fn(8, 1, 1 << 22, st) == 6             # one arrival short: SPM_ETIMEOUT
    assert fn(1, 3, 1 << 20, st) == 6
    # the context is still usable: a library call afterwards succeeds
    A = torch.randn(200, 100, device="cuda", dtype=torch.float64)
    S = spm.Sketch(100, 30, 8, 42)
    U, sg, Vt, info = spm.rsvd(S, A, 10, 1, 10, precision=spm.PREC_FP64)
    assert info["device_status"] == 0
    assert fn(4, 0, 1 << 24, st) == 0
