"""spm_rsvd_host: RandSVD of a matrix in host memory, through the C ABI.

The host entry stages A into device memory in row chunks and starts the
sketch product of each chunk as it arrives; every kernel computes what the
device entry computes on the same data (the sketch kernel's 32-row blocks do
not straddle chunks), so U, sigma and Vt must equal spm_rsvd's bit for bit.
The device entry itself is checked against the oracle elsewhere.
"""
import numpy as np
import pytest
import torch

from paper_2605_09755_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spm():
    from paper_2605_09755_gb300 import _build, spm as _spm
    _build.build()
    _spm.lib()
    return _spm


@pytest.mark.parametrize("prec,dtype", [("mixed", torch.float32), ("fp64", torch.float64),
                                        ("fp32", torch.float32)])
@pytest.mark.parametrize("m,n,r1,r2,q,pad,pinned", [(3000, 1500, 300, 100, 2, 0, True),
                                                    (2100, 700, 140, 60, 1, 5, False),
                                                    (64, 40, 20, 10, 0, 0, True)])
def test_rsvd_host_equals_device(spm, prec, dtype, m, n, r1, r2, q, pad, pinned):
    p = {"mixed": spm.PREC_MIXED, "fp64": spm.PREC_FP64, "fp32": spm.PREC_FP32}[prec]
    A, _ = wl.noisy_exp_numpy(m, n, seed=77, noise=1e-3 / np.sqrt(n))
    Ah = torch.zeros(m, n + pad, dtype=dtype)
    Ah[:, :n] = torch.tensor(A, dtype=dtype)
    if pinned:
        Ah = Ah.pin_memory()
    Ah_view = Ah[:, :n]
    S = spm.Sketch(n, r1, 8, 42)
    Uh, sh, Vh, info = spm.rsvd_host(S, Ah_view, r2, q, r2, precision=p)
    assert info["device_status"] == 0
    Ud, sd, Vd, _ = spm.rsvd(S, Ah_view.cuda(), r2, q, r2, precision=p)
    torch.cuda.synchronize()
    assert torch.equal(Uh, Ud.cpu())
    assert torch.equal(sh, sd.cpu())
    assert torch.equal(Vh, Vd.cpu())
    assert abs(info["fro_a"] - np.linalg.norm(A)) <= 1e-5 * np.linalg.norm(A)


def test_rsvd_host_rejects_device_input(spm):
    S = spm.Sketch(100, 20, 8, 42)
    with pytest.raises(ValueError):
        spm.rsvd_host(S, torch.zeros(50, 100, device="cuda"), 10, 1, 10)


def test_trim_memory_then_reuse(spm):
    """The library pool keeps freed workspace between calls; trimming hands it
    back and the next call allocates afresh."""
    A = torch.randn(500, 300, device="cuda")
    S = spm.Sketch(300, 60, 8, 42)
    U1, s1, V1, _ = spm.rsvd(S, A, 30, 1, 30, precision=spm.PREC_MIXED)
    torch.cuda.synchronize()
    spm.trim_memory()
    U2, s2, V2, _ = spm.rsvd(S, A, 30, 1, 30, precision=spm.PREC_MIXED)
    torch.cuda.synchronize()
    assert torch.equal(U1, U2) and torch.equal(s1, s2) and torch.equal(V1, V2)
