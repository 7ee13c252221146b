"""Split-K autotuning (spm_set_autotune): a tuned RandSVD agrees with the
cost-model one to rounding, the tuned classes are cached, and once tuned the
calls repeat bit for bit (the choice is fixed and every product deterministic)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spm():
    from paper_2605_09755_gb300 import _build, spm as _spm
    _build.build()
    _spm.lib()
    return _spm


def test_autotuned_rsvd_matches_model_and_repeats(spm):
    from paper_2605_09755_gb300 import workloads as wl
    m, n, r1, k = 6000, 3000, 400, 150
    A, _ = wl.noisy_exp_torch(m, n, seed=11, noise=1e-3)
    S = spm.Sketch(n, r1, 8, 42)
    spm.autotune_entries(clear=True)
    spm.set_autotune(0)
    U0, s0, V0, _ = spm.rsvd(S, A, k, 2, k, precision=spm.PREC_MIXED)
    try:
        spm.set_autotune(1)
        U1, s1, V1, _ = spm.rsvd(S, A, k, 2, k, precision=spm.PREC_MIXED)
        assert spm.autotune_entries() > 0
        U2, s2, V2, _ = spm.rsvd(S, A, k, 2, k, precision=spm.PREC_MIXED)
    finally:
        spm.set_autotune(0)
        spm.autotune_entries(clear=True)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(s1 - s0)) <= 1e-4 * s0[0]
    assert torch.equal(s1, s2) and torch.equal(U1, U2) and torch.equal(V1, V2)
    with pytest.raises(spm.SpmError):
        spm.set_autotune(2)
