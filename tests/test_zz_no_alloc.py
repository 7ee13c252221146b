"""The no-allocation product entry point (spm_gemm_bf16_noalloc).

Some callers may not allocate device memory (a plug-in inside an engine that owns
the device pool, a serving process with a fixed reservation).  This checks that
the variant which keeps its split-K partial sums in a fixed library-owned device
array returns what the allocating entry point returns, on two calls in a row
(the second with different inputs, so stale scratch contents would show), and
that requests larger than the array are refused.  Kept in its own file, named to
be collected last.
"""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spm():
    from paper_2605_09755_gb300 import _build, spm as _spm
    _build.build()
    _spm.lib()
    assert torch.cuda.is_available()
    return _spm


def _operands(M, N, K, seed, a_mn, b_mn):
    g = torch.Generator(device="cuda").manual_seed(seed)
    Am = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    Bm = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    A = Am.t().contiguous() if a_mn else Am.contiguous()
    B = Bm.t().contiguous() if b_mn else Bm.contiguous()
    return Am, Bm, A, B


@pytest.mark.parametrize("a_mn,b_mn", [(False, False), (True, True)])
def test_noalloc_matches_allocating_entry_point_twice(spm, a_mn, b_mn):
    M, N, K, splitk = 384, 512, 4096, 4      # 4 * 384 * 512 floats fit the scratch array
    spm.gemm_bf16_status(clear=True)
    for call, seed in enumerate((11, 12)):
        Am, Bm, A, B = _operands(M, N, K, seed, a_mn, b_mn)
        ref = spm.gemm_bf16([A], [B], M, N, K, a_mn=a_mn, b_mn=b_mn, splitk=splitk)
        D = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float32)
        spm.gemm_bf16_noalloc([A], [B], M, N, K, D, a_mn=a_mn, b_mn=b_mn, splitk=splitk)
        torch.cuda.synchronize()
        # the same kernels and the same fixed split-K order: equal bit for bit
        assert torch.equal(D, ref), call
        tol = 1e-4 * (K ** 0.5) * 4
        exact = Am.double() @ Bm.double().T
        assert (D.double() - exact).abs().max().item() <= tol, call
    assert spm.gemm_bf16_status(clear=True) == 0


def test_noalloc_ragged_tail_after_a_larger_call(spm):
    # a larger split-K call fills more of the shared scratch array first; a
    # following call with M not a multiple of 128 must not pick up its stale tail
    Am, Bm, A, B = _operands(1000, 500, 2048, 21, False, False)
    D = torch.empty(1000, 500, device="cuda", dtype=torch.float32)
    spm.gemm_bf16_noalloc([A], [B], 1000, 500, 2048, D, splitk=4)
    for M, N, K, splitk in [(300, 200, 3072, 3), (129, 257, 1000, 2)]:
        Am, Bm, A, B = _operands(M, N, K, 22 + M, False, False)
        ref = spm.gemm_bf16([A], [B], M, N, K, splitk=splitk)
        D = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float32)
        spm.gemm_bf16_noalloc([A], [B], M, N, K, D, splitk=splitk)
        torch.cuda.synchronize()
        assert torch.equal(D, ref), (M, N, K, splitk)
    assert spm.gemm_bf16_status(clear=True) == 0


def test_noalloc_split_precision_and_single_split(spm):
    M, N, K = 200, 130, 1024
    g = torch.Generator(device="cuda").manual_seed(3)
    X = torch.randn(M, K, device="cuda", generator=g, dtype=torch.float64)
    Y = torch.randn(N, K, device="cuda", generator=g, dtype=torch.float64)
    xh = X.float().to(torch.bfloat16)
    xl = (X.float() - xh.float()).to(torch.bfloat16)
    yh = Y.float().to(torch.bfloat16)
    yl = (Y.float() - yh.float()).to(torch.bfloat16)
    for splitk in (1, 3):
        ref = spm.gemm_bf16([xh, xh, xl], [yh, yl, yh], M, N, K, splitk=splitk)
        D = torch.empty(M, N, device="cuda", dtype=torch.float32)
        spm.gemm_bf16_noalloc([xh, xh, xl], [yh, yl, yh], M, N, K, D, splitk=splitk)
        torch.cuda.synchronize()
        assert torch.equal(D, ref), splitk
        assert (D.double() - X @ Y.T).abs().max().item() <= 1e-4 * (K ** 0.5) * 4


def test_noalloc_rejects_requests_beyond_the_scratch_array(spm):
    M, N, K = 1024, 1024, 4096               # 4 * 1024 * 1024 floats > 2 Mi
    A = torch.zeros(M, K, device="cuda", dtype=torch.bfloat16)
    B = torch.zeros(N, K, device="cuda", dtype=torch.bfloat16)
    D = torch.empty(M, N, device="cuda", dtype=torch.float32)
    with pytest.raises(spm.SpmError) as e:
        spm.gemm_bf16_noalloc([A], [B], M, N, K, D, splitk=4)
    assert e.value.code == 1
