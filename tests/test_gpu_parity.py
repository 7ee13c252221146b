"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Inputs come from the shared seeded generators; expected values come from the
oracle only.  Tolerances:
  * sketch tables: bit-exact (integer work);
  * Omega: a few ulp (libm vs CUDA log/sin/cos), |diff| <= 1e-13;
  * FP64 path: elementwise products <= 1e-12 relative to the operand scale;
    relative Frobenius residual of the range finder / RandSVD within 1e-10 of
    the oracle's at the same seed;
  * mixed path: residual <= 1.01 x the oracle's, top-k singular values within
    1e-4 relative.
"""
import numpy as np
import pytest
import torch

from oracle import algorithms as alg
from oracle import sketch as osk
from paper_2605_09755_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spm():
    from paper_2605_09755_gb300 import _build, spm as _spm
    _build.build()
    _spm.lib()
    assert torch.cuda.is_available()
    return _spm


def dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


# ------------------------------------------------------------------ a1 sketch tables
@pytest.mark.parametrize("n,r1,s,seed", [(1000, 100, 8, 42), (1537, 700, 8, 7), (513, 40, 1, 3),
                                         (64, 64, 64, 5), (16384, 2000, 8, 42), (3, 2, 2, 9)])
def test_sketch_tables_bit_exact(spm, n, r1, s, seed):
    S = spm.Sketch(n, r1, s, seed)
    cols, signs, bptr, brows, bsg = (t.cpu().numpy() for t in S.tables())
    So = osk.Sketch(n, r1, s, seed)
    assert np.array_equal(cols.reshape(n, s), So.cols)
    assert np.array_equal(signs.reshape(n, s).astype(np.int64), So.signs)
    ptr, rows, sg = So.buckets()
    assert np.array_equal(bptr, ptr)
    assert np.array_equal(brows, rows)
    assert np.array_equal(bsg.astype(np.int64), sg)


def test_identity_sketch_tables(spm):
    S = spm.Sketch(700, 700, 1, 0, kind=spm.IDENTITY)
    cols, signs, bptr, brows, bsg = (t.cpu().numpy() for t in S.tables())
    assert np.array_equal(cols, np.arange(700)) and np.all(signs == 1)
    assert np.array_equal(bptr, np.arange(701)) and np.array_equal(brows, np.arange(700))


# ------------------------------------------------------------------ a2 Omega
@pytest.mark.parametrize("rows,cols", [(100, 50), (7, 3), (2000, 1000)])
def test_gaussian_matches_oracle(spm, rows, cols):
    g = host(spm.gaussian(rows, cols, 43, torch.float64))
    o = osk.gaussian(rows, cols, 43)
    assert np.max(np.abs(g - o)) <= 1e-13
    g32 = spm.gaussian(rows, cols, 43, torch.float32).cpu().numpy()
    assert np.array_equal(g32, o.astype(np.float32)) or np.max(np.abs(g32 - o)) < 1e-6


# ------------------------------------------------------------------ a3 A S and S^T X
@pytest.mark.parametrize("m,n,r1,s", [(100, 1100, 700, 8), (33, 513, 1025, 3), (1, 5, 4, 2),
                                      (257, 2048, 2000, 8)])
def test_sketch_apply_parity(spm, m, n, r1, s):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    So = osk.Sketch(n, r1, s, 42)
    ref = osk.apply_right(A, So)
    S = spm.Sketch(n, r1, s, 42)
    out64 = host(spm.sketch_apply(S, dev(A)))
    scale = np.sqrt(s) * np.abs(A).max()
    assert np.max(np.abs(out64 - ref)) <= 1e-13 * scale
    out32 = host(spm.sketch_apply(S, dev(A, torch.float32)))
    assert np.max(np.abs(out32 - ref)) <= 1e-5 * scale
    X = rng.standard_normal((n, 37))
    refT = osk.apply_left_t(So, X)
    outT = host(spm.sketch_apply_t(S, dev(X)))
    assert np.max(np.abs(outT - refT)) <= 1e-13 * np.sqrt(s) * np.abs(X).max() * n / r1 * 4


def test_sketch_apply_identity_is_copy(spm):
    A = np.random.default_rng(1).standard_normal((70, 600))
    S = spm.Sketch(600, 600, 1, 0, kind=spm.IDENTITY)
    assert np.array_equal(host(spm.sketch_apply(S, dev(A))), A)


# ------------------------------------------------------------------ tcgen05 product
@pytest.mark.parametrize("a_mn,b_mn", [(False, False), (False, True), (True, False), (True, True)])
@pytest.mark.parametrize("M,N,K", [(300, 200, 500), (128, 256, 64), (1000, 77, 130)])
def test_gemm_bf16_layouts(spm, a_mn, b_mn, M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * N + K)
    Am = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    Bm = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    ref = Am.double() @ Bm.double().T
    Ast = Am.t().contiguous() if a_mn else Am.contiguous()
    Bst = Bm.t().contiguous() if b_mn else Bm.contiguous()
    # the ABI wants leading dimensions that are multiples of 8
    def pad(t):
        c = t.shape[1]
        cp = (c + 7) // 8 * 8
        out = torch.zeros(t.shape[0], cp, dtype=t.dtype, device=t.device)
        out[:, :c] = t
        return out
    D = spm.gemm_bf16([pad(Ast)], [pad(Bst)], M, N, K, a_mn=a_mn, b_mn=b_mn)
    err = (D.double() - ref).abs().max().item()
    assert err <= 1e-4 * (K ** 0.5) * 4, err
    D2 = spm.gemm_bf16([pad(Ast)], [pad(Bst)], M, N, K, a_mn=a_mn, b_mn=b_mn, splitk=3)
    assert (D2.double() - ref).abs().max().item() <= 1e-4 * (K ** 0.5) * 4


def test_gemm_bf16_rejects_operands_off_the_current_device(spm):
    # the tensor maps cover only this GPU's memory: a host operand (pinned or
    # pageable) or a host D is refused before anything is launched
    M = N = K = 64
    dev = torch.zeros(K, M, dtype=torch.bfloat16, device="cuda")
    for host in (torch.zeros(K, M, dtype=torch.bfloat16).pin_memory(),
                 torch.zeros(K, M, dtype=torch.bfloat16)):
        with pytest.raises(spm.SpmError):
            spm.gemm_bf16([host], [dev], M, N, K, a_mn=True, b_mn=True)
        with pytest.raises(spm.SpmError):
            spm.gemm_bf16([dev], [host], M, N, K, a_mn=True, b_mn=True)
    D = spm.gemm_bf16([dev], [dev], M, N, K, a_mn=True, b_mn=True)
    assert torch.count_nonzero(D).item() == 0


def test_gemm_bf16_split_precision(spm):
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn(700, 304, device="cuda", generator=g, dtype=torch.float64)
    Y = torch.randn(150, 304, device="cuda", generator=g, dtype=torch.float64)
    def split(t):
        hi = t.float().to(torch.bfloat16)
        lo = (t.float() - hi.float()).to(torch.bfloat16)
        return hi.contiguous(), lo.contiguous()
    xh, xl = split(X)
    yh, yl = split(Y)
    D = spm.gemm_bf16([xh, xh, xl], [yh, yl, yh], 700, 150, 304)
    ref = X @ Y.T
    rel = ((D.double() - ref).abs().max() / ref.abs().max()).item()
    assert rel < 2e-5, rel


# ------------------------------------------------------------------ Algorithm 1 / RandSVD, FP64
def _oracle_rsvd(A, n, r1, s, r2, q, k, sseed=42, oseed=43, kind=osk.SPARSE_SIGN):
    So = osk.Sketch(n, r1, s, sseed, kind=kind)
    Om = osk.gaussian(r1, r2, oseed)
    return alg.rsvd(A, So, Om, q, k)


@pytest.mark.parametrize("m,n,r1,r2,q,s", [(2000, 1000, 100, 50, 2, 8), (777, 513, 130, 40, 1, 4),
                                           (300, 200, 60, 60, 0, 8), (129, 65, 65, 33, 3, 1)])
def test_rsvd_fp64_parity(spm, m, n, r1, r2, q, s):
    A, sigma = wl.plain_fp64(m, n, seed=1001)
    k = r2
    U_o, s_o, Vt_o, Q_o = _oracle_rsvd(A, n, r1, s, r2, q, k)
    res_o = np.linalg.norm(A - (U_o * s_o) @ Vt_o)
    S = spm.Sketch(n, r1, s, 42)
    U, sg, Vt, info = spm.rsvd(S, dev(A), r2, q, k, omega_seed=43, precision=spm.PREC_FP64)
    U, sg, Vt = host(U), host(sg), host(Vt)
    res = np.linalg.norm(A - (U * sg) @ Vt)
    opt = alg.optimal_fro(sigma, k)
    assert abs(res / opt - res_o / opt) <= 1e-10 * (res_o / opt)
    assert np.max(np.abs(sg - s_o) / s_o) <= 1e-10
    assert np.linalg.norm(U.T @ U - np.eye(k)) <= 1e-12
    # singular vectors agree up to the shared sign convention where the gaps allow
    gap = np.min(np.abs(np.diff(s_o))) / s_o[0]
    if gap > 1e-6:
        assert np.max(np.abs(U - U_o)) <= 1e-7
    assert info["device_status"] == 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("m,n,r1,r2,q,noise", [(1500, 700, 200, 80, 1, 1e-2), (600, 900, 120, 60, 2, 1e-1),
                                                (2048, 512, 256, 100, 0, 3e-2)])
def test_resid_est_matches_oracle_residual(spm, prec, m, n, r1, r2, q, noise):
    """info.resid_est = sqrt(|A|_F^2 - |Q^T A|_F^2) against the oracle's
    residual_fro(A, Q) = |A - Q Q^T A|_F formed directly, for the library's own
    basis (k = r2, so U spans Q).  The subtraction loses relative accuracy
    |A|_F^2 / resid^2 times the working precision."""
    A, _ = wl.noisy_exp_numpy(m, n, seed=m + n, noise=noise)
    p = {"fp64": spm.PREC_FP64, "mixed": spm.PREC_MIXED}[prec]
    dt = torch.float64 if prec == "fp64" else torch.float32
    S = spm.Sketch(n, r1, 8, 42)
    U, sg, Vt, info = spm.rsvd(S, dev(A, dt), r2, q, r2, omega_seed=43, precision=p)
    U = host(U)
    Qg, _ = np.linalg.qr(U)              # the same range, exactly orthonormal
    res = alg.residual_fro(A, Qg)
    fro = np.linalg.norm(A)
    assert abs(info["fro_a"] - fro) <= (1e-12 if prec == "fp64" else 1e-6) * fro
    u = 1e-15 if prec == "fp64" else 2e-6
    assert abs(info["resid_est"] - res) <= 10 * u * fro ** 2 / res + 1e-12 * fro


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rsvd_truncated_rank_below_r2(spm, prec):
    """k < r2: the finish keeps the k largest of the r2 computed directions (the
    rows of V^T and columns of U~ gathered in the order of sigma)."""
    m, n, r1, r2, k, q = 1500, 700, 120, 60, 25, 2
    A, sigma = wl.plain_fp64(m, n, seed=1001)
    if prec == "mixed":
        A = A.astype(np.float32).astype(np.float64)
    U_o, s_o, Vt_o, _ = _oracle_rsvd(A, n, r1, 8, r2, q, k)
    res_o = np.linalg.norm(A - (U_o * s_o) @ Vt_o)
    S = spm.Sketch(n, r1, 8, 42)
    if prec == "fp64":
        U, sg, Vt, info = spm.rsvd(S, dev(A), r2, q, k, omega_seed=43, precision=spm.PREC_FP64)
    else:
        U, sg, Vt, info = spm.rsvd(S, dev(A, torch.float32), r2, q, k, precision=spm.PREC_MIXED)
    U, sg, Vt = host(U), host(sg), host(Vt)
    assert U.shape == (m, k) and sg.shape == (k,) and Vt.shape == (k, n)
    res = np.linalg.norm(A - (U * sg) @ Vt)
    if prec == "fp64":
        assert abs(res - res_o) <= 1e-10 * res_o
        assert np.max(np.abs(sg - s_o) / s_o) <= 1e-10
        assert np.linalg.norm(U.T @ U - np.eye(k)) <= 1e-12
    else:
        assert res <= 1.01 * res_o, (res, res_o)
        assert np.max(np.abs(sg - s_o) / s_o) <= 1e-4
        assert np.linalg.norm(U.T @ U - np.eye(k)) <= 1e-3
    assert np.all(sg[:-1] >= sg[1:])
    assert info["device_status"] == 0


def test_range_finder_fp64_identity_sketch_is_classical(spm):
    """S = I: the CUDA path reproduces the classical range finder of the oracle."""
    A, sigma = wl.plain_fp64(400, 200, seed=3)
    So = osk.Sketch(200, 200, 1, 0, kind=osk.IDENTITY)
    Q_o = alg.range_finder(A, So, osk.gaussian(200, 20, 43), q=3)
    S = spm.Sketch(200, 200, 1, 0, kind=spm.IDENTITY)
    Q, info = spm.range_finder(S, dev(A), 20, 3, omega_seed=43)
    Q = host(Q)
    assert np.linalg.norm(Q @ Q.T - Q_o @ Q_o.T) <= 1e-9
    assert abs(alg.residual_fro(A, Q) / alg.residual_fro(A, Q_o) - 1) <= 1e-10


def test_range_finder_caller_omega(spm):
    A, _ = wl.plain_fp64(300, 150, seed=4)
    Om = np.random.default_rng(2).standard_normal((50, 10))
    Q_o = alg.range_finder(A, osk.Sketch(150, 50, 8, 42), Om, q=2)
    S = spm.Sketch(150, 50, 8, 42)
    Q, _ = spm.range_finder(S, dev(A), 10, 2, omega=dev(Om))
    Q = host(Q)
    assert np.linalg.norm(Q @ Q.T - Q_o @ Q_o.T) <= 1e-9


def test_range_finder_exact_low_rank(spm):
    A, _ = wl.dense_lowrank(500, 300, np.array([5.0, 4.0, 3.0, 2.0, 1.0]), seed=8)
    S = spm.Sketch(300, 40, 8, 42)
    for prec, dt, tol in [(spm.PREC_FP64, torch.float64, 1e-11), (spm.PREC_MIXED, torch.float32, 1e-4)]:
        Q, _ = spm.range_finder(S, dev(A, dt), 10, 1, precision=prec)
        assert alg.residual_fro(A, host(Q)) <= tol * np.linalg.norm(A)


# ------------------------------------------------------------------ mixed precision
@pytest.mark.parametrize("m,n,r1,r2,q", [(4096, 2048, 256, 128, 2), (3000, 1500, 300, 100, 0),
                                         (2000, 1000, 100, 50, 2)])
def test_rsvd_mixed_parity(spm, m, n, r1, r2, q):
    if m == 2000:
        A, sigma = wl.plain_fp64(m, n, seed=1001)
    else:
        A, sigma = wl.noisy_exp_numpy(m, n, seed=1002, noise=1e-3 / np.sqrt(n))
    k = r2
    U_o, s_o, Vt_o, _ = _oracle_rsvd(A, n, r1, 8, r2, q, k)
    res_o = np.linalg.norm(A - (U_o * s_o) @ Vt_o)
    S = spm.Sketch(n, r1, 8, 42)
    U, sg, Vt, info = spm.rsvd(S, dev(A, torch.float32), r2, q, k, precision=spm.PREC_MIXED)
    U, sg, Vt = host(U), host(sg), host(Vt)
    res = np.linalg.norm(A - (U * sg) @ Vt)
    assert res <= 1.01 * res_o, (res, res_o)
    assert np.max(np.abs(sg - s_o) / s_o) <= 1e-4, np.max(np.abs(sg - s_o) / s_o)
    assert np.linalg.norm(U.T @ U - np.eye(k)) <= 1e-3
    assert info["device_status"] == 0


def test_rsvd_mixed_parity_wide(spm):
    """r2 = 600: the Gram products span several clusters of output tiles, so the
    symmetric Gram path (tiles below the diagonal skipped, then mirrored) is
    exercised, and the FP32 eigensolver runs ~6000 rotations per index (its
    eigenvector normalisation keeps the eigenvalues unbiased: before it, all
    sigma came out ~3e-4 low here).  q = 0 keeps kappa(Y) ~ sigma_1 / sigma_600
    ~ 30, so the single-precision basis keeps the tail.  Orthogonality: observed
    ~4e-7 k (Frobenius), bound 2e-6 k."""
    m, n, r1, r2, q = 3000, 1500, 1200, 600, 0
    A, sigma = wl.noisy_exp_numpy(m, n, seed=1002, noise=1e-3 / np.sqrt(n))
    U_o, s_o, Vt_o, _ = _oracle_rsvd(A, n, r1, 8, r2, q, r2)
    res_o = np.linalg.norm(A - (U_o * s_o) @ Vt_o)
    S = spm.Sketch(n, r1, 8, 42)
    U, sg, Vt, info = spm.rsvd(S, dev(A, torch.float32), r2, q, r2, precision=spm.PREC_MIXED)
    U, sg, Vt = host(U), host(sg), host(Vt)
    res = np.linalg.norm(A - (U * sg) @ Vt)
    assert res <= 1.01 * res_o, (res, res_o)
    assert np.max(np.abs(sg - s_o) / s_o) <= 1e-4, np.max(np.abs(sg - s_o) / s_o)
    assert np.linalg.norm(U.T @ U - np.eye(r2)) <= 2e-6 * r2
    assert info["device_status"] == 0


@pytest.mark.parametrize("m,n,r1,r2,q", [(2000, 1000, 100, 50, 2), (1500, 1100, 1000, 700, 1)])
def test_rsvd_fp32_parity(spm, m, n, r1, r2, q):
    """FP32 on CUDA cores: residual within 1% of the oracle's.
    With r2 = 700 of sigma_i = 1/i the iterates A~^T Y are conditioned like
    kappa(A~)^2 ~ 5e5, beyond what an FP32 Gram resolves, so Y is re-orthonormalised
    before each A~^T product too (reorth = 2)."""
    A, sigma = wl.plain_fp64(m, n, seed=1001)
    A = A.astype(np.float32).astype(np.float64)
    k = r2
    U_o, s_o, Vt_o, _ = _oracle_rsvd(A, n, r1, 8, r2, q, k)
    res_o = np.linalg.norm(A - (U_o * s_o) @ Vt_o)
    S = spm.Sketch(n, r1, 8, 42)
    U, sg, Vt, info = spm.rsvd(S, dev(A, torch.float32), r2, q, k, precision=spm.PREC_FP32,
                               reorth=2)
    U, sg, Vt = host(U), host(sg), host(Vt)
    res = np.linalg.norm(A - (U * sg) @ Vt)
    assert res <= 1.01 * res_o, (res, res_o)
    # sigma from an FP32 Gram eigensolver: absolute error ~ sqrt(r2) u32 sigma_1 times a
    # modest constant (observed < 15); bound 1e-6 sqrt(r2) sigma_1
    assert np.max(np.abs(sg - s_o)) <= 1e-6 * np.sqrt(r2) * s_o[0]
    # FP32 loss of orthogonality grows with k (a few hundred u32 per entry at k = 700)
    assert np.linalg.norm(U.T @ U - np.eye(k)) <= 3e-5 * k
    assert info["device_status"] == 0


def test_rsvd_mixed_small_fp64_option(spm):
    A, sigma = wl.plain_fp64(1500, 700, seed=11)
    U_o, s_o, Vt_o, _ = _oracle_rsvd(A, 700, 120, 8, 40, 2, 40)
    res_o = np.linalg.norm(A - (U_o * s_o) @ Vt_o)
    S = spm.Sketch(700, 120, 8, 42)
    U, sg, Vt, info = spm.rsvd(S, dev(A, torch.float32), 40, 2, 40, precision=spm.PREC_MIXED,
                               small_fp64=True)
    res = np.linalg.norm(A - (host(U) * host(sg)) @ host(Vt))
    assert res <= 1.01 * res_o
    assert np.max(np.abs(host(sg) - s_o) / s_o) <= 1e-4


# ------------------------------------------------------------------ Algorithm 2
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lowrank_parity(spm, prec):
    m, n, r1, r2, q = 900, 600, 120, 30, 2
    A, sigma = wl.plain_fp64(m, n, seed=21)
    S1o, S2o = osk.Sketch(n, r1, 8, 42), osk.Sketch(m, r1, 8, 44)
    Y_o, X_o = alg.lowrank(A, S1o, S2o, osk.gaussian(r1, r2, 43), q)
    ref = Y_o @ X_o
    S1, S2 = spm.Sketch(n, r1, 8, 42), spm.Sketch(m, r1, 8, 44)
    if prec == "fp64":
        Y, X, _ = spm.lowrank(S1, S2, dev(A), r2, q)
        assert np.linalg.norm(host(Y) @ host(X) - ref) <= 1e-9 * np.linalg.norm(A)
    else:
        Y, X, _ = spm.lowrank(S1, S2, dev(A, torch.float32), r2, q, precision=spm.PREC_MIXED)
        e = np.linalg.norm(A - host(Y) @ host(X))
        assert e <= 1.01 * np.linalg.norm(A - ref)


# ------------------------------------------------------------------ Algorithm 3
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nystrom_parity(spm, prec):
    K, h, X = wl.gmm_kernel(800, seed=1004)
    r1, r2, q = 200, 50, 1
    So = osk.Sketch(800, r1, 8, 42)
    C_o, W_o = alg.nystrom(K, So, osk.gaussian(r1, r2, 43), q)
    Ah_o = alg.nystrom_apply(C_o, W_o)
    S = spm.Sketch(800, r1, 8, 42)
    if prec == "fp64":
        Cm, W, _ = spm.nystrom(S, dev(K), r2, q)
        Ah = alg.nystrom_apply(host(Cm), host(W))
        assert np.linalg.norm(Ah - Ah_o) <= 1e-8 * np.linalg.norm(K)
    else:
        Cm, W, _ = spm.nystrom(S, dev(K, torch.float32), r2, q, precision=spm.PREC_MIXED)
        Ah = alg.nystrom_apply(host(Cm), host(W))
        assert np.linalg.norm(K - Ah) <= 1.01 * np.linalg.norm(K - Ah_o)


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("n,r1,r2,q,s", [(600, 120, 40, 1, 8), (1500, 300, 100, 2, 4), (333, 80, 80, 0, 8)])
def test_nystrom_eig_parity(spm, prec, n, r1, r2, q, s):
    """Algorithm 3 in factored form against the oracle's (same steps, FP64):
    A_hat = U diag(lam) U^T.  FP64: |A_hat - A_hat_o| <= 1e-9 |A|; mixed and FP32:
    the approximation error within 1% of the oracle's; lam >= 0 descending, U
    orthonormal."""
    rng = np.random.default_rng(n + r2)
    X = rng.standard_normal((n, 6))
    D2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    A = np.exp(-D2 / (2.0 * np.median(D2)))           # a Gaussian kernel matrix (psd)
    So = osk.Sketch(n, r1, s, 42)
    U_o, lam_o = alg.nystrom_eig(A, So, osk.gaussian(r1, r2, 43), q)
    Ah_o = (U_o * lam_o) @ U_o.T
    err_o = np.linalg.norm(A - Ah_o)
    p = {"fp64": spm.PREC_FP64, "mixed": spm.PREC_MIXED, "fp32": spm.PREC_FP32}[prec]
    dt = torch.float64 if prec == "fp64" else torch.float32
    S = spm.Sketch(n, r1, s, 42)
    U, lam, info = spm.nystrom_eig(S, dev(A, dt), r2, q, omega_seed=43, precision=p)
    assert info["device_status"] == 0
    U, lam = host(U), host(lam)
    Ah = (U * lam) @ U.T
    assert np.all(lam >= 0) and np.all(np.diff(lam) <= 1e-12 * lam[0])
    if prec == "fp64":
        assert np.linalg.norm(Ah - Ah_o) <= 1e-9 * np.linalg.norm(A)
        assert np.linalg.norm(U.T @ U - np.eye(r2)) <= 1e-10
        assert np.max(np.abs(lam - lam_o)) <= 1e-9 * lam_o[0]
    else:
        assert np.linalg.norm(A - Ah) <= 1.01 * err_o + 1e-5 * np.linalg.norm(A)
        assert np.linalg.norm(U.T @ U - np.eye(r2)) <= 1e-3
        assert np.max(np.abs(lam - lam_o)) <= 1e-4 * lam_o[0]


def test_invalid_arguments_are_rejected(spm):
    A = torch.zeros(10, 20, device="cuda", dtype=torch.float64)
    S = spm.Sketch(20, 8, 2, 1)
    with pytest.raises(spm.SpmError):
        spm.range_finder(S, A, 9, 1)          # r2 > r1
    with pytest.raises(spm.SpmError):
        spm.range_finder(S, A, 11, 1)         # r2 > m
    with pytest.raises(spm.SpmError):
        spm.rsvd(S, A, 4, 1, 5)               # k > r2
    S2 = spm.Sketch(21, 8, 2, 1)
    with pytest.raises(spm.SpmError):
        spm.range_finder(S2, A, 4, 1)         # sketch rows != columns of A


def test_rsvd_mixed_one_pass_power_residual(spm):
    """power_passes = 1 (plain BF16 power products): the residual bar still holds."""
    A, sigma = wl.noisy_exp_numpy(3000, 1500, seed=1002, noise=1e-3 / np.sqrt(1500))
    U_o, s_o, Vt_o, _ = _oracle_rsvd(A, 1500, 300, 8, 100, 2, 100)
    res_o = np.linalg.norm(A - (U_o * s_o) @ Vt_o)
    S = spm.Sketch(1500, 300, 8, 42)
    U, sg, Vt, _ = spm.rsvd(S, dev(A, torch.float32), 100, 2, 100, precision=spm.PREC_MIXED,
                            power_passes=1)
    res = np.linalg.norm(A - (host(U) * host(sg)) @ host(Vt))
    assert res <= 1.01 * res_o


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rank_deficient_input_deflates(spm, prec):
    """rank(A) = 5 < r2 = 12: CholeskyQR deflates the dependent columns, refills them at
    random, and still returns an orthonormal Q whose range contains range(A)."""
    A, _ = wl.dense_lowrank(600, 400, np.array([5.0, 4.0, 3.0, 2.0, 1.0]), seed=8)
    S = spm.Sketch(400, 48, 8, 42)
    p, dt, tol = (spm.PREC_FP64, torch.float64, 1e-11) if prec == "fp64" else \
        (spm.PREC_MIXED, torch.float32, 1e-4)
    Q, info = spm.range_finder(S, dev(A, dt), 12, 2, precision=p)
    Q = host(Q)
    assert np.linalg.norm(Q.T @ Q - np.eye(12)) <= (1e-10 if prec == "fp64" else 1e-3)
    assert alg.residual_fro(A, Q) <= tol * np.linalg.norm(A)
    assert info["device_status"] == 0


def test_rsvd_fp64_multi_cta_eigensolver(spm):
    """r2 = 300 runs the Jacobi eigensolver across many CTAs with grid barriers."""
    A, sigma = wl.plain_fp64(1200, 700, seed=17)
    U_o, s_o, Vt_o, _ = _oracle_rsvd(A, 700, 400, 8, 300, 1, 300)
    S = spm.Sketch(700, 400, 8, 42)
    U, sg, Vt, info = spm.rsvd(S, dev(A), 300, 1, 300)
    assert np.max(np.abs(host(sg) - s_o) / s_o) <= 1e-9
    res_o = np.linalg.norm(A - (U_o * s_o) @ Vt_o)
    res = np.linalg.norm(A - (host(U) * host(sg)) @ host(Vt))
    assert abs(res / res_o - 1) <= 1e-10
