"""Dense sign (Lemma 3.2 item 1) and SRHT (Lemma 3.2 item 3) sketches through the C ABI.

Expected values come from the oracle (``oracle/sketch.py``: S written out from
its definition, A S as a dense product).  Tolerances follow the arithmetic, per
row i of A S (every entry has magnitude about ||A_i||_2 / sqrt(r1)):
  * dense sign, a length-n dot product of A_i with +-1 entries: |error| <=
    n u ||A_i||_2 / sqrt(r1) (u = 2^-53 for FP64, 2^-24 for FP32);
  * SRHT, L = log2 n' butterfly stages, each adding at most u times a partial
    sum of size <= sqrt(n') ||A_i||_2: |error| <= 2 L u sqrt(n') ||A_i||_2 / sqrt(r1).
A wrong sign, index or scale gives errors of the size of the entries themselves.
RandSVD with these sketches: the same bounds as the sparse sign sketch's parity
tests (FP64 residual and sigma within 1e-10 of the oracle's; mixed residual
<= 1.01x, sigma within 1e-4).
"""
import numpy as np
import pytest
import torch

from oracle import algorithms as alg
from oracle import sketch as osk
from paper_2605_09755_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

KINDS = [osk.DENSE_SIGN, osk.SRHT]


@pytest.fixture(scope="module")
def spm():
    from paper_2605_09755_gb300 import _build, spm as _spm
    _build.build()
    _spm.lib()
    assert (_spm.DENSE_SIGN, _spm.SRHT) == (osk.DENSE_SIGN, osk.SRHT)
    return _spm


def dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def _row_bound(A, kind, n, r1, u):
    rn = np.linalg.norm(A, axis=1)
    if kind == osk.DENSE_SIGN:
        f = n
    else:
        L = osk.hadamard_order(n)
        f = 2 * max(L, 1) * np.sqrt(1 << L)
    return f * u * rn / np.sqrt(r1) + 1e-300


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype,u", [(torch.float64, 2.0 ** -53), (torch.float32, 2.0 ** -24)])
@pytest.mark.parametrize("m,n,r1", [(300, 700, 140), (257, 1024, 1024), (64, 40, 9), (33, 3, 2),
                                    (1, 1, 1), (700, 16384, 500), (91, 8193, 77)])
def test_apply_matches_oracle(spm, kind, dtype, u, m, n, r1):
    """Ragged rows (several rows per CTA for short rows), n' from 1 to 2^14, r1 = n."""
    rng = np.random.default_rng(m + n + r1)
    A = rng.standard_normal((m, n))
    if dtype == torch.float32:
        A = A.astype(np.float32).astype(np.float64)
    S = spm.Sketch(n, r1, 1, 42, kind=kind)
    got = host(spm.sketch_apply(S, dev(A, dtype)))
    ref = osk.apply_right(A, osk.Sketch(n, r1, 1, 42, kind=kind))
    err = np.max(np.abs(got - ref), axis=1)
    assert np.all(err <= _row_bound(A, kind, n, r1, u)), np.max(err / _row_bound(A, kind, n, r1, u))


@pytest.mark.parametrize("dtype,u", [(torch.float32, 2.0 ** -24)])
def test_srht_apply_largest_order(spm, dtype, u):
    """n' = 2^15 (four 32-element groups per thread); FP64 needs n' <= 2^14."""
    m, n, r1 = 50, 20000, 300
    A = np.random.default_rng(1).standard_normal((m, n)).astype(np.float32).astype(np.float64)
    S = spm.Sketch(n, r1, 1, 7, kind=spm.SRHT)
    got = host(spm.sketch_apply(S, dev(A, dtype)))
    ref = osk.apply_right(A, osk.Sketch(n, r1, 1, 7, kind=osk.SRHT))
    assert np.all(np.max(np.abs(got - ref), axis=1) <= _row_bound(A, osk.SRHT, n, r1, u))
    with pytest.raises(spm.SpmError) as ei:
        spm.sketch_apply(S, dev(A))
    assert ei.value.code == spm.EUNSUPPORTED


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype,u", [(torch.float64, 2.0 ** -53), (torch.float32, 2.0 ** -24)])
@pytest.mark.parametrize("n,p,r1", [(700, 33, 140), (1024, 5, 64), (40, 17, 40)])
def test_apply_t_matches_oracle(spm, kind, dtype, u, n, p, r1):
    X = np.random.default_rng(n + p).standard_normal((n, p))
    if dtype == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
    S = spm.Sketch(n, r1, 1, 5, kind=kind)
    got = host(spm.sketch_apply_t(S, dev(X, dtype)))
    ref = osk.apply_left_t(osk.Sketch(n, r1, 1, 5, kind=kind), X)
    bound = _row_bound(X.T, kind, n, r1, u)           # column j of S^T X is row j of X^T S
    assert np.all(np.max(np.abs(got - ref), axis=0) <= bound)


def _oracle_rsvd(A, n, r1, r2, q, k, kind):
    return alg.rsvd(A, osk.Sketch(n, r1, 1, 42, kind=kind), osk.gaussian(r1, r2, 43), q, k)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("m,n,r1,r2,q", [(2000, 1000, 100, 50, 2), (777, 513, 130, 40, 1),
                                         (300, 200, 60, 60, 0)])
def test_rsvd_fp64_matches_oracle(spm, kind, m, n, r1, r2, q):
    A, sigma = wl.plain_fp64(m, n, seed=1001)
    U_o, s_o, Vt_o, _ = _oracle_rsvd(A, n, r1, r2, q, r2, kind)
    res_o = np.linalg.norm(A - (U_o * s_o) @ Vt_o)
    S = spm.Sketch(n, r1, 1, 42, kind=kind)
    U, sg, Vt, info = spm.rsvd(S, dev(A), r2, q, r2, omega_seed=43, precision=spm.PREC_FP64)
    U, sg, Vt = host(U), host(sg), host(Vt)
    res = np.linalg.norm(A - (U * sg) @ Vt)
    assert abs(res - res_o) <= 1e-10 * res_o
    assert np.max(np.abs(sg - s_o) / s_o) <= 1e-10
    assert np.linalg.norm(U.T @ U - np.eye(r2)) <= 1e-12
    assert info["device_status"] == 0


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("m,n,r1,r2,q", [(4096, 2048, 256, 128, 2), (2000, 1000, 100, 50, 2)])
def test_rsvd_mixed_matches_oracle(spm, kind, m, n, r1, r2, q):
    """Mixed precision: the dense sign product on the tensor cores (A as two BF16
    parts, +-1 exact), the SRHT in FP32 with a hi/lo BF16 result."""
    if m == 2000:
        A, _ = wl.plain_fp64(m, n, seed=1001)
    else:
        A, _ = wl.noisy_exp_numpy(m, n, seed=1002, noise=1e-3 / np.sqrt(n))
    A = A.astype(np.float32).astype(np.float64)
    U_o, s_o, Vt_o, _ = _oracle_rsvd(A, n, r1, r2, q, r2, kind)
    res_o = np.linalg.norm(A - (U_o * s_o) @ Vt_o)
    S = spm.Sketch(n, r1, 1, 42, kind=kind)
    U, sg, Vt, info = spm.rsvd(S, dev(A, torch.float32), r2, q, r2, precision=spm.PREC_MIXED)
    U, sg, Vt = host(U), host(sg), host(Vt)
    res = np.linalg.norm(A - (U * sg) @ Vt)
    assert res <= 1.01 * res_o, (res, res_o)
    assert np.max(np.abs(sg - s_o) / s_o) <= 1e-4
    assert np.linalg.norm(U.T @ U - np.eye(r2)) <= 1e-3
    assert info["device_status"] == 0


@pytest.mark.parametrize("kind", KINDS)
def test_nystrom_and_lowrank_with_dense_sketches(spm, kind):
    """Algorithm 3 (A S and S^T (A S)) and Algorithm 2 (S2^T Q, S2^T A) with the
    dense families, FP64, against the oracle (the sparse sign tests' bounds)."""
    K, h, X = wl.gmm_kernel(800, seed=1004)
    r1, r2, q = 200, 50, 1
    C_o, W_o = alg.nystrom(K, osk.Sketch(800, r1, 1, 42, kind=kind), osk.gaussian(r1, r2, 43), q)
    Ah_o = alg.nystrom_apply(C_o, W_o)
    Cm, W, _ = spm.nystrom(spm.Sketch(800, r1, 1, 42, kind=kind), dev(K), r2, q)
    Ah = alg.nystrom_apply(host(Cm), host(W))
    assert np.linalg.norm(Ah - Ah_o) <= 1e-8 * np.linalg.norm(K)

    m, n, r1, r2, q = 900, 600, 120, 30, 2
    A, _ = wl.plain_fp64(m, n, seed=21)
    S1o, S2o = osk.Sketch(n, r1, 1, 42, kind=kind), osk.Sketch(m, r1, 1, 44, kind=kind)
    Y_o, X_o = alg.lowrank(A, S1o, S2o, osk.gaussian(r1, r2, 43), q)
    S1, S2 = spm.Sketch(n, r1, 1, 42, kind=kind), spm.Sketch(m, r1, 1, 44, kind=kind)
    Y, Xg, _ = spm.lowrank(S1, S2, dev(A), r2, q)
    assert np.linalg.norm(host(Y) @ host(Xg) - Y_o @ X_o) <= 1e-9 * np.linalg.norm(A)


def test_dense_kinds_argument_errors(spm):
    with pytest.raises(spm.SpmError) as ei:
        spm.Sketch(100, 101, 1, 1, kind=spm.SRHT)               # r1 > n
    assert ei.value.code == spm.EINVAL
    with pytest.raises(spm.SpmError) as ei:
        spm.Sketch(40000, 100, 1, 1, kind=spm.SRHT)             # n' = 2^16
    assert ei.value.code == spm.EUNSUPPORTED
    with pytest.raises(spm.SpmError) as ei:
        spm.Sketch(100, 10, 1, 1, kind=4)
    assert ei.value.code == spm.EINVAL
    for kind in KINDS:
        S = spm.Sketch(100, 10, 1, 1, kind=kind)
        with pytest.raises(spm.SpmError) as ei:
            S.tables()
        assert ei.value.code == spm.EUNSUPPORTED
        indptr, indices, values, _, _, _ = wl.sparse_planted(50, 100, 3, 0, seed=2, factors=False)
        Acsr = spm.CsrMatrix(torch.tensor(indptr, device="cuda"),
                             torch.tensor(indices, dtype=torch.int32, device="cuda"),
                             torch.tensor(values, dtype=torch.float64, device="cuda"), 100)
        with pytest.raises(spm.SpmError) as ei:
            spm.sketch_apply_csr(S, Acsr)
        assert ei.value.code == spm.EUNSUPPORTED
