"""Algorithm 3 on a Gaussian kernel matrix that is never formed.

spm_gauss_sketch generates K[i, j] = exp(-|x_i - x_j|^2 / (2 h^2)) inside the
product K S; spm_nystrom_gauss is the factored Nystrom approximation built on it.
Both against the oracle (the kernel formed by its definition in FP64, then the
oracle's K S and factored Nystrom).

Tolerances.  FP64: 1e-12 of the sum of |terms| of each output entry.  FP32: each
kernel value carries the base-2 exponential's relative error (about 2^-21) plus
the rounding of the squared distance times |exponent| (at most 2^-23 (1 + |t|)
relative, t = d2 / (2 h^2)); the terms are then summed in 32-bit fixed point
with 2^-F resolution (F = 22 for every case here: F is the largest value <= 22
with b_max 2^F / sqrt(s) <= 2^30), each term rounded once by at most 2^-23.
The test bound is 2^-20 (1 + t_max) times the sum of |terms| of the entry plus
b_c 2^-23 (b_c: entries of S in the column).
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
    return _spm


def _dev(x, dtype):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def _points(n, d, seed):
    if d == 16:
        return wl.gmm_points(n, 16, 8, seed=seed)
    return np.random.default_rng(seed).standard_normal((n, d))


# (n, d, r1, s): tiles of 32 rows with a ragged tail, d not a multiple of 4, one
# column, r1 past one FP32 column group (1705 accumulator rows) and past the FP64
# group (852), s = 1 and s not a multiple of 4
CASES = [(3000, 16, 300, 8), (1001, 3, 40, 1), (777, 32, 1500, 8), (100, 1, 20, 3),
         (600, 5, 2500, 4), (33, 7, 900, 5)]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n,d,r1,s", CASES)
def test_gauss_sketch_parity(spm, dtype, n, d, r1, s):
    X = _points(n, d, n + d)
    h = wl.lower_median_distance(X) if n <= 3000 else 1.0
    K = alg.gaussian_kernel(X, h)
    So = osk.Sketch(n, r1, s, 42)
    ref = osk.apply_right(K, So)
    absS = np.abs(So.dense())
    mag = K @ absS                               # sum of |terms| of each entry
    S = spm.Sketch(n, r1, s, 42)
    out = spm.gauss_sketch(S, _dev(X, dtype), h).double().cpu().numpy()
    err = np.abs(out - ref)
    if dtype == torch.float64:
        assert np.all(err <= 1e-12 * mag + 1e-300)
    else:
        b = np.count_nonzero(absS, axis=0)[None, :]
        assert int(b.max()) * 2.0 ** 22 / np.sqrt(s) <= 2.0 ** 30     # F = 22
        D2 = -2.0 * h * h * np.log(np.maximum(K, 1e-300))
        t_max = float(np.max(D2) / (2.0 * h * h))
        bound = 2.0 ** -20 * (1.0 + t_max) * mag + b * 2.0 ** -23
        assert np.all(err <= bound), float(np.max(err / bound))
        # integer accumulation: the same bits on every call
        out2 = spm.gauss_sketch(S, _dev(X, dtype), h).double().cpu().numpy()
        assert np.array_equal(out, out2)


def test_gauss_sketch_padded_rows_and_invalid_arguments(spm):
    n, d, r1, s = 500, 6, 64, 8
    X = np.random.default_rng(1).standard_normal((n, d + 3))
    Xd = _dev(X, torch.float64)[:, :d]           # ldx = d + 3
    S = spm.Sketch(n, r1, s, 7)
    out = spm.gauss_sketch(S, Xd, 1.5).cpu().numpy()
    ref = osk.apply_right(alg.gaussian_kernel(X[:, :d], 1.5), osk.Sketch(n, r1, s, 7))
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.sqrt(s) * n / r1 * 4
    with pytest.raises(spm.SpmError):
        spm.gauss_sketch(S, Xd, 0.0)             # h = 0
    with pytest.raises(spm.SpmError):
        spm.gauss_sketch(S, Xd, float("nan"))
    with pytest.raises(spm.SpmError):
        spm.gauss_sketch(S, _dev(np.zeros((n, 33)), torch.float64), 1.0)   # d > 32
    with pytest.raises(spm.SpmError):
        spm.gauss_sketch(spm.Sketch(n + 1, r1, s, 7), Xd, 1.0)             # S.n != n


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("n,d,r1,r2,q,s", [(2000, 16, 300, 100, 1, 8), (700, 3, 120, 40, 2, 4),
                                           (333, 6, 80, 80, 0, 8)])
def test_nystrom_gauss_parity(spm, prec, n, d, r1, r2, q, s):
    """The fused Nystrom against the oracle's factored Nystrom of the formed kernel:
    FP64 |K_hat - K_hat_o| <= 1e-9 |K|; mixed and FP32: the approximation error
    within 1% of the oracle's, lam within 1e-4 lam_1; U orthonormal."""
    X = _points(n, d, 7 * n + d)
    h = wl.lower_median_distance(X)
    K = alg.gaussian_kernel(X, h)
    So = osk.Sketch(n, r1, s, 42)
    U_o, lam_o = alg.nystrom_gauss(X, h, So, osk.gaussian(r1, r2, 43), q)
    err_o = np.linalg.norm(K - (U_o * lam_o) @ U_o.T)
    p = {"fp64": spm.PREC_FP64, "mixed": spm.PREC_MIXED, "fp32": spm.PREC_FP32}[prec]
    dt = torch.float64 if prec == "fp64" else torch.float32
    S = spm.Sketch(n, r1, s, 42)
    U, lam, info = spm.nystrom_gauss(S, _dev(X, dt), h, r2, q, omega_seed=43, precision=p)
    assert info["device_status"] == 0
    U, lam = U.double().cpu().numpy(), lam.double().cpu().numpy()
    Kh = (U * lam) @ U.T
    assert np.all(lam >= 0) and np.all(np.diff(lam) <= 1e-12 * lam[0])
    if prec == "fp64":
        assert np.linalg.norm(Kh - (U_o * lam_o) @ U_o.T) <= 1e-9 * np.linalg.norm(K)
        assert np.max(np.abs(lam - lam_o)) <= 1e-9 * lam_o[0]
        assert np.linalg.norm(U.T @ U - np.eye(r2)) <= 1e-10
    else:
        assert np.linalg.norm(K - Kh) <= 1.01 * err_o + 1e-5 * np.linalg.norm(K)
        assert np.max(np.abs(lam - lam_o)) <= 1e-4 * lam_o[0]
        assert np.linalg.norm(U.T @ U - np.eye(r2)) <= 1e-3


def test_nystrom_gauss_matches_nystrom_of_the_formed_kernel(spm):
    # FP64: the fused product and the formed-kernel path give the same factors
    n, d, r1, r2 = 1500, 16, 200, 60
    X = _points(n, d, 99)
    h = wl.lower_median_distance(X)
    S = spm.Sketch(n, r1, 8, 42)
    U1, l1, _ = spm.nystrom_gauss(S, _dev(X, torch.float64), h, r2, 1, precision=spm.PREC_FP64)
    K = _dev(alg.gaussian_kernel(X, h), torch.float64)
    U2, l2, _ = spm.nystrom_eig(S, K, r2, 1, precision=spm.PREC_FP64)
    assert torch.max(torch.abs(l1 - l2)) <= 1e-10 * l2[0]
    assert torch.linalg.norm((U1 * l1) @ U1.T - (U2 * l2) @ U2.T) <= 1e-9 * torch.linalg.norm(K)
