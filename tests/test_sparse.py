"""Sparse input A = A_csr + U diag(sig) V^T (spm_sketch_apply_csr, spm_rsvd_csr).

Parity against the oracle on the densified matrix at sizes the oracle handles;
at the 10^6 x 2*10^5 workload (20 non-zeros per row, planted rank 200), sampled
rows of A S against the oracle's row-by-row product and properties of the
factors that hold at any size.
"""
import numpy as np
import pytest
import scipy.sparse as sp
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


def _csr(spm, m, n, nnz_row, p, dtype, seed):
    indptr, indices, values, U, sig, V = wl.sparse_planted(m, n, nnz_row, p, seed=seed,
                                                           factors=p > 0)
    dense = sp.csr_matrix((values, indices, indptr), shape=(m, n)).toarray()
    kw = {}
    if p > 0:
        dense = dense + (U * sig) @ V.T
        kw = dict(U=torch.tensor(U, dtype=dtype, device="cuda"),
                  sig=torch.tensor(sig, dtype=dtype, device="cuda"),
                  V=torch.tensor(V, dtype=dtype, device="cuda"))
    A = spm.CsrMatrix(torch.tensor(indptr, device="cuda"),
                      torch.tensor(indices, dtype=torch.int32, device="cuda"),
                      torch.tensor(values, dtype=dtype, device="cuda"), n, **kw)
    return A, dense


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-6)])
@pytest.mark.parametrize("m,n,nnz_row,p,r1,s", [(1500, 700, 20, 0, 140, 8), (1500, 700, 20, 15, 140, 8),
                                                (301, 513, 7, 4, 1025, 3), (64, 40, 3, 2, 40, 1)])
def test_csr_sketch_matches_oracle(spm, dtype, tol, m, n, nnz_row, p, r1, s):
    A, dense = _csr(spm, m, n, nnz_row, p, dtype, seed=5)
    got = spm.sketch_apply_csr(spm.Sketch(n, r1, s, 42), A).double().cpu().numpy()
    ref = osk.apply_right(dense, osk.Sketch(n, r1, s, 42))
    assert np.max(np.abs(got - ref)) <= tol * max(1.0, np.abs(ref).max())


def test_csr_sketch_identity(spm):
    A, dense = _csr(spm, 200, 90, 6, 3, torch.float64, seed=6)
    S = spm.Sketch(90, 90, 1, 0, kind=spm.IDENTITY)
    got = spm.sketch_apply_csr(S, A).cpu().numpy()
    assert np.max(np.abs(got - dense)) <= 1e-12 * np.abs(dense).max()


def _oracle(dense, n, r1, s, r2, q, k):
    return alg.rsvd(dense, osk.Sketch(n, r1, s, 42), osk.gaussian(r1, r2, 43), q, k)


def test_rsvd_csr_fp64_matches_oracle(spm):
    m, n, r1, r2, q = 2000, 900, 120, 60, 2
    A, dense = _csr(spm, m, n, 20, 30, torch.float64, seed=7)
    U_o, s_o, Vt_o, _ = _oracle(dense, n, r1, 8, r2, q, r2)
    U, sg, Vt, info = spm.rsvd_csr(spm.Sketch(n, r1, 8, 42), A, r2, q, r2, precision=spm.PREC_FP64)
    U, sg, Vt = U.cpu().numpy(), sg.cpu().numpy(), Vt.cpu().numpy()
    res_o = np.linalg.norm(dense - (U_o * s_o) @ Vt_o)
    res = np.linalg.norm(dense - (U * sg) @ Vt)
    assert abs(res - res_o) <= 1e-10 * res_o
    assert np.max(np.abs(sg - s_o) / s_o) <= 1e-10
    assert info["device_status"] == 0 and info["fro_a"] == -1.0


def test_rsvd_csr_mixed_matches_oracle(spm):
    m, n, r1, r2, q = 3000, 1200, 160, 40, 2
    A, dense = _csr(spm, m, n, 20, 30, torch.float32, seed=8)
    dense = dense.astype(np.float32).astype(np.float64)
    U_o, s_o, Vt_o, _ = _oracle(dense, n, r1, 8, r2, q, r2)
    U, sg, Vt, info = spm.rsvd_csr(spm.Sketch(n, r1, 8, 42), A, r2, q, r2, precision=spm.PREC_MIXED)
    U, sg, Vt = (t.double().cpu().numpy() for t in (U, sg, Vt))
    res_o = np.linalg.norm(dense - (U_o * s_o) @ Vt_o)
    res = np.linalg.norm(dense - (U * sg) @ Vt)
    assert res <= 1.01 * res_o, (res, res_o)
    assert np.max(np.abs(sg - s_o) / s_o) <= 1e-4
    assert np.linalg.norm(U.T @ U - np.eye(r2)) <= 1e-3
    assert info["device_status"] == 0


def test_csr_bad_column_reported(spm):
    """An out-of-range column index is skipped by the kernels (bounds-checked)
    and reported as device status SPM_EINVAL."""
    m, n = 300, 200
    indptr, indices, values, _, _, _ = wl.sparse_planted(m, n, 5, 0, seed=9, factors=False)
    indices = indices.copy()
    indices[17] = n
    A = spm.CsrMatrix(torch.tensor(indptr, device="cuda"),
                      torch.tensor(indices, dtype=torch.int32, device="cuda"),
                      torch.tensor(values, dtype=torch.float64, device="cuda"), n)
    with pytest.raises(spm.SpmError) as ei:
        spm.rsvd_csr(spm.Sketch(n, 40, 8, 42), A, 20, 1, 20, precision=spm.PREC_FP64)
    assert ei.value.code == spm.EINVAL


def test_rsvd_csr_full_size_sampled(spm):
    """10^6 x 2*10^5, 20 non-zeros per row, planted rank 200 (sigma_i = 100 i^-1/2),
    r1 = 400, k = 200, q = 2: sampled rows of A S against the oracle's row-by-row
    product, then the mixed-precision run against the FP64 run of the same path
    (itself pinned to the oracle at small sizes above).  (At this size the sparse
    part's Frobenius mass, folded by S into r1 directions of ~4472 / 20 ~ 224 each,
    outweighs the planted sigma_1 = 100, so the rank-k factors follow the sketched
    noise; both precisions must agree on them.)"""
    m, n, p, r1, k = 1_000_000, 200_000, 200, 400, 200
    indptr, indices, values, U, sig, V = wl.sparse_planted(m, n, 20, p, seed=1003)
    values = values.astype(np.float32).astype(np.float64)
    U, sig, V = (x.astype(np.float32).astype(np.float64) for x in (U, sig, V))

    def dev_csr(dtype):
        t = lambda x: torch.tensor(x, dtype=dtype, device="cuda")
        return spm.CsrMatrix(torch.tensor(indptr, device="cuda"),
                             torch.tensor(indices, dtype=torch.int32, device="cuda"), t(values), n,
                             U=t(U), sig=t(sig), V=t(V))

    S = spm.Sketch(n, r1, 8, 42)
    A32 = dev_csr(torch.float32)
    At = spm.sketch_apply_csr(S, A32).double().cpu().numpy()
    So = osk.Sketch(n, r1, 8, 42)
    SV = osk.apply_left_t(So, V)     # r1 x p
    rng = np.random.default_rng(11)
    Sd = So.sparse()
    for i in rng.choice(m, 64, replace=False):
        e0, e1 = indptr[i], indptr[i + 1]
        row = np.asarray(Sd[indices[e0:e1]].T @ values[e0:e1]).ravel() + (U[i] * sig) @ SV.T
        assert np.max(np.abs(At[i] - row)) <= 1e-4 * max(1.0, np.abs(row).max()), i
    del At
    Um, sm, Vm, im = spm.rsvd_csr(S, A32, k, 2, k, precision=spm.PREC_MIXED)
    Ud, sd, Vd, idd = spm.rsvd_csr(S, dev_csr(torch.float64), k, 2, k, precision=spm.PREC_FP64)
    torch.cuda.synchronize()
    assert im["device_status"] == 0 and idd["device_status"] == 0
    sm, sd = sm.double(), sd
    assert torch.all(sm[:-1] >= sm[1:]) and sm[-1] > 0
    assert float(torch.max(torch.abs(sm - sd) / sd)) <= 1e-4
    # single-precision inner products over m = 10^6 rows: ~u32 sqrt(m) per entry,
    # so ||U^T U - I||_F ~ k u32 sqrt(m) = 200 * 6e-8 * 1e3 = 1.2e-2 (observed 2.6e-3)
    eye = torch.eye(k, device="cuda", dtype=torch.float64)
    assert float(torch.linalg.norm(Um.double().T @ Um.double() - eye)) <= 1.2e-2
    assert float(torch.linalg.norm(Vm.double() @ Vm.double().T - eye)) <= 1.2e-2
