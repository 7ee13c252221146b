"""Seeded synthetic inputs shaped like the paper's workloads.

This module builds test matrices only; it holds none of the method's arithmetic
(no sketching, no power iteration, no orthonormalisation of iterates).  Both the
CUDA path and the CPU oracle take their inputs from here.

Recipes (sizes and spectra follow the workloads this library is measured on;
the paper's own datasets, smallnorb and ImageNet, are not available, and its
synthetic ``polydecay`` matrix -- Section 4: diagonal 30000/i between random
orthogonal factors -- is the model for all dense cases):

  * ``dense_lowrank``: A = U diag(sigma) V^T with U, V Haar-distributed
    (QR of a seeded Gaussian matrix with the sign of diag(R) folded in).
  * ``plain_fp64``: 2000 x 1000, sigma_i = 1/i.
  * ``noisy_exp``: m x n, sigma_i = exp(-i/200) truncated where sigma < 1e-9,
    plus noise_scale * N(0,1) entries (default 1e-3, as the workload states).
  * ``sparse_planted``: CSR with `nnz_row` uniform distinct columns per row and
    N(0,1) values, plus a planted rank-p term U diag(100 i^-1/2) V^T kept as factors.
  * ``gmm_kernel``: Gaussian kernel exp(-|x_i - x_j|^2 / (2 h^2)) over points
    from an 8-component mixture in R^16 (means N(0, 3^2 I), unit covariance,
    equal weights), h = lower median of the pairwise distances.
  * ``batch_specs``: uneven batch, m in [512, 8192], n in [256, 4096]
    log-uniform, k in [16, 256], decay i^-alpha or exp(-i/tau).
  * ``polydecay_torch``: Section 4's synthetic matrix, 30000 x 15000 with
    sigma_i = 30000 / i between Haar factors, generated on the device.
"""
import math

import numpy as np


def load_torch_linalg():
    """Load torch's CUDA linear-algebra library by absolute path before the first
    device QR (its lazy load by name fails under some profilers' injection)."""
    import ctypes
    import os

    import torch
    path = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
    if os.path.exists(path):
        ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def haar(rows, cols, rng):
    """rows x cols matrix with orthonormal columns, Haar-distributed (Mezzadri 2007)."""
    G = rng.standard_normal((rows, cols))
    Q, R = np.linalg.qr(G, mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d


def dense_lowrank(m, n, sigma, seed, noise=0.0):
    """A = U diag(sigma) V^T (+ noise * N(0,1)); returns (A float64, sigma)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.size
    rng = _rng(seed)
    U = haar(m, r, rng)
    V = haar(n, r, rng)
    A = (U * sigma) @ V.T
    if noise:
        A = A + noise * rng.standard_normal((m, n))
    return A, sigma


def plain_fp64(m=2000, n=1000, seed=1001):
    """Dense A = U diag(1/i) V^T, the FP64 parity workload (k = 50 at full size)."""
    sigma = 1.0 / np.arange(1, min(m, n) + 1, dtype=np.float64)
    return dense_lowrank(m, n, sigma, seed)


def exp_decay_sigma(count, tau=200.0, floor=1e-9):
    i = np.arange(1, count + 1, dtype=np.float64)
    s = np.exp(-i / tau)
    return s[s >= floor]


def noisy_exp_numpy(m, n, seed=1002, noise=1e-3, tau=200.0):
    """Small-size version of the noisy exponential-decay workload (numpy, float64)."""
    sigma = exp_decay_sigma(min(m, n), tau)
    return dense_lowrank(m, n, sigma, seed, noise)


def noisy_exp_torch(m, n, seed=1002, noise=1e-3, tau=200.0, device="cuda", chunk=8192):
    """Full-size noisy exponential-decay matrix generated on the device (float32).

    U and V come from a float32 QR of seeded Gaussians on the device; A is built
    in row chunks so that no m x n float64 temporary exists.
    """
    import torch
    load_torch_linalg()
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    sigma = torch.tensor(exp_decay_sigma(min(m, n), tau), dtype=torch.float32, device=device)
    r = sigma.numel()
    U, Ru = torch.linalg.qr(torch.randn(m, r, generator=g, device=device, dtype=torch.float32))
    U *= torch.sign(torch.diagonal(Ru))
    V, Rv = torch.linalg.qr(torch.randn(n, r, generator=g, device=device, dtype=torch.float32))
    V *= torch.sign(torch.diagonal(Rv))
    del Ru, Rv
    A = torch.empty(m, n, device=device, dtype=torch.float32)
    Vs = (V * sigma).t().contiguous()
    for i0 in range(0, m, chunk):
        i1 = min(m, i0 + chunk)
        A[i0:i1] = U[i0:i1] @ Vs
        if noise:
            A[i0:i1] += noise * torch.randn(i1 - i0, n, generator=g, device=device, dtype=torch.float32)
    del U, V, Vs
    return A, sigma.cpu().numpy().astype(np.float64)


def polydecay_torch(m=30000, n=15000, seed=1006, device="cuda", chunk=8192):
    """Section 4's polydecay matrix on the device (float32): sigma_i = m / i for
    i = 1..min(m, n) between Haar factors (float32 QR of seeded Gaussians, sign of
    diag(R) folded in).  Returns (A, sigma as float64 numpy)."""
    import torch
    if str(device).startswith("cuda"):
        load_torch_linalg()
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    r = min(m, n)
    sigma = torch.tensor(float(m) / np.arange(1, r + 1), dtype=torch.float32, device=device)
    U, Ru = torch.linalg.qr(torch.randn(m, r, generator=g, device=device, dtype=torch.float32))
    U *= torch.sign(torch.diagonal(Ru))
    V, Rv = torch.linalg.qr(torch.randn(n, r, generator=g, device=device, dtype=torch.float32))
    V *= torch.sign(torch.diagonal(Rv))
    del Ru, Rv
    A = torch.empty(m, n, device=device, dtype=torch.float32)
    Vs = (V * sigma).t().contiguous()
    for i0 in range(0, m, chunk):
        i1 = min(m, i0 + chunk)
        A[i0:i1] = U[i0:i1] @ Vs
    del U, V, Vs
    return A, sigma.cpu().numpy().astype(np.float64)


def psd_lowrank(n, sigma, seed):
    """Symmetric psd A = U diag(sigma) U^T with Haar U."""
    rng = _rng(seed)
    U = haar(n, len(sigma), rng)
    return (U * np.asarray(sigma)) @ U.T


def gmm_points(npts, dim=16, comps=8, seed=1004, mean_scale=3.0):
    rng = _rng(seed)
    means = mean_scale * rng.standard_normal((comps, dim))
    lab = rng.integers(0, comps, size=npts)
    return means[lab] + rng.standard_normal((npts, dim))


def lower_median_distance(X):
    """Lower median of the pairwise Euclidean distances over i < j."""
    X = np.asarray(X, dtype=np.float64)
    sq = np.sum(X * X, axis=1)
    D2 = sq[:, None] + sq[None, :] - 2.0 * (X @ X.T)
    iu = np.triu_indices(X.shape[0], 1)
    d = np.sqrt(np.maximum(D2[iu], 0.0))
    d.sort()
    return float(d[(d.size - 1) // 2])


def gmm_kernel(npts, dim=16, comps=8, seed=1004):
    """Gaussian kernel matrix over mixture points; returns (K float64, h, X)."""
    X = gmm_points(npts, dim, comps, seed)
    h = lower_median_distance(X)
    sq = np.sum(X * X, axis=1)
    D2 = np.maximum(sq[:, None] + sq[None, :] - 2.0 * (X @ X.T), 0.0)
    K = np.exp(-D2 / (2.0 * h * h))
    return 0.5 * (K + K.T), h, X


def sparse_planted(m, n, nnz_row, p, seed=1003, amp=100.0, factors=True):
    """CSR (indptr, indices, values) + planted factors U (m x p), sig (p), V (n x p).

    Each row holds `nnz_row` distinct uniform columns (ascending) with N(0, 1)
    values; the planted term is U diag(amp i^-1/2) V^T with Haar U, V (None for
    the factors when factors=False)."""
    rng = _rng(seed)
    cols = np.sort(rng.integers(0, n, size=(m, nnz_row)), axis=1)
    dup = np.nonzero((cols[:, 1:] == cols[:, :-1]).any(axis=1))[0]
    for i in dup:  # rare: redraw the row without replacement
        cols[i] = np.sort(rng.choice(n, nnz_row, replace=False))
    indices = cols.reshape(-1)
    indptr = np.arange(0, m * nnz_row + 1, nnz_row, dtype=np.int64)
    values = rng.standard_normal(m * nnz_row)
    if not factors:
        return indptr, indices, values, None, None, None
    U = haar(m, p, rng)
    V = haar(n, p, rng)
    sig = amp * np.arange(1, p + 1, dtype=np.float64) ** -0.5
    return indptr, indices, values, U, sig, V


def batch_specs(count=512, seed=1005):
    """Shapes, ranks and spectra of an uneven batch of dense problems."""
    rng = _rng(seed)
    specs = []
    for _ in range(count):
        m = int(round(math.exp(rng.uniform(math.log(512), math.log(8192)))))
        n = int(round(math.exp(rng.uniform(math.log(256), math.log(4096)))))
        k = int(rng.integers(16, 257))
        k = min(k, m, n)
        if rng.uniform() < 0.5:
            kind, par = "poly", float(rng.uniform(0.5, 2.0))
        else:
            kind, par = "exp", float(rng.uniform(10.0, 200.0))
        specs.append(dict(m=m, n=n, k=k, kind=kind, par=par, seed=int(rng.integers(1 << 31))))
    return specs


def batch_sigma(spec):
    i = np.arange(1, min(spec["m"], spec["n"]) + 1, dtype=np.float64)
    if spec["kind"] == "poly":
        return i ** -spec["par"]
    return np.exp(-i / spec["par"])
