"""Row-sharded Algorithm 1 + Randomized SVD finish (paper_2605_09755_gb300.sharded)
over world-size-2 gloo ranks on the CPU, against the oracle's single-rank RandSVD.

Each rank holds an uneven block of A's rows; the local arithmetic (A S, QR, the
Cholesky factor, the SVD of B) is FP64 on the CPU, the sketch product taken from
the oracle.  The exchange logic under test: the all-reduces of A~^T Y, of the
CholeskyQR Gram and of Q^T A, and the all-gather behind the sign convention.
Bar: U (rows gathered in rank order), sigma and V^T equal the oracle's within
1e-10 (different orthonormalisation of the same spans: rounding only).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import algorithms as alg
from oracle import sketch as osk

M, N, R1, K, Q = 123, 90, 30, 8, 2
SPLIT = (70, 53)


class CpuOps:
    def sketch(self, A, S):
        return torch.from_numpy(osk.apply_right(A.numpy(), S))

    def orth(self, Z):
        return torch.linalg.qr(Z, mode="reduced")[0]

    def chol_upper(self, G):
        return torch.linalg.cholesky(G).T

    def svd(self, B):
        return torch.linalg.svd(B, full_matrices=False)


def _problem():
    rng = np.random.default_rng(5)
    Uo, _ = np.linalg.qr(rng.standard_normal((M, M)))
    Vo, _ = np.linalg.qr(rng.standard_normal((N, N)))
    sig = 0.8 ** np.arange(N)
    A = (Uo[:, :N] * sig) @ Vo.T
    return A, osk.Sketch(N, R1, 4, 42), osk.gaussian(R1, K, 43)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    from paper_2605_09755_gb300 import sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, S, Om = _problem()
        r0 = sum(SPLIT[:rank])
        A_r = torch.from_numpy(A[r0:r0 + SPLIT[rank]].copy())
        U, sg, Vt = sharded.rsvd_row_sharded(A_r, S, torch.from_numpy(Om), Q, K, CpuOps())
        out[rank] = (U.numpy(), sg.numpy(), Vt.numpy())
    finally:
        dist.destroy_process_group()


def test_row_sharded_rsvd_matches_single_rank_oracle():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    A, S, Om = _problem()
    U_o, s_o, Vt_o, _ = alg.rsvd(A, S, Om, Q, K)
    U = np.vstack([out[r][0] for r in range(world)])
    for r in range(world):
        assert np.allclose(out[r][1], s_o, rtol=0, atol=1e-10 * s_o[0])
        assert np.allclose(out[r][2], Vt_o, rtol=0, atol=1e-10)
    assert np.allclose(U, U_o, rtol=0, atol=1e-10)


def test_single_rank_without_a_process_group_is_the_same_arithmetic():
    from paper_2605_09755_gb300 import sharded
    A, S, Om = _problem()
    U, sg, Vt = sharded.rsvd_row_sharded(torch.from_numpy(A), S, torch.from_numpy(Om), Q, K,
                                         CpuOps())
    U_o, s_o, Vt_o, _ = alg.rsvd(A, S, Om, Q, K)
    assert np.allclose(U.numpy(), U_o, rtol=0, atol=1e-10)
    assert np.allclose(sg.numpy(), s_o, rtol=0, atol=1e-10 * s_o[0])
    assert np.allclose(Vt.numpy(), Vt_o, rtol=0, atol=1e-10)

