"""Row-sharded Algorithm 1 and Randomized SVD finish: the exchange steps of the
data-parallel form, one block of A's rows per rank.

With A split by rows over the ranks (A = [A_0; A_1; ...]), every row-local step
stays local and the only data exchanged are small sums over the ranks:

  * A~ = A S and Y = A~ Omega: local (rows of A~ are rows of A times S);
  * the power step's A~^T Y = sum_r A~_r^T Y_r: one all-reduce of r1 x r2;
  * the re-orthonormalisation of Z (r1 x r2): replicated on every rank;
  * the re-orthonormalisation of the row-sharded Y (CholeskyQR2): one all-reduce
    of the r2 x r2 Gram per pass, R^{-1} applied locally;
  * B = Q^T A = sum_r Q_r^T A_r: one all-reduce of r2 x n;
  * the SVD of B: replicated; U_r = Q_r U~ local;
  * the sign convention (largest-magnitude entry of each column of U positive):
    one all-gather of each rank's per-column extreme entry.

The arithmetic of each local step is supplied by `ops` (an object with the methods
listed in `ShardOps`), so that the exchange logic is the same whatever runs the
local products; collectives go through torch.distributed on the ranks' group.
Each call of this library uses one GPU: a multi-GPU run of these steps is not
part of it, and the logic is exercised by world-size-2 gloo runs on the CPU.
"""
import torch
import torch.distributed as dist


class ShardOps:
    """Local arithmetic of one rank (arrays: torch tensors on one device)."""

    def sketch(self, A, S):            # A S: (m_r x n) -> (m_r x r1)
        raise NotImplementedError

    def orth(self, Z):                 # orthonormal basis of a replicated r1 x r2 matrix
        raise NotImplementedError

    def chol_upper(self, G):           # R upper-triangular with R^T R = G
        raise NotImplementedError

    def svd(self, B):                  # thin SVD of the replicated r2 x n matrix
        raise NotImplementedError


def _allreduce(x, group):
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)
    return x


def orth_rows(Y, ops, group=None, passes=2):
    """CholeskyQR of a row-sharded Y: per pass the Gram sum_r Y_r^T Y_r (one
    all-reduce), its Cholesky factor R (replicated), Y_r <- Y_r R^{-1} (local)."""
    for _ in range(passes):
        G = _allreduce(Y.T @ Y, group)
        R = ops.chol_upper(G)
        Y = torch.linalg.solve_triangular(R, Y, upper=True, left=False)
    return Y


def rsvd_row_sharded(A, S, Omega, q, k, ops, group=None):
    """Rank-k Randomized SVD of the row-sharded A (this rank's rows), Algorithm 1
    with Y and Z re-orthonormalised every step.  Returns (U_r, sigma, Vt): this
    rank's rows of U, and sigma, Vt replicated on every rank."""
    At = ops.sketch(A, S)
    Y = At @ Omega
    for _ in range(q):
        Y = orth_rows(Y, ops, group)
        Z = _allreduce(At.T @ Y, group)         # r1 x r2
        Z = ops.orth(Z)
        Y = At @ Z
    Q = orth_rows(Y, ops, group)
    B = _allreduce(Q.T @ A, group)              # r2 x n
    Ub, sig, Vt = ops.svd(B)
    U = Q @ Ub[:, :k]
    Vt = Vt[:k]
    # sign: the entry of largest magnitude of each column of U, over all ranks,
    # made positive (ties: the lowest rank)
    idx = torch.argmax(U.abs(), dim=0)
    ext = U[idx, torch.arange(U.shape[1])]
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        parts = [torch.empty_like(ext) for _ in range(dist.get_world_size(group))]
        dist.all_gather(parts, ext, group=group)
        allx = torch.stack(parts)                # ranks x k
        ext = allx[torch.argmax(allx.abs(), dim=0), torch.arange(allx.shape[1])]
    sg = torch.sign(ext)
    sg[sg == 0] = 1.0
    return U * sg, sig[:k], Vt * sg[:, None]
