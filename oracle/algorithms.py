"""Plain FP64 statements of Algorithms 1-3 and the Randomized SVD finish.

TEST INFRASTRUCTURE ONLY: imported by tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the product path.  Shares no code with
the CUDA library.

Each function follows the paper's steps in order, with numpy/LAPACK primitives
(matrix product, Householder QR, SVD, symmetric eigendecomposition) as steps:

  * range_finder  -- Algorithm 1 (Sketch-Powered Range Finder), with the
    intermediate re-orthonormalisation that Section 2 ("Comparison with Classical
    Range Finder") says is done after each power step in practice and does not
    change the output in exact arithmetic.  orth() is Householder thin QR.
  * rsvd          -- Section 2 "Sketch-Powered Low-Rank Factorization", first
    paragraph: B = Q^T A, SVD of B = U~ Sigma V^T, U = Q U~.
  * lowrank       -- Algorithm 2: X = (S2^T Y)^+ (S2^T A).  The product Y X is
    unchanged when Y is replaced by Q = Y R^{-1} (R invertible), so Q is used.
  * nystrom       -- Algorithm 3: C~ = A S, W~ = S^T A S, Y = W~^q Omega,
    C = C~ Y, W = Y^T W~ Y; A_hat = C W^+ C^T.  Re-orthonormalising Y between
    the q products changes Y by an invertible right factor, which leaves
    C W^+ C^T unchanged (Section 3, proof of Theorem 2.3).
  * nystrom_eig   -- the same approximation in factored form A_hat = U diag(lam) U^T,
    computed stably: with the test matrix T = S Y (so that C = A T and
    W = T^T A T), the Nystrom approximation of A + nu I is formed instead
    (C_nu = C + nu T, W_nu = T^T C_nu, positive definite), as
    F = C_nu L^{-T} with L L^T = W_nu, then F = U Sigma V^T and
    lam = max(Sigma^2 - nu, 0).  The paper leaves W^+ unspecified; the shift
    nu = sqrt(n) * 2^-52 * |C|_F is the reading used for the stable factored
    output (the shifted Nystrom approximation of Tropp, Yurtsever, Udell and
    Cevher, 2017).

Readings (listed in the design notes): r2 = k; W^+ drops eigenvalues at or below
r2 * eps * lambda_max; singular vectors are sign-fixed so that the entry of
largest magnitude of each left vector is positive.
"""
import numpy as np

from .sketch import apply_right, apply_left_t, apply_left


def orth(Y):
    """Orthonormal basis of range(Y) (notation paragraph of Section 1): Householder QR."""
    Q, _ = np.linalg.qr(np.asarray(Y, dtype=np.float64), mode="reduced")
    return Q


def sketched_power(At, Omega, q, reorth=True):
    """Y = (A~ A~^T)^q A~ Omega (Algorithm 1 line 1), re-orthonormalised per step."""
    Y = At @ Omega
    for _ in range(q):
        if reorth:
            Y = orth(Y)
        Z = At.T @ Y
        if reorth:
            Z = orth(Z)
        Y = At @ Z
    return Y


def range_finder(A, S, Omega, q, reorth=True, return_sketch=False):
    """Algorithm 1: Q = orth((A~ A~^T)^q A~ Omega) with A~ = A S."""
    A = np.asarray(A, dtype=np.float64)
    At = apply_right(A, S)
    Q = orth(sketched_power(At, np.asarray(Omega, dtype=np.float64), q, reorth))
    return (Q, At) if return_sketch else Q


def sign_fix(U, Vt=None):
    """Make the largest-magnitude entry of each column of U positive (flip Vt rows too)."""
    idx = np.argmax(np.abs(U), axis=0)
    sg = np.sign(U[idx, np.arange(U.shape[1])])
    sg[sg == 0] = 1.0
    U = U * sg
    if Vt is not None:
        Vt = Vt * sg[:, None]
    return U, Vt


def rsvd(A, S, Omega, q, k, reorth=True):
    """Randomized SVD on the Algorithm 1 range finder: returns U (m x k), sigma (k), Vt (k x n), Q."""
    A = np.asarray(A, dtype=np.float64)
    Q = range_finder(A, S, Omega, q, reorth)
    B = Q.T @ A
    Ub, sig, Vt = np.linalg.svd(B, full_matrices=False)
    U = Q @ Ub
    U, Vt = sign_fix(U[:, :k], Vt[:k])
    return U, sig[:k], Vt, Q


def lowrank(A, S1, S2, Omega, q, reorth=True):
    """Algorithm 2: Y (m x r2), X (r2 x n) with A ~ Y X; X = (S2^T Y)^+ (S2^T A)."""
    A = np.asarray(A, dtype=np.float64)
    Y = range_finder(A, S1, Omega, q, reorth)
    M = apply_left_t(S2, Y)          # S2^T Y, r1' x r2
    N = apply_left_t(S2, A)          # S2^T A, r1' x n
    X, *_ = np.linalg.lstsq(M, N, rcond=None)   # minimum-norm solution = M^+ N
    return Y, X


def psd_pinv(W):
    """Pseudo-inverse of a symmetric psd matrix via its eigendecomposition."""
    W = 0.5 * (W + W.T)
    lam, V = np.linalg.eigh(W)
    tol = W.shape[0] * np.finfo(np.float64).eps * max(lam.max(), 0.0)
    inv = np.where(lam > tol, 1.0 / np.where(lam > tol, lam, 1.0), 0.0)
    return (V * inv) @ V.T


def nystrom(A, S, Omega, q, reorth=True):
    """Algorithm 3: returns C (n x r2), W (r2 x r2) with A_hat = C W^+ C^T."""
    A = np.asarray(A, dtype=np.float64)
    Ct = apply_right(A, S)                 # C~ = A S
    Wt = apply_left_t(S, Ct)               # W~ = S^T A S
    Wt = 0.5 * (Wt + Wt.T)
    Y = np.asarray(Omega, dtype=np.float64)
    for _ in range(q):
        Y = Wt @ Y                         # Y = W~^q Omega
        if reorth:
            Y = orth(Y)
    C = Ct @ Y
    W = Y.T @ Wt @ Y
    return C, 0.5 * (W + W.T)


def nystrom_eig(A, S, Omega, q, reorth=True):
    """Algorithm 3 in factored form: (U, lam) with A_hat = U diag(lam) U^T, U
    orthonormal (n x r2), lam descending and >= 0 (see the module notes)."""
    import scipy.linalg
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    Ct = apply_right(A, S)                 # C~ = A S
    Wt = apply_left_t(S, Ct)               # W~ = S^T A S
    Wt = 0.5 * (Wt + Wt.T)
    Y = np.asarray(Omega, dtype=np.float64)
    for _ in range(q):
        Y = Wt @ Y                         # Y = W~^q Omega
        if reorth:
            Y = orth(Y)
    T = apply_left(S, Y)                   # test matrix: C = A T
    C = Ct @ Y
    nu = np.sqrt(n) * 2.0 ** -52 * np.linalg.norm(C)
    Cn = C + nu * T                        # (A + nu I) T
    Wn = T.T @ Cn                          # T^T (A + nu I) T
    Wn = 0.5 * (Wn + Wn.T)
    L = np.linalg.cholesky(Wn)
    F = scipy.linalg.solve_triangular(L, Cn.T, lower=True).T   # C_nu L^{-T}
    U, sig, _ = np.linalg.svd(F, full_matrices=False)
    lam = np.maximum(sig ** 2 - nu, 0.0)
    U, _ = sign_fix(U)
    return U, lam


def gaussian_kernel(X, h):
    """The Gaussian kernel matrix K[i, j] = exp(-|x_i - x_j|^2 / (2 h^2)) of the
    rows of X (Section 5's kernel experiments), by its definition: squared
    distances as sums of squared coordinate differences, in FP64."""
    X = np.asarray(X, dtype=np.float64)
    D2 = np.zeros((X.shape[0], X.shape[0]))
    for k in range(X.shape[1]):
        diff = X[:, k][:, None] - X[:, k][None, :]
        D2 += diff * diff
    return np.exp(-D2 / (2.0 * h * h))


def nystrom_gauss(X, h, S, Omega, q, reorth=True):
    """Algorithm 3 in factored form on the Gaussian kernel matrix of the rows of X."""
    return nystrom_eig(gaussian_kernel(X, h), S, Omega, q, reorth)


def nystrom_apply(C, W):
    """A_hat = C W^+ C^T."""
    return C @ psd_pinv(W) @ C.T


def residual_fro(A, Q):
    """||A - Q Q^T A||_F, formed directly (no norm subtraction)."""
    A = np.asarray(A, dtype=np.float64)
    return float(np.linalg.norm(A - Q @ (Q.T @ A)))


def residual_spec(A, Q):
    """||A - Q Q^T A||_2 by a dense SVD (small inputs)."""
    A = np.asarray(A, dtype=np.float64)
    return float(np.linalg.norm(A - Q @ (Q.T @ A), 2))


def optimal_fro(sigma, k):
    """Eckart-Young: min over rank-k of ||A - A_k||_F = sqrt(sum_{i>k} sigma_i^2)."""
    sigma = np.sort(np.asarray(sigma, dtype=np.float64))[::-1]
    return float(np.sqrt(np.sum(sigma[k:] ** 2)))
