"""Pins of the CPU oracle to facts outside itself (no GPU).

Each test ties an oracle function to something it does not compute itself:
published known-answer vectors, brute force on tiny inputs, closed forms,
library routines on special cases, or exact identities the paper states.
"""
import os

import numpy as np
import pytest
import scipy.special
import scipy.stats

from oracle import algorithms as alg
from oracle import sketch as sk
from oracle.philox import philox4x32_10
from paper_2605_09755_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- generator
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (SC'11 / Random123)."""
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = philox4x32_10(*r[:6])
        assert [int(w) for w in out] == r[6:]


def test_philox_vectorised_matches_scalar():
    c = np.arange(37, dtype=np.uint64) * np.uint64(2654435761) & np.uint64(0xFFFFFFFF)
    vec = philox4x32_10(c, 7, 11, 13, 5, 9)
    for i in [0, 5, 36]:
        sc = philox4x32_10(int(c[i]), 7, 11, 13, 5, 9)
        assert [int(v[i]) for v in vec] == [int(s) for s in sc]


# ---------------------------------------------------------------- sketch (Lemma 3.2 item 2)
@pytest.mark.parametrize("n,r1,s", [(500, 40, 8), (300, 8, 8), (1000, 100, 1), (64, 64, 3)])
def test_sketch_rows_have_s_distinct_columns(n, r1, s):
    cols, signs = sk.sketch_entries(n, r1, s, seed=42)
    assert cols.shape == (n, s) and signs.shape == (n, s)
    assert cols.min() >= 0 and cols.max() < r1
    for j in range(n):
        assert len(set(cols[j].tolist())) == s
    assert set(np.unique(signs).tolist()) <= {-1, 1}
    S = sk.Sketch(n, r1, s, 42)
    D = S.dense()
    # each row: exactly s non-zeros of magnitude 1/sqrt(s)
    nz = np.count_nonzero(D, axis=1)
    assert np.all(nz == s)
    assert np.allclose(np.abs(D[D != 0]), 1.0 / np.sqrt(s))
    ptr, rows, sg = S.buckets()
    assert ptr[-1] == n * s
    for c in range(r1):
        rr = rows[ptr[c]:ptr[c + 1]]
        assert np.all(np.diff(rr) > 0)           # ascending row order inside a bucket
        assert np.allclose(D[rr, c], sg[ptr[c]:ptr[c + 1]] / np.sqrt(s))


def test_sketch_column_and_sign_distribution():
    """Columns uniform over [0, r1) and signs fair (chi-square / binomial, s = 1)."""
    n, r1 = 200000, 50
    cols, signs = sk.sketch_entries(n, r1, 1, seed=7)
    counts = np.bincount(cols[:, 0], minlength=r1)
    stat, p = scipy.stats.chisquare(counts)
    assert p > 1e-4
    plus = int((signs == 1).sum())
    assert abs(plus - n / 2) < 5 * np.sqrt(n / 4)


def test_sketch_seed_changes_draws_and_is_reproducible():
    a = sk.sketch_entries(300, 30, 4, seed=1)
    b = sk.sketch_entries(300, 30, 4, seed=1)
    c = sk.sketch_entries(300, 30, 4, seed=2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])


def test_apply_matches_brute_force():
    """A S by the definition sum_j A[i,j] S[j,c], looped in pure Python on a tiny case."""
    rng = np.random.default_rng(3)
    m, n, r1, s = 5, 17, 6, 3
    A = rng.standard_normal((m, n))
    S = sk.Sketch(n, r1, s, seed=99)
    cols, signs = S.cols, S.signs
    ref = [[0.0] * r1 for _ in range(m)]
    for i in range(m):
        for j in range(n):
            for t in range(s):
                ref[i][int(cols[j, t])] += float(signs[j, t]) / np.sqrt(s) * A[i, j]
    assert np.allclose(sk.apply_right(A, S), np.array(ref), rtol=0, atol=1e-14)
    X = rng.standard_normal((n, 4))
    refT = np.zeros((r1, 4))
    for j in range(n):
        for t in range(s):
            refT[int(cols[j, t])] += float(signs[j, t]) / np.sqrt(s) * X[j]
    assert np.allclose(sk.apply_left_t(S, X), refT, rtol=0, atol=1e-14)


def test_identity_sketch():
    S = sk.Sketch(12, 12, 1, 0, kind=sk.IDENTITY)
    assert np.array_equal(S.dense(), np.eye(12))


# ---------------------------------------------------------------- dense sketches (Lemma 3.2 items 1, 3)
@pytest.mark.parametrize("n", [1, 2, 16, 256])
def test_hadamard_entries_match_library(n):
    import scipy.linalg
    j = np.arange(n)
    assert np.array_equal(sk.hadamard_entries(j, j), scipy.linalg.hadamard(n))


@pytest.mark.parametrize("n,r1", [(64, 10), (64, 64), (1024, 100), (1024, 1024), (1, 1)])
def test_srht_columns_orthogonal_when_n_is_a_power_of_two(n, r1):
    """S = D H I_{:,T} / sqrt(r1) with H^T H = n I and D^2 = I: S^T S = (n / r1) I exactly
    when T has r1 distinct columns (a repeated or mis-signed column breaks it)."""
    S = sk.Sketch(n, r1, 1, 17, kind=sk.SRHT)
    assert S.npad == n and len(set(S.T.tolist())) == r1
    assert S.T.min() >= 0 and S.T.max() < n
    D = S.dense()
    assert np.allclose(np.abs(D), 1.0 / np.sqrt(r1), rtol=1e-15, atol=0)
    assert np.allclose(D.T @ D, (n / r1) * np.eye(r1), rtol=0, atol=1e-12)


def test_srht_apply_matches_fast_walsh_hadamard_transform():
    """A S against the butterfly recursion of the Walsh-Hadamard transform on the
    D-signed, zero-padded rows of A, then the columns of T (n = 300 -> n' = 512)."""
    rng = np.random.default_rng(4)
    m, n, r1 = 7, 300, 40
    A = rng.standard_normal((m, n))
    S = sk.Sketch(n, r1, 1, 29, kind=sk.SRHT)
    assert S.npad == 512
    X = np.zeros((m, 512))
    X[:, :n] = A * S.d[:n]
    h = 1
    while h < 512:                       # in-place butterflies (x + y, x - y)
        X = X.reshape(m, -1, 2, h)
        X = np.stack([X[:, :, 0] + X[:, :, 1], X[:, :, 0] - X[:, :, 1]], axis=2).reshape(m, 512)
        h *= 2
    ref = X[:, S.T] / np.sqrt(r1)
    assert np.allclose(sk.apply_right(A, S), ref, rtol=0, atol=1e-12)
    # zero columns appended up to n' change nothing (the padding reading)
    Ap = np.zeros((m, 512))
    Ap[:, :n] = A
    S512 = sk.Sketch(512, r1, 1, 29, kind=sk.SRHT)
    assert np.allclose(sk.apply_right(Ap, S512), sk.apply_right(A, S), rtol=0, atol=1e-12)


def test_srht_column_draws_uniform():
    """Each of the n' = 16 columns lands in T (r1 = 4) with probability 1/4, and the
    first drawn column is uniform over the 16."""
    counts = np.zeros(16)
    first = np.zeros(16)
    trials = 3000
    for seed in range(trials):
        T = sk.srht_columns(4, 4, seed)
        assert len(set(T.tolist())) == 4
        counts[T] += 1
        first[T[0]] += 1
    assert scipy.stats.chisquare(counts).pvalue > 1e-4
    assert scipy.stats.chisquare(first).pvalue > 1e-4
    d = sk.srht_signs(1 << 16, 5)
    assert abs(d.mean()) < 5 / np.sqrt(d.size)


def test_dense_sign_entries():
    n, r1 = 2000, 300
    S = sk.Sketch(n, r1, 1, 42, kind=sk.DENSE_SIGN)
    D = S.dense()
    assert np.array_equal(np.abs(D), np.full((n, r1), 1.0 / np.sqrt(r1)))
    G = D.T @ D
    assert np.allclose(np.diag(G), n / r1, rtol=1e-14)
    off = (G - np.diag(np.diag(G))) * r1 / np.sqrt(n)      # ~ N(0, 1) per entry
    assert abs(off.std() - 1.0) < 0.03 and np.abs(off).max() < 6.0
    sg = S.signs.astype(np.float64)
    assert abs(sg.mean()) < 5 / np.sqrt(sg.size)
    # neighbouring entries come from neighbouring bits of one draw: uncorrelated
    assert abs(np.mean(sg[:, :-1] * sg[:, 1:])) < 5 / np.sqrt(sg.size)
    assert abs(np.mean(sg[:-1] * sg[1:])) < 5 / np.sqrt(sg.size)
    assert np.array_equal(sk.dense_signs(5, 7, 42), S.signs[:5, :7])


@pytest.mark.parametrize("kind", [sk.DENSE_SIGN, sk.SRHT, sk.SPARSE_SIGN])
@pytest.mark.parametrize("n", [1024, 600])
def test_sketch_families_are_subspace_embeddings(kind, n):
    """Lemma 3.2: for U (n x k) with orthonormal columns, U^T S S^T U is close to
    I once r1 >> k; each family's scale makes E[S S^T] = I (a wrong scale fails).
    For the SRHT with n < n' (zero padding) E[S S^T] = (1/r1)(r1/n') D H H^T D = I
    still holds on the first n rows."""
    rng = np.random.default_rng(8)
    k, r1 = 8, 512
    U, _ = np.linalg.qr(rng.standard_normal((n, k)))
    S = sk.Sketch(n, r1, 8, 77, kind=kind)
    SU = sk.apply_left_t(S, U)
    assert np.linalg.norm(SU.T @ SU - np.eye(k), 2) < 0.5


@pytest.mark.parametrize("kind", [sk.DENSE_SIGN, sk.SRHT])
def test_exact_low_rank_is_recovered_with_dense_sketches(kind):
    sigma = np.array([5.0, 3.0, 2.0, 1.0, 0.5])
    A, _ = wl.dense_lowrank(90, 60, sigma, seed=12)
    S = sk.Sketch(60, 20, 1, 3, kind=kind)
    Q = alg.range_finder(A, S, sk.gaussian(20, 8, 4), q=1)
    assert alg.residual_fro(A, Q) < 1e-13 * np.linalg.norm(A)


def test_gaussian_omega_is_standard_normal():
    z = sk.gaussian(300, 400, seed=43).reshape(-1)
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 0.02
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-4
    # neighbouring entries come from one Box-Muller pair: still uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 0.02
    assert np.array_equal(sk.gaussian(3, 5, 43), sk.gaussian(300, 400, 43).reshape(-1)[:15].reshape(3, 5))


# ---------------------------------------------------------------- Algorithm 1
def test_orth_is_orthonormal_and_spans():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((80, 12))
    Q = alg.orth(Y)
    assert np.linalg.norm(Q.T @ Q - np.eye(12)) < 1e-13
    assert np.linalg.norm(Q @ (Q.T @ Y) - Y) < 1e-12 * np.linalg.norm(Y)


def test_q0_with_identity_omega_spans_AS():
    """q = 0 and Omega = I_{r1}: Y = A S exactly, so range(Q) = range(A S)."""
    A, _ = wl.dense_lowrank(60, 40, np.linspace(3, 1, 40), seed=5)
    S = sk.Sketch(40, 10, 4, seed=11)
    Q = alg.range_finder(A, S, np.eye(10), q=0)
    AS = A @ S.dense()
    assert Q.shape == (60, 10)
    assert np.linalg.norm(Q @ (Q.T @ AS) - AS) < 1e-12 * np.linalg.norm(AS)


def test_identity_sketch_is_subspace_iteration_converging_to_optimum():
    """S = I recovers the classical range finder (Section 2); with many power steps and a
    spectral gap, Q spans the top singular subspace, so the residual equals Eckart-Young."""
    sigma = np.concatenate([np.linspace(10, 5, 8), 0.5 * np.linspace(1, 0.1, 32)])
    A, _ = wl.dense_lowrank(70, 40, sigma, seed=8)
    S = sk.Sketch(40, 40, 1, 0, kind=sk.IDENTITY)
    Om = sk.gaussian(40, 8, seed=3)
    Q = alg.range_finder(A, S, Om, q=25)
    res = alg.residual_fro(A, Q)
    opt = alg.optimal_fro(sigma, 8)
    assert abs(res - opt) < 1e-9 * opt
    # and the projection matches the truncated SVD (library routine)
    U, s, Vt = np.linalg.svd(A)
    P_true = U[:, :8] @ U[:, :8].T
    assert np.linalg.norm(Q @ Q.T - P_true) < 1e-8


def test_reorth_does_not_change_output_in_exact_arithmetic():
    """Section 2: intermediate re-orthonormalisation leaves range(Y) unchanged."""
    A, _ = wl.dense_lowrank(50, 30, np.linspace(2, 1, 30), seed=9)
    S = sk.Sketch(30, 15, 3, seed=1)
    Om = sk.gaussian(15, 5, seed=2)
    Q1 = alg.range_finder(A, S, Om, q=2, reorth=True)
    Q2 = alg.range_finder(A, S, Om, q=2, reorth=False)
    assert np.linalg.norm(Q1 @ Q1.T - Q2 @ Q2.T) < 1e-10


def test_power_step_direction():
    """One power step uses A~ A~^T (not A~^T A~): compare with the definition on a tiny case."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((9, 7))
    S = sk.Sketch(7, 5, 2, seed=6)
    Om = rng.standard_normal((5, 3))
    At = A @ S.dense()
    Y = At @ At.T @ At @ Om
    Q = alg.range_finder(A, S, Om, q=1)
    assert np.linalg.norm(Q @ (Q.T @ Y) - Y) < 1e-12 * np.linalg.norm(Y)


def test_exact_low_rank_is_recovered():
    sigma = np.array([5.0, 3.0, 2.0, 1.0, 0.5])
    A, _ = wl.dense_lowrank(90, 60, sigma, seed=12)
    S = sk.Sketch(60, 20, 4, seed=3)
    Q = alg.range_finder(A, S, sk.gaussian(20, 8, 4), q=1)
    assert alg.residual_fro(A, Q) < 1e-13 * np.linalg.norm(A)


def test_eckart_young_lower_bound_and_cfg1_closed_form():
    """Residual never beats Eckart-Young; the 2000 x 1000, sigma_i = 1/i optimum at k = 50
    is sqrt(sum_{i=51}^{1000} i^-2) = sqrt(psi1(51) - psi1(1001))."""
    closed = np.sqrt(scipy.special.polygamma(1, 51) - scipy.special.polygamma(1, 1001))
    sig = 1.0 / np.arange(1, 1001)
    assert abs(alg.optimal_fro(sig, 50) - closed) < 1e-14
    assert abs(closed - 0.1371197763272333) < 1e-12
    A, sigma = wl.plain_fp64(200, 100, seed=1001)
    assert np.allclose(np.linalg.svd(A, compute_uv=False), sigma, atol=1e-13)
    for seed in range(3):
        S = sk.Sketch(100, 20, 8, seed=seed)
        Q = alg.range_finder(A, S, sk.gaussian(20, 10, seed + 50), q=2)
        assert alg.residual_fro(A, Q) >= alg.optimal_fro(sigma, 10) * (1 - 1e-12)


def test_sketched_power_improves_then_plateau_falls_with_sketch_size():
    """Theorem 2.1 and Section 4, qualitatively: error drops with q, and the level it
    settles at is lower for a larger sketch (averaged over seeds)."""
    A, sigma = wl.plain_fp64(400, 300, seed=21)
    k = 10
    opt = alg.optimal_fro(sigma, k)

    def err(r1, q):
        e = []
        for sd in range(6):
            S = sk.Sketch(300, r1, 4, seed=100 + sd)
            Q = alg.range_finder(A, S, sk.gaussian(r1, k, 200 + sd), q=q)
            e.append(alg.residual_fro(A, Q) / opt)
        return float(np.mean(e))

    assert err(40, 3) < err(40, 0)
    assert err(160, 6) < err(40, 6)


# ---------------------------------------------------------------- Randomized SVD finish
def test_rsvd_factors_reproduce_projection():
    A, sigma = wl.plain_fp64(120, 80, seed=31)
    S = sk.Sketch(80, 30, 8, seed=42)
    U, s, Vt, Q = alg.rsvd(A, S, sk.gaussian(30, 12, 43), q=2, k=12)
    assert np.linalg.norm(U.T @ U - np.eye(12)) < 1e-13
    assert np.linalg.norm(Vt @ Vt.T - np.eye(12)) < 1e-13
    assert np.all(np.diff(s) <= 0)
    # U S V^T equals Q Q^T A (k = r2) and s are the singular values of Q Q^T A
    P = Q @ (Q.T @ A)
    assert np.linalg.norm((U * s) @ Vt - P) < 1e-12 * np.linalg.norm(A)
    assert np.allclose(s, np.linalg.svd(P, compute_uv=False)[:12], rtol=1e-12)
    # sign convention: largest-magnitude entry of each u_i is positive
    idx = np.argmax(np.abs(U), axis=0)
    assert np.all(U[idx, np.arange(12)] > 0)


# ---------------------------------------------------------------- Algorithm 2
def test_lowrank_with_identity_S2_is_projection():
    """S2 = I: X = Y^+ A, so Y X = Q Q^T A."""
    A, _ = wl.plain_fp64(70, 50, seed=41)
    S1 = sk.Sketch(50, 20, 4, seed=1)
    S2 = sk.Sketch(70, 70, 1, 0, kind=sk.IDENTITY)
    Om = sk.gaussian(20, 8, 2)
    Y, X = alg.lowrank(A, S1, S2, Om, q=1)
    Q = alg.range_finder(A, S1, Om, q=1)
    assert np.linalg.norm(Y @ X - Q @ (Q.T @ A)) < 1e-12 * np.linalg.norm(A)


def test_lowrank_exact_on_low_rank_input():
    sigma = np.array([4.0, 2.0, 1.0])
    A, _ = wl.dense_lowrank(80, 60, sigma, seed=43)
    Y, X = alg.lowrank(A, sk.Sketch(60, 20, 4, 1), sk.Sketch(80, 20, 4, 2), sk.gaussian(20, 6, 3), q=1)
    assert np.linalg.norm(Y @ X - A) < 1e-12 * np.linalg.norm(A)


# ---------------------------------------------------------------- Algorithm 3
def test_nystrom_identity_with_range_finder_on_sqrt():
    """Proof of Theorem 2.3: C W^+ C^T = A^{1/2} Q Q^T A^{1/2} with Q from Algorithm 1
    applied to A^{1/2} with the same S and Omega."""
    n = 60
    sigma = np.linspace(4.0, 0.01, n) ** 2
    A = wl.psd_lowrank(n, sigma, seed=51)
    lam, V = np.linalg.eigh(A)
    Ah = (V * np.sqrt(np.maximum(lam, 0))) @ V.T
    S = sk.Sketch(n, 25, 4, seed=5)
    Om = sk.gaussian(25, 8, 6)
    for q in (0, 1, 2):
        C, W = alg.nystrom(A, S, Om, q)
        Ahat = alg.nystrom_apply(C, W)
        Q = alg.range_finder(Ah, S, Om, q)
        ref = Ah @ Q @ Q.T @ Ah
        assert np.linalg.norm(Ahat - ref) < 1e-9 * np.linalg.norm(A)
        # A - A_hat is psd
        assert np.linalg.eigvalsh(A - Ahat).min() > -1e-9 * np.linalg.norm(A)


def test_nystrom_exact_on_low_rank_psd():
    A = wl.psd_lowrank(50, np.array([3.0, 2.0, 1.0, 0.5]), seed=52)
    C, W = alg.nystrom(A, sk.Sketch(50, 20, 4, 1), sk.gaussian(20, 6, 2), q=1)
    assert np.linalg.norm(alg.nystrom_apply(C, W) - A) < 1e-11 * np.linalg.norm(A)


def test_gmm_kernel_is_psd_with_unit_diagonal():
    K, h, X = wl.gmm_kernel(200, seed=3)
    assert np.allclose(np.diag(K), 1.0)
    assert np.linalg.eigvalsh(K).min() > -1e-10
    assert h > 0


# ---------------------------------------------------------------- selector network (oracle)
def test_mlp_gradient_matches_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(0)
    p = mlp.init_params(3) * 0.5
    X = rng.standard_normal((5, mlp.D_IN))
    T = rng.standard_normal((5, mlp.D_OUT))
    M = (rng.uniform(size=(5, mlp.D_OUT)) > 0.3).astype(float)
    loss, g = mlp.loss_grad(p, X, T, M)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = 1e-6
        fd = (mlp.loss_grad(p + e, X, T, M)[0] - mlp.loss_grad(p - e, X, T, M)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_mlp_forward_small_case_by_hand():
    """Identity-like weights: check the forward pass against a hand evaluation."""
    from oracle import mlp
    p = np.zeros(mlp.N_PARAMS)
    layers = mlp.unpack(p)  # views into p
    layers[0][0][0, 0] = 2.0      # h1_0 = relu(2 x0 - 1)
    layers[0][1][0] = -1.0
    layers[1][0][0, 0] = 1.0      # h2_0 = h1_0
    layers[2][0][0, 0] = -3.0     # h3_0 = relu(-3 h2_0 + 10)
    layers[2][1][0] = 10.0
    layers[3][0][4, 0] = 0.5      # y_4 = 0.5 h3_0 + 7
    layers[3][1][4] = 7.0
    x = np.zeros((1, mlp.D_IN))
    x[0, 0] = 2.0
    y, _ = mlp.forward(p, x)
    h1 = max(2 * 2.0 - 1, 0)
    h3 = max(-3 * h1 + 10, 0)
    assert y[0, 4] == 0.5 * h3 + 7 and np.count_nonzero(y) == 1


def test_adam_first_step_is_sign_times_lr():
    """With bias correction the first Adam step moves each parameter by lr * g / (|g| + eps)."""
    from oracle import mlp
    p = np.arange(6.0)
    g = np.array([1.0, -2.0, 3.0, -4.0, 0.5, -0.25])
    p1, m1, v1 = mlp.adam(p, np.zeros(6), np.zeros(6), g, step=1, lr=0.01)
    assert np.allclose(p1, p - 0.01 * np.sign(g), atol=1e-9)


def test_selector_features_closed_form():
    """Features of a sketch with known singular values s_i = 2^-i."""
    from oracle import mlp
    r2 = 8
    s = 2.0 ** -np.arange(r2)
    U, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((50, r2)))
    V, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((r2, r2)))
    Y0 = (U * s) @ V.T
    f = mlp.features_from_sketch(Y0, m=50, n=30, r1=32)
    assert np.isclose(f[0], np.log10(s[1]))
    assert np.isclose(f[1], np.log10(s[3]))
    assert np.isclose(f[2], np.log10(s[7]))
    assert np.isclose(f[3], np.log10(r2 * s[7] ** 2 / np.sum(s ** 2)))
    assert np.isclose(f[7], 2.0 / 3)


def test_polydecay_generator_spectrum():
    """Section 4's polydecay matrix: singular values m / i exactly up to FP32 rounding
    (the benchmark's Section 4 protocol builds it the same way at 30000 x 15000)."""
    import torch
    A, sigma = wl.polydecay_torch(300, 150, seed=3, device="cpu")
    assert A.shape == (300, 150) and A.dtype == torch.float32
    assert np.allclose(sigma, 300.0 / np.arange(1, 151))
    s = np.linalg.svd(A.double().numpy(), compute_uv=False)
    assert np.max(np.abs(s - sigma) / sigma[0]) < 1e-5


def test_residual_norms_closed_form():
    """A = U diag(sigma) V^T with orthonormal U, V and Q = the first k columns of
    U: ||A - Q Q^T A||_2 = sigma_{k+1} and ||.||_F = sqrt(sum_{i>k} sigma_i^2)
    (Eckart-Young attained); a Q missing the top direction gives sigma_1."""
    rng = np.random.default_rng(5)
    m, n, k = 60, 40, 7
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sigma = np.sort(rng.uniform(0.1, 3.0, n))[::-1]
    A = (U * sigma) @ V.T
    Q = U[:, :k]
    assert abs(alg.residual_spec(A, Q) - sigma[k]) <= 1e-12 * sigma[0]
    assert abs(alg.residual_fro(A, Q) - np.sqrt(np.sum(sigma[k:] ** 2))) <= 1e-12 * sigma[0]
    assert abs(alg.residual_fro(A, Q) - alg.optimal_fro(sigma, k)) <= 1e-12 * sigma[0]
    Qm = U[:, 1:k + 1]                   # skips the largest direction
    assert abs(alg.residual_spec(A, Qm) - sigma[0]) <= 1e-12 * sigma[0]
    # a rotated basis of the same range gives the same residuals
    R, _ = np.linalg.qr(rng.standard_normal((k, k)))
    assert abs(alg.residual_spec(A, Q @ R) - sigma[k]) <= 1e-12 * sigma[0]


def test_apply_left_is_the_adjoint_of_apply_left_t():
    """<S Y, X> = <Y, S^T X> for the sparse sign sketch: S Y (the test matrix of
    the factored Nystrom output) against the independently written S^T X."""
    rng = np.random.default_rng(8)
    n, r1, p = 300, 40, 7
    S = sk.Sketch(n, r1, 5, 17)
    Y = rng.standard_normal((r1, p))
    X = rng.standard_normal((n, p))
    lhs = np.sum(sk.apply_left(S, Y) * X)
    rhs = np.sum(Y * sk.apply_left_t(S, X))
    assert abs(lhs - rhs) <= 1e-12 * np.abs(lhs)
    assert np.allclose(sk.apply_left(S, Y), S.dense() @ Y, rtol=0, atol=1e-14)


def _psd(n, rank, rng, decay=1.0):
    V, _ = np.linalg.qr(rng.standard_normal((n, rank)))
    mu = decay ** np.arange(rank) * rng.uniform(0.5, 1.5, rank)
    return (V * mu) @ V.T


def test_factored_nystrom_recovers_exact_low_rank():
    """rank(A) <= r2 and a sketch that sees the range: A_hat = A (the shift nu
    is O(u |A|))."""
    rng = np.random.default_rng(9)
    n, rank, r1, r2 = 200, 10, 60, 20
    A = _psd(n, rank, rng)
    S = sk.Sketch(n, r1, 8, 3)
    U, lam = alg.nystrom_eig(A, S, sk.gaussian(r1, r2, 4), 1)
    Ah = (U * lam) @ U.T
    assert np.linalg.norm(A - Ah) <= 1e-10 * np.linalg.norm(A)
    assert np.all(lam >= 0) and np.all(np.diff(lam) <= 0)
    assert np.linalg.norm(U.T @ U - np.eye(r2)) <= 1e-12


def test_factored_nystrom_equals_c_w_pinv_c():
    """For a positive definite W the shifted factored form and C W^+ C^T agree to
    O(nu kappa(W)); A - A_hat stays positive semidefinite (Theorem 2.3's proof)."""
    rng = np.random.default_rng(10)
    n, r1, r2 = 150, 50, 15
    A = _psd(n, n, rng, decay=0.9) + 1e-3 * np.eye(n)
    S = sk.Sketch(n, r1, 8, 5)
    Om = sk.gaussian(r1, r2, 6)
    C, W = alg.nystrom(A, S, Om, 2)
    U, lam = alg.nystrom_eig(A, S, Om, 2)
    Ah1 = alg.nystrom_apply(C, W)
    Ah2 = (U * lam) @ U.T
    assert np.linalg.norm(Ah1 - Ah2) <= 1e-8 * np.linalg.norm(A)
    assert np.linalg.eigvalsh(A - Ah2).min() >= -1e-9 * np.linalg.norm(A, 2)


def test_gaussian_kernel_hand_values():
    # points 0, 1, 3 on a line, h = 1: exp(-1/2), exp(-9/2), exp(-2) off the diagonal
    K = alg.gaussian_kernel(np.array([[0.0], [1.0], [3.0]]), 1.0)
    e = np.exp
    want = np.array([[1.0, e(-0.5), e(-4.5)], [e(-0.5), 1.0, e(-2.0)], [e(-4.5), e(-2.0), 1.0]])
    assert np.allclose(K, want, rtol=1e-15, atol=0.0)
    # h = 2 in R^2: |(0,0) - (3,4)|^2 = 25, 25 / 8
    K = alg.gaussian_kernel(np.array([[0.0, 0.0], [3.0, 4.0]]), 2.0)
    assert abs(K[0, 1] - np.exp(-25.0 / 8.0)) <= 1e-16


def test_gaussian_kernel_invariances_and_generator_agreement():
    # shifting or rotating the points leaves K unchanged; K is psd with unit
    # diagonal; and it matches the input generator's kernel (norm expansion)
    rng = np.random.default_rng(8)
    X = rng.standard_normal((60, 5))
    h = 1.7
    K = alg.gaussian_kernel(X, h)
    Q, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    assert np.allclose(alg.gaussian_kernel(X + 3.0, h), K, rtol=0, atol=1e-14)
    assert np.allclose(alg.gaussian_kernel(X @ Q, h), K, rtol=0, atol=1e-14)
    assert np.allclose(np.diag(K), 1.0) and np.allclose(K, K.T)
    assert np.linalg.eigvalsh(K).min() >= -1e-12
    sq = np.sum(X * X, axis=1)
    Kg = np.exp(-np.maximum(sq[:, None] + sq[None, :] - 2.0 * X @ X.T, 0.0) / (2.0 * h * h))
    assert np.allclose(K, Kg, rtol=0, atol=1e-13)


def test_nystrom_gauss_is_nystrom_of_the_formed_kernel():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((200, 3))
    S = sk.Sketch(200, 40, 4, 5)
    Om = sk.gaussian(40, 10, 6)
    U1, l1 = alg.nystrom_gauss(X, 1.3, S, Om, 1)
    U2, l2 = alg.nystrom_eig(alg.gaussian_kernel(X, 1.3), S, Om, 1)
    assert np.array_equal(U1, U2) and np.array_equal(l1, l2)
