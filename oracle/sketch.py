"""Sketch matrices S and the Gaussian start block Omega (oracle side).

TEST INFRASTRUCTURE ONLY: imported by tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the product path.

Paper anchors (Chenakkod & Derezinski, "Accelerating Power Method with Fast
Sketching for Stronger Low-Rank Approximation"):
  * Lemma 3.2, item 2: S in R^{n x r} is a CountSketch-type matrix with s random
    non-zero entries per row, each of the form +-1/sqrt(s).
  * Algorithm 1 inputs: S in R^{n x r1}, Omega in R^{r1 x r2} Gaussian
    (Section 2; Theorem 2.1 asks for a Gaussian Omega of size r2 = O(k)).
  * Section 4: S = CountSketch with one non-zero per row is the s = 1 case.
  * Lemma 3.2, item 1: S with independent sub-Gaussian entries scaled by
    1/sqrt(r), e.g. +-1/sqrt(r) (the dense sign sketch here).
  * Lemma 3.2, item 3: the subsampled randomized Hadamard transform
    S = (1/sqrt(r)) D H I_{:,T}: D diagonal with random +-1 entries, H a
    Hadamard matrix, T a uniformly random subset of r of the n columns.

Readings of points the paper leaves open (each listed in the design notes):
  * the s non-zeros of row j sit in s *distinct* columns drawn uniformly, by
    rejection of repeats; column = floor(u * r1 / 2^32) for a 32-bit draw u;
  * the t-th non-zero of row j takes its sign from one bit of a separate draw;
  * the value is sign / sqrt(s).
  * dense sign sketch (item 1): entry (j, c) is an independent fair sign / sqrt(r1);
  * SRHT (item 3): the Hadamard matrix is Sylvester's, H[j, k] = (-1)^popcount(j & k),
    of order n' = the smallest power of two >= n; A is read as padded with n' - n
    zero columns, so S is the first n rows of the n' x r1 product; T holds r1
    distinct columns of H in the order they are drawn (column c of S is the c-th
    drawn); a draw is floor(u n' / 2^32) = u >> (32 - log2 n') for a 32-bit u and
    repeats of earlier draws are rejected.

Counter layout of the draws (Philox4x32-10, key = 64-bit seed):
  * candidate number u of row j: counter (j_lo, j_hi, u >> 2, 0), word u & 3;
  * sign of entry t of row j:     counter (j_lo, j_hi, t >> 7, 1),
                                  word (t >> 5) & 3, bit t & 31 (1 -> minus);
  * Omega entry e (row-major index): pair p = e >> 1, counter (p_lo, p_hi, 0, 2);
    Box-Muller on two 53-bit uniforms u1 = (x1 + 1) 2^-53 in (0, 1] from words
    (w0, w1) and u2 = x2 2^-53 in [0, 1) from (w2, w3):
    radius sqrt(-2 ln u1), angle 2 pi u2; even e -> cos, odd e -> sin.
  * dense sign of entry (j, c):   counter (j_lo, j_hi, c >> 7, 4),
                                  word (c >> 5) & 3, bit c & 31 (1 -> minus);
  * SRHT sign D_j (j < n'):       counter (b_lo, b_hi, 0, 5) with b = j >> 7,
                                  word (j >> 5) & 3, bit j & 31 (1 -> minus);
  * SRHT draw number u:           counter (b_lo, b_hi, 0, 6) with b = u >> 2, word u & 3.
"""
import numpy as np
import scipy.sparse as sp

from .philox import philox4x32_10, seed_key

SPARSE_SIGN = 0
IDENTITY = 1
DENSE_SIGN = 2
SRHT = 3

_S32 = np.uint64(32)
_MASK32 = np.uint64(0xFFFFFFFF)


def sketch_entries(n, r1, s, seed):
    """Column indices (n, s) and signs (n, s) of the sparse sign sketch.

    Entry t of row j is the t-th accepted draw of row j (draw order, not sorted).
    """
    if not (1 <= s <= r1):
        raise ValueError("need 1 <= s <= r1")
    k0, k1 = seed_key(seed)
    j = np.arange(n, dtype=np.uint64)
    jlo, jhi = j & _MASK32, j >> _S32
    cols = np.full((n, s), -1, dtype=np.int64)
    used = np.zeros(n, dtype=np.uint64)          # candidates consumed per row
    for t in range(s):
        pend = np.arange(n)
        while pend.size:
            u = used[pend]
            w = philox4x32_10(jlo[pend], jhi[pend], u >> np.uint64(2), 0, k0, k1)
            sel = (u & np.uint64(3)).astype(np.int64)
            word = np.choose(sel, w)
            cand = ((word * np.uint64(r1)) >> _S32).astype(np.int64)
            dup = (cols[pend, :t] == cand[:, None]).any(axis=1)
            used[pend] += np.uint64(1)
            ok = ~dup
            cols[pend[ok], t] = cand[ok]
            pend = pend[dup]
    signs = np.empty((n, s), dtype=np.int64)
    for t in range(s):
        w = philox4x32_10(jlo, jhi, np.uint64(t >> 7), 1, k0, k1)
        word = w[(t >> 5) & 3]
        bit = (word >> np.uint64(t & 31)) & np.uint64(1)
        signs[:, t] = 1 - 2 * bit.astype(np.int64)
    return cols, signs


def _bits(words, pos):
    """Bit pos & 31 of word (pos >> 5) & 3 of a Philox output (words: 4 arrays)."""
    W = np.stack(words)
    sel = (pos >> np.uint64(5)) & np.uint64(3)
    word = np.take_along_axis(W, sel.astype(np.int64)[None], axis=0)[0]
    return (word >> (pos & np.uint64(31))) & np.uint64(1)


def dense_signs(n, r1, seed):
    """Signs (n, r1) of the dense sign sketch (Lemma 3.2 item 1), as +-1 int8."""
    k0, k1 = seed_key(seed)
    j = np.arange(n, dtype=np.uint64)[:, None]
    blk = np.arange((r1 + 127) // 128, dtype=np.uint64)[None, :]
    W = np.stack(philox4x32_10(j & _MASK32, j >> _S32, blk, 4, k0, k1))   # (4, n, blocks)
    c = np.arange(r1, dtype=np.uint64)
    words = W[((c >> np.uint64(5)) & np.uint64(3)).astype(np.int64), :,
              (c >> np.uint64(7)).astype(np.int64)]                          # (r1, n)
    bit = (words >> (c & np.uint64(31))[:, None]) & np.uint64(1)
    return np.ascontiguousarray((1 - 2 * bit.astype(np.int64)).T).astype(np.int8)


def hadamard_order(n):
    """log2 of n' = the smallest power of two >= n."""
    L = 0
    while (1 << L) < n:
        L += 1
    return L


def srht_signs(npad, seed):
    """The diagonal D (npad entries, +-1) of the SRHT (Lemma 3.2 item 3)."""
    k0, k1 = seed_key(seed)
    j = np.arange(npad, dtype=np.uint64)
    b = j >> np.uint64(7)
    bit = _bits(philox4x32_10(b & _MASK32, b >> _S32, 0, 5, k0, k1), j)
    return 1 - 2 * bit.astype(np.int64)


def srht_columns(L, r1, seed):
    """The r1 sampled Hadamard columns T of the SRHT, in draw order.

    Draw u gives column word_u >> (32 - L) of the n' = 2^L columns; a column
    drawn before is skipped; the first r1 distinct draws are kept.
    """
    npad = 1 << L
    if not (1 <= r1 <= npad):
        raise ValueError("need 1 <= r1 <= n'")
    k0, k1 = seed_key(seed)
    taken = np.zeros(npad, dtype=bool)
    out = []
    u = 0
    while len(out) < r1:
        blk = np.arange(u, u + 1024, dtype=np.uint64)
        b = blk >> np.uint64(2)
        w = philox4x32_10(b & _MASK32, b >> _S32, 0, 6, k0, k1)
        word = np.choose((blk & np.uint64(3)).astype(np.int64), w)
        cand = (word >> np.uint64(32 - L)).astype(np.int64) if L > 0 else np.zeros(1024, np.int64)
        for c in cand.tolist():          # the draws in order
            if not taken[c]:
                taken[c] = True
                out.append(c)
                if len(out) == r1:
                    break
        u += 1024
    return np.array(out, dtype=np.int64)


def hadamard_entries(rows, cols):
    """Sylvester Hadamard entries H[rows, cols] = (-1)^popcount(rows & cols)."""
    r = np.asarray(rows, dtype=np.uint64)[:, None]
    c = np.asarray(cols, dtype=np.uint64)[None, :]
    return 1 - 2 * (np.bitwise_count(r & c) & 1).astype(np.int64)


class Sketch:
    """The matrix S in R^{n x r1} of Lemma 3.2 (item 2 by default; item 1 with
    kind=DENSE_SIGN, item 3 with kind=SRHT) or the identity."""

    def __init__(self, n, r1, s, seed, kind=SPARSE_SIGN):
        self.n, self.r1, self.s, self.seed, self.kind = int(n), int(r1), int(s), int(seed), kind
        if kind == IDENTITY:
            if r1 != n:
                raise ValueError("identity sketch needs r1 == n")
            self.cols = np.arange(n, dtype=np.int64)[:, None]
            self.signs = np.ones((n, 1), dtype=np.int64)
            self.scale = 1.0
        elif kind == DENSE_SIGN:
            self.signs = dense_signs(n, r1, seed)
            self.scale = 1.0 / np.sqrt(r1)
        elif kind == SRHT:
            if r1 > n:
                raise ValueError("SRHT needs r1 <= n")
            self.L = hadamard_order(n)
            self.npad = 1 << self.L
            self.d = srht_signs(self.npad, seed)
            self.T = srht_columns(self.L, r1, seed)
            self.scale = 1.0 / np.sqrt(r1)
        else:
            self.cols, self.signs = sketch_entries(n, r1, s, seed)
            self.scale = 1.0 / np.sqrt(s)

    def sparse(self):
        """S as a scipy CSR matrix (values sign * scale)."""
        if self.kind in (DENSE_SIGN, SRHT):
            return sp.csr_matrix(self.dense())
        n, w = self.cols.shape
        rows = np.repeat(np.arange(n), w)
        vals = self.signs.reshape(-1) * self.scale
        return sp.csr_matrix((vals, (rows, self.cols.reshape(-1))), shape=(self.n, self.r1))

    def dense(self):
        if self.kind == DENSE_SIGN:
            return self.signs.astype(np.float64) * self.scale
        if self.kind == SRHT:
            j = np.arange(self.n)
            return (self.d[:self.n, None] * hadamard_entries(j, self.T)) * self.scale
        return self.sparse().toarray()

    def buckets(self):
        """Column-bucketed (CSC) form: ptr[r1+1], rows (j ascending per column), signs."""
        n, w = self.cols.shape
        c = self.cols.reshape(-1)
        j = np.repeat(np.arange(n), w)
        sg = self.signs.reshape(-1)
        order = np.lexsort((j, c))
        counts = np.bincount(c, minlength=self.r1)
        ptr = np.concatenate([[0], np.cumsum(counts)])
        return ptr, j[order], sg[order]

def apply_right(A, S):
    """A_tilde = A S  (Algorithm 1 line 1; A is m x n, returns m x r1)."""
    if S.kind in (DENSE_SIGN, SRHT):
        return np.asarray(A, dtype=np.float64) @ S.dense()
    return np.asarray((S.sparse().T @ np.asarray(A, dtype=np.float64).T).T)


def apply_left_t(S, X):
    """S^T X  (Algorithm 2 line 2 and Algorithm 3 line 1; X is n x p)."""
    if S.kind in (DENSE_SIGN, SRHT):
        return S.dense().T @ np.asarray(X, dtype=np.float64)
    return np.asarray(S.sparse().T @ np.asarray(X, dtype=np.float64))


def gaussian(rows, cols, seed):
    """Omega in R^{rows x cols} with i.i.d. N(0,1) entries (Algorithm 1 input)."""
    k0, k1 = seed_key(seed)
    e = np.arange(rows * cols, dtype=np.uint64)
    p = e >> np.uint64(1)
    w0, w1, w2, w3 = philox4x32_10(p & _MASK32, p >> _S32, 0, 2, k0, k1)
    x1 = (w1 << np.uint64(21)) | (w0 >> np.uint64(11))
    x2 = (w3 << np.uint64(21)) | (w2 >> np.uint64(11))
    u1 = (x1 + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = x2.astype(np.float64) * 2.0 ** -53
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 6.283185307179586 * u2
    z = np.where((e & np.uint64(1)) == 0, rad * np.cos(ang), rad * np.sin(ang))
    return z.reshape(rows, cols)


def apply_left(S, Y):
    """S Y  (n x p) for Y of r1 x p: the test matrix T = S Y of Algorithm 3's
    output C = C~ Y = A (S Y)."""
    if S.kind in (DENSE_SIGN, SRHT):
        return S.dense() @ np.asarray(Y, dtype=np.float64)
    return np.asarray(S.sparse() @ np.asarray(Y, dtype=np.float64))
