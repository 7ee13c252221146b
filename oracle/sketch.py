"""Sparse sign sketch S and Gaussian start block Omega (oracle side).

TEST INFRASTRUCTURE ONLY: imported by tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the product path.

Paper anchors (Chenakkod & Derezinski, "Accelerating Power Method with Fast
Sketching for Stronger Low-Rank Approximation"):
  * Lemma 3.2, item 2: S in R^{n x r} is a CountSketch-type matrix with s random
    non-zero entries per row, each of the form +-1/sqrt(s).
  * Algorithm 1 inputs: S in R^{n x r1}, Omega in R^{r1 x r2} Gaussian
    (Section 2; Theorem 2.1 asks for a Gaussian Omega of size r2 = O(k)).
  * Section 4: S = CountSketch with one non-zero per row is the s = 1 case.

Readings of points the paper leaves open (each listed in the design notes):
  * the s non-zeros of row j sit in s *distinct* columns drawn uniformly, by
    rejection of repeats; column = floor(u * r1 / 2^32) for a 32-bit draw u;
  * the t-th non-zero of row j takes its sign from one bit of a separate draw;
  * the value is sign / sqrt(s).

Counter layout of the draws (Philox4x32-10, key = 64-bit seed):
  * candidate number u of row j: counter (j_lo, j_hi, u >> 2, 0), word u & 3;
  * sign of entry t of row j:     counter (j_lo, j_hi, t >> 7, 1),
                                  word (t >> 5) & 3, bit t & 31 (1 -> minus);
  * Omega entry e (row-major index): pair p = e >> 1, counter (p_lo, p_hi, 0, 2);
    Box-Muller on two 53-bit uniforms u1 = (x1 + 1) 2^-53 in (0, 1] from words
    (w0, w1) and u2 = x2 2^-53 in [0, 1) from (w2, w3):
    radius sqrt(-2 ln u1), angle 2 pi u2; even e -> cos, odd e -> sin.
"""
import numpy as np
import scipy.sparse as sp

from .philox import philox4x32_10, seed_key

SPARSE_SIGN = 0
IDENTITY = 1

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


class Sketch:
    """The matrix S in R^{n x r1} of Lemma 3.2 item 2 (or the identity)."""

    def __init__(self, n, r1, s, seed, kind=SPARSE_SIGN):
        self.n, self.r1, self.s, self.seed, self.kind = int(n), int(r1), int(s), int(seed), kind
        if kind == IDENTITY:
            if r1 != n:
                raise ValueError("identity sketch needs r1 == n")
            self.cols = np.arange(n, dtype=np.int64)[:, None]
            self.signs = np.ones((n, 1), dtype=np.int64)
            self.scale = 1.0
        else:
            self.cols, self.signs = sketch_entries(n, r1, s, seed)
            self.scale = 1.0 / np.sqrt(s)

    def sparse(self):
        """S as a scipy CSR matrix (values sign * scale)."""
        n, w = self.cols.shape
        rows = np.repeat(np.arange(n), w)
        vals = self.signs.reshape(-1) * self.scale
        return sp.csr_matrix((vals, (rows, self.cols.reshape(-1))), shape=(self.n, self.r1))

    def dense(self):
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
    return np.asarray((S.sparse().T @ np.asarray(A, dtype=np.float64).T).T)


def apply_left_t(S, X):
    """S^T X  (Algorithm 2 line 2 and Algorithm 3 line 1; X is n x p)."""
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
