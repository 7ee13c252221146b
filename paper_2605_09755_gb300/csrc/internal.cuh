// Internal (C++) interfaces shared by the libspm translation units.
#pragma once
#include "common.cuh"

namespace spm {

// Element types used inside the library.
enum Dt : int { DT_F32 = 0, DT_F64 = 1, DT_BF16 = 2 };

inline size_t dt_size(int dt) { return dt == DT_F64 ? 8 : (dt == DT_F32 ? 4 : 2); }

// A strided matrix view: element (i, j) at p[i*rs + j*cs] (in elements).
struct View {
  const void* p;
  int dt;
  int64_t rs, cs;
};
struct MView {
  void* p;
  int dt;
  int64_t rs, cs;
};
inline View rowmajor(const void* p, int dt, int64_t ld) { return View{p, dt, ld, 1}; }
inline View colmajor(const void* p, int dt, int64_t ld) { return View{p, dt, 1, ld}; }
inline View transpose(View v) { return View{v.p, v.dt, v.cs, v.rs}; }
inline MView mrowmajor(void* p, int dt, int64_t ld) { return MView{p, dt, ld, 1}; }
inline View cview(MView v) { return View{v.p, v.dt, v.rs, v.cs}; }

// ---------------------------------------------------------------- sketch.cu
// out (m x r1) = A (m x n) S ; out_dt in {F32, F64, BF16}; accumulates |A|_F^2
// into *fro2 (device double) when fro2 != nullptr.
// out_lo (BF16 outputs only): second half of a hi/lo split, out_lo = bf16(v - hi).
// status (device int, may be null): device-side errors (an expired bounded wait).
// a_hi, a_lo (BF16, row stride lds, may be null): where the kernel can, the
// (hi, lo) BF16 split of A is written in the same pass; *a_split (may be null)
// tells whether it was.
int sketch_apply_dev(const spm_sketch* S, const void* A, int a_dt, int64_t m, int64_t lda,
                     void* out, int out_dt, int64_t ldo, double* fro2, cudaStream_t st,
                     void* out_lo = nullptr, int* status = nullptr, void* a_hi = nullptr,
                     void* a_lo = nullptr, int64_t lds = 0, bool* a_split = nullptr);

// ---------------------------------------------------------------- sketch_sched.cu
// A S for FP32 A (n and lda multiples of 4, A 16-byte aligned, rows that fit
// whole in shared memory) by the scheduled kernel, into FP32 or BF16 (hi, and
// lo when out_lo is set) outputs; fro2 (may be null) accumulates |A|_F^2; with
// a_hi, a_lo (BF16, row stride lds: a multiple of 4, >= n; 8-byte aligned) A's
// (hi, lo) split is written in the same pass.  Plans the sketch on first use
// (not during stream capture).  Returns SPM_EUNSUPPORTED, with nothing
// launched, when the request or the sketch does not fit the kernel.
int sched_apply(spm_sketch* S, const float* A, int64_t m, int64_t lda, void* out, int out_dt,
                int64_t ldo, double* fro2, int* status, cudaStream_t st, void* out_lo,
                void* a_hi = nullptr, void* a_lo = nullptr, int64_t lds = 0);
void sched_init(spm_sketch* S);
void sched_free(spm_sketch* S);
// out (r1 x p) = S^T X, X (n x p, row stride ldx)
int sketch_apply_t_dev(const spm_sketch* S, const void* X, int x_dt, int64_t p, int64_t ldx,
                       void* out, int out_dt, int64_t ldo, cudaStream_t st);
int gaussian_dev(void* out, int dt, int64_t rows, int64_t cols, int64_t ld, uint64_t seed,
                 cudaStream_t st);

// ---------------------------------------------------------------- sketch_dense.cu
// Dense sign (Lemma 3.2 item 1) and SRHT (item 3) sketches: tables, A S and
// S^T X with the contracts of sketch_apply_dev / sketch_apply_t_dev.
int dense_sketch_create(spm_sketch* S, cudaStream_t st);
void dense_sketch_free(spm_sketch* S);
int dense_sketch_apply(const spm_sketch* S, const void* A, int a_dt, int64_t m, int64_t lda,
                       void* out, int out_dt, int64_t ldo, double* fro2, cudaStream_t st,
                       void* out_lo);
int dense_sketch_apply_t(const spm_sketch* S, const void* X, int x_dt, int64_t p, int64_t ldx,
                         void* out, int out_dt, int64_t ldo, cudaStream_t st);
inline bool dense_kind(const spm_sketch* S) {
  return S->kind == SPM_SKETCH_DENSE_SIGN || S->kind == SPM_SKETCH_SRHT;
}

// ---------------------------------------------------------------- nystrom.cu
// out (n x p) = S Y for Y (r1 x p) (row j: s terms of Y's rows); sparse kinds only
int sketch_left_dev(const spm_sketch* S, const void* Y, int dt, int64_t ldy, int64_t p, void* out,
                    int64_t ldo, cudaStream_t st);
// nu = sqrt(n) 2^-52 sqrt(*c_sumsq) into *nu_out, and C += nu T (n x p)
int nys_shift_dev(int64_t n, int64_t p, void* C, int64_t ldc, const void* Tm, int64_t ldt, int dt,
                  const double* c_sumsq, double* nu_out, cudaStream_t st);
// sigma = sqrt(sig2) (1 where 0), lam = max(sig2 - *nu, 0) in type ldt
int nys_lambda_dev(int64_t r, const void* sig2, int sdt, const double* nu, double* sigma, void* lam,
                   int ldt, cudaStream_t st);

// out (n x r1, type odt, ld ldo) = K S for the Gaussian kernel of the points X
// (n x d, type xdt, ld ldx): K[i, j] = exp(-|x_i - x_j|^2 / (2 h^2)), K never formed;
// an expired bounded wait is recorded in *status (nullable)
int gauss_sketch_dev(const spm_sketch* S, const void* X, int xdt, int64_t n, int64_t d, int64_t ldx,
                     double h, void* out, int odt, int64_t ldo, cudaStream_t st, int* status);

// ---------------------------------------------------------------- gemm_simt.cu
// C = alpha * A(MxK) * B(KxN) + beta * C  on CUDA cores.  Accumulates in FP64 if
// any operand is FP64, else FP32.  batch > 1: pointers advance by the strides.
int gemm_simt(int64_t M, int64_t N, int64_t K, double alpha, View A, View B, double beta, MView C,
              cudaStream_t st, int batch = 1, int64_t sA = 0, int64_t sB = 0, int64_t sC = 0);

// ---------------------------------------------------------------- sparse.cu
// Column index of a CSR matrix (rows ascending inside each column).
struct CscIndex {
  int64_t* colptr;  // n + 1
  int32_t* rowind;  // nnz
  void* vals;       // nnz, the matrix's type
};
int csr_check(const spm_csr* A, int64_t n);
// out (m x r1, ld ldo, type dt) = A S for A = A_csr + U diag(sig) V^T; an
// out-of-range column index sets SPM_EINVAL in *status and is skipped
int csr_sketch_dev(const spm_sketch* S, const spm_csr* A, int dt, void* out, int64_t ldo, int* status,
                   cudaStream_t st, bool tc = false);
int csc_build(const spm_csr* A, int dt, Arena& ar, CscIndex& out, cudaStream_t st);
// B (r2 x n, ld ldb) = Q^T A, Q (m x r2, ld ldq), all of type dt
// tc (FP32 only): the low-rank terms as split-BF16 tensor-core products, with
// Q's split (Qhi, Qlo, ld ldqh) for Q^T U
int csr_project_dev(const spm_csr* A, const CscIndex& csc, int dt, const void* Q, int64_t ldq,
                    int64_t r2, void* B, int64_t ldb, cudaStream_t st,
                    const __nv_bfloat16* Qhi = nullptr, const __nv_bfloat16* Qlo = nullptr,
                    int64_t ldqh = 0);

// ---------------------------------------------------------------- gemm_tc.cu
// One BF16 operand of a tcgen05 product.  `p` points at a row-major array with
// leading dimension `ld` (elements, multiple of 8).  For the A operand (M x K):
// mn_major = false -> array is M x K (K contiguous); true -> array is K x M.
// For the B operand (N x K): mn_major = false -> array is N x K; true -> K x N.
struct TcOp {
  const __nv_bfloat16* p;
  int64_t ld;
  bool mn_major;
};
// D(M x N, fp32) = alpha * sum_{q < npass} A[q] * B[q]^T, written at
// D[i*d_rs + j*d_cs].  splitk > 1 splits K in equal chunks; partial sums are
// reduced deterministically (fixed order) before D is written.
// sym_upper (M == N, the product symmetric by construction, e.g. a Gram
// matrix): only the output tiles that meet the upper triangle are computed and
// the strictly lower triangle is then copied from the upper one.
// status (device int, may be null): an expired bounded wait records SPM_ETIMEOUT there.
int gemm_tc(int64_t M, int64_t N, int64_t K, int npass, const TcOp* A, const TcOp* B, float alpha,
            float* D, int64_t d_rs, int64_t d_cs, int splitk, cudaStream_t st,
            bool sym_upper = false, int* status = nullptr);
// Device address of the status word that the public product entry points
// (spm_gemm_bf16, spm_gemm_bf16_noalloc) record into on the current device.
int gemm_public_status(int** status);
bool tc_available();
// split-K factor of a tensor-core product (a wave and traffic cost model; api.cu)
int auto_splitk(int64_t M, int64_t N, int64_t K, bool sym = false);

// ---------------------------------------------------------------- dense.cu
// y = convert(x) elementwise on a strided 2-D view (rows x cols).
int convert2d(int64_t rows, int64_t cols, View x, MView y, cudaStream_t st);
// hi = bf16(x), lo = bf16(x - hi)  (split-precision operands)
int split_bf16(int64_t rows, int64_t cols, View x, MView hi, MView lo, cudaStream_t st);
// x (row-major, FP32 or FP64, ld ldx) ~ p1 + p2 + p3 in BF16 (row-major, ld ldp)
int split3_bf16(int64_t rows, int64_t cols, const void* x, int dt, int64_t ldx, __nv_bfloat16* p1,
                __nv_bfloat16* p2, __nv_bfloat16* p3, int64_t ldp, cudaStream_t st);
// D += T, FP32 row-major
int add2d_f32(int64_t rows, int64_t cols, float* D, int64_t ldd, const float* T, int64_t ldt,
              cudaStream_t st);
// Cholesky G = L L^T of an r x r SPD matrix (row-major, ld), lower L in place,
// and Linv = L^{-1} (row-major, ldi).  dt: F32 or F64.  Breakdown -> status.
// Deflated columns (pivot <= tol * max diag) are flagged in defl[r] (may be
// nullptr) and get a unit L column; see fill_deflated.
// With defl == nullptr the caller cannot use a deflated factor: a deflated
// column then records SPM_EBREAKDOWN in *status.
// Cholesky + inverse in one cooperative kernel (r <= 8192); SPM_EUNSUPPORTED
// when it cannot be launched.
int cholesky_inv_coop(int64_t r, void* G, int64_t ldg, void* Linv, int64_t ldi, int dt, int* defl,
                      int* status, cudaStream_t st);
int cholesky_inv(int64_t r, void* G, int64_t ldg, void* Linv, int64_t ldi, int dt, int* defl,
                 int* status, cudaStream_t st);
// Replace flagged columns of X (rows x c) by random Gaussian columns.
int fill_deflated(int64_t rows, int64_t c, void* X, int64_t ldx, int dt, const int* defl,
                  uint32_t seed, cudaStream_t st);
// Add shift * I to the diagonal, where shift = coef * (sum of diag) (device-computed).
int add_trace_shift(int64_t r, void* G, int64_t ldg, int dt, double coef, cudaStream_t st);
// Symmetric eigendecomposition by parallel cyclic Jacobi: A (r x r, row-major,
// overwritten), V (r x r row-major eigenvectors in columns), lam (r) sorted
// descending, V columns permuted accordingly.  dt F32 or F64.
// sweeps (device int, may be nullptr): atomic max of the Jacobi sweeps executed.
int sym_eig(int64_t r, void* A, int64_t lda, void* V, int64_t ldv, void* lam, int dt, int* status,
            cudaStream_t st, int* sweeps = nullptr);
// out[j] = sqrt(sum_i X[i,j]^2) for columns (col = true) or rows (col = false), in FP64.
int norms(int64_t rows, int64_t cols, View X, bool by_col, double* out, cudaStream_t st);
// Descending order of x (r values; NaN last; ties by index): perm[pos] = i and
// xs[pos] = x[i] (device arrays).
int desc_order(int64_t r, const double* x, int* perm, double* xs, cudaStream_t st);
// dst line l = src line perm[l] for l < lines (rows when by_row, else columns;
// each line has len elements).  src and dst of the same type.
int gather_lines(int64_t lines, int64_t len, View src, MView dst, const int* perm, bool by_row,
                 cudaStream_t st);
// Scale rows (or columns) of X by s[i] (or 1/s[i] when inv).
int scale_lines(int64_t rows, int64_t cols, MView X, bool rows_not_cols, const double* s, bool inv,
                cudaStream_t st);
// Sum of squares of a strided view into *acc (device double, accumulated).
int sumsq(int64_t rows, int64_t cols, View X, double* acc, cudaStream_t st);
// Sign convention: for each column j < k of U (m x k), flip column j of U and
// row j of Vt (k x n) so that the largest-magnitude entry of U[:, j] is > 0.
int sign_fix(int64_t m, int64_t k, int64_t n, MView U, MView Vt, cudaStream_t st);
// Copy sigma (FP64 device) to the output dtype.
int copy_vec(int64_t n, const double* src, void* dst, int dt, cudaStream_t st);
// Symmetrise in place: A = (A + A^T) / 2.
int symmetrize(int64_t r, void* A, int64_t lda, int dt, cudaStream_t st);
// Eigenvector refinement (dense.cu), FP32 r x r arrays with ld r.  oa_update:
// from Gm = X^T X and S = X^T G X, the correction E of X <- X + X E (one
// Ogita-Aishima step; a pair whose first-order correction would exceed theta
// gets -Gm_ij / 2).  oa_keep_best: scores X by max_{i!=j} |S_ij| / sqrt(S_jj S_00)
// + max |Gm - I|; when the score beats *best (device), *best = score and
// Xbest = X (always on the first call).  mx: 2 words, zero on entry and on
// return; keep: 2 ints, zero before the first call.
int oa_update(int64_t r, const float* S, const float* Gm, float* E, double theta, cudaStream_t st);
int oa_keep_best(int64_t r, const float* S, const float* Gm, const float* X, float* Xbest,
                 unsigned long long* mx, double* best, int* keep, cudaStream_t st);
// Scan a strided view for NaN/Inf; sets *status to SPM_ENONFINITE.
int check_finite(int64_t rows, int64_t cols, View X, int* status, cudaStream_t st);

}  // namespace spm
