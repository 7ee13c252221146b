// C ABI entry points: Algorithm 1 (Sketch-Powered Range Finder), the
// Randomized SVD finish, Algorithm 2 (Sketch-Powered Low-Rank Factorization)
// and Algorithm 3 (Sketch-Powered Nystrom Approximation).
//
// Three precision modes share one schedule:
//   SPM_PREC_FP64  -- every product on CUDA cores in FP64 (the plain form);
//   SPM_PREC_FP32  -- the same on CUDA cores in FP32;
//   SPM_PREC_MIXED -- A~ in BF16, power products on tcgen05 tensor cores with
//                     FP32 accumulation; the products whose accuracy reaches the
//                     output (CholeskyQR Gram and triangular products, Q^T A,
//                     B B^T, U~^T B, Q U~) use split-precision hi*hi + hi*lo +
//                     lo*hi BF16 passes; small factorisations in FP32 (or FP64
//                     with opts->small_fp64).
// Re-orthonormalisation (Section 2): Z = orth(A~^T Y) after every A~^T product;
// the final basis is orth(Y).  In exact arithmetic this equals Algorithm 1.
#include <math.h>

#include <algorithm>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.cuh"

namespace spm {

std::atomic<unsigned long long> g_launches{0};

struct Call {
  cudaStream_t st;
  Arena ar;
  int prec = SPM_PREC_FP64;
  int adt = DT_F64;
  bool small64 = false;
  int final_passes = 3;
  int power_passes = 3;
  int eig_refine = 3;      // eigenvector refinement steps after the FP32 eigensolver (mixed)
  bool reorth = true;     // orthonormalise Z = A~^T Y after every A~^T product
  bool reorth_y = false;  // also orthonormalise Y before every A~^T product
  const void* omega = nullptr;
  int* status = nullptr;
  double* acc = nullptr;  // [0] = |A|_F^2, [1] = |B|_F^2
  bool want_fro = false;  // |A|_F is reported (info given): the sketch pass sums squares
  StageTimer timer;
  int cholqr_passes = 0;
  // A fed from the host (spm_rsvd_host): row chunks of feed_rows rows arrive
  // on another stream, chunk c usable on st after feed_ev[c]
  int feed_n = 0;
  int64_t feed_rows = 0;
  const cudaEvent_t* feed_ev = nullptr;
  // sparse input: A~ made beforehand (at_pre, dtype adt, ld at_pre_ld), and
  // B = Q^T A made by make_b(rf, B, ldb) in B's precision (FP32 in MIXED);
  // |A|_F is not formed (no_fro)
  const void* at_pre = nullptr;
  int64_t at_pre_ld = 0;
  std::function<int(const struct RF&, void*, int64_t)> make_b;
  bool no_fro = false;
  // the mixed finish's BF16 split of A (ld pad8(n)): requested by the caller
  // (want_asplit), written by the sketch pass where its kernel can (asplit)
  bool want_asplit = false;
  __nv_bfloat16* a_hi = nullptr;
  __nv_bfloat16* a_lo = nullptr;
  bool asplit = false;
  explicit Call(cudaStream_t s) : st(s), ar(s) { timer.stream = s; }
};

// Make st wait for every chunk of a host-fed A (a no-op otherwise).
static int await_feed(const Call& C) {
  for (int c = 0; c < C.feed_n; ++c) SPM_CUDA_TRY(cudaStreamWaitEvent(C.st, C.feed_ev[c], 0));
  return SPM_OK;
}

static int64_t pad8(int64_t x) { return round_up(x, 8); }

cudaMemPool_t lib_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[16] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    uint64_t keep = ~0ull;  // keep freed memory for the next call
    if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return nullptr;
    }
    pools[dev] = p;
  }
  return pools[dev];
}

// One non-blocking stream per device for host staging copies (kept for the
// life of the process).
static cudaStream_t copy_stream() {
  static std::mutex mu;
  static cudaStream_t cs[16] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!cs[dev] && cudaStreamCreateWithFlags(&cs[dev], cudaStreamNonBlocking) != cudaSuccess)
    cs[dev] = nullptr;
  return cs[dev];
}

static int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      sms = v;
    else
      return 152;
  }
  return sms;
}

// Split-K factor of a tensor-core product from a small cost model:
//   waves(sk) x (t0 + ceil(kt / sk) x tk) + [sk > 1] (t0 + sk M N 8 B / HBM)
// (waves of the tiles x splits work units over the SMs; a CTA's set-up t0,
// one 64-deep k-tile of a 128 x 256 tile in three passes tk; the split-K
// partials written and read back once).  Whole waves matter for the few
// large products (1000 x 16384 output tiles: 3.4 waves unsplit, 6.7 at two
// splits); the partials' traffic for the short-K ones.  sym: only the tiles a
// symmetric product computes (the 128-row tiles that reach the upper
// triangle) count.
int auto_splitk(int64_t M, int64_t N, int64_t K, bool sym) {
  const int BN = (N >= 192) ? 256 : 128;
  int64_t tiles = cdiv(M, 128) * cdiv(N, BN);
  if (sym) {
    const int64_t mt = cdiv(M, 128);
    tiles = 0;
    for (int64_t j = 0; j < cdiv(N, BN); ++j)
      for (int64_t i = 0; i < mt; ++i)
        if (i * 128 < (j + 1) * BN) tiles += 1;
  }
  const int64_t kt = cdiv(K, 64);
  const int64_t sms = sm_count();
  const double t0 = 3e-6, tk = 1.3e-6, hbm = 6.5e12;
  const int64_t skmax = max64(1, min64(kt / 4, 32));
  auto cost = [&](int64_t sk) {
    const double waves = (double)cdiv(tiles * sk, sms);
    double c = waves * (t0 + (double)cdiv(kt, sk) * tk);
    if (sk > 1) c += t0 + (double)sk * (double)M * (double)N * 8.0 / hbm;
    return c;
  };
  double cmin = cost(1);
  for (int64_t sk = 2; sk <= skmax; ++sk) cmin = std::min(cmin, cost(sk));
  // the fewest splits within 2% of the best (the model is coarse)
  for (int64_t sk = 1; sk <= skmax; ++sk)
    if (cost(sk) <= 1.02 * cmin) return (int)sk;
  return 1;
}

// ------------------------------------------------------------------ split-K autotuning
// With spm_set_autotune(1), the split-K of each tensor-core product shape class
// (M, N, K, passes, operand majors, symmetric output, device) is measured on its
// first use instead of taken from the cost model: every candidate (the model's
// pick and 1, 2, 4, 8, 16 splits, at most a quarter of the K tiles) runs twice on
// the call's stream, timed by CUDA events, the faster of each pair counts, and the
// fastest candidate is cached for the process and run once more, so that the
// product the caller gets is the chosen configuration's.  Tuning synchronises the
// stream; inside a stream capture the model's pick is used.
static int g_autotune = 0;
static std::mutex g_tune_mu;
static std::map<std::tuple<int64_t, int64_t, int64_t, int, int, int, int, int>, int> g_tune;

static int tuned_gemm(int64_t M, int64_t N, int64_t K, int npass, const TcOp* A, const TcOp* B,
                      float* D, int64_t d_rs, int64_t d_cs, bool sym, cudaStream_t st, int* status) {
  const int model = auto_splitk(M, N, K, sym);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (!g_autotune || cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return gemm_tc(M, N, K, npass, A, B, 1.0f, D, d_rs, d_cs, model, st, sym, status);
  int dev = 0;
  SPM_CUDA_TRY(cudaGetDevice(&dev));
  const auto key = std::make_tuple(M, N, K, npass, (int)A[0].mn_major, (int)B[0].mn_major, (int)sym, dev);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto f = g_tune.find(key);
    if (f != g_tune.end())
      return gemm_tc(M, N, K, npass, A, B, 1.0f, D, d_rs, d_cs, f->second, st, sym, status);
  }
  const int64_t kt = cdiv(K, 64);
  std::vector<int> cand{model};
  for (int c : {1, 2, 4, 8, 16})
    if ((c == 1 || c <= kt / 4) && std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
  cudaEvent_t e0, e1;
  SPM_CUDA_TRY(cudaEventCreate(&e0));
  SPM_CUDA_TRY(cudaEventCreate(&e1));
  int best = model;
  float best_ms = 1e30f;
  int rc = SPM_OK;
  for (int c : cand) {
    float ms = 1e30f;
    for (int rep = 0; rep < 2 && rc == SPM_OK; ++rep) {
      if (cudaEventRecord(e0, st) != cudaSuccess) rc = SPM_ECUDA;
      if (rc == SPM_OK) rc = gemm_tc(M, N, K, npass, A, B, 1.0f, D, d_rs, d_cs, c, st, sym, status);
      if (rc == SPM_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = SPM_ECUDA;
      if (rc == SPM_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = SPM_ECUDA;
      float t = 0.f;
      if (rc == SPM_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms = std::min(ms, t);
    }
    if (rc != SPM_OK) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SPM_TRY(rc);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[key] = best;
  }
  return gemm_tc(M, N, K, npass, A, B, 1.0f, D, d_rs, d_cs, best, st, sym, status);
}

// Split-precision tensor-core product: D = sum of npass terms over (hi, lo) pairs.
static int tc_split(int64_t M, int64_t N, int64_t K, const __nv_bfloat16* Ahi,
                    const __nv_bfloat16* Alo, int64_t lda, bool a_mn, const __nv_bfloat16* Bhi,
                    const __nv_bfloat16* Blo, int64_t ldb, bool b_mn, int npass, float* D,
                    int64_t d_rs, int64_t d_cs, cudaStream_t st, int* status, bool sym = false) {
  TcOp A[3] = {{Ahi, lda, a_mn}, {Ahi, lda, a_mn}, {Alo, lda, a_mn}};
  TcOp B[3] = {{Bhi, ldb, b_mn}, {Blo, ldb, b_mn}, {Bhi, ldb, b_mn}};
  return tuned_gemm(M, N, K, npass, A, B, D, d_rs, d_cs, sym, st, status);
}

// ------------------------------------------------------------------ CholeskyQR
// Relative diagonal shift of the first CholeskyQR pass (shifted CholeskyQR3).
// FP64 Gram: 11 (rows c + c (c + 1)) u, the bound of Fukaya et al. (2020);
// Gram formed from FP32 / split-BF16 data (relative error about 1e-5): 1e-4.
static double shift_coef(bool fp64_gram, int64_t rows, int64_t c) {
  if (fp64_gram) return 11.0 * ((double)rows * c + (double)c * (c + 1)) * 1.1102230246251565e-16;
  return 1e-4;
}

// Shifted CholeskyQR3 in FP64 on CUDA cores: X (rows x c, ld ldx) <- orth(X).
// The first pass adds a small multiple of trace(G) to the Gram diagonal, so a
// rank-deficient or ill-conditioned X never breaks the Cholesky factorisation;
// the next passes restore orthonormality to working precision.
static int orth_f64(Call& C, double* X, int64_t rows, int64_t c, int64_t ldx, int passes) {
  Arena ar(C.st);  // scratch of this call only (freed in stream order on return)
  SPM_ALLOC(ar, double, G, c * c);
  SPM_ALLOC(ar, double, Li, c * c);
  SPM_ALLOC(ar, double, Xn, rows * c);
  SPM_ALLOC(ar, int, defl, c);
  for (int ps = 0; ps < passes; ++ps) {
    SPM_TRY(gemm_simt(c, c, rows, 1.0, transpose(rowmajor(X, DT_F64, ldx)),
                      rowmajor(X, DT_F64, ldx), 0.0, mrowmajor(G, DT_F64, c), C.st));
    if (ps == 0)
      SPM_TRY(add_trace_shift(c, G, c, DT_F64, shift_coef(true, rows, c), C.st));
    SPM_TRY(cholesky_inv(c, G, c, Li, c, DT_F64, defl, C.status, C.st));
    SPM_TRY(gemm_simt(rows, c, c, 1.0, rowmajor(X, DT_F64, ldx), transpose(rowmajor(Li, DT_F64, c)),
                      0.0, mrowmajor(Xn, DT_F64, c), C.st));
    SPM_TRY(fill_deflated(rows, c, Xn, c, DT_F64, defl, 0x5EED0000u + ps, C.st));
    SPM_TRY(convert2d(rows, c, rowmajor(Xn, DT_F64, c), mrowmajor(X, DT_F64, ldx), C.st));
  }
  return SPM_OK;
}

// Shifted CholeskyQR on an FP32 matrix with the small factorisation in FP32 or
// FP64 and the Gram / triangular products on CUDA cores (used for the r1 x r2
// iterate Z and other small bases).  First pass shifted, then `passes - 1` plain.
static int orth_small_f32(Call& C, float* X, int64_t rows, int64_t c, int64_t ldx, int passes) {
  Arena ar(C.st);  // scratch of this call only (freed in stream order on return)
  const int sdt = C.small64 ? DT_F64 : DT_F32;
  const size_t es = dt_size(sdt);
  void* G = ar.alloc<unsigned char>(c * c * es);
  void* Li = ar.alloc<unsigned char>(c * c * es);
  float* Xn = ar.alloc<float>(rows * c);
  int* defl = ar.alloc<int>(c);
  if (!G || !Li || !Xn || !defl) return SPM_ENOMEM;
  for (int ps = 0; ps < passes; ++ps) {
    SPM_TRY(gemm_simt(c, c, rows, 1.0, transpose(rowmajor(X, DT_F32, ldx)),
                      rowmajor(X, DT_F32, ldx), 0.0, mrowmajor(G, sdt, c), C.st));
    if (ps == 0) SPM_TRY(add_trace_shift(c, G, c, sdt, shift_coef(false, rows, c), C.st));
    SPM_TRY(cholesky_inv(c, G, c, Li, c, sdt, defl, C.status, C.st));
    SPM_TRY(gemm_simt(rows, c, c, 1.0, rowmajor(X, DT_F32, ldx), transpose(rowmajor(Li, sdt, c)), 0.0,
                      mrowmajor(Xn, DT_F32, c), C.st));
    SPM_TRY(fill_deflated(rows, c, Xn, c, DT_F32, defl, 0x5EED0100u + ps, C.st));
    SPM_TRY(convert2d(rows, c, rowmajor(Xn, DT_F32, c), mrowmajor(X, DT_F32, ldx), C.st));
  }
  return SPM_OK;
}

// Shifted CholeskyQR (3 passes by default) of the tall m x c FP32 basis Y on
// tensor cores: Gram and Y R^{-1} as split-precision (3-pass) BF16 products.  On return Y holds Q and
// (Qhi, Qlo) its BF16 split (row-major, ld pad8(c)).
static int orth_big_mixed(Call& C, float* Y, int64_t m, int64_t c, int64_t ldy,
                          __nv_bfloat16* Qhi, __nv_bfloat16* Qlo, int passes = 3) {
  Arena ar(C.st);  // scratch of this call only (freed in stream order on return)
  const int sdt = C.small64 ? DT_F64 : DT_F32;
  const size_t es = dt_size(sdt);
  const int64_t cp = pad8(c);
  SPM_ALLOC(ar, float, G, c * c);
  void* Gs = ar.alloc<unsigned char>(c * c * es);
  void* Li = ar.alloc<unsigned char>(c * c * es);
  if (!Gs || !Li) return SPM_ENOMEM;
  SPM_ALLOC(ar, __nv_bfloat16, Lhi, c * cp);
  SPM_ALLOC(ar, __nv_bfloat16, Llo, c * cp);
  SPM_ALLOC(ar, int, defl, c);
  for (int ps = 0; ps < passes; ++ps) {
    SPM_TRY(split_bf16(m, c, rowmajor(Y, DT_F32, ldy), mrowmajor(Qhi, DT_BF16, cp),
                       mrowmajor(Qlo, DT_BF16, cp), C.st));
    // G = Y^T Y: A-op Y^T (M = c, K = m) and B-op (N = c, K = m) both MN-major
    SPM_TRY(tc_split(c, c, m, Qhi, Qlo, cp, true, Qhi, Qlo, cp, true, 3, G, c, 1, C.st, C.status, true));
    if (sdt == DT_F64)
      SPM_TRY(convert2d(c, c, rowmajor(G, DT_F32, c), mrowmajor(Gs, DT_F64, c), C.st));
    else
      SPM_TRY(convert2d(c, c, rowmajor(G, DT_F32, c), mrowmajor(Gs, DT_F32, c), C.st));
    if (ps == 0) SPM_TRY(add_trace_shift(c, Gs, c, sdt, shift_coef(false, m, c), C.st));
    SPM_TRY(cholesky_inv(c, Gs, c, Li, c, sdt, defl, C.status, C.st));
    // Y <- Y L^{-T}: A-op Y (M = m, K = c) K-major; B-op (N = c, K = c) element
    // (n, k) = Linv[n][k], i.e. Linv row-major is K-major.
    SPM_TRY(split_bf16(c, c, rowmajor(Li, sdt, c), mrowmajor(Lhi, DT_BF16, cp),
                       mrowmajor(Llo, DT_BF16, cp), C.st));
    SPM_TRY(tc_split(m, c, c, Qhi, Qlo, cp, false, Lhi, Llo, cp, false, 3, Y, ldy, 1, C.st, C.status));
    SPM_TRY(fill_deflated(m, c, Y, ldy, DT_F32, defl, 0x5EED0200u + ps, C.st));
    C.cholqr_passes++;
  }
  SPM_TRY(split_bf16(m, c, rowmajor(Y, DT_F32, ldy), mrowmajor(Qhi, DT_BF16, cp),
                     mrowmajor(Qlo, DT_BF16, cp), C.st));
  return SPM_OK;
}

// D = X Y^T from three-part BF16 splits of both operands, keeping the six
// terms of order >= 2^-16 (FP32-equivalent): (1,1) (1,2) (2,1) in one product,
// (1,3) (2,2) (3,1) in a second one added on.  T: scratch of M x N floats.
static int tc_six(int64_t M, int64_t N, int64_t K, const __nv_bfloat16* const* X, int64_t ldx,
                  bool x_mn, const __nv_bfloat16* const* Y, int64_t ldy, bool y_mn, float* D,
                  int64_t ldd, bool sym, float* T, cudaStream_t st, int* status) {
  TcOp a1[3] = {{X[0], ldx, x_mn}, {X[0], ldx, x_mn}, {X[1], ldx, x_mn}};
  TcOp b1[3] = {{Y[0], ldy, y_mn}, {Y[1], ldy, y_mn}, {Y[0], ldy, y_mn}};
  TcOp a2[3] = {{X[0], ldx, x_mn}, {X[1], ldx, x_mn}, {X[2], ldx, x_mn}};
  TcOp b2[3] = {{Y[2], ldy, y_mn}, {Y[1], ldy, y_mn}, {Y[0], ldy, y_mn}};
  SPM_TRY(tuned_gemm(M, N, K, 3, a1, b1, D, ldd, 1, sym, st, status));
  SPM_TRY(tuned_gemm(M, N, K, 3, a2, b2, T, N, 1, sym, st, status));
  return add2d_f32(M, N, D, ldd, T, N, st);
}

// Shifted CholeskyQR of the FP32 basis X (rows x c) on tensor cores with
// Ogita-Aishima refinement of the eigenvectors X (r x r, column i = vector i,
// row-major FP32) of the symmetric FP32 matrix G, `steps` updates: Gm = X^T X
// and S = X^T (G X) as FP32-equivalent six-term products (the residuals I - Gm
// and S - diag are of the order of the eigensolver's error, and have to be
// formed to the working precision's unit roundoff), then X <- X + X E (the
// correction is small: a three-term product).  Every estimate, the solver's
// own output first, is scored by the largest off-diagonal entry it leaves in
// U^T A V relative to sigma_1 plus its loss of orthonormality, and the best one
// is returned: a step that does not improve is discarded, so the refinement
// never leaves X worse by that measure.  All on the device, no host sync.
static int eig_refine_mixed(Call& C, int64_t r, const float* G, float* X, int steps) {
  if (steps <= 0) return SPM_OK;
  Arena ar(C.st);
  const int64_t rp = pad8(r);
  SPM_ALLOC(ar, __nv_bfloat16, g1, r * rp);
  SPM_ALLOC(ar, __nv_bfloat16, g2, r * rp);
  SPM_ALLOC(ar, __nv_bfloat16, g3, r * rp);
  SPM_ALLOC(ar, __nv_bfloat16, x1, r * rp);
  SPM_ALLOC(ar, __nv_bfloat16, x2, r * rp);
  SPM_ALLOC(ar, __nv_bfloat16, x3, r * rp);
  SPM_ALLOC(ar, __nv_bfloat16, p1, r * rp);
  SPM_ALLOC(ar, __nv_bfloat16, p2, r * rp);
  SPM_ALLOC(ar, __nv_bfloat16, p3, r * rp);
  SPM_ALLOC(ar, float, Gm, r * r);
  SPM_ALLOC(ar, float, P, r * r);
  SPM_ALLOC(ar, float, Sm, r * r);
  SPM_ALLOC(ar, float, E, r * r);
  SPM_ALLOC(ar, float, T, r * r);
  SPM_ALLOC(ar, float, Xbest, r * r);
  SPM_ALLOC(ar, unsigned long long, mx, 2);
  SPM_ALLOC(ar, double, best, 1);
  SPM_ALLOC(ar, int, keep, 2);
  const __nv_bfloat16* gs[3] = {g1, g2, g3};
  const __nv_bfloat16* xs[3] = {x1, x2, x3};
  const __nv_bfloat16* ps[3] = {p1, p2, p3};
  SPM_CUDA_TRY(cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned long long), C.st));
  SPM_CUDA_TRY(cudaMemsetAsync(keep, 0, 2 * sizeof(int), C.st));
  SPM_TRY(split3_bf16(r, r, G, DT_F32, r, g1, g2, g3, rp, C.st));
  for (int it = 0; it <= steps; ++it) {
    SPM_TRY(split3_bf16(r, r, X, DT_F32, r, x1, x2, x3, rp, C.st));
    // Gm = X^T X: both operands X^T (M = N = r, K = r), stored K x M: MN-major
    SPM_TRY(tc_six(r, r, r, xs, rp, true, xs, rp, true, Gm, r, true, T, C.st, C.status));
    // P = G X: A-op G (M = r, K = r) K-major; B-op X (N = r, K = r) stored K x N: MN-major
    SPM_TRY(tc_six(r, r, r, gs, rp, false, xs, rp, true, P, r, false, T, C.st, C.status));
    SPM_TRY(split3_bf16(r, r, P, DT_F32, r, p1, p2, p3, rp, C.st));
    // S = X^T P: A-op X^T (MN-major), B-op P (N = r, K = r) stored K x N: MN-major
    SPM_TRY(tc_six(r, r, r, xs, rp, true, ps, rp, true, Sm, r, false, T, C.st, C.status));
    SPM_TRY(oa_keep_best(r, Sm, Gm, X, Xbest, mx, best, keep, C.st));
    if (it == steps) break;
    SPM_TRY(oa_update(r, Sm, Gm, E, 0.25, C.st));
    // X <- X + X E: A-op X (M = r, K = r) K-major; B-op E (N = r, K = r) stored K x N: MN-major
    SPM_TRY(split_bf16(r, r, rowmajor(E, DT_F32, r), mrowmajor(p1, DT_BF16, rp),
                       mrowmajor(p2, DT_BF16, rp), C.st));
    SPM_TRY(tc_split(r, r, r, x1, x2, rp, false, p1, p2, rp, true, 3, T, r, 1, C.st, C.status));
    SPM_TRY(add2d_f32(r, r, X, r, T, r, C.st));
  }
  SPM_CUDA_TRY(cudaMemcpyAsync(X, Xbest, r * r * sizeof(float), cudaMemcpyDeviceToDevice, C.st));
  return SPM_OK;
}

// FP32-equivalent products (tc_six): the Gram X^T X and X L^{-T}.  For the
// sketch-side iterate Z = A~^T Y, conditioned like kappa(A~)^2, whose tail a
// two-part split resolves too coarsely (the leading singular values moved by
// ~1.6e-4 on the sigma_i = 1/i workload).  On return X holds Q and (Xhi, Xlo)
// its two-part split (row-major, ld pad8(c)).
static int orth_mixed6(Call& C, float* X, int64_t rows, int64_t c, int64_t ldx,
                       __nv_bfloat16* Xhi, __nv_bfloat16* Xlo, int passes) {
  Arena ar(C.st);  // scratch of this call only (freed in stream order on return)
  const int sdt = C.small64 ? DT_F64 : DT_F32;
  const size_t es = dt_size(sdt);
  const int64_t cp = pad8(c);
  SPM_ALLOC(ar, float, G, c * c);
  SPM_ALLOC(ar, float, T, max64(c, rows) * c);
  void* Gs = ar.alloc<unsigned char>(c * c * es);
  void* Li = ar.alloc<unsigned char>(c * c * es);
  if (!Gs || !Li) return SPM_ENOMEM;
  SPM_ALLOC(ar, __nv_bfloat16, X3, rows * cp);
  SPM_ALLOC(ar, __nv_bfloat16, L1, c * cp);
  SPM_ALLOC(ar, __nv_bfloat16, L2, c * cp);
  SPM_ALLOC(ar, __nv_bfloat16, L3, c * cp);
  SPM_ALLOC(ar, int, defl, c);
  const __nv_bfloat16* xs[3] = {Xhi, Xlo, X3};
  const __nv_bfloat16* ls[3] = {L1, L2, L3};
  for (int ps = 0; ps < passes; ++ps) {
    SPM_TRY(split3_bf16(rows, c, X, DT_F32, ldx, Xhi, Xlo, X3, cp, C.st));
    // G = X^T X: both operands X^T (M = N = c, K = rows), MN-major
    SPM_TRY(tc_six(c, c, rows, xs, cp, true, xs, cp, true, G, c, true, T, C.st, C.status));
    if (sdt == DT_F64)
      SPM_TRY(convert2d(c, c, rowmajor(G, DT_F32, c), mrowmajor(Gs, DT_F64, c), C.st));
    else
      SPM_TRY(convert2d(c, c, rowmajor(G, DT_F32, c), mrowmajor(Gs, DT_F32, c), C.st));
    if (ps == 0) SPM_TRY(add_trace_shift(c, Gs, c, sdt, shift_coef(false, rows, c), C.st));
    SPM_TRY(cholesky_inv(c, Gs, c, Li, c, sdt, defl, C.status, C.st));
    // X <- X L^{-T}: A-op X (M = rows, K = c) K-major; B-op L^{-1} row-major (K-major)
    SPM_TRY(split3_bf16(c, c, Li, sdt, c, L1, L2, L3, cp, C.st));
    SPM_TRY(tc_six(rows, c, c, xs, cp, false, ls, cp, false, X, ldx, false, T, C.st, C.status));
    SPM_TRY(fill_deflated(rows, c, X, ldx, DT_F32, defl, 0x5EED0400u + ps, C.st));
    C.cholqr_passes++;
  }
  SPM_TRY(split_bf16(rows, c, rowmajor(X, DT_F32, ldx), mrowmajor(Xhi, DT_BF16, cp),
                     mrowmajor(Xlo, DT_BF16, cp), C.st));
  return SPM_OK;
}

// ------------------------------------------------------------------ Algorithm 1
// Result of the range finder, kept on the device for the finishing steps.
struct RF {
  int64_t m = 0, r2 = 0;
  double* Q64 = nullptr;       // FP64 mode: m x r2 (ld r2)
  float* Q32 = nullptr;        // MIXED and FP32: m x r2 (ld r2)
  __nv_bfloat16* Qhi = nullptr;  // MIXED: BF16 split of Q (ld pad8(r2))
  __nv_bfloat16* Qlo = nullptr;
};

static void store_q(RF& out, double* Y) { out.Q64 = Y; }
static void store_q(RF& out, float* Y) { out.Q32 = Y; }
static const double* rf_q(const RF& rf, double*) { return rf.Q64; }
static const float* rf_q(const RF& rf, float*) { return rf.Q32; }
static int orth_simt(Call& C, double* X, int64_t rows, int64_t c, int64_t ldx, int passes) {
  return orth_f64(C, X, rows, c, ldx, passes);
}
static int orth_simt(Call& C, float* X, int64_t rows, int64_t c, int64_t ldx, int passes) {
  return orth_small_f32(C, X, rows, c, ldx, passes);
}

// Algorithm 1 on CUDA cores in one precision T (FP64: the plain form; FP32:
// every product and factorisation in FP32).
template <typename T>
static int range_finder_simt(Call& C, const spm_sketch* S, const void* A, int64_t m, int64_t lda,
                             int64_t r2, int q, uint64_t seed, RF& out) {
  const int64_t r1 = S->r1;
  const int dt = std::is_same<T, double>::value ? DT_F64 : DT_F32;
  SPM_ALLOC(C.ar, T, At, m * r1);
  SPM_ALLOC(C.ar, T, Om, r1 * r2);
  SPM_ALLOC(C.ar, T, Y, m * r2);
  SPM_ALLOC(C.ar, T, Z, r1 * r2);
  {
    StageScope sc(C.timer, SPM_STAGE_SKETCH);
    if (C.omega)
      SPM_TRY(convert2d(r1, r2, rowmajor(C.omega, C.adt, r2), mrowmajor(Om, dt, r2), C.st));
    else
      SPM_TRY(gaussian_dev(Om, dt, r1, r2, r2, seed, C.st));
  }
  {
    StageScope sc(C.timer, SPM_STAGE_APPLY);
    if (C.at_pre)
      SPM_TRY(convert2d(m, r1, rowmajor(C.at_pre, C.adt, C.at_pre_ld), mrowmajor(At, dt, r1), C.st));
    else
      SPM_TRY(sketch_apply_dev(S, A, C.adt, m, lda, At, dt, r1, C.want_fro ? C.acc : nullptr, C.st,
                               nullptr, C.status));
  }
  {
    StageScope sc(C.timer, SPM_STAGE_POWER);
    SPM_TRY(gemm_simt(m, r2, r1, 1.0, rowmajor(At, dt, r1), rowmajor(Om, dt, r2), 0.0,
                      mrowmajor(Y, dt, r2), C.st));
  }
  for (int t = 0; t < q; ++t) {
    if (C.reorth_y) {
      StageScope sc(C.timer, SPM_STAGE_ORTH);
      SPM_TRY(orth_simt(C, Y, m, r2, r2, 2));
    }
    {
      StageScope sc(C.timer, SPM_STAGE_POWER);
      SPM_TRY(gemm_simt(r1, r2, m, 1.0, transpose(rowmajor(At, dt, r1)),
                        rowmajor(Y, dt, r2), 0.0, mrowmajor(Z, dt, r2), C.st));
    }
    if (C.reorth) {
      StageScope sc(C.timer, SPM_STAGE_ORTH);
      SPM_TRY(orth_simt(C, Z, r1, r2, r2, 2));  // shifted pass + one plain pass
    }
    {
      StageScope sc(C.timer, SPM_STAGE_POWER);
      SPM_TRY(gemm_simt(m, r2, r1, 1.0, rowmajor(At, dt, r1), rowmajor(Z, dt, r2), 0.0,
                        mrowmajor(Y, dt, r2), C.st));
    }
  }
  {
    StageScope sc(C.timer, SPM_STAGE_ORTH);
    SPM_TRY(orth_simt(C, Y, m, r2, r2, 3));
    C.cholqr_passes = 3;
  }
  store_q(out, Y);
  return SPM_OK;
}

static int range_finder_core(Call& C, const spm_sketch* S, const void* A, int64_t m, int64_t lda,
                             int64_t r2, int q, uint64_t seed, RF& out) {
  const int64_t n = S->n, r1 = S->r1;
  out.m = m;
  out.r2 = r2;
  if (C.prec != SPM_PREC_MIXED) SPM_TRY(await_feed(C));
  if (C.prec == SPM_PREC_FP64) return range_finder_simt<double>(C, S, A, m, lda, r2, q, seed, out);
  if (C.prec == SPM_PREC_FP32) return range_finder_simt<float>(C, S, A, m, lda, r2, q, seed, out);
  // ---------------- mixed precision
  const int64_t r1p = pad8(r1), r2p = pad8(r2);
  const int pp = C.power_passes;
  SPM_ALLOC(C.ar, __nv_bfloat16, At, m * r1p);
  __nv_bfloat16* Atlo = nullptr;
  if (pp > 1) {
    Atlo = C.ar.alloc<__nv_bfloat16>(m * r1p);
    if (!Atlo) return SPM_ENOMEM;
  }
  SPM_ALLOC(C.ar, float, Om32, r1 * r2);
  SPM_ALLOC(C.ar, __nv_bfloat16, Zhi, r1 * r2p);
  SPM_ALLOC(C.ar, __nv_bfloat16, Zlo, r1 * r2p);
  SPM_ALLOC(C.ar, float, Y, m * r2);
  SPM_ALLOC(C.ar, float, Z, r1 * r2);
  SPM_ALLOC(C.ar, __nv_bfloat16, Qhi, m * r2p);   // also the BF16 split of Y between steps
  SPM_ALLOC(C.ar, __nv_bfloat16, Qlo, m * r2p);
  {
    StageScope sc(C.timer, SPM_STAGE_SKETCH);
    if (C.omega)
      SPM_TRY(convert2d(r1, r2, rowmajor(C.omega, C.adt, r2), mrowmajor(Om32, DT_F32, r2), C.st));
    else
      SPM_TRY(gaussian_dev(Om32, DT_F32, r1, r2, r2, seed, C.st));
    SPM_TRY(split_bf16(r1, r2, rowmajor(Om32, DT_F32, r2), mrowmajor(Zhi, DT_BF16, r2p),
                       mrowmajor(Zlo, DT_BF16, r2p), C.st));
  }
  // A's split for the projection, written by the sketch pass when its kernel can
  const int64_t np_ = pad8(n);
  if (C.want_asplit && !C.at_pre && C.adt == DT_F32) {
    C.a_hi = C.ar.alloc<__nv_bfloat16>(m * np_);
    C.a_lo = C.ar.alloc<__nv_bfloat16>(m * np_);
    if (!C.a_hi || !C.a_lo) return SPM_ENOMEM;
  }
  {
    StageScope sc(C.timer, SPM_STAGE_APPLY);
    if (C.at_pre) {
      const View src = rowmajor(C.at_pre, C.adt, C.at_pre_ld);
      if (Atlo)
        SPM_TRY(split_bf16(m, r1, src, mrowmajor(At, DT_BF16, r1p), mrowmajor(Atlo, DT_BF16, r1p), C.st));
      else
        SPM_TRY(convert2d(m, r1, src, mrowmajor(At, DT_BF16, r1p), C.st));
    } else if (C.feed_n > 0) {
      // host-fed A: each row chunk's sketch product as soon as the chunk is here
      const size_t es = dt_size(C.adt);
      bool all = C.a_hi != nullptr;
      for (int c = 0; c < C.feed_n; ++c) {
        const int64_t r0 = (int64_t)c * C.feed_rows, rows = min64(C.feed_rows, m - r0);
        SPM_CUDA_TRY(cudaStreamWaitEvent(C.st, C.feed_ev[c], 0));
        bool done = false;
        SPM_TRY(sketch_apply_dev(S, (const unsigned char*)A + (size_t)r0 * lda * es, C.adt, rows,
                                 lda, At + r0 * r1p, DT_BF16, r1p, C.want_fro ? C.acc : nullptr,
                                 C.st, Atlo ? Atlo + r0 * r1p : nullptr, C.status,
                                 C.a_hi ? C.a_hi + r0 * np_ : nullptr,
                                 C.a_lo ? C.a_lo + r0 * np_ : nullptr, np_, &done));
        all = all && done;
      }
      C.asplit = all;
    } else {
      SPM_TRY(sketch_apply_dev(S, A, C.adt, m, lda, At, DT_BF16, r1p, C.want_fro ? C.acc : nullptr,
                               C.st, Atlo, C.status, C.a_hi, C.a_lo, np_, &C.asplit));
    }
  }
  const __nv_bfloat16* Alo = Atlo ? Atlo : At;
  {
    // Y = A~ Omega: A-op A~ (M = m, K = r1) K-major; B-op Omega (N = r2, K = r1) MN-major
    StageScope sc(C.timer, SPM_STAGE_POWER);
    SPM_TRY(tc_split(m, r2, r1, At, Alo, r1p, false, Zhi, Zlo, r2p, true, pp, Y, r2, 1, C.st, C.status));
  }
  for (int t = 0; t < q; ++t) {
    if (C.reorth_y) {
      // Y <- orth(Y); (Qhi, Qlo) is then its split
      StageScope sc(C.timer, SPM_STAGE_ORTH);
      const int keep = C.cholqr_passes;
      SPM_TRY(orth_big_mixed(C, Y, m, r2, r2, Qhi, Qlo, 2));
      C.cholqr_passes = keep;
    }
    {
      // Z = A~^T Y: A-op A~^T (M = r1, K = m) MN-major; B-op Y (N = r2, K = m) MN-major
      StageScope sc(C.timer, SPM_STAGE_POWER);
      if (!C.reorth_y)
        SPM_TRY(split_bf16(m, r2, rowmajor(Y, DT_F32, r2), mrowmajor(Qhi, DT_BF16, r2p),
                           mrowmajor(Qlo, DT_BF16, r2p), C.st));
      SPM_TRY(tc_split(r1, r2, m, At, Alo, r1p, true, Qhi, Qlo, r2p, true, pp, Z, r2, 1, C.st, C.status));
    }
    if (C.reorth) {
      // Z <- orth(Z) on tensor cores with FP32-equivalent products (shifted
      // pass + one plain pass); (Zhi, Zlo) is then its split
      StageScope sc(C.timer, SPM_STAGE_ORTH);
      const int keep = C.cholqr_passes;
      SPM_TRY(orth_mixed6(C, Z, r1, r2, r2, Zhi, Zlo, 2));
      C.cholqr_passes = keep;
    }
    {
      StageScope sc(C.timer, SPM_STAGE_POWER);
      if (!C.reorth)
        SPM_TRY(split_bf16(r1, r2, rowmajor(Z, DT_F32, r2), mrowmajor(Zhi, DT_BF16, r2p),
                           mrowmajor(Zlo, DT_BF16, r2p), C.st));
      SPM_TRY(tc_split(m, r2, r1, At, Alo, r1p, false, Zhi, Zlo, r2p, true, pp, Y, r2, 1, C.st, C.status));
    }
  }
  {
    StageScope sc(C.timer, SPM_STAGE_ORTH);
    SPM_TRY(orth_big_mixed(C, Y, m, r2, r2, Qhi, Qlo));
  }
  out.Q32 = Y;
  out.Qhi = Qhi;
  out.Qlo = Qlo;
  return SPM_OK;
}

// ------------------------------------------------------------------ argument checks
static int check_common(const spm_sketch* S, const void* A, int32_t dtype, int64_t m, int64_t lda,
                        int64_t r2, int32_t q, const spm_opts* o) {
  if (!S || !A) return SPM_EINVAL;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_EINVAL;
  if (m < 1 || lda < S->n || r2 < 1 || r2 > S->r1 || r2 > m || q < 0) return SPM_EINVAL;
  if (o) {
    if (o->precision != SPM_PREC_FP64 && o->precision != SPM_PREC_MIXED &&
        o->precision != SPM_PREC_FP32)
      return SPM_EINVAL;
    if (o->final_passes != 0 && o->final_passes != 1 && o->final_passes != 3) return SPM_EINVAL;
    if (o->reorth < 0 || o->reorth > 2) return SPM_EINVAL;
    if (o->power_passes != 0 && o->power_passes != 1 && o->power_passes != 3) return SPM_EINVAL;
    if (o->eig_refine > 8) return SPM_EINVAL;
  }
  return SPM_OK;
}

static void setup_call(Call& C, int32_t dtype, const spm_opts* o, spm_info* info) {
  C.adt = dtype == SPM_F64 ? DT_F64 : DT_F32;
  if (o) {
    C.prec = o->precision;
    C.reorth = o->reorth != 0;
    C.reorth_y = o->reorth == 2;
    C.final_passes = o->final_passes == 0 ? 3 : o->final_passes;
    C.power_passes = o->power_passes == 0 ? 3 : o->power_passes;
    C.small64 = o->small_fp64 != 0;
    C.eig_refine = o->eig_refine == 0 ? 3 : (o->eig_refine < 0 ? 0 : o->eig_refine);
    C.omega = o->omega;
  }
  if (info && info->want_timing) C.timer.on = true;
  C.want_fro = info != nullptr && info->want_timing != 2;
}

static int prepare(Call& C) {
  C.status = C.ar.alloc<int>(4);  // [0] device status, [1] eigensolver sweeps
  C.acc = C.ar.alloc<double>(2);
  if (!C.status || !C.acc) return SPM_ENOMEM;
  SPM_CUDA_TRY(cudaMemsetAsync(C.status, 0, 4 * sizeof(int), C.st));
  SPM_CUDA_TRY(cudaMemsetAsync(C.acc, 0, 2 * sizeof(double), C.st));
  if (C.prec == SPM_PREC_MIXED && !tc_available()) return SPM_ECUDA;
  return SPM_OK;
}

static int finish(Call& C, spm_info* info, int rc, bool has_b) {
  if (rc != SPM_OK) return rc;
  if (!info) return SPM_OK;
  int stw[4] = {0, 0, 0, 0};
  double acc[2] = {0.0, 0.0};
  SPM_CUDA_TRY(cudaMemcpyAsync(stw, C.status, 4 * sizeof(int), cudaMemcpyDeviceToHost, C.st));
  SPM_CUDA_TRY(cudaMemcpyAsync(acc, C.acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, C.st));
  SPM_CUDA_TRY(cudaStreamSynchronize(C.st));
  for (int i = 0; i < SPM_NSTAGES; ++i) info->stage_ms[i] = 0.f;
  C.timer.collect(info->stage_ms);
  const int dst = stw[0];
  info->device_status = dst;
  info->eig_sweeps = stw[1];
  info->cholqr_passes = C.cholqr_passes;
  info->auto_q = -1;
  info->auto_fp32 = 0;
  info->a_split = C.asplit ? 1 : 0;
  const bool fro = !C.no_fro && C.want_fro;
  info->fro_a = fro ? sqrt(acc[0]) : -1.0;
  info->resid_est = (has_b && fro) ? sqrt(fmax(acc[0] - acc[1], 0.0)) : -1.0;
  return dst == 0 ? SPM_OK : dst;
}

// Write an FP32 or FP64 device matrix into the caller's buffer of dtype adt.
static int store_out(int64_t rows, int64_t cols, View src, void* dst, int adt, int64_t ld,
                     cudaStream_t st) {
  return convert2d(rows, cols, src, mrowmajor(dst, adt, ld), st);
}

// ------------------------------------------------------------------ RandSVD finish
// SVD of B = Q^T A on CUDA cores in one precision T.
template <typename T>
static int rsvd_finish_simt(Call& C, const void* A, int64_t m, int64_t n, int64_t lda, const RF& rf,
                            int64_t k, void* U, int64_t ldu, void* sigma, void* Vt, int64_t ldvt) {
  const int64_t r2 = rf.r2;
  const int edt = C.adt;
  const int dt = std::is_same<T, double>::value ? DT_F64 : DT_F32;
  const T* Q = rf_q(rf, (T*)nullptr);
  SPM_ALLOC(C.ar, T, B, r2 * n);
  SPM_ALLOC(C.ar, T, G, r2 * r2);
  SPM_ALLOC(C.ar, T, Ut, r2 * r2);
  SPM_ALLOC(C.ar, T, lam, r2);
  SPM_ALLOC(C.ar, T, W, r2 * n);
  SPM_ALLOC(C.ar, double, sig, r2);
  SPM_ALLOC(C.ar, T, Uo, m * k);
  SPM_ALLOC(C.ar, int, perm, r2);
  SPM_ALLOC(C.ar, double, sigs, r2);
  SPM_ALLOC(C.ar, T, Wk, k * n);
  SPM_ALLOC(C.ar, T, Utk, r2 * k);
  {
    StageScope sc(C.timer, SPM_STAGE_PROJECT);
    if (C.make_b)
      SPM_TRY(C.make_b(rf, B, n));
    else
      SPM_TRY(gemm_simt(r2, n, m, 1.0, transpose(rowmajor(Q, dt, r2)),
                        rowmajor(A, edt, lda), 0.0, mrowmajor(B, dt, n), C.st));
  }
  {
    StageScope sc(C.timer, SPM_STAGE_SMALL);
    SPM_TRY(sumsq(r2, n, rowmajor(B, dt, n), C.acc + 1, C.st));
    SPM_TRY(gemm_simt(r2, r2, n, 1.0, rowmajor(B, dt, n), transpose(rowmajor(B, dt, n)),
                      0.0, mrowmajor(G, dt, r2), C.st));
    SPM_TRY(symmetrize(r2, G, r2, dt, C.st));
    SPM_TRY(sym_eig(r2, G, r2, Ut, r2, lam, dt, C.status, C.st, C.status + 1));
  }
  {
    StageScope sc(C.timer, SPM_STAGE_FINISH);
    SPM_TRY(gemm_simt(r2, n, r2, 1.0, transpose(rowmajor(Ut, dt, r2)),
                      rowmajor(B, dt, n), 0.0, mrowmajor(W, dt, n), C.st));
    SPM_TRY(norms(r2, n, rowmajor(W, dt, n), false, sig, C.st));
    // sigma_i = |row i of W|, ordered by the eigenvalues; order them by their
    // own values (the two can swap neighbours that agree to rounding)
    SPM_TRY(desc_order(r2, sig, perm, sigs, C.st));
    SPM_TRY(gather_lines(k, n, rowmajor(W, dt, n), mrowmajor(Wk, dt, n), perm, true, C.st));
    SPM_TRY(gather_lines(k, r2, rowmajor(Ut, dt, r2), mrowmajor(Utk, dt, k), perm, false, C.st));
    SPM_TRY(scale_lines(k, n, mrowmajor(Wk, dt, n), true, sigs, true, C.st));
    SPM_TRY(gemm_simt(m, k, r2, 1.0, rowmajor(Q, dt, r2), rowmajor(Utk, dt, k), 0.0,
                      mrowmajor(Uo, dt, k), C.st));
    SPM_TRY(sign_fix(m, k, n, mrowmajor(Uo, dt, k), mrowmajor(Wk, dt, n), C.st));
    SPM_TRY(store_out(m, k, rowmajor(Uo, dt, k), U, edt, ldu, C.st));
    SPM_TRY(store_out(k, n, rowmajor(Wk, dt, n), Vt, edt, ldvt, C.st));
    SPM_TRY(copy_vec(k, sigs, sigma, edt, C.st));
  }
  return SPM_OK;
}

static int rsvd_finish(Call& C, const void* A, int64_t m, int64_t n, int64_t lda, const RF& rf,
                       int64_t k, void* U, int64_t ldu, void* sigma, void* Vt, int64_t ldvt) {
  const int64_t r2 = rf.r2;
  const int edt = C.adt;
  if (C.prec == SPM_PREC_FP64)
    return rsvd_finish_simt<double>(C, A, m, n, lda, rf, k, U, ldu, sigma, Vt, ldvt);
  if (C.prec == SPM_PREC_FP32)
    return rsvd_finish_simt<float>(C, A, m, n, lda, rf, k, U, ldu, sigma, Vt, ldvt);
  // ---------------- mixed precision
  const int64_t np_ = pad8(n), r2p = pad8(r2);
  const int sdt = C.small64 ? DT_F64 : DT_F32;
  const size_t es = dt_size(sdt);
  __nv_bfloat16 *Ahi = nullptr, *Alo = nullptr;
  if (!C.make_b && C.asplit) {
    Ahi = C.a_hi;  // written by the sketch pass
    Alo = C.a_lo;
  } else if (!C.make_b) {
    Ahi = C.a_hi ? C.a_hi : C.ar.alloc<__nv_bfloat16>(m * np_);
    Alo = C.a_lo ? C.a_lo : C.ar.alloc<__nv_bfloat16>(m * np_);
    if (!Ahi || !Alo) return SPM_ENOMEM;
  }
  SPM_ALLOC(C.ar, float, B, r2 * n);
  SPM_ALLOC(C.ar, __nv_bfloat16, Bhi, r2 * np_);
  SPM_ALLOC(C.ar, __nv_bfloat16, Blo, r2 * np_);
  SPM_ALLOC(C.ar, float, G, r2 * r2);
  void* Gs = C.ar.alloc<unsigned char>(r2 * r2 * es);
  void* Ut = C.ar.alloc<unsigned char>(r2 * r2 * es);
  void* lam = C.ar.alloc<unsigned char>(r2 * es);
  if (!Gs || !Ut || !lam) return SPM_ENOMEM;
  SPM_ALLOC(C.ar, __nv_bfloat16, Uhi, r2 * r2p);
  SPM_ALLOC(C.ar, __nv_bfloat16, Ulo, r2 * r2p);
  SPM_ALLOC(C.ar, float, W, r2 * n);
  SPM_ALLOC(C.ar, double, sig, r2);
  SPM_ALLOC(C.ar, float, Uo, m * k);
  const int64_t kp = pad8(k);
  SPM_ALLOC(C.ar, int, perm, r2);
  SPM_ALLOC(C.ar, double, sigs, r2);
  SPM_ALLOC(C.ar, float, Wk, k * n);
  SPM_ALLOC(C.ar, __nv_bfloat16, Ukhi, r2 * kp);
  SPM_ALLOC(C.ar, __nv_bfloat16, Uklo, r2 * kp);
  {
    StageScope sc(C.timer, SPM_STAGE_PROJECT);
    if (C.make_b) {
      SPM_TRY(C.make_b(rf, B, n));
    } else {
      if (!C.asplit)
        SPM_TRY(split_bf16(m, n, rowmajor(A, edt, lda), mrowmajor(Ahi, DT_BF16, np_),
                           mrowmajor(Alo, DT_BF16, np_), C.st));
      // B = Q^T A: A-op Q^T (M = r2, K = m) MN-major; B-op A (N = n, K = m) MN-major
      SPM_TRY(tc_split(r2, n, m, rf.Qhi, rf.Qlo, r2p, true, Ahi, Alo, np_, true, C.final_passes,
                       B, n, 1, C.st, C.status));
    }
  }
  {
    StageScope sc(C.timer, SPM_STAGE_SMALL);
    SPM_TRY(sumsq(r2, n, rowmajor(B, DT_F32, n), C.acc + 1, C.st));
    SPM_TRY(split_bf16(r2, n, rowmajor(B, DT_F32, n), mrowmajor(Bhi, DT_BF16, np_),
                       mrowmajor(Blo, DT_BF16, np_), C.st));
    // G = B B^T: both operands B (r2 x n), K-major
    SPM_TRY(tc_split(r2, r2, n, Bhi, Blo, np_, false, Bhi, Blo, np_, false, 3, G, r2, 1, C.st, C.status, true));
    SPM_TRY(convert2d(r2, r2, rowmajor(G, DT_F32, r2), mrowmajor(Gs, sdt, r2), C.st));
    SPM_TRY(symmetrize(r2, Gs, r2, sdt, C.st));
    SPM_TRY(sym_eig(r2, Gs, r2, Ut, r2, lam, sdt, C.status, C.st, C.status + 1));
    if (sdt == DT_F32) SPM_TRY(eig_refine_mixed(C, r2, (const float*)Gs, (float*)Ut, C.eig_refine));
    SPM_TRY(split_bf16(r2, r2, rowmajor(Ut, sdt, r2), mrowmajor(Uhi, DT_BF16, r2p),
                       mrowmajor(Ulo, DT_BF16, r2p), C.st));
  }
  {
    StageScope sc(C.timer, SPM_STAGE_FINISH);
    // W = U~^T B: A-op U~^T (M = r2, K = r2) MN-major; B-op B (N = n, K = r2) MN-major
    SPM_TRY(tc_split(r2, n, r2, Uhi, Ulo, r2p, true, Bhi, Blo, np_, true, 3, W, n, 1, C.st, C.status));
    SPM_TRY(norms(r2, n, rowmajor(W, DT_F32, n), false, sig, C.st));
    // sigma_i = |row i of W|, ordered by the eigenvalues; order them by their
    // own values (the two can swap neighbours that agree to rounding)
    SPM_TRY(desc_order(r2, sig, perm, sigs, C.st));
    SPM_TRY(gather_lines(k, n, rowmajor(W, DT_F32, n), mrowmajor(Wk, DT_F32, n), perm, true, C.st));
    SPM_TRY(gather_lines(k, r2, rowmajor(Uhi, DT_BF16, r2p), mrowmajor(Ukhi, DT_BF16, kp), perm,
                         false, C.st));
    SPM_TRY(gather_lines(k, r2, rowmajor(Ulo, DT_BF16, r2p), mrowmajor(Uklo, DT_BF16, kp), perm,
                         false, C.st));
    SPM_TRY(scale_lines(k, n, mrowmajor(Wk, DT_F32, n), true, sigs, true, C.st));
    // U = Q U~[:, :k]: A-op Q (M = m, K = r2) K-major; B-op U~ (N = k, K = r2) MN-major
    SPM_TRY(tc_split(m, k, r2, rf.Qhi, rf.Qlo, r2p, false, Ukhi, Uklo, kp, true, 3, Uo, k, 1, C.st, C.status));
    SPM_TRY(sign_fix(m, k, n, mrowmajor(Uo, DT_F32, k), mrowmajor(Wk, DT_F32, n), C.st));
    SPM_TRY(store_out(m, k, rowmajor(Uo, DT_F32, k), U, edt, ldu, C.st));
    SPM_TRY(store_out(k, n, rowmajor(Wk, DT_F32, n), Vt, edt, ldvt, C.st));
    SPM_TRY(copy_vec(k, sigs, sigma, edt, C.st));
  }
  return SPM_OK;
}

// spm_rsvd without any host synchronisation: the device status word of the
// call (0 or an SPM_E* code set by a kernel) is copied to dev_status (device,
// may be null) instead of being read back, so the call can be captured.
int rsvd_async(const spm_sketch* S, const void* A, int32_t dtype, int64_t m, int64_t lda, int64_t r2,
               int32_t q, uint64_t omega_seed, int64_t k, const spm_opts* opts, void* U, int64_t ldu,
               void* sigma, void* Vt, int64_t ldvt, int32_t* dev_status, cudaStream_t st) {
  SPM_TRY(check_common(S, A, dtype, m, lda, r2, q, opts));
  if (!U || !sigma || !Vt || k < 1 || k > r2 || ldu < k || ldvt < S->n) return SPM_EINVAL;
  Call C(st);
  setup_call(C, dtype, opts, nullptr);
  SPM_TRY(prepare(C));
  RF rf;
  C.want_asplit = C.prec == SPM_PREC_MIXED;
  SPM_TRY(range_finder_core(C, S, A, m, lda, r2, q, omega_seed, rf));
  SPM_TRY(rsvd_finish(C, A, m, S->n, lda, rf, k, U, ldu, sigma, Vt, ldvt));
  if (dev_status)
    SPM_CUDA_TRY(cudaMemcpyAsync(dev_status, C.status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  return SPM_OK;
}

}  // namespace spm

using namespace spm;

extern "C" {

int spm_version(void) { return 100; }

const char* spm_status_string(int s) {
  switch (s) {
    case SPM_OK: return "ok";
    case SPM_EINVAL: return "invalid argument";
    case SPM_ENOMEM: return "out of device memory";
    case SPM_ECUDA: return "CUDA error or no usable sm_103 device";
    case SPM_EBREAKDOWN: return "Cholesky breakdown";
    case SPM_ENONFINITE: return "non-finite value";
    case SPM_ETIMEOUT: return "bounded device wait expired";
    case SPM_EUNSUPPORTED: return "unsupported request";
    default: return "unknown status";
  }
}

int spm_device_ok(void) { return tc_available() ? 1 : 0; }

}  // extern "C"

namespace spm {
// `blocks` CTAs (co-resident: cooperative launch) meet at a counter that waits
// for blocks + extra arrivals; each waits at most `limit` clock cycles and then
// records SPM_ETIMEOUT and returns.
__global__ void k_selftest_wait(unsigned* count, unsigned expected, long long limit, int* status) {
  if (threadIdx.x != 0) return;
  atomicAdd(count, 1u);
  const long long t0 = clock64();
  while (atomicAdd(count, 0u) < expected) {
    if (clock64() - t0 > limit) {
      set_status(status, DEV_TIMEOUT);
      return;
    }
  }
}
}  // namespace spm

extern "C" {

int spm_selftest_bounded_wait(int32_t blocks, int32_t extra, int64_t limit_cycles, void* stream) {
  if (blocks < 1 || blocks > 1024 || extra < 0 || extra > 1024 || limit_cycles < 1 ||
      limit_cycles > ((int64_t)1 << 34))
    return SPM_EINVAL;
  cudaStream_t st = as_stream(stream);
  int dev = 0, coop = 0, sms = 0;
  SPM_CUDA_TRY(cudaGetDevice(&dev));
  SPM_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  SPM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (!coop || blocks > sms) return SPM_EUNSUPPORTED;
  Arena ar(st);
  SPM_ALLOC(ar, unsigned, count, 1);
  SPM_ALLOC(ar, int, status, 1);
  SPM_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(unsigned), st));
  SPM_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  unsigned expected = (unsigned)(blocks + extra);
  long long limit = (long long)limit_cycles;
  void* args[] = {(void*)&count, (void*)&expected, (void*)&limit, (void*)&status};
  SPM_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_selftest_wait, dim3((unsigned)blocks),
                                           dim3(32), args, 0, st));
  count_launch();
  int h = 0;
  SPM_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  SPM_CUDA_TRY(cudaStreamSynchronize(st));
  return h;
}

int spm_trim_memory(void) {
  cudaMemPool_t p = lib_pool();
  if (!p) return SPM_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return SPM_ECUDA;
  return cudaMemPoolTrimTo(p, 0) == cudaSuccess ? SPM_OK : SPM_ECUDA;
}

uint64_t spm_launch_count(void) { return (uint64_t)g_launches.load(); }

// The tensor maps of a product cover device memory of the current device only:
// p must be a device allocation of that device, or managed memory.
static bool on_current_device(const void* p) {
  int dev = 0;
  cudaPointerAttributes at{};
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error of an unknown pointer
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;  // migrates to the device that reads it
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

int spm_gemm_bf16(int64_t M, int64_t N, int64_t K, int32_t npass, const void* const* A,
                  int64_t lda, int32_t a_mn, const void* const* B, int64_t ldb, int32_t b_mn,
                  float* D, int64_t ldd, int32_t splitk, void* stream) {
  if (M < 1 || N < 1 || K < 1 || npass < 1 || npass > 3 || !A || !B || !D || ldd < N || splitk < 1)
    return SPM_EINVAL;
  if (!tc_available()) return SPM_ECUDA;
  TcOp a[3], b[3];
  if (!on_current_device(D)) return SPM_EINVAL;
  for (int q = 0; q < npass; ++q) {
    if (!A[q] || !B[q] || !on_current_device(A[q]) || !on_current_device(B[q])) return SPM_EINVAL;
    a[q] = TcOp{(const __nv_bfloat16*)A[q], lda, a_mn != 0};
    b[q] = TcOp{(const __nv_bfloat16*)B[q], ldb, b_mn != 0};
  }
  if (lda < (a_mn ? M : K) || ldb < (b_mn ? N : K)) return SPM_EINVAL;
  int* status = nullptr;
  SPM_TRY(gemm_public_status(&status));
  return gemm_tc(M, N, K, npass, a, b, 1.0f, D, ldd, 1, splitk, as_stream(stream), false, status);
}

int spm_range_finder(const spm_sketch* S, const void* A, int32_t dtype, int64_t m, int64_t lda,
                     int64_t r2, int32_t q, uint64_t omega_seed, const spm_opts* opts, void* Q,
                     int64_t ldq, spm_info* info, void* stream) {
  SPM_TRY(check_common(S, A, dtype, m, lda, r2, q, opts));
  if (!Q || ldq < r2) return SPM_EINVAL;
  Call C(as_stream(stream));
  setup_call(C, dtype, opts, info);
  SPM_TRY(prepare(C));
  RF rf;
  int rc = range_finder_core(C, S, A, m, lda, r2, q, omega_seed, rf);
  if (rc == SPM_OK) {
    if (C.prec == SPM_PREC_FP64)
      rc = store_out(m, r2, rowmajor(rf.Q64, DT_F64, r2), Q, C.adt, ldq, C.st);
    else
      rc = store_out(m, r2, rowmajor(rf.Q32, DT_F32, r2), Q, C.adt, ldq, C.st);
  }
  return finish(C, info, rc, false);
}

int spm_rsvd(const spm_sketch* S, const void* A, int32_t dtype, int64_t m, int64_t lda, int64_t r2,
             int32_t q, uint64_t omega_seed, int64_t k, const spm_opts* opts, void* U, int64_t ldu,
             void* sigma, void* Vt, int64_t ldvt, spm_info* info, void* stream) {
  SPM_TRY(check_common(S, A, dtype, m, lda, r2, q, opts));
  if (!U || !sigma || !Vt || k < 1 || k > r2 || ldu < k || ldvt < S->n) return SPM_EINVAL;
  Call C(as_stream(stream));
  setup_call(C, dtype, opts, info);
  SPM_TRY(prepare(C));
  RF rf;
  C.want_asplit = C.prec == SPM_PREC_MIXED;
  int rc = range_finder_core(C, S, A, m, lda, r2, q, omega_seed, rf);
  if (rc == SPM_OK) rc = rsvd_finish(C, A, m, S->n, lda, rf, k, U, ldu, sigma, Vt, ldvt);
  return finish(C, info, rc, true);
}

int spm_rsvd_host(const spm_sketch* S, const void* A, int32_t dtype, int64_t m, int64_t lda,
                  int64_t r2, int32_t q, uint64_t omega_seed, int64_t k, const spm_opts* opts,
                  void* U, int64_t ldu, void* sigma, void* Vt, int64_t ldvt, spm_info* info,
                  void* stream) {
  SPM_TRY(check_common(S, A, dtype, m, lda, r2, q, opts));
  if (!U || !sigma || !Vt || k < 1 || k > r2 || ldu < k || ldvt < S->n) return SPM_EINVAL;
  const int64_t n = S->n;
  const size_t es = dtype == SPM_F64 ? 8 : 4;
  cudaStream_t cs = copy_stream();
  if (!cs) return SPM_ECUDA;
  Call C(as_stream(stream));
  setup_call(C, dtype, opts, info);
  SPM_TRY(prepare(C));
  void* Ad = C.ar.alloc<unsigned char>((size_t)m * n * es);
  void* Ud = C.ar.alloc<unsigned char>((size_t)m * k * es);
  void* sd = C.ar.alloc<unsigned char>((size_t)k * es);
  void* Vd = C.ar.alloc<unsigned char>((size_t)k * n * es);
  if (!Ad || !Ud || !sd || !Vd) return SPM_ENOMEM;
  // row chunks (whole 32-row blocks of the sketch kernel), copied on cs once
  // the device buffer exists in C.st's order
  const int64_t rows = round_up(cdiv(m, min64(16, max64(1, cdiv(m, 1024)))), 32);
  const int nch = (int)cdiv(m, rows);
  std::vector<cudaEvent_t> ev(nch + 1, nullptr);
  int rc = SPM_OK;
  for (int c = 0; c <= nch && rc == SPM_OK; ++c)
    if (cudaEventCreateWithFlags(&ev[c], cudaEventDisableTiming) != cudaSuccess) rc = SPM_ECUDA;
  if (rc == SPM_OK && (cudaEventRecord(ev[nch], C.st) != cudaSuccess ||
                       cudaStreamWaitEvent(cs, ev[nch], 0) != cudaSuccess))
    rc = SPM_ECUDA;
  for (int c = 0; c < nch && rc == SPM_OK; ++c) {
    const int64_t r0 = (int64_t)c * rows, rc_rows = min64(rows, m - r0);
    if (cudaMemcpy2DAsync((unsigned char*)Ad + (size_t)r0 * n * es, n * es,
                          (const unsigned char*)A + (size_t)r0 * lda * es, lda * es, n * es,
                          rc_rows, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaEventRecord(ev[c], cs) != cudaSuccess)
      rc = SPM_ECUDA;
  }
  if (rc == SPM_OK) {
    C.feed_n = nch;
    C.feed_rows = rows;
    C.feed_ev = ev.data();
    RF rf;
    C.want_asplit = C.prec == SPM_PREC_MIXED;
    rc = range_finder_core(C, S, Ad, m, n, r2, q, omega_seed, rf);
    if (rc == SPM_OK) rc = rsvd_finish(C, Ad, m, n, n, rf, k, Ud, k, sd, Vd, n);
  }
  // the staged A and the events are released only after every copy is done
  const int wrc = await_feed(C);
  if (rc == SPM_OK) rc = wrc;
  if (rc == SPM_OK &&
      (cudaMemcpy2DAsync(U, ldu * es, Ud, k * es, k * es, m, cudaMemcpyDeviceToHost, C.st) !=
           cudaSuccess ||
       cudaMemcpyAsync(sigma, sd, k * es, cudaMemcpyDeviceToHost, C.st) != cudaSuccess ||
       cudaMemcpy2DAsync(Vt, ldvt * es, Vd, n * es, n * es, k, cudaMemcpyDeviceToHost, C.st) !=
           cudaSuccess))
    rc = SPM_ECUDA;
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  return finish(C, info, rc, true);
}

int spm_sketch_apply_csr(const spm_sketch* S, const spm_csr* A, int32_t dtype, void* out, int64_t ldo,
                         void* stream) {
  if (!S || !out || (dtype != SPM_F32 && dtype != SPM_F64)) return SPM_EINVAL;
  SPM_TRY(csr_check(A, S->n));
  if (ldo < S->r1) return SPM_EINVAL;
  return csr_sketch_dev(S, A, dtype == SPM_F64 ? DT_F64 : DT_F32, out, ldo, nullptr,
                        as_stream(stream));
}

int spm_rsvd_csr(const spm_sketch* S, const spm_csr* A, int32_t dtype, int64_t r2, int32_t q,
                 uint64_t omega_seed, int64_t k, const spm_opts* opts, void* U, int64_t ldu,
                 void* sigma, void* Vt, int64_t ldvt, spm_info* info, void* stream) {
  if (!S || !A) return SPM_EINVAL;
  SPM_TRY(csr_check(A, S->n));
  // the dense checks on a stand-in pointer (A itself is never read as dense)
  SPM_TRY(check_common(S, A, dtype, A->m, S->n, r2, q, opts));
  if (!U || !sigma || !Vt || k < 1 || k > r2 || ldu < k || ldvt < S->n) return SPM_EINVAL;
  const int64_t m = A->m, n = S->n, r1 = S->r1;
  Call C(as_stream(stream));
  setup_call(C, dtype, opts, info);
  const int qdt = C.prec == SPM_PREC_FP64 ? DT_F64 : DT_F32;
  if (qdt != C.adt) return SPM_EUNSUPPORTED;  // FP64 mode wants FP64 values, the others FP32
  SPM_TRY(prepare(C));
  // A~ in the call's type (FP32 in MIXED: split into BF16 by the range finder)
  void* At = C.ar.alloc<unsigned char>((size_t)m * r1 * dt_size(C.adt));
  if (!At) return SPM_ENOMEM;
  {
    StageScope sc(C.timer, SPM_STAGE_APPLY);
    SPM_TRY(csr_sketch_dev(S, A, C.adt, At, r1, C.status, C.st, C.prec == SPM_PREC_MIXED));
  }
  CscIndex csc{};
  SPM_TRY(csc_build(A, C.adt, C.ar, csc, C.st));
  C.at_pre = At;
  C.at_pre_ld = r1;
  C.no_fro = true;
  C.make_b = [&](const RF& rf, void* B, int64_t ldb) {
    const void* Q = qdt == DT_F64 ? (const void*)rf.Q64 : (const void*)rf.Q32;
    if (C.prec == SPM_PREC_MIXED)
      return csr_project_dev(A, csc, qdt, Q, rf.r2, rf.r2, B, ldb, C.st, rf.Qhi, rf.Qlo,
                             round_up(rf.r2, 8));
    return csr_project_dev(A, csc, qdt, Q, rf.r2, rf.r2, B, ldb, C.st);
  };
  RF rf;
  int rc = range_finder_core(C, S, At, m, r1, r2, q, omega_seed, rf);
  if (rc == SPM_OK) rc = rsvd_finish(C, nullptr, m, n, n, rf, k, U, ldu, sigma, Vt, ldvt);
  return finish(C, info, rc, true);
}

int spm_lowrank(const spm_sketch* S1, const spm_sketch* S2, const void* A, int32_t dtype,
                int64_t m, int64_t lda, int64_t r2, int32_t q, uint64_t omega_seed,
                const spm_opts* opts, void* Y, int64_t ldy, void* X, int64_t ldx, spm_info* info,
                void* stream) {
  SPM_TRY(check_common(S1, A, dtype, m, lda, r2, q, opts));
  if (!S2 || S2->n != m || S2->r1 < r2 || !Y || !X || ldy < r2 || ldx < S1->n) return SPM_EINVAL;
  Call C(as_stream(stream));
  setup_call(C, dtype, opts, info);
  SPM_TRY(prepare(C));
  const int64_t n = S1->n, r1b = S2->r1;
  RF rf;
  int rc = range_finder_core(C, S1, A, m, lda, r2, q, omega_seed, rf);
  if (rc != SPM_OK) return finish(C, info, rc, false);
  // X = (S2^T Q)^+ (S2^T A) via CholeskyQR2 of M = S2^T Q: M = QM R, X = R^{-1} QM^T N
  const bool f64 = C.prec == SPM_PREC_FP64;
  const int wdt = f64 ? DT_F64 : DT_F32;
  const size_t es = dt_size(wdt);
  void* M = C.ar.alloc<unsigned char>(r1b * r2 * es);
  void* N = C.ar.alloc<unsigned char>(r1b * n * es);
  void* T1 = C.ar.alloc<unsigned char>(r2 * n * es);
  void* T2 = C.ar.alloc<unsigned char>(r2 * n * es);
  void* G = C.ar.alloc<unsigned char>(r2 * r2 * es);
  void* L1 = C.ar.alloc<unsigned char>(r2 * r2 * es);
  void* L2 = C.ar.alloc<unsigned char>(r2 * r2 * es);
  void* Mn = C.ar.alloc<unsigned char>(r1b * r2 * es);
  if (!M || !N || !T1 || !T2 || !G || !L1 || !L2 || !Mn) return finish(C, info, SPM_ENOMEM, false);
  do {
    {
      StageScope sc(C.timer, SPM_STAGE_PROJECT);
      const void* Qp = f64 ? (const void*)rf.Q64 : (const void*)rf.Q32;
      rc = sketch_apply_t_dev(S2, Qp, wdt, r2, r2, M, wdt, r2, C.st);
      if (rc) break;
      rc = sketch_apply_t_dev(S2, A, C.adt, n, lda, N, wdt, n, C.st);
      if (rc) break;
    }
    StageScope sc(C.timer, SPM_STAGE_SMALL);
    void* Ls[2] = {L1, L2};
    for (int ps = 0; ps < 2 && rc == SPM_OK; ++ps) {
      rc = gemm_simt(r2, r2, r1b, 1.0, transpose(rowmajor(M, wdt, r2)), rowmajor(M, wdt, r2), 0.0,
                     mrowmajor(G, wdt, r2), C.st);
      if (rc) break;
      rc = cholesky_inv(r2, G, r2, Ls[ps], r2, wdt, nullptr, C.status, C.st);
      if (rc) break;
      rc = gemm_simt(r1b, r2, r2, 1.0, rowmajor(M, wdt, r2), transpose(rowmajor(Ls[ps], wdt, r2)),
                     0.0, mrowmajor(Mn, wdt, r2), C.st);
      if (rc) break;
      rc = convert2d(r1b, r2, rowmajor(Mn, wdt, r2), mrowmajor(M, wdt, r2), C.st);
    }
    if (rc) break;
    // T1 = QM^T N ; T2 = L2^{-T} T1 ; T1 = L1^{-T} T2
    rc = gemm_simt(r2, n, r1b, 1.0, transpose(rowmajor(M, wdt, r2)), rowmajor(N, wdt, n), 0.0,
                   mrowmajor(T1, wdt, n), C.st);
    if (rc) break;
    rc = gemm_simt(r2, n, r2, 1.0, transpose(rowmajor(L2, wdt, r2)), rowmajor(T1, wdt, n), 0.0,
                   mrowmajor(T2, wdt, n), C.st);
    if (rc) break;
    rc = gemm_simt(r2, n, r2, 1.0, transpose(rowmajor(L1, wdt, r2)), rowmajor(T2, wdt, n), 0.0,
                   mrowmajor(T1, wdt, n), C.st);
    if (rc) break;
    StageScope sc2(C.timer, SPM_STAGE_FINISH);
    rc = store_out(r2, n, rowmajor(T1, wdt, n), X, C.adt, ldx, C.st);
    if (rc) break;
    if (f64)
      rc = store_out(m, r2, rowmajor(rf.Q64, DT_F64, r2), Y, C.adt, ldy, C.st);
    else
      rc = store_out(m, r2, rowmajor(rf.Q32, DT_F32, r2), Y, C.adt, ldy, C.st);
  } while (0);
  return finish(C, info, rc, false);
}

}  // extern "C"

namespace spm {

// Algorithm 3 up to C: C~ = A S (n x r1), W~ = S^T C~ (r1 x r1, symmetrised),
// Y = W~^q Omega (r1 x r2, re-orthonormalised between the q products) and
// C = C~ Y (n x r2), in the working type wdt (FP64 in FP64 mode, else FP32).
// In mixed precision C = C~ Y is a split-BF16 tensor-core product.
struct Nys {
  void* Ct = nullptr;  // n x r1
  void* Wt = nullptr;  // r1 x r1
  void* Y = nullptr;   // r1 x r2
  void* C = nullptr;   // n x r2
  int wdt = DT_F64;
};

// The Gaussian kernel matrix of a point set, generated inside the first product
// (A = nullptr in nystrom_core): K[i, j] = exp(-|x_i - x_j|^2 / (2 h^2)).
struct GaussSrc {
  const void* X;
  int64_t d, ldx;
  double h;
};

static int nystrom_core(Call& C, const spm_sketch* S, const void* A, int64_t n, int64_t lda,
                        int64_t r2, int q, uint64_t omega_seed, Nys& o,
                        const GaussSrc* gs = nullptr) {
  const int64_t r1 = S->r1;
  const bool f64 = C.prec == SPM_PREC_FP64;
  const int wdt = f64 ? DT_F64 : DT_F32;
  const size_t es = dt_size(wdt);
  o.wdt = wdt;
  o.Ct = C.ar.alloc<unsigned char>(n * r1 * es);
  o.Wt = C.ar.alloc<unsigned char>(r1 * r1 * es);
  o.Y = C.ar.alloc<unsigned char>(r1 * r2 * es);
  o.C = C.ar.alloc<unsigned char>(n * r2 * es);
  void* Yn = C.ar.alloc<unsigned char>(r1 * r2 * es);
  if (!o.Ct || !o.Wt || !o.Y || !o.C || !Yn) return SPM_ENOMEM;
  {
    StageScope sc(C.timer, SPM_STAGE_SKETCH);
    if (C.omega)
      SPM_TRY(convert2d(r1, r2, rowmajor(C.omega, C.adt, r2), mrowmajor(o.Y, wdt, r2), C.st));
    else
      SPM_TRY(gaussian_dev(o.Y, wdt, r1, r2, r2, omega_seed, C.st));
  }
  {
    StageScope sc(C.timer, SPM_STAGE_APPLY);
    if (gs)                                                               // C~ = K S
      SPM_TRY(gauss_sketch_dev(S, gs->X, C.adt, n, gs->d, gs->ldx, gs->h, o.Ct, wdt, r1, C.st,
                               C.status));
    else
      SPM_TRY(sketch_apply_dev(S, A, C.adt, n, lda, o.Ct, wdt, r1, C.want_fro ? C.acc : nullptr,
                               C.st, nullptr, C.status));                // C~ = A S
    SPM_TRY(sketch_apply_t_dev(S, o.Ct, wdt, r1, r1, o.Wt, wdt, r1, C.st));  // W~ = S^T C~
    SPM_TRY(symmetrize(r1, o.Wt, r1, wdt, C.st));
  }
  for (int t = 0; t < q; ++t) {
    StageScope sc(C.timer, SPM_STAGE_POWER);
    SPM_TRY(gemm_simt(r1, r2, r1, 1.0, rowmajor(o.Wt, wdt, r1), rowmajor(o.Y, wdt, r2), 0.0,
                      mrowmajor(Yn, wdt, r2), C.st));
    SPM_TRY(convert2d(r1, r2, rowmajor(Yn, wdt, r2), mrowmajor(o.Y, wdt, r2), C.st));
    if (C.reorth) {
      if (f64)
        SPM_TRY(orth_f64(C, (double*)o.Y, r1, r2, r2, 3));
      else
        SPM_TRY(orth_small_f32(C, (float*)o.Y, r1, r2, r2, 3));
    }
  }
  StageScope sc(C.timer, SPM_STAGE_PROJECT);
  if (C.prec == SPM_PREC_MIXED) {
    // C = C~ Y as hi*hi + hi*lo + lo*hi BF16 products: A-op C~ (M = n, K = r1)
    // K-major; B-op Y (N = r2, K = r1) stored K x N, MN-major
    const int64_t r1p = pad8(r1), r2p = pad8(r2);
    Arena ar(C.st);
    SPM_ALLOC(ar, __nv_bfloat16, Chi, n * r1p);
    SPM_ALLOC(ar, __nv_bfloat16, Clo, n * r1p);
    SPM_ALLOC(ar, __nv_bfloat16, Yhi, r1 * r2p);
    SPM_ALLOC(ar, __nv_bfloat16, Ylo, r1 * r2p);
    SPM_TRY(split_bf16(n, r1, rowmajor(o.Ct, DT_F32, r1), mrowmajor(Chi, DT_BF16, r1p),
                       mrowmajor(Clo, DT_BF16, r1p), C.st));
    SPM_TRY(split_bf16(r1, r2, rowmajor(o.Y, DT_F32, r2), mrowmajor(Yhi, DT_BF16, r2p),
                       mrowmajor(Ylo, DT_BF16, r2p), C.st));
    SPM_TRY(tc_split(n, r2, r1, Chi, Clo, r1p, false, Yhi, Ylo, r2p, true, 3, (float*)o.C, r2, 1,
                     C.st, C.status));
  } else {
    SPM_TRY(gemm_simt(n, r2, r1, 1.0, rowmajor(o.Ct, wdt, r1), rowmajor(o.Y, wdt, r2), 0.0,
                      mrowmajor(o.C, wdt, r2), C.st));
  }
  return SPM_OK;
}

// D (M x N, FP32) = X^T Y or X Y (op_x = true for X^T) as split-BF16 tensor-core
// products of FP32 operands; `sym` for a symmetric result (X^T X).
static int tc_f32(Call& C, int64_t M, int64_t N, int64_t K, const float* X, int64_t ldx, bool xt,
                  const float* Yp, int64_t ldy, bool yt, float* D, int64_t ldd, bool sym = false) {
  // A-op (M x K): X^T stored K x M (MN-major) or X stored M x K (K-major)
  // B-op (N x K): Y stored K x N (MN-major) unless yt: Y^T, i.e. Y stored N x K
  Arena ar(C.st);
  const int64_t xr = xt ? K : M, xc = xt ? M : K, yr = yt ? N : K, yc = yt ? K : N;
  const int64_t xcp = pad8(xc), ycp = pad8(yc);
  SPM_ALLOC(ar, __nv_bfloat16, Xh, xr * xcp);
  SPM_ALLOC(ar, __nv_bfloat16, Xl, xr * xcp);
  SPM_TRY(split_bf16(xr, xc, rowmajor(X, DT_F32, ldx), mrowmajor(Xh, DT_BF16, xcp),
                     mrowmajor(Xl, DT_BF16, xcp), C.st));
  const __nv_bfloat16 *Yh = Xh, *Yl = Xl;
  if (Yp != X || yr != xr || yc != xc) {
    __nv_bfloat16* h = ar.alloc<__nv_bfloat16>(yr * ycp);
    __nv_bfloat16* l = ar.alloc<__nv_bfloat16>(yr * ycp);
    if (!h || !l) return SPM_ENOMEM;
    SPM_TRY(split_bf16(yr, yc, rowmajor(Yp, DT_F32, ldy), mrowmajor(h, DT_BF16, ycp),
                       mrowmajor(l, DT_BF16, ycp), C.st));
    Yh = h;
    Yl = l;
  }
  return tc_split(M, N, K, Xh, Xl, xcp, xt, Yh, Yl, ycp, !yt, 3, D, ldd, 1, C.st, C.status, sym);
}

// Factored Nystrom finish: U (n x r2) and lam (r2) with A_hat = U diag(lam) U^T
// (see nystrom.cu for the construction).  The Cholesky of W_nu is FP64 in every mode.
static int nystrom_eig_finish(Call& C, const spm_sketch* S, Nys& o, int64_t n, int64_t r2, void* Uout,
                              int64_t ldu, void* lam_out) {
  const int wdt = o.wdt;
  const size_t es = dt_size(wdt);
  const bool mixed = C.prec == SPM_PREC_MIXED;
  const int sdt = (C.prec == SPM_PREC_FP64 || C.small64) ? DT_F64 : DT_F32;
  Arena ar(C.st);
  void* T = ar.alloc<unsigned char>(n * r2 * es);
  void* F = ar.alloc<unsigned char>(n * r2 * es);
  void* U = ar.alloc<unsigned char>(n * r2 * es);
  double* Wn = ar.alloc<double>(r2 * r2);
  double* Li = ar.alloc<double>(r2 * r2);
  void* Lw = ar.alloc<unsigned char>(r2 * r2 * es);
  void* G = ar.alloc<unsigned char>(r2 * r2 * es);
  void* Gs = ar.alloc<unsigned char>(r2 * r2 * dt_size(sdt));
  void* V = ar.alloc<unsigned char>(r2 * r2 * dt_size(sdt));
  void* Vw = ar.alloc<unsigned char>(r2 * r2 * es);
  void* sig2 = ar.alloc<unsigned char>(r2 * dt_size(sdt));
  double* scal = ar.alloc<double>(4);  // [0] |C|_F^2, [1] nu
  double* sigma = ar.alloc<double>(r2);
  if (!T || !F || !U || !Wn || !Li || !Lw || !G || !Gs || !V || !Vw || !sig2 || !scal || !sigma)
    return SPM_ENOMEM;
  {
    StageScope sc(C.timer, SPM_STAGE_SMALL);
    SPM_CUDA_TRY(cudaMemsetAsync(scal, 0, 4 * sizeof(double), C.st));
    SPM_TRY(sketch_left_dev(S, o.Y, wdt, r2, r2, T, r2, C.st));     // T = S Y: C = A T
    SPM_TRY(sumsq(n, r2, rowmajor(o.C, wdt, r2), scal, C.st));
    SPM_TRY(nys_shift_dev(n, r2, o.C, r2, T, r2, wdt, scal, scal + 1, C.st));  // C_nu = C + nu T
    // W_nu = T^T C_nu (r2 x r2), symmetrised, in FP64
    if (mixed) {
      SPM_TRY(tc_f32(C, r2, r2, n, (const float*)T, r2, true, (const float*)o.C, r2, false, (float*)G,
                     r2));
      SPM_TRY(convert2d(r2, r2, rowmajor(G, DT_F32, r2), mrowmajor(Wn, DT_F64, r2), C.st));
    } else {
      SPM_TRY(gemm_simt(r2, r2, n, 1.0, transpose(rowmajor(T, wdt, r2)), rowmajor(o.C, wdt, r2), 0.0,
                        mrowmajor(Wn, DT_F64, r2), C.st));
    }
    SPM_TRY(symmetrize(r2, Wn, r2, DT_F64, C.st));
    SPM_TRY(cholesky_inv(r2, Wn, r2, Li, r2, DT_F64, nullptr, C.status, C.st));  // L L^T = W_nu
  }
  {
    StageScope sc(C.timer, SPM_STAGE_FINISH);
    // F = C_nu L^{-T}
    if (mixed) {
      SPM_TRY(convert2d(r2, r2, rowmajor(Li, DT_F64, r2), mrowmajor(Lw, DT_F32, r2), C.st));
      SPM_TRY(tc_f32(C, n, r2, r2, (const float*)o.C, r2, false, (const float*)Lw, r2, true, (float*)F,
                     r2));
    } else {
      SPM_TRY(gemm_simt(n, r2, r2, 1.0, rowmajor(o.C, wdt, r2), transpose(rowmajor(Li, DT_F64, r2)),
                        0.0, mrowmajor(F, wdt, r2), C.st));
    }
    // F = Q_F R with Q_F orthonormal (shifted CholeskyQR3, in place); R = Q_F^T F
    SPM_TRY(convert2d(n, r2, rowmajor(F, wdt, r2), mrowmajor(U, wdt, r2), C.st));  // keep F
    if (mixed) {
      const int64_t r2p = pad8(r2);
      __nv_bfloat16* Qh = ar.alloc<__nv_bfloat16>(n * r2p);
      __nv_bfloat16* Ql = ar.alloc<__nv_bfloat16>(n * r2p);
      if (!Qh || !Ql) return SPM_ENOMEM;
      SPM_TRY(orth_big_mixed(C, (float*)F, n, r2, r2, Qh, Ql));
      SPM_TRY(tc_f32(C, r2, r2, n, (const float*)F, r2, true, (const float*)U, r2, false, (float*)G, r2));
    } else {
      if (wdt == DT_F64)
        SPM_TRY(orth_f64(C, (double*)F, n, r2, r2, 3));
      else
        SPM_TRY(orth_small_f32(C, (float*)F, n, r2, r2, 3));
      SPM_TRY(gemm_simt(r2, r2, n, 1.0, transpose(rowmajor(F, wdt, r2)), rowmajor(U, wdt, r2), 0.0,
                        mrowmajor(G, wdt, r2), C.st));
    }
    // R R^T = U~ diag(sig2) U~^T (small, in sdt): F = Q_F U~ Sigma V^T
    SPM_TRY(convert2d(r2, r2, rowmajor(G, wdt, r2), mrowmajor(Lw, wdt, r2), C.st));
    SPM_TRY(gemm_simt(r2, r2, r2, 1.0, rowmajor(Lw, wdt, r2), transpose(rowmajor(Lw, wdt, r2)), 0.0,
                      mrowmajor(Gs, sdt, r2), C.st));
    SPM_TRY(symmetrize(r2, Gs, r2, sdt, C.st));
    SPM_TRY(sym_eig(r2, Gs, r2, V, r2, sig2, sdt, C.status, C.st, C.status + 1));
    // U = Q_F U~, lam = max(sig2 - nu, 0)
    SPM_TRY(convert2d(r2, r2, rowmajor(V, sdt, r2), mrowmajor(Vw, wdt, r2), C.st));
    if (mixed)
      SPM_TRY(tc_f32(C, n, r2, r2, (const float*)F, r2, false, (const float*)Vw, r2, false, (float*)U,
                     r2));
    else
      SPM_TRY(gemm_simt(n, r2, r2, 1.0, rowmajor(F, wdt, r2), rowmajor(Vw, wdt, r2), 0.0,
                        mrowmajor(U, wdt, r2), C.st));
    SPM_TRY(nys_lambda_dev(r2, sig2, sdt, scal + 1, sigma, lam_out, C.adt, C.st));
    SPM_TRY(sign_fix(n, r2, 0, mrowmajor(U, wdt, r2), mrowmajor(U, wdt, r2), C.st));
    SPM_TRY(store_out(n, r2, rowmajor(U, wdt, r2), Uout, C.adt, ldu, C.st));
  }
  return SPM_OK;
}

}  // namespace spm

extern "C" {

int spm_nystrom(const spm_sketch* S, const void* A, int32_t dtype, int64_t n, int64_t lda,
                int64_t r2, int32_t q, uint64_t omega_seed, const spm_opts* opts, void* Cout,
                int64_t ldc, void* Wout, int64_t ldw, spm_info* info, void* stream) {
  SPM_TRY(check_common(S, A, dtype, n, lda, r2, q, opts));
  if (S->n != n || !Cout || !Wout || ldc < r2 || ldw < r2) return SPM_EINVAL;
  Call C(as_stream(stream));
  setup_call(C, dtype, opts, info);
  SPM_TRY(prepare(C));
  const int64_t r1 = S->r1;
  Nys o;
  int rc = nystrom_core(C, S, A, n, lda, r2, q, omega_seed, o);
  if (rc != SPM_OK) return finish(C, info, rc, false);
  const int wdt = o.wdt;
  const size_t es = dt_size(wdt);
  void* T = C.ar.alloc<unsigned char>(r1 * r2 * es);
  void* Ww = C.ar.alloc<unsigned char>(r2 * r2 * es);
  if (!T || !Ww) return finish(C, info, SPM_ENOMEM, false);
  do {
    StageScope sc(C.timer, SPM_STAGE_FINISH);
    rc = gemm_simt(r1, r2, r1, 1.0, rowmajor(o.Wt, wdt, r1), rowmajor(o.Y, wdt, r2), 0.0,
                   mrowmajor(T, wdt, r2), C.st);
    if (rc) break;
    rc = gemm_simt(r2, r2, r1, 1.0, transpose(rowmajor(o.Y, wdt, r2)), rowmajor(T, wdt, r2), 0.0,
                   mrowmajor(Ww, wdt, r2), C.st);  // W = Y^T W~ Y
    if (rc) break;
    rc = symmetrize(r2, Ww, r2, wdt, C.st);
    if (rc) break;
    rc = store_out(n, r2, rowmajor(o.C, wdt, r2), Cout, C.adt, ldc, C.st);
    if (rc) break;
    rc = store_out(r2, r2, rowmajor(Ww, wdt, r2), Wout, C.adt, ldw, C.st);
  } while (0);
  return finish(C, info, rc, false);
}

int spm_nystrom_eig(const spm_sketch* S, const void* A, int32_t dtype, int64_t n, int64_t lda,
                    int64_t r2, int32_t q, uint64_t omega_seed, const spm_opts* opts, void* U,
                    int64_t ldu, void* lam, spm_info* info, void* stream) {
  SPM_TRY(check_common(S, A, dtype, n, lda, r2, q, opts));
  if (S->n != n || !U || !lam || ldu < r2) return SPM_EINVAL;
  if (dense_kind(S)) return SPM_EUNSUPPORTED;
  Call C(as_stream(stream));
  setup_call(C, dtype, opts, info);
  SPM_TRY(prepare(C));
  Nys o;
  int rc = nystrom_core(C, S, A, n, lda, r2, q, omega_seed, o);
  if (rc == SPM_OK) rc = nystrom_eig_finish(C, S, o, n, r2, U, ldu, lam);
  return finish(C, info, rc, false);
}

int spm_set_autotune(int32_t mode) {
  if (mode != 0 && mode != 1) return SPM_EINVAL;
  g_autotune = mode;
  return SPM_OK;
}

int spm_autotune_entries(int32_t clear) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  const int n = (int)g_tune.size();
  if (clear) g_tune.clear();
  return n;
}

int spm_gauss_sketch(const spm_sketch* S, const void* X, int32_t dtype, int64_t n, int64_t d,
                     int64_t ldx, double h, void* out, int64_t ldo, void* stream) {
  if (!S || !X || !out || (dtype != SPM_F32 && dtype != SPM_F64)) return SPM_EINVAL;
  if (n < 0 || d < 1 || ldx < d || ldo < S->r1) return SPM_EINVAL;
  const int dt = dtype == SPM_F64 ? DT_F64 : DT_F32;
  int* status = nullptr;
  SPM_TRY(gemm_public_status(&status));
  return gauss_sketch_dev(S, X, dt, n, d, ldx, h, out, dt, ldo, as_stream(stream), status);
}

int spm_nystrom_gauss(const spm_sketch* S, const void* X, int32_t dtype, int64_t n, int64_t d,
                      int64_t ldx, double h, int64_t r2, int32_t q, uint64_t omega_seed,
                      const spm_opts* opts, void* U, int64_t ldu, void* lam, spm_info* info,
                      void* stream) {
  if (!S || !X || d < 1 || ldx < d || !(h > 0.0)) return SPM_EINVAL;
  SPM_TRY(check_common(S, X, dtype, n, S->n, r2, q, opts));
  if (S->n != n || !U || !lam || ldu < r2) return SPM_EINVAL;
  if (dense_kind(S)) return SPM_EUNSUPPORTED;
  Call C(as_stream(stream));
  setup_call(C, dtype, opts, info);
  C.want_fro = false;                         // |K|_F is not read by the fused product
  SPM_TRY(prepare(C));
  Nys o;
  const GaussSrc gs{X, d, ldx, h};
  int rc = nystrom_core(C, S, nullptr, n, 0, r2, q, omega_seed, o, &gs);
  if (rc == SPM_OK) rc = nystrom_eig_finish(C, S, o, n, r2, U, ldu, lam);
  return finish(C, info, rc, false);
}

}  // extern "C"
