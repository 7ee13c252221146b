// Learned choice of the power count q and the sketch size r1.
//
// Theorems 2.1-2.3 size q and r1 only up to unspecified constants, so in
// practice they are tuned.  This file computes cheap features of the q = 0
// sketch (Algorithm 1 with q = 0: Y0 = A S Omega), feeds them to the selector
// network (mlp.cu) and runs the Randomized SVD with the cheapest candidate the
// network predicts to meet a requested residual ratio.
//
// Features (one FP32 vector of 8, see spm.h), from the singular values
// s_1 >= ... >= s_r2 of Y0 (square roots of the eigenvalues of Y0^T Y0):
//   log10(s_{r2/4}/s_1), log10(s_{r2/2}/s_1), log10(s_{r2}/s_1),
//   log10(r2 s_{r2}^2 / sum s_i^2), log10(m)/4, log10(n)/4, log10(r2)/3,
//   log2(r1/r2)/3.
#include <math.h>

#include <algorithm>
#include <functional>
#include <map>
#include <tuple>
#include <vector>

#include "internal.cuh"

namespace spm {

int mlp_forward_dev(const float* params, const float* X, int64_t batch, float* Y, cudaStream_t st);
int on_side_streams(int count, const int* order, int ns, cudaStream_t st,
                    const std::function<int(int, cudaStream_t)>& body);

__global__ void k_selector_features(const float* __restrict__ lam, int r2, double m, double n,
                                    double r1, float* __restrict__ feat) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s0 = sqrt(fmax((double)lam[0], 0.0));
  if (!(s0 > 0.0)) s0 = 1e-300;
  double tot = 0.0;
  for (int i = 0; i < r2; ++i) {
    const double si = fmax(sqrt(fmax((double)lam[i], 0.0)), 1e-30 * s0);
    tot += si * si;
  }
  auto sv = [&](int i) { return fmax(sqrt(fmax((double)lam[i], 0.0)), 1e-30 * s0); };
  const int i4 = max(1, r2 / 4), i2 = max(1, r2 / 2);
  const double sl = sv(r2 - 1);
  feat[0] = (float)log10(sv(i4 - 1) / s0);
  feat[1] = (float)log10(sv(i2 - 1) / s0);
  feat[2] = (float)log10(sl / s0);
  feat[3] = (float)log10(r2 * sl * sl / tot);
  feat[4] = (float)(log10(m) / 4.0);
  feat[5] = (float)(log10(n) / 4.0);
  feat[6] = (float)(log10((double)r2) / 3.0);
  feat[7] = (float)(log2(r1 / r2) / 3.0);
}

static int64_t pad8s(int64_t x) { return round_up(x, 8); }

// The cheapest candidate predicted to reach the target; cost ~ (2q + 1) r1 for
// the power products, ties broken towards smaller q; if no candidate is
// predicted to reach it, the one with the smallest predicted error.
void choose_candidate(const float* pred, double target_ratio, int* q_out, int* c_out) {
  const double thr = log10(target_ratio - 1.0);
  const int cs[3] = {2, 4, 8};
  int best = -1, best_any = 0;
  double best_cost = 1e300;
  for (int q = 0; q <= 4; ++q)
    for (int c = 0; c < 3; ++c) {
      const int idx = 3 * q + c;
      if (pred[idx] < pred[best_any]) best_any = idx;
      const double cost = (2.0 * q + 1.0) * cs[c];
      if (pred[idx] <= thr && cost < best_cost) {
        best_cost = cost;
        best = idx;
      }
    }
  if (best < 0) best = best_any;
  *q_out = best / 3;
  *c_out = cs[best % 3];
}

int selector_features_dev(const spm_sketch* S, const void* A, int adt, int64_t m, int64_t lda,
                          int64_t r2, uint64_t seed, float* feat, cudaStream_t st) {
  const int64_t r1 = S->r1, r1p = pad8s(r1), r2p = pad8s(r2);
  Arena ar(st);
  SPM_ALLOC(ar, __nv_bfloat16, Ahi, m * r1p);
  SPM_ALLOC(ar, __nv_bfloat16, Alo, m * r1p);
  SPM_ALLOC(ar, float, Om, r1 * r2);
  SPM_ALLOC(ar, __nv_bfloat16, Ohi, r1 * r2p);
  SPM_ALLOC(ar, __nv_bfloat16, Olo, r1 * r2p);
  SPM_ALLOC(ar, float, Y, m * r2);
  SPM_ALLOC(ar, float, G, r2 * r2);
  SPM_ALLOC(ar, float, V, r2 * r2);
  SPM_ALLOC(ar, float, lam, r2);
  SPM_ALLOC(ar, int, status, 1);
  SPM_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  SPM_TRY(gaussian_dev(Om, DT_F32, r1, r2, r2, seed, st));
  SPM_TRY(split_bf16(r1, r2, rowmajor(Om, DT_F32, r2), mrowmajor(Ohi, DT_BF16, r2p),
                     mrowmajor(Olo, DT_BF16, r2p), st));
  SPM_TRY(sketch_apply_dev(S, A, adt, m, lda, Ahi, DT_BF16, r1p, nullptr, st, Alo));
  // Y0 = A~ Omega as a split-precision product (A~ K-major, Omega MN-major)
  TcOp a[3] = {{Ahi, r1p, false}, {Ahi, r1p, false}, {Alo, r1p, false}};
  TcOp b[3] = {{Ohi, r2p, true}, {Olo, r2p, true}, {Ohi, r2p, true}};
  SPM_TRY(gemm_tc(m, r2, r1, 3, a, b, 1.0f, Y, r2, 1, 1, st));
  SPM_TRY(gemm_simt(r2, r2, m, 1.0, transpose(rowmajor(Y, DT_F32, r2)), rowmajor(Y, DT_F32, r2), 0.0,
                    mrowmajor(G, DT_F32, r2), st));
  SPM_TRY(symmetrize(r2, G, r2, DT_F32, st));
  SPM_TRY(sym_eig(r2, G, r2, V, r2, lam, DT_F32, status, st));
  k_selector_features<<<1, 32, 0, st>>>(lam, (int)r2, (double)m, (double)S->n, (double)r1, feat);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

// ---------------------------------------------------------------- residual judge
// After the chosen (q, r1) has run, the result is judged by the a-posteriori
// residual estimate e = sqrt(|A|_F^2 - |B|_F^2) (B = Q^T A; with k = r2 its
// squared Frobenius norm is the sum of the k squared singular values).  The
// problem is re-run with one more power step; once a step improves e by less
// than a quarter of the target's margin (e <= (1 + (target - 1) / 4) e_next)
// the power iteration has settled, and the error left is the sketch-size term of
// Theorem 3.1: the sketch is then doubled (r1 -> min(2 r1, n); r1 = n is the
// classical range finder) at the same q, and if that helps by more than the
// margin the power steps resume, else the problem is settled.  A power step
// that makes e worse (e_next > (1 + 1e-3) e) marks the working precision's
// limit: the problem is re-run in FP32 at the end.  The result kept is always
// the one with the smallest estimate.  e^2 is a difference of two nearly equal
// squared norms, each with the products' relative error (~1e-5 in the mixed and
// FP32 paths); a problem whose estimate is below JUDGE_FLOOR |A|_F (0.014:
// e^2 >= 2e-4 |A|_F^2, where a 5% change of e is 10x that error) is kept as
// run, since its estimate cannot resolve the target's margin.  FP64 runs use a
// floor of 1e-6.
static constexpr int JUDGE_ROUNDS = 4;
static constexpr double JUDGE_FLOOR = 0.014, JUDGE_FLOOR64 = 1e-6;

enum JudgeMode { JUDGE_DONE = 0, JUDGE_Q = 1, JUDGE_R1 = 2 };

// out[i] = sum of squares of item i's A (what = 0) or sigma (what = 1)
static int batch_sumsq(const std::vector<spm_batch_item>& it, int adt, int what, double* out,
                       cudaStream_t st) {
  SPM_CUDA_TRY(cudaMemsetAsync(out, 0, it.size() * sizeof(double), st));
  for (size_t i = 0; i < it.size(); ++i) {
    if (what == 0)
      SPM_TRY(sumsq(it[i].m, it[i].n, rowmajor(it[i].A, adt, it[i].lda), out + i, st));
    else
      SPM_TRY(sumsq(1, it[i].k, rowmajor(it[i].sigma, adt, it[i].k), out + i, st));
  }
  return SPM_OK;
}

static int copy_outputs(const spm_batch_item& from, const spm_batch_item& to, size_t es,
                        cudaStream_t st) {
  SPM_CUDA_TRY(cudaMemcpy2DAsync(to.U, to.ldu * es, from.U, from.ldu * es, from.k * es, from.m,
                                 cudaMemcpyDeviceToDevice, st));
  SPM_CUDA_TRY(cudaMemcpyAsync(to.sigma, from.sigma, from.k * es, cudaMemcpyDeviceToDevice, st));
  SPM_CUDA_TRY(cudaMemcpy2DAsync(to.Vt, to.ldvt * es, from.Vt, from.ldvt * es, from.n * es, from.k,
                                 cudaMemcpyDeviceToDevice, st));
  return SPM_OK;
}

// Scratch outputs (U m x k, sigma k, Vt k x n, each 256-byte aligned, ld k and n)
// for the given items, carved from one arena block.
static int scratch_outputs(Arena& ar, std::vector<spm_batch_item>& nx, size_t es) {
  auto up = [](int64_t b) { return (b + 255) & ~(int64_t)255; };
  int64_t total = 0;
  for (const auto& t : nx) total += up(t.m * t.k * es) + up(t.k * es) + up(t.k * t.n * es);
  unsigned char* base = ar.alloc<unsigned char>(total);
  if (!base) return SPM_ENOMEM;
  for (auto& t : nx) {
    t.U = base;
    base += up(t.m * t.k * es);
    t.sigma = base;
    base += up(t.k * es);
    t.Vt = base;
    base += up(t.k * t.n * es);
    t.ldu = t.k;
    t.ldvt = t.n;
  }
  return SPM_OK;
}

// The judge over a batch whose chosen run is in items (outputs written); items[i].q
// is updated to the q of the kept result.  One host synchronisation per round.
static int judge_batch(int count, spm_batch_item* items, int32_t dtype, double target,
                       const spm_opts* opts, int nstreams, cudaStream_t st,
                       std::vector<int>* used_fp32 = nullptr) {
  const int adt = dtype == SPM_F64 ? DT_F64 : DT_F32;
  const size_t es = dt_size(adt);
  spm_opts o32{};
  if (opts) o32 = *opts;
  o32.precision = SPM_PREC_FP32;
  std::vector<spm_batch_item> all(items, items + count);
  std::vector<double> a2(count), e(count), tmp(count);
  {
    Arena ar(st);
    double* d = ar.alloc<double>(2 * (int64_t)count);
    if (!d) return SPM_ENOMEM;
    SPM_TRY(batch_sumsq(all, adt, 0, d, st));
    SPM_TRY(batch_sumsq(all, adt, 1, d + count, st));
    SPM_CUDA_TRY(cudaMemcpyAsync(a2.data(), d, count * sizeof(double), cudaMemcpyDeviceToHost, st));
    SPM_CUDA_TRY(cudaMemcpyAsync(tmp.data(), d + count, count * sizeof(double), cudaMemcpyDeviceToHost, st));
    SPM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  for (int i = 0; i < count; ++i) e[i] = sqrt(fmax(a2[i] - tmp[i], 0.0));
  const double floor_rel = (opts && opts->precision == SPM_PREC_FP64) || !opts ? JUDGE_FLOOR64 : JUDGE_FLOOR;
  std::vector<int> active, fp32;
  for (int i = 0; i < count; ++i)
    if (e[i] >= floor_rel * sqrt(a2[i])) active.push_back(i);
  std::vector<int> mode(count, JUDGE_Q);
  for (int round = 0; round < JUDGE_ROUNDS && !active.empty(); ++round) {
    // the active problems once more, one power step or a doubled sketch further
    // than their current result, into scratch outputs
    Arena ar(st);
    std::vector<spm_batch_item> nx;
    for (int i : active) {
      spm_batch_item t = items[i];
      if (mode[i] == JUDGE_Q) {
        t.q += 1;
      } else {
        t.r1 = std::min<int64_t>(2 * t.r1, t.n);
        t.s = (int32_t)std::min<int64_t>(t.s, t.r1);
      }
      nx.push_back(t);
    }
    SPM_TRY(scratch_outputs(ar, nx, es));
    const int na = (int)nx.size();
    int32_t* dst = ar.alloc<int32_t>(na);
    double* d = ar.alloc<double>(na);
    if (!dst || !d) return SPM_ENOMEM;
    SPM_TRY(spm_rsvd_batched(na, nx.data(), dtype, opts, nstreams, dst, st));
    SPM_TRY(batch_sumsq(nx, adt, 1, d, st));
    std::vector<double> s2(na);
    std::vector<int32_t> hs(na);
    SPM_CUDA_TRY(cudaMemcpyAsync(s2.data(), d, na * sizeof(double), cudaMemcpyDeviceToHost, st));
    SPM_CUDA_TRY(cudaMemcpyAsync(hs.data(), dst, na * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SPM_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int> next;
    const double settle = 1.0 + 0.25 * (target - 1.0);
    for (int j = 0; j < na; ++j) {
      const int i = active[j];
      const double e0 = e[i];
      const double e2 = hs[j] == 0 ? sqrt(fmax(a2[i] - s2[j], 0.0)) : -1.0;
      if (e2 < 0.0) continue;  // the re-run failed: keep what there is
      if (mode[i] == JUDGE_Q && e2 > e0 * (1.0 + 1e-3) && opts && opts->precision == SPM_PREC_MIXED &&
          std::find(fp32.begin(), fp32.end(), i) == fp32.end())
        fp32.push_back(i);
      const bool helped = e0 > settle * e2;
      if (e2 < e0) {
        SPM_TRY(copy_outputs(nx[j], items[i], es, st));
        e[i] = e2;
        items[i].q = nx[j].q;
        items[i].r1 = nx[j].r1;
        items[i].s = nx[j].s;
      }
      if (mode[i] == JUDGE_Q)
        mode[i] = helped ? JUDGE_Q : (items[i].r1 < items[i].n ? JUDGE_R1 : JUDGE_DONE);
      else
        mode[i] = helped ? JUDGE_Q : JUDGE_DONE;
      if (mode[i] != JUDGE_DONE) next.push_back(i);
    }
    // scratch outputs are released in stream order after the copies above
    active.swap(next);
  }
  if (!fp32.empty()) {
    Arena ar(st);
    std::vector<spm_batch_item> nx;
    for (int i : fp32) nx.push_back(items[i]);
    SPM_TRY(scratch_outputs(ar, nx, es));
    const int na = (int)nx.size();
    int32_t* dst = ar.alloc<int32_t>(na);
    double* d = ar.alloc<double>(na);
    if (!dst || !d) return SPM_ENOMEM;
    SPM_TRY(spm_rsvd_batched(na, nx.data(), dtype, &o32, nstreams, dst, st));
    SPM_TRY(batch_sumsq(nx, adt, 1, d, st));
    std::vector<double> s2(na);
    std::vector<int32_t> hs(na);
    SPM_CUDA_TRY(cudaMemcpyAsync(s2.data(), d, na * sizeof(double), cudaMemcpyDeviceToHost, st));
    SPM_CUDA_TRY(cudaMemcpyAsync(hs.data(), dst, na * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SPM_CUDA_TRY(cudaStreamSynchronize(st));
    for (int j = 0; j < na; ++j) {
      const int i = fp32[j];
      const double e2 = hs[j] == 0 ? sqrt(fmax(a2[i] - s2[j], 0.0)) : -1.0;
      if (e2 >= 0.0 && e2 < e[i]) {
        SPM_TRY(copy_outputs(nx[j], items[i], es, st));
        if (used_fp32) used_fp32->push_back(i);
      }
    }
  }
  return SPM_OK;
}

}  // namespace spm

using namespace spm;

extern "C" {

int spm_selector_features(const spm_sketch* S, const void* A, int32_t dtype, int64_t m,
                          int64_t lda, int64_t r2, uint64_t omega_seed, float* feat, void* stream) {
  if (!S || !A || !feat || m < 1 || lda < S->n || r2 < 1 || r2 > S->r1 || r2 > m) return SPM_EINVAL;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_EINVAL;
  if (!tc_available()) return SPM_ECUDA;
  return selector_features_dev(S, A, dtype == SPM_F64 ? DT_F64 : DT_F32, m, lda, r2, omega_seed, feat,
                               as_stream(stream));
}

int spm_rsvd_auto(const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda, int64_t k,
                  double target_ratio, const float* params, uint64_t seed, const spm_opts* opts,
                  void* U, int64_t ldu, void* sigma, void* Vt, int64_t ldvt, int32_t* choice,
                  spm_info* info, void* stream) {
  if (!A || !params || !U || !sigma || !Vt || m < 1 || n < 1 || lda < n || k < 1 || k > m ||
      k > n || ldu < k || ldvt < n || !(target_ratio > 1.0))
    return SPM_EINVAL;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_EINVAL;
  cudaStream_t st = as_stream(stream);
  const int s = 8;
  const int64_t r1p = (4 * k < n) ? 4 * k : n;
  spm_sketch* P = nullptr;
  SPM_TRY(spm_sketch_create(&P, n, r1p, (int32_t)(s < r1p ? s : r1p), seed, SPM_SKETCH_SPARSE_SIGN, st));
  // the probe is used once, by the general kernels, as in the batched selector
  int rc = spm_sketch_set_plan(P, 0);
  float pred[SPM_MLP_OUT];
  {
    Arena ar(st);
    float* feat = ar.alloc<float>(SPM_MLP_IN);
    float* out = ar.alloc<float>(SPM_MLP_OUT);
    if (!feat || !out) rc = SPM_ENOMEM;
    if (rc == SPM_OK) rc = spm_selector_features(P, A, dtype, m, lda, k, seed + 1, feat, stream);
    if (rc == SPM_OK) rc = mlp_forward_dev(params, feat, 1, out, st);
    if (rc == SPM_OK && cudaMemcpyAsync(pred, out, sizeof(pred), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      rc = SPM_ECUDA;
    if (rc == SPM_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = SPM_ECUDA;
  }
  if (rc != SPM_OK) {
    spm_sketch_destroy(P);
    return rc;
  }
  int q = 0, c = 2;
  choose_candidate(pred, target_ratio, &q, &c);
  int64_t r1 = c * k;
  if (r1 > n) r1 = n;
  if (choice) {
    choice[0] = q;
    choice[1] = c;
  }
  spm_sketch* S = P;
  if (r1 != r1p) {
    spm_sketch_destroy(P);
    P = nullptr;
    SPM_TRY(spm_sketch_create(&S, n, r1, (int32_t)(s < r1 ? s : r1), seed, SPM_SKETCH_SPARSE_SIGN, st));
  }
  rc = spm_rsvd(S, A, dtype, m, lda, k, q, seed + 1, k, opts, U, ldu, sigma, Vt, ldvt, info, stream);
  spm_sketch_destroy(S);
  if (rc != SPM_OK) return rc;
  spm_batch_item it{A, m, n, lda, k, r1, (int32_t)(s < r1 ? s : r1), q, seed, U, ldu, sigma, Vt, ldvt};
  std::vector<int> f32;
  SPM_TRY(judge_batch(1, &it, dtype, target_ratio, opts, 1, st, &f32));
  if (info) {
    info->auto_q = it.q;
    info->auto_fp32 = f32.empty() ? 0 : 1;
  }
  return SPM_OK;
}

int spm_rsvd_batched_auto(int32_t count, spm_batch_item* items, int32_t dtype, double target_ratio,
                          const float* params, const spm_opts* opts, int32_t nstreams,
                          int32_t* dev_status, int32_t* choices, void* stream) {
  if (count < 0 || (count > 0 && !items) || !params || !(target_ratio > 1.0) || nstreams < 0 ||
      nstreams > 32)
    return SPM_EINVAL;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_EINVAL;
  for (int i = 0; i < count; ++i) {
    const spm_batch_item& it = items[i];
    if (!it.A || !it.U || !it.sigma || !it.Vt || it.m < 1 || it.n < 1 || it.lda < it.n ||
        it.k < 1 || it.k > it.m || it.k > it.n || it.ldu < it.k || it.ldvt < it.n)
      return SPM_EINVAL;
  }
  if (count == 0) return SPM_OK;
  if (!tc_available()) return SPM_ECUDA;
  cudaStream_t st = as_stream(stream);
  const int ns = nstreams == 0 ? 16 : nstreams;
  const int adt = dtype == SPM_F64 ? DT_F64 : DT_F32;
  // probe sketches: r1 = 4k (at most n), s = 8 (at most r1), one per distinct shape and seed
  std::map<std::tuple<int64_t, int64_t, uint64_t>, spm_sketch*> probes;
  std::vector<spm_sketch*> of(count, nullptr);
  int rc = SPM_OK;
  for (int i = 0; i < count && rc == SPM_OK; ++i) {
    const spm_batch_item& it = items[i];
    const int64_t r1p = std::min<int64_t>(4 * it.k, it.n);
    const auto key = std::make_tuple(it.n, r1p, it.seed);
    auto f = probes.find(key);
    if (f == probes.end()) {
      spm_sketch* P = nullptr;
      rc = spm_sketch_create(&P, it.n, r1p, (int32_t)std::min<int64_t>(8, r1p), it.seed,
                             SPM_SKETCH_SPARSE_SIGN, st);
      if (rc == SPM_OK) rc = spm_sketch_set_plan(P, 0);  // no plan: no synchronisation
      if (rc == SPM_OK) probes[key] = of[i] = P;
    } else {
      of[i] = f->second;
    }
  }
  std::vector<float> pred((size_t)count * SPM_MLP_OUT);
  {
    Arena ar(st);
    float* feat = ar.alloc<float>((int64_t)count * SPM_MLP_IN);
    float* out = ar.alloc<float>((int64_t)count * SPM_MLP_OUT);
    if (rc == SPM_OK && (!feat || !out)) rc = SPM_ENOMEM;
    if (rc == SPM_OK)
      rc = on_side_streams(count, nullptr, ns, st, [&](int i, cudaStream_t s) {
        const spm_batch_item& it = items[i];
        return selector_features_dev(of[i], it.A, adt, it.m, it.lda, it.k, it.seed + 1,
                                     feat + (int64_t)i * SPM_MLP_IN, s);
      });
    if (rc == SPM_OK) rc = mlp_forward_dev(params, feat, count, out, st);
    if (rc == SPM_OK && cudaMemcpyAsync(pred.data(), out, pred.size() * sizeof(float),
                                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
      rc = SPM_ECUDA;
    if (rc == SPM_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = SPM_ECUDA;
  }
  for (auto& kv : probes) spm_sketch_destroy(kv.second);
  if (rc != SPM_OK) return rc;
  for (int i = 0; i < count; ++i) {
    spm_batch_item& it = items[i];
    int q = 0, c = 2;
    choose_candidate(pred.data() + (size_t)i * SPM_MLP_OUT, target_ratio, &q, &c);
    it.q = q;
    it.r1 = std::min<int64_t>((int64_t)c * it.k, it.n);
    it.s = (int32_t)std::min<int64_t>(8, it.r1);
    if (choices) {
      choices[2 * i] = q;
      choices[2 * i + 1] = c;
    }
  }
  SPM_TRY(spm_rsvd_batched(count, items, dtype, opts, nstreams, dev_status, stream));
  return judge_batch(count, items, dtype, target_ratio, opts, ns, st);
}

}  // extern "C"
