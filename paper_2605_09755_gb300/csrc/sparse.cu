// Sparse input: A = A_csr + U diag(sig) V^T, the CSR matrix with an optional
// planted low-rank term kept as factors (never densified).
//
//   A~ = A S (Algorithm 1 line 1):  A_csr S by a warp per row (the row's r1
//        accumulators in shared memory, its non-zeros in order, the s entries
//        of row j of S added by s lanes at once: they hit distinct columns), plus
//        U (diag(sig) (S^T V)^T) as one product;
//   B = Q^T A (the RandSVD finish):  B^T = A_csr^T Q by a warp per column of A
//        over a column index of A built on the device (rows ascending inside a
//        column, so sums run in a fixed order), plus (Q^T U) diag(sig) V^T.
//
// The range finder and the SVD of B are the dense path's (`api.cu`), fed with
// A~ and B from here.
#include "internal.cuh"

namespace spm {

template <typename T, typename TACC>
__global__ void k_csr_sketch(int64_t m, int64_t n, int64_t nnz, int r1, int s,
                             const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                             const T* __restrict__ vals, const int32_t* __restrict__ scols,
                             const int8_t* __restrict__ ssigns, TACC scale, TACC* __restrict__ out,
                             int64_t ldo, int* __restrict__ status, bool add) {
  extern __shared__ __align__(16) unsigned char csr_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  TACC* acc = reinterpret_cast<TACC*>(csr_smem) + (size_t)wib * r1;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; i < m; i += nw) {
    for (int c = lane; c < r1; c += 32) acc[c] = (TACC)0;
    __syncwarp();
    // clamped, so that a malformed row pointer cannot send the loop out of range
    const int64_t e0 = max64(0, min64(rowptr[i], nnz)), e1 = max64(e0, min64(rowptr[i + 1], nnz));
    for (int64_t e = e0; e < e1; ++e) {
      const int64_t j = colind[e];
      if (j < 0 || j >= n) {
        bad = true;
        continue;
      }
      const TACC v = (TACC)vals[e];
      for (int t = lane; t < s; t += 32) {
        const int c = scols[j * s + t];
        acc[c] += ssigns[j * s + t] < 0 ? -v : v;
      }
      __syncwarp();
    }
    for (int c = lane; c < r1; c += 32)
      out[i * ldo + c] = add ? out[i * ldo + c] + acc[c] * scale : acc[c] * scale;
    __syncwarp();
  }
  if (bad && lane == 0) set_status(status, SPM_EINVAL);
}

// X[i][c] *= sig[c]
template <typename T>
__global__ void k_scale_cols(int64_t rows, int64_t cols, T* __restrict__ X, int64_t ld,
                             const T* __restrict__ sig) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    X[(e / cols) * ld + e % cols] *= sig[e % cols];
}

// ---------------------------------------------------------------- column index
__global__ void k_csc_count(int64_t nnz, int64_t n, const int32_t* __restrict__ colind,
                            unsigned long long* __restrict__ cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = colind[e];
    if (j >= 0 && j < n) atomicAdd(cnt + j, 1ull);
  }
}

// exclusive scan of cnt[0..n) into ptr[0..n], one CTA of 1024 threads
__global__ void __launch_bounds__(1024) k_scan_1cta(int64_t n, const unsigned long long* __restrict__ cnt,
                                                    int64_t* __restrict__ ptr) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int64_t chunk = (n + 1023) / 1024;
  const int64_t b = t * chunk, e = min64(n, b + chunk);
  int64_t sum = 0;
  for (int64_t i = b; i < e; ++i) sum += (int64_t)cnt[i];
  part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int u = 0; u < 1024; ++u) {
      const int64_t v = part[u];
      part[u] = run;
      run += v;
    }
  }
  __syncthreads();
  int64_t run = part[t];
  for (int64_t i = b; i < e; ++i) {
    ptr[i] = run;
    run += (int64_t)cnt[i];
  }
  if (t == 1023) ptr[n] = run;
}

template <typename T>
__global__ void k_csc_fill(int64_t m, int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
                           const int32_t* __restrict__ colind, const T* __restrict__ vals,
                           const int64_t* __restrict__ colptr, unsigned long long* __restrict__ cursor,
                           int32_t* __restrict__ rowind, T* __restrict__ cvals) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = max64(0, min64(rowptr[i], nnz)), e1 = max64(e0, min64(rowptr[i + 1], nnz));
    for (int64_t e = e0; e < e1; ++e) {
      const int64_t j = colind[e];
      if (j < 0 || j >= n) continue;
      const int64_t pos = colptr[j] + (int64_t)atomicAdd(cursor + j, 1ull);
      rowind[pos] = (int32_t)i;
      cvals[pos] = vals[e];
    }
  }
}

// rows ascending inside each column (insertion sort; columns hold ~nnz/n entries)
template <typename T>
__global__ void k_csc_sort(int64_t n, const int64_t* __restrict__ colptr, int32_t* __restrict__ rowind,
                           T* __restrict__ cvals) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = colptr[j], e = colptr[j + 1];
    for (int64_t p = b + 1; p < e; ++p) {
      const int32_t r = rowind[p];
      const T v = cvals[p];
      int64_t q = p - 1;
      while (q >= b && rowind[q] > r) {
        rowind[q + 1] = rowind[q];
        cvals[q + 1] = cvals[q];
        --q;
      }
      rowind[q + 1] = r;
      cvals[q + 1] = v;
    }
  }
}

// Bt[j][c] = sum over the non-zeros (i, v) of column j of v Q[i][c]; a warp per
// column, eight output columns per lane at a time
template <typename T>
__global__ void k_csc_spmm_t(int64_t n, int r2, const int64_t* __restrict__ colptr,
                             const int32_t* __restrict__ rowind, const T* __restrict__ cvals,
                             const T* __restrict__ Q, int64_t ldq, T* __restrict__ Bt, int64_t ldb) {
  constexpr int U = 8;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n; j += nw) {
    const int64_t b = colptr[j], e = colptr[j + 1];
    for (int c0 = 0; c0 < r2; c0 += 32 * U) {
      T acc[U];
#pragma unroll
      for (int u = 0; u < U; ++u) acc[u] = (T)0;
      for (int64_t p = b; p < e; ++p) {
        const int64_t i = rowind[p];
        const T v = cvals[p];
        const T* qr = Q + i * ldq;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int c = c0 + lane + 32 * u;
          if (c < r2) acc[u] = fma(v, qr[c], acc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = c0 + lane + 32 * u;
        if (c < r2) Bt[j * ldb + c] = acc[u];
      }
    }
  }
}

static int blocks_for(int64_t work, int per_block) {
  return (int)max64(1, min64(cdiv(work, per_block), 152 * 32));
}

// D (M x N, FP32, ld ldd) = X Y^T from the BF16 splits of X (M x K) and Y
// (N x K), both row-major FP32 with ld ldx / ldy; x_mn / y_mn: the operand is
// stored transposed (K x M, K x N) instead.  Three passes (hi hi + hi lo + lo hi).
static int tc_split_f32(int64_t M, int64_t N, int64_t K, const float* X, int64_t ldx, bool x_mn,
                        const float* Y, int64_t ldy, bool y_mn, float* D, int64_t ldd, Arena& ar,
                        cudaStream_t st) {
  const int64_t xr = x_mn ? K : M, xc = x_mn ? M : K, yr = y_mn ? K : N, yc = y_mn ? N : K;
  const int64_t xp = round_up(xc, 8), yp = round_up(yc, 8);
  __nv_bfloat16* xh = ar.alloc<__nv_bfloat16>(xr * xp);
  __nv_bfloat16* xl = ar.alloc<__nv_bfloat16>(xr * xp);
  __nv_bfloat16* yh = ar.alloc<__nv_bfloat16>(yr * yp);
  __nv_bfloat16* yl = ar.alloc<__nv_bfloat16>(yr * yp);
  if (!xh || !xl || !yh || !yl) return SPM_ENOMEM;
  SPM_TRY(split_bf16(xr, xc, rowmajor(X, DT_F32, ldx), mrowmajor(xh, DT_BF16, xp),
                     mrowmajor(xl, DT_BF16, xp), st));
  SPM_TRY(split_bf16(yr, yc, rowmajor(Y, DT_F32, ldy), mrowmajor(yh, DT_BF16, yp),
                     mrowmajor(yl, DT_BF16, yp), st));
  TcOp a[3] = {{xh, xp, x_mn}, {xh, xp, x_mn}, {xl, xp, x_mn}};
  TcOp b[3] = {{yh, yp, y_mn}, {yl, yp, y_mn}, {yh, yp, y_mn}};
  return gemm_tc(M, N, K, 3, a, b, 1.0f, D, ldd, 1, auto_splitk(M, N, K), st);
}

// out[e] = sum_c parts[c * len + e], c ascending
template <typename T>
__global__ void k_sum_parts(int count, int64_t len, const T* __restrict__ parts, T* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len;
       e += (int64_t)gridDim.x * blockDim.x) {
    T acc = (T)0;
    for (int c = 0; c < count; ++c) acc += parts[(int64_t)c * len + e];
    out[e] = acc;
  }
}

// out (M x N, ld N) = X^T Y for tall X (K x M, ld ldx) and Y (K x N, ld ldy):
// K split into chunks whose partial products (the CUDA-core GEMM, one batch
// entry per chunk) are summed in a fixed order.
static int gemm_tn_tall(int64_t M, int64_t N, int64_t K, int dt, const void* X, int64_t ldx,
                        const void* Y, int64_t ldy, void* out, cudaStream_t st) {
  const size_t es = dt == DT_F64 ? 8 : 4;
  const int64_t ks = max64(1, min64(256, K / 2048));
  const int64_t kc = cdiv(K, ks);
  const int64_t full = K / kc, rem = K - full * kc;
  const int64_t parts = full + (rem > 0 ? 1 : 0);
  Arena ar(st);
  void* P = ar.alloc<unsigned char>((size_t)parts * M * N * es);
  if (!P) return SPM_ENOMEM;
  SPM_TRY(gemm_simt(M, N, kc, 1.0, transpose(rowmajor(X, dt, ldx)), rowmajor(Y, dt, ldy), 0.0,
                    mrowmajor(P, dt, N), st, (int)full, kc * ldx, kc * ldy, M * N));
  if (rem > 0)
    SPM_TRY(gemm_simt(M, N, rem, 1.0,
                      transpose(rowmajor((const unsigned char*)X + (size_t)full * kc * ldx * es, dt, ldx)),
                      rowmajor((const unsigned char*)Y + (size_t)full * kc * ldy * es, dt, ldy), 0.0,
                      mrowmajor((unsigned char*)P + (size_t)full * M * N * es, dt, N), st));
  if (dt == DT_F64)
    k_sum_parts<double><<<blocks_for(M * N, 256), 256, 0, st>>>((int)parts, M * N, (const double*)P,
                                                               (double*)out);
  else
    k_sum_parts<float><<<blocks_for(M * N, 256), 256, 0, st>>>((int)parts, M * N, (const float*)P,
                                                              (float*)out);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

int csr_check(const spm_csr* A, int64_t n) {
  if (!A || A->m < 1 || A->n != n || A->nnz < 0 || A->p < 0 || !A->rowptr) return SPM_EINVAL;
  if (A->nnz > 0 && (!A->colind || !A->vals)) return SPM_EINVAL;
  if (A->nnz > 0x7FFFFFFFll * 8 || A->m > 0x7FFFFFFF) return SPM_EUNSUPPORTED;
  if (A->p > 0 && (!A->U || !A->sig || !A->V || A->ldu < A->p || A->ldv < A->p)) return SPM_EINVAL;
  return SPM_OK;
}

int csr_sketch_dev(const spm_sketch* S, const spm_csr* A, int dt, void* out, int64_t ldo, int* status,
                   cudaStream_t st, bool tc) {
  if (S->kind != SPM_SKETCH_SPARSE_SIGN && S->kind != SPM_SKETCH_IDENTITY) return SPM_EUNSUPPORTED;
  const int64_t m = A->m, n = A->n, r1 = S->r1;
  const int s = S->s;
  const size_t es = dt == DT_F64 ? 8 : 4;
  const int threads = 256, wpb = threads / 32;
  const size_t smem = (size_t)wpb * r1 * es;
  if (smem > 200 * 1024) return SPM_EUNSUPPORTED;
  const int grid = blocks_for(m, wpb);
  const double scale = (S->kind == SPM_SKETCH_IDENTITY) ? 1.0 : 1.0 / sqrt((double)s);
  const bool tc_factor = tc && dt == DT_F32 && A->p > 0 && tc_available();
  if (tc_factor) {
    // out = U (diag(sig) (S^T V)^T) on tensor cores first; the sparse part is added below
    Arena ar(st);
    float* SV = ar.alloc<float>(r1 * A->p);
    if (!SV) return SPM_ENOMEM;
    SPM_TRY(sketch_apply_t_dev(S, A->V, dt, A->p, A->ldv, SV, dt, A->p, st));
    k_scale_cols<float><<<blocks_for(r1 * A->p, 256), 256, 0, st>>>(r1, A->p, SV, A->p,
                                                                     (const float*)A->sig);
    SPM_LAUNCH_CHECK();
    SPM_TRY(tc_split_f32(m, r1, A->p, (const float*)A->U, A->ldu, false, SV, A->p, false,
                         (float*)out, ldo, ar, st));
  }
  if (dt == DT_F64) {
    auto kern = k_csr_sketch<double, double>;
    SPM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, threads, smem, st>>>(m, n, A->nnz, (int)r1, s, A->rowptr, A->colind,
                                      (const double*)A->vals, S->cols, S->signs, scale, (double*)out,
                                      ldo, status, false);
  } else {
    auto kern = k_csr_sketch<float, float>;
    SPM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, threads, smem, st>>>(m, n, A->nnz, (int)r1, s, A->rowptr, A->colind,
                                      (const float*)A->vals, S->cols, S->signs, (float)scale,
                                      (float*)out, ldo, status, tc_factor);
  }
  SPM_LAUNCH_CHECK();
  if (A->p > 0 && !tc_factor) {
    // A~ += U diag(sig) (S^T V)^T
    Arena ar(st);
    void* SV = ar.alloc<unsigned char>((size_t)r1 * A->p * es);
    if (!SV) return SPM_ENOMEM;
    SPM_TRY(sketch_apply_t_dev(S, A->V, dt, A->p, A->ldv, SV, dt, A->p, st));
    if (dt == DT_F64)
      k_scale_cols<double><<<blocks_for(r1 * A->p, 256), 256, 0, st>>>(r1, A->p, (double*)SV, A->p,
                                                                        (const double*)A->sig);
    else
      k_scale_cols<float><<<blocks_for(r1 * A->p, 256), 256, 0, st>>>(r1, A->p, (float*)SV, A->p,
                                                                       (const float*)A->sig);
    SPM_LAUNCH_CHECK();
    SPM_TRY(gemm_simt(m, r1, A->p, 1.0, rowmajor(A->U, dt, A->ldu), transpose(rowmajor(SV, dt, A->p)),
                      1.0, mrowmajor(out, dt, ldo), st));
  }
  return SPM_OK;
}

int csc_build(const spm_csr* A, int dt, Arena& ar, CscIndex& out, cudaStream_t st) {
  const int64_t m = A->m, n = A->n, nnz = A->nnz;
  const size_t es = dt == DT_F64 ? 8 : 4;
  out.colptr = ar.alloc<int64_t>(n + 1);
  out.rowind = ar.alloc<int32_t>(max64(nnz, 1));
  out.vals = ar.alloc<unsigned char>((size_t)max64(nnz, 1) * es);
  unsigned long long* cnt = ar.alloc<unsigned long long>(n);
  unsigned long long* cur = ar.alloc<unsigned long long>(n);
  if (!out.colptr || !out.rowind || !out.vals || !cnt || !cur) return SPM_ENOMEM;
  SPM_CUDA_TRY(cudaMemsetAsync(cnt, 0, n * sizeof(unsigned long long), st));
  SPM_CUDA_TRY(cudaMemsetAsync(cur, 0, n * sizeof(unsigned long long), st));
  if (nnz > 0) {
    k_csc_count<<<blocks_for(nnz, 256), 256, 0, st>>>(nnz, n, A->colind, cnt);
    SPM_LAUNCH_CHECK();
  }
  k_scan_1cta<<<1, 1024, 0, st>>>(n, cnt, out.colptr);
  SPM_LAUNCH_CHECK();
  if (nnz > 0) {
    if (dt == DT_F64) {
      k_csc_fill<double><<<blocks_for(m, 256), 256, 0, st>>>(m, n, nnz, A->rowptr, A->colind,
                                                             (const double*)A->vals, out.colptr, cur,
                                                             out.rowind, (double*)out.vals);
      k_csc_sort<double><<<blocks_for(n, 128), 128, 0, st>>>(n, out.colptr, out.rowind,
                                                             (double*)out.vals);
    } else {
      k_csc_fill<float><<<blocks_for(m, 256), 256, 0, st>>>(m, n, nnz, A->rowptr, A->colind,
                                                            (const float*)A->vals, out.colptr, cur,
                                                            out.rowind, (float*)out.vals);
      k_csc_sort<float><<<blocks_for(n, 128), 128, 0, st>>>(n, out.colptr, out.rowind,
                                                            (float*)out.vals);
    }
    SPM_LAUNCH_CHECK();
  }
  return SPM_OK;
}

int csr_project_dev(const spm_csr* A, const CscIndex& csc, int dt, const void* Q, int64_t ldq,
                    int64_t r2, void* B, int64_t ldb, cudaStream_t st, const __nv_bfloat16* Qhi,
                    const __nv_bfloat16* Qlo, int64_t ldqh) {
  const int64_t m = A->m, n = A->n;
  const size_t es = dt == DT_F64 ? 8 : 4;
  Arena ar(st);
  void* Bt = ar.alloc<unsigned char>((size_t)n * r2 * es);
  if (!Bt) return SPM_ENOMEM;
  const int grid = blocks_for(n, 8);
  if (dt == DT_F64)
    k_csc_spmm_t<double><<<grid, 256, 0, st>>>(n, (int)r2, csc.colptr, csc.rowind,
                                               (const double*)csc.vals, (const double*)Q, ldq,
                                               (double*)Bt, r2);
  else
    k_csc_spmm_t<float><<<grid, 256, 0, st>>>(n, (int)r2, csc.colptr, csc.rowind,
                                              (const float*)csc.vals, (const float*)Q, ldq, (float*)Bt,
                                              r2);
  SPM_LAUNCH_CHECK();
  SPM_TRY(convert2d(r2, n, transpose(rowmajor(Bt, dt, r2)), mrowmajor(B, dt, ldb), st));
  if (A->p > 0 && dt == DT_F32 && Qhi && Qlo && tc_available()) {
    // B += (Q^T U) diag(sig) V^T on tensor cores: Q^T U from Q's split and U's,
    // then (Q^T U diag(sig)) V^T into a scratch added to B
    const int64_t p = A->p, pp = round_up(p, 8);
    float* QU = ar.alloc<float>(r2 * p);
    float* Bf = ar.alloc<float>(r2 * n);
    __nv_bfloat16* uh = ar.alloc<__nv_bfloat16>(m * pp);
    __nv_bfloat16* ul = ar.alloc<__nv_bfloat16>(m * pp);
    if (!QU || !Bf || !uh || !ul) return SPM_ENOMEM;
    SPM_TRY(split_bf16(m, p, rowmajor(A->U, DT_F32, A->ldu), mrowmajor(uh, DT_BF16, pp),
                       mrowmajor(ul, DT_BF16, pp), st));
    // A-op Q^T (M = r2, K = m) and B-op U (N = p, K = m), both MN-major
    TcOp a[3] = {{Qhi, ldqh, true}, {Qhi, ldqh, true}, {Qlo, ldqh, true}};
    TcOp b[3] = {{uh, pp, true}, {ul, pp, true}, {uh, pp, true}};
    SPM_TRY(gemm_tc(r2, p, m, 3, a, b, 1.0f, QU, p, 1, auto_splitk(r2, p, m), st));
    k_scale_cols<float><<<blocks_for(r2 * p, 256), 256, 0, st>>>(r2, p, QU, p, (const float*)A->sig);
    SPM_LAUNCH_CHECK();
    SPM_TRY(tc_split_f32(r2, n, p, QU, p, false, (const float*)A->V, A->ldv, false, Bf, n, ar, st));
    SPM_TRY(add2d_f32(r2, n, (float*)B, ldb, Bf, n, st));
  } else if (A->p > 0) {
    // B += (Q^T U) diag(sig) V^T
    void* QU = ar.alloc<unsigned char>((size_t)r2 * A->p * es);
    if (!QU) return SPM_ENOMEM;
    SPM_TRY(gemm_tn_tall(r2, A->p, m, dt, Q, ldq, A->U, A->ldu, QU, st));
    if (dt == DT_F64)
      k_scale_cols<double><<<blocks_for(r2 * A->p, 256), 256, 0, st>>>(r2, A->p, (double*)QU, A->p,
                                                                        (const double*)A->sig);
    else
      k_scale_cols<float><<<blocks_for(r2 * A->p, 256), 256, 0, st>>>(r2, A->p, (float*)QU, A->p,
                                                                       (const float*)A->sig);
    SPM_LAUNCH_CHECK();
    SPM_TRY(gemm_simt(r2, n, A->p, 1.0, rowmajor(QU, dt, A->p), transpose(rowmajor(A->V, dt, A->ldv)),
                      1.0, mrowmajor(B, dt, ldb), st));
  }
  return SPM_OK;
}

}  // namespace spm
