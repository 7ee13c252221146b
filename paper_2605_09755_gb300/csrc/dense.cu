// Small dense building blocks of the hot path: CholeskyQR pieces (Gram
// Cholesky and triangular inverse, Section 2 "Orthonormalize the columns of Y"),
// the symmetric eigensolver behind the core SVD of B = Q^T A (Section 2,
// Randomized SVD finish) and of W (Algorithm 3), and elementwise helpers
// (split-precision conversion, norms, sign convention).
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "internal.cuh"
#include "rng.cuh"

namespace spm {

// ------------------------------------------------------------------ elementwise
template <typename T>
__device__ __forceinline__ double ldd(const T* p) { return (double)*p; }
template <>
__device__ __forceinline__ double ldd<__nv_bfloat16>(const __nv_bfloat16* p) {
  return (double)__bfloat162float(*p);
}
template <typename T>
__device__ __forceinline__ void std_(T* p, double v) { *p = (T)v; }
template <>
__device__ __forceinline__ void std_<__nv_bfloat16>(__nv_bfloat16* p, double v) {
  *p = __float2bfloat16_rn((float)v);
}

// Direct element conversions; FP32 paths avoid FP64 intermediates (the FP64
// pipe, conversions included, is far slower than FP32 on this part).
template <typename TY, typename TX>
__device__ __forceinline__ TY cvt(TX x) { return (TY)x; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, float>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, double>(double x) {
  return __float2bfloat16_rn((float)x);
}
template <>
__device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, __nv_bfloat16>(__nv_bfloat16 x) { return x; }

template <typename TX, typename TY>
__global__ void k_convert(int64_t rows, int64_t cols, const TX* __restrict__ x, int64_t xrs,
                          int64_t xcs, TY* __restrict__ y, int64_t yrs, int64_t ycs) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    // iterate so that the faster-moving index follows the destination's unit stride
    int64_t i, j;
    if (ycs == 1) {
      i = e / cols;
      j = e % cols;
    } else {
      j = e / rows;
      i = e % rows;
    }
    y[i * yrs + j * ycs] = cvt<TY, TX>(x[i * xrs + j * xcs]);
  }
}

template <typename TX>
__global__ void k_split(int64_t rows, int64_t cols, const TX* __restrict__ x, int64_t xrs,
                        int64_t xcs, __nv_bfloat16* __restrict__ hi, int64_t hrs, int64_t hcs,
                        __nv_bfloat16* __restrict__ lo, int64_t lrs, int64_t lcs) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i, j;
    if (hcs == 1) {
      i = e / cols;
      j = e % cols;
    } else {
      j = e / rows;
      i = e % rows;
    }
    const float v = (float)x[i * xrs + j * xcs];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const float r = v - __bfloat162float(h);
    hi[i * hrs + j * hcs] = h;
    lo[i * lrs + j * lcs] = __float2bfloat16_rn(r);
  }
}

static int grid_for(int64_t total) { return (int)min64(max64(cdiv(total, 256), 1), 152 * 16); }

// Row-major FP32 -> (hi, lo) BF16 split, four consecutive elements per thread:
// one 16-byte load and two 8-byte stores, rows from the grid's y dimension
// (no 64-bit division per element).
__global__ void k_split_rows4(int64_t rows, int64_t cols4, const float* __restrict__ x, int64_t xrs,
                              __nv_bfloat16* __restrict__ hi, int64_t hrs, __nv_bfloat16* __restrict__ lo,
                              int64_t lrs) {
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
    const float4* xr = reinterpret_cast<const float4*>(x + i * xrs);
    uint2* hr = reinterpret_cast<uint2*>(hi + i * hrs);
    uint2* lr = reinterpret_cast<uint2*>(lo + i * lrs);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols4;
         j += (int64_t)gridDim.x * blockDim.x) {
      const float4 v = __ldcs(xr + j);
      const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y);
      const __nv_bfloat162 h23 = __floats2bfloat162_rn(v.z, v.w);
      const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
      const __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
      const __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
      uint2 hv, lv;
      hv.x = *reinterpret_cast<const uint32_t*>(&h01);
      hv.y = *reinterpret_cast<const uint32_t*>(&h23);
      lv.x = *reinterpret_cast<const uint32_t*>(&l01);
      lv.y = *reinterpret_cast<const uint32_t*>(&l23);
      hr[j] = hv;
      lr[j] = lv;
    }
  }
}

int convert2d(int64_t rows, int64_t cols, View x, MView y, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return SPM_OK;
  const int g = grid_for(rows * cols);
#define SPM_CV(TX, TY)                                                                          \
  k_convert<TX, TY><<<g, 256, 0, st>>>(rows, cols, (const TX*)x.p, x.rs, x.cs, (TY*)y.p, y.rs, \
                                       y.cs)
  if (x.dt == DT_F32 && y.dt == DT_F32) SPM_CV(float, float);
  else if (x.dt == DT_F32 && y.dt == DT_F64) SPM_CV(float, double);
  else if (x.dt == DT_F64 && y.dt == DT_F32) SPM_CV(double, float);
  else if (x.dt == DT_F64 && y.dt == DT_F64) SPM_CV(double, double);
  else if (x.dt == DT_F32 && y.dt == DT_BF16) SPM_CV(float, __nv_bfloat16);
  else if (x.dt == DT_F64 && y.dt == DT_BF16) SPM_CV(double, __nv_bfloat16);
  else if (x.dt == DT_BF16 && y.dt == DT_F32) SPM_CV(__nv_bfloat16, float);
  else return SPM_EINVAL;
#undef SPM_CV
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

int split_bf16(int64_t rows, int64_t cols, View x, MView hi, MView lo, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return SPM_OK;
  const bool rows4 = x.dt == DT_F32 && x.cs == 1 && hi.cs == 1 && lo.cs == 1 && cols % 4 == 0 &&
                     x.rs % 4 == 0 && hi.rs % 4 == 0 && lo.rs % 4 == 0 &&
                     ((uintptr_t)x.p & 15) == 0 && ((uintptr_t)hi.p & 7) == 0 &&
                     ((uintptr_t)lo.p & 7) == 0;
  if (rows4) {
    const int64_t cols4 = cols / 4;
    const int gx = (int)min64(cdiv(cols4, 256), 64);
    const int gy = (int)min64(rows, max64(1, (152 * 32) / gx));
    k_split_rows4<<<dim3(gx, gy), 256, 0, st>>>(rows, cols4, (const float*)x.p, x.rs,
                                                 (__nv_bfloat16*)hi.p, hi.rs, (__nv_bfloat16*)lo.p,
                                                 lo.rs);
    SPM_LAUNCH_CHECK();
    return SPM_OK;
  }
  const int g = grid_for(rows * cols);
  if (x.dt == DT_F32)
    k_split<float><<<g, 256, 0, st>>>(rows, cols, (const float*)x.p, x.rs, x.cs,
                                      (__nv_bfloat16*)hi.p, hi.rs, hi.cs, (__nv_bfloat16*)lo.p,
                                      lo.rs, lo.cs);
  else if (x.dt == DT_F64)
    k_split<double><<<g, 256, 0, st>>>(rows, cols, (const double*)x.p, x.rs, x.cs,
                                       (__nv_bfloat16*)hi.p, hi.rs, hi.cs, (__nv_bfloat16*)lo.p,
                                       lo.rs, lo.cs);
  else
    return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

// Three-part BF16 split x ~ p1 + p2 + p3 (24 significant bits: each part is
// the BF16 rounding of what the previous parts leave), row-major outputs.
template <typename TX>
__global__ void k_split3(int64_t rows, int64_t cols, const TX* __restrict__ x, int64_t xrs,
                         __nv_bfloat16* __restrict__ p1, __nv_bfloat16* __restrict__ p2,
                         __nv_bfloat16* __restrict__ p3, int64_t prs) {
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y)
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols;
         j += (int64_t)gridDim.x * blockDim.x) {
      const float v = (float)x[i * xrs + j];
      const __nv_bfloat16 a = __float2bfloat16_rn(v);
      const float r1 = v - __bfloat162float(a);
      const __nv_bfloat16 b = __float2bfloat16_rn(r1);
      const __nv_bfloat16 c = __float2bfloat16_rn(r1 - __bfloat162float(b));
      p1[i * prs + j] = a;
      p2[i * prs + j] = b;
      p3[i * prs + j] = c;
    }
}

int split3_bf16(int64_t rows, int64_t cols, const void* x, int dt, int64_t ldx, __nv_bfloat16* p1,
                __nv_bfloat16* p2, __nv_bfloat16* p3, int64_t ldp, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return SPM_OK;
  const int gx = (int)min64(cdiv(cols, 256), 64);
  const int gy = (int)min64(rows, max64(1, (152 * 32) / gx));
  if (dt == DT_F32)
    k_split3<float><<<dim3(gx, gy), 256, 0, st>>>(rows, cols, (const float*)x, ldx, p1, p2, p3, ldp);
  else if (dt == DT_F64)
    k_split3<double><<<dim3(gx, gy), 256, 0, st>>>(rows, cols, (const double*)x, ldx, p1, p2, p3, ldp);
  else
    return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

// D += T (rows x cols FP32, row-major)
__global__ void k_add2d(int64_t rows, int64_t cols, float* __restrict__ D, int64_t ldd,
                        const float* __restrict__ T, int64_t ldt) {
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y)
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols;
         j += (int64_t)gridDim.x * blockDim.x)
      D[i * ldd + j] += T[i * ldt + j];
}

int add2d_f32(int64_t rows, int64_t cols, float* D, int64_t ldd, const float* T, int64_t ldt,
              cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return SPM_OK;
  const int gx = (int)min64(cdiv(cols, 256), 64);
  const int gy = (int)min64(rows, max64(1, (152 * 32) / gx));
  k_add2d<<<dim3(gx, gy), 256, 0, st>>>(rows, cols, D, ldd, T, ldt);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

// ------------------------------------------------------------------ Cholesky
// Leaf size of the blocked Cholesky: 128 in FP32, 64 in FP64 (shared memory).
template <typename T>
struct ChNB {
  static constexpr int v = 64;
};
static constexpr int CH_THREADS = 512;

// Factor one diagonal block G_kk = L L^T in shared memory (right-looking), write
// L (lower, zeros above) back in place and L^{-1} into Linv.
// Deflation: a pivot at or below tol * max(diag G) means that column is, to
// working precision, in the span of the earlier ones (the Gram matrix of a
// rank-deficient basis).  Its L column becomes e_j, defl[j] is set, and the
// caller replaces that column of the orthonormalised basis by a fresh random
// direction which the next CholeskyQR pass orthonormalises.
template <typename T>
__global__ void __launch_bounds__(CH_THREADS)
    k_chol_diag(int b, T* __restrict__ G, int64_t ldg, T* __restrict__ Li, int64_t ldi,
                const T* __restrict__ maxd, T tol, int* __restrict__ defl,
                int* __restrict__ status) {
  constexpr int NB = ChNB<T>::v;
  extern __shared__ __align__(16) unsigned char ch_smem[];
  T(*a)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(ch_smem);
  T(*inv)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(ch_smem + sizeof(T) * NB * (NB + 1));
  __shared__ T rdiag[NB];  // 1/sqrt(pivot), 0 for a deflated column
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  const T thr = tol * (*maxd);
  for (int e = tid; e < b * b; e += CH_THREADS) {
    const int i = e / b, j = e % b;
    a[i][j] = (j <= i) ? G[(int64_t)i * ldg + j] : (T)0;
  }
  __syncthreads();
  // Right-looking elimination with one barrier per pivot: column j is final
  // (unscaled) when step j starts, so every thread reads the pivot itself and
  // applies a[i][k] -= a[i][j] a[k][j] / a[j][j] to its own 2 x 4 elements of
  // the trailing square (rows ty + 32 v, columns tx + 16 u; entries above the
  // diagonal are skipped).  All loads of a step are issued before any store.
  const int ty = tid / 16, tx = tid % 16;
  static_assert(NB == 64 && CH_THREADS == 512, "2 x 4 elements per thread");
  for (int j = 0; j < b; ++j) {
    const T d = a[j][j];
    const bool fin = isfinite((double)d);
    const bool piv = fin && (d > thr);
    const T invd = piv ? (T)1 / d : (T)0;
    if (tid == 0) {
      rdiag[j] = piv ? (T)1 / sqrt(d) : (T)0;
      if (defl) defl[j] = piv ? 0 : 1;
      if (!fin) bad = 1;
    }
    if (piv) {
      T ci[2], ck[4], val[2][4];
      int ii[2], kk[4];
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        ii[v] = j + 1 + ty + 32 * v;
        ci[v] = (ii[v] < b) ? a[ii[v]][j] * invd : (T)0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        kk[u] = j + 1 + tx + 16 * u;
        ck[u] = (kk[u] < b) ? a[kk[u]][j] : (T)0;
      }
#pragma unroll
      for (int v = 0; v < 2; ++v)
#pragma unroll
        for (int u = 0; u < 4; ++u)
          val[v][u] = (ii[v] < b && kk[u] <= ii[v]) ? a[ii[v]][kk[u]] : (T)0;
#pragma unroll
      for (int v = 0; v < 2; ++v)
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (ii[v] < b && kk[u] <= ii[v]) a[ii[v]][kk[u]] = val[v][u] - ci[v] * ck[u];
    }
    __syncthreads();
  }
  // scale columns: L[i][j] = a[i][j] / sqrt(pivot j); deflated columns become e_j
  for (int e = tid; e < b * b; e += CH_THREADS) {
    const int i = e / b, j = e % b;
    const T r = rdiag[j];
    T v;
    if (j > i) v = (T)0;
    else if (r == (T)0) v = (i == j) ? (T)1 : (T)0;
    else v = (i == j) ? (T)1 / r : a[i][j] * r;
    a[i][j] = v;
  }
  __syncthreads();
  // inverse of the lower-triangular block: column c by 4 threads, each summing
  // every fourth term of the substitution, combined with warp shuffles
  for (int c0 = 0; c0 < NB; c0 += CH_THREADS / 4) {
    const int c = c0 + (tid >> 2), part = tid & 3;
    for (int i = 0; i < b; ++i) {
      T sacc = (T)0;
      if (c < b && i > c)
        for (int k = c + part; k < i; k += 4) sacc += a[i][k] * inv[k][c];
      sacc += __shfl_xor_sync(0xFFFFFFFFu, sacc, 1);
      sacc += __shfl_xor_sync(0xFFFFFFFFu, sacc, 2);
      if (part == 0 && c < b) inv[i][c] = (i < c) ? (T)0 : (((i == c) ? (T)1 : (T)0) - sacc) / a[i][i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = tid; e < b * b; e += CH_THREADS) {
    const int i = e / b, j = e % b;
    G[(int64_t)i * ldg + j] = a[i][j];
    Li[(int64_t)i * ldi + j] = inv[i][j];
  }
  if (tid == 0 && bad) set_status(status, DEV_NONFINITE);
}

template <typename T>
__global__ void k_maxdiag(int64_t r, const T* __restrict__ G, int64_t ldg, T* __restrict__ out) {
  __shared__ double red[256];
  double mx = 0.0;
  for (int64_t i = threadIdx.x; i < r; i += blockDim.x) mx = fmax(mx, (double)G[i * ldg + i]);
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (T)red[0];
}

// zero the columns j of P (rows x b) whose defl[j] is set
template <typename T>
__global__ void k_zero_defl_cols(int64_t rows, int b, T* __restrict__ P, int64_t ldp,
                                 const int* __restrict__ defl) {
  const int64_t total = rows * b;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % b);
    if (defl[j]) P[(e / b) * ldp + j] = (T)0;
  }
}

template <typename T>
__global__ void k_copy_block(int rows, int cols, const T* __restrict__ src, int64_t lds,
                             T* __restrict__ dst, int64_t ldd_) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    dst[i * ldd_ + j] = src[i * lds + j];
  }
}

template <typename T>
__global__ void k_zero2d(int64_t rows, int64_t cols, T* __restrict__ p, int64_t ld) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    p[(e / cols) * ld + (e % cols)] = (T)0;
}

template <typename T>
static int cholesky_inv_t(int64_t r, T* G, int64_t ldg, T* Li, int64_t ldi, int* defl,
                          int* status, cudaStream_t st) {
  constexpr int NB = ChNB<T>::v;
  const int dt = std::is_same<T, double>::value ? DT_F64 : DT_F32;
  const T tol = std::is_same<T, double>::value ? (T)1e-12 : (T)1e-6;
  Arena ar(st);
  SPM_ALLOC(ar, T, P, r * NB);
  SPM_ALLOC(ar, T, Tm, r * r);
  SPM_ALLOC(ar, T, maxd, 1);
  if (!defl) {
    defl = ar.alloc<int>(r);
    if (!defl) return SPM_ENOMEM;
  }
  k_zero2d<T><<<grid_for(r * r), 256, 0, st>>>(r, r, Li, ldi);
  SPM_LAUNCH_CHECK();
  k_maxdiag<T><<<1, 256, 0, st>>>(r, G, ldg, maxd);
  SPM_LAUNCH_CHECK();
  const int smem = (int)(2 * sizeof(T) * NB * (NB + 1));
  SPM_CUDA_TRY(cudaFuncSetAttribute(k_chol_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  for (int64_t kb = 0; kb < r; kb += NB) {
    const int b = (int)min64(NB, r - kb);
    k_chol_diag<T><<<1, CH_THREADS, smem, st>>>(b, G + kb * ldg + kb, ldg, Li + kb * ldi + kb, ldi,
                                                 maxd, tol, defl + kb, status);
    SPM_LAUNCH_CHECK();
    const int64_t rest = r - kb - b;
    if (rest > 0) {
      // P = G21 * Linv_kk^T (rest x b), deflated columns forced to zero
      T* g21 = G + (kb + b) * ldg + kb;
      View lkT = transpose(rowmajor(Li + kb * ldi + kb, dt, ldi));
      SPM_TRY(gemm_simt(rest, b, b, 1.0, rowmajor(g21, dt, ldg), lkT, 0.0, mrowmajor(P, dt, NB), st));
      k_zero_defl_cols<T><<<grid_for(rest * b), 256, 0, st>>>(rest, b, P, NB, defl + kb);
      SPM_LAUNCH_CHECK();
      // G22 -= P P^T
      SPM_TRY(gemm_simt(rest, rest, b, -1.0, rowmajor(P, dt, NB), transpose(rowmajor(P, dt, NB)), 1.0,
                        mrowmajor(G + (kb + b) * ldg + (kb + b), dt, ldg), st));
      // L21 = P
      k_copy_block<T><<<grid_for(rest * b), 256, 0, st>>>((int)rest, b, P, NB, g21, ldg);
      SPM_LAUNCH_CHECK();
    }
  }
  // Off-diagonal blocks of L^{-1} by recursive doubling: with the inverses of
  // the two diagonal halves of a 2s x 2s diagonal block known,
  //   Linv[o+s:o+2s, o:o+s] = -Linv[o+s:o+2s, o+s:o+2s] * L[o+s:o+2s, o:o+s] * Linv[o:o+s, o:o+s].
  // All such blocks of one level are independent: two batched products per level.
  for (int64_t sz = NB; sz < r; sz *= 2) {
    const int64_t full = r / (2 * sz);            // complete 2s blocks
    const int64_t o_tail = full * 2 * sz;
    const int64_t tail2 = r - o_tail - sz;        // size of a ragged lower half, if any
    const int64_t bstride_g = 2 * sz * (ldg + 1), bstride_i = 2 * sz * (ldi + 1);
    if (full > 0) {
      // Tm[t] = L21 * Linv11   (s x s each)
      SPM_TRY(gemm_simt(sz, sz, sz, 1.0, rowmajor(G + sz * ldg, dt, ldg), rowmajor(Li, dt, ldi), 0.0,
                        mrowmajor(Tm, dt, sz), st, (int)full, bstride_g, bstride_i, sz * sz));
      // Linv21 = -Linv22 * Tm
      SPM_TRY(gemm_simt(sz, sz, sz, -1.0, rowmajor(Li + sz * ldi + sz, dt, ldi), rowmajor(Tm, dt, sz),
                        0.0, mrowmajor(Li + sz * ldi, dt, ldi), st, (int)full, bstride_i, sz * sz,
                        bstride_i));
    }
    if (tail2 > 0) {
      const int64_t o = o_tail;
      SPM_TRY(gemm_simt(tail2, sz, sz, 1.0, rowmajor(G + (o + sz) * ldg + o, dt, ldg),
                        rowmajor(Li + o * ldi + o, dt, ldi), 0.0, mrowmajor(Tm, dt, sz), st));
      SPM_TRY(gemm_simt(tail2, sz, tail2, -1.0, rowmajor(Li + (o + sz) * ldi + (o + sz), dt, ldi),
                        rowmajor(Tm, dt, sz), 0.0, mrowmajor(Li + (o + sz) * ldi + o, dt, ldi), st));
    }
  }
  return SPM_OK;
}

// A caller that passes no deflation flags cannot use a deflated factor (a
// least-squares solve, not an orthonormalisation): any deflated column is then
// a breakdown.
__global__ void k_defl_breakdown(int64_t r, const int* __restrict__ defl, int* status) {
  int any = 0;
  for (int64_t j = threadIdx.x; j < r; j += blockDim.x) any |= defl[j];
  if (__syncthreads_or(any) && threadIdx.x == 0) set_status(status, DEV_BREAKDOWN);
}

int cholesky_inv(int64_t r, void* G, int64_t ldg, void* Linv, int64_t ldi, int dt, int* defl,
                 int* status, cudaStream_t st) {
  Arena ar(st);
  int* dd = defl;
  if (!dd) {
    dd = ar.alloc<int>(r);
    if (!dd) return SPM_ENOMEM;
  }
  // one cooperative kernel where the grid fits; the multi-launch path otherwise
  int rc = cholesky_inv_coop(r, G, ldg, Linv, ldi, dt, dd, status, st);
  if (rc == SPM_EUNSUPPORTED) {
    if (dt == DT_F64) rc = cholesky_inv_t<double>(r, (double*)G, ldg, (double*)Linv, ldi, dd, status, st);
    else if (dt == DT_F32) rc = cholesky_inv_t<float>(r, (float*)G, ldg, (float*)Linv, ldi, dd, status, st);
    else rc = SPM_EINVAL;
  }
  if (rc == SPM_OK && !defl) {
    k_defl_breakdown<<<1, 256, 0, st>>>(r, dd, status);
    SPM_LAUNCH_CHECK();
  }
  return rc;
}

// Replace the deflated columns of X (rows x c) by Gaussian columns scaled by
// 1/sqrt(rows); Philox4x32-10 keyed by `seed`, counter (row, column, 0, 3).
template <typename T>
__global__ void k_fill_deflated(int64_t rows, int64_t c, T* __restrict__ X, int64_t ldx,
                                const int* __restrict__ defl, uint32_t seed) {
  // nothing to do unless some column was deflated (the common case)
  int any = 0;
  for (int64_t j = threadIdx.x; j < c; j += blockDim.x) any |= defl[j];
  if (!__syncthreads_or(any)) return;
  const int64_t total = rows * c;
  const double sc = 1.0 / sqrt((double)rows);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / c, j = e % c;
    if (!defl[j]) continue;
    const u32x4 w = philox4x32_10((uint32_t)i, (uint32_t)j, 0u, 3u, seed, 0x2545F491u);
    const double u1 = ((double)w.x + 1.0) * 0x1.0p-32;
    const double u2 = (double)w.y * 0x1.0p-32;
    X[i * ldx + j] = (T)(sc * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
  }
}

int fill_deflated(int64_t rows, int64_t c, void* X, int64_t ldx, int dt, const int* defl,
                  uint32_t seed, cudaStream_t st) {
  if (dt == DT_F64) k_fill_deflated<double><<<grid_for(rows * c), 256, 0, st>>>(rows, c, (double*)X, ldx, defl, seed);
  else if (dt == DT_F32) k_fill_deflated<float><<<grid_for(rows * c), 256, 0, st>>>(rows, c, (float*)X, ldx, defl, seed);
  else return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

template <typename T>
__global__ void k_trace_shift(int64_t r, T* G, int64_t ldg, double coef) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < r; i += blockDim.x) s += (double)G[i * ldg + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double shift = coef * red[0];
  for (int64_t i = threadIdx.x; i < r; i += blockDim.x) G[i * ldg + i] = (T)((double)G[i * ldg + i] + shift);
}

int add_trace_shift(int64_t r, void* G, int64_t ldg, int dt, double coef, cudaStream_t st) {
  if (dt == DT_F64) k_trace_shift<double><<<1, 256, 0, st>>>(r, (double*)G, ldg, coef);
  else if (dt == DT_F32) k_trace_shift<float><<<1, 256, 0, st>>>(r, (float*)G, ldg, coef);
  else return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

template <typename T>
__global__ void k_symmetrize(int64_t r, T* A, int64_t lda) {
  const int64_t total = r * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / r, j = e % r;
    if (j < i) {
      const T v = (T)0.5 * (A[i * lda + j] + A[j * lda + i]);
      A[i * lda + j] = v;
      A[j * lda + i] = v;
    }
  }
}

int symmetrize(int64_t r, void* A, int64_t lda, int dt, cudaStream_t st) {
  if (dt == DT_F64) k_symmetrize<double><<<grid_for(r * r), 256, 0, st>>>(r, (double*)A, lda);
  else if (dt == DT_F32) k_symmetrize<float><<<grid_for(r * r), 256, 0, st>>>(r, (float*)A, lda);
  else return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

// ------------------------------------------------------------------ Jacobi eig
// Block cyclic Jacobi for the symmetric eigenproblem G = V diag(lam) V^T.
//
// G is padded to NB blocks of JB = 16 (NB even) with zero rows/columns, which
// never couple to the real ones.  A sweep runs NB - 1 rounds of the
// round-robin ("chess tournament") pairing of the blocks.  In a round:
//   phase 1: CTA c < NB/2 takes block pair c, loads the 32 x 32 subproblem
//            [G_PP G_PQ; G_QP G_QQ] into shared memory and diagonalises it by
//            one cyclic sweep of 2 x 2 rotations, accumulating the 32 x 32
//            rotation J_c;
//   phase 2: every warp applies the rotations as small dense products:
//            G[i, j] <- J_i^T G[i, j] J_j for every pair of block pairs (each
//            32 x 32 tile is read and written by one warp only, so in place), and
//            V[:, j] <- V[:, j] J_j.
// Bounded grid barriers separate the phases; the kernel is launched
// cooperatively so that all CTAs are resident.  A sweep starts with the
// off-diagonal mass test.
__device__ __forceinline__ int rr_player(int pos, int r, int np) {
  return pos == 0 ? 0 : 1 + ((pos - 1 + r) % (np - 1));
}
// pair i of round r among np (even) players
__device__ __forceinline__ void rr_pair(int i, int r, int np, int& p, int& q) {
  const int a = rr_player(i, r, np), b = rr_player(np - 1 - i, r, np);
  p = min(a, b);
  q = max(a, b);
}

static constexpr int JB = 16;          // block size
static constexpr int JS = 2 * JB;      // subproblem size
static constexpr int JLD = JS + 1;     // padded shared-memory row
// threads per CTA (512 in FP32 was measured slower: register spills in the
// rotation products outweigh the single wave of warp items)
template <typename T>
struct JT {
  static constexpr int v = 256;
};
// row stride of the per-warp product tiles: 16-byte aligned rows for vector
// shared loads and for the asynchronous 16-byte copies of the J tiles
template <typename T>
constexpr int JL4 = sizeof(T) == 4 ? JS + 4 : JS + 2;

// 16-byte asynchronous copy global -> shared through L2 only (.cg): the J tiles
// are rewritten every round by other CTAs
__device__ __forceinline__ void cp_async16_cg(void* sdst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// One warp copies a JS x JS row-major rotation tile into a shared tile with
// row stride JL4 (16-byte pieces, JS * sizeof(T) / 16 per row).
template <typename T>
__device__ __forceinline__ void j_tile_async(T (*dst)[JL4<T>], const T* __restrict__ src, int lane) {
  constexpr int CH = JS * (int)sizeof(T) / 16;
#pragma unroll
  for (int e = lane; e < JS * CH; e += 32) {
    const int row = e / CH, ch = e % CH;
    cp_async16_cg(reinterpret_cast<char*>(&dst[row][0]) + 16 * ch,
                  reinterpret_cast<const char*>(src + row * JS) + 16 * ch);
  }
}

__device__ __forceinline__ void ld4(const float* p, float v[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4]) {
  const double2 t0 = *reinterpret_cast<const double2*>(p);
  const double2 t1 = *reinterpret_cast<const double2*>(p + 2);
  v[0] = t0.x;
  v[1] = t0.y;
  v[2] = t1.x;
  v[3] = t1.y;
}
__device__ __forceinline__ void st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double* v) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

template <typename T>
__device__ __forceinline__ void rot_params(T app, T aqq, T apq, T& c, T& s) {
  c = (T)1;
  s = (T)0;
  if (fabs(apq) <= (T)1e-300) return;
  const T tau = (aqq - app) / ((T)2 * apq);
  const T t = (tau >= (T)0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
  c = (T)1 / sqrt((T)1 + t * t);
  s = t * c;
}
// FP32: approximate reciprocal intrinsics keep the rotation on the critical
// path short.  The angle (t) may carry their error; c must not: c^2 (1 + t^2)
// has to be 1 to rounding, or every rotation scales its rows and the bias adds
// up over the ~r^2 rotations of a solve (a uniform relative loss of ~1e-7 per
// rotation shrank all eigenvalues by ~3e-4 at r = 600).  So the approximate
// rsqrt gets one Newton-Raphson step, r' = r + r (1 - x r^2) / 2.
template <>
__device__ __forceinline__ void rot_params<float>(float app, float aqq, float apq, float& c, float& s) {
  c = 1.f;
  s = 0.f;
  if (fabsf(apq) <= 1e-37f) return;
  const float tau = (aqq - app) * __fdividef(0.5f, apq);
  const float at = fabsf(tau);
  const float y = fmaf(at, at, 1.f);  // sqrt(y) as y rsqrt(y): only the angle sees its error
  const float t = copysignf(at > 1e15f ? __fdividef(0.5f, at) : __fdividef(1.f, at + y * rsqrtf(y)), tau);
  const float x = fmaf(t, t, 1.f);
  const float r = rsqrtf(x);
  c = fmaf(0.5f * r, fmaf(-(x * r), r, 1.f), r);
  s = t * c;
}

// global index of local row a (0..63) of block pair (P, Q)
__device__ __forceinline__ int pair_index(int P, int Q, int a) {
  return a < JB ? P * JB + a : Q * JB + (a - JB);
}

// Phase 1: eigendecomposition of a JS x JS symmetric tile in shared memory by
// cyclic 2 x 2 Jacobi.  Each inner round first tabulates its JB index pairs and
// rotations (one thread per pair), then every thread updates whole 2 x 2
// blocks of M and row pairs of J from the tables.
template <typename T>
__device__ void inner_jacobi(T (*__restrict__ M)[JLD], T (*__restrict__ J)[JLD], T* __restrict__ cs,
                             T* __restrict__ sn, int max_inner, double tol2, int r_first = 0) {
  const int tid = threadIdx.x;
  __shared__ double red[2];
  for (int e = tid; e < JS * JS; e += JT<T>::v) J[e / JS][e % JS] = (e / JS == e % JS) ? (T)1 : (T)0;
  __syncthreads();
  for (int sw = 0; sw < max_inner; ++sw) {
    if (max_inner > 1) {
      if (tid < 2) red[tid] = 0.0;
      __syncthreads();
      double off = 0.0, tot = 0.0;
      for (int e = tid; e < JS * JS; e += JT<T>::v) {
        const double v = (double)M[e / JS][e % JS];
        tot += v * v;
        if (e / JS != e % JS) off += v * v;
      }
      atomicAdd(&red[0], off);
      atomicAdd(&red[1], tot);
      __syncthreads();
      const bool done = red[0] <= tol2 * red[1];
      __syncthreads();
      if (done) break;
    }
    for (int r = r_first; r < JS - 1; ++r) {
      // XOR ordering: round x = r + 1 pairs i with i ^ x (all pairs once per
      // sweep); pair t's low member is t with a 0 inserted at the top set bit
      // of x.  Indices come from this formula, not from a table, so the loads
      // of M and J do not wait on index loads.
      const int x = r + 1, hb = 31 - __clz(x);
      auto low = [&](int t) { return ((t >> hb) << (hb + 1)) | (t & ((1 << hb) - 1)); };
      if (tid < JB) {
        const int p = low(tid), q = p ^ x;
        T c, s;
        rot_params<T>(M[p][p], M[q][q], M[p][q], c, s);
        cs[tid] = c;
        sn[tid] = s;
      }
      __syncthreads();
      // all loads of a thread (its 2 x 2 block of M and its J row pairs) are
      // issued before any store, so their latencies overlap
      static_assert(JB * JB == JT<T>::v && JS * JB == 2 * JT<T>::v, "one block, two J items per thread");
      {
        const int bi = tid / JB, bj = tid % JB;
        const int pi = low(bi), qi = pi ^ x, pj = low(bj), qj = pj ^ x;
        const int row0 = tid / JB, row1 = row0 + JS / 2;
        const T m00 = M[pi][pj], m01 = M[pi][qj], m10 = M[qi][pj], m11 = M[qi][qj];
        const T j0p = J[row0][pj], j0q = J[row0][qj], j1p = J[row1][pj], j1q = J[row1][qj];
        const T ci = cs[bi], si = sn[bi], cj = cs[bj], sj = sn[bj];
        const T t00 = ci * m00 - si * m10, t01 = ci * m01 - si * m11;
        const T t10 = si * m00 + ci * m10, t11 = si * m01 + ci * m11;
        T n00 = cj * t00 - sj * t01, n01 = sj * t00 + cj * t01;
        T n10 = cj * t10 - sj * t11, n11 = sj * t10 + cj * t11;
        if (bi == bj) {
          n01 = (T)0;
          n10 = (T)0;
        }
        M[pi][pj] = n00;
        M[pi][qj] = n01;
        M[qi][pj] = n10;
        M[qi][qj] = n11;
        J[row0][pj] = cj * j0p - sj * j0q;
        J[row0][qj] = sj * j0p + cj * j0q;
        J[row1][pj] = cj * j1p - sj * j1q;
        J[row1][qj] = sj * j1p + cj * j1q;
      }
      __syncthreads();
    }
  }
}

// Where block X sits in round r: pair index i and half h (0 = the lower block).
__device__ __forceinline__ void rr_locate(int X, int r, int np, int& i, int& h) {
  const int pos = (X == 0) ? 0 : (((X - 1 - r) % (np - 1)) + (np - 1)) % (np - 1) + 1;
  i = min(pos, np - 1 - pos);
  int P, Q;
  rr_pair(i, r, np, P, Q);
  h = (X == P) ? 0 : 1;
}

// Subproblem of pair c of round r + 1, built from G^(r) and the round-r
// rotations (the rounds' products G^(r+1) = J^T G^(r) J restricted to the
// pair's blocks): quadrant (X, Y) = J_iX[:, hX]^T G^(r)[pair iX, pair iY] J_iY[:, hY].
// The three tiles and two rotations are copied into shared memory with 16-byte
// asynchronous copies (buf: 5 JS x JL4 tiles, then 3 JS x (JB + 4) products);
// the two products run as 4 x 4 register tiles, each sum taken over l in order.
template <typename T>
__device__ void build_next_subproblem(const T* __restrict__ Gc, int64_t ld, const T* __restrict__ Jc,
                                      int c, int r, int NB, T (*S0)[JLD], unsigned char* buf) {
  constexpr int BL = JL4<T>;
  constexpr int WL = JB + 4;
  const int tid = threadIdx.x;
  T(*Tl)[BL] = reinterpret_cast<T(*)[BL]>(buf);                // 3 tiles: (P,P), (P,Q), (Q,Q)
  T(*Jl)[BL] = Tl + 3 * JS;                                     // J_iP, J_iQ
  T(*Wl)[WL] = reinterpret_cast<T(*)[WL]>(buf + 5 * sizeof(T) * JS * BL);  // 3 x (JS x JB)
  int P2, Q2;
  rr_pair(c, r + 1, NB, P2, Q2);
  int ib[2], hb[2];
  rr_locate(P2, r, NB, ib[0], hb[0]);
  rr_locate(Q2, r, NB, ib[1], hb[1]);
  int Pb[2], Qb[2];
  rr_pair(ib[0], r, NB, Pb[0], Qb[0]);
  rr_pair(ib[1], r, NB, Pb[1], Qb[1]);
  // 16-byte pieces: a row of a G tile is two runs of JB elements (the pair's
  // blocks), a row of a J tile one run of JS
  constexpr int CR = JB * (int)sizeof(T) / 16;   // pieces per run
  constexpr int CT = 3 * JS * 2 * CR;            // G tiles
  constexpr int CJ = 2 * JS * 2 * CR;            // J tiles
  for (int e = tid; e < CT + CJ; e += JT<T>::v) {
    if (e < CT) {
      const int qd = e / (JS * 2 * CR), a = (e / (2 * CR)) % JS, k = (e / CR) % 2, ch = e % CR;
      const int X = (qd == 2) ? 1 : 0, Y = (qd == 0) ? 0 : 1;
      const T* src = Gc + (int64_t)pair_index(Pb[X], Qb[X], a) * ld + (k ? Qb[Y] : Pb[Y]) * JB;
      cp_async16_cg(reinterpret_cast<char*>(&Tl[qd * JS + a][k * JB]) + 16 * ch,
                    reinterpret_cast<const char*>(src) + 16 * ch);
    } else {
      const int f = e - CT;
      const int t = f / (JS * 2 * CR), a = (f / (2 * CR)) % JS, ch = f % (2 * CR);
      cp_async16_cg(reinterpret_cast<char*>(&Jl[t * JS + a][0]) + 16 * ch,
                    reinterpret_cast<const char*>(Jc + (size_t)ib[t] * JS * JS + (size_t)a * JS) + 16 * ch);
    }
  }
  cp_async_commit_group();
  cp_async_wait_all();
  __syncthreads();
  // W_qd = T_qd J_iY[:, hY]   (32 x 16 each): thread -> (qd, 4 rows, 4 columns)
  if (tid < 3 * (JS / 4) * (JB / 4)) {
    const int qd = tid / ((JS / 4) * (JB / 4)), a0 = ((tid / (JB / 4)) % (JS / 4)) * 4,
              b0 = (tid % (JB / 4)) * 4;
    const int Y = (qd == 0) ? 0 : 1;
    const T(*Tq)[BL] = Tl + qd * JS;
    const T(*Jy)[BL] = Jl + Y * JS;
    const int jc = hb[Y] * JB + b0;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
#pragma unroll 2
    for (int l = 0; l < JS; l += 4) {
      T tv[4][4], jv[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) ld4(&Tq[a0 + i][l], tv[i]);
#pragma unroll
      for (int k = 0; k < 4; ++k) ld4(&Jy[l + k][jc], jv[k]);
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(tv[i][k], jv[k][j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) st4(&Wl[qd * JS + a0 + i][b0], acc[i]);
  }
  __syncthreads();
  // S0 quadrant = J_iX[:, hX]^T W_qd   (16 x 16 each); (Q, P) is the transpose of (P, Q)
  if (tid < 3 * (JB / 4) * (JB / 4)) {
    const int qd = tid / ((JB / 4) * (JB / 4)), a0 = ((tid / (JB / 4)) % (JB / 4)) * 4,
              b0 = (tid % (JB / 4)) * 4;
    const int X = (qd == 2) ? 1 : 0, Y = (qd == 0) ? 0 : 1;
    const T(*Jx)[BL] = Jl + X * JS;
    const int jc = hb[X] * JB + a0;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
#pragma unroll 4
    for (int l = 0; l < JS; ++l) {
      T jv[4], wv[4];
      ld4(&Jx[l][jc], jv);
      ld4(&Wl[qd * JS + l][b0], wv);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(jv[i], wv[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        S0[X * JB + a0 + i][Y * JB + b0 + j] = acc[i][j];
        if (qd == 1) S0[JB + b0 + j][a0 + i] = acc[i][j];
      }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(JT<T>::v)
    k_block_jacobi(int n, int NB, T* __restrict__ G, T* __restrict__ Gb, T* __restrict__ V,
                   T* __restrict__ Jbuf, int max_sweeps, double tol2, int max_inner,
                   double tol2_inner, GridBar gb, double* __restrict__ offacc,
                   int* __restrict__ status, int* __restrict__ sweeps_out) {
  extern __shared__ __align__(16) unsigned char jsm[];
  T(*S0)[JLD] = reinterpret_cast<T(*)[JLD]>(jsm);
  T(*S1)[JLD] = S0 + JS;
  unsigned char* bbuf = jsm + 2 * sizeof(T) * JS * JLD;  // staging of build_next_subproblem
  __shared__ T cs[JB], sn[JB];
  __shared__ double red2[2];
  const unsigned nb = gridDim.x;
  const int tid = threadIdx.x;
  const int npad = NB * JB;
  const int hp = NB / 2;
  const int64_t ld = npad;
  // CTAs [0, L) build and solve the next round's subproblems while CTAs
  // [p2_first, nb) apply the current round's rotations (all CTAs when too few)
  const int L = max(1, min(hp, (int)nb / 2));
  const int p2_first = ((int)nb > L) ? L : 0;
  const int nworkers = (int)nb - p2_first, worker = (int)blockIdx.x - p2_first;
  const size_t jstride = (size_t)hp * JS * JS;
  T* Gc = G;
  T* Gn = Gb;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // off-diagonal mass
    double off = 0.0, tot = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)JT<T>::v + tid; e < (int64_t)npad * npad;
         e += (int64_t)nb * JT<T>::v) {
      const double v = (double)Gc[e];
      tot += v * v;
      if (e / npad != e % npad) off += v * v;
    }
    if (tid < 2) red2[tid] = 0.0;
    if (blockIdx.x == 0 && tid == 0) {
      offacc[2 * (sweep & 1)] = 0.0;
      offacc[2 * (sweep & 1) + 1] = 0.0;
    }
    if (!grid_sync(gb, nb, status)) return;
    atomicAdd(&red2[0], off);
    atomicAdd(&red2[1], tot);
    __syncthreads();
    if (tid == 0) {
      atomicAdd(&offacc[2 * (sweep & 1)], red2[0]);
      atomicAdd(&offacc[2 * (sweep & 1) + 1], red2[1]);
    }
    if (!grid_sync(gb, nb, status)) return;
    const double offv = *((volatile double*)&offacc[2 * (sweep & 1)]);
    const double totv = *((volatile double*)&offacc[2 * (sweep & 1) + 1]);
    if (offv <= tol2 * totv) break;
    // The look-ahead subproblems (rounds 1.. of the sweep) run only the inner
    // rounds that pair the two blocks (x >= JB); pairs inside one block are
    // annihilated once per sweep, in round 0.  Full inner sweeps in the last
    // sweeps cost ~3 us a round (the look-ahead is the round's critical path)
    // and, with the eigenvector refinement that follows the solve, bought no
    // accuracy: the largest off-diagonal of U^T A V at 65536 x 16384 went from
    // 2.9e-6 / 1.2e-6 / 6.3e-4 sigma_1 (sparse, dense, SRHT) to 8.4e-6 / 1.9e-5 / 1.5e-6.
    const int r_first = JB - 1;
    // round 0 subproblems straight from G
    for (int c = blockIdx.x; c < hp; c += nb) {
      int P, Q;
      rr_pair(c, 0, NB, P, Q);
      for (int e = tid; e < JS * JS; e += JT<T>::v) {
        const int a = e / JS, b = e % JS;
        S0[a][b] = Gc[(int64_t)pair_index(P, Q, a) * ld + pair_index(P, Q, b)];
      }
      __syncthreads();
      inner_jacobi<T>(S0, S1, cs, sn, max_inner, tol2_inner);
      T* Jo = Jbuf + (size_t)c * JS * JS;
      for (int e = tid; e < JS * JS; e += JT<T>::v) Jo[e] = S1[e / JS][e % JS];
      __syncthreads();
    }
    if (!grid_sync(gb, nb, status)) return;
    for (int r = 0; r < NB - 1; ++r) {
      const T* Jc = Jbuf + (size_t)(r & 1) * jstride;
      T* Jn = Jbuf + (size_t)((r + 1) & 1) * jstride;
      // ---------------- lookahead: round r + 1 subproblems from G^(r) and J^(r)
      if ((int)blockIdx.x < L && r + 1 < NB - 1) {
        for (int c = blockIdx.x; c < hp; c += L) {
          build_next_subproblem<T>(Gc, ld, Jc, c, r, NB, S0, bbuf);
          inner_jacobi<T>(S0, S1, cs, sn, max_inner, tol2_inner, r_first);
          T* Jo = Jn + (size_t)c * JS * JS;
          for (int e = tid; e < JS * JS; e += JT<T>::v) Jo[e] = S1[e / JS][e % JS];
          __syncthreads();
        }
      }
      if ((int)blockIdx.x >= p2_first) {
      // ---------------- phase 2: G <- J^T G J (tile pairs), V <- V J
      // One warp per item.  Its operands sit in shared memory and each lane
      // computes a 4 x 8 block of the 32 x 32 product (rows 4 (lane % 8),
      // columns 8 (lane / 8)) from one 16-byte load of the left operand's
      // column and two of the right operand's row per step: 32 multiply-adds
      // for 3 shared loads.  The J tiles (and a G item's tile) are copied in
      // asynchronously; a V item's tile goes through registers, where it is
      // transposed for the left operand.  Every sum runs over l in order.
      {
        constexpr int W = JT<T>::v / 32;
        constexpr int BL = JL4<T>;
        static_assert(W % 4 == 0, "warps come in sub-partition groups of four");
        const int lane = tid & 31, warp = tid >> 5;
        const int a0 = 4 * (lane & 7), c0 = 8 * (lane >> 3);
        T(*R0)[BL] = reinterpret_cast<T(*)[BL]>(jsm + (size_t)warp * 3 * sizeof(T) * JS * BL);
        T(*R1)[BL] = R0 + JS;
        T(*R2)[BL] = R0 + 2 * JS;
        const int gitems = hp * (hp + 1) / 2;  // tile pairs i <= j; G_ji is the transpose
        const int vitems = (npad / JS) * hp;
        const int nwarps = nworkers * W;
        // acc[i][j] += sum_l A[l][a0 + i] B[l][c0 + j] for l = 0 .. JS - 1
        auto product = [&](const T(*A)[BL], const T(*B)[BL], T(&acc)[4][8]) {
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = (T)0;
#pragma unroll 4
          for (int l = 0; l < JS; ++l) {
            T av[4], bv[8];
            ld4(&A[l][a0], av);
            ld4(&B[l][c0], bv);
            ld4(&B[l][c0 + 4], bv + 4);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 8; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
          }
        };
        // Warps w and w + 4 of a CTA share a sub-partition's issue slots.  Slots
        // are numbered so that the first warps of all sub-partitions come
        // before the second ones, and items (G pairs, two products each, then
        // V blocks, one product) are dealt over the slots forwards, then
        // backwards: a sub-partition gets at most one more product than the
        // mean.
        const int slot = (warp / 4) * (nworkers * 4) + worker * 4 + (warp % 4);
        for (int pass = 0; pass * nwarps < gitems + vitems; ++pass) {
          const int w = pass * nwarps + ((pass & 1) ? nwarps - 1 - slot : slot);
          if (w >= gitems + vitems) continue;
          T acc[4][8];
          if (w < gitems) {
            // w -> (i, j), i <= j, row-wise over the upper triangle of pair indices
            int i = (int)(((2.0f * hp + 1.0f) - sqrtf((2.0f * hp + 1.0f) * (2.0f * hp + 1.0f) - 8.0f * w)) * 0.5f);
            if (i < 0) i = 0;
            while (i > 0 && i * hp - i * (i - 1) / 2 > w) --i;
            while ((i + 1) * hp - (i + 1) * i / 2 <= w) ++i;
            const int j = i + (w - (i * hp - i * (i - 1) / 2));
            int Pi, Qi, Pj, Qj;
            rr_pair(i, r, NB, Pi, Qi);
            rr_pair(j, r, NB, Pj, Qj);
            // R0 = X (rows of pair i, columns of pair j), R1 = J_i, R2 = J_j
            {
              constexpr int CR = JB * (int)sizeof(T) / 16;  // 16-byte pieces per block run
#pragma unroll
              for (int e = lane; e < JS * 2 * CR; e += 32) {
                const int a = e / (2 * CR), k = (e / CR) % 2, ch = e % CR;
                const T* src = Gc + (int64_t)pair_index(Pi, Qi, a) * ld + (k ? Qj : Pj) * JB;
                cp_async16_cg(reinterpret_cast<char*>(&R0[a][k * JB]) + 16 * ch,
                              reinterpret_cast<const char*>(src) + 16 * ch);
              }
            }
            j_tile_async<T>(R1, Jc + (size_t)i * JS * JS, lane);
            j_tile_async<T>(R2, Jc + (size_t)j * JS * JS, lane);
            cp_async_commit_group();
            cp_async_wait_all();
            __syncwarp();
            // T = Ji^T X:  T[a][c] = sum_l Ji[l][a] X[l][c]
            product(R1, R0, acc);
            __syncwarp();
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {  // R1[c][a] = T[a][c]
              const T v[4] = {acc[0][jj], acc[1][jj], acc[2][jj], acc[3][jj]};
              st4(&R1[c0 + jj][a0], v);
            }
            __syncwarp();
            // X' = T Jj:  X'[a][c] = sum_l T[a][l] Jj[l][c] = sum_l R1[l][a] Jj[l][c]
            product(R1, R2, acc);
            // G_ij = X' (rows of pair i, columns of pair j); G_ji = X'^T
            const int64_t cj = pair_index(Pj, Qj, c0);
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) {
              T* dst = Gn + (int64_t)pair_index(Pi, Qi, a0 + ii) * ld + cj;
              st4(dst, acc[ii]);
              st4(dst + 4, acc[ii] + 4);
            }
            if (i != j) {
              const int64_t ci = pair_index(Pi, Qi, a0);
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {
                const T v[4] = {acc[0][jj], acc[1][jj], acc[2][jj], acc[3][jj]};
                st4(Gn + (int64_t)pair_index(Pj, Qj, c0 + jj) * ld + ci, v);
              }
            }
            __syncwarp();
          } else {
            const int v = w - gitems;
            const int rb = v / hp, j = v % hp;
            int Pj, Qj;
            rr_pair(j, r, NB, Pj, Qj);
            j_tile_async<T>(R2, Jc + (size_t)j * JS * JS, lane);
            cp_async_commit_group();
            {
              // lane l loads column l of the V tile and writes it as row l of R1
              T x[JS];
              const int64_t coll = pair_index(Pj, Qj, lane);
#pragma unroll
              for (int a = 0; a < JS; ++a) x[a] = V[(int64_t)(rb * JS + a) * ld + coll];
#pragma unroll
              for (int a = 0; a < JS; a += 4) st4(&R1[lane][a], &x[a]);
            }
            cp_async_wait_all();
            __syncwarp();
            // X' = X Jj:  X'[a][c] = sum_l X[a][l] Jj[l][c] = sum_l R1[l][a] Jj[l][c]
            product(R1, R2, acc);
            const int64_t cj = pair_index(Pj, Qj, c0);
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) {
              T* dst = V + (int64_t)(rb * JS + a0 + ii) * ld + cj;
              st4(dst, acc[ii]);
              st4(dst + 4, acc[ii] + 4);
            }
            __syncwarp();
          }
        }
      }
      }
      if (!grid_sync(gb, nb, status)) return;
      T* tmp = Gc;
      Gc = Gn;
      Gn = tmp;
    }
  }
  // the eigenvalues are read from G's diagonal
  if (Gc != G)
    for (int i = blockIdx.x * JT<T>::v + tid; i < npad; i += nb * JT<T>::v)
      G[(int64_t)i * ld + i] = Gc[(int64_t)i * ld + i];
  if (blockIdx.x == 0 && tid == 0 && sweeps_out) atomicMax(sweeps_out, sweep);
}

template <typename T>
__global__ void k_eye_pad(int n, int npad, const T* __restrict__ A, int64_t lda, T* __restrict__ G,
                          T* __restrict__ V) {
  const int64_t total = (int64_t)npad * npad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / npad, j = e % npad;
    G[e] = (i < n && j < n) ? A[i * lda + j] : (T)0;
    V[e] = (i == j) ? (T)1 : (T)0;
  }
}

// Column norms of the accumulated rotations.  A rotation whose cosine rounds
// to 1 (|t| < 2^-12 in FP32) is sqrt(1 + t^2) times an orthogonal one, and the
// late sweeps consist of such rotations: to first order V = W D with W
// orthogonal and D diagonal, and the same products turn G into D W^T G0 W D.
// So each eigenvector is normalised and its eigenvalue divided by the squared
// norm (the Rayleigh quotient of the unit vector): lamc[i] = G_ii / |v_i|^2,
// inv[i] = 1 / |v_i|.  A block takes 32 columns (one per lane, rows read
// coalesced), its 8 warps every 8th row; the 8 partial sums are added in FP64.
template <typename T>
__global__ void k_eig_colnorm(int n, int64_t ldg, const T* __restrict__ G, const T* __restrict__ V,
                              T* __restrict__ lamc, T* __restrict__ inv) {
  __shared__ double part[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (i < n)
    for (int row = w; row < n; row += 8) {
      const double v = (double)V[(int64_t)row * ldg + i];
      s += v * v;
    }
  part[w][lane] = s;
  __syncthreads();
  if (w == 0 && i < n) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += part[k][lane];
    lamc[i] = (T)((double)G[(int64_t)i * ldg + i] / t);
    inv[i] = (T)(1.0 / sqrt(t));
  }
}

// Sort the first n (corrected) eigenvalues descending and gather the normalised
// eigenvector columns; padded positions (>= n) hold the decoupled zero rows and
// are skipped.
template <typename T>
__global__ void k_eig_sort(int n, int64_t ldg, const T* __restrict__ lamc, const T* __restrict__ inv,
                           const T* __restrict__ Vin, T* __restrict__ Vout, int64_t ldvo,
                           T* __restrict__ lam) {
  __shared__ int rk;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const T li = lamc[i];
    const T sc = inv[i];
    if (threadIdx.x == 0) rk = 0;
    __syncthreads();
    int cnt = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const T lj = lamc[j];
      if (lj > li || (lj == li && j < i)) ++cnt;
    }
    atomicAdd(&rk, cnt);
    __syncthreads();
    const int pos = rk;
    if (threadIdx.x == 0) lam[pos] = li;
    for (int row = threadIdx.x; row < n; row += blockDim.x)
      Vout[(int64_t)row * ldvo + pos] = Vin[(int64_t)row * ldg + i] * sc;
    __syncthreads();
  }
}

template <typename T>
static int sym_eig_t(int64_t r, T* A, int64_t lda, T* V, int64_t ldv, T* lam, int* status,
                     cudaStream_t st, int* sweeps) {
  const int n = (int)r;
  int NB = (int)cdiv(n, JB);
  if (NB < 2) NB = 2;
  if (NB & 1) ++NB;
  const int npad = NB * JB;
  Arena ar(st);
  SPM_ALLOC(ar, T, G, (int64_t)npad * npad);
  SPM_ALLOC(ar, T, Vw, (int64_t)npad * npad);
  SPM_ALLOC(ar, T, Gb, (int64_t)npad * npad);            // second buffer of G (rounds alternate)
  SPM_ALLOC(ar, T, Jbuf, 2 * (int64_t)(NB / 2) * JS * JS);  // this round's and the next round's J
  SPM_ALLOC(ar, unsigned, bar, 2);
  SPM_ALLOC(ar, double, offacc, 4);
  SPM_ALLOC(ar, T, lamc, 2 * (int64_t)n);  // corrected eigenvalues, then inverse column norms
  SPM_CUDA_TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
  k_eye_pad<T><<<grid_for((int64_t)npad * npad), 256, 0, st>>>(n, npad, A, lda, G, Vw);
  SPM_LAUNCH_CHECK();
  int dev = 0, sms = 0, per_sm = 0;
  SPM_CUDA_TRY(cudaGetDevice(&dev));
  SPM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  constexpr int JTHREADS = JT<T>::v;
  // subproblems: 2 JS x JLD tiles, 5 JS x JL4 ones and 3 JS x (JB + 4) ones;
  // products: per warp 3 JS x JL4 tiles
  const int smem = (int)std::max(2 * sizeof(T) * JS * JLD + 5 * sizeof(T) * JS * JL4<T> +
                                     3 * sizeof(T) * JS * (JB + 4),
                                 (JTHREADS / 32) * 3 * sizeof(T) * JS * JL4<T>);
  auto kern = k_block_jacobi<T>;
  SPM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  SPM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, JTHREADS, smem));
  if (per_sm < 1) return SPM_ECUDA;
  const int hp = NB / 2;
  const int items = hp * (hp + 1) / 2 + (npad / JS) * hp;
  // one CTA per SM: the grid barrier's arrival count stays small (two per SM
  // measured slower: the barriers and the phase-1 CTAs lose more than the
  // rotation products gain)
  // (items count warps: small problems take only the CTAs they can fill, which
  // also keeps their grid barriers cheap and leaves SMs to concurrent work)
  int blocks = min((items + JTHREADS / 32 - 1) / (JTHREADS / 32), sms);
  blocks = max(blocks, hp);
  if (blocks > sms * per_sm) return SPM_EUNSUPPORTED;  // too large for one resident grid
  const bool is64 = std::is_same<T, double>::value;
  const double eps = is64 ? 1.1102230246251565e-16 : 5.960464477539063e-08;
  double tol2 = (4.0 * npad * eps) * (4.0 * npad * eps);
  double tol2i = (4.0 * JS * eps) * (4.0 * JS * eps);
  int max_sweeps = is64 ? 25 : 20;
  int max_inner = 1;  // one inner sweep per round: the outer sweeps converge the rest
  GridBar gb{bar, bar + 1};
  int NBv = NB;
  void* args[] = {(void*)&n, (void*)&NBv, (void*)&G, (void*)&Gb, (void*)&Vw, (void*)&Jbuf,
                  (void*)&max_sweeps, (void*)&tol2, (void*)&max_inner, (void*)&tol2i,
                  (void*)&gb, (void*)&offacc, (void*)&status, (void*)&sweeps};
  SPM_CUDA_TRY(cudaLaunchCooperativeKernel((void*)kern, dim3(blocks), dim3(JTHREADS), args, smem, st));
  count_launch();
  k_eig_colnorm<T><<<(unsigned)cdiv(n, 32), 256, 0, st>>>(n, npad, G, Vw, lamc, lamc + n);
  SPM_LAUNCH_CHECK();
  k_eig_sort<T><<<(unsigned)min(n, 1024), 128, 0, st>>>(n, npad, lamc, lamc + n, Vw, V, ldv, lam);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

int sym_eig(int64_t r, void* A, int64_t lda, void* V, int64_t ldv, void* lam, int dt, int* status,
            cudaStream_t st, int* sweeps) {
  if (r <= 0) return SPM_OK;
  if (r > 16384) return SPM_EUNSUPPORTED;
  if (dt == DT_F64) return sym_eig_t<double>(r, (double*)A, lda, (double*)V, ldv, (double*)lam, status, st, sweeps);
  if (dt == DT_F32) return sym_eig_t<float>(r, (float*)A, lda, (float*)V, ldv, (float*)lam, status, st, sweeps);
  return SPM_EINVAL;
}

// ------------------------------------------------------------------ eigenvector refinement
// One step of the Ogita-Aishima refinement (Ogita & Aishima, 2018) of approximate
// eigenvectors X of a symmetric G: with Gm = X^T X and S = X^T G X,
//   lam_i = S_ii / Gm_ii                             (Rayleigh quotients),
//   E_ii  = (1 - Gm_ii) / 2,
//   E_ij  = (S_ij - lam_j Gm_ij) / (lam_j - lam_i)   (i != j; R = I - Gm),
// and X <- X + X E.  The paper switches a pair to E_ij = R_ij / 2 = -Gm_ij / 2
// (orthogonality only) when the two eigenvalues are closer than a global bound;
// here the switch is per pair: when the first-order correction would exceed
// theta in magnitude (a pair too close for one Newton step).  S and Gm are read
// symmetrised.  One thread per element.
template <typename T>
__global__ void k_oa_update(int64_t r, const T* __restrict__ S, int64_t lds, const T* __restrict__ Gm,
                            int64_t ldg, T* __restrict__ E, int64_t lde, T theta) {
  const int64_t total = r * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / r, j = e % r;
    const T gi = Gm[i * ldg + i], gj = Gm[j * ldg + j];
    T v;
    if (i == j) {
      v = ((T)1 - gi) * (T)0.5;
    } else {
      const T li = S[i * lds + i] / gi, lj = S[j * lds + j] / gj;
      const T sij = (S[i * lds + j] + S[j * lds + i]) * (T)0.5;
      const T gij = (Gm[i * ldg + j] + Gm[j * ldg + i]) * (T)0.5;
      const T num = sij - lj * gij, den = lj - li;
      v = (fabs(num) <= theta * fabs(den)) ? num / den : -gij * (T)0.5;
    }
    E[i * lde + j] = v;
  }
}

int oa_update(int64_t r, const float* S, const float* Gm, float* E, double theta, cudaStream_t st) {
  if (r <= 0) return SPM_OK;
  k_oa_update<float><<<grid_for(r * r), 256, 0, st>>>(r, S, r, Gm, r, E, r, (float)theta);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

// Score of an eigenvector estimate X from S = X^T G X and Gm = X^T X:
//   m = max_{i != j} |S_ij| / sqrt(S_jj S_00) + max_{i, j} |Gm_ij - delta_ij|,
// the largest off-diagonal entry of U^T A V relative to sigma_1 that X would
// leave in the Randomized SVD finish (S_00 = sigma_1^2: the columns come in
// descending order), plus the loss of orthonormality.  Nonnegative doubles
// compare like their bit patterns, so the maxima are integer atomics into
// mx[0..1]; a NaN anywhere gives a NaN bit pattern above every finite one.
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v) {
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}
template <typename T>
__global__ void k_oa_metric(int64_t r, const T* __restrict__ S, const T* __restrict__ Gm,
                            unsigned long long* __restrict__ mx) {
  // FP32 arithmetic: the score only ranks estimates
  float f1 = 0.f, f2 = 0.f;
  const float s00 = (float)S[0];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < r * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / r, j = e % r;
    const float g = fabsf((float)Gm[e] - (i == j ? 1.f : 0.f));
    f2 = (g > f2 || g != g) ? g : f2;
    if (i != j) {
      const float q = fabsf((float)S[e]) * rsqrtf(fabsf((float)S[j * r + j] * s00));
      f1 = (q > f1 || q != q) ? q : f1;
    }
  }
  double m1 = f1, m2 = f2;
  for (int o = 16; o > 0; o >>= 1) {
    const double a = __shfl_xor_sync(0xFFFFFFFFu, m1, o), b = __shfl_xor_sync(0xFFFFFFFFu, m2, o);
    m1 = (a > m1 || a != a) ? a : m1;
    m2 = (b > m2 || b != b) ? b : m2;
  }
  // one atomic per block: the warps' maxima through shared memory
  __shared__ double w1[32], w2[32];
  const int warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) {
    w1[warp] = m1;
    w2[warp] = m2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      m1 = (w1[w] > m1 || w1[w] != w1[w]) ? w1[w] : m1;
      m2 = (w2[w] > m2 || w2[w] != w2[w]) ? w2[w] : m2;
    }
    atomic_max_nonneg(mx, m1);
    atomic_max_nonneg(mx + 1, m2);
  }
}

// keep[0] = 1 when the score in mx beats *best (which is then updated), and
// always on the first evaluation (keep[1] = 0); mx cleared for the next one.
__global__ void k_oa_decide(unsigned long long* __restrict__ mx, double* __restrict__ best,
                            int* __restrict__ keep) {
  const double m = __longlong_as_double((long long)mx[0]) + __longlong_as_double((long long)mx[1]);
  const bool better = keep[1] == 0 || m < *best;  // a NaN score never replaces a kept one
  if (better) *best = m;
  keep[0] = better ? 1 : 0;
  keep[1] = 1;
  mx[0] = mx[1] = 0ull;
}

template <typename T>
__global__ void k_copy_if(int64_t n, const T* __restrict__ src, T* __restrict__ dst,
                          const int* __restrict__ keep) {
  if (!*keep) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

int oa_keep_best(int64_t r, const float* S, const float* Gm, const float* X, float* Xbest,
                 unsigned long long* mx, double* best, int* keep, cudaStream_t st) {
  k_oa_metric<float><<<grid_for(r * r), 256, 0, st>>>(r, S, Gm, mx);
  SPM_LAUNCH_CHECK();
  k_oa_decide<<<1, 1, 0, st>>>(mx, best, keep);
  SPM_LAUNCH_CHECK();
  k_copy_if<float><<<grid_for(r * r), 256, 0, st>>>(r * r, X, Xbest, keep);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

// ------------------------------------------------------------------ norms etc.
template <typename T>
__global__ void k_line_norms(int64_t rows, int64_t cols, const T* __restrict__ X, int64_t rs,
                             int64_t cs, bool by_col, double* __restrict__ out) {
  // one CTA per line
  const int64_t nl = by_col ? cols : rows;
  const int64_t len = by_col ? rows : cols;
  __shared__ double red[256];
  for (int64_t l = blockIdx.x; l < nl; l += gridDim.x) {
    // per-thread partial sums in T (FP32 for FP32 data: len / 256 terms each),
    // combined in FP64
    T sp = (T)0;
    for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
      const T v = by_col ? X[t * rs + l * cs] : X[l * rs + t * cs];
      sp = fma(v, v, sp);
    }
    red[threadIdx.x] = (double)sp;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[l] = sqrt(red[0]);
    __syncthreads();
  }
}

int norms(int64_t rows, int64_t cols, View X, bool by_col, double* out, cudaStream_t st) {
  const int64_t nl = by_col ? cols : rows;
  const int g = (int)min64(nl, 152 * 8);
  if (X.dt == DT_F32) k_line_norms<float><<<g, 256, 0, st>>>(rows, cols, (const float*)X.p, X.rs, X.cs, by_col, out);
  else if (X.dt == DT_F64) k_line_norms<double><<<g, 256, 0, st>>>(rows, cols, (const double*)X.p, X.rs, X.cs, by_col, out);
  else return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

template <typename T>
__global__ void k_scale_lines(int64_t rows, int64_t cols, T* __restrict__ X, int64_t rs, int64_t cs,
                              bool by_rows, const double* __restrict__ s, bool inv) {
  // blockIdx.y walks the lines (rows or columns), threads the other index; the
  // factor is formed once per line and applied in T
  const int64_t nl = by_rows ? rows : cols, len = by_rows ? cols : rows;
  __shared__ T fs;
  for (int64_t l = blockIdx.y; l < nl; l += gridDim.y) {
    __syncthreads();  // the previous line's factor has been read
    if (threadIdx.x == 0) {
      double f = s[l];
      if (inv) f = (f != 0.0) ? 1.0 / f : 0.0;
      fs = (T)f;
    }
    __syncthreads();
    const T ft = fs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < len;
         t += (int64_t)gridDim.x * blockDim.x) {
      T* p = by_rows ? X + l * rs + t * cs : X + t * rs + l * cs;
      *p = *p * ft;
    }
  }
}

int scale_lines(int64_t rows, int64_t cols, MView X, bool rows_not_cols, const double* s, bool inv,
                cudaStream_t st) {
  const int64_t nl = rows_not_cols ? rows : cols, len = rows_not_cols ? cols : rows;
  const dim3 g((unsigned)min64(cdiv(len, 256), 64), (unsigned)min64(nl, 65535));
  if (X.dt == DT_F32) k_scale_lines<float><<<g, 256, 0, st>>>(rows, cols, (float*)X.p, X.rs, X.cs, rows_not_cols, s, inv);
  else if (X.dt == DT_F64) k_scale_lines<double><<<g, 256, 0, st>>>(rows, cols, (double*)X.p, X.rs, X.cs, rows_not_cols, s, inv);
  else return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

// Descending order of x[0..r): pos(i) = #{j : x_j > x_i, or x_j = x_i and j < i}
// (NaN ranks last, as -inf), so every position is taken exactly once;
// perm[pos(i)] = i, xs[pos(i)] = x_i.  The comparisons run on 64-bit integer
// keys that order like the values (-0 taken as +0; the bits of a negative
// value with its 63 low bits inverted), staged through shared memory.
__device__ __forceinline__ long long order_key(double v) {
  if (!(v == v)) v = -INFINITY;
  if (v == 0.0) v = 0.0;
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFll);
}

__global__ void k_desc_order(int r, const double* __restrict__ x, int* __restrict__ perm,
                             double* __restrict__ xs) {
  __shared__ long long tile[1024];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const long long ki = i < r ? order_key(x[i]) : 0ll;
  int pos = 0;
  for (int j0 = 0; j0 < r; j0 += 1024) {
    const int nt = min(1024, r - j0);
    __syncthreads();
    for (int t = threadIdx.x; t < nt; t += blockDim.x) tile[t] = order_key(x[j0 + t]);
    __syncthreads();
    if (i < r)
      for (int t = 0; t < nt; ++t) {
        const long long kj = tile[t];
        pos += (kj > ki) || (kj == ki && j0 + t < i);
      }
  }
  if (i < r) {
    perm[pos] = i;
    xs[pos] = x[i];
  }
}

int desc_order(int64_t r, const double* x, int* perm, double* xs, cudaStream_t st) {
  if (r <= 0) return SPM_OK;
  if (r > 0x7FFFFFFF) return SPM_EUNSUPPORTED;
  k_desc_order<<<(unsigned)cdiv(r, 256), 256, 0, st>>>((int)r, x, perm, xs);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

// dst line l = src line perm[l] (rows when by_row, else columns), l < lines.
template <typename T>
__global__ void k_gather_lines(int64_t lines, int64_t len, const T* __restrict__ src, int64_t srs,
                               int64_t scs, T* __restrict__ dst, int64_t drs, int64_t dcs,
                               const int* __restrict__ perm, bool by_row) {
  for (int64_t l = blockIdx.y; l < lines; l += gridDim.y) {
    const int64_t from = perm[l];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
      if (by_row)
        dst[l * drs + e * dcs] = src[from * srs + e * scs];
      else
        dst[e * drs + l * dcs] = src[e * srs + from * scs];
    }
  }
}

int gather_lines(int64_t lines, int64_t len, View src, MView dst, const int* perm, bool by_row,
                 cudaStream_t st) {
  if (lines <= 0 || len <= 0) return SPM_OK;
  if (src.dt != dst.dt) return SPM_EINVAL;
  const dim3 g((unsigned)min64(cdiv(len, 256), 64), (unsigned)min64(lines, 65535));
#define SPM_GL(T)                                                                              \
  k_gather_lines<T><<<g, 256, 0, st>>>(lines, len, (const T*)src.p, src.rs, src.cs, (T*)dst.p, \
                                       dst.rs, dst.cs, perm, by_row)
  if (src.dt == DT_F32) SPM_GL(float);
  else if (src.dt == DT_F64) SPM_GL(double);
  else if (src.dt == DT_BF16) SPM_GL(__nv_bfloat16);
  else return SPM_EINVAL;
#undef SPM_GL
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

template <typename T>
__global__ void k_sumsq(int64_t rows, int64_t cols, const T* __restrict__ X, int64_t rs, int64_t cs,
                        double* acc) {
  __shared__ double red[256];
  // rows from blockIdx.y, per-thread partial sums in T, combined in FP64
  T sp = (T)0;
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y)
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols;
         j += (int64_t)gridDim.x * blockDim.x) {
      const T v = X[i * rs + j * cs];
      sp = fma(v, v, sp);
    }
  red[threadIdx.x] = (double)sp;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(acc, red[0]);
}

int sumsq(int64_t rows, int64_t cols, View X, double* acc, cudaStream_t st) {
  const dim3 g((unsigned)min64(cdiv(cols, 256), 16), (unsigned)min64(rows, 1024));
  if (X.dt == DT_F32) k_sumsq<float><<<g, 256, 0, st>>>(rows, cols, (const float*)X.p, X.rs, X.cs, acc);
  else if (X.dt == DT_F64) k_sumsq<double><<<g, 256, 0, st>>>(rows, cols, (const double*)X.p, X.rs, X.cs, acc);
  else return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

// column argmax |U[:, j]| (smallest index on ties) -> sign flag
template <typename T>
__global__ void k_sign_flags(int64_t m, int64_t k, const T* __restrict__ U, int64_t rs, int64_t cs,
                             int* __restrict__ flip) {
  __shared__ double bv[256];
  __shared__ int64_t bi[256];
  for (int64_t j = blockIdx.x; j < k; j += gridDim.x) {
    T best = (T)-1;
    int64_t idx = 0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
      const T v = fabs(U[i * rs + j * cs]);
      if (v > best) {
        best = v;
        idx = i;
      }
    }
    bv[threadIdx.x] = (double)best;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        const double v2 = bv[threadIdx.x + o];
        const int64_t i2 = bi[threadIdx.x + o];
        if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
          bv[threadIdx.x] = v2;
          bi[threadIdx.x] = i2;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) flip[j] = (U[bi[0] * rs + j * cs] < (T)0) ? 1 : 0;
    __syncthreads();
  }
}

// The same argmax in two passes for a row-major U (cs == 1): a CTA scans a
// block of rows with its threads on columns (coalesced rows) and keeps, per
// column, the largest |U| and its first row; then each column's block results
// are combined in block order.  Ties go to the smallest row, as above.
template <typename T>
__global__ void k_sign_part(int64_t m, int64_t k, const T* __restrict__ U, int64_t rs, int64_t rows_per,
                            T* __restrict__ pv, int64_t* __restrict__ pi) {
  const int64_t r0 = blockIdx.x * rows_per, r1 = min64(m, r0 + rows_per);
  for (int64_t j = threadIdx.x; j < k; j += blockDim.x) {
    T best = (T)-1;
    int64_t idx = r0;
    for (int64_t i = r0; i < r1; ++i) {
      const T v = fabs(U[i * rs + j]);
      if (v > best) {
        best = v;
        idx = i;
      }
    }
    pv[blockIdx.x * k + j] = best;
    pi[blockIdx.x * k + j] = idx;
  }
}

// a warp per column: lane l takes blocks l, l + 32, ... in order, then the warp
// keeps the largest value and, among equal ones, the smallest row (the result
// of a scan over the blocks in order)
template <typename T>
__global__ void k_sign_combine(int nblk, int64_t k, const T* __restrict__ U, int64_t rs,
                               const T* __restrict__ pv, const int64_t* __restrict__ pi,
                               int* __restrict__ flip) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < k; j += nw) {
    T best = (T)-1;
    int64_t idx = 0;
    for (int b = lane; b < nblk; b += 32) {
      const T v = pv[b * k + j];
      if (v > best) {
        best = v;
        idx = pi[b * k + j];
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T v2 = __shfl_xor_sync(0xFFFFFFFFu, best, o);
      const int64_t i2 = __shfl_xor_sync(0xFFFFFFFFu, idx, o);
      if (v2 > best || (v2 == best && i2 < idx)) {
        best = v2;
        idx = i2;
      }
    }
    if (lane == 0) flip[j] = (U[idx * rs + j] < (T)0) ? 1 : 0;
  }
}

template <typename T>
__global__ void k_apply_flags(int64_t rows, int64_t cols, T* __restrict__ X, int64_t rs, int64_t cs,
                              bool by_col, const int* __restrict__ flip) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    if (flip[by_col ? j : i]) X[i * rs + j * cs] = -X[i * rs + j * cs];
  }
}

template <typename T>
static void sign_flags_rows(int64_t m, int64_t k, const T* U, int64_t rs, int* flip, Arena& ar,
                            cudaStream_t st, bool& done) {
  done = false;
  const int64_t nblk = min64(cdiv(m, 64), 152 * 4);
  const int64_t rows_per = cdiv(m, nblk);
  T* pv = ar.alloc<T>(nblk * k);
  int64_t* pi = ar.alloc<int64_t>(nblk * k);
  if (!pv || !pi) return;
  k_sign_part<T><<<(unsigned)cdiv(m, rows_per), 256, 0, st>>>(m, k, U, rs, rows_per, pv, pi);
  k_sign_combine<T><<<(unsigned)min64(cdiv(k, 8), 152 * 8), 256, 0, st>>>((int)cdiv(m, rows_per), k, U,
                                                                          rs, pv, pi, flip);
  done = true;
}

int sign_fix(int64_t m, int64_t k, int64_t n, MView U, MView Vt, cudaStream_t st) {
  Arena ar(st);
  SPM_ALLOC(ar, int, flip, k);
  const int g = (int)min64(k, 152 * 8);
  bool rows_done = false;
  if (U.cs == 1 && U.dt == DT_F32)
    sign_flags_rows<float>(m, k, (const float*)U.p, U.rs, flip, ar, st, rows_done);
  else if (U.cs == 1 && U.dt == DT_F64)
    sign_flags_rows<double>(m, k, (const double*)U.p, U.rs, flip, ar, st, rows_done);
  if (U.dt == DT_F32) {
    if (!rows_done) k_sign_flags<float><<<g, 256, 0, st>>>(m, k, (const float*)U.p, U.rs, U.cs, flip);
    k_apply_flags<float><<<grid_for(m * k), 256, 0, st>>>(m, k, (float*)U.p, U.rs, U.cs, true, flip);
    k_apply_flags<float><<<grid_for(k * n), 256, 0, st>>>(k, n, (float*)Vt.p, Vt.rs, Vt.cs, false, flip);
  } else if (U.dt == DT_F64) {
    if (!rows_done) k_sign_flags<double><<<g, 256, 0, st>>>(m, k, (const double*)U.p, U.rs, U.cs, flip);
    k_apply_flags<double><<<grid_for(m * k), 256, 0, st>>>(m, k, (double*)U.p, U.rs, U.cs, true, flip);
    k_apply_flags<double><<<grid_for(k * n), 256, 0, st>>>(k, n, (double*)Vt.p, Vt.rs, Vt.cs, false, flip);
  } else {
    return SPM_EINVAL;
  }
  count_launch(2);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

template <typename T>
__global__ void k_copy_vec(int64_t n, const double* __restrict__ s, T* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = (T)s[i];
}

int copy_vec(int64_t n, const double* src, void* dst, int dt, cudaStream_t st) {
  if (dt == DT_F32) k_copy_vec<float><<<grid_for(n), 256, 0, st>>>(n, src, (float*)dst);
  else if (dt == DT_F64) k_copy_vec<double><<<grid_for(n), 256, 0, st>>>(n, src, (double*)dst);
  else return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

template <typename T>
__global__ void k_check_finite(int64_t rows, int64_t cols, const T* __restrict__ X, int64_t rs,
                               int64_t cs, int* status) {
  const int64_t total = rows * cols;
  bool bad = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite((double)X[(e / cols) * rs + (e % cols) * cs]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(status, DEV_NONFINITE);
}

int check_finite(int64_t rows, int64_t cols, View X, int* status, cudaStream_t st) {
  const int g = grid_for(rows * cols);
  if (X.dt == DT_F32) k_check_finite<float><<<g, 256, 0, st>>>(rows, cols, (const float*)X.p, X.rs, X.cs, status);
  else if (X.dt == DT_F64) k_check_finite<double><<<g, 256, 0, st>>>(rows, cols, (const double*)X.p, X.rs, X.cs, status);
  else return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

}  // namespace spm
