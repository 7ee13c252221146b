// Small dense building blocks of the hot path: CholeskyQR pieces (Gram
// Cholesky and triangular inverse, Section 2 "Orthonormalize the columns of Y"),
// the symmetric eigensolver behind the core SVD of B = Q^T A (Section 2,
// Randomized SVD finish) and of W (Algorithm 3), and elementwise helpers
// (split-precision conversion, norms, sign convention).
#include <math.h>

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
    std_<TY>(y + i * yrs + j * ycs, ldd<TX>(x + i * xrs + j * xcs));
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
    const float v = (float)ldd<TX>(x + i * xrs + j * xcs);
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const float r = v - __bfloat162float(h);
    hi[i * hrs + j * hcs] = h;
    lo[i * lrs + j * lcs] = __float2bfloat16_rn(r);
  }
}

static int grid_for(int64_t total) { return (int)min64(max64(cdiv(total, 256), 1), 152 * 16); }

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

// ------------------------------------------------------------------ Cholesky
static constexpr int CH_NB = 64;

// Factor one diagonal block G_kk = L L^T in shared memory (right-looking), write
// L (lower, zeros above) back in place and L^{-1} into Linv.
// Deflation: a pivot at or below tol * max(diag G) means that column is, to
// working precision, in the span of the earlier ones (the Gram matrix of a
// rank-deficient basis).  Its L column becomes e_j, defl[j] is set, and the
// caller replaces that column of the orthonormalised basis by a fresh random
// direction which the next CholeskyQR pass orthonormalises.
template <typename T>
__global__ void __launch_bounds__(256)
    k_chol_diag(int b, T* __restrict__ G, int64_t ldg, T* __restrict__ Li, int64_t ldi,
                const T* __restrict__ maxd, T tol, int* __restrict__ defl,
                int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char ch_smem[];
  T(*a)[CH_NB + 1] = reinterpret_cast<T(*)[CH_NB + 1]>(ch_smem);
  T(*inv)[CH_NB + 1] = reinterpret_cast<T(*)[CH_NB + 1]>(ch_smem + sizeof(T) * CH_NB * (CH_NB + 1));
  __shared__ int bad, dj;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  const T thr = tol * (*maxd);
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    a[i][j] = (j <= i) ? G[(int64_t)i * ldg + j] : (T)0;
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      const T d = a[j][j];
      int f = 0;
      if (!isfinite((double)d)) {
        bad = 1;
        f = 1;
      } else if (!(d > thr)) {
        f = 1;
      }
      dj = f;
      a[j][j] = f ? (T)1 : sqrt(d);
      if (defl) defl[j] = f;
    }
    __syncthreads();
    const T djj = a[j][j];
    const int f = dj;
    for (int i = j + 1 + tid; i < b; i += blockDim.x) a[i][j] = f ? (T)0 : a[i][j] / djj;
    __syncthreads();
    const int rem = b - j - 1;
    if (!f) {
      for (int e = tid; e < rem * rem; e += blockDim.x) {
        const int i = j + 1 + e / rem, k = j + 1 + e % rem;
        if (k <= i) a[i][k] -= a[i][j] * a[k][j];
      }
    }
    __syncthreads();
  }
  // inverse of the lower-triangular block, one column per thread
  for (int c = tid; c < b; c += blockDim.x) {
    for (int i = 0; i < b; ++i) {
      T sacc = (i == c) ? (T)1 : (T)0;
      for (int k = c; k < i; ++k) sacc -= a[i][k] * inv[k][c];
      inv[i][c] = (i < c) ? (T)0 : sacc / a[i][i];
    }
  }
  __syncthreads();
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    G[(int64_t)i * ldg + j] = (j <= i) ? a[i][j] : (T)0;
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
  const int dt = std::is_same<T, double>::value ? DT_F64 : DT_F32;
  const T tol = std::is_same<T, double>::value ? (T)1e-12 : (T)1e-6;
  Arena ar(st);
  SPM_ALLOC(ar, T, P, r * CH_NB);
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
  const int smem = (int)(2 * sizeof(T) * CH_NB * (CH_NB + 1));
  SPM_CUDA_TRY(cudaFuncSetAttribute(k_chol_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  for (int64_t kb = 0; kb < r; kb += CH_NB) {
    const int b = (int)min64(CH_NB, r - kb);
    k_chol_diag<T><<<1, 256, smem, st>>>(b, G + kb * ldg + kb, ldg, Li + kb * ldi + kb, ldi, maxd,
                                         tol, defl + kb, status);
    SPM_LAUNCH_CHECK();
    const int64_t rest = r - kb - b;
    if (rest > 0) {
      // P = G21 * Linv_kk^T   (rest x b), deflated columns forced to zero
      View g21 = rowmajor(G + (kb + b) * ldg + kb, dt, ldg);
      View lkT = transpose(rowmajor(Li + kb * ldi + kb, dt, ldi));
      SPM_TRY(gemm_simt(rest, b, b, 1.0, g21, lkT, 0.0, mrowmajor(P, dt, CH_NB), st));
      k_zero_defl_cols<T><<<grid_for(rest * b), 256, 0, st>>>(rest, b, P, CH_NB, defl + kb);
      SPM_LAUNCH_CHECK();
      // G22 -= P P^T
      SPM_TRY(gemm_simt(rest, rest, b, -1.0, rowmajor(P, dt, CH_NB),
                        transpose(rowmajor(P, dt, CH_NB)), 1.0,
                        mrowmajor(G + (kb + b) * ldg + (kb + b), dt, ldg), st));
      // L21 = P
      k_copy_block<T><<<grid_for(rest * b), 256, 0, st>>>((int)rest, b, P, CH_NB,
                                                           G + (kb + b) * ldg + kb, ldg);
      SPM_LAUNCH_CHECK();
    }
  }
  // off-diagonal blocks of L^{-1}: Linv[i, 0:ib] = -Linv_ii * (L[i, 0:ib] * Linv[0:ib, 0:ib])
  for (int64_t ib = CH_NB; ib < r; ib += CH_NB) {
    const int b = (int)min64(CH_NB, r - ib);
    SPM_TRY(gemm_simt(b, ib, ib, 1.0, rowmajor(G + ib * ldg, dt, ldg), rowmajor(Li, dt, ldi), 0.0,
                      mrowmajor(Tm, dt, ib), st));
    SPM_TRY(gemm_simt(b, ib, b, -1.0, rowmajor(Li + ib * ldi + ib, dt, ldi), rowmajor(Tm, dt, ib),
                      0.0, mrowmajor(Li + ib * ldi, dt, ldi), st));
  }
  return SPM_OK;
}

int cholesky_inv(int64_t r, void* G, int64_t ldg, void* Linv, int64_t ldi, int dt, int* defl,
                 int* status, cudaStream_t st) {
  if (dt == DT_F64) return cholesky_inv_t<double>(r, (double*)G, ldg, (double*)Linv, ldi, defl, status, st);
  if (dt == DT_F32) return cholesky_inv_t<float>(r, (float*)G, ldg, (float*)Linv, ldi, defl, status, st);
  return SPM_EINVAL;
}

// Replace the deflated columns of X (rows x c) by Gaussian columns scaled by
// 1/sqrt(rows); Philox4x32-10 keyed by `seed`, counter (row, column, 0, 3).
template <typename T>
__global__ void k_fill_deflated(int64_t rows, int64_t c, T* __restrict__ X, int64_t ldx,
                                const int* __restrict__ defl, uint32_t seed) {
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
// Parallel cyclic Jacobi (round-robin ordering): every round rotates n/2
// disjoint index pairs at once.  The new matrix is J^T A J with J a direct sum
// of 2 x 2 rotations, so each 2 x 2 block of the new matrix depends only on
// one 2 x 2 block of the old one; the kernel double-buffers A and needs one
// grid-wide barrier per round.  Launched cooperatively (all CTAs resident);
// the barrier spin is bounded and reports SPM_ETIMEOUT on expiry.
struct GridBar {
  unsigned* count;
  unsigned* gen;
};

__device__ __forceinline__ bool grid_sync(GridBar gb, unsigned nblocks, int* status) {
  __syncthreads();
  __shared__ int timed_out;
  if (threadIdx.x == 0) {
    timed_out = 0;
    volatile unsigned* vgen = gb.gen;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(gb.count, 1u) + 1u;
    if (arrived == nblocks) {
      *gb.count = 0;
      __threadfence();
      atomicAdd(gb.gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (clock64() - t0 > (1ll << 32)) {
          set_status(status, DEV_TIMEOUT);
          timed_out = 1;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return timed_out == 0;
}

__device__ __forceinline__ int rr_player(int pos, int r, int np) {
  return pos == 0 ? 0 : 1 + ((pos - 1 + r) % (np - 1));
}

template <typename T>
__device__ __forceinline__ void rr_pair(int i, int r, int np, int n, int& p, int& q, bool& active) {
  const int a = rr_player(i, r, np), b = rr_player(np - 1 - i, r, np);
  p = min(a, b);
  q = max(a, b);
  active = q < n;
}

template <typename T>
__device__ __forceinline__ void rot_params(const T* A, int64_t lda, int p, int q, bool active, T& c,
                                           T& s) {
  c = (T)1;
  s = (T)0;
  if (!active) return;
  const T apq = A[(int64_t)p * lda + q];
  const T app = A[(int64_t)p * lda + p];
  const T aqq = A[(int64_t)q * lda + q];
  const T eps = std::is_same<T, double>::value ? (T)1e-300 : (T)1e-37;
  if (fabs((double)apq) <= (double)eps) return;
  const T tau = (aqq - app) / ((T)2 * apq);
  const T t = (tau >= (T)0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
  c = (T)1 / sqrt((T)1 + t * t);
  s = t * c;
}

template <typename T>
__global__ void __launch_bounds__(512)
    k_jacobi(int n, int np, T* __restrict__ A0, T* __restrict__ A1, int64_t lda, T* __restrict__ V,
             int64_t ldv, int max_sweeps, double tol2, GridBar gb, double* __restrict__ offacc,
             int* __restrict__ status, int* __restrict__ which) {
  const unsigned nb = gridDim.x;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
  const int hp = np / 2;
  T* Acur = A0;
  T* Anew = A1;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // convergence test on the current matrix
    double off = 0.0, dia = 0.0;
    for (int64_t e = gtid; e < (int64_t)n * n; e += gsz) {
      const int64_t i = e / n, j = e % n;
      const double v = (double)Acur[i * lda + j];
      if (i == j) dia += v * v;
      else off += v * v;
    }
    if (gtid == 0) {
      offacc[2 * (sweep & 1)] = 0.0;
      offacc[2 * (sweep & 1) + 1] = 0.0;
    }
    if (!grid_sync(gb, nb, status)) return;
    {
      __shared__ double red_off[32], red_dia[32];
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xFFFFFFFFu, off, o);
        dia += __shfl_xor_sync(0xFFFFFFFFu, dia, o);
      }
      if ((threadIdx.x & 31) == 0) {
        red_off[threadIdx.x >> 5] = off;
        red_dia[threadIdx.x >> 5] = dia;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double so = 0.0, sd = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
          so += red_off[w];
          sd += red_dia[w];
        }
        atomicAdd(&offacc[2 * (sweep & 1)], so);
        atomicAdd(&offacc[2 * (sweep & 1) + 1], sd);
      }
    }
    if (!grid_sync(gb, nb, status)) return;
    const double offv = *((volatile double*)&offacc[2 * (sweep & 1)]);
    const double diav = *((volatile double*)&offacc[2 * (sweep & 1) + 1]);
    if (offv <= tol2 * (offv + diav)) break;
    for (int r = 0; r < np - 1; ++r) {
      // 2x2 blocks of the new matrix
      for (int64_t w = gtid; w < (int64_t)hp * hp; w += gsz) {
        const int bi = (int)(w / hp), bj = (int)(w % hp);
        int pi, qi, pj, qj;
        bool ai, aj;
        rr_pair<T>(bi, r, np, n, pi, qi, ai);
        rr_pair<T>(bj, r, np, n, pj, qj, aj);
        T ci, si, cj, sj;
        rot_params<T>(Acur, lda, pi, qi, ai, ci, si);
        rot_params<T>(Acur, lda, pj, qj, aj, cj, sj);
        // rows present: pi always (< n unless pi itself is the dummy, impossible: p < q)
        const bool rq = qi < n, cq = qj < n;
        const T m00 = Acur[(int64_t)pi * lda + pj];
        const T m01 = cq ? Acur[(int64_t)pi * lda + qj] : (T)0;
        const T m10 = rq ? Acur[(int64_t)qi * lda + pj] : (T)0;
        const T m11 = (rq && cq) ? Acur[(int64_t)qi * lda + qj] : (T)0;
        // J_i^T M
        const T t00 = ci * m00 - si * m10, t01 = ci * m01 - si * m11;
        const T t10 = si * m00 + ci * m10, t11 = si * m01 + ci * m11;
        // (J_i^T M) J_j
        T n00 = cj * t00 - sj * t01, n01 = sj * t00 + cj * t01;
        T n10 = cj * t10 - sj * t11, n11 = sj * t10 + cj * t11;
        if (bi == bj && ai) {
          n01 = (T)0;
          n10 = (T)0;
        }
        Anew[(int64_t)pi * lda + pj] = n00;
        if (cq) Anew[(int64_t)pi * lda + qj] = n01;
        if (rq) Anew[(int64_t)qi * lda + pj] = n10;
        if (rq && cq) Anew[(int64_t)qi * lda + qj] = n11;
      }
      // V <- V J (column pairs)
      for (int64_t w = gtid; w < (int64_t)n * hp; w += gsz) {
        const int row = (int)(w / hp), bj = (int)(w % hp);
        int pj, qj;
        bool aj;
        rr_pair<T>(bj, r, np, n, pj, qj, aj);
        if (!aj) continue;
        T cj, sj;
        rot_params<T>(Acur, lda, pj, qj, aj, cj, sj);
        const T vp = V[(int64_t)row * ldv + pj], vq = V[(int64_t)row * ldv + qj];
        V[(int64_t)row * ldv + pj] = cj * vp - sj * vq;
        V[(int64_t)row * ldv + qj] = sj * vp + cj * vq;
      }
      if (!grid_sync(gb, nb, status)) return;
      T* tmp = Acur;
      Acur = Anew;
      Anew = tmp;
    }
  }
  if (gtid == 0) *which = (Acur == A0) ? 0 : 1;
}

template <typename T>
__global__ void k_eye(int64_t n, T* V, int64_t ldv) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    V[(e / n) * ldv + (e % n)] = (e / n == e % n) ? (T)1 : (T)0;
}

// Sort eigenvalues descending and permute eigenvector columns accordingly.
template <typename T>
__global__ void k_eig_sort(int n, const T* __restrict__ A0, const T* __restrict__ A1, int64_t lda,
                           const int* __restrict__ which, const T* __restrict__ Vin, int64_t ldvi,
                           T* __restrict__ Vout, int64_t ldvo, T* __restrict__ lam) {
  const T* A = (*which == 0) ? A0 : A1;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const T li = A[(int64_t)i * lda + i];
    __shared__ int rk;
    if (threadIdx.x == 0) rk = 0;
    __syncthreads();
    int cnt = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const T lj = A[(int64_t)j * lda + j];
      if (lj > li || (lj == li && j < i)) ++cnt;
    }
    atomicAdd(&rk, cnt);
    __syncthreads();
    const int pos = rk;
    if (threadIdx.x == 0) lam[pos] = li;
    for (int row = threadIdx.x; row < n; row += blockDim.x)
      Vout[(int64_t)row * ldvo + pos] = Vin[(int64_t)row * ldvi + i];
    __syncthreads();
  }
}

template <typename T>
static int sym_eig_t(int64_t r, T* A, int64_t lda, T* V, int64_t ldv, T* lam, int* status,
                     cudaStream_t st) {
  const int n = (int)r;
  const int np = n + (n & 1);
  Arena ar(st);
  SPM_ALLOC(ar, T, A1, r * r);
  SPM_ALLOC(ar, T, Vw, r * r);
  SPM_ALLOC(ar, unsigned, bar, 2);
  SPM_ALLOC(ar, double, offacc, 4);
  SPM_ALLOC(ar, int, which, 1);
  SPM_CUDA_TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
  k_eye<T><<<grid_for(r * r), 256, 0, st>>>(r, Vw, r);
  SPM_LAUNCH_CHECK();
  k_copy_block<T><<<grid_for(r * r), 256, 0, st>>>(n, n, A, lda, A1, r);
  SPM_LAUNCH_CHECK();
  SPM_CUDA_TRY(cudaMemsetAsync(which, 0, sizeof(int), st));
  int dev = 0, sms = 0, per_sm = 0;
  SPM_CUDA_TRY(cudaGetDevice(&dev));
  SPM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  auto kern = k_jacobi<T>;
  SPM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, 0));
  if (per_sm < 1) return SPM_ECUDA;
  const int64_t work = (int64_t)(np / 2) * (np / 2) + (int64_t)n * (np / 2);
  int blocks = (int)min64(cdiv(work, 512 * 4), (int64_t)sms);
  if (blocks < 1) blocks = 1;
  const bool is64 = std::is_same<T, double>::value;
  const int max_sweeps = is64 ? 30 : 20;
  // stop when the off-diagonal mass reaches the rounding floor: (10 n eps)^2 relative
  const double eps = is64 ? 1.1102230246251565e-16 : 5.960464477539063e-08;
  const double tol = (10.0 * n * eps) * (10.0 * n * eps);
  GridBar gb{bar, bar + 1};
  SPM_ALLOC(ar, T, A2, r * r);
  T* a0 = A1;  // the kernel works on two private copies (ld r)
  T* a1 = A2;
  int64_t ldw = r;
  int mx = max_sweeps;
  double tl = tol;
  void* args[] = {(void*)&n, (void*)&np, (void*)&a0, (void*)&a1, (void*)&ldw, (void*)&Vw,
                  (void*)&ldw, (void*)&mx, (void*)&tl, (void*)&gb, (void*)&offacc,
                  (void*)&status, (void*)&which};
  SPM_CUDA_TRY(cudaLaunchCooperativeKernel((void*)kern, dim3(blocks), dim3(512), args, 0, st));
  count_launch();
  k_eig_sort<T><<<(unsigned)min(n, 1024), 128, 0, st>>>(n, a0, a1, ldw, which, Vw, ldw, V, ldv, lam);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

int sym_eig(int64_t r, void* A, int64_t lda, void* V, int64_t ldv, void* lam, int dt, int* status,
            cudaStream_t st) {
  if (r <= 0) return SPM_OK;
  if (r > 0x3FFFFFFF) return SPM_EUNSUPPORTED;
  if (dt == DT_F64) return sym_eig_t<double>(r, (double*)A, lda, (double*)V, ldv, (double*)lam, status, st);
  if (dt == DT_F32) return sym_eig_t<float>(r, (float*)A, lda, (float*)V, ldv, (float*)lam, status, st);
  return SPM_EINVAL;
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
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
      const double v = by_col ? ldd<T>(X + t * rs + l * cs) : ldd<T>(X + l * rs + t * cs);
      s += v * v;
    }
    red[threadIdx.x] = s;
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
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    double f = s[by_rows ? i : j];
    if (inv) f = (f != 0.0) ? 1.0 / f : 0.0;
    T* p = X + i * rs + j * cs;
    *p = (T)((double)*p * f);
  }
}

int scale_lines(int64_t rows, int64_t cols, MView X, bool rows_not_cols, const double* s, bool inv,
                cudaStream_t st) {
  const int g = grid_for(rows * cols);
  if (X.dt == DT_F32) k_scale_lines<float><<<g, 256, 0, st>>>(rows, cols, (float*)X.p, X.rs, X.cs, rows_not_cols, s, inv);
  else if (X.dt == DT_F64) k_scale_lines<double><<<g, 256, 0, st>>>(rows, cols, (double*)X.p, X.rs, X.cs, rows_not_cols, s, inv);
  else return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

template <typename T>
__global__ void k_sumsq(int64_t rows, int64_t cols, const T* __restrict__ X, int64_t rs, int64_t cs,
                        double* acc) {
  __shared__ double red[256];
  double s = 0.0;
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = ldd<T>(X + (e / cols) * rs + (e % cols) * cs);
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(acc, red[0]);
}

int sumsq(int64_t rows, int64_t cols, View X, double* acc, cudaStream_t st) {
  const int g = grid_for(rows * cols);
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
    double best = -1.0;
    int64_t idx = 0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
      const double v = fabs((double)U[i * rs + j * cs]);
      if (v > best) {
        best = v;
        idx = i;
      }
    }
    bv[threadIdx.x] = best;
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

int sign_fix(int64_t m, int64_t k, int64_t n, MView U, MView Vt, cudaStream_t st) {
  Arena ar(st);
  SPM_ALLOC(ar, int, flip, k);
  const int g = (int)min64(k, 152 * 8);
  if (U.dt == DT_F32) {
    k_sign_flags<float><<<g, 256, 0, st>>>(m, k, (const float*)U.p, U.rs, U.cs, flip);
    k_apply_flags<float><<<grid_for(m * k), 256, 0, st>>>(m, k, (float*)U.p, U.rs, U.cs, true, flip);
    k_apply_flags<float><<<grid_for(k * n), 256, 0, st>>>(k, n, (float*)Vt.p, Vt.rs, Vt.cs, false, flip);
  } else if (U.dt == DT_F64) {
    k_sign_flags<double><<<g, 256, 0, st>>>(m, k, (const double*)U.p, U.rs, U.cs, flip);
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
