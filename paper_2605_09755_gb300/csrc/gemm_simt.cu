// CUDA-core GEMM on strided views: the FP64 path of every product (the plain
// FP64 form of Algorithms 1-3) and the small FP32 products of the mixed path.
// C = alpha * A (M x K) * B (K x N) + beta * C.
#include <type_traits>

#include "internal.cuh"

namespace spm {

static constexpr int SG_BM = 64, SG_BN = 64, SG_BK = 16, SG_THREADS = 256;

// Load one element converted straight to the accumulator type (an FP32
// product never goes through FP64, whose conversions are slow on this part).
template <typename TACC, typename T>
__device__ __forceinline__ TACC ld_as(const T* p) {
  return (TACC)*p;
}
template <>
__device__ __forceinline__ float ld_as<float, __nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <>
__device__ __forceinline__ double ld_as<double, __nv_bfloat16>(const __nv_bfloat16* p) {
  return (double)__bfloat162float(*p);
}

template <typename TA, typename TB, typename TC, typename TACC>
__global__ void __launch_bounds__(SG_THREADS)
    k_gemm_simt(int64_t M, int64_t N, int64_t K, TACC alpha, const TA* __restrict__ A, int64_t ars,
                int64_t acs, const TB* __restrict__ B, int64_t brs, int64_t bcs, TACC beta,
                TC* __restrict__ C, int64_t crs, int64_t ccs, int64_t sA, int64_t sB, int64_t sC) {
  __shared__ TACC As[SG_BK][SG_BM + 1];
  __shared__ TACC Bs[SG_BK][SG_BN + 1];
  const int64_t bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int64_t row0 = (int64_t)blockIdx.y * SG_BM, col0 = (int64_t)blockIdx.x * SG_BN;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  TACC acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (TACC)0;
  const bool a_kfast = (acs == 1);
  const bool b_nfast = (bcs == 1);
  for (int64_t k0 = 0; k0 < K; k0 += SG_BK) {
#pragma unroll
    for (int q = 0; q < (SG_BM * SG_BK) / SG_THREADS; ++q) {
      const int e = tid + q * SG_THREADS;
      const int kk = a_kfast ? (e % SG_BK) : (e / SG_BM);
      const int ii = a_kfast ? (e / SG_BK) : (e % SG_BM);
      const int64_t gi = row0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < M && gk < K) ? ld_as<TACC>(A + gi * ars + gk * acs) : (TACC)0;
    }
#pragma unroll
    for (int q = 0; q < (SG_BN * SG_BK) / SG_THREADS; ++q) {
      const int e = tid + q * SG_THREADS;
      const int kk = b_nfast ? (e / SG_BN) : (e % SG_BK);
      const int jj = b_nfast ? (e % SG_BN) : (e / SG_BK);
      const int64_t gj = col0 + jj, gk = k0 + kk;
      Bs[kk][jj] = (gj < N && gk < K) ? ld_as<TACC>(B + gk * brs + gj * bcs) : (TACC)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SG_BK; ++kk) {
      TACC a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gi = row0 + ty + 16 * i;
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gj = col0 + tx + 16 * j;
      if (gj >= N) continue;
      TC* c = C + gi * crs + gj * ccs;
      TACC v = alpha * acc[i][j];
      if (beta != (TACC)0) v += beta * ld_as<TACC>(c);
      *c = (TC)v;
    }
  }
}

template <typename TA, typename TB, typename TC>
static int launch(int64_t M, int64_t N, int64_t K, double alpha, View A, View B, double beta,
                  MView C, cudaStream_t st, int batch, int64_t sA, int64_t sB, int64_t sC) {
  dim3 grid((unsigned)cdiv(N, SG_BN), (unsigned)cdiv(M, SG_BM), (unsigned)batch);
  if (cdiv(M, SG_BM) > 65535 || batch > 65535) return SPM_EUNSUPPORTED;
  constexpr bool any64 = sizeof(TA) == 8 || sizeof(TB) == 8 || sizeof(TC) == 8;
  using TACC = typename std::conditional<any64, double, float>::type;
  k_gemm_simt<TA, TB, TC, TACC><<<grid, SG_THREADS, 0, st>>>(
      M, N, K, (TACC)alpha, (const TA*)A.p, A.rs, A.cs, (const TB*)B.p, B.rs, B.cs, (TACC)beta,
      (TC*)C.p, C.rs, C.cs, sA, sB, sC);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

template <typename TA, typename TB>
static int dispatch_c(int64_t M, int64_t N, int64_t K, double alpha, View A, View B, double beta,
                      MView C, cudaStream_t st, int batch, int64_t sA, int64_t sB, int64_t sC) {
  if (C.dt == DT_F32) return launch<TA, TB, float>(M, N, K, alpha, A, B, beta, C, st, batch, sA, sB, sC);
  if (C.dt == DT_F64) return launch<TA, TB, double>(M, N, K, alpha, A, B, beta, C, st, batch, sA, sB, sC);
  return SPM_EINVAL;
}

template <typename TA>
static int dispatch_b(int64_t M, int64_t N, int64_t K, double alpha, View A, View B, double beta,
                      MView C, cudaStream_t st, int batch, int64_t sA, int64_t sB, int64_t sC) {
  if (B.dt == DT_F32) return dispatch_c<TA, float>(M, N, K, alpha, A, B, beta, C, st, batch, sA, sB, sC);
  if (B.dt == DT_F64) return dispatch_c<TA, double>(M, N, K, alpha, A, B, beta, C, st, batch, sA, sB, sC);
  return SPM_EINVAL;
}

int gemm_simt(int64_t M, int64_t N, int64_t K, double alpha, View A, View B, double beta, MView C,
              cudaStream_t st, int batch, int64_t sA, int64_t sB, int64_t sC) {
  if (M <= 0 || N <= 0) return SPM_OK;
  if (A.dt == DT_F32) return dispatch_b<float>(M, N, K, alpha, A, B, beta, C, st, batch, sA, sB, sC);
  if (A.dt == DT_F64) return dispatch_b<double>(M, N, K, alpha, A, B, beta, C, st, batch, sA, sB, sC);
  return SPM_EINVAL;
}

}  // namespace spm
