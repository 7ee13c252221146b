// Kernels of the factored Nystrom output (Algorithm 3 with a shifted Cholesky
// finish): the test matrix T = S Y, the shift C <- C + nu T with nu computed on
// the device, and the eigenvalues lam = max(sigma^2 - nu, 0).
//
// With T = S Y the Nystrom output of Algorithm 3 is C = C~ Y = A T and
// W = Y^T W~ Y = T^T A T.  The factored form approximates A + nu I instead
// (C_nu = C + nu T, W_nu = T^T C_nu, positive definite), factors
// W_nu = L L^T, F = C_nu L^{-T} = Q_F R (orthonormal Q_F), R = U~ Sigma V^T,
// and returns U = Q_F U~ (orthonormal to working precision however small
// Sigma gets) and
// lam = max(Sigma^2 - nu, 0): A_hat = U diag(lam) U^T.  The paper leaves W^+
// unspecified; nu = sqrt(n) 2^-52 |C|_F is the reading used.
#include <math.h>

#include "internal.cuh"

namespace spm {

// out[j, c] = sum_t sign(j, t) / sqrt(s) * Y[col(j, t), c]  (row j of S times Y)
template <typename T>
__global__ void k_sketch_left(int64_t n, int s, const int32_t* __restrict__ cols,
                              const int8_t* __restrict__ signs, const T* __restrict__ Y, int64_t ldy,
                              int64_t p, T* __restrict__ out, int64_t ldo, T scale) {
  const int64_t total = n * p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / p, c = e % p;
    T acc = (T)0;
    for (int t = 0; t < s; ++t) {
      const T y = Y[(int64_t)cols[j * s + t] * ldy + c];
      acc += signs[j * s + t] < 0 ? -y : y;
    }
    out[j * ldo + c] = acc * scale;
  }
}

int sketch_left_dev(const spm_sketch* S, const void* Y, int dt, int64_t ldy, int64_t p, void* out,
                    int64_t ldo, cudaStream_t st) {
  if (dense_kind(S)) return SPM_EUNSUPPORTED;
  if (S->n <= 0 || p <= 0) return SPM_OK;
  const int s = S->kind == SPM_SKETCH_IDENTITY ? 1 : S->s;
  const double scale = S->kind == SPM_SKETCH_IDENTITY ? 1.0 : 1.0 / sqrt((double)S->s);
  const int g = (int)min64(cdiv(S->n * p, 256), 152 * 16);
  if (dt == DT_F64)
    k_sketch_left<double><<<g, 256, 0, st>>>(S->n, s, S->cols, S->signs, (const double*)Y, ldy, p,
                                             (double*)out, ldo, scale);
  else if (dt == DT_F32)
    k_sketch_left<float><<<g, 256, 0, st>>>(S->n, s, S->cols, S->signs, (const float*)Y, ldy, p,
                                            (float*)out, ldo, (float)scale);
  else
    return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

// nu = sqrt(n) 2^-52 sqrt(*c_sumsq); C += nu T; *nu_out = nu (written by one thread)
template <typename T>
__global__ void k_nys_shift(int64_t n, int64_t p, T* __restrict__ C, int64_t ldc,
                            const T* __restrict__ Tm, int64_t ldt, const double* __restrict__ c_sumsq,
                            double* __restrict__ nu_out) {
  const double nu = sqrt((double)n) * 0x1.0p-52 * sqrt(*c_sumsq);
  if (blockIdx.x == 0 && threadIdx.x == 0) *nu_out = nu;
  const int64_t total = n * p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / p, c = e % p;
    C[j * ldc + c] = (T)((double)C[j * ldc + c] + nu * (double)Tm[j * ldt + c]);
  }
}

int nys_shift_dev(int64_t n, int64_t p, void* C, int64_t ldc, const void* Tm, int64_t ldt, int dt,
                  const double* c_sumsq, double* nu_out, cudaStream_t st) {
  const int g = (int)min64(cdiv(n * p, 256), 152 * 16);
  if (dt == DT_F64)
    k_nys_shift<double><<<g, 256, 0, st>>>(n, p, (double*)C, ldc, (const double*)Tm, ldt, c_sumsq, nu_out);
  else if (dt == DT_F32)
    k_nys_shift<float><<<g, 256, 0, st>>>(n, p, (float*)C, ldc, (const float*)Tm, ldt, c_sumsq, nu_out);
  else
    return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

// From the squared singular values sig2 of F (descending): lam = max(sig2 - nu, 0)
// in the output type, and sigma = sqrt(sig2) (1 where sig2 is 0).
template <typename TS, typename TO>
__global__ void k_nys_lambda(int64_t r, const TS* __restrict__ sig2, const double* __restrict__ nu,
                             double* __restrict__ sigma, TO* __restrict__ lam) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= r) return;
  const double v = fmax((double)sig2[i], 0.0);
  sigma[i] = v > 0.0 ? sqrt(v) : 1.0;
  lam[i] = (TO)fmax(v - *nu, 0.0);
}

int nys_lambda_dev(int64_t r, const void* sig2, int sdt, const double* nu, double* sigma, void* lam,
                   int ldt, cudaStream_t st) {
  const int g = (int)cdiv(r, 256);
#define SPM_NL(TS, TO) \
  k_nys_lambda<TS, TO><<<g, 256, 0, st>>>(r, (const TS*)sig2, nu, sigma, (TO*)lam)
  if (sdt == DT_F64 && ldt == DT_F64) SPM_NL(double, double);
  else if (sdt == DT_F64 && ldt == DT_F32) SPM_NL(double, float);
  else if (sdt == DT_F32 && ldt == DT_F64) SPM_NL(float, double);
  else if (sdt == DT_F32 && ldt == DT_F32) SPM_NL(float, float);
  else return SPM_EINVAL;
#undef SPM_NL
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

}  // namespace spm
