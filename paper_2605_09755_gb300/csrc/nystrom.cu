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

#include "bulk.cuh"
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

// ------------------------------------------------------------------ fused Gaussian kernel
// C~ = K S for the Gaussian kernel K[i, j] = exp(-|x_i - x_j|^2 / (2 h^2)) of the
// points x_1..x_n in R^d (rows of X), K never formed: Algorithm 3's first
// product on a kernel matrix, the setting of the paper's kernel experiments.
//
// One CTA owns 32 rows i (lane = row) and a group of cw output columns, whose
// accumulators live in shared memory: acc[c][33] (a warp adding to one column
// for its 32 rows hits 32 distinct banks; the row-major write-out reads 32
// consecutive columns of one row, again 32 distinct banks), plus a trash row
// cw for padding entries and for entries of other column groups.  The CTA's
// warps split the points j: each lane forms its kernel value from its own point
// (registers) and x_j (a shared-memory broadcast), then adds value * sign /
// sqrt(s) into the accumulator of each column of row j of S.  Two warps may meet
// in a column, so the adds are shared-memory reductions.
//
// FP32 accumulates in 32-bit fixed point with 2^-F resolution: a kernel value
// kv becomes the bit pattern P of kv 2^F / sqrt(s) + 1.5 * 2^23, which for
// |kv 2^F / sqrt(s)| <= 2^22 is 0x4B400000 + round(kv 2^F / sqrt(s)) (one
// multiply-add per point); a positive entry adds P, a negative one adds ~P =
// -(0x4B400000 + round(...)) - 1, both as integers (red.shared.add.u32: native,
// unlike a floating-point add into shared memory).  The constants are taken off
// at the write-out: (p_c - m_c) 0x4B400000 - m_c for a column with p_c positive
// and m_c negative entries.  Integer addition is exact and associative, so the
// result does not depend on the order of the adds: it is reproducible bit for
// bit, and wrap-around of the partial sums cancels.  F = min(22,
// floor(log2(2^30 sqrt(s) / b_max))) (b_max: the most entries in one column)
// keeps the true sum of every column below 2^30 in magnitude; each term is
// rounded once, by at most 2^-(F+1).
//
// The entries of S are pre-expanded per column group into (byte offset of the
// accumulator row, sign mask) pairs, sp = round_up(s, 4) per point, padding
// entries naming the trash row.  The points and the pairs stream through a
// ring of shared-memory slots, GS_CHUNK points per slot, each filled by two
// 1-D bulk copies behind an mbarrier (waits bounded; a timeout stops the CTA
// and is recorded in the status word).  FP64 (the accuracy mode) reads points
// and (offset, value) pairs through L1/L2 and adds doubles.
namespace spm {

static constexpr int GS_WARPS = 32;
static constexpr int GS_DMAX = 32;
static constexpr int GS_CHUNK = 128;  // points per ring slot
static constexpr int GS_NSLOT = 4;
static constexpr int GS_SMEM_LIMIT = 227 * 1024;
static constexpr uint32_t GS_MAGIC = 0x4B400000u;  // bit pattern of 1.5 * 2^23

// Xp (n x dp, zero-padded) in the compute type TO
template <typename TI, typename TO>
__global__ void k_gauss_points(int64_t n, int d, const TI* __restrict__ X, int64_t ldx, int dp,
                               TO* __restrict__ Xp) {
  const int64_t total = n * dp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / dp;
    const int k = (int)(e % dp);
    Xp[e] = k < d ? (TO)X[i * ldx + k] : (TO)0;
  }
}

// Local column of entry t of point j in group g (cw: the trash row, when the
// column is outside the group or t >= s) and whether its sign is negative.
__device__ __forceinline__ int gs_local(int64_t j, int t, int s, int g, int cw,
                                        const int32_t* __restrict__ cols,
                                        const int8_t* __restrict__ signs, bool* neg) {
  *neg = false;
  if (t >= s) return cw;
  const int c = cols[j * s + t] - g * cw;
  if (c < 0 || c >= cw) return cw;
  *neg = signs[j * s + t] < 0;
  return c;
}

// FP32 entries, per group g and point j in quads of 4: {4 byte offsets of the
// accumulator rows, 4 sign masks (0 or ~0)}
__global__ void k_gauss_codes(int64_t n, int s, int sp, const int32_t* __restrict__ cols,
                              const int8_t* __restrict__ signs, int cw, int groups,
                              uint32_t* __restrict__ code) {
  const int64_t per = n * sp, total = per * groups;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(e / per);
    const int64_t r = e % per, j = r / sp;
    const int t = (int)(r % sp);
    bool neg;
    const int lc = gs_local(j, t, s, g, cw, cols, signs, &neg);
    uint32_t* q = code + ((int64_t)g * n * sp + j * sp + (t & ~3)) * 2;
    q[t & 3] = (uint32_t)lc * 132u;
    q[4 + (t & 3)] = neg ? 0xFFFFFFFFu : 0u;
  }
}

// FP64 pairs: offs = byte offset of the accumulator row, vals = sign / sqrt(s)
__global__ void k_gauss_pairs(int64_t n, int s, const int32_t* __restrict__ cols,
                              const int8_t* __restrict__ signs, int cw, int groups, double scale,
                              int32_t* __restrict__ offs, double* __restrict__ vals) {
  const int64_t per = n * s, total = per * groups;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(e / per);
    const int64_t r = e % per;
    bool neg;
    const int lc = gs_local(r / s, (int)(r % s), s, g, cw, cols, signs, &neg);
    offs[e] = lc * 33 * 8;
    vals[e] = lc == cw ? 0.0 : (neg ? -scale : scale);
  }
}

// entries per column (all points): cnt[c] += 1, and cnt[r1 + c] += 1 when negative
__global__ void k_gauss_count(int64_t nnz, int r1, const int32_t* __restrict__ cols,
                              const int8_t* __restrict__ signs, int* __restrict__ cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    atomicAdd(cnt + cols[e], 1);
    if (signs[e] < 0) atomicAdd(cnt + r1 + cols[e], 1);
  }
}

// prm[0] = 2^F / sqrt(s), prm[1] = 2^-F (one block)
__global__ void k_gauss_scale(int r1, const int* __restrict__ cnt, double inv_sqrt_s,
                              float* __restrict__ prm) {
  __shared__ int red[32];
  int m = 0;
  for (int c = threadIdx.x; c < r1; c += blockDim.x) m = max(m, cnt[c]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
    m = max(m, 1);
    int F = 22;
    // largest F <= 22 with b_max 2^F / sqrt(s) <= 2^30
    while (F > 0 && ldexp((double)m * inv_sqrt_s, F) > 1073741824.0) --F;
    prm[0] = (float)ldexp(inv_sqrt_s, F);
    prm[1] = (float)ldexp(1.0, -F);
  }
}

__device__ __forceinline__ uint64_t gs_sub2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t gs_fma2(uint64_t a, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(d) : "l"(a), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t gs_pack(float lo, float hi) {
  return ((uint64_t)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
// 2^t (t <= 0): the kernel value exp(-d2 / (2 h^2)) = 2^(d2 * (-log2(e) / (2 h^2)))
__device__ __forceinline__ float gs_exp2(float t) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(t));
  return y;
}
// Reductions into the accumulators.  Volatile without a memory clobber: they
// stay in program order with each other and with the barriers, while the
// loads around them may be scheduled freely.
__device__ __forceinline__ void gs_red(uint32_t addr, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}
__device__ __forceinline__ void gs_red(uint32_t addr, double v) {
  asm volatile("red.shared.add.f64 [%0], %1;" ::"r"(addr), "d"(v));
}

template <typename T>
__device__ __forceinline__ void gs_zero(T* acc, int cw) {
  for (int e = threadIdx.x; e < (cw + 1) * 33; e += blockDim.x) acc[e] = (T)0;
}

struct GsArgs {
  int64_t n;
  const float4* Xp;      // n x DP4 float4
  const uint4* code;     // groups x n x SP4 x {offsets, masks}
  float c2;              // -log2(e) / (2 h^2)
  const float* prm;      // 2^F / sqrt(s), 2^-F
  const int* cnt;        // entries per column (r1), negative entries per column (r1)
  int cw, r1;
  uint32_t acc_bytes;    // (cw + 1) x 33 words, rounded up to 16 bytes
  float* out;
  int64_t ldo;
  int* status;
};

// FP32: squared distances by packed f32x2 arithmetic, fixed-point reductions,
// the ring described above; DP4 float4 per point, SP4 quads of entries per point
template <int DP4, int SP4>
__global__ void __launch_bounds__(GS_WARPS * 32, 1) k_gauss_sketch_f32(const __grid_constant__ GsArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t* acc = reinterpret_cast<uint32_t*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = blockIdx.y;
  const int64_t n = a.n;
  const int64_t i0 = (int64_t)blockIdx.x * 32, i = i0 + lane;
  constexpr uint32_t xbytes = GS_CHUNK * DP4 * 16, tbytes = GS_CHUNK * SP4 * 32;
  constexpr uint32_t slot_bytes = xbytes + tbytes;
  const uint32_t ring0 = smem_u32(smem_raw) + a.acc_bytes;
  const uint32_t bar0 = ring0 + GS_NSLOT * slot_bytes;
  const unsigned char* ring = smem_raw + a.acc_bytes;
  const int nchunks = (int)((n + GS_CHUNK - 1) / GS_CHUNK);
  const uint4* ctab = a.code + (int64_t)g * n * SP4 * 2;
  gs_zero(acc, a.cw);
  if (tid == 0) {
    for (int k = 0; k < GS_NSLOT; ++k) mbar_init(bar0 + 8 * k, 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int c) {
    const int64_t j0 = (int64_t)c * GS_CHUNK;
    const uint32_t rows = (uint32_t)min64(GS_CHUNK, n - j0);
    const uint32_t dst = ring0 + (uint32_t)(c % GS_NSLOT) * slot_bytes, bar = bar0 + 8 * (c % GS_NSLOT);
    mbar_expect(bar, rows * (DP4 * 16 + SP4 * 32));
    bulk_g2s(dst, a.Xp + j0 * DP4, rows * DP4 * 16, bar);
    bulk_g2s(dst + xbytes, ctab + j0 * SP4 * 2, rows * SP4 * 32, bar);
  };
  if (tid == 0)
    for (int c = 0; c < GS_NSLOT && c < nchunks; ++c) issue(c);
  uint64_t xi[2 * DP4];
#pragma unroll
  for (int k = 0; k < DP4; ++k) {
    const float4 v = i < n ? a.Xp[i * DP4 + k] : make_float4(0.f, 0.f, 0.f, 0.f);
    xi[2 * k] = gs_pack(v.x, v.y);
    xi[2 * k + 1] = gs_pack(v.z, v.w);
  }
  const uint32_t base = smem_u32(acc) + 4u * lane;
  const float c2 = a.c2, wf = a.prm[0];
  const float magic = __uint_as_float(GS_MAGIC);
  int c = 0;
  bool timed_out = false;
  for (; c < nchunks; ++c) {
    const int sl = c % GS_NSLOT;
    const bool to = !mbar_wait(bar0 + 8 * sl, (uint32_t)(c / GS_NSLOT) & 1u);
    if (!to) {
      const int rows = (int)min64(GS_CHUNK, n - (int64_t)c * GS_CHUNK);
      const float4* xs = reinterpret_cast<const float4*>(ring + (size_t)sl * slot_bytes);
      const uint4* ts = reinterpret_cast<const uint4*>(ring + (size_t)sl * slot_bytes + xbytes);
#pragma unroll 2
      for (int u = 0; u < GS_CHUNK / GS_WARPS; ++u) {
        const int jj = warp + GS_WARPS * u;
        if (jj >= rows) break;
        uint64_t a0 = 0, a1 = 0;
#pragma unroll
        for (int k = 0; k < DP4; ++k) {
          const float4 v = xs[jj * DP4 + k];
          a0 = gs_fma2(gs_sub2(xi[2 * k], gs_pack(v.x, v.y)), a0);
          a1 = gs_fma2(gs_sub2(xi[2 * k + 1], gs_pack(v.z, v.w)), a1);
        }
        const float d2 = (__uint_as_float((uint32_t)a0) + __uint_as_float((uint32_t)(a0 >> 32))) +
                         (__uint_as_float((uint32_t)a1) + __uint_as_float((uint32_t)(a1 >> 32)));
        const uint32_t P = __float_as_uint(fmaf(gs_exp2(d2 * c2), wf, magic));
#pragma unroll
        for (int q = 0; q < SP4; ++q) {
          const uint4 o = ts[(jj * SP4 + q) * 2], m = ts[(jj * SP4 + q) * 2 + 1];
          gs_red(base + o.x, P ^ m.x);
          gs_red(base + o.y, P ^ m.y);
          gs_red(base + o.z, P ^ m.z);
          gs_red(base + o.w, P ^ m.w);
        }
      }
    }
    // the slot has been read by every warp; a timeout anywhere stops the CTA
    if (__syncthreads_or(to ? 1 : 0)) {
      timed_out = true;
      break;
    }
    if (tid == 0 && c + GS_NSLOT < nchunks) {
      proxy_async_fence();
      issue(c + GS_NSLOT);
    }
  }
  if (timed_out) {
    if (tid == 0) {
      set_status(a.status, DEV_TIMEOUT);
      for (int k = c; k < c + GS_NSLOT && k < nchunks; ++k)   // copies still in flight
        mbar_wait(bar0 + 8 * (k % GS_NSLOT), (uint32_t)(k / GS_NSLOT) & 1u);
    }
    __syncthreads();
    return;
  }
  // write-out: take off the constants of the column's p_c positive and m_c
  // negative terms, (p_c - m_c) 0x4B400000 - m_c, then scale by 2^-F
  const int c0 = g * a.cw;
  const int cols = min(a.cw, a.r1 - c0);
  const int64_t rows = (n - i0) < 32 ? (n - i0) : 32;
  const float inv = a.prm[1];
  for (int64_t e = tid; e < rows * cols; e += blockDim.x) {
    const int64_t r = e / cols, cc = e % cols;
    const uint32_t all = (uint32_t)__ldg(a.cnt + c0 + cc), neg = (uint32_t)__ldg(a.cnt + a.r1 + c0 + cc);
    const uint32_t off = (all - 2u * neg) * GS_MAGIC - neg;
    a.out[(i0 + r) * a.ldo + c0 + cc] = (float)(int32_t)(acc[cc * 33 + r] - off) * inv;
  }
}

// FP64: plain per-dimension differences, points and pairs read through L1/L2;
// 16 warps (the point lives in 64 registers)
static constexpr int GS_WARPS64 = 16;
__global__ void __launch_bounds__(GS_WARPS64 * 32, 1)
    k_gauss_sketch_f64(int64_t n, int dp, const double* __restrict__ Xp, double c, int sp,
                       const int32_t* __restrict__ offs, const double* __restrict__ vals, int cw, int r1,
                       double* __restrict__ out, int64_t ldo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* acc = reinterpret_cast<double*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.y;
  const int64_t i0 = (int64_t)blockIdx.x * 32, i = i0 + lane;
  gs_zero(acc, cw);
  double xi[GS_DMAX];
#pragma unroll
  for (int k = 0; k < GS_DMAX; ++k) xi[k] = (i < n && k < dp) ? Xp[i * dp + k] : 0.0;
  const uint32_t base = smem_u32(acc) + 8u * lane;
  const int32_t* ot = offs + (int64_t)g * n * sp;
  const double* vt = vals + (int64_t)g * n * sp;
  __syncthreads();
  for (int64_t j = warp; j < n; j += GS_WARPS64) {
    const double* xj = Xp + j * dp;
    double d2 = 0.0;
#pragma unroll
    for (int k = 0; k < GS_DMAX; ++k)
      if (k < dp) {
        const double t = xi[k] - __ldg(xj + k);
        d2 = fma(t, t, d2);
      }
    const double kv = exp(d2 * c);
    for (int t = 0; t < sp; ++t) gs_red(base + __ldg(ot + j * sp + t), kv * __ldg(vt + j * sp + t));
  }
  __syncthreads();
  const int c0 = g * cw;
  const int ncols = min(cw, r1 - c0);
  const int64_t rows = (n - i0) < 32 ? (n - i0) : 32;
  for (int64_t e = threadIdx.x; e < rows * ncols; e += blockDim.x) {
    const int64_t r = e / ncols, cc = e % ncols;
    out[(i0 + r) * ldo + c0 + cc] = acc[cc * 33 + r];
  }
}

template <int DP4, int SP4>
static int launch_gs_f32(dim3 grid, size_t smem, cudaStream_t st, const GsArgs& a) {
  SPM_CUDA_TRY(cudaFuncSetAttribute(k_gauss_sketch_f32<DP4, SP4>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_gauss_sketch_f32<DP4, SP4><<<grid, GS_WARPS * 32, smem, st>>>(a);
  return SPM_OK;
}
template <int DP4>
static int launch_gs_f32_sp(int sp4, dim3 grid, size_t smem, cudaStream_t st, const GsArgs& a) {
  switch (sp4) {
    case 1: return launch_gs_f32<DP4, 1>(grid, smem, st, a);
    case 2: return launch_gs_f32<DP4, 2>(grid, smem, st, a);
    case 4: return launch_gs_f32<DP4, 4>(grid, smem, st, a);
    case 16: return launch_gs_f32<DP4, 16>(grid, smem, st, a);
    default: return SPM_EINVAL;
  }
}

// FP32 widths: points padded to 4, 8, 16 or 32 coordinates, entries to 4, 8,
// 16 or 64 per point
static int gs_dp(int64_t d) { return d <= 4 ? 4 : d <= 8 ? 8 : d <= 16 ? 16 : 32; }
static int gs_sp(int s) { return s <= 4 ? 4 : s <= 8 ? 8 : s <= 16 ? 16 : 64; }

int gauss_sketch_dev(const spm_sketch* S, const void* X, int xdt, int64_t n, int64_t d, int64_t ldx,
                     double h, void* out, int odt, int64_t ldo, cudaStream_t st, int* status) {
  if (dense_kind(S) || S->n != n) return SPM_EUNSUPPORTED;
  if (d < 1 || d > GS_DMAX || !(h > 0.0) || !std::isfinite(h)) return SPM_EINVAL;
  if ((xdt != DT_F32 && xdt != DT_F64) || (odt != DT_F32 && odt != DT_F64)) return SPM_EINVAL;
  if (n <= 0) return SPM_OK;
  const int64_t r1 = S->r1;
  const int s = S->kind == SPM_SKETCH_IDENTITY ? 1 : S->s;
  const double scale = S->kind == SPM_SKETCH_IDENTITY ? 1.0 : 1.0 / sqrt((double)S->s);
  const bool f32 = odt == DT_F32;
  const int es = (int)dt_size(odt);
  const int dp = f32 ? gs_dp(d) : (int)d;
  const int sp = f32 ? gs_sp(s) : s;
  // shared memory: (cw + 1) rows of 33 accumulators, and for FP32 the ring
  const int64_t ring = f32 ? (int64_t)GS_NSLOT * GS_CHUNK * (dp * 4 + sp * 8) + 8 * GS_NSLOT : 0;
  const int64_t cw_max = (GS_SMEM_LIMIT - ring - 16) / (33 * es) - 1;
  if (cw_max < 1) return SPM_EUNSUPPORTED;
  const int64_t groups = cdiv(r1, cw_max);
  const int64_t cw = cdiv(r1, groups);
  const int64_t blocks = cdiv(n, 32);
  if (blocks > 0x7FFFFFFF || groups > 65535 || cw > 0x7FFF) return SPM_EUNSUPPORTED;
  const int64_t acc_bytes = round_up((cw + 1) * 33 * es, 16);
  const size_t smem = (size_t)(acc_bytes + ring);
  Arena ar(st);
  void* Xp = ar.alloc<unsigned char>(n * dp * es);
  if (!Xp) return SPM_ENOMEM;
  const int ge = (int)min64(cdiv(n * dp, 256), 152 * 8);
  const int gt = (int)min64(cdiv(groups * n * sp, 256), 152 * 8);
#define SPM_GP(TI, TO) \
  k_gauss_points<TI, TO><<<ge, 256, 0, st>>>(n, (int)d, (const TI*)X, ldx, dp, (TO*)Xp)
  if (xdt == DT_F32 && odt == DT_F32) SPM_GP(float, float);
  else if (xdt == DT_F32) SPM_GP(float, double);
  else if (odt == DT_F32) SPM_GP(double, float);
  else SPM_GP(double, double);
#undef SPM_GP
  SPM_LAUNCH_CHECK();
  const dim3 grid((unsigned)blocks, (unsigned)groups);
  if (f32) {
    uint32_t* code = ar.alloc<uint32_t>(groups * n * sp * 2);
    int* cnt = ar.alloc<int>(2 * r1);
    float* prm = ar.alloc<float>(2);
    if (!code || !cnt || !prm) return SPM_ENOMEM;
    k_gauss_codes<<<gt, 256, 0, st>>>(n, s, sp, S->cols, S->signs, (int)cw, (int)groups, code);
    SPM_LAUNCH_CHECK();
    SPM_CUDA_TRY(cudaMemsetAsync(cnt, 0, 2 * r1 * sizeof(int), st));
    k_gauss_count<<<(int)min64(cdiv(n * s, 256), 152 * 8), 256, 0, st>>>(n * s, (int)r1, S->cols,
                                                                         S->signs, cnt);
    SPM_LAUNCH_CHECK();
    k_gauss_scale<<<1, 1024, 0, st>>>((int)r1, cnt, scale, prm);
    SPM_LAUNCH_CHECK();
    GsArgs a;
    a.n = n;
    a.Xp = (const float4*)Xp;
    a.code = (const uint4*)code;
    a.c2 = (float)(-1.0 / (2.0 * h * h * log(2.0)));   // 2^(d2 c2) = exp(-d2 / (2 h^2))
    a.prm = prm;
    a.cnt = cnt;
    a.cw = (int)cw;
    a.r1 = (int)r1;
    a.acc_bytes = (uint32_t)acc_bytes;
    a.out = (float*)out;
    a.ldo = ldo;
    a.status = status;
    int rc = SPM_EINVAL;
    switch (dp / 4) {
      case 1: rc = launch_gs_f32_sp<1>(sp / 4, grid, smem, st, a); break;
      case 2: rc = launch_gs_f32_sp<2>(sp / 4, grid, smem, st, a); break;
      case 4: rc = launch_gs_f32_sp<4>(sp / 4, grid, smem, st, a); break;
      case 8: rc = launch_gs_f32_sp<8>(sp / 4, grid, smem, st, a); break;
      default: break;
    }
    if (rc != SPM_OK) return rc;
  } else {
    int32_t* offs = ar.alloc<int32_t>(groups * n * s);
    double* vals = ar.alloc<double>(groups * n * s);
    if (!offs || !vals) return SPM_ENOMEM;
    k_gauss_pairs<<<gt, 256, 0, st>>>(n, s, S->cols, S->signs, (int)cw, (int)groups, scale, offs, vals);
    SPM_LAUNCH_CHECK();
    SPM_CUDA_TRY(cudaFuncSetAttribute(k_gauss_sketch_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    k_gauss_sketch_f64<<<grid, GS_WARPS64 * 32, smem, st>>>(n, dp, (const double*)Xp, -1.0 / (2.0 * h * h),
                                                            s, offs, vals, (int)cw, (int)r1,
                                                            (double*)out, ldo);
  }
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

}  // namespace spm
