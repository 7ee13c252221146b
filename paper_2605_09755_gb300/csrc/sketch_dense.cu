// The two dense sketch families of Lemma 3.2 next to the sparse sign sketch:
//   item 1 -- S with independent entries +-1/sqrt(r1) (dense sign sketch);
//   item 3 -- the subsampled randomized Hadamard transform
//             S = (1/sqrt(r1)) D H I_{:,T}, D a random +-1 diagonal, H the
//             Sylvester Hadamard matrix H[j, k] = (-1)^popcount(j & k) of order
//             n' = 2^L >= n (A read as padded with zero columns), T r1 distinct
//             columns of H in the order they are drawn.
//
// Random draws (Philox4x32-10 keyed by the 64-bit seed, bit 1 = minus):
//   dense sign of (j, c):  counter (j_lo, j_hi, c >> 7, 4), word (c >> 5) & 3, bit c & 31;
//   SRHT sign D_j:         counter (b_lo, b_hi, 0, 5), b = j >> 7, word (j >> 5) & 3, bit j & 31;
//   SRHT draw u:           counter (b_lo, b_hi, 0, 6), b = u >> 2, word u & 3;
//                          column = word >> (32 - L); repeats of earlier draws are skipped.
//
// A S for the dense sign sketch is a dense contraction: the tensor cores take it
// (A split into BF16 parts, the +-1 entries exact in BF16) when the product is
// stored in BF16, the CUDA-core GEMM when it is stored in FP32 or FP64.  A S for
// the SRHT is a fast Walsh-Hadamard transform of each row of A: one CTA holds a
// block of rows in shared memory, every thread keeps 32 elements that differ in
// five index bits in registers and applies the butterflies of those bits there,
// so a row of n' = 2^14 takes one pass straight from global memory and two
// passes through shared memory; the r1 sampled entries are then gathered.
// S^T X for both families runs the same products on X^T.
#include <math.h>

#include <type_traits>

#include "internal.cuh"
#include "rng.cuh"

namespace spm {

static constexpr int SRHT_THREADS = 256;
static constexpr int SRHT_ROW_ELEMS = 8192;   // elements of a CTA's row block when rows are short
static constexpr int SRHT_MAX_GROUPS = 4;     // 32-element groups per thread (n' <= 32768)
static constexpr int SRHT_MAX_L = 15;

static int64_t pad8_(int64_t x) { return round_up(x, 8); }

// ------------------------------------------------------------------ generation
// Dense sign sketch as BF16 +-1 (exact), n x ld row-major; one thread per
// (row j, 32 columns).  Columns [r1, ld) are zero.
__global__ void k_dense_sign(int64_t n, int r1, int64_t ld, uint32_t k0, uint32_t k1,
                             __nv_bfloat16* __restrict__ out) {
  const int nw = (int)((ld + 31) >> 5);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nw) return;
  const int64_t j = t / nw;
  const int w = (int)(t - j * nw);
  const u32x4 d = philox4x32_10((uint32_t)j, (uint32_t)(j >> 32), (uint32_t)(w >> 2), 4u, k0, k1);
  const uint32_t bits = pick(d, (uint32_t)(w & 3));
  const __nv_bfloat16 one = __float2bfloat16(1.f), mone = __float2bfloat16(-1.f),
                      zero = __float2bfloat16(0.f);
  for (int b = 0; b < 32; ++b) {
    const int c = w * 32 + b;
    if (c >= ld) break;
    out[j * ld + c] = c < r1 ? (((bits >> b) & 1u) ? mone : one) : zero;
  }
}

// SRHT diagonal as bits: word w holds D_j for j = 32 w .. 32 w + 31 (1 = minus).
__global__ void k_srht_signs(int words, uint32_t k0, uint32_t k1, uint32_t* __restrict__ dbits) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= words) return;
  const uint32_t b = (uint32_t)w >> 2;   // j >> 7 for j = 32 w
  const u32x4 d = philox4x32_10(b, 0u, 0u, 5u, k0, k1);
  dbits[w] = pick(d, (uint32_t)(w & 3));
}

// SRHT columns: one warp consumes the draws 32 at a time in order.  A draw is
// kept when its column was not taken by an earlier batch (bitmap in shared
// memory) nor by a lower lane of this batch; kept draws are written in lane
// order until r1 are held.  Bounded: stops after 2^26 draws, which r1 <= n'
// <= 2^15 never needs (about n' ln n' draws at most); cols is zeroed first, so
// every entry is a valid column whatever happens.
__global__ void k_srht_cols(int L, int r1, uint32_t k0, uint32_t k1, int32_t* __restrict__ cols) {
  extern __shared__ uint32_t taken[];
  const int lane = threadIdx.x;
  const int words = L >= 5 ? (1 << (L - 5)) : 1;
  for (int w = lane; w < words; w += 32) taken[w] = 0u;
  __syncwarp();
  int held = 0;
  uint32_t u = 0;
  while (held < r1) {
    const uint32_t uu = u + (uint32_t)lane;
    const u32x4 d = philox4x32_10(uu >> 2, 0u, 0u, 6u, k0, k1);
    const uint32_t word = pick(d, uu & 3u);
    const int cand = L > 0 ? (int)(word >> (32 - L)) : 0;
    const bool seen = (taken[cand >> 5] >> (cand & 31)) & 1u;
    const unsigned same = __match_any_sync(0xffffffffu, cand);
    const bool keep = !seen && (__ffs(same) - 1) == lane;
    const unsigned kept = __ballot_sync(0xffffffffu, keep);
    const int rank = __popc(kept & ((1u << lane) - 1u));
    if (keep && held + rank < r1) {
      cols[held + rank] = cand;
      atomicOr(&taken[cand >> 5], 1u << (cand & 31));
    }
    held = min(r1, held + __popc(kept));
    __syncwarp();
    u += 32;
    if (u >= (1u << 26)) break;
  }
}

// ------------------------------------------------------------------ SRHT apply
template <typename TO, typename T>
__device__ __forceinline__ void store_out(TO* out, TO* out_lo, int64_t off, T v) {
  if constexpr (std::is_same<TO, __nv_bfloat16>::value) {
    const float f = (float)v;
    const __nv_bfloat16 h = __float2bfloat16(f);
    out[off] = h;
    if (out_lo) out_lo[off] = __float2bfloat16(f - __bfloat162float(h));
  } else {
    out[off] = (TO)v;
  }
}

// Element j of row slot r in shared memory: rows are 2^Ls elements apart and
// the low five index bits are XORed with bits 5..9 and the row slot, so that
// the 32 lanes of a warp hit 32 banks in every pass.
__device__ __forceinline__ int srht_slot(int r, int j, int Ls) {
  return (r << Ls) + (j ^ (((j >> 5) ^ r) & 31));
}

// Index of element e of group g in the window of bits [lo, lo + 5).
__device__ __forceinline__ int srht_win(int g, int e, int lo) {
  return (g & ((1 << lo) - 1)) | (e << lo) | ((g >> lo) << (lo + 5));
}

// Butterflies (x + y, x - y) over the window bits flagged in `act`.
template <typename T>
__device__ __forceinline__ void fwht32(T (&v)[32], int act) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    if (act & (1 << s)) {
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        if (e & (1 << s)) continue;
        const T x = v[e], y = v[e | (1 << s)];
        v[e] = x + y;
        v[e | (1 << s)] = x - y;
      }
    }
  }
}

// out (m x r1) = A (m x n) S for the SRHT.  Ls = max(L, 5): rows are held as
// 2^Ls elements (zero beyond n); R rows per CTA iteration (R 2^Ls <= 8192 when
// rows are short, else R = 1, and each thread then handles 2^Ls / 8192 groups).
// Persistent over row blocks.  The per-thread sign masks of the first window do
// not depend on the row and are built once.
template <typename TA, typename TO, int Ls>
__global__ void __launch_bounds__(SRHT_THREADS)
    k_srht_apply(const TA* __restrict__ A, int64_t m, int64_t n, int64_t lda, int L, int R,
                 const uint32_t* __restrict__ dbits, const int32_t* __restrict__ cols, int r1,
                 TO* __restrict__ out, int64_t ldo, TO* __restrict__ out_lo, TA scale,
                 double* __restrict__ fro2) {
  extern __shared__ __align__(16) unsigned char srht_smem[];
  TA* sm = reinterpret_cast<TA*>(srht_smem);
  constexpr int gpr = 1 << (Ls - 5);             // groups per row
  const int gtot = R * gpr;                      // groups per iteration: 256, 512 or 1024
  constexpr int lo0 = Ls - 5;                    // first window: bits [lo0, Ls)
  const int act0 = L >= 5 ? 31 : ((1 << L) - 1); // bits >= L exist only as padding (L < 5)
  const int ng = gtot / SRHT_THREADS;
  uint32_t dmask[SRHT_MAX_GROUPS];
#pragma unroll
  for (int q = 0; q < SRHT_MAX_GROUPS; ++q) {
    uint32_t mk = 0u;
    if (q < ng) {
      const int g = (threadIdx.x + SRHT_THREADS * q) & (gpr - 1);
      for (int e = 0; e < 32; ++e) {
        const int j = g | (e << lo0);
        if (j < n) mk |= ((__ldg(dbits + (j >> 5)) >> (j & 31)) & 1u) << e;
      }
    }
    dmask[q] = mk;
  }
  TA psum = (TA)0;
  double facc = 0.0;
  const int64_t nblk = (m + R - 1) / R;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t i0 = blk * R;
    // pass 1: global memory -> registers (signs of D) -> butterflies -> shared memory
#pragma unroll 1
    for (int q = 0; q < SRHT_MAX_GROUPS; ++q) {
      if (q >= ng) break;
      const int gt = threadIdx.x + SRHT_THREADS * q;
      const int r = gt >> (Ls - 5), g = gt & (gpr - 1);
      const int64_t i = i0 + r;
      const TA* arow = A + i * lda;
      TA v[32];
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const int j = g | (e << lo0);
        TA x = (TA)0;
        if (i < m && j < n) x = __ldcs(arow + j);
        psum = fma(x, x, psum);
        v[e] = ((dmask[q] >> e) & 1u) ? -x : x;
      }
      fwht32(v, act0);
#pragma unroll
      for (int e = 0; e < 32; ++e) sm[srht_slot(r, g | (e << lo0), Ls)] = v[e];
    }
    facc += (double)psum;
    psum = (TA)0;
    __syncthreads();
    // remaining bits [0, lo0), five at a time (bits of the window at or above
    // lo0 were done in pass 1 and are only carried)
#pragma unroll
    for (int lo = 0; lo < lo0; lo += 5) {
      const int act = (1 << (min(lo + 5, lo0) - lo)) - 1;
#pragma unroll 1
      for (int q = 0; q < SRHT_MAX_GROUPS; ++q) {
        if (q >= ng) break;
        const int gt = threadIdx.x + SRHT_THREADS * q;
        const int r = gt >> (Ls - 5), g = gt & (gpr - 1);
        TA v[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = sm[srht_slot(r, srht_win(g, e, lo), Ls)];
        fwht32(v, act);
#pragma unroll
        for (int e = 0; e < 32; ++e) sm[srht_slot(r, srht_win(g, e, lo), Ls)] = v[e];
      }
      __syncthreads();
    }
    // gather the sampled columns
    const int tot = R * r1;
    for (int t = threadIdx.x; t < tot; t += SRHT_THREADS) {
      const int r = t / r1, c = t - r * r1;
      const int64_t i = i0 + r;
      if (i >= m) break;
      const TA y = sm[srht_slot(r, __ldg(cols + c), Ls)] * scale;
      store_out<TO, TA>(out, out_lo, i * ldo + c, y);
    }
    __syncthreads();
  }
  if (fro2) {
    __shared__ double red[SRHT_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) facc += __shfl_xor_sync(0xffffffffu, facc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = facc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < SRHT_THREADS / 32; ++w) s += red[w];
      atomicAdd(fro2, s);
    }
  }
}

template <typename TA, typename TO, int Ls>
static int launch_srht_ls(const spm_sketch* S, const TA* A, int64_t m, int64_t lda, TO* out,
                          int64_t ldo, TO* out_lo, double* fro2, cudaStream_t st) {
  constexpr int64_t Ns = (int64_t)1 << Ls;
  const int R = Ns <= SRHT_ROW_ELEMS ? (int)(SRHT_ROW_ELEMS / Ns) : 1;
  const size_t smem = (size_t)R * Ns * sizeof(TA);
  if (smem > 227 * 1024) return SPM_EUNSUPPORTED;
  auto kern = k_srht_apply<TA, TO, Ls>;
  SPM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0, per_sm = 0;
  SPM_CUDA_TRY(cudaGetDevice(&dev));
  SPM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SPM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SRHT_THREADS, smem));
  const int64_t nblk = cdiv(m, R);
  const int grid = (int)min64(nblk, (int64_t)max64(per_sm, 1) * sms);
  kern<<<grid, SRHT_THREADS, smem, st>>>(A, m, S->n, lda, S->hl, R, S->dbits, S->hcols, (int)S->r1,
                                         out, ldo, out_lo, (TA)(1.0 / sqrt((double)S->r1)), fro2);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

template <typename TA, typename TO>
static int launch_srht(const spm_sketch* S, const TA* A, int64_t m, int64_t lda, TO* out,
                       int64_t ldo, TO* out_lo, double* fro2, cudaStream_t st) {
  switch (S->hl > 5 ? S->hl : 5) {
#define SPM_LS(LS) \
  case LS: return launch_srht_ls<TA, TO, LS>(S, A, m, lda, out, ldo, out_lo, fro2, st)
    SPM_LS(5); SPM_LS(6); SPM_LS(7); SPM_LS(8); SPM_LS(9); SPM_LS(10);
    SPM_LS(11); SPM_LS(12); SPM_LS(13); SPM_LS(14); SPM_LS(15);
#undef SPM_LS
    default: return SPM_EUNSUPPORTED;
  }
}

static int srht_apply(const spm_sketch* S, const void* A, int a_dt, int64_t m, int64_t lda,
                      void* out, int out_dt, int64_t ldo, double* fro2, cudaStream_t st,
                      void* out_lo) {
  if (a_dt == DT_F32) {
    const float* a = (const float*)A;
    if (out_dt == DT_F32) return launch_srht<float, float>(S, a, m, lda, (float*)out, ldo, nullptr, fro2, st);
    if (out_dt == DT_F64) return launch_srht<float, double>(S, a, m, lda, (double*)out, ldo, nullptr, fro2, st);
    if (out_dt == DT_BF16)
      return launch_srht<float, __nv_bfloat16>(S, a, m, lda, (__nv_bfloat16*)out, ldo,
                                               (__nv_bfloat16*)out_lo, fro2, st);
  } else if (a_dt == DT_F64) {
    const double* a = (const double*)A;
    if (out_dt == DT_F64) return launch_srht<double, double>(S, a, m, lda, (double*)out, ldo, nullptr, fro2, st);
    if (out_dt == DT_F32) return launch_srht<double, float>(S, a, m, lda, (float*)out, ldo, nullptr, fro2, st);
    if (out_dt == DT_BF16)
      return launch_srht<double, __nv_bfloat16>(S, a, m, lda, (__nv_bfloat16*)out, ldo,
                                                (__nv_bfloat16*)out_lo, fro2, st);
  }
  return SPM_EINVAL;
}

// ------------------------------------------------------------------ dense sign apply
static int dense_sign_apply(const spm_sketch* S, const void* A, int a_dt, int64_t m, int64_t lda,
                            void* out, int out_dt, int64_t ldo, double* fro2, cudaStream_t st,
                            void* out_lo) {
  const int64_t n = S->n, r1 = S->r1;
  const double scale = 1.0 / sqrt((double)r1);
  Arena ar(st);
  if (fro2) SPM_TRY(sumsq(m, n, rowmajor(A, a_dt, lda), fro2, st));
  if (out_dt == DT_BF16) {
    // tensor cores: A ~ sum of BF16 parts (two when a hi/lo result is kept, else one)
    if (!tc_available()) return SPM_ECUDA;
    const int npass = out_lo ? 2 : 1;
    const int64_t np = pad8_(n);
    __nv_bfloat16* part[2] = {nullptr, nullptr};
    for (int q = 0; q < npass; ++q) {
      part[q] = ar.alloc<__nv_bfloat16>(m * np);
      if (!part[q]) return SPM_ENOMEM;
    }
    if (npass == 2)
      SPM_TRY(split_bf16(m, n, rowmajor(A, a_dt, lda), mrowmajor(part[0], DT_BF16, np),
                         mrowmajor(part[1], DT_BF16, np), st));
    else
      SPM_TRY(convert2d(m, n, rowmajor(A, a_dt, lda), mrowmajor(part[0], DT_BF16, np), st));
    SPM_ALLOC(ar, float, D, m * r1);
    TcOp a[2], b[2];
    for (int q = 0; q < npass; ++q) {
      a[q] = TcOp{part[q], np, false};
      b[q] = TcOp{S->dsign, S->ld_dsign, true};
    }
    SPM_TRY(gemm_tc(m, r1, n, npass, a, b, (float)scale, D, r1, 1, auto_splitk(m, r1, n), st));
    if (out_lo)
      return split_bf16(m, r1, rowmajor(D, DT_F32, r1), mrowmajor(out, DT_BF16, ldo),
                        mrowmajor(out_lo, DT_BF16, ldo), st);
    return convert2d(m, r1, rowmajor(D, DT_F32, r1), mrowmajor(out, DT_BF16, ldo), st);
  }
  if (out_dt != DT_F32 && out_dt != DT_F64) return SPM_EINVAL;
  // CUDA cores in the output's precision; the +-1 entries as FP32 (exact)
  SPM_ALLOC(ar, float, S32, n * r1);
  SPM_TRY(convert2d(n, r1, rowmajor(S->dsign, DT_BF16, S->ld_dsign), mrowmajor(S32, DT_F32, r1), st));
  return gemm_simt(m, r1, n, scale, rowmajor(A, a_dt, lda), rowmajor(S32, DT_F32, r1), 0.0,
                   mrowmajor(out, out_dt, ldo), st);
}

// ------------------------------------------------------------------ entry points
int dense_sketch_create(spm_sketch* S, cudaStream_t st) {
  const uint32_t k0 = (uint32_t)S->seed, k1 = (uint32_t)(S->seed >> 32);
  if (S->kind == SPM_SKETCH_DENSE_SIGN) {
    S->ld_dsign = pad8_(S->r1);
    const int64_t nw = (S->ld_dsign + 31) >> 5;
    if (cudaMallocAsync((void**)&S->dsign, S->n * S->ld_dsign * sizeof(__nv_bfloat16), st) != cudaSuccess)
      return SPM_ENOMEM;
    const int64_t threads = S->n * nw;
    k_dense_sign<<<(unsigned)cdiv(threads, 256), 256, 0, st>>>(S->n, (int)S->r1, S->ld_dsign, k0, k1,
                                                               S->dsign);
    SPM_LAUNCH_CHECK();
    return SPM_OK;
  }
  if (S->kind == SPM_SKETCH_SRHT) {
    int L = 0;
    while (((int64_t)1 << L) < S->n) ++L;
    if (L > SRHT_MAX_L) return SPM_EUNSUPPORTED;
    S->hl = L;
    const int words = L >= 5 ? (1 << (L - 5)) : 1;
    if (cudaMallocAsync((void**)&S->dbits, words * sizeof(uint32_t), st) != cudaSuccess) return SPM_ENOMEM;
    if (cudaMallocAsync((void**)&S->hcols, S->r1 * sizeof(int32_t), st) != cudaSuccess) return SPM_ENOMEM;
    SPM_CUDA_TRY(cudaMemsetAsync(S->hcols, 0, S->r1 * sizeof(int32_t), st));
    k_srht_signs<<<(unsigned)cdiv(words, 256), 256, 0, st>>>(words, k0, k1, S->dbits);
    SPM_LAUNCH_CHECK();
    k_srht_cols<<<1, 32, words * sizeof(uint32_t), st>>>(L, (int)S->r1, k0, k1, S->hcols);
    SPM_LAUNCH_CHECK();
    return SPM_OK;
  }
  return SPM_EINVAL;
}

void dense_sketch_free(spm_sketch* S) {
  if (S->dsign) cudaFreeAsync(S->dsign, S->stream);
  if (S->dbits) cudaFreeAsync(S->dbits, S->stream);
  if (S->hcols) cudaFreeAsync(S->hcols, S->stream);
}

int dense_sketch_apply(const spm_sketch* S, const void* A, int a_dt, int64_t m, int64_t lda,
                       void* out, int out_dt, int64_t ldo, double* fro2, cudaStream_t st,
                       void* out_lo) {
  if (S->kind == SPM_SKETCH_SRHT) return srht_apply(S, A, a_dt, m, lda, out, out_dt, ldo, fro2, st, out_lo);
  return dense_sign_apply(S, A, a_dt, m, lda, out, out_dt, ldo, fro2, st, out_lo);
}

// S^T X = (X^T S)^T: X^T and the product go through row-major scratch copies.
int dense_sketch_apply_t(const spm_sketch* S, const void* X, int x_dt, int64_t p, int64_t ldx,
                         void* out, int out_dt, int64_t ldo, cudaStream_t st) {
  if ((x_dt != DT_F32 && x_dt != DT_F64) || (out_dt != DT_F32 && out_dt != DT_F64))
    return SPM_EUNSUPPORTED;
  const int64_t n = S->n, r1 = S->r1;
  Arena ar(st);
  void* Xt = x_dt == DT_F64 ? (void*)ar.alloc<double>(p * n) : (void*)ar.alloc<float>(p * n);
  void* Yt = out_dt == DT_F64 ? (void*)ar.alloc<double>(p * r1) : (void*)ar.alloc<float>(p * r1);
  if (!Xt || !Yt) return SPM_ENOMEM;
  SPM_TRY(convert2d(p, n, transpose(rowmajor(X, x_dt, ldx)), mrowmajor(Xt, x_dt, n), st));
  SPM_TRY(dense_sketch_apply(S, Xt, x_dt, p, n, Yt, out_dt, r1, nullptr, st, nullptr));
  return convert2d(r1, p, transpose(rowmajor(Yt, out_dt, r1)), mrowmajor(out, out_dt, ldo), st);
}

}  // namespace spm
