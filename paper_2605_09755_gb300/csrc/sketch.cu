// Sparse sign sketch S (Lemma 3.2 item 2), Gaussian Omega (Algorithm 1 input)
// and the sketch products A S (Algorithm 1 line 1, Algorithm 3 line 1) and
// S^T X (Algorithm 2 line 2, Algorithm 3 line 1).
//
// Layout of a sketch on the device
//   cols[n*s], signs[n*s]: entry t of row j in draw order (bit-exact with the
//     CPU oracle for the same seed).
//   Chunked CSC: rows j are grouped into chunks of CHUNK = 512; inside a chunk,
//   entries are sorted by column c and, within a column, by ascending j.
//   cptr[k*r1 + c] is the start of the (chunk k, column c) segment in ent[];
//   ent[] packs j (bits 0..30) and the sign (bit 31 set = minus).
//   The segments of chunk k form the contiguous range [k*CHUNK*s, ...).
#include <math.h>

#include <type_traits>

#include "internal.cuh"
#include "rng.cuh"

namespace spm {

static constexpr int CHUNK = 512;          // rows of S (columns of A) per tile
static constexpr int APPLY_ROWS = 32;      // rows of A per CTA (one per lane)
static constexpr int APPLY_WARPS = 32;
static constexpr int APPLY_THREADS = APPLY_WARPS * 32;
static constexpr int APPLY_TILE_LD = APPLY_ROWS + 1;   // padded: conflict-free
static constexpr uint32_t SIGN_BIT = 0x80000000u;
static constexpr int SACC_MAX_CG = 1100;   // accumulator columns per CTA (x 33 floats)
static constexpr int SACC_MAX_S = 8;       // entries of one chunk staged: CHUNK * s words

// ------------------------------------------------------------------ a1: generation
__global__ void k_sketch_gen(int64_t n, uint32_t r1, int s, uint32_t k0, uint32_t k1,
                             int32_t* __restrict__ cols, int8_t* __restrict__ signs,
                             int* __restrict__ status) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint32_t jlo = (uint32_t)j, jhi = (uint32_t)(j >> 32);
  int32_t chosen[64];
  uint32_t u = 0, blk = 0xFFFFFFFFu;
  u32x4 w = {0, 0, 0, 0};
  for (int t = 0; t < s; ++t) {
    for (;;) {
      const uint32_t b = u >> 2;
      if (b != blk) {
        w = philox4x32_10(jlo, jhi, b, 0u, k0, k1);
        blk = b;
      }
      const uint32_t word = pick(w, u & 3u);
      ++u;
      const int32_t cand = (int32_t)(((uint64_t)word * r1) >> 32);
      bool dup = false;
      for (int q = 0; q < t; ++q) dup |= (chosen[q] == cand);
      if (!dup) {
        chosen[t] = cand;
        break;
      }
      if (u > (1u << 26)) {  // cannot happen for s <= r1; bounded anyway
        set_status(status, DEV_TIMEOUT);
        chosen[t] = 0;
        break;
      }
    }
  }
  uint32_t sblk = 0xFFFFFFFFu;
  u32x4 sw = {0, 0, 0, 0};
  for (int t = 0; t < s; ++t) {
    const uint32_t b = (uint32_t)(t >> 7);
    if (b != sblk) {
      sw = philox4x32_10(jlo, jhi, b, 1u, k0, k1);
      sblk = b;
    }
    const uint32_t word = pick(sw, (uint32_t)((t >> 5) & 3));
    const uint32_t bit = (word >> (t & 31)) & 1u;
    cols[j * s + t] = chosen[t];
    signs[j * s + t] = bit ? (int8_t)-1 : (int8_t)1;
  }
}

__global__ void k_sketch_identity(int64_t n, int32_t* cols, int8_t* signs, uint32_t* ent,
                                  int64_t* cptr, int nchunks) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) {
    cols[j] = (int32_t)j;
    signs[j] = 1;
    ent[j] = (uint32_t)j;
  }
  // cptr[k*n + c]: column c lives only in chunk c / CHUNK
  const int64_t total = (int64_t)nchunks * n;
  for (int64_t q = j; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = q / n, c = q % n;
    const int64_t base = k * CHUNK;
    const int64_t len = min64(CHUNK, n - base);
    // segment (k, c) holds entry c only when c lies in chunk k
    cptr[q] = base + min64(max64(c - base, 0), len);
  }
  if (j == 0) cptr[total] = n;
}

// Stable counting sort of one chunk's entries by column (one CTA per chunk).
__global__ void k_chunk_sort(int64_t n, int r1, int s, const int32_t* __restrict__ cols,
                             const int8_t* __restrict__ signs, int64_t* __restrict__ cptr,
                             uint32_t* __restrict__ ent) {
  extern __shared__ int hist[];  // r1 + 1 ints
  const int k = blockIdx.x;
  const int64_t j0 = (int64_t)k * CHUNK;
  const int64_t j1 = min(n, j0 + CHUNK);
  const int64_t e0 = j0 * s, e1 = j1 * s;
  for (int c = threadIdx.x; c <= r1; c += blockDim.x) hist[c] = 0;
  __syncthreads();
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) atomicAdd(&hist[cols[e]], 1);
  __syncthreads();
  // exclusive scan over r1 bins by thread 0 of each warp-sized slice (simple, r1 small)
  if (threadIdx.x == 0) {
    int run = 0;
    for (int c = 0; c < r1; ++c) {
      const int v = hist[c];
      hist[c] = run;
      run += v;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < r1; c += blockDim.x) cptr[(int64_t)k * r1 + c] = e0 + hist[c];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t base = e0; base < e1; base += 32) {
      const int64_t e = base + lane;
      const bool valid = e < e1;
      const int c = valid ? cols[e] : -1 - lane;
      const unsigned mask = __match_any_sync(0xFFFFFFFFu, c);
      const int rank = __popc(mask & lt);
      const int leader = __ffs(mask) - 1;
      int pos = 0;
      if (valid) pos = hist[c] + rank;
      __syncwarp();
      if (valid && lane == leader) hist[c] += __popc(mask);
      __syncwarp();
      if (valid) {
        const uint32_t j = (uint32_t)(e / s);
        ent[e0 + pos] = j | (signs[e] < 0 ? SIGN_BIT : 0u);
      }
    }
  }
}

__global__ void k_set_i64(int64_t* p, int64_t v) { *p = v; }

// Segment bounds relative to each chunk's first entry, and per-entry tile offsets.
__global__ void k_apply_tables(int64_t nnz, int r1, int nchunks, const int64_t* __restrict__ cptr,
                               const uint32_t* __restrict__ ent, int2* __restrict__ seg,
                               uint32_t* __restrict__ entoff) {
  const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
  const int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t q = g0; q < (int64_t)nchunks * r1; q += gsz) {
    const int64_t base = cptr[(q / r1) * r1];
    seg[q] = make_int2((int)(cptr[q] - base), (int)(cptr[q + 1] - base));
  }
  for (int64_t e = g0; e < nnz; e += gsz) {
    const uint32_t v = ent[e];
    const uint32_t jj = (v & ~SIGN_BIT) % (uint32_t)CHUNK;
    entoff[e] = (jj * (uint32_t)APPLY_TILE_LD) | (v & SIGN_BIT);
  }
}

// Entry words of the shared-accumulator apply: tile offset, accumulator offset
// of the column inside its group of cg columns, sign.  ent[] is sorted by
// column inside each chunk, so the column of entry e is found by bisection of
// the chunk's segment starts.
__global__ void k_acc_tables(int64_t nnz, int r1, int nchunks, int cg,
                             const int64_t* __restrict__ cptr, const uint32_t* __restrict__ ent,
                             uint32_t* __restrict__ entacc) {
  const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += gsz) {
    const uint32_t v = ent[e];
    const uint32_t j = v & ~SIGN_BIT;
    const int64_t k = (int64_t)j / CHUNK;
    const int64_t* cp = cptr + k * r1;
    int lo = 0, hi = r1 - 1;  // last column c with cp[c] <= e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cp[mid] <= e) lo = mid;
      else hi = mid - 1;
    }
    const uint32_t c = (uint32_t)lo;
    const uint32_t jj = j % (uint32_t)CHUNK;
    entacc[e] = (jj * (uint32_t)APPLY_TILE_LD) | (((c % (uint32_t)cg) * (uint32_t)APPLY_TILE_LD) << 15) |
                (v & SIGN_BIT);
  }
}

// Plain CSC view for spm_sketch_tables: count per column over all chunks.
__global__ void k_bucket_counts(int r1, int nchunks, const int64_t* __restrict__ cptr,
                                int64_t* __restrict__ cnt) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= r1) return;
  int64_t tot = 0;
  for (int k = 0; k < nchunks; ++k) {
    const int64_t b = cptr[(int64_t)k * r1 + c];
    const int64_t e = cptr[(int64_t)k * r1 + c + 1];
    tot += e - b;
  }
  cnt[c] = tot;
}

__global__ void k_exclusive_scan_small(int64_t count, const int64_t* __restrict__ in,
                                       int64_t* __restrict__ out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int64_t run = 0;
    for (int64_t i = 0; i < count; ++i) {
      out[i] = run;
      run += in[i];
    }
    out[count] = run;
  }
}

__global__ void k_bucket_fill(int r1, int nchunks, const int64_t* __restrict__ cptr,
                              const uint32_t* __restrict__ ent, const int64_t* __restrict__ bptr,
                              int32_t* __restrict__ rows, int8_t* __restrict__ sg) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= r1) return;
  int64_t o = bptr[c];
  for (int k = 0; k < nchunks; ++k) {
    const int64_t b = cptr[(int64_t)k * r1 + c];
    const int64_t e = cptr[(int64_t)k * r1 + c + 1];
    for (int64_t p = b; p < e; ++p, ++o) {
      const uint32_t v = ent[p];
      if (rows) rows[o] = (int32_t)(v & ~SIGN_BIT);
      if (sg) sg[o] = (v & SIGN_BIT) ? (int8_t)-1 : (int8_t)1;
    }
  }
}

// ------------------------------------------------------------------ a2: Omega
// Box-Muller on Philox: elements 2p and 2p + 1 are rad cos(ang) and rad sin(ang)
// of the pair drawn with counter p.  One thread per pair (the logarithm, the
// square root and the angle's reduction shared), one 64-bit division per pair.
template <typename T>
__global__ void k_gaussian(int64_t rows, int64_t cols, int64_t ld, uint32_t k0, uint32_t k1,
                           T* __restrict__ out) {
  const int64_t total = rows * cols;
  const int64_t npairs = (total + 1) >> 1;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npairs;
       p += (int64_t)gridDim.x * blockDim.x) {
    const u32x4 w = philox4x32_10((uint32_t)p, (uint32_t)((uint64_t)p >> 32), 0u, 2u, k0, k1);
    const uint64_t x1 = ((uint64_t)w.y << 21) | (uint64_t)(w.x >> 11);
    const uint64_t x2 = ((uint64_t)w.w << 21) | (uint64_t)(w.z >> 11);
    const double u1 = (double)(x1 + 1ull) * 0x1.0p-53;
    const double u2 = (double)x2 * 0x1.0p-53;
    const double rad = sqrt(-2.0 * log(u1));
    const double ang = 6.283185307179586 * u2;
    double sn, cs;
    sincos(ang, &sn, &cs);
    const int64_t e0 = 2 * p;
    int64_t i = e0 / cols, j = e0 - i * cols;
    out[i * ld + j] = (T)(rad * cs);
    if (e0 + 1 < total) {
      if (++j == cols) {
        j = 0;
        ++i;
      }
      out[i * ld + j] = (T)(rad * sn);
    }
  }
}

// ------------------------------------------------------------------ a3: A S
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* sdst, const T* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(sdst);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_elem8(void* sdst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc));
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ double as_double(float x) { return (double)x; }
__device__ __forceinline__ double as_double(double x) { return x; }
__device__ __forceinline__ double as_double(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

template <typename TO, typename TV>
__device__ __forceinline__ TO cvt_out(TV v) { return (TO)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16, double>(double v) {
  return __float2bfloat16_rn((float)v);
}

template <typename TO>
__device__ __forceinline__ TO to_out(double v);
template <>
__device__ __forceinline__ float to_out<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ double to_out<double>(double v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn((float)v);
}

// One CTA: 32 rows of A (lane = row) x a group of CG = 16 warps * CPW output
// columns.  Per chunk of CHUNK = 512 columns of A (rows of S):
//   * the A tile (32 x 512) is staged transposed in shared memory ([jj][row],
//     row stride 33), so one warp-wide read of column jj hits 32 distinct banks;
//   * the CTA's segment bounds and bucket entries for this chunk (one
//     contiguous range) are staged next to it; each entry already holds the
//     tile offset of its column and its sign bit;
//   all with cp.async into a double buffer, so chunk k+1 streams in while
//   chunk k is reduced.  Each warp owns CPW output columns with one accumulator
//   per lane and column in registers across all chunks; an entry costs one
//   broadcast shared load, one conflict-free shared load of A, a sign flip and
//   an add per lane.
template <typename TA, typename TACC>
__device__ __forceinline__ TACC signed_val(TA a, uint32_t e) {
  return (e & SIGN_BIT) ? -(TACC)a : (TACC)a;
}
template <>
__device__ __forceinline__ float signed_val<float, float>(float a, uint32_t e) {
  return __int_as_float(__float_as_int(a) ^ (int)(e & SIGN_BIT));
}

// Sum of the signed tile values of one (chunk, column) segment [p, pe) of the
// staged entries; entries past the staged capacity are read from global memory.
template <typename TA, typename TACC>
__device__ __noinline__ TACC segment_sum(const uint32_t* es, const TA* t, const uint32_t* eg, int p,
                                         int pe, int ent_cap) {
  TACC a0 = (TACC)0, a1 = (TACC)0;
  if (pe <= ent_cap) {
    for (; p + 1 < pe; p += 2) {
      const uint32_t e0 = es[p], e1 = es[p + 1];
      a0 += signed_val<TA, TACC>(t[e0 & ~SIGN_BIT], e0);
      a1 += signed_val<TA, TACC>(t[e1 & ~SIGN_BIT], e1);
    }
    if (p < pe) {
      const uint32_t e0 = es[p];
      a0 += signed_val<TA, TACC>(t[e0 & ~SIGN_BIT], e0);
    }
  } else {
    for (; p < pe; ++p) {
      const uint32_t e0 = (p < ent_cap) ? es[p] : __ldg(eg + p);
      a0 += signed_val<TA, TACC>(t[e0 & ~SIGN_BIT], e0);
    }
  }
  return a0 + a1;
}

template <typename TA, typename TACC, typename TO, int CPW, int NBUF, bool GENT>
__global__ void __launch_bounds__(APPLY_THREADS, 1)
    k_sketch_apply(const TA* __restrict__ A, int64_t m, int64_t n, int64_t lda, int r1,
                   int nchunks, const int64_t* __restrict__ cptr, const int2* __restrict__ seg,
                   const uint32_t* __restrict__ entoff, TO* __restrict__ out, int64_t ldo,
                   int col_groups, double scale, double* __restrict__ fro2,
                   TO* __restrict__ out_lo, int ent_cap) {
  constexpr int CG = APPLY_WARPS * CPW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TA* tile = reinterpret_cast<TA*>(smem_raw);
  int2* seg_s = reinterpret_cast<int2*>(smem_raw + (size_t)NBUF * CHUNK * APPLY_TILE_LD * sizeof(TA));
  uint32_t* ent_s = reinterpret_cast<uint32_t*>(seg_s + (size_t)NBUF * CG);  // NBUF x ent_cap
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t rb = blockIdx.x / col_groups;
  const int cg = blockIdx.x % col_groups;
  const int64_t row0 = rb * APPLY_ROWS;
  const int nrows = (int)min64(APPLY_ROWS, m - row0);
  const int c0 = cg * CG;
  const int c1 = (int)min64(c0 + CG, r1);
  const int ncols = c1 - c0;
  const int wc0 = warp * CPW;  // first column of this warp, relative to c0
  const bool do_fro = (fro2 != nullptr) && (cg == 0);
  TACC acc[CPW];
#pragma unroll
  for (int i = 0; i < CPW; ++i) acc[i] = (TACC)0;
  double fro_local = 0.0;

  // stage chunk k into buffer b (A tile, segment bounds, entries)
  auto stage = [&](int k, int b) {
    TA* t = tile + (size_t)b * CHUNK * APPLY_TILE_LD;
    const int64_t j0 = (int64_t)k * CHUNK;
    const int wcnt = (int)min64(CHUNK, n - j0);
    for (int jj = tid; jj < CHUNK; jj += APPLY_THREADS) {
#pragma unroll 8
      for (int r = 0; r < APPLY_ROWS; ++r) {
        TA* dst = t + jj * APPLY_TILE_LD + r;
        if (r < nrows && jj < wcnt)
          cp_async_elem(dst, A + (row0 + r) * lda + j0 + jj);
        else
          *dst = (TA)0;
      }
    }
    const int2* sg = seg + (int64_t)k * r1 + c0;
    int2* ss = seg_s + (size_t)b * CG;
    for (int i = tid; i < ncols; i += APPLY_THREADS) cp_async_elem8(ss + i, sg + i);
    const int e_beg = __ldg(&sg[0].x), e_end = __ldg(&sg[ncols - 1].y);
    // columns past ncols (last group) get empty segments: no bounds test in the loop
    for (int i = ncols + tid; i < CG; i += APPLY_THREADS) ss[i] = make_int2(e_end, e_end);
    const int cnt = min(e_end - e_beg, ent_cap);
    const uint32_t* src = entoff + __ldg(cptr + (int64_t)k * r1) + e_beg;
    uint32_t* es = ent_s + (size_t)b * ent_cap;
    if (!GENT)
      for (int i = tid; i < cnt; i += APPLY_THREADS) cp_async_elem(es + i, src + i);
    cp_async_commit();
  };

  if (NBUF == 2) stage(0, 0);
  for (int k = 0; k < nchunks; ++k) {
    const int b = (NBUF == 2) ? (k & 1) : 0;
    if (NBUF == 2) {
      if (k + 1 < nchunks) {
        stage(k + 1, b ^ 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
    } else {
      stage(k, 0);
      cp_async_wait<0>();
    }
    __syncthreads();
    const TA* t = tile + (size_t)b * CHUNK * APPLY_TILE_LD + lane;
    const int2* ss = seg_s + (size_t)b * CG;
    const uint32_t* es = ent_s + (size_t)b * ent_cap;
    if (do_fro) {
      // |A|_F^2: per-chunk partial in the tile's type, one FP64 add per chunk
      const TA* tt = tile + (size_t)b * CHUNK * APPLY_TILE_LD;
      TA part = (TA)0;
      for (int jj = tid; jj < CHUNK; jj += APPLY_THREADS) {
#pragma unroll 8
        for (int r = 0; r < APPLY_ROWS; ++r) {
          const TA v = tt[jj * APPLY_TILE_LD + r];
          part += v * v;
        }
      }
      fro_local += (double)part;
    }
    const int base = ss[0].x;
    const uint32_t* eglob = entoff + __ldg(cptr + (int64_t)k * r1);  // for entries beyond ent_cap
    // The accumulators need static register indices, so the column loop is
    // unrolled; each copy is a minimal loop (a few instructions per entry) so
    // that the unrolled code stays within the instruction cache.
    if (GENT) es = eglob + base;  // very dense sketches: entries straight from global
#pragma unroll
    for (int i = 0; i < CPW; ++i) {
      const int2 se = ss[wc0 + i];
      TACC a = (TACC)0;
      // a segment holds about two entries: a plain loop, not an unrolled one
      // with a remainder (whose set-up would cost more than the entries)
#pragma unroll 1
      for (int p = se.x - base; p < se.y - base; ++p) {
        const uint32_t e0 = es[p];
        a += signed_val<TA, TACC>(t[e0 & ~SIGN_BIT], e0);
      }
      acc[i] += a;
    }
    __syncthreads();
  }
  // epilogue: transpose the 32 x CPW accumulator block of each warp through
  // shared memory so that stores are row-contiguous.
  TACC* st = reinterpret_cast<TACC*>(smem_raw) + (size_t)warp * APPLY_ROWS * (CPW + 1);
#pragma unroll
  for (int i = 0; i < CPW; ++i) st[lane * (CPW + 1) + i] = acc[i];
  __syncwarp();
  for (int r = 0; r < nrows; ++r) {
    for (int i = lane; i < CPW; i += 32) {
      const int c = c0 + wc0 + i;
      if (wc0 + i < ncols) {
        // epilogue arithmetic stays in the accumulator type (FP64 is slow on this part)
        const TACC v = st[r * (CPW + 1) + i] * (TACC)scale;
        const TO h = cvt_out<TO>(v);
        out[(row0 + r) * ldo + c] = h;
        // split-precision copy: lo = v - hi, rounded (only for BF16 outputs)
        if (out_lo) out_lo[(row0 + r) * ldo + c] = cvt_out<TO>(v - (TACC)as_double(h));
      }
    }
  }
  if (do_fro) {
    for (int o = 16; o > 0; o >>= 1) fro_local += __shfl_xor_sync(0xFFFFFFFFu, fro_local, o);
    __syncthreads();
    double* red = reinterpret_cast<double*>(smem_raw);
    if (lane == 0) red[warp] = fro_local;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int w = 0; w < APPLY_WARPS; ++w) sum += red[w];
      atomicAdd(fro2, sum);
    }
  }
}

// ------------------------------------------------------------------ A S, shared accumulators
// FP32 A, sparse sign S with s <= 8.  One CTA: 32 rows of A (lane = row) x a
// group of cg output columns, whose accumulators live in shared memory
// (acc[c][33], FP32).  Per chunk of 512 columns of A, each warp walks a flat,
// contiguous list of the entries of its own columns (the chunk's CSC segment
// of those columns) and adds sign * tile[jj][lane] into acc[c][lane]: one
// entry word, one tile value and one accumulator read-modify-write per entry,
// no per-column loop.  A column belongs to one warp, so there are no races.
// The next chunk's tile and entry words are loaded into registers while the
// current chunk is processed.
template <typename TO>
__global__ void __launch_bounds__(APPLY_THREADS, 1)
    k_sketch_apply_sacc(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda, int r1,
                        int nchunks, int cg, int ngroups, const int64_t* __restrict__ cptr,
                        const uint32_t* __restrict__ entacc, TO* __restrict__ out, int64_t ldo,
                        double scale, double* __restrict__ fro2, TO* __restrict__ out_lo,
                        int ent_cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* tile = reinterpret_cast<float*>(smem_raw);                       // CHUNK x 33
  float* acc = tile + CHUNK * APPLY_TILE_LD;                               // cg x 33
  uint32_t* es = reinterpret_cast<uint32_t*>(acc + (size_t)cg * APPLY_TILE_LD);  // ent_cap
  int* wb = reinterpret_cast<int*>(es + ent_cap);  // 2 x 33 warp bounds (this chunk, next chunk)
  constexpr int PER = CHUNK * APPLY_ROWS / APPLY_THREADS;                  // 16 tile values per thread
  constexpr int EPER = (CHUNK * SACC_MAX_S) / APPLY_THREADS;               // 4 entry words per thread
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t rb = blockIdx.x / ngroups;
  const int g = blockIdx.x % ngroups;
  const int64_t row0 = rb * APPLY_ROWS;
  const int nrows = (int)min64(APPLY_ROWS, m - row0);
  const int c0 = g * cg;
  const int ncols = min(cg, r1 - c0);
  const bool do_fro = (fro2 != nullptr) && (g == 0);
  for (int i = tid; i < cg * APPLY_TILE_LD; i += APPLY_THREADS) acc[i] = 0.f;
  double fro_local = 0.0;

  float tv[PER];
  uint32_t ev[EPER];
  int e_cnt = 0;
  // load chunk k into registers (tile values: element q = tid + 1024 u is row q / 512,
  // column q % 512, so a warp reads 32 consecutive floats of one row)
  auto load = [&](int k) {
    const int64_t j0 = (int64_t)k * CHUNK;
    const int wcnt = (int)min64(CHUNK, n - j0);
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int q = tid + APPLY_THREADS * u;
      const int r = q / CHUNK, jj = q % CHUNK;
      tv[u] = (r < nrows && jj < wcnt) ? __ldcs(A + (row0 + r) * lda + j0 + jj) : 0.f;
    }
    const int64_t base = __ldg(cptr + (int64_t)k * r1 + c0);
    const int64_t end = __ldg(cptr + (int64_t)k * r1 + c0 + ncols);
    e_cnt = (int)(end - base);
#pragma unroll
    for (int u = 0; u < EPER; ++u) {
      const int q = tid + APPLY_THREADS * u;
      ev[u] = (q < e_cnt) ? __ldg(entacc + base + q) : 0u;
    }
    // warp w owns columns [c0 + w cg / 32, c0 + (w + 1) cg / 32)
    if (tid <= APPLY_WARPS) {
      const int cw = min(ncols, (int)(((int64_t)tid * ncols) / APPLY_WARPS));
      wb[APPLY_WARPS + 1 + tid] = (int)(__ldg(cptr + (int64_t)k * r1 + c0 + cw) - base);
    }
  };
  load(0);
  for (int k = 0; k < nchunks; ++k) {
    // registers -> shared (tile transposed: tile[jj][row])
    float part = 0.f;  // |A|_F^2: one FP64 add per chunk
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int q = tid + APPLY_THREADS * u;
      tile[(q % CHUNK) * APPLY_TILE_LD + q / CHUNK] = tv[u];
      part = fmaf(tv[u], tv[u], part);
    }
    if (do_fro) fro_local += (double)part;
#pragma unroll
    for (int u = 0; u < EPER; ++u) {
      const int q = tid + APPLY_THREADS * u;
      if (q < e_cnt) es[q] = ev[u];
    }
    if (tid <= APPLY_WARPS) wb[tid] = wb[APPLY_WARPS + 1 + tid];
    __syncthreads();
    if (k + 1 < nchunks) load(k + 1);  // in flight while this chunk is reduced
    {
      const int p0 = wb[warp], p1 = wb[warp + 1];
      const float* tl = tile + lane;
      float* al = acc + lane;
#pragma unroll 4
      for (int p = p0; p < p1; ++p) {
        const uint32_t e = es[p];
        const float v = __int_as_float(__float_as_int(tl[e & 0x7FFFu]) ^ (int)(e & SIGN_BIT));
        float* a = al + ((e >> 15) & 0xFFFFu);
        *a += v;
      }
    }
    __syncthreads();
  }
  // epilogue: acc[c][r] -> out[row0 + r][c0 + c], consecutive threads on consecutive c
  for (int q = tid; q < nrows * ncols; q += APPLY_THREADS) {
    const int r = q / ncols, c = q % ncols;
    const float v = acc[c * APPLY_TILE_LD + r] * (float)scale;
    const TO h = cvt_out<TO>(v);
    out[(row0 + r) * ldo + c0 + c] = h;
    if (out_lo) out_lo[(row0 + r) * ldo + c0 + c] = cvt_out<TO>(v - (float)as_double(h));
  }
  if (do_fro) {
    for (int o = 16; o > 0; o >>= 1) fro_local += __shfl_xor_sync(0xFFFFFFFFu, fro_local, o);
    __syncthreads();
    double* red = reinterpret_cast<double*>(smem_raw);
    if (lane == 0) red[warp] = fro_local;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int w = 0; w < APPLY_WARPS; ++w) sum += red[w];
      atomicAdd(fro2, sum);
    }
  }
}

// ------------------------------------------------------------------ S^T X
// One CTA per (output row c, strip of 256 columns of X); c varies fastest so
// that all CTAs of one strip run together and re-reads of X rows hit L2.
template <typename TX, typename TACC, typename TO>
__global__ void __launch_bounds__(256)
    k_sketch_apply_t(const TX* __restrict__ X, int64_t p, int64_t ldx, int r1, int nchunks,
                     const int64_t* __restrict__ cptr, const uint32_t* __restrict__ ent,
                     TO* __restrict__ out, int64_t ldo, double scale) {
  const int c = blockIdx.x % r1;
  const int64_t strip = blockIdx.x / r1;
  const int64_t col = strip * 256 + threadIdx.x;
  TACC acc = 0;
  if (col < p) {
    for (int k = 0; k < nchunks; ++k) {
      const int64_t b = __ldg(cptr + (int64_t)k * r1 + c);
      const int64_t e = __ldg(cptr + (int64_t)k * r1 + c + 1);
      for (int64_t q = b; q < e; ++q) {
        const uint32_t v = __ldg(ent + q);
        const int64_t j = (int64_t)(v & ~SIGN_BIT);
        const TACC x = (TACC)X[j * ldx + col];
        acc += (v & SIGN_BIT) ? -x : x;
      }
    }
    out[(int64_t)c * ldo + col] = to_out<TO>((double)acc * scale);
  }
}

// ------------------------------------------------------------------ host side
static int64_t nchunks_of(int64_t n) { return cdiv(n, CHUNK); }

int gaussian_dev(void* out, int dt, int64_t rows, int64_t cols, int64_t ld, uint64_t seed,
                 cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return SPM_OK;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int64_t total = rows * cols;
  const int blocks = (int)min64(cdiv((total + 1) / 2, 256), 152 * 16);
  if (dt == DT_F64)
    k_gaussian<double><<<blocks, 256, 0, st>>>(rows, cols, ld, k0, k1, (double*)out);
  else if (dt == DT_F32)
    k_gaussian<float><<<blocks, 256, 0, st>>>(rows, cols, ld, k0, k1, (float*)out);
  else
    return SPM_EINVAL;
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

// Shared-accumulator apply (FP32 A, FP32 or BF16 out); SPM_EUNSUPPORTED when
// the sketch has no entacc table or the CTA's shared memory would not fit.
template <typename TO>
static int launch_apply_sacc(const spm_sketch* S, const float* A, int64_t m, int64_t lda, TO* out,
                             int64_t ldo, double* fro2, cudaStream_t st, TO* out_lo) {
  if (!S->entacc || S->kind != SPM_SKETCH_SPARSE_SIGN || S->s > SACC_MAX_S) return SPM_EUNSUPPORTED;
  const int64_t nch = nchunks_of(S->n);
  const int cg = S->acc_cg;
  const int ngroups = (int)cdiv(S->r1, cg);
  const int ent_cap = CHUNK * S->s;
  const size_t smem = ((size_t)CHUNK * APPLY_TILE_LD + (size_t)cg * APPLY_TILE_LD) * sizeof(float) +
                      (size_t)ent_cap * sizeof(uint32_t) + 2 * (APPLY_WARPS + 1) * sizeof(int);
  if (smem > 227 * 1024) return SPM_EUNSUPPORTED;
  const int64_t grid = cdiv(m, APPLY_ROWS) * ngroups;
  if (grid > 0x7FFFFFFF) return SPM_EUNSUPPORTED;
  const double scale = 1.0 / sqrt((double)S->s);
  auto kern = k_sketch_apply_sacc<TO>;
  SPM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)grid, APPLY_THREADS, smem, st>>>(A, m, S->n, lda, (int)S->r1, (int)nch, cg, ngroups,
                                                    S->bucket_ptr, S->entacc, out, ldo, scale, fro2,
                                                    out_lo, ent_cap);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

template <typename TA, typename TACC, typename TO, int CPW, int NBUF>
static int launch_apply(const spm_sketch* S, const TA* A, int64_t m, int64_t lda, TO* out,
                        int64_t ldo, double* fro2, cudaStream_t st, TO* out_lo = nullptr) {
  if constexpr (std::is_same<TA, float>::value && std::is_same<TACC, float>::value) {
    const int rc = launch_apply_sacc<TO>(S, A, m, lda, out, ldo, fro2, st, out_lo);
    if (rc != SPM_EUNSUPPORTED) return rc;
  }
  const int64_t nch = nchunks_of(S->n);
  constexpr int CG = APPLY_WARPS * CPW;
  const int col_groups = (int)cdiv(S->r1, CG);
  const int64_t row_blocks = cdiv(m, APPLY_ROWS);
  const int64_t grid = row_blocks * col_groups;
  if (grid > 0x7FFFFFFF) return SPM_EUNSUPPORTED;
  const size_t tile_bytes = (size_t)NBUF * CHUNK * APPLY_TILE_LD * sizeof(TA);
  const size_t seg_bytes = (size_t)NBUF * CG * sizeof(int2);
  const size_t epi_bytes = (size_t)APPLY_WARPS * APPLY_ROWS * (CPW + 1) * sizeof(TACC);
  // all entries of one chunk (at most CHUNK * s) are staged when they fit;
  // otherwise the kernel reads them from global memory
  const size_t budget = 225 * 1024;
  int ent_cap = CHUNK * (S->kind == SPM_SKETCH_IDENTITY ? 1 : S->s);
  const bool gent = tile_bytes + seg_bytes + (size_t)NBUF * ent_cap * 4 > budget;
  if (gent) ent_cap = 0;
  size_t smem = tile_bytes + seg_bytes + (size_t)NBUF * ent_cap * 4;
  if (epi_bytes > smem) smem = epi_bytes;
  const double scale = (S->kind == SPM_SKETCH_IDENTITY) ? 1.0 : 1.0 / sqrt((double)S->s);
  auto go = [&](auto kern) -> int {
    SPM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)grid, APPLY_THREADS, smem, st>>>(A, m, S->n, lda, (int)S->r1, (int)nch,
                                                     S->bucket_ptr, S->seg, S->entoff, out, ldo,
                                                     col_groups, scale, fro2, out_lo, ent_cap);
    SPM_LAUNCH_CHECK();
    return SPM_OK;
  };
  if (gent) return go(k_sketch_apply<TA, TACC, TO, CPW, NBUF, true>);
  return go(k_sketch_apply<TA, TACC, TO, CPW, NBUF, false>);
}

int sketch_apply_dev(const spm_sketch* S, const void* A, int a_dt, int64_t m, int64_t lda,
                     void* out, int out_dt, int64_t ldo, double* fro2, cudaStream_t st,
                     void* out_lo, int* status, void* a_hi, void* a_lo, int64_t lds,
                     bool* a_split) {
  if (a_split) *a_split = false;
  if (m <= 0) return SPM_OK;
  if (dense_kind(S)) return dense_sketch_apply(S, A, a_dt, m, lda, out, out_dt, ldo, fro2, st, out_lo);
  if (a_dt == DT_F32 && (out_dt == DT_F32 || out_dt == DT_BF16)) {
    // whole rows in shared memory, conflict-free gather schedule (the plan is
    // the sketch's own, built on first use)
    const bool sp = a_hi != nullptr && out_dt == DT_BF16;
    int rc = sched_apply(const_cast<spm_sketch*>(S), (const float*)A, m, lda, out, out_dt, ldo,
                         fro2, status, st, out_dt == DT_BF16 ? out_lo : nullptr,
                         sp ? a_hi : nullptr, sp ? a_lo : nullptr, lds);
    if (rc == SPM_OK && a_split) *a_split = sp;
    if (rc != SPM_EUNSUPPORTED) return rc;
  }
  if (a_dt == DT_F32) {
    const float* a = (const float*)A;
    if (out_dt == DT_F32) return launch_apply<float, float, float, 32, 2>(S, a, m, lda, (float*)out, ldo, fro2, st);
    if (out_dt == DT_BF16)
      return launch_apply<float, float, __nv_bfloat16, 32, 2>(S, a, m, lda, (__nv_bfloat16*)out, ldo, fro2, st,
                                                              (__nv_bfloat16*)out_lo);
    if (out_dt == DT_F64) return launch_apply<float, double, double, 16, 2>(S, a, m, lda, (double*)out, ldo, fro2, st);
  } else if (a_dt == DT_F64) {
    const double* a = (const double*)A;
    if (out_dt == DT_F64) return launch_apply<double, double, double, 16, 1>(S, a, m, lda, (double*)out, ldo, fro2, st);
    if (out_dt == DT_F32) return launch_apply<double, double, float, 16, 1>(S, a, m, lda, (float*)out, ldo, fro2, st);
    if (out_dt == DT_BF16)
      return launch_apply<double, double, __nv_bfloat16, 16, 1>(S, a, m, lda, (__nv_bfloat16*)out, ldo, fro2, st,
                                                                (__nv_bfloat16*)out_lo);
  }
  return SPM_EINVAL;
}

int sketch_apply_t_dev(const spm_sketch* S, const void* X, int x_dt, int64_t p, int64_t ldx,
                       void* out, int out_dt, int64_t ldo, cudaStream_t st) {
  if (p <= 0) return SPM_OK;
  if (dense_kind(S)) return dense_sketch_apply_t(S, X, x_dt, p, ldx, out, out_dt, ldo, st);
  const int64_t strips = cdiv(p, 256);
  const int64_t grid = strips * S->r1;
  if (grid > 0x7FFFFFFF) return SPM_EUNSUPPORTED;
  const double scale = (S->kind == SPM_SKETCH_IDENTITY) ? 1.0 : 1.0 / sqrt((double)S->s);
  const int nch = (int)nchunks_of(S->n);
  const int r1 = (int)S->r1;
#define SPM_APT(TX, TACC, TO)                                                                 \
  k_sketch_apply_t<TX, TACC, TO><<<(unsigned)grid, 256, 0, st>>>((const TX*)X, p, ldx, r1, nch, \
                                                                 S->bucket_ptr, S->bucket_ent, \
                                                                 (TO*)out, ldo, scale)
  if (x_dt == DT_F32 && out_dt == DT_F32) SPM_APT(float, float, float);
  else if (x_dt == DT_F32 && out_dt == DT_F64) SPM_APT(float, double, double);
  else if (x_dt == DT_F64 && out_dt == DT_F64) SPM_APT(double, double, double);
  else if (x_dt == DT_F64 && out_dt == DT_F32) SPM_APT(double, double, float);
  else if (x_dt == DT_F32 && out_dt == DT_BF16) SPM_APT(float, float, __nv_bfloat16);
  else if (x_dt == DT_BF16 && out_dt == DT_F32) SPM_APT(__nv_bfloat16, float, float);
  else return SPM_EINVAL;
#undef SPM_APT
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

}  // namespace spm

using namespace spm;

extern "C" {

int spm_sketch_create(spm_sketch** out, int64_t n, int64_t r1, int32_t s, uint64_t seed,
                      int32_t kind, void* stream) {
  if (!out) return SPM_EINVAL;
  *out = nullptr;
  if (n < 1 || r1 < 1 || s < 1 || n > 0x7FFFFFFF || r1 > 0x7FFFFFFF) return SPM_EINVAL;
  if (kind == SPM_SKETCH_SPARSE_SIGN) {
    if (s > r1 || s > 64) return SPM_EINVAL;
    if (r1 > 48 * 1024) return SPM_EUNSUPPORTED;  // per-chunk histogram lives in shared memory
  } else if (kind == SPM_SKETCH_IDENTITY) {
    if (r1 != n || s != 1) return SPM_EINVAL;
  } else if (kind == SPM_SKETCH_DENSE_SIGN) {
    if (n * round_up(r1, 8) > ((int64_t)1 << 36)) return SPM_EUNSUPPORTED;
  } else if (kind == SPM_SKETCH_SRHT) {
    if (r1 > n) return SPM_EINVAL;
    if (n > 32768) return SPM_EUNSUPPORTED;  // one row of the transform per CTA in shared memory
  } else {
    return SPM_EINVAL;
  }
  if (kind == SPM_SKETCH_DENSE_SIGN || kind == SPM_SKETCH_SRHT) {
    spm_sketch* S = new spm_sketch();
    S->n = n;
    S->r1 = r1;
    S->s = s;
    S->kind = kind;
    S->seed = seed;
    S->stream = as_stream(stream);
    const int rc = dense_sketch_create(S, S->stream);
    if (rc != SPM_OK) {
      spm_sketch_destroy(S);
      return rc;
    }
    *out = S;
    return SPM_OK;
  }
  if (n * (int64_t)s > 0x7FFFFFFF) return SPM_EUNSUPPORTED;
  cudaStream_t st = as_stream(stream);
  spm_sketch* S = new spm_sketch();
  S->n = n;
  S->r1 = r1;
  S->s = s;
  S->kind = kind;
  S->seed = seed;
  S->stream = st;
  const int64_t nnz = n * s;
  const int64_t nch = nchunks_of(n);
  auto fail = [&](int code) {
    spm_sketch_destroy(S);
    return code;
  };
  if (cudaMallocAsync((void**)&S->cols, nnz * sizeof(int32_t), st) != cudaSuccess) return fail(SPM_ENOMEM);
  if (cudaMallocAsync((void**)&S->signs, nnz * sizeof(int8_t), st) != cudaSuccess) return fail(SPM_ENOMEM);
  if (cudaMallocAsync((void**)&S->bucket_ent, nnz * sizeof(uint32_t), st) != cudaSuccess) return fail(SPM_ENOMEM);
  if (cudaMallocAsync((void**)&S->bucket_ptr, (nch * r1 + 1) * sizeof(int64_t), st) != cudaSuccess)
    return fail(SPM_ENOMEM);
  if (cudaMallocAsync((void**)&S->seg, nch * r1 * sizeof(int2), st) != cudaSuccess) return fail(SPM_ENOMEM);
  if (cudaMallocAsync((void**)&S->entoff, nnz * sizeof(uint32_t), st) != cudaSuccess) return fail(SPM_ENOMEM);
  if (kind == SPM_SKETCH_IDENTITY) {
    const int64_t blocks = cdiv(max64(n, 1), 256);
    k_sketch_identity<<<(unsigned)min64(blocks, 65535 * 16), 256, 0, st>>>(
        n, S->cols, S->signs, S->bucket_ent, S->bucket_ptr, (int)nch);
    if (cudaGetLastError() != cudaSuccess) return fail(SPM_ECUDA);
  } else {
    k_sketch_gen<<<(unsigned)cdiv(n, 128), 128, 0, st>>>(n, (uint32_t)r1, s, (uint32_t)seed,
                                                         (uint32_t)(seed >> 32), S->cols,
                                                         S->signs, nullptr);
    if (cudaGetLastError() != cudaSuccess) return fail(SPM_ECUDA);
    const size_t hist_bytes = (size_t)(r1 + 1) * sizeof(int);
    if (cudaFuncSetAttribute(k_chunk_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)hist_bytes) != cudaSuccess)
      return fail(SPM_ECUDA);
    k_chunk_sort<<<(unsigned)nch, 256, hist_bytes, st>>>(n, (int)r1, s, S->cols, S->signs,
                                                         S->bucket_ptr, S->bucket_ent);
    if (cudaGetLastError() != cudaSuccess) return fail(SPM_ECUDA);
    k_set_i64<<<1, 1, 0, st>>>(S->bucket_ptr + nch * r1, nnz);
    if (cudaGetLastError() != cudaSuccess) return fail(SPM_ECUDA);
  }
  {
    const int64_t work = max64(nnz, nch * r1);
    k_apply_tables<<<(unsigned)min64(cdiv(work, 256), 152 * 16), 256, 0, st>>>(
        nnz, (int)r1, (int)nch, S->bucket_ptr, S->bucket_ent, S->seg, S->entoff);
    if (cudaGetLastError() != cudaSuccess) return fail(SPM_ECUDA);
  }
  if (kind == SPM_SKETCH_SPARSE_SIGN) sched_init(S);
  if (kind == SPM_SKETCH_SPARSE_SIGN && s <= SACC_MAX_S && r1 <= 65535) {
    const int64_t ng = cdiv(r1, SACC_MAX_CG);
    S->acc_cg = (int32_t)cdiv(r1, ng);
    if (cudaMallocAsync((void**)&S->entacc, nnz * sizeof(uint32_t), st) != cudaSuccess)
      return fail(SPM_ENOMEM);
    k_acc_tables<<<(unsigned)min64(cdiv(nnz, 256), 152 * 16), 256, 0, st>>>(
        nnz, (int)r1, (int)nch, S->acc_cg, S->bucket_ptr, S->bucket_ent, S->entacc);
    if (cudaGetLastError() != cudaSuccess) return fail(SPM_ECUDA);
  }
  *out = S;
  return SPM_OK;
}

int spm_sketch_destroy(spm_sketch* S) {
  if (!S) return SPM_EINVAL;
  if (S->cols) cudaFreeAsync(S->cols, S->stream);
  if (S->signs) cudaFreeAsync(S->signs, S->stream);
  if (S->bucket_ent) cudaFreeAsync(S->bucket_ent, S->stream);
  if (S->bucket_ptr) cudaFreeAsync(S->bucket_ptr, S->stream);
  if (S->seg) cudaFreeAsync(S->seg, S->stream);
  if (S->entoff) cudaFreeAsync(S->entoff, S->stream);
  if (S->entacc) cudaFreeAsync(S->entacc, S->stream);
  sched_free(S);
  dense_sketch_free(S);
  delete S;
  return SPM_OK;
}

int spm_sketch_shape(const spm_sketch* S, int64_t* n, int64_t* r1, int32_t* s, int32_t* kind) {
  if (!S) return SPM_EINVAL;
  if (n) *n = S->n;
  if (r1) *r1 = S->r1;
  if (s) *s = S->s;
  if (kind) *kind = S->kind;
  return SPM_OK;
}

int spm_sketch_tables(const spm_sketch* S, int32_t* cols, int8_t* signs, int64_t* bucket_ptr,
                      int32_t* bucket_rows, int8_t* bucket_signs, void* stream) {
  if (!S) return SPM_EINVAL;
  if (dense_kind(S)) return SPM_EUNSUPPORTED;  // no sparse tables
  cudaStream_t st = as_stream(stream);
  const int64_t nnz = S->n * S->s;
  if (cols) SPM_CUDA_TRY(cudaMemcpyAsync(cols, S->cols, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  if (signs) SPM_CUDA_TRY(cudaMemcpyAsync(signs, S->signs, nnz, cudaMemcpyDeviceToDevice, st));
  if (bucket_ptr || bucket_rows || bucket_signs) {
    Arena ar(st);
    const int nch = (int)nchunks_of(S->n);
    const int r1 = (int)S->r1;
    SPM_ALLOC(ar, int64_t, cnt, r1);
    SPM_ALLOC(ar, int64_t, bptr, r1 + 1);
    k_bucket_counts<<<(unsigned)cdiv(r1, 256), 256, 0, st>>>(r1, nch, S->bucket_ptr, cnt);
    SPM_LAUNCH_CHECK();
    k_exclusive_scan_small<<<1, 1, 0, st>>>(r1, cnt, bptr);
    SPM_LAUNCH_CHECK();
    if (bucket_ptr)
      SPM_CUDA_TRY(cudaMemcpyAsync(bucket_ptr, bptr, (r1 + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    if (bucket_rows || bucket_signs) {
      k_bucket_fill<<<(unsigned)cdiv(r1, 128), 128, 0, st>>>(r1, nch, S->bucket_ptr, S->bucket_ent,
                                                              bptr, bucket_rows, bucket_signs);
      SPM_LAUNCH_CHECK();
    }
  }
  return SPM_OK;
}

int spm_gaussian(void* out, int32_t dtype, int64_t rows, int64_t cols, int64_t ld, uint64_t seed,
                 void* stream) {
  if (!out || rows < 1 || cols < 1 || ld < cols) return SPM_EINVAL;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_EINVAL;
  return gaussian_dev(out, dtype == SPM_F64 ? DT_F64 : DT_F32, rows, cols, ld, seed,
                      as_stream(stream));
}

int spm_sketch_apply(const spm_sketch* S, const void* A, int32_t dtype, int64_t m, int64_t lda,
                     void* out, int64_t ldo, void* stream) {
  if (!S || !A || !out || m < 1 || lda < S->n || ldo < S->r1) return SPM_EINVAL;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_EINVAL;
  const int dt = dtype == SPM_F64 ? DT_F64 : DT_F32;
  return sketch_apply_dev(S, A, dt, m, lda, out, dt, ldo, nullptr, as_stream(stream));
}

int spm_sketch_apply_t(const spm_sketch* S, const void* X, int32_t dtype, int64_t p, int64_t ldx,
                       void* out, int64_t ldo, void* stream) {
  if (!S || !X || !out || p < 1 || ldx < p || ldo < p) return SPM_EINVAL;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_EINVAL;
  const int dt = dtype == SPM_F64 ? DT_F64 : DT_F32;
  return sketch_apply_t_dev(S, X, dt, p, ldx, out, dt, ldo, as_stream(stream));
}

}  // extern "C"
