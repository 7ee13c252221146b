// Cholesky factorisation G = L L^T of a small Gram matrix and the inverse
// L^{-1}, in one cooperative kernel (the small factorisation of CholeskyQR).
//
// The matrix is cut into 64 x 64 tiles; nt = ceil(r / 64).  Per panel p:
//   * CTA 0 factors the diagonal tile (blocked by 16 inside the tile: a warp
//     factors each 16 x 16 block in registers, then a panel solve and a
//     trailing update in shared memory) and inverts it;
//   * the CTAs form the panel L[ib][p] = G[ib][p] L_pp^{-T} (ib > p), CTA 0
//     the tile p + 1, each tile published by a flag;
//   * the CTAs apply the trailing update G[ib][jb] -= L[ib][p] L[jb][p]^T,
//     each waiting only for the flags of its two panel tiles; the tile
//     (p + 1, p + 1) goes to CTA 0, which factors it right away, so the
//     diagonal chain does not wait for the rest of the panel.
// One bounded grid barrier per panel.  The off-diagonal tiles of L^{-1} then
// follow by recursive doubling: for a lower-triangular [L11 0; L21 L22],
//   inv(L)_21 = -inv(L22) (L21 inv(L11)),
// applied level by level over groups of 1, 2, 4, ... tiles, two products and
// two barriers per level.
//
// Deflation follows the unblocked rule: a pivot (Schur complement diagonal)
// at or below tol * max(diag G) marks its column deflated; that column of L
// becomes e_j, the elimination step is skipped and the column of every panel
// below is zeroed.
#include <algorithm>
#include <type_traits>

#include "internal.cuh"

namespace spm {

static constexpr int CT = 64;
static constexpr int CLD = CT + 4;  // 16-byte aligned rows: vector shared loads
static constexpr int CTHREADS = 512;

// A tile in registers: thread t holds elements t + 512 u (u = 0..7), row-major.
template <typename T>
struct TileRegs {
  T v[CT * CT / CTHREADS];
};
template <typename T>
__device__ __forceinline__ void ld_regs(TileRegs<T>& t, const T* M, int64_t ld, int r0, int c0, int R,
                                        int Cc) {
#pragma unroll
  for (int u = 0; u < CT * CT / CTHREADS; ++u) {
    const int e = threadIdx.x + CTHREADS * u;
    const int gi = r0 + (e >> 6), gj = c0 + (e & 63);
    t.v[u] = (gi < R && gj < Cc) ? __ldcg(M + (int64_t)gi * ld + gj) : (T)0;
  }
}
template <typename T>
__device__ __forceinline__ void st_regs(T (*s)[CLD], const TileRegs<T>& t, bool trans) {
#pragma unroll
  for (int u = 0; u < CT * CT / CTHREADS; ++u) {
    const int e = threadIdx.x + CTHREADS * u;
    const int i = e >> 6, j = e & 63;
    if (trans)
      s[j][i] = t.v[u];
    else
      s[i][j] = t.v[u];
  }
}

// s = tile (r0.., c0..) of a row-major matrix, zero outside [0, R) x [0, Cc);
// trans: s[j][i] = M[r0 + i][c0 + j].  Loads bypass L1 (the data may have been
// written by another CTA since this SM last read it) and are all issued
// before the first shared store.
template <typename T>
__device__ __forceinline__ void ld_tile(T (*s)[CLD], const T* M, int64_t ld, int r0, int c0, int R,
                                        int Cc, bool trans) {
  TileRegs<T> t;
  ld_regs(t, M, ld, r0, c0, R, Cc);
  st_regs(s, t, trans);
}

// 2- and 4-element shared loads and stores (8- and 16-byte aligned addresses)
static __device__ __forceinline__ void vld2(const float* p, float v[2]) {
  const float2 t = *reinterpret_cast<const float2*>(p);
  v[0] = t.x;
  v[1] = t.y;
}
static __device__ __forceinline__ void vld2(const double* p, double v[2]) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  v[0] = t.x;
  v[1] = t.y;
}
static __device__ __forceinline__ void vld4(const float* p, float v[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
static __device__ __forceinline__ void vld4(const double* p, double v[4]) {
  vld2(p, v);
  vld2(p + 2, v + 2);
}
static __device__ __forceinline__ void vst4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
static __device__ __forceinline__ void vst4(double* p, const double v[4]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

// acc[v][u] += sum_k Xt[k][row_v] Y[k][col_u]; rows 2 ty + v, columns 4 tx + u
// (ty = tid / 16, tx = tid % 16): per k, one 2-element load of Xt and one
// 4-element load of Y for eight multiply-adds.
template <typename T>
__device__ __forceinline__ void tile_mma(T acc[2][4], const T (*Xt)[CLD], const T (*Y)[CLD]) {
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll 8
  for (int k = 0; k < CT; ++k) {
    T x[2], y[4];
    vld2(&Xt[k][2 * ty], x);
    vld4(&Y[k][4 * tx], y);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc[0][u] = fma(x[0], y[u], acc[0][u]);
      acc[1][u] = fma(x[1], y[u], acc[1][u]);
    }
  }
}

template <typename T>
__device__ __forceinline__ void acc_zero(T acc[2][4]) {
#pragma unroll
  for (int v = 0; v < 2; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[v][u] = (T)0;
}

// acc += sum_{kb in [k0, k1)} X(kb) Y(kb) with X(kb) staged transposed; the
// next pair of tiles is loaded into registers while the current product runs.
template <typename T, typename FX, typename FY>
__device__ __forceinline__ void tile_chain(T acc[2][4], int k0, int k1, FX fx, FY fy, T (*s0)[CLD],
                                           T (*s1)[CLD]) {
  if (k0 >= k1) return;
  TileRegs<T> rx, ry;
  fx(rx, k0);
  fy(ry, k0);
  for (int kb = k0; kb < k1; ++kb) {
    st_regs(s0, rx, true);
    st_regs(s1, ry, false);
    __syncthreads();
    if (kb + 1 < k1) {
      fx(rx, kb + 1);
      fy(ry, kb + 1);
    }
    tile_mma<T>(acc, s0, s1);
    __syncthreads();
  }
}

// 1 / sqrt(d): the fast reciprocal square root in FP32 (a few ulp; CholeskyQR
// repeats its passes), the exact quotient in FP64.
__device__ __forceinline__ float rsqrt_t(float d) { return rsqrtf(d); }
__device__ __forceinline__ double rsqrt_t(double d) { return 1.0 / sqrt(d); }

// Factor the 64 x 64 tile in a (lower part valid, padded with the identity
// beyond b) in place into L, and write L^{-1} into inv.  Deflated columns get
// flag 1 in defl[0..b) (global) and are e_j in L.
template <typename T>
__device__ __forceinline__ void diag_factor(T (*a)[CLD], T (*inv)[CLD], int b, T thr, int* defl, int* bad) {
  __shared__ unsigned dfl16;
  __shared__ T rdg[CT];  // 1 / L_ii (1 for a deflated column)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int o = 0; o < CT; o += 16) {
    // (1) one warp factors the 16 x 16 diagonal block in registers (lane = row).
    // Branch-free: the pivot test is uniform and every per-lane choice is a
    // select, so the column-to-column chain holds only the pivot broadcast,
    // its rsqrt and the broadcasts of the new column.
    if (warp == 0) {
      T row[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) row[c] = (lane < 16 && c <= lane) ? a[o + lane][o + c] : (T)0;
      unsigned df = 0;
      bool nonfinite = false;
      T my_rdg = (T)1;
      T dnext = __shfl_sync(0xFFFFFFFFu, row[0], 0);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const T d = dnext;
        // a pivot is finite and above the threshold (false for NaN); the
        // reciprocal square root is taken unconditionally and only used when
        // it is one, so the chain from one pivot to the next is rsqrt, a
        // multiply, a select, a multiply-add and a broadcast
        const bool piv = (d > thr) && (d < (T)INFINITY);
        nonfinite |= !isfinite(d);
        const T isd = rsqrt_t(d);
        const T base = (lane == c) ? d : ((lane > c) ? row[c] : (T)0);
        const T lraw = base * isd;
        const T lc = piv ? lraw : ((lane == c) ? (T)1 : (T)0);
        my_rdg = (lane == c) ? (piv ? isd : (T)1) : my_rdg;
        df |= piv ? 0u : (1u << c);
        row[c] = lc;
        const T nlc = piv ? -lraw : (T)0;
        // the next pivot, from lane c + 1's own entry (the same multiply-add
        // as its update below), broadcast before the other lanes' updates
        if (c + 1 < 16) dnext = __shfl_sync(0xFFFFFFFFu, fma(nlc, lc, row[c + 1]), c + 1);
#pragma unroll
        for (int k = c + 1; k < 16; ++k) {
          const T lkc = __shfl_sync(0xFFFFFFFFu, lc, k);
          row[k] = fma((lane >= k) ? nlc : (T)0, lkc, row[k]);
        }
      }
      if (lane < 16) {
#pragma unroll
        for (int c = 0; c < 16; ++c) a[o + lane][o + c] = (c <= lane) ? row[c] : (T)0;
        rdg[o + lane] = my_rdg;
        if (defl && o + lane < b) defl[o + lane] = (df >> lane) & 1u;
      }
      if (lane == 0) {
        dfl16 = df;
        if (nonfinite) *bad = 1;
      }
    }
    __syncthreads();
    const int nbelow = CT - o - 16;
    if (nbelow <= 0) break;
    // (2) panel: rows below solve x L_oo^T = a (forward substitution per row)
    if (tid < nbelow) {
      const int i = o + 16 + tid;
      const unsigned df = dfl16;
      T x[16];
#pragma unroll
      for (int c = 0; c < 16; c += 4) vld4(&a[i][o + c], x + c);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        T s = x[c];
#pragma unroll
        for (int j = 0; j < c; ++j) s = fma(-x[j], a[o + c][o + j], s);
        x[c] = ((df >> c) & 1u) ? (T)0 : s * rdg[o + c];
      }
#pragma unroll
      for (int c = 0; c < 16; c += 4) vst4(&a[i][o + c], x + c);
    }
    __syncthreads();
    // (3) trailing update of the lower part below the block, in 4 x 4 blocks
    // (one per thread): a[i][k] -= sum_c a[i][o + c] a[k][o + c], c in order
    {
      const int n4 = nbelow / 4;
      if (tid < n4 * (n4 + 1) / 2) {
        int bi = (int)((sqrtf(8.0f * tid + 1.0f) - 1.0f) * 0.5f);
        while ((bi + 1) * (bi + 2) / 2 <= tid) ++bi;
        while (bi * (bi + 1) / 2 > tid) --bi;
        const int bj = tid - bi * (bi + 1) / 2;
        const int i0 = o + 16 + 4 * bi, k0 = o + 16 + 4 * bj;
        T acc[4][4];
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) vld4(&a[i0 + ii][k0], acc[ii]);
#pragma unroll
        for (int c = 0; c < 16; c += 4) {
          T xi[4][4], xk[4][4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            vld4(&a[i0 + q][o + c], xi[q]);
            vld4(&a[k0 + q][o + c], xk[q]);
          }
#pragma unroll
          for (int cc = 0; cc < 4; ++cc)
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) acc[ii][kk] = fma(-xi[ii][cc], xk[kk][cc], acc[ii][kk]);
        }
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            if (bi > bj || kk <= ii) a[i0 + ii][k0 + kk] = acc[ii][kk];
      }
    }
    __syncthreads();
  }
  // inverse of the lower-triangular tile by blocks, with
  //   inv([A 0; B C]) = [inv(A) 0; -inv(C) B inv(A), inv(C)]:
  // (1) each 16 x 16 diagonal block by one warp (lane = column, forward
  //     substitution in registers, 1 / L_ii from the table), the blocks above
  //     the diagonal zeroed by the other warps;
  // (2) the two 32 x 32 diagonal blocks: off-diagonal 16 x 16 blocks (1, 0), (3, 2);
  // (3) the 64 x 64 tile: off-diagonal 32 x 32 block.
  __shared__ __align__(16) T tmp[32][34];
  if (warp < 4) {
    const int o = warp * 16, c = lane;
    if (c < 16) {
      T x[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        T s = (i == c) ? (T)1 : (T)0;
#pragma unroll
        for (int k = 0; k < i; ++k) s = fma(-a[o + i][o + k], x[k], s);
        x[i] = s * rdg[o + i];  // x_i = 0 above the diagonal (i < c) by the same formula
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) inv[o + i][o + c] = x[i];
    }
  } else {
    for (int e = tid - 128; e < CT * CT; e += CTHREADS - 128) {
      const int i = e >> 6, j = e & 63;
      if ((j >> 4) > (i >> 4)) inv[i][j] = (T)0;
    }
  }
  __syncthreads();
  {
    // (2) T = L[b+1][b] inv(D_b) for b = 0, 2 (one element per thread), then
    //     inv[b+1][b] = -inv(D_{b+1}) T
    const int q = tid >> 8, e = tid & 255, i = e >> 4, j = e & 15, b = 32 * q;
    T acc = (T)0;
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(a[b + 16 + i][b + k], inv[b + k][b + j], acc);
    tmp[16 * q + i][j] = acc;
    __syncthreads();
    acc = (T)0;
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(inv[b + 16 + i][b + 16 + k], tmp[16 * q + k][j], acc);
    inv[b + 16 + i][b + j] = -acc;
    __syncthreads();
  }
  {
    // (3) T = L[32:64][0:32] inv[0:32][0:32] (two adjacent elements per
    //     thread, one 2-element load of inv per k), then
    //     inv[32:64][0:32] = -inv[32:64][32:64] T
    const int i = tid >> 4, j = 2 * (tid & 15);
    T acc0 = (T)0, acc1 = (T)0;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      T v[2];
      vld2(&inv[k][j], v);
      const T x = a[32 + i][k];
      acc0 = fma(x, v[0], acc0);
      acc1 = fma(x, v[1], acc1);
    }
    tmp[i][j] = acc0;
    tmp[i][j + 1] = acc1;
    __syncthreads();
    acc0 = (T)0;
    acc1 = (T)0;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      T v[2];
      vld2(&tmp[k][j], v);
      const T x = inv[32 + i][32 + k];
      acc0 = fma(x, v[0], acc0);
      acc1 = fma(x, v[1], acc1);
    }
    inv[32 + i][j] = -acc0;
    inv[32 + i][j + 1] = -acc1;
  }
  __syncthreads();
}

// CTA-wide: factor diagonal tile p, held (lower part, identity padding beyond
// the matrix) in shared memory a, and store L into G and L^{-1} into Li.
template <typename T>
__device__ __forceinline__ void factor_tile_smem(int p, int r, T* G, int64_t ldg, T* Li, int64_t ldi,
                                                 T thr, int* defl, T (*a)[CLD], T (*inv)[CLD],
                                                 int* bad) {
  const int o = p * CT, b = min(CT, r - o);
  diag_factor<T>(a, inv, b, thr, defl ? defl + o : nullptr, bad);
  for (int e = threadIdx.x; e < CT * CT; e += CTHREADS) {
    const int i = e >> 6, j = e & 63;
    if (i < b && j < b) {
      G[(int64_t)(o + i) * ldg + o + j] = a[i][j];
      Li[(int64_t)(o + i) * ldi + o + j] = inv[i][j];
    }
  }
  __syncthreads();
}

// CTA-wide: factor diagonal tile p of G into G (L) and Li (L^{-1}).
template <typename T>
__device__ __forceinline__ void factor_tile(int p, int r, T* G, int64_t ldg, T* Li, int64_t ldi, T thr,
                                            int* defl, T (*s0)[CLD], T (*s1)[CLD], int* bad) {
  const int o = p * CT, b = min(CT, r - o);
  for (int e = threadIdx.x; e < CT * CT; e += CTHREADS) {
    const int i = e >> 6, j = e & 63;
    T v;
    if (i < b && j < b)
      v = (j <= i) ? __ldcg(G + (int64_t)(o + i) * ldg + o + j) : (T)0;
    else
      v = (i == j) ? (T)1 : (T)0;
    s0[i][j] = v;
  }
  __syncthreads();
  factor_tile_smem<T>(p, r, G, ldg, Li, ldi, thr, defl, s0, s1, bad);
}

// Point-to-point publication of a finished tile: the CTA's writes, then the
// flag (epochs only grow, so the flags need no reset between panels).
__device__ __forceinline__ void post_flag(int* flag, int epoch) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicMax(flag, epoch);
  }
}
// Bounded wait (thread 0) until *flag >= epoch; false, with the status set,
// if it never came.
__device__ __forceinline__ bool wait_flag(const int* flag, int epoch, int* status) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile const int* vf = flag;
    if (*vf < epoch) {
      const long long t0 = clock64();
      while (*vf < epoch) {
        if (clock64() - t0 > (1ll << 32)) {
          set_status(status, DEV_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(CTHREADS, 1)
    k_chol_coop(int r, T* __restrict__ G, int64_t ldg, T* __restrict__ Li, int64_t ldi,
                T* __restrict__ Tm, int64_t ldt, T tol, int* __restrict__ defl,
                int* __restrict__ flags, int* __restrict__ status, GridBar gb) {
  extern __shared__ __align__(16) unsigned char cc_smem[];
  T(*s0)[CLD] = reinterpret_cast<T(*)[CLD]>(cc_smem);
  T(*s1)[CLD] = s0 + CT;
  __shared__ int bad;
  __shared__ T thr_s;
  __shared__ T red[CTHREADS / 32];
  const unsigned nb = gridDim.x;
  const int cta = blockIdx.x, tid = threadIdx.x;
  const int nt = (r + CT - 1) / CT;
  const int ty = tid >> 4, tx = tid & 15;
  if (tid == 0) bad = 0;
  if (cta == 0) {
    T mx = (T)0;
    for (int i = tid; i < r; i += CTHREADS) mx = fmax(mx, G[(int64_t)i * ldg + i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
      T m2 = red[0];
      for (int w = 1; w < CTHREADS / 32; ++w) m2 = fmax(m2, red[w]);
      thr_s = tol * m2;
    }
    __syncthreads();
    factor_tile<T>(0, r, G, ldg, Li, ldi, thr_s, defl, s0, s1, &bad);
  }
  // strictly upper tiles of L^{-1} are zero
  for (int t = cta; t < nt * nt; t += nb) {
    const int ib = t / nt, jb = t - ib * nt;
    if (jb <= ib) continue;
    for (int e = tid; e < CT * CT; e += CTHREADS) {
      const int i = ib * CT + (e >> 6), j = jb * CT + (e & 63);
      if (i < r && j < r) Li[(int64_t)i * ldi + j] = (T)0;
    }
  }
  if (!grid_sync(gb, nb, status)) return;

  for (int p = 0; p + 1 < nt; ++p) {
    const int o = p * CT;
    // panel: L[ib][p] = G[ib][p] inv(L_pp)^T, deflated columns zeroed, each
    // tile published by its flag (epoch p + 1), which the trailing updates
    // wait for.  CTA 0 takes tile p + 1 and, without a round trip through
    // global memory, updates the next diagonal tile with it and factors it
    // (the chain every later panel waits for); CTAs 1.. take the tiles below.
    if (nb > 1 && cta == 0) {
      const int ib = p + 1, od = ib * CT, b = min(CT, r - od);
      ld_tile<T>(s0, G, ldg, od, o, r, r, true);
      ld_tile<T>(s1, Li, ldi, o, o, r, r, true);
      TileRegs<T> gd;  // the diagonal tile before this panel's update (in flight during the product)
      ld_regs(gd, (const T*)G, ldg, od, od, r, r);
      __syncthreads();
      T acc[2][4];
      acc_zero(acc);
      tile_mma<T>(acc, s0, s1);
      __syncthreads();
      int dj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) dj[u] = (o + 4 * tx + u < r) ? __ldcg(defl + o + 4 * tx + u) : 1;
#pragma unroll
      for (int v = 0; v < 2; ++v)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = od + 2 * ty + v, j = o + 4 * tx + u;
          const bool in = i < r && j < r;
          const T val = (in && !dj[u]) ? acc[v][u] : (T)0;
          if (in) G[(int64_t)i * ldg + j] = val;
          s0[4 * tx + u][2 * ty + v] = val;  // transposed: s0[k][i] = L[i][k]
        }
      post_flag(flags + ib, p + 1);
      acc_zero(acc);
      tile_mma<T>(acc, s0, s0);  // L L^T of the diagonal tile
      st_regs(s1, gd, false);
      __syncthreads();
#pragma unroll
      for (int v = 0; v < 2; ++v)
#pragma unroll
        for (int u = 0; u < 4; ++u) s1[2 * ty + v][4 * tx + u] -= acc[v][u];
      __syncthreads();
      // lower part only, identity beyond the matrix
      for (int e = tid; e < CT * CT; e += CTHREADS) {
        const int i = e >> 6, j = e & 63;
        if (i >= b || j >= b)
          s1[i][j] = (i == j) ? (T)1 : (T)0;
        else if (j > i)
          s1[i][j] = (T)0;
      }
      __syncthreads();
      factor_tile_smem<T>(ib, r, G, ldg, Li, ldi, thr_s, defl, s1, s0, &bad);
    } else {
      const int ib0 = (nb == 1) ? p + 1 : p + 1 + cta;
      const int ibs = (nb == 1) ? 1 : (int)nb - 1;
      for (int ib = ib0; ib < nt; ib += ibs) {
        ld_tile<T>(s0, G, ldg, ib * CT, o, r, r, true);
        ld_tile<T>(s1, Li, ldi, o, o, r, r, true);
        __syncthreads();
        T acc[2][4];
        acc_zero(acc);
        int dj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) dj[u] = (o + 4 * tx + u < r) ? __ldcg(defl + o + 4 * tx + u) : 1;
        tile_mma<T>(acc, s0, s1);
#pragma unroll
        for (int v = 0; v < 2; ++v)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = ib * CT + 2 * ty + v, j = o + 4 * tx + u;
            if (i < r && j < r) G[(int64_t)i * ldg + j] = dj[u] ? (T)0 : acc[v][u];
          }
        post_flag(flags + ib, p + 1);
      }
      // trailing update G[ib][jb] -= L[ib][p] L[jb][p]^T, p + 1 <= jb <= ib,
      // row-major over the lower triangle; tile t = 0, the next diagonal tile,
      // is CTA 0's (above) unless one CTA does all
      const int rest = nt - p - 1;
      const int ntr = rest * (rest + 1) / 2;
      const int t0 = (nb == 1) ? 0 : cta;
      const int step = (nb == 1) ? 1 : (int)nb - 1;
      for (int t = t0; t < ntr; t += step) {
        int ii = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
        while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
        while (ii * (ii + 1) / 2 > t) --ii;
        const int jj = t - ii * (ii + 1) / 2;
        const int ib = p + 1 + ii, jb = p + 1 + jj;
        if (!wait_flag(flags + ib, p + 1, status) || !wait_flag(flags + jb, p + 1, status)) return;
        ld_tile<T>(s0, G, ldg, ib * CT, o, r, r, true);
        ld_tile<T>(s1, G, ldg, jb * CT, o, r, r, true);
        __syncthreads();
        T acc[2][4];
        acc_zero(acc);
        tile_mma<T>(acc, s0, s1);
#pragma unroll
        for (int v = 0; v < 2; ++v)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = ib * CT + 2 * ty + v, j = jb * CT + 4 * tx + u;
            if (i < r && j < r && j <= i) {
              T* g = G + (int64_t)i * ldg + j;
              *g = __ldcg(g) - acc[v][u];
            }
          }
        __syncthreads();
      }
      if (nb == 1) factor_tile<T>(p + 1, r, G, ldg, Li, ldi, thr_s, defl, s0, s1, &bad);
    }
    if (!grid_sync(gb, nb, status)) return;
  }

  // off-diagonal tiles of L^{-1}, recursive doubling over tile groups
  for (int h = 1; h < nt; h *= 2) {
    const int groups = (nt + 2 * h - 1) / (2 * h);
    const int total = groups * h * h;
    // Tm[ib][jb] = sum_{kb = jb}^{o + h - 1} L[ib][kb] inv(L)[kb][jb]
    for (int it = cta; it < total; it += nb) {
      const int g = it / (h * h), rem = it - g * h * h;
      const int og = 2 * h * g;
      const int ib = og + h + rem / h, jb = og + rem % h;
      if (ib >= nt) continue;
      T acc[2][4];
      acc_zero(acc);
      tile_chain<T>(
          acc, jb, og + h,
          [&](TileRegs<T>& t, int kb) { ld_regs(t, (const T*)G, ldg, ib * CT, kb * CT, r, r); },
          [&](TileRegs<T>& t, int kb) { ld_regs(t, (const T*)Li, ldi, kb * CT, jb * CT, r, r); }, s0, s1);
#pragma unroll
      for (int v = 0; v < 2; ++v)
#pragma unroll
        for (int u = 0; u < 4; ++u)
          Tm[(int64_t)(ib * CT + 2 * ty + v) * ldt + jb * CT + 4 * tx + u] = acc[v][u];
    }
    if (!grid_sync(gb, nb, status)) return;
    // inv(L)[ib][jb] = -sum_{kb = o + h}^{ib} inv(L)[ib][kb] Tm[kb][jb]
    for (int it = cta; it < total; it += nb) {
      const int g = it / (h * h), rem = it - g * h * h;
      const int og = 2 * h * g;
      const int ib = og + h + rem / h, jb = og + rem % h;
      if (ib >= nt) continue;
      T acc[2][4];
      acc_zero(acc);
      tile_chain<T>(
          acc, og + h, ib + 1,
          [&](TileRegs<T>& t, int kb) { ld_regs(t, (const T*)Li, ldi, ib * CT, kb * CT, r, r); },
          [&](TileRegs<T>& t, int kb) {
            ld_regs(t, (const T*)Tm, ldt, kb * CT, jb * CT, nt * CT, nt * CT);
          },
          s0, s1);
#pragma unroll
      for (int v = 0; v < 2; ++v)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = ib * CT + 2 * ty + v, j = jb * CT + 4 * tx + u;
          if (i < r && j < r) Li[(int64_t)i * ldi + j] = -acc[v][u];
        }
    }
    if (!grid_sync(gb, nb, status)) return;
  }
  if (tid == 0 && bad) set_status(status, DEV_NONFINITE);
}

// Returns SPM_EUNSUPPORTED (nothing launched) when the cooperative grid does
// not fit; the caller then takes the multi-launch path.
template <typename T>
static int cholesky_inv_coop_t(int64_t r, T* G, int64_t ldg, T* Li, int64_t ldi, int* defl,
                               int* status, cudaStream_t st) {
  const int nt = (int)cdiv(r, CT);
  const T tol = std::is_same<T, double>::value ? (T)1e-12 : (T)1e-6;
  int dev = 0, sms = 0, per_sm = 0;
  SPM_CUDA_TRY(cudaGetDevice(&dev));
  SPM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int smem = (int)(2 * CT * CLD * sizeof(T));
  auto kern = k_chol_coop<T>;
  SPM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  SPM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CTHREADS, smem));
  if (per_sm < 1) return SPM_EUNSUPPORTED;
  const int want = std::max(1, nt * (nt - 1) / 2 + 1);
  const int blocks = std::min(want, sms);
  Arena ar(st);
  SPM_ALLOC(ar, T, Tm, (int64_t)nt * CT * nt * CT);
  SPM_ALLOC(ar, unsigned, bar, 2);
  SPM_ALLOC(ar, int, flags, nt);
  if (!defl) {
    defl = ar.alloc<int>(r);
    if (!defl) return SPM_ENOMEM;
  }
  SPM_CUDA_TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
  SPM_CUDA_TRY(cudaMemsetAsync(flags, 0, nt * sizeof(int), st));
  GridBar gb{bar, bar + 1};
  int rr = (int)r;
  int64_t ldt = (int64_t)nt * CT;
  T tolv = tol;
  void* args[] = {(void*)&rr, (void*)&G, (void*)&ldg, (void*)&Li, (void*)&ldi, (void*)&Tm,
                  (void*)&ldt, (void*)&tolv, (void*)&defl, (void*)&flags, (void*)&status,
                  (void*)&gb};
  SPM_CUDA_TRY(cudaLaunchCooperativeKernel((void*)kern, dim3(blocks), dim3(CTHREADS), args, smem, st));
  count_launch();
  return SPM_OK;
}

int cholesky_inv_coop(int64_t r, void* G, int64_t ldg, void* Linv, int64_t ldi, int dt, int* defl,
                      int* status, cudaStream_t st) {
  if (r < 1 || r > 8192) return SPM_EUNSUPPORTED;
  if (dt == DT_F64)
    return cholesky_inv_coop_t<double>(r, (double*)G, ldg, (double*)Linv, ldi, defl, status, st);
  if (dt == DT_F32)
    return cholesky_inv_coop_t<float>(r, (float*)G, ldg, (float*)Linv, ldi, defl, status, st);
  return SPM_EINVAL;
}

}  // namespace spm
