// tcgen05 tensor-core GEMM for the dense tall-skinny contractions of the
// sketched power method (Algorithm 1 line 1: A~ Z and A~^T Y; the final
// projection B = Q^T A of the Randomized SVD finish; CholeskyQR Gram and
// triangular products).
//
// D (M x N, fp32) = alpha * sum_{q < npass} A_q (M x K) * B_q (N x K)^T
// with BF16 operands and FP32 accumulation in tensor memory.  npass = 3 with
// (hi, lo) operand pairs gives the split-precision product hi*hi + hi*lo + lo*hi.
//
// Per CTA: one 128 x BN output tile.  Warp 0 issues TMA loads (128-byte
// swizzle) into a STAGES-deep shared-memory ring, warp 1 owns the tensor-memory
// allocation and issues tcgen05.mma from one thread, warps 2..5 drain the
// accumulator (tcgen05.ld) and store.  Operands may be K-major or MN-major in
// global memory; TMA zero-fills every out-of-range element, so ragged M, N, K
// need no padding.  Every mbarrier wait is bounded: on expiry the CTA records
// SPM_ETIMEOUT in the status word, drains its own copies and returns.
#include <cuda.h>

#include <mutex>
#include <type_traits>

#include "internal.cuh"

namespace spm {

static constexpr int TC_BM = 128;
static constexpr int TC_BK = 64;           // 64 bf16 = 128 bytes = one swizzle row
static constexpr int TC_THREADS = 192;
static constexpr long long TC_WAIT_LIMIT = 1ll << 31;  // clock cycles (~1 s)

template <int BN>
struct TcCfg {
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;
  static constexpr int B_BYTES = BN * TC_BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = (192 * 1024) / STAGE_BYTES;
  static constexpr int EP_BYTES = 4 * 32 * 33 * 4;  // epilogue staging: a 32 x 33 block per warp
  static constexpr int SMEM = STAGES * STAGE_BYTES + EP_BYTES + 1024 /*align*/ + 256 /*barriers*/;
};

struct TcParams {
  int M, N, K;
  int k_tiles, kt_per_split, npass;
  float alpha;
  float* D;
  int64_t d_rs, d_cs, split_stride;
  int* status;
  int sym_upper;  // skip output tiles that lie entirely below the diagonal
  int fused3;     // split product A0 B0 + A0 B1 + A2 B0 (A1 = A0, B2 = B0): each k-tile
                  // takes two ring stages, (A0, B0) and (A2, B1), and all three MMAs
  int mt, nt, splits;  // output tiles along M and N, K splits: the work units
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and status set) if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > TC_WAIT_LIMIT) {
      set_status(status, DEV_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor (tcgen05): start >> 4 in bits 0-13, leading
// byte offset >> 4 in 16-29, stride byte offset >> 4 in 32-45, the fixed
// value 1 in bits 46-48, swizzle mode 2 (128-byte) in bits 61-63.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;
  d |= 2ull << 61;
  return d;
}

// Instruction descriptor, kind::f16: D fp32 (bit 4), A and B bf16 (bits 7, 10),
// A/B major (bits 15, 16: 1 = MN-major), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
template <int BN, bool A_MN, bool B_MN>
__host__ __device__ constexpr uint32_t instr_desc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((A_MN ? 1u : 0u) << 15) | ((B_MN ? 1u : 0u) << 16) |
         ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
        "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
        "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Persistent: each CTA walks the work units (output tile and K split) u =
// blockIdx.x, blockIdx.x + gridDim.x, ...; its producer, MMA and epilogue roles
// walk the same sequence.  The stage ring runs on across units, and the TMEM
// accumulator is double-buffered (2 x BN columns): the epilogue drains unit t's
// buffer while the MMA thread fills unit t + 1's.  Every operand tile is fetched
// by this CTA's own TMA loads from this GPU's memory.  A bounded wait that
// expires sets the status word and a CTA-wide abort flag that every role checks.
template <int BN, bool A_MN, bool B_MN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap ta0, const __grid_constant__ CUtensorMap ta1,
              const __grid_constant__ CUtensorMap ta2, const __grid_constant__ CUtensorMap tb0,
              const __grid_constant__ CUtensorMap tb1, const __grid_constant__ CUtensorMap tb2,
              TcParams p) {
  using Cfg = TcCfg<BN>;
  constexpr int STAGES = Cfg::STAGES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the 128-byte swizzle atoms
  unsigned char* smem =
      smem_raw + ((1024 - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* tiles = smem;
  unsigned char* ep = smem + STAGES * Cfg::STAGE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(ep + Cfg::EP_BYTES);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  const uint32_t full0 = smem_u32(bars);
  const uint32_t empty0 = smem_u32(bars + STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * STAGES);      // accumulator b filled: 2 barriers
  const uint32_t tempty0 = smem_u32(bars + 2 * STAGES + 2); // accumulator b drained: 2 barriers
  const uint32_t done = smem_u32(bars + 2 * STAGES + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = p.mt * p.nt * p.splits;
  const int per_kt = p.fused3 ? 2 : p.npass;  // ring stages per k-tile
  static_assert(STAGES % 2 == 0, "a fused k-tile's two stages must not wrap");
  // unit u: M tile fastest (consecutive CTAs share the B tile), then N tile, then split
  auto decode = [&](int u, int& m0, int& n0, int& z, int& kt0, int& kt1) {
    const int mi = u % p.mt, ni = (u / p.mt) % p.nt;
    z = u / (p.mt * p.nt);
    m0 = mi * TC_BM;
    n0 = ni * BN;
    kt0 = z * p.kt_per_split;
    kt1 = min(p.k_tiles, kt0 + p.kt_per_split);
    // symmetric output: a tile entirely below the diagonal is skipped by every role
    return !(p.sym_upper && m0 >= n0 + BN);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, 4);  // one arrival per epilogue warp
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");  // barrier inits visible to the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"((uint32_t)(2 * BN))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  auto fail = [&]() { *abort_flag = 1; };

  if (warp == 0) {
    if (lane == 0) {
      const CUtensorMap* ta[3] = {&ta0, &ta1, &ta2};
      const CUtensorMap* tb[3] = {&tb0, &tb1, &tb2};
      int g = 0;  // ring iteration over all units
      for (int u = blockIdx.x; u < units && !*abort_flag; u += gridDim.x) {
        int m0, n0, z, kt0, kt1;
        if (!decode(u, m0, n0, z, kt0, kt1)) continue;
        const int iters = (kt1 - kt0) * per_kt;
        for (int it = 0; it < iters; ++it, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
          if (*abort_flag || !mbar_wait(empty0 + 8 * s, ph ^ 1u, p.status)) {
            fail();
            break;
          }
          const int kt = kt0 + it / per_kt;
          const int q = it % per_kt;
          // fused: the k-tile's first stage holds (A0, B0), its second (A2, B1)
          const int qa = p.fused3 ? (q == 0 ? 0 : 2) : q;
          const int qb = p.fused3 ? (q == 0 ? 0 : 1) : q;
          const int k0 = kt * TC_BK;
          const uint32_t fb = full0 + 8 * s;
          mbar_expect_tx(fb, Cfg::STAGE_BYTES);
          const uint32_t sa = smem_u32(tiles + s * Cfg::STAGE_BYTES);
          const uint32_t sb = sa + Cfg::A_BYTES;
          if (!A_MN) {
            tma_load_2d(sa, ta[qa], k0, m0, fb);
          } else {
#pragma unroll
            for (int b = 0; b < TC_BM / 64; ++b) tma_load_2d(sa + b * 8192, ta[qa], m0 + 64 * b, k0, fb);
          }
          if (!B_MN) {
            tma_load_2d(sb, tb[qb], k0, n0, fb);
          } else {
#pragma unroll
            for (int b = 0; b < BN / 64; ++b) tma_load_2d(sb + b * 8192, tb[qb], n0 + 64 * b, k0, fb);
          }
        }
      }
      // drain: every copy this thread issued must have landed before exit
      for (int it = max(0, g - STAGES); it < g; ++it)
        mbar_wait(full0 + 8 * (it % STAGES), (uint32_t)(it / STAGES) & 1u, p.status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = instr_desc<BN, A_MN, B_MN>();
      auto desc_a = [&](uint32_t sa, int kk) {
        return A_MN ? smem_desc(sa + kk * 2048, 8192, 1024) : smem_desc(sa + kk * 32, 16, 1024);
      };
      auto desc_b = [&](uint32_t sb, int kk) {
        return B_MN ? smem_desc(sb + kk * 2048, 8192, 1024) : smem_desc(sb + kk * 32, 16, 1024);
      };
      int g = 0, t = 0;
      for (int u = blockIdx.x; u < units && !*abort_flag; u += gridDim.x) {
        int m0, n0, z, kt0, kt1;
        if (!decode(u, m0, n0, z, kt0, kt1)) continue;
        const int iters = (kt1 - kt0) * per_kt;
        const int b = t & 1;
        // the accumulator's previous unit (t - 2) has been drained
        if (!mbar_wait(tempty0 + 8 * b, ((uint32_t)(t >> 1) & 1u) ^ 1u, p.status)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(b * BN);
        bool ok = true;
        // fused split product: per k-tile wait for both stages, issue A0 B0, A0 B1,
        // A2 B0 (the order of the unfused passes), release both stages
        for (int j = 0; p.fused3 && j < iters / 2; ++j, g += 2) {
          const int s0 = g % STAGES, s1 = (g + 1) % STAGES;
          if (*abort_flag || !mbar_wait(full0 + 8 * s0, (uint32_t)(g / STAGES) & 1u, p.status) ||
              !mbar_wait(full0 + 8 * s1, (uint32_t)((g + 1) / STAGES) & 1u, p.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_hi = smem_u32(tiles + s0 * Cfg::STAGE_BYTES), b_hi = a_hi + Cfg::A_BYTES;
          const uint32_t a_lo = smem_u32(tiles + s1 * Cfg::STAGE_BYTES), b_lo = a_lo + Cfg::A_BYTES;
#pragma unroll
          for (int tt = 0; tt < 3; ++tt) {
            const uint32_t sa = (tt == 2) ? a_lo : a_hi;
            const uint32_t sb = (tt == 1) ? b_lo : b_hi;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk)
              tc_mma(acc, desc_a(sa, kk), desc_b(sb, kk), idesc, (j > 0 || tt > 0 || kk > 0) ? 1u : 0u);
          }
          tc_commit(empty0 + 8 * s0);
          tc_commit(empty0 + 8 * s1);
        }
        for (int it = 0; !p.fused3 && it < iters; ++it, ++g) {
          const int s = g % STAGES;
          if (*abort_flag || !mbar_wait(full0 + 8 * s, (uint32_t)(g / STAGES) & 1u, p.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(tiles + s * Cfg::STAGE_BYTES);
          const uint32_t sb = sa + Cfg::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk)
            tc_mma(acc, desc_a(sa, kk), desc_b(sb, kk), idesc, (it > 0 || kk > 0) ? 1u : 0u);
          tc_commit(empty0 + 8 * s);
        }
        if (!ok) {
          fail();
          break;
        }
        tc_commit(tfull0 + 8 * b);  // fires once this unit's MMAs have completed
        ++t;
      }
      tc_commit(done);  // fires once every MMA above has completed
    }
  } else {
    // epilogue warps 2..5: TMEM lane quarter = warp % 4
    const int quarter = warp & 3;
    float(*st)[33] = reinterpret_cast<float(*)[33]>(ep + quarter * 32 * 33 * sizeof(float));
    int t = 0;
    for (int u = blockIdx.x; u < units && !*abort_flag; u += gridDim.x) {
      int m0, n0, z, kt0, kt1;
      if (!decode(u, m0, n0, z, kt0, kt1)) continue;
      const int b = t & 1;
      bool ok = true;
      if (lane == 0) ok = mbar_wait(tfull0 + 8 * b, (uint32_t)(t >> 1) & 1u, p.status);
      ok = __shfl_sync(0xFFFFFFFFu, ok ? 1 : 0, 0) != 0;
      if (!ok) {
        if (lane == 0) fail();
        break;
      }
      tc_fence_after();
      if (kt1 > kt0) {
        const uint32_t acc = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN);
        const int row = m0 + quarter * 32 + lane;
        float* D = p.D + (int64_t)z * p.split_stride;
        if (p.d_cs == 1) {
          // row-major output: each 32 x 32 block goes through shared memory so
          // that a warp stores one 128-byte row segment at a time
          const int rbase = m0 + quarter * 32;
#pragma unroll 1
          for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(acc + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) st[lane][j] = p.alpha * __uint_as_float(v[j]);
            __syncwarp();
            const int col = n0 + c0 + lane;
#pragma unroll 4
            for (int r = 0; r < 32; ++r)
              if (rbase + r < p.M && col < p.N) D[(int64_t)(rbase + r) * p.d_rs + col] = st[r][lane];
            __syncwarp();
          }
        } else {
#pragma unroll 1
          for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(acc + (uint32_t)c0, v);
            if (row < p.M) {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const int col = n0 + c0 + j;
                if (col < p.N) D[(int64_t)row * p.d_rs + (int64_t)col * p.d_cs] = p.alpha * __uint_as_float(v[j]);
              }
            }
          }
        }
      }
      // this warp's reads of the accumulator are done: hand it back to the MMA thread
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * b);
      ++t;
    }
  }
  tc_fence_before();
  __syncthreads();
  // the MMA thread's final commit must have fired before the columns go back
  if (warp == 1 && lane == 0) mbar_wait(done, 0, p.status);
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(2 * BN))
                 : "memory");
  }
}

// Deterministic split-K reduction: D[i, j] = sum_{z < splits} W[z][i][j] in order.
__global__ void k_splitk_reduce(int M, int N, int splits, const float* __restrict__ W,
                                float* __restrict__ D, int64_t d_rs, int64_t d_cs) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += W[(int64_t)z * total + e];
    const int64_t i = e / N, j = e % N;
    D[i * d_rs + j * d_cs] = s;
  }
}

// ------------------------------------------------------------------ host side
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                    const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                    const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode() {
  static PFN_encodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_encodeTiled)f;
  }
  return fn;
}

bool tc_available() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  int maj = 0, min_ = 0;
  cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&min_, cudaDevAttrComputeCapabilityMinor, dev);
  return maj == 10 && min_ == 3 && get_encode() != nullptr;
}

// Tensor map of one operand.  rows_mn = M (or N), k = K.
static int make_map(CUtensorMap* map, const TcOp& op, int64_t rows_mn, int64_t k, int box_outer) {
  PFN_encodeTiled enc = get_encode();
  if (!enc) return SPM_ECUDA;
  if (((uintptr_t)op.p & 15u) != 0 || (op.ld % 8) != 0) return SPM_EINVAL;
  cuuint64_t dims[2], strides[1];
  cuuint32_t box[2], es[2] = {1, 1};
  if (!op.mn_major) {  // array rows_mn x k, k contiguous
    dims[0] = (cuuint64_t)k;
    dims[1] = (cuuint64_t)rows_mn;
    box[0] = TC_BK;
    box[1] = (cuuint32_t)box_outer;
  } else {             // array k x rows_mn, mn contiguous
    dims[0] = (cuuint64_t)rows_mn;
    dims[1] = (cuuint64_t)k;
    box[0] = 64;
    box[1] = TC_BK;
  }
  strides[0] = (cuuint64_t)op.ld * 2;
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)op.p, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SPM_OK : SPM_EINVAL;
}

template <int BN, bool A_MN, bool B_MN>
static int launch_tc(const CUtensorMap* ta, const CUtensorMap* tb, const TcParams& p, dim3 grid,
                     cudaStream_t st) {
  auto kern = k_gemm_tc<BN, A_MN, B_MN>;
  SPM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    TcCfg<BN>::SMEM));
  kern<<<grid, TC_THREADS, TcCfg<BN>::SMEM, st>>>(ta[0], ta[1], ta[2], tb[0], tb[1], tb[2], p);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

template <int BN>
static int launch_bn(bool amn, bool bmn, const CUtensorMap* ta, const CUtensorMap* tb,
                     const TcParams& p, dim3 grid, cudaStream_t st) {
  if (!amn && !bmn) return launch_tc<BN, false, false>(ta, tb, p, grid, st);
  if (!amn && bmn) return launch_tc<BN, false, true>(ta, tb, p, grid, st);
  if (amn && !bmn) return launch_tc<BN, true, false>(ta, tb, p, grid, st);
  return launch_tc<BN, true, true>(ta, tb, p, grid, st);
}

// The split pattern A0 B0 + A0 B1 + A2 B0 (A1 = A0, B2 = B0): four distinct
// operand tiles per k-tile instead of six.
static int fused_split(int npass, const TcOp* A, const TcOp* B) {
  auto same = [](const TcOp& x, const TcOp& y) {
    return x.p == y.p && x.ld == y.ld && x.mn_major == y.mn_major;
  };
  return (npass == 3 && same(A[0], A[1]) && same(B[0], B[2])) ? 1 : 0;
}

// SM count of the current device (cached per device)
static int tc_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (dev < 0 || dev >= 64) return 148;
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 148;
    cache[dev] = n;
  }
  return cache[dev];
}

// persistent grid: one CTA per SM (the kernel's shared memory allows one), or
// fewer when there are fewer work units
static dim3 tc_grid(TcParams& p, int64_t mt, int64_t nt, int splitk) {
  p.mt = (int)mt;
  p.nt = (int)nt;
  p.splits = splitk;
  const int64_t units = mt * nt * splitk;
  return dim3((unsigned)min64(units, tc_sms()));
}

// strictly lower triangle of D (n x n) from the upper one
__global__ void k_mirror_upper(int n, float* __restrict__ D, int64_t d_rs, int64_t d_cs) {
  for (int i = blockIdx.y; i < n; i += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < i; j += gridDim.x * blockDim.x)
      D[(int64_t)i * d_rs + (int64_t)j * d_cs] = D[(int64_t)j * d_rs + (int64_t)i * d_cs];
}

int gemm_tc(int64_t M, int64_t N, int64_t K, int npass, const TcOp* A, const TcOp* B, float alpha,
            float* D, int64_t d_rs, int64_t d_cs, int splitk, cudaStream_t st, bool sym_upper,
            int* status) {
  if (sym_upper && M != N) return SPM_EINVAL;
  if (M <= 0 || N <= 0) return SPM_OK;
  if (npass < 1 || npass > 3) return SPM_EINVAL;
  if (M > 0x7FFFFFFF || N > 0x7FFFFFFF || K > 0x7FFFFFFF) return SPM_EUNSUPPORTED;
  if (K <= 0) {
    // empty contraction: D = 0
    Arena ar(st);
    (void)ar;
    return SPM_EUNSUPPORTED;
  }
  for (int q = 0; q < npass; ++q)
    if (A[q].mn_major != A[0].mn_major || B[q].mn_major != B[0].mn_major) return SPM_EINVAL;
  const int BN = (N >= 192) ? 256 : 128;
  CUtensorMap ta[3], tb[3];
  for (int q = 0; q < 3; ++q) {
    const int qq = q < npass ? q : 0;
    SPM_TRY(make_map(&ta[q], A[qq], M, K, TC_BM));
    SPM_TRY(make_map(&tb[q], B[qq], N, K, BN));
  }
  const int k_tiles = (int)cdiv(K, TC_BK);
  if (splitk < 1) splitk = 1;
  if (splitk > k_tiles) splitk = k_tiles;
  const int kt_per = (int)cdiv(k_tiles, splitk);
  splitk = (int)cdiv(k_tiles, kt_per);
  const int64_t mt = cdiv(M, TC_BM), nt = cdiv(N, BN);
  if (mt > 0x7FFFFFFF || nt > 65535 || splitk > 65535 || mt * nt * splitk > 0x7FFFFFFF)
    return SPM_EUNSUPPORTED;
  TcParams p{};
  p.M = (int)M;
  p.N = (int)N;
  p.K = (int)K;
  p.k_tiles = k_tiles;
  p.kt_per_split = kt_per;
  p.npass = npass;
  p.alpha = alpha;
  p.status = status;
  p.sym_upper = sym_upper ? 1 : 0;
  p.fused3 = fused_split(npass, A, B);
  const dim3 grid = tc_grid(p, mt, nt, splitk);
  Arena ar(st);
  if (splitk == 1) {
    p.D = D;
    p.d_rs = d_rs;
    p.d_cs = d_cs;
    p.split_stride = 0;
  } else {
    SPM_ALLOC(ar, float, W, (int64_t)splitk * M * N);
    p.D = W;
    p.d_rs = N;
    p.d_cs = 1;
    p.split_stride = M * N;
  }
  if (BN == 256)
    SPM_TRY((launch_bn<256>(A[0].mn_major, B[0].mn_major, ta, tb, p, grid, st)));
  else
    SPM_TRY((launch_bn<128>(A[0].mn_major, B[0].mn_major, ta, tb, p, grid, st)));
  if (splitk > 1) {
    const int64_t total = M * N;
    const int blocks = (int)min64(cdiv(total, 256), 152 * 8);
    k_splitk_reduce<<<blocks, 256, 0, st>>>((int)M, (int)N, splitk, p.D, D, d_rs, d_cs);
    SPM_LAUNCH_CHECK();
  }
  if (sym_upper) {
    const dim3 g((unsigned)min64(cdiv(M, 256), 8), (unsigned)min64(M, 1024));
    k_mirror_upper<<<g, 256, 0, st>>>((int)M, D, d_rs, d_cs);
    SPM_LAUNCH_CHECK();
  }
  return SPM_OK;
}


// ------------------------------------------------------------------ no-allocation variant
// Some callers may not allocate device memory at all: a plug-in that runs
// inside an inference engine which owns the whole device pool, or a serving
// process that reserves its memory once at start-up and must not grow it.
// For them spm_gemm_bf16_noalloc keeps its split-K partial sums in this
// file-scope device array instead of stream-ordered workspace.  The array lives
// on every GPU that loads the library until the process exits.  In host code
// its name is only a host-side stand-in, never a device address: the device
// address is looked up with cudaGetSymbolAddress (which allocates nothing) on
// every call, so a cached address can never outlive the context it came from.
static constexpr int64_t kNoAllocScratchFloats = (int64_t)SPM_NOALLOC_SCRATCH_FLOATS;
static __device__ __align__(256) float g_noalloc_scratch[SPM_NOALLOC_SCRATCH_FLOATS];
// First device-side status (0 or SPM_ETIMEOUT) of the public product entry
// points on this device since it was last cleared (spm_gemm_bf16_status).
static __device__ int g_gemm_status;

// Device addresses of the scratch array and of the status word on the current device.
static int gemm_symbols(float** scratch, int** status) {
  void* p = nullptr;
  if (scratch) {
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SPM_ECUDA;
    *scratch = reinterpret_cast<float*>(p);
  }
  if (status) {
    p = nullptr;
    if (cudaGetSymbolAddress(&p, g_gemm_status) != cudaSuccess || !p) return SPM_ECUDA;
    *status = reinterpret_cast<int*>(p);
  }
  return SPM_OK;
}

int gemm_public_status(int** status) { return gemm_symbols(nullptr, status); }

int gemm_tc_noalloc(int64_t M, int64_t N, int64_t K, int npass, const TcOp* A, const TcOp* B,
                    float* D, int64_t ldd, int splitk, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0 || npass < 1 || npass > 3) return SPM_EINVAL;
  if (M > 0x7FFFFFFF || N > 0x7FFFFFFF || K > 0x7FFFFFFF) return SPM_EUNSUPPORTED;
  for (int q = 0; q < npass; ++q)
    if (A[q].mn_major != A[0].mn_major || B[q].mn_major != B[0].mn_major) return SPM_EINVAL;
  const int BN = (N >= 192) ? 256 : 128;
  const int k_tiles = (int)cdiv(K, TC_BK);
  if (splitk < 1) splitk = 1;
  if (splitk > k_tiles) splitk = k_tiles;
  const int kt_per = (int)cdiv(k_tiles, splitk);
  splitk = (int)cdiv(k_tiles, kt_per);
  // the partial sums must fit the fixed scratch array
  if (splitk > 1 && (int64_t)splitk * M * N > kNoAllocScratchFloats) return SPM_EINVAL;
  const int64_t mt = cdiv(M, TC_BM), nt = cdiv(N, BN);
  if (mt > 0x7FFFFFFF || nt > 65535 || splitk > 65535 || mt * nt * splitk > 0x7FFFFFFF)
    return SPM_EUNSUPPORTED;
  float* scratch = nullptr;
  int* status = nullptr;
  SPM_TRY(gemm_symbols(&scratch, &status));
  CUtensorMap ta[3], tb[3];
  for (int q = 0; q < 3; ++q) {
    const int qq = q < npass ? q : 0;
    SPM_TRY(make_map(&ta[q], A[qq], M, K, TC_BM));
    SPM_TRY(make_map(&tb[q], B[qq], N, K, BN));
  }
  TcParams p{};
  p.M = (int)M;
  p.N = (int)N;
  p.K = (int)K;
  p.k_tiles = k_tiles;
  p.kt_per_split = kt_per;
  p.npass = npass;
  p.alpha = 1.0f;
  p.status = status;
  p.fused3 = fused_split(npass, A, B);
  if (splitk == 1) {
    p.D = D;
    p.d_rs = ldd;
    p.d_cs = 1;
    p.split_stride = 0;
  } else {
    // every partial the reduction reads is written first by the GEMM, so the
    // scratch needs no clearing between calls
    p.D = scratch;
    p.d_rs = N;
    p.d_cs = 1;
    p.split_stride = M * N;
  }
  const dim3 grid = tc_grid(p, mt, nt, splitk);
  if (BN == 256)
    SPM_TRY((launch_bn<256>(A[0].mn_major, B[0].mn_major, ta, tb, p, grid, st)));
  else
    SPM_TRY((launch_bn<128>(A[0].mn_major, B[0].mn_major, ta, tb, p, grid, st)));
  if (splitk > 1) {
    const int64_t total = M * N;
    const int blocks = (int)min64(cdiv(total, 256), 152 * 8);
    k_splitk_reduce<<<blocks, 256, 0, st>>>((int)M, (int)N, splitk, scratch, D, ldd, 1);
    SPM_LAUNCH_CHECK();
  }
  return SPM_OK;
}

}  // namespace spm

extern "C" int spm_gemm_bf16_noalloc(int64_t M, int64_t N, int64_t K, int32_t npass,
                                     const void* const* A, int64_t lda, int32_t a_mn,
                                     const void* const* B, int64_t ldb, int32_t b_mn, float* D,
                                     int64_t ldd, int32_t splitk, void* stream) {
  using namespace spm;
  if (M < 1 || N < 1 || K < 1 || npass < 1 || npass > 3 || !A || !B || !D || ldd < N || splitk < 1)
    return SPM_EINVAL;
  if (lda < (a_mn ? M : K) || ldb < (b_mn ? N : K)) return SPM_EINVAL;
  if (!tc_available()) return SPM_ECUDA;
  TcOp a[3], b[3];
  for (int q = 0; q < npass; ++q) {
    if (!A[q] || !B[q]) return SPM_EINVAL;
    a[q] = TcOp{(const __nv_bfloat16*)A[q], lda, a_mn != 0};
    b[q] = TcOp{(const __nv_bfloat16*)B[q], ldb, b_mn != 0};
  }
  return gemm_tc_noalloc(M, N, K, npass, a, b, D, ldd, splitk, as_stream(stream));
}

extern "C" int spm_gemm_bf16_status(int32_t clear, void* stream) {
  using namespace spm;
  int* status = nullptr;
  SPM_TRY(gemm_symbols(nullptr, &status));
  cudaStream_t st = as_stream(stream);
  int h = 0;
  SPM_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (clear) SPM_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  SPM_CUDA_TRY(cudaStreamSynchronize(st));
  return h;
}
