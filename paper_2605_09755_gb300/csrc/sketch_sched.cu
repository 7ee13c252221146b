// Scheduled sketch product A~ = A S (Algorithm 1 line 1; Algorithm 3 line 1)
// for FP32 A whose rows fit whole in shared memory.
//
// Column c of A~ is the sum over the bucket of c of sign(j, c) A[:, j] / sqrt(s)
// (Lemma 3.2 item 2).  One CTA (1024 threads) owns a group of up to 1008 output
// columns, one lane per column part, and a stream of rows i = p, p + P, ...;
// the G column groups of a row run in G CTAs.  Each row of A arrives whole in
// a three-slot shared-memory ring by one 1D TMA bulk copy (cp.async.bulk)
// issued three rows ahead, behind a 32-float zero pad.  A lane then reads the
// row elements of its bucket, one per step, from offsets it holds in 48
// registers (two 15-bit offsets each): the plan (sched_plan.h) has coloured
// every step of every warp so that its 32 reads fall in 32 distinct banks, one
// shared-memory wavefront per step, and has put the + entries and the -
// entries of each lane in two phases, so a step is one offset extraction, one
// address, one shared load and one add.  A lane enters each phase at its
// warp's step count through a jump table (Duff's device over the unrolled
// steps).  Each lane leaves its sum in a staging row; after one CTA barrier the
// staging row is scaled and written out coalesced (BF16 hi + lo, or FP32),
// while the ring slot it came from is refilled.  With FRO the lanes also sum
// the squares of what they read: every element of A is read exactly s times
// over all groups, so the sum over all CTAs, divided by s, is |A|_F^2.
//
// With a split output (ahi set) each row is also written out as its (hi, lo)
// BF16 split, hi = bf16(a), lo = bf16(a - hi), while it sits in shared memory:
// group g's CTA splits the g-th of G equal column ranges of the row (four
// elements per thread and pass), so A is read from HBM once for the sketch
// product and the tensor-core projection Q^T A that follows.
//
// Every wait on a ring slot is bounded; on expiry the CTA records
// SPM_ETIMEOUT, waits (bounded) for the copies it still has in flight and
// returns.
#include <math.h>

#include <mutex>
#include <vector>

#include "internal.cuh"
#include "bulk.cuh"
#include "sched_plan.h"

namespace spm {

static constexpr int SCHED_TT = sched::kTT;
static constexpr int SCHED_THREADS = sched::kLanes;
static constexpr int SCHED_WARPS = sched::kWarps;
static constexpr int SCHED_PAD = sched::kPad;
static constexpr int SCHED_GROUP_COLS = 1008;  // columns per group: 16 lanes left for split parts
static constexpr int64_t SCHED_SEARCH = 300000;
// Without spm_sketch_set_plan(S, 1), a sketch is planned only by a product over
// at least this many elements of A (the plan costs ~0.1 s of host time).
static constexpr int64_t SCHED_AUTO_ELEMS = (int64_t)1 << 24;
static constexpr int SCHED_SMEM_LIMIT = 227 * 1024;

static_assert(SCHED_TT == 96, "the phase sequences below are written for 96 steps");

// One row of A (bytes, a multiple of 16) into shared memory; completion is
// counted on the barrier at `bar`.
__device__ __forceinline__ void sched_load_row(uint32_t dst, const float* src, uint32_t bytes,
                                               uint32_t bar) {
  mbar_expect(bar, bytes);
  bulk_g2s(dst, src, bytes, bar);
}


// Shared-memory load at a 32-bit shared address.  Not volatile, so the
// compiler may schedule the loads of a phase freely; the address it takes is
// laundered after the row's barrier wait (see the kernel), which keeps every
// load behind that wait.
__device__ __forceinline__ float sched_lds(uint32_t addr) {
  float v;
  asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
  return v;
}

// Shared address of the row element a register step names: the even step's
// offset sits in bits 0-14 of its register, the odd step's in bits 17-31 with
// bits 15-16 clear, so that (w >> 15) is already the odd step's byte offset.
// Volatile: the extractions stay inside the row loop (the offsets are
// loop-invariant, and hoisting all 96 of them would need 96 registers).
__device__ __forceinline__ uint32_t sched_even(uint32_t w, uint32_t rowa) {
  uint32_t a;
  asm volatile("{\n .reg .u32 t;\n and.b32 t, %1, 32767;\n mad.lo.u32 %0, t, 4, %2;\n}"
               : "=r"(a)
               : "r"(w), "r"(rowa));
  return a;
}
__device__ __forceinline__ uint32_t sched_odd(uint32_t w, uint32_t rowa) {
  uint32_t a;
  asm volatile("{\n .reg .u32 t;\n shr.u32 t, %1, 15;\n add.u32 %0, t, %2;\n}"
               : "=r"(a)
               : "r"(w), "r"(rowa));
  return a;
}
// Address of register step i (a compile-time index into R).
#define SCHED_A(i) (((i)&1) ? sched_odd(R[(i) >> 1], rowa) : sched_even(R[(i) >> 1], rowa))
#define SCHED_ADD(i, OP, ri)                           \
  {                                                    \
    const float v_ = sched_lds(SCHED_A(ri));           \
    a0 OP v_;                                          \
    if (FRO) f0 = fmaf(v_, v_, f0);                    \
  }

// Phase sequences.  The + phase runs register steps [e, TT) with e = TT - T+,
// the - phase runs "positions" [e, TT) with e = TT - T-, position i reading
// register step TT-1-i.  Entry: a jump to the 8-step block that holds e; that
// block's steps are predicated on (step >= e), every later block runs
// unguarded, so the code has a merge point only every 8 steps.
#define SCHED_PSTEP(i) SCHED_ADD(i, +=, (i))
#define SCHED_MSTEP(i) SCHED_ADD(i, -=, (SCHED_TT - 1 - (i)))
#define SCHED_G(ST, i) \
  if ((i) >= e) ST(i)
#define SCHED_GB(ST, b)                                                                      \
  SCHED_G(ST, 8 * (b)) SCHED_G(ST, 8 * (b) + 1) SCHED_G(ST, 8 * (b) + 2) SCHED_G(ST, 8 * (b) + 3) \
      SCHED_G(ST, 8 * (b) + 4) SCHED_G(ST, 8 * (b) + 5) SCHED_G(ST, 8 * (b) + 6)                \
          SCHED_G(ST, 8 * (b) + 7)
#define SCHED_UB(ST, b)                                                                   \
  ST(8 * (b)) ST(8 * (b) + 1) ST(8 * (b) + 2) ST(8 * (b) + 3) ST(8 * (b) + 4) ST(8 * (b) + 5) \
      ST(8 * (b) + 6) ST(8 * (b) + 7)
#define SCHED_PHASE(ST, L)                                                                  \
  switch (e >> 3) {                                                                        \
    case 0: SCHED_GB(ST, 0) goto L##1;                                                     \
    case 1: SCHED_GB(ST, 1) goto L##2;                                                     \
    case 2: SCHED_GB(ST, 2) goto L##3;                                                     \
    case 3: SCHED_GB(ST, 3) goto L##4;                                                     \
    case 4: SCHED_GB(ST, 4) goto L##5;                                                     \
    case 5: SCHED_GB(ST, 5) goto L##6;                                                     \
    case 6: SCHED_GB(ST, 6) goto L##7;                                                     \
    case 7: SCHED_GB(ST, 7) goto L##8;                                                     \
    case 8: SCHED_GB(ST, 8) goto L##9;                                                     \
    case 9: SCHED_GB(ST, 9) goto L##10;                                                    \
    case 10: SCHED_GB(ST, 10) goto L##11;                                                  \
    case 11: SCHED_GB(ST, 11) goto L##12;                                                  \
    default: goto L##12;                                                                   \
  }                                                                                        \
  L##1 : SCHED_UB(ST, 1) L##2 : SCHED_UB(ST, 2) L##3 : SCHED_UB(ST, 3) L##4 : SCHED_UB(ST, 4) \
  L##5 : SCHED_UB(ST, 5) L##6 : SCHED_UB(ST, 6) L##7 : SCHED_UB(ST, 7) L##8 : SCHED_UB(ST, 8) \
  L##9 : SCHED_UB(ST, 9) L##10 : SCHED_UB(ST, 10) L##11 : SCHED_UB(ST, 11) L##12 :;

template <typename TO>
__device__ __forceinline__ TO sched_out(float v);
template <>
__device__ __forceinline__ float sched_out<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 sched_out<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// Launch constants (read from the kernel's parameter space where they are used).
template <typename TO>
struct SchedArgs {
  const float* A;
  TO* out;
  TO* out_lo;
  const int2* wsteps;
  const int* slots;
  const int* partner;
  double* fro2;
  int* status;
  __nv_bfloat16* ahi;  // split of A (null: none), row stride lds
  __nv_bfloat16* alo;
  int64_t lds;
  int64_t lda, ldo;
  int m, n, G, P, cw, r1;
  float scale;
  double inv_s;
};

template <typename TO, bool FRO, int NSLOT, bool SPLIT>
__global__ void __launch_bounds__(SCHED_THREADS, 1)
    k_sketch_sched(const __grid_constant__ SchedArgs<TO> args, const uint32_t* __restrict__ words) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int n = args.n;
  const int slot_floats = (SCHED_PAD + n + 31) & ~31;  // 128-byte slots
  float* ring = reinterpret_cast<float*>(smem_raw);
  float* stage = ring + (size_t)NSLOT * slot_floats;  // 2 x SCHED_THREADS
  double* fro_part = reinterpret_cast<double*>(stage + 2 * SCHED_THREADS);  // SCHED_THREADS
  uint64_t* bars = reinterpret_cast<uint64_t*>(fro_part + SCHED_THREADS);
  const int tid = threadIdx.x;
  const int g = (int)(blockIdx.x % (unsigned)args.G);
  const int p0 = (int)(blockIdx.x / (unsigned)args.G);
  // this lane's offsets, its warp's phase entries and its staging slot: the
  // per-lane state kept in registers
  uint32_t R[SCHED_TT / 2];
  {
    const uint32_t* wp =
        words + ((size_t)(g * SCHED_WARPS + (tid >> 5)) * (SCHED_TT / 2)) * 32 + (tid & 31);
#pragma unroll
    for (int i = 0; i < SCHED_TT / 2; ++i) R[i] = __ldg(wp + (size_t)i * 32);
  }
  const int2 tpm = __ldg(args.wsteps + g * SCHED_WARPS + (tid >> 5));
  const uint32_t enter = (uint32_t)(SCHED_TT - tpm.x) | ((uint32_t)(SCHED_TT - tpm.y) << 8);
  const int sl = __ldg(args.slots + g * SCHED_THREADS + tid);
  for (int i = tid; i < NSLOT * SCHED_PAD; i += SCHED_THREADS)
    ring[(size_t)(i / SCHED_PAD) * slot_floats + (i % SCHED_PAD)] = 0.f;
  if (FRO) fro_part[tid] = 0.0;
  const uint32_t bar0 = smem_u32(bars), ring0 = smem_u32(ring);
  const uint32_t slot_bytes = (uint32_t)slot_floats * 4u;
  if (tid == 0) {
    for (int s = 0; s < NSLOT; ++s)
      mbar_init(bar0 + 8 * s, 1);
    mbar_init_fence();
    for (int s = 0; s < NSLOT; ++s) {
      const int row = p0 + s * args.P;
      if (row < args.m)
        sched_load_row(ring0 + s * slot_bytes + SCHED_PAD * 4, args.A + (int64_t)row * args.lda,
                       (uint32_t)n * 4u, bar0 + 8 * s);
    }
  }
  __syncthreads();
  int it = 0;
  bool timed_out = false;
  for (int row = p0; row < args.m; row += args.P, ++it) {
    const int s = it % NSLOT;
    const uint32_t par = (uint32_t)(it / NSLOT) & 1u;
    const bool to = !mbar_wait(bar0 + 8 * s, par);
    // the row's shared address, redefined after the wait: no load that uses it
    // can be scheduled before the copy has landed
    uint32_t rowa = ring0 + s * slot_bytes;
    asm volatile("" : "+r"(rowa)::"memory");
    float a0 = 0.f, f0 = 0.f;
    if (!to) {
      {
        const uint32_t e = enter & 0xFFu;
        SCHED_PHASE(SCHED_PSTEP, plus_)
      }
      {
        const uint32_t e = enter >> 8;
        SCHED_PHASE(SCHED_MSTEP, minus_)
      }
    }
    float* sg = stage + (it & 1) * SCHED_THREADS;
    if (sl >= 0) sg[sl & 0xFFFF] = (sl >> 16) ? -a0 : a0;
    if (FRO) fro_part[tid] += (double)f0;
    if (SPLIT && !to) {
      // this group's column range of the row, two elements per thread and pass
      const int q2 = ((n >> 1) + args.G - 1) / args.G;
      const int e2 = min((g + 1) * q2, n >> 1);
      const uint32_t rb = rowa + SCHED_PAD * 4;
#pragma unroll 1
      for (int c2 = g * q2 + tid; c2 < e2; c2 += SCHED_THREADS) {
        float vx, vy;
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(vx), "=f"(vy) : "r"(rb + 8u * (uint32_t)c2));
        const __nv_bfloat162 h = __floats2bfloat162_rn(vx, vy);
        const float2 f = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(vx - f.x, vy - f.y);
        const int64_t o = (int64_t)row * args.lds + 2 * c2;
        *reinterpret_cast<__nv_bfloat162*>(args.ahi + o) = h;
        *reinterpret_cast<__nv_bfloat162*>(args.alo + o) = l;
      }
    }
    // one barrier per row: the slot has been read by every warp, the staging
    // row is complete, and a timeout anywhere stops the whole CTA
    if (__syncthreads_or(to ? 1 : 0)) {
      timed_out = true;
      break;
    }
    if (tid == 0) {
      const int nr = row + NSLOT * args.P;
      if (nr < args.m) {
        proxy_async_fence();
        sched_load_row(ring0 + s * slot_bytes + SCHED_PAD * 4, args.A + (int64_t)nr * args.lda,
                       (uint32_t)n * 4u, bar0 + 8 * s);
      }
    }
    // write-out: thread t takes column t of the group (a group has at most
    // SCHED_THREADS columns), so consecutive threads store consecutive columns
    {
      const int cw = args.cw;
      const int c = g * cw + tid;
      if (tid < cw && c < args.r1) {
        float v = sg[tid];
        const int pt = __ldg(args.partner + g * cw + tid);
        if (pt >= 0) v += sg[pt];
        v *= args.scale;
        const TO h = sched_out<TO>(v);
        const int64_t o = (int64_t)row * args.ldo + c;
        args.out[o] = h;
        if (args.out_lo) args.out_lo[o] = sched_out<TO>(v - (float)h);
      }
    }
  }
  if (timed_out) {
    if (tid == 0) {
      set_status(args.status, DEV_TIMEOUT);
      // wait (bounded) for every copy this CTA still has in flight
      int64_t row = (int64_t)p0 + (int64_t)it * args.P;
      for (int k = 0; k < NSLOT; ++k, row += args.P) {
        if (row >= args.m) break;
        const int s = (it + k) % NSLOT;
        mbar_wait(bar0 + 8 * s, (uint32_t)((it + k) / NSLOT) & 1u);
      }
    }
    __syncthreads();
    return;
  }
  if (FRO) {
    double fro_acc = fro_part[tid];
    for (int o = 16; o > 0; o >>= 1) fro_acc += __shfl_xor_sync(0xFFFFFFFFu, fro_acc, o);
    __syncthreads();
    double* red = reinterpret_cast<double*>(stage);
    if ((tid & 31) == 0) red[tid >> 5] = fro_acc;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int w = 0; w < SCHED_WARPS; ++w) sum += red[w];
      atomicAdd(args.fro2, sum * args.inv_s);
    }
  }
}

#undef SCHED_A
#undef SCHED_ADD
#undef SCHED_PSTEP
#undef SCHED_MSTEP
#undef SCHED_G
#undef SCHED_GB
#undef SCHED_UB
#undef SCHED_PHASE

// ------------------------------------------------------------------ host side
static int sched_nslot(int64_t n) {
  const int64_t slot_bytes = ((SCHED_PAD + n + 31) & ~31ll) * 4;
  const int64_t fixed = 2 * SCHED_THREADS * 4 + SCHED_THREADS * 8 + 64;
  if (3 * slot_bytes + fixed <= SCHED_SMEM_LIMIT) return 3;
  if (2 * slot_bytes + fixed <= SCHED_SMEM_LIMIT) return 2;
  return 0;
}
static size_t sched_smem(int64_t n, int nslot) {
  return (size_t)(nslot * ((SCHED_PAD + n + 31) & ~31ll) * 4 + 2 * SCHED_THREADS * 4 +
                  SCHED_THREADS * 8 + 8 * nslot);
}

static int sched_plan_tables(int64_t n, int64_t r1, const std::vector<std::vector<uint32_t>>& cols,
                             int64_t search, int& G, int& cw, std::vector<uint32_t>& words,
                             std::vector<int32_t>& wsteps, std::vector<int32_t>& slots,
                             std::vector<int32_t>& partner, int64_t& steps) {
  G = (int)cdiv(r1, SCHED_GROUP_COLS);
  cw = (int)cdiv(r1, G);
  words.clear();
  wsteps.clear();
  slots.clear();
  partner.assign((size_t)G * cw, -1);
  steps = 0;
  for (int g = 0; g < G; ++g) {
    const int c0 = g * cw, c1 = (int)min64(r1, (int64_t)c0 + cw);
    std::vector<std::vector<uint32_t>> gc(cols.begin() + c0, cols.begin() + c1);
    sched::GroupPlan gp;
    if (!sched::plan_group(gc, search, gp)) return SPM_EUNSUPPORTED;
    words.insert(words.end(), gp.words.begin(), gp.words.end());
    wsteps.insert(wsteps.end(), gp.wsteps.begin(), gp.wsteps.end());
    slots.insert(slots.end(), gp.slot.begin(), gp.slot.end());
    for (int c = 0; c < c1 - c0; ++c) partner[(size_t)g * cw + c] = gp.partner[c];
    steps += gp.steps;
  }
  (void)n;
  return SPM_OK;
}

// Plans the sketch's scheduled product (once; not while st is being captured).
// States: 0 = plan at the first eligible product over SCHED_AUTO_ELEMS elements,
// 2 = plan at the first eligible product, 1 = ready, -1 = does not fit, -2 = off.
static bool sched_ready(spm_sketch* S, cudaStream_t st, int64_t elems) {
  if (S->kind != SPM_SKETCH_SPARSE_SIGN || !S->sched_mu) return false;
  if (S->sched_state == 0 && elems < SCHED_AUTO_ELEMS) return false;
  if (S->sched_state != 0 && S->sched_state != 2) return S->sched_state == 1;
  std::lock_guard<std::mutex> lock(*reinterpret_cast<std::mutex*>(S->sched_mu));
  if (S->sched_state != 0 && S->sched_state != 2) return S->sched_state == 1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return false;  // plan later, outside the capture
  const int64_t n = S->n, r1 = S->r1, nnz = S->n * S->s;
  if (sched_nslot(n) == 0 || n + SCHED_PAD > 0x7FFF) {
    S->sched_state = -1;
    return false;
  }
  // the column buckets on the host: chunked CSC -> one list per column
  const int64_t nch = cdiv(n, 512);
  std::vector<int64_t> cptr(nch * r1 + 1);
  std::vector<uint32_t> ent(nnz);
  cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
  cudaThreadExchangeStreamCaptureMode(&mode);
  bool ok = cudaMemcpyAsync(cptr.data(), S->bucket_ptr, cptr.size() * sizeof(int64_t),
                            cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaMemcpyAsync(ent.data(), S->bucket_ent, ent.size() * sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess;
  std::vector<std::vector<uint32_t>> cols(r1);
  if (ok)
    for (int64_t k = 0; k < nch; ++k)
      for (int64_t c = 0; c < r1; ++c)
        for (int64_t e = cptr[k * r1 + c]; e < cptr[k * r1 + c + 1]; ++e) cols[c].push_back(ent[e]);
  int G = 0, cw = 0;
  int64_t steps = 0;
  std::vector<uint32_t> words;
  std::vector<int32_t> wsteps, slots, partner;
  ok = ok && sched_plan_tables(n, r1, cols, SCHED_SEARCH, G, cw, words, wsteps, slots, partner,
                               steps) == SPM_OK;
  if (ok) {
    ok = cudaMallocAsync((void**)&S->sched_words, words.size() * 4, st) == cudaSuccess &&
         cudaMallocAsync((void**)&S->sched_wsteps, wsteps.size() * 4, st) == cudaSuccess &&
         cudaMallocAsync((void**)&S->sched_slot, slots.size() * 4, st) == cudaSuccess &&
         cudaMallocAsync((void**)&S->sched_partner, partner.size() * 4, st) == cudaSuccess &&
         cudaMemcpyAsync(S->sched_words, words.data(), words.size() * 4, cudaMemcpyHostToDevice,
                         st) == cudaSuccess &&
         cudaMemcpyAsync(S->sched_wsteps, wsteps.data(), wsteps.size() * 4,
                         cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(S->sched_slot, slots.data(), slots.size() * 4, cudaMemcpyHostToDevice,
                         st) == cudaSuccess &&
         cudaMemcpyAsync(S->sched_partner, partner.data(), partner.size() * 4,
                         cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaStreamSynchronize(st) == cudaSuccess;
  }
  cudaThreadExchangeStreamCaptureMode(&mode);
  if (ok) {
    S->sched_groups = G;
    S->sched_cw = cw;
    S->sched_steps = steps;
    S->sched_state = 1;
  } else {
    S->sched_state = -1;
  }
  return ok;
}

void sched_free(spm_sketch* S) {
  if (S->sched_words) cudaFreeAsync(S->sched_words, S->stream);
  if (S->sched_wsteps) cudaFreeAsync(S->sched_wsteps, S->stream);
  if (S->sched_slot) cudaFreeAsync(S->sched_slot, S->stream);
  if (S->sched_partner) cudaFreeAsync(S->sched_partner, S->stream);
  delete reinterpret_cast<std::mutex*>(S->sched_mu);
  S->sched_mu = nullptr;
}

void sched_init(spm_sketch* S) { S->sched_mu = new std::mutex(); }

static int sm_count_dev() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
    return 152;
  return v;
}

template <typename TO, bool FRO, int NSLOT, bool SPLIT>
static int sched_launch(const spm_sketch* S, const float* A, int64_t m, int64_t lda, TO* out,
                        TO* out_lo, int64_t ldo, double* fro2, int* status, cudaStream_t st,
                        __nv_bfloat16* ahi, __nv_bfloat16* alo, int64_t lds) {
  const int G = S->sched_groups;
  const int P = (int)max64(1, min64(m, sm_count_dev() / G));
  const size_t smem = sched_smem(S->n, NSLOT);
  SchedArgs<TO> a{};
  a.A = A;
  a.out = out;
  a.out_lo = out_lo;
  a.wsteps = S->sched_wsteps;
  a.slots = S->sched_slot;
  a.partner = S->sched_partner;
  a.fro2 = fro2;
  a.status = status;
  a.ahi = ahi;
  a.alo = alo;
  a.lds = lds;
  a.lda = lda;
  a.ldo = ldo;
  a.m = (int)m;
  a.n = (int)S->n;
  a.G = G;
  a.P = P;
  a.cw = S->sched_cw;
  a.r1 = (int)S->r1;
  a.scale = (float)(1.0 / sqrt((double)S->s));
  a.inv_s = 1.0 / (double)S->s;
  auto kern = k_sketch_sched<TO, FRO, NSLOT, SPLIT>;
  SPM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)(G * P), SCHED_THREADS, smem, st>>>(a, S->sched_words);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

int sched_apply(spm_sketch* S, const float* A, int64_t m, int64_t lda, void* out, int out_dt,
                int64_t ldo, double* fro2, int* status, cudaStream_t st, void* out_lo, void* a_hi,
                void* a_lo, int64_t lds) {
  if (S->kind != SPM_SKETCH_SPARSE_SIGN || m < 1 || m > 0x7FFFFFFF) return SPM_EUNSUPPORTED;
  if (a_hi && (!a_lo || lds < S->n || (lds & 3) != 0 || ((uintptr_t)a_hi & 7u) != 0 ||
               ((uintptr_t)a_lo & 7u) != 0))
    return SPM_EINVAL;
  if ((S->n & 3) != 0 || (lda & 3) != 0 || ((uintptr_t)A & 15u) != 0) return SPM_EUNSUPPORTED;
  if (out_dt != DT_F32 && out_dt != DT_BF16) return SPM_EUNSUPPORTED;
  const int nslot = sched_nslot(S->n);
  if (nslot == 0 || !sched_ready(S, st, m * S->n)) return SPM_EUNSUPPORTED;
  // the split of A is a separate instantiation (BF16 outputs only: the mixed
  // path), so the kernel without it keeps its registers for the offsets
#define SPM_SCHED_GO(TO, NS, SP)                                                                    \
  (fro2 ? sched_launch<TO, true, NS, SP>(S, A, m, lda, (TO*)out, (TO*)out_lo, ldo, fro2, status, st, \
                                         (__nv_bfloat16*)a_hi, (__nv_bfloat16*)a_lo, lds)               \
        : sched_launch<TO, false, NS, SP>(S, A, m, lda, (TO*)out, (TO*)out_lo, ldo, fro2, status, st, \
                                          (__nv_bfloat16*)a_hi, (__nv_bfloat16*)a_lo, lds))
  if (out_dt == DT_BF16 && a_hi)
    return nslot == 3 ? SPM_SCHED_GO(__nv_bfloat16, 3, true) : SPM_SCHED_GO(__nv_bfloat16, 2, true);
  if (a_hi) return SPM_EUNSUPPORTED;
  if (out_dt == DT_BF16)
    return nslot == 3 ? SPM_SCHED_GO(__nv_bfloat16, 3, false) : SPM_SCHED_GO(__nv_bfloat16, 2, false);
  return nslot == 3 ? SPM_SCHED_GO(float, 3, false) : SPM_SCHED_GO(float, 2, false);
#undef SPM_SCHED_GO
}

}  // namespace spm

using namespace spm;

extern "C" int spm_sketch_set_plan(spm_sketch* S, int32_t mode) {
  if (!S || mode < 0 || mode > 2) return SPM_EINVAL;
  if (S->kind != SPM_SKETCH_SPARSE_SIGN || !S->sched_mu) return mode ? SPM_EUNSUPPORTED : SPM_OK;
  std::lock_guard<std::mutex> lock(*reinterpret_cast<std::mutex*>(S->sched_mu));
  if (S->sched_state == 1 || S->sched_state == -1) return mode == 0 ? SPM_EINVAL : SPM_OK;
  S->sched_state = mode == 0 ? -2 : (mode == 1 ? 2 : 0);
  return SPM_OK;
}

extern "C" int spm_sketch_plan(const spm_sketch* S, int32_t* state, int64_t* steps_per_row,
                               int32_t* groups) {
  if (!S) return SPM_EINVAL;
  if (state) *state = S->sched_state == -2 ? -1 : (S->sched_state == 2 ? 0 : S->sched_state);
  if (steps_per_row) *steps_per_row = S->sched_state == 1 ? S->sched_steps : 0;
  if (groups) *groups = S->sched_state == 1 ? S->sched_groups : 0;
  return SPM_OK;
}

extern "C" int spm_sched_plan_host(int64_t n, int64_t r1, const int64_t* col_ptr,
                                   const uint32_t* col_ent, int64_t search, int32_t* groups,
                                   int64_t* steps_per_row, uint32_t* words, int32_t* wsteps,
                                   int32_t* slots, int32_t* partner) {
  if (n < 1 || r1 < 1 || !col_ptr || !col_ent || search < 0) return SPM_EINVAL;
  std::vector<std::vector<uint32_t>> cols(r1);
  for (int64_t c = 0; c < r1; ++c) {
    if (col_ptr[c + 1] < col_ptr[c]) return SPM_EINVAL;
    cols[c].assign(col_ent + col_ptr[c], col_ent + col_ptr[c + 1]);
  }
  int G = 0, cw = 0;
  int64_t steps = 0;
  std::vector<uint32_t> w;
  std::vector<int32_t> ws, sl, pt;
  const int rc = sched_plan_tables(n, r1, cols, search, G, cw, w, ws, sl, pt, steps);
  if (groups) *groups = rc == SPM_OK ? G : 0;
  if (steps_per_row) *steps_per_row = rc == SPM_OK ? steps : 0;
  if (rc != SPM_OK) return rc;
  if (words) std::copy(w.begin(), w.end(), words);
  if (wsteps) std::copy(ws.begin(), ws.end(), wsteps);
  if (slots) std::copy(sl.begin(), sl.end(), slots);
  if (partner) std::copy(pt.begin(), pt.end(), partner);
  return SPM_OK;
}
