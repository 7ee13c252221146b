// Shared host/device helpers of libspm: status plumbing, stream-ordered
// workspace, device status word, small math helpers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>

#include "../../include/spm.h"

namespace spm {

// Device-side error codes written into the status word (first error wins).
enum DevStatus : int {
  DEV_OK = 0,
  DEV_BREAKDOWN = SPM_EBREAKDOWN,
  DEV_NONFINITE = SPM_ENONFINITE,
  DEV_TIMEOUT = SPM_ETIMEOUT,
};

__device__ __forceinline__ void set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

#define SPM_CUDA_TRY(expr)                                                   \
  do {                                                                       \
    cudaError_t _e = (expr);                                                 \
    if (_e != cudaSuccess) {                                                 \
      if (_e == cudaErrorMemoryAllocation) return SPM_ENOMEM;                \
      return SPM_ECUDA;                                                      \
    }                                                                        \
  } while (0)

#define SPM_TRY(expr)               \
  do {                              \
    int _s = (expr);                \
    if (_s != SPM_OK) return _s;    \
  } while (0)

// Host-side count of kernel launches issued by the library (spm_launch_count).
extern std::atomic<unsigned long long> g_launches;
inline void count_launch(unsigned long long k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

#define SPM_LAUNCH_CHECK()          \
  do {                              \
    ::spm::count_launch();          \
    SPM_CUDA_TRY(cudaGetLastError()); \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

// Stream-ordered scratch arena: every buffer is cudaMallocAsync'ed on the
// call's stream and released by cudaFreeAsync when the arena dies.
// The library's stream-ordered memory pool on the current device: freed
// blocks stay reserved for the next call instead of being handed back to the
// device at every synchronisation (the default pool's behaviour), until
// spm_trim_memory.  Null if it cannot be created (allocations then fail).
cudaMemPool_t lib_pool();

struct Arena {
  cudaStream_t stream;
  void* ptrs[128];
  int count = 0;
  bool failed = false;
  explicit Arena(cudaStream_t s) : stream(s) {}
  ~Arena() {
    for (int i = count - 1; i >= 0; --i) cudaFreeAsync(ptrs[i], stream);
  }
  template <typename T>
  T* alloc(int64_t elems) {
    if (elems <= 0) elems = 1;
    if (count >= 128) { failed = true; return nullptr; }
    void* p = nullptr;
    // round to 256 B so that every TMA base is aligned
    size_t bytes = (size_t)round_up(elems * (int64_t)sizeof(T), 256);
    cudaMemPool_t pool = lib_pool();
    if (!pool || cudaMallocFromPoolAsync(&p, bytes, pool, stream) != cudaSuccess) {
      failed = true;
      return nullptr;
    }
    ptrs[count++] = p;
    return reinterpret_cast<T*>(p);
  }
};

#define SPM_ALLOC(arena, T, name, elems)          \
  T* name = (arena).template alloc<T>(elems);     \
  if (!name) return SPM_ENOMEM

// Event-based stage timer, used only when the caller asks for timing.
struct StageTimer {
  bool on = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev[2 * SPM_NSTAGES * 8];
  int stage_of[SPM_NSTAGES * 8];
  int n = 0;
  int cur = -1;
  void begin(int stage) {
    if (!on) return;
    if (cur >= 0) end();  // a nested stage closes the enclosing one
    if (n >= SPM_NSTAGES * 8) return;
    cudaEventCreate(&ev[2 * n]);
    cudaEventCreate(&ev[2 * n + 1]);
    cudaEventRecord(ev[2 * n], stream);
    stage_of[n] = stage;
    cur = n;
  }
  void end() {
    if (!on || cur < 0) return;
    cudaEventRecord(ev[2 * cur + 1], stream);
    ++n;
    cur = -1;
  }
  void collect(float* out) {
    if (!on) return;
    cudaStreamSynchronize(stream);
    for (int i = 0; i < n; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
      out[stage_of[i]] += ms;
      cudaEventDestroy(ev[2 * i]);
      cudaEventDestroy(ev[2 * i + 1]);
    }
    n = 0;
  }
  ~StageTimer() {
    for (int i = 0; i < n; ++i) {
      cudaEventDestroy(ev[2 * i]);
      cudaEventDestroy(ev[2 * i + 1]);
    }
  }
};

struct StageScope {
  StageTimer& t;
  StageScope(StageTimer& tt, int stage) : t(tt) { t.begin(stage); }
  ~StageScope() { t.end(); }
};

// Bounded grid-wide barrier for cooperative kernels.  The arrival counter only
// grows within a launch (it starts at 0): the k-th barrier is complete when it
// reaches nblocks (k + 1).  Thread 0 of each CTA adds 1 with release semantics
// (after the CTA barrier, so the CTA's writes are ordered before it) and polls
// the counter with acquire loads until it reaches the next multiple of
// nblocks above its own arrival; nobody resets or flips a second word, so the
// last arrival is seen after one trip through L2.  A CTA arriving at barrier
// k finds the counter in [nblocks k, nblocks (k + 1)), since barrier k cannot
// complete without it.  The wait is bounded (~2^32 clocks); on expiry it
// records DEV_TIMEOUT and the caller returns.
struct GridBar {
  unsigned* count;
  unsigned* gen;  // spare word (zeroed with the counter)
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool grid_sync(GridBar gb, unsigned nblocks, int* status) {
  __syncthreads();
  __shared__ int timed_out;
  if (threadIdx.x == 0) {
    timed_out = 0;
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;\n" : "=r"(old) : "l"(gb.count) : "memory");
    const unsigned target = (old / nblocks + 1u) * nblocks;
    if ((int)(ld_acquire_gpu(gb.count) - target) < 0) {
      const long long t0 = clock64();
      while ((int)(ld_acquire_gpu(gb.count) - target) < 0) {
        if (clock64() - t0 > (1ll << 32)) {
          set_status(status, DEV_TIMEOUT);
          timed_out = 1;
          break;
        }
      }
    }
  }
  __syncthreads();
  return timed_out == 0;
}

}  // namespace spm

// The sketch handle (opaque to C callers).
struct spm_sketch {
  int64_t n;
  int64_t r1;
  int32_t s;
  int32_t kind;
  uint64_t seed;
  cudaStream_t stream;
  int32_t* cols;          // n*s, draw order
  int8_t* signs;          // n*s
  int64_t* bucket_ptr;    // r1+1
  uint32_t* bucket_ent;   // n*s: row index j in bits 0..30, sign (1 = minus) in bit 31
  int2* seg;              // chunks x r1: [start, end) of each (chunk, column) segment,
                          // relative to the chunk's first entry
  uint32_t* entoff;       // n*s: (j mod 512) * 33 | sign bit -- shared-memory offset of the
                          // entry's column in the transposed A tile
  uint32_t* entacc;       // n*s (sparse sign, r1 <= 65535): tile offset (j mod 512) * 33 in
                          // bits 0..14, accumulator offset (c mod cg) * 33 in bits 15..30,
                          // sign in bit 31 (the shared-accumulator apply kernel); or null
  int32_t acc_cg;         // column-group size of entacc (at most SACC_MAX_CG)
  // dense families (Lemma 3.2 items 1 and 3); null for the sparse kinds
  __nv_bfloat16* dsign;   // dense sign: n x ld_dsign, +-1 (exact in BF16)
  int64_t ld_dsign;
  uint32_t* dbits;        // SRHT: D as bits (1 = minus), max(1, n'/32) words
  int32_t* hcols;         // SRHT: the r1 sampled Hadamard columns, in draw order
  int32_t hl;             // SRHT: log2 n'
  // Scheduled A S for FP32 rows held whole in shared memory (sketch_sched.cu),
  // planned on the host at the first eligible call: 0 = not planned yet,
  // 1 = ready, -1 = this sketch does not fit the kernel.
  int32_t sched_state;
  int32_t sched_groups;   // column groups G (CTAs per row)
  int32_t sched_cw;       // columns per group
  int64_t sched_steps;    // shared-memory gather steps per row, all groups together
  uint32_t* sched_words;  // G x 32 warps x (SCHED_TT / 2) words x 32 lanes: two 16-bit row offsets each
  int2* sched_wsteps;     // G x 32: steps of the + and the - phase of each warp
  int32_t* sched_slot;    // G x 1024: staging slot of each lane's column part (-1: idle)
  int32_t* sched_partner; // G x cw: staging slot of a column's second part (-1: none)
  void* sched_mu;         // std::mutex guarding the lazy planning
};
