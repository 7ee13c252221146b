// Batched Randomized SVD over many matrices of uneven shapes and ranks.
//
// Each problem runs the stream-ordered RandSVD pipeline (Algorithm 1 followed
// by the SVD of B = Q^T A) with no host synchronisation.  The problems are
// spread round-robin over a fixed pool of side streams that fork from and join
// back into the caller's stream through events, so independent problems fill
// the GPU concurrently, and the whole call can be captured into one CUDA graph
// (cudaStreamBeginCapture on the caller's stream) and replayed as one launch.
// Problems with the same (n, r1, s, seed) share one set of sketch tables.
//
// Problems are issued largest first (by m n r1), so the long ones start early
// and the short ones fill in behind them.
#include <algorithm>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.cuh"

namespace spm {

int rsvd_async(const spm_sketch* S, const void* A, int32_t dtype, int64_t m, int64_t lda, int64_t r2,
               int32_t q, uint64_t omega_seed, int64_t k, const spm_opts* opts, void* U, int64_t ldu,
               void* sigma, void* Vt, int64_t ldvt, int32_t* dev_status, cudaStream_t st);

static constexpr int kMaxSide = 32;

// Side streams and fork/join events, created once per device and kept for the
// life of the process (a capture may not destroy streams it forked into).
struct SidePool {
  int dev = -1;
  cudaStream_t s[kMaxSide] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kMaxSide] = {};
};

static std::mutex g_pool_mu;
static SidePool g_pools[16];

static SidePool* side_pool(int dev) {
  if (dev < 0 || dev >= 16) return nullptr;
  SidePool& p = g_pools[dev];
  if (p.dev == dev) return &p;
  for (int i = 0; i < kMaxSide; ++i) {
    if (cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming) != cudaSuccess) return nullptr;
  }
  if (cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  p.dev = dev;
  return &p;
}

// Fork `ns` side streams from st, run body(i, stream) for i in `order` round
// robin over them, and join them back into st (also after an error).
int on_side_streams(int count, const int* order, int ns, cudaStream_t st,
                    const std::function<int(int, cudaStream_t)>& body) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  int dev = 0;
  SPM_CUDA_TRY(cudaGetDevice(&dev));
  SidePool* pool = side_pool(dev);
  if (!pool) return SPM_ECUDA;
  SPM_CUDA_TRY(cudaEventRecord(pool->fork, st));
  int rc = SPM_OK;
  int forked = 0;
  for (; forked < ns && rc == SPM_OK; ++forked)
    if (cudaStreamWaitEvent(pool->s[forked], pool->fork, 0) != cudaSuccess) rc = SPM_ECUDA;
  for (int o = 0; o < count && rc == SPM_OK; ++o) rc = body(order ? order[o] : o, pool->s[o % ns]);
  for (int j = 0; j < forked; ++j) {
    const bool ok = cudaEventRecord(pool->join[j], pool->s[j]) == cudaSuccess &&
                    cudaStreamWaitEvent(st, pool->join[j], 0) == cudaSuccess;
    if (!ok && rc == SPM_OK) rc = SPM_ECUDA;
  }
  return rc;
}

}  // namespace spm

using namespace spm;

extern "C" int spm_rsvd_batched(int32_t count, const spm_batch_item* items, int32_t dtype,
                                const spm_opts* opts, int32_t nstreams, int32_t* dev_status,
                                void* stream) {
  if (count < 0 || (count > 0 && !items) || nstreams < 0 || nstreams > kMaxSide) return SPM_EINVAL;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_EINVAL;
  for (int i = 0; i < count; ++i) {
    const spm_batch_item& it = items[i];
    if (!it.A || !it.U || !it.sigma || !it.Vt || it.m < 1 || it.n < 1 || it.lda < it.n ||
        it.k < 1 || it.k > it.m || it.k > it.n || it.r1 < it.k || it.r1 > it.n || it.s < 1 ||
        it.s > it.r1 || it.q < 0 || it.ldu < it.k || it.ldvt < it.n)
      return SPM_EINVAL;
  }
  if (count == 0) return SPM_OK;
  cudaStream_t st = as_stream(stream);
  const int ns = nstreams == 0 ? 16 : nstreams;
  // sketch tables, on the caller's stream before the fork
  std::map<std::tuple<int64_t, int64_t, int32_t, uint64_t>, spm_sketch*> sketches;
  std::vector<spm_sketch*> of(count, nullptr);
  int rc = SPM_OK;
  for (int i = 0; i < count && rc == SPM_OK; ++i) {
    const spm_batch_item& it = items[i];
    const auto key = std::make_tuple(it.n, it.r1, it.s, it.seed);
    auto f = sketches.find(key);
    if (f == sketches.end()) {
      spm_sketch* S = nullptr;
      rc = spm_sketch_create(&S, it.n, it.r1, it.s, it.seed, SPM_SKETCH_SPARSE_SIGN, st);
      // no plan (it would synchronise a stream): the batch runs the general
      // sketch kernels, the same whether it is captured or not
      if (rc == SPM_OK) rc = spm_sketch_set_plan(S, 0);
      if (rc == SPM_OK) sketches[key] = of[i] = S;
    } else {
      of[i] = f->second;
    }
  }
  if (dev_status && rc == SPM_OK &&
      cudaMemsetAsync(dev_status, 0, (size_t)count * sizeof(int32_t), st) != cudaSuccess)
    rc = SPM_ECUDA;

  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  auto work = [&](int i) { return (double)items[i].m * (double)items[i].n * (double)items[i].r1; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
  if (rc == SPM_OK)
    rc = on_side_streams(count, order.data(), ns, st, [&](int i, cudaStream_t s) {
      const spm_batch_item& it = items[i];
      return rsvd_async(of[i], it.A, dtype, it.m, it.lda, it.k, it.q, it.seed + 1, it.k, opts, it.U,
                        it.ldu, it.sigma, it.Vt, it.ldvt, dev_status ? dev_status + i : nullptr, s);
    });
  for (auto& kv : sketches) spm_sketch_destroy(kv.second);
  return rc;
}
