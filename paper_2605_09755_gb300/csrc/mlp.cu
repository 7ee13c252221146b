// The learned (q, sketch size) selector: a multilayer perceptron with three
// hidden layers of 64 ReLU units, trained and evaluated by these kernels.
//
// Parameters are one packed FP32 vector, layer by layer: W_l (out x in,
// row-major) followed by b_l; layer sizes 8 -> 64 -> 64 -> 64 -> 15.  The
// network reads features of the q = 0 sketch (see spm_selector_features) and
// predicts log10(residual / optimal - 1) for 15 candidates (q in 0..4) x (sketch
// size r1 in {2, 4, 8} x r2).
//
// One warp evaluates one sample: lane u computes hidden units u and u + 32;
// the CTA keeps the weights transposed in shared memory ([in][out]) so that a
// warp reads one input column with consecutive lanes.  The backward pass
// accumulates the CTA's gradients in shared memory and adds them to global
// memory once per CTA.
#include "internal.cuh"

namespace spm {

static constexpr int MLP_IN = SPM_MLP_IN, MLP_H = 64, MLP_OUT = SPM_MLP_OUT;
static constexpr int MLP_THREADS = 256, MLP_WARPS = MLP_THREADS / 32;
__host__ __device__ __forceinline__ constexpr int l_in(int l) { return l == 0 ? MLP_IN : MLP_H; }
__host__ __device__ __forceinline__ constexpr int l_out(int l) { return l == 3 ? MLP_OUT : MLP_H; }
// packed offsets: 0, 64*8+64, +64*64+64, +64*64+64; total + 15*64+15
__host__ __device__ __forceinline__ constexpr int layer_off(int l) {
  return l == 0 ? 0 : (l == 1 ? 576 : (l == 2 ? 4736 : 8896));
}
static_assert(8896 + MLP_OUT * MLP_H + MLP_OUT == SPM_MLP_PARAMS, "packed size");

// load all parameters into shared memory, weights transposed to [in][out]
__device__ void load_params_t(const float* __restrict__ p, float* sp) {
  for (int l = 0; l < 4; ++l) {
    const int in = l_in(l), out = l_out(l), off = layer_off(l);
    for (int e = threadIdx.x; e < in * out; e += blockDim.x) {
      const int o = e / in, i = e % in;
      sp[off + i * out + o] = p[off + e];
    }
    for (int e = threadIdx.x; e < out; e += blockDim.x) sp[off + in * out + e] = p[off + in * out + e];
  }
}

// forward of one sample by one warp; acts: [x (8) | h1 (64) | h2 (64) | h3 (64) | y (15)]
__device__ __forceinline__ void warp_forward(const float* sp, float* acts) {
  const int lane = threadIdx.x & 31;
  const float* h_in = acts;
  float* h_out = acts + MLP_IN;
  for (int l = 0; l < 4; ++l) {
    const int in = l_in(l), out = l_out(l), off = layer_off(l);
    const float* WT = sp + off;
    const float* b = sp + off + in * out;
    for (int u = lane; u < out; u += 32) {
      float z = b[u];
      for (int i = 0; i < in; ++i) z = fmaf(WT[i * out + u], h_in[i], z);
      h_out[u] = (l < 3) ? fmaxf(z, 0.f) : z;
    }
    __syncwarp();
    h_in = h_out;
    h_out += out;
  }
}

__global__ void __launch_bounds__(MLP_THREADS)
    k_mlp_forward(const float* __restrict__ params, const float* __restrict__ X, int64_t batch,
                  float* __restrict__ Y) {
  extern __shared__ float msm[];
  float* sp = msm;
  float* acts = msm + SPM_MLP_PARAMS + (threadIdx.x >> 5) * 256;
  load_params_t(params, sp);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int64_t s = (int64_t)blockIdx.x * MLP_WARPS + (threadIdx.x >> 5); s < batch;
       s += (int64_t)gridDim.x * MLP_WARPS) {
    if (lane < MLP_IN) acts[lane] = X[s * MLP_IN + lane];
    __syncwarp();
    warp_forward(sp, acts);
    const float* y = acts + MLP_IN + 3 * MLP_H;
    if (lane < MLP_OUT) Y[s * MLP_OUT + lane] = y[lane];
    __syncwarp();
  }
}

__global__ void k_mask_count(int64_t n, const float* __restrict__ M, float* __restrict__ cnt) {
  float s = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    s += M[e];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(cnt, s);
}

// Masked MSE loss and its gradient: grad += dL/dp, loss += L (both pre-zeroed).
__global__ void __launch_bounds__(MLP_THREADS)
    k_mlp_grad(const float* __restrict__ params, const float* __restrict__ X,
               const float* __restrict__ T, const float* __restrict__ M, int64_t batch,
               const float* __restrict__ cnt_p, float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ float msm[];
  float* sp = msm;                                  // transposed params
  float* sg = msm + SPM_MLP_PARAMS;                 // gradient accumulator (packed layout)
  float* acts = sg + SPM_MLP_PARAMS + (threadIdx.x >> 5) * 512;
  float* dl = acts + 256;                           // deltas of the current layer
  load_params_t(params, sp);
  for (int e = threadIdx.x; e < SPM_MLP_PARAMS; e += blockDim.x) sg[e] = 0.f;
  __syncthreads();
  const float cnt = fmaxf(*cnt_p, 1.f);
  const int lane = threadIdx.x & 31;
  float lsum = 0.f;
  for (int64_t s = (int64_t)blockIdx.x * MLP_WARPS + (threadIdx.x >> 5); s < batch;
       s += (int64_t)gridDim.x * MLP_WARPS) {
    if (lane < MLP_IN) acts[lane] = X[s * MLP_IN + lane];
    __syncwarp();
    warp_forward(sp, acts);
    // output delta
    const float* y = acts + MLP_IN + 3 * MLP_H;
    if (lane < MLP_OUT) {
      const float r = y[lane] - T[s * MLP_OUT + lane];
      const float mk = M[s * MLP_OUT + lane];
      lsum += mk * r * r;
      dl[lane] = 2.f * mk * r / cnt;
    }
    __syncwarp();
    for (int l = 3; l >= 0; --l) {
      const int in = l_in(l), out = l_out(l), off = layer_off(l);
      const float* h_in = acts + (l == 0 ? 0 : MLP_IN + (l - 1) * MLP_H);
      // dW[o][i] += d[o] h_in[i]; db[o] += d[o]   (packed, untransposed layout)
      for (int e = lane; e < in * out; e += 32) {
        const int o = e / in, i = e % in;
        atomicAdd(&sg[off + e], dl[o] * h_in[i]);
      }
      for (int o = lane; o < out; o += 32) atomicAdd(&sg[off + in * out + o], dl[o]);
      __syncwarp();
      if (l > 0) {
        // d_in[i] = (sum_o W[o][i] d[o]) * [h_in[i] > 0]
        const float* WT = sp + off;
        float nd[2];
        for (int q = 0; q < 2; ++q) {
          const int i = lane + 32 * q;
          float acc = 0.f;
          if (i < in)
            for (int o = 0; o < out; ++o) acc = fmaf(WT[i * out + o], dl[o], acc);
          nd[q] = (i < in && h_in[i] > 0.f) ? acc : 0.f;
        }
        __syncwarp();
        for (int q = 0; q < 2; ++q)
          if (lane + 32 * q < in) dl[lane + 32 * q] = nd[q];
        __syncwarp();
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < SPM_MLP_PARAMS; e += blockDim.x)
    if (sg[e] != 0.f) atomicAdd(&grad[e], sg[e]);
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xFFFFFFFFu, lsum, o);
  if (lane == 0) atomicAdd(loss, lsum / cnt);
}

__global__ void k_adam(int n, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
}

int mlp_forward_dev(const float* params, const float* X, int64_t batch, float* Y, cudaStream_t st) {
  if (batch <= 0) return SPM_OK;
  const int smem = (SPM_MLP_PARAMS + MLP_WARPS * 256) * 4;
  SPM_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int blocks = (int)min64(cdiv(batch, MLP_WARPS), 152 * 2);
  k_mlp_forward<<<blocks, MLP_THREADS, smem, st>>>(params, X, batch, Y);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

}  // namespace spm

using namespace spm;

extern "C" {

int spm_mlp_forward(const float* params, const float* X, int64_t batch, float* Y, void* stream) {
  if (!params || !X || !Y || batch < 0) return SPM_EINVAL;
  return mlp_forward_dev(params, X, batch, Y, as_stream(stream));
}

int spm_mlp_loss_grad(const float* params, const float* X, const float* T, const float* M,
                      int64_t batch, float* grad, float* loss, void* stream) {
  if (!params || !X || !T || !M || !grad || !loss || batch < 1) return SPM_EINVAL;
  cudaStream_t st = as_stream(stream);
  Arena ar(st);
  SPM_ALLOC(ar, float, cnt, 1);
  SPM_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(float), st));
  SPM_CUDA_TRY(cudaMemsetAsync(grad, 0, SPM_MLP_PARAMS * sizeof(float), st));
  SPM_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
  k_mask_count<<<(unsigned)min64(cdiv(batch * MLP_OUT, 256), 1024), 256, 0, st>>>(batch * MLP_OUT, M, cnt);
  SPM_LAUNCH_CHECK();
  const int smem = (2 * SPM_MLP_PARAMS + MLP_WARPS * 512) * 4;
  SPM_CUDA_TRY(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int blocks = (int)min64(cdiv(batch, MLP_WARPS), 152);
  k_mlp_grad<<<blocks, MLP_THREADS, smem, st>>>(params, X, T, M, batch, cnt, grad, loss);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

int spm_mlp_adam(float* params, float* m, float* v, const float* grad, int32_t step, float lr,
                 float b1, float b2, float eps, void* stream) {
  if (!params || !m || !v || !grad || step < 1) return SPM_EINVAL;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<(SPM_MLP_PARAMS + 255) / 256, 256, 0, as_stream(stream)>>>(SPM_MLP_PARAMS, params, m, v,
                                                                      grad, lr, b1, b2, eps, c1, c2);
  SPM_LAUNCH_CHECK();
  return SPM_OK;
}

}  // extern "C"
