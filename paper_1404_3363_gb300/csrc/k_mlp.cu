// Learned initial guess for the inverse geometry map (not in the paper): per
// block, a 3-64-64-3 perceptron with ReLU hidden layers maps a world point
// normalised to the block's control-point box, g_hat = (g - c) / h per axis, to a
// parameter-space guess p_hat.  It is trained on samples of the forward map
// the method itself evaluates (p uniform in [0,1]^3, g = phi(p)).
//
//   K7a mlp_samples  -- counter-based uniform p per (block, index), g = phi(p)
//   K7b mlp_fwd_bwd  -- forward, squared-error loss and backward for one
//                       mini-batch, one thread per sample; the weight
//                       gradients of a CTA's 128 samples are reduced in shared
//                       memory into one partial gradient per CTA (no atomics,
//                       so training is deterministic)
//   K7c mlp_adam     -- sums the partial gradients and applies Adam; also
//                       refreshes the FP16 copy used for inference
//   K6  mlp_infer    -- FP16 weights, FP32 accumulation on tensor cores
//                       (warp-level mma.sync m16n8k16): 16 points per warp
//                       tile; layer 1 (K = 3) on the FP32 pipe straight into the
//                       A fragments, layers 2 and 3 as MMAs whose accumulator
//                       fragments feed the next layer's A fragments directly.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "ivv_device.cuh"
#include "mlp.cuh"

namespace ivv {

namespace {

// ----------------------------------------------------------- sampling
__device__ __forceinline__ unsigned hash32(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

__device__ __forceinline__ float unit_float(unsigned long long seed, unsigned a, unsigned b, unsigned c) {
  unsigned h = hash32((unsigned)seed ^ hash32(a * 0x9e3779b9u ^ hash32(b + 0x632be5abu * c + (unsigned)(seed >> 32))));
  return ((h >> 8) + 0.5f) * (1.0f / 16777216.0f);
}

template <int P>
__global__ void k_mlp_samples(DevVolume V, MlpNorm norm, int block, int S, unsigned long long seed,
                              float4* __restrict__ x_out, float4* __restrict__ p_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S) return;
  float p[3] = {unit_float(seed, block, i, 0), unit_float(seed, block, i, 1), unit_float(seed, block, i, 2)};
  const BlockInfo B = V.blocks[block];
  float phi[3], J[3][3], rho;
  eval_block<P, float, false>(V, B, p, phi, J, rho);
  x_out[i] = make_float4((phi[0] - norm.c[0]) * norm.inv_h[0], (phi[1] - norm.c[1]) * norm.inv_h[1],
                         (phi[2] - norm.c[2]) * norm.inv_h[2], 0.f);
  p_out[i] = make_float4(p[0], p[1], p[2], 0.f);
}

// ----------------------------------------------------------- training
constexpr int kTrainThreads = 128;
constexpr int kLd = kMlpH + 1;          // padded row stride of activation tiles

struct TrainSmem {
  float w[kMlpParams];
  float h1[kTrainThreads][kLd];         // h1, later dh1
  float h2[kTrainThreads][kLd];
  float dh2[kTrainThreads][kLd];
  float x[kTrainThreads][3];
  float dy[kTrainThreads][3];
  float loss[kTrainThreads];
};

// Forward + backward of samples [first, first + n) (n <= 128 per CTA,
// CTA b takes samples first + 128 b ...); writes this CTA's gradient sum to
// partial[cta][kMlpParams] and its loss sum to partial_loss[cta].  scale is
// the 1/N of the mean over the whole batch.
__global__ void __launch_bounds__(kTrainThreads) k_mlp_fwd_bwd(const float* __restrict__ theta,
                                                               const float4* __restrict__ xs,
                                                               const float4* __restrict__ ps, int S, int first,
                                                               int n, float scale, float* __restrict__ partial,
                                                               float* __restrict__ partial_loss) {
  extern __shared__ float smem_raw[];
  TrainSmem& sm = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int tid = threadIdx.x;
  for (int i = tid; i < kMlpParams; i += kTrainThreads) sm.w[i] = theta[i];
  const int local = blockIdx.x * kTrainThreads + tid;
  const bool valid = local < n;
  const int idx = (first + local) % S;
  float x[3] = {0, 0, 0}, pt[3] = {0, 0, 0};
  if (valid) {
    const float4 a = xs[idx], b = ps[idx];
    x[0] = a.x; x[1] = a.y; x[2] = a.z;
    pt[0] = b.x; pt[1] = b.y; pt[2] = b.z;
  }
  __syncthreads();
  const float* W1 = sm.w + kOffW1;
  const float* b1 = sm.w + kOffB1;
  const float* W2 = sm.w + kOffW2;
  const float* b2 = sm.w + kOffB2;
  const float* W3 = sm.w + kOffW3;
  const float* b3 = sm.w + kOffB3;
  // forward
  for (int i = 0; i < kMlpH; ++i) {
    const float z = b1[i] + W1[3 * i] * x[0] + W1[3 * i + 1] * x[1] + W1[3 * i + 2] * x[2];
    sm.h1[tid][i] = z > 0.f ? z : 0.f;
  }
  for (int i = 0; i < kMlpH; ++i) {
    float z = b2[i];
#pragma unroll 16
    for (int k = 0; k < kMlpH; ++k) z += W2[i * kMlpH + k] * sm.h1[tid][k];
    sm.h2[tid][i] = z > 0.f ? z : 0.f;
  }
  float dy[3], l = 0.f;
  for (int c = 0; c < 3; ++c) {
    float z = b3[c];
#pragma unroll 16
    for (int k = 0; k < kMlpH; ++k) z += W3[c * kMlpH + k] * sm.h2[tid][k];
    const float e = valid ? z - pt[c] : 0.f;
    l += e * e;
    dy[c] = 2.f * e * scale;
  }
  // backward to the hidden layers (per sample)
  for (int i = 0; i < kMlpH; ++i) {
    const float g = W3[i] * dy[0] + W3[kMlpH + i] * dy[1] + W3[2 * kMlpH + i] * dy[2];
    sm.dh2[tid][i] = sm.h2[tid][i] > 0.f ? g : 0.f;
  }
  for (int c = 0; c < 3; ++c) {
    sm.x[tid][c] = x[c];
    sm.dy[tid][c] = dy[c];
  }
  sm.loss[tid] = valid ? l * scale : 0.f;
  // dh1 = W2^T dh2 (masked by h1 > 0); kept in registers until h1 is consumed
  float dh1[kMlpH];
#pragma unroll
  for (int k = 0; k < kMlpH; ++k) dh1[k] = 0.f;
  for (int i = 0; i < kMlpH; ++i) {
    const float g = sm.dh2[tid][i];
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) dh1[k] += W2[i * kMlpH + k] * g;
  }
  __syncthreads();
  // per-CTA weight gradients: each thread owns whole output entries
  float* out = partial + (size_t)blockIdx.x * kMlpParams;
  for (int e = tid; e < kMlpH * kMlpH; e += kTrainThreads) {           // dW2[i][k] = sum dh2_i h1_k
    const int i = e / kMlpH, k = e % kMlpH;
    float acc = 0.f;
    for (int s = 0; s < kTrainThreads; ++s) acc += sm.dh2[s][i] * sm.h1[s][k];
    out[kOffW2 + e] = acc;
  }
  for (int e = tid; e < 3 * kMlpH; e += kTrainThreads) {               // dW3[c][k] = sum dy_c h2_k
    const int c = e / kMlpH, k = e % kMlpH;
    float acc = 0.f;
    for (int s = 0; s < kTrainThreads; ++s) acc += sm.dy[s][c] * sm.h2[s][k];
    out[kOffW3 + e] = acc;
  }
  for (int i = tid; i < kMlpH; i += kTrainThreads) {                   // db2
    float acc = 0.f;
    for (int s = 0; s < kTrainThreads; ++s) acc += sm.dh2[s][i];
    out[kOffB2 + i] = acc;
  }
  if (tid < 3) {                                                       // db3
    float acc = 0.f;
    for (int s = 0; s < kTrainThreads; ++s) acc += sm.dy[s][tid];
    out[kOffB3 + tid] = acc;
  }
  if (tid == 0) {
    float acc = 0.f;
    for (int s = 0; s < kTrainThreads; ++s) acc += sm.loss[s];
    partial_loss[blockIdx.x] = acc;
  }
  __syncthreads();
  // dh1 replaces h1 (h1 > 0 mask first)
#pragma unroll
  for (int k = 0; k < kMlpH; ++k) {
    const float h = sm.h1[tid][k];
    sm.h1[tid][k] = h > 0.f ? dh1[k] : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < 3 * kMlpH; e += kTrainThreads) {               // dW1[i][c] = sum dh1_i x_c
    const int i = e / 3, c = e % 3;
    float acc = 0.f;
    for (int s = 0; s < kTrainThreads; ++s) acc += sm.h1[s][i] * sm.x[s][c];
    out[kOffW1 + e] = acc;
  }
  for (int i = tid; i < kMlpH; i += kTrainThreads) {                   // db1
    float acc = 0.f;
    for (int s = 0; s < kTrainThreads; ++s) acc += sm.h1[s][i];
    out[kOffB1 + i] = acc;
  }
}

// Sum of the per-CTA partial gradients (fixed order) -> grad, loss.
__global__ void k_mlp_reduce(const float* __restrict__ partial, const float* __restrict__ partial_loss, int nparts,
                             float* __restrict__ grad, float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kMlpParams) {
    float acc = 0.f;
    for (int c = 0; c < nparts; ++c) acc += partial[(size_t)c * kMlpParams + i];
    grad[i] = acc;
  }
  if (i == 0) {
    float acc = 0.f;
    for (int c = 0; c < nparts; ++c) acc += partial_loss[c];
    *loss = acc;
  }
}

// Adam (Kingma & Ba) on one block's parameters, then the FP16 inference copy.
__global__ void k_mlp_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ grad, float lr, float b1, float b2, float eps, float bc1,
                           float bc2, __half* __restrict__ theta16) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float t = theta[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  theta[i] = t;
  theta16[i] = __float2half_rn(t);
}

__global__ void k_mlp_to_half(const float* __restrict__ theta, __half* __restrict__ theta16, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) theta16[i] = __float2half_rn(theta[i]);
}

}  // namespace

void launch_mlp_samples(const DevVolume& V, const MlpNorm& norm, int block, int S, unsigned long long seed,
                        float4* x_out, float4* p_out, cudaStream_t s) {
  if (V.P == 2)
    k_mlp_samples<2><<<(S + 255) / 256, 256, 0, s>>>(V, norm, block, S, seed, x_out, p_out);
  else
    k_mlp_samples<3><<<(S + 255) / 256, 256, 0, s>>>(V, norm, block, S, seed, x_out, p_out);
}

size_t mlp_train_smem() { return sizeof(TrainSmem); }

cudaError_t launch_mlp_fwd_bwd(const float* theta, const float4* xs, const float4* ps, int S, int first, int n,
                               float scale, float* partial, float* partial_loss, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(TrainSmem));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int ctas = (n + kTrainThreads - 1) / kTrainThreads;
  k_mlp_fwd_bwd<<<ctas, kTrainThreads, sizeof(TrainSmem), s>>>(theta, xs, ps, S, first, n, scale, partial,
                                                              partial_loss);
  return cudaGetLastError();
}

int mlp_train_ctas(int n) { return (n + kTrainThreads - 1) / kTrainThreads; }

void launch_mlp_reduce(const float* partial, const float* partial_loss, int nparts, float* grad, float* loss,
                       cudaStream_t s) {
  k_mlp_reduce<<<(kMlpParams + 255) / 256, 256, 0, s>>>(partial, partial_loss, nparts, grad, loss);
}

void launch_mlp_adam(float* theta, float* m, float* v, const float* grad, float lr, int step, __half* theta16,
                     cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(theta, m, v, grad, lr, b1, b2, 1e-8f, bc1, bc2, theta16);
}

void launch_mlp_to_half(const float* theta, __half* theta16, int n, cudaStream_t s) {
  k_mlp_to_half<<<(n + 255) / 256, 256, 0, s>>>(theta, theta16, n);
}


}  // namespace ivv
