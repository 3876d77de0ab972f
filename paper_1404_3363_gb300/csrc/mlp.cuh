// Layout and launchers of the learned initial-guess network (k_mlp.cu).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "ivv_device.cuh"

namespace ivv {

constexpr int kMlpH = 64;
// flat parameter vector: W1 [64][3], b1 [64], W2 [64][64], b2 [64], W3 [3][64], b3 [3]
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpH * 3;
constexpr int kOffW2 = kOffB1 + kMlpH;
constexpr int kOffB2 = kOffW2 + kMlpH * kMlpH;
constexpr int kOffW3 = kOffB2 + kMlpH;
constexpr int kOffB3 = kOffW3 + 3 * kMlpH;
constexpr int kMlpParams = kOffB3 + 3;      // 4611
// per-block stride of the parameter arrays on the device: a multiple of 8 so
// every block's FP16 copy starts on a 16-byte boundary (the inference kernel
// reads weight pairs as 32-bit words)
constexpr int kMlpStride = (kMlpParams + 7) / 8 * 8;   // 4616
static_assert(kMlpStride % 8 == 0 && kOffW2 % 2 == 0 && kOffW3 % 2 == 0, "FP16 weight pairs must stay word aligned");

// Input normalisation of a block: g_hat_r = (g_r - c_r) * inv_h_r, mapping
// the block's control-point box to [-1, 1]^3.
struct MlpNorm {
  float c[3];
  float inv_h[3];
};

void launch_mlp_samples(const DevVolume& V, const MlpNorm& norm, int block, int S, unsigned long long seed,
                        float4* x_out, float4* p_out, cudaStream_t s);
size_t mlp_train_smem();
int mlp_train_ctas(int n);
cudaError_t launch_mlp_fwd_bwd(const float* theta, const float4* xs, const float4* ps, int S, int first, int n,
                               float scale, float* partial, float* partial_loss, cudaStream_t s);
void launch_mlp_reduce(const float* partial, const float* partial_loss, int nparts, float* grad, float* loss,
                       cudaStream_t s);
void launch_mlp_adam(float* theta, float* m, float* v, const float* grad, float lr, int step, __half* theta16,
                     cudaStream_t s);
void launch_mlp_to_half(const float* theta, __half* theta16, int n, cudaStream_t s);
// Tensor-core inference (k_mlp_tc.cu): p_out[i] = network of block gblk[i]
// at world point g[i], for i < *n_ptr (or n_static when n_ptr is null).
// perm (optional): the order in which the entries are taken (block after
// block, from launch_block_sort), so that a tile of 128 holds one block.
void launch_mlp_infer(const __half* theta16, const MlpNorm* norms, const float4* g, const int* gblk, const int* n_ptr,
                      int n_static, float4* p_out, DevStats* st, int num_sms, cudaStream_t s,
                      const int* perm = nullptr);
// Counting sort of the n = *n_ptr entries by block into perm [n]; hist:
// [n_blocks + 1] ints of scratch.
void launch_block_sort(const int* gblk, const int* n_ptr, int n_blocks, int* hist, int* perm, int num_sms,
                       cudaStream_t s);

}  // namespace ivv
