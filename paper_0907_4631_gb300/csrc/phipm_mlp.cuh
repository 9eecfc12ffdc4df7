// The learned (tau, m) controller network: 8 inputs, two hidden layers of 64
// GELU units, 2 outputs, FP32.  Inference runs on one warp inside the solver;
// training (mean squared error, Adam) runs in the kernels of phipm_mlp_train.cuh.
//
// Parameter layout (4866 floats): W1 [64 x 8] row-major at 0, b1 [64] at 512,
// W2 [64 x 64] at 576, b2 [64] at 4672, W3 [2 x 64] at 4736, b3 [2] at 4864.
// A controller blob appends x_mean[8], x_std[8], y_mean[2], y_std[2]
// (inputs are normalised, outputs de-normalised).
#pragma once
#include <cuda_runtime.h>

#define MLP_IN 8
#define MLP_H 64
#define MLP_OUT 2
#define MLP_OFF_W1 0
#define MLP_OFF_B1 512
#define MLP_OFF_W2 576
#define MLP_OFF_B2 4672
#define MLP_OFF_W3 4736
#define MLP_OFF_B3 4864
#define MLP_NP 4866
#define MLP_BLOB (MLP_NP + 20)
#define MLP_WARPS 8                     // warps per training CTA
#define MLP_PART (MLP_NP + 1)           // per-CTA partial: gradient + loss

__device__ __forceinline__ float mlp_gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float mlp_gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// One warp evaluates the network on x (8 values, identical in every lane).
// h1 / h2 are per-warp scratch of 64 floats (shared memory).  Returns y in every lane.
__device__ __forceinline__ void mlp_warp_forward(const float* __restrict__ w, const float* x, float* h1, float* h2,
                                                 float y[2]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int h = lane + 32 * q;
    float z = w[MLP_OFF_B1 + h];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) z = fmaf(w[MLP_OFF_W1 + h * MLP_IN + i], x[i], z);
    h1[h] = mlp_gelu(z);
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int h = lane + 32 * q;
    float z = w[MLP_OFF_B2 + h];
    for (int k = 0; k < MLP_H; ++k) z = fmaf(w[MLP_OFF_W2 + h * MLP_H + k], h1[k], z);
    h2[h] = mlp_gelu(z);
  }
  __syncwarp();
#pragma unroll
  for (int o = 0; o < MLP_OUT; ++o) {
    float a = w[MLP_OFF_W3 + o * MLP_H + lane] * h2[lane] + w[MLP_OFF_W3 + o * MLP_H + lane + 32] * h2[lane + 32];
#pragma unroll
    for (int off = 16; off; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    y[o] = a + w[MLP_OFF_B3 + o];
  }
  __syncwarp();
}

