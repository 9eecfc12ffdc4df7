// Training and batch-inference kernels of the controller network (phipm_mlp.cuh):
// per-CTA gradients, the fixed-order Adam step and a batched forward pass.  Only
// the C ABI's translation unit includes this file, so each kernel is defined once.
#pragma once
#include "phipm_mlp.cuh"

struct MlpSmem {
  float w[MLP_NP];
  float g[MLP_WARPS][MLP_NP];          // per-warp gradient accumulators (deterministic order)
  float act[MLP_WARPS][4][MLP_H];      // z1, h1, z2/dz2, h2 per warp
  float loss[MLP_WARPS];
};

// Per-CTA partial gradient (and loss) of mean((y - t)^2) over rows [0, n):
// warps take rows round-robin; each lane owns fixed parameters in its warp's
// accumulator; the 8 warp copies are summed in a fixed order.
__global__ void __launch_bounds__(MLP_WARPS * 32)
k_mlp_grad(const float* __restrict__ wg, const float* __restrict__ X, const float* __restrict__ T, long long n,
           float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char mlp_smem_raw[];
  MlpSmem& sm = *reinterpret_cast<MlpSmem*>(mlp_smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < MLP_NP; i += blockDim.x) sm.w[i] = wg[i];
  for (int i = threadIdx.x; i < MLP_WARPS * MLP_NP; i += blockDim.x) (&sm.g[0][0])[i] = 0.f;
  __syncthreads();
  const float* w = sm.w;
  float* g = sm.g[warp];
  float* z1 = sm.act[warp][0];
  float* h1 = sm.act[warp][1];
  float* dz2 = sm.act[warp][2];
  float* h2 = sm.act[warp][3];
  const float scale = 2.0f / (float)(n * MLP_OUT);
  float lsum = 0.f;
  const long long wid = (long long)blockIdx.x * MLP_WARPS + warp, nw = (long long)gridDim.x * MLP_WARPS;
  for (long long r = wid; r < n; r += nw) {
    float x[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) x[i] = X[r * MLP_IN + i];
    float zz[2], hh2[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int h = lane + 32 * q;
      float z = w[MLP_OFF_B1 + h];
#pragma unroll
      for (int i = 0; i < MLP_IN; ++i) z = fmaf(w[MLP_OFF_W1 + h * MLP_IN + i], x[i], z);
      z1[h] = z;
      h1[h] = mlp_gelu(z);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int h = lane + 32 * q;
      float z = w[MLP_OFF_B2 + h];
      for (int k = 0; k < MLP_H; ++k) z = fmaf(w[MLP_OFF_W2 + h * MLP_H + k], h1[k], z);
      zz[q] = z;
      hh2[q] = mlp_gelu(z);
      h2[h] = hh2[q];
    }
    __syncwarp();
    float dy[MLP_OUT];
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) {
      float a = w[MLP_OFF_W3 + o * MLP_H + lane] * hh2[0] + w[MLP_OFF_W3 + o * MLP_H + lane + 32] * hh2[1];
#pragma unroll
      for (int off = 16; off; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
      const float res = a + w[MLP_OFF_B3 + o] - T[r * MLP_OUT + o];
      lsum += res * res;
      dy[o] = scale * res;
    }
    // output layer
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int k = lane + 32 * q;
      g[MLP_OFF_W3 + k] += dy[0] * hh2[q];
      g[MLP_OFF_W3 + MLP_H + k] += dy[1] * hh2[q];
      const float dh2 = w[MLP_OFF_W3 + k] * dy[0] + w[MLP_OFF_W3 + MLP_H + k] * dy[1];
      dz2[k] = dh2 * mlp_gelu_grad(zz[q]);
    }
    if (lane == 0) { g[MLP_OFF_B3] += dy[0]; g[MLP_OFF_B3 + 1] += dy[1]; }
    __syncwarp();
    // second hidden layer: lane owns rows h = lane, lane + 32 of W2
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int h = lane + 32 * q;
      const float d = dz2[h];
      for (int k = 0; k < MLP_H; ++k) g[MLP_OFF_W2 + h * MLP_H + k] += d * h1[k];
      g[MLP_OFF_B2 + h] += d;
    }
    // first hidden layer: dh1[k] = sum_h W2[h][k] dz2[h]
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int k = lane + 32 * q;
      float dh1 = 0.f;
      for (int h = 0; h < MLP_H; ++h) dh1 = fmaf(w[MLP_OFF_W2 + h * MLP_H + k], dz2[h], dh1);
      const float dz1 = dh1 * mlp_gelu_grad(z1[k]);
#pragma unroll
      for (int i = 0; i < MLP_IN; ++i) g[MLP_OFF_W1 + k * MLP_IN + i] += dz1 * x[i];
      g[MLP_OFF_B1 + k] += dz1;
    }
    __syncwarp();
  }
  if (lane == 0) sm.loss[warp] = lsum;
  __syncthreads();
  float* out = part + (size_t)blockIdx.x * MLP_PART;
  for (int i = threadIdx.x; i < MLP_NP; i += blockDim.x) {
    float a = 0.f;
    for (int q = 0; q < MLP_WARPS; ++q) a += sm.g[q][i];
    out[i] = a;
  }
  if (threadIdx.x == 0) {
    float a = 0.f;
    for (int q = 0; q < MLP_WARPS; ++q) a += sm.loss[q];
    out[MLP_NP] = a / (float)(n * MLP_OUT);
  }
}

// Sum the per-CTA partials in a fixed order; optionally write the gradient and
// the loss, and apply one Adam step (t counts from 1) when lr > 0.
__global__ void k_mlp_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ part, int G, float* __restrict__ grad_out,
                           float* __restrict__ loss_out, long long t, float lr, float beta1, float beta2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > MLP_NP) return;
  float a = 0.f;
  for (int q = 0; q < G; ++q) a += part[(size_t)q * MLP_PART + i];
  if (i == MLP_NP) {
    if (loss_out) *loss_out = a;
    return;
  }
  if (grad_out) grad_out[i] = a;
  if (lr > 0.f) {
    const float mi = beta1 * m[i] + (1.f - beta1) * a;
    const float vi = beta2 * v[i] + (1.f - beta2) * a * a;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(beta1, (float)t));
    const float vh = vi / (1.f - powf(beta2, (float)t));
    w[i] -= lr * mh / (sqrtf(vh) + eps);
  }
}

// Y = f(X) for n rows, one warp per row.
__global__ void __launch_bounds__(256) k_mlp_forward(const float* __restrict__ w, const float* __restrict__ X, long long n,
                                                     float* __restrict__ Y) {
  __shared__ float hs[8][2][MLP_H];
  const int warp = threadIdx.x >> 5;
  const long long wid = (long long)blockIdx.x * 8 + warp, nw = (long long)gridDim.x * 8;
  for (long long r = wid; r < n; r += nw) {
    float x[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) x[i] = X[r * MLP_IN + i];
    float y[2];
    mlp_warp_forward(w, x, hs[warp][0], hs[warp][1], y);
    if ((threadIdx.x & 31) == 0) { Y[r * 2] = y[0]; Y[r * 2 + 1] = y[1]; }
  }
}
