// The signed-distance surrogate network shared by the training (mlp.cu) and
// inference (mlp_infer.cu) kernels: parameter offsets, the device state
// layout and the activation.
//
// f(u) = w4 . s(W3 s(W2 s(W1 u + b1) + b2) + b3) + b4, s(z) = z sigmoid(z),
// hidden width 256.  Master parameters are float32; W2 and W3 also live as
// bfloat16 (and transposed, for the backward pass), the operands of the
// tcgen05 GEMMs.
#pragma once

#include <cuda_bf16.h>

#include "tc_gemm.cuh"

namespace vapr {

constexpr int MH = VAPR_MLP_HIDDEN;
constexpr int64_t MLP_P = VAPR_MLP_PARAMS;
constexpr int64_t OFF_W1 = 0, OFF_B1 = 3 * MH, OFF_W2 = OFF_B1 + MH, OFF_B2 = OFF_W2 + MH * MH,
                  OFF_W3 = OFF_B2 + MH, OFF_B3 = OFF_W3 + MH * MH, OFF_W4 = OFF_B3 + MH,
                  OFF_B4 = OFF_W4 + MH;
static_assert(OFF_B4 + 1 == MLP_P, "parameter layout");

typedef __nv_bfloat16 bf16;

__host__ __device__ constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device state: master parameters, Adam moments, Adam step, bf16 weights.
struct MlpState {
  float* p;
  float* m;
  float* v;
  int* step;
  bf16* W2;   // [256 out][256 in]
  bf16* W3;
  bf16* W2T;  // [256 in][256 out]
  bf16* W3T;
};

constexpr size_t MLP_PBYTES = align256(MLP_P * sizeof(float));
constexpr size_t MLP_WBYTES = (size_t)MH * MH * sizeof(bf16);
constexpr size_t MLP_STATE_BYTES = 3 * MLP_PBYTES + 256 + 4 * MLP_WBYTES;

__host__ __device__ inline MlpState mlp_state(void* base) {
  uint8_t* b = static_cast<uint8_t*>(base);
  MlpState s;
  s.p = reinterpret_cast<float*>(b);
  s.m = reinterpret_cast<float*>(b + MLP_PBYTES);
  s.v = reinterpret_cast<float*>(b + 2 * MLP_PBYTES);
  s.step = reinterpret_cast<int*>(b + 3 * MLP_PBYTES);
  uint8_t* w = b + 3 * MLP_PBYTES + 256;
  s.W2 = reinterpret_cast<bf16*>(w);
  s.W3 = reinterpret_cast<bf16*>(w + MLP_WBYTES);
  s.W2T = reinterpret_cast<bf16*>(w + 2 * MLP_WBYTES);
  s.W3T = reinterpret_cast<bf16*>(w + 3 * MLP_WBYTES);
  return s;
}

// sigmoid through the hardware tanh (PTX tanh.approx.f32, relative error
// about 2^-11, below the bfloat16 rounding that follows):
// sigmoid(z) = (1 + tanh(z / 2)) / 2.
__device__ __forceinline__ float tanh_hw(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sigmoid_hw(float z) { return fmaf(0.5f, tanh_hw(0.5f * z), 0.5f); }
__device__ __forceinline__ float silu(float z) { return z * sigmoid_hw(z); }
// d/dz z sigmoid(z) = sigmoid(z) (1 + z (1 - sigmoid(z)))
__device__ __forceinline__ float silu_grad(float z) {
  const float sg = sigmoid_hw(z);
  return sg * fmaf(z, 1.f - sg, 1.f);
}

// Two floats to a bf16x2 word, first in the low half (round to nearest even).
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

cudaError_t launch_mlp_refresh(const MlpState& s, bool bump_step, cudaStream_t st);

}  // namespace vapr
