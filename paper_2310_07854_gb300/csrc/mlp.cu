// Training of the signed-distance surrogate (mlp.cuh): one batch's loss and
// gradient, the Adam step, and the bfloat16 weight copies.
//
// A batch of Nb samples (Nb a multiple of 128) goes through
//   l1        u -> Z1 = W1 u + b1 (float32), A1 = s(Z1) (bf16, also transposed)
//   GEMM      A1 W2^T, epilogue + b2 -> Z2, A2 = s(Z2) (bf16, also transposed)
//   GEMM      A2 W3^T, head epilogue: + b3, A3 = s(Z3), f = w4 . A3 + b4,
//             r = f - y, dL/df = 2 w r / Nb (w = over_weight if r > 0,
//             else 1), then a second pass over the
//             accumulator: dZ3 = dL/df w4 s'(Z3)
//   GEMM      dZ3^T A2 (split over the batch)          -> dL/dW3
//   GEMM      dZ3 W3, epilogue x s'(Z2)                -> dZ2
//   GEMM      dZ2^T A1 (split over the batch)          -> dL/dW2
//   GEMM      dZ2 W2, epilogue x s'(Z1)                -> dZ1 (float32, transposed)
//   sums      dL/dW1, db1, db2, db3, dw4, db4 and the loss (fixed-order trees)
// The GEMMs are the tcgen05 kernel of tc_gemm.cuh with the epilogues below;
// every operand is K-major, which is why the epilogues also write the
// transposed (batch-contiguous) copies that the weight-gradient GEMMs read.
#include "mlp.cuh"

namespace vapr {

constexpr int MAX_MLP_BATCH = 1 << 20;

// ---- workspace of one batch
struct MlpWork {
  float* Z1;    // [Nb][256]
  bf16* A1;     // [Nb][256]
  bf16* A1T;    // [256][Nb]
  float* Z2;    // [Nb][256]
  bf16* A2;
  bf16* A2T;
  float* A3T;   // [256][Nb]
  float* dF;    // [Nb]
  float* rsq;   // [Nb] weighted squared residuals
  bf16* dZ3;    // [Nb][256]
  bf16* dZ3T;   // [256][Nb]
  bf16* dZ2;
  bf16* dZ2T;
  float* dZ1T;  // [256][Nb]
  float* slab;  // [splits][256][256]
  float* grads; // [MLP_P]
  int splits, k_split;
  size_t bytes;
};

// Split of the batch for the weight-gradient GEMMs: about 64 slabs of whole
// 64-sample slices, so that 2 x 64 CTAs share the GPU.
static void weight_split(int64_t Nb, int& splits, int& k_split) {
  const int64_t slices = Nb / TG_K;
  const int64_t per = (slices + 63) / 64;
  k_split = (int)(per * TG_K);
  splits = (int)((Nb + k_split - 1) / k_split);
}

static MlpWork carve_work(void* base, int64_t Nb) {
  MlpWork w;
  weight_split(Nb, w.splits, w.k_split);
  uint8_t* b = static_cast<uint8_t*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    uint8_t* p = b ? b + off : nullptr;
    off += align256(bytes);
    return p;
  };
  const size_t NH = (size_t)Nb * MH;
  w.Z1 = reinterpret_cast<float*>(take(NH * 4));
  w.A1 = reinterpret_cast<bf16*>(take(NH * 2));
  w.A1T = reinterpret_cast<bf16*>(take(NH * 2));
  w.Z2 = reinterpret_cast<float*>(take(NH * 4));
  w.A2 = reinterpret_cast<bf16*>(take(NH * 2));
  w.A2T = reinterpret_cast<bf16*>(take(NH * 2));
  w.A3T = reinterpret_cast<float*>(take(NH * 4));
  w.dF = reinterpret_cast<float*>(take((size_t)Nb * 4));
  w.rsq = reinterpret_cast<float*>(take((size_t)Nb * 4));
  w.dZ3 = reinterpret_cast<bf16*>(take(NH * 2));
  w.dZ3T = reinterpret_cast<bf16*>(take(NH * 2));
  w.dZ2 = reinterpret_cast<bf16*>(take(NH * 2));
  w.dZ2T = reinterpret_cast<bf16*>(take(NH * 2));
  w.dZ1T = reinterpret_cast<float*>(take(NH * 4));
  w.slab = reinterpret_cast<float*>(take((size_t)w.splits * MH * MH * 4));
  w.grads = reinterpret_cast<float*>(take(MLP_P * 4));
  w.bytes = off;
  return w;
}

// ---- layer 1 on the CUDA cores: one thread per sample
__global__ void __launch_bounds__(128) mlp_l1_kernel(const float* __restrict__ u,
                                                     const float* __restrict__ p, MlpWork w,
                                                     int Nb) {
  __shared__ float sW[3 * MH + MH];
  for (int i = threadIdx.x; i < 4 * MH; i += blockDim.x) sW[i] = p[OFF_W1 + i];  // W1 then b1
  __syncthreads();
  const int row = blockIdx.x * 128 + threadIdx.x;
  const float x0 = u[3 * row], x1 = u[3 * row + 1], x2 = u[3 * row + 2];
#pragma unroll 1
  for (int c8 = 0; c8 < MH / 8; ++c8) {
    float z[8];
    uint32_t a[4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = c8 * 8 + j;
      z[j] = fmaf(sW[3 * c], x0, fmaf(sW[3 * c + 1], x1, fmaf(sW[3 * c + 2], x2, sW[3 * MH + c])));
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = pack_bf16x2(silu(z[2 * j]), silu(z[2 * j + 1]));
    float4* zr = reinterpret_cast<float4*>(w.Z1 + (int64_t)row * MH + c8 * 8);
    zr[0] = make_float4(z[0], z[1], z[2], z[3]);
    zr[1] = make_float4(z[4], z[5], z[6], z[7]);
    *reinterpret_cast<uint4*>(w.A1 + (int64_t)row * MH + c8 * 8) = make_uint4(a[0], a[1], a[2], a[3]);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t h = a[j >> 1] >> (16 * (j & 1));
      reinterpret_cast<uint16_t*>(w.A1T)[(int64_t)(c8 * 8 + j) * Nb + row] = (uint16_t)h;
    }
  }
}

// ---- GEMM epilogues (thread = one row of the 128 x 256 tile; n0 = 0)

// + bias, Z (float32), A = s(Z) row-major and transposed (bf16)
struct EpiHidden {
  const float* bias;
  float* Z;
  bf16* A;
  bf16* AT;
  int Nb;
  __device__ __forceinline__ void operator()(uint32_t taddr, int row, int, int) const {
#pragma unroll 1
    for (int c = 0; c < MH / 32; ++c) {
      uint32_t r[32];
      tmem_ld32(taddr + (uint32_t)(c * 32), r);
      float z[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) z[j] = __uint_as_float(r[j]) + __ldg(bias + c * 32 + j);
      float4* zr = reinterpret_cast<float4*>(Z + (int64_t)row * MH + c * 32);
#pragma unroll
      for (int j = 0; j < 8; ++j) zr[j] = make_float4(z[4 * j], z[4 * j + 1], z[4 * j + 2], z[4 * j + 3]);
      uint32_t a[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) a[j] = pack_bf16x2(silu(z[2 * j]), silu(z[2 * j + 1]));
      uint4* ar = reinterpret_cast<uint4*>(A + (int64_t)row * MH + c * 32);
#pragma unroll
      for (int j = 0; j < 4; ++j) ar[j] = make_uint4(a[4 * j], a[4 * j + 1], a[4 * j + 2], a[4 * j + 3]);
      uint16_t* at = reinterpret_cast<uint16_t*>(AT);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        at[(int64_t)(c * 32 + j) * Nb + row] = (uint16_t)(a[j >> 1] >> (16 * (j & 1)));
    }
  }
};

// Output layer and the start of the backward pass.
struct EpiHead {
  const float* b3;
  const float* w4;
  const float* b4;
  const float* y;
  float* A3T;
  float* dF;
  float* rsq;
  bf16* dZ3;
  bf16* dZ3T;
  int Nb;
  float inv_n;
  float over_w;
  __device__ __forceinline__ void operator()(uint32_t taddr, int row, int, int) const {
    float f = 0.f;
#pragma unroll 1
    for (int c = 0; c < MH / 32; ++c) {
      uint32_t r[32];
      tmem_ld32(taddr + (uint32_t)(c * 32), r);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int col = c * 32 + j;
        const float a = silu(__uint_as_float(r[j]) + __ldg(b3 + col));
        A3T[(int64_t)col * Nb + row] = a;
        f = fmaf(__ldg(w4 + col), a, f);
      }
    }
    f += __ldg(b4);
    const float res = f - __ldg(y + row);
    const float wt = res > 0.f ? over_w : 1.f;
    const float df = 2.f * wt * res * inv_n;
    dF[row] = df;
    rsq[row] = wt * res * res;
#pragma unroll 1
    for (int c = 0; c < MH / 32; ++c) {
      uint32_t r[32];
      tmem_ld32(taddr + (uint32_t)(c * 32), r);
      uint32_t g[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = c * 32 + 2 * j;
        const float g0 = df * __ldg(w4 + col) * silu_grad(__uint_as_float(r[2 * j]) + __ldg(b3 + col));
        const float g1 =
            df * __ldg(w4 + col + 1) * silu_grad(__uint_as_float(r[2 * j + 1]) + __ldg(b3 + col + 1));
        g[j] = pack_bf16x2(g0, g1);
      }
      uint4* dr = reinterpret_cast<uint4*>(dZ3 + (int64_t)row * MH + c * 32);
#pragma unroll
      for (int j = 0; j < 4; ++j) dr[j] = make_uint4(g[4 * j], g[4 * j + 1], g[4 * j + 2], g[4 * j + 3]);
      uint16_t* dt = reinterpret_cast<uint16_t*>(dZ3T);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        dt[(int64_t)(c * 32 + j) * Nb + row] = (uint16_t)(g[j >> 1] >> (16 * (j & 1)));
    }
  }
};

// dZ = dA x s'(Z): bf16 row-major and transposed (hidden layer 2)
struct EpiBackHidden {
  const float* Z;
  bf16* dZ;
  bf16* dZT;
  int Nb;
  __device__ __forceinline__ void operator()(uint32_t taddr, int row, int, int) const {
#pragma unroll 1
    for (int c = 0; c < MH / 32; ++c) {
      uint32_t r[32];
      tmem_ld32(taddr + (uint32_t)(c * 32), r);
      const float4* zr = reinterpret_cast<const float4*>(Z + (int64_t)row * MH + c * 32);
      uint32_t g[16];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float4 z = zr[j];
        g[2 * j] = pack_bf16x2(__uint_as_float(r[4 * j]) * silu_grad(z.x),
                               __uint_as_float(r[4 * j + 1]) * silu_grad(z.y));
        g[2 * j + 1] = pack_bf16x2(__uint_as_float(r[4 * j + 2]) * silu_grad(z.z),
                                   __uint_as_float(r[4 * j + 3]) * silu_grad(z.w));
      }
      uint4* dr = reinterpret_cast<uint4*>(dZ + (int64_t)row * MH + c * 32);
#pragma unroll
      for (int j = 0; j < 4; ++j) dr[j] = make_uint4(g[4 * j], g[4 * j + 1], g[4 * j + 2], g[4 * j + 3]);
      uint16_t* dt = reinterpret_cast<uint16_t*>(dZT);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        dt[(int64_t)(c * 32 + j) * Nb + row] = (uint16_t)(g[j >> 1] >> (16 * (j & 1)));
    }
  }
};

// dZ1 = dA1 x s'(Z1), float32 transposed (for the layer-1 sums)
struct EpiBackFirst {
  const float* Z;
  float* dZT;
  int Nb;
  __device__ __forceinline__ void operator()(uint32_t taddr, int row, int, int) const {
#pragma unroll 1
    for (int c = 0; c < MH / 32; ++c) {
      uint32_t r[32];
      tmem_ld32(taddr + (uint32_t)(c * 32), r);
      const float4* zr = reinterpret_cast<const float4*>(Z + (int64_t)row * MH + c * 32);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float4 z = zr[j];
        const int col = c * 32 + 4 * j;
        dZT[(int64_t)col * Nb + row] = __uint_as_float(r[4 * j]) * silu_grad(z.x);
        dZT[(int64_t)(col + 1) * Nb + row] = __uint_as_float(r[4 * j + 1]) * silu_grad(z.y);
        dZT[(int64_t)(col + 2) * Nb + row] = __uint_as_float(r[4 * j + 2]) * silu_grad(z.z);
        dZT[(int64_t)(col + 3) * Nb + row] = __uint_as_float(r[4 * j + 3]) * silu_grad(z.w);
      }
    }
  }
};

// ---- sums over the batch

// out[i] = sum_z slab[z][i] (z in order)
__global__ void mlp_reduce_slabs(const float* __restrict__ slab, int splits, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= MH * MH) return;
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += slab[(int64_t)z * MH * MH + i];
  out[i] = s;
}

// Block-wide sum in a fixed order (256 threads).
__device__ __forceinline__ float block_sum(float v, float* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  const float s = red[0];
  __syncthreads();
  return s;
}

// blockIdx.y: 0 dW1 and db1, 1 db2, 2 db3, 3 dw4, 4 db4 and the loss
// (block 0 only); blockIdx.x = hidden unit.
__global__ void __launch_bounds__(256) mlp_small_grads(const float* __restrict__ u, MlpWork w, int Nb,
                                                       float inv_n, float* __restrict__ loss) {
  __shared__ float red[256];
  const int c = blockIdx.x, kind = blockIdx.y;
  float* g = w.grads;
  if (kind == 0) {
    const float* d = w.dZ1T + (int64_t)c * Nb;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, sb = 0.f;
    for (int r = threadIdx.x; r < Nb; r += 256) {
      const float v = d[r];
      sb += v;
      s0 = fmaf(v, u[3 * r], s0);
      s1 = fmaf(v, u[3 * r + 1], s1);
      s2 = fmaf(v, u[3 * r + 2], s2);
    }
    s0 = block_sum(s0, red);
    s1 = block_sum(s1, red);
    s2 = block_sum(s2, red);
    sb = block_sum(sb, red);
    if (threadIdx.x == 0) {
      g[OFF_W1 + 3 * c] = s0;
      g[OFF_W1 + 3 * c + 1] = s1;
      g[OFF_W1 + 3 * c + 2] = s2;
      g[OFF_B1 + c] = sb;
    }
  } else if (kind == 1 || kind == 2) {
    const uint16_t* d = reinterpret_cast<const uint16_t*>(kind == 1 ? w.dZ2T : w.dZ3T) + (int64_t)c * Nb;
    float s = 0.f;
    for (int r = threadIdx.x; r < Nb; r += 256) s += __uint_as_float((uint32_t)d[r] << 16);
    s = block_sum(s, red);
    if (threadIdx.x == 0) g[(kind == 1 ? OFF_B2 : OFF_B3) + c] = s;
  } else if (kind == 3) {
    const float* a = w.A3T + (int64_t)c * Nb;
    float s = 0.f;
    for (int r = threadIdx.x; r < Nb; r += 256) s = fmaf(a[r], w.dF[r], s);
    s = block_sum(s, red);
    if (threadIdx.x == 0) g[OFF_W4 + c] = s;
  } else if (c == 0) {
    float sf = 0.f, sl = 0.f;
    for (int r = threadIdx.x; r < Nb; r += 256) {
      sf += w.dF[r];
      sl += w.rsq[r];
    }
    sf = block_sum(sf, red);
    sl = block_sum(sl, red);
    if (threadIdx.x == 0) {
      g[OFF_B4] = sf;
      if (loss) *loss = sl * inv_n;
    }
  }
}

// ---- optimiser and weight copies

__global__ void mlp_adam(MlpState s, const float* __restrict__ g, vapr_train_params hp) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= MLP_P) return;
  const int t = *s.step + 1;
  const float c1 = 1.f - powf(hp.beta1, (float)t), c2 = 1.f - powf(hp.beta2, (float)t);
  const float gi = g[i];
  const float m = fmaf(hp.beta1, s.m[i], (1.f - hp.beta1) * gi);
  const float v = fmaf(hp.beta2, s.v[i], (1.f - hp.beta2) * gi * gi);
  s.m[i] = m;
  s.v[i] = v;
  s.p[i] -= hp.lr * (m / c1) / (sqrtf(v / c2) + hp.eps);
}

// bf16 W2, W3 and their transposes; 32 x 32 tiles through shared memory.
__global__ void mlp_refresh_kernel(MlpState s, int bump_step) {
  __shared__ float tile[32][33];
  const float* W = s.p + (blockIdx.z == 0 ? OFF_W2 : OFF_W3);
  bf16* D = blockIdx.z == 0 ? s.W2 : s.W3;
  bf16* DT = blockIdx.z == 0 ? s.W2T : s.W3T;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const float v = W[(r0 + k) * MH + c0 + threadIdx.x];
    tile[k][threadIdx.x] = v;
    D[(r0 + k) * MH + c0 + threadIdx.x] = __float2bfloat16_rn(v);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y)
    DT[(c0 + k) * MH + r0 + threadIdx.x] = __float2bfloat16_rn(tile[threadIdx.x][k]);
  if (bump_step && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
      threadIdx.y == 0)
    *s.step += 1;
}

cudaError_t launch_mlp_refresh(const MlpState& s, bool bump_step, cudaStream_t st) {
  mlp_refresh_kernel<<<dim3(MH / 32, MH / 32, 2), dim3(32, 8), 0, st>>>(s, bump_step ? 1 : 0);
  return cudaGetLastError();
}

static cudaError_t run_grads(const MlpState& s, const float* u, const float* y, int64_t Nb64,
                             float over_w, const MlpWork& w, float* loss, cudaStream_t st) {
  const int Nb = (int)Nb64;
  int* err = tc_error_word();
  if (!err) return cudaErrorUnknown;
  const float inv_n = 1.f / (float)Nb;
  cudaError_t e;
  mlp_l1_kernel<<<Nb / 128, 128, 0, st>>>(u, s.p, w, Nb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const TgShape fwd{Nb, MH, MH, MH};
  if ((e = tg_launch(w.A1, s.W2, fwd, EpiHidden{s.p + OFF_B2, w.Z2, w.A2, w.A2T, Nb}, err, st)) != cudaSuccess)
    return e;
  EpiHead head{s.p + OFF_B3, s.p + OFF_W4, s.p + OFF_B4, y,     w.A3T, w.dF, w.rsq,
               w.dZ3,      w.dZ3T,         Nb,              inv_n, over_w};
  if ((e = tg_launch(w.A2, s.W3, fwd, head, err, st)) != cudaSuccess) return e;
  const TgShape wg{MH, MH, Nb, w.k_split};
  const int rb = (MH * MH + 255) / 256;
  if ((e = tg_launch(w.dZ3T, w.A2T, wg, StoreF32{w.slab, MH, (int64_t)MH * MH}, err, st)) != cudaSuccess)
    return e;
  mlp_reduce_slabs<<<rb, 256, 0, st>>>(w.slab, w.splits, w.grads + OFF_W3);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = tg_launch(w.dZ3, s.W3T, fwd, EpiBackHidden{w.Z2, w.dZ2, w.dZ2T, Nb}, err, st)) != cudaSuccess)
    return e;
  if ((e = tg_launch(w.dZ2T, w.A1T, wg, StoreF32{w.slab, MH, (int64_t)MH * MH}, err, st)) != cudaSuccess)
    return e;
  mlp_reduce_slabs<<<rb, 256, 0, st>>>(w.slab, w.splits, w.grads + OFF_W2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = tg_launch(w.dZ2, s.W2T, fwd, EpiBackFirst{w.Z1, w.dZ1T, Nb}, err, st)) != cudaSuccess) return e;
  mlp_small_grads<<<dim3(MH, 5), 256, 0, st>>>(u, w, Nb, inv_n, loss);
  return cudaGetLastError();
}

static vapr_status check_batch(const void* state, const float* u, const float* y, int64_t batch,
                               void* ws, size_t ws_bytes) {
  if (!state || !u || !y || !ws) return VAPR_ERR_INVALID_ARG;
  if (batch <= 0 || batch % 128) return VAPR_ERR_INVALID_ARG;
  if (batch > MAX_MLP_BATCH) return VAPR_ERR_TOO_LARGE;
  if (((uintptr_t)state | (uintptr_t)ws) % 256 || (uintptr_t)u % 16 || (uintptr_t)y % 4)
    return VAPR_ERR_MISALIGNED;
  if (ws_bytes < carve_work(nullptr, batch).bytes) return VAPR_ERR_INVALID_ARG;
  return VAPR_OK;
}

}  // namespace vapr

using namespace vapr;

extern "C" size_t vapr_mlp_state_bytes(void) { return MLP_STATE_BYTES; }

extern "C" vapr_status vapr_mlp_init(void* state, const float* params, void* stream) {
  if (!state || !params) return VAPR_ERR_INVALID_ARG;
  if ((uintptr_t)state % 256 || (uintptr_t)params % 4) return VAPR_ERR_MISALIGNED;
  cudaStream_t st = (cudaStream_t)stream;
  const MlpState s = mlp_state(state);
  cudaError_t e = cudaMemcpyAsync(s.p, params, MLP_P * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.m, 0, 2 * MLP_PBYTES + 256, st);  // m, v, step
  if (e == cudaSuccess) e = launch_mlp_refresh(s, false, st);
  return cuda_status(e);
}

extern "C" vapr_status vapr_mlp_get_params(const void* state, float* params, void* stream) {
  if (!state || !params) return VAPR_ERR_INVALID_ARG;
  if ((uintptr_t)state % 256 || (uintptr_t)params % 4) return VAPR_ERR_MISALIGNED;
  const MlpState s = mlp_state(const_cast<void*>(state));
  return cuda_status(cudaMemcpyAsync(params, s.p, MLP_P * sizeof(float), cudaMemcpyDeviceToDevice,
                                     (cudaStream_t)stream));
}

extern "C" size_t vapr_mlp_workspace_bytes(int64_t batch) {
  if (batch <= 0 || batch % 128 || batch > MAX_MLP_BATCH) return 0;
  return carve_work(nullptr, batch).bytes;
}

extern "C" vapr_status vapr_mlp_grads(const void* state, const float* u, const float* y,
                                      int64_t batch, float over_weight, void* workspace,
                                      size_t workspace_bytes, float* grads, float* loss,
                                      void* stream) {
  const vapr_status v = check_batch(state, u, y, batch, workspace, workspace_bytes);
  if (v != VAPR_OK) return v;
  if (!(over_weight > 0.f) || !isfinite(over_weight)) return VAPR_ERR_INVALID_ARG;
  if ((grads && (uintptr_t)grads % 4) || (loss && (uintptr_t)loss % 4)) return VAPR_ERR_MISALIGNED;
  cudaStream_t st = (cudaStream_t)stream;
  const MlpState s = mlp_state(const_cast<void*>(state));
  const MlpWork w = carve_work(workspace, batch);
  cudaError_t e = run_grads(s, u, y, batch, over_weight, w, loss, st);
  if (e == cudaSuccess && grads)
    e = cudaMemcpyAsync(grads, w.grads, MLP_P * sizeof(float), cudaMemcpyDeviceToDevice, st);
  return cuda_status(e);
}

extern "C" vapr_status vapr_mlp_train_step(void* state, const float* u, const float* y,
                                           int64_t batch, const vapr_train_params* hp,
                                           void* workspace, size_t workspace_bytes, float* loss,
                                           void* stream) {
  const vapr_status v = check_batch(state, u, y, batch, workspace, workspace_bytes);
  if (v != VAPR_OK) return v;
  if (!hp || !(hp->lr >= 0.f) || !isfinite(hp->lr) || !(hp->beta1 >= 0.f && hp->beta1 < 1.f) ||
      !(hp->beta2 >= 0.f && hp->beta2 < 1.f) || !(hp->eps > 0.f) || !(hp->over_weight > 0.f) ||
      !isfinite(hp->over_weight))
    return VAPR_ERR_INVALID_ARG;
  if (loss && (uintptr_t)loss % 4) return VAPR_ERR_MISALIGNED;
  cudaStream_t st = (cudaStream_t)stream;
  const MlpState s = mlp_state(state);
  const MlpWork w = carve_work(workspace, batch);
  cudaError_t e = run_grads(s, u, y, batch, hp->over_weight, w, loss, st);
  if (e == cudaSuccess) {
    mlp_adam<<<(int)((MLP_P + 255) / 256), 256, 0, st>>>(s, w.grads, *hp);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_mlp_refresh(s, true, st);
  return cuda_status(e);
}
