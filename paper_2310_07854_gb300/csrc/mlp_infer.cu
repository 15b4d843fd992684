// Inference of the signed-distance surrogate (mlp.cuh) in one persistent
// launch, the exact scene distance that labels its training data, and the
// collision stage with the network as a broad phase.
//
// mlp_infer_kernel, one CTA per SM, 10 warps, two tiles of 128 inputs in
// flight so that the CUDA-core work of one overlaps the tensor-core work of
// the other:
//   warp 8 lane 0   TMA producer: streams 16 KB weight slices (128 output
//                   units x 64 inputs of W2 or W3, 128-byte swizzled)
//                   through a 5-stage ring, 16 slices per tile, for every
//                   tile of the CTA;
//   warp 9 lane 0   MMA issuer: layer 2 of tile t (A1 x W2^T into TMEM
//                   columns 0-255, one N=128 half at a time), then layer 3
//                   (A2 x W3^T into columns 256-511); each half is
//                   signalled with tcgen05.commit;
//   warps 0-7       per tile: layer 1 (3 -> 256, CUDA cores) into the
//                   swizzled A1 operand; the layer-2 epilogue (bias, SiLU,
//                   bf16) into A2; the layer-3 epilogue (bias, SiLU, dot
//                   with w4).  Warp w reads TMEM lanes 32(w%4).. (its rows)
//                   and the column half w/4.
// Order of the compute warps: epi2(t), L1(t+1), epi3(t), so that layer 3 of
// tile t runs under L1(t+1) and layer 2 of tile t+1 under epi3(t).
// Buffers: A1 (written by L1, read by layer 2), A2 (epi2 / layer 3), the two
// TMEM accumulators; each is reused only after the commit that ends its
// last reader.  The activations never leave the SM; only the weights (from
// L2) and 12 input and 4 output bytes per query touch memory.
// Waits are bounded.  On a timeout the CTA records VAPR_ERR_TIMEOUT and runs
// to its end without waiting again (compute warps still pass every named
// barrier, so none is left behind), lets its copies and MMAs land, and frees
// its tensor memory.
#include <cfloat>

#include "mlp.cuh"

namespace vapr {

constexpr int MI_STAGES = 5;
constexpr int MI_CWARPS = 8;
constexpr int MI_THREADS = (MI_CWARPS + 2) * 32;
constexpr uint32_t MI_SLICE = 128 * 128;       // 128 rows x 64 bf16 (128 B), swizzled
constexpr uint32_t MI_A_BYTES = 4 * MI_SLICE;  // 128 x 256 bf16 activations
constexpr size_t MI_SMEM = 1024 + 2 * MI_A_BYTES + MI_STAGES * MI_SLICE + 3 * 128 * 16 +
                           3 * MH * 4 + 2 * 128 * 4 + 24 * 8 + 16;

__device__ __forceinline__ void cw_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_addr(bar)) : "memory");
}

// Inputs given as domain coordinates u [n][3].
struct InPlain {
  const float* u;
  __device__ __forceinline__ float4 operator()(int64_t q) const {
    return make_float4(__ldg(u + 3 * q), __ldg(u + 3 * q + 1), __ldg(u + 3 * q + 2), -1.f);
  }
};

// Inputs = sphere centres of packed P rows (query q = configuration q / S,
// sphere q % S); .w = the outside-the-box lower bound of sdf, or -1 inside.
struct InSpheres {
  const uint8_t* pos;
  int64_t stride;
  DevFmt f;
  int S;
  float lo[3], hi[3], ctr[3], ihalf[3], pad;
  __device__ __forceinline__ float4 operator()(int64_t q) const {
    const int64_t c = q / S;
    const int s = (int)(q - c * S);
    const uint32_t* row = reinterpret_cast<const uint32_t*>(pos + c * stride);
    float x[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int i = 3 * s + j, w = i / f.k;
      x[j] = unpack_slot(__ldg(row + w), i - w * f.k, f);
    }
    float o2 = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float e = fmaxf(fmaxf(lo[j] - x[j], x[j] - hi[j]), 0.f);
      o2 = fmaf(e, e, o2);
    }
    const float lb = o2 > 0.f ? sqrtf(o2) + pad : -1.f;
    return make_float4((x[0] - ctr[0]) * ihalf[0], (x[1] - ctr[1]) * ihalf[1],
                       (x[2] - ctr[2]) * ihalf[2], lb);
  }
};

template <class In>
__global__ void __launch_bounds__(MI_THREADS, 1)
    mlp_infer_kernel(const __grid_constant__ CUtensorMap tmW2, const __grid_constant__ CUtensorMap tmW3,
                     const float* __restrict__ p, In in, int64_t n, float* __restrict__ out, int* err) {
  extern __shared__ uint8_t mi_raw[];
  uint8_t* base = mi_raw + ((1024u - (sm_addr(mi_raw) & 1023u)) & 1023u);
  uint8_t* sA1 = base;
  uint8_t* sA2 = base + MI_A_BYTES;
  uint8_t* ring = base + 2 * MI_A_BYTES;
  float4* xin = reinterpret_cast<float4*>(ring + MI_STAGES * MI_SLICE);  // [3][128]
  float* sb2 = reinterpret_cast<float*>(xin + 3 * 128);
  float* sb3 = sb2 + MH;
  float* sw4 = sb3 + MH;
  float* red = sw4 + MH;  // [2][128]
  uint64_t* full = reinterpret_cast<uint64_t*>(red + 2 * 128);
  uint64_t* empty = full + MI_STAGES;
  uint64_t* a1_full = empty + MI_STAGES;  // L1(t) written (256 arrivals)
  uint64_t* a2_full = a1_full + 1;        // epi2(t) done (256 arrivals)
  uint64_t* acc2 = a2_full + 1;           // [2] layer-2 half done
  uint64_t* acc3 = acc2 + 2;              // [2] layer-3 half done
  uint64_t* drain = acc3 + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (n + 127) / 128;
  const int my_tiles = ntiles > (int64_t)blockIdx.x ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < MI_STAGES; ++s) {
      mb_init(full + s, 1);
      mb_init(empty + s, 1);
    }
    mb_init(a1_full, MI_CWARPS * 32);
    mb_init(a2_full, MI_CWARPS * 32);
    for (int h = 0; h < 2; ++h) {
      mb_init(acc2 + h, 1);
      mb_init(acc3 + h, 1);
    }
    mb_init(drain, 1);
    *abort_flag = 0;
    mb_init_fence();
  }
  for (int i = threadIdx.x; i < MH; i += blockDim.x) {
    sb2[i] = p[OFF_B2 + i];
    sb3[i] = p[OFF_B3 + i];
    sw4[i] = p[OFF_W4 + i];
  }
  if (warp == 0) tmem_alloc(tslot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t IDESC = idesc_bf16_f32(128, 128);

  if (warp == MI_CWARPS) {  // ---- TMA producer
    if (lane == 0) {
      const int total = my_tiles * 16;
      int issued = 0;
      for (int it = 0; it < total; ++it) {
        const int s = it % MI_STAGES;
        if (it >= MI_STAGES && !mb_wait(empty + s, ((it / MI_STAGES) - 1) & 1, TG_WAIT)) {
          *abort_flag = 1;
          break;
        }
        if (*abort_flag) break;
        mb_expect_tx(full + s, MI_SLICE);
        const int j = it & 15;  // layer (j >> 3), output half ((j >> 2) & 1), K slice (j & 3)
        tma_load_2d(ring + s * MI_SLICE, (j & 8) ? &tmW3 : &tmW2, (j & 3) * TG_K, ((j >> 2) & 1) * 128,
                    full + s);
        issued = it + 1;
      }
      if (*abort_flag)  // let every issued copy land before the CTA can exit
        for (int it = (issued > MI_STAGES ? issued - MI_STAGES : 0); it < issued; ++it)
          mb_wait(full + it % MI_STAGES, (it / MI_STAGES) & 1, TG_WAIT);
    }
    __syncwarp();
  } else if (warp == MI_CWARPS + 1) {  // ---- MMA issuer
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int t = 0; t < my_tiles && ok; ++t) {
        for (int layer = 0; layer < 2 && ok; ++layer) {
          if (!mb_wait(layer ? a2_full : a1_full, t & 1, TG_WAIT) || *abort_flag) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint8_t* sA = layer ? sA2 : sA1;
          for (int nh = 0; nh < 2 && ok; ++nh) {
            const uint32_t d = tmem + (uint32_t)(layer * 256 + nh * 128);
            for (int ks = 0; ks < 4; ++ks, ++it) {
              const int s = it % MI_STAGES;
              if (!mb_wait(full + s, (it / MI_STAGES) & 1, TG_WAIT)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint64_t ad = sw128_desc(sA + ks * MI_SLICE), bd = sw128_desc(ring + s * MI_SLICE);
#pragma unroll
              for (int kk = 0; kk < TG_K / 16; ++kk) umma_bf16(d, ad + 2 * kk, bd + 2 * kk, IDESC, (ks | kk) != 0);
              umma_commit(empty + s);
            }
            if (ok) umma_commit((layer ? acc3 : acc2) + nh);
          }
        }
      }
      if (!ok) *abort_flag = 1;
      umma_commit(drain);  // arrives once every MMA issued above has completed
      mb_wait(drain, 0, TG_WAIT);
    }
    __syncwarp();
  } else {  // ---- compute warps
    const int tid = threadIdx.x;  // 0..255
    float w1[8][3], b1[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = 8 * lane + j;
      w1[j][0] = p[OFF_W1 + 3 * col];
      w1[j][1] = p[OFF_W1 + 3 * col + 1];
      w1[j][2] = p[OFF_W1 + 3 * col + 2];
      b1[j] = p[OFF_B1 + col];
    }
    const float b4 = p[OFF_B4];
    const int qd = warp & 3, half = warp >> 2;
    const int rr = 32 * qd + lane;  // this thread's row in the epilogues
    const uint32_t trow = tmem + ((uint32_t)(32 * qd) << 16);
    bool failed = false;
    // bounded wait on a phase; once one wait has failed, none waits again
    auto wait = [&](uint64_t* bar, int parity) {
      if (!failed) failed = !mb_wait(bar, (uint32_t)parity, TG_WAIT);
      failed = __any_sync(0xffffffffu, failed);
      tc_fence_after();
    };
    // stage the inputs of tile t, then layer 1 into A1 (rows warp, warp+8, ...;
    // lane = one 16-byte chunk of 8 columns)
    auto layer1 = [&](int t) {
      const int64_t q0 = ((int64_t)blockIdx.x + (int64_t)t * gridDim.x) * 128;
      float4* xt = xin + (t % 3) * 128;
      if (tid < 128) xt[tid] = q0 + tid < n ? in(q0 + tid) : make_float4(0.f, 0.f, 0.f, -1.f);
      cw_bar();
      const int slice = lane >> 3, ch = lane & 7;
#pragma unroll 2
      for (int r = warp; r < 128; r += MI_CWARPS) {
        const float4 x = xt[r];
        uint32_t a[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float z0 = fmaf(w1[2 * j][0], x.x, fmaf(w1[2 * j][1], x.y, fmaf(w1[2 * j][2], x.z, b1[2 * j])));
          const float z1 = fmaf(w1[2 * j + 1][0], x.x,
                                fmaf(w1[2 * j + 1][1], x.y, fmaf(w1[2 * j + 1][2], x.z, b1[2 * j + 1])));
          a[j] = pack_bf16x2(silu(z0), silu(z1));
        }
        *reinterpret_cast<uint4*>(sA1 + slice * MI_SLICE + r * 128 + ((ch ^ (r & 7)) << 4)) =
            make_uint4(a[0], a[1], a[2], a[3]);
      }
      proxy_fence();
      mb_arrive(a1_full);
    };
    if (my_tiles > 0) layer1(0);
    for (int t = 0; t < my_tiles; ++t) {
      const int64_t q0 = ((int64_t)blockIdx.x + (int64_t)t * gridDim.x) * 128;
      // ---- epi2(t): + b2, SiLU, bf16 into A2 (free: layer 3 of t-1 is done)
      wait(acc2 + half, t & 1);
      if (!failed) {
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
          const int col0 = 128 * half + 32 * c;
          uint32_t r[32];
          tmem_ld32(trow + (uint32_t)col0, r);
          uint32_t a[16];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            a[j] = pack_bf16x2(silu(__uint_as_float(r[2 * j]) + sb2[col0 + 2 * j]),
                               silu(__uint_as_float(r[2 * j + 1]) + sb2[col0 + 2 * j + 1]));
          uint8_t* rowp = sA2 + (col0 >> 6) * MI_SLICE + rr * 128;
          const int ch0 = (col0 & 63) >> 3;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            *reinterpret_cast<uint4*>(rowp + (((ch0 + k) ^ (rr & 7)) << 4)) =
                make_uint4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
        }
      }
      tc_fence_before();
      proxy_fence();
      mb_arrive(a2_full);
      // ---- L1(t+1) into A1 (free once both halves of layer 2 of t are done)
      if (t + 1 < my_tiles) {
        wait(acc2 + 1, t & 1);
        layer1(t + 1);
      }
      // ---- epi3(t): + b3, SiLU, dot with w4; the two halves meet in red
      wait(acc3 + half, t & 1);
      float part = 0.f;
      if (!failed) {
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
          const int col0 = 128 * half + 32 * c;
          uint32_t r[32];
          tmem_ld32(trow + (uint32_t)(256 + col0), r);
#pragma unroll
          for (int j = 0; j < 32; ++j)
            part = fmaf(sw4[col0 + j], silu(__uint_as_float(r[j]) + sb3[col0 + j]), part);
        }
      }
      tc_fence_before();
      float* rt = red + (t & 1) * 128;
      if (half == 1) rt[rr] = part;
      cw_bar();
      if (half == 0 && q0 + rr < n) {
        const float lb = xin[(t % 3) * 128 + rr].w;
        out[q0 + rr] = lb >= 0.f ? lb : (b4 + part) + rt[rr];
      }
      // A2 is rewritten by epi2(t+1): both halves of layer 3 of t must be done
      wait(acc3 + 1, t & 1);
    }
    if (failed && lane == 0) atomicCAS(err, 0, (int)VAPR_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

template <class In>
static cudaError_t launch_infer(const MlpState& s, In in, int64_t n, float* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int* err = tc_error_word();
  if (!err) return cudaErrorUnknown;
  CUtensorMap m2, m3;
  if (!tg_tensor_map(&m2, s.W2, MH, MH, 128) || !tg_tensor_map(&m3, s.W3, MH, MH, 128))
    return cudaErrorInvalidValue;
  const int per_sm = blocks_per_sm((const void*)mlp_infer_kernel<In>, MI_THREADS, MI_SMEM);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t tiles = (n + 127) / 128;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  mlp_infer_kernel<In><<<(int)(tiles < cap ? tiles : cap), MI_THREADS, MI_SMEM, st>>>(m2, m3, s.p, in, n,
                                                                                      out, err);
  return cudaGetLastError();
}

// ---- exact scene signed distance: one thread per point, cuboids in shared memory
__global__ void scene_sdf_kernel(SceneArgs sc, const float* __restrict__ pts, int64_t n,
                                 float* __restrict__ sdf, float* __restrict__ u, float3 ctr, float3 ihalf,
                                 float y_min, float y_max) {
  extern __shared__ float ss[];
  float* pose = ss;             // [O][12]
  float* half = ss + 12 * sc.O; // [O][3]
  for (int i = threadIdx.x; i < 12 * sc.O; i += blockDim.x) pose[i] = sc.pose[i];
  for (int i = threadIdx.x; i < 3 * sc.O; i += blockDim.x) half[i] = sc.half[i];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float px = pts[3 * i], py = pts[3 * i + 1], pz = pts[3 * i + 2];
    float best = FLT_MAX;
    for (int o = 0; o < sc.O; ++o) {
      const float* R = pose + 12 * o;
      const float dx = px - R[9], dy = py - R[10], dz = pz - R[11];
      // box frame: x = R^T (p - t)
      const float x0 = fmaf(R[0], dx, fmaf(R[3], dy, R[6] * dz));
      const float x1 = fmaf(R[1], dx, fmaf(R[4], dy, R[7] * dz));
      const float x2 = fmaf(R[2], dx, fmaf(R[5], dy, R[8] * dz));
      const float u0 = fabsf(x0) - half[3 * o], u1 = fabsf(x1) - half[3 * o + 1],
                  u2 = fabsf(x2) - half[3 * o + 2];
      const float v0 = fmaxf(u0, 0.f), v1 = fmaxf(u1, 0.f), v2 = fmaxf(u2, 0.f);
      const float d = sqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2))) + fminf(fmaxf(u0, fmaxf(u1, u2)), 0.f);
      best = fminf(best, d);
    }
    sdf[i] = fminf(fmaxf(best, y_min), y_max);
    if (u) {
      u[3 * i] = (px - ctr.x) * ihalf.x;
      u[3 * i + 1] = (py - ctr.y) * ihalf.y;
      u[3 * i + 2] = (pz - ctr.z) * ihalf.z;
    }
  }
}

static cudaError_t launch_sdf(const SceneArgs& sc, const float* pts, int64_t n, float* sdf, float* u,
                              float3 ctr, float3 ihalf, float y_min, float y_max, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t smem = (size_t)15 * sc.O * sizeof(float);
  const int per_sm = blocks_per_sm((const void*)scene_sdf_kernel, 256, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t blocks = (n + 255) / 256, cap = (int64_t)sm_count() * per_sm;
  scene_sdf_kernel<<<(int)(blocks < cap ? blocks : cap), 256, smem, st>>>(sc, pts, n, sdf, u, ctr, ihalf,
                                                                         y_min, y_max);
  return cudaGetLastError();
}

static vapr_status check_scene_args(const vapr_scene* scene, SceneArgs& sc) {
  return check_scene(scene, &sc);
}

static vapr_status check_domain(const vapr_surrogate_domain* d) {
  if (!d) return VAPR_ERR_INVALID_ARG;
  for (int j = 0; j < 3; ++j)
    if (!(d->hi[j] > d->lo[j]) || !isfinite(d->lo[j]) || !isfinite(d->hi[j])) return VAPR_ERR_INVALID_ARG;
  if (!(d->pad >= 0.f) || !(d->margin >= 0.f) || !isfinite(d->pad) || !isfinite(d->margin))
    return VAPR_ERR_INVALID_ARG;
  return VAPR_OK;
}

}  // namespace vapr

using namespace vapr;

extern "C" vapr_status vapr_mlp_forward(const void* state, const float* u, int64_t n, float* out,
                                        void* stream) {
  if (n < 0) return VAPR_ERR_INVALID_ARG;
  if (n == 0) return VAPR_OK;
  if (!state || !u || !out) return VAPR_ERR_INVALID_ARG;
  if ((uintptr_t)state % 256 || (uintptr_t)u % 4 || (uintptr_t)out % 4) return VAPR_ERR_MISALIGNED;
  if (n > ((int64_t)1 << 40)) return VAPR_ERR_TOO_LARGE;
  const MlpState s = mlp_state(const_cast<void*>(state));
  return cuda_status(launch_infer(s, InPlain{u}, n, out, (cudaStream_t)stream));
}

extern "C" vapr_status vapr_scene_sdf(const vapr_scene* scene, const float* pts, int64_t n, float* sdf,
                                      void* stream) {
  SceneArgs sc;
  const vapr_status v = check_scene_args(scene, sc);
  if (v != VAPR_OK) return v;
  if (n < 0) return VAPR_ERR_INVALID_ARG;
  if (n == 0) return VAPR_OK;
  if (!pts || !sdf) return VAPR_ERR_INVALID_ARG;
  if ((uintptr_t)pts % 4 || (uintptr_t)sdf % 4) return VAPR_ERR_MISALIGNED;
  return cuda_status(
      launch_sdf(sc, pts, n, sdf, nullptr, float3{}, float3{}, -FLT_MAX, FLT_MAX, (cudaStream_t)stream));
}

extern "C" vapr_status vapr_surrogate_samples(const vapr_scene* scene, const vapr_surrogate_domain* domain,
                                              const float* pts, int64_t n, float y_min, float y_max,
                                              float* u, float* y, void* stream) {
  SceneArgs sc;
  vapr_status v = check_scene_args(scene, sc);
  if (v == VAPR_OK) v = check_domain(domain);
  if (v != VAPR_OK) return v;
  if (!(y_min <= y_max)) return VAPR_ERR_INVALID_ARG;
  if (n < 0) return VAPR_ERR_INVALID_ARG;
  if (n == 0) return VAPR_OK;
  if (!pts || !u || !y) return VAPR_ERR_INVALID_ARG;
  if ((uintptr_t)pts % 4 || (uintptr_t)u % 4 || (uintptr_t)y % 4) return VAPR_ERR_MISALIGNED;
  const float3 ctr{0.5f * (domain->lo[0] + domain->hi[0]), 0.5f * (domain->lo[1] + domain->hi[1]),
                   0.5f * (domain->lo[2] + domain->hi[2])};
  const float3 ih{2.f / (domain->hi[0] - domain->lo[0]), 2.f / (domain->hi[1] - domain->lo[1]),
                  2.f / (domain->hi[2] - domain->lo[2])};
  return cuda_status(launch_sdf(sc, pts, n, y, u, ctr, ih, y_min, y_max, (cudaStream_t)stream));
}

extern "C" vapr_status vapr_surrogate_collision_cost(const vapr_robot* robot, const vapr_scene* scene,
                                                     const vapr_cost_params* params, const void* net,
                                                     const vapr_surrogate_domain* domain,
                                                     const void* pos_packed, int64_t n,
                                                     const vapr_format_table* table, float* cost,
                                                     void* dist_packed, void* grad_packed, float* estimate,
                                                     void* stream) {
  RobotArgs r;
  vapr_status v = check_robot(robot, &r);
  if (v != VAPR_OK) return v;
  SceneArgs sc;
  if ((v = check_scene_args(scene, sc)) != VAPR_OK) return v;
  if ((v = check_table(table)) != VAPR_OK) return v;
  if ((v = check_domain(domain)) != VAPR_OK) return v;
  if (!params) return VAPR_ERR_INVALID_ARG;
  if (n < 0) return VAPR_ERR_INVALID_ARG;
  if (n > VAPR_MAX_CONFIGS) return VAPR_ERR_TOO_LARGE;
  if (n == 0) return VAPR_OK;
  if (!net || !pos_packed || !estimate) return VAPR_ERR_INVALID_ARG;
  if ((uintptr_t)net % 256 || (uintptr_t)estimate % 4) return VAPR_ERR_MISALIGNED;
  if (((uintptr_t)pos_packed | (uintptr_t)dist_packed | (uintptr_t)grad_packed) % 16 ||
      (uintptr_t)cost % 4)
    return VAPR_ERR_MISALIGNED;
  cudaStream_t st = (cudaStream_t)stream;
  Packed pos{(uint8_t*)pos_packed, (int64_t)row_bytes(3 * r.S, table->pos), make_dev_fmt(table->pos)};
  Packed dist{(uint8_t*)dist_packed, (int64_t)row_bytes(r.S, table->dist), make_dev_fmt(table->dist)};
  Packed grad{(uint8_t*)grad_packed, (int64_t)row_bytes(3 * r.S, table->grad), make_dev_fmt(table->grad)};
  InSpheres in;
  in.pos = pos.ptr;
  in.stride = pos.stride;
  in.f = pos.f;
  in.S = r.S;
  for (int j = 0; j < 3; ++j) {
    in.lo[j] = domain->lo[j];
    in.hi[j] = domain->hi[j];
    in.ctr[j] = 0.5f * (domain->lo[j] + domain->hi[j]);
    in.ihalf[j] = 2.f / (domain->hi[j] - domain->lo[j]);
  }
  in.pad = domain->pad;
  const MlpState s = mlp_state(const_cast<void*>(net));
  cudaError_t e = launch_infer(s, in, n * r.S, estimate, st);
  if (e == cudaSuccess)
    e = launch_collision(r, sc, *params, pos, n, cost, dist, grad, st, estimate, domain->margin);
  return cuda_status(e);
}
