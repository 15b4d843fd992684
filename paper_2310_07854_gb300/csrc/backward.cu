// Backward kinematics (iteration step 5 of Sec. III-B): the gradient with
// respect to the sphere centres (grad_out_spheres, Sec. III-C) becomes the
// joint-space gradient.
//
// For a revolute joint j with axis a_j and origin o_j (z-axis and origin of
// T_j), every sphere on link j or beyond moves as dc_s/dq_j = a_j x (c_s - o_j),
// so  J_j = a_j . (M_{>=j} - o_j x F_{>=j})  with  F = sum G_s  and
// M = sum c_s x G_s  over those spheres.  Writing b_j = a_j x o_j,
//   J_j = a_j . M_{>=j} - b_j . F_{>=j}
//       = (a_j . M - b_j . F) - (a_j . M_{<j} - b_j . F_{<j}),
// so one pass over the links in chain order suffices: when joint j is
// reached the thread records a_j, b_j and K_j = a_j . M_{<j} - b_j . F_{<j},
// and the totals finish every J_j at the end.  Zero gradients are skipped
// (the sparsity of Sec. III-C).
//
// One thread per configuration; a warp owns 32 consecutive configurations.
// Their gradient rows are contiguous in global memory, so lane 0 stages
// them into shared memory with a single TMA bulk copy (cp.async.bulk,
// completion counted in bytes on an mbarrier) while the lanes start on the
// joint chain; each lane then reads its own row with 16-byte shared loads.
// Every wait on the mbarrier is bounded: on timeout the kernel records
// VAPR_ERR_TIMEOUT in a device word (vapr_device_error), drains its own copy
// (again bounded) and stops.
//
// Spheres are visited link by link in a block-wide order built once in
// shared memory, so the sphere table may list spheres in any order.
#include "common.cuh"

namespace vapr {

constexpr int BW_WARPS = 4;
constexpr int BW_BLOCK = 32 * BW_WARPS;
constexpr int BW_BARS = (BW_WARPS + 1) & ~1;  // mbarriers, rounded to 16 bytes
constexpr unsigned long long BW_WAIT_LIMIT = 1ull << 24;  // ~1 s of 64 ns sleeps

__device__ int g_backward_error;  // sticky: first error code, 0 if none

// ---- mbarrier / bulk-copy wrappers (PTX ISA: mbarrier, cp.async.bulk)
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return done != 0;
}
// Bounded wait for the phase to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  for (unsigned long long it = 0; it < BW_WAIT_LIMIT; ++it) {
    if (mbar_test(bar, phase)) return true;
    __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

struct BwArgs {
  RobotArgs r;
  const float* q;
  int64_t n;
  Packed xform, grad, jgrad;
  const float* dcost;
  int kstride;   // float4 per thread in sK (2J rounded up to odd)
  int gbuf;      // bytes of one warp's staging buffer (32 rows)
};

// Streams the words of one packed row, caching the current 16-byte chunk.
// GLOBAL selects read-only global loads; otherwise the row is in shared memory.
template <bool GLOBAL>
struct RowReader {
  const uint8_t* row;
  int chunk = -1;
  uint4 v;
  __device__ __forceinline__ uint32_t word(int w) {
    const int c = w >> 2;
    if (c != chunk) {
      if constexpr (GLOBAL) v = __ldg(reinterpret_cast<const uint4*>(row) + c);
      else v = *(reinterpret_cast<const uint4*>(row) + c);
      chunk = c;
    }
    const int q = w & 3;
    return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
  }
  __device__ __forceinline__ float value(int i, const DevFmt& f) {  // runtime format
    const int w = i / f.k;
    return unpack_slot(word(w), i - w * f.k, f);
  }
  template <int K>
  __device__ __forceinline__ float value_k(int i, const DevFmt& f) {  // compile-time format
    return row_value<K>(i, f, [&](int w) { return word(w); });
  }
};

// GK: format kind of the gradient rows (the hot input), fixed at compile time.
// STAGED: rows come through the TMA staging buffer; otherwise (rows too large
// for shared memory) each lane streams its own row from global memory.
template <int GK, bool STAGED>
__global__ void __launch_bounds__(BW_BLOCK) backward_kernel(BwArgs a) {
  extern __shared__ float4 smem4[];
  const int J = a.r.J, S = a.r.S;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t* gbuf_all = reinterpret_cast<uint8_t*>(smem4);                       // [W][gbuf]
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbuf_all + BW_WARPS * a.gbuf);  // [W]
  float4* sF = reinterpret_cast<float4*>(bars + BW_BARS);          // [3J] rows of F_j
  float4* sSph = sF + 3 * J;                                        // [S] (p, r)
  float4* sK = sSph + S;                                            // [BW_BLOCK][kstride]
  int* sOrder = reinterpret_cast<int*>(sK + BW_BLOCK * a.kstride);  // [S] by link
  int* sStart = sOrder + S;                                         // [J+1]

  for (int i = threadIdx.x; i < 3 * J; i += blockDim.x) {
    const int j = i / 3, d = i - 3 * j;
    const float* F = a.r.joint_fixed + 12 * j;
    sF[i] = make_float4(F[3 * d], F[3 * d + 1], F[3 * d + 2], F[9 + d]);
  }
  for (int s = threadIdx.x; s < S; s += blockDim.x)
    sSph[s] = reinterpret_cast<const float4*>(a.r.sphere_local)[s];
  if (threadIdx.x == 0) {  // stable counting sort of the spheres by link
    for (int j = 0; j <= J; ++j) sStart[j] = 0;
    for (int s = 0; s < S; ++s) ++sStart[clampi(a.r.sphere_link[s], 1, J)];
    for (int j = 1; j <= J; ++j) sStart[j] += sStart[j - 1];
    for (int s = S - 1; s >= 0; --s) sOrder[--sStart[clampi(a.r.sphere_link[s], 1, J)]] = s;
    for (int j = 0; j < J; ++j) sStart[j] = sStart[j + 1];  // first slot of 0-based link j
    sStart[J] = S;
  }
  uint8_t* gbuf = gbuf_all + warp * a.gbuf;
  uint64_t* bar = bars + warp;
  if (STAGED && lane == 0) mbar_init(bar, 1);
  __syncthreads();

  float4* myK = sK + threadIdx.x * a.kstride;
  uint32_t phase = 0;
  const int64_t n_tiles = (a.n + 31) / 32;
  for (int64_t tile = (int64_t)blockIdx.x * BW_WARPS + warp; tile < n_tiles;
       tile += (int64_t)gridDim.x * BW_WARPS) {
    const int64_t c0 = tile * 32;
    const int rows = (int)(a.n - c0 < 32 ? a.n - c0 : 32);
    if (STAGED && lane == 0) {  // stage the warp's gradient rows (contiguous in global)
      const uint32_t bytes = (uint32_t)(rows * a.grad.stride);
      mbar_expect_tx(bar, bytes);
      bulk_g2s(gbuf, a.grad.ptr + c0 * a.grad.stride, bytes, bar);
    }
    const int64_t c = c0 + lane;
    const bool live = lane < rows;
    RowReader<!STAGED> g{STAGED ? gbuf + lane * a.grad.stride
                                : (live ? a.grad.ptr + c * a.grad.stride : a.grad.ptr)};
    RowReader<true> x{a.xform.ptr && live ? a.xform.ptr + c * a.xform.stride : nullptr};
    const float* qc = a.q && live ? a.q + c * J : nullptr;
    float R[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
    float t[3] = {0.f, 0.f, 0.f};
    float F0 = 0.f, F1 = 0.f, F2 = 0.f, M0 = 0.f, M1 = 0.f, M2 = 0.f;
    bool staged = !STAGED;
    for (int j = 0; j < J; ++j) {
      if (live) {
        if (a.xform.ptr) {  // stored transforms: element e of T_j is value 12j + e
#pragma unroll
          for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int k = 0; k < 3; ++k) R[r][k] = x.value(12 * j + 3 * r + k, a.xform.f);
            t[r] = x.value(12 * j + 9 + r, a.xform.f);
          }
        } else {  // recompute T_j = T_{j-1} F_j Rz(q_j)
          const float4 f0 = sF[3 * j], f1 = sF[3 * j + 1], f2 = sF[3 * j + 2];
          float B[3][3], tb[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            B[r][0] = fmaf(R[r][0], f0.x, fmaf(R[r][1], f1.x, R[r][2] * f2.x));
            B[r][1] = fmaf(R[r][0], f0.y, fmaf(R[r][1], f1.y, R[r][2] * f2.y));
            B[r][2] = fmaf(R[r][0], f0.z, fmaf(R[r][1], f1.z, R[r][2] * f2.z));
            tb[r] = fmaf(R[r][0], f0.w, fmaf(R[r][1], f1.w, fmaf(R[r][2], f2.w, t[r])));
          }
          float sn, cs;
          sincosf(qc[j], &sn, &cs);
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            R[r][0] = fmaf(cs, B[r][0], sn * B[r][1]);
            R[r][1] = fmaf(cs, B[r][1], -sn * B[r][0]);
            R[r][2] = B[r][2];
            t[r] = tb[r];
          }
        }
      }
      // axis a_j, b_j = a_j x o_j, and the correction K_j
      const float ax = R[0][2], ay = R[1][2], az = R[2][2];
      const float bx = ay * t[2] - az * t[1];
      const float by = az * t[0] - ax * t[2];
      const float bz = ax * t[1] - ay * t[0];
      const float K = (ax * M0 + ay * M1 + az * M2) - (bx * F0 + by * F1 + bz * F2);
      myK[2 * j] = make_float4(ax, ay, az, K);
      myK[2 * j + 1] = make_float4(bx, by, bz, 0.f);
      if (!staged && sStart[j + 1] > sStart[j]) {  // first link with spheres: need the rows
        const bool ok = mbar_wait(bar, phase);
        if (!__all_sync(0xffffffffu, ok)) {
          if (lane == 0) atomicCAS(&g_backward_error, 0, (int)VAPR_ERR_TIMEOUT);
          mbar_wait(bar, phase);  // let the copy in flight land before leaving
          return;
        }
        staged = true;
      }
      // spheres on link j: accumulate F += G and M += c x G
      if (live) {
        for (int idx = sStart[j]; idx < sStart[j + 1]; ++idx) {
          const int s = sOrder[idx];
          const float g0 = g.template value_k<GK>(3 * s, a.grad.f);
          const float g1 = g.template value_k<GK>(3 * s + 1, a.grad.f);
          const float g2 = g.template value_k<GK>(3 * s + 2, a.grad.f);
          if (g0 == 0.f && g1 == 0.f && g2 == 0.f) continue;
          const float4 p = sSph[s];
          const float c0_ = fmaf(R[0][0], p.x, fmaf(R[0][1], p.y, fmaf(R[0][2], p.z, t[0])));
          const float c1_ = fmaf(R[1][0], p.x, fmaf(R[1][1], p.y, fmaf(R[1][2], p.z, t[1])));
          const float c2_ = fmaf(R[2][0], p.x, fmaf(R[2][1], p.y, fmaf(R[2][2], p.z, t[2])));
          F0 += g0;
          F1 += g1;
          F2 += g2;
          M0 += c1_ * g2 - c2_ * g1;
          M1 += c2_ * g0 - c0_ * g2;
          M2 += c0_ * g1 - c1_ * g0;
        }
      }
    }
    if (!staged) {  // no sphere at all: still consume the phase before reusing the buffer
      const bool ok = mbar_wait(bar, phase);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicCAS(&g_backward_error, 0, (int)VAPR_ERR_TIMEOUT);
        mbar_wait(bar, phase);
        return;
      }
    }
    if (STAGED) phase ^= 1u;
    if (live) {
      const float dc = a.dcost ? a.dcost[c] : 1.f;
      for (int j = 0; j < J; ++j) {
        const float4 ak = myK[2 * j], b = myK[2 * j + 1];
        const float Jj =
            (ak.x * M0 + ak.y * M1 + ak.z * M2) - (b.x * F0 + b.y * F1 + b.z * F2) - ak.w;
        myK[2 * j + 1].w = dc * Jj;
      }
      // packed joint-gradient row (its padding words are written as zero)
      uint4* out = reinterpret_cast<uint4*>(a.jgrad.ptr + c * a.jgrad.stride);
      const int chunks = (int)(a.jgrad.stride / 16);
      for (int cc = 0; cc < chunks; ++cc)
        out[cc] = pack_chunk_dyn(cc, J, a.jgrad.f, [&](int i) { return myK[2 * i + 1].w; });
    }
    // every lane is done with the staged rows before the next copy overwrites them
    __syncwarp();
    if (STAGED) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
}

static size_t bw_smem(const RobotArgs& r, int kstride, int gbuf) {
  return (size_t)BW_WARPS * gbuf + sizeof(uint64_t) * BW_BARS +
         sizeof(float4) * (3 * r.J + r.S + (size_t)BW_BLOCK * kstride) +
         sizeof(int) * (r.S + r.J + 1);
}

int backward_device_error(bool reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_backward_error, sizeof(int)) != cudaSuccess) return -1;
  if (reset && v) {
    const int z = 0;
    cudaMemcpyToSymbol(g_backward_error, &z, sizeof(int));
  }
  return v;
}

cudaError_t launch_backward(const RobotArgs& r, const float* q, Packed xform, Packed grad,
                            const float* dcost, int64_t n, Packed jgrad, cudaStream_t st) {
  BwArgs a;
  a.r = r;
  a.q = q;
  a.n = n;
  a.xform = xform;
  a.grad = grad;
  a.jgrad = jgrad;
  a.dcost = dcost;
  a.kstride = (2 * r.J) | 1;
  // Stage the rows through shared memory when a block's buffers fit and at
  // least one block per SM still fits; otherwise stream them from global.
  void (*kern)(BwArgs) = nullptr;
  size_t smem = 0;
  int per_sm = 0;
  for (int staged = 1; staged >= 0 && per_sm <= 0; --staged) {
    a.gbuf = staged ? (int)(32 * grad.stride) : 0;
    smem = bw_smem(r, a.kstride, a.gbuf);
#define VAPR_BW_CASE(K) \
  case K: kern = staged ? backward_kernel<K, true> : backward_kernel<K, false>; break;
    switch (grad.f.kind) {
      VAPR_BW_CASE(KIND_F32)
      VAPR_BW_CASE(KIND_F16)
      VAPR_BW_CASE(KIND_BF16)
      VAPR_BW_CASE(KIND_E4M3)
      VAPR_BW_CASE(KIND_E5M2)
      VAPR_BW_CASE(KIND_E2M1)
      VAPR_BW_CASE(KIND_E3M2)
      VAPR_BW_CASE(KIND_E2M3)
      default: kern = staged ? backward_kernel<KIND_GENERIC, true>
                             : backward_kernel<KIND_GENERIC, false>;
    }
#undef VAPR_BW_CASE
    per_sm = blocks_per_sm((const void*)kern, BW_BLOCK, smem);
  }
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t tiles = (n + 31) / 32;
  const int64_t blocks = (tiles + BW_WARPS - 1) / BW_WARPS;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  kern<<<(int)(blocks < cap ? blocks : cap), BW_BLOCK, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace vapr
