// Backward kinematics (iteration step 5 of Sec. III-B): the gradient with
// respect to the sphere centres (grad_out_spheres, Sec. III-C) becomes the
// joint-space gradient (backward_config in stages.cuh).
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
// (again bounded) and stops.  When a block's staging buffers would not fit
// in shared memory, lanes stream their rows from global memory instead.
#include "stages.cuh"

namespace vapr {

constexpr int BW_WARPS = 4;
constexpr int BW_BLOCK = 32 * BW_WARPS;
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
  int kstride;  // float4 per thread in sK (2J rounded up to odd)
  int gbuf;     // bytes of one warp's staging buffer (32 rows), 0 if unstaged
};

__host__ __device__ inline void carve_bw(Bump& b, const BwArgs& a, RobotSm& rb, uint8_t*& gbuf_all,
                                         uint64_t*& bars, float4*& sK) {
  gbuf_all = b.take<uint8_t>((size_t)BW_WARPS * a.gbuf);
  bars = b.take<uint64_t>(BW_WARPS);
  carve_robot(b, a.r.J, a.r.S, rb);
  sK = b.take<float4>((size_t)BW_BLOCK * a.kstride);
}

// GK: format kind of the gradient rows (the hot input), fixed at compile time.
// STAGED: rows come through the TMA staging buffer, else straight from global.
template <int GK, bool STAGED>
__global__ void __launch_bounds__(BW_BLOCK) backward_kernel(BwArgs a) {
  extern __shared__ float4 smem4[];
  const int J = a.r.J;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Bump b(smem4);
  RobotSm rb;
  uint8_t* gbuf_all;
  uint64_t* bars;
  float4* sK;
  carve_bw(b, a, rb, gbuf_all, bars, sK);
  load_robot(a.r, rb);
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
    RowReader<STAGED ? ROW_SHARED : ROW_GLOBAL_RO> g{
        STAGED ? gbuf + lane * a.grad.stride
               : (live ? a.grad.ptr + c * a.grad.stride : a.grad.ptr)};
    RowReader<ROW_GLOBAL_RO> x{a.xform.ptr && live ? a.xform.ptr + c * a.xform.stride : nullptr};
    const float dc = live && a.dcost ? a.dcost[c] : 1.f;
    const bool ok = backward_config<GK, STAGED ? ROW_SHARED : ROW_GLOBAL_RO>(
        rb, J, live, a.q && live ? a.q + c * J : nullptr, x, a.xform.f, g, a.grad.f, dc, myK,
        [&]() {
          if (!STAGED) return true;
          const bool done = mbar_wait(bar, phase);
          if (__all_sync(FULL_MASK, done)) return true;
          if (lane == 0) atomicCAS(&g_backward_error, 0, (int)VAPR_ERR_TIMEOUT);
          mbar_wait(bar, phase);  // let the copy in flight land before leaving
          return false;
        });
    if (!ok) return;
    if (STAGED) phase ^= 1u;
    if (live) backward_store(J, myK, a.jgrad.ptr + c * a.jgrad.stride, a.jgrad.stride, a.jgrad.f);
    // every lane is done with the staged rows before the next copy overwrites them
    __syncwarp();
    if (STAGED) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
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
  // Stage the rows through shared memory when a block's buffers fit at
  // least one block per SM; otherwise stream them from global memory.
  void (*kern)(BwArgs) = nullptr;
  size_t smem = 0;
  int per_sm = 0;
  for (int staged = 1; staged >= 0 && per_sm <= 0; --staged) {
    a.gbuf = staged ? (int)(32 * grad.stride) : 0;
    Bump b(nullptr);
    RobotSm rb;
    uint8_t* gb;
    uint64_t* bars;
    float4* sK;
    carve_bw(b, a, rb, gb, bars, sK);
    smem = b.bytes();
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
