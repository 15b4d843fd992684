// Forward kinematics (Sec. II-B robot kinematics; iteration step 2 of
// Sec. III-B): joint configurations -> link transforms -> sphere centres,
// stored in the ExMy format of out_spheres (Sec. III-C).
//
// A block takes tiles of FK_TILE configurations, with two kinds of warps
// and two transform buffers: FK_PRODUCERS warps (one configuration per
// thread) run the joint chains of a tile (fk_chain) into one buffer while
// FK_WRITERS warps write the packed rows of the previous tile from the other
// one (fk_store_pos_staged: lanes take spheres, then words).  The hand-over
// uses named barriers: a buffer's FULL barrier (producers arrive, writers
// wait) and its EMPTY barrier (writers arrive, producers wait before
// refilling it); both sides walk the same tiles, so every arrival has its
// matching wait and no wait can be left open.  (Measured on GB300, 2^20
// configurations of the particle arm: with the per-word row writer of an
// earlier version the writers were the bottleneck and this split did not
// pay; with the staged writer the chains are.)
#include "stages.cuh"

namespace vapr {

constexpr int FK_TILE = 128;
constexpr int FK_PRODUCERS = FK_TILE / 32;
constexpr int FK_WRITERS = 12;
constexpr int FK_THREADS = 32 * (FK_PRODUCERS + FK_WRITERS);
constexpr int BAR_PROD = 1, BAR_FULL = 2, BAR_EMPTY = 4;  // named barriers (0: __syncthreads)

struct FkArgs {
  RobotArgs r;
  const float* q;
  int64_t n;
  Packed pos, xform;
  int tstride;    // float4 per configuration in the transform tile (3J rounded up to odd)
  int stage_len;  // floats of a writer warp's staging row
};

// stage_len: floats of a writer warp's staging row (the packed row's words, >= 3S)
__host__ __device__ inline void carve_fk(Bump& b, int J, int S, int tstride, int stage_len, RobotSm& rb,
                                         float4*& sT, float*& sQ, float*& sStage) {
  carve_robot(b, J, S, rb);
  sT = b.take<float4>((size_t)2 * FK_TILE * tstride);  // two buffers
  sQ = b.take<float>((size_t)FK_TILE * J);
  sStage = b.take<float>((size_t)FK_WRITERS * stage_len);
}

template <int ID, int COUNT>
__device__ __forceinline__ void bar_sync() {
  asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(COUNT) : "memory");
}
template <int ID, int COUNT>
__device__ __forceinline__ void bar_arrive() {
  asm volatile("bar.arrive %0, %1;" ::"n"(ID), "n"(COUNT) : "memory");
}
__device__ __forceinline__ void full_arrive(int buf) {
  if (buf) bar_arrive<BAR_FULL + 1, FK_THREADS>(); else bar_arrive<BAR_FULL, FK_THREADS>();
}
__device__ __forceinline__ void full_wait(int buf) {
  if (buf) bar_sync<BAR_FULL + 1, FK_THREADS>(); else bar_sync<BAR_FULL, FK_THREADS>();
}
__device__ __forceinline__ void empty_arrive(int buf) {
  if (buf) bar_arrive<BAR_EMPTY + 1, FK_THREADS>(); else bar_arrive<BAR_EMPTY, FK_THREADS>();
}
__device__ __forceinline__ void empty_wait(int buf) {
  if (buf) bar_sync<BAR_EMPTY + 1, FK_THREADS>(); else bar_sync<BAR_EMPTY, FK_THREADS>();
}

__global__ void __launch_bounds__(FK_THREADS, 2) fk_kernel(FkArgs a) {
  extern __shared__ float4 smem4[];
  const int J = a.r.J, S = a.r.S;
  Bump b(smem4);
  RobotSm rb;
  float4* sT;
  float *sQ, *sStage;
  carve_fk(b, J, S, a.tstride, a.stage_len, rb, sT, sQ, sStage);
  load_robot(a.r, rb);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n_tiles = (a.n + FK_TILE - 1) / FK_TILE;
  const int my_tiles = blockIdx.x < n_tiles ? (int)((n_tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  const size_t buf_len = (size_t)FK_TILE * a.tstride;

  if (warp < FK_PRODUCERS) {
    const int t = threadIdx.x;
    for (int k = 0; k < my_tiles; ++k) {
      const int64_t base = (blockIdx.x + (int64_t)k * gridDim.x) * FK_TILE;
      const int rows = (int)(a.n - base < FK_TILE ? a.n - base : FK_TILE);
      bar_sync<BAR_PROD, 32 * FK_PRODUCERS>();  // the previous chains are done with sQ
      for (int i = t; i < rows * J; i += 32 * FK_PRODUCERS) sQ[i] = a.q[base * J + i];
      bar_sync<BAR_PROD, 32 * FK_PRODUCERS>();
      if (k >= 2) empty_wait(k & 1);  // the writers are done with this buffer
      if (t < rows) fk_chain(rb, J, sQ + t * J, sT + (k & 1) * buf_len + t * a.tstride);
      full_arrive(k & 1);
    }
    for (int k = my_tiles - 2 > 0 ? my_tiles - 2 : 0; k < my_tiles; ++k)
      empty_wait(k & 1);  // the writers' last two hand-backs
  } else {
    const int wr = warp - FK_PRODUCERS;
    float* stage = sStage + wr * a.stage_len;
    for (int i = 3 * S + lane; i < a.stage_len; i += 32) stage[i] = 0.f;  // padding words stay zero
    __syncwarp();
    for (int k = 0; k < my_tiles; ++k) {
      const int64_t base = (blockIdx.x + (int64_t)k * gridDim.x) * FK_TILE;
      const int rows = (int)(a.n - base < FK_TILE ? a.n - base : FK_TILE);
      const float4* T = sT + (k & 1) * buf_len;
      full_wait(k & 1);
      {
        const int words = (int)(a.pos.stride / 4);
        dispatch_kind(a.pos.f.kind, [&](auto kc) {
          constexpr int K = decltype(kc)::value;
          for (int r = wr; r < rows; r += FK_WRITERS)
            fk_store_pos_staged<K>(rb, S, T + r * a.tstride,
                                   reinterpret_cast<uint32_t*>(a.pos.ptr + (base + r) * a.pos.stride),
                                   words, a.pos.f, lane, stage);
        });
      }
      if (a.xform.ptr) {
        const int words = (int)(a.xform.stride / 4);
        dispatch_kind(a.xform.f.kind, [&](auto kc) {
          constexpr int K = decltype(kc)::value;
          for (int r = wr; r < rows; r += FK_WRITERS)
            fk_store_xform<K>(J, T + r * a.tstride,
                              reinterpret_cast<uint32_t*>(a.xform.ptr + (base + r) * a.xform.stride),
                              words, a.xform.f, lane);
        });
      }
      empty_arrive(k & 1);
    }
  }
}

cudaError_t launch_fk(const RobotArgs& r, const float* q, int64_t n, Packed pos,
                      Packed xform, cudaStream_t st) {
  FkArgs a;
  a.r = r;
  a.q = q;
  a.n = n;
  a.pos = pos;
  a.xform = xform;
  a.tstride = (3 * r.J) | 1;  // odd float4 stride: conflict-free 16-byte stores
  a.stage_len = (int)(pos.stride / 4) > 3 * r.S ? (int)(pos.stride / 4) : 3 * r.S;
  a.stage_len = (a.stage_len + 3) & ~3;
  Bump b(nullptr);
  RobotSm rb;
  float4* sT;
  float *sQ, *sStage;
  carve_fk(b, r.J, r.S, a.tstride, a.stage_len, rb, sT, sQ, sStage);
  const size_t smem = b.bytes();
  const int per_sm = blocks_per_sm((const void*)fk_kernel, FK_THREADS, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t tiles = (n + FK_TILE - 1) / FK_TILE;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  fk_kernel<<<(int)(tiles < cap ? tiles : cap), FK_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace vapr
