// Forward kinematics (Sec. II-B robot kinematics; iteration step 2 of
// Sec. III-B): joint configurations -> link transforms -> sphere centres,
// stored in the ExMy format of out_spheres (Sec. III-C).
//
// A block takes tiles of FK_TILE configurations.  FK_TILE of its threads
// each run the joint chain of one configuration (fk_chain) and leave the J
// transforms in shared memory; then all its warps write the tile's packed
// rows: warps take rows, lanes take the 32-bit words of a row, so every warp
// store is 128 contiguous bytes.
#include "stages.cuh"

namespace vapr {

constexpr int FK_TILE = 128;
// Threads per block: the chain runs on FK_TILE of them, the row stores on
// all; more warps than configurations hide the store latency (measured on
// GB300: 512 threads take 0.22 ns per configuration at 2^20 configurations,
// 128 threads 0.33 ns).
constexpr int FK_THREADS = 512;

struct FkArgs {
  RobotArgs r;
  const float* q;
  int64_t n;
  Packed pos, xform;
  int tstride;  // float4 per configuration in the transform tile (3J rounded up to odd)
};

__host__ __device__ inline void carve_fk(Bump& b, int J, int S, int tstride, RobotSm& rb,
                                         float4*& sT, float*& sQ) {
  carve_robot(b, J, S, rb);
  sT = b.take<float4>((size_t)FK_TILE * tstride);
  sQ = b.take<float>((size_t)FK_TILE * J);
}

__global__ void __launch_bounds__(FK_THREADS) fk_kernel(FkArgs a) {
  extern __shared__ float4 smem4[];
  const int J = a.r.J, S = a.r.S;
  Bump b(smem4);
  RobotSm rb;
  float4* sT;
  float* sQ;
  carve_fk(b, J, S, a.tstride, rb, sT, sQ);
  load_robot(a.r, rb);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

  const int64_t n_tiles = (a.n + FK_TILE - 1) / FK_TILE;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t base = tile * FK_TILE;
    const int rows = (int)(a.n - base < FK_TILE ? a.n - base : FK_TILE);
    __syncthreads();  // tables ready / previous tile's readers done
    for (int i = threadIdx.x; i < rows * J; i += blockDim.x) sQ[i] = a.q[base * J + i];
    __syncthreads();
    if (threadIdx.x < rows) fk_chain(rb, J, sQ + threadIdx.x * J, sT + threadIdx.x * a.tstride);
    __syncthreads();
    {
      const int words = (int)(a.pos.stride / 4);
      dispatch_kind(a.pos.f.kind, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        for (int r = warp; r < rows; r += nwarps)
          fk_store_pos<K>(rb, S, sT + r * a.tstride,
                          reinterpret_cast<uint32_t*>(a.pos.ptr + (base + r) * a.pos.stride),
                          words, a.pos.f, lane);
      });
    }
    if (a.xform.ptr) {
      const int words = (int)(a.xform.stride / 4);
      dispatch_kind(a.xform.f.kind, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        for (int r = warp; r < rows; r += nwarps)
          fk_store_xform<K>(J, sT + r * a.tstride,
                            reinterpret_cast<uint32_t*>(a.xform.ptr + (base + r) * a.xform.stride),
                            words, a.xform.f, lane);
      });
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
  Bump b(nullptr);
  RobotSm rb;
  float4* sT;
  float* sQ;
  carve_fk(b, r.J, r.S, a.tstride, rb, sT, sQ);
  const size_t smem = b.bytes();
  const int per_sm = blocks_per_sm((const void*)fk_kernel, FK_THREADS, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t tiles = (n + FK_TILE - 1) / FK_TILE;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  fk_kernel<<<(int)(tiles < cap ? tiles : cap), FK_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace vapr
