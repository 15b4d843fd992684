// Collision cost (iteration steps 3-4 of Sec. III-B): robot-environment
// distance queries against oriented cuboids plus robot self-collision
// (Sec. II-B), the per-configuration cost aggregation, and the gradient with
// respect to the sphere centres.  Reads out_spheres (P) and writes the
// per-sphere penetration (D) and dC/dP (G) in their ExMy formats.
//
// One warp per configuration (collision_config in stages.cuh); a block runs
// COLL_WARPS of them at a time over tables staged once in shared memory.
// The environment term is sphere-major: each lane owns up to two spheres and
// walks the cuboids in order, accumulating penetration and gradient in
// registers.  Most sphere/cuboid pairs are far apart, so a sphere runs the
// exact distance for cuboid o only when its centre lies within o's bounding
// sphere grown by r + eta (a skipped pair provably has zero penetration,
// since d_o(c) >= |c - t_o| - |h_o|; SLACK metres cover float32 rounding),
// and the warp skips cuboid o outright when none of its spheres does.
// (Measured on the 40-cuboid particle workload, this plain scheme issues
// fewer instructions than per-link candidate lists or a compacted queue of
// surviving pairs: the bounding test is cheaper than the bookkeeping.)
// With a broad-phase grid (grid.cuh) each sphere visits only the cuboids
// listed for its cell, with the same tests in the same order.
//
// Self pairs: the block groups the pair table by cluster pair (runs of up to
// three spheres of one link, load_self); per configuration, cluster pairs
// whose bounding spheres are apart are skipped and the pairs of the others
// tested in table order (self_pairs in stages.cuh).
//
// Determinism: every sphere adds its terms in cuboid order in one register,
// and a skipped pair would have added exactly zero, so the result of a
// configuration does not depend on the batch it is in or on which pairs the
// bounding test lets through.  Active self pairs are applied sphere-major in
// table order; which lane sums a pair's penetration follows from the
// configuration's own kept cluster pairs.
#include "stages.cuh"

namespace vapr {

constexpr int COLL_WARPS = 8;

struct CollArgs {
  RobotArgs r;
  SceneArgs sc;
  float eta, eta_s, w_c, w_s;
  Packed pos, dist, grad;
  float* cost;
  int64_t n;
  const float* est;  // MASKED: per-sphere distance estimates [n][S]
  float margin;
};

// Carves the block's tables and every warp's working set; keeps warp `mine`'s.
// The self-table scratch lies over the warps' working sets (built first).
__host__ __device__ inline void carve_coll(Bump& b, const RobotArgs& r, int O, RobotSm& rb,
                                           SceneSm& sm, CollWarp& w_mine, int mine,
                                           SelfScratch& scratch) {
  carve_robot(b, r.J, r.S, rb);
  carve_scene(b, O, r.NP, cluster_bound(r.S, r.J), sm);
  Bump t(b.base);
  t.off = b.bytes();
  for (int w = 0; w < COLL_WARPS; ++w) {
    CollWarp cw;
    carve_coll_warp(b, r.S, r.J, cw);
    if (w == mine) w_mine = cw;
  }
  carve_self_scratch(t, r.NP, cluster_bound(r.S, r.J), scratch);
  if (t.off > b.off) b.off = t.off;
}

template <bool MASKED>
__global__ void __launch_bounds__(COLL_WARPS * 32, 4) collision_kernel(CollArgs a) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Bump b(smem4);
  RobotSm rb;
  SceneSm sm;
  CollWarp w;
  SelfScratch scratch;
  carve_coll(b, a.r, a.sc.O, rb, sm, w, wid, scratch);
  load_robot(a.r, rb);
  load_scene(a.r, a.sc, a.eta, a.eta_s, sm);
  __syncthreads();
  load_clusters(a.r.J, a.r.S, rb);
  load_self(a.r, rb, sm, scratch, a.eta_s);
  init_coll_warp(a.r, w, lane);
  __syncthreads();
  const GridHeader* grid = grid_check(a.sc, a.r, a.eta);  // null: visit every cuboid
  const uint2* cells = grid ? grid_cells(a.sc) : nullptr;

  CollOut out;
  out.dist_words = (int)(a.dist.stride / 4);
  out.grad_words = (int)(a.grad.stride / 4);
  // the block owns a contiguous range of configurations; its warps take them
  // one at a time from a shared counter, so uneven per-configuration work
  // evens out within the block (measured: -4 % at 32768 configurations)
  __shared__ int s_next;
  const int64_t per_block = (a.n + gridDim.x - 1) / gridDim.x;
  const int64_t c_begin = blockIdx.x * per_block;
  const int64_t c_end = c_begin + per_block < a.n ? c_begin + per_block : a.n;
  if (threadIdx.x == 0) s_next = 0;
  __syncthreads();
  for (;;) {
    int k = 0;
    if (lane == 0) k = atomicAdd(&s_next, 1);
    k = __shfl_sync(0xffffffffu, k, 0);
    const int64_t c = c_begin + k;
    if (c >= c_end) break;
    out.cost = a.cost ? a.cost + c : nullptr;
    out.dist = a.dist.ptr ? reinterpret_cast<uint32_t*>(a.dist.ptr + c * a.dist.stride) : nullptr;
    out.grad = a.grad.ptr ? reinterpret_cast<uint32_t*>(a.grad.ptr + c * a.grad.stride) : nullptr;
    collision_config<false, MASKED>(a.r, a.sc.O, rb, sm, w,
                                    reinterpret_cast<const uint32_t*>(a.pos.ptr + c * a.pos.stride),
                                    a.pos.f, a.dist.f, a.grad.f, a.eta, a.w_c, a.w_s, out, lane,
                                    MASKED ? a.est + c * a.r.S : nullptr, a.margin, grid, cells);
  }
}

cudaError_t launch_collision(const RobotArgs& r, const SceneArgs& sc, const vapr_cost_params& p,
                             Packed pos, int64_t n, float* cost, Packed dist, Packed grad,
                             cudaStream_t st, const float* est, float margin) {
  CollArgs a;
  a.r = r;
  a.sc = sc;
  a.eta = p.eta;
  a.eta_s = p.eta_self;
  a.w_c = p.w_coll;
  a.w_s = p.w_self;
  a.pos = pos;
  a.dist = dist;
  a.grad = grad;
  a.cost = cost;
  a.n = n;
  a.est = est;
  a.margin = margin;
  Bump b(nullptr);
  RobotSm rb;
  SceneSm sm;
  CollWarp w;
  SelfScratch scratch;
  carve_coll(b, r, sc.O, rb, sm, w, 0, scratch);
  const size_t smem = b.bytes();
  const void* fn = est ? (const void*)collision_kernel<true> : (const void*)collision_kernel<false>;
  const int per_sm = blocks_per_sm(fn, COLL_WARPS * 32, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t blocks = (n + COLL_WARPS - 1) / COLL_WARPS;
  const int grid = (int)(blocks < (int64_t)sm_count() * per_sm ? blocks : (int64_t)sm_count() * per_sm);
  if (est)
    collision_kernel<true><<<grid, COLL_WARPS * 32, smem, st>>>(a);
  else
    collision_kernel<false><<<grid, COLL_WARPS * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace vapr
