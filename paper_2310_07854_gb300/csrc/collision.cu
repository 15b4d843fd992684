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
// listed for its cell (those it can penetrate) and runs the exact term on
// them alone, in the same order.
//
// Self pairs: the block groups the pair table by cluster pair (runs of up to
// CL spheres of one link, load_self), or copies the robot's prebuilt
// tables (load_block_tables: a hash-checked copy instead of about 10 us
// of building per block); per configuration, cluster pairs whose bounding
// spheres are apart are skipped and the pairs of the others tested in
// table order (self_pairs in stages.cuh).
//
// Determinism: every sphere adds its terms in cuboid order in one register,
// and a skipped pair would have added exactly zero, so the result of a
// configuration does not depend on the batch it is in or on which pairs the
// bounding test lets through.  The self terms' gradients are summed in
// fixed point (integer sums, the same in any order); which lane sums a
// pair's penetration follows from the configuration's own kept cluster
// pairs.
#include <map>
#include <mutex>

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
  int slot;          // ticket slot, or -1: each block takes a contiguous range
};

// Ticket scheduling: the warps of a launch take configurations one at a
// time from a counter of their own (measured at 262,144 configurations:
// -9 % against contiguous ranges per block, since faster SMs take more).
// The counters are slots of a fixed device array, and the last block of a
// launch to finish puts its slot back to zero.  Launches made outside
// stream capture take slots round-robin, skipping any slot whose previous
// launch has not completed (an event recorded after each launch); a
// captured launch, which may be replayed at any later time, gets a slot of
// its own for good.  With no slot free, a launch falls back to contiguous
// ranges per block.
constexpr int SCHED_ROUND = 1024, SCHED_CAPTURED = 4096;
struct SchedSlot {
  unsigned int next, done;
};
__device__ SchedSlot g_sched[SCHED_ROUND + SCHED_CAPTURED];

// Carves the block's tables and every warp's working set; keeps warp `mine`'s.
// The self-table scratch lies over the warps' working sets (built first).
__host__ __device__ inline void carve_coll(Bump& b, const RobotArgs& r, int O, RobotSm& rb,
                                           SceneSm& sm, CollWarp& w_mine, int mine,
                                           SelfScratch& scratch) {
  carve_robot(b, r.J, r.S, rb);
  carve_scene(b, O, r.NP, cluster_bound(r.S, r.J), sm);
  Bump t(b.base);
  t.off = b.bytes();
  carve_warps(b, COLL_WARPS, mine, [&](Bump& wb) { carve_coll_warp(wb, r.S, r.J, w_mine); });
  carve_self_scratch(t, r.NP, cluster_bound(r.S, r.J), r.S, scratch);
  if (t.off > b.off) b.off = t.off;
}

// F32: P, D and G are float32 (the loop body without the other formats'
// code, which keeps it within the instruction cache).
template <bool MASKED, bool F32>
__global__ void __launch_bounds__(COLL_WARPS * 32, 4) collision_kernel(CollArgs a) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Bump b(smem4);
  RobotSm rb;
  SceneSm sm;
  CollWarp w;
  SelfScratch scratch;
  carve_coll(b, a.r, a.sc.O, rb, sm, w, wid, scratch);
  __shared__ int s_next;
  if (threadIdx.x == 0) s_next = 0;  // (visible after the prologue's barriers)
  // null grid: visit every cuboid
  const GridHeader* grid = load_block_tables(a.r, a.sc, a.eta, a.eta_s, rb, sm, scratch, w);
  const uint2* cells = grid ? grid_cells(a.sc) : nullptr;

  CollOut out;
  out.dist_words = (int)(a.dist.stride / 4);
  out.grad_words = (int)(a.grad.stride / 4);
  // configurations come one at a time per warp: from the launch's ticket
  // slot, or (no slot) from a shared counter over the block's contiguous range
  const int64_t per_block = (a.n + gridDim.x - 1) / gridDim.x;
  const int64_t c_begin = a.slot >= 0 ? 0 : blockIdx.x * per_block;
  const int64_t c_end = a.slot >= 0 ? a.n : (c_begin + per_block < a.n ? c_begin + per_block : a.n);
  grid_dependents_may_launch();  // (the next stage waits for this grid to finish)
  grid_dependency_wait();        // the P rows are complete from here on
  auto draw = [&]() -> unsigned int {  // lane 0's ticket (the other lanes get 0)
    if (lane != 0) return 0u;
    return a.slot >= 0 ? atomicAdd(&g_sched[a.slot].next, 1u) : (unsigned int)atomicAdd(&s_next, 1);
  };
  unsigned int k_next = draw();
  for (;;) {
    const unsigned int k = __shfl_sync(0xffffffffu, k_next, 0);
    const int64_t c = c_begin + k;
    if (c >= c_end) break;
    // the next ticket is drawn now and read after this configuration: its
    // latency overlaps this configuration's work
    k_next = draw();
    out.cost = a.cost ? a.cost + c : nullptr;
    out.dist = a.dist.ptr ? reinterpret_cast<uint32_t*>(a.dist.ptr + c * a.dist.stride) : nullptr;
    out.grad = a.grad.ptr ? reinterpret_cast<uint32_t*>(a.grad.ptr + c * a.grad.stride) : nullptr;
    // between the environment and self terms (the next ticket is back by
    // then): lanes prefetch the next configuration's P row into L1
    auto prefetch_next = [&]() {
      const int64_t cn = c_begin + __shfl_sync(0xffffffffu, k_next, 0);
      if (cn < c_end && 128 * lane < a.pos.stride)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.pos.ptr + cn * a.pos.stride + 128 * lane));
    };
    collision_config<false, MASKED, F32>(a.r, a.sc.O, rb, sm, w,
                                    reinterpret_cast<const uint32_t*>(a.pos.ptr + c * a.pos.stride),
                                    a.pos.f, a.dist.f, a.grad.f, a.eta, a.w_c, a.w_s, out, lane,
                                    MASKED ? a.est + c * a.r.S : nullptr, a.margin, grid, cells, prefetch_next);
  }
  if (a.slot >= 0) {  // every warp of this block has drawn its last ticket
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(&g_sched[a.slot].done, 1u) == gridDim.x - 1) {
      atomicExch(&g_sched[a.slot].next, 0u);  // the whole launch is past its draws
      atomicExch(&g_sched[a.slot].done, 0u);
    }
  }
}

// Host side of the ticket slots, per device.
struct SchedPool {
  std::mutex mu;
  unsigned int next = 0;
  int captured = 0;
  cudaEvent_t done[SCHED_ROUND] = {};
};

static SchedPool& sched_pool() {
  static std::mutex m;
  static std::map<int, SchedPool*> pools;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(m);
  SchedPool*& p = pools[dev];
  if (!p) p = new SchedPool;  // kept for the life of the process
  return *p;
}

// Picks the ticket slot of a launch on stream st (with P.mu held), or -1;
// *rec receives the event to record after the launch (round-robin slots).
static int sched_slot(SchedPool& P, cudaStream_t st, int64_t n, cudaEvent_t* rec) {
  *rec = nullptr;
  if (n > (int64_t)INT32_MAX) return -1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (cs == cudaStreamCaptureStatusActive) return P.captured < SCHED_CAPTURED ? SCHED_ROUND + P.captured++ : -1;
  if (cs != cudaStreamCaptureStatusNone) return -1;
  for (int t = 0; t < SCHED_ROUND; ++t) {
    const int k = (int)(P.next++ % SCHED_ROUND);
    if (!P.done[k]) {
      if (cudaEventCreateWithFlags(&P.done[k], cudaEventDisableTiming) != cudaSuccess) {
        P.done[k] = nullptr;
        cudaGetLastError();
        return -1;
      }
    } else if (cudaEventQuery(P.done[k]) != cudaSuccess) {  // still running (or unknown)
      cudaGetLastError();
      continue;
    }
    *rec = P.done[k];
    return k;
  }
  return -1;
}

cudaError_t launch_collision(const RobotArgs& r, const SceneArgs& sc, const vapr_cost_params& p,
                             Packed pos, int64_t n, float* cost, Packed dist, Packed grad,
                             cudaStream_t st, const float* est, float margin, bool overlap) {
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
  const bool f32 = pos.f.kind == KIND_F32 && (!dist.ptr || dist.f.kind == KIND_F32) &&
                   (!grad.ptr || grad.f.kind == KIND_F32);
  auto kernel = est ? (f32 ? collision_kernel<true, true> : collision_kernel<true, false>)
                    : (f32 ? collision_kernel<false, true> : collision_kernel<false, false>);
  const int per_sm = blocks_per_sm((const void*)kernel, COLL_WARPS * 32, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t blocks = (n + COLL_WARPS - 1) / COLL_WARPS;
  const int grid = (int)(blocks < (int64_t)sm_count() * per_sm ? blocks : (int64_t)sm_count() * per_sm);
  SchedPool& P = sched_pool();
  std::lock_guard<std::mutex> hold(P.mu);  // slot choice, launch and its event together
  cudaEvent_t rec;
  a.slot = sched_slot(P, st, n, &rec);
  cudaError_t e = launch_after(overlap, kernel, grid, COLL_WARPS * 32, smem, st, a);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess && rec) return cudaEventRecord(rec, st);
  return e;
}

}  // namespace vapr
