// Uneven multi-problem evaluation in one persistent launch.
//
// Many planning problems -- different numbers of trajectories, horizons and
// cuboids, and per-problem sphere radii -- are cut into work items of `tile`
// configurations.  A host-built plan holds the problem descriptors, the
// work list (longest first), one ready word per problem and a work counter.
// Each resident block repeatedly claims the next item and runs the whole
// path on it with the same stage functions as the single-problem kernels:
//   FK (thread per configuration)  -> packed P rows in the block's scratch
//   collision (warp per configuration) -> cost, D to the caller, packed G
//                                          rows in the block's scratch
//   backward (thread per configuration) -> packed J rows to the caller
// P and G never leave the block's small scratch slice, which stays in L2.
// A block reloads the robot and scene tables only when the problem changes.
//
// A deferred problem waits for vapr_batched_publish; the wait is bounded
// (wait_limit_us), after which the item is skipped and VAPR_ERR_TIMEOUT is
// recorded in the caller's status word.
#include <algorithm>
#include <cstring>
#include <vector>

#include "stages.cuh"

namespace vapr {

constexpr int BT_WARPS = 8;
constexpr int BT_BLOCK = 32 * BT_WARPS;

struct ProblemDev {
  RobotArgs r;
  SceneArgs sc;
  float eta, eta_s, w_c, w_s;
  const float* q;
  int64_t n;
  const float* dcost;
  float* cost;
  uint8_t* dist;
  uint8_t* jgrad;
  int64_t pos_stride, dist_stride, grad_stride, jgrad_stride;
};

struct WorkItem {
  int32_t problem;
  int32_t rows;
  int64_t first;
};

struct BatchArgs {
  const ProblemDev* probs;
  const WorkItem* items;
  int n_items;
  int* counter;
  const int* ready;
  uint8_t* scratch;        // [grid][tile * (pos_row + grad_row)]
  int64_t scratch_block;   // bytes per block
  int64_t scratch_grad;    // offset of the G rows within a block's slice
  int tile, maxJ, maxS, maxO, maxNP;
  DevFmt fP, fD, fG, fJ;
  int* status;
  long long wait_ns;
};

// Host handle stored in vapr_batch_plan::opaque.
struct PlanHost {
  uint64_t magic;
  BatchArgs args;
  int grid;
  size_t smem;
  int n_problems;
  int kind_g;
};
static_assert(sizeof(PlanHost) <= sizeof(vapr_batch_plan), "plan handle too small");
constexpr uint64_t PLAN_MAGIC = 0x5641505242415443ull;

// The self-table scratch lies over the warps' working sets, sU and sQ (not
// live while a problem's tables are built).
__host__ __device__ inline void carve_batch(Bump& b, const BatchArgs& a, RobotSm& rb, SceneSm& sm,
                                            CollWarp& w_mine, int mine, float4*& sU, float*& sQ,
                                            int*& sItem, SelfScratch& scratch) {
  carve_robot(b, a.maxJ, a.maxS, rb);
  carve_scene(b, a.maxO, a.maxNP, cluster_bound(a.maxS, a.maxJ), sm);
  Bump t(b.base);
  t.off = b.bytes();
  carve_warps(b, BT_WARPS, mine, [&](Bump& wb) { carve_coll_warp(wb, a.maxS, a.maxJ, w_mine); });
  const int tstride = (3 * a.maxJ) | 1, kstride = (2 * a.maxJ) | 1;
  sU = b.take<float4>((size_t)a.tile * (tstride > kstride ? tstride : kstride));  // T, then K
  sQ = b.take<float>((size_t)a.tile * a.maxJ);
  carve_self_scratch(t, a.maxNP, cluster_bound(a.maxS, a.maxJ), a.maxS, scratch);
  if (t.off > b.off) b.off = t.off;
  sItem = b.take<int>(4);
}

__host__ __device__ inline int64_t packed_stride(int row_len, const DevFmt& f) {
  const int64_t words = (row_len + f.k - 1) / f.k;
  return ((4 * words + 15) / 16) * 16;
}

template <int GK>
__global__ void __launch_bounds__(BT_BLOCK) batched_kernel(BatchArgs a) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Bump b(smem4);
  RobotSm rb;
  SceneSm sm;
  CollWarp w;
  float4* sU;
  float* sQ;
  int* sItem;
  SelfScratch self_scr;
  carve_batch(b, a, rb, sm, w, warp, sU, sQ, sItem, self_scr);
  uint8_t* scratch = a.scratch + (int64_t)blockIdx.x * a.scratch_block;
  int cur = -1;
  const GridHeader* grid = nullptr;  // the current problem's scene grid, when usable
  const uint2* cells = nullptr;
  for (;;) {
    if (threadIdx.x == 0) {
      const int item = atomicAdd(a.counter, 1);
      int ok = 1;
      if (item < a.n_items) {  // bounded wait for the problem to be published
        const int p = a.items[item].problem;
        const volatile int* rd = a.ready + p;
        const long long t0 = clock64();
        long long spins = 0;
        while (*rd == 0) {
          __nanosleep(1000);
          // clock64 counts SM cycles; spins bounds the loop even if the clock stalls
          if (++spins > a.wait_ns / 1000 + 1 || clock64() - t0 > 4 * a.wait_ns) {
            ok = 0;
            atomicCAS(a.status, 0, (int)VAPR_ERR_TIMEOUT);
            break;
          }
        }
      }
      sItem[0] = item;
      sItem[1] = ok;
    }
    __syncthreads();
    const int item = sItem[0], ok = sItem[1];
    if (item >= a.n_items) break;
    if (!ok) {
      __syncthreads();
      continue;
    }
    const WorkItem it = a.items[item];
    const ProblemDev& P = a.probs[it.problem];
    const int J = P.r.J, S = P.r.S, rows = it.rows;
    if (it.problem != cur) {  // this problem's arm and obstacles into shared memory
      load_scene(P.r, P.sc, P.eta, P.eta_s, sm);
      load_robot_self(P.r, rb, sm, self_scr, P.eta_s);
      init_coll_warp(P.r, w, lane);
      grid = grid_check(P.sc, P.r, P.eta);  // block-wide; null: every cuboid
      cells = grid ? grid_cells(P.sc) : nullptr;
      cur = it.problem;
    }
    const int tstride = (3 * J) | 1, kstride = (2 * J) | 1;
    uint8_t* prow0 = scratch;
    uint8_t* grow0 = scratch + a.scratch_grad;
    // ---- FK: chains into sU, packed P rows into scratch
    for (int i = threadIdx.x; i < rows * J; i += blockDim.x) sQ[i] = P.q[it.first * J + i];
    __syncthreads();
    if (threadIdx.x < rows) fk_chain(rb, J, sQ + threadIdx.x * J, sU + threadIdx.x * tstride);
    __syncthreads();
    dispatch_kind(a.fP.kind, [&](auto kc) {
      constexpr int K = decltype(kc)::value;
      for (int r = warp; r < rows; r += BT_WARPS)
        fk_store_pos<K>(rb, S, sU + r * tstride,
                        reinterpret_cast<uint32_t*>(prow0 + r * P.pos_stride),
                        (int)(P.pos_stride / 4), a.fP, lane);
    });
    __syncthreads();
    // ---- collision: one warp per configuration
    CollOut out;
    out.dist_words = (int)(P.dist_stride / 4);
    out.grad_words = (int)(P.grad_stride / 4);
    for (int r = warp; r < rows; r += BT_WARPS) {
      const int64_t c = it.first + r;
      out.cost = P.cost + c;
      out.dist = P.dist ? reinterpret_cast<uint32_t*>(P.dist + c * P.dist_stride) : nullptr;
      out.grad = reinterpret_cast<uint32_t*>(grow0 + r * P.grad_stride);
      collision_config<true>(P.r, P.sc.O, rb, sm, w,
                             reinterpret_cast<const uint32_t*>(prow0 + r * P.pos_stride), a.fP, a.fD,
                             a.fG, P.eta, P.w_c, P.w_s, out, lane, nullptr, 0.f, grid, cells);
    }
    __syncthreads();
    // ---- backward: one thread per configuration, G from scratch
    if (threadIdx.x < rows) {
      const int r = threadIdx.x;
      const int64_t c = it.first + r;
      RowReader<ROW_GLOBAL_COHERENT> g{grow0 + r * P.grad_stride};
      RowReader<ROW_GLOBAL_RO> x{nullptr};
      float4* myK = sU + r * kstride;
      backward_config<GK>(rb, J, true, sQ + r * J, x, a.fJ, g, a.fG, P.dcost ? P.dcost[c] : 1.f, myK, 1,
                          [&](int j, float v) { myK[2 * j + 1].w = v; });
      backward_store(J, [&](int i) { return myK[2 * i + 1].w; }, P.jgrad + c * P.jgrad_stride,
                     P.jgrad_stride, a.fJ);
    }
    __syncthreads();
  }
}

static void (*batched_for(int kind))(BatchArgs) {
  switch (kind) {
    case KIND_F32: return batched_kernel<KIND_F32>;
    case KIND_F16: return batched_kernel<KIND_F16>;
    case KIND_BF16: return batched_kernel<KIND_BF16>;
    case KIND_E4M3: return batched_kernel<KIND_E4M3>;
    case KIND_E5M2: return batched_kernel<KIND_E5M2>;
    case KIND_E2M1: return batched_kernel<KIND_E2M1>;
    case KIND_E3M2: return batched_kernel<KIND_E3M2>;
    case KIND_E2M3: return batched_kernel<KIND_E2M3>;
    default: return batched_kernel<KIND_GENERIC>;
  }
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Everything the plan needs, computed on the host.
struct Layout {
  std::vector<ProblemDev> probs;
  std::vector<WorkItem> items;
  BatchArgs args;
  int grid = 0;
  size_t smem = 0;
  size_t off_items = 0, off_ready = 0, off_counter = 0, off_scratch = 0, total = 0;
  void (*kern)(BatchArgs) = nullptr;
};

static vapr_status layout(const vapr_problem* pr, int32_t np, const vapr_format_table* table,
                          const vapr_batch_tuning* tuning, Layout& L) {
  if (!pr || np < 1 || !tuning) return VAPR_ERR_INVALID_ARG;
  vapr_status st = check_table(table);
  if (st != VAPR_OK) return st;
  const int tile = tuning->tile;
  if (tile != 32 && tile != 64 && tile != 128 && tile != 256) return VAPR_ERR_INVALID_ARG;
  if (tuning->wait_limit_us < 0) return VAPR_ERR_INVALID_ARG;
  BatchArgs& a = L.args;
  std::memset(&a, 0, sizeof(a));
  a.tile = tile;
  a.fP = make_dev_fmt(table->pos);
  a.fD = make_dev_fmt(table->dist);
  a.fG = make_dev_fmt(table->grad);
  a.fJ = make_dev_fmt(table->jgrad);
  a.wait_ns = 1000ll * (tuning->wait_limit_us ? tuning->wait_limit_us : 1000000);
  auto al = [](const void* p, uintptr_t k) { return ((uintptr_t)p % k) == 0; };
  for (int32_t i = 0; i < np; ++i) {
    const vapr_problem& p = pr[i];
    ProblemDev d;
    std::memset(&d, 0, sizeof(d));
    if ((st = check_robot(&p.robot, &d.r)) != VAPR_OK) return st;
    if (p.scene.n_cuboids < 0 || p.n < 0 || p.reserved != 0 || (p.deferred != 0 && p.deferred != 1))
      return VAPR_ERR_INVALID_ARG;
    if (p.scene.n_cuboids > VAPR_MAX_CUBOIDS || p.n > VAPR_MAX_CONFIGS) return VAPR_ERR_TOO_LARGE;
    if (p.scene.n_cuboids > 0 && (!p.scene.pose || !p.scene.half_ext)) return VAPR_ERR_INVALID_ARG;
    if (p.n > 0 && (!p.q || !p.cost || !p.jgrad_packed)) return VAPR_ERR_INVALID_ARG;
    if ((p.scene.n_cuboids > 0 && (!al(p.scene.pose, 16) || !al(p.scene.half_ext, 4))) ||
        !al(p.q, 4) || !al(p.cost, 4) || !al(p.dcost, 4) || !al(p.dist_packed, 16) ||
        !al(p.jgrad_packed, 16) || !al(p.scene.grid, 16))
      return VAPR_ERR_MISALIGNED;
    d.sc.O = p.scene.n_cuboids;
    d.sc.pose = p.scene.pose;
    d.sc.half = p.scene.half_ext;
    d.sc.grid = p.scene.grid;  // checked against the problem on the device, as everywhere
    d.eta = p.params.eta;
    d.eta_s = p.params.eta_self;
    d.w_c = p.params.w_coll;
    d.w_s = p.params.w_self;
    d.q = p.q;
    d.n = p.n;
    d.dcost = p.dcost;
    d.cost = p.cost;
    d.dist = (uint8_t*)p.dist_packed;
    d.jgrad = (uint8_t*)p.jgrad_packed;
    d.pos_stride = (int64_t)row_bytes(3 * (int64_t)d.r.S, table->pos);
    d.dist_stride = (int64_t)row_bytes(d.r.S, table->dist);
    d.grad_stride = (int64_t)row_bytes(3 * (int64_t)d.r.S, table->grad);
    d.jgrad_stride = (int64_t)row_bytes(d.r.J, table->jgrad);
    a.maxJ = std::max(a.maxJ, d.r.J);
    a.maxS = std::max(a.maxS, d.r.S);
    a.maxO = std::max(a.maxO, d.sc.O);
    a.maxNP = std::max(a.maxNP, d.r.NP);
    L.probs.push_back(d);
    for (int64_t f = 0; f < p.n; f += tile) {
      WorkItem w;
      w.problem = i;
      w.rows = (int32_t)std::min<int64_t>(tile, p.n - f);
      w.first = f;
      L.items.push_back(w);
    }
  }
  // longest first: estimated cost of an item ~ rows * (cuboids + self pairs / 16 + spheres)
  auto cost = [&](const WorkItem& w) {
    const ProblemDev& d = L.probs[w.problem];
    return (double)w.rows * (d.sc.O + d.r.NP / 16.0 + d.r.S);
  };
  std::stable_sort(L.items.begin(), L.items.end(),
                   [&](const WorkItem& x, const WorkItem& y) { return cost(x) > cost(y); });
  a.n_items = (int)L.items.size();
  // shared memory and resident blocks
  Bump b(nullptr);
  RobotSm rb;
  SceneSm sm;
  CollWarp w;
  float4* sU;
  float* sQ;
  int* sItem;
  SelfScratch scratch;
  carve_batch(b, a, rb, sm, w, 0, sU, sQ, sItem, scratch);
  L.smem = b.bytes();
  L.kern = batched_for(a.fG.kind);
  const int per_sm = blocks_per_sm((const void*)L.kern, BT_BLOCK, L.smem);
  if (per_sm <= 0) return VAPR_ERR_TOO_LARGE;
  L.grid = sm_count() * per_sm;
  if (a.n_items > 0 && L.grid > a.n_items) L.grid = a.n_items;
  if (L.grid < 1) L.grid = 1;
  // device layout
  const int64_t prow = (int64_t)row_bytes(3 * (int64_t)a.maxS, table->pos);
  const int64_t grow = (int64_t)row_bytes(3 * (int64_t)a.maxS, table->grad);
  a.scratch_grad = (int64_t)align256((size_t)(tile * prow));
  a.scratch_block = (int64_t)align256((size_t)(a.scratch_grad + tile * grow));
  L.off_items = align256(sizeof(ProblemDev) * L.probs.size());
  L.off_ready = L.off_items + align256(sizeof(WorkItem) * std::max<size_t>(1, L.items.size()));
  L.off_counter = L.off_ready + align256(sizeof(int) * L.probs.size());
  L.off_scratch = L.off_counter + 256;
  L.total = L.off_scratch + (size_t)L.grid * (size_t)a.scratch_block;
  return VAPR_OK;
}

}  // namespace vapr

using namespace vapr;

extern "C" {

size_t vapr_batched_plan_bytes(const vapr_problem* problems, int32_t n_problems,
                               const vapr_format_table* table, const vapr_batch_tuning* tuning) {
  Layout L;
  return layout(problems, n_problems, table, tuning, L) == VAPR_OK ? L.total : 0;
}

vapr_status vapr_batched_plan(const vapr_problem* problems, int32_t n_problems,
                              const vapr_format_table* table, const vapr_batch_tuning* tuning,
                              void* plan_dev, size_t plan_bytes, vapr_batch_plan* plan) {
  if (!plan || !plan_dev) return VAPR_ERR_INVALID_ARG;
  if (((uintptr_t)plan_dev % 256) != 0) return VAPR_ERR_MISALIGNED;
  Layout L;
  vapr_status st = layout(problems, n_problems, table, tuning, L);
  if (st != VAPR_OK) return st;
  if (plan_bytes < L.total) return VAPR_ERR_INVALID_ARG;
  uint8_t* base = (uint8_t*)plan_dev;
  std::vector<int> ready(L.probs.size());
  for (size_t i = 0; i < ready.size(); ++i) ready[i] = problems[i].deferred ? 0 : 1;
  cudaError_t e = cudaMemcpy(base, L.probs.data(), sizeof(ProblemDev) * L.probs.size(),
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !L.items.empty())
    e = cudaMemcpy(base + L.off_items, L.items.data(), sizeof(WorkItem) * L.items.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(base + L.off_ready, ready.data(), sizeof(int) * ready.size(),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_status(e);
  PlanHost h;
  std::memset(&h, 0, sizeof(h));
  h.magic = PLAN_MAGIC;
  h.args = L.args;
  h.args.probs = (const ProblemDev*)base;
  h.args.items = (const WorkItem*)(base + L.off_items);
  h.args.ready = (const int*)(base + L.off_ready);
  h.args.counter = (int*)(base + L.off_counter);
  h.args.scratch = base + L.off_scratch;
  h.grid = L.grid;
  h.smem = L.smem;
  h.n_problems = n_problems;
  h.kind_g = L.args.fG.kind;
  std::memset(plan, 0, sizeof(*plan));
  std::memcpy(plan, &h, sizeof(h));
  return VAPR_OK;
}

vapr_status vapr_batched_publish(const vapr_batch_plan* plan, int32_t problem, void* stream) {
  if (!plan) return VAPR_ERR_INVALID_ARG;
  PlanHost h;
  std::memcpy(&h, plan, sizeof(h));
  if (h.magic != PLAN_MAGIC || problem < 0 || problem >= h.n_problems) return VAPR_ERR_INVALID_ARG;
  return cuda_status(cudaMemsetAsync((void*)(h.args.ready + problem), 1, sizeof(int),
                                     (cudaStream_t)stream));
}

vapr_status vapr_batched_eval(const vapr_batch_plan* plan, int32_t* dev_status, void* stream) {
  if (!plan || !dev_status) return VAPR_ERR_INVALID_ARG;
  if (((uintptr_t)dev_status % 4) != 0) return VAPR_ERR_MISALIGNED;
  PlanHost h;
  std::memcpy(&h, plan, sizeof(h));
  if (h.magic != PLAN_MAGIC) return VAPR_ERR_INVALID_ARG;
  h.args.status = dev_status;
  const cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(h.args.counter, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev_status, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return cuda_status(e);
  if (h.args.n_items == 0) return VAPR_OK;
  void (*kern)(BatchArgs) = batched_for(h.kind_g);
  if (blocks_per_sm((const void*)kern, BT_BLOCK, h.smem) <= 0) return cuda_status(cudaErrorInvalidConfiguration);
  kern<<<h.grid, BT_BLOCK, h.smem, st>>>(h.args);
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
