// The whole cost-and-gradient step of a batch in one kernel, with the
// sphere centres P and their gradient G kept on the SM: the upper bound of
// what not storing those tensors buys (the staged path stores them in
// their ExMy formats, Sec. III-C).  It computes what vapr_fk,
// vapr_collision_cost and vapr_backward compute (iteration steps 2-5 of
// Sec. III-B):
//   FK         T_j = T_{j-1} F_j Rz(q_j), c_s = T_link(s) [p_s; 1]
//   collision  C = w_c sum_s D_s + w_s sum P_ij, G = dC/dc
//   backward   J_j = dC (a_j . M_{>=j} - b_j . F_{>=j}), F = sum G_s,
//              M = sum c_s x G_s over the spheres on links >= j
// and rounds P and G to the table's formats in registers, as storing and
// loading them would.
//
// A block of FU_WARPS warps takes a contiguous range of mini-tiles of
// FU_MT = 8 configurations, which its warps draw one at a time from a block
// counter.  A warp runs its mini-tile's joint chains (lanes 0..7, one
// configuration each) into its own transform rows in shared memory, then
// takes the configurations one by one: it computes the sphere centres from
// the transforms (lanes over spheres), runs the collision stage's
// environment and self terms on them (collision_terms: the same code, so
// cost and D are the staged path's bit for bit), writes cost and D, and
// runs the backward pass cooperatively: lanes form each sphere's F = G and
// M = c x G (G rounded to its format), lane l sums link l's in index order,
// the suffix sums over links run from the last link down, and lane j forms
// J_j.  (The staged backward sums in one running pass over all spheres, so
// J agrees with it to rounding, not bit for bit.)  A first version shared
// 32-configuration tiles across the block, behind block barriers: warps
// idled at each tile's end, 0.61 of the staged speed at 2^20.
#include "stages.cuh"

namespace vapr {

constexpr int FU_WARPS = 8;
constexpr int FU_MT = 8;  // configurations per mini-tile (a warp's chains)

struct FusedArgs {
  RobotArgs r;
  SceneArgs sc;
  float eta, eta_s, w_c, w_s;
  const float* q;
  const float* dcost;
  int64_t n;
  DevFmt fP, fG;
  Packed dist, jgrad;
  float* cost;
  int tstride;  // float4 per configuration in the transform rows (3J rounded up to odd)
  int64_t mt_per_block;  // mini-tiles of each block's contiguous range
};

struct FusedWarp {
  float4* C;    // [S] centres before rounding to the P format; then c x G
  float4* lk;   // [2 VAPR_MAX_JOINTS] per-link sums (F, -), (M, -)
  float* jrow;  // [VAPR_MAX_JOINTS] this configuration's joint gradient
  float4* T;    // [FU_MT][tstride] transforms of the mini-tile
};

__host__ __device__ inline void carve_fused(Bump& b, const FusedArgs& a, RobotSm& rb, SceneSm& sm,
                                            CollWarp& w_mine, FusedWarp& f_mine, int mine,
                                            SelfScratch& scratch) {
  const RobotArgs& r = a.r;
  carve_robot(b, r.J, r.S, rb);
  carve_scene(b, a.sc.O, r.NP, cluster_bound(r.S, r.J), sm);
  Bump t(b.base);
  t.off = b.bytes();
  for (int w = 0; w < FU_WARPS; ++w) {
    CollWarp cw;
    carve_coll_warp(b, r.S, r.J, cw);
    FusedWarp fw;
    fw.C = b.take<float4>(r.S);
    fw.lk = b.take<float4>(2 * VAPR_MAX_JOINTS);
    fw.jrow = b.take<float>(VAPR_MAX_JOINTS);
    if (w == mine) {
      w_mine = cw;
      f_mine = fw;
    }
  }
  carve_self_scratch(t, r.NP, cluster_bound(r.S, r.J), scratch);  // over the warps' sets (built first)
  if (t.off > b.off) b.off = t.off;
  for (int w = 0; w < FU_WARPS; ++w) {  // (after the scratch: written once the tables are built)
    float4* T = b.take<float4>((size_t)FU_MT * a.tstride);
    if (w == mine) f_mine.T = T;
  }
}

// dec(enc(x)) in format f: the value a stored and reloaded x has.
__device__ __forceinline__ float round_trip(float x, const DevFmt& f) {
  return f.kind == KIND_F32 ? x : decode(encode(x, f), f);
}

__global__ void __launch_bounds__(FU_WARPS * 32, 4) fused_kernel(FusedArgs a) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int J = a.r.J, S = a.r.S;
  Bump b(smem4);
  RobotSm rb;
  SceneSm sm;
  CollWarp w;
  FusedWarp fw;
  SelfScratch scratch;
  carve_fused(b, a, rb, sm, w, fw, wid, scratch);
  load_robot(a.r, rb);
  load_scene(a.r, a.sc, a.eta, a.eta_s, sm);
  __syncthreads();
  load_clusters(J, S, rb);
  load_self(a.r, rb, sm, scratch, a.eta_s);
  init_coll_warp(a.r, w, lane);
  __shared__ int s_next;
  if (threadIdx.x == 0) s_next = 0;
  __syncthreads();
  const GridHeader* grid = grid_check(a.sc, a.r, a.eta);  // null: visit every cuboid
  const uint2* cells = grid ? grid_cells(a.sc) : nullptr;

  const int64_t n_mt = (a.n + FU_MT - 1) / FU_MT;
  const int64_t mt0 = blockIdx.x * a.mt_per_block;
  const int64_t mt1 = mt0 + a.mt_per_block < n_mt ? mt0 + a.mt_per_block : n_mt;
  for (;;) {
    int k = 0;
    if (lane == 0) k = atomicAdd(&s_next, 1);
    k = __shfl_sync(FULL_MASK, k, 0);
    const int64_t mt = mt0 + k;
    if (mt >= mt1) break;
    const int64_t c0 = mt * FU_MT;
    const int rows = (int)(a.n - c0 < FU_MT ? a.n - c0 : FU_MT);
    if (lane < rows) fk_chain(rb, J, a.q + (c0 + lane) * J, fw.T + lane * a.tstride);
    __syncwarp();
    for (int i = 0; i < rows; ++i) {
      const int64_t c = c0 + i;
      const float4* T = fw.T + i * a.tstride;
      // ---- FK: centres c_s (lanes over spheres), P rounded to its format
      for (int s = lane; s < S; s += 32) {
        const int l = rb.link0[s];
        const float4 r0 = T[3 * l], r1 = T[3 * l + 1], r2 = T[3 * l + 2];
        const float4 p = rb.sph[s];
        const float cx = fmaf(r0.x, p.x, fmaf(r0.y, p.y, fmaf(r0.z, p.z, r0.w)));
        const float cy = fmaf(r1.x, p.x, fmaf(r1.y, p.y, fmaf(r1.z, p.z, r1.w)));
        const float cz = fmaf(r2.x, p.x, fmaf(r2.y, p.y, fmaf(r2.z, p.z, r2.w)));
        fw.C[s] = make_float4(cx, cy, cz, 0.f);
        const float4 old = w.P[s];  // .w: the radius
        w.P[s] = make_float4(round_trip(cx, a.fP), round_trip(cy, a.fP), round_trip(cz, a.fP), old.w);
      }
      __syncwarp();
      // ---- collision: environment and self terms, cost and D out
      const float selfsum =
          collision_terms<false>(a.r, a.sc.O, rb, sm, w, a.eta, a.w_c, a.w_s, lane, nullptr, 0.f, grid, cells);
      CollOut out;
      out.cost = a.cost ? a.cost + c : nullptr;
      out.dist = a.dist.ptr ? reinterpret_cast<uint32_t*>(a.dist.ptr + c * a.dist.stride) : nullptr;
      out.dist_words = (int)(a.dist.stride / 4);
      out.grad = nullptr;
      out.grad_words = 0;
      coll_cost_dist(w, S, a.dist.f, a.w_c, a.w_s * selfsum, out, lane);
      __syncwarp();
      // ---- backward: per sphere F = G (rounded to its format) and M = c x G,
      //      then per link (lane l: link l's spheres in index order)
      for (int s = lane; s < S; s += 32) {
        const float4 gg = w.acc[s];
        const float g0 = round_trip(gg.y, a.fG), g1 = round_trip(gg.z, a.fG), g2 = round_trip(gg.w, a.fG);
        const float4 cc = fw.C[s];
        w.acc[s] = make_float4(gg.x, g0, g1, g2);
        fw.C[s] = make_float4(cc.y * g2 - cc.z * g1, cc.z * g0 - cc.x * g2, cc.x * g1 - cc.y * g0, 0.f);
      }
      __syncwarp();
      if (lane < J) {
        float F0 = 0.f, F1 = 0.f, F2 = 0.f, M0 = 0.f, M1 = 0.f, M2 = 0.f;
        for (int k2 = rb.start[lane]; k2 < rb.start[lane + 1]; ++k2) {
          const int s = rb.order[k2];
          const float4 g = w.acc[s], m = fw.C[s];
          F0 += g.y;
          F1 += g.z;
          F2 += g.w;
          M0 += m.x;
          M1 += m.y;
          M2 += m.z;
        }
        fw.lk[2 * lane] = make_float4(F0, F1, F2, 0.f);
        fw.lk[2 * lane + 1] = make_float4(M0, M1, M2, 0.f);
      }
      __syncwarp();
      if (lane < J) {  // suffix sums from the last link down, then J_j
        float F0 = 0.f, F1 = 0.f, F2 = 0.f, M0 = 0.f, M1 = 0.f, M2 = 0.f;
        for (int l = J - 1; l >= lane; --l) {
          const float4 f = fw.lk[2 * l], m = fw.lk[2 * l + 1];
          F0 += f.x;
          F1 += f.y;
          F2 += f.z;
          M0 += m.x;
          M1 += m.y;
          M2 += m.z;
        }
        const int j = lane;
        const float4 r0 = T[3 * j], r1 = T[3 * j + 1], r2 = T[3 * j + 2];
        const float ax = r0.z, ay = r1.z, az = r2.z;  // axis a_j: z-column of T_j
        const float bx = ay * r2.w - az * r1.w;       // b_j = a_j x o_j
        const float by = az * r0.w - ax * r2.w;
        const float bz = ax * r1.w - ay * r0.w;
        const float dc = a.dcost ? a.dcost[c] : 1.f;
        fw.jrow[j] = dc * ((ax * M0 + ay * M1 + az * M2) - (bx * F0 + by * F1 + bz * F2));
      }
      __syncwarp();
      {
        uint4* row = reinterpret_cast<uint4*>(a.jgrad.ptr + c * a.jgrad.stride);
        for (int cc = lane; cc < (int)(a.jgrad.stride / 16); cc += 32)
          row[cc] = pack_chunk_dyn(cc, J, a.jgrad.f, [&](int i2) { return fw.jrow[i2]; });
      }
      coll_reset(w, S, lane);
    }
  }
}

cudaError_t launch_fused(const RobotArgs& r, const SceneArgs& sc, const vapr_cost_params& p, const float* q,
                         const float* dcost, int64_t n, const vapr_format_table& t, float* cost, Packed dist,
                         Packed jgrad, cudaStream_t st) {
  FusedArgs a;
  a.r = r;
  a.sc = sc;
  a.eta = p.eta;
  a.eta_s = p.eta_self;
  a.w_c = p.w_coll;
  a.w_s = p.w_self;
  a.q = q;
  a.dcost = dcost;
  a.n = n;
  a.fP = make_dev_fmt(t.pos);
  a.fG = make_dev_fmt(t.grad);
  a.dist = dist;
  a.jgrad = jgrad;
  a.cost = cost;
  a.tstride = (3 * r.J) | 1;
  Bump b(nullptr);
  RobotSm rb;
  SceneSm sm;
  CollWarp w;
  FusedWarp fw;
  SelfScratch scratch;
  carve_fused(b, a, rb, sm, w, fw, 0, scratch);
  const size_t smem = b.bytes();
  const int per_sm = blocks_per_sm((const void*)fused_kernel, FU_WARPS * 32, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t n_mt = (n + FU_MT - 1) / FU_MT;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  const int64_t want = (n_mt + FU_WARPS - 1) / FU_WARPS;  // at least a mini-tile per warp
  const int grid = (int)(want < cap ? want : cap);
  a.mt_per_block = (n_mt + grid - 1) / grid;
  fused_kernel<<<grid, FU_WARPS * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace vapr
