// The whole cost-and-gradient step of a batch in one kernel, with the
// sphere centres P and their gradient G kept on the SM: the upper bound of
// what not storing those tensors buys (the staged path stores them in
// their ExMy formats, Sec. III-C).  It computes what vapr_fk,
// vapr_collision_cost and vapr_backward compute (iteration steps 2-5 of
// Sec. III-B):
//   FK         T_j = T_{j-1} F_j Rz(q_j), c_s = T_link(s) [p_s; 1]
//   collision  C = w_c sum_s D_s + w_s sum P_ij, G = dC/dc
//   backward   J_j = dC (a_j . M_{>=j} - b_j . F_{>=j}), F = sum G_s,
//              M = sum c_s x G_s over the spheres on links >= j (from
//              per-link sums in the link's frame, LinkSums)
// and rounds P and G to the table's formats in registers, as storing and
// loading them would.
//
// A block of FU_WARPS warps takes a contiguous range of mini-tiles of
// FU_MT = 4 configurations, which its warps draw one at a time from a block
// counter.  A warp runs its mini-tile's joint chains (lanes 0..3, one
// configuration each) into its own transform rows in shared memory, then
// takes the configurations one by one: it computes the sphere centres from
// the transforms (lanes over spheres), runs the collision stage's
// environment and self terms on them (collision_terms: the same code, so
// cost and D are the staged path's bit for bit), writes cost and D, and
// runs the backward pass cooperatively: lanes round G to its format, lane l
// forms link l's sums and moment (LinkSums, spheres in the robot's order),
// and lane j runs the staged backward's running totals over the links to
// form K_j and J_j.  Every sum is taken in the staged pass's order with the
// same operations, so J is the staged path's bit for bit too (with the
// transforms recomputed there, not stored).  A first version shared
// 32-configuration tiles across the block, behind block barriers: warps
// idled at each tile's end, 0.61 of the staged speed at 2^20.  Mini-tiles
// of 8 configurations (twice the transform rows, and a longer serial chain
// phase per warp) ran at 0.71 of the staged speed at 32,768 configurations,
// against 0.86 with 4.  Splitting each chain over three
// lanes (one transform row each) gained nothing: the chains are a small
// part of a mini-tile's time next to its sphere tests.
#include "stages.cuh"

namespace vapr {

constexpr int FU_WARPS = 8;
constexpr int FU_MT = 4;  // configurations per mini-tile (a warp's chains)

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
  carve_warps(b, FU_WARPS, mine, [&](Bump& wb) {
    carve_coll_warp(wb, r.S, r.J, w_mine);
    f_mine.lk = wb.take<float4>(2 * VAPR_MAX_JOINTS);
    f_mine.jrow = wb.take<float>(VAPR_MAX_JOINTS);
  });
  carve_self_scratch(t, r.NP, cluster_bound(r.S, r.J), r.S, scratch);  // over the warps' sets (built first)
  if (t.off > b.off) b.off = t.off;
  // (after the scratch: written once the tables are built)
  carve_warps(b, FU_WARPS, mine, [&](Bump& wb) { f_mine.T = wb.take<float4>((size_t)FU_MT * a.tstride); });
}

// dec(enc(x)) in format f: the value a stored and reloaded x has.
__device__ __forceinline__ float round_trip(float x, const DevFmt& f) {
  return f.kind == KIND_F32 ? x : decode(encode(x, f), f);
}

// F32: P, G, D and J are float32 (the loop body without the other formats'
// code, for the instruction cache).
template <bool F32>
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
  __shared__ int s_next;
  if (threadIdx.x == 0) s_next = 0;  // (visible after the prologue's barriers)
  // null grid: visit every cuboid
  const GridHeader* grid = load_block_tables(a.r, a.sc, a.eta, a.eta_s, rb, sm, scratch, w);
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
      // ---- FK: centres c_s (lanes over spheres), rounded to the P format
      for (int s = lane; s < S; s += 32) {
        const int l = rb.link0[s];
        const float4 r0 = T[3 * l], r1 = T[3 * l + 1], r2 = T[3 * l + 2];
        const float4 p = rb.sph[s];
        const float cx = fmaf(r0.x, p.x, fmaf(r0.y, p.y, fmaf(r0.z, p.z, r0.w)));
        const float cy = fmaf(r1.x, p.x, fmaf(r1.y, p.y, fmaf(r1.z, p.z, r1.w)));
        const float cz = fmaf(r2.x, p.x, fmaf(r2.y, p.y, fmaf(r2.z, p.z, r2.w)));
        const float4 old = w.P[s];  // .w: the radius
        w.P[s] = F32 ? make_float4(cx, cy, cz, old.w)
                     : make_float4(round_trip(cx, a.fP), round_trip(cy, a.fP), round_trip(cz, a.fP), old.w);
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
      coll_cost_dist<F32>(w, S, a.dist.f, a.w_c, a.w_s * selfsum, out, lane);
      __syncwarp();
      // ---- backward: G rounded to its format (lanes over spheres), then
      //      lane l forms link l's sums and moment, and lane j runs the
      //      staged pass's running totals over the links to form J_j
      if (!F32 && a.fG.kind != KIND_F32) {
        for (int s = lane; s < S; s += 32) {
          const float4 gg = w.acc[s];
          w.acc[s] = make_float4(gg.x, round_trip(gg.y, a.fG), round_trip(gg.z, a.fG), round_trip(gg.w, a.fG));
        }
        __syncwarp();
      }
      float R[3][3], t[3];
      if (lane < J) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float4 rk = T[3 * lane + k];
          R[k][0] = rk.x;
          R[k][1] = rk.y;
          R[k][2] = rk.z;
          t[k] = rk.w;
        }
        LinkSums ls;
        ls.zero();
        for (int k2 = rb.start[lane]; k2 < rb.start[lane + 1]; ++k2) {
          const int s = rb.order[k2];
          const float4 g = w.acc[s];
          ls.add(g.y, g.z, g.w, rb.sph[s]);
        }
        float mo[3];
        ls.moment(R, t, mo);
        fw.lk[2 * lane] = make_float4(ls.f[0], ls.f[1], ls.f[2], 0.f);
        fw.lk[2 * lane + 1] = make_float4(mo[0], mo[1], mo[2], 0.f);
      }
      __syncwarp();
      if (lane < J) {
        float ax, ay, az, bx, by, bz;
        joint_axis(R, t, ax, ay, az, bx, by, bz);
        float M[3] = {0.f, 0.f, 0.f}, F[3] = {0.f, 0.f, 0.f};
        float K = 0.f;
        for (int l = 0; l < J; ++l) {
          if (l == lane) K = axis_term(ax, ay, az, bx, by, bz, M, F);
          const float4 f = fw.lk[2 * l], m = fw.lk[2 * l + 1];
          M[0] = __fadd_rn(M[0], m.x);
          M[1] = __fadd_rn(M[1], m.y);
          M[2] = __fadd_rn(M[2], m.z);
          F[0] = __fadd_rn(F[0], f.x);
          F[1] = __fadd_rn(F[1], f.y);
          F[2] = __fadd_rn(F[2], f.z);
        }
        const float dc = a.dcost ? a.dcost[c] : 1.f;
        fw.jrow[lane] = __fmul_rn(dc, __fsub_rn(axis_term(ax, ay, az, bx, by, bz, M, F), K));
      }
      __syncwarp();
      {
        uint4* row = reinterpret_cast<uint4*>(a.jgrad.ptr + c * a.jgrad.stride);
        for (int cc = lane; cc < (int)(a.jgrad.stride / 16); cc += 32) {
          if constexpr (F32) {
            auto v = [&](int i2) { return i2 < J ? __float_as_uint(fw.jrow[i2]) : 0u; };
            row[cc] = make_uint4(v(4 * cc), v(4 * cc + 1), v(4 * cc + 2), v(4 * cc + 3));
          } else {
            row[cc] = pack_chunk_dyn(cc, J, a.jgrad.f, [&](int i2) { return fw.jrow[i2]; });
          }
        }
      }
      __syncwarp();  // (collision_terms rewrites acc whole for the next configuration)
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
  const bool f32 = a.fP.kind == KIND_F32 && a.fG.kind == KIND_F32 && jgrad.f.kind == KIND_F32 &&
                   (!dist.ptr || dist.f.kind == KIND_F32);
  auto kernel = f32 ? fused_kernel<true> : fused_kernel<false>;
  const int per_sm = blocks_per_sm((const void*)kernel, FU_WARPS * 32, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t n_mt = (n + FU_MT - 1) / FU_MT;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  const int64_t want = (n_mt + FU_WARPS - 1) / FU_WARPS;  // at least a mini-tile per warp
  const int grid = (int)(want < cap ? want : cap);
  a.mt_per_block = (n_mt + grid - 1) / grid;
  kernel<<<grid, FU_WARPS * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace vapr
