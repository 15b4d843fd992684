// Swept-sphere environment cost for trajectory optimisation: the cost whose
// gradient is the paper's closest_pt_swept tensor (Sec. III-C).  The paper
// names the tensor but prints no formula; the reading here:
//   rows are trajectories of `horizon` consecutive configurations; row h
//   sweeps each sphere toward row h' = h+1 (h' = h on the last row) at K
//   points p_k = c_h + a_k (c_h' - c_h), a_k = k/K;
//   D_s = sum_k sum_o max(0, r_s + eta - d_o(p_k)),  C = w_c sum_s D_s;
//   G = d(sum of C over the trajectory)/dc_h: (1 - a_k) times the hinge
//   gradient at the row's own points (1 on the last row, whose points do
//   not move with a next row) plus a_k times it at the previous row's points.
// With K = 1 this is the environment term of vapr_collision_cost exactly.
//
// One warp per chunk of SW_CHUNK consecutive rows of one trajectory: the
// warp walks its rows in order, decoding each P row once (the next row's
// centres become the current ones).  Lanes own up to two spheres and run the
// sphere-major cuboid loop of the collision stage at each swept point; a
// point's gradient goes to its own row with weight 1 - a_k and is carried to
// the next row with weight a_k, so every point is evaluated once.  The first
// row of a chunk recomputes the carry from the previous row's points.
// Deterministic: a row's sums do not depend on where chunks start.
#include "stages.cuh"

namespace vapr {

constexpr int SW_WARPS = 8;
constexpr int SW_CHUNK = 8;  // rows per warp

struct SweptArgs {
  RobotArgs r;
  SceneArgs sc;
  float eta, w_c;
  Packed pos, dist, grad;
  float* cost;
  int64_t n;
  int horizon, samples;
};

__host__ __device__ inline void carve_swept(Bump& b, const RobotArgs& r, int O, RobotSm& rb, SceneSm& sm,
                                            CollWarp& w_mine, float4*& Pn, float4*& Pp, int mine) {
  carve_robot(b, r.J, r.S, rb);
  carve_scene(b, O, 0, 0, sm);
  carve_warps(b, SW_WARPS, mine, [&](Bump& wb) {
    carve_coll_warp(wb, r.S, r.J, w_mine);
    Pn = wb.take<float4>(r.S);
    Pp = wb.take<float4>(r.S);
  });
}

// Hinge terms of the point (x, radius x.w) against every cuboid, into t.
__device__ __forceinline__ void point_terms(const SceneSm& m, int O, const float4& xa, bool va,
                                            const float4& xb, bool vb, float eta, float w_c, float4& ta,
                                            float4& tb) {
  for (int o = 0; o < O; ++o) {
    const float4 C = m.cubC[o];
    const float ax = xa.x - C.x, ay = xa.y - C.y, az = xa.z - C.z, sa = xa.w + C.w;
    const float bx = xb.x - C.x, by = xb.y - C.y, bz = xb.z - C.z, sb = xb.w + C.w;
    const bool na = va && fmaf(ax, ax, fmaf(ay, ay, az * az)) < sa * sa;
    const bool nb = vb && fmaf(bx, bx, fmaf(by, by, bz * bz)) < sb * sb;
    if (__any_sync(FULL_MASK, na || nb)) {
      if (na) box_term(m, o, xa, eta, w_c, ta);
      if (nb) box_term(m, o, xb, eta, w_c, tb);
    }
  }
}

__device__ __forceinline__ float4 lerp4(const float4& c, const float4& d, float a) {
  return make_float4(fmaf(a, d.x - c.x, c.x), fmaf(a, d.y - c.y, c.y), fmaf(a, d.z - c.z, c.z), c.w);
}

__global__ void __launch_bounds__(SW_WARPS * 32) swept_kernel(SweptArgs a) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Bump b(smem4);
  RobotSm rb;
  SceneSm sm;
  CollWarp w;
  float4 *Pn, *Pp;
  carve_swept(b, a.r, a.sc.O, rb, sm, w, Pn, Pp, wid);
  load_robot(a.r, rb);
  RobotArgs r0 = a.r;
  r0.NP = 0;
  load_scene(r0, a.sc, a.eta, 0.f, sm);
  init_coll_warp(a.r, w, lane);
  for (int s = lane; s < a.r.S; s += 32) {
    Pn[s] = w.P[s];
    Pp[s] = w.P[s];
  }
  __syncthreads();
  const GridHeader* grid = grid_check(a.sc, a.r, a.eta);  // null: every cuboid
  const uint2* cells = grid ? grid_cells(a.sc) : nullptr;
  // the terms of two points, through the scene grid when there is one
  auto terms = [&](const float4& xa, bool va, const float4& xb, bool vb, float4& ta, float4& tb) {
    if (grid) {
      env_grid2(sm, *grid, cells, va, xa, vb, xb, a.eta, a.w_c, ta, tb);
    } else {
      point_terms(sm, a.sc.O, xa, va, xb, vb, a.eta, a.w_c, ta, tb);
    }
  };

  const int S = a.r.S, K = a.samples, H = a.horizon;
  const float invK = 1.f / (float)K;
  const int64_t chunks_per_traj = (H + SW_CHUNK - 1) / SW_CHUNK;
  const int64_t n_chunks = (a.n / H) * chunks_per_traj;
  auto row = [&](int64_t cc) { return reinterpret_cast<const uint32_t*>(a.pos.ptr + cc * a.pos.stride); };
  float4* cur = w.P;  // centres of the row being finished (.w = radius)
  float4* nxt = Pn;
  CollOut out;
  out.dist_words = (int)(a.dist.stride / 4);
  out.grad_words = (int)(a.grad.stride / 4);
  for (int64_t ch = blockIdx.x * (int64_t)SW_WARPS + wid; ch < n_chunks; ch += (int64_t)gridDim.x * SW_WARPS) {
    const int64_t traj = ch / chunks_per_traj;
    const int h0 = (int)(ch - traj * chunks_per_traj) * SW_CHUNK;
    const int h1 = min(H, h0 + SW_CHUNK);
    const int64_t base_row = traj * H;
    load_centres<false>(row(base_row + h0), a.pos.f, S, cur, lane);
    if (h0 > 0) load_centres<false>(row(base_row + h0 - 1), a.pos.f, S, Pp, lane);
    __syncwarp();
    // carry into the chunk's first row: the previous row's points, weight
    // a_k; each lane keeps the carries of its spheres in Pp[s].xyz (the
    // previous row's centres are no longer needed once read)
    for (int pass = 0; pass * 64 < S; ++pass) {
      const int sa = pass * 64 + lane, sb = sa + 32;
      const bool va = sa < S, vb = sb < S;
      float3 c0 = make_float3(0.f, 0.f, 0.f), c1 = c0;
      if (h0 > 0) {
        const float4 ca = va ? cur[sa] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 cb = vb ? cur[sb] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 pa = va ? make_float4(Pp[sa].x, Pp[sa].y, Pp[sa].z, ca.w) : ca;
        const float4 pb = vb ? make_float4(Pp[sb].x, Pp[sb].y, Pp[sb].z, cb.w) : cb;
        for (int k = 1; k < K; ++k) {
          const float al = (float)k * invK;
          float4 ta = make_float4(0.f, 0.f, 0.f, 0.f), tb = ta;
          terms(lerp4(pa, ca, al), va, lerp4(pb, cb, al), vb, ta, tb);
          c0 = make_float3(fmaf(al, ta.y, c0.x), fmaf(al, ta.z, c0.y), fmaf(al, ta.w, c0.z));
          c1 = make_float3(fmaf(al, tb.y, c1.x), fmaf(al, tb.z, c1.y), fmaf(al, tb.w, c1.z));
        }
      }
      if (va) Pp[sa] = make_float4(c0.x, c0.y, c0.z, Pp[sa].w);
      if (vb) Pp[sb] = make_float4(c1.x, c1.y, c1.z, Pp[sb].w);
    }
    for (int h = h0; h < h1; ++h) {
      const int64_t c = base_row + h;
      const bool last = h + 1 == H;
      if (!last) load_centres<false>(row(c + 1), a.pos.f, S, nxt, lane);
      __syncwarp();
      for (int pass = 0; pass * 64 < S; ++pass) {
        const int sa = pass * 64 + lane, sb = sa + 32;
        const bool va = sa < S, vb = sb < S;
        const float4 ca = va ? cur[sa] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 cb = vb ? cur[sb] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 na = va && !last ? make_float4(nxt[sa].x, nxt[sa].y, nxt[sa].z, ca.w) : ca;
        const float4 nb = vb && !last ? make_float4(nxt[sb].x, nxt[sb].y, nxt[sb].z, cb.w) : cb;
        float Da = 0.f, Db = 0.f;
        float3 ga = make_float3(0.f, 0.f, 0.f), gb = ga, fa = ga, fb = ga;
        for (int k = 0; k < K; ++k) {
          const float al = (float)k * invK;
          float4 ta = make_float4(0.f, 0.f, 0.f, 0.f), tb = ta;
          terms(lerp4(ca, na, al), va, lerp4(cb, nb, al), vb, ta, tb);
          const float wo = last ? 1.f : 1.f - al;
          Da += ta.x;
          Db += tb.x;
          ga = make_float3(fmaf(wo, ta.y, ga.x), fmaf(wo, ta.z, ga.y), fmaf(wo, ta.w, ga.z));
          gb = make_float3(fmaf(wo, tb.y, gb.x), fmaf(wo, tb.z, gb.y), fmaf(wo, tb.w, gb.z));
          if (!last && k > 0) {  // the same point moves with the next row (weight a_k)
            fa = make_float3(fmaf(al, ta.y, fa.x), fmaf(al, ta.z, fa.y), fmaf(al, ta.w, fa.z));
            fb = make_float3(fmaf(al, tb.y, fb.x), fmaf(al, tb.z, fb.y), fmaf(al, tb.w, fb.z));
          }
        }
        // own points, then the carry from the previous row; store the next carry
        if (va) {
          const float4 cr = Pp[sa];
          w.acc[sa] = make_float4(Da, ga.x + cr.x, ga.y + cr.y, ga.z + cr.z);
          Pp[sa] = make_float4(fa.x, fa.y, fa.z, cr.w);
        }
        if (vb) {
          const float4 cr = Pp[sb];
          w.acc[sb] = make_float4(Db, gb.x + cr.x, gb.y + cr.y, gb.z + cr.z);
          Pp[sb] = make_float4(fb.x, fb.y, fb.z, cr.w);
        }
      }
      __syncwarp();
      out.cost = a.cost ? a.cost + c : nullptr;
      out.dist = a.dist.ptr ? reinterpret_cast<uint32_t*>(a.dist.ptr + c * a.dist.stride) : nullptr;
      out.grad = a.grad.ptr ? reinterpret_cast<uint32_t*>(a.grad.ptr + c * a.grad.stride) : nullptr;
      coll_outputs(w, S, a.dist.f, a.grad.f, a.w_c, 0.f, out, lane);
      if (!last) {  // the next row's centres become the current ones
        float4* t = cur;
        cur = nxt;
        nxt = t;
      }
    }
  }
}

static cudaError_t launch_swept(const SweptArgs& a, cudaStream_t st) {
  Bump b(nullptr);
  RobotSm rb;
  SceneSm sm;
  CollWarp w;
  float4 *Pn, *Pp;
  carve_swept(b, a.r, a.sc.O, rb, sm, w, Pn, Pp, 0);
  const size_t smem = b.bytes();
  const int per_sm = blocks_per_sm((const void*)swept_kernel, SW_WARPS * 32, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t chunks = (a.n / a.horizon) * ((a.horizon + SW_CHUNK - 1) / SW_CHUNK);
  const int64_t blocks = (chunks + SW_WARPS - 1) / SW_WARPS;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  swept_kernel<<<(int)(blocks < cap ? blocks : cap), SW_WARPS * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace vapr

using namespace vapr;

extern "C" vapr_status vapr_swept_cost(const vapr_robot* robot, const vapr_scene* scene,
                                       const vapr_cost_params* params, const void* pos_packed, int64_t n,
                                       int32_t horizon, int32_t samples, const vapr_format_table* table,
                                       float* cost, void* dist_packed, void* grad_packed, void* stream) {
  RobotArgs r;
  vapr_status v = check_robot(robot, &r);
  if (v != VAPR_OK) return v;
  if ((v = check_table(table)) != VAPR_OK) return v;
  if (!params) return VAPR_ERR_INVALID_ARG;
  SceneArgs sc;
  if ((v = check_scene(scene, &sc)) != VAPR_OK) return v;
  if (n < 0 || horizon < 1 || samples < 1) return VAPR_ERR_INVALID_ARG;
  if (samples > VAPR_MAX_SWEPT_SAMPLES || n > VAPR_MAX_CONFIGS) return VAPR_ERR_TOO_LARGE;
  if (n % horizon) return VAPR_ERR_INVALID_ARG;
  if (n == 0) return VAPR_OK;
  if (!pos_packed) return VAPR_ERR_INVALID_ARG;
  if ((uintptr_t)pos_packed % 16 || (uintptr_t)dist_packed % 16 || (uintptr_t)grad_packed % 16 ||
      (uintptr_t)cost % 4)
    return VAPR_ERR_MISALIGNED;
  SweptArgs a;
  a.r = r;
  a.sc = sc;
  a.eta = params->eta;
  a.w_c = params->w_coll;
  a.pos = Packed{(uint8_t*)pos_packed, (int64_t)row_bytes(3 * (int64_t)r.S, table->pos), make_dev_fmt(table->pos)};
  a.dist = Packed{(uint8_t*)dist_packed, (int64_t)row_bytes(r.S, table->dist), make_dev_fmt(table->dist)};
  a.grad = Packed{(uint8_t*)grad_packed, (int64_t)row_bytes(3 * (int64_t)r.S, table->grad), make_dev_fmt(table->grad)};
  a.cost = cost;
  a.n = n;
  a.horizon = horizon;
  a.samples = samples;
  return cuda_status(launch_swept(a, (cudaStream_t)stream));
}
