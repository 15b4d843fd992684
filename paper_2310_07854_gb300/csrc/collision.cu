// Collision cost (iteration steps 3-4 of Sec. III-B): robot-environment
// distance queries against oriented cuboids plus robot self-collision
// (Sec. II-B), the per-configuration cost aggregation, and the gradient with
// respect to the sphere centres.  Reads out_spheres (P) and writes the
// per-sphere penetration (D) and dC/dP (G) in their ExMy formats.
//
//   box distance: x = R^T (c - t), u = |x| - h,
//                 d = |max(u, 0)| + min(max_k u_k, 0)
//   D_s  = sum_o max(0, r_s + eta - d_o(c_s))
//   P_ij = max(0, r_i + r_j + eta_self - |c_i - c_j|)
//   C    = w_coll sum_s D_s + w_self sum_pairs P_ij,   G_s = dC/dc_s
//
// One warp per configuration (a block runs COLL_WARPS of them at a time).
// Most sphere/cuboid pairs are far apart, so the exact distance is only
// evaluated where a conservative test cannot rule the pair out:
//   1. a bounding sphere per link (centroid of its spheres, radius from the
//      actual positions) against each cuboid's bounding sphere -> a 64-bit
//      mask of candidate cuboids per link;
//   2. each sphere against the candidates of its link;
//   3. pairs that survive are compacted into a warp queue (ballot + popc)
//      and evaluated 32 at a time, one per lane.
// Every skipped pair provably has zero penetration: d_o(c) >= |c - t_o| - |h_o|,
// and a slack of SLACK metres covers float32 rounding of the tests.
// Contributions to a sphere are summed in queue order by the lane group
// that shares it (__match_any_sync), so results do not depend on timing.
#include "common.cuh"

namespace vapr {

constexpr int COLL_WARPS = 8;
constexpr int QCAP = 64;
constexpr float SLACK = 1e-4f;
constexpr unsigned FULL = 0xffffffffu;

struct CollArgs {
  RobotArgs r;
  SceneArgs sc;
  float eta, eta_s, w_c, w_s;
  Packed pos, dist, grad;
  float* cost;
  int64_t n;
};

struct CollSmem {
  float4* cub;     // [O][4]: (col_k of R, t_k) for k = 0..2, then (h, bound)
  float4* P;       // [COLL_WARPS][S]: (x, y, z, r)
  float4* acc;     // [COLL_WARPS][S]: (D, gx, gy, gz)
  float4* lb;      // [COLL_WARPS][J]: link bounding sphere (centre, radius)
  uint64_t* mask;  // [COLL_WARPS][J]
  uint32_t* queue; // [COLL_WARPS][QCAP]: sphere | cuboid << 16
  uint32_t* pairs; // [NP]: i | j << 16
  int* order;      // [S] spheres grouped by link
  int* start;      // [J+1]
  int* linkof;     // [S] 0-based link
};

__device__ __forceinline__ CollSmem carve(void* base, int O, int S, int J, int NP) {
  CollSmem m;
  float4* f4 = reinterpret_cast<float4*>(base);
  m.cub = f4;
  f4 += 4 * O;
  m.P = f4;
  f4 += COLL_WARPS * S;
  m.acc = f4;
  f4 += COLL_WARPS * S;
  m.lb = f4;
  f4 += COLL_WARPS * J;
  m.mask = reinterpret_cast<uint64_t*>(f4);
  uint32_t* u = reinterpret_cast<uint32_t*>(m.mask + COLL_WARPS * J);
  m.queue = u;
  u += COLL_WARPS * QCAP;
  m.pairs = u;
  u += NP;
  m.order = reinterpret_cast<int*>(u);
  m.start = m.order + S;
  m.linkof = m.start + J + 1;
  return m;
}

static size_t coll_smem(int O, int S, int J, int NP) {
  return sizeof(float4) * (4 * (size_t)O + 2 * COLL_WARPS * (size_t)S + COLL_WARPS * (size_t)J) +
         sizeof(uint64_t) * COLL_WARPS * J + sizeof(uint32_t) * (COLL_WARPS * QCAP + (size_t)NP) +
         sizeof(int) * (2 * (size_t)S + J + 1);
}

// Sums (a, b, c, d) over the lanes that share `key`, in lane order, and adds
// the total into acc[key] from the group's lowest lane.  Lanes with
// active == false neither contribute nor write.
__device__ __forceinline__ void group_add(float4* acc, bool active, int key, float a, float b,
                                          float c, float d) {
  const int lane = threadIdx.x & 31;
  const unsigned grp = __match_any_sync(FULL, active ? key : -1);
  unsigned rem = active ? grp : 0u;
  float sa = 0.f, sb = 0.f, sc = 0.f, sd = 0.f;
  while (__any_sync(FULL, rem != 0u)) {
    const int src = rem ? __ffs(rem) - 1 : lane;
    const float va = __shfl_sync(FULL, a, src), vb = __shfl_sync(FULL, b, src);
    const float vc = __shfl_sync(FULL, c, src), vd = __shfl_sync(FULL, d, src);
    if (rem) {
      sa += va;
      sb += vb;
      sc += vc;
      sd += vd;
      rem &= rem - 1u;
    }
  }
  if (active && lane == __ffs(grp) - 1) {
    float4 v = acc[key];
    v.x += sa;
    v.y += sb;
    v.z += sc;
    v.w += sd;
    acc[key] = v;
  }
}

// Exact narrow phase of queue entries 0..cnt-1, one per lane.
__device__ __forceinline__ void flush(const CollSmem& m, float4* P, float4* acc,
                                      const uint32_t* queue, int cnt, float eta, float w_c) {
  const int lane = threadIdx.x & 31;
  const bool have = lane < cnt;
  const uint32_t e = have ? queue[lane] : 0u;
  const int s = (int)(e & 0xffffu), o = (int)(e >> 16);
  float dD = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
  if (have) {
    const float4 c = P[s];
    const float4 A0 = m.cub[4 * o], A1 = m.cub[4 * o + 1], A2 = m.cub[4 * o + 2];
    const float4 H = m.cub[4 * o + 3];
    const float dx = c.x - A0.w, dy = c.y - A1.w, dz = c.z - A2.w;
    const float x0 = fmaf(A0.x, dx, fmaf(A0.y, dy, A0.z * dz));
    const float x1 = fmaf(A1.x, dx, fmaf(A1.y, dy, A1.z * dz));
    const float x2 = fmaf(A2.x, dx, fmaf(A2.y, dy, A2.z * dz));
    const float u0 = fabsf(x0) - H.x, u1 = fabsf(x1) - H.y, u2 = fabsf(x2) - H.z;
    float d, l0, l1, l2;
    if (u0 > 0.f || u1 > 0.f || u2 > 0.f) {
      const float v0 = fmaxf(u0, 0.f), v1 = fmaxf(u1, 0.f), v2 = fmaxf(u2, 0.f);
      d = sqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
      const float inv = 1.0f / d;
      l0 = copysignf(v0 * inv, x0 >= 0.f ? 1.f : -1.f);
      l1 = copysignf(v1 * inv, x1 >= 0.f ? 1.f : -1.f);
      l2 = copysignf(v2 * inv, x2 >= 0.f ? 1.f : -1.f);
    } else {  // inside: nearest face, lowest axis on ties, sgn(0) = +1
      int k = 0;
      d = u0;
      if (u1 > d) { d = u1; k = 1; }
      if (u2 > d) { d = u2; k = 2; }
      const float xs = k == 0 ? x0 : k == 1 ? x1 : x2;
      const float sg = xs >= 0.f ? 1.f : -1.f;
      l0 = k == 0 ? sg : 0.f;
      l1 = k == 1 ? sg : 0.f;
      l2 = k == 2 ? sg : 0.f;
    }
    const float pen = c.w + eta - d;
    if (pen > 0.f) {
      dD = pen;  // gradient of the hinge: -grad d, scaled by w_coll
      gx = -w_c * fmaf(A0.x, l0, fmaf(A1.x, l1, A2.x * l2));
      gy = -w_c * fmaf(A0.y, l0, fmaf(A1.y, l1, A2.y * l2));
      gz = -w_c * fmaf(A0.z, l0, fmaf(A1.z, l1, A2.z * l2));
    }
  }
  group_add(acc, have, s, dD, gx, gy, gz);
}

__global__ void __launch_bounds__(COLL_WARPS * 32) collision_kernel(CollArgs a) {
  extern __shared__ float4 smem4[];
  const int J = a.r.J, S = a.r.S, NP = a.r.NP, O = a.sc.O;
  const CollSmem m = carve(smem4, O, S, J, NP);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  // ---- block-wide tables
  for (int o = threadIdx.x; o < O; o += blockDim.x) {
    const float* p = a.sc.pose + 12 * o;
    const float hx = a.sc.half[3 * o], hy = a.sc.half[3 * o + 1], hz = a.sc.half[3 * o + 2];
    m.cub[4 * o + 0] = make_float4(p[0], p[3], p[6], p[9]);
    m.cub[4 * o + 1] = make_float4(p[1], p[4], p[7], p[10]);
    m.cub[4 * o + 2] = make_float4(p[2], p[5], p[8], p[11]);
    m.cub[4 * o + 3] = make_float4(hx, hy, hz, sqrtf(hx * hx + hy * hy + hz * hz) + a.eta + SLACK);
  }
  for (int p = threadIdx.x; p < NP; p += blockDim.x) {
    const int i = clampi(a.r.pairs[2 * p], 0, S - 1), j = clampi(a.r.pairs[2 * p + 1], 0, S - 1);
    m.pairs[p] = (uint32_t)i | ((uint32_t)j << 16);
  }
  for (int i = threadIdx.x; i < COLL_WARPS * S; i += blockDim.x) {
    const int s = i % S;
    m.P[i] = make_float4(0.f, 0.f, 0.f, a.r.sphere_local[4 * s + 3]);
  }
  if (threadIdx.x == 0) {  // stable counting sort of the spheres by link
    for (int j = 0; j <= J; ++j) m.start[j] = 0;
    for (int s = 0; s < S; ++s) {
      const int L = clampi(a.r.sphere_link[s], 1, J);
      m.linkof[s] = L - 1;
      ++m.start[L];
    }
    for (int j = 1; j <= J; ++j) m.start[j] += m.start[j - 1];
    for (int s = S - 1; s >= 0; --s) m.order[--m.start[m.linkof[s] + 1]] = s;
    for (int j = 0; j < J; ++j) m.start[j] = m.start[j + 1];
    m.start[J] = S;
  }
  __syncthreads();

  float4* P = m.P + wid * S;
  float4* acc = m.acc + wid * S;
  float4* lb = m.lb + wid * J;
  uint64_t* mask = m.mask + wid * J;
  uint32_t* queue = m.queue + wid * QCAP;
  const unsigned lt_mask = (1u << lane) - 1u;

  for (int64_t c = blockIdx.x * (int64_t)COLL_WARPS + wid; c < a.n;
       c += (int64_t)gridDim.x * COLL_WARPS) {
    // ---- 1. sphere centres of this configuration (coalesced 16-byte loads)
    {
      const uint8_t* row = a.pos.ptr + c * a.pos.stride;
      const int cpr = (int)(a.pos.stride / 16), nv = 3 * S, k = a.pos.f.k;
      for (int cc = lane; cc < cpr; cc += 32) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(row) + cc);
        const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i0 = (4 * cc + q) * k;
          for (int j = 0; j < k; ++j) {
            const int i = i0 + j;
            if (i < nv) {
              const int s = i / 3;
              reinterpret_cast<float*>(P + s)[i - 3 * s] = unpack_slot(w4[q], j, a.pos.f);
            }
          }
        }
      }
    }
    for (int s = lane; s < S; s += 32) acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();

    // ---- 2. link bounding spheres from the actual positions
    if (lane < J) {
      const int b = m.start[lane], e = m.start[lane + 1];
      float4 v = make_float4(0.f, 0.f, 0.f, -1.f);  // empty link: never near
      if (e > b) {
        float mx = 0.f, my = 0.f, mz = 0.f;
        for (int idx = b; idx < e; ++idx) {
          const float4 p = P[m.order[idx]];
          mx += p.x;
          my += p.y;
          mz += p.z;
        }
        const float inv = 1.0f / (float)(e - b);
        mx *= inv;
        my *= inv;
        mz *= inv;
        float rad = 0.f;
        for (int idx = b; idx < e; ++idx) {
          const float4 p = P[m.order[idx]];
          const float dx = p.x - mx, dy = p.y - my, dz = p.z - mz;
          rad = fmaxf(rad, sqrtf(dx * dx + dy * dy + dz * dz) + p.w);
        }
        v = make_float4(mx, my, mz, rad + SLACK);
      }
      lb[lane] = v;
    }
    __syncwarp();

    // ---- 3. environment: cull, compact, evaluate
    int qn = 0;
    for (int base = 0; base < O; base += 64) {
      for (int L = 0; L < J; ++L) {
        const float4 b = lb[L];
        bool n0 = false, n1 = false;
        const int o0 = base + lane, o1 = base + 32 + lane;
        if (b.w >= 0.f && o0 < O) {
          const float4 H = m.cub[4 * o0 + 3];
          const float dx = b.x - m.cub[4 * o0].w, dy = b.y - m.cub[4 * o0 + 1].w,
                      dz = b.z - m.cub[4 * o0 + 2].w;
          const float thr = b.w + H.w;
          n0 = dx * dx + dy * dy + dz * dz < thr * thr;
        }
        if (b.w >= 0.f && o1 < O) {
          const float4 H = m.cub[4 * o1 + 3];
          const float dx = b.x - m.cub[4 * o1].w, dy = b.y - m.cub[4 * o1 + 1].w,
                      dz = b.z - m.cub[4 * o1 + 2].w;
          const float thr = b.w + H.w;
          n1 = dx * dx + dy * dy + dz * dz < thr * thr;
        }
        const uint32_t b0 = __ballot_sync(FULL, n0), b1 = __ballot_sync(FULL, n1);
        if (lane == 0) mask[L] = (uint64_t)b0 | ((uint64_t)b1 << 32);
      }
      __syncwarp();
      for (int sb = 0; sb < S; sb += 32) {
        const int idx = sb + lane;
        const bool valid = idx < S;
        const int s = valid ? m.order[idx] : 0;
        uint64_t cand = valid ? mask[m.linkof[s]] : 0ull;
        const float4 cs = P[s];
        while (__any_sync(FULL, cand != 0ull)) {
          bool nr = false;
          int o = 0;
          if (cand) {
            o = base + __ffsll((long long)cand) - 1;
            cand &= cand - 1ull;
            const float4 H = m.cub[4 * o + 3];
            const float dx = cs.x - m.cub[4 * o].w, dy = cs.y - m.cub[4 * o + 1].w,
                        dz = cs.z - m.cub[4 * o + 2].w;
            const float thr = cs.w + H.w;
            nr = dx * dx + dy * dy + dz * dz < thr * thr;
          }
          const unsigned bal = __ballot_sync(FULL, nr);
          if (nr) queue[qn + __popc(bal & lt_mask)] = (uint32_t)s | ((uint32_t)o << 16);
          qn += __popc(bal);
          if (qn >= 32) {
            __syncwarp();
            flush(m, P, acc, queue, 32, a.eta, a.w_c);
            __syncwarp();
            const int rest = qn - 32;
            const uint32_t moved = lane < rest ? queue[32 + lane] : 0u;
            __syncwarp();
            if (lane < rest) queue[lane] = moved;
            qn = rest;
            __syncwarp();
          }
        }
      }
    }
    __syncwarp();
    if (qn > 0) flush(m, P, acc, queue, qn, a.eta, a.w_c);

    // ---- 4. self-collision over the pair list
    float selfsum = 0.f;
    for (int pb = 0; pb < NP; pb += 32) {
      const int p = pb + lane;
      const bool ok = p < NP;
      const uint32_t pr = ok ? m.pairs[p] : 0u;
      const int i = (int)(pr & 0xffffu), j = (int)(pr >> 16);
      const float4 ci = P[i], cj = P[j];
      const float dx = ci.x - cj.x, dy = ci.y - cj.y, dz = ci.z - cj.z;
      const float d2 = dx * dx + dy * dy + dz * dz;
      const float thr = ci.w + cj.w + a.eta_s;
      bool act = ok && d2 < thr * thr;
      if (__any_sync(FULL, act)) {
        float ux = 0.f, uy = 0.f, uz = 0.f;
        if (act) {
          const float dd = sqrtf(d2);
          const float pen = thr - dd;
          if (pen > 0.f) {
            selfsum += pen;
            if (dd > 0.f) {
              const float inv = a.w_s / dd;
              ux = dx * inv;
              uy = dy * inv;
              uz = dz * inv;
            }
          } else {
            act = false;
          }
        }
        __syncwarp();
        group_add(acc, act, i, 0.f, -ux, -uy, -uz);
        __syncwarp();
        group_add(acc, act, j, 0.f, ux, uy, uz);
      }
    }
    __syncwarp();

    // ---- 5. cost and packed outputs
    float local = 0.f;
    for (int s = lane; s < S; s += 32) local += acc[s].x;
    local = a.w_c * local + a.w_s * selfsum;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(FULL, local, off);
    if (a.cost && lane == 0) a.cost[c] = local;
    if (a.dist.ptr) {
      const int cpr = (int)(a.dist.stride / 16);
      auto get = [&](int i) { return acc[i].x; };
      for (int cc = lane; cc < cpr; cc += 32) {
        uint4 v;
        v.x = pack_word(4 * cc + 0, S, a.dist.f, get);
        v.y = pack_word(4 * cc + 1, S, a.dist.f, get);
        v.z = pack_word(4 * cc + 2, S, a.dist.f, get);
        v.w = pack_word(4 * cc + 3, S, a.dist.f, get);
        *reinterpret_cast<uint4*>(a.dist.ptr + c * a.dist.stride + 16 * cc) = v;
      }
    }
    if (a.grad.ptr) {
      const int cpr = (int)(a.grad.stride / 16), nv = 3 * S;
      auto get = [&](int i) {
        const int s = i / 3, d = i - 3 * s;
        return reinterpret_cast<const float*>(acc + s)[1 + d];
      };
      for (int cc = lane; cc < cpr; cc += 32) {
        uint4 v;
        v.x = pack_word(4 * cc + 0, nv, a.grad.f, get);
        v.y = pack_word(4 * cc + 1, nv, a.grad.f, get);
        v.z = pack_word(4 * cc + 2, nv, a.grad.f, get);
        v.w = pack_word(4 * cc + 3, nv, a.grad.f, get);
        *reinterpret_cast<uint4*>(a.grad.ptr + c * a.grad.stride + 16 * cc) = v;
      }
    }
    __syncwarp();
  }
}

cudaError_t launch_collision(const RobotArgs& r, const SceneArgs& sc, const vapr_cost_params& p,
                             Packed pos, int64_t n, float* cost, Packed dist, Packed grad,
                             cudaStream_t st) {
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
  const size_t smem = coll_smem(sc.O, r.S, r.J, r.NP);
  const int per_sm = blocks_per_sm((const void*)collision_kernel, COLL_WARPS * 32, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t blocks = (n + COLL_WARPS - 1) / COLL_WARPS;
  const int64_t cap = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1);
  collision_kernel<<<(int)(blocks < cap ? blocks : cap), COLL_WARPS * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace vapr
