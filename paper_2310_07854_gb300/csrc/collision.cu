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
// evaluated where a conservative test cannot rule the pair out.  Cuboids
// are taken 64 at a time (lane l holds cuboids l and l + 32):
//   1. each link's bounding sphere (centroid of its spheres, radius from the
//      actual positions) is tested against every cuboid's bounding sphere;
//      the ballot of each test directly writes the link's candidate list;
//   2. every (sphere of the link, candidate) pair is enumerated densely over
//      the lanes and tested sphere-against-bounding-sphere;
//   3. survivors are compacted into a warp queue (ballot + popc) and the exact
//      distance runs 32 pairs at a time, branch-free, one pair per lane.
// A skipped pair provably has zero penetration (d_o(c) >= |c - t_o| - |h_o|);
// SLACK metres cover the float32 rounding of the tests.
//
// Determinism: queue entries of one sphere are contiguous and in ascending
// cuboid order, and they are added to the sphere's accumulator one per
// round (lanes of rank r in round r).  Every sphere therefore sums its
// contributions sequentially in cuboid order, independent of where queue
// flushes fall or which zero-penetration pairs survive the culling, so the
// result of a configuration does not depend on the batch it is in.  Active
// self pairs are applied one lane at a time in pair order.
#include "common.cuh"

namespace vapr {

constexpr int COLL_WARPS = 8;
constexpr int QCAP = 64;
constexpr int CHUNK = 64;  // cuboids per culling pass
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
  float4* cubA;     // [O][3]: (column k of R, t_k), k = 0..2
  float4* cubH;     // [O]: (h, unused)
  float4* cubC;     // [O]: (t, bounding radius + eta + slack)
  float4* P;        // [W][S]: (x, y, z, r)
  float4* acc;      // [W][S]: (D, gx, gy, gz)
  float4* lb;       // [W][J]: link bounding sphere (centre, radius)
  uint32_t* queue;  // [W][QCAP]: sphere | cuboid << 16
  uint16_t* cand;   // [W][J][CHUNK] candidate cuboids of each link
  int* ccount;      // [W][J]
  uint2* pairs;     // [NP]: (i | j << 16, bits of r_i + r_j + eta_s)
  int* order;       // [S] spheres grouped by link
  int* start;       // [J+1]
  int* linkof;      // [S] 0-based link
};

__host__ __device__ __forceinline__ size_t coll_smem_bytes(int O, int S, int J, int NP) {
  return sizeof(float4) * (5 * (size_t)O + 2 * COLL_WARPS * (size_t)S + COLL_WARPS * (size_t)J) +
         sizeof(uint2) * (size_t)NP + sizeof(uint32_t) * COLL_WARPS * QCAP +
         sizeof(int) * COLL_WARPS * (size_t)J +
         sizeof(int) * (2 * (size_t)S + J + 1) +
         sizeof(uint16_t) * COLL_WARPS * (size_t)J * CHUNK + 16;
}

__device__ __forceinline__ CollSmem carve(void* base, int O, int S, int J, int NP) {
  CollSmem m;
  float4* f4 = reinterpret_cast<float4*>(base);
  m.cubA = f4;
  f4 += 3 * O;
  m.cubH = f4;
  f4 += O;
  m.cubC = f4;
  f4 += O;
  m.P = f4;
  f4 += COLL_WARPS * S;
  m.acc = f4;
  f4 += COLL_WARPS * S;
  m.lb = f4;
  f4 += COLL_WARPS * J;
  m.pairs = reinterpret_cast<uint2*>(f4);
  uint32_t* u = reinterpret_cast<uint32_t*>(m.pairs + NP);
  m.queue = u;
  u += COLL_WARPS * QCAP;
  m.ccount = reinterpret_cast<int*>(u);
  u += COLL_WARPS * J;
  m.order = reinterpret_cast<int*>(u);
  m.start = m.order + S;
  m.linkof = m.start + J + 1;
  m.cand = reinterpret_cast<uint16_t*>(m.linkof + S);
  return m;
}

// Exact narrow phase of queue entries 0..cnt-1 (one per lane) and their
// accumulation, rank by rank, into acc (entries of a sphere are contiguous).
__device__ __forceinline__ void flush(const CollSmem& m, const float4* P, float4* acc,
                                      const uint32_t* queue, int cnt, float eta, float w_c) {
  const int lane = threadIdx.x & 31;
  const bool have = lane < cnt;
  const uint32_t e = have ? queue[lane] : 0xffffffffu;
  const int s = (int)(e & 0xffffu), o = (int)(e >> 16);
  float dD = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
  if (have) {
    const float4 c = P[s];
    const float4 A0 = m.cubA[3 * o], A1 = m.cubA[3 * o + 1], A2 = m.cubA[3 * o + 2];
    const float4 H = m.cubH[o];
    const float dx = c.x - A0.w, dy = c.y - A1.w, dz = c.z - A2.w;
    const float x0 = fmaf(A0.x, dx, fmaf(A0.y, dy, A0.z * dz));
    const float x1 = fmaf(A1.x, dx, fmaf(A1.y, dy, A1.z * dz));
    const float x2 = fmaf(A2.x, dx, fmaf(A2.y, dy, A2.z * dz));
    const float u0 = fabsf(x0) - H.x, u1 = fabsf(x1) - H.y, u2 = fabsf(x2) - H.z;
    const float v0 = fmaxf(u0, 0.f), v1 = fmaxf(u1, 0.f), v2 = fmaxf(u2, 0.f);
    const float n2 = fmaf(v0, v0, fmaf(v1, v1, v2 * v2));
    const bool outside = u0 > 0.f || u1 > 0.f || u2 > 0.f;
    // inside: the face of the largest u (lowest axis on ties)
    const int k = (u0 >= u1 && u0 >= u2) ? 0 : (u1 >= u2 ? 1 : 2);
    const float umax = fmaxf(u0, fmaxf(u1, u2));
    const float rs = n2 > 0.f ? rsqrtf(n2) : 0.f;  // 1/|max(u,0)|
    const float d = outside ? n2 * rs : umax;
    const float pen = c.w + eta - d;
    if (pen > 0.f) {
      const float inv = outside ? rs : 0.f;
      const float s0 = x0 >= 0.f ? 1.f : -1.f, s1 = x1 >= 0.f ? 1.f : -1.f,
                  s2 = x2 >= 0.f ? 1.f : -1.f;
      const float l0 = outside ? s0 * v0 * inv : (k == 0 ? s0 : 0.f);
      const float l1 = outside ? s1 * v1 * inv : (k == 1 ? s1 : 0.f);
      const float l2 = outside ? s2 * v2 * inv : (k == 2 ? s2 : 0.f);
      dD = pen;  // gradient of the hinge: -grad d, scaled by w_coll
      gx = -w_c * fmaf(A0.x, l0, fmaf(A1.x, l1, A2.x * l2));
      gy = -w_c * fmaf(A0.y, l0, fmaf(A1.y, l1, A2.y * l2));
      gz = -w_c * fmaf(A0.z, l0, fmaf(A1.z, l1, A2.z * l2));
    }
  }
  // rank of each entry within its sphere's (contiguous) run
  const int prev = __shfl_up_sync(FULL, s, 1);
  const bool head = lane == 0 || !have || s != prev;
  const unsigned heads = __ballot_sync(FULL, head);
  const int rank = lane - (31 - __clz(heads & (FULL >> (31 - lane))));
  const int rounds = __reduce_max_sync(FULL, have ? rank : 0);
  for (int r = 0; r <= rounds; ++r) {
    if (have && rank == r) {
      float4 a = acc[s];
      a.x += dD;
      a.y += gx;
      a.z += gy;
      a.w += gz;
      acc[s] = a;
    }
    __syncwarp();
  }
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
    m.cubA[3 * o + 0] = make_float4(p[0], p[3], p[6], p[9]);
    m.cubA[3 * o + 1] = make_float4(p[1], p[4], p[7], p[10]);
    m.cubA[3 * o + 2] = make_float4(p[2], p[5], p[8], p[11]);
    m.cubH[o] = make_float4(hx, hy, hz, 0.f);
    m.cubC[o] = make_float4(p[9], p[10], p[11],
                            sqrtf(hx * hx + hy * hy + hz * hz) + a.eta + SLACK);
  }
  for (int p = threadIdx.x; p < NP; p += blockDim.x) {
    const int i = clampi(a.r.pairs[2 * p], 0, S - 1), j = clampi(a.r.pairs[2 * p + 1], 0, S - 1);
    m.pairs[p] = make_uint2((uint32_t)i | ((uint32_t)j << 16),
                            __float_as_uint(a.r.sphere_local[4 * i + 3] +
                                            a.r.sphere_local[4 * j + 3] + a.eta_s));
  }
  for (int i = threadIdx.x; i < COLL_WARPS * S; i += blockDim.x) {
    const int s = i % S;
    m.P[i] = make_float4(0.f, 0.f, 0.f, a.r.sphere_local[4 * s + 3]);
    m.acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
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
  uint32_t* queue = m.queue + wid * QCAP;
  uint16_t* cand = m.cand + wid * J * CHUNK;
  int* ccount = m.ccount + wid * J;
  const unsigned lt_mask = (1u << lane) - 1u;

  for (int64_t c = blockIdx.x * (int64_t)COLL_WARPS + wid; c < a.n;
       c += (int64_t)gridDim.x * COLL_WARPS) {
    // ---- 1. sphere centres of this configuration (coalesced 16-byte loads)
    {
      const uint32_t* row = reinterpret_cast<const uint32_t*>(a.pos.ptr + c * a.pos.stride);
      const int nv = 3 * S;
      dispatch_kind(a.pos.f.kind, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        const int kw = per_word<K>(a.pos.f);
        const int nw = (nv + kw - 1) / kw;
        for (int w = lane; w < nw; w += 32)
          unpack_word_t<K>(__ldg(row + w), w, nv, a.pos.f, [&](int i, float x) {
            const int s = i / 3;
            reinterpret_cast<float*>(P + s)[i - 3 * s] = x;
          });
      });
    }
    // ---- 2. link bounding spheres: centred on the link's middle sphere, the
    //      radius the largest |c_s - centre| + r_s over the link (integer
    //      atomicMax on non-negative float bits)
    if (lane < J) {
      const int b = m.start[lane], e = m.start[lane + 1];
      const float4 ctr = e > b ? P[m.order[b + (e - b) / 2]] : make_float4(0.f, 0.f, 0.f, 0.f);
      lb[lane] = make_float4(ctr.x, ctr.y, ctr.z, e > b ? 0.f : -1.f);
    }
    __syncwarp();
    for (int s = lane; s < S; s += 32) {
      const float4 p = P[s];
      const float4 b = lb[m.linkof[s]];
      const float dx = p.x - b.x, dy = p.y - b.y, dz = p.z - b.z;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const float rad = (d2 > 0.f ? d2 * rsqrtf(d2) : 0.f) + p.w + SLACK;
      atomicMax(reinterpret_cast<int*>(lb + m.linkof[s]) + 3, __float_as_int(rad));
    }
    __syncwarp();

    // ---- 3. environment: cull, compact, evaluate
    for (int base = 0; base < O; base += CHUNK) {
      const int o0 = base + lane, o1 = base + 32 + lane;
      const float4 C0 = o0 < O ? m.cubC[o0] : make_float4(0.f, 0.f, 0.f, -1e30f);
      const float4 C1 = o1 < O ? m.cubC[o1] : make_float4(0.f, 0.f, 0.f, -1e30f);
      for (int L = 0; L < J; ++L) {
        const float4 b = lb[L];
        bool n0 = false, n1 = false;
        if (b.w >= 0.f) {
          const float ax = b.x - C0.x, ay = b.y - C0.y, az = b.z - C0.z;
          const float t0 = b.w + C0.w;
          n0 = C0.w > 0.f && fmaf(ax, ax, fmaf(ay, ay, az * az)) < t0 * t0;
          const float bx = b.x - C1.x, by = b.y - C1.y, bz = b.z - C1.z;
          const float t1 = b.w + C1.w;
          n1 = C1.w > 0.f && fmaf(bx, bx, fmaf(by, by, bz * bz)) < t1 * t1;
        }
        const unsigned m0 = __ballot_sync(FULL, n0), m1 = __ballot_sync(FULL, n1);
        uint16_t* cl = cand + L * CHUNK;
        if (n0) cl[__popc(m0 & lt_mask)] = (uint16_t)o0;
        if (n1) cl[__popc(m0) + __popc(m1 & lt_mask)] = (uint16_t)o1;
        if (lane == 0) ccount[L] = __popc(m0) + __popc(m1);
      }
      __syncwarp();
      // (sphere of link L, candidate) pairs, sphere-major, densely over lanes
      int qn = 0;
      for (int L = 0; L < J; ++L) {
        const int cl_n = ccount[L];
        const int s0 = m.start[L], ns = m.start[L + 1] - s0;
        const int total = cl_n * ns;
        if (total == 0) continue;
        const float rcp = 1.0f / (float)cl_n;
        const uint16_t* cl = cand + L * CHUNK;
        for (int t = 0; t < total; t += 32) {
          const int idx = t + lane;
          bool nr = false;
          int s = 0, o = 0;
          if (idx < total) {
            int js = __float2int_rd(((float)idx + 0.5f) * rcp);  // idx / cl_n
            int jc = idx - js * cl_n;
            if (jc >= cl_n) { ++js; jc -= cl_n; }  // exact quotient whatever the rounding
            if (jc < 0) { --js; jc += cl_n; }
            s = m.order[s0 + js];
            o = cl[jc];
            const float4 p = P[s];
            const float4 C = m.cubC[o];
            const float dx = p.x - C.x, dy = p.y - C.y, dz = p.z - C.z;
            const float thr = p.w + C.w;
            nr = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < thr * thr;
          }
          const unsigned bal = __ballot_sync(FULL, nr);
          if (nr) queue[qn + __popc(bal & lt_mask)] = (uint32_t)s | ((uint32_t)o << 16);
          qn += __popc(bal);
          if (qn >= 32) {
            __syncwarp();
            flush(m, P, acc, queue, 32, a.eta, a.w_c);
            const int rest = qn - 32;
            const uint32_t moved = lane < rest ? queue[32 + lane] : 0u;
            __syncwarp();
            if (lane < rest) queue[lane] = moved;
            qn = rest;
            __syncwarp();
          }
        }
      }
      __syncwarp();
      if (qn > 0) flush(m, P, acc, queue, qn, a.eta, a.w_c);  // keep runs within a chunk
      __syncwarp();
    }

    // ---- 4. self-collision over the pair list
    float selfsum = 0.f;
    for (int pb = 0; pb < NP; pb += 32) {
      const int p = pb + lane;
      bool act = false;
      float pen = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
      int i = 0, j = 0;
      if (p < NP) {
        const uint2 pr = m.pairs[p];
        i = (int)(pr.x & 0xffffu);
        j = (int)(pr.x >> 16);
        const float4 ci = P[i], cj = P[j];
        const float dx = ci.x - cj.x, dy = ci.y - cj.y, dz = ci.z - cj.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float thr = __uint_as_float(pr.y);
        if (d2 < thr * thr) {
          const float rs = d2 > 0.f ? rsqrtf(d2) : 0.f;
          pen = thr - d2 * rs;
          act = pen > 0.f;
          const float inv = a.w_s * rs;  // 0 at zero distance: no gradient
          ux = dx * inv;
          uy = dy * inv;
          uz = dz * inv;
        }
      }
      unsigned am = __ballot_sync(FULL, act);
      if (act) selfsum += pen;
      while (am) {  // active pairs are rare: apply them one lane at a time, in pair order
        const int l = __ffs(am) - 1;
        if (lane == l) {
          float4 vi = acc[i];
          vi.y -= ux;
          vi.z -= uy;
          vi.w -= uz;
          acc[i] = vi;
          float4 vj = acc[j];
          vj.y += ux;
          vj.z += uy;
          vj.w += uz;
          acc[j] = vj;
        }
        __syncwarp();
        am &= am - 1u;
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
      uint32_t* out = reinterpret_cast<uint32_t*>(a.dist.ptr + c * a.dist.stride);
      const int words = (int)(a.dist.stride / 4);
      dispatch_kind(a.dist.f.kind, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        for (int w = lane; w < words; w += 32)
          out[w] = pack_word_t<K>(w, S, a.dist.f, [&](int i) { return acc[i].x; });
      });
    }
    if (a.grad.ptr) {
      uint32_t* out = reinterpret_cast<uint32_t*>(a.grad.ptr + c * a.grad.stride);
      const int words = (int)(a.grad.stride / 4), nv = 3 * S;
      dispatch_kind(a.grad.f.kind, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        for (int w = lane; w < words; w += 32)
          out[w] = pack_word_t<K>(w, nv, a.grad.f, [&](int i) {
            const int s = i / 3;
            return reinterpret_cast<const float*>(acc + s)[1 + i - 3 * s];
          });
      });
    }
    __syncwarp();
    for (int s = lane; s < S; s += 32) acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
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
  const size_t smem = coll_smem_bytes(sc.O, r.S, r.J, r.NP);
  const int per_sm = blocks_per_sm((const void*)collision_kernel, COLL_WARPS * 32, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t blocks = (n + COLL_WARPS - 1) / COLL_WARPS;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  collision_kernel<<<(int)(blocks < cap ? blocks : cap), COLL_WARPS * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace vapr
