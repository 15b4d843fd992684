// The three stages of the path as block-, warp- and thread-level device
// functions, shared by the single-problem kernels (fk.cu, collision.cu,
// backward.cu) and the uneven multi-problem kernel (batched.cu), so every
// entry point runs the same arithmetic on a configuration.
//
//   FK         (Sec. II-B; iteration step 2 of Sec. III-B):
//              T_0 = I, T_j = T_{j-1} F_j Rz(q_j), c_s = T_link(s) [p_s; 1]
//   collision  (iteration steps 3-4): box distance d = |max(u,0)| +
//              min(max u, 0), u = |R^T (c - t)| - h;
//              D_s = sum_o max(0, r_s + eta - d_o(c_s));
//              P_ij = max(0, r_i + r_j + eta_s - |c_i - c_j|);
//              C = w_c sum D + w_s sum P;  G = dC/dc
//   backward   (iteration step 5): J_j = a_j . M_{>=j} - b_j . F_{>=j},
//              F = sum G_s, M = sum c_s x G_s, b_j = a_j x o_j
#pragma once

#include "common.cuh"
#include "grid.cuh"

namespace vapr {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Hands out 16-byte-aligned slices of a buffer in a fixed order.  With a
// null base it only counts bytes, so the host sizes shared memory with the
// same code the device uses to carve it.
struct Bump {
  char* base;
  size_t off;
  __host__ __device__ explicit Bump(void* b) : base((char*)b), off(0) {}
  template <typename T>
  __host__ __device__ T* take(size_t n) {
    off = (off + 15) & ~(size_t)15;
    T* r = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += n * sizeof(T);
    return r;
  }
  __host__ __device__ size_t bytes() const { return (off + 15) & ~(size_t)15; }
};

// nw equal per-warp working sets, carve(Bump&) each, one after another from
// b's next 16-byte boundary: the layout of nw calls of carve(b) in turn,
// computed with two calls (one for the stride, one for warp mine's
// pointers, left in carve's outputs).
template <typename Carve>
__host__ __device__ inline void carve_warps(Bump& b, int nw, int mine, Carve carve) {
  Bump probe(nullptr);
  carve(probe);
  const size_t stride = probe.bytes();
  b.off = b.bytes();
  Bump mb(b.base);
  mb.off = b.off + (size_t)mine * stride;
  carve(mb);
  b.off += (size_t)nw * stride;
}

// ------------------------------------------------------------ robot tables
// Self-collision clusters: runs of at most CL consecutive spheres of one
// link (in the link-grouped order), at most cluster_bound(S, J) of them.
constexpr int CL = 3;
__host__ __device__ constexpr int cluster_bound(int S, int J) { return (S + (CL - 1) * J) / CL + 1; }

struct RobotSm {
  float4* F;      // [3J] rows of F_j: (R_d0, R_d1, R_d2, t_d)
  float4* sph;    // [S] (p, r)
  int* link0;     // [S] 0-based link, clamped into range
  int* order;     // [S] spheres grouped by link (stable)
  int* start;     // [J+1] first slot of each link in order
  int* cl_start;  // [NC+1] cluster c = spheres order[cl_start[c] .. cl_start[c+1])
  int* cl_of;     // [S] cluster of each sphere
  int* cl_sph;    // [NC] cluster c's spheres: s0 | s1 << 8 | s2 << 16 | count << 24
  int* n_cl;      // [2] NC, and the exponent e of the self terms' fixed point (self_pairs)
};

__host__ __device__ inline void carve_robot(Bump& b, int J, int S, RobotSm& r) {
  r.F = b.take<float4>(3 * J);
  r.sph = b.take<float4>(S);
  r.link0 = b.take<int>(S);
  r.order = b.take<int>(S);
  r.start = b.take<int>(J + 1);
  r.cl_start = b.take<int>(cluster_bound(S, J) + 1);
  r.cl_of = b.take<int>(S);
  r.cl_sph = b.take<int>(cluster_bound(S, J));
  r.n_cl = b.take<int>(2);
}

// Block-cooperative (every thread calls it); the caller synchronises the
// block afterwards.  The spheres are sorted by link (stably) in parallel:
// each sphere's slot counts the spheres before it in (link, index) order.
__device__ inline void load_robot(const RobotArgs& a, const RobotSm& r) {
  const int J = a.J, S = a.S;
  for (int i = threadIdx.x; i < 3 * J; i += blockDim.x) {
    const int j = i / 3, d = i - 3 * j;
    const float* F = a.joint_fixed + 12 * j;
    r.F[i] = make_float4(F[3 * d], F[3 * d + 1], F[3 * d + 2], F[9 + d]);
  }
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    r.sph[s] = reinterpret_cast<const float4*>(a.sphere_local)[s];
    r.link0[s] = clampi(a.sphere_link[s], 1, J) - 1;
  }
  __syncthreads();
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const int l = r.link0[s];
    int slot = 0;
    for (int t = 0; t < S; ++t) {
      const int lt = r.link0[t];
      slot += (lt < l) || (lt == l && t < s);
    }
    r.order[slot] = s;
  }
  for (int j = threadIdx.x; j <= J; j += blockDim.x) {  // first slot of each link
    int c = 0;
    for (int t = 0; t < S; ++t) c += r.link0[t] < j;
    r.start[j] = c;
  }
}

// Block-cooperative, after load_robot and a block synchronisation: the
// self-collision clusters (runs of up to CL spheres of one link in the
// link-sorted order).  Ends with the block synchronised.
__device__ inline void load_clusters(int J, int S, const RobotSm& r) {
  auto clusters_before = [&](int j) {
    int c = 0;
    for (int i = 0; i < j; ++i) c += (r.start[i + 1] - r.start[i] + CL - 1) / CL;
    return c;
  };
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    const int c0 = clusters_before(j), nj = r.start[j + 1] - r.start[j];
    for (int c = 0; c * CL < nj; ++c) r.cl_start[c0 + c] = r.start[j] + c * CL;
    if (j == J - 1) {
      const int nc = c0 + (nj + CL - 1) / CL;
      r.cl_start[nc] = S;
      r.n_cl[0] = nc;
    }
  }
  for (int k = threadIdx.x; k < S; k += blockDim.x) {
    const int s = r.order[k], j = r.link0[s];
    r.cl_of[s] = clusters_before(j) + (k - r.start[j]) / CL;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < r.n_cl[0]; c += blockDim.x) {
    const int k0 = r.cl_start[c], k1 = r.cl_start[c + 1];
    int packed = (k1 - k0) << 24;
    for (int k = k0; k < k1; ++k) packed |= r.order[k] << (8 * (k - k0));
    r.cl_sph[c] = packed;
  }
  __syncthreads();
}

// ------------------------------------------------------------ FK (thread)
// One step of the joint chain: (R, t) = T_{j-1} becomes T_j = T_{j-1} F_j Rz(q_j).
// sin and cos of a joint angle, to about one float32 ulp.  Cody-Waite
// reduction to r = q - k pi/2 in [-pi/4, pi/4] (k the integer nearest
// 2q/pi; pi/2 split into its float and the float of the remainder, each
// subtracted by one fused multiply-add: exact first step for |k| < 2^21,
// and r off by about 1e-15 |k| plus one rounding), then the Taylor series
// of sin r to r^9 and of cos r to r^10, whose truncation errors on
// [-pi/4, pi/4] are below 2e-9 and 2e-10, evaluated by Horner's rule; the
// quadrant k mod 4 picks (sin, cos) = (s, c), (c, -s), (-s, -c), (-c, s).
__device__ __forceinline__ void joint_sincos(float q, float& sn, float& cs) {
  const float k = rintf(q * 0.636619772f);  // 2 / pi
  float r = fmaf(-k, 1.57079637f, q);       // float(pi/2) = pi/2 + 4.3711388e-8
  r = fmaf(k, 4.37113883e-8f, r);
  const float r2 = r * r;
  // sin r = r (1 - r^2/3! + r^4/5! - r^6/7! + r^8/9!)
  float ps = fmaf(r2, 2.75573192e-6f, -1.98412698e-4f);
  ps = fmaf(r2, ps, 8.33333333e-3f);
  ps = fmaf(r2, ps, -1.66666667e-1f);
  const float sr = fmaf(r * r2, ps, r);
  // cos r = 1 - r^2/2! + r^4/4! - r^6/6! + r^8/8! - r^10/10!
  float pc = fmaf(r2, -2.75573192e-7f, 2.48015873e-5f);
  pc = fmaf(r2, pc, -1.38888889e-3f);
  pc = fmaf(r2, pc, 4.16666667e-2f);
  pc = fmaf(r2, pc, -0.5f);
  const float cr = fmaf(r2, pc, 1.f);
  const int quad = (int)k & 3;
  const float s_ = (quad & 1) ? cr : sr, c_ = (quad & 1) ? sr : cr;
  sn = (quad & 2) ? -s_ : s_;
  cs = ((quad + 1) & 2) ? -c_ : c_;
}

__device__ __forceinline__ void joint_step(const RobotSm& r, int j, float qj, float (&R)[3][3], float (&t)[3]) {
  const float4 f0 = r.F[3 * j], f1 = r.F[3 * j + 1], f2 = r.F[3 * j + 2];
  float B[3][3], tb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {  // T_{j-1} F_j
    B[k][0] = fmaf(R[k][0], f0.x, fmaf(R[k][1], f1.x, R[k][2] * f2.x));
    B[k][1] = fmaf(R[k][0], f0.y, fmaf(R[k][1], f1.y, R[k][2] * f2.y));
    B[k][2] = fmaf(R[k][0], f0.z, fmaf(R[k][1], f1.z, R[k][2] * f2.z));
    tb[k] = fmaf(R[k][0], f0.w, fmaf(R[k][1], f1.w, fmaf(R[k][2], f2.w, t[k])));
  }
  float sn, cs;
  joint_sincos(qj, sn, cs);
#pragma unroll
  for (int k = 0; k < 3; ++k) {  // ... Rz(q_j)
    R[k][0] = fmaf(cs, B[k][0], sn * B[k][1]);
    R[k][1] = fmaf(cs, B[k][1], -sn * B[k][0]);
    R[k][2] = B[k][2];
    t[k] = tb[k];
  }
}

// The joint chain of one configuration into myT: 3 float4 per joint, rows
// (R_d0, R_d1, R_d2, t_d).
__device__ __forceinline__ void fk_chain(const RobotSm& r, int J, const float* q, float4* myT) {
  float R[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
  float t[3] = {0.f, 0.f, 0.f};
  for (int j = 0; j < J; ++j) {
    joint_step(r, j, q[j], R, t);
#pragma unroll
    for (int k = 0; k < 3; ++k) myT[3 * j + k] = make_float4(R[k][0], R[k][1], R[k][2], t[k]);
  }
}

// The q rows of configurations c0 .. c0+31 into dst (32 x J floats,
// row-major): rows below n by 4-byte asynchronous copies (cp.async),
// committed as one group of this thread, rows past n as zeros; q_wait makes
// them visible to the warp.
__device__ __forceinline__ void q_prefetch(float* dst, const float* q, int64_t c0, int64_t n, int J, int lane) {
  const int rows = (int)(n - c0 < 32 ? n - c0 : 32);
  const float* src = q + c0 * J;
  for (int i = lane; i < rows * J; i += 32)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst + i)),
                 "l"(src + i)
                 : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int i = rows * J + lane; i < 32 * J; i += 32) dst[i] = 0.f;
}
__device__ __forceinline__ void q_wait() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
}
// The same when `after` (0..3) later commit groups of this thread may stay
// in flight (copies issued after the q rows).
__device__ __forceinline__ void q_wait_after(int after) {
  switch (after) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
  }
  __syncwarp();
}

// Packed sphere-centre row of one configuration from its transforms T;
// lanes take the row's 32-bit words (padding words written as zero).
template <int K>
__device__ __forceinline__ void fk_store_pos(const RobotSm& r, int S, const float4* T,
                                             uint32_t* out, int words, const DevFmt& f, int lane) {
  const int nv = 3 * S;
  for (int w = lane; w < words; w += 32)
    out[w] = pack_word_t<K>(w, nv, f, [&](int i) {
      const int s = i / 3, d = i - 3 * s;
      const float4 row = T[3 * r.link0[s] + d];
      const float4 p = r.sph[s];
      return fmaf(row.x, p.x, fmaf(row.y, p.y, fmaf(row.z, p.z, row.w)));
    });
}

// ------------------------------------------------------- collision (warp)
// (SLACK, the metres that cover float32 rounding of the culls: grid.cuh)

struct SceneSm {
  float4* cubA;  // [O][3]: (column k of R, t_k), k = 0..2
  float4* cubH;  // [O]: (half extents, unused)
  float4* cubC;  // [O]: (centre, bounding radius + eta + SLACK)
  // self pairs, grouped by cluster pair (load_self)
  uint32_t* pairs;      // [NP]: i | j << 16, cluster-pair major (threshold (r_i + r_j) + eta_s from the radii)
  uint16_t* cp;         // [NG]: cluster pair a | b << 8 (a <= b), in increasing a * NC + b
  uint16_t* cp_start;   // [NG+1]: its pairs are pairs[cp_start[g] .. cp_start[g+1])
  int* self_meta;       // [2]: NG, bits of eta_s
};

__host__ __device__ inline int pair_groups_bound(int NP, int NCB) {
  return NP < NCB * NCB ? NP : NCB * NCB;
}

// NCB: cluster_bound of the largest robot the tables serve.
__host__ __device__ inline void carve_scene(Bump& b, int O, int NP, int NCB, SceneSm& s) {
  s.cubA = b.take<float4>(3 * O);
  s.cubH = b.take<float4>(O);
  s.cubC = b.take<float4>(O);
  const int NG = pair_groups_bound(NP, NCB);
  s.pairs = b.take<uint32_t>(NP);
  s.cp = b.take<uint16_t>(NG);
  s.cp_start = b.take<uint16_t>(NG + 1);
  s.self_meta = b.take<int>(2);
}

// Scratch of load_self; callers lay it over buffers that are not live
// while the tables are built (the warps' working sets).
struct SelfScratch {
  uint32_t* word;      // [NP] per pair: i | j << 7 | (key, then cluster pair) << 14
  int* cursor;         // [NG] pair counts, then fill cursors
  uint16_t* g_of_key;  // [NC^2]
  uint32_t* keymap;    // [NC^2 / 32] keys that occur
  int* keybase;        // [NC^2 / 32] keys that occur in earlier keymap words
  int* deg;            // [S] pairs naming each sphere (a pair (i, i) twice)
};

__host__ __device__ inline void carve_self_scratch(Bump& b, int NP, int NCB, int S, SelfScratch& t) {
  const int keys = NP > 0 ? NCB * NCB : 0;
  t.deg = b.take<int>(S);
  t.word = b.take<uint32_t>(NP);
  t.cursor = b.take<int>(pair_groups_bound(NP, NCB));
  t.g_of_key = b.take<uint16_t>(keys);
  t.keymap = b.take<uint32_t>((keys + 31) / 32);
  t.keybase = b.take<int>((keys + 31) / 32);
}
static_assert(VAPR_MAX_SPHERES <= 128, "sphere indices are packed in 7 bits");

__device__ inline void load_scene(const RobotArgs& r, const SceneArgs& sc, float eta, float eta_s,
                                  const SceneSm& m) {
  const int O = sc.O, S = r.S;
  for (int o = threadIdx.x; o < O; o += blockDim.x) {
    const float* p = sc.pose + 12 * o;
    const float hx = sc.half[3 * o], hy = sc.half[3 * o + 1], hz = sc.half[3 * o + 2];
    m.cubA[3 * o + 0] = make_float4(p[0], p[3], p[6], p[9]);
    m.cubA[3 * o + 1] = make_float4(p[1], p[4], p[7], p[10]);
    m.cubA[3 * o + 2] = make_float4(p[2], p[5], p[8], p[11]);
    m.cubH[o] = make_float4(hx, hy, hz, 0.f);
    m.cubC[o] = make_float4(p[9], p[10], p[11], sqrtf(hx * hx + hy * hy + hz * hz) + eta + SLACK);
  }
  (void)S;
  (void)eta_s;
}

// Inclusive warp scan of v.
__device__ __forceinline__ int warp_scan(int v, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int t = __shfl_up_sync(FULL_MASK, v, off);
    if (lane >= off) v += t;
  }
  return v;
}

// Block-cooperative (all threads, block converged; load_robot's and
// load_clusters' tables complete): the self-pair table grouped by cluster
// pair.  Cluster pairs are numbered in increasing key a * NC + b and the
// pairs within one keep the robot's order (a stable counting sort, so the
// table does not depend on thread timing).  The robot's pair list is read
// once, in parallel; the one serial pass (the scatter, a warp over 32 pairs
// at a time) touches shared memory only.  Ends with the block synchronised.
__device__ inline void load_self(const RobotArgs& r, const RobotSm& rb, const SceneSm& m,
                                 const SelfScratch& t, float eta_s) {
  const int NP = r.NP, NC = rb.n_cl[0], keys = NC * NC, kw = (keys + 31) / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (NP == 0) {  // no pairs: an empty table (the scratch is sized for none)
    if (threadIdx.x == 0) {
      m.self_meta[0] = 0;
      m.self_meta[1] = (int)__float_as_uint(eta_s);
      m.cp_start[0] = 0;
      rb.n_cl[1] = 30;
    }
    __syncthreads();
    return;
  }
  __shared__ int s_maxdeg;
  for (int k = threadIdx.x; k < kw; k += blockDim.x) t.keymap[k] = 0u;
  for (int k = threadIdx.x; k < r.S; k += blockDim.x) t.deg[k] = 0;
  if (threadIdx.x == 0) s_maxdeg = 1;
  __syncthreads();
  for (int p = threadIdx.x; p < NP; p += blockDim.x) {
    const int i = clampi(r.pairs[2 * p], 0, r.S - 1), j = clampi(r.pairs[2 * p + 1], 0, r.S - 1);
    const int a = rb.cl_of[i], b = rb.cl_of[j];
    const int key = a <= b ? a * NC + b : b * NC + a;
    t.word[p] = (uint32_t)i | ((uint32_t)j << 7) | ((uint32_t)key << 14);
    atomicOr(&t.keymap[key >> 5], 1u << (key & 31));
    atomicAdd(&t.deg[i], 1);
    atomicAdd(&t.deg[j], 1);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < r.S; k += blockDim.x) atomicMax(&s_maxdeg, t.deg[k]);
  __syncthreads();
  // The self terms' fixed point (self_pairs): a sphere's sum of at most
  // maxdeg unit-vector components times 2^e, e = 30 - floor(log2 maxdeg),
  // stays below 2^31 (maxdeg 2^(30-e+1) - 1 at most: 2^31 - 2^e).
  if (threadIdx.x == 0) rb.n_cl[1] = __clz(s_maxdeg) - 1;
  if (warp == 0) {  // keys occurring in earlier words
    int base = 0;
    for (int k0 = 0; k0 < kw; k0 += 32) {
      const int c = k0 + lane < kw ? __popc(t.keymap[k0 + lane]) : 0;
      const int incl = warp_scan(c, lane);
      if (k0 + lane < kw) t.keybase[k0 + lane] = base + incl - c;
      base += __shfl_sync(FULL_MASK, incl, 31);
    }
    if (lane == 0) {
      m.self_meta[0] = base;
      m.self_meta[1] = (int)__float_as_uint(eta_s);
    }
  }
  __syncthreads();
  for (int key = threadIdx.x; key < keys; key += blockDim.x) {  // number the keys that occur
    const uint32_t bits = t.keymap[key >> 5], bit = 1u << (key & 31);
    if (bits & bit) {
      const int g = t.keybase[key >> 5] + __popc(bits & (bit - 1u));
      const int a = key / NC;
      t.g_of_key[key] = (uint16_t)g;
      m.cp[g] = (uint16_t)(a | ((key - a * NC) << 8));
      t.cursor[g] = 0;
    }
  }
  __syncthreads();
  const int NG = m.self_meta[0];
  for (int p = threadIdx.x; p < NP; p += blockDim.x) {  // pairs per cluster pair
    const uint32_t wd = t.word[p];
    const int g = t.g_of_key[wd >> 14];
    t.word[p] = (wd & 0x3fffu) | ((uint32_t)g << 14);
    atomicAdd(&t.cursor[g], 1);
  }
  __syncthreads();
  if (warp == 0) {
    int base = 0;  // exclusive scan of the counts: group starts, and the fill cursors
    for (int g0 = 0; g0 < NG; g0 += 32) {
      const int g = g0 + lane;
      const int c = g < NG ? t.cursor[g] : 0;
      const int incl = warp_scan(c, lane);
      if (g < NG) {
        m.cp_start[g] = (uint16_t)(base + incl - c);
        t.cursor[g] = base + incl - c;
      }
      base += __shfl_sync(FULL_MASK, incl, 31);
    }
    if (lane == 0) m.cp_start[NG] = (uint16_t)base;
    __syncwarp();
    for (int p0 = 0; p0 < NP; p0 += 32) {  // stable scatter, in pair order
      const int p = p0 + lane;
      const uint32_t wd = p < NP ? t.word[p] : 0u;
      const int g = p < NP ? (int)(wd >> 14) : -1 - lane;
      const unsigned same = __match_any_sync(FULL_MASK, g);
      if (p < NP) {
        const int i = (int)(wd & 0x7fu), j = (int)((wd >> 7) & 0x7fu);
        m.pairs[t.cursor[g] + __popc(same & ((1u << lane) - 1u))] = (uint32_t)i | ((uint32_t)j << 16);
      }
      __syncwarp();
      if (p < NP && lane == __ffs(same) - 1) t.cursor[g] += __popc(same);
      __syncwarp();
    }
  }
  __syncthreads();
}

// ------------------------------------------------- prebuilt robot tables
// What load_robot, load_clusters and load_self build in shared memory
// depends on the robot alone: vapr_robot_tables_build stores it once in
// global memory (RobotImage: a header, then the shared-memory arrays in the
// same order and 16-byte alignment), and a block whose robot carries such
// tables copies them (load_robot_self) instead of building them, after
// checking that they were made for the robot's current contents (a hash of
// its arrays, as the scene grid is checked) and are intact (a checksum of
// the image body).  Copied and built tables are the same bytes.
constexpr uint32_t TABLES_MAGIC = 0x56525443u;

struct TablesHeader {
  uint32_t magic, J, S, NP, hash, NG;
  uint32_t body_words, body_hash;  // the 32-bit words after the header, and their hash
  uint32_t pad[8];  // 64 bytes
};
static_assert(sizeof(TablesHeader) == 64, "the arrays after the header stay 16-byte aligned");

struct RobotImage {
  TablesHeader* h;
  RobotSm rb;
  uint32_t* pairs;
  uint16_t* cp;
  uint16_t* cp_start;
};

__host__ __device__ inline void carve_image(Bump& b, int J, int S, int NP, RobotImage& im) {
  im.h = b.take<TablesHeader>(1);
  carve_robot(b, J, S, im.rb);
  const int NG = pair_groups_bound(NP, cluster_bound(S, J));
  im.pairs = b.take<uint32_t>(NP);
  im.cp = b.take<uint16_t>(NG);
  im.cp_start = b.take<uint16_t>(NG + 1);
}

// Hash of the robot's arrays (and sizes): the sum of hash_word over the
// joint, sphere, link and pair words in that order, as the scene grid's
// hash (all four arrays are 16-byte aligned).
__device__ __forceinline__ uint32_t robot_hash_part(const RobotArgs& r, int tid, int stride) {
  const int n0 = 12 * r.J, n1 = 4 * r.S, n2 = r.S, n3 = 2 * r.NP;
  uint32_t s = hash_words<true>(reinterpret_cast<const uint32_t*>(r.joint_fixed), n0, 0u, tid, stride) +
               hash_words<true>(reinterpret_cast<const uint32_t*>(r.sphere_local), n1, (uint32_t)n0, tid, stride) +
               hash_words<true>(reinterpret_cast<const uint32_t*>(r.sphere_link), n2, (uint32_t)(n0 + n1), tid,
                                stride);
  if (n3 > 0)
    s += hash_words<true>(reinterpret_cast<const uint32_t*>(r.pairs), n3, (uint32_t)(n0 + n1 + n2), tid, stride);
  if (tid == 0) s += hash_word((uint32_t)r.J ^ (uint32_t)r.S << 8 ^ (uint32_t)r.NP << 16, 0xffffffffu);
  return s;
}

// Checksum of words [0, nw) of a table image's body (16-byte aligned, nw a
// multiple of 4): the sum of word i times 2i + 1 (mod 2^32), which any
// change of a single word alters (odd factors are invertible), at one
// multiply-add per word, four words per load.
__device__ __forceinline__ uint32_t body_hash_part(const uint32_t* body, uint32_t nw, int tid, int stride) {
  uint32_t s = 0;
  for (uint32_t q = tid; q < nw / 4u; q += stride) {
    const uint4 v = __ldcg(reinterpret_cast<const uint4*>(body) + q);
    const uint32_t i = 8u * q + 1u;  // 2 (4q) + 1
    s += v.x * i + v.y * (i + 2u) + v.z * (i + 4u) + v.w * (i + 6u);
  }
  return s;
}

// 16-byte granules of an array (its padding to 16 bytes included).
__device__ __forceinline__ void copy_granules(void* dst, const void* src, size_t bytes) {
  const int n = (int)((bytes + 15) / 16);
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    reinterpret_cast<uint4*>(dst)[i] = __ldg(reinterpret_cast<const uint4*>(src) + i);
}

// Block-cooperative (every thread calls it, the block converged): rb
// (load_robot, load_clusters) and m's self tables (load_self) for eta_s,
// copied from r.tables when they were made for this robot, else built.
// Ends with the block synchronised.
__device__ inline void load_robot_self(const RobotArgs& r, const RobotSm& rb, const SceneSm& m,
                                       const SelfScratch& t, float eta_s) {
  __shared__ uint32_t s_hash, s_body;
  __shared__ int s_ok;
  const TablesHeader* h = static_cast<const TablesHeader*>(r.tables);
  bool ok = false;
  Bump b(const_cast<void*>(r.tables));
  RobotImage im;
  if (h) {  // uniform over the block
    carve_image(b, r.J, r.S, r.NP, im);
    const uint32_t nw = (uint32_t)((b.bytes() - sizeof(TablesHeader)) / 4);
    if (threadIdx.x == 0) {
      s_hash = 0u;
      s_body = 0u;
    }
    __syncthreads();
    atomicAdd(&s_hash, robot_hash_part(r, threadIdx.x, blockDim.x));
    const bool sized = __ldcg(&h->body_words) == nw;  // the body read below stays inside the image
    if (sized) atomicAdd(&s_body, body_hash_part(reinterpret_cast<const uint32_t*>(h + 1), nw, threadIdx.x,
                                                 blockDim.x));
    __syncthreads();
    if (threadIdx.x == 0)
      s_ok = sized && h->magic == TABLES_MAGIC && h->J == (uint32_t)r.J && h->S == (uint32_t)r.S &&
             h->NP == (uint32_t)r.NP && h->hash == s_hash && h->body_hash == s_body;
    __syncthreads();
    ok = s_ok != 0;
  }
  if (!ok) {
    load_robot(r, rb);
    __syncthreads();
    load_clusters(r.J, r.S, rb);
    load_self(r, rb, m, t, eta_s);
    return;
  }
  const int J = r.J, S = r.S, NCB = cluster_bound(S, J), NG = (int)h->NG;
  const char *ib = reinterpret_cast<const char*>(im.rb.F), *sb = reinterpret_cast<const char*>(rb.F);
  const char *ip = reinterpret_cast<const char*>(im.pairs), *sp = reinterpret_cast<const char*>(m.pairs);
  // the robot arrays, and the pair tables, lie in the same order and
  // alignment in the image as in a block carved for this robot's sizes:
  // one copy each then
  const bool same_robot = reinterpret_cast<const char*>(rb.n_cl) - sb == reinterpret_cast<const char*>(im.rb.n_cl) - ib &&
                          reinterpret_cast<const char*>(rb.cl_of) - sb == reinterpret_cast<const char*>(im.rb.cl_of) - ib;
  const bool same_self = reinterpret_cast<const char*>(m.cp) - sp == reinterpret_cast<const char*>(im.cp) - ip &&
                         reinterpret_cast<const char*>(m.cp_start) - sp == reinterpret_cast<const char*>(im.cp_start) - ip;
  if (same_robot) {
    copy_granules(rb.F, im.rb.F, reinterpret_cast<const char*>(im.rb.n_cl + 2) - ib);
  } else {
    copy_granules(rb.F, im.rb.F, 3 * J * sizeof(float4));
    copy_granules(rb.sph, im.rb.sph, S * sizeof(float4));
    copy_granules(rb.link0, im.rb.link0, S * sizeof(int));
    copy_granules(rb.order, im.rb.order, S * sizeof(int));
    copy_granules(rb.start, im.rb.start, (J + 1) * sizeof(int));
    copy_granules(rb.cl_start, im.rb.cl_start, (NCB + 1) * sizeof(int));
    copy_granules(rb.cl_of, im.rb.cl_of, S * sizeof(int));
    copy_granules(rb.cl_sph, im.rb.cl_sph, NCB * sizeof(int));
    copy_granules(rb.n_cl, im.rb.n_cl, 2 * sizeof(int));
  }
  if (same_self) {
    copy_granules(m.pairs, im.pairs, reinterpret_cast<const char*>(im.cp_start + NG + 1) - ip);
  } else {
    copy_granules(m.cp, im.cp, NG * sizeof(uint16_t));
    copy_granules(m.cp_start, im.cp_start, (NG + 1) * sizeof(uint16_t));
    copy_granules(m.pairs, im.pairs, r.NP * sizeof(uint32_t));
  }
  if (threadIdx.x == 0) {
    m.self_meta[0] = NG;
    m.self_meta[1] = (int)__float_as_uint(eta_s);
  }
  __syncthreads();
}

// One warp's working set for one configuration.
constexpr int KEPT_CAP = 128;  // cluster pairs tested before their kept ones are expanded

struct CollWarp {
  float4* P;       // [S] (x, y, z, r)
  float4* acc;     // [S] (D, gx, gy, gz)
  float4* cls;     // [NC] cluster bounding spheres of this configuration (centre, radius)
  int4* gi;        // [S] self-term gradient sums of this configuration, fixed point 2^-e (.w unused)
  uint16_t* kept;  // [KEPT_CAP] kept cluster pairs, in table order
};

__host__ __device__ inline void carve_coll_warp(Bump& b, int S, int J, CollWarp& w) {
  w.P = b.take<float4>(S);
  w.acc = b.take<float4>(S);
  w.cls = b.take<float4>(cluster_bound(S, J));
  w.gi = b.take<int4>(S);
  w.kept = b.take<uint16_t>(KEPT_CAP);
}

// Radii into P[].w and zero accumulators (once per robot).
__device__ __forceinline__ void init_coll_warp(const RobotArgs& r, const CollWarp& w, int lane) {
  for (int s = lane; s < r.S; s += 32) {
    w.P[s] = make_float4(0.f, 0.f, 0.f, r.sphere_local[4 * s + 3]);
    w.acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Block-cooperative prologue of a block carved for this robot's own sizes
// (every thread calls it, the block converged): the scene arrays
// (load_scene), the robot and self tables (as load_robot_self: copied from
// r.tables when they were made for this robot, else built) and the scene
// grid's header (as grid_check: null when there is no usable grid), with
// every global read of the checks and the copies issued in one phase: the
// three hashes are summed per warp and checked by thread 0 behind one
// barrier, and the tables are copied before their check (a failed check
// builds them over the copy; the copy reads only as far as the image's own
// header says it reaches).  Then each warp's working set (init_coll_warp,
// radii from the tables).  Three block barriers; ends with the block
// synchronised.
__device__ inline const GridHeader* load_block_tables(const RobotArgs& r, const SceneArgs& sc, float eta,
                                                      float eta_s, const RobotSm& rb, const SceneSm& m,
                                                      const SelfScratch& t, const CollWarp& w) {
  __shared__ uint32_t s_part[32][3];  // per warp: robot, body and scene hash shares
  __shared__ int s_rad[32][2];        // per warp: smallest and largest radius bits
  __shared__ GridHeader s_g;
  __shared__ int s_ok[2];             // tables, grid
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (int)(blockDim.x >> 5);
  const TablesHeader* h = static_cast<const TablesHeader*>(r.tables);
  const GridHeader* g = static_cast<const GridHeader*>(sc.grid);
  load_scene(r, sc, eta, eta_s, m);
  uint32_t hr = 0u, hb = 0u, hs = 0u;
  int rmin = 0x7fffffff, rmax = (int)0x80000000;
  bool sized = false;
  if (h) {  // uniform over the block
    Bump b(const_cast<void*>(r.tables));
    RobotImage im;
    carve_image(b, r.J, r.S, r.NP, im);
    const uint32_t nw = (uint32_t)((b.bytes() - sizeof(TablesHeader)) / 4);
    hr = robot_hash_part(r, threadIdx.x, blockDim.x);
    sized = __ldcg(&h->body_words) == nw;  // the reads below stay inside the image
    if (sized) {
      hb = body_hash_part(reinterpret_cast<const uint32_t*>(h + 1), nw, threadIdx.x, blockDim.x);
      const int NGb = pair_groups_bound(r.NP, cluster_bound(r.S, r.J));
      copy_granules(rb.F, im.rb.F, reinterpret_cast<const char*>(im.rb.n_cl + 2) - reinterpret_cast<const char*>(im.rb.F));
      copy_granules(m.pairs, im.pairs, reinterpret_cast<const char*>(im.cp_start + NGb + 1) -
                                           reinterpret_cast<const char*>(im.pairs));
    }
  }
  if (g) {
    hs = scene_hash_part(sc, threadIdx.x, blockDim.x);
    for (int s = threadIdx.x; s < r.S; s += blockDim.x) {
      const int bits = __float_as_int(r.sphere_local[4 * s + 3]);
      rmin = min(rmin, bits);
      rmax = max(rmax, bits);
    }
    if (threadIdx.x < (int)(sizeof(GridHeader) / 4))
      reinterpret_cast<uint32_t*>(&s_g)[threadIdx.x] = reinterpret_cast<const uint32_t*>(g)[threadIdx.x];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    hr += __shfl_xor_sync(FULL_MASK, hr, off);
    hb += __shfl_xor_sync(FULL_MASK, hb, off);
    hs += __shfl_xor_sync(FULL_MASK, hs, off);
    rmin = min(rmin, __shfl_xor_sync(FULL_MASK, rmin, off));
    rmax = max(rmax, __shfl_xor_sync(FULL_MASK, rmax, off));
  }
  if (lane == 0) {
    s_part[warp][0] = hr;
    s_part[warp][1] = hb;
    s_part[warp][2] = hs;
    s_rad[warp][0] = rmin;
    s_rad[warp][1] = rmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t sr = 0u, sb = 0u, ss = 0u;
    int mn = 0x7fffffff, mx = (int)0x80000000;
    for (int k = 0; k < nwarps; ++k) {
      sr += s_part[k][0];
      sb += s_part[k][1];
      ss += s_part[k][2];
      mn = min(mn, s_rad[k][0]);
      mx = max(mx, s_rad[k][1]);
    }
    const bool tok = h && sized && h->magic == TABLES_MAGIC && h->J == (uint32_t)r.J && h->S == (uint32_t)r.S &&
                     h->NP == (uint32_t)r.NP && h->hash == sr && h->body_hash == sb;
    s_ok[0] = tok;
    s_ok[1] = g && grid_header_ok(s_g, sc, eta, ss, mn, mx);
    if (tok) {
      m.self_meta[0] = (int)h->NG;
      m.self_meta[1] = (int)__float_as_uint(eta_s);
    }
  }
  __syncthreads();
  if (!s_ok[0]) {  // uniform: build the tables over whatever was copied
    load_robot(r, rb);
    __syncthreads();
    load_clusters(r.J, r.S, rb);
    load_self(r, rb, m, t, eta_s);
  }
  for (int s = lane; s < r.S; s += 32) {  // this warp's working set (over the scratch)
    w.P[s] = make_float4(0.f, 0.f, 0.f, rb.sph[s].w);
    w.acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  return s_ok[1] ? &s_g : nullptr;
}

// Exact sphere-cuboid term: penetration max(0, r + eta - d) of the sphere
// (c, c.w = r) against cuboid o, and its gradient -w_c grad d, as
// (D, gx, gy, gz); all zero when the sphere is clear of the cuboid.
__device__ __forceinline__ float4 box_term_value(const SceneSm& m, int o, const float4& c, float eta,
                                                 float w_c) {
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 A0 = m.cubA[3 * o], A1 = m.cubA[3 * o + 1], A2 = m.cubA[3 * o + 2];
  const float4 H = m.cubH[o];
  const float dx = c.x - A0.w, dy = c.y - A1.w, dz = c.z - A2.w;
  const float x0 = fmaf(A0.x, dx, fmaf(A0.y, dy, A0.z * dz));
  const float x1 = fmaf(A1.x, dx, fmaf(A1.y, dy, A1.z * dz));
  const float x2 = fmaf(A2.x, dx, fmaf(A2.y, dy, A2.z * dz));
  const float u0 = fabsf(x0) - H.x, u1 = fabsf(x1) - H.y, u2 = fabsf(x2) - H.z;
  const float v0 = fmaxf(u0, 0.f), v1 = fmaxf(u1, 0.f), v2 = fmaxf(u2, 0.f);
  const float n2 = fmaf(v0, v0, fmaf(v1, v1, v2 * v2));
  const float umax = fmaxf(u0, fmaxf(u1, u2));
  const bool outside = umax > 0.f;  // some u > 0 (fmaxf passes over a NaN as the comparisons do)
  const float rs = n2 > 0.f ? rsqrtf(n2) : 0.f;  // 1/|max(u,0)|
  const float d = outside ? n2 * rs : umax;
  const float pen = c.w + eta - d;
  if (pen > 0.f) {
    // outside: s v / |v| (s = sign of x, +1 at 0; a product with s is its
    // sign bit on s v |v|^-1, so copysignf gives the same bits); inside: s
    // on the face of the largest u (lowest axis on ties)
    const int k = (u0 >= u1 && u0 >= u2) ? 0 : (u1 >= u2 ? 1 : 2);
    const float s0 = x0 >= 0.f ? 1.f : -1.f, s1 = x1 >= 0.f ? 1.f : -1.f, s2 = x2 >= 0.f ? 1.f : -1.f;
    const float l0 = outside ? copysignf(v0 * rs, s0) : (k == 0 ? s0 : 0.f);
    const float l1 = outside ? copysignf(v1 * rs, s1) : (k == 1 ? s1 : 0.f);
    const float l2 = outside ? copysignf(v2 * rs, s2) : (k == 2 ? s2 : 0.f);
    acc.x = pen;  // gradient of the hinge: -grad d, scaled by w_coll
    acc.y = -w_c * fmaf(A0.x, l0, fmaf(A1.x, l1, A2.x * l2));
    acc.z = -w_c * fmaf(A0.y, l0, fmaf(A1.y, l1, A2.y * l2));
    acc.w = -w_c * fmaf(A0.z, l0, fmaf(A1.z, l1, A2.z * l2));
  }
  return acc;
}

// The term added to acc (x: D, yzw: G) when the sphere penetrates the cuboid.
__device__ __forceinline__ void add_term(float4& acc, const float4& t) {
  if (t.x > 0.f) {
    acc.x += t.x;
    acc.y += t.y;
    acc.z += t.z;
    acc.w += t.w;
  }
}

__device__ __forceinline__ void box_term(const SceneSm& m, int o, const float4& c, float eta, float w_c,
                                         float4& acc) {
  add_term(acc, box_term_value(m, o, c, eta, w_c));
}

struct CollOut {
  float* cost;        // this configuration's cost, or null
  uint32_t* dist;     // packed D row, or null
  int dist_words;
  uint32_t* grad;     // packed G row, or null
  int grad_words;
};

// Decodes the sphere centres of one packed P row into P[s].xyz (one word per
// lane; .w is left alone).  COHERENT: loads that see writes made earlier in
// the same kernel.  F32: the row is float32 (no other format's code is
// compiled in: a smaller loop body for the instruction cache).
template <bool COHERENT, bool F32 = false>
__device__ __forceinline__ void load_centres(const uint32_t* prow, const DevFmt& fP, int S, float4* P,
                                             int lane) {
  const int nv = 3 * S;
  if (F32 || fP.kind == KIND_F32) {  // float32: lane s takes sphere s's three words
    for (int s = lane; s < S; s += 32) {
      const uint32_t* r = prow + 3 * s;
      float* d = reinterpret_cast<float*>(P + s);
      d[0] = __uint_as_float(COHERENT ? __ldcg(r) : __ldg(r));
      d[1] = __uint_as_float(COHERENT ? __ldcg(r + 1) : __ldg(r + 1));
      d[2] = __uint_as_float(COHERENT ? __ldcg(r + 2) : __ldg(r + 2));
    }
    return;
  }
  if constexpr (!F32) dispatch_kind(fP.kind, [&](auto kc) {
    constexpr int K = decltype(kc)::value;
    const int kw = per_word<K>(fP);
    const int nw = (nv + kw - 1) / kw;
    for (int wd = lane; wd < nw; wd += 32) {
      const uint32_t word = COHERENT ? __ldcg(prow + wd) : __ldg(prow + wd);
      unpack_word_t<K>(word, wd, nv, fP, [&](int i, float x) {
        const int s = i / 3;
        reinterpret_cast<float*>(P + s)[i - 3 * s] = x;
      });
    }
  });
}

// Cost (w_c sum_s acc[s].x + extra) and the packed D row (acc.x) of one
// configuration, one word per lane.  F32: D is float32.
template <bool F32 = false>
__device__ __forceinline__ void coll_cost_dist(const CollWarp& w, int S, const DevFmt& fD, float w_c, float extra,
                                               const CollOut& out, int lane) {
  float local = 0.f;
  for (int s = lane; s < S; s += 32) local += w.acc[s].x;
  local = w_c * local + extra;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(FULL_MASK, local, off);
  if (out.cost && lane == 0) *out.cost = local;
  if (F32 && out.dist) {
    for (int wd = lane; wd < out.dist_words; wd += 32) out.dist[wd] = wd < S ? __float_as_uint(w.acc[wd].x) : 0u;
  } else if (out.dist) {
    dispatch_kind(fD.kind, [&](auto kc) {
      constexpr int K = decltype(kc)::value;
      for (int wd = lane; wd < out.dist_words; wd += 32)
        out.dist[wd] = pack_word_t<K>(wd, S, fD, [&](int i) { return w.acc[i].x; });
    });
  }
}

// Zeroes acc for the next configuration.
__device__ __forceinline__ void coll_reset(const CollWarp& w, int S, int lane) {
  __syncwarp();
  for (int s = lane; s < S; s += 32) w.acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncwarp();
}

// Cost, the packed D (acc.x) and G (acc.yzw) rows of one configuration, one
// word per lane (every caller rewrites acc whole for the next configuration,
// after the closing warp barrier).  F32: D and G are float32.
template <bool F32 = false>
__device__ __forceinline__ void coll_outputs(const CollWarp& w, int S, const DevFmt& fD, const DevFmt& fG,
                                             float w_c, float extra, const CollOut& out, int lane) {
  coll_cost_dist<F32>(w, S, fD, w_c, extra, out, lane);
  if (out.grad && (F32 || fG.kind == KIND_F32)) {  // float32: lane s writes sphere s's three words
    for (int s = lane; s < S; s += 32) {
      const float4 a = w.acc[s];
      uint32_t* r = out.grad + 3 * s;
      r[0] = __float_as_uint(a.y);
      r[1] = __float_as_uint(a.z);
      r[2] = __float_as_uint(a.w);
    }
    for (int wd = 3 * S + lane; wd < out.grad_words; wd += 32) out.grad[wd] = 0u;  // row padding
  } else if (!F32 && out.grad) {
    const int nv = 3 * S;
    dispatch_kind(fG.kind, [&](auto kc) {
      constexpr int K = decltype(kc)::value;
      for (int wd = lane; wd < out.grad_words; wd += 32)
        out.grad[wd] = pack_word_t<K>(wd, nv, fG, [&](int i) {
          const int s = i / 3;
          return reinterpret_cast<const float*>(w.acc + s)[1 + i - 3 * s];
        });
    });
  }
  __syncwarp();
}

// Environment terms of sphere p over the cuboids obase + b for the set bits
// b of mm, in increasing cuboid order: the bounding test and exact term of
// the plain loop below, on the lanes' own candidates (lanes with different
// candidate counts idle once theirs run out).
__device__ __forceinline__ void env_bits(const SceneSm& m, int obase, unsigned long long mm,
                                         const float4& p, float eta, float w_c, float4& acc) {
  while (__any_sync(FULL_MASK, mm != 0ull)) {
    if (mm != 0ull) {
      const int o = obase + __ffsll((long long)mm) - 1;
      mm &= mm - 1ull;
      const float4 C = m.cubC[o];
      const float ax = p.x - C.x, ay = p.y - C.y, az = p.z - C.z, ta = p.w + C.w;
      if (fmaf(ax, ax, fmaf(ay, ay, az * az)) < ta * ta) box_term(m, o, p, eta, w_c, acc);
    }
  }
}

// Environment terms of sphere p over the cuboids obase + b for the set bits
// b of mm (a scene-grid cell's candidates), in increasing cuboid order: the
// exact term alone.  A candidate of the grid's cell is one the sphere can
// penetrate, and a pair the bounding test would reject has a negative
// penetration (SLACK), so the sums equal the plain loop's bit for bit.
__device__ __forceinline__ void env_bits_direct(const SceneSm& m, int obase, unsigned long long mm,
                                                const float4& p, float eta, float w_c, float4& acc) {
  while (__any_sync(FULL_MASK, mm != 0ull)) {
    if (mm != 0ull) {
      const int o = obase + __ffsll((long long)mm) - 1;
      mm &= mm - 1ull;
      box_term(m, o, p, eta, w_c, acc);
    }
  }
}

// Self-collision of one configuration (P in w.P, acc receiving gradients):
// returns this lane's share of the penetration sum.
//
// Each cluster's bounding sphere comes from the decoded centres: the
// centroid, radius rho = the largest |c_s - centroid| + r_s.  A cluster
// pair (a, b) whose spheres are apart by d_ab - rho_a - rho_b >= eta_s (+ a
// rounding margin) holds no pair with |c_i - c_j| < r_i + r_j + eta_s, since
// |c_i - c_j| >= d_ab - (rho_a - r_i) - (rho_b - r_j): its pairs are skipped.
// (A NaN anywhere keeps the cluster pair.)  The cluster pairs are tested
// KEPT_CAP at a time and the kept ones listed in table order; 32 listed
// cluster pairs at a time are expanded into their pairs through a warp
// prefix sum of their pair counts (lane t of a round finds its cluster pair
// from a warp OR of the cluster pairs' start positions), and the pairs are
// tested in table order; each active
// pair's gradient is added to its two spheres in fixed point (w.gi), and
// the sums are added to G at the end.
__device__ __forceinline__ float self_pairs(const RobotSm& rb, const SceneSm& m, const CollWarp& w,
                                            int S, float w_s, int lane) {
  const int NC = rb.n_cl[0], NG = m.self_meta[0], e = rb.n_cl[1];
  const float eta_s = __int_as_float(m.self_meta[1]);
  const float fix = __int_as_float((127 + e) << 23);  // 2^e
  const float eta_m = eta_s + 1e-4f;                  // eta_s and the margin's 1e-4 m
  for (int s = lane; s < S; s += 32) w.gi[s] = make_int4(0, 0, 0, 0);
  static_assert(CL <= 3, "a cluster's spheres are packed, 8 bits each, in one word with their count");
  for (int c = lane; c < NC; c += 32) {
    const int packed = rb.cl_sph[c], cnt = packed >> 24;
    float4 p[CL];
#pragma unroll
    for (int k = 0; k < CL; ++k) p[k] = w.P[k < cnt ? (packed >> (8 * k)) & 0xff : packed & 0xff];
    float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
    for (int k = 0; k < CL; ++k)
      if (k < cnt) {
        sx += p[k].x;
        sy += p[k].y;
        sz += p[k].z;
      }
    const float inv = __fdividef(1.f, (float)cnt);
    const float cx = sx * inv, cy = sy * inv, cz = sz * inv;
    float rho = 0.f;
#pragma unroll
    for (int k = 0; k < CL; ++k)
      if (k < cnt) {
        const float dx = p[k].x - cx, dy = p[k].y - cy, dz = p[k].z - cz;
        const float e2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        // |c_s - centroid| from the hardware reciprocal square root, rounded up
        rho = fmaxf(rho, fmaf(e2 > 0.f ? e2 * rsqrtf(e2) : 0.f, 1.000001f, p[k].w));
      }
    // grown by this cluster's share of the test's rounding margin,
    // 4e-6 (|centre|_1 + rho) (the pair test adds 1e-4 m on top)
    w.cls[c] = make_float4(cx, cy, cz, fmaf(4e-6f, fabsf(cx) + fabsf(cy) + fabsf(cz) + rho, rho));
  }
  __syncwarp();
  float selfsum = 0.f;
  for (int G0 = 0; G0 < NG; G0 += KEPT_CAP) {
    // the kept cluster pairs of the next KEPT_CAP, in table order, into w.kept
    int K = 0;
#pragma unroll
    for (int q = 0; q < KEPT_CAP / 32; ++q) {
      const int g = G0 + 32 * q + lane;
      bool keep = false;
      if (g < NG) {
        const uint32_t ab = m.cp[g];
        const float4 A = w.cls[ab & 0xffu], B = w.cls[ab >> 8];
        const float dx = A.x - B.x, dy = A.y - B.y, dz = A.z - B.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float rhs = A.w + B.w + eta_m;
        keep = !(rhs <= 0.f || d2 >= rhs * rhs);
      }
      const unsigned km = __ballot_sync(FULL_MASK, keep);
      if (keep) w.kept[K + __popc(km & ((1u << lane) - 1u))] = (uint16_t)g;
      K += __popc(km);
    }
    __syncwarp();
    for (int k0 = 0; k0 < K; k0 += 32) {  // their pairs, 32 cluster pairs at a time
      int cnt = 0, st = 0;
      if (k0 + lane < K) {
        const int g = w.kept[k0 + lane];
        st = m.cp_start[g];
        cnt = m.cp_start[g + 1] - st;
      }
      const int incl = warp_scan(cnt, lane), excl = incl - cnt;
      const int total = __shfl_sync(FULL_MASK, incl, 31);
      int before = 0;  // listed cluster pairs whose pairs start before t0
      for (int t0 = 0; t0 < total; t0 += 32) {
        const int v = t0 + lane;
        // the cluster pairs whose pairs start in [t0, t0 + 32), as bits
        // (every listed cluster pair has at least one pair): v's owner is
        // the last of them starting at or before v
        const unsigned starts =
            __reduce_or_sync(FULL_MASK, cnt > 0 && excl >= t0 && excl < t0 + 32 ? 1u << (excl - t0) : 0u);
        const int owner = before + __popc(starts & ((2u << lane) - 1u)) - 1;
        before += __popc(starts);
        const int pst = __shfl_sync(FULL_MASK, st, owner & 31), pex = __shfl_sync(FULL_MASK, excl, owner & 31);
        bool act = false;
        float pen = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;  // (c_i - c_j) / |c_i - c_j|
        int i = 0, j = 0;
        if (v < total) {
          const uint32_t pr = m.pairs[pst + v - pex];
          i = (int)(pr & 0xffffu);
          j = (int)(pr >> 16);
          const float4 ci = w.P[i], cj = w.P[j];
          const float dx = ci.x - cj.x, dy = ci.y - cj.y, dz = ci.z - cj.z;
          const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          const float thr = (ci.w + cj.w) + eta_s;
          if (d2 < thr * thr) {
            const float rs = d2 > 0.f ? rsqrtf(d2) : 0.f;
            pen = thr - d2 * rs;
            act = pen > 0.f;
            ux = dx * rs;  // 0 at zero distance: no gradient
            uy = dy * rs;
            uz = dz * rs;
          }
        }
        // each active pair adds -u to sphere i and +u to sphere j, in fixed
        // point (u times 2^e, rounded to an integer): integer sums do not
        // depend on the order of the additions, so the lanes add them at
        // once with shared-memory atomics and the result is still the same
        // bits every time.  (Measured and slower: float sums in table order
        // by lane 0 from staged pairs, which also set the launch's tail on
        // configurations with many contacts; each pair's own lane applying
        // it behind a warp barrier per pair; the spheres' owners receiving
        // the pairs by shuffles or from shared memory.)
        if (act) {
          selfsum += pen;
          const int vx = __float2int_rn(ux * fix), vy = __float2int_rn(uy * fix), vz = __float2int_rn(uz * fix);
          atomicAdd(&w.gi[i].x, -vx);
          atomicAdd(&w.gi[i].y, -vy);
          atomicAdd(&w.gi[i].z, -vz);
          atomicAdd(&w.gi[j].x, vx);
          atomicAdd(&w.gi[j].y, vy);
          atomicAdd(&w.gi[j].z, vz);
        }
      }
    }
    __syncwarp();  // w.kept is rewritten by the next KEPT_CAP
  }
  __syncwarp();
  // G += w_s 2^-e (the fixed-point sums)
  const float unit = w_s * __int_as_float((127 - e) << 23);
  for (int s = lane; s < S; s += 32) {
    float4 a = w.acc[s];
    const int4 g = w.gi[s];
    a.y = fmaf(unit, (float)g.x, a.y);
    a.z = fmaf(unit, (float)g.y, a.z);
    a.w = fmaf(unit, (float)g.z, a.w);
    w.acc[s] = a;
  }
  __syncwarp();
  return selfsum;
}

// Environment terms of sphere p (when v) over the candidates of its grid cell.
// first: the cell's first mask chunk, already loaded (the caller issues the
// loads of both its spheres' first chunks before either loop starts).
// DIRECT runs the exact term on the candidates alone (env_bits_direct),
// else the bounding test first (env_bits).
template <bool DIRECT>
__device__ __forceinline__ void env_grid(const SceneSm& m, const GridHeader& g, const uint2* c,
                                         uint2 first, const float4& p, float eta, float w_c, float4& acc) {
  for (int k = 0; k < (g.words >> 1); ++k) {
    const uint2 wd = k == 0 ? first : (c ? __ldg(c + k) : make_uint2(0u, 0u));
    unsigned long long mm = ((unsigned long long)wd.y << 32) | wd.x;
    const int left = g.O - 64 * k;  // bits past the last cuboid stay clear
    if (left < 64) mm &= left > 0 ? (1ull << left) - 1ull : 0ull;
    if constexpr (DIRECT) env_bits_direct(m, 64 * k, mm, p, eta, w_c, acc);
    else env_bits(m, 64 * k, mm, p, eta, w_c, acc);
  }
}

// Environment terms of spheres pa and pb (when va, vb) over their cells'
// candidates.
template <bool DIRECT = false>
__device__ __forceinline__ void env_grid2(const SceneSm& m, const GridHeader& g, const uint2* cells,
                                          bool va, const float4& pa, bool vb, const float4& pb, float eta,
                                          float w_c, float4& acca, float4& accb) {
  const uint2* ca = va ? grid_cell(g, cells, pa) : nullptr;
  const uint2* cb = vb ? grid_cell(g, cells, pb) : nullptr;
  const uint2 fa = ca ? __ldg(ca) : make_uint2(0u, 0u);
  const uint2 fb = cb ? __ldg(cb) : make_uint2(0u, 0u);
  env_grid<DIRECT>(m, g, ca, fa, pa, eta, w_c, acca);
  env_grid<DIRECT>(m, g, cb, fb, pb, eta, w_c, accb);
}

// The whole collision stage of one configuration by one warp: P row in,
// cost, D and G rows out (see collision.cu for the scheme).
// COHERENT reads the P row with loads that see writes made earlier in the
// same kernel (the fused multi-problem kernel); otherwise through the
// read-only cache.  MASKED takes a per-sphere distance estimate `est` (this
// configuration's row): spheres with est - r >= margin skip the cuboid
// tests.
// The environment and self terms of one configuration by one warp, on the
// centres in w.P: per-sphere penetration and gradient in w.acc (D, G);
// returns this lane's share of the self-penetration sum.  MASKED takes a
// per-sphere distance estimate `est` (this configuration's row): spheres
// with est - r >= margin skip the cuboid tests.
struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// between(): called by every lane after the environment terms, before the
// self terms (the collision kernel prefetches its next row there).
template <bool MASKED = false, typename Between = NoHook>
__device__ __forceinline__ float collision_terms(const RobotArgs& r, int O, const RobotSm& rb, const SceneSm& m,
                                                 const CollWarp& w, float eta, float w_c, float w_s, int lane,
                                                 const float* est = nullptr, float margin = 0.f,
                                                 const GridHeader* grid = nullptr,
                                                 const uint2* cells = nullptr, Between between = Between{}) {
  const int S = r.S;
  // ---- environment, sphere-major: lane owns spheres base + lane and
  //      base + 32 + lane and sums their terms in registers, cuboid by
  //      cuboid in order.  A sphere takes cuboid o's exact test only when it
  //      lies within the cuboid's bounding sphere grown by r + eta (+ SLACK);
  //      the warp skips o when none of its spheres does.
  for (int base = 0; base < S; base += 64) {
    const int sa = base + lane, sb = base + 32 + lane;
    bool va = sa < S, vb = sb < S;
    const float4 pa = va ? w.P[sa] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 pb = vb ? w.P[sb] : make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (MASKED) {
      va = va && __ldg(est + sa) - pa.w < margin;
      vb = vb && __ldg(est + sb) - pb.w < margin;
    }
    float4 acca = make_float4(0.f, 0.f, 0.f, 0.f), accb = acca;
    if (grid) {  // broad phase: each sphere visits its cell's candidates only
      env_grid2<true>(m, *grid, cells, va, pa, vb, pb, eta, w_c, acca, accb);
    } else if (__any_sync(FULL_MASK, va || vb)) {
#pragma unroll 2  // measured at 40 cuboids: 4.68 ns per configuration unrolled by 1, 4.59 by 2, 4.74 by 4
      for (int o = 0; o < O; ++o) {
        const float4 C = m.cubC[o];
        const float ax = pa.x - C.x, ay = pa.y - C.y, az = pa.z - C.z, ta = pa.w + C.w;
        const float bx = pb.x - C.x, by = pb.y - C.y, bz = pb.z - C.z, tb = pb.w + C.w;
        const bool na = va && fmaf(ax, ax, fmaf(ay, ay, az * az)) < ta * ta;
        const bool nb = vb && fmaf(bx, bx, fmaf(by, by, bz * bz)) < tb * tb;
        if (__any_sync(FULL_MASK, na || nb)) {
          if (na) box_term(m, o, pa, eta, w_c, acca);
          if (nb) box_term(m, o, pb, eta, w_c, accb);
        }
      }
    }
    if (sa < S) w.acc[sa] = acca;
    if (sb < S) w.acc[sb] = accb;
  }
  __syncwarp();
  between();
  // ---- self-collision: cluster bounding spheres, then the pairs of the
  //      cluster pairs whose spheres can touch (self_pairs)
  return self_pairs(rb, m, w, S, w_s, lane);
}

// The whole collision stage of one configuration by one warp: P row in,
// cost, D and G rows out (see collision.cu for the scheme).
// COHERENT reads the P row with loads that see writes made earlier in the
// same kernel (the fused multi-problem kernel); otherwise through the
// read-only cache.
template <bool COHERENT = false, bool MASKED = false, bool F32 = false, typename Between = NoHook>
__device__ __forceinline__ void collision_config(const RobotArgs& r, int O, const RobotSm& rb,
                                                 const SceneSm& m, const CollWarp& w,
                                                 const uint32_t* prow, const DevFmt& fP,
                                                 const DevFmt& fD, const DevFmt& fG, float eta,
                                                 float w_c, float w_s, const CollOut& out,
                                                 int lane, const float* est = nullptr,
                                                 float margin = 0.f,
                                                 const GridHeader* grid = nullptr,
                                                 const uint2* cells = nullptr, Between between = Between{}) {
  // ---- 1. sphere centres (one word per lane)
  load_centres<COHERENT, F32>(prow, fP, r.S, w.P, lane);
  __syncwarp();
  // ---- 2.-4. environment and self terms
  const float selfsum =
      collision_terms<MASKED>(r, O, rb, m, w, eta, w_c, w_s, lane, est, margin, grid, cells, between);
  // ---- 5. cost and packed outputs, then reset acc
  coll_outputs<F32>(w, r.S, fD, fG, w_c, w_s * selfsum, out, lane);
}

// ------------------------------------------------------- backward (thread)
// Streams the words of one packed row, caching the current 16-byte chunk.
// Where the row lives: shared memory, global through the read-only cache,
// or global written earlier in the same kernel (coherent L2 loads).
enum RowSrc : int { ROW_SHARED = 0, ROW_GLOBAL_RO = 1, ROW_GLOBAL_COHERENT = 2 };

template <int SRC>
struct RowReader {
  const uint8_t* row;
  int chunk = -1;
  uint4 v;
  __device__ __forceinline__ uint32_t word(int w) {
    const int c = w >> 2;
    if (c != chunk) {
      const uint4* p = reinterpret_cast<const uint4*>(row) + c;
      if constexpr (SRC == ROW_GLOBAL_RO) v = __ldg(p);
      else if constexpr (SRC == ROW_GLOBAL_COHERENT) v = __ldcg(p);
      else v = *p;
      chunk = c;
    }
    const int q = w & 3;
    return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
  }
  __device__ __forceinline__ float value(int i, const DevFmt& f) {  // runtime format
    const int w = i / f.k;
    return unpack_slot(word(w), i - w * f.k, f);
  }
  template <int K>
  __device__ __forceinline__ float value_k(int i, const DevFmt& f) {  // compile-time format
    return row_value<K>(i, f, [&](int w) { return word(w); });
  }
  // the three values of sphere s (values 3s .. 3s+2)
  template <int K>
  __device__ __forceinline__ void sphere(int s, const DevFmt& f, float& g0, float& g1, float& g2) {
    g0 = value_k<K>(3 * s, f);
    g1 = value_k<K>(3 * s + 1, f);
    g2 = value_k<K>(3 * s + 2, f);
  }
};

// Backward pass building blocks, shared by every kernel that forms the
// joint gradient so that they all round alike.  Link l's spheres enter
// through sums in the link's own frame,
//   f = sum_s G_s,   W = sum_s G_s p_s^T   (p_s the sphere's offset on the link),
// which need no pose; with the link's pose (R, t), c_s = R p_s + t gives
//   sum_s c_s x G_s = t x f + sum_s (R p_s) x G_s,
// and (R p_s) x G_s summed over s is the antisymmetric part of U = R W^T
// (U_km = sum_l R_kl W_ml = sum_s (R p_s)_k G_s,m):
//   (U_12 - U_21, U_20 - U_02, U_01 - U_10).
// 12 multiply-adds per sphere instead of 21 for forming c_s and c_s x G_s.
struct LinkSums {
  float f[3], W[3][3];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      f[m] = 0.f;
#pragma unroll
      for (int l = 0; l < 3; ++l) W[m][l] = 0.f;
    }
  }
  __device__ __forceinline__ void add(float g0, float g1, float g2, const float4& p) {
    const float g[3] = {g0, g1, g2};
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      f[m] = __fadd_rn(f[m], g[m]);
      W[m][0] = fmaf(g[m], p.x, W[m][0]);
      W[m][1] = fmaf(g[m], p.y, W[m][1]);
      W[m][2] = fmaf(g[m], p.z, W[m][2]);
    }
  }
  // sum_s c_s x G_s for the link at pose (R, t)
  __device__ __forceinline__ void moment(const float (&R)[3][3], const float (&t)[3], float (&mo)[3]) const {
    float U[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int m = 0; m < 3; ++m) U[k][m] = fmaf(R[k][0], W[m][0], fmaf(R[k][1], W[m][1], __fmul_rn(R[k][2], W[m][2])));
    mo[0] = __fadd_rn(fmaf(t[1], f[2], -__fmul_rn(t[2], f[1])), __fsub_rn(U[1][2], U[2][1]));
    mo[1] = __fadd_rn(fmaf(t[2], f[0], -__fmul_rn(t[0], f[2])), __fsub_rn(U[2][0], U[0][2]));
    mo[2] = __fadd_rn(fmaf(t[0], f[1], -__fmul_rn(t[1], f[0])), __fsub_rn(U[0][1], U[1][0]));
  }
};

// a . M - b . F
__device__ __forceinline__ float axis_term(float ax, float ay, float az, float bx, float by, float bz,
                                           const float (&M)[3], const float (&F)[3]) {
  return __fsub_rn(fmaf(ax, M[0], fmaf(ay, M[1], __fmul_rn(az, M[2]))),
                   fmaf(bx, F[0], fmaf(by, F[1], __fmul_rn(bz, F[2]))));
}

// The axis a_j (z-column of R_j) and b_j = a_j x o_j (o_j = t_j) of joint j.
__device__ __forceinline__ void joint_axis(const float (&R)[3][3], const float (&t)[3], float& ax, float& ay,
                                           float& az, float& bx, float& by, float& bz) {
  ax = R[0][2];
  ay = R[1][2];
  az = R[2][2];
  bx = fmaf(ay, t[2], -__fmul_rn(az, t[1]));
  by = fmaf(az, t[0], -__fmul_rn(ax, t[2]));
  bz = fmaf(ax, t[1], -__fmul_rn(ay, t[0]));
}

// Joint gradient of one configuration: put(j, dc * J_j) for j < J, with the
// per-joint terms (a_j, K_j), (b_j, -) in myK[0], myK[kst], .. myK[(2J-1) kst].
// One pass over the links in chain order: at joint j the running totals
// M, F hold links < j, so K_j = a_j . M - b_j . F, and at the end
// J_j = (a_j . M - b_j . F) - K_j over all links (= links >= j).
// sums(j, ls) adds link j's spheres to ls (LinkSums, zeroed), in the
// robot's sphere order.  live == false runs the same control flow (its
// results are not stored).
template <typename XR, typename Sums, typename Put>
__device__ __forceinline__ void backward_chain(const RobotSm& rb, int J, bool live, const float* q, XR& x,
                                               const DevFmt& fx, float dc, float4* myK, int kst, Sums sums,
                                               Put put) {
  float R[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
  float t[3] = {0.f, 0.f, 0.f};
  float F[3] = {0.f, 0.f, 0.f}, M[3] = {0.f, 0.f, 0.f};
  for (int j = 0; j < J; ++j) {
    if (live) {
      if (x.row) {  // stored transforms: element e of T_j is value 12j + e
#pragma unroll
        for (int k = 0; k < 3; ++k) {
#pragma unroll
          for (int l = 0; l < 3; ++l) R[k][l] = x.value(12 * j + 3 * k + l, fx);
          t[k] = x.value(12 * j + 9 + k, fx);
        }
      } else {  // recompute T_j = T_{j-1} F_j Rz(q_j)
        joint_step(rb, j, q[j], R, t);
      }
    }
    float ax, ay, az, bx, by, bz;
    joint_axis(R, t, ax, ay, az, bx, by, bz);
    myK[2 * j * kst] = make_float4(ax, ay, az, axis_term(ax, ay, az, bx, by, bz, M, F));
    myK[(2 * j + 1) * kst] = make_float4(bx, by, bz, 0.f);
    LinkSums ls;
    ls.zero();
    sums(j, ls);
    float mo[3];
    ls.moment(R, t, mo);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      M[k] = __fadd_rn(M[k], mo[k]);
      F[k] = __fadd_rn(F[k], ls.f[k]);
    }
  }
  for (int j = 0; j < J; ++j) {
    const float4 ak = myK[2 * j * kst], b = myK[(2 * j + 1) * kst];
    put(j, __fmul_rn(dc, __fsub_rn(axis_term(ak.x, ak.y, ak.z, b.x, b.y, b.z, M, F), ak.w)));
  }
}

// backward_chain with the gradient reader g, which gives the three values
// of a sphere (g.sphere); all lanes of a warp ask for the same sphere at
// the same time (the sphere order is the robot's, shared by all lanes).
template <int GK, typename XR, typename GR, typename Put>
__device__ __forceinline__ void backward_config(const RobotSm& rb, int J, bool live, const float* q, XR& x,
                                                const DevFmt& fx, GR& g, const DevFmt& fg, float dc,
                                                float4* myK, int kst, Put put) {
  backward_chain(rb, J, live, q, x, fx, dc, myK, kst, [&](int j, LinkSums& ls) {
    for (int idx = rb.start[j]; idx < rb.start[j + 1]; ++idx) {
      const int s = rb.order[idx];
      float g0, g1, g2;
      g.template sphere<GK>(s, fg, g0, g1, g2);
      ls.add(g0, g1, g2, rb.sph[s]);
    }
  }, put);
}

// Packed joint-gradient row of J values get(i) (padding words written as zero).
template <typename Get>
__device__ __forceinline__ void backward_store(int J, Get get, uint8_t* row, int64_t stride,
                                               const DevFmt& fj) {
  uint4* out = reinterpret_cast<uint4*>(row);
  const int chunks = (int)(stride / 16);
  for (int cc = 0; cc < chunks; ++cc) out[cc] = pack_chunk_dyn(cc, J, fj, get);
}

}  // namespace vapr
