// Backward kinematics (iteration step 5 of Sec. III-B): the gradient with
// respect to the sphere centres (grad_out_spheres, Sec. III-C) becomes the
// joint-space gradient (backward_config in stages.cuh).
//
// For a revolute joint j with axis a_j and origin o_j (z-axis and origin of
// T_j), every sphere on link j or beyond moves as dc_s/dq_j = a_j x (c_s - o_j),
// so  J_j = a_j . (M_{>=j} - o_j x F_{>=j})  with  F = sum G_s  and
// M = sum c_s x G_s  over those spheres.  Writing b_j = a_j x o_j,
//   J_j = a_j . M_{>=j} - b_j . F_{>=j}
//       = (a_j . M - b_j . F) - (a_j . M_{<j} - b_j . F_{<j}),
// so one pass over the links in chain order suffices: when joint j is
// reached the thread records a_j, b_j and K_j = a_j . M_{<j} - b_j . F_{<j},
// and the totals finish every J_j at the end.  A link's spheres enter
// through sums in the link's frame, f = sum G_s and W = sum G_s p_s^T, and
// its moment sum c_s x G_s = t x f + (antisymmetric part of R W^T) costs a
// few multiply-adds per link (LinkSums in stages.cuh): 12 multiply-adds
// per sphere.
//
// One thread per configuration; a warp owns tiles of 32 consecutive
// configurations, whose gradient rows are contiguous in global memory.  The
// kernel is bound by streaming those rows (624 bytes per configuration in
// float32), so each warp streams them through a small ring of shared-memory
// slots (SegReader): a slot holds one segment of the tile, SEG_W = 12 words
// of each of the 32 rows, copied in by the lanes with 16-byte cp.async
// copies laid out so that each copy instruction reads whole runs of about
// 11 consecutive rows.  The threads read their rows' values in increasing
// order; when a segment is done the warp hands its slot to the copy
// SEG_SLOTS segments ahead, so copies stay in flight while the warp
// computes.  A segment row of 12 words holds whole spheres (4k of them at k
// values per word), so each sphere costs one segment check and three 32-bit
// shared loads.  A slot is small (1.5 KB), so many warps fit per SM.  (A
// 2-D TMA copy per segment was measured first: the TMA unit took about 210
// cycles per 32-row box of 48-byte rows, which held the kernel to
// 2.3 TB/s.)  The q rows of the next tile are copied the same way while
// the warp works on the current one.  The joint loop stays a loop (the
// per-joint terms go to shared memory): unrolling it over 7 joints made the
// code too large for the instruction cache.
//
// Reading values in increasing order needs the robot's spheres grouped by
// link in increasing link order (the order the pass walks them in); the
// block checks this, and otherwise the threads read their rows straight
// from global memory.  The kernel has no waits other than on its own
// asynchronous copies.
#include "stages.cuh"

namespace vapr {

constexpr int BW_WARPS = 4;
constexpr int BW_BLOCK = 32 * BW_WARPS;
constexpr int SEG_W = 12;     // words of each row per segment (48 B)
constexpr int SEG_SLOTS = 3;  // ring slots per warp
constexpr uint32_t SEG_BYTES = 32u * SEG_W * 4u;
static_assert(SEG_W == 12, "a segment row holds 12k values = 4k whole spheres");

__device__ int g_backward_error;  // sticky: first error code, 0 if none (no wait here can time out)

struct BwArgs {
  RobotArgs r;
  const float* q;
  int64_t n;
  Packed xform, grad, jgrad;
  const float* dcost;
};

__host__ __device__ inline void carve_bw(Bump& b, const BwArgs& a, RobotSm& rb, uint8_t*& ring,
                                         float4*& sK, float*& sQ) {
  ring = b.take<uint8_t>((size_t)BW_WARPS * SEG_SLOTS * SEG_BYTES);
  carve_robot(b, a.r.J, a.r.S, rb);
  sK = b.take<float4>((size_t)BW_BLOCK * 2 * a.r.J);  // per warp [2J][32 lanes]
  sQ = b.take<float>((size_t)BW_WARPS * 2 * 32 * a.r.J);  // two q tiles per warp
}

// One warp's view of its gradient rows through the segment ring.  Every
// lane holds the same copy of the bookkeeping (all calls are warp-uniform).
// A segment holds 12k values (k per word) of each row, i.e. spheres
// 4k c .. 4k c + 4k - 1 of segment c, so a sphere's three values never
// straddle two segments; segments are used in increasing order.
//
// A segment of the warp's 32 rows is 96 chunks of 16 bytes; lane m copies
// chunks m, m + 32 and m + 64 (chunk i: row i / 3, third i % 3 of the
// segment row) with cp.async, so each copy instruction reads whole runs of
// about 11 consecutive rows and the slot fills linearly.  The lane's three
// chunks sit at fixed offsets from the tile's first row, so a copy costs an
// add and two compares.  Every segment is one commit group of each lane,
// and every release commits one group (empty past the last segment), so
// waiting until at most SEG_SLOTS - 1 groups are pending always means the
// segment in hand has landed.
struct SegReader {
  uint8_t* slots;       // this warp's [SEG_SLOTS][32 rows][SEG_W words]
  int nseg, kw;         // segments per tile, values per word
  // issue side
  int off[3], lim[3], rt[3];  // this lane's chunks: offset from the tile's first row, end of
                              // the row's bytes (copy while col < lim), row in the tile
  const uint8_t* tile = nullptr;  // first row of the tile being issued
  int64_t row0 = 0, row_step = 0, n = 0;  // its first row, rows between this warp's tiles, rows
  int64_t tile_step = 0;  // bytes between this warp's tiles
  int tile_rows = 0;    // rows of the tile being issued below n (clamped to 32)
  int col = 0;          // byte offset in the rows of the next segment to issue
  int seg_bytes = 0;    // bytes of the rows that one tile's segments cover
  int left = 0;         // segments still to issue
  int iss_slot = 0;     // slot of the next segment to issue
  // use side
  int use_slot = 0;     // slot of the segment in hand (or of the next one)
  int cur = -1;         // segment of the current tile in hand, -1: none
  int s_end = 0;        // first sphere past the segment in hand
  const uint32_t* row = nullptr;  // this lane's row in the slot in hand
  int lane;

  __device__ __forceinline__ void init(uint8_t* sl, const uint8_t* rows, int64_t stride, int64_t n_, int S, int k,
                                       int ln, int64_t first, int64_t step, int64_t tiles) {
    slots = sl;
    kw = k;
    lane = ln;
    nseg = (3 * S + 12 * k - 1) / (12 * k);
    seg_bytes = nseg * SEG_W * 4;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int i = ln + 32 * t, r = i / 3, third = i - 3 * r;
      off[t] = (int)(r * stride) + 16 * third;
      lim[t] = (int)stride - 16 * third;
      rt[t] = r;
    }
    n = n_;
    row0 = first * 32;
    row_step = step * 32;
    tile = rows + row0 * stride;
    tile_step = row_step * stride;
    tile_rows = (int)(n - row0 < 32 ? (n - row0 > 0 ? n - row0 : 0) : 32);
    left = (int)(tiles * nseg);
  }
  __device__ __forceinline__ void issue_next() {  // warp-uniform
    if (left > 0) {
      const uint32_t slot = (uint32_t)__cvta_generic_to_shared(slots + iss_slot * SEG_BYTES) + 16 * lane;
#pragma unroll
      for (int t = 0; t < 3; ++t)
        if (rt[t] < tile_rows && col < lim[t])  // rows past n and past the row's end stay as they are
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(slot + 512 * t), "l"(tile + off[t] + col)
                       : "memory");
      --left;
      col += SEG_W * 4;
      if (col == seg_bytes) {  // next tile
        col = 0;
        row0 += row_step;
        tile += tile_step;
        tile_rows = (int)(n - row0 < 32 ? (n - row0 > 0 ? n - row0 : 0) : 32);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    iss_slot = iss_slot == SEG_SLOTS - 1 ? 0 : iss_slot + 1;
  }
  __device__ __forceinline__ void start() {
    for (int i = 0; i < SEG_SLOTS; ++i) issue_next();
  }
  __device__ __forceinline__ void acquire(int c) {
    row = reinterpret_cast<const uint32_t*>(slots + use_slot * SEG_BYTES) + lane * SEG_W;
    s_end = 4 * kw * (c + 1);
    asm volatile("cp.async.wait_group %0;" ::"n"(SEG_SLOTS - 1) : "memory");
    __syncwarp();  // every lane's copies of this segment are visible
  }
  __device__ __forceinline__ void release() {
    __syncwarp();  // every lane is done reading the slot
    issue_next();
    use_slot = use_slot == SEG_SLOTS - 1 ? 0 : use_slot + 1;
  }
  __device__ __forceinline__ void advance_to(int c) {
    while (cur < c) {
      if (cur >= 0) release();
      ++cur;
      acquire(cur);
    }
  }
  __device__ __forceinline__ void end_tile() {
    advance_to(nseg - 1);
    release();
    cur = -1;
    s_end = 0;
  }
  __device__ __forceinline__ void finish() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
  // Words wi WW .. wi WW + WW - 1 of this lane's row in the segment in hand
  // (16-, 8- or 4-byte shared loads: a row is 48 bytes, 16-byte aligned).
  template <int WW>
  __device__ __forceinline__ void window(int wi, uint32_t (&wd)[WW]) const {
    const uint32_t* p = row + wi * WW;
    if constexpr (WW % 4 == 0) {
#pragma unroll
      for (int v = 0; v < WW / 4; ++v) {
        const uint4 x = reinterpret_cast<const uint4*>(p)[v];
        wd[4 * v] = x.x;
        wd[4 * v + 1] = x.y;
        wd[4 * v + 2] = x.z;
        wd[4 * v + 3] = x.w;
      }
    } else if constexpr (WW % 2 == 0) {
#pragma unroll
      for (int v = 0; v < WW / 2; ++v) {
        const uint2 x = reinterpret_cast<const uint2*>(p)[v];
        wd[2 * v] = x.x;
        wd[2 * v + 1] = x.y;
      }
    } else {
#pragma unroll
      for (int v = 0; v < WW; ++v) wd[v] = p[v];
    }
  }
  // The three values of sphere s: one segment check, then one 32-bit
  // shared load per value (the formats without a window, below).
  template <int K>
  __device__ __forceinline__ void sphere(int s, const DevFmt& f, float& g0_, float& g1_, float& g2_) {
    while (s >= s_end) advance_to(cur + 1);  // spheres come in increasing order
    const int base = 12 * kw * cur;  // first value of the segment
    float v[3];
    if constexpr (K == KIND_F32) {
#pragma unroll
      for (int d = 0; d < 3; ++d) v[d] = __uint_as_float(row[3 * s + d - base]);
    } else {
      int k = kw;
      if constexpr (K != KIND_GENERIC) k = Fmt<K>::k;
      const int i0 = 3 * s - base;
      int w = i0 / k, r = i0 - w * k;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const uint32_t word = row[w];
        if constexpr (K == KIND_GENERIC) {
          v[d] = decode_generic((word >> (f.bits * r)) & f.mask, f);
        } else {
          constexpr int b = Fmt<K>::bits;
          v[d] = dec_pair<K>((word >> (b * r)) & ((1u << b) - 1u), 0u).x;
        }
        if (++r == k) {
          r = 0;
          ++w;
        }
      }
    }
    g0_ = v[0];
    g1_ = v[1];
    g2_ = v[2];
  }
};

// Windows: WS whole spheres whose 3 WS values fill WW whole words (k values
// per word, fixed at compile time: GKW for the generic kind); a segment
// holds WPS windows.  A window's words are read at once and decoded with
// every bit position fixed at compile time.
template <int GK, int GKW>
constexpr int values_per_word() {
  if constexpr (GK == KIND_GENERIC) return GKW;  // 0: runtime
  else return Fmt<GK>::k;
}
template <int GK, int GKW = 0>
struct Win {
  static constexpr int k = values_per_word<GK, GKW>();
  // the fewest whole spheres that fill whole words: 3 WS a multiple of k
  static constexpr int WS = k == 8 ? 8 : k == 5 ? 5 : k == 6 ? 2 : k == 3 ? 1 : 4;
  static constexpr bool ok = k >= 1 && k <= 8 && k != 7;
  static constexpr int WW = ok ? 3 * WS / k : 1;
  static constexpr int WPS = SEG_W / WW;
  static_assert(!ok || (3 * WS) % k == 0, "a window holds whole words");
  static_assert(!ok || SEG_W % WW == 0, "a segment holds whole windows");
};

// Values 0 .. 3 WS - 1 of a window's words.
template <int GK, int WS, int WW>
__device__ __forceinline__ void decode_window(const uint32_t (&wd)[WW], float (&v)[3 * WS], const DevFmt& f) {
  constexpr int k = 3 * WS / WW;
  if constexpr (GK == KIND_GENERIC) {
#pragma unroll
    for (int i = 0; i < 3 * WS; ++i) v[i] = decode_generic((wd[i / k] >> (f.bits * (i % k))) & f.mask, f);
  } else if constexpr (k == 1) {
#pragma unroll
    for (int i = 0; i < 3 * WS; ++i) v[i] = __uint_as_float(wd[i]);
  } else {
    constexpr int b = Fmt<GK>::bits;
    constexpr uint32_t m = (1u << b) - 1u;
#pragma unroll
    for (int w = 0; w < WW; ++w) {  // the k values of each word, two at a time
#pragma unroll
      for (int r = 0; r < k; r += 2) {
        const float2 x = dec_pair<GK>((wd[w] >> (b * r)) & m, r + 1 < k ? (wd[w] >> (b * (r + 1))) & m : 0u);
        v[w * k + r] = x.x;
        if (r + 1 < k) v[w * k + r + 1] = x.y;
      }
    }
  }
}

// GK: format kind of the gradient rows (the hot input), fixed at compile
// time; GKW: values per word of a generic kind (0: runtime).
template <int GK, int GKW>
__global__ void __launch_bounds__(BW_BLOCK, 4) backward_kernel(BwArgs a) {
  extern __shared__ float4 smem4[];
  const int J = a.r.J;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Bump b(smem4);
  RobotSm rb;
  uint8_t* ring;
  float4* sK;
  float* sQ;
  carve_bw(b, a, rb, ring, sK, sQ);
  load_robot(a.r, rb);
  __syncthreads();
  int in_order = 1;  // spheres grouped by link in increasing link order
  for (int k = threadIdx.x; k < a.r.S; k += blockDim.x) in_order &= rb.order[k] == k;
  const bool use_ring = __syncthreads_and(in_order);

  float4* myK = sK + (size_t)warp * 2 * J * 32 + lane;  // term i at myK[32 i]
  float* qbuf = sQ + (size_t)warp * 2 * 32 * J;
  const int64_t n_tiles = (a.n + 31) / 32;
  const int64_t first = (int64_t)blockIdx.x * BW_WARPS + warp, step = (int64_t)gridDim.x * BW_WARPS;
  const int64_t my_tiles = first < n_tiles ? (n_tiles - 1 - first) / step + 1 : 0;
  SegReader sr;
  sr.init(ring + (size_t)warp * SEG_SLOTS * SEG_BYTES, a.grad.ptr, a.grad.stride, a.n, a.r.S, a.grad.f.k, lane,
          first, step, use_ring ? my_tiles : 0);
  if (a.q && my_tiles > 0) q_prefetch(qbuf, a.q, first * 32, a.n, J, lane);
  grid_dependents_may_launch();
  grid_dependency_wait();  // the gradient rows are complete from here on
  if (use_ring) sr.start();

  // Between two tiles' q copies each lane commits one ring group per
  // segment (nseg of them, the ring's start() the first time), so the q rows
  // of a tile have landed once at most min(nseg, SEG_SLOTS) groups are
  // pending: the ring's copies stay in flight across the wait.
  static_assert(SEG_SLOTS <= 3, "q_wait_after takes at most 3 groups in flight");
  const int q_after = use_ring ? (sr.nseg < SEG_SLOTS ? sr.nseg : SEG_SLOTS) : 0;
  for (int64_t k = 0; k < my_tiles; ++k) {
    const int64_t c = (first + k * step) * 32 + lane;
    const bool live = c < a.n;
    const float* qp = nullptr;
    if (a.q) {  // this tile's q rows, and the next tile's in flight
      q_wait_after(q_after);
      if (k + 1 < my_tiles) q_prefetch(qbuf + ((k + 1) & 1) * 32 * J, a.q, (first + (k + 1) * step) * 32, a.n, J, lane);
      qp = qbuf + (k & 1) * 32 * J + lane * J;
    }
    const float dc = live && a.dcost ? a.dcost[c] : 1.f;
    RowReader<ROW_GLOBAL_RO> x{a.xform.ptr && live ? a.xform.ptr + c * a.xform.stride : nullptr};
    auto put = [&](int j, float v) { myK[32 * (2 * j + 1)].w = v; };  // after b_j is read
    if (use_ring) {
      if constexpr (Win<GK, GKW>::ok) {
        // link j's spheres [s0, s1) by windows: every window that holds one
        // of them, with the others of the window left out (warp-uniform)
        using W = Win<GK, GKW>;
        backward_chain(rb, J, live, qp, x, a.xform.f, dc, myK, 32, [&](int j, LinkSums& ls) {
          const int s0 = rb.start[j], s1 = rb.start[j + 1];
          if (s0 < s1) {
            for (int wdx = s0 / W::WS; wdx * W::WS < s1; ++wdx) {
              const int seg = wdx / W::WPS;
              sr.advance_to(seg);
              uint32_t wd[W::WW];
              sr.window<W::WW>(wdx - seg * W::WPS, wd);
              float v[3 * W::WS];
              decode_window<GK, W::WS, W::WW>(wd, v, a.grad.f);
              const int w0 = wdx * W::WS;
              if (w0 >= s0 && w0 + W::WS <= s1) {  // the whole window is on the link
#pragma unroll
                for (int u = 0; u < W::WS; ++u) ls.add(v[3 * u], v[3 * u + 1], v[3 * u + 2], rb.sph[w0 + u]);
              } else {
#pragma unroll
                for (int u = 0; u < W::WS; ++u) {
                  const int sp = w0 + u;
                  if (sp >= s0 && sp < s1) ls.add(v[3 * u], v[3 * u + 1], v[3 * u + 2], rb.sph[sp]);
                }
              }
            }
          }
        }, put);
      } else {
        backward_config<GK>(rb, J, live, qp, x, a.xform.f, sr, a.grad.f, dc, myK, 32, put);
      }
      sr.end_tile();
    } else {
      RowReader<ROW_GLOBAL_RO> g{live ? a.grad.ptr + c * a.grad.stride : a.grad.ptr};
      backward_config<GK>(rb, J, live, qp, x, a.xform.f, g, a.grad.f, dc, myK, 32, put);
    }
    if (live)
      backward_store(J, [&](int i) { return myK[32 * (2 * i + 1)].w; }, a.jgrad.ptr + c * a.jgrad.stride,
                     a.jgrad.stride, a.jgrad.f);
    __syncwarp();  // every lane is done with this tile's q rows
  }
  sr.finish();
}

int backward_device_error(bool reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_backward_error, sizeof(int)) != cudaSuccess) return -1;
  if (reset && v) {
    const int z = 0;
    cudaMemcpyToSymbol(g_backward_error, &z, sizeof(int));
  }
  return v;
}

static void (*bw_kernel_for(const DevFmt& f))(BwArgs) {
  switch (f.kind) {
    case KIND_F32: return backward_kernel<KIND_F32, 0>;
    case KIND_F16: return backward_kernel<KIND_F16, 0>;
    case KIND_BF16: return backward_kernel<KIND_BF16, 0>;
    case KIND_E4M3: return backward_kernel<KIND_E4M3, 0>;
    case KIND_E5M2: return backward_kernel<KIND_E5M2, 0>;
    case KIND_E2M1: return backward_kernel<KIND_E2M1, 0>;
    case KIND_E3M2: return backward_kernel<KIND_E3M2, 0>;
    case KIND_E2M3: return backward_kernel<KIND_E2M3, 0>;
    default:
      switch (f.k) {  // the widths of the searched formats (4 to 16 bits)
        case 2: return backward_kernel<KIND_GENERIC, 2>;
        case 3: return backward_kernel<KIND_GENERIC, 3>;
        case 4: return backward_kernel<KIND_GENERIC, 4>;
        case 5: return backward_kernel<KIND_GENERIC, 5>;
        case 6: return backward_kernel<KIND_GENERIC, 6>;
        default: return backward_kernel<KIND_GENERIC, 0>;
      }
  }
}

cudaError_t launch_backward(const RobotArgs& r, const float* q, Packed xform, Packed grad,
                            const float* dcost, int64_t n, Packed jgrad, cudaStream_t st, bool overlap) {
  BwArgs a;
  a.r = r;
  a.q = q;
  a.n = n;
  a.xform = xform;
  a.grad = grad;
  a.jgrad = jgrad;
  a.dcost = dcost;
  void (*kern)(BwArgs) = bw_kernel_for(grad.f);
  Bump b(nullptr);
  RobotSm rb;
  uint8_t* ring;
  float4* sK;
  float* sQ;
  carve_bw(b, a, rb, ring, sK, sQ);
  const size_t smem = b.bytes();
  const int per_sm = blocks_per_sm((const void*)kern, BW_BLOCK, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t tiles = (n + 31) / 32;
  const int64_t blocks = (tiles + BW_WARPS - 1) / BW_WARPS;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  const cudaError_t e = launch_after(overlap, kern, (int)(blocks < cap ? blocks : cap), BW_BLOCK, smem, st, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace vapr
