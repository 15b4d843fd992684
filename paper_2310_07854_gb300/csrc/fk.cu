// Forward kinematics (Sec. II-B robot kinematics; iteration step 2 of
// Sec. III-B): joint configurations -> link transforms -> sphere centres,
// stored in the ExMy format of out_spheres (Sec. III-C).
//
// The kernel is bound by writing the packed P rows (624 bytes per
// configuration in float32), so it is laid out around the stores.  One
// thread per configuration; a warp owns tiles of 32 consecutive
// configurations, whose P rows are one contiguous range of global memory.
// The q rows of the warp's next tile are copied into shared memory
// (cp.async) while it works on the current one.
//
// A thread walks the spheres in index order and keeps one link transform
// in registers, advancing the joint chain (joint_step) when a sphere's link
// is further down the chain, and restarting it from the base when a
// sphere's link is nearer the base (only for robots whose spheres are not
// grouped by link); all lanes walk the same spheres, so the branches are
// warp-uniform.  No transform is stored.  The thread packs its row one
// segment at a time: a segment is PSEG_W = 12 words of the row, i.e. 4k
// spheres for k values per word, packed in registers with every bit position
// fixed at compile time (for k <= 2; for k >= 3 three words at a time), and
// written into its row of the warp's shared tile (rows an odd number of
// 16-byte chunks apart: conflict-free 16-byte stores).  The tile's 32 rows
// are one contiguous range of global memory, so the warp then copies them
// out as whole lines: by one bulk copy (cp.async.bulk) when the rows need
// no padding (float32: 39 chunks), else lane i taking 16-byte chunk i,
// i + 32, ...  (Writing
// 48-byte pieces of 32 rows at a time, by a 2-D TMA store per segment or by
// plain stores, was measured first: about 2.2 TB/s in float32 either way.)
// The segments cover the padded row, so padding words are written as zero.
//
// With the optional transform rows T (table->xform), each thread also keeps
// its transforms in shared memory and writes its T row from there.
#include "stages.cuh"
#include "tcgen05.cuh"

namespace vapr {

constexpr int FK_WARPS = 2;
constexpr int FK_BLOCK = 32 * FK_WARPS;
constexpr int PSEG_W = 12;     // words of each row per segment (48 B)
static_assert(PSEG_W == 12, "a segment holds 12k values = 4k whole spheres");

struct FkArgs {
  RobotArgs r;
  const float* q;
  int64_t n;
  Packed pos, xform;
  int tstride;  // float4 per thread of transform rows (3J rounded up to odd), 0 without T
  int nseg;     // segments per (padded) P row
  int pitch;    // bytes per row in the warp's shared tile: >= 48 nseg, an odd number of 16-byte chunks
  int bulk;     // pitch == row stride: the tile leaves by one bulk copy (cp.async.bulk)
};

__host__ __device__ inline void carve_fk(Bump& b, const FkArgs& a, RobotSm& rb, uint8_t*& tiles,
                                         float*& sQ, float4*& sT) {
  tiles = b.take<uint8_t>((size_t)FK_WARPS * 32 * a.pitch);  // 32 rows per warp
  carve_robot(b, a.r.J, a.r.S, rb);
  sQ = b.take<float>((size_t)FK_WARPS * 2 * 32 * a.r.J);  // two q tiles per warp
  sT = b.take<float4>((size_t)FK_BLOCK * a.tstride);
}

// One packed word from KW values v[0..KW-1] (compile-time positions);
// the same codes and bit layout as pack_word_t.
template <int PK, int KW>
__device__ __forceinline__ uint32_t enc_word(const float* v, const DevFmt& f) {
  if constexpr (PK == KIND_F32) {
    return __float_as_uint(v[0]);
  } else if constexpr (PK == KIND_GENERIC) {
    uint32_t w = 0u;
#pragma unroll
    for (int j = 0; j < KW; ++j) w |= (encode_generic(v[j], f) & f.mask) << (f.bits * j);
    return w;
  } else {
    constexpr int b = Fmt<PK>::bits;
    static_assert(Fmt<PK>::k == KW, "values per word of the kind");
    uint32_t w = 0u;
#pragma unroll
    for (int j = 0; j < KW; j += 2) {
      uint32_t pr = enc_pair<PK>(v[j], j + 1 < KW ? v[j + 1] : 0.f, f);
      if (j + 1 >= KW) pr &= (1u << b) - 1u;
      w |= pr << (b * j);
    }
    return w;
  }
}

// A thread's walk over its configuration's spheres: the transform of link
// cl in (R, t), advanced (or restarted) on demand.
struct ChainWalk {
  float R[3][3], t[3];
  int cl;
  __device__ __forceinline__ void reset() {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int b = 0; b < 3; ++b) R[a][b] = a == b ? 1.f : 0.f;
      t[a] = 0.f;
    }
    cl = -1;
  }
  // to link l (warp-uniform); every transform computed goes to myT (if any)
  __device__ __forceinline__ void to(const RobotSm& rb, int l, const float* q, float4* myT) {
    if (l < cl) reset();
    while (cl < l) {
      ++cl;
      joint_step(rb, cl, q[cl], R, t);
      if (myT) {
#pragma unroll
        for (int k = 0; k < 3; ++k) myT[3 * cl + k] = make_float4(R[k][0], R[k][1], R[k][2], t[k]);
      }
    }
  }
  __device__ __forceinline__ void centre(const float4& p, float* v) const {
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = fmaf(R[k][0], p.x, fmaf(R[k][1], p.y, fmaf(R[k][2], p.z, t[k])));
  }
};

// Values of spheres s0 .. s0+ns-1 (compile-time ns) into v[3 ns]; zeros past
// the last sphere.
template <int NS>
__device__ __forceinline__ void sphere_values(const RobotSm& rb, int S, int s0, ChainWalk& cw, const float* q,
                                              float4* myT, float* v) {
#pragma unroll
  for (int u = 0; u < NS; ++u) {
    const int s = s0 + u;
    if (s < S) {
      const int l = rb.link0[s];
      if (l != cw.cl) cw.to(rb, l, q, myT);
      cw.centre(rb.sph[s], v + 3 * u);
    } else {
      v[3 * u] = v[3 * u + 1] = v[3 * u + 2] = 0.f;
    }
  }
}

// PK: format kind of P; KW: its values per word, both fixed at compile time.
// XF: the transform rows are written too.
template <int PK, int KW, bool XF>
__global__ void __launch_bounds__(FK_BLOCK) fk_kernel(FkArgs a) {
  extern __shared__ float4 smem4[];
  const int J = a.r.J, S = a.r.S;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Bump b(smem4);
  RobotSm rb;
  uint8_t* tiles;
  float* sQ;
  float4* sT;
  carve_fk(b, a, rb, tiles, sQ, sT);
  load_robot(a.r, rb);
  __syncthreads();
  grid_dependents_may_launch();  // (the next stage waits for this grid to finish)

  float4* myT = XF ? sT + threadIdx.x * a.tstride : nullptr;
  uint8_t* tb = tiles + (size_t)warp * 32 * a.pitch;  // this warp's 32 rows
  uint4* myrow = reinterpret_cast<uint4*>(tb + (size_t)lane * a.pitch);
  float* qbuf = sQ + (size_t)warp * 2 * 32 * J;
  const int cpr = (int)(a.pos.stride / 16);  // 16-byte chunks per row
  const int64_t n_tiles = (a.n + 31) / 32;
  const int64_t first = (int64_t)blockIdx.x * FK_WARPS + warp, step = (int64_t)gridDim.x * FK_WARPS;
  if (first < n_tiles) q_prefetch(qbuf, a.q, first * 32, a.n, J, lane);
  int buf = 0;
  for (int64_t tile = first; tile < n_tiles; tile += step, buf ^= 1) {
    q_wait();  // this tile's q rows
    if (tile + step < n_tiles) q_prefetch(qbuf + (buf ^ 1) * 32 * J, a.q, (tile + step) * 32, a.n, J, lane);
    const int64_t c = tile * 32 + lane;
    const bool live = c < a.n;
    const float* myq = qbuf + buf * 32 * J + lane * J;  // (rows past n: zeros, never stored)
    ChainWalk cw;
    cw.reset();
    if (a.bulk) {  // the previous tile's bulk store has read the rows before they are rewritten
      if (lane == 0) bulk_wait_read<0>();
      __syncwarp();
    }
    for (int g = 0; g < a.nseg; ++g) {
      if constexpr (KW <= 2) {  // all 4 KW spheres of the segment at once
        float v[12 * KW];
        sphere_values<4 * KW>(rb, S, 4 * KW * g, cw, myq, myT, v);
        uint32_t wd[PSEG_W];
#pragma unroll
        for (int w = 0; w < PSEG_W; ++w) wd[w] = enc_word<PK, KW>(v + w * KW, a.pos.f);
        myrow[3 * g] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        myrow[3 * g + 1] = make_uint4(wd[4], wd[5], wd[6], wd[7]);
        myrow[3 * g + 2] = make_uint4(wd[8], wd[9], wd[10], wd[11]);
      } else {  // KW spheres -> 3 words at a time
        uint32_t* dst = reinterpret_cast<uint32_t*>(myrow + 3 * g);
        for (int sb = 0; sb < 4; ++sb) {
          float v[3 * KW];
          sphere_values<KW>(rb, S, (4 * g + sb) * KW, cw, myq, myT, v);
#pragma unroll
          for (int w = 0; w < 3; ++w) dst[3 * sb + w] = enc_word<PK, KW>(v + w * KW, a.pos.f);
        }
      }
    }
    __syncwarp();
    if (a.bulk) {  // rows packed back to back, as in global memory: one bulk copy of the tile
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the rows' writes before the copy reads them
      __syncwarp();
      if (lane == 0) {
        const int rows = (int)(a.n - tile * 32 < 32 ? a.n - tile * 32 : 32);
        bulk_s2g(a.pos.ptr + tile * 32 * a.pos.stride, tb, (uint32_t)(rows * a.pos.stride));
        bulk_commit();
      }
    } else {  // the tile's rows are one contiguous range: lanes take its 16-byte chunks in order
      const int rows = (int)(a.n - tile * 32 < 32 ? a.n - tile * 32 : 32);
      uint4* out = reinterpret_cast<uint4*>(a.pos.ptr + tile * 32 * a.pos.stride);
      int r = lane / cpr, ch = lane - r * cpr;  // chunk i = r cpr + ch, i = lane + 32 t
      const int dr = 32 / cpr, dc = 32 - dr * cpr;
      for (int i = lane; i < rows * cpr; i += 32) {
        out[i] = reinterpret_cast<const uint4*>(tb + (size_t)r * a.pitch)[ch];
        r += dr;
        ch += dc;
        if (ch >= cpr) {
          ch -= cpr;
          ++r;
        }
      }
    }
    if constexpr (XF) {  // every joint's transform, then the packed T row
      cw.to(rb, J - 1, myq, myT);
      __syncwarp();
      if (live) {  // element e of T_j is value 12 j + e
        uint4* out = reinterpret_cast<uint4*>(a.xform.ptr + c * a.xform.stride);
        const int chunks = (int)(a.xform.stride / 16);
        for (int cc = 0; cc < chunks; ++cc)
          out[cc] = pack_chunk_dyn(cc, 12 * J, a.xform.f, [&](int i) {
            const int j = i / 12, e = i - 12 * j;
            const int d = e < 9 ? e / 3 : e - 9;
            const int col = e < 9 ? e - 3 * d : 3;
            const float4 row = myT[3 * j + d];
            return col == 0 ? row.x : col == 1 ? row.y : col == 2 ? row.z : row.w;
          });
      }
    }
    __syncwarp();  // the rows are copied out and this tile's q rows read before they are reused
  }
  if (a.bulk && lane == 0) bulk_wait<0>();
}

using FkKernel = void (*)(FkArgs);

template <bool XF>
static FkKernel fk_kernel_for(const DevFmt& f) {
  switch (f.kind) {
    case KIND_F32: return fk_kernel<KIND_F32, 1, XF>;
    case KIND_F16: return fk_kernel<KIND_F16, 2, XF>;
    case KIND_BF16: return fk_kernel<KIND_BF16, 2, XF>;
    case KIND_E4M3: return fk_kernel<KIND_E4M3, 4, XF>;
    case KIND_E5M2: return fk_kernel<KIND_E5M2, 4, XF>;
    case KIND_E2M1: return fk_kernel<KIND_E2M1, 8, XF>;
    case KIND_E3M2: return fk_kernel<KIND_E3M2, 5, XF>;
    case KIND_E2M3: return fk_kernel<KIND_E2M3, 5, XF>;
    default:
      switch (f.k) {
        case 1: return fk_kernel<KIND_GENERIC, 1, XF>;
        case 2: return fk_kernel<KIND_GENERIC, 2, XF>;
        case 3: return fk_kernel<KIND_GENERIC, 3, XF>;
        case 4: return fk_kernel<KIND_GENERIC, 4, XF>;
        case 5: return fk_kernel<KIND_GENERIC, 5, XF>;
        case 6: return fk_kernel<KIND_GENERIC, 6, XF>;
        case 8: return fk_kernel<KIND_GENERIC, 8, XF>;
        default: return nullptr;
      }
  }
}

cudaError_t launch_fk(const RobotArgs& r, const float* q, int64_t n, Packed pos,
                      Packed xform, cudaStream_t st) {
  FkArgs a;
  a.r = r;
  a.q = q;
  a.n = n;
  a.pos = pos;
  a.xform = xform;
  const bool xf = xform.ptr != nullptr;
  a.tstride = xf ? (3 * r.J) | 1 : 0;  // odd float4 stride: conflict-free 16-byte accesses
  const int64_t words = pos.stride / 4;
  a.nseg = (int)((words + PSEG_W - 1) / PSEG_W);
  a.pitch = 16 * ((3 * a.nseg) | 1);  // odd chunk count: conflict-free 16-byte row stores
  a.bulk = a.pitch == pos.stride;
  const FkKernel kern = xf ? fk_kernel_for<true>(pos.f) : fk_kernel_for<false>(pos.f);
  if (!kern) return cudaErrorInvalidValue;
  Bump b(nullptr);
  RobotSm rb;
  uint8_t* ring;
  float* sQ;
  float4* sT;
  carve_fk(b, a, rb, ring, sQ, sT);
  const size_t smem = b.bytes();
  const int per_sm = blocks_per_sm((const void*)kern, FK_BLOCK, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t tiles = (n + 31) / 32;
  const int64_t blocks = (tiles + FK_WARPS - 1) / FK_WARPS;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  kern<<<(int)(blocks < cap ? blocks : cap), FK_BLOCK, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace vapr
