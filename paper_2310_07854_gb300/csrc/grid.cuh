// Broad-phase grid of a scene: a uniform grid of cubic cells over the
// region where any sphere can touch a cuboid's bounding sphere, each cell
// holding the bitmask of the cuboids that a sphere centred in that cell can
// both pass the bounding test of and penetrate (grid.cu: a bounding-sphere
// test and a box-distance test of the cell).  It is scene preprocessing and
// only narrows which cuboids the environment loop visits: the loop runs the
// same exact distance, in cuboid order, on the cuboids it visits, and a
// cuboid left out of a cell is one that no sphere in it penetrates (its
// term would be exactly zero), so the results are the same as the plain
// loop over all cuboids, bit for bit.
//
// Layout (device memory, 16-byte aligned):
//   GridHeader (GRID_HEADER_BYTES), then cells[dims_z][dims_y][dims_x] of
//   `words` uint32 (an even count: 64-bit chunks, cuboid 64 k + b is bit b
//   of chunk k, low word first).
#pragma once

#include "common.cuh"

namespace vapr {

constexpr int GRID_HEADER_BYTES = 128;
constexpr int GRID_MAGIC = 0x56475244;  // marks a header the builder completed
constexpr int GRID_MAX_CELLS = VAPR_GRID_MAX_CELLS;
constexpr float SLACK = 1e-4f;  // metres: covers float32 rounding of the culls

struct GridHeader {
  float lo[3];        // corner of cell (0,0,0)
  float inv_h;        // 1 / cell side
  int dims[3];        // cells per axis (0 when no cell can hold a candidate)
  int words;          // mask words per cell (even)
  int O;              // cuboids of the scene it was built for
  uint32_t eta_bits;  // eta it was built for
  float reach;        // largest sphere radius it serves
  uint32_t hash;      // scene_hash of the pose and half-extent words
  float h;            // cell side
  int magic;          // GRID_MAGIC, or 0 when the builder gave up
  int pad[2];
};
static_assert(sizeof(GridHeader) <= GRID_HEADER_BYTES, "grid header");

__host__ __device__ constexpr int grid_words(int O) { return 2 * (((O > 0 ? O : 1) + 63) / 64); }

// Term of word w at position i of a hashed sequence: w xor a Weyl-sequence
// key of i, times an odd constant, then an xorshift, so each step (and the
// term, for a fixed i) is a bijection of w: changing any one word changes
// the sum of the terms.  Three integer operations and an index multiply-add
// per word.
__device__ __forceinline__ uint32_t hash_word(uint32_t w, uint32_t i) {
  const uint32_t h = (w ^ (i * 0x9e3779b9u + 0x7f4a7c15u)) * 0x85ebca6bu;
  return h ^ (h >> 15);
}

// One thread's share (words tid, tid + stride, ... in 16-byte groups when
// VEC) of the sum of hash_word(p[k], base + k) over k < n.  VEC: p is
// 16-byte aligned.  The sum does not depend on how the words are split, so
// a block adds its threads' shares with atomics.
template <bool VEC>
__device__ __forceinline__ uint32_t hash_words(const uint32_t* p, int n, uint32_t base, int tid, int stride) {
  uint32_t s = 0;
  int k0 = 0;
  if constexpr (VEC) {
    const int nq = n >> 2;
    for (int q = tid; q < nq; q += stride) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(p) + q);
      const uint32_t i = base + 4u * (uint32_t)q;
      s += hash_word(v.x, i) + hash_word(v.y, i + 1u) + hash_word(v.z, i + 2u) + hash_word(v.w, i + 3u);
    }
    k0 = 4 * nq;
  }
  for (int k = k0 + tid; k < n; k += stride) s += hash_word(__ldg(p + k), base + (uint32_t)k);
  return s;
}

// One thread's share of the scene hash: the sum (mod 2^32) of hash_word
// over the 12 O pose words, then the 3 O half-extent words.
__device__ __forceinline__ uint32_t scene_hash_part(const SceneArgs& sc, int tid, int stride) {
  const int np = 12 * sc.O;
  return hash_words<true>(reinterpret_cast<const uint32_t*>(sc.pose), np, 0u, tid, stride) +
         hash_words<false>(reinterpret_cast<const uint32_t*>(sc.half), 3 * sc.O, (uint32_t)np, tid, stride);
}

// Bounding radius of cuboid o's test as the collision stage computes it
// (half diagonal + eta + SLACK metres; see load_scene), grown by the
// largest sphere radius.  The test is |c - t_o| < r + R_o; for r in
// [0, reach] its threshold's magnitude is at most |R_o| + reach.
__device__ __forceinline__ float grid_reach_of(const SceneArgs& sc, int o, float eta, float reach) {
  const float hx = sc.half[3 * o], hy = sc.half[3 * o + 1], hz = sc.half[3 * o + 2];
  return fabsf(sqrtf(hx * hx + hy * hy + hz * hz) + eta + SLACK) + reach;
}

// Whether header g was built for this scene (hash: the scene's current
// hash), this eta and radii covering every sphere (rmin, rmax: the
// smallest and largest radius as int bits; non-negative floats order like
// their bits, and a negative radius, -0 or a NaN fails the range check).
__device__ __forceinline__ bool grid_header_ok(const GridHeader& g, const SceneArgs& sc, float eta, uint32_t hash,
                                               int rmin, int rmax) {
  return g.magic == GRID_MAGIC && g.O == sc.O && g.eta_bits == __float_as_uint(eta) && g.hash == hash &&
         rmin >= 0 && rmax <= __float_as_int(g.reach) && g.words == grid_words(sc.O) && g.dims[0] >= 0 &&
         g.dims[0] <= GRID_MAX_CELLS && g.dims[1] >= 0 && g.dims[1] <= GRID_MAX_CELLS && g.dims[2] >= 0 &&
         g.dims[2] <= GRID_MAX_CELLS;
}

// Block-cooperative (every thread calls it; the block must be converged):
// a shared-memory copy of the scene's grid header when the grid was built
// for this scene's current contents, this eta and radii covering every
// sphere of the robot (all in [0, reach]); else null, and the caller runs
// the plain loop.
__device__ inline const GridHeader* grid_check(const SceneArgs& sc, const RobotArgs& r, float eta) {
  __shared__ GridHeader s_g;
  __shared__ uint32_t s_hash;
  __shared__ int s_rmin, s_rmax, s_ok;
  const GridHeader* g = static_cast<const GridHeader*>(sc.grid);
  if (!g) return nullptr;  // uniform over the block
  if (threadIdx.x == 0) {
    s_hash = 0;
    s_rmin = 0x7fffffff;
    s_rmax = (int)0x80000000;
  }
  __syncthreads();
  atomicAdd(&s_hash, scene_hash_part(sc, threadIdx.x, blockDim.x));
  int rmin = 0x7fffffff, rmax = (int)0x80000000;
  for (int s = threadIdx.x; s < r.S; s += blockDim.x) {
    const int b = __float_as_int(r.sphere_local[4 * s + 3]);
    rmin = min(rmin, b);
    rmax = max(rmax, b);
  }
  atomicMin(&s_rmin, rmin);
  atomicMax(&s_rmax, rmax);
  if (threadIdx.x < (int)(sizeof(GridHeader) / 4))
    reinterpret_cast<uint32_t*>(&s_g)[threadIdx.x] = reinterpret_cast<const uint32_t*>(g)[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) s_ok = grid_header_ok(s_g, sc, eta, s_hash, s_rmin, s_rmax);
  __syncthreads();
  return s_ok ? &s_g : nullptr;
}

// The first mask chunk of the cell holding centre p (cells: the chunks after
// the header), or null when p lies outside the grid (then no cuboid's
// bounding test passes for it; a NaN centre lands here too, and fails every
// test as well).
__device__ __forceinline__ const uint2* grid_cell(const GridHeader& g, const uint2* cells,
                                                  const float4& p) {
  const float fx = (p.x - g.lo[0]) * g.inv_h;
  const float fy = (p.y - g.lo[1]) * g.inv_h;
  const float fz = (p.z - g.lo[2]) * g.inv_h;
  if (!(fx >= 0.f && fx < (float)g.dims[0] && fy >= 0.f && fy < (float)g.dims[1] && fz >= 0.f &&
        fz < (float)g.dims[2]))
    return nullptr;
  const int ix = min((int)fx, g.dims[0] - 1), iy = min((int)fy, g.dims[1] - 1),
            iz = min((int)fz, g.dims[2] - 1);
  return cells + ((size_t)(iz * g.dims[1] + iy) * g.dims[0] + ix) * (g.words >> 1);
}

__device__ __forceinline__ const uint2* grid_cells(const SceneArgs& sc) {
  return reinterpret_cast<const uint2*>(static_cast<const uint8_t*>(sc.grid) + GRID_HEADER_BYTES);
}

}  // namespace vapr
