// Builds the broad-phase grid of a scene (layout and use: grid.cuh).
//
// One block computes the scene hash and the region: the union of the
// cuboids' bounding spheres, each grown by eta, SLACK and the largest sphere
// radius, padded, with cubic cells whose side is the longest extent divided
// by the requested cells per axis.  Then a thread per (cell, 64-bit chunk)
// sets bit b when the cell, widened by a thousandth of its side, comes
// within 1.0001 R + 1e-5 m of cuboid 64 k + b's centre (R its grown
// bounding radius) and the box distance from the cell's centre to the
// cuboid, less the cell's half diagonal, is below reach + eta + 2 SLACK.
// The widening covers the rounding of the cell index the collision stage
// computes, the factor and SLACK the float32 rounding of the distance
// tests; the box distance is 1-Lipschitz, so a sphere's cell lists every
// cuboid whose bounding test can pass for it and that it can penetrate.
#include <cmath>

#include "stages.cuh"

namespace vapr {

struct GridBuild {
  SceneArgs sc;
  float reach, eta;
  int cells;       // requested cells per axis
  GridHeader* g;
  uint2* out;      // the cells' mask chunks
};

__global__ void __launch_bounds__(256) grid_header_kernel(GridBuild a) {
  __shared__ uint32_t s_hash;
  __shared__ float s_lo[3][256], s_hi[3][256];
  __shared__ int s_bad;
  if (threadIdx.x == 0) {
    s_hash = 0;
    s_bad = 0;
  }
  __syncthreads();
  atomicAdd(&s_hash, scene_hash_part(a.sc, threadIdx.x, blockDim.x));
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  for (int o = threadIdx.x; o < a.sc.O; o += blockDim.x) {
    const float R = grid_reach_of(a.sc, o, a.eta, a.reach);
    bad |= !isfinite(R);
    for (int k = 0; k < 3; ++k) {
      const float c = a.sc.pose[12 * o + 9 + k];
      bad |= !isfinite(c);
      lo[k] = fminf(lo[k], c - R);
      hi[k] = fmaxf(hi[k], c + R);
    }
  }
  for (int k = 0; k < 3; ++k) {
    s_lo[k][threadIdx.x] = lo[k];
    s_hi[k][threadIdx.x] = hi[k];
  }
  if (bad) s_bad = 1;
  __syncthreads();
  if (threadIdx.x != 0) return;
  GridHeader g = {};
  g.words = grid_words(a.sc.O);
  g.O = a.sc.O;
  g.eta_bits = __float_as_uint(a.eta);
  g.reach = a.reach;
  g.hash = s_hash;
  g.magic = GRID_MAGIC;
  g.h = 1.f;
  g.inv_h = 1.f;
  if (a.sc.O > 0) {  // (no cuboids: no cells, every sphere is outside)
    for (int k = 0; k < 3; ++k) {
      lo[k] = INFINITY;
      hi[k] = -INFINITY;
      for (int t = 0; t < (int)blockDim.x; ++t) {
        lo[k] = fminf(lo[k], s_lo[k][t]);
        hi[k] = fmaxf(hi[k], s_hi[k][t]);
      }
    }
    float E = fmaxf(hi[0] - lo[0], fmaxf(hi[1] - lo[1], hi[2] - lo[2]));
    const float pad = 1e-3f * E / (float)a.cells + 1e-5f;
    for (int k = 0; k < 3; ++k) {
      lo[k] -= pad;
      hi[k] += pad;
    }
    E = fmaxf(hi[0] - lo[0], fmaxf(hi[1] - lo[1], hi[2] - lo[2]));
    if (s_bad || !(E <= 1e6f)) {
      g.magic = 0;  // unusable: the collision stage runs the plain loop
    } else {
      g.h = E / (float)a.cells;
      g.inv_h = 1.f / g.h;
      for (int k = 0; k < 3; ++k) {
        g.lo[k] = lo[k];
        g.dims[k] = min(a.cells, max(1, (int)ceilf((hi[k] - lo[k]) * g.inv_h)));
      }
    }
  }
  *a.g = g;
}

__global__ void __launch_bounds__(256) grid_fill_kernel(GridBuild a) {
  const GridHeader g = *a.g;
  if (g.magic != GRID_MAGIC) return;
  const int nch = g.words >> 1;
  const int64_t total = (int64_t)g.dims[0] * g.dims[1] * g.dims[2] * nch;
  const float widen = 1e-3f * g.h;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = t / nch;
    const int k = (int)(t - cell * nch);
    const int ix = (int)(cell % g.dims[0]);
    const int iy = (int)((cell / g.dims[0]) % g.dims[1]);
    const int iz = (int)(cell / ((int64_t)g.dims[0] * g.dims[1]));
    const int idx[3] = {ix, iy, iz};
    float bmin[3], bmax[3];
    for (int d = 0; d < 3; ++d) {
      bmin[d] = g.lo[d] + (float)idx[d] * g.h - widen;
      bmax[d] = g.lo[d] + (float)(idx[d] + 1) * g.h + widen;
    }
    // the widened cell's centre and half diagonal
    float cc[3];
    for (int d = 0; d < 3; ++d) cc[d] = 0.5f * (bmin[d] + bmax[d]);
    const float hd = 0.8660254f * (g.h + 2.f * widen);
    const float near = a.reach + a.eta + hd + 2.f * SLACK;
    unsigned long long bits = 0ull;
    for (int b = 0; b < 64; ++b) {
      const int o = 64 * k + b;
      if (o >= a.sc.O) break;
      const float R = grid_reach_of(a.sc, o, a.eta, a.reach);
      const float* P = a.sc.pose + 12 * o;
      float d2 = 0.f;
      for (int d = 0; d < 3; ++d) {
        const float c = P[9 + d];
        const float e = fmaxf(fmaxf(bmin[d] - c, c - bmax[d]), 0.f);
        d2 = fmaf(e, e, d2);
      }
      const float thr = fmaf(R, 1.0001f, 1e-5f);
      if (!(d2 < thr * thr)) continue;
      // box distance at the cell centre; the distance is 1-Lipschitz, so no
      // point of the cell is nearer than that minus the half diagonal
      const float dx = cc[0] - P[9], dy = cc[1] - P[10], dz = cc[2] - P[11];
      float u[3];
      for (int e = 0; e < 3; ++e)  // x_e = (R^T (c - t))_e, R row-major
        u[e] = fabsf(fmaf(P[e], dx, fmaf(P[3 + e], dy, P[6 + e] * dz))) - a.sc.half[3 * o + e];
      const float v0 = fmaxf(u[0], 0.f), v1 = fmaxf(u[1], 0.f), v2 = fmaxf(u[2], 0.f);
      const float dbox = sqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2))) + fminf(fmaxf(u[0], fmaxf(u[1], u[2])), 0.f);
      if (dbox < near) bits |= 1ull << b;
    }
    a.out[t] = make_uint2((uint32_t)bits, (uint32_t)(bits >> 32));
  }
}

}  // namespace vapr

using namespace vapr;

extern "C" size_t vapr_scene_grid_bytes(int32_t n_cuboids, int32_t cells_per_axis) {
  if (n_cuboids < 0 || n_cuboids > VAPR_MAX_CUBOIDS || cells_per_axis < 1 ||
      cells_per_axis > VAPR_GRID_MAX_CELLS)
    return 0;
  const size_t c = (size_t)cells_per_axis;
  return GRID_HEADER_BYTES + c * c * c * (size_t)grid_words(n_cuboids) * 4;
}

extern "C" vapr_status vapr_scene_grid_build(const vapr_scene* scene, float reach, float eta,
                                             int32_t cells_per_axis, void* grid, size_t grid_bytes,
                                             void* stream) {
  SceneArgs sc;
  const vapr_status v = check_scene(scene, &sc);
  if (v != VAPR_OK) return v;
  sc.grid = nullptr;
  if (!(reach >= 0.f) || !std::isfinite(reach) || !std::isfinite(eta)) return VAPR_ERR_INVALID_ARG;
  if (cells_per_axis < 1 || cells_per_axis > VAPR_GRID_MAX_CELLS || !grid) return VAPR_ERR_INVALID_ARG;
  if ((uintptr_t)grid % 16) return VAPR_ERR_MISALIGNED;
  if (grid_bytes < vapr_scene_grid_bytes(sc.O, cells_per_axis)) return VAPR_ERR_INVALID_ARG;
  GridBuild a;
  a.sc = sc;
  a.reach = reach;
  a.eta = eta;
  a.cells = cells_per_axis;
  a.g = static_cast<GridHeader*>(grid);
  a.out = reinterpret_cast<uint2*>(static_cast<uint8_t*>(grid) + GRID_HEADER_BYTES);
  const cudaStream_t st = (cudaStream_t)stream;
  grid_header_kernel<<<1, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  const int64_t cap = (int64_t)cells_per_axis * cells_per_axis * cells_per_axis * (grid_words(sc.O) >> 1);
  const int64_t want = (cap + 255) / 256;
  const int64_t most = (int64_t)sm_count() * 8;
  grid_fill_kernel<<<(int)(want < most ? want : most), 256, 0, st>>>(a);
  return cuda_status(cudaGetLastError());
}
