// Forward kinematics (Sec. II-B robot kinematics; iteration step 2 of
// Sec. III-B): joint configurations -> link transforms -> sphere centres,
// stored in the ExMy format of out_spheres (Sec. III-C).
//
// T_0 = I, T_j = T_{j-1} F_j Rz(q_j); c_s = T_link(s) [p_s; 1].
//
// A block takes tiles of FK_TILE configurations.  Each thread runs the joint
// chain of one configuration and leaves its J transforms in shared memory;
// then the block writes the tile's packed rows: warps take rows, lanes take
// the 32-bit words of a row, so every warp store is 128 contiguous bytes.
#include "common.cuh"

namespace vapr {

constexpr int FK_TILE = 128;

struct FkArgs {
  RobotArgs r;
  const float* q;
  int64_t n;
  Packed pos, xform;
  int tstride;  // float4 per configuration in sT (3J rounded up to odd)
};

__global__ void __launch_bounds__(FK_TILE) fk_kernel(FkArgs a) {
  extern __shared__ float4 smem4[];
  const int J = a.r.J, S = a.r.S;
  float4* sF = smem4;                       // [J*3] rows of F_j: (R_d0, R_d1, R_d2, t_d)
  float4* sSph = sF + 3 * J;                // [S] (p, r)
  float4* sT = sSph + S;                    // [FK_TILE][tstride]
  int* sLink = reinterpret_cast<int*>(sT + FK_TILE * a.tstride);  // [S] 0-based
  float* sQ = reinterpret_cast<float*>(sLink + S);                // [FK_TILE][J]

  for (int i = threadIdx.x; i < 3 * J; i += blockDim.x) {
    const int j = i / 3, d = i - 3 * j;
    const float* F = a.r.joint_fixed + 12 * j;
    sF[i] = make_float4(F[3 * d], F[3 * d + 1], F[3 * d + 2], F[9 + d]);
  }
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    sSph[s] = reinterpret_cast<const float4*>(a.r.sphere_local)[s];
    sLink[s] = clampi(a.r.sphere_link[s], 1, J) - 1;
  }

  const int64_t n_tiles = (a.n + FK_TILE - 1) / FK_TILE;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t base = tile * FK_TILE;
    const int rows = (int)(a.n - base < FK_TILE ? a.n - base : FK_TILE);
    __syncthreads();  // tables ready / previous tile's readers done
    for (int i = threadIdx.x; i < rows * J; i += blockDim.x) sQ[i] = a.q[base * J + i];
    __syncthreads();

    if (threadIdx.x < rows) {
      // the joint chain of one configuration, in registers
      float R[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
      float t[3] = {0.f, 0.f, 0.f};
      float4* myT = sT + threadIdx.x * a.tstride;
      for (int j = 0; j < J; ++j) {
        const float4 f0 = sF[3 * j], f1 = sF[3 * j + 1], f2 = sF[3 * j + 2];
        float B[3][3], tb[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {  // (T_{j-1} F_j): rotation and translation
          B[r][0] = fmaf(R[r][0], f0.x, fmaf(R[r][1], f1.x, R[r][2] * f2.x));
          B[r][1] = fmaf(R[r][0], f0.y, fmaf(R[r][1], f1.y, R[r][2] * f2.y));
          B[r][2] = fmaf(R[r][0], f0.z, fmaf(R[r][1], f1.z, R[r][2] * f2.z));
          tb[r] = fmaf(R[r][0], f0.w, fmaf(R[r][1], f1.w, fmaf(R[r][2], f2.w, t[r])));
        }
        float sn, cs;
        sincosf(sQ[threadIdx.x * J + j], &sn, &cs);
#pragma unroll
        for (int r = 0; r < 3; ++r) {  // ... Rz(q_j)
          R[r][0] = fmaf(cs, B[r][0], sn * B[r][1]);
          R[r][1] = fmaf(cs, B[r][1], -sn * B[r][0]);
          R[r][2] = B[r][2];
          t[r] = tb[r];
          myT[3 * j + r] = make_float4(R[r][0], R[r][1], R[r][2], t[r]);
        }
      }
    }
    __syncthreads();

    // Packed rows: warps take the tile's rows, lanes the words of a row, so
    // each warp store covers 128 consecutive bytes.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    {  // sphere centres: value i of a row is coordinate i % 3 of sphere i / 3
      const int words = (int)(a.pos.stride / 4), nv = 3 * S;
      dispatch_kind(a.pos.f.kind, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        for (int r = warp; r < rows; r += nwarps) {
          const float4* T = sT + r * a.tstride;
          uint32_t* out = reinterpret_cast<uint32_t*>(a.pos.ptr + (base + r) * a.pos.stride);
          for (int w = lane; w < words; w += 32)
            out[w] = pack_word_t<K>(w, nv, a.pos.f, [&](int i) {
              const int s = i / 3, d = i - 3 * s;
              const float4 row = T[3 * sLink[s] + d];
              const float4 p = sSph[s];
              return fmaf(row.x, p.x, fmaf(row.y, p.y, fmaf(row.z, p.z, row.w)));
            });
        }
      });
    }
    if (a.xform.ptr) {  // link transforms: value i is element i % 12 (R row-major, t) of T_{i/12}
      const int words = (int)(a.xform.stride / 4), nv = 12 * J;
      dispatch_kind(a.xform.f.kind, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        for (int r = warp; r < rows; r += nwarps) {
          const float4* T = sT + r * a.tstride;
          uint32_t* out = reinterpret_cast<uint32_t*>(a.xform.ptr + (base + r) * a.xform.stride);
          for (int w = lane; w < words; w += 32)
            out[w] = pack_word_t<K>(w, nv, a.xform.f, [&](int i) {
              const int j = i / 12, e = i - 12 * j;
              const int d = e < 9 ? e / 3 : e - 9;
              const int col = e < 9 ? e - 3 * d : 3;
              const float4 row = T[3 * j + d];
              return col == 0 ? row.x : col == 1 ? row.y : col == 2 ? row.z : row.w;
            });
        }
      });
    }
  }
}

static size_t fk_smem(int J, int S, int tstride) {
  return sizeof(float4) * (3 * J + S + (size_t)FK_TILE * tstride) + sizeof(int) * S +
         sizeof(float) * (size_t)FK_TILE * J;
}

cudaError_t launch_fk(const RobotArgs& r, const float* q, int64_t n, Packed pos,
                      Packed xform, cudaStream_t st) {
  FkArgs a;
  a.r = r;
  a.q = q;
  a.n = n;
  a.pos = pos;
  a.xform = xform;
  a.tstride = (3 * r.J) | 1;  // odd float4 stride: conflict-free 16-byte stores
  const size_t smem = fk_smem(r.J, r.S, a.tstride);
  const int per_sm = blocks_per_sm((const void*)fk_kernel, FK_TILE, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t tiles = (n + FK_TILE - 1) / FK_TILE;
  const int64_t cap = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1);
  const int grid = (int)(tiles < cap ? tiles : cap);
  fk_kernel<<<grid, FK_TILE, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace vapr
