// Backward kinematics (iteration step 5 of Sec. III-B): the gradient with
// respect to the sphere centres (grad_out_spheres, Sec. III-C) becomes the
// joint-space gradient.
//
// For a revolute joint j with axis a_j and origin o_j (z-axis and origin of
// T_j), every sphere on link j or beyond moves as dc_s/dq_j = a_j x (c_s - o_j),
// so  J_j = a_j . (M_{>=j} - o_j x F_{>=j})  with  F = sum G_s  and
// M = sum c_s x G_s  over those spheres.  Writing b_j = a_j x o_j,
//   J_j = a_j . M_{>=j} - b_j . F_{>=j}
//       = (a_j . M - b_j . F) - (a_j . M_{<j} - b_j . F_{<j}),
// so one pass over the links in chain order suffices: when joint j is
// reached the thread records a_j, b_j and K_j = a_j . M_{<j} - b_j . F_{<j},
// and the totals finish every J_j at the end.  Zero gradients are skipped
// (the sparsity of Sec. III-C).
//
// One thread per configuration.  Spheres are visited link by link in a
// block-wide order built once in shared memory, so the sphere table may
// list spheres in any order.
#include "common.cuh"

namespace vapr {

constexpr int BW_BLOCK = 128;

struct BwArgs {
  RobotArgs r;
  const float* q;
  int64_t n;
  Packed xform, grad, jgrad;
  const float* dcost;
  int kstride;  // float4 per thread in sK (2J rounded up to odd)
};

// Streams the words of one packed row, caching the current 16-byte chunk.
struct RowReader {
  const uint8_t* row;
  int chunk = -1;
  uint4 v;
  __device__ __forceinline__ uint32_t word(int w) {
    const int c = w >> 2;
    if (c != chunk) {
      v = __ldg(reinterpret_cast<const uint4*>(row) + c);
      chunk = c;
    }
    const int q = w & 3;
    return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
  }
  __device__ __forceinline__ float value(int i, const DevFmt& f) {
    const int w = i / f.k;
    return unpack_slot(word(w), i - w * f.k, f);
  }
};

__global__ void __launch_bounds__(BW_BLOCK) backward_kernel(BwArgs a) {
  extern __shared__ float4 smem4[];
  const int J = a.r.J, S = a.r.S;
  float4* sF = smem4;                          // [3J] rows of F_j
  float4* sSph = sF + 3 * J;                   // [S] (p, r)
  float4* sK = sSph + S;                       // [BW_BLOCK][kstride]
  int* sOrder = reinterpret_cast<int*>(sK + BW_BLOCK * a.kstride);  // [S] by link
  int* sStart = sOrder + S;                                         // [J+1]

  for (int i = threadIdx.x; i < 3 * J; i += blockDim.x) {
    const int j = i / 3, d = i - 3 * j;
    const float* F = a.r.joint_fixed + 12 * j;
    sF[i] = make_float4(F[3 * d], F[3 * d + 1], F[3 * d + 2], F[9 + d]);
  }
  for (int s = threadIdx.x; s < S; s += blockDim.x)
    sSph[s] = reinterpret_cast<const float4*>(a.r.sphere_local)[s];
  if (threadIdx.x == 0) {  // stable counting sort of the spheres by link
    for (int j = 0; j <= J; ++j) sStart[j] = 0;
    for (int s = 0; s < S; ++s) ++sStart[clampi(a.r.sphere_link[s], 1, J)];
    for (int j = 1; j <= J; ++j) sStart[j] += sStart[j - 1];  // sStart[j] = end of link j
    for (int s = S - 1; s >= 0; --s) sOrder[--sStart[clampi(a.r.sphere_link[s], 1, J)]] = s;
    // now sStart[j] = first slot of link j (1-based), sStart[0] = 0
    for (int j = 0; j < J; ++j) sStart[j] = sStart[j + 1];
    sStart[J] = S;
  }
  __syncthreads();

  float4* myK = sK + threadIdx.x * a.kstride;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < a.n;
       c += (int64_t)gridDim.x * blockDim.x) {
    RowReader g{a.grad.ptr + c * a.grad.stride};
    RowReader x{a.xform.ptr ? a.xform.ptr + c * a.xform.stride : nullptr};
    const float* qc = a.q ? a.q + c * J : nullptr;
    float R[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
    float t[3] = {0.f, 0.f, 0.f};
    float F0 = 0.f, F1 = 0.f, F2 = 0.f, M0 = 0.f, M1 = 0.f, M2 = 0.f;
    for (int j = 0; j < J; ++j) {
      if (a.xform.ptr) {  // stored transforms: element e of T_j is value 12j + e
#pragma unroll
        for (int r = 0; r < 3; ++r) {
#pragma unroll
          for (int k = 0; k < 3; ++k) R[r][k] = x.value(12 * j + 3 * r + k, a.xform.f);
          t[r] = x.value(12 * j + 9 + r, a.xform.f);
        }
      } else {  // recompute T_j = T_{j-1} F_j Rz(q_j)
        const float4 f0 = sF[3 * j], f1 = sF[3 * j + 1], f2 = sF[3 * j + 2];
        float B[3][3], tb[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          B[r][0] = fmaf(R[r][0], f0.x, fmaf(R[r][1], f1.x, R[r][2] * f2.x));
          B[r][1] = fmaf(R[r][0], f0.y, fmaf(R[r][1], f1.y, R[r][2] * f2.y));
          B[r][2] = fmaf(R[r][0], f0.z, fmaf(R[r][1], f1.z, R[r][2] * f2.z));
          tb[r] = fmaf(R[r][0], f0.w, fmaf(R[r][1], f1.w, fmaf(R[r][2], f2.w, t[r])));
        }
        float sn, cs;
        sincosf(qc[j], &sn, &cs);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          R[r][0] = fmaf(cs, B[r][0], sn * B[r][1]);
          R[r][1] = fmaf(cs, B[r][1], -sn * B[r][0]);
          R[r][2] = B[r][2];
          t[r] = tb[r];
        }
      }
      // axis a_j, b_j = a_j x o_j, and the correction K_j
      const float ax = R[0][2], ay = R[1][2], az = R[2][2];
      const float bx = ay * t[2] - az * t[1];
      const float by = az * t[0] - ax * t[2];
      const float bz = ax * t[1] - ay * t[0];
      const float K = (ax * M0 + ay * M1 + az * M2) - (bx * F0 + by * F1 + bz * F2);
      myK[2 * j] = make_float4(ax, ay, az, K);
      myK[2 * j + 1] = make_float4(bx, by, bz, 0.f);
      // spheres on link j: accumulate F += G and M += c x G
      for (int idx = sStart[j]; idx < sStart[j + 1]; ++idx) {
        const int s = sOrder[idx];
        const float g0 = g.value(3 * s, a.grad.f);
        const float g1 = g.value(3 * s + 1, a.grad.f);
        const float g2 = g.value(3 * s + 2, a.grad.f);
        if (g0 == 0.f && g1 == 0.f && g2 == 0.f) continue;
        const float4 p = sSph[s];
        const float c0 = fmaf(R[0][0], p.x, fmaf(R[0][1], p.y, fmaf(R[0][2], p.z, t[0])));
        const float c1 = fmaf(R[1][0], p.x, fmaf(R[1][1], p.y, fmaf(R[1][2], p.z, t[1])));
        const float c2 = fmaf(R[2][0], p.x, fmaf(R[2][1], p.y, fmaf(R[2][2], p.z, t[2])));
        F0 += g0;
        F1 += g1;
        F2 += g2;
        M0 += c1 * g2 - c2 * g1;
        M1 += c2 * g0 - c0 * g2;
        M2 += c0 * g1 - c1 * g0;
      }
    }
    const float dc = a.dcost ? a.dcost[c] : 1.f;
    for (int j = 0; j < J; ++j) {
      const float4 ak = myK[2 * j], b = myK[2 * j + 1];
      const float Jj = (ak.x * M0 + ak.y * M1 + ak.z * M2) - (b.x * F0 + b.y * F1 + b.z * F2) - ak.w;
      myK[2 * j + 1].w = dc * Jj;
    }
    // packed joint-gradient row (its padding words are written as zero)
    uint32_t* out = reinterpret_cast<uint32_t*>(a.jgrad.ptr + c * a.jgrad.stride);
    const int words = (int)(a.jgrad.stride / 4);
    auto get = [&](int i) { return myK[2 * i + 1].w; };
    for (int w = 0; w < words; ++w) out[w] = pack_word(w, J, a.jgrad.f, get);
  }
}

cudaError_t launch_backward(const RobotArgs& r, const float* q, Packed xform, Packed grad,
                            const float* dcost, int64_t n, Packed jgrad, cudaStream_t st) {
  BwArgs a;
  a.r = r;
  a.q = q;
  a.n = n;
  a.xform = xform;
  a.grad = grad;
  a.jgrad = jgrad;
  a.dcost = dcost;
  a.kstride = (2 * r.J) | 1;
  const size_t smem = sizeof(float4) * (3 * r.J + r.S + (size_t)BW_BLOCK * a.kstride) +
                      sizeof(int) * (r.S + r.J + 1);
  const int per_sm = blocks_per_sm((const void*)backward_kernel, BW_BLOCK, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  const int64_t blocks = (n + BW_BLOCK - 1) / BW_BLOCK;
  const int64_t cap = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1);
  backward_kernel<<<(int)(blocks < cap ? blocks : cap), BW_BLOCK, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace vapr
