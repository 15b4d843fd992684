// Compute ceiling of the collision stage's environment pair test: the
// denominator against which the rate of vapr_collision_cost is reported (a
// measurement aid of this library; the paper has no counterpart).
//
// The collision stage is bound by FP32 arithmetic and instruction issue,
// not by HBM, so its roofline needs a compute ceiling.  This kernel runs the
// stage's own environment loop -- the bounding-sphere test of every
// sphere/cuboid pair, and the exact box term (box_term) where it passes,
// two spheres per lane, the warp skipping a cuboid none of its spheres can
// touch, cuboids staged in shared memory exactly as the stage stages them
// -- on sphere centres held in registers: no packed rows to decode, no
// self pairs, no outputs until the end.  Each 64-sphere group repeats the
// loop `reps` times; an empty asm statement makes the centres opaque at the
// start of every repetition and consumes its sums at the end, so the
// compiler can neither hoist a repetition out of the loop nor drop one.
// On spheres that clear every cuboid's bounding sphere the loop is the
// bounding tests alone (10 FLOP each): the rate it reaches is the ceiling of
// the method's pair-test work.  Outputs are those of the last repetition:
// per sphere (D, G) of the environment term, equal to what the collision
// stage computes for it.
#include "stages.cuh"

namespace vapr {

constexpr int CEIL_WARPS = 8;

struct CeilArgs {
  SceneArgs sc;
  float eta, w_c;
  const float4* spheres;  // [n] (x, y, z, r)
  int64_t n;
  int reps;
  float4* out;  // [n] (D, G)
};

// The optimiser must assume v changed here (and read it).
__device__ __forceinline__ void opaque(float4& v) {
  asm volatile("" : "+f"(v.x), "+f"(v.y), "+f"(v.z), "+f"(v.w));
}

__global__ void __launch_bounds__(CEIL_WARPS * 32) env_ceiling_kernel(CeilArgs a) {
  extern __shared__ float4 smem4[];
  Bump b(smem4);
  SceneSm m;
  carve_scene(b, a.sc.O, 0, 0, m);
  RobotArgs r{};  // load_scene reads the scene only
  load_scene(r, a.sc, a.eta, 0.f, m);
  __syncthreads();
  const int lane = threadIdx.x & 31, O = a.sc.O;
  const float eta = a.eta, w_c = a.w_c;
  const int64_t stride = (int64_t)gridDim.x * CEIL_WARPS;
  // warp-uniform loop over 64-sphere groups: lane owns spheres 64g + lane and
  // 64g + 32 + lane, as in the collision stage
  for (int64_t g = (int64_t)blockIdx.x * CEIL_WARPS + (threadIdx.x >> 5); g * 64 < a.n; g += stride) {
    const int64_t sa = g * 64 + lane, sb = sa + 32;
    const bool va = sa < a.n, vb = sb < a.n;
    float4 pa = va ? a.spheres[sa] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 pb = vb ? a.spheres[sb] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 acca = make_float4(0.f, 0.f, 0.f, 0.f), accb = acca;
    for (int k = 0; k < a.reps; ++k) {
      opaque(pa);
      opaque(pb);
      acca = make_float4(0.f, 0.f, 0.f, 0.f);
      accb = acca;
#pragma unroll 2
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
      opaque(acca);
      opaque(accb);
    }
    if (va) a.out[sa] = acca;
    if (vb) a.out[sb] = accb;
  }
}

static size_t ceiling_smem(int O) {
  Bump b(nullptr);
  SceneSm m;
  carve_scene(b, O, 0, 0, m);
  return b.bytes();
}

// Resident warps of one launch on the current device (0 on error).
static int64_t ceiling_warps(int O) {
  const int per_sm = blocks_per_sm((const void*)env_ceiling_kernel, CEIL_WARPS * 32, ceiling_smem(O));
  if (per_sm <= 0) return 0;
  return (int64_t)sm_count() * per_sm * CEIL_WARPS;
}

}  // namespace vapr

using namespace vapr;

extern "C" int64_t vapr_env_ceiling_warps(int32_t n_cuboids) {
  if (n_cuboids < 0 || n_cuboids > VAPR_MAX_CUBOIDS) return 0;
  return ceiling_warps(n_cuboids);
}

extern "C" vapr_status vapr_env_ceiling(const vapr_scene* scene, const float* spheres, int64_t n,
                                        float eta, float w_coll, int32_t reps, float* out,
                                        void* stream) {
  SceneArgs sc;
  vapr_status v = check_scene(scene, &sc);
  if (v != VAPR_OK) return v;
  if (n < 0 || reps < 1) return VAPR_ERR_INVALID_ARG;
  if (n == 0) return VAPR_OK;
  if (!spheres || !out) return VAPR_ERR_INVALID_ARG;
  if ((uintptr_t)spheres % 16 || (uintptr_t)out % 16) return VAPR_ERR_MISALIGNED;
  const int64_t warps = ceiling_warps(sc.O);
  if (warps <= 0) return cuda_status(cudaErrorInvalidConfiguration);
  CeilArgs a;
  a.sc = sc;
  a.sc.grid = nullptr;  // the plain loop: every pair gets its bounding test
  a.eta = eta;
  a.w_c = w_coll;
  a.spheres = reinterpret_cast<const float4*>(spheres);
  a.n = n;
  a.reps = reps;
  a.out = reinterpret_cast<float4*>(out);
  const int64_t groups = (n + 63) / 64;
  int64_t blocks = (groups + CEIL_WARPS - 1) / CEIL_WARPS;
  const int64_t cap = warps / CEIL_WARPS;
  if (blocks > cap) blocks = cap;
  env_ceiling_kernel<<<(int)blocks, CEIL_WARPS * 32, ceiling_smem(sc.O), (cudaStream_t)stream>>>(a);
  return cuda_status(cudaGetLastError());
}
