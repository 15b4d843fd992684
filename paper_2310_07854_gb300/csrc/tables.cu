// Prebuilt robot tables (vapr_robot_tables_build): the robot's link-grouped
// sphere order, self-collision clusters and self pairs grouped by cluster
// pair (the broad phase of iteration step 3 of Sec. III-B), built once by
// the same block-cooperative code the kernels run (load_robot,
// load_clusters, load_self) and stored in global memory for blocks to copy
// (load_robot_self in stages.cuh).
#include "stages.cuh"

namespace vapr {

constexpr int TB_THREADS = 256;

struct TablesSm {
  RobotSm rb;
  SceneSm sm;
  SelfScratch t;
};

__host__ __device__ inline void carve_tables(Bump& b, const RobotArgs& r, TablesSm& s) {
  carve_robot(b, r.J, r.S, s.rb);
  carve_scene(b, 0, r.NP, cluster_bound(r.S, r.J), s.sm);
  carve_self_scratch(b, r.NP, cluster_bound(r.S, r.J), r.S, s.t);
}

__device__ __forceinline__ void store_granules(void* dst, const void* src, size_t bytes) {
  const int n = (int)((bytes + 15) / 16);
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
}

__global__ void __launch_bounds__(TB_THREADS) robot_tables_kernel(RobotArgs r, uint8_t* out) {
  extern __shared__ float4 smem4[];
  Bump b(smem4);
  TablesSm s;
  carve_tables(b, r, s);
  load_robot(r, s.rb);
  __syncthreads();
  load_clusters(r.J, r.S, s.rb);
  load_self(r, s.rb, s.sm, s.t, 0.f);  // (eta_s is not part of the tables)
  __shared__ uint32_t s_hash;
  if (threadIdx.x == 0) s_hash = 0u;
  __syncthreads();
  atomicAdd(&s_hash, robot_hash_part(r, threadIdx.x, blockDim.x));
  Bump g(out);
  RobotImage im;
  carve_image(g, r.J, r.S, r.NP, im);
  const int J = r.J, S = r.S, NCB = cluster_bound(S, J), NG = s.sm.self_meta[0];
  store_granules(im.rb.F, s.rb.F, 3 * J * sizeof(float4));
  store_granules(im.rb.sph, s.rb.sph, S * sizeof(float4));
  store_granules(im.rb.link0, s.rb.link0, S * sizeof(int));
  store_granules(im.rb.order, s.rb.order, S * sizeof(int));
  store_granules(im.rb.start, s.rb.start, (J + 1) * sizeof(int));
  store_granules(im.rb.cl_start, s.rb.cl_start, (NCB + 1) * sizeof(int));
  store_granules(im.rb.cl_of, s.rb.cl_of, S * sizeof(int));
  store_granules(im.rb.cl_sph, s.rb.cl_sph, NCB * sizeof(int));
  store_granules(im.rb.n_cl, s.rb.n_cl, 2 * sizeof(int));
  store_granules(im.pairs, s.sm.pairs, r.NP * sizeof(uint32_t));
  store_granules(im.cp, s.sm.cp, NG * sizeof(uint16_t));
  store_granules(im.cp_start, s.sm.cp_start, (NG + 1) * sizeof(uint16_t));
  __syncthreads();
  const uint32_t nw = (uint32_t)((g.bytes() - sizeof(TablesHeader)) / 4);
  __shared__ uint32_t s_body;
  if (threadIdx.x == 0) s_body = 0u;
  __syncthreads();
  atomicAdd(&s_body, body_hash_part(reinterpret_cast<const uint32_t*>(im.h + 1), nw, threadIdx.x, blockDim.x));
  __threadfence();  // the arrays before the header that validates them, for every observer
  __syncthreads();
  if (threadIdx.x == 0) {
    TablesHeader h;
    for (int i = 0; i < 8; ++i) h.pad[i] = 0u;
    h.body_words = nw;
    h.body_hash = s_body;
    h.magic = TABLES_MAGIC;
    h.J = (uint32_t)J;
    h.S = (uint32_t)S;
    h.NP = (uint32_t)r.NP;
    h.hash = s_hash;
    h.NG = (uint32_t)NG;
    *im.h = h;
  }
}

size_t robot_tables_bytes(const RobotArgs& r) {
  Bump b(nullptr);
  RobotImage im;
  carve_image(b, r.J, r.S, r.NP, im);
  return b.bytes();
}

cudaError_t launch_robot_tables(RobotArgs r, void* out, cudaStream_t st) {
  r.tables = nullptr;
  Bump b(nullptr);
  TablesSm s;
  carve_tables(b, r, s);
  const size_t smem = b.bytes();
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(robot_tables_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
  }
  robot_tables_kernel<<<1, TB_THREADS, smem, st>>>(r, static_cast<uint8_t*>(out));
  return cudaGetLastError();
}

}  // namespace vapr
