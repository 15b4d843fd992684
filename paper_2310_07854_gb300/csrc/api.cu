// C ABI entry points (include/vapr.h): argument checks, format tables and
// the pack/unpack converter kernels.  Every check happens before anything is
// enqueued; kernels themselves never abort.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace vapr {

static thread_local int g_last_cuda_error = 0;

vapr_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return VAPR_OK;
  g_last_cuda_error = (int)e;
  return VAPR_ERR_CUDA;
}

bool fmt_ok(vapr_format f) {
  const int E = f.exp_bits, M = f.man_bits, fl = f.flags;
  if (f.reserved != 0) return false;
  if (E < 2 || E > 8 || M < 1 || M > 23) return false;
  if (fl & ~(VAPR_FMT_IEEE | VAPR_FMT_FN | VAPR_FMT_SATFINITE)) return false;
  if ((fl & VAPR_FMT_IEEE) && (fl & VAPR_FMT_FN)) return false;
  if (E == 8 && M == 23) return fl == VAPR_FMT_IEEE;  // float32 itself
  if (1 + E + M > 16) return false;
  if (E == 8 && !(fl & VAPR_FMT_IEEE)) return false;  // would exceed float32
  if ((fl & VAPR_FMT_FN) && M < 1) return false;
  return true;
}

DevFmt make_dev_fmt(vapr_format fm) {
  DevFmt f;
  std::memset(&f, 0, sizeof(f));
  f.E = fm.exp_bits;
  f.M = fm.man_bits;
  f.bits = 1 + f.E + f.M;
  f.k = 32 / f.bits;
  f.mask = f.bits >= 32 ? 0xffffffffu : ((1u << f.bits) - 1u);
  f.ieee = (fm.flags & VAPR_FMT_IEEE) != 0;
  f.fn = (fm.flags & VAPR_FMT_FN) != 0;
  const int sat = (fm.flags & VAPR_FMT_SATFINITE) != 0;
  if (f.E == 8 && f.M == 23) {
    f.kind = KIND_F32;
    return f;
  }
  f.bias = (1 << (f.E - 1)) - 1;
  f.emin = 1 - f.bias;
  f.all_e = (1u << f.E) - 1u;
  f.all_m = (1u << f.M) - 1u;
  if (f.ieee) {
    f.emax_field = f.all_e - 1u;
    f.mmax = f.all_m;
  } else if (f.fn) {
    f.emax_field = f.all_e;
    f.mmax = f.all_m - 1u;
  } else {
    f.emax_field = f.all_e;
    f.mmax = f.all_m;
  }
  f.max_code = (f.emax_field << f.M) | f.mmax;
  f.inf_code = f.all_e << f.M;
  f.nan_code = (f.ieee || f.fn) ? ((f.all_e << f.M) | f.all_m) : f.max_code;
  f.ovf_inf = f.ieee && !sat;
  const unsigned fl = fm.flags;
  f.fastdec = f.E < 8 && !f.ieee && !f.fn;
  f.dec_scale = std::ldexp(1.0f, 127 - f.bias);
  f.enc_scale = std::ldexp(1.0f, f.bias - 127);
  f.enc_lo = (uint32_t)(127 + f.emin) << 23;
  f.kind = KIND_GENERIC;
  if (f.E == 5 && f.M == 10 && fl == VAPR_FMT_IEEE) f.kind = KIND_F16;
  if (f.E == 8 && f.M == 7 && fl == VAPR_FMT_IEEE) f.kind = KIND_BF16;
  if (f.E == 4 && f.M == 3 && fl == (VAPR_FMT_FN | VAPR_FMT_SATFINITE)) f.kind = KIND_E4M3;
  if (f.E == 5 && f.M == 2 && fl == (VAPR_FMT_IEEE | VAPR_FMT_SATFINITE)) f.kind = KIND_E5M2;
  if (f.E == 2 && f.M == 1 && fl == VAPR_FMT_SATFINITE) f.kind = KIND_E2M1;
  if (f.E == 3 && f.M == 2 && fl == VAPR_FMT_SATFINITE) f.kind = KIND_E3M2;
  if (f.E == 2 && f.M == 3 && fl == VAPR_FMT_SATFINITE) f.kind = KIND_E2M3;
#ifdef VAPR_GENERIC_CONVERTERS_ONLY
  f.kind = KIND_GENERIC;
#endif
  return f;
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 148;
  }
  return cached[dev];
}

int blocks_per_sm(const void* fn, int threads, size_t smem) {
  struct Entry {
    const void* fn;
    int dev, threads;
    size_t smem;
    int blocks;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  static std::vector<std::pair<const void*, int>> raised;  // (kernel, device) done
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  std::lock_guard<std::mutex> lock(mu);
  for (const Entry& e : cache)
    if (e.fn == fn && e.dev == dev && e.threads == threads && e.smem == smem) return e.blocks;
  bool done = false;
  for (const auto& r : raised) done |= (r.first == fn && r.second == dev);
  if (!done) {  // allow up to the device's opt-in maximum once; launches use less
    int optin = 0;
    cudaFuncAttributes fa;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, fn) != cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes) != cudaSuccess) {  // minus static shared
      cudaGetLastError();  // clear it: a later launch check must not see this
      return -1;
    }
    raised.emplace_back(fn, dev);
  }
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    blocks = 0;  // does not fit (e.g. too much shared memory): cache the answer
  }
  cache.push_back(Entry{fn, dev, threads, smem, blocks});
  return blocks;
}

size_t row_bytes(int64_t row_len, vapr_format f) {
  if (row_len <= 0 || !fmt_ok(f)) return 0;
  const int64_t k = 32 / (1 + f.exp_bits + f.man_bits);
  const int64_t words = (row_len + k - 1) / k;
  return (size_t)(((4 * words + 15) / 16) * 16);
}

static bool aligned(const void* p, uintptr_t a) { return ((uintptr_t)p % a) == 0; }

// ---------------------------------------------------------------- pack/unpack
// One thread per 16-byte chunk of a packed row; the float source is read
// contiguously by consecutive threads.
__global__ void pack_kernel(const float* __restrict__ src, int64_t rows, int row_len,
                            Packed dst) {
  const int cpr = (int)(dst.stride / 16);
  const int64_t total = rows * cpr;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = c / cpr;
    const int cc = (int)(c - r * cpr);
    const float* row = src + r * row_len;
    *reinterpret_cast<uint4*>(dst.ptr + r * dst.stride + 16 * cc) =
        pack_chunk_dyn(cc, row_len, dst.f, [&](int i) { return row[i]; });
  }
}

__global__ void unpack_kernel(Packed src, int64_t rows, int row_len, float* __restrict__ dst) {
  const int cpr = (int)(src.stride / 16);
  const int64_t total = rows * cpr;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = c / cpr;
    const int cc = (int)(c - r * cpr);
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(src.ptr + r * src.stride + 16 * cc));
    float* row = dst + r * row_len;
    unpack_chunk_dyn(v, cc, row_len, src.f, [&](int i, float x) { row[i] = x; });
  }
}

static int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  const int64_t cap = (int64_t)sm_count() * 16;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_pack(const float* src, int64_t rows, int64_t row_len, Packed dst,
                        cudaStream_t st) {
  const int64_t work = rows * (dst.stride / 16);
  pack_kernel<<<grid_for(work, 256), 256, 0, st>>>(src, rows, (int)row_len, dst);
  return cudaGetLastError();
}

cudaError_t launch_unpack(Packed src, int64_t rows, int64_t row_len, float* dst,
                          cudaStream_t st) {
  const int64_t work = rows * (src.stride / 16);
  unpack_kernel<<<grid_for(work, 256), 256, 0, st>>>(src, rows, (int)row_len, dst);
  return cudaGetLastError();
}

vapr_status check_robot(const vapr_robot* r, RobotArgs* out) {
  if (!r) return VAPR_ERR_INVALID_ARG;
  if (r->n_joints < 1 || r->n_joints > VAPR_MAX_JOINTS) return VAPR_ERR_INVALID_ARG;
  if (r->n_spheres < 1 || r->n_spheres > VAPR_MAX_SPHERES) return VAPR_ERR_INVALID_ARG;
  if (r->n_pairs < 0 || r->n_pairs > VAPR_MAX_PAIRS) return VAPR_ERR_INVALID_ARG;
  if (!r->joint_fixed || !r->sphere_local || !r->sphere_link) return VAPR_ERR_INVALID_ARG;
  if (r->n_pairs > 0 && !r->pairs) return VAPR_ERR_INVALID_ARG;
  if (!aligned(r->joint_fixed, 16) || !aligned(r->sphere_local, 16) ||
      !aligned(r->sphere_link, 16) || (r->pairs && !aligned(r->pairs, 16)) ||
      (r->tables && !aligned(r->tables, 16)))
    return VAPR_ERR_MISALIGNED;
  out->J = r->n_joints;
  out->S = r->n_spheres;
  out->NP = r->n_pairs;
  out->joint_fixed = r->joint_fixed;
  out->sphere_local = r->sphere_local;
  out->sphere_link = r->sphere_link;
  out->pairs = r->pairs;
  out->tables = r->tables;
  return VAPR_OK;
}

vapr_status check_scene(const vapr_scene* s, SceneArgs* out) {
  if (!s || s->n_cuboids < 0) return VAPR_ERR_INVALID_ARG;
  if (s->n_cuboids > VAPR_MAX_CUBOIDS) return VAPR_ERR_TOO_LARGE;
  if (s->n_cuboids > 0 && (!s->pose || !s->half_ext)) return VAPR_ERR_INVALID_ARG;
  if (s->n_cuboids > 0 && (!aligned(s->pose, 16) || !aligned(s->half_ext, 4)))
    return VAPR_ERR_MISALIGNED;
  if (s->grid && !aligned(s->grid, 16)) return VAPR_ERR_MISALIGNED;
  out->O = s->n_cuboids;
  out->pose = s->pose;
  out->half = s->half_ext;
  out->grid = s->grid;
  return VAPR_OK;
}

vapr_status check_table(const vapr_format_table* t) {
  if (!t) return VAPR_ERR_INVALID_ARG;
  if (!fmt_ok(t->pos) || !fmt_ok(t->dist) || !fmt_ok(t->grad) || !fmt_ok(t->jgrad) ||
      !fmt_ok(t->xform))
    return VAPR_ERR_UNSUPPORTED_FORMAT;
  return VAPR_OK;
}

static Packed packed(const void* p, int64_t row_len, vapr_format f) {
  Packed x;
  x.ptr = (uint8_t*)p;
  x.stride = (int64_t)row_bytes(row_len, f);
  x.f = make_dev_fmt(f);
  return x;
}

}  // namespace vapr

using namespace vapr;

extern "C" {

size_t vapr_robot_tables_bytes(const vapr_robot* robot) {
  RobotArgs r;
  if (check_robot(robot, &r) != VAPR_OK) return 0;
  return robot_tables_bytes(r);
}

vapr_status vapr_robot_tables_build(const vapr_robot* robot, void* tables, size_t bytes, void* stream) {
  RobotArgs r;
  const vapr_status st = check_robot(robot, &r);
  if (st != VAPR_OK) return st;
  if (!tables) return VAPR_ERR_INVALID_ARG;
  if (!aligned(tables, 16)) return VAPR_ERR_MISALIGNED;
  if (bytes < robot_tables_bytes(r)) return VAPR_ERR_INVALID_ARG;
  return launch_robot_tables(r, tables, (cudaStream_t)stream) == cudaSuccess ? VAPR_OK : VAPR_ERR_CUDA;
}

const char* vapr_status_string(vapr_status s) {
  switch (s) {
    case VAPR_OK: return "ok";
    case VAPR_ERR_INVALID_ARG: return "invalid argument";
    case VAPR_ERR_UNSUPPORTED_FORMAT: return "unsupported format";
    case VAPR_ERR_MISALIGNED: return "misaligned pointer";
    case VAPR_ERR_CUDA: return "CUDA error";
    case VAPR_ERR_TIMEOUT: return "device wait timed out";
    case VAPR_ERR_TOO_LARGE: return "size above the documented maximum";
  }
  return "unknown status";
}

int vapr_last_cuda_error(void) { return g_last_cuda_error; }

vapr_format vapr_format_default(int E, int M) {
  vapr_format f;
  f.exp_bits = (uint8_t)E;
  f.man_bits = (uint8_t)M;
  f.reserved = 0;
  if ((E == 8 && M == 23) || (E == 8 && M == 7) || (E == 5 && M == 10))
    f.flags = VAPR_FMT_IEEE;
  else if (E == 5 && M == 2)
    f.flags = VAPR_FMT_IEEE | VAPR_FMT_SATFINITE;
  else if (E == 4 && M == 3)
    f.flags = VAPR_FMT_FN | VAPR_FMT_SATFINITE;
  else if (E == 8)
    f.flags = VAPR_FMT_IEEE | VAPR_FMT_SATFINITE;
  else
    f.flags = VAPR_FMT_SATFINITE;
  return f;
}

int vapr_format_supported(vapr_format f) { return fmt_ok(f) ? 1 : 0; }

size_t vapr_packed_row_bytes(int64_t row_len, vapr_format f) { return row_bytes(row_len, f); }

vapr_status vapr_device_error(int32_t* code) {
  if (!code) return VAPR_ERR_INVALID_ARG;
  const int v = backward_device_error(true);
  const int w = tc_device_error(true);
  if (v < 0 || w < 0) return cuda_status(cudaErrorUnknown);
  *code = v ? v : w;
  return VAPR_OK;
}

vapr_status vapr_robot_check(const vapr_robot* robot) {
  RobotArgs r;
  vapr_status st = check_robot(robot, &r);
  if (st != VAPR_OK) return st;
  std::vector<float> local((size_t)r.S * 4);
  std::vector<int32_t> link((size_t)r.S), pairs((size_t)r.NP * 2);
  cudaError_t e = cudaMemcpy(local.data(), r.sphere_local, local.size() * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(link.data(), r.sphere_link, link.size() * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && r.NP)
    e = cudaMemcpy(pairs.data(), r.pairs, pairs.size() * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  for (int s = 0; s < r.S; ++s) {
    if (link[s] < 1 || link[s] > r.J) return VAPR_ERR_INVALID_ARG;
    if (!(local[4 * s + 3] >= 0.0f)) return VAPR_ERR_INVALID_ARG;
  }
  for (int p = 0; p < r.NP; ++p) {
    const int i = pairs[2 * p], j = pairs[2 * p + 1];
    if (i < 0 || j < 0 || i >= r.S || j >= r.S || i == j) return VAPR_ERR_INVALID_ARG;
  }
  return VAPR_OK;
}

vapr_status vapr_pack(const float* src, int64_t rows, int64_t row_len, vapr_format f,
                      void* dst, void* stream) {
  if (!fmt_ok(f)) return VAPR_ERR_UNSUPPORTED_FORMAT;
  if (rows < 0 || row_len < 0) return VAPR_ERR_INVALID_ARG;
  if (row_len > (int64_t)1 << 30) return VAPR_ERR_TOO_LARGE;
  if (rows == 0 || row_len == 0) return VAPR_OK;
  if (!src || !dst) return VAPR_ERR_INVALID_ARG;
  if (!aligned(src, 4) || !aligned(dst, 16)) return VAPR_ERR_MISALIGNED;
  return cuda_status(launch_pack(src, rows, row_len, packed(dst, row_len, f),
                                 (cudaStream_t)stream));
}

vapr_status vapr_unpack(const void* src, int64_t rows, int64_t row_len, vapr_format f,
                        float* dst, void* stream) {
  if (!fmt_ok(f)) return VAPR_ERR_UNSUPPORTED_FORMAT;
  if (rows < 0 || row_len < 0) return VAPR_ERR_INVALID_ARG;
  if (row_len > (int64_t)1 << 30) return VAPR_ERR_TOO_LARGE;
  if (rows == 0 || row_len == 0) return VAPR_OK;
  if (!src || !dst) return VAPR_ERR_INVALID_ARG;
  if (!aligned(src, 16) || !aligned(dst, 4)) return VAPR_ERR_MISALIGNED;
  return cuda_status(launch_unpack(packed(src, row_len, f), rows, row_len, dst,
                                   (cudaStream_t)stream));
}

vapr_status vapr_fk(const vapr_robot* robot, const float* q, int64_t n,
                    const vapr_format_table* table, void* pos_packed, void* xform_packed,
                    void* stream) {
  RobotArgs r;
  vapr_status st = check_robot(robot, &r);
  if (st != VAPR_OK) return st;
  if ((st = check_table(table)) != VAPR_OK) return st;
  if (n < 0) return VAPR_ERR_INVALID_ARG;
  if (n > VAPR_MAX_CONFIGS) return VAPR_ERR_TOO_LARGE;
  if (n == 0) return VAPR_OK;
  if (!q || !pos_packed) return VAPR_ERR_INVALID_ARG;
  if (!aligned(q, 4) || !aligned(pos_packed, 16) || (xform_packed && !aligned(xform_packed, 16)))
    return VAPR_ERR_MISALIGNED;
  Packed pos = packed(pos_packed, 3 * (int64_t)r.S, table->pos);
  Packed xf = packed(xform_packed, 12 * (int64_t)r.J, table->xform);
  return cuda_status(launch_fk(r, q, n, pos, xf, (cudaStream_t)stream));
}

vapr_status vapr_collision_cost(const vapr_robot* robot, const vapr_scene* scene,
                                const vapr_cost_params* params, const void* pos_packed,
                                int64_t n, const vapr_format_table* table, float* cost,
                                void* dist_packed, void* grad_packed, void* stream) {
  RobotArgs r;
  vapr_status st = check_robot(robot, &r);
  if (st != VAPR_OK) return st;
  if ((st = check_table(table)) != VAPR_OK) return st;
  if (!params) return VAPR_ERR_INVALID_ARG;
  SceneArgs sc;
  if ((st = check_scene(scene, &sc)) != VAPR_OK) return st;
  if (n < 0) return VAPR_ERR_INVALID_ARG;
  if (n > VAPR_MAX_CONFIGS) return VAPR_ERR_TOO_LARGE;
  if (n == 0) return VAPR_OK;
  if (!pos_packed) return VAPR_ERR_INVALID_ARG;
  if (!aligned(pos_packed, 16) || (cost && !aligned(cost, 4)) ||
      (dist_packed && !aligned(dist_packed, 16)) || (grad_packed && !aligned(grad_packed, 16)))
    return VAPR_ERR_MISALIGNED;
  return cuda_status(launch_collision(
      r, sc, *params, packed(pos_packed, 3 * (int64_t)r.S, table->pos), n, cost,
      packed(dist_packed, r.S, table->dist), packed(grad_packed, 3 * (int64_t)r.S, table->grad),
      (cudaStream_t)stream));
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t vapr_cost_grad_workspace_bytes(const vapr_robot* robot, int64_t n,
                                      const vapr_format_table* table) {
  RobotArgs r;
  if (check_robot(robot, &r) != VAPR_OK || check_table(table) != VAPR_OK || n < 0 ||
      n > VAPR_MAX_CONFIGS)
    return 0;
  const size_t P = row_bytes(3 * (int64_t)r.S, table->pos) * (size_t)n;
  const size_t G = row_bytes(3 * (int64_t)r.S, table->grad) * (size_t)n;
  return align256(P) + align256(G);
}

vapr_status vapr_cost_grad(const vapr_robot* robot, const vapr_scene* scene,
                           const vapr_cost_params* params, const float* q, int64_t n,
                           const vapr_format_table* table, const float* dcost, float* cost,
                           void* dist_packed, void* jgrad_packed, void* workspace,
                           size_t workspace_bytes, void* stream) {
  RobotArgs r;
  vapr_status st = check_robot(robot, &r);
  if (st != VAPR_OK) return st;
  if ((st = check_table(table)) != VAPR_OK) return st;
  if (!params) return VAPR_ERR_INVALID_ARG;
  SceneArgs sc;
  if ((st = check_scene(scene, &sc)) != VAPR_OK) return st;
  if (n < 0) return VAPR_ERR_INVALID_ARG;
  if (n > VAPR_MAX_CONFIGS) return VAPR_ERR_TOO_LARGE;
  if (n == 0) return VAPR_OK;
  if (!q || !cost || !jgrad_packed || !workspace) return VAPR_ERR_INVALID_ARG;
  if (workspace_bytes < vapr_cost_grad_workspace_bytes(robot, n, table)) return VAPR_ERR_INVALID_ARG;
  if (!aligned(q, 4) || !aligned(cost, 4) || (dcost && !aligned(dcost, 4)) ||
      !aligned(jgrad_packed, 16) || (dist_packed && !aligned(dist_packed, 16)) ||
      !aligned(workspace, 256))
    return VAPR_ERR_MISALIGNED;
  const cudaStream_t s = (cudaStream_t)stream;
  uint8_t* ws = (uint8_t*)workspace;
  Packed pos = packed(ws, 3 * (int64_t)r.S, table->pos);
  Packed grad = packed(ws + align256((size_t)pos.stride * (size_t)n), 3 * (int64_t)r.S, table->grad);
  Packed none = packed(nullptr, 12 * (int64_t)r.J, table->xform);
  cudaError_t e = launch_fk(r, q, n, pos, none, s);
  // the collision and backward kernels may load their tables while the
  // stage before them finishes (programmatic dependent launch), up to 2^18
  // configurations: beyond that the stage before runs several waves, and
  // the early blocks' hold on the SMs costs more than the overlap saves
  // (measured on the particle arm: -20 us at 32,768, even at 2^18, +85 us
  // at 2^20)
  const bool overlap = n <= ((int64_t)1 << 18);
  if (e == cudaSuccess)
    e = launch_collision(r, sc, *params, pos, n, cost, packed(dist_packed, r.S, table->dist), grad, s,
                         nullptr, 0.f, overlap);
  if (e == cudaSuccess)
    e = launch_backward(r, q, none, grad, dcost, n, packed(jgrad_packed, r.J, table->jgrad), s, overlap);
  return cuda_status(e);
}

vapr_status vapr_cost_grad_fused(const vapr_robot* robot, const vapr_scene* scene,
                                 const vapr_cost_params* params, const float* q, int64_t n,
                                 const vapr_format_table* table, const float* dcost, float* cost,
                                 void* dist_packed, void* jgrad_packed, void* stream) {
  RobotArgs r;
  vapr_status st = check_robot(robot, &r);
  if (st != VAPR_OK) return st;
  if ((st = check_table(table)) != VAPR_OK) return st;
  if (!params) return VAPR_ERR_INVALID_ARG;
  SceneArgs sc;
  if ((st = check_scene(scene, &sc)) != VAPR_OK) return st;
  if (n < 0) return VAPR_ERR_INVALID_ARG;
  if (n > VAPR_MAX_CONFIGS) return VAPR_ERR_TOO_LARGE;
  if (n == 0) return VAPR_OK;
  if (!q || !cost || !jgrad_packed) return VAPR_ERR_INVALID_ARG;
  if (!aligned(q, 4) || !aligned(cost, 4) || (dcost && !aligned(dcost, 4)) || !aligned(jgrad_packed, 16) ||
      (dist_packed && !aligned(dist_packed, 16)))
    return VAPR_ERR_MISALIGNED;
  return cuda_status(launch_fused(r, sc, *params, q, dcost, n, *table, cost, packed(dist_packed, r.S, table->dist),
                                  packed(jgrad_packed, r.J, table->jgrad), (cudaStream_t)stream));
}

vapr_status vapr_backward(const vapr_robot* robot, const float* q, const void* xform_packed,
                          const void* grad_packed, const float* dcost, int64_t n,
                          const vapr_format_table* table, void* jgrad_packed, void* stream) {
  RobotArgs r;
  vapr_status st = check_robot(robot, &r);
  if (st != VAPR_OK) return st;
  if ((st = check_table(table)) != VAPR_OK) return st;
  if (n < 0) return VAPR_ERR_INVALID_ARG;
  if (n > VAPR_MAX_CONFIGS) return VAPR_ERR_TOO_LARGE;
  if (n == 0) return VAPR_OK;
  if (!grad_packed || !jgrad_packed || (!q && !xform_packed)) return VAPR_ERR_INVALID_ARG;
  if ((q && !aligned(q, 4)) || !aligned(grad_packed, 16) || !aligned(jgrad_packed, 16) ||
      (xform_packed && !aligned(xform_packed, 16)) || (dcost && !aligned(dcost, 4)))
    return VAPR_ERR_MISALIGNED;
  return cuda_status(launch_backward(
      r, q, packed(xform_packed, 12 * (int64_t)r.J, table->xform),
      packed(grad_packed, 3 * (int64_t)r.S, table->grad), dcost, n,
      packed(jgrad_packed, r.J, table->jgrad), (cudaStream_t)stream));
}

}  // extern "C"
