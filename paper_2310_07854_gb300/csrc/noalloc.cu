// vapr_cost_grad_noalloc: the whole step with its scratch in a fixed,
// library-owned device array, for callers that must not allocate device
// memory while they run -- a real-time planning or control loop whose
// latency budget cannot absorb cudaMalloc (which may synchronise the
// device), or a host program whose device memory is fixed at start-up or
// owned by another allocator.  The caller still owns every input and
// output; only the intermediate P and G rows live here.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds VAPR_NOALLOC_SCRATCH_BYTES of it until the process exits.
// In host code its name is only a host-side stand-in, so its device address
// is looked up once per device with cudaGetSymbolAddress (with that device
// current) and cached.
#include <mutex>

#include "common.cuh"

namespace vapr {

static __device__ __align__(256) unsigned char g_noalloc_scratch[VAPR_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices];
static std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (set up on
// the first call per device).
static cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace vapr

extern "C" vapr_status vapr_cost_grad_noalloc(const vapr_robot* robot, const vapr_scene* scene,
                                              const vapr_cost_params* params, const float* q,
                                              int64_t n, const vapr_format_table* table,
                                              const float* dcost, float* cost,
                                              void* dist_packed, void* jgrad_packed,
                                              void* stream) {
  vapr::RobotArgs r;
  vapr_status st = vapr::check_robot(robot, &r);
  if (st != VAPR_OK) return st;
  if ((st = vapr::check_table(table)) != VAPR_OK) return st;
  if (n < 0) return VAPR_ERR_INVALID_ARG;
  if (n > VAPR_MAX_CONFIGS) return VAPR_ERR_TOO_LARGE;
  if (n == 0) return VAPR_OK;
  const size_t need = vapr_cost_grad_workspace_bytes(robot, n, table);
  if (need == 0) return VAPR_ERR_INVALID_ARG;
  if (need > (size_t)VAPR_NOALLOC_SCRATCH_BYTES) return VAPR_ERR_TOO_LARGE;
  void* scratch = nullptr;
  const cudaError_t e = vapr::scratch_address(&scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return VAPR_ERR_CUDA;
  }
  // Nothing in the scratch has to start at zero: FK writes every word of
  // P and the collision kernel every word of G before anything reads them.
  return vapr_cost_grad(robot, scene, params, q, n, table, dcost, cost, dist_packed,
                        jgrad_packed, scratch, (size_t)VAPR_NOALLOC_SCRATCH_BYTES, stream);
}
