// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/vapr.h"
#include "exmy.cuh"

namespace vapr {

// Robot tables as the kernels read them (device pointers).
struct RobotArgs {
  int J, S, NP;
  const float* joint_fixed;   // [J][12]
  const float* sphere_local;  // [S][4]
  const int32_t* sphere_link; // [S]
  const int32_t* pairs;       // [NP][2]
  const void* tables = nullptr;  // prebuilt self-collision tables (stages.cuh), or null
};

struct SceneArgs {
  int O;
  const float* pose;  // [O][12]
  const float* half;  // [O][3]
  const void* grid = nullptr;  // broad-phase grid (grid.cuh), or null
};

// A packed tensor: base pointer, row stride in bytes, format.
struct Packed {
  uint8_t* ptr;
  int64_t stride;
  DevFmt f;
};

DevFmt make_dev_fmt(vapr_format f);
// Argument checks shared by the entry points (api.cu).
bool fmt_ok(vapr_format f);
size_t row_bytes(int64_t row_len, vapr_format f);  // packed row, padded to 16 B
vapr_status check_robot(const vapr_robot* r, RobotArgs* out);
// Checks a scene (counts, pointers, alignment) and fills out, grid included.
vapr_status check_scene(const vapr_scene* s, SceneArgs* out);
vapr_status check_table(const vapr_format_table* t);
vapr_status cuda_status(cudaError_t e);           // records the error for vapr_last_cuda_error
int sm_count();  // SMs of the current device (cached per device)
// Resident blocks per SM of `fn` at `threads` and `smem` dynamic bytes on the
// current device.  The first call for a (kernel, device, smem) also raises
// the kernel's dynamic shared-memory limit; later calls hit a cache, so a
// launch costs no attribute or occupancy query.  Returns <= 0 on error.
int blocks_per_sm(const void* fn, int threads, size_t smem);
size_t robot_tables_bytes(const RobotArgs& r);
cudaError_t launch_robot_tables(RobotArgs r, void* out, cudaStream_t st);

int backward_device_error(bool reset);  // sticky device word of vapr_backward
int tc_device_error(bool reset);        // sticky device word of the tensor-core kernels
int* tc_error_word();                   // its device address (for kernel arguments)

cudaError_t launch_fk(const RobotArgs& r, const float* q, int64_t n, Packed pos,
                      Packed xform, cudaStream_t st);
// overlap: launched right after the step's previous stage (vapr_cost_grad),
// whose tail its table loading may overlap (launch_after)
cudaError_t launch_collision(const RobotArgs& r, const SceneArgs& sc,
                             const vapr_cost_params& p, Packed pos, int64_t n,
                             float* cost, Packed dist, Packed grad, cudaStream_t st,
                             const float* est = nullptr, float margin = 0.f, bool overlap = false);
cudaError_t launch_backward(const RobotArgs& r, const float* q, Packed xform,
                            Packed grad, const float* dcost, int64_t n,
                            Packed jgrad, cudaStream_t st, bool overlap = false);
cudaError_t launch_fused(const RobotArgs& r, const SceneArgs& sc, const vapr_cost_params& p, const float* q,
                         const float* dcost, int64_t n, const vapr_format_table& t, float* cost, Packed dist,
                         Packed jgrad, cudaStream_t st);
cudaError_t launch_pack(const float* src, int64_t rows, int64_t row_len, Packed dst,
                        cudaStream_t st);
cudaError_t launch_unpack(Packed src, int64_t rows, int64_t row_len, float* dst,
                          cudaStream_t st);

// Programmatic dependent launch (the stages of a step launched back to back
// on one stream): a kernel launched with launch_after() may start while the
// kernel before it finishes; it must call grid_dependency_wait() before it
// reads anything that kernel writes (until then it only loads its tables).
// grid_dependents_may_launch() lets the next kernel start as this one's
// blocks retire.  Both are no-ops for a kernel launched plainly.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_may_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launches kern<<<grid, block, smem, st>>>(args...); with overlap, so that
// it may start while the kernel launched before it on st finishes (it waits
// for that kernel's results with grid_dependency_wait()).  Only the step's
// own stages are launched this way (vapr_cost_grad): a kernel's work before
// its wait reads only what the kernel before it does not write.
template <typename... Params, typename... Args>
cudaError_t launch_after(bool overlap, void (*kern)(Params...), int grid, int block, size_t smem,
                         cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = overlap ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Params>(args)...);
}

// Clamps a device-table index into [lo, hi] so that a bad table can give a
// wrong answer but never an out-of-bounds access.
__device__ __forceinline__ int clampi(int v, int lo, int hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

}  // namespace vapr
