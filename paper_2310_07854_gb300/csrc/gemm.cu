// Host side of the tcgen05 GEMM (tc_gemm.cuh): tensor-map encoding through
// the runtime's driver entry point (no link against libcuda), and the plain
// FP32-output entry point vapr_gemm_bf16.
#include <cudaTypedefs.h>

#include <mutex>

#include "tc_gemm.cuh"

namespace vapr {

__device__ int g_tc_error;  // sticky: first error code of a tensor-core kernel, 0 if none

int* tc_error_word() {
  static int* p = nullptr;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (!p && cudaGetSymbolAddress((void**)&p, g_tc_error) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

int tc_device_error(bool reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess) return -1;
  if (reset && v) {
    const int z = 0;
    cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
  }
  return v;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  });
  return fn;
}

bool tg_tensor_map(CUtensorMap* map, const void* ptr, uint64_t K, uint64_t rows, uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {K, rows};
  const cuuint64_t strides[1] = {K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TG_K, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace vapr

using namespace vapr;

extern "C" vapr_status vapr_gemm_bf16(const void* A, const void* B, float* C, int64_t M, int64_t N,
                                      int64_t K, void* stream) {
  if (M < 0 || N < 0 || K < 0) return VAPR_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return VAPR_OK;
  if (!A || !B || !C || K == 0) return VAPR_ERR_INVALID_ARG;
  if (M % TG_M || N % TG_N || K % TG_K) return VAPR_ERR_INVALID_ARG;
  if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30)) return VAPR_ERR_TOO_LARGE;
  if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C) % 16) return VAPR_ERR_MISALIGNED;
  int* err = tc_error_word();
  if (!err) return cuda_status(cudaErrorUnknown);
  TgShape sh{(int)M, (int)N, (int)K, (int)K};
  StoreF32 epi{C, (int)N, 0};
  return cuda_status(tg_launch(A, B, sh, epi, err, (cudaStream_t)stream));
}
