// C[M x N] = A[M x K] * B[N x K]^T on the tcgen05 tensor cores, BF16
// operands (row-major, K contiguous), FP32 accumulation in tensor memory,
// with a pluggable epilogue.
//
// One CTA of 4 warps computes a 128 x 256 tile over its K range:
//   warp 0 lane 0  TMA producer: 64-wide K slices of A (128 rows) and B
//                  (256 rows), 128-byte swizzled, into a 3-stage ring;
//   warp 1 lane 0  MMA issuer: four K=16 tcgen05.mma per slice into one
//                  128 x 256 FP32 accumulator (256 TMEM columns), then
//                  tcgen05.commit onto the slice's "empty" mbarrier;
//   all 4 warps    epilogue: warp w owns TMEM lanes 32w..32w+31 (its 32
//                  rows); the epilogue functor epi(taddr, row, n0, z) reads
//                  them with tcgen05.ld (taddr = the warp's lane base).
// Every mbarrier wait is bounded; on timeout the CTA records
// VAPR_ERR_TIMEOUT, skips the rest, lets copies in flight land (bounded)
// and frees its tensor memory.
#pragma once

#include "common.cuh"
#include "tcgen05.cuh"

namespace vapr {

constexpr int TG_M = 128, TG_N = 256, TG_K = 64, TG_STAGES = 3;
constexpr uint32_t TG_A_BYTES = TG_M * TG_K * 2;  // 16 KB
constexpr uint32_t TG_B_BYTES = TG_N * TG_K * 2;  // 32 KB
constexpr uint32_t TG_WAIT = 1u << 22;
constexpr size_t TG_SMEM = 1024 + TG_STAGES * (TG_A_BYTES + TG_B_BYTES) + 256;

struct TgShape {
  int M, N, K;
  int k_split;  // K columns per CTA along grid z (multiple of 64)
};

template <class Epi>
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   TgShape sh, Epi epi, int* err) {
  extern __shared__ uint8_t tg_raw[];
  uint8_t* base = tg_raw + ((1024u - (sm_addr(tg_raw) & 1023u)) & 1023u);
  uint8_t* sA = base;
  uint8_t* sB = base + TG_STAGES * TG_A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + TG_STAGES * TG_B_BYTES);
  uint64_t* empty = full + TG_STAGES;
  uint64_t* done = empty + TG_STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TG_M, n0 = blockIdx.y * TG_N;
  const int kb = blockIdx.z * sh.k_split;
  const int ke = min(sh.K, kb + sh.k_split);
  const int nk = (ke - kb) / TG_K;  // >= 1 (host guarantees)

  if (threadIdx.x == 0) {
    for (int s = 0; s < TG_STAGES; ++s) {
      mb_init(full + s, 1);
      mb_init(empty + s, 1);
    }
    mb_init(done, 1);
    *abort_flag = 0;
    mb_init_fence();
  }
  if (warp == 0) tmem_alloc(tslot, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t IDESC = idesc_bf16_f32(TG_M, TG_N);

  if (warp == 0 && lane == 0) {  // ---- TMA producer
    int issued = 0;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % TG_STAGES;
      if (kt >= TG_STAGES && !mb_wait(empty + s, ((kt / TG_STAGES) - 1) & 1, TG_WAIT)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      mb_expect_tx(full + s, TG_A_BYTES + TG_B_BYTES);
      tma_load_2d(sA + s * TG_A_BYTES, &tmA, kb + kt * TG_K, m0, full + s);
      tma_load_2d(sB + s * TG_B_BYTES, &tmB, kb + kt * TG_K, n0, full + s);
      issued = kt + 1;
    }
    if (*abort_flag)  // let every issued copy land before the CTA can exit
      for (int kt = (issued > TG_STAGES ? issued - TG_STAGES : 0); kt < issued; ++kt)
        mb_wait(full + kt % TG_STAGES, (kt / TG_STAGES) & 1, TG_WAIT);
  } else if (warp == 1 && lane == 0) {  // ---- MMA issuer
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % TG_STAGES;
      if (!mb_wait(full + s, (kt / TG_STAGES) & 1, TG_WAIT)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint64_t ad = sw128_desc(sA + s * TG_A_BYTES), bd = sw128_desc(sB + s * TG_B_BYTES);
#pragma unroll
      for (int kk = 0; kk < TG_K / 16; ++kk)  // K step of 16 bf16 = 32 bytes = 2 descriptor units
        umma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, IDESC, (kt | kk) != 0);
      umma_commit(empty + s);
    }
    umma_commit(done);
  }
  __syncwarp();
  // ---- epilogue: this warp's 32 accumulator rows
  const bool landed = mb_wait(done, 0, TG_WAIT);
  const bool ok = __all_sync(0xffffffffu, landed) && !*abort_flag;
  tc_fence_after();
  if (ok) {
    // the epilogue reads its row's 256 accumulator columns from tensor memory
    // (lane field = TMEM lane, column field = column) with tmem_ld32
    epi(tmem + ((uint32_t)(warp * 32) << 16), m0 + warp * 32 + lane, n0, (int)blockIdx.z);
  } else if (lane == 0) {
    atomicCAS(err, 0, (int)VAPR_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

// Epilogue: FP32 rows of C (split z writes its own C slab).
struct StoreF32 {
  float* C;
  int N;
  int64_t slab;  // elements per split
  __device__ __forceinline__ void operator()(uint32_t taddr, int row, int n0, int z) const {
#pragma unroll 1
    for (int c = 0; c < TG_N / 32; ++c) {
      uint32_t r[32];
      tmem_ld32(taddr + (uint32_t)(c * 32), r);
      float4* out = reinterpret_cast<float4*>(C + z * slab + (int64_t)row * N + n0 + c * 32);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        out[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                             __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
    }
  }
};

// Host: tensor map of a row-major bf16 matrix [rows][K] read in 64 x box_rows
// tiles with 128-byte swizzle.  False if the driver rejects it.
bool tg_tensor_map(CUtensorMap* map, const void* ptr, uint64_t K, uint64_t rows, uint32_t box_rows);

// Host: launches tc_gemm_kernel over M/128 x N/256 x ceil(K/k_split) CTAs.
template <class Epi>
cudaError_t tg_launch(const void* A, const void* B, TgShape sh, Epi epi, int* err, cudaStream_t st) {
  CUtensorMap ma, mb;
  if (!tg_tensor_map(&ma, A, (uint64_t)sh.K, (uint64_t)sh.M, TG_M) ||
      !tg_tensor_map(&mb, B, (uint64_t)sh.K, (uint64_t)sh.N, TG_N))
    return cudaErrorInvalidValue;
  const int per_sm = blocks_per_sm((const void*)tc_gemm_kernel<Epi>, 128, TG_SMEM);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  dim3 grid(sh.M / TG_M, sh.N / TG_N, (sh.K + sh.k_split - 1) / sh.k_split);
  tc_gemm_kernel<Epi><<<grid, 128, TG_SMEM, st>>>(ma, mb, sh, epi, err);
  return cudaGetLastError();
}

}  // namespace vapr
