// ExMy storage converters used on every load and store of a packed tensor.
//
// Sec. IV-A: a format has 1 sign bit, E exponent bits and M mantissa bits,
// and one 32-bit register holds k = floor(32 / (1+E+M)) values.  Sec. V-B:
// float32 -> format conversion rounds to nearest, ties to even ("_rn").
// Special values follow the flags documented in include/vapr.h.
//
// Two implementations share one contract and must agree bit for bit:
//  * a generic integer path valid for every supported (E, M, flags);
//  * hardware cvt paths (sm_100-family cvt instructions) for the standard
//    formats: half, bfloat16, E4M3, E5M2, E2M1, E3M2, E2M3.  Sec. VIII of
//    the paper proposes a fast converter unit for sub-16-bit formats; on
//    sm_103a such conversions exist as instructions, so the "proposed"
//    converter is real here.  NaN inputs are mapped in software before the
//    instruction so that every path gives the documented code.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace vapr {

enum FmtKind : int {
  KIND_F32 = 0,   // E8M23: identity on bits
  KIND_GENERIC,   // integer rounding, any format
  KIND_F16,       // E5M10 IEEE
  KIND_BF16,      // E8M7 IEEE
  KIND_E4M3,      // OCP fn, saturating
  KIND_E5M2,      // IEEE-style, saturating
  KIND_E2M1,      // finite, saturating
  KIND_E3M2,
  KIND_E2M3,
};

// Everything a kernel needs to convert one tensor; built on the host.
struct DevFmt {
  int kind;
  int E, M, bits, k;      // k values per 32-bit word
  uint32_t mask;          // low `bits` ones
  int bias, emin;         // emin: exponent of the smallest normal
  uint32_t all_e, all_m;
  uint32_t emax_field;    // largest exponent field of a finite value
  uint32_t mmax;          // largest mantissa at emax_field
  uint32_t max_code, inf_code, nan_code;
  int ovf_inf;            // overflow -> Inf (IEEE without saturation)
  int ieee, fn;
};

__device__ __forceinline__ uint32_t encode_generic(float x, const DevFmt& f) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t a = u & 0x7fffffffu;
  if (a > 0x7f800000u) return f.nan_code;
  const uint32_t sbit = (u >> 31) << (f.E + f.M);
  if (a == 0x7f800000u) return sbit | (f.ovf_inf ? f.inf_code : f.max_code);
  if (a == 0u) return sbit;
  const int e32 = (int)(a >> 23);
  const uint32_t sig = e32 ? ((a & 0x7fffffu) | 0x800000u) : (a & 0x7fffffu);
  const int ex = e32 ? e32 - 150 : -149;                    // value = sig * 2^ex
  const int elog = e32 ? e32 - 127 : (-149 + 31 - __clz(sig));  // floor(log2 value)
  int qe = (elog > f.emin ? elog : f.emin) - f.M;            // quantum exponent
  const int shift = qe - ex;                                  // >= 1 for every format
  if (shift > 24) return sbit;                                // below half a quantum
  uint32_t n = sig >> shift;
  const uint32_t rem = sig & ((1u << shift) - 1u);
  const uint32_t half = 1u << (shift - 1);
  if (rem > half || (rem == half && (n & 1u))) ++n;
  if (n == 0u) return sbit;
  if (qe == f.emin - f.M && n < (1u << f.M)) return sbit | n;  // subnormal
  if (n == (2u << f.M)) {  // rounding carried into the next binade
    n >>= 1;
    ++qe;
  }
  const uint32_t efield = (uint32_t)(qe + f.M + f.bias);
  const uint32_t mant = n - (1u << f.M);
  if (efield > f.emax_field || (efield == f.emax_field && mant > f.mmax))
    return sbit | (f.ovf_inf ? f.inf_code : f.max_code);
  return sbit | (efield << f.M) | mant;
}

__device__ __forceinline__ float decode_generic(uint32_t code, const DevFmt& f) {
  const uint32_t s = ((code >> (f.E + f.M)) & 1u) << 31;
  const uint32_t ef = (code >> f.M) & f.all_e;
  const uint32_t mf = code & f.all_m;
  if (f.ieee && ef == f.all_e) return __uint_as_float(mf ? 0x7fc00000u : (s | 0x7f800000u));
  if (f.fn && ef == f.all_e && mf == f.all_m) return __uint_as_float(0x7fc00000u);
  if (ef == 0u) {
    if (mf == 0u) return __uint_as_float(s);
    const int p = 31 - __clz(mf);                 // leading one of the mantissa
    const int ev = f.emin - f.M + p;              // exponent of the value
    if (ev >= -126)
      return __uint_as_float(s | ((uint32_t)(ev + 127) << 23) | ((mf << (23 - p)) & 0x7fffffu));
    return __uint_as_float(s | (mf << (23 - f.M)));  // float32 subnormal (E = 8)
  }
  return __uint_as_float(s | ((uint32_t)((int)ef - f.bias + 127) << 23) | (mf << (23 - f.M)));
}

// ---- hardware conversions (one value in the low part of the result) ----
__device__ __forceinline__ uint32_t cvt_e4m3(float x) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(0.0f), "f"(x));
  return r & 0xffu;
}
__device__ __forceinline__ uint32_t cvt_e5m2(float x) {
  uint16_t r;
  asm("cvt.rn.satfinite.e5m2x2.f32 %0, %1, %2;" : "=h"(r) : "f"(0.0f), "f"(x));
  return r & 0xffu;
}
__device__ __forceinline__ uint32_t cvt_e2m1(float x) {
  uint32_t r;
  asm("{ .reg .b8 t; cvt.rn.satfinite.e2m1x2.f32 t, %1, %2; cvt.u32.u8 %0, t; }"
      : "=r"(r) : "f"(0.0f), "f"(x));
  return r & 0xfu;
}
__device__ __forceinline__ uint32_t cvt_e3m2(float x) {
  uint16_t r;
  asm("cvt.rn.satfinite.e3m2x2.f32 %0, %1, %2;" : "=h"(r) : "f"(0.0f), "f"(x));
  return r & 0x3fu;
}
__device__ __forceinline__ uint32_t cvt_e2m3(float x) {
  uint16_t r;
  asm("cvt.rn.satfinite.e2m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(0.0f), "f"(x));
  return r & 0x3fu;
}
// sub-16-bit code (low byte) -> half (low half) -> float
__device__ __forceinline__ float from_h2lo(uint32_t h2) {
  return __half2float(__ushort_as_half((unsigned short)(h2 & 0xffffu)));
}
__device__ __forceinline__ float dec_e4m3(uint32_t c) {
  uint32_t h2;
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"((uint16_t)c));
  return from_h2lo(h2);
}
__device__ __forceinline__ float dec_e5m2(uint32_t c) {
  uint32_t h2;
  asm("cvt.rn.f16x2.e5m2x2 %0, %1;" : "=r"(h2) : "h"((uint16_t)c));
  return from_h2lo(h2);
}
__device__ __forceinline__ float dec_e2m1(uint32_t c) {
  uint32_t h2;
  asm("{ .reg .b8 t; cvt.u8.u32 t, %1; cvt.rn.f16x2.e2m1x2 %0, t; }" : "=r"(h2) : "r"(c));
  return from_h2lo(h2);
}
__device__ __forceinline__ float dec_e3m2(uint32_t c) {
  uint32_t h2;
  asm("cvt.rn.f16x2.e3m2x2 %0, %1;" : "=r"(h2) : "h"((uint16_t)c));
  return from_h2lo(h2);
}
__device__ __forceinline__ float dec_e2m3(uint32_t c) {
  uint32_t h2;
  asm("cvt.rn.f16x2.e2m3x2 %0, %1;" : "=r"(h2) : "h"((uint16_t)c));
  return from_h2lo(h2);
}

__device__ __forceinline__ uint32_t encode(float x, const DevFmt& f) {
  switch (f.kind) {
    case KIND_F32:
      return __float_as_uint(x);
    case KIND_F16:
      return x != x ? f.nan_code : (uint32_t)__half_as_ushort(__float2half_rn(x));
    case KIND_BF16:
      return x != x ? f.nan_code : (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
    case KIND_E4M3:
      return x != x ? f.nan_code : cvt_e4m3(x);
    case KIND_E5M2:
      return x != x ? f.nan_code : cvt_e5m2(x);
    case KIND_E2M1:
      return x != x ? f.nan_code : cvt_e2m1(x);
    case KIND_E3M2:
      return x != x ? f.nan_code : cvt_e3m2(x);
    case KIND_E2M3:
      return x != x ? f.nan_code : cvt_e2m3(x);
    default:
      return encode_generic(x, f);
  }
}

__device__ __forceinline__ float decode(uint32_t c, const DevFmt& f) {
  switch (f.kind) {
    case KIND_F32:
      return __uint_as_float(c);
    case KIND_F16:
      return __half2float(__ushort_as_half((unsigned short)c));
    case KIND_BF16:
      return __uint_as_float(c << 16);
    case KIND_E4M3:
      return dec_e4m3(c);
    case KIND_E5M2:
      return dec_e5m2(c);
    case KIND_E2M1:
      return dec_e2m1(c);
    case KIND_E3M2:
      return dec_e3m2(c);
    case KIND_E2M3:
      return dec_e2m3(c);
    default:
      return decode_generic(c, f);
  }
}

// Value j (0 <= j < k) of a packed word.
__device__ __forceinline__ float unpack_slot(uint32_t word, int j, const DevFmt& f) {
  return decode((word >> (f.bits * j)) & f.mask, f);
}

// Packs the values i = w*k .. w*k+k-1 (those < n) of a row into word w;
// get(i) returns value i as float.
template <typename Get>
__device__ __forceinline__ uint32_t pack_word(int w, int n, const DevFmt& f, Get get) {
  uint32_t word = 0u;
  const int i0 = w * f.k;
  for (int j = 0; j < f.k; ++j) {
    const int i = i0 + j;
    if (i < n) word |= (encode(get(i), f) & f.mask) << (f.bits * j);
  }
  return word;
}

}  // namespace vapr
