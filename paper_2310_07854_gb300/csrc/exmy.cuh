// ExMy storage converters used on every load and store of a packed tensor.
//
// Sec. IV-A: a format has 1 sign bit, E exponent bits and M mantissa bits,
// and one 32-bit register holds k = floor(32 / (1+E+M)) values.  Sec. V-B:
// float32 -> format conversion rounds to nearest, ties to even ("_rn").
// Special values follow the flags documented in include/vapr.h.
//
// Two implementations share one contract and must agree bit for bit:
//  * a generic integer path valid for every supported (E, M, flags);
//  * hardware cvt paths for the standard formats (half, bfloat16, E4M3,
//    E5M2, E2M1, E3M2, E2M3), two values per instruction.  Appendix A of
//    the paper proposes a fast converter unit for sub-16-bit formats; on
//    sm_103a those conversions are instructions.  NaN inputs are patched in
//    software after the instruction so every path gives the documented code.
//
// Kernels move whole 16-byte chunks (4 words = 4k values).  pack_chunk /
// unpack_chunk are templated on the format kind, so k, the bit offsets and
// the conversion are compile-time; the *_dyn dispatchers switch on the kind
// once per chunk.
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
  int fastdec;            // finite-only, all codes numeric, E < 8: decode by one multiply,
                          // and encode |x| >= 2^emin by one multiply and an integer rounding
  float dec_scale;        // 2^(127 - bias)
  float enc_scale;        // 2^(bias - 127)
  uint32_t enc_lo;        // float32 bits of 2^emin, the smallest normal value
};

// ------------------------------------------------------------ generic path
__device__ __forceinline__ uint32_t encode_exact(float x, const DevFmt& f) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t a = u & 0x7fffffffu;
  if (a > 0x7f800000u) return f.nan_code;
  const uint32_t sbit = (u >> 31) << (f.E + f.M);
  if (a == 0x7f800000u) return sbit | (f.ovf_inf ? f.inf_code : f.max_code);
  if (a == 0u) return sbit;
  const int e32 = (int)(a >> 23);
  const uint32_t sig = e32 ? ((a & 0x7fffffu) | 0x800000u) : (a & 0x7fffffu);
  const int ex = e32 ? e32 - 150 : -149;                        // value = sig * 2^ex
  const int elog = e32 ? e32 - 127 : (-149 + 31 - __clz(sig));  // floor(log2 value)
  int qe = (elog > f.emin ? elog : f.emin) - f.M;               // quantum exponent
  const int shift = qe - ex;                                     // >= 1 for every format
  if (shift > 24) return sbit;                                   // below half a quantum
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

// encode_exact's codes, faster for the finite formats with E < 8 (fastdec):
// for |x| >= 2^emin (or 0), |x| 2^(bias - 127) is an exact float32 whose
// exponent field is the format's, so rounding its bits to M mantissa bits
// (an integer add of half a unit less one, plus the lowest kept bit: ties
// to even, carries into the exponent included) gives the code's magnitude;
// past the largest value it saturates, as the format does.  Values below
// 2^emin (the format's subnormals), Inf and NaN take the exact path.
__device__ __forceinline__ uint32_t encode_generic(float x, const DevFmt& f) {
  if (f.fastdec) {
    const uint32_t u = __float_as_uint(x), a = u & 0x7fffffffu;
    if ((a == 0u || a >= f.enc_lo) && a < 0x7f800000u) {
      const uint32_t y = __float_as_uint(__uint_as_float(a) * f.enc_scale);
      const int sh = 23 - f.M;
      const uint32_t mag = (y + ((1u << (sh - 1)) - 1u) + ((y >> sh) & 1u)) >> sh;
      return ((u >> 31) << (f.E + f.M)) | (mag < f.max_code ? mag : f.max_code);
    }
  }
  return encode_exact(x, f);
}

__device__ __forceinline__ float decode_generic(uint32_t code, const DevFmt& f) {
  const uint32_t s = ((code >> (f.E + f.M)) & 1u) << 31;
  if (f.fastdec) {
    // The code's exponent and mantissa fields placed at float32's mantissa
    // point read as 2^(e - 127) (1 + m 2^-M) (e > 0) or m 2^(-126 - M)
    // (e = 0); times 2^(127 - bias) that is the format's value, normal or
    // subnormal, exactly (E < 8 keeps every value a normal float32 or zero).
    const uint32_t mag = code & ((1u << (f.E + f.M)) - 1u);
    return __uint_as_float(__float_as_uint(__uint_as_float(mag << (23 - f.M)) * f.dec_scale) | s);
  }
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

// ------------------------------------------------- hardware pair conversions
// Each returns the codes of (lo, hi) with lo in the low bits.
__device__ __forceinline__ uint32_t cvt2_f16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ uint32_t cvt2_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ uint32_t cvt2_e4m3(float lo, float hi) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ uint32_t cvt2_e5m2(float lo, float hi) {
  uint16_t r;
  asm("cvt.rn.satfinite.e5m2x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ uint32_t cvt2_e2m1(float lo, float hi) {  // 8 bits
  uint32_t r;
  asm("{ .reg .b8 t; cvt.rn.satfinite.e2m1x2.f32 t, %1, %2; cvt.u32.u8 %0, t; }"
      : "=r"(r) : "f"(hi), "f"(lo));
  return r & 0xffu;
}
__device__ __forceinline__ uint32_t cvt2_e3m2(float lo, float hi) {  // one code per byte
  uint16_t r;
  asm("cvt.rn.satfinite.e3m2x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ uint32_t cvt2_e2m3(float lo, float hi) {
  uint16_t r;
  asm("cvt.rn.satfinite.e2m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
  return r;
}
// two codes (lo in the low byte / half) -> two floats
__device__ __forceinline__ float2 h2_to_f2(uint32_t h2) {
  return make_float2(__half2float(__ushort_as_half((unsigned short)(h2 & 0xffffu))),
                     __half2float(__ushort_as_half((unsigned short)(h2 >> 16))));
}
__device__ __forceinline__ float2 dec2_e4m3(uint32_t c16) {
  uint32_t h2;
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"((uint16_t)c16));
  return h2_to_f2(h2);
}
__device__ __forceinline__ float2 dec2_e5m2(uint32_t c16) {
  uint32_t h2;
  asm("cvt.rn.f16x2.e5m2x2 %0, %1;" : "=r"(h2) : "h"((uint16_t)c16));
  return h2_to_f2(h2);
}
__device__ __forceinline__ float2 dec2_e2m1(uint32_t c8) {
  uint32_t h2;
  asm("{ .reg .b8 t; cvt.u8.u32 t, %1; cvt.rn.f16x2.e2m1x2 %0, t; }" : "=r"(h2) : "r"(c8));
  return h2_to_f2(h2);
}
__device__ __forceinline__ float2 dec2_e3m2(uint32_t c16) {
  uint32_t h2;
  asm("cvt.rn.f16x2.e3m2x2 %0, %1;" : "=r"(h2) : "h"((uint16_t)c16));
  return h2_to_f2(h2);
}
__device__ __forceinline__ float2 dec2_e2m3(uint32_t c16) {
  uint32_t h2;
  asm("cvt.rn.f16x2.e2m3x2 %0, %1;" : "=r"(h2) : "h"((uint16_t)c16));
  return h2_to_f2(h2);
}

// ------------------------------------------------------- per-kind traits
template <int K> struct Fmt;
template <> struct Fmt<KIND_F32> { static constexpr int bits = 32, k = 1; };
template <> struct Fmt<KIND_F16> { static constexpr int bits = 16, k = 2; };
template <> struct Fmt<KIND_BF16> { static constexpr int bits = 16, k = 2; };
template <> struct Fmt<KIND_E4M3> { static constexpr int bits = 8, k = 4; };
template <> struct Fmt<KIND_E5M2> { static constexpr int bits = 8, k = 4; };
template <> struct Fmt<KIND_E2M1> { static constexpr int bits = 4, k = 8; };
template <> struct Fmt<KIND_E3M2> { static constexpr int bits = 6, k = 5; };
template <> struct Fmt<KIND_E2M3> { static constexpr int bits = 6, k = 5; };

// codes of two values, low value in the low `bits`
template <int K>
__device__ __forceinline__ uint32_t enc_pair(float lo, float hi, const DevFmt& f) {
  uint32_t r;
  constexpr int b = Fmt<K>::bits;
  if (K == KIND_F16) r = cvt2_f16(lo, hi);
  else if (K == KIND_BF16) r = cvt2_bf16(lo, hi);
  else if (K == KIND_E4M3) r = cvt2_e4m3(lo, hi);
  else if (K == KIND_E5M2) r = cvt2_e5m2(lo, hi);
  else if (K == KIND_E2M1) r = cvt2_e2m1(lo, hi);
  else if (K == KIND_E3M2) r = cvt2_e3m2(lo, hi);
  else r = cvt2_e2m3(lo, hi);
  uint32_t c0, c1;
  if (K == KIND_E3M2 || K == KIND_E2M3) {  // one 6-bit code per byte
    c0 = r & 0x3fu;
    c1 = (r >> 8) & 0x3fu;
  } else {
    c0 = r & ((1u << b) - 1u);
    c1 = (r >> b) & ((1u << b) - 1u);
  }
  if (lo != lo) c0 = f.nan_code;
  if (hi != hi) c1 = f.nan_code;
  return c0 | (c1 << b);
}

template <int K>
__device__ __forceinline__ float2 dec_pair(uint32_t c0, uint32_t c1) {  // codes, low bits
  constexpr int b = Fmt<K>::bits;
  if (K == KIND_F16)
    return make_float2(__half2float(__ushort_as_half((unsigned short)c0)),
                       __half2float(__ushort_as_half((unsigned short)c1)));
  if (K == KIND_BF16) return make_float2(__uint_as_float(c0 << 16), __uint_as_float(c1 << 16));
  if (K == KIND_E4M3) return dec2_e4m3(c0 | (c1 << 8));
  if (K == KIND_E5M2) return dec2_e5m2(c0 | (c1 << 8));
  if (K == KIND_E2M1) return dec2_e2m1(c0 | (c1 << 4));
  if (K == KIND_E3M2) return dec2_e3m2(c0 | (c1 << 8));
  (void)b;
  return dec2_e2m3(c0 | (c1 << 8));
}

// ---------------------------------------------------------- single values
__device__ __forceinline__ uint32_t encode(float x, const DevFmt& f) {
  switch (f.kind) {
    case KIND_F32: return __float_as_uint(x);
    case KIND_F16: return enc_pair<KIND_F16>(x, 0.f, f) & 0xffffu;
    case KIND_BF16: return enc_pair<KIND_BF16>(x, 0.f, f) & 0xffffu;
    case KIND_E4M3: return enc_pair<KIND_E4M3>(x, 0.f, f) & 0xffu;
    case KIND_E5M2: return enc_pair<KIND_E5M2>(x, 0.f, f) & 0xffu;
    case KIND_E2M1: return enc_pair<KIND_E2M1>(x, 0.f, f) & 0xfu;
    case KIND_E3M2: return enc_pair<KIND_E3M2>(x, 0.f, f) & 0x3fu;
    case KIND_E2M3: return enc_pair<KIND_E2M3>(x, 0.f, f) & 0x3fu;
    default: return encode_generic(x, f);
  }
}

__device__ __forceinline__ float decode(uint32_t c, const DevFmt& f) {
  switch (f.kind) {
    case KIND_F32: return __uint_as_float(c);
    case KIND_F16: return dec_pair<KIND_F16>(c, 0u).x;
    case KIND_BF16: return dec_pair<KIND_BF16>(c, 0u).x;
    case KIND_E4M3: return dec_pair<KIND_E4M3>(c, 0u).x;
    case KIND_E5M2: return dec_pair<KIND_E5M2>(c, 0u).x;
    case KIND_E2M1: return dec_pair<KIND_E2M1>(c, 0u).x;
    case KIND_E3M2: return dec_pair<KIND_E3M2>(c, 0u).x;
    case KIND_E2M3: return dec_pair<KIND_E2M3>(c, 0u).x;
    default: return decode_generic(c, f);
  }
}

// Value j (0 <= j < k) of a packed word (runtime format).
__device__ __forceinline__ float unpack_slot(uint32_t word, int j, const DevFmt& f) {
  return decode((word >> (f.bits * j)) & f.mask, f);
}

// ------------------------------------------------------------- words
// Compile-time kind dispatch: dispatch_kind(kind, body) calls
// body(KindC<K>{}) for the tensor's kind, so a whole loop runs with k, the
// bit offsets and the conversion fixed at compile time.
template <int K> struct KindC { static constexpr int value = K; };

template <typename Body>
__device__ __forceinline__ void dispatch_kind(int kind, Body&& body) {
  switch (kind) {
    case KIND_F32: body(KindC<KIND_F32>{}); break;
    case KIND_F16: body(KindC<KIND_F16>{}); break;
    case KIND_BF16: body(KindC<KIND_BF16>{}); break;
    case KIND_E4M3: body(KindC<KIND_E4M3>{}); break;
    case KIND_E5M2: body(KindC<KIND_E5M2>{}); break;
    case KIND_E2M1: body(KindC<KIND_E2M1>{}); break;
    case KIND_E3M2: body(KindC<KIND_E3M2>{}); break;
    case KIND_E2M3: body(KindC<KIND_E2M3>{}); break;
    default: body(KindC<KIND_GENERIC>{}); break;
  }
}

// Values per word of a kind (runtime for the generic kind).
template <int K>
__device__ __forceinline__ int per_word(const DevFmt& f) {
  if constexpr (K == KIND_GENERIC) return f.k;
  else return Fmt<K>::k;
}

// Word w of a row: values w*k .. w*k+k-1 from get(i), i < n; unused slots 0.
template <int K, typename Get>
__device__ __forceinline__ uint32_t pack_word_t(int w, int n, const DevFmt& f, Get get) {
  if constexpr (K == KIND_F32) {
    return w < n ? __float_as_uint(get(w)) : 0u;
  } else if constexpr (K == KIND_GENERIC) {
    const int i0 = w * f.k;
    uint32_t word = 0u;
    for (int j = 0; j < f.k; ++j)
      if (i0 + j < n) word |= (encode_generic(get(i0 + j), f) & f.mask) << (f.bits * j);
    return word;
  } else {
    constexpr int b = Fmt<K>::bits, k = Fmt<K>::k;
    const int i0 = w * k;
    uint32_t word = 0u;
#pragma unroll
    for (int j = 0; j < k; j += 2) {
      const float lo = i0 + j < n ? get(i0 + j) : 0.f;
      const float hi = (j + 1 < k && i0 + j + 1 < n) ? get(i0 + j + 1) : 0.f;
      uint32_t pr = enc_pair<K>(lo, hi, f);
      if (j + 1 >= k) pr &= (1u << b) - 1u;
      word |= pr << (b * j);
    }
    return word;
  }
}

// put(i, value) for the values of word w that are < n.
template <int K, typename Put>
__device__ __forceinline__ void unpack_word_t(uint32_t word, int w, int n, const DevFmt& f, Put put) {
  if constexpr (K == KIND_F32) {
    if (w < n) put(w, __uint_as_float(word));
  } else if constexpr (K == KIND_GENERIC) {
    const int i0 = w * f.k;
    for (int j = 0; j < f.k; ++j)
      if (i0 + j < n) put(i0 + j, decode_generic((word >> (f.bits * j)) & f.mask, f));
  } else {
    constexpr int b = Fmt<K>::bits, k = Fmt<K>::k;
    constexpr uint32_t m = (1u << b) - 1u;
    const int i0 = w * k;
#pragma unroll
    for (int j = 0; j < k; j += 2) {
      const float2 x = dec_pair<K>((word >> (b * j)) & m,
                                   j + 1 < k ? (word >> (b * (j + 1))) & m : 0u);
      if (i0 + j < n) put(i0 + j, x.x);
      if (j + 1 < k && i0 + j + 1 < n) put(i0 + j + 1, x.y);
    }
  }
}

// ------------------------------------------------------------- chunks
// A chunk is 16 bytes = words 4c .. 4c+3 of a row = values 4kc .. 4kc+4k-1.
// pack_chunk: value i comes from get(i) for i < n; slots past n are zero.
template <int K, typename Get>
__device__ __forceinline__ uint4 pack_chunk(int c, int n, const DevFmt& f, Get get) {
  uint32_t w[4];
  if constexpr (K == KIND_F32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = 4 * c + q;
      w[q] = i < n ? __float_as_uint(get(i)) : 0u;
    }
  } else {
    constexpr int b = Fmt<K>::bits, k = Fmt<K>::k;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i0 = (4 * c + q) * k;
      uint32_t word = 0u;
#pragma unroll
      for (int j = 0; j < k; j += 2) {
        const float lo = i0 + j < n ? get(i0 + j) : 0.f;
        const float hi = (j + 1 < k && i0 + j + 1 < n) ? get(i0 + j + 1) : 0.f;
        uint32_t pr = enc_pair<K>(lo, hi, f);
        if (j + 1 >= k) pr &= (1u << b) - 1u;  // odd k: the last pair has one value
        word |= pr << (b * j);
      }
      w[q] = word;
    }
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

template <typename Get>
__device__ __forceinline__ uint4 pack_chunk_generic(int c, int n, const DevFmt& f, Get get) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i0 = (4 * c + q) * f.k;
    uint32_t word = 0u;
    for (int j = 0; j < f.k; ++j)
      if (i0 + j < n) word |= (encode_generic(get(i0 + j), f) & f.mask) << (f.bits * j);
    w[q] = word;
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

template <typename Get>
__device__ __forceinline__ uint4 pack_chunk_dyn(int c, int n, const DevFmt& f, Get get) {
  switch (f.kind) {
    case KIND_F32: return pack_chunk<KIND_F32>(c, n, f, get);
    case KIND_F16: return pack_chunk<KIND_F16>(c, n, f, get);
    case KIND_BF16: return pack_chunk<KIND_BF16>(c, n, f, get);
    case KIND_E4M3: return pack_chunk<KIND_E4M3>(c, n, f, get);
    case KIND_E5M2: return pack_chunk<KIND_E5M2>(c, n, f, get);
    case KIND_E2M1: return pack_chunk<KIND_E2M1>(c, n, f, get);
    case KIND_E3M2: return pack_chunk<KIND_E3M2>(c, n, f, get);
    case KIND_E2M3: return pack_chunk<KIND_E2M3>(c, n, f, get);
    default: return pack_chunk_generic(c, n, f, get);
  }
}

// unpack_chunk: put(i, value) for every value i < n of chunk c.
template <int K, typename Put>
__device__ __forceinline__ void unpack_chunk(uint4 v, int c, int n, const DevFmt& f, Put put) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  if constexpr (K == KIND_F32) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (4 * c + q < n) put(4 * c + q, __uint_as_float(w[q]));
  } else {
    constexpr int b = Fmt<K>::bits, k = Fmt<K>::k;
    constexpr uint32_t m = (1u << b) - 1u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i0 = (4 * c + q) * k;
#pragma unroll
      for (int j = 0; j < k; j += 2) {
        const float2 x = dec_pair<K>((w[q] >> (b * j)) & m,
                                     j + 1 < k ? (w[q] >> (b * (j + 1))) & m : 0u);
        if (i0 + j < n) put(i0 + j, x.x);
        if (j + 1 < k && i0 + j + 1 < n) put(i0 + j + 1, x.y);
      }
    }
  }
  (void)f;
}

template <typename Put>
__device__ __forceinline__ void unpack_chunk_generic(uint4 v, int c, int n, const DevFmt& f, Put put) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i0 = (4 * c + q) * f.k;
    for (int j = 0; j < f.k; ++j)
      if (i0 + j < n) put(i0 + j, decode_generic((w[q] >> (f.bits * j)) & f.mask, f));
  }
}

template <typename Put>
__device__ __forceinline__ void unpack_chunk_dyn(uint4 v, int c, int n, const DevFmt& f, Put put) {
  switch (f.kind) {
    case KIND_F32: unpack_chunk<KIND_F32>(v, c, n, f, put); break;
    case KIND_F16: unpack_chunk<KIND_F16>(v, c, n, f, put); break;
    case KIND_BF16: unpack_chunk<KIND_BF16>(v, c, n, f, put); break;
    case KIND_E4M3: unpack_chunk<KIND_E4M3>(v, c, n, f, put); break;
    case KIND_E5M2: unpack_chunk<KIND_E5M2>(v, c, n, f, put); break;
    case KIND_E2M1: unpack_chunk<KIND_E2M1>(v, c, n, f, put); break;
    case KIND_E3M2: unpack_chunk<KIND_E3M2>(v, c, n, f, put); break;
    case KIND_E2M3: unpack_chunk<KIND_E2M3>(v, c, n, f, put); break;
    default: unpack_chunk_generic(v, c, n, f, put);
  }
}

// Value i of a row (runtime format) from a word fetcher word(w).
template <int K, typename Word>
__device__ __forceinline__ float row_value(int i, const DevFmt& f, Word word) {
  if constexpr (K == KIND_F32) {
    return __uint_as_float(word(i));
  } else if constexpr (K == KIND_GENERIC) {
    const int w = i / f.k;
    return decode_generic((word(w) >> (f.bits * (i - w * f.k))) & f.mask, f);
  } else {
    constexpr int b = Fmt<K>::bits, k = Fmt<K>::k;
    const int w = i / k;
    return dec_pair<K>((word(w) >> (b * (i - w * k))) & ((1u << b) - 1u), 0u).x;
  }
}

}  // namespace vapr
