// Exact fixed-point sums of block values, shared by the frame reduction and the tensor-core
// kernel's fused reduction of a batched tick (so that both give the same FP64 features).
//
// Every block value the analyzer writes is 0 or a float in [1, 2^30), a multiple of 2^-23, so
// v * 2^23 is an integer below 2^53 (fixed23).  Sums of those integers are kept in 128 bits and
// rounded to FP64 once (to_double).
#pragma once

#include <cstdint>

#include "vca_internal.h"

namespace vca {
namespace {

// v * 2^23 truncated to an integer, for a block value v in [0, 2^30): the significand shifted by
// the unbiased exponent.  Every value the analyzer writes is 0 or at least 1 (a multiple of
// 2^-23), so nothing is truncated for them.  Values outside [0, 2^30) -- negative (also -0.0),
// NaN, infinite or 2^30 and above -- and values below 2^-24 count as 0.
__device__ __forceinline__ unsigned long long fixed23(float v) {
  const uint32_t b = __float_as_uint(v);
  const int e = (int)(b >> 23) - 127;  // 128 for NaN and infinities
  if ((b >> 31) != 0u || e >= 30 || e < -24) return 0ull;
  const unsigned long long m = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
  return e >= 0 ? m << e : m >> -e;
}

struct U128 {
  unsigned long long lo, hi;
};

__device__ __forceinline__ void add_to(U128& a, unsigned long long v) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(a.lo), "+l"(a.hi) : "l"(v));
}

__device__ __forceinline__ void add_to(U128& a, const U128& b) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(b.lo), "l"(b.hi));
}

// The 128-bit integer as the nearest double (ties to even): its leading 64 bits, with a sticky
// bit for anything below them, rounded once by the 64-bit conversion and scaled.
__device__ __forceinline__ double to_double(const U128& a) {
  if (a.hi == 0ull) return __ull2double_rn(a.lo);
  const int lz = __clzll((long long)a.hi);
  const unsigned long long top = lz ? (a.hi << lz) | (a.lo >> (64 - lz)) : a.hi;
  const unsigned long long rest = lz ? a.lo << lz : a.lo;
  const double scale = __hiloint2double((1023 + 64 - lz) << 20, 0);  // 2^(64 - lz)
  return __ull2double_rn(top | (rest != 0ull ? 1ull : 0ull)) * scale;
}

// Sums of a frame reduction: the six block-value rows (BlockValueRow order), then |dH_Y|.
constexpr int kSums = kRedSums;

// Feature of sum r with exact total t (in units of 2^-23): its slot in a feature row (E_Y, h, L_Y,
// E_U, E_V, L_U, L_V) and its value, the total rounded once to FP64 and divided by its norm (C w^2
// for the luma energies, C Nv Nh for the chroma energies, C for the brightness sums).
__device__ __forceinline__ double feature_of_sum(int r, const U128& t, double C, double normY, double normC,
                                                 int& slot) {
  const double total = to_double(t) * 1.1920928955078125e-07;  // x 2^-23 (exact)
  double norm;
  switch (r) {
    case ROW_H_Y: slot = 0; norm = normY; break;
    case ROW_L_Y: slot = 2; norm = C; break;
    case ROW_H_U: slot = 3; norm = normC; break;
    case ROW_L_U: slot = 5; norm = C; break;
    case ROW_H_V: slot = 4; norm = normC; break;
    case ROW_L_V: slot = 6; norm = C; break;
    default: slot = 1; norm = normY; break;  // the |dH_Y| sum: h
  }
  return total / norm;
}

}  // namespace
}  // namespace vca
