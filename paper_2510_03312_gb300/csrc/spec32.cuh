// spec32.cuh -- float32 rule set for every float->integer decision of the
// rasterizer (culling, depth keys, tile rectangles) and the values that feed
// them.
//
// Rules (the translation unit that includes this header is compiled with
// --fmad=false -prec-div=true -prec-sqrt=true -ftz=false):
//  * each + - * is one IEEE binary32 operation rounded to nearest-even; no
//    contraction into FMA; expressions are evaluated exactly as written,
//    sums left to right;
//  * division and square root are correctly rounded;
//  * exp and log below are this project's own functions:
//      exp: Cody & Waite (1980) reduction x = k ln2 + r with ln2 split into a
//           16-significant-bit head and a rounded tail, the degree-7 Taylor
//           polynomial of e^r in Horner form with binary32-rounded 1/k!
//           coefficients, and the scale 2^k assembled from exponent bits;
//           x is clamped to [-87, 88] and x < -87 returns 0;
//      log: x = m 2^e with m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1),
//           log m = 2 atanh(s) summed as s (2 + z(2/3 + z(2/5 + z(2/7 +
//           z(2/9 + z 2/11))))) with z = s^2; log x = e ln2_hi + (poly +
//           e ln2_lo); x <= 0 (or NaN) returns -inf.
#pragma once

#ifndef UBS_HD
#define UBS_HD __host__ __device__ __forceinline__
#endif

#include <math.h>
#include <stdint.h>
#include <string.h>

namespace ubs {
namespace spec {

UBS_HD float bits_to_float(int32_t i) {
#ifdef __CUDA_ARCH__
  return __int_as_float(i);
#else
  float f;
  memcpy(&f, &i, 4);
  return f;
#endif
}

UBS_HD int32_t float_to_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_int(f);
#else
  int32_t i;
  memcpy(&i, &f, 4);
  return i;
#endif
}

// exact binary32 constants (1/k! and 2/(2k+1) are the binary32 roundings)
constexpr float kLog2e = 0x1.715476p+0f;   // 1/ln 2
constexpr float kLn2 = 0x1.62e430p-1f;     // ln 2
constexpr float kLn2Hi = 0x1.62e4p-1f;     // 16 significant bits
constexpr float kLn2Lo = 0x1.7f7d1cp-20f;  // ln 2 - kLn2Hi
constexpr float kSqrt2 = 0x1.6a09e6p+0f;
constexpr float kMargR = 0x1.004p+0f;      // 1 + 2^-10
constexpr float kMargA = 0x1p-6f;          // 2^-6 px

UBS_HD float exp32(float x) {
  const bool under = x < -87.0f;
  float xc = fminf(fmaxf(x, -87.0f), 88.0f);
  float k = rintf(xc * kLog2e);
  float r = (xc - k * kLn2Hi) - k * kLn2Lo;
  float p = 0x1.a01a02p-13f;
  p = p * r + 0x1.6c16c2p-10f;
  p = p * r + 0x1.111112p-7f;
  p = p * r + 0x1.555556p-5f;
  p = p * r + 0x1.555556p-3f;
  p = p * r + 0.5f;
  p = p * r + 1.0f;
  p = p * r + 1.0f;
  float scale = bits_to_float(((int32_t)k + 127) << 23);
  float out = p * scale;
  return under ? 0.0f : out;
}

UBS_HD float log32(float x) {
  if (!(x > 0.0f)) return -INFINITY;
  int32_t bits = float_to_bits(x);
  int32_t e = ((bits >> 23) & 0xFF) - 127;
  float m = bits_to_float((bits & 0x7FFFFF) | 0x3F800000);
  if (m > kSqrt2) {
    m = m * 0.5f;
    e = e + 1;
  }
  float s = (m - 1.0f) / (m + 1.0f);
  float z = s * s;
  float p = 0x1.745d18p-3f;
  p = p * z + 0x1.c71c72p-3f;
  p = p * z + 0x1.24924ap-2f;
  p = p * z + 0x1.99999ap-2f;
  p = p * z + 0x1.555556p-1f;
  p = p * z + 2.0f;
  float poly = s * p;
  float ef = (float)e;
  return ef * kLn2Hi + (poly + ef * kLn2Lo);
}

}  // namespace spec
}  // namespace ubs
