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
//      sin, cos (x >= 0): Cody & Waite reduction x = j pi/2 + r, j =
//           rint(x 2/pi), with pi/2 split into three parts of at most 12
//           significant bits each but the last, r = ((x - j P1) - j P2) -
//           j P3; with z = r^2, sin r = r + r (z (-1/3! + z (1/5! + z (-1/7!
//           + z 1/9!)))) and cos r = 1 + z (-1/2! + z (1/4! + z (-1/6! +
//           z (1/8! - z 1/10!)))) (binary32-rounded coefficients); the
//           quadrant j mod 4 picks (s, c), (c, -s), (-s, -c) or (-c, s).
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

// pi/2 = kPio2a + kPio2b + kPio2c (12, 12 and 24 significant bits)
constexpr float kTwoOverPi = 0x1.45f306p-1f;
constexpr float kPio2a = 0x1.92p+0f;
constexpr float kPio2b = 0x1.fb4p-12f;
constexpr float kPio2c = 0x1.4442d2p-24f;
// 1/k! with alternating signs, binary32-rounded
constexpr float kInv3 = -0x1.555556p-3f, kInv5 = 0x1.111112p-7f, kInv7 = -0x1.a01a02p-13f,
                kInv9 = 0x1.71de3ap-19f;
constexpr float kInv2 = -0.5f, kInv4 = 0x1.555556p-5f, kInv6 = -0x1.6c16c2p-10f, kInv8 = 0x1.a01a02p-16f,
                kInv10 = -0x1.27e4fcp-22f;

UBS_HD void sincos32(float x, float* s_out, float* c_out) {
  const float j = rintf(x * kTwoOverPi);
  const float r = ((x - j * kPio2a) - j * kPio2b) - j * kPio2c;
  const float z = r * r;
  const float s = r + r * (z * (kInv3 + z * (kInv5 + z * (kInv7 + z * kInv9))));
  const float c = 1.0f + z * (kInv2 + z * (kInv4 + z * (kInv6 + z * (kInv8 + z * kInv10))));
  const int q = ((int)j) & 3;
  *s_out = q == 0 ? s : q == 1 ? c : q == 2 ? -s : -c;
  *c_out = q == 0 ? c : q == 1 ? -s : q == 2 ? -c : s;
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
