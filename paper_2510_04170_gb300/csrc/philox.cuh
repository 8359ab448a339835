// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications with the Weyl key schedule.  Device-side
// implementation used for the features (Sec. 2.2) and the sketches (Sec. 4.1).
#pragma once
#include <stdint.h>

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// 53-bit uniform on [0,1) from two words: ((a >> 5) * 2^26 + (b >> 6)) * 2^-53.
__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b) {
  const uint64_t v = ((uint64_t)(a >> 5) << 26) + (uint64_t)(b >> 6);
  return (double)v * 0x1p-53;
}

// Nearest bfloat16 (ties to even) of a double in the bf16 normal range,
// returned as the 16 stored bits.
__device__ __forceinline__ uint16_t bf16_bits_rne(double x) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  b = (b + 0x0FFFFFFFFFFFull + ((b >> 45) & 1ull)) & ~((1ull << 45) - 1ull);
  const double r = __longlong_as_double((long long)b);
  const float f = (float)r;  // exact: r has 8 significant bits
  return (uint16_t)(__float_as_uint(f) >> 16);
}

__device__ __forceinline__ double bf16_bits_to_double(uint16_t h) {
  return (double)__uint_as_float(((uint32_t)h) << 16);
}

// Gaussian sketch entries rounded to the grid 2^-4: (rint(16 z0), rint(16 z1))
// for the Box-Muller pair z0 = r cos(t), z1 = r sin(t), r = sqrt(-2 log(1-u1)),
// t = 2 pi u2, identical to evaluating Box-Muller in FP64 and rounding.
// The pair is evaluated in FP32 (w = 1 - u1 is formed exactly in FP64 first);
// with r >= 0.01 the FP32 error of 16 z is below 2.5e-4 (logf 1 ulp, sinf/cosf
// 2 ulp, sqrtf correctly rounded, inputs rounded once), so an FP32 result more
// than 1e-3 away from a rounding tie decides the same integer; only the rest
// (about 0.2%) is recomputed in FP64.  For r < 0.01, |16 z| < 0.17 and the
// integer is 0 either way.
__device__ __forceinline__ void gauss_pair_q16(const uint32_t c[4], float* d0, float* d1) {
  const double u1 = uniform53(c[0], c[1]);
  const double u2 = uniform53(c[2], c[3]);
  const double w = 1.0 - u1;  // exact
  const float rf = sqrtf(-2.0f * logf((float)w));
  float sf, cf;
  sincosf(6.2831853f * (float)u2, &sf, &cf);
  const float t0 = 16.0f * (rf * cf), t1 = 16.0f * (rf * sf);
  const float q0 = rintf(t0), q1 = rintf(t1);
  if (rf < 0.01f) {
    *d0 = 0.0f;
    *d1 = 0.0f;
    return;
  }
  const bool safe = fabsf(fabsf(t0 - q0) - 0.5f) > 1e-3f && fabsf(fabsf(t1 - q1) - 0.5f) > 1e-3f;
  if (safe) {
    *d0 = q0;
    *d1 = q1;
    return;
  }
  const double rad = sqrt(-2.0 * log(w));
  const double th = 6.283185307179586 * u2;
  *d0 = (float)rint(16.0 * (rad * cos(th)));
  *d1 = (float)rint(16.0 * (rad * sin(th)));
}
