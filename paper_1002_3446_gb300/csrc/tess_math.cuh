// Device primitives: counter-based random numbers and complex Minkowski
// four-vector algebra, templated on the arithmetic type (float / double).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tess {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32 -> 64-bit products (multipliers 0xD2511F53, 0xCD9E8D57) with the
// high halves xored into the other words; the two key words advance by the
// Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// 52 random bits (26 from each word) -> (k + 1/2) 2^-52, exact in double and
// strictly inside (0, 1).
__device__ __forceinline__ double unit_from_words(uint32_t a, uint32_t b) {
  const double hi = (double)(a >> 6), lo = (double)(b >> 6);
  return (hi * 67108864.0 + lo + 0.5) * 0x1p-52;
}

// Uniforms number 2*blk and 2*blk+1 of event `ev` in stream `seed`: one
// Philox block with counter (ev_lo, ev_hi, blk, 0) and key (seed_lo, seed_hi).
__device__ __forceinline__ double2 uniform_pair(uint64_t seed, uint64_t ev, uint32_t blk) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)ev, (uint32_t)(ev >> 32), blk, 0u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  return make_double2(unit_from_words(w.x, w.y), unit_from_words(w.z, w.w));
}

// Single uniform j of an event (used for scattered draws).
__device__ __forceinline__ double uniform_at(uint64_t seed, uint64_t ev, uint32_t j) {
  const double2 p = uniform_pair(seed, ev, j >> 1);
  return (j & 1u) ? p.y : p.x;
}

// ---------------------------------------------------------------------------
// Complex numbers and complex / real four-vectors, metric (+,-,-,-).
// ---------------------------------------------------------------------------
template <typename R>
struct Cx {
  R re, im;
};
template <typename R>
struct CV4 {
  Cx<R> c[4];
};
template <typename R>
struct RV4 {
  R v[4];
};

template <typename R>
__device__ __forceinline__ Cx<R> cx(R re, R im) {
  Cx<R> z;
  z.re = re;
  z.im = im;
  return z;
}

template <typename R>
__device__ __forceinline__ CV4<R> cv_zero() {
  CV4<R> z;
#pragma unroll
  for (int m = 0; m < 4; ++m) z.c[m] = cx<R>(R(0), R(0));
  return z;
}

// a.b = a0 b0 - a1 b1 - a2 b2 - a3 b3, complex x complex (no conjugation)
template <typename R>
__device__ __forceinline__ Cx<R> mdot(const CV4<R> &a, const CV4<R> &b) {
  R re = a.c[0].re * b.c[0].re;
  R im = a.c[0].re * b.c[0].im;
  re = fma(-a.c[0].im, b.c[0].im, re);
  im = fma(a.c[0].im, b.c[0].re, im);
#pragma unroll
  for (int m = 1; m < 4; ++m) {
    re = fma(-a.c[m].re, b.c[m].re, re);
    re = fma(a.c[m].im, b.c[m].im, re);
    im = fma(-a.c[m].re, b.c[m].im, im);
    im = fma(-a.c[m].im, b.c[m].re, im);
  }
  return cx<R>(re, im);
}

// complex x real
template <typename R>
__device__ __forceinline__ Cx<R> mdot(const CV4<R> &a, const RV4<R> &k) {
  R re = a.c[0].re * k.v[0];
  R im = a.c[0].im * k.v[0];
#pragma unroll
  for (int m = 1; m < 4; ++m) {
    re = fma(-a.c[m].re, k.v[m], re);
    im = fma(-a.c[m].im, k.v[m], im);
  }
  return cx<R>(re, im);
}

template <typename R>
__device__ __forceinline__ R mdot(const RV4<R> &a, const RV4<R> &b) {
  R s = a.v[0] * b.v[0];
#pragma unroll
  for (int m = 1; m < 4; ++m) s = fma(-a.v[m], b.v[m], s);
  return s;
}

// acc += s * v  (complex scalar, complex vector)
template <typename R>
__device__ __forceinline__ void axpy(CV4<R> &acc, const Cx<R> &s, const CV4<R> &v) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    acc.c[m].re = fma(s.re, v.c[m].re, acc.c[m].re);
    acc.c[m].re = fma(-s.im, v.c[m].im, acc.c[m].re);
    acc.c[m].im = fma(s.re, v.c[m].im, acc.c[m].im);
    acc.c[m].im = fma(s.im, v.c[m].re, acc.c[m].im);
  }
}

// acc += s * k  (complex scalar, real vector)
template <typename R>
__device__ __forceinline__ void axpy(CV4<R> &acc, const Cx<R> &s, const RV4<R> &k) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    acc.c[m].re = fma(s.re, k.v[m], acc.c[m].re);
    acc.c[m].im = fma(s.im, k.v[m], acc.c[m].im);
  }
}

template <typename R>
__device__ __forceinline__ RV4<R> rsub(const RV4<R> &a, const RV4<R> &b) {
  RV4<R> d;
#pragma unroll
  for (int m = 0; m < 4; ++m) d.v[m] = a.v[m] - b.v[m];
  return d;
}

template <typename R>
__device__ __forceinline__ RV4<R> radd(const RV4<R> &a, const RV4<R> &b) {
  RV4<R> d;
#pragma unroll
  for (int m = 0; m < 4; ++m) d.v[m] = a.v[m] + b.v[m];
  return d;
}

}  // namespace tess
