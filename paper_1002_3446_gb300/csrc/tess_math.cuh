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
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;  // one wide multiply each
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
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

// Philox4x32-10 with the ten round keys given (rk[2r], rk[2r+1] = key of
// round r); the same function of (counter, key) as philox4x32_10.  Kernels
// take the round keys from their launch constants, so the key schedule is
// not recomputed per block.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t *rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1],
                   (uint32_t)p0);
  }
  return c;
}

// Round keys of philox4x32_10 for key (seed_lo, seed_hi).
__host__ __device__ inline void philox_round_keys(uint64_t seed, uint32_t *rk) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk[2 * r] = k0;
    rk[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// The 52-bit integer k of uniform u = (k + 1/2) 2^-52 from its two words.
__device__ __forceinline__ uint64_t unit_bits(uint32_t a, uint32_t b) {
  return ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
}

// floor(u * c) exactly as the double-precision product rounds it (single
// rounding to 53 bits, ties to even), in integer arithmetic: u * c =
// (2k+1) c 2^-53 and scaling by 2^-53 is exact.  c <= 2^10.
__device__ __forceinline__ int floor_unit_times(uint64_t k, uint32_t c) {
  uint64_t X = (2 * k + 1) * (uint64_t)c;
  const int e = 63 - __clzll((long long)X);
  if (e >= 53) {
    const int s = e - 52;
    const uint64_t mask = (1ull << s) - 1, half = 1ull << (s - 1);
    uint64_t q = X >> s;
    const uint64_t rem = X & mask;
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    X = q << s;
  }
  return (int)(X >> 53);
}

// A uniform in single precision from the same two words: hi 2^-26 +
// (lo + 1/2) 2^-52 with one rounding when hi < 2^24 (u < 1/4, exactly
// float(u)); within 2 ulp of float(u) above.  Strictly inside (0, 1).
__device__ __forceinline__ float unit_f32(uint32_t a, uint32_t b) {
  const float hi = (float)(a >> 6), lo = (float)(b >> 6);
  const float u = fmaf(lo + 0.5f, 0x1p-52f, hi * 0x1p-26f);
  return fminf(u, 0x1.fffffep-1f);
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

namespace tess {

// ---------------------------------------------------------------------------
// Double-float ("two-float") arithmetic: a value is hi + lo with |lo| <=
// ulp(hi)/2, about 47-48 significant bits, evaluated on the FP32 pipe.  Built
// from the error-free transformations two-sum (Knuth) and two-product (one
// FMA); reciprocal and reciprocal square root take one Newton step in
// double-float from the FP32 estimate.  Rounding a normalised value to FP32
// gives hi.
// ---------------------------------------------------------------------------
struct DS {
  float hi, lo;
};

__device__ __forceinline__ DS ds(float x) { return DS{x, 0.f}; }

__device__ __forceinline__ DS ds_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return DS{s, b - (s - a)};
}

__device__ __forceinline__ DS ds_add(DS a, DS b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  return ds_fast_two_sum(s, e + a.lo + b.lo);
}

__device__ __forceinline__ DS ds_add(DS a, float b) {
  const float s = a.hi + b;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b - bb);
  return ds_fast_two_sum(s, e + a.lo);
}

__device__ __forceinline__ DS ds_neg(DS a) { return DS{-a.hi, -a.lo}; }

__device__ __forceinline__ DS ds_sub(DS a, DS b) { return ds_add(a, ds_neg(b)); }

__device__ __forceinline__ DS ds_mul(DS a, DS b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return ds_fast_two_sum(p, e);
}

__device__ __forceinline__ DS ds_mul(DS a, float b) {
  const float p = a.hi * b;
  const float e = fmaf(a.lo, b, fmaf(a.hi, b, -p));
  return ds_fast_two_sum(p, e);
}

// 1/a: y0 = rcp(hi), y = y0 + y0 (1 - a y0)
__device__ __forceinline__ DS ds_rcp(DS a) {
  const float y0 = 1.f / a.hi;
  const DS r = ds_add(ds(1.f), ds_neg(ds_mul(a, y0)));  // 1 - a y0, small
  return ds_add(ds(y0), r.hi * y0);
}

// 1/sqrt(a): y0 = rsqrt(hi), y = y0 + y0 (1 - a y0^2) / 2
__device__ __forceinline__ DS ds_rsqrt(DS a) {
  const float y0 = rsqrtf(a.hi);
  const DS t = ds_mul(ds_mul(a, y0), y0);  // a y0^2, close to 1
  const DS r = ds_add(ds(1.f), ds_neg(t));
  return ds_add(ds(y0), 0.5f * y0 * r.hi);
}

__device__ __forceinline__ DS ds_sqrt(DS a) { return ds_mul(a, ds_rsqrt(a)); }

// Unnormalised pairs (h, l) for chains whose result is needed only rounded to
// FP32: error-free products and sums as above, without renormalising between
// steps (|l| stays within a few ulp of h), rounded once at the end.
__device__ __forceinline__ float two_sum(float a, float b, float &t) {  // s + t = a + b exactly
  const float s = a + b;
  const float bb = s - a;
  t = (a - (s - bb)) + (b - bb);
  return s;
}

// (ah, al) (bh, bl) as a pair
__device__ __forceinline__ float pair_mul(float ah, float al, float bh, float bl, float &l) {
  const float h = ah * bh;
  l = fmaf(ah, bl, fmaf(al, bh, fmaf(ah, bh, -h)));
  return h;
}

// (ah, al) b as a pair
__device__ __forceinline__ float pair_mul(float ah, float al, float b, float &l) {
  const float h = ah * b;
  l = fmaf(al, b, fmaf(ah, b, -h));
  return h;
}

// FP32 rounding of (ah, al) (bh, bl)
__device__ __forceinline__ float pair_mul_round(float ah, float al, float bh, float bl) {
  float l;
  const float h = pair_mul(ah, al, bh, bl, l);
  return h + l;
}

}  // namespace tess
