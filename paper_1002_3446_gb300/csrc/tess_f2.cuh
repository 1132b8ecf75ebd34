// Packed FP32 pairs on sm_100-class GPUs: one 64-bit register pair holds two
// floats and fma.rn.f32x2 / mul / add / sub operate on both halves with one
// instruction.  The FMA pipe still does 128 lanes of FP32 work per SM per
// clock, but a packed instruction takes one issue slot for two lanes' work,
// which leaves the other slots to loads, addresses and control (measured:
// packed FMAs interleaved 1:1 with integer instructions keep the FMA pipe at
// its peak).
//
// Four-vectors are packed by component pairs, (x0, x1) and (x2, x3).  With
// the metric (+,-,-,-) folded into one operand -- its "signed" form (x0, -x1,
// -x2, -x3) -- a Minkowski dot is the plain sum of the four products.
#pragma once
#include <cstdint>

#include "tess_math.cuh"

namespace tess {

struct P2 {
  unsigned long long v;
};

__device__ __forceinline__ P2 p2(float lo, float hi) {
  P2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ P2 pbc(float x) { return p2(x, x); }
__device__ __forceinline__ float plo(P2 a) {
  float x, y;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.v));
  return x;
}
__device__ __forceinline__ float phi(P2 a) {
  float x, y;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.v));
  return y;
}
__device__ __forceinline__ P2 pfma(P2 a, P2 b, P2 c) {
  P2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}
__device__ __forceinline__ P2 pmul(P2 a, P2 b) {
  P2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ P2 padd(P2 a, P2 b) {
  P2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ P2 psub(P2 a, P2 b) {
  P2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ P2 pzero() { return p2(0.f, 0.f); }

// Real four-vector (x0, x1), (x2, x3) and complex four-vector (real and
// imaginary parts packed the same way).
struct PV4 {
  P2 a, b;
};
struct PC4 {
  PV4 re, im;
};

__device__ __forceinline__ PV4 pv4(float4 v) { return PV4{p2(v.x, v.y), p2(v.z, v.w)}; }
__device__ __forceinline__ float4 f4(PV4 v) { return make_float4(plo(v.a), phi(v.a), plo(v.b), phi(v.b)); }
__device__ __forceinline__ PV4 pv_zero() { return PV4{pzero(), pzero()}; }
__device__ __forceinline__ PC4 pc_zero() { return PC4{pv_zero(), pv_zero()}; }
__device__ __forceinline__ PV4 pv_add(PV4 x, PV4 y) { return PV4{padd(x.a, y.a), padd(x.b, y.b)}; }

// The signed form of a raised vector (metric applied): (x0, -x1), (-x2, -x3).
__device__ __forceinline__ PV4 pv_signed(PV4 x) {
  return PV4{pmul(x.a, p2(1.f, -1.f)), pmul(x.b, pbc(-1.f))};
}
__device__ __forceinline__ PC4 pc_signed(PC4 x) { return PC4{pv_signed(x.re), pv_signed(x.im)}; }

// Component products summed over the four components, as one pair (the
// caller adds its two halves): x . y with one of them signed.
__device__ __forceinline__ P2 pdot_pair(PV4 x, PV4 y) { return pfma(x.b, y.b, pmul(x.a, y.a)); }

// Complex dot of a signed and a raised complex four-vector as the two pairs
// whose halves add to the real and the imaginary part:
// re = sum (ar br - ai bi), im = sum (ar bi + ai br).
__device__ __forceinline__ void pcdot_pairs(const PC4 &s, const PC4 &r, P2 &pre, P2 &pim) {
  pre = psub(pdot_pair(s.re, r.re), pdot_pair(s.im, r.im));
  pim = pfma(s.im.b, r.re.b, pfma(s.im.a, r.re.a, pdot_pair(s.re, r.im)));
}

// acc += c v for a complex scalar c given as broadcast pairs (c.re, c.re),
// (c.im, c.im), (-c.im, -c.im) and a complex four-vector v.
__device__ __forceinline__ void pc_axpy(PC4 &acc, P2 cre, P2 cim, P2 ncim, const PC4 &v) {
  acc.re.a = pfma(ncim, v.im.a, pfma(cre, v.re.a, acc.re.a));
  acc.re.b = pfma(ncim, v.im.b, pfma(cre, v.re.b, acc.re.b));
  acc.im.a = pfma(cim, v.re.a, pfma(cre, v.im.a, acc.im.a));
  acc.im.b = pfma(cim, v.re.b, pfma(cre, v.im.b, acc.im.b));
}

// acc += c k for a complex scalar c (broadcast pairs) and a real four-vector k.
__device__ __forceinline__ void pr_axpy(PC4 &acc, P2 cre, P2 cim, const PV4 &k) {
  acc.re.a = pfma(cre, k.a, acc.re.a);
  acc.re.b = pfma(cre, k.b, acc.re.b);
  acc.im.a = pfma(cim, k.a, acc.im.a);
  acc.im.b = pfma(cim, k.b, acc.im.b);
}

}  // namespace tess
