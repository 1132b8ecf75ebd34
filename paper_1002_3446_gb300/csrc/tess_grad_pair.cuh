// Event weights and gradients, FP32 current forms: LN threads ("lanes") per
// event sharing the event's Berends-Giele table in shared memory (the layout
// of the lane-pair amplitude form, tess_pair.cuh), with the reverse sweep in
// pull form.
//
// The reverse sweep of the recursion (Sec. 3) is usually written in push
// form: each set X, in decreasing length, adds its contributions into the
// gradient accumulators of its parts (left, right, and the three parts of
// every four-vertex triple).  Lanes sharing an event would then write the
// same accumulators.  Here every set Y instead gathers its own gradient from
// all of its parents X (longer sets, already final): as the left part of X =
// [c..b], as the right part of X = [a..d], as the first or last part of a
// triple of those X, and as the middle part of a triple of X = [a..b] with
// a < c, d < b.  Every term is the same as in the push form; only who adds it
// changes, so the lanes split the sets of one length (lane j: sets starting
// at c = j, j + LN, ...) with no shared accumulator, one barrier per length.
// Momentum gradients go through the prefix sums P (K[c..d] = P[d+1] - P[c]):
// each set adds its K-gradient to P[d+1] and subtracts it from P[c] in the
// lane's own prefix-gradient row; the rows are added in a fixed order at the
// end.  Kinematics, polarisations and the output stage run thread per event
// in kernels of their own (the split pipeline below).
#pragma once
#include <algorithm>

#include "tess_grad.cuh"
#include "tess_grad_f32.cuh"
#include "tess_pair.cuh"

namespace tess {

template <int L, int NEV, int LN>
struct GradPairSmem {
  static constexpr int T = L * (L + 1) / 2;
  static constexpr size_t j_off = 0;                                               // float4 [2 T][NEV] currents
  static constexpr size_t g_off = j_off + (size_t)2 * T * NEV * sizeof(float4);    // float4 [2 T][NEV] adjoints
  static constexpr size_t p_off = g_off + (size_t)2 * T * NEV * sizeof(float4);    // float4 [L + 1][NEV]
  static constexpr size_t gp_off = p_off + (size_t)(L + 1) * NEV * sizeof(float4);  // float4 [LN][L + 1][NEV]
  static constexpr size_t e_off = gp_off + (size_t)LN * (L + 1) * NEV * sizeof(float4);  // float4 [2][NEV]
  static constexpr size_t s_off = e_off + (size_t)2 * NEV * sizeof(float4);        // float2 [T][NEV]
  static constexpr size_t gs_off = s_off + (size_t)T * NEV * sizeof(float2);       // float2 [T][NEV]
  static constexpr size_t bytes = gs_off + (size_t)T * NEV * sizeof(float2);
};

template <int NEV>
__device__ __forceinline__ CV4<float> ld_cv4(const float4 *base, int X, int g) {
  const float4 u = base[(2 * X) * NEV + g], v = base[(2 * X + 1) * NEV + g];
  CV4<float> r;
  r.c[0] = cx<float>(u.x, u.y);
  r.c[1] = cx<float>(u.z, u.w);
  r.c[2] = cx<float>(v.x, v.y);
  r.c[3] = cx<float>(v.z, v.w);
  return r;
}

template <int NEV>
__device__ __forceinline__ void st_cv4(float4 *base, int X, int g, const CV4<float> &r) {
  base[(2 * X) * NEV + g] = make_float4(r.c[0].re, r.c[0].im, r.c[1].re, r.c[1].im);
  base[(2 * X + 1) * NEV + g] = make_float4(r.c[2].re, r.c[2].im, r.c[3].re, r.c[3].im);
}

__device__ __forceinline__ RV4<float> rv4(const float4 p) {
  RV4<float> r = {{p.x, p.y, p.z, p.w}};
  return r;
}

// Minkowski metric sign of component m
__device__ __forceinline__ float eta_of(int m) { return m == 0 ? 1.f : -1.f; }

// sum_m conj(v^m) G^m
__device__ __forceinline__ Cx<float> conj_dot4(const CV4<float> &v, const CV4<float> &G) {
  float re = 0.f, im = 0.f;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    re = fmaf(v.c[m].re, G.c[m].re, fmaf(v.c[m].im, G.c[m].im, re));
    im = fmaf(v.c[m].re, G.c[m].im, fmaf(-v.c[m].im, G.c[m].re, im));
  }
  return cx<float>(re, im);
}

// g += conj(z) G
__device__ __forceinline__ void add_conj(CV4<float> &g, const Cx<float> &z, const CV4<float> &G) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    g.c[m].re = fmaf(z.re, G.c[m].re, fmaf(z.im, G.c[m].im, g.c[m].re));
    g.c[m].im = fmaf(z.re, G.c[m].im, fmaf(-z.im, G.c[m].re, g.c[m].im));
  }
}

// g^m += eta_m conj(v^m) z
__device__ __forceinline__ void add_eta_conj(CV4<float> &g, const CV4<float> &v, const Cx<float> &z) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const float e = eta_of(m);
    g.c[m].re = fmaf(e, v.c[m].re * z.re + v.c[m].im * z.im, g.c[m].re);
    g.c[m].im = fmaf(e, v.c[m].re * z.im - v.c[m].im * z.re, g.c[m].im);
  }
}

// Gathers the gradient of set Y = [c..d] (L legs, shared tables): GJ =
// df/dJ_Y, GS = df/dS_Y, GK = df/dK_Y, from all parents of Y.
template <int L, int NEV>
__device__ void pull_set(const float4 *J4, const float4 *G4, const float4 *P4, const float2 *S2, const float2 *gS2,
                         int g, int c, int d, CV4<float> &GJ, Cx<float> &GS, RV4<float> &GK) {
  GJ = cv_zero<float>();
  GS = cx<float>(0.f, 0.f);
  GK.v[0] = GK.v[1] = GK.v[2] = GK.v[3] = 0.f;
  const RV4<float> Pc = rv4(P4[c * NEV + g]), Pd1 = rv4(P4[(d + 1) * NEV + g]);
  const RV4<float> KY = rsub(Pd1, Pc);
  const CV4<float> JY = ld_cv4<NEV>(J4, pair_tri<L>(c, d), g);
  // Y as the left part of X = [c..b] (split after d), and as the first part
  // A of the triples of X with A = Y
#pragma unroll 1
  for (int b = d + 1; b < L; ++b) {
    const int X = pair_tri<L>(c, b), r = pair_tri<L>(d + 1, b);
    const CV4<float> GX = ld_cv4<NEV>(G4, X, g), Jr = ld_cv4<NEV>(J4, r, g);
    const float2 gsx = gS2[X * NEV + g], sr = S2[r * NEV + g];
    const RV4<float> Kr = rsub(rv4(P4[(b + 1) * NEV + g]), Pd1);
    const Cx<float> dd = mdot(JY, Jr);
    const Cx<float> krjl = mdot(Jr, KY);
    const Cx<float> cl = cx<float>(fmaf(-2.f, krjl.re, -sr.x), fmaf(-2.f, krjl.im, -sr.y));
    const Cx<float> gcr = conj_dot4(Jr, GX), gcl = conj_dot4(JY, GX);
    add_conj(GJ, cl, GX);
    Cx<float> gd = cx<float>(gsx.x, gsx.y);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float dk = KY.v[m] - Kr.v[m];
      gd.re = fmaf(dk, GX.c[m].re, gd.re);
      gd.im = fmaf(dk, GX.c[m].im, gd.im);
      GK.v[m] += dd.re * GX.c[m].re + dd.im * GX.c[m].im;  // Re(conj(d) G), as K_l
    }
    GS.re -= gcr.re;  // cr = 2 J_l.K_r - S_l
    GS.im -= gcr.im;
    const Cx<float> gjlkr = cx<float>(2.f * gcr.re, 2.f * gcr.im);
    const Cx<float> gkrjl = cx<float>(-2.f * gcl.re, -2.f * gcl.im);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float e = eta_of(m);
      GJ.c[m].re = fmaf(e * Kr.v[m], gjlkr.re, GJ.c[m].re);  // from J_l.K_r
      GJ.c[m].im = fmaf(e * Kr.v[m], gjlkr.im, GJ.c[m].im);
      GK.v[m] += e * (Jr.c[m].re * gkrjl.re + Jr.c[m].im * gkrjl.im);  // from J_r.K_l
    }
    add_eta_conj(GJ, Jr, gd);  // from d = J_l.J_r
    // triples (Y, [d+1..j], [j+1..b])
#pragma unroll 1
    for (int j = d + 1; j < b; ++j) {
      const CV4<float> JB = ld_cv4<NEV>(J4, pair_tri<L>(d + 1, j), g);
      const CV4<float> JC = ld_cv4<NEV>(J4, pair_tri<L>(j + 1, b), g);
      const Cx<float> gt0 = conj_dot4(JB, GX);
      add_eta_conj(GJ, JC, cx<float>(2.f * gt0.re, 2.f * gt0.im));
    }
  }
  // Y as the right part of X = [a..d] (split before c), and as the last part
  // C of the triples of X with C = Y
#pragma unroll 1
  for (int a = 0; a < c; ++a) {
    const int X = pair_tri<L>(a, d), l = pair_tri<L>(a, c - 1);
    const CV4<float> GX = ld_cv4<NEV>(G4, X, g), Jl = ld_cv4<NEV>(J4, l, g);
    const float2 gsx = gS2[X * NEV + g], sl = S2[l * NEV + g];
    const RV4<float> Kl = rsub(Pc, rv4(P4[a * NEV + g]));
    const Cx<float> dd = mdot(Jl, JY);
    const Cx<float> jlkr = mdot(Jl, KY);
    const Cx<float> cr = cx<float>(fmaf(2.f, jlkr.re, -sl.x), fmaf(2.f, jlkr.im, -sl.y));
    const Cx<float> gcr = conj_dot4(JY, GX), gcl = conj_dot4(Jl, GX);
    add_conj(GJ, cr, GX);
    Cx<float> gd = cx<float>(gsx.x, gsx.y);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float dk = Kl.v[m] - KY.v[m];
      gd.re = fmaf(dk, GX.c[m].re, gd.re);
      gd.im = fmaf(dk, GX.c[m].im, gd.im);
      GK.v[m] -= dd.re * GX.c[m].re + dd.im * GX.c[m].im;  // as K_r
    }
    GS.re -= gcl.re;  // cl = -2 J_r.K_l - S_r
    GS.im -= gcl.im;
    const Cx<float> gjlkr = cx<float>(2.f * gcr.re, 2.f * gcr.im);
    const Cx<float> gkrjl = cx<float>(-2.f * gcl.re, -2.f * gcl.im);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float e = eta_of(m);
      GK.v[m] += e * (Jl.c[m].re * gjlkr.re + Jl.c[m].im * gjlkr.im);  // from J_l.K_r
      GJ.c[m].re = fmaf(e * Kl.v[m], gkrjl.re, GJ.c[m].re);            // from J_r.K_l
      GJ.c[m].im = fmaf(e * Kl.v[m], gkrjl.im, GJ.c[m].im);
    }
    add_eta_conj(GJ, Jl, gd);
    // triples ([a..i], [i+1..c-1], Y)
#pragma unroll 1
    for (int i = a; i + 1 < c; ++i) {
      const CV4<float> JA = ld_cv4<NEV>(J4, pair_tri<L>(a, i), g);
      const CV4<float> JB = ld_cv4<NEV>(J4, pair_tri<L>(i + 1, c - 1), g);
      const Cx<float> gt0 = conj_dot4(JB, GX);
      add_eta_conj(GJ, JA, cx<float>(2.f * gt0.re, 2.f * gt0.im));
    }
    // Y as the middle part of X = [a..b], b > d: ([a..c-1], Y, [d+1..b])
#pragma unroll 1
    for (int b = d + 1; b < L; ++b) {
      const CV4<float> GXb = ld_cv4<NEV>(G4, pair_tri<L>(a, b), g);
      const Cx<float> t = mdot(Jl, ld_cv4<NEV>(J4, pair_tri<L>(d + 1, b), g));
      add_conj(GJ, cx<float>(2.f * t.re, 2.f * t.im), GXb);
    }
  }
}

// ---------------------------------------------------------------------------
// Split gradient pipeline (FP32 forms), per chunk of events:
//   G1 grad_in_kernel   thread per event: kinematics -> amplitude inputs
//                       (rows as InRows: momenta in the unit c and the five
//                       nonzero eps components per colour position)
//   G2 grad_amp_kernel  LN lanes per event: recursion, |m|^2 and the pull-form
//                       reverse sweep -> df/dk and df/deps per position
//   G3 grad_out_kernel  thread per event: kinematics again -> weights and
//                       gradients (grad_outputs_f32)
// so that the table-bound middle stage keeps all its lanes busy and the
// kinematics run at full occupancy.  The eps gradients keep the five
// components the polarisation adjoint reads (Re x, y, z; Im x, y).
// ---------------------------------------------------------------------------
struct GradChunk {
  float *in;  // [InRows<L>::rows][cap]
  float *gr;  // [InRows<L>::rows][cap]: df/dk (4) and df/deps (5) per position 1..L, then df/deps_0
  double *f;  // [cap] |m|^2
  int cap;
};

template <int N>
__global__ void __launch_bounds__(kBlock) grad_in_kernel(GradParams G, uint64_t first, int count, GradChunk B) {
  constexpr int M = N - 2, L = N - 1, NU = 2 + 4 * M;
  const int e = blockIdx.x * kBlock + threadIdx.x;
  if (e >= count) return;
  const uint64_t ev = first + (uint64_t)e;
  GradKinF<N> K;
  grad_kin_f32<N>(G.P, G.u + ev * NU, G.order + ev * N, K);
  const uint32_t hel = G.hel[ev];
  const size_t cap = (size_t)B.cap;
#pragma unroll
  for (int a = 0; a <= L; ++a) {
    RV4<float> k;
    CV4<float> eps;
    grad_amp_input_f32<N>(K, hel, a, k, eps);
    float *o = B.in + (size_t)(a == 0 ? InRows<L>::eps0 : InRows<L>::eps(a - 1)) * cap + e;
    if (a > 0) {
      float *ok = B.in + (size_t)InRows<L>::k(a - 1) * cap + e;
#pragma unroll
      for (int m = 0; m < 4; ++m) ok[m * cap] = k.v[m];
    }
    o[0] = eps.c[1].re;
    o[cap] = eps.c[2].re;
    o[2 * cap] = eps.c[3].re;
    o[3 * cap] = eps.c[1].im;
    o[4 * cap] = eps.c[2].im;
  }
}

template <int N, int NEV, int LN>
__global__ void __launch_bounds__(LN * NEV) grad_amp_kernel(int count, GradChunk B) {
  constexpr int L = N - 1;
  using PS = GradPairSmem<L, NEV, LN>;
  static_assert(LN >= 2 && LN - 1 <= PS::T, "the lanes' partial top sums use adjoint-table slots 0 .. LN-2");
  extern __shared__ __align__(16) char smem_ga[];
  float4 *J4 = (float4 *)(smem_ga + PS::j_off), *G4 = (float4 *)(smem_ga + PS::g_off);
  float4 *P4 = (float4 *)(smem_ga + PS::p_off), *E4 = (float4 *)(smem_ga + PS::e_off);
  float2 *S2 = (float2 *)(smem_ga + PS::s_off), *gS2 = (float2 *)(smem_ga + PS::gs_off);
  const int lane = threadIdx.x / NEV, g = threadIdx.x % NEV;
  float4 *GP4 = (float4 *)(smem_ga + PS::gp_off) + (size_t)lane * (L + 1) * NEV;
  const int e = blockIdx.x * NEV + g;
  const bool live = e < count;
  const size_t cap = (size_t)B.cap;
  if (live) {
    if (lane == 0) {  // momenta -> prefix sums, eps_0
      RV4<float> p = {{0.f, 0.f, 0.f, 0.f}};
      P4[g] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
      for (int a = 0; a < L; ++a) {
        RV4<float> k;
        load_k(B.in + (size_t)InRows<L>::k(a) * cap + e, cap, k);
        p = radd(p, k);
        P4[(a + 1) * NEV + g] = make_float4(p.v[0], p.v[1], p.v[2], p.v[3]);
      }
      CV4<float> e0;
      load_eps(B.in + (size_t)InRows<L>::eps0 * cap + e, cap, e0);
      E4[g] = make_float4(e0.c[0].re, e0.c[0].im, e0.c[1].re, e0.c[1].im);
      E4[NEV + g] = make_float4(e0.c[2].re, e0.c[2].im, e0.c[3].re, e0.c[3].im);
    } else {  // single-leg currents, shared by the other lanes
#pragma unroll 1
      for (int a = lane - 1; a < L; a += LN - 1) {
        CV4<float> ea;
        load_eps(B.in + (size_t)InRows<L>::eps(a) * cap + e, cap, ea);
        const int X = pair_tri<L>(a, a);
        st_cv4<NEV>(J4, X, g, ea);
        S2[X * NEV + g] = make_float2(0.f, 0.f);
      }
    }
  }
#pragma unroll 1
  for (int i = 0; i <= L; ++i) GP4[i * NEV + g] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  PairView<NEV> V;
  V.J4 = J4;
  V.P4 = P4;
  V.E4 = E4;
  V.S2 = S2;
  V.g = g;
#pragma unroll 1
  for (int len = 2; len < L; ++len) {
    if (live) {
#pragma unroll 1
      for (int a = lane; a + len - 1 < L; a += LN) {
        const int b = a + len - 1;
        CV4<float> acc;
        Cx<float> s;
        pair_sums<L, NEV>(V, a, b, 0, 1, acc, s);
        const RV4<float> Kab = rsub(V.P(b + 1), V.P(a));
        const float inv = 1.f / mdot(Kab, Kab);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          acc.c[m].re *= inv;
          acc.c[m].im *= inv;
        }
        const int X = pair_tri<L>(a, b);
        V.setJ(X, acc);
        S2[X * NEV + g] = make_float2(s.re, s.im);
      }
    }
    __syncthreads();
  }
  const int top = pair_tri<L>(0, L - 1);
  CV4<float> num = cv_zero<float>();
  if (live) {
    Cx<float> s;
    pair_sums<L, NEV>(V, 0, L - 1, lane, LN, num, s);
    // the adjoint table is free until the sweep: scratch for the partial sums
    if (lane > 0) st_cv4<NEV>(G4, lane - 1, g, num);
  }
  __syncthreads();
  if (live && lane == 0) {
#pragma unroll 1
    for (int j = 1; j < LN; ++j) {
      const CV4<float> other = ld_cv4<NEV>(G4, j - 1, g);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        num.c[m].re += other.c[m].re;
        num.c[m].im += other.c[m].im;
      }
    }
    const float4 u0 = E4[g], v0 = E4[NEV + g];
    CV4<float> e0;
    e0.c[0] = cx<float>(u0.x, u0.y);
    e0.c[1] = cx<float>(u0.z, u0.w);
    e0.c[2] = cx<float>(v0.x, v0.y);
    e0.c[3] = cx<float>(v0.z, v0.w);
    const Cx<float> mamp = mdot(e0, num);
    B.f[e] = (double)mamp.re * (double)mamp.re + (double)mamp.im * (double)mamp.im;
    const Cx<float> gm = cx<float>(2.f * mamp.re, 2.f * mamp.im);
    CV4<float> ge0 = cv_zero<float>(), gtop = cv_zero<float>();
    add_eta_conj(ge0, num, gm);
    add_eta_conj(gtop, e0, gm);
    st_cv4<NEV>(G4, top, g, gtop);
    gS2[top * NEV + g] = make_float2(0.f, 0.f);
    float *o = B.gr + (size_t)InRows<L>::eps0 * cap + e;
    o[0] = ge0.c[1].re;
    o[cap] = ge0.c[2].re;
    o[2 * cap] = ge0.c[3].re;
    o[3 * cap] = ge0.c[1].im;
    o[4 * cap] = ge0.c[2].im;
  }
  __syncthreads();
#pragma unroll 1
  for (int len = L - 1; len >= 1; --len) {
    if (live) {
#pragma unroll 1
      for (int c = lane; c + len - 1 < L; c += LN) {
        const int d = c + len - 1, Y = pair_tri<L>(c, d);
        CV4<float> GJ;
        Cx<float> GS;
        RV4<float> GK;
        pull_set<L, NEV>(J4, G4, P4, S2, gS2, g, c, d, GJ, GS, GK);
        if (len >= 2) {
          const RV4<float> KY = rsub(rv4(P4[(d + 1) * NEV + g]), rv4(P4[c * NEV + g]));
          const float inv = 1.f / mdot(KY, KY);
          const Cx<float> cj = conj_dot4(V.J(Y), GJ);
          const float gk2 = -2.f * cj.re * inv;
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            GK.v[m] = fmaf(gk2 * eta_of(m), KY.v[m], GK.v[m]);
            GJ.c[m].re *= inv;
            GJ.c[m].im *= inv;
          }
          gS2[Y * NEV + g] = make_float2(GS.re, GS.im);
          st_cv4<NEV>(G4, Y, g, GJ);
        } else {  // a single leg: df/deps of position c + 1
          float *o = B.gr + (size_t)InRows<L>::eps(c) * cap + e;
          o[0] = GJ.c[1].re;
          o[cap] = GJ.c[2].re;
          o[2 * cap] = GJ.c[3].re;
          o[3 * cap] = GJ.c[1].im;
          o[4 * cap] = GJ.c[2].im;
        }
        float4 hi = GP4[(d + 1) * NEV + g], lo = GP4[c * NEV + g];
        GP4[(d + 1) * NEV + g] = make_float4(hi.x + GK.v[0], hi.y + GK.v[1], hi.z + GK.v[2], hi.w + GK.v[3]);
        GP4[c * NEV + g] = make_float4(lo.x - GK.v[0], lo.y - GK.v[1], lo.z - GK.v[2], lo.w - GK.v[3]);
      }
    }
    __syncthreads();
  }
  if (live && lane == 0) {  // df/dk of BG leg t = sum over i > t of every lane's prefix rows
    const float4 *GPa = (const float4 *)(smem_ga + PS::gp_off);
    RV4<float> acc = {{0.f, 0.f, 0.f, 0.f}};
#pragma unroll 1
    for (int t = L - 1; t >= 0; --t) {
#pragma unroll
      for (int j = 0; j < LN; ++j) {
        const float4 a0 = GPa[((size_t)j * (L + 1) + t + 1) * NEV + g];
        acc.v[0] += a0.x;
        acc.v[1] += a0.y;
        acc.v[2] += a0.z;
        acc.v[3] += a0.w;
      }
      float *ok = B.gr + (size_t)InRows<L>::k(t) * cap + e;
#pragma unroll
      for (int m = 0; m < 4; ++m) ok[m * cap] = acc.v[m];
    }
  }
}

template <int N>
__global__ void __launch_bounds__(kBlock) grad_out_kernel(GradParams G, uint64_t first, int count, GradChunk B) {
  constexpr int M = N - 2, L = N - 1, NU = 2 + 4 * M;
  const int e = blockIdx.x * kBlock + threadIdx.x;
  if (e >= count) return;
  const uint64_t ev = first + (uint64_t)e;
  GradKinF<N> K;
  grad_kin_f32<N>(G.P, G.u + ev * NU, G.order + ev * N, K);
  const uint32_t hel = G.hel[ev];
  const size_t cap = (size_t)B.cap;
  grad_outputs_f32<N>(G, ev, K, hel, B.f[e], [&](int a, float(&g4)[4], CV4<float> &ge) {
    const float *o = B.gr + (size_t)(a == 0 ? InRows<L>::eps0 : InRows<L>::eps(a - 1)) * cap + e;
    ge = cv_zero<float>();
    ge.c[1].re = o[0];
    ge.c[2].re = o[cap];
    ge.c[3].re = o[2 * cap];
    ge.c[1].im = o[3 * cap];
    ge.c[2].im = o[4 * cap];
    if (a > 0) {
      const float *ok = B.gr + (size_t)InRows<L>::k(a - 1) * cap + e;
#pragma unroll
      for (int m = 0; m < 4; ++m) g4[m] = ok[m * cap];
    }
  });
}

// Lanes per event of the amplitude stage (measured at 2^20 events: n <= 5
// two, n = 6, 7 four, n >= 8 eight; more lanes split the sets of a length
// finer and raise the warps per SM for the same table).
template <int N>
__host__ __device__ constexpr int grad_lanes() {
  return N <= 5 ? 2 : (N <= 7 ? 4 : 8);
}

// Events per chunk of the split pipeline: two chunk buffers (input rows,
// gradient rows, |m|^2) of TESS_GRAD_CHUNK_MB each.  Measured (2^22 events,
// weights and all gradients): 32 MB chunks 6.5e8 / 2.48e8 events/s at
// n = 6 / 8, 256 MB 7.1e8 / 2.54e8, 1 GB 7.2e8 / 2.57e8 -- fewer launches,
// each with its ramp-up and tail (the buffers do not stay in L2 either way).
#ifndef TESS_GRAD_CHUNK_MB
#define TESS_GRAD_CHUNK_MB 1024
#endif
template <int N>
__host__ inline int grad_chunk_cap(uint64_t n_events, size_t chunk_bytes) {
  constexpr int L = N - 1;
  const size_t per_event = (size_t)2 * InRows<L>::rows * sizeof(float) + sizeof(double);
  const uint64_t bytes = chunk_bytes ? chunk_bytes : ((uint64_t)TESS_GRAD_CHUNK_MB << 20);
  const uint64_t target = std::min<uint64_t>(std::max<uint64_t>(128, (bytes / per_event) / 128 * 128),
                                             (uint64_t)INT32_MAX / 256 * 128);
  const uint64_t want = (std::max<uint64_t>(n_events, 1) + 127) / 128 * 128;
  return (int)std::min(target, want);
}

template <int N>
__host__ inline size_t grad_buffer_bytes(int cap) {
  constexpr int L = N - 1;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return 2 * al((size_t)InRows<L>::rows * cap * sizeof(float)) + al((size_t)cap * sizeof(double));
}

// One chunk buffer when a single chunk holds every event, else two.
template <int N>
__host__ inline size_t grad_workspace_bytes(uint64_t n_events, size_t chunk_bytes) {
  const int cap = grad_chunk_cap<N>(n_events, chunk_bytes);
  return (n_events > (uint64_t)cap ? 2 : 1) * grad_buffer_bytes<N>(cap);
}

// Gradient launch for n: FP64 one kernel, thread per event (push form, tables
// in local memory); FP32 forms the split pipeline over chunks of the
// caller's workspace (grad_workspace_bytes).  With two buffers and an aux
// stream, G3 of chunk c (aux stream) runs beside G1/G2 of chunk c+1 (caller's
// stream): the amplitude stage is held to few warps per SM by its shared
// tables, and the output stage fills the issue slots it leaves.  Buffer c % 2
// is rewritten by G2 of chunk c only after G3 of chunk c-2 has read it.
template <int N>
cudaError_t launch_grad_n(bool fp64, const GradParams &G, void *ws, cudaStream_t s, const GradStreams &gs) {
  if (fp64) {
    grad_kernel<N, double><<<(unsigned)((G.n_events + kBlock - 1) / kBlock), kBlock, 0, s>>>(G);
    return cudaGetLastError();
  }
  constexpr int L = N - 1, NEV = 32, LN = grad_lanes<N>();
  const int cap = grad_chunk_cap<N>(G.n_events, G.chunk_bytes);
  const size_t bb = grad_buffer_bytes<N>(cap);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int nbuf = G.n_events > (uint64_t)cap ? 2 : 1;
  GradChunk BB[2];
  for (int b = 0; b < nbuf; ++b) {
    char *base = (char *)ws + b * bb;
    BB[b].cap = cap;
    BB[b].in = (float *)base;
    BB[b].gr = (float *)(base + al((size_t)InRows<L>::rows * cap * sizeof(float)));
    BB[b].f = (double *)((char *)BB[b].gr + al((size_t)InRows<L>::rows * cap * sizeof(float)));
  }
  cudaError_t e = allow_max_smem((const void *)grad_amp_kernel<N, NEV, LN>);
  if (e != cudaSuccess) return e;
  const bool ovl = nbuf == 2 && gs.aux != nullptr;
  if (ovl && ((e = cudaEventRecord(gs.fork, s)) != cudaSuccess || (e = cudaStreamWaitEvent(gs.aux, gs.fork, 0)) != cudaSuccess))
    return e;
  int c = 0;
  for (uint64_t off = 0; off < G.n_events; off += (uint64_t)cap, ++c) {
    const int b = ovl ? (c & 1) : 0;
    const GradChunk &B = BB[b];
    const int count = (int)std::min<uint64_t>((uint64_t)cap, G.n_events - off);
    const unsigned tb = (unsigned)((count + kBlock - 1) / kBlock);
    grad_in_kernel<N><<<tb, kBlock, 0, s>>>(G, off, count, B);
    if (ovl && c >= 2 && (e = cudaStreamWaitEvent(s, gs.g3done[b], 0)) != cudaSuccess) return e;
    grad_amp_kernel<N, NEV, LN>
        <<<(unsigned)((count + NEV - 1) / NEV), LN * NEV, GradPairSmem<L, NEV, LN>::bytes, s>>>(count, B);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ovl) {
      if ((e = cudaEventRecord(gs.g2done[b], s)) != cudaSuccess || (e = cudaStreamWaitEvent(gs.aux, gs.g2done[b], 0)) != cudaSuccess)
        return e;
      grad_out_kernel<N><<<tb, kBlock, 0, gs.aux>>>(G, off, count, B);
      if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventRecord(gs.g3done[b], gs.aux)) != cudaSuccess) return e;
    } else {
      grad_out_kernel<N><<<tb, kBlock, 0, s>>>(G, off, count, B);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  if (ovl && ((e = cudaEventRecord(gs.join, gs.aux)) != cudaSuccess || (e = cudaStreamWaitEvent(s, gs.join, 0)) != cudaSuccess))
    return e;
  return cudaSuccess;
}

}  // namespace tess
