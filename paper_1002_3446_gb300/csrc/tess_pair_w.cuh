// K2, tensor form (FP32, any n): the O(n^3) rewrite of the four-vertex sum
// (Sec. 3, W-tensor equations) in the lane-pair layout.  Every set S keeps,
// besides its current J[S], the antisymmetric tensor
//   T[S]^{mu nu} = sum over the splits (L', R') of S of
//                  J[L']^mu J[R']^nu - J[R']^mu J[L']^nu,
// and the four-vertex part of a current is then a sum over splits only:
//   sum over the triples (A, B, C) of X of {J_A, J_B, J_C}
//     = sum over the splits (L, R) of X of T[R].J[L] - T[L].J[R],
// (T.J)^mu = T^{mu nu} J_nu, metric (+,-,-,-).  The three-vertex bracket is
// evaluated as written in the recursion.  Per split 434 FLOPs and no triple
// loop; the table holds 80 B per set (J: two float4, T's six complex
// components: three float4) against 40 B for the split-sum form, so fewer
// events fit per SM.  Two lanes per event share the sets of one length, as
// in bg_pair_kernel.
#pragma once
#include "tess_pair.cuh"

namespace tess {

template <int L, int NEV>
struct PairWSmem {
  static constexpr int T = L * (L + 1) / 2;
  static constexpr size_t j_off = 0;                                             // float4 [2 T][NEV]
  static constexpr size_t t_off = j_off + (size_t)2 * T * NEV * sizeof(float4);  // float4 [3 T][NEV]
  static constexpr size_t p_off = t_off + (size_t)3 * T * NEV * sizeof(float4);  // float4 [L + 1][NEV]
  static constexpr size_t e_off = p_off + (size_t)(L + 1) * NEV * sizeof(float4);  // float4 [2][NEV]
  static constexpr size_t bytes = e_off + (size_t)2 * NEV * sizeof(float4);
};

// The six independent components of an antisymmetric complex tensor, in the
// order 01, 02, 03, 12, 13, 23.
struct AT6 {
  Cx<float> c[6];
};

__device__ __forceinline__ Cx<float> cmul(const Cx<float> &a, const Cx<float> &b) {
  return cx<float>(fmaf(a.re, b.re, -a.im * b.im), fmaf(a.re, b.im, a.im * b.re));
}

// t += l^mu r^nu - r^mu l^nu for mu < nu
__device__ __forceinline__ void at6_add_wedge(AT6 &t, const CV4<float> &l, const CV4<float> &r) {
  int q = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
#pragma unroll
    for (int nu = mu + 1; nu < 4; ++nu, ++q) {
      const Cx<float> x = cmul(l.c[mu], r.c[nu]), y = cmul(r.c[mu], l.c[nu]);
      t.c[q].re += x.re - y.re;
      t.c[q].im += x.im - y.im;
    }
}

// acc += s (T.J), (T.J)^mu = sum_nu T^{mu nu} eta_nu J^nu, s = +1 or -1
__device__ __forceinline__ void at6_apply(CV4<float> &acc, const AT6 &t, const CV4<float> &j, float s) {
  // index of T^{mu nu} (mu < nu) in the six-component order
  constexpr int idx[4][4] = {{-1, 0, 1, 2}, {0, -1, 3, 4}, {1, 3, -1, 5}, {2, 4, 5, -1}};
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    Cx<float> sum = cx<float>(0.f, 0.f);
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
      if (nu == mu) continue;
      const float sign = (mu < nu ? 1.f : -1.f) * (nu == 0 ? 1.f : -1.f);  // antisymmetry x metric
      const Cx<float> p = cmul(t.c[idx[mu][nu]], j.c[nu]);
      sum.re = fmaf(sign, p.re, sum.re);
      sum.im = fmaf(sign, p.im, sum.im);
    }
    acc.c[mu].re = fmaf(s, sum.re, acc.c[mu].re);
    acc.c[mu].im = fmaf(s, sum.im, acc.c[mu].im);
  }
}

template <int NEV>
__device__ __forceinline__ AT6 ld_at6(const float4 *T4, int X, int g) {
  const float4 a = T4[(3 * X) * NEV + g], b = T4[(3 * X + 1) * NEV + g], c = T4[(3 * X + 2) * NEV + g];
  AT6 t;
  t.c[0] = cx<float>(a.x, a.y);
  t.c[1] = cx<float>(a.z, a.w);
  t.c[2] = cx<float>(b.x, b.y);
  t.c[3] = cx<float>(b.z, b.w);
  t.c[4] = cx<float>(c.x, c.y);
  t.c[5] = cx<float>(c.z, c.w);
  return t;
}

template <int NEV>
__device__ __forceinline__ void st_at6(float4 *T4, int X, int g, const AT6 &t) {
  T4[(3 * X) * NEV + g] = make_float4(t.c[0].re, t.c[0].im, t.c[1].re, t.c[1].im);
  T4[(3 * X + 1) * NEV + g] = make_float4(t.c[2].re, t.c[2].im, t.c[3].re, t.c[3].im);
  T4[(3 * X + 2) * NEV + g] = make_float4(t.c[4].re, t.c[4].im, t.c[5].re, t.c[5].im);
}

// Over the splits i = a + i0, a + i0 + di, ... of X = [a..b]: the
// three-vertex brackets plus T[R].J[L] - T[L].J[R] into acc, and (when
// want_t) the wedge products J[L] ^ J[R] into t.
template <int L, int NEV>
__device__ __forceinline__ void pair_sums_w(const PairView<NEV> &V, const float4 *T4, int a, int b, int i0, int di,
                                            bool want_t, CV4<float> &acc, AT6 &t) {
  const RV4<float> Pa = V.P(a), Pb = V.P(b + 1);
  acc = cv_zero<float>();
#pragma unroll
  for (int q = 0; q < 6; ++q) t.c[q] = cx<float>(0.f, 0.f);
#pragma unroll 1
  for (int i = a + i0; i < b; i += di) {
    const int l = pair_tri<L>(a, i), r = pair_tri<L>(i + 1, b);
    const CV4<float> Jl = V.J(l), Jr = V.J(r);
    const RV4<float> Pi = V.P(i + 1);
    const RV4<float> Kl = rsub(Pi, Pa), Kr = rsub(Pb, Pi);
    const Cx<float> d = mdot(Jl, Jr);
    const Cx<float> jlkr = mdot(Jl, Kr);
    const Cx<float> krjl = mdot(Jr, Kl);
    axpy(acc, cx<float>(2.f * jlkr.re, 2.f * jlkr.im), Jr);
    axpy(acc, cx<float>(-2.f * krjl.re, -2.f * krjl.im), Jl);
    axpy(acc, d, rsub(Kl, Kr));
    if (i + 1 < b) at6_apply(acc, ld_at6<NEV>(T4, r, V.g), Jl, 1.f);   // T[R].J[L] (zero for one leg)
    if (i > a) at6_apply(acc, ld_at6<NEV>(T4, l, V.g), Jr, -1.f);     // -T[L].J[R]
    if (want_t) at6_add_wedge(t, Jl, Jr);
  }
}

template <int N, int NEV>
__global__ void __launch_bounds__(2 * NEV) bg_pair_w_kernel(ChunkParams C, ChunkBuf<float> B, double *partials) {
  constexpr int L = N - 1, NB = 2 * NEV;
  using PS = PairWSmem<L, NEV>;
  extern __shared__ __align__(16) char smem_pw[];
  PairView<NEV> V;
  V.J4 = (float4 *)(smem_pw + PS::j_off);
  V.P4 = (float4 *)(smem_pw + PS::p_off);
  V.E4 = (float4 *)(smem_pw + PS::e_off);
  V.S2 = nullptr;
  float4 *T4 = (float4 *)(smem_pw + PS::t_off);
  const int lane = threadIdx.x / NEV;
  V.g = threadIdx.x % NEV;
  const int nb2 = C.P.hist_bins > 0 ? C.P.hist_bins + 2 : 0;
  EpiSmem<NB> ES(smem_pw + PS::bytes, nb2);
  epi_init(ES, nb2);
  Accum<NB> A;
  const int count = k2_count(C, B);
  const int ntiles = (count + NEV - 1) / NEV;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile * NEV + V.g;
    const bool live = j < count;
    const int e = live ? k2_col(C, B, j) : 0;
    if (live) {
      if (lane == 0) {  // momenta -> prefix sums, and eps of position 0
        RV4<float> p = {{0.f, 0.f, 0.f, 0.f}};
        V.P4[V.g] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
        for (int a = 0; a < L; ++a) {
          RV4<float> k;
          load_k(B.in + (size_t)InRows<L>::k(a) * B.cap + e, (size_t)B.cap, k);
          p = radd(p, k);
          V.P4[(a + 1) * NEV + V.g] = make_float4(p.v[0], p.v[1], p.v[2], p.v[3]);
        }
        CV4<float> e0;
        load_eps(B.in + (size_t)InRows<L>::eps0 * B.cap + e, (size_t)B.cap, e0);
        V.E4[V.g] = make_float4(e0.c[0].re, e0.c[0].im, e0.c[1].re, e0.c[1].im);
        V.E4[NEV + V.g] = make_float4(e0.c[2].re, e0.c[2].im, e0.c[3].re, e0.c[3].im);
      } else {  // single-leg currents (their tensors are never read)
#pragma unroll 1
        for (int a = 0; a < L; ++a) {
          CV4<float> ea;
          load_eps(B.in + (size_t)InRows<L>::eps(a) * B.cap + e, (size_t)B.cap, ea);
          V.setJ(pair_tri<L>(a, a), ea);
        }
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int len = 2; len < L; ++len) {
      if (live) {
#pragma unroll 1
        for (int a = lane; a + len - 1 < L; a += 2) {
          const int b = a + len - 1;
          CV4<float> acc;
          AT6 t;
          pair_sums_w<L, NEV>(V, T4, a, b, 0, 1, true, acc, t);
          const RV4<float> K = rsub(V.P(b + 1), V.P(a));
          const float inv = 1.f / mdot(K, K);
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            acc.c[m].re *= inv;
            acc.c[m].im *= inv;
          }
          const int X = pair_tri<L>(a, b);
          V.setJ(X, acc);
          st_at6<NEV>(T4, X, V.g, t);
        }
      }
      __syncthreads();
    }
    // top current [0..L-1] (numerator only, no tensor): splits shared
    const int top = pair_tri<L>(0, L - 1);
    CV4<float> part = cv_zero<float>();
    if (live) {
      AT6 t;
      pair_sums_w<L, NEV>(V, T4, 0, L - 1, lane, 2, false, part, t);
      if (lane == 1) V.setJ(top, part);
    }
    __syncthreads();
    double w = 0.0;
    int bin = -1;
    if (live && lane == 0) {
      const CV4<float> other = V.J(top);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        part.c[m].re += other.c[m].re;
        part.c[m].im += other.c[m].im;
      }
      const float4 u = V.E4[V.g], v = V.E4[NEV + V.g];
      CV4<float> e0;
      e0.c[0] = cx<float>(u.x, u.y);
      e0.c[1] = cx<float>(u.z, u.w);
      e0.c[2] = cx<float>(v.x, v.y);
      e0.c[3] = cx<float>(v.z, v.w);
      finish_event<NB, float>(C, B, e, amp2_of(mdot(e0, part)), A, w, bin);
    }
    epi_tile<NB>(ES, nb2, w, bin);
    __syncthreads();  // the table is refilled by the next tile
  }
  epi_flush<NB>(ES, nb2, A, partials, C.P.hist_bins);
}

}  // namespace tess
