// K2, lane-pair form (FP32, any n): two threads per event with the event's
// Berends-Giele table in shared memory.
//
// Thread t of a block of 2 NEV threads serves event slot g = t % NEV as lane
// j = t / NEV, so the two lanes of an event sit in different warps and every
// warp-wide access reads one table entry for 32 consecutive events
// (conflict-free 16-byte loads).  The table holds, per event, the currents
// J[a..b] (complex four-vectors as two float4), the split sums S[a..b] (Sec.
// 3 recursion, reorganised four-vertex sum as in tess_bg.cuh) and the prefix
// momenta P[i] = k_0 + ... + k_{i-1}, so K[a..b] = P[b+1] - P[a] needs no
// table of its own.  Currents of one length are shared between the lanes
// (lane j builds the sets starting at a = j, j + 2, ...), with one block
// barrier per length; the top current's splits and four-vertex triples are
// split between the two lanes by parity of the left part's end and the two
// partial sums are added in a fixed order.  All loops are runtime loops, so
// the code stays small for every n (the unrolled row form outgrows the
// instruction cache at n >= 10), and the table costs 44 B/current/event.
#pragma once
#include "tess_pipeline.cuh"

namespace tess {

template <int L>
__host__ __device__ constexpr int pair_tri(int a, int b) {
  return a * L - (a * (a - 1)) / 2 + (b - a);
}

template <int L, int NEV>
struct PairSmem {
  static constexpr int T = L * (L + 1) / 2;
  static constexpr size_t j_off = 0;                                           // float4 [2 T][NEV]
  static constexpr size_t p_off = j_off + (size_t)2 * T * NEV * sizeof(float4);  // float4 [L + 1][NEV]
  static constexpr size_t e_off = p_off + (size_t)(L + 1) * NEV * sizeof(float4);  // float4 [2][NEV]
  static constexpr size_t s_off = e_off + (size_t)2 * NEV * sizeof(float4);      // float2 [T][NEV]
  static constexpr size_t bytes = s_off + (size_t)T * NEV * sizeof(float2);
};

template <int NEV>
struct PairView {
  float4 *J4, *P4, *E4;
  float2 *S2;
  int g;
  __device__ __forceinline__ CV4<float> J(int X) const {
    const float4 u = J4[(2 * X) * NEV + g], v = J4[(2 * X + 1) * NEV + g];
    CV4<float> r;
    r.c[0] = cx<float>(u.x, u.y);
    r.c[1] = cx<float>(u.z, u.w);
    r.c[2] = cx<float>(v.x, v.y);
    r.c[3] = cx<float>(v.z, v.w);
    return r;
  }
  __device__ __forceinline__ void setJ(int X, const CV4<float> &r) const {
    J4[(2 * X) * NEV + g] = make_float4(r.c[0].re, r.c[0].im, r.c[1].re, r.c[1].im);
    J4[(2 * X + 1) * NEV + g] = make_float4(r.c[2].re, r.c[2].im, r.c[3].re, r.c[3].im);
  }
  __device__ __forceinline__ RV4<float> P(int i) const {
    const float4 p = P4[i * NEV + g];
    RV4<float> r = {{p.x, p.y, p.z, p.w}};
    return r;
  }
  __device__ __forceinline__ Cx<float> S(int X) const {
    const float2 s = S2[X * NEV + g];
    return cx<float>(s.x, s.y);
  }
};

// Sum over the splits i = a + i0, a + i0 + di, ... of X = [a..b] of the
// three-vertex brackets (with the -S terms of the reorganised four-vertex
// sum), plus 2 x the triples whose left part ends at one of those i; s
// receives the split sum of J_l.J_r over the same splits.  Table entries are
// reached through pointers advanced incrementally (the triangular index of
// [a..i] grows by 1 with i, that of [i+1..b] by L - i - 2, ...), so the
// loops carry no index arithmetic beyond a few adds.
template <int L, int NEV>
__device__ __forceinline__ void pair_sums(const PairView<NEV> &V, int a, int b, int i0, int di, CV4<float> &acc,
                                          Cx<float> &s) {
  constexpr int JS = 2 * NEV;  // float4 stride between table entries of one event
  const RV4<float> Pa = V.P(a), Pb = V.P(b + 1);
  CV4<float> acc1 = cv_zero<float>(), acc2 = cv_zero<float>(), trs = cv_zero<float>();
  s = cx<float>(0.f, 0.f);
  auto ldJ = [](const float4 *q) {
    const float4 u = q[0], v = q[NEV];
    CV4<float> r;
    r.c[0] = cx<float>(u.x, u.y);
    r.c[1] = cx<float>(u.z, u.w);
    r.c[2] = cx<float>(v.x, v.y);
    r.c[3] = cx<float>(v.z, v.w);
    return r;
  };
  const float4 *Jg = V.J4 + V.g;
  const float2 *Sg = V.S2 + V.g;
  const float4 *Pg = V.P4 + V.g;
  int i = a + i0;
  int xl = pair_tri<L>(a, i), xr = pair_tri<L>(i + 1, b);
#pragma unroll 1
  for (; i < b; i += di) {
    const CV4<float> Jl = ldJ(Jg + xl * JS), Jr = ldJ(Jg + xr * JS);
    const float4 p4 = Pg[(i + 1) * NEV];
    const RV4<float> Pi = {{p4.x, p4.y, p4.z, p4.w}};
    const RV4<float> Kl = rsub(Pi, Pa), Kr = rsub(Pb, Pi);
    const Cx<float> d = mdot(Jl, Jr);
    const Cx<float> jlkr = mdot(Jl, Kr);
    const Cx<float> krjl = mdot(Jr, Kl);
    const float2 sl = Sg[xl * NEV], sr = Sg[xr * NEV];  // zero for single legs
    const Cx<float> cr = cx<float>(fmaf(2.f, jlkr.re, -sl.x), fmaf(2.f, jlkr.im, -sl.y));
    const Cx<float> cl = cx<float>(fmaf(-2.f, krjl.re, -sr.x), fmaf(-2.f, krjl.im, -sr.y));
    axpy(acc1, cr, Jr);
    axpy(acc2, cl, Jl);
    axpy(acc1, d, rsub(Kl, Kr));
    s.re += d.re;
    s.im += d.im;
    // triples (J[a..i] . J[c+1..b]) J[i+1..c], i < c < b: [c+1..b] starts at
    // [i+2..b] (index xr + L - i - 2) and steps by L - c - 2; [i+1..c] starts
    // at [i+1..i+1] (index xr - (b - i - 1)) and steps by 1
    int xc = xr + (L - i - 2), xm = xr - (b - i - 1);
#pragma unroll 1
    for (int c = i + 1; c < b; ++c) {
      axpy(trs, mdot(Jl, ldJ(Jg + xc * JS)), ldJ(Jg + xm * JS));
      xc += L - c - 2;
      xm += 1;
    }
    // next split: [a..i+di] is di entries on; [i+di+1..b] is sum_{t=1..di} (L - i - t - 1) on
#pragma unroll 1
    for (int t = 1; t <= di; ++t) xr += L - i - t - 1;
    xl += di;
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    acc.c[m].re = fmaf(2.f, trs.c[m].re, acc1.c[m].re + acc2.c[m].re);
    acc.c[m].im = fmaf(2.f, trs.c[m].im, acc1.c[m].im + acc2.c[m].im);
  }
}

template <int N, int NEV>
__global__ void __launch_bounds__(2 * NEV) bg_pair_kernel(ChunkParams C, ChunkBuf<float> B, double *partials) {
  constexpr int L = N - 1, NB = 2 * NEV;
  using PS = PairSmem<L, NEV>;
  extern __shared__ __align__(16) char smem_pair[];
  PairView<NEV> V;
  V.J4 = (float4 *)(smem_pair + PS::j_off);
  V.P4 = (float4 *)(smem_pair + PS::p_off);
  V.E4 = (float4 *)(smem_pair + PS::e_off);
  V.S2 = (float2 *)(smem_pair + PS::s_off);
  const int lane = threadIdx.x / NEV;
  V.g = threadIdx.x % NEV;
  const int nb2 = C.P.hist_bins > 0 ? C.P.hist_bins + 2 : 0;
  EpiSmem<NB> ES(smem_pair + PS::bytes, nb2);
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
      } else {  // eps of positions 1..L: the single-leg currents
#pragma unroll 1
        for (int a = 0; a < L; ++a) {
          CV4<float> ea;
          load_eps(B.in + (size_t)InRows<L>::eps(a) * B.cap + e, (size_t)B.cap, ea);
          const int X = pair_tri<L>(a, a);
          V.setJ(X, ea);
          V.S2[X * NEV + V.g] = make_float2(0.f, 0.f);
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
          Cx<float> s;
          pair_sums<L, NEV>(V, a, b, 0, 1, acc, s);
          const RV4<float> K = rsub(V.P(b + 1), V.P(a));
          const float inv = 1.f / mdot(K, K);
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            acc.c[m].re *= inv;
            acc.c[m].im *= inv;
          }
          const int X = pair_tri<L>(a, b);
          V.setJ(X, acc);
          V.S2[X * NEV + V.g] = make_float2(s.re, s.im);
        }
      }
      __syncthreads();
    }
    // top current [0..L-1] (numerator only): splits and triples shared
    const int top = pair_tri<L>(0, L - 1);
    CV4<float> part = cv_zero<float>();
    if (live) {
      Cx<float> s;
      pair_sums<L, NEV>(V, 0, L - 1, lane, 2, part, s);
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
