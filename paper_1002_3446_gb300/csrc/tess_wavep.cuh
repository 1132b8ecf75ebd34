// K2, wavefront row form in packed FP32 pairs (FP32, large n).  The schedule
// of tess_wave.cuh -- two lanes of a warp per event, each building one row of
// the current table, the two rows in step, a warp barrier between steps --
// with the arithmetic of every split and four-vertex triple in packed pairs
// (tess_f2.cuh), which halves the issue slots of the vertex algebra.
//
// Recursion (Sec. 3, Eq. (BG-recursion), four-vertex sum reorganised as in
// the other forms): for the set [a..b],
//   Num = sum_splits ( cr J_r + cl J_l + d (K_l - K_r) ) + 2 sum_triples (J_A.J_C) J_B,
//   cr = 2 J_l.K_r - S_l,  cl = -2 J_r.K_l - S_r,  d = J_l.J_r,  S = sum_splits d,
// and J[a..b] = Num / K[a..b]^2.  The table (shared memory) holds the
// currents raised, the lane's row (registers) holds them signed, so every
// dot product above is a plain sum of component products; contributions
// along a signed vector go to a second accumulator that is signed back once
// per set.  The table is laid out by set length (the sets of one length are
// consecutive), so the address of a triple's middle set is a compile-time
// offset from the row's start.
#pragma once
#include "tess_f2.cuh"
#include "tess_wave.cuh"

namespace tess {

// Current of set index t: raised real parts (x0..x3) in plane 2t, imaginary
// parts in plane 2t + 1 (event slot e of NE).
template <int NE>
__device__ __forceinline__ PC4 pld_cv(const float4 *J4, int t, int e) {
  return PC4{pv4(J4[(2 * t) * NE + e]), pv4(J4[(2 * t + 1) * NE + e])};
}

template <int NE>
__device__ __forceinline__ void pst_cv(float4 *J4, int t, int e, const PC4 &v) {
  J4[(2 * t) * NE + e] = f4(v.re);
  J4[(2 * t + 1) * NE + e] = f4(v.im);
}

template <int NE>
__device__ __forceinline__ PV4 pld_k(const float4 *K4, int leg, int e) {
  return pv4(K4[leg * NE + e]);
}

__device__ __forceinline__ PC4 pc_of(const CV4<float> &v) {
  return PC4{PV4{p2(v.c[0].re, v.c[1].re), p2(v.c[2].re, v.c[3].re)},
             PV4{p2(v.c[0].im, v.c[1].im), p2(v.c[2].im, v.c[3].im)}};
}

__device__ __forceinline__ float phsum(P2 x) { return plo(x) + phi(x); }

template <int L>
__device__ __forceinline__ void wavep_keep(int d, const PC4 &cur, float2 s, const PV4 &k, PC4 (&row)[L - 1],
                                           float2 (&srow)[L - 1], PV4 (&krow)[L - 1]) {
  switch (d) {
#define TESS_WAVEP_KEEP(D)           \
  case D:                            \
    if constexpr (D < L - 1) {       \
      row[D] = cur;                  \
      srow[D] = s;                   \
      krow[D] = k;                   \
    }                                \
    break;
    TESS_WAVEP_KEEP(1)
    TESS_WAVEP_KEEP(2)
    TESS_WAVEP_KEEP(3)
    TESS_WAVEP_KEEP(4)
    TESS_WAVEP_KEEP(5)
    TESS_WAVEP_KEEP(6)
    TESS_WAVEP_KEEP(7)
    TESS_WAVEP_KEEP(8)
    TESS_WAVEP_KEEP(9)
    TESS_WAVEP_KEEP(10)
#undef TESS_WAVEP_KEEP
    default:
      break;
  }
}

// As bg_wave (tess_wave.cuh) with packed arithmetic; S2 holds -S.
template <int L, int NE, int G, bool UNR>
__device__ __forceinline__ Cx<float> bg_wavep(const float4 *K4, float4 *J4, float2 *S2, int e, int g,
                                              const float *in_eps0, const float *in_e0, size_t cap) {
  Cx<float> amp = cx<float>(0.f, 0.f);
  const P2 sg_a = p2(1.f, -1.f), sg_b = pbc(-1.f), two = pbc(2.f);
#pragma unroll 1
  for (int a0 = wave_top_group<L, G>(); a0 >= 0; a0 -= G) {
    const int a = a0 - g;            // this lane's row
    const int len = L - a;           // its entries (the leaf and len - 1 sets)
    const int steps = L - (a0 - G + 1) - 1;
    PC4 row[L - 1];                  // signed currents J[a..a+dp]
    float2 srow[L - 1];              // -S[a..a+dp] (0 for the leaf)
    PV4 krow[L - 1];                 // signed K[a..a+dp]
    PV4 kcur;                        // raised K[a..b]
    if (a == 0) {
      CV4<float> v;
      load_eps(in_eps0, cap, v);
      row[0] = pc_signed(pc_of(v));
    } else {
      row[0] = pc_signed(pld_cv<NE>(J4, dsx<L>(a, 1), e));
    }
    kcur = pld_k<NE>(K4, a, e);
    srow[0] = make_float2(0.f, 0.f);
    krow[0] = pv_signed(kcur);
    auto step = [&](const int d) {
      if (d < len) {
        const int b = a + d;
        kcur = pv_add(kcur, pld_k<NE>(K4, b, e));
        PC4 accR = pc_zero(), accS = pc_zero(), tri = pc_zero();
        float sre = 0.f, sim = 0.f;
        PV4 kr = pv_zero();
#pragma unroll
        for (int dp = L - 2; dp >= 0; --dp) {
          if (dp < d) {  // split: left [a..a+dp] (row register dp), right [a+dp+1..b]
            const int r0 = a + dp + 1;
            kr = pv_add(kr, pld_k<NE>(K4, r0, e));
            const int ir = dsx<L>(r0, d - dp);
            const PC4 Jr = pld_cv<NE>(J4, ir, e);
            const PC4 &Jl = row[dp];
            P2 tre, tim;
            pcdot_pairs(Jl, Jr, tre, tim);
            const float d0re = phsum(tre), d0im = phsum(tim);
            sre += d0re;
            sim += d0im;
            const float crre = fmaf(2.f, phsum(pdot_pair(Jl.re, kr)), srow[dp].x);
            const float crim = fmaf(2.f, phsum(pdot_pair(Jl.im, kr)), srow[dp].y);
            float clre = -2.f * phsum(pdot_pair(Jr.re, krow[dp]));
            float clim = -2.f * phsum(pdot_pair(Jr.im, krow[dp]));
            if (dp + 1 < d) {  // right part has more than one leg: its -S
              const float2 sr = S2[ir * NE + e];
              clre += sr.x;
              clim += sr.y;
            }
            pc_axpy(accR, pbc(crre), pbc(crim), pbc(-crim), Jr);
            pc_axpy(accS, pbc(clre), pbc(clim), pbc(-clim), Jl);
            pr_axpy(accS, pbc(d0re), pbc(d0im), krow[dp]);
            pr_axpy(accR, pbc(-d0re), pbc(-d0im), kr);
            // four-vertex triples whose last part is [r0..b]: middle [a+dpp+1..a+dp]
#pragma unroll
            for (int dpp = 0; dpp < dp; ++dpp) {
              const PC4 JB = pld_cv<NE>(J4, dsx<L>(1, dp - dpp) + a + dpp, e);
              P2 xre, xim;
              pcdot_pairs(row[dpp], Jr, xre, xim);
              const float dre = phsum(xre), dim = phsum(xim);
              pc_axpy(tri, pbc(dre), pbc(dim), pbc(-dim), JB);
            }
          }
        }
        // Num (raised) = accR + g accS + 2 tri
        PC4 acc;
        acc.re.a = pfma(two, tri.re.a, pfma(sg_a, accS.re.a, accR.re.a));
        acc.re.b = pfma(two, tri.re.b, pfma(sg_b, accS.re.b, accR.re.b));
        acc.im.a = pfma(two, tri.im.a, pfma(sg_a, accS.im.a, accR.im.a));
        acc.im.b = pfma(two, tri.im.b, pfma(sg_b, accS.im.b, accR.im.b));
        if (a == 0 && d == L - 1) {
          CV4<float> v;
          load_eps(in_e0, cap, v);
          P2 xre, xim;
          pcdot_pairs(pc_signed(pc_of(v)), acc, xre, xim);
          amp = cx<float>(phsum(xre), phsum(xim));
        } else {
          // K^2 as the other forms evaluate it (one rounded product, then fused
          // multiply-adds): nearly collinear legs make it a small difference of
          // large terms, and the events failing the cuts are evaluated too
          float k2 = plo(kcur.a) * plo(kcur.a);
          k2 = fmaf(-phi(kcur.a), phi(kcur.a), k2);
          k2 = fmaf(-plo(kcur.b), plo(kcur.b), k2);
          k2 = fmaf(-phi(kcur.b), phi(kcur.b), k2);
          const float inv = 1.f / k2;
          const P2 ib = pbc(inv), isa = p2(inv, -inv), isb = pbc(-inv);
          const PC4 cur = PC4{PV4{pmul(acc.re.a, ib), pmul(acc.re.b, ib)}, PV4{pmul(acc.im.a, ib), pmul(acc.im.b, ib)}};
          const PC4 curs =
              PC4{PV4{pmul(acc.re.a, isa), pmul(acc.re.b, isb)}, PV4{pmul(acc.im.a, isa), pmul(acc.im.b, isb)}};
          const float2 sneg = make_float2(-sre, -sim);
          wavep_keep<L>(d, curs, sneg, pv_signed(kcur), row, srow, krow);
          if (a > 0) {
            const int t = dsx<L>(a, d + 1);
            pst_cv<NE>(J4, t, e, cur);
            S2[t * NE + e] = sneg;
          }
        }
      }
      if (G > 1) __syncwarp();  // the set stored at step d is the partner's right part at d + 1
    };
    if constexpr (UNR) {
#pragma unroll
      for (int d = 1; d < L; ++d) {
        if (d > steps) break;
        step(d);
      }
    } else {
#pragma unroll 1
      for (int d = 1; d <= steps; ++d) step(d);
    }
    if (G > 1) __syncwarp();
  }
  return amp;
}

template <int N, int NE, int G, bool UNR = false>
__global__ void __launch_bounds__(NE * G) bg_wavep_kernel(ChunkParams C, ChunkBuf<float> B, double *partials) {
  static_assert(G == 1 || G == 2, "one or two lanes per event");
  static_assert(G == 1 || NE % 16 == 0, "two-lane groups fill half warps");
  constexpr int L = N - 1, T1 = L * (L - 1) / 2, NT = NE * G;
  extern __shared__ __align__(16) char smem_raw[];
  float4 *J4 = (float4 *)smem_raw;
  float4 *K4 = J4 + 2 * T1 * NE;
  float2 *S2 = (float2 *)(K4 + L * NE);
  const int nb2 = C.P.hist_bins > 0 ? C.P.hist_bins + 2 : 0;
  EpiSmem<NT> S((char *)(S2 + T1 * NE), nb2);
  epi_init(S, nb2);
  Accum<NT> A;
  int slot, g;
  wave_slot<G>(slot, g);
  const int count = k2_count(C, B);
  const int ntiles = (count + NE - 1) / NE;
  const size_t cap = (size_t)B.cap;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile * NE + slot;
    const bool has = j < count;
    const int e = has ? k2_col(C, B, j) : 0;  // lanes without an event compute on column 0's data, unused
    if (G > 1) __syncwarp();
    // leg momenta and polarisations (positions 1..L-1) into the event's column
    for (int a = g; a < L; a += G) {
      const float *base = B.in + (size_t)InRows<L>::k(a) * cap + e;
      K4[a * NE + slot] = make_float4(base[0], base[cap], base[2 * cap], base[3 * cap]);
      if (a > 0) {
        CV4<float> ea;
        load_eps(B.in + (size_t)InRows<L>::eps(a) * cap + e, cap, ea);
        pst_cv<NE>(J4, dsx<L>(a, 1), slot, pc_of(ea));
      }
    }
    if (G > 1) __syncwarp();
    wave_prefetch_next<L, NE, NT>(C, B, tile, ntiles);
    const Cx<float> amp = bg_wavep<L, NE, G, UNR>(K4, J4, S2, slot, g, B.in + (size_t)InRows<L>::eps(0) * cap + e,
                                                  B.in + (size_t)InRows<L>::eps0 * cap + e, cap);
    double w = 0.0;
    int bin = -1;
    if (has && g == G - 1) finish_event<NT, float>(C, B, e, amp2_of(amp), A, w, bin);
    epi_tile<NT>(S, nb2, w, bin);
  }
  epi_flush<NT>(S, nb2, A, partials, C.P.hist_bins);
}

}  // namespace tess
