// K2, wavefront row form (FP32, large n): the Berends-Giele recursion of one
// event split over G lanes of one warp, each lane building one row of the
// current table, the G rows of a group advancing in step over their sets.
//
// Recursion (Sec. 3, Eq. (BG-recursion), with the four-vertex sum reorganised
// as in the other forms): row a holds the currents J[a..b], b >= a.  Set
// [a..a+d] needs the left parts J[a..a+dp] (the lane's own row, in its
// registers), the right parts J[a+dp+1..a+d] and the middle parts of its
// four-vertex triples, all from rows > a.  Sec. 3 assigns one thread per
// current of a given length; here the G rows a0, a0-1, ..., a0-G+1 run
// together: at step d lane g builds [a0-g .. a0-g+d], whose right part of
// one leg fewer, [a0-g+1 .. a0-g+d], is the set lane g-1 built at step d-1.
// So a step needs only what the previous steps stored (in the event's
// shared-memory column) and a warp-level barrier between steps, and an event
// occupies G threads instead of one: G times the resident warps for the same
// shared memory per event.  Lanes whose row is shorter than the group's
// longest idle at its last steps (for n = 10 and G = 2 the lanes do 83 % of
// the thread-steps' work).
//
// Within a step the split loop over dp is unrolled with a uniform branch per
// dp (dp < d), so the row's registers are addressed with compile-time
// indices while the step loop itself stays a runtime loop: one copy of the
// code serves every step and every row (a fraction of the fully unrolled
// row body, so that it stays in the instruction cache).
//
// Each lane's arithmetic per set is the row form's (tess_pipeline.cuh,
// bg_rows), in the same order.
#pragma once
#include "tess_pipeline.cuh"

namespace tess {

// Per-event shared-memory column: J of the sets [a..b], 1 <= a <= b <= L-1
// (two float4 each, index wix<L, UNR>), the leg momenta (float4), the split
// sums S (float2).  Event slot e of NE, element (plane p, slot e) at
// p * NE + e.
//
// Index of the set [s..s+len-1] (1 <= s, s + len - 1 <= L-1) in the
// length-major layout: the sets of length 1, then of length 2, ...  A set of
// row a with a given length sits at a + (a constant of the length), so in
// the unrolled step code, where every length is known at compile time,
// every table address is one register per row plus an immediate offset
// (measured at n = 10: 2.7 % faster than the row-major t1 layout).  The
// rolled step code, whose lengths are runtime values, keeps the row-major
// layout (7 % slower with this one).
template <int L>
__host__ __device__ constexpr int dsx(int s, int len) {
  return (len - 1) * L - ((len - 1) * len) / 2 + (s - 1);
}
template <int L, bool LENGTH_MAJOR>
__host__ __device__ constexpr int wix(int s, int len) {
  return LENGTH_MAJOR ? dsx<L>(s, len) : t1<L>(s, s + len - 1);
}
template <int L>
__host__ __device__ constexpr size_t wave_smem_per_event() {
  return (size_t)(L * (L - 1) / 2) * (2 * sizeof(float4) + sizeof(float2)) + (size_t)L * sizeof(float4);
}

template <int NE>
__device__ __forceinline__ void wst_cv(float4 *J4, int t, int e, const CV4<float> &v) {
  J4[(2 * t) * NE + e] = make_float4(v.c[0].re, v.c[0].im, v.c[1].re, v.c[1].im);
  J4[(2 * t + 1) * NE + e] = make_float4(v.c[2].re, v.c[2].im, v.c[3].re, v.c[3].im);
}

template <int NE>
__device__ __forceinline__ CV4<float> wld_cv(const float4 *J4, int t, int e) {
  const float4 a = J4[(2 * t) * NE + e];
  const float4 b = J4[(2 * t + 1) * NE + e];
  CV4<float> v;
  v.c[0] = cx<float>(a.x, a.y);
  v.c[1] = cx<float>(a.z, a.w);
  v.c[2] = cx<float>(b.x, b.y);
  v.c[3] = cx<float>(b.z, b.w);
  return v;
}

template <int NE>
__device__ __forceinline__ RV4<float> wld_k(const float4 *K4, int leg, int e) {
  const float4 v = K4[leg * NE + e];
  RV4<float> r = {{v.x, v.y, v.z, v.w}};
  return r;
}

// row[d] = cur, srow[d] = s, krow[d] = k for the runtime step d (1 <= d <=
// L-2): one uniform jump to the copy for that d instead of a predicated
// copy into every candidate register.
template <int L>
__device__ __forceinline__ void wave_keep(int d, const CV4<float> &cur, const Cx<float> &s, const RV4<float> &k,
                                          CV4<float> (&row)[L - 1], Cx<float> (&srow)[L - 1],
                                          RV4<float> (&krow)[L - 1]) {
  switch (d) {
#define TESS_WAVE_KEEP(D)            \
  case D:                            \
    if constexpr (D < L - 1) {       \
      row[D] = cur;                  \
      srow[D] = s;                   \
      krow[D] = k;                   \
    }                                \
    break;
    TESS_WAVE_KEEP(1)
    TESS_WAVE_KEEP(2)
    TESS_WAVE_KEEP(3)
    TESS_WAVE_KEEP(4)
    TESS_WAVE_KEEP(5)
    TESS_WAVE_KEEP(6)
    TESS_WAVE_KEEP(7)
    TESS_WAVE_KEEP(8)
    TESS_WAVE_KEEP(9)
    TESS_WAVE_KEEP(10)
#undef TESS_WAVE_KEEP
    default:
      break;
  }
}

// First row of the group that holds row a (rows are grouped from the top so
// that row 0 closes the last group): groups {a0, ..., a0-G+1} with a0 = G-1,
// 2G-1, ...; the first group processed is the highest one with a set.
template <int L, int G>
__host__ __device__ constexpr int wave_top_group() {
  // rows with at least one set: 0..L-2
  return ((L - 2) / G) * G + G - 1;
}

// The amplitude m = e0 . Num[0..L-1] of the event in slot e (returned by the
// lane that builds row 0, g = G-1; other lanes return 0).  in_e0 / in_eps0:
// the event's rows of the contraction vector and of position 0's
// polarisation (read from the chunk buffer by that lane).
template <int L, int NE, int G, bool UNR>
__device__ __forceinline__ Cx<float> bg_wave(const float4 *K4, float4 *J4, float2 *S2, int e, int g,
                                             const float *in_eps0, const float *in_e0, size_t cap) {
  Cx<float> amp = cx<float>(0.f, 0.f);
#pragma unroll 1
  for (int a0 = wave_top_group<L, G>(); a0 >= 0; a0 -= G) {
    const int a = a0 - g;            // this lane's row
    const int len = L - a;           // its entries (the leaf and len - 1 sets); <= 0: no row
    const int steps = L - (a0 - G + 1) - 1;  // sets of the group's longest row
    CV4<float> row[L - 1];
    Cx<float> srow[L - 1];
    RV4<float> krow[L - 1];
    RV4<float> kcur = {{0.f, 0.f, 0.f, 0.f}};
    if (len > 0) {
      if (a == 0) {
        load_eps(in_eps0, cap, row[0]);
      } else {
        row[0] = wld_cv<NE>(J4, wix<L, UNR>(a, 1), e);
      }
      kcur = wld_k<NE>(K4, a, e);
    } else {
      row[0] = cv_zero<float>();
    }
    srow[0] = cx<float>(0.f, 0.f);
    krow[0] = kcur;
    auto step = [&](const int d) {
      if (d < len) {
        const int b = a + d;
        kcur = radd(kcur, wld_k<NE>(K4, b, e));
        CV4<float> acc = cv_zero<float>(), tri = cv_zero<float>();
        Cx<float> s = cx<float>(0.f, 0.f);
        RV4<float> kr = {{0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int dp = L - 2; dp >= 0; --dp) {
          if (dp < d) {  // split: left [a..a+dp] (row register dp), right [a+dp+1..b]
            const int r0 = a + dp + 1;
            kr = radd(kr, wld_k<NE>(K4, r0, e));
            const int tr = wix<L, UNR>(r0, d - dp);  // [r0..b]
            const CV4<float> Jr = wld_cv<NE>(J4, tr, e);
            const CV4<float> &Jl = row[dp];
            // the left part [a..a] (dp = 0) is a single leg: its polarisation
            // vector's exact zeros are left out (tess_bg.cuh, mdot_l); so are
            // the right part's when it is one ([b..b], dp = d - 1), where the
            // step is known at compile time (UNR)
            const bool rl = UNR && dp + 1 == d;
            const Cx<float> d0 = leaf_sel(dp == 0, rl, [&](auto la, auto lb) {
              return mdot_l<decltype(la)::value, decltype(lb)::value>(Jl, Jr);
            });
            const Cx<float> jlkr = dp == 0 ? mdot_leaf(Jl, kr) : mdot(Jl, kr);
            const Cx<float> krjl = rl ? mdot_leaf(Jr, krow[dp]) : mdot(Jr, krow[dp]);
            Cx<float> cr = cx<float>(2.f * jlkr.re - srow[dp].re, 2.f * jlkr.im - srow[dp].im);
            Cx<float> cl = cx<float>(-2.f * krjl.re, -2.f * krjl.im);
            if (dp + 1 < d) {  // right part has more than one leg
              const float2 sr = S2[tr * NE + e];
              cl.re -= sr.x;
              cl.im -= sr.y;
            }
            if (rl)
              axpy_leaf(acc, cr, Jr);
            else
              axpy(acc, cr, Jr);
            if (dp == 0)
              axpy_leaf(acc, cl, Jl);
            else
              axpy(acc, cl, Jl);
            axpy(acc, d0, rsub(krow[dp], kr));
            s.re += d0.re;
            s.im += d0.im;
            // four-vertex triples whose last part is [r0..b] (first part
            // [a..a+dpp] a single leg for dpp = 0, middle part one for dpp = dp - 1)
#pragma unroll
            for (int dpp = 0; dpp < dp; ++dpp) {
              const CV4<float> JB = wld_cv<NE>(J4, wix<L, UNR>(a + dpp + 1, dp - dpp), e);  // [a+dpp+1..a+dp]
              const Cx<float> x = leaf_sel(dpp == 0, rl, [&](auto la, auto lb) {
                return mdot_l<decltype(la)::value, decltype(lb)::value>(row[dpp], Jr);
              });
              if (dpp + 1 == dp)
                axpy_leaf(tri, x, JB);
              else
                axpy(tri, x, JB);
            }
          }
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          acc.c[m].re = fmaf(2.f, tri.c[m].re, acc.c[m].re);
          acc.c[m].im = fmaf(2.f, tri.c[m].im, acc.c[m].im);
        }
        if (a == 0 && d == L - 1) {
          CV4<float> e0;
          load_eps(in_e0, cap, e0);
          amp = mdot(e0, acc);
        } else {
          const float inv = 1.f / mdot(kcur, kcur);
          CV4<float> cur;
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            cur.c[m].re = acc.c[m].re * inv;
            cur.c[m].im = acc.c[m].im * inv;
          }
          wave_keep<L>(d, cur, s, kcur, row, srow, krow);
          if (a > 0) {
            const int t = wix<L, UNR>(a, d + 1);  // [a..b]
            wst_cv<NE>(J4, t, e, cur);
            S2[t * NE + e] = make_float2(s.re, s.im);
          }
        }
      }
      if (G > 1) __syncwarp();  // the set stored at step d is the partner's right part at d + 1
    };
    if constexpr (UNR) {  // every step its own code: compile-time register and table indices
#pragma unroll
      for (int d = 1; d < L; ++d) {
        if (d > steps) break;
        step(d);
      }
    } else {
#pragma unroll 1
      for (int d = 1; d <= steps; ++d) step(d);
    }
    if (G > 1) __syncwarp();  // the group's rows are complete before the next group reads them
  }
  return amp;
}

// Lean form of bg_wave: only the row's currents stay in registers.  The left
// part's momentum sum is K[a..b] - K[r0..b] (both at hand in the split
// loop), and its split sum S is read back from the table (row 0's split
// sums, not otherwise stored, in their own slots S0[d]).  About 50 registers
// fewer per lane, so that 12 warps fit on an SM beside the tables (6 blocks
// of 32 events).  Subtracting momentum sums instead of adding legs changes
// only the rounding: its absolute error, eps |K[r0..b]|, is of the order of
// the rounding already present in the K[r0..b] terms of the same bracket.
template <int L, int NE, int G>
__device__ __forceinline__ Cx<float> bg_wave_lean(const float4 *K4, float4 *J4, float2 *S2, float2 *S0, int e, int g,
                                                  const float *in_eps0, const float *in_e0, size_t cap) {
  Cx<float> amp = cx<float>(0.f, 0.f);
#pragma unroll 1
  for (int a0 = wave_top_group<L, G>(); a0 >= 0; a0 -= G) {
    const int a = a0 - g;
    const int len = L - a;
    const int steps = L - (a0 - G + 1) - 1;
    CV4<float> row[L - 1];
    RV4<float> kcur;
    if (a == 0) {
      load_eps(in_eps0, cap, row[0]);
    } else {
      row[0] = wld_cv<NE>(J4, t1<L>(a, a), e);
    }
    kcur = wld_k<NE>(K4, a, e);
#pragma unroll 1
    for (int d = 1; d <= steps; ++d) {
      if (d < len) {
        const int b = a + d;
        kcur = radd(kcur, wld_k<NE>(K4, b, e));
        CV4<float> acc = cv_zero<float>(), tri = cv_zero<float>();
        Cx<float> s = cx<float>(0.f, 0.f);
        RV4<float> kr = {{0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int dp = L - 2; dp >= 0; --dp) {
          if (dp < d) {  // split: left [a..a+dp] (row register dp), right [a+dp+1..b]
            const int r0 = a + dp + 1;
            kr = radd(kr, wld_k<NE>(K4, r0, e));
            const RV4<float> kl = rsub(kcur, kr);
            const int tr = t1<L>(r0, b);
            const CV4<float> Jr = wld_cv<NE>(J4, tr, e);
            const CV4<float> &Jl = row[dp];
            const Cx<float> d0 = dp == 0 ? mdot_l<true, false>(Jl, Jr) : mdot(Jl, Jr);  // leaf left part
            const Cx<float> jlkr = dp == 0 ? mdot_leaf(Jl, kr) : mdot(Jl, kr);
            const Cx<float> krjl = mdot(Jr, kl);
            Cx<float> cr = cx<float>(2.f * jlkr.re, 2.f * jlkr.im);
            if (dp > 0) {  // left part has more than one leg
              const float2 sl = a > 0 ? S2[t1<L>(a, a + dp) * NE + e] : S0[dp * NE + e];
              cr.re -= sl.x;
              cr.im -= sl.y;
            }
            Cx<float> cl = cx<float>(-2.f * krjl.re, -2.f * krjl.im);
            if (dp + 1 < d) {  // right part has more than one leg
              const float2 sr = S2[tr * NE + e];
              cl.re -= sr.x;
              cl.im -= sr.y;
            }
            axpy(acc, cr, Jr);
            if (dp == 0)
              axpy_leaf(acc, cl, Jl);
            else
              axpy(acc, cl, Jl);
            axpy(acc, d0, rsub(kl, kr));
            s.re += d0.re;
            s.im += d0.im;
#pragma unroll
            for (int dpp = 0; dpp < dp; ++dpp) {
              const CV4<float> JB = wld_cv<NE>(J4, t1<L>(a + dpp + 1, a + dp), e);
              const Cx<float> x = dpp == 0 ? mdot_l<true, false>(row[dpp], Jr) : mdot(row[dpp], Jr);
              if (dpp + 1 == dp)
                axpy_leaf(tri, x, JB);
              else
                axpy(tri, x, JB);
            }
          }
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          acc.c[m].re = fmaf(2.f, tri.c[m].re, acc.c[m].re);
          acc.c[m].im = fmaf(2.f, tri.c[m].im, acc.c[m].im);
        }
        if (a == 0 && d == L - 1) {
          CV4<float> e0;
          load_eps(in_e0, cap, e0);
          amp = mdot(e0, acc);
        } else {
          const float inv = 1.f / mdot(kcur, kcur);
          CV4<float> cur;
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            cur.c[m].re = acc.c[m].re * inv;
            cur.c[m].im = acc.c[m].im * inv;
          }
          switch (d) {
#define TESS_WAVE_LEAN_KEEP(D) \
  case D:                      \
    if constexpr (D < L - 1) row[D] = cur; \
    break;
            TESS_WAVE_LEAN_KEEP(1)
            TESS_WAVE_LEAN_KEEP(2)
            TESS_WAVE_LEAN_KEEP(3)
            TESS_WAVE_LEAN_KEEP(4)
            TESS_WAVE_LEAN_KEEP(5)
            TESS_WAVE_LEAN_KEEP(6)
            TESS_WAVE_LEAN_KEEP(7)
            TESS_WAVE_LEAN_KEEP(8)
            TESS_WAVE_LEAN_KEEP(9)
            TESS_WAVE_LEAN_KEEP(10)
#undef TESS_WAVE_LEAN_KEEP
            default:
              break;
          }
          if (a > 0) {
            const int t = t1<L>(a, b);
            wst_cv<NE>(J4, t, e, cur);
            S2[t * NE + e] = make_float2(s.re, s.im);
          } else {
            S0[d * NE + e] = make_float2(s.re, s.im);
          }
        }
      }
      if (G > 1) __syncwarp();
    }
    if (G > 1) __syncwarp();
  }
  return amp;
}

// Event slot and group lane of this thread: G = 1, one thread per event; G =
// 2, lanes l and l + 16 of a warp share event slot 16 w + (l & 15), so that
// the eight lanes of a shared-memory phase read eight consecutive slots.
template <int G>
__device__ __forceinline__ void wave_slot(int &slot, int &g) {
  if (G == 1) {
    slot = threadIdx.x;
    g = 0;
  } else {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    slot = warp * 16 + (lane & 15);
    g = lane >> 4;
  }
}

template <int L>
__host__ __device__ constexpr size_t wave_lean_smem_per_event() {
  return wave_smem_per_event<L>() + (size_t)(L - 1) * sizeof(float2);
}

// The block's next tile of amplitude inputs (NE consecutive chunk columns, one
// 128-byte line per input row when NE = 32) and event factors into L2 while
// the current tile is computed: the chunk buffer is read once, mostly from
// DRAM, so every tile otherwise starts with a DRAM-latency wait.  Columns
// past the chunk's count are inside the buffer (its capacity is a multiple of
// 128 columns), so no prefetch leaves it.  Not for cut-first chunks, whose
// tiles are gathered through a column list.  Used by the packed-pair forms
// (measured at n = 10 / 12: +4 / +5 %) and the unrolled scalar form (+6 % at
// n = 10 with the histogram deferred); the rolled scalar forms measured 2-4 %
// slower with it (n = 10, 11) and do without.
template <int L, int NE, int NT>
__device__ __forceinline__ void wave_prefetch_next(const ChunkParams &C, const ChunkBuf<float> &B, int tile,
                                                   int ntiles) {
  const int nt = tile + (int)gridDim.x;
  if (C.P.cut_first || nt >= ntiles) return;
  static_assert(NE % 32 == 0, "whole 128-byte lines per input row");
  const size_t col = (size_t)nt * NE;
  const size_t cap = (size_t)B.cap;
  constexpr int R = InRows<L>::rows, LF = NE / 32, LD = NE / 16;  // lines per float row, per double row
  for (int i = threadIdx.x; i < R * LF + 2 * LD; i += NT) {
    const char *p;
    if (i < R * LF)
      p = (const char *)(B.in + (size_t)(i / LF) * cap + col) + (i % LF) * 128;
    else {
      const int k = i - R * LF;
      p = (const char *)((k < LD ? B.efac : B.wfac) + col) + (k % LD) * 128;
    }
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
  }
}

template <int N, int NE, int G, bool UNR = false, bool LEAN = false, int MINB = 1>
__global__ void __launch_bounds__(NE * G, MINB) bg_wave_kernel(ChunkParams C, ChunkBuf<float> B, double *partials) {
  static_assert(G == 1 || G == 2, "one or two lanes per event");
  static_assert(G == 1 || NE % 16 == 0, "two-lane groups fill half warps");
  constexpr int L = N - 1, T1 = L * (L - 1) / 2, NT = NE * G;
  extern __shared__ __align__(16) char smem_raw[];
  float4 *J4 = (float4 *)smem_raw;
  float4 *K4 = J4 + 2 * T1 * NE;
  float2 *S2 = (float2 *)(K4 + L * NE);
  float2 *S0 = S2 + T1 * NE;  // lean form only: row 0's split sums
  const int nb2 = C.P.hist_bins > 0 ? C.P.hist_bins + 2 : 0;
  EpiSmem<NT> S((char *)(LEAN ? S0 + (L - 1) * NE : S0), nb2);
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
    if (G > 1) __syncwarp();  // the previous tile's reads of this slot are done
    // leg momenta and polarisations (positions 1..L-1) into the event's column
#pragma unroll
    for (int a = g; a < L; a += G) {
      const float *base = B.in + (size_t)InRows<L>::k(a) * cap + e;
      K4[a * NE + slot] = make_float4(base[0], base[cap], base[2 * cap], base[3 * cap]);
      if (a > 0) {
        CV4<float> ea;
        load_eps(B.in + (size_t)InRows<L>::eps(a) * cap + e, cap, ea);
        wst_cv<NE>(J4, wix<L, UNR && !LEAN>(a, 1), slot, ea);
      }
    }
    if (G > 1) __syncwarp();
    if constexpr (UNR) wave_prefetch_next<L, NE, NT>(C, B, tile, ntiles);
    Cx<float> amp;
    if constexpr (LEAN)
      amp = bg_wave_lean<L, NE, G>(K4, J4, S2, S0, slot, g, B.in + (size_t)InRows<L>::eps(0) * cap + e,
                                   B.in + (size_t)InRows<L>::eps0 * cap + e, cap);
    else
      amp = bg_wave<L, NE, G, UNR>(K4, J4, S2, slot, g, B.in + (size_t)InRows<L>::eps(0) * cap + e,
                                   B.in + (size_t)InRows<L>::eps0 * cap + e, cap);
    double w = 0.0;
    int bin = -1;
    if (has && g == G - 1) finish_event<NT, float>(C, B, e, amp2_of(amp), A, w, bin);
    epi_tile<NT>(S, nb2, w, bin);
  }
  epi_flush<NT>(S, nb2, A, partials, C.P.hist_bins);
}

}  // namespace tess
