// K2, warp-lanes form (FP32, large n): LN lanes of one warp per event
// (32 / LN events per warp), the event's Berends-Giele table in shared
// memory, the currents of one length built together.
//
// Sec. 3 assigns one thread per current of a given length, so that the
// recursion runs in n - 2 steps; here the LN lanes of an event share the
// sets of one length, and where a length has fewer sets than lanes (the long
// sets), q lanes (a power of two) share one set: lane r of the q takes the
// splits i = a + r, a + r + q, ... of X = [a..b] together with the
// four-vertex triples whose left part ends at those i, and the q partial
// sums (current numerator and split sum S, Sec. 3 recursion with the
// reorganised four-vertex sum of tess_bg.cuh) are added by a butterfly of
// __shfl_xor_sync in a fixed order, so the result does not depend on timing.
// A __syncwarp separates the lengths (the event's lanes are one warp's).
//
// Table layout per event slot g (all in float4 / float2 units, event-major
// so that the lanes of one event, reading consecutive entries, fall on
// distinct banks): the two halves of the current J[X] in separate planes
// (Jlo, Jhi), the split sums S[X], the prefix momenta P[i] = k_0 + ... +
// k_{i-1} (K[a..b] = P[b+1] - P[a]) and the contraction vector e0.
#pragma once
#include "tess_pair.cuh"

namespace tess {

template <int L>
struct LanesLayout {
  static constexpr int T = L * (L + 1) / 2;  // sets [a..b], 0 <= a <= b <= L-1 (index pair_tri)
  // float4 slots per event: Jlo[T], Jhi[T], P[L + 1], e0[2]; then float2 S[T]
  static constexpr int f4 = 2 * T + (L + 1) + 2;
  // rounded up to 16 bytes so that every event's float4 planes stay aligned
  static constexpr size_t bytes_per_event =
      ((size_t)f4 * sizeof(float4) + (size_t)T * sizeof(float2) + 15) / 16 * 16;
};

template <int L>
struct LanesView {
  float4 *Jlo, *Jhi, *P4, *E4;
  float2 *S2;
  __device__ LanesView(char *base, int g) {
    constexpr int T = LanesLayout<L>::T;
    float4 *f = (float4 *)(base + (size_t)g * LanesLayout<L>::bytes_per_event);
    Jlo = f;
    Jhi = f + T;
    P4 = f + 2 * T;
    E4 = P4 + (L + 1);
    S2 = (float2 *)(E4 + 2);
  }
  __device__ __forceinline__ CV4<float> J(int X) const {
    const float4 u = Jlo[X], v = Jhi[X];
    CV4<float> r;
    r.c[0] = cx<float>(u.x, u.y);
    r.c[1] = cx<float>(u.z, u.w);
    r.c[2] = cx<float>(v.x, v.y);
    r.c[3] = cx<float>(v.z, v.w);
    return r;
  }
  __device__ __forceinline__ void setJ(int X, const CV4<float> &r) const {
    Jlo[X] = make_float4(r.c[0].re, r.c[0].im, r.c[1].re, r.c[1].im);
    Jhi[X] = make_float4(r.c[2].re, r.c[2].im, r.c[3].re, r.c[3].im);
  }
  __device__ __forceinline__ RV4<float> P(int i) const {
    const float4 p = P4[i];
    RV4<float> r = {{p.x, p.y, p.z, p.w}};
    return r;
  }
};

// Partial sums of X = [a..b] over the splits i = a + i0, a + i0 + di, ... <
// b: the three-vertex brackets (with the -S terms of the reorganised
// four-vertex sum) plus 2 x the triples whose left part ends at one of those
// i, and the split sum s of J_l.J_r over the same splits.  The arithmetic per
// split and per triple is the lane-pair form's (pair_sums); table indices
// advance by adds.
template <int L>
__device__ __forceinline__ void lanes_sums(const LanesView<L> &V, int a, int b, int i0, int di, CV4<float> &acc,
                                           Cx<float> &s) {
  const RV4<float> Pa = V.P(a), Pb = V.P(b + 1);
  CV4<float> acc1 = cv_zero<float>(), acc2 = cv_zero<float>(), trs = cv_zero<float>();
  s = cx<float>(0.f, 0.f);
  int i = a + i0;
  int xl = pair_tri<L>(a, i), xr = i < b ? pair_tri<L>(i + 1, b) : 0;
#pragma unroll 1
  for (; i < b; i += di) {
    const CV4<float> Jl = V.J(xl), Jr = V.J(xr);
    const RV4<float> Pi = V.P(i + 1);
    const RV4<float> Kl = rsub(Pi, Pa), Kr = rsub(Pb, Pi);
    const Cx<float> d = mdot(Jl, Jr);
    const Cx<float> jlkr = mdot(Jl, Kr);
    const Cx<float> krjl = mdot(Jr, Kl);
    const float2 sl = V.S2[xl], sr = V.S2[xr];  // zero for single legs
    const Cx<float> cr = cx<float>(fmaf(2.f, jlkr.re, -sl.x), fmaf(2.f, jlkr.im, -sl.y));
    const Cx<float> cl = cx<float>(fmaf(-2.f, krjl.re, -sr.x), fmaf(-2.f, krjl.im, -sr.y));
    axpy(acc1, cr, Jr);
    axpy(acc2, cl, Jl);
    axpy(acc1, d, rsub(Kl, Kr));
    s.re += d.re;
    s.im += d.im;
    // triples (J[a..i] . J[c+1..b]) J[i+1..c], i < c < b
    int xc = xr + (L - i - 2), xm = xr - (b - i - 1);
#pragma unroll 1
    for (int c = i + 1; c < b; ++c) {
      axpy(trs, mdot(Jl, V.J(xc)), V.J(xm));
      xc += L - c - 2;
      xm += 1;
    }
    // next split of this lane: [a..i+di] is di entries on; [i+di+1..b] is
    // sum_{t=1..di} (L - i - t - 1) = di (L - i - 1) - di (di + 1) / 2 on
    xr += di * (L - i - 1) - (di * (di + 1)) / 2;
    xl += di;
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    acc.c[m].re = fmaf(2.f, trs.c[m].re, acc1.c[m].re + acc2.c[m].re);
    acc.c[m].im = fmaf(2.f, trs.c[m].im, acc1.c[m].im + acc2.c[m].im);
  }
}

// Sum over the q lanes (aligned groups, q a power of two <= LN) of the
// current numerator and split sum; every lane of the warp takes part.
template <int LN>
__device__ __forceinline__ void lanes_reduce(int q, CV4<float> &acc, Cx<float> &s) {
#pragma unroll
  for (int m = 1; m < LN; m <<= 1) {
    if (m >= q) break;  // q is uniform across the warp
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc.c[c].re += __shfl_xor_sync(0xffffffffu, acc.c[c].re, m);
      acc.c[c].im += __shfl_xor_sync(0xffffffffu, acc.c[c].im, m);
    }
    s.re += __shfl_xor_sync(0xffffffffu, s.re, m);
    s.im += __shfl_xor_sync(0xffffffffu, s.im, m);
  }
}

// Lanes per set at length len: the largest power of two q with q times the
// number of sets within LN (at least 1).
template <int L, int LN>
__device__ __forceinline__ int lanes_per_set(int len) {
  const int ns = L - len + 1;
  int q = 1;
  while (2 * q * ns <= LN) q *= 2;
  return q;
}

// The event's amplitude numerator Num[0..L-1] contracted with e0, returned
// by lane 0 of the event (the other lanes return 0).  r: lane within the
// event.  live: the event exists (all lanes still run every shuffle).
template <int L, int LN>
__device__ __forceinline__ Cx<float> bg_lanes(const LanesView<L> &V, int r, bool live) {
  // lengths 2..L-1: the sets a = pass * (LN / q) + r / q, split share r % q
#pragma unroll 1
  for (int len = 2; len < L; ++len) {
    const int ns = L - len + 1;
    const int q = lanes_per_set<L, LN>(len);
    const int per_pass = LN / q;
#pragma unroll 1
    for (int base = 0; base < ns; base += per_pass) {
      const int a = base + r / q;
      const bool has = live && a < ns;
      CV4<float> acc = cv_zero<float>();
      Cx<float> s = cx<float>(0.f, 0.f);
      if (has) lanes_sums<L>(V, a, a + len - 1, r % q, q, acc, s);
      lanes_reduce<LN>(q, acc, s);
      if (has && r % q == 0) {
        const int b = a + len - 1;
        const RV4<float> K = rsub(V.P(b + 1), V.P(a));
        const float inv = 1.f / mdot(K, K);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          acc.c[m].re *= inv;
          acc.c[m].im *= inv;
        }
        const int X = pair_tri<L>(a, b);
        V.setJ(X, acc);
        V.S2[X] = make_float2(s.re, s.im);
      }
    }
    __syncwarp();  // this length's sets are the next lengths' parts
  }
  // the top set [0..L-1] (numerator only), shared by all LN lanes
  CV4<float> num = cv_zero<float>();
  Cx<float> s = cx<float>(0.f, 0.f);
  if (live) lanes_sums<L>(V, 0, L - 1, r, LN, num, s);
  lanes_reduce<LN>(LN, num, s);
  Cx<float> amp = cx<float>(0.f, 0.f);
  if (live && r == 0) {
    const float4 u = V.E4[0], v = V.E4[1];
    CV4<float> e0;
    e0.c[0] = cx<float>(u.x, u.y);
    e0.c[1] = cx<float>(u.z, u.w);
    e0.c[2] = cx<float>(v.x, v.y);
    e0.c[3] = cx<float>(v.z, v.w);
    amp = mdot(e0, num);
  }
  return amp;
}

template <int L, int NW, int LN>
__host__ __device__ constexpr size_t lanes_smem_bytes() {
  return (size_t)NW * (32 / LN) * LanesLayout<L>::bytes_per_event;
}

// NW warps per block, 32 / LN events per warp: NE = NW * 32 / LN events per
// tile.  Event slot g = warp * (32 / LN) + lane / LN, lane within the event
// r = lane % LN.
template <int N, int LN, int NW>
__global__ void __launch_bounds__(32 * NW) bg_lanes_kernel(ChunkParams C, ChunkBuf<float> B, double *partials) {
  static_assert(LN == 4 || LN == 8 || LN == 16 || LN == 32, "lanes per event: a power of two dividing 32");
  constexpr int L = N - 1, NB = 32 * NW, EPW = 32 / LN, NE = NW * EPW;
  extern __shared__ __align__(16) char smem_lanes[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int g = warp * EPW + lane / LN, r = lane % LN;
  const LanesView<L> V(smem_lanes, g);
  const int nb2 = C.P.hist_bins > 0 ? C.P.hist_bins + 2 : 0;
  EpiSmem<NB> ES(smem_lanes + lanes_smem_bytes<L, NW, LN>(), nb2);
  epi_init(ES, nb2);
  Accum<NB> A;
  const int count = k2_count(C, B);
  const int ntiles = (count + NE - 1) / NE;
  const size_t cap = (size_t)B.cap;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile * NE + g;
    const bool live = j < count;
    const int e = live ? k2_col(C, B, j) : 0;
    __syncwarp();  // the previous tile's reads of this warp's tables are done
    if (live) {
      // leaves and momenta: lane r loads legs r, r + LN, ...
#pragma unroll 1
      for (int a = r; a < L; a += LN) {
        CV4<float> ea;
        load_eps(B.in + (size_t)InRows<L>::eps(a) * cap + e, cap, ea);
        const int X = pair_tri<L>(a, a);
        V.setJ(X, ea);
        V.S2[X] = make_float2(0.f, 0.f);
        RV4<float> k;
        load_k(B.in + (size_t)InRows<L>::k(a) * cap + e, cap, k);
        V.P4[a + 1] = make_float4(k.v[0], k.v[1], k.v[2], k.v[3]);  // k_a, summed below
      }
      if (r == 0) {
        CV4<float> e0;
        load_eps(B.in + (size_t)InRows<L>::eps0 * cap + e, cap, e0);
        V.E4[0] = make_float4(e0.c[0].re, e0.c[0].im, e0.c[1].re, e0.c[1].im);
        V.E4[1] = make_float4(e0.c[2].re, e0.c[2].im, e0.c[3].re, e0.c[3].im);
      }
    }
    __syncwarp();
    if (live && r == 0) {  // prefix sums P[i] = k_0 + ... + k_{i-1}, in leg order
      RV4<float> p = {{0.f, 0.f, 0.f, 0.f}};
      V.P4[0] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
      for (int a = 0; a < L; ++a) {
        p = radd(p, V.P(a + 1));
        V.P4[a + 1] = make_float4(p.v[0], p.v[1], p.v[2], p.v[3]);
      }
    }
    __syncwarp();
    const Cx<float> amp = bg_lanes<L, LN>(V, r, live);
    double w = 0.0;
    int bin = -1;
    if (live && r == 0) finish_event<NB, float>(C, B, e, amp2_of(amp), A, w, bin);
    epi_tile<NB>(ES, nb2, w, bin);
  }
  epi_flush<NB>(ES, nb2, A, partials, C.P.hist_bins);
}

}  // namespace tess
