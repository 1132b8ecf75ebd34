// Berends-Giele colour-ordered amplitude for one event, one thread.
//
// Recursion (Sec. 3, Eq. (BG-recursion) and its shorthand): for a contiguous
// set X = [a..b] of the L = n-1 legs,
//   J[X] = 1/K[X]^2 ( sum_splits [J_l, J_r] + sum_triples {J_l, J_m, J_r} ).
// The triple (four-gluon vertex) sum is reorganised here without changing
// its value.  With S[Y] = sum_{splits (l,r) of Y} J_l.J_r (a scalar per set),
//   sum_{A,B,C} {A,B,C} = 2 sum_{A,B,C} (J_A.J_C) J_B
//                         - sum_{splits (l,r) of X} ( S[l] J_r + S[r] J_l ),
// so each split costs one three-vertex bracket plus two scalar multiply-adds
// and only the (J_A.J_C) J_B term keeps the O(n^4) triple loop.  S[Y] is
// accumulated for free while Y itself is built (it is the sum of the J_l.J_r
// dot products the brackets already need).
//
// All loops have compile-time trip counts, so after full unrolling every
// table index is a constant and the tables live in registers.
#pragma once
#include <type_traits>

#include "tess_math.cuh"

namespace tess {

// Single-leg currents are polarisation vectors of the helicity basis, whose
// components eps^0 and Im eps^3 are exact zeros (e1 and e2 have no time
// component, e2 no z component).  Where a part of a split or a triple is a
// single leg (a "leaf"), the products with those components are left out:
// each would add an exact +-0 to a finite partial sum, so the results are the
// full products' (up to the sign of an exactly zero sum).  LA / LB: a / b is
// a leaf.  The order of the remaining operations is that of mdot / axpy.
template <bool LA, bool LB, typename R>
__device__ __forceinline__ Cx<R> mdot_l(const CV4<R> &a, const CV4<R> &b) {
  R re, im;
  if constexpr (!LA && !LB) {
    re = a.c[0].re * b.c[0].re;
    im = a.c[0].re * b.c[0].im;
    re = fma(-a.c[0].im, b.c[0].im, re);
    im = fma(a.c[0].im, b.c[0].re, im);
  } else {
    re = -a.c[1].re * b.c[1].re;
    im = -a.c[1].re * b.c[1].im;
  }
#pragma unroll
  for (int m = 1; m < 4; ++m) {
    const bool first = (LA || LB) && m == 1;  // its leading products are already in re, im
    if (!first) re = fma(-a.c[m].re, b.c[m].re, re);
    if (m < 3 || (!LA && !LB)) re = fma(a.c[m].im, b.c[m].im, re);
    if (!first && (m < 3 || !LB)) im = fma(-a.c[m].re, b.c[m].im, im);
    if (m < 3 || !LA) im = fma(-a.c[m].im, b.c[m].re, im);
  }
  return cx<R>(re, im);
}

// leaf a (complex) . k (real)
template <typename R>
__device__ __forceinline__ Cx<R> mdot_leaf(const CV4<R> &a, const RV4<R> &k) {
  R re = -a.c[1].re * k.v[1];
  R im = -a.c[1].im * k.v[1];
  re = fma(-a.c[2].re, k.v[2], re);
  im = fma(-a.c[2].im, k.v[2], im);
  re = fma(-a.c[3].re, k.v[3], re);
  return cx<R>(re, im);
}

// acc += s * v for a leaf v
template <typename R>
__device__ __forceinline__ void axpy_leaf(CV4<R> &acc, const Cx<R> &s, const CV4<R> &v) {
#pragma unroll
  for (int m = 1; m < 4; ++m) {
    acc.c[m].re = fma(s.re, v.c[m].re, acc.c[m].re);
    if (m < 3) acc.c[m].re = fma(-s.im, v.c[m].im, acc.c[m].re);
    if (m < 3) acc.c[m].im = fma(s.re, v.c[m].im, acc.c[m].im);
    acc.c[m].im = fma(s.im, v.c[m].re, acc.c[m].im);
  }
}

// f(integral_constant<la>, integral_constant<lb>) for runtime flags that are
// constants after unrolling (so only one branch survives)
template <typename F>
__device__ __forceinline__ auto leaf_sel(bool la, bool lb, F &&f) {
  if (la && lb) return f(std::true_type{}, std::true_type{});
  if (la) return f(std::true_type{}, std::false_type{});
  if (lb) return f(std::false_type{}, std::true_type{});
  return f(std::false_type{}, std::false_type{});
}

template <typename R, int L>
struct BGTables {
  CV4<R> J[L][L];  // J[a][b], a <= b: current of legs a..b
  RV4<R> K[L][L];  // K[a][b]: sum of the momenta of legs a..b
  Cx<R> S[L][L];   // S[a][b]: sum over splits of J_l . J_r (b > a)
};

// Un-propagated top current Num = K^2 J[0..L-1] for leg momenta k[0..L) and
// polarisations e[0..L) (already in the colour order), then the amplitude
// m = e0 . Num (amplitude equation of Sec. 3, leg 1 off-shell).
template <typename R, int L>
__device__ __forceinline__ Cx<R> bg_amplitude(const RV4<R> (&k)[L], const CV4<R> (&e)[L], const CV4<R> &e0) {
  BGTables<R, L> t;
#pragma unroll
  for (int a = 0; a < L; ++a) {
    t.J[a][a] = e[a];
    t.K[a][a] = k[a];
  }
  CV4<R> num = cv_zero<R>();
#pragma unroll
  for (int len = 2; len <= L; ++len) {
#pragma unroll
    for (int a = 0; a + len - 1 < L; ++a) {
      const int b = a + len - 1;
      t.K[a][b] = radd(t.K[a][b - 1], k[b]);
      CV4<R> acc = cv_zero<R>();
      CV4<R> tri = cv_zero<R>();
      Cx<R> s = cx<R>(R(0), R(0));
#pragma unroll
      for (int i = a; i < b; ++i) {
        // split l = [a..i], r = [i+1..b] (leaves: i == a, i + 1 == b)
        const CV4<R> &Jl = t.J[a][i];
        const CV4<R> &Jr = t.J[i + 1][b];
        const bool ll = i == a, lr = i + 1 == b;
        const Cx<R> d = leaf_sel(ll, lr, [&](auto la, auto lb) { return mdot_l<decltype(la)::value, decltype(lb)::value>(Jl, Jr); });
        const Cx<R> jlkr = ll ? mdot_leaf(Jl, t.K[i + 1][b]) : mdot(Jl, t.K[i + 1][b]);
        const Cx<R> krjl = lr ? mdot_leaf(Jr, t.K[a][i]) : mdot(Jr, t.K[a][i]);
        Cx<R> cr = cx<R>(R(2) * jlkr.re, R(2) * jlkr.im);
        Cx<R> cl = cx<R>(R(-2) * krjl.re, R(-2) * krjl.im);
        if (i > a) {
          cr.re -= t.S[a][i].re;
          cr.im -= t.S[a][i].im;
        }
        if (b > i + 1) {
          cl.re -= t.S[i + 1][b].re;
          cl.im -= t.S[i + 1][b].im;
        }
        if (lr)
          axpy_leaf(acc, cr, Jr);
        else
          axpy(acc, cr, Jr);
        if (ll)
          axpy_leaf(acc, cl, Jl);
        else
          axpy(acc, cl, Jl);
        axpy(acc, d, rsub(t.K[a][i], t.K[i + 1][b]));
        s.re += d.re;
        s.im += d.im;
      }
#pragma unroll
      for (int i = a; i + 1 < b; ++i) {
#pragma unroll
        for (int j = i + 1; j < b; ++j) {
          // triple ([a..i], [i+1..j], [j+1..b]): leaves i == a, j == i + 1, j + 1 == b
          const Cx<R> x = leaf_sel(i == a, j + 1 == b, [&](auto la, auto lb) {
            return mdot_l<decltype(la)::value, decltype(lb)::value>(t.J[a][i], t.J[j + 1][b]);
          });
          if (j == i + 1)
            axpy_leaf(tri, x, t.J[i + 1][j]);
          else
            axpy(tri, x, t.J[i + 1][j]);
        }
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        acc.c[m].re = fma(R(2), tri.c[m].re, acc.c[m].re);
        acc.c[m].im = fma(R(2), tri.c[m].im, acc.c[m].im);
      }
      if (len < L) {
        const R inv = R(1) / mdot(t.K[a][b], t.K[a][b]);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          t.J[a][b].c[m].re = acc.c[m].re * inv;
          t.J[a][b].c[m].im = acc.c[m].im * inv;
        }
        t.S[a][b] = s;
      } else {
        num = acc;
      }
    }
  }
  return mdot_l<true, false>(e0, num);  // e0: leg 0's polarisation vector
}

// The same recursion with real polarisation vectors (Sec. 3's random real
// polarisations): every current is then a real four-vector, so each complex
// multiply-add of the helicity form becomes one real FMA.  Same splits, same
// reorganised four-vertex sum, same operation order per component.
template <typename R>
__device__ __forceinline__ void raxpy(RV4<R> &acc, R s, const RV4<R> &v) {
#pragma unroll
  for (int m = 0; m < 4; ++m) acc.v[m] = fma(s, v.v[m], acc.v[m]);
}

// Real polarisation vectors cos(phi) e1 + sin(phi) e2 have eps^0 = 0
// exactly: where a part is a single leg its time component is left out
// (products with an exact zero; the same argument as mdot_l).
template <bool LA, bool LB, typename R>
__device__ __forceinline__ R rdot_l(const RV4<R> &a, const RV4<R> &b) {
  R s;
  if constexpr (!LA && !LB) {
    s = a.v[0] * b.v[0];
    s = fma(-a.v[1], b.v[1], s);
  } else {
    s = -a.v[1] * b.v[1];
  }
  s = fma(-a.v[2], b.v[2], s);
  s = fma(-a.v[3], b.v[3], s);
  return s;
}

template <typename R>
__device__ __forceinline__ void raxpy_leaf(RV4<R> &acc, R s, const RV4<R> &v) {
#pragma unroll
  for (int m = 1; m < 4; ++m) acc.v[m] = fma(s, v.v[m], acc.v[m]);
}

template <typename R, int L>
__device__ __forceinline__ R bg_amplitude_real(const RV4<R> (&k)[L], const RV4<R> (&e)[L], const RV4<R> &e0) {
  RV4<R> J[L][L], K[L][L];
  R S[L][L];
#pragma unroll
  for (int a = 0; a < L; ++a) {
    J[a][a] = e[a];
    K[a][a] = k[a];
  }
  RV4<R> num = {{R(0), R(0), R(0), R(0)}};
#pragma unroll
  for (int len = 2; len <= L; ++len) {
#pragma unroll
    for (int a = 0; a + len - 1 < L; ++a) {
      const int b = a + len - 1;
      K[a][b] = radd(K[a][b - 1], k[b]);
      RV4<R> acc = {{R(0), R(0), R(0), R(0)}}, tri = {{R(0), R(0), R(0), R(0)}};
      R sum = R(0);
#pragma unroll
      for (int i = a; i < b; ++i) {
        // split l = [a..i], r = [i+1..b]
        const RV4<R> &Jl = J[a][i];
        const RV4<R> &Jr = J[i + 1][b];
        const bool ll = i == a, lr = i + 1 == b;  // single-leg parts
        const R d = leaf_sel(ll, lr, [&](auto la, auto lb) {
          return rdot_l<decltype(la)::value, decltype(lb)::value>(Jl, Jr);
        });
        R cr = R(2) * (ll ? rdot_l<true, false>(Jl, K[i + 1][b]) : mdot(Jl, K[i + 1][b]));
        R cl = R(-2) * (lr ? rdot_l<true, false>(Jr, K[a][i]) : mdot(Jr, K[a][i]));
        if (i > a) cr -= S[a][i];
        if (b > i + 1) cl -= S[i + 1][b];
        if (lr)
          raxpy_leaf(acc, cr, Jr);
        else
          raxpy(acc, cr, Jr);
        if (ll)
          raxpy_leaf(acc, cl, Jl);
        else
          raxpy(acc, cl, Jl);
        raxpy(acc, d, rsub(K[a][i], K[i + 1][b]));
        sum += d;
      }
#pragma unroll
      for (int i = a; i + 1 < b; ++i) {
#pragma unroll
        for (int j = i + 1; j < b; ++j) {
          const R x = leaf_sel(i == a, j + 1 == b, [&](auto la, auto lb) {
            return rdot_l<decltype(la)::value, decltype(lb)::value>(J[a][i], J[j + 1][b]);
          });
          if (j == i + 1)
            raxpy_leaf(tri, x, J[i + 1][j]);
          else
            raxpy(tri, x, J[i + 1][j]);
        }
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) acc.v[m] = fma(R(2), tri.v[m], acc.v[m]);
      if (len < L) {
        const R inv = R(1) / mdot(K[a][b], K[a][b]);
#pragma unroll
        for (int m = 0; m < 4; ++m) J[a][b].v[m] = acc.v[m] * inv;
        S[a][b] = sum;
      } else {
        num = acc;
      }
    }
  }
  return rdot_l<true, false>(e0, num);  // e0: leg 0's polarisation vector
}

// ---------------------------------------------------------------------------
// Loop form of the same recursion for large tables (FP64, and FP32 with
// n >= 8): runtime loops over lengths, sets and splits, the table in
// per-thread local memory indexed by tri(a, b).  Compiles in O(1) code size.
// The caller fills the single-leg entries J[tri(a,a)] (polarisations) and
// K[tri(a,a)] (momenta) in colour order, then calls run().
// ---------------------------------------------------------------------------
template <typename R, int L>
struct BGLoop {
  static constexpr int T = L * (L + 1) / 2;
  CV4<R> J[T];
  RV4<R> K[T];
  Cx<R> S[T];

  __device__ __forceinline__ static int tri(int a, int b) { return a * L - (a * (a - 1)) / 2 + (b - a); }

  __device__ Cx<R> run(const CV4<R> &e0) {
#pragma unroll 1
    for (int a = 0; a < L; ++a) S[tri(a, a)] = cx<R>(R(0), R(0));
    CV4<R> num = cv_zero<R>();
#pragma unroll 1
    for (int len = 2; len <= L; ++len) {
#pragma unroll 1
      for (int a = 0; a + len - 1 < L; ++a) {
        const int b = a + len - 1;
        const int X = tri(a, b);
        K[X] = radd(K[tri(a, b - 1)], K[tri(b, b)]);
        CV4<R> acc = cv_zero<R>();
        CV4<R> trs = cv_zero<R>();
        Cx<R> s = cx<R>(R(0), R(0));
#pragma unroll 1
        for (int i = a; i < b; ++i) {
          const int l = tri(a, i), r = tri(i + 1, b);
          const CV4<R> Jl = J[l], Jr = J[r];
          const RV4<R> Kl = K[l], Kr = K[r];
          const Cx<R> d = mdot(Jl, Jr);
          const Cx<R> jlkr = mdot(Jl, Kr);
          const Cx<R> krjl = mdot(Jr, Kl);
          const Cx<R> Sl = S[l], Sr = S[r];
          const Cx<R> cr = cx<R>(fma(R(2), jlkr.re, -Sl.re), fma(R(2), jlkr.im, -Sl.im));
          const Cx<R> cl = cx<R>(fma(R(-2), krjl.re, -Sr.re), fma(R(-2), krjl.im, -Sr.im));
          axpy(acc, cr, Jr);
          axpy(acc, cl, Jl);
          axpy(acc, d, rsub(Kl, Kr));
          s.re += d.re;
          s.im += d.im;
        }
#pragma unroll 1
        for (int i = a; i + 1 < b; ++i) {
          const CV4<R> JA = J[tri(a, i)];
#pragma unroll 1
          for (int j = i + 1; j < b; ++j) axpy(trs, mdot(JA, J[tri(j + 1, b)]), J[tri(i + 1, j)]);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          acc.c[m].re = fma(R(2), trs.c[m].re, acc.c[m].re);
          acc.c[m].im = fma(R(2), trs.c[m].im, acc.c[m].im);
        }
        if (len < L) {
          const R inv = R(1) / mdot(K[X], K[X]);
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            J[X].c[m].re = acc.c[m].re * inv;
            J[X].c[m].im = acc.c[m].im * inv;
          }
          S[X] = s;
        } else {
          num = acc;
        }
      }
    }
    return mdot(e0, num);
  }
};

}  // namespace tess
