// Event weights and their gradients (reverse mode, written by hand):
//   w(u) for caller-given uniforms u = (u_x1, u_x2, Rambo 4m), fixed helicity
//   labels and colour ordering;
//   dw/du (total derivative), dw/dk at fixed x1, x2 (all-outgoing momentum
//   components, polarisation vectors and K-sums varying with k), and
//   dw/d ln mu_R.
// Kinematics and their adjoints run in FP64; the Berends-Giele forward pass
// and its adjoint in R (float or double).  Cuts enter as a step function
// (zero derivative almost everywhere): failing events have w = 0 and zero
// gradients.
#pragma once
#include <cstdint>

#include "tess_bg.cuh"
#include "tess_event.cuh"
#include "tess_kernels.cuh"

namespace tess {

struct GradParams {
  EventParams P;  // process constants (seed/first_event unused)
  const double *u;
  const uint32_t *hel;
  const uint8_t *order;
  double *w, *dw_du, *dw_dk, *dw_dlnmu;
  const double *dL_dw;  // optional upstream gradient
  uint64_t n_events;
  size_t chunk_bytes;  // bytes per chunk buffer of the FP32 split pipeline (0 = default)
};

// Streams and events of the overlapped split pipeline of the FP32 forms
// (aux == nullptr: all stages on the caller's stream).
struct GradStreams {
  cudaStream_t aux = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t g2done[2] = {nullptr, nullptr}, g3done[2] = {nullptr, nullptr};
};

// Berends-Giele forward pass and adjoint of f = |m|^2 for one ordering.
// Inputs in colour-position order: k[a], eps[a] (a = 0..L-1), e0.  Outputs
// the gradients g_k[a] (real), g_eps[a], g_e0 in the convention
// g(z) = df/dRe z + i df/dIm z, and returns f.
template <typename R, int L>
struct BGAdjoint {
  static constexpr int T = L * (L + 1) / 2;
  CV4<R> J[T], GJ[T];
  RV4<R> K[T], GK[T];
  Cx<R> S[T], GS[T];
  CV4<R> num;

  __device__ __forceinline__ static int tri(int a, int b) { return a * L - (a * (a - 1)) / 2 + (b - a); }

  __device__ void forward() {
#pragma unroll 1
    for (int a = 0; a < L; ++a) S[tri(a, a)] = cx<R>(R(0), R(0));
#pragma unroll 1
    for (int len = 2; len <= L; ++len) {
#pragma unroll 1
      for (int a = 0; a + len - 1 < L; ++a) {
        const int b = a + len - 1, X = tri(a, b);
        K[X] = radd(K[tri(a, b - 1)], K[tri(b, b)]);
        CV4<R> acc = cv_zero<R>();
        Cx<R> s = cx<R>(R(0), R(0));
#pragma unroll 1
        for (int i = a; i < b; ++i) {
          const int l = tri(a, i), r = tri(i + 1, b);
          const Cx<R> d = mdot(J[l], J[r]);
          const Cx<R> jlkr = mdot(J[l], K[r]);
          const Cx<R> krjl = mdot(J[r], K[l]);
          const Cx<R> cr = cx<R>(R(2) * jlkr.re - S[l].re, R(2) * jlkr.im - S[l].im);
          const Cx<R> cl = cx<R>(R(-2) * krjl.re - S[r].re, R(-2) * krjl.im - S[r].im);
          axpy(acc, cr, J[r]);
          axpy(acc, cl, J[l]);
          axpy(acc, d, rsub(K[l], K[r]));
          s.re += d.re;
          s.im += d.im;
        }
#pragma unroll 1
        for (int i = a; i + 1 < b; ++i)
#pragma unroll 1
          for (int j = i + 1; j < b; ++j) {
            const Cx<R> t = mdot(J[tri(a, i)], J[tri(j + 1, b)]);
            axpy(acc, cx<R>(R(2) * t.re, R(2) * t.im), J[tri(i + 1, j)]);
          }
        if (len < L) {
          const R inv = R(1) / mdot(K[X], K[X]);
#pragma unroll
          for (int m = 0; m < 4; ++m) J[X].c[m] = cx<R>(acc.c[m].re * inv, acc.c[m].im * inv);
          S[X] = s;
        } else {
          num = acc;
        }
      }
    }
  }

  // helpers for adjoints: g(a) += conj(c) * G (component-wise), Re(conj(c) G)
  __device__ __forceinline__ static void add_conj_scaled(CV4<R> &g, const Cx<R> &c, const CV4<R> &G) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      g.c[m].re += c.re * G.c[m].re + c.im * G.c[m].im;
      g.c[m].im += c.re * G.c[m].im - c.im * G.c[m].re;
    }
  }
  // sum_m conj(v^m) G^m (plain component sum)
  __device__ __forceinline__ static Cx<R> conj_dot(const CV4<R> &v, const CV4<R> &G) {
    R re = 0, im = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      re += v.c[m].re * G.c[m].re + v.c[m].im * G.c[m].im;
      im += v.c[m].re * G.c[m].im - v.c[m].im * G.c[m].re;
    }
    return cx<R>(re, im);
  }
  // adjoint of z = a.b (Minkowski, complex a, b): g(a^m) += eta_m conj(b^m) g(z)
  __device__ __forceinline__ static void dot_adj(CV4<R> &ga, const CV4<R> &b, const Cx<R> &gz) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const R e = m == 0 ? R(1) : R(-1);
      ga.c[m].re += e * (b.c[m].re * gz.re + b.c[m].im * gz.im);
      ga.c[m].im += e * (b.c[m].re * gz.im - b.c[m].im * gz.re);
    }
  }
  // adjoint of z = a.K (complex a, real K): g(a) += eta K g(z); g(K^m) += Re(eta conj(a^m) g(z))
  __device__ __forceinline__ static void dot_adj_ck(CV4<R> &ga, RV4<R> &gK, const CV4<R> &a, const RV4<R> &K,
                                                    const Cx<R> &gz) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const R e = m == 0 ? R(1) : R(-1);
      ga.c[m].re += e * K.v[m] * gz.re;
      ga.c[m].im += e * K.v[m] * gz.im;
      gK.v[m] += e * (a.c[m].re * gz.re + a.c[m].im * gz.im);
    }
  }

  // Reverse sweep.  g_m = df/dm (complex, f = |m|^2 gives 2m).  Leaves the
  // gradients of the single-leg entries in GJ[tri(a,a)], GK[tri(a,a)].
  __device__ void adjoint(const CV4<R> &e0, const Cx<R> &gm, CV4<R> &g_e0) {
#pragma unroll 1
    for (int X = 0; X < T; ++X) {
      GJ[X] = cv_zero<R>();
      GS[X] = cx<R>(R(0), R(0));
#pragma unroll
      for (int m = 0; m < 4; ++m) GK[X].v[m] = R(0);
    }
    // m = sum_m eta_m e0^m num^m
    g_e0 = cv_zero<R>();
    CV4<R> gtop = cv_zero<R>();
    dot_adj(g_e0, num, gm);
    dot_adj(gtop, e0, gm);
#pragma unroll 1
    for (int len = L; len >= 2; --len) {
#pragma unroll 1
      for (int a = 0; a + len - 1 < L; ++a) {
        const int b = a + len - 1, X = tri(a, b);
        CV4<R> G;  // adjoint of the un-propagated sum acc_X
        if (len == L) {
          G = gtop;
        } else {
          const R k2 = mdot(K[X], K[X]);
          const R inv = R(1) / k2;
#pragma unroll
          for (int m = 0; m < 4; ++m) G.c[m] = cx<R>(GJ[X].c[m].re * inv, GJ[X].c[m].im * inv);
          // inv = 1/K^2: g(inv) = Re sum conj(acc) g(J) = K^2 Re sum conj(J) g(J)
          const Cx<R> cj = conj_dot(J[X], GJ[X]);
          const R ginv = k2 * cj.re;
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const R e = m == 0 ? R(1) : R(-1);
            GK[X].v[m] += ginv * (-inv * inv) * R(2) * e * K[X].v[m];
          }
        }
        const Cx<R> gsX = GS[X];
#pragma unroll 1
        for (int i = a; i < b; ++i) {
          const int l = tri(a, i), r = tri(i + 1, b);
          const Cx<R> d = mdot(J[l], J[r]);
          const Cx<R> jlkr = mdot(J[l], K[r]);
          const Cx<R> krjl = mdot(J[r], K[l]);
          const Cx<R> cr = cx<R>(R(2) * jlkr.re - S[l].re, R(2) * jlkr.im - S[l].im);
          const Cx<R> cl = cx<R>(R(-2) * krjl.re - S[r].re, R(-2) * krjl.im - S[r].im);
          // acc += cr J_r + cl J_l + d (K_l - K_r); s += d
          const Cx<R> gcr = conj_dot(J[r], G);
          const Cx<R> gcl = conj_dot(J[l], G);
          add_conj_scaled(GJ[r], cr, G);
          add_conj_scaled(GJ[l], cl, G);
          RV4<R> dk = rsub(K[l], K[r]);
          Cx<R> gd = cx<R>(gsX.re, gsX.im);
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            gd.re += dk.v[m] * G.c[m].re;
            gd.im += dk.v[m] * G.c[m].im;
            const R gk = d.re * G.c[m].re + d.im * G.c[m].im;  // Re(conj(d) G^m)
            GK[l].v[m] += gk;
            GK[r].v[m] -= gk;
          }
          // cr = 2 jlkr - S_l ; cl = -2 krjl - S_r
          GS[l].re -= gcr.re;
          GS[l].im -= gcr.im;
          GS[r].re -= gcl.re;
          GS[r].im -= gcl.im;
          const Cx<R> gjlkr = cx<R>(R(2) * gcr.re, R(2) * gcr.im);
          const Cx<R> gkrjl = cx<R>(R(-2) * gcl.re, R(-2) * gcl.im);
          dot_adj_ck(GJ[l], GK[r], J[l], K[r], gjlkr);
          dot_adj_ck(GJ[r], GK[l], J[r], K[l], gkrjl);
          dot_adj(GJ[l], J[r], gd);
          dot_adj(GJ[r], J[l], gd);
        }
#pragma unroll 1
        for (int i = a; i + 1 < b; ++i)
#pragma unroll 1
          for (int j = i + 1; j < b; ++j) {
            const int A = tri(a, i), B = tri(i + 1, j), C = tri(j + 1, b);
            const Cx<R> t = mdot(J[A], J[C]);
            // acc += 2 t J_B
            const Cx<R> gt0 = conj_dot(J[B], G);
            const Cx<R> gt = cx<R>(R(2) * gt0.re, R(2) * gt0.im);
            add_conj_scaled(GJ[B], cx<R>(R(2) * t.re, R(2) * t.im), G);
            dot_adj(GJ[A], J[C], gt);
            dot_adj(GJ[C], J[A], gt);
          }
        // K_X = K[a][b-1] + k_b
        const RV4<R> gK = GK[X];
        GK[tri(a, b - 1)] = radd(GK[tri(a, b - 1)], gK);
        GK[tri(b, b)] = radd(GK[tri(b, b)], gK);
      }
    }
  }
};

// Gradient of the polarisation vector of direction p (3-vector, FP64) with
// respect to p: g_p += Re sum conj(d eps / d p) g_eps for eps = eps_{+/-}.
template <typename T>
__device__ __forceinline__ void polvec_adjoint(const T (&p)[3], bool minus, const T (&ge_re)[4], const T (&ge_im)[4],
                                               T (&gp)[3]) {
  const T px = p[0], py = p[1], pz = p[2];
  const T pt2 = px * px + py * py;
  const T pt = sqrt(pt2), r = sqrt(pt2 + pz * pz);
  if (!(pt > T(0))) return;  // beam axis: the basis is fixed by convention
  const T ct = pz / r, cf = px / pt, sf = py / pt;
  const T s2 = T(0.70710678118654752440);
  // Re eps = sgn e1 / sqrt2, Im eps = -e2 / sqrt2 with sgn = -1 (eps_+) or +1 (eps_-)
  const T sg = minus ? T(1) : T(-1);
  const T G1x = sg * s2 * ge_re[1], G1y = sg * s2 * ge_re[2], G1z = sg * s2 * ge_re[3];
  const T G2x = -s2 * ge_im[1], G2y = -s2 * ge_im[2];
  // e1 = (ct cf, ct sf, -st), e2 = (-sf, cf, 0)
  const T g_ct = G1x * cf + G1y * sf;
  const T g_cf = G1x * ct + G2y;
  const T g_sf = G1y * ct - G2x;
  const T g_st = -G1z;
  const T r3 = r * r * r, pt3 = pt2 * pt;
  gp[0] += g_ct * (-pz * px / r3) + g_st * (px / (pt * r) - pt * px / r3) + g_cf * (T(1) / pt - px * px / pt3) +
           g_sf * (-px * py / pt3);
  gp[1] += g_ct * (-pz * py / r3) + g_st * (py / (pt * r) - pt * py / r3) + g_cf * (-px * py / pt3) +
           g_sf * (T(1) / pt - py * py / pt3);
  gp[2] += g_ct * (T(1) / r - pz * pz / r3) + g_st * (-pt * pz / r3);
}

}  // namespace tess

namespace tess {

// Kinematics of one event for the gradient kernels, with every intermediate
// the reverse sweep needs (T: the FP32-split type, see grad_kinematics).
template <int N, typename T>
struct GradKin {
  static constexpr int M = N - 2;
  T tx1, tx2, tht;
  double x1, x2, shat, rs, ht, c, Q0, Q1, Q2, Q3, Mq, gam, aa, xs;
  double q[M][4], cth[M], sth[M], cph[M], sph[M], q0v[M], bv[3], kk[N][4], bq[M], fq[M], kp[N][4];
  int legp[N];
  int pass;
};

// Forward kinematics of one event from its uniforms u (x1, x2, Rambo 4m) and
// colour order: x, Rambo (keeping its intermediates), cuts, observables, the
// colour-ordered momenta and the exact power-of-two momentum unit c of the
// amplitude.  Precision split of the FP32-current forms (as the kinematics
// kernel): x, the Rambo seeds, cuts, observables, alpha_s, PDF and the
// polarisation basis in T; the boost/rescale and the weight scalings in FP64
// (T = double: everything FP64).
template <int N, typename T>
__device__ __forceinline__ void grad_kinematics(const EventParams &P, const double *u, const uint8_t *order,
                                                GradKin<N, T> &K) {
  constexpr int M = N - 2;
  const T lnx = (T)P.lnxmin;
  const T tx1 = exp((T)u[0] * lnx), tx2 = exp((T)u[1] * lnx);
  const double x1 = tx1, x2 = tx2;
  const double shat = x1 * x2 * P.S, rs = sqrt(shat);
  double q[M][4], cth[M], sth[M], cph[M], sph[M], q0v[M];
  double Q0 = 0, Q1 = 0, Q2 = 0, Q3 = 0;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const T c = T(2) * (T)u[2 + 4 * i] - T(1);
    const T s = sqrt(T(1) - c * c);
    T sn, cs;
    sincospi(T(2) * (T)u[2 + 4 * i + 1], &sn, &cs);
    const T q0 = -log((T)u[2 + 4 * i + 2] * (T)u[2 + 4 * i + 3]);
    cth[i] = c; sth[i] = s; cph[i] = cs; sph[i] = sn; q0v[i] = q0;
    q[i][0] = q0; q[i][1] = q0 * s * cs; q[i][2] = q0 * s * sn; q[i][3] = q0 * c;
    Q0 += q[i][0]; Q1 += q[i][1]; Q2 += q[i][2]; Q3 += q[i][3];
  }
  const double Mq = sqrt(Q0 * Q0 - Q1 * Q1 - Q2 * Q2 - Q3 * Q3);
  const double iMq = 1.0 / Mq;
  const double bv[3] = {-Q1 * iMq, -Q2 * iMq, -Q3 * iMq};
  const double gam = Q0 * iMq, aa = 1.0 / (1.0 + gam), xs = rs * iMq;
  double kk[N][4];
  const double h = 0.5 * rs;
  kk[0][0] = -h; kk[0][1] = 0.0; kk[0][2] = 0.0; kk[0][3] = -h;
  kk[1][0] = -h; kk[1][1] = 0.0; kk[1][2] = 0.0; kk[1][3] = h;
  double bq[M], fq[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    bq[i] = bv[0] * q[i][1] + bv[1] * q[i][2] + bv[2] * q[i][3];
    fq[i] = aa * bq[i] + q[i][0];
    kk[2 + i][0] = xs * (gam * q[i][0] + bq[i]);
#pragma unroll
    for (int j = 0; j < 3; ++j) kk[2 + i][1 + j] = xs * (q[i][1 + j] + bv[j] * fq[i]);
  }
  const T y = T(0.5) * lnx * ((T)u[0] - (T)u[1]);  // 0.5 ln(x1 / x2)
  int pass = 1;
  T tht = T(0), eta[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const T px = (T)kk[2 + i][1], py = (T)kk[2 + i][2], pz = (T)kk[2 + i][3];
    const T pt = sqrt(px * px + py * py), pa = sqrt(px * px + py * py + pz * pz);
    eta[i] = T(0.5) * log((pa + pz) / (pa - pz)) + y;
    tht += pt;
    pass &= (pt > (T)P.pt_min) & (fabs(eta[i]) < (T)P.eta_max);
  }
#pragma unroll
  for (int i = 0; i < M; ++i)
#pragma unroll
    for (int j = i + 1; j < M; ++j) {
      const T pxi = (T)kk[2 + i][1], pyi = (T)kk[2 + i][2], pxj = (T)kk[2 + j][1], pyj = (T)kk[2 + j][2];
      const T dphi = atan2(fabs(pxi * pyj - pyi * pxj), pxi * pxj + pyi * pyj);
      const T de = eta[i] - eta[j];
      pass &= (de * de + dphi * dphi > (T)P.dr2_min);
    }
  const double ht = tht;

  // ---- colour order and the momentum unit of the amplitude (exact power of two)
  int perm[N];
#pragma unroll
  for (int i = 0; i < N; ++i) perm[i] = order[i];
  double kp[N][4];
  int legp[N];
  gather_positions<N>(kk, perm, kp, legp);
  const double c = pow2_unit_inv(rs);
  K.tx1 = tx1;
  K.tx2 = tx2;
  K.tht = tht;
  K.x1 = x1;
  K.x2 = x2;
  K.shat = shat;
  K.rs = rs;
  K.ht = ht;
  K.c = c;
  K.Q0 = Q0;
  K.Q1 = Q1;
  K.Q2 = Q2;
  K.Q3 = Q3;
  K.Mq = Mq;
  K.gam = gam;
  K.aa = aa;
  K.xs = xs;
  K.pass = pass;
#pragma unroll
  for (int i = 0; i < M; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) K.q[i][m] = q[i][m];
#pragma unroll
  for (int i = 0; i < M; ++i) K.cth[i] = cth[i];
#pragma unroll
  for (int i = 0; i < M; ++i) K.sth[i] = sth[i];
#pragma unroll
  for (int i = 0; i < M; ++i) K.cph[i] = cph[i];
#pragma unroll
  for (int i = 0; i < M; ++i) K.sph[i] = sph[i];
#pragma unroll
  for (int i = 0; i < M; ++i) K.q0v[i] = q0v[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) K.bv[i] = bv[i];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) K.kk[i][m] = kk[i][m];
#pragma unroll
  for (int i = 0; i < M; ++i) K.bq[i] = bq[i];
#pragma unroll
  for (int i = 0; i < M; ++i) K.fq[i] = fq[i];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) K.kp[i][m] = kp[i][m];
#pragma unroll
  for (int i = 0; i < N; ++i) K.legp[i] = legp[i];
}

// Amplitude inputs of colour position a: the momentum in the unit c and the
// polarisation vector of its helicity label (position 0: eps only is used).
template <int N, typename R, typename T>
__device__ __forceinline__ void grad_amp_input(const GradKin<N, T> &K, uint32_t hel, int a, RV4<R> &k, CV4<R> &eps) {
  CV4<R> ep, em;
  const T sg = K.legp[a] < 2 ? T(-1) : T(1);
  polarisations<R, T>(sg * (T)K.kp[a][1], sg * (T)K.kp[a][2], sg * (T)K.kp[a][3], ep, em);
  eps = ((hel >> K.legp[a]) & 1u) ? em : ep;
#pragma unroll
  for (int m = 0; m < 4; ++m) k.v[m] = R(K.kp[a][m] * K.c);
}

// Weights and gradients of one event from its kinematics and the amplitude
// stage's result: f = |m|^2 and, through get(a, g4, ge) for every colour
// position a, df/dk of the position's momentum in the unit c (g4; zero for
// position 0, whose momentum the amplitude does not take) and df/d eps (ge,
// convention g(z) = df/dRe z + i df/dIm z).  Writes w, dw/du, dw/dk,
// dw/dlnmu of event e.
template <int N, typename R, typename T, typename Get>
__device__ __forceinline__ void grad_outputs(const GradParams &G, uint64_t e, const GradKin<N, T> &K, uint32_t hel,
                                             double f, Get get) {
  constexpr int M = N - 2, L = N - 1, NU = 2 + 4 * M;
  const EventParams &P = G.P;
  const double *u = G.u + e * NU;
  const T tx1 = K.tx1;
  const T tx2 = K.tx2;
  const T tht = K.tht;
  const double x1 = K.x1;
  const double x2 = K.x2;
  const double shat = K.shat;
  const double rs = K.rs;
  const double ht = K.ht;
  const double c = K.c;
  const double Q0 = K.Q0;
  const double Q1 = K.Q1;
  const double Q2 = K.Q2;
  const double Q3 = K.Q3;
  const double Mq = K.Mq;
  const double gam = K.gam;
  const double aa = K.aa;
  const double xs = K.xs;
  const int pass = K.pass;
  const double(&q)[M][4] = K.q;
  const double(&cth)[M] = K.cth;
  const double(&sth)[M] = K.sth;
  const double(&cph)[M] = K.cph;
  const double(&sph)[M] = K.sph;
  const double(&q0v)[M] = K.q0v;
  const double(&bv)[3] = K.bv;
  const double(&kk)[N][4] = K.kk;
  const double(&bq)[M] = K.bq;
  const double(&fq)[M] = K.fq;
  const double(&kp)[N][4] = K.kp;
  const int(&legp)[N] = K.legp;
  double ufac = P.efac;  // E = efac c^(2(N-4)) f
#pragma unroll
  for (int i = 0; i < N - 4; ++i) ufac *= c * c;
  const double E = ufac * f;

  // ---- dE/dk per leg (k unscaled): K-sum path and polarisation path
  double gk[N][4];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) gk[i][m] = 0.0;
#pragma unroll
  for (int a = 0; a <= L; ++a) {
    const int leg = legp[a];
    double g4[4] = {0, 0, 0, 0};
    CV4<R> ge;
    get(a, g4, ge);
    const double sg = leg < 2 ? -1.0 : 1.0;
    const T pphys[3] = {T(sg * kp[a][1]), T(sg * kp[a][2]), T(sg * kp[a][3])};
    T gre[4], gim[4], gp[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      gre[m] = (T)ge.c[m].re;
      gim[m] = (T)ge.c[m].im;
    }
    polvec_adjoint<T>(pphys, (hel >> leg) & 1u, gre, gim, gp);
    // f depends on k' = c k through the K sums (g4) and on the direction of k
    // through eps (gp, scale-free)
    const double scale = ufac * c;
#pragma unroll
    for (int s2 = 0; s2 < N; ++s2) {
      if (s2 == leg) {
        gk[s2][0] += scale * g4[0];
#pragma unroll
        for (int j = 0; j < 3; ++j) gk[s2][1 + j] += scale * g4[1 + j] + ufac * sg * gp[j];
      }
    }
  }

  // ---- weight, and its gradients
  double w = 0.0, gw_lnmu = 0.0, wfac = 0.0, dwfac_dht = 0.0, as = 0.0;
  if (pass) {
    const T mu = (T)P.mu_r_factor * tht;
    as = (T)P.alphas_mz / (T(1) + (T)P.alphas_mz * (T)P.b0 * (log(mu * mu) - (T)P.ln_mz2));
    const double g2 = 4.0 * 3.14159265358979323846 * as;
    double gp_ = 1.0, sp = 1.0;
#pragma unroll
    for (int i = 0; i < N - 2; ++i) gp_ *= g2;
#pragma unroll
    for (int i = 0; i < M - 2; ++i) sp *= shat;
    const double f1 = T(1.7) * pow(tx1, T(-0.2)) * pow(T(1) - tx1, T(5)),
                 f2 = T(1.7) * pow(tx2, T(-0.2)) * pow(T(1) - tx2, T(5));
    wfac = P.wconst * (P.lnxmin * P.lnxmin * f1 * f2) / (2.0 * shat) * (P.phiconst * sp) * gp_;
    w = wfac * E;
    // d ln alpha_s / d ln mu = -2 b0 alpha_s (one loop)
    gw_lnmu = -2.0 * (N - 2) * P.b0 * as * w;
    dwfac_dht = wfac * (N - 2) * (-2.0 * P.b0 * as) / ht;
  }
  const double up = G.dL_dw ? G.dL_dw[e] : 1.0;
  if (G.w) G.w[e] = w;
  if (G.dw_dlnmu) G.dw_dlnmu[e] = up * gw_lnmu;
  // dw/dk at fixed x: wfac dE/dk + E dwfac/dH_T dH_T/dk
  double gt[N][4];
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int m = 0; m < 4; ++m) gt[i][m] = pass ? wfac * gk[i][m] : 0.0;
    if (pass && i >= 2) {
      const double px = kk[i][1], py = kk[i][2], pt = sqrt(px * px + py * py);
      const double ept = E * dwfac_dht * (double)(T(1) / (T)pt);  // reciprocal in T
      gt[i][1] += ept * px;
      gt[i][2] += ept * py;
    }
  }
  if (G.dw_dk)
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) G.dw_dk[(e * N + i) * 4 + m] = up * gt[i][m];
  if (!G.dw_du) return;
  double *gu = G.dw_du + e * NU;
  // x uniforms: w is homogeneous in the momenta (degree 8 - 2n) and H_T
  // scales with sqrt(s_hat):
  // d ln w / d ln x = x f'/f + (m - 3) - (n - 2) b0 alpha_s + (4 - n)
  const double xs_[2] = {x1, x2};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const double x = xs_[j];
    const double dl = -0.2 - 5.0 * x / (1.0 - x) + (M - 3) - (N - 2) * P.b0 * as + (4 - N);
    gu[j] = pass ? up * w * dl * P.lnxmin : 0.0;
  }
  if (!pass) {  // failing events: zero gradients, whatever the (possibly non-finite) kinematics
#pragma unroll
    for (int j = 2; j < NU; ++j) gu[j] = 0.0;
    return;
  }
  // Rambo uniforms: reverse through the boost/rescale and the seed map
  double gx = 0.0, ggam = 0.0, gaa = 0.0, gM = 0.0, gb[3] = {0, 0, 0}, gQ[4] = {0, 0, 0, 0};
  double gq[M][4], gbq[M], gf[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const double *gpi = gt[2 + i];
    gx += gpi[0] * (gam * q[i][0] + bq[i]);
    ggam += gpi[0] * xs * q[i][0];
    gq[i][0] = gpi[0] * xs * gam;
    gbq[i] = gpi[0] * xs;
    gf[i] = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      gx += gpi[1 + j] * (q[i][1 + j] + bv[j] * fq[i]);
      gq[i][1 + j] = gpi[1 + j] * xs;
      gb[j] += gpi[1 + j] * xs * fq[i];
      gf[i] += gpi[1 + j] * xs * bv[j];
    }
    gq[i][0] += gf[i];
    gaa += gf[i] * bq[i];
    gbq[i] += gf[i] * aa;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      gb[j] += gbq[i] * q[i][1 + j];
      gq[i][1 + j] += gbq[i] * bv[j];
    }
  }
  ggam += gaa * (-aa * aa);
  const double iMq = 1.0 / Mq;
  gM += gx * (-xs * iMq);
  gQ[0] += ggam * iMq;
  gM += ggam * (-gam * iMq);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    gQ[1 + j] += -gb[j] * iMq;
    gM += gb[j] * (-bv[j] * iMq);
  }
  gQ[0] += gM * Q0 * iMq;
  gQ[1] += gM * (-Q1 * iMq);
  gQ[2] += gM * (-Q2 * iMq);
  gQ[3] += gM * (-Q3 * iMq);
#pragma unroll
  for (int i = 0; i < M; ++i) {
#pragma unroll
    for (int m = 0; m < 4; ++m) gq[i][m] += gQ[m];
    const double q0 = q0v[i], s = sth[i], cc = cth[i], cs = cph[i], sn = sph[i];
    const double gq0 = gq[i][0] + gq[i][1] * s * cs + gq[i][2] * s * sn + gq[i][3] * cc;
    const double gs = gq[i][1] * q0 * cs + gq[i][2] * q0 * sn;
    const double gc = gq[i][3] * q0 + gs * (-cc * (double)(T(1) / (T)s));
    const double gphi = gq[i][1] * (-q0 * s * sn) + gq[i][2] * (q0 * s * cs);
    gu[2 + 4 * i + 0] = up * 2.0 * gc;
    gu[2 + 4 * i + 1] = up * 2.0 * 3.14159265358979323846 * gphi;
    gu[2 + 4 * i + 2] = up * (-gq0 * (double)(T(1) / (T)u[2 + 4 * i + 2]));
    gu[2 + 4 * i + 3] = up * (-gq0 * (double)(T(1) / (T)u[2 + 4 * i + 3]));
  }
}

template <int N, typename R>
__global__ void __launch_bounds__(kBlock) grad_kernel(GradParams G) {
  constexpr int M = N - 2, L = N - 1, NU = 2 + 4 * M;
  const uint64_t e = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (e >= G.n_events) return;
  GradKin<N, R> K;
  grad_kinematics<N, R>(G.P, G.u + e * NU, G.order + e * N, K);
  const uint32_t hel = G.hel[e];
  BGAdjoint<R, L> bg;
  CV4<R> e0;
  {
    RV4<R> k0;
    grad_amp_input<N, R, R>(K, hel, 0, k0, e0);
  }
#pragma unroll
  for (int a = 0; a < L; ++a) {
    const int X = BGAdjoint<R, L>::tri(a, a);
    grad_amp_input<N, R, R>(K, hel, a + 1, bg.K[X], bg.J[X]);
  }
  bg.forward();
  const Cx<R> mamp = mdot(e0, bg.num);
  CV4<R> ge0;
  bg.adjoint(e0, cx<R>(R(2) * mamp.re, R(2) * mamp.im), ge0);
  const double f = (double)mamp.re * (double)mamp.re + (double)mamp.im * (double)mamp.im;
  grad_outputs<N, R, R>(G, e, K, hel, f, [&](int a, double(&g4)[4], CV4<R> &ge) {
    if (a == 0) {
      ge = ge0;
    } else {
      const int X = BGAdjoint<R, L>::tri(a - 1, a - 1);
#pragma unroll
      for (int m = 0; m < 4; ++m) g4[m] = (double)bg.GK[X].v[m];
      ge = bg.GJ[X];
    }
  });
}

// The generator's own draws for events [first, first + n): the x and Rambo
// uniforms (FP64), helicity labels and colour ordering, so that
// tess_gradients on them reproduces tess_generate's events.
template <int N>
__global__ void __launch_bounds__(kBlock) draws_kernel(EventParams P, double *u, uint32_t *hel, uint8_t *order) {
  constexpr int M = N - 2, NU = 2 + 4 * M;
  const uint64_t e = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (e >= P.n_events) return;
  const uint64_t ev = P.first_event + e;
#pragma unroll
  for (int b = 0; b < NU / 2; ++b) {
    const double2 v = uniform_pair(P.seed, ev, b);
    u[e * NU + 2 * b] = v.x;
    u[e * NU + 2 * b + 1] = v.y;
  }
  int perm[N];
  const uint32_t h = sample_config<N>(P, ev, perm);
  hel[e] = h;
#pragma unroll
  for (int i = 0; i < N; ++i) order[e * N + i] = (uint8_t)perm[i];
}

}  // namespace tess
