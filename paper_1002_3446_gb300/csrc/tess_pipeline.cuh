// Two-kernel event pipeline for sampled helicity / colour ordering:
//   K1 (kin_kernel): draws -> x1, x2 -> Rambo -> luminosity, alpha_s, cuts,
//       observables -> polarisation vectors; writes the colour-ordered
//       Berends-Giele inputs of a chunk of events to workspace (SoA).
//   K2 (bg_*_kernel): Berends-Giele amplitude of every event of the chunk ->
//       |A|^2 estimator, weight -> per-block partial sums (deterministic).
// The chunk buffer is streamed through HBM between the two launches (its
// size is the caller's trade between workspace and per-launch cost).
//
// Precision: with R = double every step is FP64 (the plain FP64 form).  With
// R = float (FP32 currents) the Rambo seeds, cuts, observables, alpha_s and
// PDF are FP32, while Rambo's mass-conserving boost and rescale, the
// polarisation-vector construction and all accumulation stay FP64.
#pragma once
#include <cstdint>

#include "tess_async.cuh"
#include "tess_event.cuh"
#include "tess_kernels.cuh"

namespace tess {

// Chunk buffers inside the caller's workspace, element e of slot s at
// base[s * cap + e] (coalesced across consecutive events).
template <typename R>
struct ChunkBuf {
  R *in;          // [InRows<L>::rows * cap] amplitude inputs, rows as InRows
  double *efac;   // [cap] |m|^2 -> estimator E (includes the momentum unit)
  double *wfac;   // [cap] E -> weight (0 if the event fails the cuts)
  double *hval;   // [cap] histogram observable
  uint8_t *pass;  // [cap] pass flag
  int cap;
  // cut-first generation only (else null): the kinematics kernel puts the
  // events that pass the cuts in the first columns of its tile (in event
  // order) and counts them per tile; the index kernel lists their columns.
  int *col = nullptr;     // [cap] column of the j-th kept event of the chunk
  int *orig = nullptr;    // [cap] chunk index of the event in a kept column
  int *tcount = nullptr;  // [cap / kBlock] kept events per kinematics tile
  int *toff = nullptr;    // [cap / kBlock] kept events before the tile
  int *dcount = nullptr;  // [1] kept events of the chunk
  // deferred histogram only (else null): the amplitude kernel's event
  // weights, which the histogram kernel bins after it
  double *wev = nullptr;  // [cap]
};

struct ChunkParams {
  EventParams P;
  uint64_t chunk_first;  // index of the chunk's first event within the call
  int count;             // events in this chunk
};

// Rows of the amplitude inputs in a chunk buffer (each row cap events).  For
// colour positions 1..L (block b = position - 1): k^0..k^3, Re eps^x, eps^y,
// eps^z, Im eps^x, eps^y; then for position 0: Re eps^x, eps^y, eps^z, Im
// eps^x, eps^y.  eps^0 = 0 and Im eps^z = 0 in the helicity basis of the
// polarisation vectors (eps_+- = (-+e1 - i e2)/sqrt2 with e1, e2 spatial and
// e2 transverse to z), so those components are not stored.
template <int L>
struct InRows {
  static constexpr int rows = 9 * L + 5;
  __host__ __device__ static constexpr int k(int b) { return 9 * b; }
  __host__ __device__ static constexpr int eps(int b) { return 9 * b + 4; }
  static constexpr int eps0 = 9 * L;
};

// Momentum and polarisation vector from their rows (row stride s elements).
template <typename R>
__device__ __forceinline__ void load_k(const R *p, size_t s, RV4<R> &k) {
#pragma unroll
  for (int m = 0; m < 4; ++m) k.v[m] = p[m * s];
}

template <typename R>
__device__ __forceinline__ void load_eps(const R *p, size_t s, CV4<R> &v) {
  v.c[0].re = R(0);
  v.c[0].im = R(0);
  v.c[1].re = p[0];
  v.c[2].re = p[s];
  v.c[3].re = p[2 * s];
  v.c[1].im = p[3 * s];
  v.c[2].im = p[4 * s];
  v.c[3].im = R(0);
}

template <typename R>
__device__ __forceinline__ R r_exp(R x);
template <>
__device__ __forceinline__ float r_exp<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double r_exp<double>(double x) { return exp(x); }

template <typename R>
__device__ __forceinline__ R r_log(R x);
template <>
__device__ __forceinline__ float r_log<float>(float x) { return logf(x); }
template <>
__device__ __forceinline__ double r_log<double>(double x) { return log(x); }

template <typename R>
__device__ __forceinline__ R r_atan2(R y, R x);
template <>
__device__ __forceinline__ float r_atan2<float>(float y, float x) { return atan2f(y, x); }
template <>
__device__ __forceinline__ double r_atan2<double>(double y, double x) { return atan2(y, x); }

template <typename R>
__device__ __forceinline__ void r_sincospi(R x, R *s, R *c);
template <>
__device__ __forceinline__ void r_sincospi<float>(float x, float *s, float *c) { sincospif(x, s, c); }
template <>
__device__ __forceinline__ void r_sincospi<double>(double x, double *s, double *c) { sincospi(x, s, c); }

template <typename R>
__device__ __forceinline__ R r_pow(R x, R y);
template <>
__device__ __forceinline__ float r_pow<float>(float x, float y) { return powf(x, y); }
template <>
__device__ __forceinline__ double r_pow<double>(double x, double y) { return pow(x, y); }

// A uniform rounded to R, kept strictly below 1.
template <typename R>
__device__ __forceinline__ R r_unit(double u) {
  R v = R(u);
  return v < R(1) ? v : R(1) - R(1) / R(1 << 24);
}

// Random real polarisations (Sec. 3): cos and sin of the angle phi = 2 pi u of
// every leg, from the draws after the colour-ordering draws (positions
// 2 + 4m + 1 + (n - 2) + l of the event's draw layout).
template <int N, typename T>
__device__ __forceinline__ void polarisation_angles(const EventParams &P, uint64_t ev, T (&cphi)[N], T (&sphi)[N]) {
  constexpr uint32_t j0 = 2 + 4 * (N - 2) + 1 + (N - 2);
#pragma unroll
  for (uint32_t b = j0 >> 1; b <= (j0 + N - 1) >> 1; ++b) {
    const uint4 w = event_block(P, ev, b);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int l = (int)(2 * b + h) - (int)j0;
      if (l >= 0 && l < N) {
        if constexpr (sizeof(T) == 4) {
          const float u = h ? unit_f32(w.z, w.w) : unit_f32(w.x, w.y);
          sincospif(2.f * u, &sphi[l], &cphi[l]);
        } else {
          const double u = h ? unit_from_words(w.z, w.w) : unit_from_words(w.x, w.y);
          sincospi(2.0 * u, &sphi[l], &cphi[l]);
        }
      }
    }
  }
}

// Cuts and observables of the FP32 kinematics forms from the rounded
// momenta pk (E, px, py, pz of the final-state gluons) and the partonic
// rapidity y: pT, eta (lab), H_T, leading pT, and the pT / |eta| cuts.
// Every operation's rounding is written out (no contraction left to the
// compiler), so the kernels' instantiations (cut-first or not) give
// bit-identical observables.
template <int M>
__device__ __forceinline__ void cuts_observables(const EventParams &P, const float (&pk)[M][4], float y, float (&px)[M],
                                                 float (&py)[M], float (&pt)[M], float (&eta)[M], int &pass, float &sum,
                                                 float &lead) {
#pragma unroll
  for (int i = 0; i < M; ++i) {
    px[i] = pk[i][1];
    py[i] = pk[i][2];
    const float pz = pk[i][3];
    const float pt2 = __fmaf_rn(px[i], px[i], __fmul_rn(py[i], py[i]));
    const float pabs = sqrtf(__fmaf_rn(pz, pz, pt2));
    pt[i] = sqrtf(pt2);
    eta[i] = __fadd_rn(__fmul_rn(0.5f, logf(__fdiv_rn(__fadd_rn(pabs, pz), __fsub_rn(pabs, pz)))), y);
    sum = __fadd_rn(sum, pt[i]);
    lead = fmaxf(lead, pt[i]);
    pass &= (pt[i] > P.f_pt_min) & (fabsf(eta[i]) < P.f_eta_max);
  }
}

// Delta R of every pair (the Delta R cut); returns the smallest Delta R^2.
// Azimuths once per gluon (m arctangents instead of m(m-1)/2), the pair's
// Delta phi = |phi_i - phi_j| folded into [0, pi]; each azimuth is within an
// ulp or two of the exact one, so Delta phi is within ~1e-6 absolute, far
// inside the FP32 forms' tolerance on cut decisions and R_min.
template <int M>
__device__ __forceinline__ float pair_cuts(const EventParams &P, const float (&px)[M], const float (&py)[M],
                                           const float (&eta)[M], int &pass) {
  float dr2min = 1e30f;
  float phi[M];
#pragma unroll
  for (int i = 0; i < M; ++i) phi[i] = atan2f(py[i], px[i]);
#pragma unroll
  for (int i = 0; i < M; ++i) {
#pragma unroll
    for (int j = i + 1; j < M; ++j) {
      float dphi = fabsf(__fsub_rn(phi[i], phi[j]));
      dphi = dphi > 3.14159265358979f ? __fsub_rn(6.28318530717959f, dphi) : dphi;
      const float de = __fsub_rn(eta[i], eta[j]);
      const float dr2 = __fmaf_rn(de, de, __fmul_rn(dphi, dphi));
      dr2min = fminf(dr2min, dr2);
      pass &= (dr2 > P.f_dr2_min);
    }
  }
  return dr2min;
}

// One-loop alpha_s at mu_R = mu_r_factor H_T, FP32, roundings written out.
__device__ __forceinline__ float alphas_f32(const EventParams &P, float ht) {
  const float mu = __fmul_rn(P.f_mu_r_factor, ht);
  const float l = __fsub_rn(logf(__fmul_rn(mu, mu)), P.f_ln_mz2);
  return __fdiv_rn(P.f_alphas_mz, __fmaf_rn(P.f_asb0, l, 1.f));
}

// Grid mode (Sec. 3's tabulated PDF and alpha_s): the tables, built once per
// call from the functions in FP64 and rounded to FP32 ...
template <int NT>
__global__ void __launch_bounds__(NT) grid_fill_kernel(EventParams P, float *g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kPdfNodes) {
    const double x = exp((double)i / (double)kPdfSegments * P.lnxmin);
    g[i] = (float)(1.7 * pow(x, -0.2) * pow(1.0 - x, 5.0));
  } else if (i < kPdfNodes + kAsNodes) {
    const int j = i - kPdfNodes;
    const double mu = exp(0.5 * (P.as_vlo + (P.as_vhi - P.as_vlo) * j / (double)kAsSegments));
    g[i] = (float)(P.alphas_mz / (1.0 + P.alphas_mz * P.b0 * (log(mu * mu) - P.ln_mz2)));
  }
}

// ... and read by linear interpolation in FP32: s in node units, clamped,
// i = min(floor(s), nseg - 1), t = s - i, value fma(t, g[i+1] - g[i], g[i]).
__device__ __forceinline__ float grid_blend(const float *__restrict__ g, int nseg, float s) {
  s = fminf(fmaxf(s, 0.f), (float)nseg);
  const int i = min((int)s, nseg - 1);
  const float t = __fsub_rn(s, (float)i);
  const float g0 = __ldg(g + i), g1 = __ldg(g + i + 1);
  return __fmaf_rn(t, __fsub_rn(g1, g0), g0);
}

// x g(x) at the float x draw u (ln x = u ln x_min)
__device__ __forceinline__ float grid_pdf(const EventParams &P, float u) {
  return grid_blend(P.grid_pdf, kPdfSegments, __fmul_rn(u, (float)kPdfSegments));
}

// alpha_s at mu_R = mu_r_factor H_T from the table in ln mu^2
__device__ __forceinline__ float grid_alphas(const EventParams &P, float ht) {
  const float mu = __fmul_rn(P.f_mu_r_factor, ht);
  const float v = logf(__fmul_rn(mu, mu));
  return grid_blend(P.grid_as, kAsSegments, __fmul_rn(__fsub_rn(v, P.f_as_vlo), P.f_as_inv));
}

// K1, FP64 form: every step in double precision.
template <int N, typename R, bool RP>
__device__ __forceinline__ void kin_generic(const ChunkParams &C, const ChunkBuf<R> &B, int e) {
  constexpr int M = N - 2, L = N - 1;
  const EventParams &P = C.P;
  const uint64_t idx = C.chunk_first + (uint64_t)e;
  const uint64_t ev = P.first_event + idx;

  // ---- x1, x2 (uniform in ln x)
  const double2 ux = uniform_pair(P.seed, ev, 0);
  const R x1 = r_exp<R>(R(ux.x) * R(P.lnxmin));
  const R x2 = r_exp<R>(R(ux.y) * R(P.lnxmin));
  const double shat = (double)x1 * (double)x2 * P.S;
  const double rs = sqrt(shat);

  // ---- Rambo: isotropic seeds in R, boost + rescale in FP64
  double q[M][4];
  double Q0 = 0.0, Q1 = 0.0, Q2 = 0.0, Q3 = 0.0;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const double2 a = uniform_pair(P.seed, ev, 1 + 2 * i);
    const double2 b = uniform_pair(P.seed, ev, 2 + 2 * i);
    const R c = R(2) * r_unit<R>(a.x) - R(1);
    const R s = sqrt(fmax(R(1) - c * c, R(0)));
    R sn, cs;
    r_sincospi<R>(R(2) * r_unit<R>(a.y), &sn, &cs);
    const R q0 = -r_log<R>(r_unit<R>(b.x) * r_unit<R>(b.y));
    q[i][0] = (double)q0;
    q[i][1] = (double)(q0 * s * cs);
    q[i][2] = (double)(q0 * s * sn);
    q[i][3] = (double)(q0 * c);
    Q0 += q[i][0];
    Q1 += q[i][1];
    Q2 += q[i][2];
    Q3 += q[i][3];
  }
  const double Mq = sqrt(Q0 * Q0 - Q1 * Q1 - Q2 * Q2 - Q3 * Q3);
  const double invM = 1.0 / Mq;
  const double bx = -Q1 * invM, by = -Q2 * invM, bz = -Q3 * invM;
  const double gam = Q0 * invM;
  const double aa = 1.0 / (1.0 + gam);
  const double xs = rs * invM;
  double kk[N][4];
  const double h = 0.5 * rs;
  kk[0][0] = -h; kk[0][1] = 0.0; kk[0][2] = 0.0; kk[0][3] = -h;
  kk[1][0] = -h; kk[1][1] = 0.0; kk[1][2] = 0.0; kk[1][3] = h;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const double bq = bx * q[i][1] + by * q[i][2] + bz * q[i][3];
    kk[2 + i][0] = xs * (gam * q[i][0] + bq);
    const double f = aa * bq + q[i][0];
    kk[2 + i][1] = xs * (q[i][1] + bx * f);
    kk[2 + i][2] = xs * (q[i][2] + by * f);
    kk[2 + i][3] = xs * (q[i][3] + bz * f);
  }

  // ---- cuts and observables (R), lab rapidity = eta + ln(x1/x2)/2
  const R y = R(0.5) * r_log<R>(x1 / x2);
  R eta[M], pt[M], px[M], py[M];
  int pass = 1;
  R sum = R(0), lead = R(0);
#pragma unroll
  for (int i = 0; i < M; ++i) {
    px[i] = R(kk[2 + i][1]);
    py[i] = R(kk[2 + i][2]);
    const R pz = R(kk[2 + i][3]);
    const R pt2 = px[i] * px[i] + py[i] * py[i];
    const R pabs = sqrt(pt2 + pz * pz);
    pt[i] = sqrt(pt2);
    eta[i] = R(0.5) * r_log<R>((pabs + pz) / (pabs - pz)) + y;
    sum += pt[i];
    lead = fmax(lead, pt[i]);
    pass &= (pt[i] > R(P.pt_min)) & (fabs(eta[i]) < R(P.eta_max));
  }
  R dr2min = R(1e30);
#pragma unroll
  for (int i = 0; i < M; ++i) {
#pragma unroll
    for (int j = i + 1; j < M; ++j) {
      const R dphi = r_atan2<R>(fabs(px[i] * py[j] - py[i] * px[j]), px[i] * px[j] + py[i] * py[j]);
      const R de = eta[i] - eta[j];
      const R dr2 = de * de + dphi * dphi;
      dr2min = fmin(dr2min, dr2);
      pass &= (dr2 > R(P.dr2_min));
    }
  }
  const double ht = (double)sum, ptlead = (double)lead, rmin = (double)sqrt(dr2min);
  if (P.ht) P.ht[idx] = ht;
  if (P.ptlead) P.ptlead[idx] = ptlead;
  if (P.rmin) P.rmin[idx] = rmin;
  if (P.pass) P.pass[idx] = (uint8_t)pass;

  // ---- weight factor (everything but the matrix element)
  double wf = 0.0;
  if (pass) {
    const R mu = R(P.mu_r_factor) * sum;
    const R as = R(P.alphas_mz) / (R(1) + R(P.alphas_mz) * R(P.b0) * (r_log<R>(mu * mu) - R(P.ln_mz2)));
    const double g2 = 4.0 * 3.14159265358979323846 * (double)as;
    double gp = 1.0;
#pragma unroll
    for (int i = 0; i < N - 2; ++i) gp *= g2;
    double sp = 1.0;
#pragma unroll
    for (int i = 0; i < M - 2; ++i) sp *= shat;
    const R f1 = R(1.7) * r_pow<R>(x1, R(-0.2)) * r_pow<R>(R(1) - x1, R(5));
    const R f2 = R(1.7) * r_pow<R>(x2, R(-0.2)) * r_pow<R>(R(1) - x2, R(5));
    const double lum = P.lnxmin * P.lnxmin * (double)f1 * (double)f2;
    wf = P.wconst * lum / (2.0 * shat) * (P.phiconst * sp) * gp;
  }
  const double inv_rs = pow2_unit_inv(rs);
  double ef = P.efac;
  const double u2 = inv_rs * inv_rs;
#pragma unroll
  for (int i = 0; i < N - 4; ++i) ef *= u2;
  B.efac[e] = ef;
  B.wfac[e] = wf;
  B.pass[e] = (uint8_t)pass;
  if (B.hval) B.hval[e] = P.hist_obs == 0 ? ptlead : (P.hist_obs == 1 ? ht : rmin);

  // ---- colour ordering, then sampled helicities or random real
  // polarisations (FP64 construction)
  int perm[N];
  const uint32_t hel = sample_config<N>(P, ev, perm);
  double cphi[N], sphi[N];
  if constexpr (RP) polarisation_angles<N, double>(P, ev, cphi, sphi);
  double kp[N][4];
  int legp[N];
  gather_positions<N>(kk, perm, kp, legp);
  const int cap = B.cap;
#pragma unroll
  for (int a = 0; a < N; ++a) {
    const double sg = legp[a] < 2 ? -1.0 : 1.0;
    CV4<double> ep, em;
    polarisations<double>(sg * kp[a][1], sg * kp[a][2], sg * kp[a][3], ep, em);
    using IR = InRows<L>;
    R *o = B.in + (size_t)(a == 0 ? IR::eps0 : IR::eps(a - 1)) * cap + e;
    if (a > 0) {
      R *ok = B.in + (size_t)IR::k(a - 1) * cap + e;
#pragma unroll
      for (int m = 0; m < 4; ++m) ok[(size_t)m * cap] = R(kp[a][m] * inv_rs);
    }
    if constexpr (RP) {
      // eps_+ = -(e1 + i e2)/sqrt2, so cos e1 + sin e2 = -sqrt2 (cos Re + sin Im) eps_+
      double cl = 0.0, sl = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l)
        if (legp[a] == l) {
          cl = cphi[l];
          sl = sphi[l];
        }
      const double r = -1.41421356237309504880;
#pragma unroll
      for (int m = 1; m < 4; ++m) o[(size_t)(m - 1) * cap] = R(r * (cl * ep.c[m].re + sl * ep.c[m].im));
      o[(size_t)3 * cap] = R(0);
      o[(size_t)4 * cap] = R(0);
    } else {
      const bool minus = (hel >> legp[a]) & 1u;
      const CV4<double> &z = minus ? em : ep;
      o[0] = R(z.c[1].re);
      o[(size_t)cap] = R(z.c[2].re);
      o[(size_t)2 * cap] = R(z.c[3].re);
      o[(size_t)3 * cap] = R(z.c[1].im);
      o[(size_t)4 * cap] = R(z.c[2].im);
    }
  }
}

// Polarisation basis of an outgoing massless momentum (E, px, py, pz) in FP64
// (the Gram products): e1 = theta-hat = (ct cf, ct sf, -st), e2 = phi-hat =
// (-sf, cf, 0), with ct = pz/E, st = pT/E, cf = px/pT, sf = py/pT (E = |p|
// for a massless momentum).  Returned rounded to FP32.
__device__ __forceinline__ void pol_basis_f32(double E, double px, double py, double pz, float (&e1)[3],
                                              float (&e2)[2]) {
  const double pt2 = px * px + py * py;
  double cf = 1.0, sf = 0.0, pt = 0.0;
  if (pt2 > 0.0) {
    const double inv_pt = rsqrt(pt2);
    pt = pt2 * inv_pt;
    cf = px * inv_pt;
    sf = py * inv_pt;
  }
  const double inv_e = 1.0 / E;
  const double ct = pz * inv_e, st = pt * inv_e;
  e1[0] = (float)(ct * cf);
  e1[1] = (float)(ct * sf);
  e1[2] = (float)(-st);
  e2[0] = (float)(-sf);
  e2[1] = (float)cf;
}

// Writes the amplitude inputs of one event -- per colour position a: the leg
// momentum (positions 1..L) and eps (eps_+ = -(e1 + i e2)/sqrt2, eps_- =
// (e1 - i e2)/sqrt2 by the leg's helicity label) -- into a shared-memory tile
// of the block's kBlock events ([12 L + 8 rows][kBlock]).  Each leg's values
// go straight to the rows of its colour position; store_tile then writes the
// tile's rows to the chunk buffer with bulk copies.
template <int N>
constexpr size_t kin_tile_bytes() {
  return (size_t)InRows<N - 1>::rows * kBlock * sizeof(float);
}

template <int N>
__device__ __forceinline__ void scatter_ordered(const EventParams &P, uint64_t ev, float *tile, int slot,
                                                const float (&lk)[N][4], const float (&le1)[N][3],
                                                const float (&le2)[N][2]) {
  constexpr int L = N - 1;
  uint64_t posw;
  const uint32_t hel = sample_positions<N>(P, ev, &posw);
  float *col = tile + slot;
  const float r2 = 0.70710678118654752440f;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    const int p = (int)((posw >> (4 * l)) & 15ull);  // colour position of leg l
    const float sre = ((hel >> l) & 1u) ? r2 : -r2;
    float *o = col + (p == 0 ? InRows<L>::eps0 : InRows<L>::eps(p - 1)) * kBlock;
    if (p > 0) {
      float *ok = col + InRows<L>::k(p - 1) * kBlock;
#pragma unroll
      for (int q = 0; q < 4; ++q) ok[q * kBlock] = lk[l][q];
    }
    o[0] = sre * le1[l][0];
    o[1 * kBlock] = sre * le1[l][1];
    o[2 * kBlock] = sre * le1[l][2];
    o[3 * kBlock] = -r2 * le2[l][0];
    o[4 * kBlock] = -r2 * le2[l][1];
  }
}

// As scatter_ordered, with the random real polarisation eps = cos(phi) e1 +
// sin(phi) e2 of every leg (imaginary rows zero); the colour ordering comes
// from the same draws.
template <int N>
__device__ __forceinline__ void scatter_ordered_real(const EventParams &P, uint64_t ev, float *tile, int slot,
                                                     const float (&lk)[N][4], const float (&le1)[N][3],
                                                     const float (&le2)[N][2]) {
  constexpr int L = N - 1;
  uint64_t posw;
  sample_positions<N>(P, ev, &posw);
  float cphi[N], sphi[N];
  polarisation_angles<N, float>(P, ev, cphi, sphi);
  float *col = tile + slot;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    const int p = (int)((posw >> (4 * l)) & 15ull);  // colour position of leg l
    float *o = col + (p == 0 ? InRows<L>::eps0 : InRows<L>::eps(p - 1)) * kBlock;
    if (p > 0) {
      float *ok = col + InRows<L>::k(p - 1) * kBlock;
#pragma unroll
      for (int q = 0; q < 4; ++q) ok[q * kBlock] = lk[l][q];
    }
    o[0] = fmaf(cphi[l], le1[l][0], sphi[l] * le2[l][0]);
    o[1 * kBlock] = fmaf(cphi[l], le1[l][1], sphi[l] * le2[l][1]);
    o[2 * kBlock] = cphi[l] * le1[l][2];
    o[3 * kBlock] = 0.f;
    o[4 * kBlock] = 0.f;
  }
}

template <int N, bool RP>
__device__ __forceinline__ void scatter_legs(const EventParams &P, uint64_t ev, float *tile, int slot,
                                             const float (&lk)[N][4], const float (&le1)[N][3],
                                             const float (&le2)[N][2]) {
  if constexpr (RP)
    scatter_ordered_real<N>(P, ev, tile, slot, lk, le1, le2);
  else
    scatter_ordered<N>(P, ev, tile, slot, lk, le1, le2);
}

// Cut-first compaction point of the kinematics kernels (CF): the block's
// events that pass the cuts take the first columns of its tile, in event
// order; returns this event's column (-1 when it is not kept, i.e. it fails
// the cuts or lies past the chunk) and records the block's count.  Failing
// events get their weight and |m|^2 outputs (0) here, since no amplitude
// kernel sees them.  Every thread of the block must call it.
template <bool CF>
__device__ __forceinline__ int cut_first_slot(const EventParams &P, const ChunkBuf<float> &B, bool live, int pass,
                                              uint64_t idx, int *kept = nullptr) {
  if constexpr (!CF) {
    return (int)threadIdx.x;
  } else {
    __shared__ int wsum[kBlock / 32];
    const bool keep = live && pass;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wsum[w] = __popc(m);
    __syncthreads();
    int base = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < kBlock / 32; ++i) {
      base += i < w ? wsum[i] : 0;
      tot += wsum[i];
    }
    if (threadIdx.x == 0) B.tcount[blockIdx.x] = tot;
    if (kept) *kept = tot;
    if (live && !pass) {
      if (P.weight) P.weight[idx] = 0.0;
      if (P.me2) P.me2[idx] = 0.0;
    }
    return keep ? base + __popc(m & ((1u << lane) - 1u)) : -1;
  }
}

// Rows of the block's tile -> chunk buffer, one bulk copy per row issued by
// warp 0.  The chunk buffers hold cap events, cap a multiple of kBlock, so a
// whole tile is in bounds (columns of threads without an event carry no data
// the amplitude kernel reads); row segments start on 512-byte boundaries.
template <int N>
__device__ __forceinline__ void store_tile(const ChunkBuf<float> &B, const float *tile) {
  constexpr int rows = InRows<N - 1>::rows;
  fence_proxy_async();  // this thread's tile writes, visible to the bulk-copy engine
  __syncthreads();
  if (threadIdx.x < 32) {
    const size_t e0 = (size_t)blockIdx.x * kBlock;
    for (int r = threadIdx.x; r < rows; r += 32)
      bulk_s2g(B.in + (size_t)r * B.cap + e0, tile + (size_t)r * kBlock, kBlock * sizeof(float));
    bulk_commit_and_wait_read();
  }
}

// K1, FP32-current form.  FP32: uniforms (from the Philox words directly),
// Rambo seeds, x1/x2, cuts, observables, alpha_s, PDF.  FP64: the Rambo boost
// and rescale (conservation and masslessness), the polarisation Gram
// products, the weight factor.  Helicity labels and colour ordering are
// exact integer functions of the draws (identical in both forms).
template <int N, bool RP, bool CF>
__device__ __forceinline__ void kin_fp32(const ChunkParams &C, const ChunkBuf<float> &B, int e, float *tile,
                                     bool live) {
  constexpr int M = N - 2;
  const EventParams &P = C.P;
  const uint64_t idx = C.chunk_first + (uint64_t)e;
  const uint64_t ev = P.first_event + idx;

  const uint4 w0 = event_block(P, ev, 0);
  const float lnxmin = P.f_lnxmin;
  const float ux1 = unit_f32(w0.x, w0.y), ux2 = unit_f32(w0.z, w0.w);
  const float x1 = expf(ux1 * lnxmin);
  const float x2 = expf(ux2 * lnxmin);
  const double shat = (double)x1 * (double)x2 * P.S;
  const double rs = sqrt(shat);

  // Rambo seeds in FP32, boost + rescale in FP64
  float qf[M][4];
  double Q0 = 0.0, Q1 = 0.0, Q2 = 0.0, Q3 = 0.0;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const uint4 wa = event_block(P, ev, 1 + 2 * i);
    const uint4 wb = event_block(P, ev, 2 + 2 * i);
    const float c = 2.f * unit_f32(wa.x, wa.y) - 1.f;
    const float sn0 = sqrtf(fmaxf(1.f - c * c, 0.f));
    float sn, cs;
    sincospif(2.f * unit_f32(wa.z, wa.w), &sn, &cs);
    const float q0 = -logf(unit_f32(wb.x, wb.y) * unit_f32(wb.z, wb.w));
    qf[i][0] = q0;
    qf[i][1] = q0 * sn0 * cs;
    qf[i][2] = q0 * sn0 * sn;
    qf[i][3] = q0 * c;
    Q0 += (double)qf[i][0];
    Q1 += (double)qf[i][1];
    Q2 += (double)qf[i][2];
    Q3 += (double)qf[i][3];
  }
  const double invM = rsqrt(Q0 * Q0 - Q1 * Q1 - Q2 * Q2 - Q3 * Q3);
  const double bx = -Q1 * invM, by = -Q2 * invM, bz = -Q3 * invM;
  const double gam = Q0 * invM;
  const double aa = 1.0 / (1.0 + gam);
  const double xs = rs * invM;
  double pk[M][4];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const double q0 = qf[i][0], q1 = qf[i][1], q2 = qf[i][2], q3 = qf[i][3];
    const double bq = bx * q1 + by * q2 + bz * q3;
    pk[i][0] = xs * (gam * q0 + bq);
    const double f = aa * bq + q0;
    pk[i][1] = xs * (q1 + bx * f);
    pk[i][2] = xs * (q2 + by * f);
    pk[i][3] = xs * (q3 + bz * f);
  }

  // cuts and observables in FP32
  const float y = __fmul_rn(0.5f, logf(__fdiv_rn(x1, x2)));
  float eta[M], pt[M], px[M], py[M], pkf[M][4];
#pragma unroll
  for (int i = 0; i < M; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) pkf[i][m] = (float)pk[i][m];
  int pass = 1;
  float sum = 0.f, lead = 0.f;
  cuts_observables<M>(P, pkf, y, px, py, pt, eta, pass, sum, lead);
  const float dr2min = pair_cuts<M>(P, px, py, eta, pass);
  const double ht = (double)sum, ptlead = (double)lead, rmin = (double)sqrtf(dr2min);
  if (live) {
    if (P.ht) P.ht[idx] = ht;
    if (P.ptlead) P.ptlead[idx] = ptlead;
    if (P.rmin) P.rmin[idx] = rmin;
    if (P.pass) P.pass[idx] = (uint8_t)pass;
  }
  const int slot = cut_first_slot<CF>(P, B, live, pass, idx);
  if (slot < 0) return;
  const int ec = CF ? (int)blockIdx.x * kBlock + slot : e;  // chunk column of the event's factors
  if constexpr (CF) B.orig[ec] = e;

  double wf = 0.0;
  if (pass) {
    const float as = P.pdf_grid ? grid_alphas(P, sum) : alphas_f32(P, sum);
    const double g2 = 4.0 * 3.14159265358979323846 * (double)as;
    double gp = 1.0;
#pragma unroll
    for (int i = 0; i < N - 2; ++i) gp *= g2;
    double sp = 1.0;
#pragma unroll
    for (int i = 0; i < M - 2; ++i) sp *= shat;
    const float f1 = P.pdf_grid ? grid_pdf(P, ux1) : 1.7f * powf(x1, -0.2f) * powf(1.f - x1, 5.f);
    const float f2 = P.pdf_grid ? grid_pdf(P, ux2) : 1.7f * powf(x2, -0.2f) * powf(1.f - x2, 5.f);
    const double lum = P.lnxmin * P.lnxmin * (double)f1 * (double)f2;
    wf = P.wconst * lum / (2.0 * shat) * (P.phiconst * sp) * gp;
  }
  const double inv_rs = pow2_unit_inv(rs);
  double ef = P.efac;
  const double u2 = inv_rs * inv_rs;
#pragma unroll
  for (int i = 0; i < N - 4; ++i) ef *= u2;
  B.efac[ec] = ef;
  B.wfac[ec] = wf;
  B.pass[ec] = (uint8_t)pass;
  if (B.hval) B.hval[ec] = P.hist_obs == 0 ? ptlead : (P.hist_obs == 1 ? ht : rmin);

  // per-leg FP32 data: momentum in units of the power-of-two scale, and the
  // polarisation basis (e1 spatial, e2 transverse); beam-axis legs are exact
  float lk[N][4], le1[N][3], le2[N][2];
  const float sc = (float)inv_rs;
  const float hs = (float)(0.5 * rs) * sc;
  lk[0][0] = -hs; lk[0][1] = 0.f; lk[0][2] = 0.f; lk[0][3] = -hs;
  lk[1][0] = -hs; lk[1][1] = 0.f; lk[1][2] = 0.f; lk[1][3] = hs;
  le1[0][0] = 1.f; le1[0][1] = 0.f; le1[0][2] = 0.f; le2[0][0] = 0.f; le2[0][1] = 1.f;   // physical +z
  le1[1][0] = -1.f; le1[1][1] = 0.f; le1[1][2] = 0.f; le2[1][0] = 0.f; le2[1][1] = 1.f;  // physical -z
#pragma unroll
  for (int i = 0; i < M; ++i) {
#pragma unroll
    for (int m = 0; m < 4; ++m) lk[2 + i][m] = (float)pk[i][m] * sc;
    pol_basis_f32(pk[i][0], pk[i][1], pk[i][2], pk[i][3], le1[2 + i], le2[2 + i]);
  }

  scatter_legs<N, RP>(P, ev, tile, slot, lk, le1, le2);
}

// Polarisation basis in FP32 from the FP32-rounded momentum components (each
// within half an ulp of the double-float value, so every product here has
// FP32 relative accuracy: no cancellation occurs); E = |p|.
__device__ __forceinline__ void pol_basis_rounded(float E, float px, float py, float pz, float (&e1)[3],
                                                  float (&e2)[2]) {
  const float pt2 = fmaf(px, px, py * py);
  float cf = 1.f, sf = 0.f, pt = 0.f;
  if (pt2 > 0.f) {
    const float ipt = rsqrtf(pt2);
    pt = pt2 * ipt;
    cf = px * ipt;
    sf = py * ipt;
  }
  const float ie = 1.f / E;
  const float ct = pz * ie, st = pt * ie;
  e1[0] = ct * cf;
  e1[1] = ct * sf;
  e1[2] = -st;
  e2[0] = -sf;
  e2[1] = cf;
}

// K1, double-float form: as kin_fp32, with the step that needs more than
// FP32 -- Rambo's boost and rescale -- in double-float (two-float)
// arithmetic on the FP32 pipe instead of native FP64 (1/64 of the FP32 rate
// on this GPU), and the polarisation basis in FP32 from the rounded momenta.
// The weight factor is assembled in FP32 with its power-of-two scale kept as
// an exact exponent.
// Second half of the double-float kinematics of one event (weight factor,
// momenta in the power-of-two unit, polarisation basis, scatter into tile
// column `slot`), from the first half's results.
template <int N, bool RP, bool CF>
__device__ __forceinline__ void kin_ds_back(const ChunkParams &C, const ChunkBuf<float> &B, float *tile, int slot,
                                            int e, uint64_t ev, float rs_hi, float shat_hi, float sum, float lead,
                                            float rmin, float x1, float x2, float ux1, float ux2, int pass,
                                            const float (&pk)[N - 2][4]) {
  constexpr int M = N - 2;
  const EventParams &P = C.P;
  const float lnxmin = P.f_lnxmin;
  const int ec = CF ? (int)blockIdx.x * kBlock + slot : e;  // chunk column of the event's factors
  if constexpr (CF) B.orig[ec] = e;

  // momentum unit 2^-ex near 1/sqrt(s_hat); s' = s_hat 2^-2ex in [1/4, 1)
  int ex;
  frexpf(rs_hi, &ex);
  const float sc = ldexpf(1.f, -ex);
  const float sp = __fmul_rn(__fmul_rn(shat_hi, sc), sc);
  double wf = 0.0;
  if (pass) {
    const float as = P.pdf_grid ? grid_alphas(P, sum) : alphas_f32(P, sum);
    const float g2 = __fmul_rn(4.f * 3.14159265358979323846f, as);
    float F;
    if (P.pdf_grid) {
      F = __fmul_rn(grid_pdf(P, ux1), grid_pdf(P, ux2));
    } else {
      // f(x1) f(x2) with f(x) = 1.7 x^-0.2 (1 - x)^5: (x1 x2)^-0.2 from ln x1 + ln x2
      const float t1 = __fsub_rn(1.f, x1), t2 = __fsub_rn(1.f, x2);
      const float t1s = __fmul_rn(t1, t1), t2s = __fmul_rn(t2, t2);
      const float p1 = __fmul_rn(__fmul_rn(t1s, t1s), t1), p2 = __fmul_rn(__fmul_rn(t2s, t2s), t2);
      F = __fmul_rn(__fmul_rn(__fmul_rn(2.89f, expf(__fmul_rn(__fmul_rn(-0.2f, lnxmin), __fadd_rn(ux1, ux2)))), p1),
                    p2);
    }
#pragma unroll
    for (int i = 0; i < N - 2; ++i) F = __fmul_rn(F, g2);
    // s_hat^(m-3) = s'^(m-3) 2^(2 ex (m-3))
    if (M >= 3) {
#pragma unroll
      for (int i = 0; i < M - 3; ++i) F = __fmul_rn(F, sp);
    } else {
      F = __fdiv_rn(F, sp);
    }
    if (F > 0.f) wf = scale_pow2(P.wk * (double)F, 2 * ex * (M - 3));
  }
  B.efac[ec] = scale_pow2(P.efac, -2 * ex * (N - 4));
  B.wfac[ec] = wf;
  B.pass[ec] = (uint8_t)pass;
  if (B.hval && P.hist_bins > 0) B.hval[ec] = (double)(P.hist_obs == 0 ? lead : (P.hist_obs == 1 ? sum : rmin));

  float lk[N][4], le1[N][3], le2[N][2];
  const float hs = 0.5f * rs_hi * sc;
  lk[0][0] = -hs; lk[0][1] = 0.f; lk[0][2] = 0.f; lk[0][3] = -hs;
  lk[1][0] = -hs; lk[1][1] = 0.f; lk[1][2] = 0.f; lk[1][3] = hs;
  le1[0][0] = 1.f; le1[0][1] = 0.f; le1[0][2] = 0.f; le2[0][0] = 0.f; le2[0][1] = 1.f;   // physical +z
  le1[1][0] = -1.f; le1[1][1] = 0.f; le1[1][2] = 0.f; le2[1][0] = 0.f; le2[1][1] = 1.f;  // physical -z
#pragma unroll
  for (int i = 0; i < M; ++i) {
#pragma unroll
    for (int m = 0; m < 4; ++m) lk[2 + i][m] = pk[i][m] * sc;
    pol_basis_rounded(pk[i][0], pk[i][1], pk[i][2], pk[i][3], le1[2 + i], le2[2 + i]);
  }
  scatter_legs<N, RP>(P, ev, tile, slot, lk, le1, le2);
}

template <int N, bool RP, bool CF>
__device__ __forceinline__ void kin_ds(const ChunkParams &C, const ChunkBuf<float> &B, int e, float *tile,
                                     bool live) {
  constexpr int M = N - 2;
  const EventParams &P = C.P;
  const uint64_t idx = C.chunk_first + (uint64_t)e;
  const uint64_t ev = P.first_event + idx;

  const uint4 w0 = event_block(P, ev, 0);
  const float lnxmin = P.f_lnxmin;
  const float ux1 = unit_f32(w0.x, w0.y), ux2 = unit_f32(w0.z, w0.w);
  const float x1 = expf(ux1 * lnxmin);  // ln x = u ln x_min
  const float x2 = expf(ux2 * lnxmin);
  const DS shat = ds_mul(ds_mul(DS{P.S_hi, P.S_lo}, x1), x2);
  const DS rs = ds_sqrt(shat);

  float qf[M][4];
  float Qh[4] = {0.f, 0.f, 0.f, 0.f}, Ql[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const uint4 wa = event_block(P, ev, 1 + 2 * i);
    const uint4 wb = event_block(P, ev, 2 + 2 * i);
    const float c = 2.f * unit_f32(wa.x, wa.y) - 1.f;
    const float sn0 = sqrtf(fmaxf(1.f - c * c, 0.f));
    float sn, cs;
    sincospif(2.f * unit_f32(wa.z, wa.w), &sn, &cs);
    const float q0 = -logf(unit_f32(wb.x, wb.y) * unit_f32(wb.z, wb.w));
    qf[i][0] = q0;
    qf[i][1] = q0 * sn0 * cs;
    qf[i][2] = q0 * sn0 * sn;
    qf[i][3] = q0 * c;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float t;
      Qh[m] = two_sum(Qh[m], qf[i][m], t);
      Ql[m] += t;
    }
  }
  DS Q[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) Q[m] = ds_fast_two_sum(Qh[m], Ql[m]);
  const DS M2 = ds_sub(ds_mul(Q[0], Q[0]), ds_add(ds_add(ds_mul(Q[1], Q[1]), ds_mul(Q[2], Q[2])), ds_mul(Q[3], Q[3])));
  const DS invM = ds_rsqrt(M2);
  const DS b[3] = {ds_neg(ds_mul(Q[1], invM)), ds_neg(ds_mul(Q[2], invM)), ds_neg(ds_mul(Q[3], invM))};
  const DS gam = ds_mul(Q[0], invM);
  const DS aa = ds_rcp(ds_add(gam, 1.f));
  const DS xs = ds_mul(rs, invM);
  // boost and rescale of each seed, k = xs (gam q0 + b.q, q + b f), f = aa b.q
  // + q0, in unnormalised pairs, each component rounded once to FP32
  float pk[M][4];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    float t, l1, l2, l3;
    const float p1 = pair_mul(b[0].hi, b[0].lo, qf[i][1], l1);
    const float p2 = pair_mul(b[1].hi, b[1].lo, qf[i][2], l2);
    const float p3 = pair_mul(b[2].hi, b[2].lo, qf[i][3], l3);
    float uh = two_sum(p1, p2, t);
    float ul = t + l1 + l2 + l3;
    uh = two_sum(uh, p3, t);
    ul += t;  // (uh, ul) = b.q
    float gl;
    const float gh = pair_mul(gam.hi, gam.lo, qf[i][0], gl);
    const float eh = two_sum(gh, uh, t);
    pk[i][0] = pair_mul_round(xs.hi, xs.lo, eh, t + gl + ul);
    float fl;
    const float fp = pair_mul(aa.hi, aa.lo, uh, ul, fl);
    const float fh = two_sum(fp, qf[i][0], t);
    fl += t;  // (fh, fl) = f
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float bl;
      const float bh = pair_mul(b[j].hi, b[j].lo, fh, fl, bl);
      const float sh = two_sum(qf[i][1 + j], bh, t);
      pk[i][1 + j] = pair_mul_round(xs.hi, xs.lo, sh, t + bl);
    }
  }

  // cuts and observables in FP32 from the rounded momenta; the partonic
  // rapidity 0.5 ln(x1 / x2) from the logarithms drawn above
  const float y = __fmul_rn(__fmul_rn(0.5f, lnxmin), __fsub_rn(ux1, ux2));
  float eta[M], pt[M], px[M], py[M];
  int pass = 1;
  float sum = 0.f, lead = 0.f;
  cuts_observables<M>(P, pk, y, px, py, pt, eta, pass, sum, lead);
  float dr2min = pair_cuts<M>(P, px, py, eta, pass);
  const float rmin = sqrtf(dr2min);
  if (live) {
    if (P.ht) P.ht[idx] = (double)sum;
    if (P.ptlead) P.ptlead[idx] = (double)lead;
    if (P.rmin) P.rmin[idx] = (double)rmin;
    if (P.pass) P.pass[idx] = (uint8_t)pass;
  }
  if constexpr (!CF) {
    kin_ds_back<N, RP, CF>(C, B, tile, (int)threadIdx.x, e, ev, rs.hi, shat.hi, sum, lead, rmin, x1, x2, ux1, ux2,
                           pass, pk);
  } else {
    // the block's kept events are finished by its first threads, one each,
    // with their first-half results staged in shared memory
    constexpr int NS = 4 * M + 12;
    __shared__ uint32_t st[NS][kBlock];
    int kept = 0;
    int slot = cut_first_slot<CF>(P, B, live, pass, idx, &kept);
    if (slot >= 0) {
      const float v[12] = {rs.hi, shat.hi, sum, lead, rmin, x1, x2, ux1, ux2, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 9; ++q) st[q][slot] = __float_as_uint(v[q]);
      st[9][slot] = (uint32_t)e;
      st[10][slot] = (uint32_t)ev;
      st[11][slot] = (uint32_t)(ev >> 32);
#pragma unroll
      for (int i = 0; i < M; ++i)
#pragma unroll
        for (int m = 0; m < 4; ++m) st[12 + 4 * i + m][slot] = __float_as_uint(pk[i][m]);
    }
    __syncthreads();
    slot = (int)threadIdx.x;
    if (slot >= kept) return;
    float q[9], pq[M][4];
#pragma unroll
    for (int i = 0; i < 9; ++i) q[i] = __uint_as_float(st[i][slot]);
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) pq[i][m] = __uint_as_float(st[12 + 4 * i + m][slot]);
    const int eo = (int)st[9][slot];
    const uint64_t evo = (uint64_t)st[10][slot] | ((uint64_t)st[11][slot] << 32);
    kin_ds_back<N, RP, CF>(C, B, tile, slot, eo, evo, q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7], q[8], 1, pq);
  }
}

// K1 kernels.  The FP32 forms take kin_tile_bytes<N>() of dynamic shared
// memory for the block's output tile.
// CF (cut-first): every thread of a block runs the kinematics (threads past
// the chunk on its last event, writing nothing) so that all reach the
// compaction point.
template <int N, typename R, bool RP = false, bool CF = false>
__global__ void __launch_bounds__(kBlock) kin_kernel(ChunkParams C, ChunkBuf<R> B) {
  const int e = blockIdx.x * kBlock + threadIdx.x;
  if constexpr (sizeof(R) == 4) {
    extern __shared__ __align__(128) float kin_tile[];
    if (CF)
      kin_fp32<N, RP, CF>(C, B, min(e, C.count - 1), kin_tile, e < C.count);
    else if (e < C.count)
      kin_fp32<N, RP, CF>(C, B, e, kin_tile, true);
    store_tile<N>(B, kin_tile);
  } else {
    if (e >= C.count) return;
    kin_generic<N, R, RP>(C, B, e);
  }
}

template <int N, bool RP = false, bool CF = false>
__global__ void __launch_bounds__(kBlock) kin_ds_kernel(ChunkParams C, ChunkBuf<float> B) {
  extern __shared__ __align__(128) float kin_tile[];
  const int e = blockIdx.x * kBlock + threadIdx.x;
  if (CF)
    kin_ds<N, RP, CF>(C, B, min(e, C.count - 1), kin_tile, e < C.count);
  else if (e < C.count)
    kin_ds<N, RP, CF>(C, B, e, kin_tile, true);
  store_tile<N>(B, kin_tile);
}

// Cut-first: exclusive scan of the kinematics tiles' kept counts (one
// block) into per-tile offsets and the chunk's kept total ...
template <int NT>
__global__ void __launch_bounds__(NT) cut_first_scan_kernel(const int *tcount, int ntiles, int *toff, int *dcount) {
  __shared__ int part[NT];
  const int t = threadIdx.x;
  const int per = (ntiles + NT - 1) / NT;
  const int t0 = min(t * per, ntiles), t1 = min(t0 + per, ntiles);
  int sum = 0;
  for (int i = t0; i < t1; ++i) sum += tcount[i];
  part[t] = sum;
  __syncthreads();
  for (int d = 1; d < NT; d <<= 1) {
    const int v = t >= d ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int off = part[t] - sum;
  for (int i = t0; i < t1; ++i) {
    toff[i] = off;
    off += tcount[i];
  }
  if (t == NT - 1) *dcount = part[NT - 1];
}

// ... then the list of kept columns in event order (kept index j -> column),
// one block per kinematics tile.
template <int NB>
__global__ void __launch_bounds__(NB) cut_first_fill_kernel(const int *tcount, const int *toff, int *col) {
  const int t = blockIdx.x;
  if ((int)threadIdx.x < tcount[t]) col[toff[t] + threadIdx.x] = t * NB + threadIdx.x;
}

// The kinematics kernel of a call: double-float or plain form, sampled
// helicities or random real polarisations.
template <int N, typename R>
__host__ inline cudaError_t launch_kin(const ChunkParams &C, const ChunkBuf<R> &B, int kin_smem, cudaStream_t s) {
  const unsigned grid = (unsigned)((C.count + kBlock - 1) / kBlock);
  if constexpr (sizeof(R) == 4) {
    const int v = (C.P.pol_random ? 1 : 0) + (C.P.cut_first ? 2 : 0);
    if (C.P.kin_ds) {
      switch (v) {
        case 0: kin_ds_kernel<N, false, false><<<grid, kBlock, kin_smem, s>>>(C, B); break;
        case 1: kin_ds_kernel<N, true, false><<<grid, kBlock, kin_smem, s>>>(C, B); break;
        case 2: kin_ds_kernel<N, false, true><<<grid, kBlock, kin_smem, s>>>(C, B); break;
        default: kin_ds_kernel<N, true, true><<<grid, kBlock, kin_smem, s>>>(C, B); break;
      }
    } else {
      switch (v) {
        case 0: kin_kernel<N, R, false, false><<<grid, kBlock, kin_smem, s>>>(C, B); break;
        case 1: kin_kernel<N, R, true, false><<<grid, kBlock, kin_smem, s>>>(C, B); break;
        case 2: kin_kernel<N, R, false, true><<<grid, kBlock, kin_smem, s>>>(C, B); break;
        default: kin_kernel<N, R, true, true><<<grid, kBlock, kin_smem, s>>>(C, B); break;
      }
    }
    if (C.P.cut_first) {
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      cut_first_scan_kernel<1024><<<1, 1024, 0, s>>>(B.tcount, (int)grid, B.toff, B.dcount);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      cut_first_fill_kernel<kBlock><<<grid, kBlock, 0, s>>>(B.tcount, B.toff, B.col);
    }
    return cudaGetLastError();
  } else {
    if (C.P.pol_random)
      kin_kernel<N, R, true><<<grid, kBlock, kin_smem, s>>>(C, B);
    else
      kin_kernel<N, R, false><<<grid, kBlock, kin_smem, s>>>(C, B);
    return cudaGetLastError();
  }
}

// ---------------------------------------------------------------------------
// K2 epilogue shared by the Berends-Giele kernels: |m|^2 -> estimator and
// weight, per-event outputs, and block-owned partial sums.  Each block owns
// partial row blockIdx.x and adds this chunk's sums to it (chunks run in order
// on one stream, so the read-modify-write is race-free and deterministic).
// ---------------------------------------------------------------------------
template <int NB>
struct Accum {
  double sw = 0.0, sw2 = 0.0;
  int npass = 0, nbad = 0;
};

// |A|^2 as the epilogue's FP64 input.  FP32 amplitudes: squared in FP32 (one
// rounding, far below the FP32 amplitude's own error) when that stays in the
// normal range, else in FP64.
// Exact widening of a positive normal FP32 value to FP64 on the integer pipe
// (binary32 -> binary64 layouts: the 23 fraction bits move up by 29, the
// exponent bias grows by 1023 - 127 = 896); FP64 conversions share the
// 1/64-rate FP64 pipe on this GPU.
__device__ __forceinline__ double widen_positive_normal(float s) {
  return __longlong_as_double((long long)((((uint64_t)__float_as_uint(s)) << 29) + (896ull << 52)));
}

__device__ __forceinline__ double amp2_of(const Cx<float> &a) {
  const float s = fmaf(a.re, a.re, a.im * a.im);
  if (s < 3.0e38f && s > 1.0e-30f) return widen_positive_normal(s);
  const double re = a.re, im = a.im;
  return re * re + im * im;
}

__device__ __forceinline__ double amp2_of(const Cx<double> &a) { return a.re * a.re + a.im * a.im; }

// Event epilogue from the chunk factors of event e (chunk index): efac, wfac,
// pass and the histogram value *hval (read only when histogramming).
template <int NB>
__device__ __forceinline__ void finish_values(const ChunkParams &C, int e, double efac, double wfac, int ok,
                                              const double *hval, double amp2, Accum<NB> &A, double &w_out,
                                              int &bin_out) {
  const EventParams &P = C.P;
  const uint64_t idx = C.chunk_first + (uint64_t)e;
  const double E = efac * amp2;
  double w = wfac * E;
  if ((__double2hiint(w) & 0x7ff00000) == 0x7ff00000) {  // not finite: exponent field all ones
    A.nbad += 1;
    w = 0.0;
  }
  if (P.me2) P.me2[idx] = E;
  if (P.weight) P.weight[idx] = w;
  A.sw += w;
  A.sw2 += w * w;
  A.npass += ok;
  w_out = w;
  bin_out = (P.hist_bins > 0 && ok) ? hist_bin(*hval, P.hist_lo, P.hist_inv_width, P.hist_bins) : -1;
}

// Events the amplitude kernel evaluates in a chunk, and the chunk column of
// the j-th: every event in order, or under cut-first the kept ones (their
// count and columns from the index kernel).
template <typename R>
__device__ __forceinline__ int k2_count(const ChunkParams &C, const ChunkBuf<R> &B) {
  return C.P.cut_first ? *B.dcount : C.count;
}

template <typename R>
__device__ __forceinline__ int k2_col(const ChunkParams &C, const ChunkBuf<R> &B, int j) {
  return C.P.cut_first ? B.col[j] : j;
}

// Epilogue of the event in chunk column e (factors at e; per-event outputs
// at its chunk index, e itself unless cut-first moved it).
template <int NB, typename R>
__device__ __forceinline__ void finish_event(const ChunkParams &C, const ChunkBuf<R> &B, int e, double amp2,
                                             Accum<NB> &A, double &w_out, int &bin_out) {
  const int o = C.P.cut_first ? B.orig[e] : e;
  finish_values<NB>(C, o, B.efac[e], B.wfac[e], B.pass[e], B.hval + e, amp2, A, w_out, bin_out);
  if (B.wev) B.wev[e] = w_out;
}

// Shared-memory scratch of the epilogue: one histogram per warp (w bins then
// w^2 bins) and the warps' (w, w^2) staging of a tile, after the bytes the
// kernel uses itself.
template <int NB>
struct EpiSmem {
  static constexpr int NW = NB / 32;
  double *hw;                  // [NW][2 nb2]
  double *stage_w, *stage_w2;  // [NB]
  __device__ EpiSmem(char *base, int nb2) {
    hw = (double *)base;
    stage_w = hw + (size_t)2 * nb2 * NW;
    stage_w2 = stage_w + NB;
  }
  static size_t bytes(int hist_bins) {
    const int nb2 = hist_bins > 0 ? hist_bins + 2 : 0;
    return (size_t)(2 * nb2 * NW + 2 * NB) * sizeof(double);
  }
};

// Zeroes the calling warp's histogram (every thread of the block calls it).
template <int NB>
__device__ __forceinline__ void epi_init(const EpiSmem<NB> &S, int nb2) {
  if (nb2 == 0) return;
  double *h = S.hw + (size_t)(threadIdx.x >> 5) * 2 * nb2;
  for (int i = (int)(threadIdx.x & 31u); i < 2 * nb2; i += 32) h[i] = 0.0;
  __syncwarp();
}

// Adds a tile's events to the warps' histograms (bin < 0: no fill).  Within
// each warp the lanes that fill the same bin are found with one match
// instruction and the lowest of them sums the group's w and w^2 in lane order
// into the warp's own histogram (a warp's groups have distinct bins), so no
// block barrier is needed and every sum has a fixed order: the histogram does
// not depend on timing.  The block's histogram is the warps' summed in warp
// order (epi_hist_sum).  (A loop of one thread per bin over all of the tile's
// events, the first form, made the amplitude kernel up to 3.7x slower with a
// histogram: one FP64 add per event and bin thread with a single active lane
// on the 1/64-rate FP64 pipe, between two block barriers per tile.)
template <int NB>
__device__ __forceinline__ void epi_tile(const EpiSmem<NB> &S, int nb2, double w, int bin) {
  static_assert(NB % 32 == 0, "whole warps");
  if (nb2 == 0) return;
  const int lane = (int)(threadIdx.x & 31u), warp = (int)(threadIdx.x >> 5);
  double *sw = S.stage_w + warp * 32, *sw2 = S.stage_w2 + warp * 32;
  __syncwarp();  // the warp's previous tile has been summed
  sw[lane] = w;
  sw2[lane] = w * w;
  const unsigned peers = __match_any_sync(0xffffffffu, bin);
  __syncwarp();
  if (bin >= 0 && (peers & ((1u << lane) - 1u)) == 0u) {  // the group's lowest lane
    double s = sw[lane], s2 = sw2[lane];
    for (unsigned rest = peers & ~(1u << lane); rest != 0u; rest &= rest - 1u) {
      const int t = __ffs(rest) - 1;
      s += sw[t];
      s2 += sw2[t];
    }
    double *h = S.hw + (size_t)warp * 2 * nb2;
    h[bin] += s;
    h[nb2 + bin] += s2;
  }
}

// Entry i of the block's histogram ([w bins | w^2 bins]): the warps' in warp
// order.  After a block barrier.
template <int NB>
__device__ __forceinline__ double epi_hist_sum(const EpiSmem<NB> &S, int nb2, int i) {
  double v = S.hw[i];
#pragma unroll
  for (int w = 1; w < EpiSmem<NB>::NW; ++w) v += S.hw[(size_t)w * 2 * nb2 + i];
  return v;
}

template <int NB>
__device__ __forceinline__ void epi_flush(const EpiSmem<NB> &S, int nb2, Accum<NB> &A, double *partials,
                                          int hist_bins, int stalled = 0) {
  __shared__ double red[4][NB];
  red[0][threadIdx.x] = A.sw;
  red[1][threadIdx.x] = A.sw2;
  red[2][threadIdx.x] = (double)A.npass;
  red[3][threadIdx.x] = (double)A.nbad;
  __syncthreads();
  for (int s = NB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    }
    __syncthreads();
  }
  double *row = partials + (size_t)blockIdx.x * partial_stride(hist_bins);
  if (threadIdx.x < 4) row[threadIdx.x] += red[threadIdx.x][0];
  if (threadIdx.x == 4 && stalled) row[4] += 1.0;
  for (int i = threadIdx.x; i < 2 * nb2; i += NB) row[kPartialHead + i] += epi_hist_sum(S, nb2, i);
}

// Deferred histogram (schedule SCHED_SERIAL_HIST): after the amplitude kernel
// of a chunk, block b bins the events of tiles b, b + gridDim.x, ... (NB
// events each) from the weights the amplitude kernel left in B.wev and the
// flags and observables the kinematics kernel left, and adds its histogram to
// the histogram columns of partial row b (the amplitude kernel, launched with
// hist_bins < 0, adds only the sums).  The histogram epilogue then runs as
// its own small kernel instead of inside the amplitude kernel, whose code
// (the unrolled wavefront forms reach ~100 KB) then keeps the instruction
// cache to itself.  Fills as epi_tile does: per-warp copies, fixed order.
template <int NB>
__global__ void __launch_bounds__(NB) hist_chunk_kernel(ChunkParams C, const double *__restrict__ wev,
                                                        const double *__restrict__ hval,
                                                        const uint8_t *__restrict__ pass, double *partials) {
  extern __shared__ __align__(16) char smem_raw[];
  const int nb2 = C.P.hist_bins + 2;
  EpiSmem<NB> S(smem_raw, nb2);
  epi_init(S, nb2);
  const int ntiles = (C.count + NB - 1) / NB;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int e = tile * NB + (int)threadIdx.x;
    double w = 0.0;
    int bin = -1;
    if (e < C.count && pass[e]) {
      w = wev[e];
      bin = hist_bin(hval[e], C.P.hist_lo, C.P.hist_inv_width, C.P.hist_bins);
    }
    epi_tile<NB>(S, nb2, w, bin);
  }
  __syncthreads();
  double *row = partials + (size_t)blockIdx.x * partial_stride(C.P.hist_bins);
  for (int i = threadIdx.x; i < 2 * nb2; i += NB) row[kPartialHead + i] += epi_hist_sum(S, nb2, i);
}

// L2 prefetch, by the whole block, of the amplitude inputs and event factors
// of the NB chunk columns starting at c0 (NB a multiple of 32: whole
// 128-byte lines of every float row, NB / 16 lines of every double row), so
// that the block's next tile starts from L2 instead of DRAM: the chunk buffer
// is streamed through HBM once.  Columns past the chunk's count stay inside
// the buffer (its capacity is a multiple of 128 columns).
template <int L, int NB, typename R>
__device__ __forceinline__ void prefetch_tile_l2(const ChunkBuf<R> &B, int c0, bool hist) {
  static_assert(NB % 32 == 0 && sizeof(R) == 4, "whole lines of FP32 rows");
  constexpr int LF = NB / 32, LD = NB / 16, RF = InRows<L>::rows * LF;
  const size_t cap = (size_t)B.cap;
  const int nd = hist ? 3 : 2;  // efac, wfac (and hval)
  for (int i = threadIdx.x; i < RF + nd * LD + 1; i += NB) {
    const char *p;
    if (i < RF) {
      p = (const char *)(B.in + (size_t)(i / LF) * cap + c0) + (i % LF) * 128;
    } else if (i < RF + nd * LD) {
      const int k = i - RF;
      const double *row = k < LD ? B.efac : (k < 2 * LD ? B.wfac : B.hval);
      p = (const char *)(row + c0) + (k % LD) * 128;
    } else {
      p = (const char *)(B.pass + c0);
    }
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
  }
}

// K2, register form (FP32, n <= 7): thread per event, the whole current table
// in registers.  PF: before each tile, the block's next tile is prefetched
// into L2 (the inputs are read once per event from the chunk buffer in HBM,
// and the tile's input loads are the kernel's long-scoreboard stall).
template <int N, typename R, int NB, int MINB = 1, bool PF = false>
__global__ void __launch_bounds__(NB, MINB) bg_reg_kernel(ChunkParams C, ChunkBuf<R> B, double *partials) {
  constexpr int L = N - 1;
  extern __shared__ __align__(16) char smem_raw[];
  const int nb2 = C.P.hist_bins > 0 ? C.P.hist_bins + 2 : 0;
  EpiSmem<NB> S(smem_raw, nb2);
  epi_init(S, nb2);
  Accum<NB> A;
  const int count = k2_count(C, B);
  const int ntiles = (count + NB - 1) / NB;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile * NB + threadIdx.x;
    if constexpr (PF) {
      const int next = tile + (int)gridDim.x;  // the block's next tile
      if (!C.P.cut_first && next < ntiles) prefetch_tile_l2<L, NB, R>(B, next * NB, nb2 > 0);
    }
    double w = 0.0;
    int bin = -1;
    if (j < count) {
      const int e = k2_col(C, B, j);
      RV4<R> k[L];
      CV4<R> ev[L], e0;
#pragma unroll
      for (int a = 0; a < L; ++a) {
        load_k(B.in + (size_t)InRows<L>::k(a) * B.cap + e, (size_t)B.cap, k[a]);
        load_eps(B.in + (size_t)InRows<L>::eps(a) * B.cap + e, (size_t)B.cap, ev[a]);
      }
      load_eps(B.in + (size_t)InRows<L>::eps0 * B.cap + e, (size_t)B.cap, e0);
      const Cx<R> amp = bg_amplitude<R, L>(k, ev, e0);
      finish_event<NB, R>(C, B, e, amp2_of(amp), A, w, bin);
    }
    epi_tile<NB>(S, nb2, w, bin);
  }
  epi_flush<NB>(S, nb2, A, partials, C.P.hist_bins);
}

// K2, real-current register form (FP32, random real polarisations, n <= 9):
// as bg_reg_kernel with the real recursion; reads the momentum rows and the
// three real polarisation rows of every position (the imaginary rows, zero,
// are not read).
template <int N, int NB, int MINB = 1>
__global__ void __launch_bounds__(NB, MINB) bg_real_kernel(ChunkParams C, ChunkBuf<float> B, double *partials) {
  constexpr int L = N - 1;
  extern __shared__ __align__(16) char smem_raw[];
  const int nb2 = C.P.hist_bins > 0 ? C.P.hist_bins + 2 : 0;
  EpiSmem<NB> S(smem_raw, nb2);
  epi_init(S, nb2);
  Accum<NB> A;
  const int count = k2_count(C, B);
  const int ntiles = (count + NB - 1) / NB;
  const size_t cap = (size_t)B.cap;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile * NB + threadIdx.x;
    double w = 0.0;
    int bin = -1;
    if (j < count) {
      const int e = k2_col(C, B, j);
      RV4<float> k[L], ev[L], e0;
#pragma unroll
      for (int a = 0; a < L; ++a) {
        load_k(B.in + (size_t)InRows<L>::k(a) * cap + e, cap, k[a]);
        const float *p = B.in + (size_t)InRows<L>::eps(a) * cap + e;
        ev[a].v[0] = 0.f;
        ev[a].v[1] = p[0];
        ev[a].v[2] = p[cap];
        ev[a].v[3] = p[2 * cap];
      }
      {
        const float *p = B.in + (size_t)InRows<L>::eps0 * cap + e;
        e0.v[0] = 0.f;
        e0.v[1] = p[0];
        e0.v[2] = p[cap];
        e0.v[3] = p[2 * cap];
      }
      const float amp = bg_amplitude_real<float, L>(k, ev, e0);
      finish_event<NB, float>(C, B, e, amp2_of(Cx<float>{amp, 0.f}), A, w, bin);
    }
    epi_tile<NB>(S, nb2, w, bin);
  }
  epi_flush<NB>(S, nb2, A, partials, C.P.hist_bins);
}

// K2, staged register form (FP32, n <= 8): as bg_reg_kernel, with each
// warp's inputs (its 32 events' slice of the InRows rows of the chunk
// buffer and of the event factors) brought into shared memory by the TMA unit
// one tile ahead: one tiled tensor copy of the box {32 events, all rows} and
// four bulk copies of the event factors.  Every warp owns two stages and
// their mbarriers (which count the copied bytes) and runs its own pipeline:
// it issues the copies of its slice of tile t + gridDim.x, then waits for
// tile t, so the next inputs arrive while this tile is computed, and warps
// never wait for one another (the block synchronises per tile only to fill a
// histogram).  A wait that does not complete within kStageWaitNs retires the
// warp: it computes nothing more, waits once more (bounded) for its copies in
// flight, and the block counts a stall in its partial row.
template <int L>
struct WarpStage {
  static constexpr int rows = InRows<L>::rows;
  static constexpr size_t in_bytes = (size_t)rows * 32 * sizeof(float);
  static constexpr size_t off_efac = in_bytes;
  static constexpr size_t off_wfac = off_efac + 32 * sizeof(double);
  static constexpr size_t off_hval = off_wfac + 32 * sizeof(double);
  static constexpr size_t off_pass = off_hval + 32 * sizeof(double);
  static constexpr size_t bytes = (off_pass + 32 + 127) / 128 * 128;
  static constexpr uint32_t tx = (uint32_t)(in_bytes + 3 * 32 * sizeof(double) + 32);
};

template <int L, int NB>
struct RegStage {
  static constexpr int warps = NB / 32;
  static constexpr size_t head = (size_t)warps * 2 * WarpStage<L>::bytes + 128;  // stages, then mbarriers
  static constexpr size_t window = head + 128;  // + alignment slack for the 128-byte stage base
  static_assert(warps * 2 * sizeof(uint64_t) <= 128, "mbarrier area");
};

// Copies of the 32 events starting at chunk index e0 into stage `st`: one
// tiled tensor copy (TMA) of the box {32 events, all input rows} of the chunk
// buffer (map: 2-D tensor [rows][cap] floats) and four bulk copies of the
// event factors.  The chunk buffers hold cap events, cap a multiple of 128,
// so a whole slice of a tile is in bounds; e0 * 4 bytes and the factor
// offsets are multiples of 128 bytes.
template <int L>
__device__ __forceinline__ void issue_slice(const ChunkBuf<float> &B, const CUtensorMap *map, size_t e0, char *st,
                                            uint64_t *bar) {
  using W = WarpStage<L>;
  const int lane = threadIdx.x & 31;
  fence_proxy_async();  // this warp's earlier reads of the stage precede the copies
  if (lane == 0) mbar_arrive_expect_tx(bar, W::tx);
  __syncwarp();
  if (lane == 0)
    tensor2d_g2s(st, map, (int)e0, 0, bar);
  else if (lane == 1)
    bulk_g2s(st + W::off_efac, B.efac + e0, 32 * sizeof(double), bar);
  else if (lane == 2)
    bulk_g2s(st + W::off_wfac, B.wfac + e0, 32 * sizeof(double), bar);
  else if (lane == 3)
    bulk_g2s(st + W::off_hval, B.hval + e0, 32 * sizeof(double), bar);
  else if (lane == 4)
    bulk_g2s(st + W::off_pass, B.pass + e0, 32, bar);
}

template <int N, int NB, int MINB = 1>
__global__ void __launch_bounds__(NB, MINB)
    bg_reg_tma_kernel(ChunkParams C, ChunkBuf<float> B, double *partials, const __grid_constant__ CUtensorMap map) {
  constexpr int L = N - 1;
  using W = WarpStage<L>;
  static_assert(NB == kBlock, "tiles must match the chunk-capacity granularity");
  extern __shared__ __align__(128) char smem_stage_raw[];
  // tensor copies land on 128-byte boundaries (the window is padded by 128 B)
  char *const smem_stage = (char *)(((uintptr_t)smem_stage_raw + 127) & ~(uintptr_t)127);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  char *const my0 = smem_stage + (size_t)warp * 2 * W::bytes, *const my1 = my0 + W::bytes;
  uint64_t *const bar = (uint64_t *)(smem_stage + (size_t)RegStage<L, NB>::warps * 2 * W::bytes) + 2 * warp;
  const int nb2 = C.P.hist_bins > 0 ? C.P.hist_bins + 2 : 0;
  EpiSmem<NB> ES(smem_stage + RegStage<L, NB>::head, nb2);
  epi_init(ES, nb2);
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_proxy_async();
  }
  __syncthreads();
  Accum<NB> A;
  const int ntiles = (C.count + NB - 1) / NB;
  // bit q of `parity`: phase of stage q's next completion; of `pending`: copies into q in flight
  uint32_t parity = 0u, pending = 0u;
  bool dead = false;
  if ((int)blockIdx.x < ntiles) {
    const size_t e0 = (size_t)blockIdx.x * NB + warp * 32;
    if (e0 < (size_t)C.count) {
      issue_slice<L>(B, &map, e0, my0, &bar[0]);
      pending = 1u;
    }
  }
  int k = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
    const int sb = k & 1;
    const int next = tile + gridDim.x;
    if (!dead && next < ntiles) {  // the other stage was read by this warp in the previous iteration
      const size_t e0n = (size_t)next * NB + warp * 32;
      if (e0n < (size_t)C.count) {
        issue_slice<L>(B, &map, e0n, sb ? my0 : my1, &bar[sb ^ 1]);
        pending |= 1u << (sb ^ 1);
      }
    }
    const size_t e0 = (size_t)tile * NB + warp * 32;
    double w = 0.0;
    int bin = -1;
    if (!dead && e0 < (size_t)C.count) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[sb], (parity >> sb) & 1u));
      if (!ok) {
        dead = true;
      } else {
        parity ^= 1u << sb;
        pending &= ~(1u << sb);
        const int e = (int)e0 + lane;
        if (e < C.count) {
          const char *st = sb ? my1 : my0;
          const float *in = (const float *)st + lane;
          RV4<float> kk[L];
          CV4<float> ev[L], e0v;
#pragma unroll
          for (int a = 0; a < L; ++a) {
            load_k(in + (size_t)InRows<L>::k(a) * 32, 32, kk[a]);
            load_eps(in + (size_t)InRows<L>::eps(a) * 32, 32, ev[a]);
          }
          load_eps(in + (size_t)InRows<L>::eps0 * 32, 32, e0v);
          const Cx<float> amp = bg_amplitude<float, L>(kk, ev, e0v);
          const double *efac = (const double *)(st + W::off_efac), *wfac = (const double *)(st + W::off_wfac);
          const double *hval = (const double *)(st + W::off_hval);
          const uint8_t *pass = (const uint8_t *)(st + W::off_pass);
          finish_values<NB>(C, e, efac[lane], wfac[lane], pass[lane], hval + lane, amp2_of(amp), A, w, bin);
          if (B.wev) B.wev[e] = w;
        }
      }
    }
    epi_tile<NB>(ES, nb2, w, bin);  // block barrier only when filling a histogram
    __syncwarp();                   // this warp's reads of the stage precede its refill
  }
  if (dead) {
    // copies still in flight into this warp's stages: wait once more (bounded)
    for (int q = 0; q < 2; ++q)
      if ((pending >> q) & 1u) (void)mbar_wait_bounded(&bar[q], (parity >> q) & 1u);
    __syncwarp();
  }
  const int stalled = __syncthreads_or(dead) ? 1 : 0;
  epi_flush<NB>(ES, nb2, A, partials, C.P.hist_bins, stalled);
}

// K2, loop form (FP64): table in per-thread local memory.
template <int N, int NB>
__global__ void __launch_bounds__(NB) bg_loop_kernel(ChunkParams C, ChunkBuf<double> B, double *partials) {
  constexpr int L = N - 1;
  extern __shared__ __align__(16) char smem_raw[];
  const int nb2 = C.P.hist_bins > 0 ? C.P.hist_bins + 2 : 0;
  EpiSmem<NB> S(smem_raw, nb2);
  epi_init(S, nb2);
  Accum<NB> A;
  const int count = k2_count(C, B);
  const int ntiles = (count + NB - 1) / NB;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile * NB + threadIdx.x;
    double w = 0.0;
    int bin = -1;
    if (j < count) {
      const int e = k2_col(C, B, j);
      BGLoop<double, L> bg;
#pragma unroll 1
      for (int a = 0; a < L; ++a) {
        const int X = BGLoop<double, L>::tri(a, a);
        load_k(B.in + (size_t)InRows<L>::k(a) * B.cap + e, (size_t)B.cap, bg.K[X]);
        load_eps(B.in + (size_t)InRows<L>::eps(a) * B.cap + e, (size_t)B.cap, bg.J[X]);
      }
      CV4<double> e0;
      load_eps(B.in + (size_t)InRows<L>::eps0 * B.cap + e, (size_t)B.cap, e0);
      const Cx<double> amp = bg.run(e0);
      finish_event<NB, double>(C, B, e, amp.re * amp.re + amp.im * amp.im, A, w, bin);
    }
    epi_tile<NB>(S, nb2, w, bin);
  }
  epi_flush<NB>(S, nb2, A, partials, C.P.hist_bins);
}

// ---------------------------------------------------------------------------
// K2, row form (FP32, n >= 8).  Thread per event; currents are computed row
// by row, rows a = L-1 down to 0 (row a = the sets [a..b], b >= a), each row
// in increasing b.  The row being built lives in registers (it supplies the
// left part J[a..i] of every split and the first part J_A of every four-
// vertex triple), older rows live in the thread's own shared-memory column
// (they supply the right parts and the middle parts).  Right-part momenta
// K[i+1..b] are summed on the fly from the leg momenta, so no momentum table
// is stored.  Shared-memory traffic is 10 floats per split and 8 per triple.
// ---------------------------------------------------------------------------
template <int L>
__host__ __device__ constexpr int t1(int a, int b) {
  // sets [a..b] with 1 <= a <= b <= L-1, triangular over the legs 1..L-1
  return (a - 1) * (L - 1) - ((a - 1) * (a - 2)) / 2 + (b - a);
}

template <int NB>
__device__ __forceinline__ void st_cv(float4 *J4, int t, const CV4<float> &v) {
  J4[(2 * t) * NB + threadIdx.x] = make_float4(v.c[0].re, v.c[0].im, v.c[1].re, v.c[1].im);
  J4[(2 * t + 1) * NB + threadIdx.x] = make_float4(v.c[2].re, v.c[2].im, v.c[3].re, v.c[3].im);
}

template <int NB>
__device__ __forceinline__ CV4<float> ld_cv(const float4 *J4, int t) {
  const float4 a = J4[(2 * t) * NB + threadIdx.x];
  const float4 b = J4[(2 * t + 1) * NB + threadIdx.x];
  CV4<float> v;
  v.c[0] = cx<float>(a.x, a.y);
  v.c[1] = cx<float>(a.z, a.w);
  v.c[2] = cx<float>(b.x, b.y);
  v.c[3] = cx<float>(b.z, b.w);
  return v;
}

template <int L, int NB>
__device__ __forceinline__ Cx<float> bg_rows(const float4 *K4, const CV4<float> &eps_pos0, const CV4<float> &e0,
                                             float4 *J4, float2 *S2) {
  Cx<float> amp = cx<float>(0.f, 0.f);
  auto kleg = [&](int leg) {
    const float4 v = K4[leg * NB + threadIdx.x];
    RV4<float> r = {{v.x, v.y, v.z, v.w}};
    return r;
  };
  // Runtime loop over rows; inside a row every register index is relative to
  // a and compile-time, so the row stays in registers and only one row's
  // worth of state is live at a time.
#pragma unroll 1
  for (int a = L - 1; a >= 0; --a) {
    const int len = L - a;  // currents in this row
    CV4<float> row[L];
    Cx<float> srow[L];
    RV4<float> krow[L];
    row[0] = (a == 0) ? eps_pos0 : ld_cv<NB>(J4, t1<L>(a, a));
    srow[0] = cx<float>(0.f, 0.f);
    krow[0] = kleg(a);
#pragma unroll
    for (int d = 1; d < L; ++d) {
      if (d >= len) break;
      const int b = a + d;
      krow[d] = radd(krow[d - 1], kleg(b));
      CV4<float> acc = cv_zero<float>(), tri = cv_zero<float>();
      Cx<float> s = cx<float>(0.f, 0.f);
      RV4<float> kr = {{0.f, 0.f, 0.f, 0.f}};
#pragma unroll
      for (int dp = d - 1; dp >= 0; --dp) {
        const int r0 = a + dp + 1;  // right part [r0..b]
        kr = radd(kr, kleg(r0));
        const CV4<float> Jr = ld_cv<NB>(J4, t1<L>(r0, b));
        const CV4<float> &Jl = row[dp];
        const Cx<float> d0 = mdot(Jl, Jr);
        const Cx<float> jlkr = mdot(Jl, kr);
        const Cx<float> krjl = mdot(Jr, krow[dp]);
        Cx<float> cr = cx<float>(2.f * jlkr.re - srow[dp].re, 2.f * jlkr.im - srow[dp].im);
        Cx<float> cl = cx<float>(-2.f * krjl.re, -2.f * krjl.im);
        if (dp + 1 < d) {  // right part has more than one leg
          const float2 sr = S2[t1<L>(r0, b) * NB + threadIdx.x];
          cl.re -= sr.x;
          cl.im -= sr.y;
        }
        axpy(acc, cr, Jr);
        axpy(acc, cl, Jl);
        axpy(acc, d0, rsub(krow[dp], kr));
        s.re += d0.re;
        s.im += d0.im;
        // four-vertex triples whose last part is [r0..b]
#pragma unroll
        for (int dpp = 0; dpp < dp; ++dpp) {
          const CV4<float> JB = ld_cv<NB>(J4, t1<L>(a + dpp + 1, a + dp));
          axpy(tri, mdot(row[dpp], Jr), JB);
        }
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        acc.c[m].re = fmaf(2.f, tri.c[m].re, acc.c[m].re);
        acc.c[m].im = fmaf(2.f, tri.c[m].im, acc.c[m].im);
      }
      if (a == 0 && d == L - 1) {
        amp = mdot(e0, acc);
      } else {
        const float inv = 1.f / mdot(krow[d], krow[d]);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          row[d].c[m].re = acc.c[m].re * inv;
          row[d].c[m].im = acc.c[m].im * inv;
        }
        srow[d] = s;
        if (a > 0) {
          st_cv<NB>(J4, t1<L>(a, b), row[d]);
          S2[t1<L>(a, b) * NB + threadIdx.x] = make_float2(s.re, s.im);
        }
      }
    }
  }
  return amp;
}

// Row form with real currents (random real polarisations): the same schedule
// as bg_rows, with the real recursion of bg_amplitude_real; the table holds
// one float4 per current and one float per split sum.
template <int L, int NB>
__device__ __forceinline__ float bg_rows_real(const float4 *K4, const RV4<float> &eps_pos0, const RV4<float> &e0,
                                              float4 *J4, float *S1) {
  float amp = 0.f;
  auto kleg = [&](int leg) {
    const float4 v = K4[leg * NB + threadIdx.x];
    RV4<float> r = {{v.x, v.y, v.z, v.w}};
    return r;
  };
  auto ldj = [&](int t) {
    const float4 v = J4[t * NB + threadIdx.x];
    RV4<float> r = {{v.x, v.y, v.z, v.w}};
    return r;
  };
#pragma unroll 1
  for (int a = L - 1; a >= 0; --a) {
    const int len = L - a;
    RV4<float> row[L], krow[L];
    float srow[L];
    row[0] = (a == 0) ? eps_pos0 : ldj(t1<L>(a, a));
    srow[0] = 0.f;
    krow[0] = kleg(a);
#pragma unroll
    for (int d = 1; d < L; ++d) {
      if (d >= len) break;
      const int b = a + d;
      krow[d] = radd(krow[d - 1], kleg(b));
      RV4<float> acc = {{0.f, 0.f, 0.f, 0.f}}, tri = {{0.f, 0.f, 0.f, 0.f}};
      float sum = 0.f;
      RV4<float> kr = {{0.f, 0.f, 0.f, 0.f}};
#pragma unroll
      for (int dp = d - 1; dp >= 0; --dp) {
        const int r0 = a + dp + 1;  // right part [r0..b]
        kr = radd(kr, kleg(r0));
        const RV4<float> Jr = ldj(t1<L>(r0, b));
        const RV4<float> &Jl = row[dp];
        const float d0 = mdot(Jl, Jr);
        const float cr = 2.f * mdot(Jl, kr) - srow[dp];
        float cl = -2.f * mdot(Jr, krow[dp]);
        if (dp + 1 < d) cl -= S1[t1<L>(r0, b) * NB + threadIdx.x];
        raxpy(acc, cr, Jr);
        raxpy(acc, cl, Jl);
        raxpy(acc, d0, rsub(krow[dp], kr));
        sum += d0;
#pragma unroll
        for (int dpp = 0; dpp < dp; ++dpp) raxpy(tri, mdot(row[dpp], Jr), ldj(t1<L>(a + dpp + 1, a + dp)));
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) acc.v[m] = fmaf(2.f, tri.v[m], acc.v[m]);
      if (a == 0 && d == L - 1) {
        amp = mdot(e0, acc);
      } else {
        const float inv = 1.f / mdot(krow[d], krow[d]);
#pragma unroll
        for (int m = 0; m < 4; ++m) row[d].v[m] = acc.v[m] * inv;
        srow[d] = sum;
        if (a > 0) {
          J4[t1<L>(a, b) * NB + threadIdx.x] = make_float4(row[d].v[0], row[d].v[1], row[d].v[2], row[d].v[3]);
          S1[t1<L>(a, b) * NB + threadIdx.x] = sum;
        }
      }
    }
  }
  return amp;
}

template <int L>
__host__ __device__ constexpr size_t rows_real_smem_per_thread() {
  return (size_t)(L * (L - 1) / 2) * (sizeof(float4) + sizeof(float)) + (size_t)L * sizeof(float4);
}

template <int N, int NB>
__global__ void __launch_bounds__(NB) bg_rows_real_kernel(ChunkParams C, ChunkBuf<float> B, double *partials) {
  constexpr int L = N - 1, T1 = L * (L - 1) / 2;
  extern __shared__ __align__(16) char smem_raw[];
  float4 *J4 = (float4 *)smem_raw;
  float4 *K4 = J4 + T1 * NB;
  float *S1 = (float *)(K4 + L * NB);
  const int nb2 = C.P.hist_bins > 0 ? C.P.hist_bins + 2 : 0;
  // epilogue scratch after the table, 16-byte aligned
  EpiSmem<NB> S((char *)smem_raw + ((rows_real_smem_per_thread<L>() * NB + 15) & ~(size_t)15), nb2);
  epi_init(S, nb2);
  Accum<NB> A;
  const int count = k2_count(C, B);
  const int ntiles = (count + NB - 1) / NB;
  const size_t cap = (size_t)B.cap;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile * NB + threadIdx.x;
    double w = 0.0;
    int bin = -1;
    if (j < count) {
      const int e = k2_col(C, B, j);
      RV4<float> eps0pos, e0;
#pragma unroll
      for (int a = 0; a < L; ++a) {
        const float *base = B.in + (size_t)InRows<L>::k(a) * cap + e;
        K4[a * NB + threadIdx.x] = make_float4(base[0], base[cap], base[2 * cap], base[3 * cap]);
        const float *pe = B.in + (size_t)InRows<L>::eps(a) * cap + e;
        const RV4<float> ea = {{0.f, pe[0], pe[cap], pe[2 * cap]}};
        if (a == 0)
          eps0pos = ea;
        else
          J4[t1<L>(a, a) * NB + threadIdx.x] = make_float4(0.f, ea.v[1], ea.v[2], ea.v[3]);
      }
      {
        const float *pe = B.in + (size_t)InRows<L>::eps0 * cap + e;
        e0.v[0] = 0.f;
        e0.v[1] = pe[0];
        e0.v[2] = pe[cap];
        e0.v[3] = pe[2 * cap];
      }
      const float amp = bg_rows_real<L, NB>(K4, eps0pos, e0, J4, S1);
      finish_event<NB, float>(C, B, e, amp2_of(Cx<float>{amp, 0.f}), A, w, bin);
    }
    epi_tile<NB>(S, nb2, w, bin);
  }
  epi_flush<NB>(S, nb2, A, partials, C.P.hist_bins);
}

template <int L>
__host__ __device__ constexpr size_t rows_smem_per_thread() {
  return (size_t)(L * (L - 1) / 2) * (2 * sizeof(float4) + sizeof(float2)) + (size_t)L * sizeof(float4);
}

template <int N, int NB>
__global__ void __launch_bounds__(NB) bg_rows_kernel(ChunkParams C, ChunkBuf<float> B, double *partials) {
  constexpr int L = N - 1, T1 = L * (L - 1) / 2;
  extern __shared__ __align__(16) char smem_raw[];
  float4 *J4 = (float4 *)smem_raw;
  float4 *K4 = J4 + 2 * T1 * NB;
  float2 *S2 = (float2 *)(K4 + L * NB);
  const int nb2 = C.P.hist_bins > 0 ? C.P.hist_bins + 2 : 0;
  EpiSmem<NB> S((char *)(S2 + T1 * NB), nb2);
  epi_init(S, nb2);
  Accum<NB> A;
  const int count = k2_count(C, B);
  const int ntiles = (count + NB - 1) / NB;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile * NB + threadIdx.x;
    double w = 0.0;
    int bin = -1;
    if (j < count) {
      const int e = k2_col(C, B, j);
      CV4<float> eps0pos, e0;
#pragma unroll
      for (int a = 0; a < L; ++a) {
        const float *base = B.in + (size_t)InRows<L>::k(a) * B.cap + e;
        K4[a * NB + threadIdx.x] =
            make_float4(base[0], base[(size_t)B.cap], base[(size_t)2 * B.cap], base[(size_t)3 * B.cap]);
        CV4<float> ea;
        load_eps(B.in + (size_t)InRows<L>::eps(a) * B.cap + e, (size_t)B.cap, ea);
        if (a == 0)
          eps0pos = ea;
        else
          st_cv<NB>(J4, t1<L>(a, a), ea);
      }
      load_eps(B.in + (size_t)InRows<L>::eps0 * B.cap + e, (size_t)B.cap, e0);
      const Cx<float> amp = bg_rows<L, NB>(K4, eps0pos, e0, J4, S2);
      finish_event<NB, float>(C, B, e, amp2_of(amp), A, w, bin);
    }
    epi_tile<NB>(S, nb2, w, bin);
  }
  epi_flush<NB>(S, nb2, A, partials, C.P.hist_bins);
}

}  // namespace tess
