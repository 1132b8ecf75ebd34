// One event of the generator, one thread: counter-based draws, Rambo, parton
// luminosity, cuts and observables, alpha_s, polarisation vectors, the
// Berends-Giele amplitude and the event weight (the four stages of Sec. 3).
#pragma once
#include <cstdint>

#include "tess_bg.cuh"
#include "tess_math.cuh"

namespace tess {

// Per-launch constants, prepared on the host from a tess_process.
// Node counts of the PDF and alpha_s tables of the grid mode.
constexpr int kPdfSegments = 1024, kPdfNodes = kPdfSegments + 1;
constexpr int kAsSegments = 512, kAsNodes = kAsSegments + 1;

struct EventParams {
  uint64_t seed;
  uint64_t first_event;
  uint64_t n_events;
  double S;            // hadronic s
  double lnxmin;       // ln x_min, x_min = (m pT_min)^2 / S
  double pt_min, eta_max, dr2_min;
  double alphas_mz, ln_mz2, b0, mu_r_factor;
  double wconst;       // N^(n-2)(N^2-1) / (256 m!) * GeV^-2 -> pb
  double phiconst;     // Phi_m(s) = phiconst * s^(m-2)
  double efac;         // sampled estimator factor 2^n (n-1)! / 2^(n-2)
  double hist_lo, hist_inv_width;
  int hist_bins;       // 0: no histogram; < 0 (amplitude kernel of a deferred
                       // histogram): -hist_bins bins filled by another kernel
  int hist_obs;
  // double-float kinematics: S split into two floats, and the weight
  // constant wconst (ln x_min)^2 phiconst / 2
  float S_hi, S_lo;
  double wk;
  uint32_t rk[20];     // Philox round keys of `seed`
  // single-precision copies of the constants the FP32 kinematics read
  float f_lnxmin, f_pt_min, f_eta_max, f_dr2_min, f_alphas_mz, f_asb0, f_ln_mz2, f_mu_r_factor;
  int kin_ds;          // 1: double-float kinematics kernel
  int pol_random;      // 1: random real polarisations instead of sampled helicities
  int cut_first;       // 1: amplitudes only for events passing the cuts (compacted)
  int pdf_grid;        // 1: PDF and alpha_s from the tables below (linear interpolation)
  const float *grid_pdf, *grid_as;  // kPdfNodes / kAsNodes values, in the workspace
  double as_vlo, as_vhi;            // alpha_s table range in ln mu^2
  float f_as_vlo, f_as_inv;         // the same as floats: v_lo and kAsSegments / (v_hi - v_lo)
  // outputs (device; may be null)
  double *weight, *me2, *ht, *ptlead, *rmin;
  uint8_t *pass;
};

struct EventResult {
  double w, me2, ht, ptlead, rmin;
  int pass;
};

// Polarisation vectors eps_+ and eps_- of the physical direction of p
// (helicity form; e1 = theta-hat, e2 = phi-hat; beam-axis legs take phi = 0):
// eps_+ = -(e1 + i e2)/sqrt2, eps_- = (e1 - i e2)/sqrt2.
template <typename R, typename T = double>
__device__ __forceinline__ void polarisations(T px, T py, T pz, CV4<R> &ep, CV4<R> &em) {
  const T pt2 = px * px + py * py;
  const T pt = sqrt(pt2);
  const T inv_p = T(1) / sqrt(pt2 + pz * pz);
  const T ct = pz * inv_p, st = pt * inv_p;
  T cf = T(1), sf = T(0);
  if (pt > T(0)) {
    const T inv_pt = T(1) / pt;
    cf = px * inv_pt;
    sf = py * inv_pt;
  }
  const T r = T(0.70710678118654752440);
  const T e1[4] = {T(0), ct * cf, ct * sf, -st};
  const T e2[4] = {T(0), -sf, cf, T(0)};
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    ep.c[m] = cx<R>(R(-e1[m] * r), R(-e2[m] * r));
    em.c[m] = cx<R>(R(e1[m] * r), R(-e2[m] * r));
  }
}

// Phase space and phase-space weight stages.  Fills the all-outgoing momenta
// kk[N][4] (k1 = -p1, k2 = -p2), the observables and the pass flag.
template <int N>
struct Kinematics {
  static constexpr int M = N - 2;
  double kk[N][4];
  double x1, x2, shat, ht, ptlead, rmin;
  int pass;
};

template <int N>
__device__ __forceinline__ void kinematics(const EventParams &P, uint64_t ev, Kinematics<N> &K) {
  constexpr int M = N - 2;
  const double2 ux = uniform_pair(P.seed, ev, 0);
  K.x1 = exp(ux.x * P.lnxmin);
  K.x2 = exp(ux.y * P.lnxmin);
  K.shat = K.x1 * K.x2 * P.S;
  const double rs = sqrt(K.shat);
  // Rambo (Kleiss-Stirling-Ellis): isotropic massless seeds q with energy
  // density q0 exp(-q0), then one boost + rescale to total (rs, 0, 0, 0).
  double q[M][4];
  double Q0 = 0.0, Q1 = 0.0, Q2 = 0.0, Q3 = 0.0;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const double2 a = uniform_pair(P.seed, ev, 1 + 2 * i);
    const double2 b = uniform_pair(P.seed, ev, 2 + 2 * i);
    const double c = 2.0 * a.x - 1.0;
    const double s = sqrt(1.0 - c * c);
    double sn, cs;
    sincospi(2.0 * a.y, &sn, &cs);
    const double q0 = -log(b.x * b.y);
    q[i][0] = q0;
    q[i][1] = q0 * s * cs;
    q[i][2] = q0 * s * sn;
    q[i][3] = q0 * c;
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
  const double h = 0.5 * rs;
  K.kk[0][0] = -h; K.kk[0][1] = 0.0; K.kk[0][2] = 0.0; K.kk[0][3] = -h;
  K.kk[1][0] = -h; K.kk[1][1] = 0.0; K.kk[1][2] = 0.0; K.kk[1][3] = h;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const double bq = bx * q[i][1] + by * q[i][2] + bz * q[i][3];
    K.kk[2 + i][0] = xs * (gam * q[i][0] + bq);
    const double f = aa * bq + q[i][0];
    K.kk[2 + i][1] = xs * (q[i][1] + bx * f);
    K.kk[2 + i][2] = xs * (q[i][2] + by * f);
    K.kk[2 + i][3] = xs * (q[i][3] + bz * f);
  }
  // jets: every final-state gluon; lab rapidity = eta + ln(x1/x2)/2
  const double y = 0.5 * log(K.x1 / K.x2);
  double eta[M], pt[M];
  int pass = 1;
  double sum = 0.0, lead = 0.0;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const double px = K.kk[2 + i][1], py = K.kk[2 + i][2], pz = K.kk[2 + i][3];
    const double pt2 = px * px + py * py;
    const double pabs = sqrt(pt2 + pz * pz);
    pt[i] = sqrt(pt2);
    eta[i] = 0.5 * log((pabs + pz) / (pabs - pz)) + y;
    sum += pt[i];
    lead = fmax(lead, pt[i]);
    pass &= (pt[i] > P.pt_min) & (fabs(eta[i]) < P.eta_max);
  }
  double dr2min = 1.0e300;
#pragma unroll
  for (int i = 0; i < M; ++i) {
#pragma unroll
    for (int j = i + 1; j < M; ++j) {
      const double pxi = K.kk[2 + i][1], pyi = K.kk[2 + i][2];
      const double pxj = K.kk[2 + j][1], pyj = K.kk[2 + j][2];
      const double dphi = atan2(fabs(pxi * pyj - pyi * pxj), pxi * pxj + pyi * pyj);
      const double de = eta[i] - eta[j];
      const double dr2 = de * de + dphi * dphi;
      dr2min = fmin(dr2min, dr2);
      pass &= (dr2 > P.dr2_min);
    }
  }
  K.ht = sum;
  K.ptlead = lead;
  K.rmin = sqrt(dr2min);
  K.pass = pass;
}

// Colour ordering (Fisher-Yates on positions 2..n) and helicity labels of a
// sampled event, from its draws.  Both are integer functions of the Philox
// words: the helicity word is the top n bits of its uniform, and each swap
// index floor(u (i-1)) is evaluated exactly as the double product rounds.
// Philox block `blk` of event `ev` of the launch's stream (round keys from
// the launch constants).
__device__ __forceinline__ uint4 event_block(const EventParams &P, uint64_t ev, uint32_t blk) {
  return philox4x32_10_rk(make_uint4((uint32_t)ev, (uint32_t)(ev >> 32), blk, 0u), P.rk);
}

template <int N>
__device__ __forceinline__ uint32_t sample_config(const EventParams &P, uint64_t ev, int (&perm)[N]) {
  constexpr int M = N - 2;
  constexpr uint32_t jh = 2 + 4 * M;  // helicity draw; ordering draws follow
  uint4 w = event_block(P, ev, jh >> 1);
  uint32_t cur = jh >> 1;
  const uint32_t a0 = (jh & 1u) ? w.z : w.x;
  const uint32_t hel = a0 >> (32 - N);  // top N bits of (a >> 6) 2^26 + (b >> 6)
#pragma unroll
  for (int i = 0; i < N; ++i) perm[i] = i;
#pragma unroll
  for (int i = N; i >= 3; --i) {
    const uint32_t j = jh + 1 + (N - i);
    if ((j >> 1) != cur) {
      cur = j >> 1;
      w = event_block(P, ev, cur);
    }
    const uint64_t k = (j & 1u) ? unit_bits(w.z, w.w) : unit_bits(w.x, w.y);
    const int r = 2 + floor_unit_times(k, (uint32_t)(i - 1));
    // swap positions i and r (1-based)
#pragma unroll
    for (int q = 2; q <= N; ++q) {
      if (q == r && q != i) {
        const int t = perm[i - 1];
        perm[i - 1] = perm[q - 1];
        perm[q - 1] = t;
      }
    }
  }
  return hel;
}

// The same draws as sample_config, with the permutation kept packed: nibble
// a of the working word holds the leg at colour position a (a swap is a few
// shifts and xors instead of selects over positions).  Returns the helicity
// word; *posw receives the inverse, nibble l = colour position of leg l.
template <int N>
__device__ __forceinline__ uint32_t sample_positions(const EventParams &P, uint64_t ev, uint64_t *posw) {
  static_assert(N <= 16, "4-bit positions");
  constexpr int M = N - 2;
  constexpr uint32_t jh = 2 + 4 * M;  // helicity draw; ordering draws follow
  uint4 w = event_block(P, ev, jh >> 1);
  uint32_t cur = jh >> 1;
  const uint32_t a0 = (jh & 1u) ? w.z : w.x;
  const uint32_t hel = a0 >> (32 - N);
  uint64_t pw = 0;
#pragma unroll
  for (int a = 0; a < N; ++a) pw |= (uint64_t)a << (4 * a);
#pragma unroll
  for (int i = N; i >= 3; --i) {
    const uint32_t j = jh + 1 + (N - i);
    if ((j >> 1) != cur) {
      cur = j >> 1;
      w = event_block(P, ev, cur);
    }
    const uint64_t k = (j & 1u) ? unit_bits(w.z, w.w) : unit_bits(w.x, w.y);
    const int r = 2 + floor_unit_times(k, (uint32_t)(i - 1));
    // swap positions i and r (1-based)
    const int si = 4 * (i - 1), sr = 4 * (r - 1);
    const uint64_t x = ((pw >> si) ^ (pw >> sr)) & 15ull;
    pw ^= (x << si) | (x << sr);
  }
  uint64_t qw = 0;
#pragma unroll
  for (int a = 0; a < N; ++a) qw |= (uint64_t)a << (4 * (int)((pw >> (4 * a)) & 15ull));
  *posw = qw;
  return hel;
}

// Which Berends-Giele form a (precision, n) uses: the unrolled register
// form while its table fits in registers (FP32 up to n = 7, FP64 up to
// n = 5), else the loop form.  The register form also leaves out the exact
// zeros of single-leg polarisation vectors, which the loop form's runtime
// indices cannot know.
template <typename R, int N>
struct UseRegisterBG {
  static constexpr bool value = sizeof(R) == 4 ? N <= 7 : N <= 5;
};

// Momentum of leg `leg` gathered into colour position order without dynamic
// register indexing (selects over the compile-time leg index).
template <int N>
__device__ __forceinline__ void gather_positions(const double (&kk)[N][4], const int (&perm)[N], double (&kp)[N][4],
                                                 int (&legp)[N]) {
#pragma unroll
  for (int a = 0; a < N; ++a) {
    const int want = perm[a];
    double v0 = kk[0][0], v1 = kk[0][1], v2 = kk[0][2], v3 = kk[0][3];
#pragma unroll
    for (int l = 1; l < N; ++l) {
      const bool hit = (want == l);
      v0 = hit ? kk[l][0] : v0;
      v1 = hit ? kk[l][1] : v1;
      v2 = hit ? kk[l][2] : v2;
      v3 = hit ? kk[l][3] : v3;
    }
    kp[a][0] = v0;
    kp[a][1] = v1;
    kp[a][2] = v2;
    kp[a][3] = v3;
    legp[a] = want;
  }
}

// |m|^2 (paper normalisation) of one colour ordering and helicity labelling,
// momenta multiplied by inv_rs (an exact power of two).  perm[0] is the leg contracted last; leg
// `leg` uses eps_{+/-} of its physical direction by bit `leg` of hel.
template <typename R, int N>
__device__ __forceinline__ double ordered_amp2(const double (&kk)[N][4], double inv_rs, const int (&perm)[N],
                                               uint32_t hel) {
  constexpr int L = N - 1;
  double kp[N][4];
  int legp[N];
  gather_positions<N>(kk, perm, kp, legp);
  CV4<R> e0, ep, em;
  {
    const double sg = legp[0] < 2 ? -1.0 : 1.0;
    polarisations<R>(sg * kp[0][1], sg * kp[0][2], sg * kp[0][3], ep, em);
    e0 = ((hel >> legp[0]) & 1u) ? em : ep;
  }
  Cx<R> amp;
  if constexpr (UseRegisterBG<R, N>::value) {
    RV4<R> k[L];
    CV4<R> e[L];
#pragma unroll
    for (int a = 0; a < L; ++a) {
#pragma unroll
      for (int m = 0; m < 4; ++m) k[a].v[m] = R(kp[a + 1][m] * inv_rs);
      const double sg = legp[a + 1] < 2 ? -1.0 : 1.0;
      polarisations<R>(sg * kp[a + 1][1], sg * kp[a + 1][2], sg * kp[a + 1][3], ep, em);
      e[a] = ((hel >> legp[a + 1]) & 1u) ? em : ep;
    }
    amp = bg_amplitude<R, L>(k, e, e0);
  } else {
    BGLoop<R, L> bg;
#pragma unroll
    for (int a = 0; a < L; ++a) {
      const int X = BGLoop<R, L>::tri(a, a);
#pragma unroll
      for (int m = 0; m < 4; ++m) bg.K[X].v[m] = R(kp[a + 1][m] * inv_rs);
      const double sg = legp[a + 1] < 2 ? -1.0 : 1.0;
      polarisations<R>(sg * kp[a + 1][1], sg * kp[a + 1][2], sg * kp[a + 1][3], ep, em);
      bg.J[X] = ((hel >> legp[a + 1]) & 1u) ? em : ep;
    }
    amp = bg.run(e0);
  }
  const double re = (double)amp.re, im = (double)amp.im;
  return re * re + im * im;
}

// Exact power-of-two unit 2^e close to sqrt(s): scaling momenta by it (for
// the FP32 dynamic range) changes no rounding, so momentum conservation and
// masslessness survive bit for bit.  Returns 2^-e; |m|^2 scales by 4^e per
// unit of mass dimension.
__device__ __forceinline__ double pow2_unit_inv(double rs) {
  int e;
  frexp(rs, &e);
  return ldexp(1.0, -e);
}

// x 2^s by adding s to the exponent field: equal to ldexp(x, s) for a normal
// nonzero x whose result is normal (the callers' factors are far inside the
// double range), in two integer operations instead of FP64 work.
__device__ __forceinline__ double scale_pow2(double x, int s) {
  return __longlong_as_double(__double_as_longlong(x) + ((long long)s << 52));
}

template <int N, typename R, bool SUM>
__device__ __forceinline__ EventResult event(const EventParams &P, uint64_t ev) {
  constexpr int M = N - 2;
  Kinematics<N> K;
  kinematics<N>(P, ev, K);
  const double inv_rs = pow2_unit_inv(sqrt(K.shat));
  double E;
  if constexpr (SUM) {
    // exact sum over (n-1)! orderings and 2^n helicities; flipping every
    // label conjugates each polarisation vector (up to a sign), which leaves
    // |m| unchanged exactly, so leg 0 keeps label 0 and the sum doubles.
    int perm[N];
#pragma unroll
    for (int i = 0; i < N; ++i) perm[i] = i;
    double acc = 0.0;
    bool more = true;
    while (more) {
      for (uint32_t hel = 0; hel < (1u << N); hel += 2) acc += ordered_amp2<R, N>(K.kk, inv_rs, perm, hel);
      // next permutation of perm[1..N) in lexicographic order
      int i = N - 2;
      while (i >= 1 && perm[i] >= perm[i + 1]) --i;
      if (i < 1) {
        more = false;
      } else {
        int j = N - 1;
        while (perm[j] <= perm[i]) --j;
        int t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        for (int a = i + 1, b = N - 1; a < b; ++a, --b) { t = perm[a]; perm[a] = perm[b]; perm[b] = t; }
      }
    }
    E = 2.0 * acc * P.efac;  // efac = 1 / 2^(n-2) in this mode
  } else {
    int perm[N];
    const uint32_t hel = sample_config<N>(P, ev, perm);
    E = P.efac * ordered_amp2<R, N>(K.kk, inv_rs, perm, hel);
  }
  // |m|^2 has mass dimension 8 - 2n: undo the momentum unit (exact)
  const double u2 = inv_rs * inv_rs;
#pragma unroll
  for (int i = 0; i < N - 4; ++i) E *= u2;
  EventResult r;
  r.me2 = E;
  r.ht = K.ht;
  r.ptlead = K.ptlead;
  r.rmin = K.rmin;
  r.pass = K.pass;
  r.w = 0.0;
  if (K.pass) {
    const double mu = P.mu_r_factor * K.ht;
    const double as = P.alphas_mz / (1.0 + P.alphas_mz * P.b0 * (log(mu * mu) - P.ln_mz2));
    const double g2 = 4.0 * 3.14159265358979323846 * as;
    double gp = 1.0;
#pragma unroll
    for (int i = 0; i < N - 2; ++i) gp *= g2;
    double sp = 1.0;
#pragma unroll
    for (int i = 0; i < M - 2; ++i) sp *= K.shat;
    const double f1 = 1.7 * pow(K.x1, -0.2) * pow(1.0 - K.x1, 5.0);
    const double f2 = 1.7 * pow(K.x2, -0.2) * pow(1.0 - K.x2, 5.0);
    const double lum = P.lnxmin * P.lnxmin * f1 * f2;
    r.w = P.wconst * lum / (2.0 * K.shat) * (P.phiconst * sp) * gp * E;
  }
  return r;
}

}  // namespace tess
