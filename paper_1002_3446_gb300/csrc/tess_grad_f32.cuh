// Kinematics, their adjoint and the gradient outputs for the FP32 forms of
// the gradient path, with no native FP64 arithmetic per component: FP64 runs
// at 1/64 of the FP32 rate on this GPU, and the FP64 forms of these stages
// kept its pipe 80 % busy while the FP32 pipe idled.
//
//   forward   as the generator's double-float kinematics kernel: FP32 seeds,
//             the Rambo boost/rescale in double-float pairs rounded once to
//             FP32, cuts and observables in FP32 from the rounded momenta;
//   adjoint   FP32, in units of A = (upstream gradient) x wfac x efac', so
//             that every quantity stays O(1); each output is A times an FP32
//             number, formed as an exact power-of-two scaling of the FP32
//             product (mantissa of A) x (number) in integer arithmetic.
// A handful of FP64 products per event remain (the weight and A).
#pragma once
#include <cstdint>

#include "tess_grad.cuh"

namespace tess {

// Rare paths of the conversions below, kept out of line: the compiler cannot
// turn a call into a predicated select, so the FP64 instructions in them are
// issued only when taken.
static __device__ __noinline__ float f32_of_f64_native(double x) { return (float)x; }
static __device__ __noinline__ double f64_of_f32_native(float x, int k) { return ldexp((double)x, k); }
static __device__ __noinline__ double f64_times_f32_native(double a, float x) { return a * (double)x; }

// binary64 -> binary32, round to nearest even, in integer operations; exact
// for results in the normal binary32 range (the native conversion otherwise).
__device__ __forceinline__ float f32_of_f64(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // rebiased for binary32
  if (e < 1 || e > 254) return f32_of_f64_native(x);
  const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // leading 23 mantissa bits
  const uint32_t rest = lo & 0x1fffffffu;                   // the 29 dropped bits
  const uint32_t up = (rest > 0x10000000u) | ((rest == 0x10000000u) & (m & 1u));
  // a carry out of the mantissa steps the exponent, as the rounding requires
  return __uint_as_float((hi & 0x80000000u) | (((uint32_t)e << 23) + m + up));
}

// x 2^k as binary64 for binary32 x, in integer operations; exact when x is
// zero or normal and x 2^k is a normal double (ldexp otherwise).
__device__ __forceinline__ double f64_of_f32_scaled(float x, int k) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t s = b & 0x80000000u;
  if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)s, 0);
  const int e = (int)((b >> 23) & 0xffu);
  const int E = e + 896 + k;
  if (e == 0 || e == 255 || E < 1 || E > 2046) return f64_of_f32_native(x, k);
  return __hiloint2double((int)(s | ((uint32_t)E << 20) | ((b & 0x7fffffu) >> 3)), (int)(b << 29));
}

// Writes a * x for FP64 a and FP32 x: a = m 2^k split once (m in (-2, 2)
// rounded to FP32), then each value is the FP32 product m x scaled by 2^k.
struct ScaledOut {
  float m;
  int k;
  double a;
  bool fast;
  __device__ __forceinline__ explicit ScaledOut(double a_) : a(a_) {
    const uint32_t hi = (uint32_t)__double2hiint(a_);
    const int ef = (int)((hi >> 20) & 0x7ffu);
    fast = ef > 0 && ef < 2047;
    k = ef - 1023;
    m = fast ? f32_of_f64(__hiloint2double((int)((hi & 0x800fffffu) | (1023u << 20)), __double2loint(a_))) : 0.f;
  }
  __device__ __forceinline__ double operator()(float x) const {
    return fast ? f64_of_f32_scaled(m * x, k) : f64_times_f32_native(a, x);
  }
};

// A caller-given uniform as FP32, kept below 1 like the generator's FP32
// draws (so that 1 - c^2 and ln u stay finite).
__device__ __forceinline__ float unit_of(double u) { return fminf(f32_of_f64(u), 0x1.fffffep-1f); }

template <int N>
struct GradKinF {
  static constexpr int M = N - 2;
  float ux1, ux2, x1, x2, ht, shat_hi;
  float q[M][4], cth[M], sth[M], cph[M], sph[M], q0v[M], u3[M], u4[M];
  float Q[4], iMq, gam, aa, xs, bv[3];
  float kk[N][4], bq[M], fq[M], kp[N][4];
  int legp[N], ex, pass;
};

// Forward kinematics of one event (uniforms u, colour order) with the
// intermediates the adjoint needs; the momentum unit is c = 2^-ex near
// 1/sqrt(s_hat).
template <int N>
__device__ __forceinline__ void grad_kin_f32(const EventParams &P, const double *u, const uint8_t *order,
                                             GradKinF<N> &K) {
  constexpr int M = N - 2;
  const float lnx = P.f_lnxmin;
  const float ux1 = unit_of(u[0]), ux2 = unit_of(u[1]);
  const float x1 = expf(ux1 * lnx), x2 = expf(ux2 * lnx);
  const DS shat = ds_mul(ds_mul(DS{P.S_hi, P.S_lo}, x1), x2);
  const DS rs = ds_sqrt(shat);
  K.ux1 = ux1;
  K.ux2 = ux2;
  K.x1 = x1;
  K.x2 = x2;
  K.shat_hi = shat.hi;

  float Qh[4] = {0.f, 0.f, 0.f, 0.f}, Ql[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const float uc = unit_of(u[2 + 4 * i]), uf = unit_of(u[2 + 4 * i + 1]);
    const float u3 = unit_of(u[2 + 4 * i + 2]), u4 = unit_of(u[2 + 4 * i + 3]);
    const float c = 2.f * uc - 1.f;
    const float s = sqrtf(fmaxf(1.f - c * c, 0.f));
    float sn, cs;
    sincospif(2.f * uf, &sn, &cs);
    const float q0 = -logf(u3 * u4);
    K.cth[i] = c;
    K.sth[i] = s;
    K.cph[i] = cs;
    K.sph[i] = sn;
    K.q0v[i] = q0;
    K.u3[i] = u3;
    K.u4[i] = u4;
    K.q[i][0] = q0;
    K.q[i][1] = q0 * s * cs;
    K.q[i][2] = q0 * s * sn;
    K.q[i][3] = q0 * c;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float t;
      Qh[m] = two_sum(Qh[m], K.q[i][m], t);
      Ql[m] += t;
    }
  }
  DS Q[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    Q[m] = ds_fast_two_sum(Qh[m], Ql[m]);
    K.Q[m] = Q[m].hi;
  }
  const DS M2 = ds_sub(ds_mul(Q[0], Q[0]), ds_add(ds_add(ds_mul(Q[1], Q[1]), ds_mul(Q[2], Q[2])), ds_mul(Q[3], Q[3])));
  const DS invM = ds_rsqrt(M2);
  const DS b[3] = {ds_neg(ds_mul(Q[1], invM)), ds_neg(ds_mul(Q[2], invM)), ds_neg(ds_mul(Q[3], invM))};
  const DS gam = ds_mul(Q[0], invM);
  const DS aa = ds_rcp(ds_add(gam, 1.f));
  const DS xs = ds_mul(rs, invM);
  K.iMq = invM.hi;
  K.gam = gam.hi;
  K.aa = aa.hi;
  K.xs = xs.hi;
#pragma unroll
  for (int j = 0; j < 3; ++j) K.bv[j] = b[j].hi;

  // k = xs (gam q0 + b.q, q + b f) with f = aa b.q + q0, in unnormalised
  // pairs, each component rounded once to FP32
  const float h = 0.5f * rs.hi;
  K.kk[0][0] = -h; K.kk[0][1] = 0.f; K.kk[0][2] = 0.f; K.kk[0][3] = -h;
  K.kk[1][0] = -h; K.kk[1][1] = 0.f; K.kk[1][2] = 0.f; K.kk[1][3] = h;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const float(&qi)[4] = K.q[i];
    float t, l1, l2, l3;
    const float p1 = pair_mul(b[0].hi, b[0].lo, qi[1], l1);
    const float p2 = pair_mul(b[1].hi, b[1].lo, qi[2], l2);
    const float p3 = pair_mul(b[2].hi, b[2].lo, qi[3], l3);
    float uh = two_sum(p1, p2, t);
    float ul = t + l1 + l2 + l3;
    uh = two_sum(uh, p3, t);
    ul += t;  // (uh, ul) = b.q
    float gl;
    const float gh = pair_mul(gam.hi, gam.lo, qi[0], gl);
    const float eh = two_sum(gh, uh, t);
    K.kk[2 + i][0] = pair_mul_round(xs.hi, xs.lo, eh, t + gl + ul);
    float fl;
    const float fp = pair_mul(aa.hi, aa.lo, uh, ul, fl);
    const float fh = two_sum(fp, qi[0], t);
    fl += t;  // (fh, fl) = f
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float bl;
      const float bh = pair_mul(b[j].hi, b[j].lo, fh, fl, bl);
      const float sh = two_sum(qi[1 + j], bh, t);
      K.kk[2 + i][1 + j] = pair_mul_round(xs.hi, xs.lo, sh, t + bl);
    }
    K.bq[i] = uh + ul;
    K.fq[i] = fh + fl;
  }

  // cuts and observables in FP32 from the rounded momenta; the partonic
  // rapidity 0.5 ln(x1 / x2) from the drawn logarithms
  const float y = 0.5f * lnx * (ux1 - ux2);
  float eta[M];
  int pass = 1;
  float sum = 0.f;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const float px = K.kk[2 + i][1], py = K.kk[2 + i][2], pz = K.kk[2 + i][3];
    const float pt2 = px * px + py * py;
    const float pabs = sqrtf(pt2 + pz * pz);
    const float pt = sqrtf(pt2);
    eta[i] = 0.5f * logf((pabs + pz) / (pabs - pz)) + y;
    sum += pt;
    pass &= (pt > P.f_pt_min) & (fabsf(eta[i]) < P.f_eta_max);
  }
#pragma unroll
  for (int i = 0; i < M; ++i)
#pragma unroll
    for (int j = i + 1; j < M; ++j) {
      const float pxi = K.kk[2 + i][1], pyi = K.kk[2 + i][2], pxj = K.kk[2 + j][1], pyj = K.kk[2 + j][2];
      const float dphi = atan2f(fabsf(pxi * pyj - pyi * pxj), pxi * pxj + pyi * pyj);
      const float de = eta[i] - eta[j];
      pass &= (de * de + dphi * dphi > P.f_dr2_min);
    }
  K.ht = sum;
  K.pass = pass;
  int ex;
  frexpf(rs.hi, &ex);
  K.ex = ex;

  // colour-ordered momenta
#pragma unroll
  for (int a = 0; a < N; ++a) {
    const int want = order[a];
    float v0 = K.kk[0][0], v1 = K.kk[0][1], v2 = K.kk[0][2], v3 = K.kk[0][3];
#pragma unroll
    for (int l = 1; l < N; ++l) {
      const bool hit = (want == l);
      v0 = hit ? K.kk[l][0] : v0;
      v1 = hit ? K.kk[l][1] : v1;
      v2 = hit ? K.kk[l][2] : v2;
      v3 = hit ? K.kk[l][3] : v3;
    }
    K.kp[a][0] = v0;
    K.kp[a][1] = v1;
    K.kp[a][2] = v2;
    K.kp[a][3] = v3;
    K.legp[a] = want;
  }
}

// Amplitude inputs of colour position a: the momentum in the unit c and the
// polarisation vector of its helicity label.
template <int N>
__device__ __forceinline__ void grad_amp_input_f32(const GradKinF<N> &K, uint32_t hel, int a, RV4<float> &k,
                                                   CV4<float> &eps) {
  CV4<float> ep, em;
  const float sg = K.legp[a] < 2 ? -1.f : 1.f;
  polarisations<float, float>(sg * K.kp[a][1], sg * K.kp[a][2], sg * K.kp[a][3], ep, em);
  eps = ((hel >> K.legp[a]) & 1u) ? em : ep;
  const float c = ldexpf(1.f, -K.ex);
#pragma unroll
  for (int m = 0; m < 4; ++m) k.v[m] = K.kp[a][m] * c;
}

// Weights and gradients of event e from its kinematics and f = |m|^2 (in the
// unit c); get(a, g4, ge) gives df/dk' of colour position a (k' = c k; zero
// for position 0) and df/d eps (g(z) = df/dRe z + i df/dIm z).  Same
// function as grad_outputs: w = wfac(x, H_T) E(k), E = efac' f; all
// gradients carried in units of A = up wfac efac'.
template <int N, typename Get>
__device__ __forceinline__ void grad_outputs_f32(const GradParams &G, uint64_t e, const GradKinF<N> &K, uint32_t hel,
                                                 double f, Get get) {
  constexpr int M = N - 2, L = N - 1, NU = 2 + 4 * M;
  const EventParams &P = G.P;
  const float lnx = P.f_lnxmin;
  const float c = ldexpf(1.f, -K.ex);

  // weight factors as the kinematics kernel forms them: wfac = wk F 2^(2 ex
  // (m-3)) with F the FP32 product of PDFs, couplings and the scaled s_hat
  double w = 0.0, A = 0.0;
  float as = 0.f;
  if (K.pass) {
    const float mu = P.f_mu_r_factor * K.ht;
    as = P.f_alphas_mz / (1.f + P.f_asb0 * (logf(mu * mu) - P.f_ln_mz2));
    const float g2 = 4.f * 3.14159265358979323846f * as;
    const float t1 = 1.f - K.x1, t2 = 1.f - K.x2;
    const float t1s = t1 * t1, t2s = t2 * t2;
    float F = 2.89f * expf(-0.2f * lnx * (K.ux1 + K.ux2)) * (t1s * t1s * t1) * (t2s * t2s * t2);
#pragma unroll
    for (int i = 0; i < N - 2; ++i) F *= g2;
    const float sp = K.shat_hi * c * c;
    if (M >= 3) {
#pragma unroll
      for (int i = 0; i < M - 3; ++i) F *= sp;
    } else {
      F /= sp;
    }
    if (F > 0.f) {
      const double wf = scale_pow2(P.wk * f64_of_f32_scaled(F, 0), 2 * K.ex * (M - 3));
      const double Aw = wf * scale_pow2(P.efac, -2 * K.ex * (N - 4));
      w = Aw * f;
      A = (G.dL_dw ? G.dL_dw[e] : 1.0) * Aw;
    }
  }
  if (G.w) G.w[e] = w;
  double *gu = G.dw_du ? G.dw_du + e * NU : nullptr;
  double *gkout = G.dw_dk ? G.dw_dk + e * N * 4 : nullptr;
  if (A == 0.0) {  // failing event or zero upstream gradient
    if (G.dw_dlnmu) G.dw_dlnmu[e] = 0.0;
    if (gkout)
#pragma unroll
      for (int i = 0; i < 4 * N; ++i) gkout[i] = 0.0;
    if (gu)
#pragma unroll
      for (int j = 0; j < NU; ++j) gu[j] = 0.0;
    return;
  }
  const ScaledOut out(A);
  const float ff = f32_of_f64(f);
  const float b0 = P.f_asb0 / P.f_alphas_mz;
  const float dlnw_dlnmu = -2.f * (float)(N - 2) * b0 * as;  // one-loop running
  if (G.dw_dlnmu) G.dw_dlnmu[e] = out(ff * dlnw_dlnmu);

  // dE/dk per leg in units of A (K-sum path through k' = c k, polarisation
  // path through the direction of k), plus E dwfac/dH_T dH_T/dk
  float gt[N][4];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) gt[i][m] = 0.f;
#pragma unroll
  for (int a = 0; a <= L; ++a) {
    const int leg = K.legp[a];
    float g4[4] = {0.f, 0.f, 0.f, 0.f};
    CV4<float> ge;
    get(a, g4, ge);
    const float sg = leg < 2 ? -1.f : 1.f;
    const float pphys[3] = {sg * K.kp[a][1], sg * K.kp[a][2], sg * K.kp[a][3]};
    float gre[4], gim[4], gp[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      gre[m] = ge.c[m].re;
      gim[m] = ge.c[m].im;
    }
    polvec_adjoint<float>(pphys, (hel >> leg) & 1u, gre, gim, gp);
#pragma unroll
    for (int s2 = 0; s2 < N; ++s2) {
      if (s2 == leg) {
        gt[s2][0] += c * g4[0];
#pragma unroll
        for (int j = 0; j < 3; ++j) gt[s2][1 + j] += c * g4[1 + j] + sg * gp[j];
      }
    }
  }
  {
    const float eht = ff * dlnw_dlnmu / K.ht;  // d ln wfac / d H_T = -2 (n-2) b0 alpha_s / H_T
#pragma unroll
    for (int i = 2; i < N; ++i) {
      const float px = K.kk[i][1], py = K.kk[i][2];
      const float ipt = rsqrtf(px * px + py * py);
      gt[i][1] += eht * px * ipt;
      gt[i][2] += eht * py * ipt;
    }
  }
  if (gkout)
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) gkout[i * 4 + m] = out(gt[i][m]);
  if (!gu) return;
  // x uniforms: w is homogeneous in the momenta (degree 8 - 2n) and H_T
  // scales with sqrt(s_hat):
  // d ln w / d ln x = x f'/f + (m - 3) - (n - 2) b0 alpha_s + (4 - n)
  const float xv[2] = {K.x1, K.x2};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float x = xv[j];
    const float dl = -0.2f - 5.f * x / (1.f - x) + (float)(M - 3) + 0.5f * dlnw_dlnmu + (float)(4 - N);
    gu[j] = out(ff * dl * lnx);
  }
  // Rambo uniforms: reverse through the boost/rescale and the seed map
  float gx = 0.f, ggam = 0.f, gaa = 0.f, gM = 0.f, gb[3] = {0.f, 0.f, 0.f}, gQ[4] = {0.f, 0.f, 0.f, 0.f};
  float gq[M][4], gbq[M], gf[M];
  const float gam = K.gam, aa = K.aa, xs = K.xs, iMq = K.iMq;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const float(&gpi)[4] = gt[2 + i];
    gx += gpi[0] * (gam * K.q[i][0] + K.bq[i]);
    ggam += gpi[0] * xs * K.q[i][0];
    gq[i][0] = gpi[0] * xs * gam;
    gbq[i] = gpi[0] * xs;
    gf[i] = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      gx += gpi[1 + j] * (K.q[i][1 + j] + K.bv[j] * K.fq[i]);
      gq[i][1 + j] = gpi[1 + j] * xs;
      gb[j] += gpi[1 + j] * xs * K.fq[i];
      gf[i] += gpi[1 + j] * xs * K.bv[j];
    }
    gq[i][0] += gf[i];
    gaa += gf[i] * K.bq[i];
    gbq[i] += gf[i] * aa;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      gb[j] += gbq[i] * K.q[i][1 + j];
      gq[i][1 + j] += gbq[i] * K.bv[j];
    }
  }
  ggam += gaa * (-aa * aa);
  gM += gx * (-xs * iMq);
  gQ[0] += ggam * iMq;
  gM += ggam * (-gam * iMq);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    gQ[1 + j] += -gb[j] * iMq;
    gM += gb[j] * (-K.bv[j] * iMq);
  }
  gQ[0] += gM * K.Q[0] * iMq;
  gQ[1] += gM * (-K.Q[1] * iMq);
  gQ[2] += gM * (-K.Q[2] * iMq);
  gQ[3] += gM * (-K.Q[3] * iMq);
#pragma unroll
  for (int i = 0; i < M; ++i) {
#pragma unroll
    for (int m = 0; m < 4; ++m) gq[i][m] += gQ[m];
    const float q0 = K.q0v[i], s = K.sth[i], cc = K.cth[i], cs = K.cph[i], sn = K.sph[i];
    const float gq0 = gq[i][0] + gq[i][1] * s * cs + gq[i][2] * s * sn + gq[i][3] * cc;
    const float gs = gq[i][1] * q0 * cs + gq[i][2] * q0 * sn;
    const float gc = gq[i][3] * q0 + gs * (-cc / s);
    const float gphi = gq[i][1] * (-q0 * s * sn) + gq[i][2] * (q0 * s * cs);
    gu[2 + 4 * i + 0] = out(2.f * gc);
    gu[2 + 4 * i + 1] = out(2.f * 3.14159265358979323846f * gphi);
    gu[2 + 4 * i + 2] = out(-gq0 / K.u3[i]);
    gu[2 + 4 * i + 3] = out(-gq0 / K.u4[i]);
  }
}

}  // namespace tess
