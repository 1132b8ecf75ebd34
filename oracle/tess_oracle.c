/*
 * tess_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for the
 * leading-order, leading-colour gg -> (n-2) gluon event generator of
 * Giele, Stavenga, Winter, "Thread-Scalable Evaluation of Multi-Jet
 * Observables" (arXiv:1002.3446).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path and must never be used as a
 * fallback for it.
 *
 * Everything is FP64 (C99 double / double complex).  Each function names
 * the section / equation of the paper it restates.  Where the paper is
 * silent the reading used is stated at the function.
 *
 * Conventions
 *   n      total number of gluons (paper's n); m = n - 2 final-state gluons.
 *   L      n - 1 legs of the Berends-Giele current (leg 1 is the off-shell
 *          leg that is finally contracted, Sec. 3 "amplitude" equation).
 *   metric (+,-,-,-); all four-vectors stored contravariantly, index 0 = E.
 *   k_i    all-outgoing momenta: k_1 = -p_1, k_2 = -p_2, k_i = p_i (i >= 3),
 *          so that sum_i k_i = 0.
 *
 * Pins (see the test-suite): Philox4x32-10 against the published known-answer
 * vectors of Salmon et al.'s Random123 library.  Conventions of this
 * implementation with nothing external to pin them: the layout of the draws
 * in the counter-based stream, the histogram range of the 2 -> 2
 * leading-jet-pT histogram, and the choice of x_min (cross-section neutral
 * by construction).
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 12
#define ORC_MAXL (ORC_MAXN - 1)

/* ------------------------------------------------------------------------
 * Process description (mirrors nothing on the CUDA side; own layout).
 * ---------------------------------------------------------------------- */
typedef struct {
  int n;               /* total gluons 4..12                              */
  int hel_mode;        /* 0: exact sum over helicities and orderings;     */
                       /* 1: one helicity + ordering sampled per event;   */
                       /* 2: random real polarisations + sampled ordering */
  double sqrt_s;       /* hadronic centre-of-mass energy, GeV             */
  double pt_min;       /* jet cuts, Sec. 4: pT > pt_min (GeV)             */
  double eta_max;      /*            |eta| < eta_max                      */
  double dr_min;       /*            Delta R > dr_min                     */
  double alphas_mz;    /* alpha_s(M_Z)                                    */
  double mz;           /* M_Z (GeV)                                       */
  int nf;              /* active flavours in the one-loop running         */
  int hist_obs;        /* 0: leading-jet pT, 1: H_T, 2: R_min             */
  double mu_r_factor;  /* mu_R = mu_r_factor * H_T                        */
  int hist_bins;       /* number of uniform bins in [hist_lo, hist_hi)    */
  int grid;            /* 1: PDF and alpha_s from interpolation grids     */
  double hist_lo, hist_hi;
} orc_process;

/* ========================================================================
 * 1. Counter-based random numbers.
 *    The paper does not name its generator (Sec. 4, discussion of Fig. 2:
 *    only that the draw count is of the order of the square root of the
 *    cycle length).  Reading: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 *    SC'11), written here from that paper's description: ten rounds of
 *    two 32x32->64 multiplications with a Weyl-sequence key schedule.
 * ====================================================================== */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
  const uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
  const uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
  const uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
  const uint32_t n0 = hi1 ^ c[1] ^ k[0];
  const uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k[0] += 0x9E3779B9u; /* golden ratio          */
      k[1] += 0xBB67AE85u; /* sqrt(3) - 1           */
    }
    philox_round(c, k);
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* The j-th uniform of event `ev`: counter (ev_lo, ev_hi, j/2, 0), key
 * (seed_lo, seed_hi); two 32-bit words (a, b) of the block give the 52-bit
 * integer k = (a >> 6) 2^26 + (b >> 6) and u = (k + 1/2) 2^-52, which is
 * exact in double precision and strictly inside (0,1):
 * 2^-53 <= u <= 1 - 2^-53.                                                */
double orc_uniform(uint64_t seed, uint64_t ev, uint32_t j) {
  const uint32_t ctr[4] = {(uint32_t)ev, (uint32_t)(ev >> 32), j >> 1, 0u};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  const uint32_t a = w[2 * (j & 1u)], b = w[2 * (j & 1u) + 1];
  const double hi = (double)(a >> 6), lo = (double)(b >> 6);
  return (hi * 67108864.0 + lo + 0.5) * (1.0 / 4503599627370496.0);
}

/* Per-event draw layout (fixed for every mode so that x and the momenta of
 * an event do not depend on how its amplitude is summed):
 *   u[0], u[1]            x1, x2
 *   u[2 .. 2+4m)          Rambo, four per final-state gluon
 *   u[2+4m]               helicity word: top n bits of u
 *   u[3+4m .. 3+4m+n-2)   colour ordering (Fisher-Yates on {2..n})
 * and, in the random-polarisation mode only,
 *   u[1+4m+n .. 1+5m+2n)  polarisation angle of leg i = 0..n-1: phi = 2 pi u */
int orc_n_uniforms(int n) { return 2 + 4 * (n - 2) + 1 + (n - 2); }
int orc_n_uniforms_mode(int n, int hel_mode) { return orc_n_uniforms(n) + (hel_mode == 2 ? n : 0); }

/* ========================================================================
 * 2. Parton luminosity.  Sec. 3, cross-section formula: the integrand has
 *    F_g(x1) F_g(x2) / (4 p1.p2).  Toy gluon density x g(x) = 1.7 x^-0.2
 *    (1-x)^5 (replacing CTEQ6L1, which is not available); x sampled
 *    uniformly in ln x on [ln x_min, 0], so dx = x |ln x_min| du and the
 *    Jacobian-weighted density is (ln x_min)^2 f(x1) f(x2).
 *    Reading: x_min = tau_min = (m pT_min)^2 / S.  Any event passing the
 *    cuts has sqrt(s_hat) >= sum_i E_i >= sum_i pT_i > m pT_min, so the
 *    choice removes no accepted event.
 * ====================================================================== */
double orc_xg(double x) { return 1.7 * pow(x, -0.2) * pow(1.0 - x, 5.0); }

/* Grid mode (the paper's mechanism, Sec. 3: PDF and alpha_s read from
 * tables by linear interpolation).  The tables are built from the functions
 * above and interpolated in single precision:
 *   PDF: 1025 nodes u_i = i/1024 of the x draw (ln x = u ln x_min), value
 *        float(xg(exp(u_i ln x_min))); at a float draw u: s = 1024 u,
 *        i = min(floor(s), 1023), t = s - i, f = fma(t, g[i+1] - g[i], g[i]).
 *   alpha_s: 513 nodes uniform in v = ln mu^2 over [v_lo, v_hi],
 *        v_lo = 2 ln(mu_r_factor m pT_min) (no passing event has a smaller
 *        H_T), v_hi = 2 ln(mu_r_factor sqrt(S)); value float(alpha_s(mu));
 *        at v: s = (v - v_lo) * float(512 / (v_hi - v_lo)) clamped to
 *        [0, 512], i = min(floor(s), 511), t = s - i, same blend.
 * Every step in float arithmetic (fmaf rounds once), as the grid-mode
 * kernels evaluate it.                                                    */
#define ORC_PDF_NODES 1025
#define ORC_AS_NODES 513
static float grid_blend(const float *g, int nseg, float s) {
  if (s < 0.0f) s = 0.0f;
  if (s > (float)nseg) s = (float)nseg;
  int i = (int)s;
  if (i > nseg - 1) i = nseg - 1;
  const float t = s - (float)i;
  return fmaf(t, g[i + 1] - g[i], g[i]);
}

float orc_grid_pdf(const orc_process *pr, float u) {
  float g[ORC_PDF_NODES];
  const int m = pr->n - 2;
  const double S = pr->sqrt_s * pr->sqrt_s;
  const double lnxmin = log((m * pr->pt_min) * (m * pr->pt_min) / S);
  for (int i = 0; i < ORC_PDF_NODES; ++i) g[i] = (float)orc_xg(exp((double)i / 1024.0 * lnxmin));
  return grid_blend(g, ORC_PDF_NODES - 1, u * 1024.0f);
}

double orc_alphas(double mu, double alphas_mz, double mz, int nf);
float orc_grid_alphas(const orc_process *pr, float v) {
  float a[ORC_AS_NODES];
  const int m = pr->n - 2;
  const double vlo = 2.0 * log(pr->mu_r_factor * m * pr->pt_min), vhi = 2.0 * log(pr->mu_r_factor * pr->sqrt_s);
  for (int i = 0; i < ORC_AS_NODES; ++i)
    a[i] = (float)orc_alphas(exp(0.5 * (vlo + (vhi - vlo) * i / 512.0)), pr->alphas_mz, pr->mz, pr->nf);
  const float inv = (float)(512.0 / (vhi - vlo));
  return grid_blend(a, ORC_AS_NODES - 1, (v - (float)vlo) * inv);
}

/* ========================================================================
 * 3. Rambo (Kleiss, Stirling, Ellis 1986), cited but not restated in
 *    Sec. 3 ("unit-weight phase-space generator").  m massless momenta in
 *    the partonic centre-of-mass frame with total energy sqrt_shat; the
 *    weight is the same for every event (flat phase space).
 * ====================================================================== */
void orc_rambo(int m, double sqrt_shat, const double *u, double *p /* m x 4 */) {
  double q[ORC_MAXN][4];
  double Q[4] = {0, 0, 0, 0};
  for (int i = 0; i < m; ++i) {
    const double c = 2.0 * u[4 * i + 0] - 1.0;
    const double s = sqrt(1.0 - c * c);
    const double phi = 2.0 * M_PI * u[4 * i + 1];
    const double q0 = -log(u[4 * i + 2] * u[4 * i + 3]);
    q[i][0] = q0;
    q[i][1] = q0 * s * cos(phi);
    q[i][2] = q0 * s * sin(phi);
    q[i][3] = q0 * c;
    for (int mu = 0; mu < 4; ++mu) Q[mu] += q[i][mu];
  }
  const double M = sqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
  const double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
  const double gamma = Q[0] / M;
  const double a = 1.0 / (1.0 + gamma);
  const double x = sqrt_shat / M;
  for (int i = 0; i < m; ++i) {
    const double bq = b[0] * q[i][1] + b[1] * q[i][2] + b[2] * q[i][3];
    p[4 * i + 0] = x * (gamma * q[i][0] + bq);
    for (int k = 0; k < 3; ++k) p[4 * i + 1 + k] = x * (q[i][1 + k] + b[k] * q[i][0] + a * bq * b[k]);
  }
}

/* Flat massless m-body phase-space volume, including the (2 pi) factors of
 * the Lorentz-invariant measure:
 *   Phi_m(s) = (2pi)^(4-3m) (pi/2)^(m-1) s^(m-2) / ((m-1)! (m-2)!).        */
double orc_rambo_weight(int m, double shat) {
  double fm1 = 1.0, fm2 = 1.0;
  for (int i = 2; i <= m - 1; ++i) fm1 *= i;
  for (int i = 2; i <= m - 2; ++i) fm2 *= i;
  return pow(2.0 * M_PI, 4.0 - 3.0 * m) * pow(M_PI / 2.0, m - 1.0) * pow(shat, m - 2.0) / (fm1 * fm2);
}

/* ========================================================================
 * 4. Cuts and observables, Sec. 3 (phase-space weight stage) and Sec. 4
 *    (jet cuts pT > pT_min, |eta| < eta_max, Delta R > dr_min; H_T;
 *    R_min = min over pairs of Delta R).  Every final-state gluon is a jet.
 *    A failing event is only flagged (Sec. 3).  Momenta p are in the
 *    partonic frame; the lab rapidity is eta + y with y = ln(x1/x2)/2.
 *    Returns the pass flag; writes H_T, leading pT and R_min.
 * ====================================================================== */
int orc_cuts(int m, const double *p, double y, double pt_min, double eta_max, double dr_min,
             double *ht, double *ptlead, double *rmin) {
  double pt[ORC_MAXN], eta[ORC_MAXN];
  int pass = 1;
  double sum = 0.0, lead = 0.0;
  for (int i = 0; i < m; ++i) {
    const double px = p[4 * i + 1], py = p[4 * i + 2], pz = p[4 * i + 3];
    const double pabs = sqrt(px * px + py * py + pz * pz);
    pt[i] = sqrt(px * px + py * py);
    eta[i] = 0.5 * log((pabs + pz) / (pabs - pz)) + y;
    sum += pt[i];
    if (pt[i] > lead) lead = pt[i];
    if (!(pt[i] > pt_min)) pass = 0;
    if (!(fabs(eta[i]) < eta_max)) pass = 0;
  }
  double dr2min = INFINITY;
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) {
      const double pxi = p[4 * i + 1], pyi = p[4 * i + 2], pxj = p[4 * j + 1], pyj = p[4 * j + 2];
      const double dphi = atan2(fabs(pxi * pyj - pyi * pxj), pxi * pxj + pyi * pyj);
      const double deta = eta[i] - eta[j];
      const double dr2 = deta * deta + dphi * dphi;
      if (dr2 < dr2min) dr2min = dr2;
      if (!(dr2 > dr_min * dr_min)) pass = 0;
    }
  *ht = sum;
  *ptlead = lead;
  *rmin = sqrt(dr2min);
  return pass;
}

/* ========================================================================
 * 5. Strong coupling, one loop (the paper interpolates a grid in mu,
 *    Sec. 3; the closed form is used here):
 *    alpha_s(mu) = a0 / (1 + a0 b0 ln(mu^2 / M_Z^2)), b0 = (33 - 2 nf)/(12 pi).
 * ====================================================================== */
double orc_alphas(double mu, double alphas_mz, double mz, int nf) {
  const double b0 = (33.0 - 2.0 * nf) / (12.0 * M_PI);
  return alphas_mz / (1.0 + alphas_mz * b0 * log(mu * mu / (mz * mz)));
}

/* ========================================================================
 * 6. Polarisation vectors (helicity form).  Sec. 3 names conventional
 *    helicity vectors as the alternative to its random real vectors.  For
 *    direction (sin t cos f, sin t sin f, cos t):
 *      e1 = (0, cos t cos f, cos t sin f, -sin t), e2 = (0, -sin f, cos f, 0)
 *      eps_+ = -(e1 + i e2)/sqrt2,  eps_- = (e1 - i e2)/sqrt2.
 *    Built from the physical momentum p of the leg (incoming legs use their
 *    physical direction); a leg along the beam axis takes f = 0.
 *    h = 0 -> eps_+, h = 1 -> eps_-.   Output: 4 complex = 8 doubles
 *    interleaved (re, im).
 * ====================================================================== */
void orc_polvec(const double *p, int h, double *eps) {
  const double px = p[1], py = p[2], pz = p[3];
  const double pt = sqrt(px * px + py * py);
  const double pabs = sqrt(px * px + py * py + pz * pz);
  const double ct = pz / pabs, st = pt / pabs;
  const double cf = pt > 0.0 ? px / pt : 1.0;
  const double sf = pt > 0.0 ? py / pt : 0.0;
  const double e1[4] = {0.0, ct * cf, ct * sf, -st};
  const double e2[4] = {0.0, -sf, cf, 0.0};
  const double r = 1.0 / sqrt(2.0);
  for (int mu = 0; mu < 4; ++mu) {
    double complex e = (h == 0) ? -(e1[mu] + I * e2[mu]) * r : (e1[mu] - I * e2[mu]) * r;
    eps[2 * mu] = creal(e);
    eps[2 * mu + 1] = cimag(e);
  }
}

/* Random real polarisation, Sec. 3 (the paper's own choice): a random unit
 * vector orthogonal to the gluon momentum, eps = cos(phi) e1 + sin(phi) e2
 * with e1, e2 the transverse basis above and phi uniform in [0, 2 pi).
 * The currents are then real.  Since the amplitude is linear in each eps and
 * E[cos^2] = E[sin^2] = 1/2, E[cos sin] = 0 for independent angles,
 * E_phi |m(eps(phi))|^2 = 2^-n sum over the basis {e1, e2}^n of |m|^2, and
 * by completeness (eps_+, eps_- and e1, e2 span the same transverse plane,
 * related by a unitary map) that basis sum equals the helicity sum: 2^n
 * |m(eps(phi))|^2 estimates sum_h |m_h|^2 without bias.
 * Output as orc_polvec: 4 complex (imaginary parts zero) = 8 doubles.      */
void orc_polvec_real(const double *p, double phi, double *eps) {
  const double px = p[1], py = p[2], pz = p[3];
  const double pt = sqrt(px * px + py * py);
  const double pabs = sqrt(px * px + py * py + pz * pz);
  const double ct = pz / pabs, st = pt / pabs;
  const double cf = pt > 0.0 ? px / pt : 1.0;
  const double sf = pt > 0.0 ? py / pt : 0.0;
  const double e1[4] = {0.0, ct * cf, ct * sf, -st};
  const double e2[4] = {0.0, -sf, cf, 0.0};
  const double c = cos(phi), s = sin(phi);
  for (int mu = 0; mu < 4; ++mu) {
    eps[2 * mu] = c * e1[mu] + s * e2[mu];
    eps[2 * mu + 1] = 0.0;
  }
}

/* ========================================================================
 * 7. Berends-Giele recursion, Sec. 3, Eq. (BG-recursion) and the shorthand
 *    equation that follows it:
 *      J[m..n] = 1/K[m..n]^2 ( sum_i [J[m..i], J[i+1..n]]
 *                             + sum_{i<j} {J[m..i], J[i+1..j], J[j+1..n]} )
 *      [a,b]   = 2 (J_a.K_b) J_b - 2 (K_a.J_b) J_a + (J_a.J_b)(K_a - K_b)
 *      {a,b,c} = 2 (J_a.J_c) J_b - (J_a.J_b) J_c - (J_c.J_b) J_a
 *    with J[i] = polarisation vector, K[m..n] = sum of the momenta.
 *    The full current is kept un-propagated (its K^2 vanishes on shell),
 *    which is the amputation of the "amplitude" equation:
 *      m = (J[2..n] . J[1]) x K^2[2..n]   (leg 1 off-shell, as in Sec. 3's
 *      implementation text and Sec. 4's gauge check).
 * ====================================================================== */
typedef double complex cvec[4];

static double complex mdot_cc(const cvec a, const cvec b) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
static double complex mdot_cr(const cvec a, const double *b) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
static double mdot_rr(const double *a, const double *b) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

/* [a,b]_mu, the three-gluon-vertex shorthand. */
static void bg_bracket(const cvec Ja, const double *Ka, const cvec Jb, const double *Kb, cvec out) {
  const double complex JaKb = mdot_cr(Ja, Kb);
  const double complex KaJb = mdot_cr(Jb, Ka);
  const double complex JaJb = mdot_cc(Ja, Jb);
  for (int mu = 0; mu < 4; ++mu)
    out[mu] = 2.0 * JaKb * Jb[mu] - 2.0 * KaJb * Ja[mu] + JaJb * (Ka[mu] - Kb[mu]);
}

/* {a,b,c}_mu, the four-gluon-vertex shorthand. */
static void bg_brace(const cvec Ja, const cvec Jb, const cvec Jc, cvec out) {
  const double complex JaJc = mdot_cc(Ja, Jc);
  const double complex JaJb = mdot_cc(Ja, Jb);
  const double complex JcJb = mdot_cc(Jc, Jb);
  for (int mu = 0; mu < 4; ++mu) out[mu] = 2.0 * JaJc * Jb[mu] - JaJb * Jc[mu] - JcJb * Ja[mu];
}

/* Currents of legs lk[0..L) with polarisations le[0..L) (complex), in the
 * order given; writes the un-propagated top current Num = K^2 J[1..L].
 * J and K tables are indexed [first leg][last leg] as in the paper.    */
static void bg_top_current(int L, double lk[][4], cvec *le, cvec num) {
  static __thread cvec J[ORC_MAXL][ORC_MAXL];
  static __thread double K[ORC_MAXL][ORC_MAXL][4];
  for (int a = 0; a < L; ++a) {
    for (int mu = 0; mu < 4; ++mu) {
      J[a][a][mu] = le[a][mu];
      K[a][a][mu] = lk[a][mu];
    }
  }
  for (int len = 2; len <= L; ++len) {
    for (int m = 0; m + len - 1 < L; ++m) {
      const int n = m + len - 1;
      for (int mu = 0; mu < 4; ++mu) K[m][n][mu] = K[m][n - 1][mu] + lk[n][mu];
      cvec acc = {0, 0, 0, 0}, t;
      for (int i = m; i <= n - 1; ++i) {
        bg_bracket(J[m][i], K[m][i], J[i + 1][n], K[i + 1][n], t);
        for (int mu = 0; mu < 4; ++mu) acc[mu] += t[mu];
      }
      for (int i = m; i <= n - 2; ++i)
        for (int j = i + 1; j <= n - 1; ++j) {
          bg_brace(J[m][i], J[i + 1][j], J[j + 1][n], t);
          for (int mu = 0; mu < 4; ++mu) acc[mu] += t[mu];
        }
      if (len < L) {
        const double K2 = mdot_rr(K[m][n], K[m][n]);
        for (int mu = 0; mu < 4; ++mu) J[m][n][mu] = acc[mu] / K2;
      } else {
        for (int mu = 0; mu < 4; ++mu) num[mu] = acc[mu];
      }
    }
  }
}

/* The same current from the rewritten recursion of Sec. 3 (the O(n^3)
 * "W tensor" equation), with the propagator 1/K^2 that the printed
 * equation omits restored (without it the two forms differ):
 *   J[m..n] = 1/K^2 sum_i ( W[i+1..n].J[m..i] - W[m..i].J[i+1..n] )
 *   W^{mu nu}[S] = 2 J^mu K^nu - K^mu J^nu
 *                  + sum_{splits (l,r) of S} (J_l^mu J_r^nu - J_r^mu J_l^nu)
 *   (W.J)^mu = W^{mu nu} J_nu.                                            */
static void bg_top_current_w(int L, double lk[][4], cvec *le, cvec num) {
  static __thread cvec J[ORC_MAXL][ORC_MAXL];
  static __thread double K[ORC_MAXL][ORC_MAXL][4];
  static __thread double complex W[ORC_MAXL][ORC_MAXL][4][4];
  static const double g[4] = {1.0, -1.0, -1.0, -1.0};
  for (int len = 1; len <= L; ++len) {
    for (int m = 0; m + len - 1 < L; ++m) {
      const int n = m + len - 1;
      if (len == 1) {
        for (int mu = 0; mu < 4; ++mu) {
          J[m][n][mu] = le[m][mu];
          K[m][n][mu] = lk[m][mu];
        }
      } else {
        for (int mu = 0; mu < 4; ++mu) K[m][n][mu] = K[m][n - 1][mu] + lk[n][mu];
        cvec acc = {0, 0, 0, 0};
        for (int i = m; i <= n - 1; ++i)
          for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu)
              acc[mu] += g[nu] * (W[i + 1][n][mu][nu] * J[m][i][nu] - W[m][i][mu][nu] * J[i + 1][n][nu]);
        if (len < L) {
          const double K2 = mdot_rr(K[m][n], K[m][n]);
          for (int mu = 0; mu < 4; ++mu) J[m][n][mu] = acc[mu] / K2;
        } else {
          for (int mu = 0; mu < 4; ++mu) num[mu] = acc[mu];
          continue; /* the top set needs no tensor */
        }
      }
      for (int mu = 0; mu < 4; ++mu)
        for (int nu = 0; nu < 4; ++nu) {
          double complex w = 2.0 * J[m][n][mu] * K[m][n][nu] - K[m][n][mu] * J[m][n][nu];
          for (int i = m; i <= n - 1; ++i) w += J[m][i][mu] * J[i + 1][n][nu] - J[i + 1][n][mu] * J[m][i][nu];
          W[m][n][mu][nu] = w;
        }
    }
  }
}

/* Colour-ordered amplitude in the paper's normalisation,
 *   m(o_0, o_1, ..., o_{n-1}) = eps_{o_0} . Num[o_1 .. o_{n-1}],
 * for the cyclic ordering `order` (0-based leg labels), all-outgoing
 * momenta k (n x 4) and polarisations eps (n x 8, interleaved re/im).
 * form 0: Eq. (BG-recursion); form 1: the W-tensor rewrite.  out = (re, im). */
void orc_amp(int n, const int *order, const double *k, const double *eps, int form, double *out) {
  double lk[ORC_MAXL][4];
  cvec le[ORC_MAXL], num, e0;
  const int L = n - 1;
  for (int a = 0; a < L; ++a) {
    const int leg = order[a + 1];
    for (int mu = 0; mu < 4; ++mu) {
      lk[a][mu] = k[4 * leg + mu];
      le[a][mu] = eps[8 * leg + 2 * mu] + I * eps[8 * leg + 2 * mu + 1];
    }
  }
  for (int mu = 0; mu < 4; ++mu) e0[mu] = eps[8 * order[0] + 2 * mu] + I * eps[8 * order[0] + 2 * mu + 1];
  if (form == 0)
    bg_top_current(L, lk, le, num);
  else
    bg_top_current_w(L, lk, le, num);
  const double complex amp = mdot_cc(e0, num);
  out[0] = creal(amp);
  out[1] = cimag(amp);
}

/* ========================================================================
 * 8. Event: Sec. 3 stages in order -- phase space (Rambo), phase-space
 *    weight (PDF, alpha_s, cuts, observables), matrix-element weight,
 *    epilogue -- and the cross-section formula at the end of Sec. 3:
 *      dsigma = dx1 dx2 F(x1)F(x2)/(4 p1.p2) 1/(n-2)! dPhi sum_pi |m|^2.
 *    Leading colour (Sec. 3, colour-summed square):
 *      sum_col |A|^2 = g^(2n-4) N^(n-2) (N^2-1) sum_{sigma in S_(n-1)} |A_D(1,sigma)|^2
 *    with A_D the colour-ordered amplitude for Tr(T^a T^b) = delta^ab.  The
 *    paper's vertex normalisation gives |A_D|^2 = |m|^2 / 2^(n-2).
 *    Average over initial colours and helicities: 1/(4 * 64).
 *    hel_mode 0: E = sum_hel sum_sigma |A_D|^2 (exact);
 *    hel_mode 1: E = 2^n (n-1)! |A_D(1, sigma; h)|^2 for one sampled
 *    (sigma, h) -- the unbiased estimator of the same sum; with the
 *    final-state symmetry 1/(n-2)! this is the paper's (n-1)|m|^2.
 *    hel_mode 2: the same with random real polarisations in place of the
 *    sampled helicities (orc_polvec_real), Sec. 3's own choice.
 * ====================================================================== */
typedef struct {
  double x1, x2, shat, y, alphas, ht, ptlead, rmin, me2, weight, pdf, phi;
  int pass, hel_bits;
  int perm[ORC_MAXN];
  double k[ORC_MAXN][4]; /* all-outgoing momenta                       */
} orc_event_out;

#define GEV2_TO_PB 0.3893793721e9
#define NC 3.0

/* Kinematics, helicity word and colour ordering from the event's uniforms
 * u[0 .. orc_n_uniforms(n)) in the layout of Sec. 1 above. */
static void event_kinematics(const orc_process *pr, const double *u, orc_event_out *o) {
  const int n = pr->n, m = n - 2;
  const double S = pr->sqrt_s * pr->sqrt_s;
  const double lnxmin = log((m * pr->pt_min) * (m * pr->pt_min) / S);
  o->x1 = exp(u[0] * lnxmin);
  o->x2 = exp(u[1] * lnxmin);
  o->shat = o->x1 * o->x2 * S;
  if (pr->grid) /* the grid-mode kernels read the draws as floats */
    o->pdf = lnxmin * lnxmin * (double)orc_grid_pdf(pr, (float)u[0]) * (double)orc_grid_pdf(pr, (float)u[1]);
  else
    o->pdf = lnxmin * lnxmin * orc_xg(o->x1) * orc_xg(o->x2);
  o->y = 0.5 * log(o->x1 / o->x2);
  const double rs = sqrt(o->shat);
  double p[ORC_MAXN * 4];
  orc_rambo(m, rs, u + 2, p);
  /* all-outgoing momenta: k1 = -p1, k2 = -p2 with p1,2 = rs/2 (1,0,0,+-1) */
  const double h = 0.5 * rs;
  const double p1[4] = {h, 0, 0, h}, p2[4] = {h, 0, 0, -h};
  for (int mu = 0; mu < 4; ++mu) {
    o->k[0][mu] = -p1[mu];
    o->k[1][mu] = -p2[mu];
  }
  for (int i = 0; i < m; ++i)
    for (int mu = 0; mu < 4; ++mu) o->k[2 + i][mu] = p[4 * i + mu];
  o->phi = orc_rambo_weight(m, o->shat);
  o->pass = orc_cuts(m, p, o->y, pr->pt_min, pr->eta_max, pr->dr_min, &o->ht, &o->ptlead, &o->rmin);
  /* helicity word and colour ordering */
  const double uh = u[2 + 4 * m];
  o->hel_bits = (int)floor(uh * (double)(1 << n));
  for (int i = 0; i < n; ++i) o->perm[i] = i;
  for (int i = n; i >= 3; --i) { /* positions 2..n (1-based) are shuffled */
    const double ui = u[3 + 4 * m + (n - i)];
    const int r = 2 + (int)floor(ui * (double)(i - 1)); /* 1-based in [2, i] */
    const int tmp = o->perm[i - 1];
    o->perm[i - 1] = o->perm[r - 1];
    o->perm[r - 1] = tmp;
  }
}

/* physical momentum of leg i (for the polarisation vector) */
static void physical_momentum(const orc_event_out *o, int leg, double *p) {
  const double s = leg < 2 ? -1.0 : 1.0;
  for (int mu = 0; mu < 4; ++mu) p[mu] = s * o->k[leg][mu];
}

static double amp2_dixon(int n, const int *order, const orc_event_out *o, int hel_bits) {
  double eps[ORC_MAXN * 8], pp[4], a[2];
  for (int i = 0; i < n; ++i) {
    physical_momentum(o, i, pp);
    orc_polvec(pp, (hel_bits >> i) & 1, eps + 8 * i);
  }
  orc_amp(n, order, &o->k[0][0], eps, 0, a);
  return (a[0] * a[0] + a[1] * a[1]) / pow(2.0, n - 2);
}

/* |A_D|^2 with the random real polarisations of the event's angle draws */
static double amp2_dixon_real(int n, const int *order, const orc_event_out *o, const double *uphi) {
  double eps[ORC_MAXN * 8], pp[4], a[2];
  for (int i = 0; i < n; ++i) {
    physical_momentum(o, i, pp);
    orc_polvec_real(pp, 2.0 * M_PI * uphi[i], eps + 8 * i);
  }
  orc_amp(n, order, &o->k[0][0], eps, 0, a);
  return (a[0] * a[0] + a[1] * a[1]) / pow(2.0, n - 2);
}

/* next permutation of v[0..len) in lexicographic order; 0 at the end */
static int next_perm(int *v, int len) {
  int i = len - 2;
  while (i >= 0 && v[i] >= v[i + 1]) --i;
  if (i < 0) return 0;
  int j = len - 1;
  while (v[j] <= v[i]) --j;
  int t = v[i]; v[i] = v[j]; v[j] = t;
  for (int a = i + 1, b = len - 1; a < b; ++a, --b) { t = v[a]; v[a] = v[b]; v[b] = t; }
  return 1;
}

static int event_from_uniforms(const orc_process *pr, const double *u, orc_event_out *o) {
  const int n = pr->n, m = n - 2;
  if (n < 4 || n > ORC_MAXN) return -1;
  event_kinematics(pr, u, o);
  double E = 0.0;
  if (pr->hel_mode == 0) {
    int order[ORC_MAXN];
    for (int i = 0; i < n; ++i) order[i] = i;
    do {
      for (int h = 0; h < (1 << n); ++h) E += amp2_dixon(n, order, o, h);
    } while (next_perm(order + 1, n - 1));
  } else {
    /* sampled ordering; one sampled helicity configuration (mode 1) or
     * random real polarisations (mode 2): both 2^n (n-1)! |A_D|^2 */
    double fact = 1.0;
    for (int i = 2; i <= n - 1; ++i) fact *= i;
    const double a2 = pr->hel_mode == 2 ? amp2_dixon_real(n, o->perm, o, u + orc_n_uniforms(n))
                                        : amp2_dixon(n, o->perm, o, o->hel_bits);
    E = (double)(1 << n) * fact * a2;
  }
  o->me2 = E;
  double w = 0.0;
  o->alphas = 0.0;
  if (o->pass) {
    double mfact = 1.0;
    for (int i = 2; i <= m; ++i) mfact *= i;
    if (pr->grid) {
      const float mu = (float)pr->mu_r_factor * (float)o->ht;
      o->alphas = (double)orc_grid_alphas(pr, logf(mu * mu));
    } else {
      o->alphas = orc_alphas(pr->mu_r_factor * o->ht, pr->alphas_mz, pr->mz, pr->nf);
    }
    const double col = pow(NC, n - 2) * (NC * NC - 1.0);
    const double g2 = 4.0 * M_PI * o->alphas;
    w = o->pdf / (2.0 * o->shat) * o->phi / mfact / 256.0 * col * pow(g2, n - 2) * E * GEV2_TO_PB;
  }
  o->weight = w;
  return 0;
}

int orc_event(const orc_process *pr, uint64_t seed, uint64_t ev, orc_event_out *o) {
  if (pr->n < 4 || pr->n > ORC_MAXN) return -1;
  double u[80];
  const int nu = orc_n_uniforms_mode(pr->n, pr->hel_mode);
  for (int j = 0; j < nu; ++j) u[j] = orc_uniform(seed, ev, (uint32_t)j);
  return event_from_uniforms(pr, u, o);
}

/* ========================================================================
 * 9. Accumulation.  Sec. 4 (Fig. 2): a single-precision running sum of
 *    ~1e11 weights underestimates sigma; compensated (Kahan) summation is
 *    used.  Neumaier's variant of compensated summation is used here.
 * ====================================================================== */
typedef struct { double s, c; } ksum;
static void ksum_add(ksum *k, double x) {
  const double t = k->s + x;
  if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
  else k->c += (x - t) + k->s;
  k->s = t;
}
static double ksum_val(const ksum *k) { return k->s + k->c; }

/* Histogram bin: 0 underflow, 1..nb uniform bins on [lo, hi), nb+1 overflow. */
int orc_hist_bin(double v, int nb, double lo, double hi) {
  if (!(v >= lo)) return 0;
  if (!(v < hi)) return nb + 1;
  int b = (int)floor((v - lo) / ((hi - lo) / nb));
  if (b > nb - 1) b = nb - 1;
  return 1 + b;
}

typedef struct {
  const orc_process *pr;
  uint64_t seed, first, count, out_offset;
  double *weight, *me2, *ht, *ptlead, *rmin;
  uint8_t *pass;
  ksum sw, sw2;
  uint64_t npass;
  ksum *hw, *hw2;
  int rc;
} orc_chunk;

static void *run_chunk(void *arg) {
  orc_chunk *c = (orc_chunk *)arg;
  const orc_process *pr = c->pr;
  orc_event_out o;
  for (uint64_t e = 0; e < c->count; ++e) {
    const uint64_t ev = c->first + e, idx = c->out_offset + e;
    if (orc_event(pr, c->seed, ev, &o) != 0) { c->rc = -1; return NULL; }
    if (c->weight) c->weight[idx] = o.weight;
    if (c->me2) c->me2[idx] = o.me2;
    if (c->pass) c->pass[idx] = (uint8_t)o.pass;
    if (c->ht) c->ht[idx] = o.ht;
    if (c->ptlead) c->ptlead[idx] = o.ptlead;
    if (c->rmin) c->rmin[idx] = o.rmin;
    ksum_add(&c->sw, o.weight);
    ksum_add(&c->sw2, o.weight * o.weight);
    if (o.pass) {
      c->npass += 1;
      if (c->hw) {
        const double v = pr->hist_obs == 0 ? o.ptlead : (pr->hist_obs == 1 ? o.ht : o.rmin);
        const int b = orc_hist_bin(v, pr->hist_bins, pr->hist_lo, pr->hist_hi);
        ksum_add(&c->hw[b], o.weight);
        ksum_add(&c->hw2[b], o.weight * o.weight);
      }
    }
  }
  return NULL;
}

/* Generate events [first, first + n_events) of stream `seed` on n_threads
 * host threads (contiguous chunks, combined in chunk order).
 * acc[0..3] = (sum w, sum w^2, n_pass, n_events); hist (optional) =
 * (sum w over bins 0..nb+1, then sum w^2 over bins 0..nb+1).
 * Per-event outputs may be NULL.  Returns 0 or -1. */
int orc_generate(const orc_process *pr, uint64_t seed, uint64_t first, uint64_t n_events, int n_threads,
                 double *weight, double *me2, uint8_t *pass, double *ht, double *ptlead, double *rmin,
                 double *acc, double *hist) {
  if (n_threads < 1) n_threads = 1;
  if ((uint64_t)n_threads > n_events && n_events > 0) n_threads = (int)n_events;
  const int nb = pr->hist_bins;
  orc_chunk *ch = calloc((size_t)n_threads, sizeof(orc_chunk));
  pthread_t *th = calloc((size_t)n_threads, sizeof(pthread_t));
  if (!ch || !th) { free(ch); free(th); return -1; }
  uint64_t start = 0;
  for (int t = 0; t < n_threads; ++t) {
    const uint64_t cnt = n_events / n_threads + ((uint64_t)t < n_events % n_threads ? 1 : 0);
    ch[t].pr = pr;
    ch[t].seed = seed;
    ch[t].first = first + start;
    ch[t].count = cnt;
    ch[t].out_offset = start;
    ch[t].weight = weight; ch[t].me2 = me2; ch[t].pass = pass;
    ch[t].ht = ht; ch[t].ptlead = ptlead; ch[t].rmin = rmin;
    if (hist) {
      ch[t].hw = calloc((size_t)(nb + 2), sizeof(ksum));
      ch[t].hw2 = calloc((size_t)(nb + 2), sizeof(ksum));
    }
    start += cnt;
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, run_chunk, &ch[t]);
  run_chunk(&ch[0]);
  for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
  int rc = 0;
  ksum sw = {0, 0}, sw2 = {0, 0};
  uint64_t npass = 0;
  for (int t = 0; t < n_threads; ++t) {
    if (ch[t].rc) rc = -1;
    ksum_add(&sw, ksum_val(&ch[t].sw));
    ksum_add(&sw2, ksum_val(&ch[t].sw2));
    npass += ch[t].npass;
  }
  if (acc) {
    acc[0] = ksum_val(&sw);
    acc[1] = ksum_val(&sw2);
    acc[2] = (double)npass;
    acc[3] = (double)n_events;
  }
  if (hist) {
    for (int b = 0; b < nb + 2; ++b) {
      ksum s = {0, 0}, s2 = {0, 0};
      for (int t = 0; t < n_threads; ++t) {
        ksum_add(&s, ksum_val(&ch[t].hw[b]));
        ksum_add(&s2, ksum_val(&ch[t].hw2[b]));
      }
      hist[b] = ksum_val(&s);
      hist[nb + 2 + b] = ksum_val(&s2);
    }
    for (int t = 0; t < n_threads; ++t) { free(ch[t].hw); free(ch[t].hw2); }
  }
  free(ch);
  free(th);
  return rc;
}

/* Single-event entry for tests: fills the fixed-layout record
 * rec[0..] = x1, x2, shat, y, alphas, ht, ptlead, rmin, me2, weight, pdf, phi,
 *            pass, hel_bits, perm[0..n), k[0..n)[4].                          */
int orc_event_record(const orc_process *pr, uint64_t seed, uint64_t ev, double *rec) {
  orc_event_out o;
  const int rc = orc_event(pr, seed, ev, &o);
  if (rc) return rc;
  const double head[12] = {o.x1, o.x2, o.shat, o.y, o.alphas, o.ht, o.ptlead, o.rmin, o.me2, o.weight, o.pdf, o.phi};
  memcpy(rec, head, sizeof head);
  rec[12] = o.pass;
  rec[13] = o.hel_bits;
  for (int i = 0; i < pr->n; ++i) rec[14 + i] = o.perm[i];
  for (int i = 0; i < pr->n; ++i)
    for (int mu = 0; mu < 4; ++mu) rec[14 + pr->n + 4 * i + mu] = o.k[i][mu];
  return 0;
}

/* The same record for caller-given uniforms u[0 .. orc_n_uniforms_mode(n, mode)). */
int orc_event_record_u(const orc_process *pr, const double *u, double *rec) {
  orc_event_out o;
  const int rc = event_from_uniforms(pr, u, &o);
  if (rc) return rc;
  const double head[12] = {o.x1, o.x2, o.shat, o.y, o.alphas, o.ht, o.ptlead, o.rmin, o.me2, o.weight, o.pdf, o.phi};
  memcpy(rec, head, sizeof head);
  rec[12] = o.pass;
  rec[13] = o.hel_bits;
  for (int i = 0; i < pr->n; ++i) rec[14 + i] = o.perm[i];
  for (int i = 0; i < pr->n; ++i)
    for (int mu = 0; mu < 4; ++mu) rec[14 + pr->n + 4 * i + mu] = o.k[i][mu];
  return 0;
}

/* Compensated sum of x[0..len), for the accumulation tests. */
double orc_compensated_sum(const double *x, uint64_t len) {
  ksum k = {0, 0};
  for (uint64_t i = 0; i < len; ++i) ksum_add(&k, x[i]);
  return ksum_val(&k);
}
