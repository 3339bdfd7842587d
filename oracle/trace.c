/*
 * CPU FP64 oracle: brute-force ray tracer with the paper's scattering models.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or runs
 * this file; only the test-suite, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code with the CUDA library.
 *
 * Every sample is traced against EVERY active primitive (no acceleration
 * structure), the K nearest hits are kept, each is shaded with the single-fibre
 * BCSDF (strands, Eq. 1) or the aggregated BCSDF (thick hairs, Eq. 5-13) and
 * the hits are composited front to back.  All arithmetic is double precision.
 *
 * Readings of the paper that this file implements are marked READING; they are
 * the same readings the CUDA library follows and are listed in the design notes.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846
#define MAXK 64

/* flag bits (same values as the library's render flags) */
#define FLAG_NO_S 1u          /* drop the shadowing-masking term S (ablation, Fig. "S-term") */
#define FLAG_SINGLE_ON_ETH 2u /* shade thick hairs with f_single (ablation, Fig. "S-term") */
#define FLAG_SHADOWS 4u       /* dual-scattering transmittance along shadow rays (Section 3.2, 6) */
/* Marschner R/TT/TRT single fibre (Section 7, "Extending to Marschner model
 * with TRT term"): the third lobe is TRT instead of D.  READING (the paper
 * prints no formula for it): A_TRT takes the D lobe's attenuation slots,
 * M_TRT = G(beta_TRT, theta_h) with beta_TRT = 2 beta_R (Marschner et al.
 * 2003's width relation) and no longitudinal shift (none of the paper's
 * lobes has one), and N_TRT = 1 / 2 pi (the paper's azimuthal simplification
 * of the R lobe, which leaves the fibre on the same side as TRT).            */
#define FLAG_TRT 8u
/* READING: the forward scattering density d_F of dual scattering (Section
 * 3.2 names it, without a value); Zinke et al. 2008 use 0.7.                */
#define D_F 0.7

typedef struct { double x, y, z; } v3;
static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double len(v3 a) { return sqrt(dot(a, a)); }
static v3 nrm(v3 a) { return scl(a, 1.0 / len(a)); }
static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* ------------------------------------------------------------------ BCSDF */

/* Single-fibre lobe parameters: A_p per RGB channel for p in {R, TT, D}, the
 * longitudinal widths beta_R, beta_TT and the TT azimuthal width gamma_TT.   */
typedef struct {
  double A[3][3]; /* [lobe R,TT,D][rgb]; [R,TT,TRT] with FLAG_TRT */
  double bR, bTT, gTT;
  int trt;        /* third lobe is TRT (FLAG_TRT) */
} material;

typedef struct {
  int n;
  const double* x; /* Gauss-Legendre nodes on [-1, 1] */
  const double* w;
} quad;

/* Gaussian with standard deviation beta (Section 3.2, definition of G).
 * Pinned by test_gaussian_definition.
 */
double oracle_gauss(double beta, double x) {
  return exp(-x * x / (2.0 * beta * beta)) / (sqrt(2.0 * PI) * beta);
}

/* IM(theta; beta) = integral over theta_o in [-pi/2, pi/2] of
 * G(beta, (theta + theta_o) / 2) cos^2(theta_o): the longitudinal factor of
 * the directional albedo of a lobe with M = G(beta, theta_h) under the
 * cos^2 measure of the rendering equation (Section 3).
 * Pinned by test_longitudinal_integral_closed_form,
 *   test_longitudinal_integral_quadrature_converged.
 */
static double im_quad(const quad* q, double theta, double beta) {
  double s = 0.0;
  for (int i = 0; i < q->n; ++i) {
    double to = 0.5 * PI * q->x[i];
    double c = cos(to);
    s += q->w[i] * oracle_gauss(beta, 0.5 * (theta + to)) * c * c;
  }
  return 0.5 * PI * s;
}

double oracle_im(int nq, const double* qx, const double* qw, double theta, double beta) {
  quad q = {nq, qx, qw};
  return im_quad(&q, theta, beta);
}

/* Single-fibre BCSDF, Eq. (1): sum over R, TT, D of A_p M_p(theta_h) N_p(phi)
 * with M_R = G(beta_R), N_R = 1/2pi; M_TT = G(beta_TT), N_TT = G(gamma_TT,
 * phi - pi); M_D = 1/pi, N_D = 1/2pi (the n = 1 case of Eq. 6).
 * phi is taken in [0, pi] from cos(phi) (the model is even in phi).
 * sg2 is the forward spread variance gathered along the light's path (zero
 * without shadow rays); READING: it adds to every lobe's variance.
 * With FLAG_TRT the third lobe is A_TRT G(2 beta_R, theta_h) / 2 pi.
 * Pinned by test_f_single_hand_values, test_spread_is_a_wider_lobe,
 *   test_trt_single_fibre_hand_values.
 */
static void f_single(const material* m, double th_i, double th_o, double cphi, double sg2,
                     double out[3]) {
  double th_h = 0.5 * (th_i + th_o);
  double phi = acos(clampd(cphi, -1.0, 1.0));
  double mR = oracle_gauss(sqrt(m->bR * m->bR + sg2), th_h) / (2.0 * PI);
  double mTT = oracle_gauss(sqrt(m->bTT * m->bTT + sg2), th_h) *
               oracle_gauss(sqrt(m->gTT * m->gTT + sg2), phi - PI);
  double mD = m->trt ? oracle_gauss(sqrt(4.0 * m->bR * m->bR + sg2), th_h) / (2.0 * PI)
                    : 1.0 / (PI * 2.0 * PI);
  for (int c = 0; c < 3; ++c) out[c] = m->A[0][c] * mR + m->A[1][c] * mTT + m->A[2][c] * mD;
}

/* Forward / backward hemispherical albedo of the single fibre, a_F and a_B
 * (Section 4, used by Eq. 7, 8, 10 and 13), and the forward spread variance
 * sigma_f^2 (Eq. 7).
 * READING: a_F(theta_d) is the albedo of f_single into the front half
 * (cos phi < 0) for light incident at |theta_d| / 2 (the mirror configuration),
 * under the cos^2 measure; a_B likewise into the back half (cos phi > 0).
 * The separable lobes make this A_p * IM_p * (azimuthal mass in the half).
 * sigma_f^2 is the mean of beta_R^2 and beta_TT^2 weighted by the RGB-mean
 * forward albedo of the R and TT lobes (and of (2 beta_R)^2, weighted by the
 * TRT lobe's, with FLAG_TRT).
 * Pinned by test_separable_albedo_equals_2d_quadrature,
 *   test_albedo_white_furnace_c1_material.
 */
static void albedo_split(const material* m, const quad* q, double theta_d, double aF[3],
                         double aB[3], double* sig2) {
  double ta = 0.5 * fabs(theta_d);
  double imR = im_quad(q, ta, m->bR);
  double imT = im_quad(q, ta, m->bTT);
  double imTRT = m->trt ? im_quad(q, ta, 2.0 * m->bR) : 0.0;
  double nF_TT = erf(PI / (2.0 * sqrt(2.0) * m->gTT));
  double nB_TT = erf(PI / (sqrt(2.0) * m->gTT)) - nF_TT;
  double wR = 0.0, wT = 0.0, w3 = 0.0;
  for (int c = 0; c < 3; ++c) {
    double r = m->A[0][c] * imR * 0.5;
    /* third lobe: D (azimuth and longitude uniform: a quarter per half) or
     * TRT (uniform azimuth: half of A_TRT IM(2 beta_R) per half) */
    double third = m->trt ? m->A[2][c] * imTRT * 0.5 : m->A[2][c] * 0.25;
    aF[c] = r + m->A[1][c] * imT * nF_TT + third;
    aB[c] = r + m->A[1][c] * imT * nB_TT + third;
    wR += r / 3.0;
    wT += m->A[1][c] * imT * nF_TT / 3.0;
    if (m->trt) w3 += third / 3.0;
  }
  *sig2 = (wR * m->bR * m->bR + wT * m->bTT * m->bTT + w3 * 4.0 * m->bR * m->bR) /
          (wR + wT + w3);
}

static void load_material(const double* row, material* m, unsigned flags);

void oracle_albedo(const double* mat12, int nq, const double* qx, const double* qw,
                   double theta_d, unsigned flags, double* aF3, double* aB3, double* sig2) {
  material m;
  load_material(mat12, &m, flags);
  quad q = {nq, qx, qw};
  albedo_split(&m, &q, theta_d, aF3, aB3, sig2);
}

/* Back-scattering attenuations of the B^ lobe for one channel.
 * Dual scattering (Zinke et al. 2008): A_1 = a_B a_F^2 / (1 - a_F^2) sums the
 * paths with one backward and an even number of forward events,
 * A_3 = a_B^3 a_F^2 / (1 - a_F^2)^3 those with three backward events.
 * Eq. (8): A_1+ = d_1+ a_B sum_{i=1..n} a_F^(2i-1) with d_1+ = 0.6, in the
 * closed form a_F (1 - a_F^(2n)) / (1 - a_F^2) of the geometric sum.
 * a_F is clamped to 1 - 1e-6 so the sums stay finite.
 * Pinned by test_back_lobe_attenuations_equal_their_series.
 */
static void back_atten(double aF, double aB, double n, double* A1, double* A3, double* A1p) {
  double f = aF < 1.0 - 1e-6 ? aF : 1.0 - 1e-6;
  double f2 = f * f, g = 1.0 - f2;
  *A1 = aB * f2 / g;
  *A3 = aB * aB * aB * f2 / (g * g * g);
  *A1p = 0.6 * aB * f * (1.0 - pow(f, 2.0 * n)) / g;
}

void oracle_back_atten(double aF, double aB, double n, double* out3) {
  back_atten(aF, aB, n, &out3[0], &out3[1], &out3[2]);
}

/* Aggregated BCSDF of a thick hair, Eq. (5):
 *   f = S(phi, theta_d) * sum over R^, TT^, D^, B^ of A_p M_p(theta_h) N_p(phi)
 * Eq. (6)/(7): A_p = a_F^(n-1) a_p with widened lobes
 *   beta_p^2 + (n-1) sigma_f^2  (READING: variances add),
 * n = 1 when the outgoing direction is in the back hemisphere (cos phi > 0).
 * Eq. (8): A_1+ = d_1+ a_B sum_{i=1..n} a_F^(2i-1), d_1+ = 0.6, summed in
 * closed form (READING: valid for real n, here n = max(1, n_view)).
 * A_1, A_3: local back-scattering of dual scattering (Zinke et al. 2008),
 *   A_1 = a_B a_F^2 / (1 - a_F^2),  A_3 = a_B^3 a_F^2 / (1 - a_F^2)^3.
 * Eq. (9): A_B^ = A_1+ + A_1 + A_3, M_B^ = G(beta_B^), N_B^ = I_B(phi) / pi;
 * READING: beta_B^2 is the RGB-mean-attenuation weighted mean of the path
 * variances beta_R^2 + 2 s^2 (A_1), 3 beta_R^2 + 2 s^2 (A_3) and
 * beta_R^2 + (n + 1) s^2 (A_1+).
 * Eq. (10)-(13): S = P_s a_F + P_n with P_s = (1 - rho)(1 - cos phi),
 * P_m = c_m (1 - rho), c_m = 0.2, P_n = 1 - P_m - P_s, applied for
 * phi in (-pi/2, pi/2) only (READING: P_n floored at 0).
 * With FLAG_TRT the third hat lobe is TRT^: a_F^(n-1) A_TRT
 * G(sqrt(4 beta_R^2 + (n-1) s^2), theta_h) / 2 pi.
 * Pinned by test_aggregated_reciprocity, test_aggregated_reduces_to_single_at_n1_front,
 *   test_back_lobe_uniform_over_back_half,
 *   test_shadowing_masking_bounds_and_ablation_order, tests/test_oracle_convergence.py.
 */
static void f_ours(const material* m, const quad* q, double th_i, double th_o, double cphi,
                   double rho, double n_view, unsigned flags, double sg2, double out[3]) {
  double th_h = 0.5 * (th_i + th_o);
  double th_d = th_i - th_o;
  double phi = acos(clampd(cphi, -1.0, 1.0));
  int back = cphi > 0.0;
  double aF[3], aB[3], s2;
  albedo_split(m, q, th_d, aF, aB, &s2);
  double n = back ? 1.0 : n_view;
  double bR = sqrt(m->bR * m->bR + (n - 1.0) * s2 + sg2);
  double bT = sqrt(m->bTT * m->bTT + (n - 1.0) * s2 + sg2);
  double gT = sqrt(m->gTT * m->gTT + (n - 1.0) * s2 + sg2);
  double mR = oracle_gauss(bR, th_h) / (2.0 * PI);
  double mTT = oracle_gauss(bT, th_h) * oracle_gauss(gT, phi - PI);
  double mD = m->trt ? oracle_gauss(sqrt(4.0 * m->bR * m->bR + (n - 1.0) * s2 + sg2), th_h) /
                          (2.0 * PI)
                    : 1.0 / (PI * 2.0 * PI);
  double lob[3];
  for (int c = 0; c < 3; ++c) {
    double att = pow(aF[c], n - 1.0);
    lob[c] = att * (m->A[0][c] * mR + m->A[1][c] * mTT + m->A[2][c] * mD);
  }
  if (back) {
    double A1[3], A3[3], A1p[3], w1 = 0, w3 = 0, w1p = 0;
    for (int c = 0; c < 3; ++c) {
      back_atten(aF[c], aB[c], n_view, &A1[c], &A3[c], &A1p[c]);
      w1 += A1[c];
      w3 += A3[c];
      w1p += A1p[c];
    }
    double bR2 = m->bR * m->bR;
    double vB = (w1 * (bR2 + 2.0 * s2) + w3 * (3.0 * bR2 + 2.0 * s2) +
                 w1p * (bR2 + (n_view + 1.0) * s2)) / (w1 + w3 + w1p);
    double mB = oracle_gauss(sqrt(vB + sg2), th_h) / PI;
    for (int c = 0; c < 3; ++c) lob[c] += (A1p[c] + A1[c] + A3[c]) * mB;
    if (!(flags & FLAG_NO_S)) {
      double Ps = (1.0 - rho) * (1.0 - cphi);
      double Pm = 0.2 * (1.0 - rho);
      double Pn = 1.0 - Pm - Ps;
      if (Pn < 0.0) Pn = 0.0;
      for (int c = 0; c < 3; ++c) lob[c] *= Ps * aF[c] + Pn;
    }
  }
  for (int c = 0; c < 3; ++c) out[c] = lob[c];
}

static void load_material(const double* row, material* m, unsigned flags) {
  for (int p = 0; p < 3; ++p)
    for (int c = 0; c < 3; ++c) m->A[p][c] = row[3 * p + c];
  m->bR = row[9];
  m->bTT = row[10];
  m->gTT = row[11];
  m->trt = (flags & FLAG_TRT) != 0;
}

void oracle_f_single(const double* mat12, double th_i, double th_o, double cphi, unsigned flags,
                     double* out3) {
  material m;
  load_material(mat12, &m, flags);
  f_single(&m, th_i, th_o, cphi, 0.0, out3);
}

void oracle_f_single_spread(const double* mat12, double th_i, double th_o, double cphi,
                            double sg2, double* out3) {
  material m;
  load_material(mat12, &m, 0u);
  f_single(&m, th_i, th_o, cphi, sg2, out3);
}

void oracle_f_ours(const double* mat12, int nq, const double* qx, const double* qw, double th_i,
                   double th_o, double cphi, double rho, double n_view, unsigned flags,
                   double* out3) {
  material m;
  load_material(mat12, &m, flags);
  quad q = {nq, qx, qw};
  f_ours(&m, &q, th_i, th_o, cphi, rho, n_view, flags, 0.0, out3);
}

/* Directional albedo of f_single by direct 2-D midpoint-free Gauss-Legendre
 * quadrature over theta_o in [-pi/2, pi/2] and phi in [0, pi] (doubled: the
 * model is even in phi), under the cos^2(theta_o) measure, split at
 * phi = pi/2 into back (phi < pi/2) and front parts.  Used only to check the
 * separable albedo above against the definition.
 * Pinned by test_albedo_2d_diffuse_closed_form.
 */
void oracle_albedo_2d(const double* mat12, int nq, const double* qx, const double* qw,
                      double theta_i, unsigned flags, double* front3, double* back3) {
  material m;
  load_material(mat12, &m, flags);
  for (int c = 0; c < 3; ++c) front3[c] = back3[c] = 0.0;
  for (int i = 0; i < nq; ++i) {
    double to = 0.5 * PI * qx[i], wt = 0.5 * PI * qw[i] * cos(to) * cos(to);
    for (int half = 0; half < 2; ++half) {
      for (int j = 0; j < nq; ++j) {
        /* phi in [0, pi/2] (back) or [pi/2, pi] (front) */
        double phi = 0.25 * PI * (qx[j] + 1.0) + (half ? 0.5 * PI : 0.0);
        double wp = 0.25 * PI * qw[j] * 2.0;
        double f[3];
        f_single(&m, theta_i, to, cos(phi), 0.0, f);
        for (int c = 0; c < 3; ++c) (half ? front3 : back3)[c] += wt * wp * f[c];
      }
    }
  }
}

/* ------------------------------------------------------------ geometry */

/* Primitive row (15 doubles): c0[3] c1[3] e1[3] a b kind mat n_tot r
 * An elliptic-cylinder segment from c0 to c1 whose cross-section has
 * semi-axis a along e1 (perpendicular to the axis) and b along e2 = t x e1.
 * kind 0: single strand segment; kind 1: thick-hair (ETH) segment.          */
#define PRIM_STRIDE 15

typedef struct {
  v3 c0, t, e1, e2;
  double L, a, b;
  int kind, mat;
  double ntot, r;
  int64_t id;
} prim;

/* Ray against an open elliptic cylinder of finite length (READING: no caps,
 * no joint fill).  Returns the nearest root whose axial coordinate lies in
 * [0, L] and whose distance exceeds tmin, and the chord length of the ray
 * inside the finite cylinder (used for the hair count n, Section 4).
 * Pinned by test_circular_cylinder_perpendicular_hit,
 *   test_elliptic_cylinder_axis_aligned_hit, test_intersection_misses_and_open_ends.
 */
static int intersect(const prim* p, v3 o, v3 d, double tmin, double* t_hit, double* chord) {
  v3 r = sub(o, p->c0);
  double u0 = dot(r, p->e1) / p->a, v0 = dot(r, p->e2) / p->b, w0 = dot(r, p->t);
  double du = dot(d, p->e1) / p->a, dv = dot(d, p->e2) / p->b, dw = dot(d, p->t);
  double A = du * du + dv * dv;
  double B = 2.0 * (u0 * du + v0 * dv);
  double C = u0 * u0 + v0 * v0 - 1.0;
  if (A <= 0.0) return 0;
  double disc = B * B - 4.0 * A * C;
  if (disc < 0.0) return 0;
  double sq = sqrt(disc);
  double tm = (-B - sq) / (2.0 * A), tp = (-B + sq) / (2.0 * A);
  double wlo, whi;
  if (dw != 0.0) {
    double ta = (0.0 - w0) / dw, tb = (p->L - w0) / dw;
    wlo = ta < tb ? ta : tb;
    whi = ta < tb ? tb : ta;
  } else {
    if (w0 < 0.0 || w0 > p->L) return 0;
    wlo = -INFINITY;
    whi = INFINITY;
  }
  double th;
  if (tm > tmin && tm >= wlo && tm <= whi)
    th = tm;
  else if (tp > tmin && tp >= wlo && tp <= whi)
    th = tp;
  else
    return 0;
  double lo = tm > wlo ? tm : wlo, hi = tp < whi ? tp : whi;
  *t_hit = th;
  *chord = hi > lo ? hi - lo : 0.0;
  return 1;
}

int oracle_intersect(const double* row, const double* o3, const double* d3, double* t_out,
                     double* chord_out) {
  prim p;
  v3 c0 = mk(row[0], row[1], row[2]), c1 = mk(row[3], row[4], row[5]);
  v3 ax = sub(c1, c0);
  p.L = len(ax);
  p.t = scl(ax, 1.0 / p.L);
  p.c0 = c0;
  p.e1 = mk(row[6], row[7], row[8]);
  p.e2 = cross(p.t, p.e1);
  p.a = row[9];
  p.b = row[10];
  return intersect(&p, mk(o3[0], o3[1], o3[2]), mk(d3[0], d3[1], d3[2]), 0.0, t_out, chord_out);
}

/* Ray interval inside the finite cylinder volume of one primitive: the part
 * of the infinite elliptic cylinder's interval [t-, t+] whose axial
 * coordinate lies in [0, L].  Returns 0 when the ray misses it.
 * Pinned by test_thick_hair_occluder_counts_its_hair_number_over_the_chord.
 */
static int span(const prim* p, v3 o, v3 d, double* lo, double* hi) {
  v3 r = sub(o, p->c0);
  double u0 = dot(r, p->e1) / p->a, v0 = dot(r, p->e2) / p->b, w0 = dot(r, p->t);
  double du = dot(d, p->e1) / p->a, dv = dot(d, p->e2) / p->b, dw = dot(d, p->t);
  double A = du * du + dv * dv;
  if (A <= 0.0) return 0;
  double B = 2.0 * (u0 * du + v0 * dv);
  double C = u0 * u0 + v0 * v0 - 1.0;
  double disc = B * B - 4.0 * A * C;
  if (disc < 0.0) return 0;
  double sq = sqrt(disc);
  double tm = (-B - sq) / (2.0 * A), tp = (-B + sq) / (2.0 * A);
  double wlo = -INFINITY, whi = INFINITY;
  if (dw != 0.0) {
    double ta = (0.0 - w0) / dw, tb = (p->L - w0) / dw;
    wlo = ta < tb ? ta : tb;
    whi = ta < tb ? tb : ta;
  } else if (w0 < 0.0 || w0 > p->L) {
    return 0;
  }
  *lo = tm > wlo ? tm : wlo;
  *hi = tp < whi ? tp : whi;
  return *hi > *lo;
}

/* Transmittance of the light path of dual scattering (Section 3.2: the light
 * reaching a hair is attenuated by the forward scattering of every hair it
 * passes; Section 6 finds those hairs by ray shooting).  READING:
 *  - the shadow ray leaves x along wi and ends at the light (t_light, +inf
 *    for a directional light); every primitive of the shading hair itself
 *    (the same material row: the same strand or thick hair) is skipped;
 *  - a primitive is crossed when the ray's interval inside its cylinder
 *    meets (0, t_light); a strand segment counts one hair, a thick-hair
 *    segment n = rho l sqrt(n_tot / (pi a b)) hairs (the hair-number estimate
 *    of Section 4, l its chord within (0, t_light));
 *  - each crossed hair attenuates by its forward albedo a_F at incidence
 *    |asin(wi . t)| (the mirror configuration of the a_F reading) and adds
 *    its forward spread variance sigma_f^2, n times;
 *  - T = d_F * prod a_F^n when at least one hair is crossed, else 1.
 * Pinned by tests/test_oracle_shadows.py.
 */
static void shadow_path(const prim* P, int64_t n_prims, const material* M, const quad* q, v3 x,
                        v3 wi, double t_light, int self_mat, double T[3], double* sg2) {
  int crossed = 0;
  T[0] = T[1] = T[2] = 1.0;
  *sg2 = 0.0;
  for (int64_t j = 0; j < n_prims; ++j) {
    const prim* p = &P[j];
    if (p->mat == self_mat) continue;
    double lo, hi;
    if (!span(p, x, wi, &lo, &hi)) continue;
    double a = lo > 0.0 ? lo : 0.0, b = hi < t_light ? hi : t_light;
    if (!(b > a)) continue;
    double n = 1.0;
    if (p->kind == 1) {
      double rho = p->ntot * p->r * p->r / (p->a * p->b);
      if (rho > 1.0) rho = 1.0;
      n = rho * (b - a) * sqrt(p->ntot / (PI * p->a * p->b));
    }
    double th = asin(clampd(dot(wi, p->t), -1.0, 1.0));
    double aF[3], aB[3], s2;
    albedo_split(&M[p->mat], q, 2.0 * th, aF, aB, &s2);
    for (int c = 0; c < 3; ++c) T[c] *= pow(aF[c], n);
    *sg2 += n * s2;
    crossed = 1;
  }
  if (crossed)
    for (int c = 0; c < 3; ++c) T[c] *= D_F;
}

/* ------------------------------------------------------------ camera */

/*
 * Pinned by test_splitmix64_published_outputs (same stream),
 *   test_camera_jitter_uses_published_stream.
 */
static uint64_t splitmix_out(uint64_t seed, uint64_t i) {
  /* output i (0-based) of SplitMix64 started at seed (Steele et al. 2014) */
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

typedef struct {
  int kind, W, H;
  double pix;
  v3 eye, right, up, fwd;
} camera;

/* Sample sid = pixel * spp + s, pixel = y * W + x.  Its position inside the
 * pixel is a pair of 24-bit uniforms drawn from SplitMix64 outputs 2 sid and
 * 2 sid + 1 of the frame seed (READING: stratification left to the spp count).
 * Pinned by test_camera_jitter_uses_published_stream, test_perspective_edge_ray_half_fov.
 */
static void camera_ray(const camera* c, uint64_t seed, int64_t sid, int spp, v3* o, v3* d) {
  int64_t pixel = sid / spp;
  int64_t x = pixel % c->W, y = pixel / c->W;
  double jx = (double)(splitmix_out(seed, 2 * (uint64_t)sid) >> 40) * (1.0 / 16777216.0);
  double jy = (double)(splitmix_out(seed, 2 * (uint64_t)sid + 1) >> 40) * (1.0 / 16777216.0);
  double sx = ((double)x + jx - 0.5 * c->W) / c->pix;
  double sy = (0.5 * c->H - ((double)y + jy)) / c->pix;
  if (c->kind == 1) {
    *o = c->eye;
    *d = nrm(add(add(c->fwd, scl(c->right, sx)), scl(c->up, sy)));
  } else {
    *o = add(add(c->eye, scl(c->right, sx)), scl(c->up, sy));
    *d = c->fwd;
  }
}

/* ------------------------------------------------------------ renderer */

static void load_prims(const double* prim_rows, int64_t n_prims, const int64_t* prim_ids,
                       prim* P) {
  for (int64_t j = 0; j < n_prims; ++j) {
    const double* r = prim_rows + PRIM_STRIDE * j;
    v3 c0 = mk(r[0], r[1], r[2]), c1 = mk(r[3], r[4], r[5]);
    v3 ax = sub(c1, c0);
    P[j].c0 = c0;
    P[j].L = len(ax);
    P[j].t = scl(ax, 1.0 / P[j].L);
    P[j].e1 = mk(r[6], r[7], r[8]);
    P[j].e2 = cross(P[j].t, P[j].e1);
    P[j].a = r[9];
    P[j].b = r[10];
    P[j].kind = (int)r[11];
    P[j].mat = (int)r[12];
    P[j].ntot = r[13];
    P[j].r = r[14];
    P[j].id = prim_ids ? prim_ids[j] : j;
  }
}

typedef struct {
  const prim* prims;
  int64_t n_prims;
  const material* mats;
  camera cam;
  const double* lights;
  int n_lights;
  const int64_t* samples;
  int64_t m;
  int spp, K;
  uint64_t seed;
  unsigned flags;
  quad q;
  double* rad;
  int64_t* hit;
  int64_t begin, end;
} job;

/* Radiance leaving hit point x toward -d: sum over lights of
 * T f(omega_i, omega_o) E cos(theta_i) (directional light E = rgb, point
 * light E = rgb / distance^2).  T = 1 and f unwidened without FLAG_SHADOWS
 * (READING: primary hits only); with it, T and the spread variance come
 * from the light path (shadow_path).  The angles are measured
 * against the segment axis t: sin(theta) = omega . t, cos(phi) from the
 * projections onto the normal plane (Section 3).
 * Pinned by test_light_sum_point_and_directional_lights,
 *   test_thick_hair_shading_uses_the_hair_number_of_its_chord.
 */
static void shade(const job* jb, const prim* p, v3 x, v3 d, double chord, double* rgb,
                  double* alpha) {
  const material* m = &jb->mats[p->mat];
  v3 wo = scl(d, -1.0);
  double so = clampd(dot(wo, p->t), -1.0, 1.0);
  double th_o = asin(so);
  v3 wop = sub(wo, scl(p->t, so));
  double nop = len(wop);
  double rho = 0.0, n_raw = 0.0, n_view = 1.0;
  if (p->kind == 1) {
    /* Section 4 "Estimation of hair number n": rho = n_tot r^2 / (|r_A||r_B|),
     * n = rho l sqrt(n_tot / (pi |r_A||r_B|)); READING: |r_A|, |r_B| are the
     * semi-axes a, b and l is the view ray's chord inside the thick hair.    */
    rho = p->ntot * p->r * p->r / (p->a * p->b);
    if (rho > 1.0) rho = 1.0;
    n_raw = rho * chord * sqrt(p->ntot / (PI * p->a * p->b));
    n_view = n_raw > 1.0 ? n_raw : 1.0;
  }
  double n_cross = 0.0;
  if (p->kind == 1) {
    /* READING (opacity; the paper renders thick hairs as opaque strips and
     * leaves order-independent transparency open, Section 5.2): the expected
     * number of member strands, centres uniform over the ellipse, whose centre
     * lies within r of the view chord, 2 r l n_tot / (pi a b).               */
    n_cross = 2.0 * p->r * chord * p->ntot / (PI * p->a * p->b);
  }
  rgb[0] = rgb[1] = rgb[2] = 0.0;
  for (int l = 0; l < jb->n_lights; ++l) {
    const double* L = jb->lights + 8 * l;
    v3 wi;
    double E = 1.0;
    if (L[3] == 0.0) {
      wi = nrm(mk(L[0], L[1], L[2]));
    } else {
      v3 to = sub(mk(L[0], L[1], L[2]), x);
      double dd = dot(to, to);
      wi = scl(to, 1.0 / sqrt(dd));
      E = 1.0 / dd;
    }
    double si = clampd(dot(wi, p->t), -1.0, 1.0);
    double th_i = asin(si);
    v3 wip = sub(wi, scl(p->t, si));
    double nip = len(wip);
    double cphi = (nip > 0.0 && nop > 0.0) ? clampd(dot(wip, wop) / (nip * nop), -1.0, 1.0) : 1.0;
    double T[3] = {1.0, 1.0, 1.0}, sg2 = 0.0;
    if (jb->flags & FLAG_SHADOWS)
      shadow_path(jb->prims, jb->n_prims, jb->mats, &jb->q, x, wi,
                  L[3] == 0.0 ? INFINITY : 1.0 / sqrt(E), p->mat, T, &sg2);
    double f[3];
    if (p->kind == 1 && !(jb->flags & FLAG_SINGLE_ON_ETH))
      f_ours(m, &jb->q, th_i, th_o, cphi, rho, n_view, jb->flags, sg2, f);
    else
      f_single(m, th_i, th_o, cphi, sg2, f);
    double g = E * sqrt(1.0 - si * si);
    for (int c = 0; c < 3; ++c) rgb[c] += f[c] * T[c] * g * L[4 + c];
  }
  /* READING: a thick hair's opacity is the Poisson probability 1 - exp(-n_c)
   * that the view chord meets at least one member strand; a strand is opaque. */
  *alpha = p->kind == 1 ? 1.0 - exp(-n_cross) : 1.0;
}

/*
 * Pinned by test_kbuffer_keeps_the_nearest_in_order_and_breaks_ties_by_id,
 *   test_composite_front_to_back_with_closed_form_opacity.
 */
static void* worker(void* arg) {
  job* jb = (job*)arg;
  double kt[MAXK], kc[MAXK];
  int64_t kp[MAXK];
  for (int64_t i = jb->begin; i < jb->end; ++i) {
    v3 o, d;
    camera_ray(&jb->cam, jb->seed, jb->samples[i], jb->spp, &o, &d);
    int cnt = 0;
    for (int64_t j = 0; j < jb->n_prims; ++j) {
      double t, ch;
      if (!intersect(&jb->prims[j], o, d, 0.0, &t, &ch)) continue;
      /* keep the K nearest hits ordered by (t, primitive id) */
      int64_t id = jb->prims[j].id;
      int pos = cnt;
      while (pos > 0 && (kt[pos - 1] > t || (kt[pos - 1] == t && jb->prims[kp[pos - 1]].id > id)))
        --pos;
      if (pos >= jb->K) continue;
      int last = cnt < jb->K ? cnt : jb->K - 1;
      for (int s = last; s > pos; --s) {
        kt[s] = kt[s - 1];
        kc[s] = kc[s - 1];
        kp[s] = kp[s - 1];
      }
      kt[pos] = t;
      kc[pos] = ch;
      kp[pos] = j;
      if (cnt < jb->K) ++cnt;
    }
    /* front-to-back compositing over the k-buffer (Section 5.2: thick hairs
     * may overlap; the paper leaves order-independent transparency open)   */
    double T = 1.0, C[3] = {0, 0, 0};
    for (int h = 0; h < cnt && T > 0.0; ++h) {
      const prim* p = &jb->prims[kp[h]];
      double rgb[3], a;
      shade(jb, p, add(o, scl(d, kt[h])), d, kc[h], rgb, &a);
      for (int c = 0; c < 3; ++c) C[c] += T * a * rgb[c];
      T *= 1.0 - a;
    }
    for (int c = 0; c < 3; ++c) jb->rad[3 * i + c] = C[c];
    /* the composited hits: nearest first, none after the first opaque one */
    int past = 0;
    for (int h = 0; h < jb->K; ++h) {
      const int live = h < cnt && !past;
      jb->hit[(int64_t)jb->K * i + h] = live ? jb->prims[kp[h]].id : -1;
      if (live && jb->prims[kp[h]].kind == 0) past = 1;
    }
  }
  return 0;
}

int oracle_render(const double* prim_rows, const int64_t* prim_ids, int64_t n_prims,
                  const double* mat_rows, int64_t n_mats, const double* cam_rec,
                  const double* lights, int n_lights, const int64_t* samples, int64_t m, int spp,
                  int K, uint64_t seed, unsigned flags, int nq, const double* qx,
                  const double* qw, double* rad_out, int64_t* hit_out, int n_threads) {
  if (K < 1 || K > MAXK || spp < 1) return 1;
  prim* P = (prim*)malloc(sizeof(prim) * (size_t)(n_prims > 0 ? n_prims : 1));
  material* M = (material*)malloc(sizeof(material) * (size_t)(n_mats > 0 ? n_mats : 1));
  if (!P || !M) return 2;
  load_prims(prim_rows, n_prims, prim_ids, P);
  for (int64_t j = 0; j < n_mats; ++j) load_material(mat_rows + 12 * j, &M[j], flags);
  camera cam;
  cam.kind = (int)cam_rec[0];
  cam.W = (int)cam_rec[1];
  cam.H = (int)cam_rec[2];
  cam.pix = cam_rec[3];
  cam.eye = mk(cam_rec[4], cam_rec[5], cam_rec[6]);
  cam.right = mk(cam_rec[7], cam_rec[8], cam_rec[9]);
  cam.up = mk(cam_rec[10], cam_rec[11], cam_rec[12]);
  cam.fwd = mk(cam_rec[13], cam_rec[14], cam_rec[15]);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  job jobs[256];
  int64_t chunk = (m + n_threads - 1) / n_threads;
  int started = 0;
  for (int t = 0; t < n_threads; ++t) {
    job* jb = &jobs[t];
    jb->prims = P;
    jb->n_prims = n_prims;
    jb->mats = M;
    jb->cam = cam;
    jb->lights = lights;
    jb->n_lights = n_lights;
    jb->samples = samples;
    jb->m = m;
    jb->spp = spp;
    jb->K = K;
    jb->seed = seed;
    jb->flags = flags;
    jb->q.n = nq;
    jb->q.x = qx;
    jb->q.w = qw;
    jb->rad = rad_out;
    jb->hit = hit_out;
    jb->begin = t * chunk;
    jb->end = (t + 1) * chunk < m ? (t + 1) * chunk : m;
    if (jb->begin >= jb->end) break;
    pthread_create(&th[t], 0, worker, jb);
    ++started;
  }
  for (int t = 0; t < started; ++t) pthread_join(th[t], 0);
  free(P);
  free(M);
  return 0;
}

/* Camera ray of one sample, exported for the ray-generation checks. */
void oracle_camera_ray(const double* cam_rec, uint64_t seed, int64_t sid, int spp, double* o3,
                       double* d3) {
  camera cam;
  cam.kind = (int)cam_rec[0];
  cam.W = (int)cam_rec[1];
  cam.H = (int)cam_rec[2];
  cam.pix = cam_rec[3];
  cam.eye = mk(cam_rec[4], cam_rec[5], cam_rec[6]);
  cam.right = mk(cam_rec[7], cam_rec[8], cam_rec[9]);
  cam.up = mk(cam_rec[10], cam_rec[11], cam_rec[12]);
  cam.fwd = mk(cam_rec[13], cam_rec[14], cam_rec[15]);
  v3 o, d;
  camera_ray(&cam, seed, sid, spp, &o, &d);
  o3[0] = o.x; o3[1] = o.y; o3[2] = o.z;
  d3[0] = d.x; d3[1] = d.y; d3[2] = d.z;
}

/* The light-path transmittance of one point, exported for the pins. */
void oracle_shadow_path(const double* prim_rows, int64_t n_prims, const double* mat_rows,
                        int64_t n_mats, int nq, const double* qx, const double* qw,
                        const double* x3, const double* wi3, double t_light, int self_mat,
                        unsigned flags, double* T3, double* sg2) {
  prim* P = (prim*)malloc(sizeof(prim) * (size_t)(n_prims > 0 ? n_prims : 1));
  material* M = (material*)malloc(sizeof(material) * (size_t)(n_mats > 0 ? n_mats : 1));
  if (!P || !M) {
    free(P);
    free(M);
    T3[0] = T3[1] = T3[2] = -1.0;
    return;
  }
  load_prims(prim_rows, n_prims, 0, P);
  for (int64_t j = 0; j < n_mats; ++j) load_material(mat_rows + 12 * j, &M[j], flags);
  quad q = {nq, qx, qw};
  shadow_path(P, n_prims, M, &q, mk(x3[0], x3[1], x3[2]), mk(wi3[0], wi3[1], wi3[2]), t_light,
              self_mat, T3, sg2);
  free(P);
  free(M);
}
