/*
 * FP64 CPU oracle for the ray-error Sim(3) Gauss-Newton path of MASt3R-SLAM
 * (arXiv 2412.12392).  TEST INFRASTRUCTURE ONLY: tests, the smoke check and
 * the benchmark's CPU-baseline leg call it; the product path never does.
 *
 * Every routine restates one passage of the paper in plain double-precision
 * C, in the paper's order of steps.  Readings where the paper is silent (the
 * bilinear cell, the LM schedule, the refinement window, the weight form) are
 * the ones listed in the design notes and are repeated at each routine.
 * OpenMP parallelises only over independent pixels or edges.
 *
 * ORC_MUTANT_<NAME> (off in every normal build): a copy compiled with one of
 * these defines carries one planted mistake (a flipped sign, a transposed
 * operand, a dropped term, a wrong branch of a weight, a wrong rounding or
 * gauge), so that the tests can show that a pin of this oracle catches it.
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* small vector / matrix helpers                                             */
/* ------------------------------------------------------------------------ */

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static int finite3(const double a[3]) { return isfinite(a[0]) && isfinite(a[1]) && isfinite(a[2]); }

static void skew(const double v[3], double S[9]) {
  S[0] = 0;     S[1] = -v[2]; S[2] = v[1];
  S[3] = v[2];  S[4] = 0;     S[5] = -v[0];
  S[6] = -v[1]; S[7] = v[0];  S[8] = 0;
}

static void matmul(const double* A, const double* B, double* C, int n, int k, int m) {
  /* C (n x m) = A (n x k) B (k x m), row-major */
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      double s = 0;
      for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * m + j];
      C[i * m + j] = s;
    }
}

static void quat_to_rot(const double q[4], double R[9]) {
  double x = q[0], y = q[1], z = q[2], w = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
  R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
  R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
}

static void quat_mul(const double a[4], const double b[4], double c[4]) {
  /* Hamilton product, (x, y, z, w) layout */
  double ax = a[0], ay = a[1], az = a[2], aw = a[3];
  double bx = b[0], by = b[1], bz = b[2], bw = b[3];
  c[0] = aw * bx + ax * bw + ay * bz - az * by;
  c[1] = aw * by - ax * bz + ay * bw + az * bx;
  c[2] = aw * bz + ax * by - ay * bx + az * bw;
  c[3] = aw * bw - ax * bx - ay * by - az * bz;
}

static void quat_normalise(double q[4]) {
  double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) q[k] /= n;
}

/* ------------------------------------------------------------------------ */
/* Sim(3), Eq. 1: T = [[sR, t], [0, 1]], left-plus T <- Exp(tau) o T         */
/* ------------------------------------------------------------------------ */

/* I_n(s) = integral_0^1 x^n e^{s x} dx */
static double int_xn_exp(int n, double s) {
  if (fabs(s) < 1.0) {
    double term = 1.0, sum = 0.0; /* sum_k s^k / (k! (n + k + 1)) */
    for (int k = 0; k < 40; ++k) {
      sum += term / (double)(n + k + 1);
      term *= s / (double)(k + 1);
    }
    return sum;
  }
  double mom = expm1(s) / s, es = exp(s);
  for (int k = 1; k <= n; ++k) mom = (es - k * mom) / s;
  return mom;
}

/* V = integral_0^1 exp(x ([phi]x + sigma I)) dx = A0 I + B [phi]x + C [phi]x^2,
 * the matrix that maps rho to the translation of Exp(tau). */
static void sim3_V(const double phi[3], double sigma, double V[9]) {
  double th = norm3(phi), A0 = int_xn_exp(0, sigma), B, C;
  if (th < 1e-4) {
    double t2 = th * th;
    B = int_xn_exp(1, sigma) - t2 * int_xn_exp(3, sigma) / 6.0 + t2 * t2 * int_xn_exp(5, sigma) / 120.0;
    C = int_xn_exp(2, sigma) / 2.0 - t2 * int_xn_exp(4, sigma) / 24.0 + t2 * t2 * int_xn_exp(6, sigma) / 720.0;
  } else {
    double es = exp(sigma), c = cos(th), sn = sin(th), den = sigma * sigma + th * th;
    double Ic = ((es * c - 1.0) * sigma + es * th * sn) / den; /* integral e^{sx} cos(th x) */
    double Is = (es * sn * sigma - (es * c - 1.0) * th) / den;  /* integral e^{sx} sin(th x) */
    B = Is / th;
    C = (A0 - Ic) / (th * th);
  }
  double S[9], S2[9];
  skew(phi, S);
  matmul(S, S, S2, 3, 3, 3);
  for (int k = 0; k < 9; ++k) V[k] = B * S[k] + C * S2[k];
  V[0] += A0; V[4] += A0; V[8] += A0;
}

void orc_sim3_exp(const double tau[7], double T[8]) {
  const double* rho = tau;
  const double* phi = tau + 3;
  double sigma = tau[6];
  double th = norm3(phi);
  double k = (th < 1e-6) ? 0.5 - th * th / 48.0 : sin(0.5 * th) / th;
  double q[4] = {k * phi[0], k * phi[1], k * phi[2], cos(0.5 * th)};
  quat_normalise(q);
  double V[9];
  sim3_V(phi, sigma, V);
#ifdef ORC_MUTANT_EXP_NO_V
  for (int r = 0; r < 3; ++r) T[r] = rho[r];
#else
  for (int r = 0; r < 3; ++r) T[r] = V[3 * r] * rho[0] + V[3 * r + 1] * rho[1] + V[3 * r + 2] * rho[2];
#endif
  for (int r = 0; r < 4; ++r) T[3 + r] = q[r];
  T[7] = exp(sigma);
}

static int solve3(const double A_in[9], const double b_in[3], double x[3]) {
  /* Gaussian elimination with partial pivoting */
  double A[9], b[3];
  memcpy(A, A_in, sizeof A);
  memcpy(b, b_in, sizeof b);
  for (int c = 0; c < 3; ++c) {
    int p = c;
    for (int r = c + 1; r < 3; ++r)
      if (fabs(A[3 * r + c]) > fabs(A[3 * p + c])) p = r;
    if (A[3 * p + c] == 0.0) return 0;
    if (p != c) {
      for (int k = 0; k < 3; ++k) { double t = A[3 * c + k]; A[3 * c + k] = A[3 * p + k]; A[3 * p + k] = t; }
      double t = b[c]; b[c] = b[p]; b[p] = t;
    }
    for (int r = c + 1; r < 3; ++r) {
      double f = A[3 * r + c] / A[3 * c + c];
      for (int k = c; k < 3; ++k) A[3 * r + k] -= f * A[3 * c + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = 2; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < 3; ++k) s -= A[3 * r + k] * x[k];
    x[r] = s / A[3 * r + r];
  }
  return 1;
}

void orc_sim3_log(const double T[8], double tau[7]) {
  double q[4] = {T[3], T[4], T[5], T[6]};
  quat_normalise(q);
  if (q[3] < 0) for (int k = 0; k < 4; ++k) q[k] = -q[k];
  double vn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
  double th = 2.0 * atan2(vn, q[3]);
  double f = (vn < 1e-12) ? 2.0 / q[3] : th / vn;
  double phi[3] = {f * q[0], f * q[1], f * q[2]};
  double sigma = log(T[7]);
  double V[9], rho[3];
  sim3_V(phi, sigma, V);
  solve3(V, T, rho);
  tau[0] = rho[0]; tau[1] = rho[1]; tau[2] = rho[2];
  tau[3] = phi[0]; tau[4] = phi[1]; tau[5] = phi[2];
  tau[6] = sigma;
}

void orc_sim3_mul(const double A[8], const double B[8], double C[8]) {
  double Ra[9], q[4], t[3];
  quat_to_rot(A + 3, Ra);
  for (int r = 0; r < 3; ++r)
    t[r] = A[7] * (Ra[3 * r] * B[0] + Ra[3 * r + 1] * B[1] + Ra[3 * r + 2] * B[2]) + A[r];
  quat_mul(A + 3, B + 3, q);
  quat_normalise(q);
  C[0] = t[0]; C[1] = t[1]; C[2] = t[2];
  C[3] = q[0]; C[4] = q[1]; C[5] = q[2]; C[6] = q[3];
  C[7] = A[7] * B[7];
}

void orc_sim3_inv(const double A[8], double Ai[8]) {
  double R[9], qi[4] = {-A[3], -A[4], -A[5], A[6]};
  quat_to_rot(A + 3, R);
  double si = 1.0 / A[7];
  for (int r = 0; r < 3; ++r) /* -(1/s) R^T t */
    Ai[r] = -si * (R[r] * A[0] + R[3 + r] * A[1] + R[6 + r] * A[2]);
  Ai[3] = qi[0]; Ai[4] = qi[1]; Ai[5] = qi[2]; Ai[6] = qi[3];
  Ai[7] = si;
}

void orc_sim3_act(const double T[8], const double x[3], double y[3]) {
  double R[9];
  quat_to_rot(T + 3, R);
  for (int r = 0; r < 3; ++r) y[r] = T[7] * (R[3 * r] * x[0] + R[3 * r + 1] * x[1] + R[3 * r + 2] * x[2]) + T[r];
}

void orc_sim3_matrix(const double T[8], double M[16]) {
  double R[9];
  quat_to_rot(T + 3, R);
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) M[4 * r + c] = T[7] * R[3 * r + c];
    M[4 * r + 3] = T[r];
  }
  M[12] = M[13] = M[14] = 0.0;
  M[15] = 1.0;
}

/* Ad_T with T Exp(tau) T^-1 = Exp(Ad_T tau):
 * [[sR, [t]x R, -t], [0, R, 0], [0, 0, 1]] (derived from hat(tau) and Eq. 1). */
void orc_sim3_adjoint(const double T[8], double Ad[49]) {
  double R[9], S[9], SR[9];
  quat_to_rot(T + 3, R);
  skew(T, S);
  matmul(S, R, SR, 3, 3, 3);
  memset(Ad, 0, 49 * sizeof(double));
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      Ad[7 * r + c] = T[7] * R[3 * r + c];
      Ad[7 * r + 3 + c] = SR[3 * r + c];
      Ad[7 * (3 + r) + 3 + c] = R[3 * r + c];
    }
  for (int r = 0; r < 3; ++r) Ad[7 * r + 6] = -T[r];
  Ad[48] = 1.0;
}

void orc_sim3_retract(const double tau[7], double T[8]) {
  double E[8], out[8];
  orc_sim3_exp(tau, E);
  orc_sim3_mul(E, T, out);
  memcpy(T, out, sizeof out);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: psi(X) = X / |X|, one ray per pixel ("each pointmap defines its   */
/* own camera model").  A non-finite or zero point gives the zero vector.     */
/* ------------------------------------------------------------------------ */
void orc_ray_image(const double* X, int64_t n, double* R) {
  for (int64_t p = 0; p < n; ++p) {
    const double* x = X + 3 * p;
    double nx = norm3(x);
    if (finite3(x) && nx > 0.0) {
      R[3 * p] = x[0] / nx; R[3 * p + 1] = x[1] / nx; R[3 * p + 2] = x[2] / nx;
    } else {
      R[3 * p] = R[3 * p + 1] = R[3 * p + 2] = 0.0;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2, Eq. 2: p* = argmin_p |psi([X_ref]_p) - psi(x)|^2 by LM, then the */
/* coarse-to-fine descriptor refinement, the 3D outlier test and q.           */
/* Readings: bilinear interpolation of the stored rays in the cell            */
/* (clamp(floor u, 0, W-2), clamp(floor v, 0, H-2)), analytic cell derivative; */
/* (J^T J + lambda I) delta = -J^T r with every step accepted and p clamped to */
/* the image; a fixed number of iterations; rounding half-up; refinement      */
/* windows of radius r with the given dilations, strict '>' in row-major      */
/* (dy, dx) order; q = sqrt(Q_ref[m] Q_qry[n]) (Sec. 3.3).                    */
/* ------------------------------------------------------------------------ */
static void bilinear_ray(const double* R, int H, int W, double u, double v, double Rp[3], double Ju[3],
                         double Jv[3]) {
  int u0 = (int)floor(u), v0 = (int)floor(v);
  if (u0 < 0) u0 = 0;
  if (u0 > W - 2) u0 = W - 2;
  if (v0 < 0) v0 = 0;
  if (v0 > H - 2) v0 = H - 2;
  double a = u - u0, b = v - v0;
  const double* R00 = R + 3 * ((int64_t)v0 * W + u0);
  const double* R10 = R + 3 * ((int64_t)v0 * W + u0 + 1);
  const double* R01 = R + 3 * ((int64_t)(v0 + 1) * W + u0);
  const double* R11 = R + 3 * ((int64_t)(v0 + 1) * W + u0 + 1);
  for (int c = 0; c < 3; ++c) {
    Rp[c] = (1 - a) * (1 - b) * R00[c] + a * (1 - b) * R10[c] + (1 - a) * b * R01[c] + a * b * R11[c];
    Ju[c] = (1 - b) * (R10[c] - R00[c]) + b * (R11[c] - R01[c]);
    Jv[c] = (1 - a) * (R01[c] - R00[c]) + a * (R11[c] - R10[c]);
  }
}

static double desc_dot(const double* a, const double* b, int d) {
  double s = 0.0;
  for (int k = 0; k < d; ++k) s += a[k] * b[k];
  return s;
}

void orc_match(const orc_params* P, int H, int W, int d, const double* X_ref, const double* X_qry,
               const double* D_ref, const double* D_qry, const double* Q_ref, const double* Q_qry,
               const int32_t* init_idx, const int64_t* pix, int64_t n_pix, int32_t* idx_out, double* q_out,
               double* diag) {
  int64_t HW = (int64_t)H * W;
  double* R = (double*)malloc(sizeof(double) * 3 * HW);
  orc_ray_image(X_ref, HW, R); /* the reference camera model psi(X^i_i) */
  int64_t count = pix ? n_pix : HW;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t s = 0; s < count; ++s) {
    int64_t n = pix ? pix[s] : s;
    double* dg = diag ? diag + 9 * s : NULL;
    if (dg) for (int k = 0; k < 9; ++k) dg[k] = 0.0;
    const double* x = X_qry + 3 * n;
    double nx = norm3(x);
    if (!(finite3(x) && nx > 0.0)) {
      idx_out[s] = -1;
      q_out[s] = 0.0;
      continue;
    }
    double tgt[3] = {x[0] / nx, x[1] / nx, x[2] / nx};
    /* initial projection: the previous match, else the identity map */
    int64_t p0 = (init_idx && init_idx[n] >= 0) ? init_idx[n] : n;
    double u = (double)(p0 % W), v = (double)(p0 / W), last = 0.0;
    for (int it = 0; it < P->lm_iters; ++it) {
      double Rp[3], Ju[3], Jv[3], r[3];
      bilinear_ray(R, H, W, u, v, Rp, Ju, Jv);
      for (int c = 0; c < 3; ++c) r[c] = Rp[c] - tgt[c];
      double a00 = dot3(Ju, Ju) + P->lm_lambda, a01 = dot3(Ju, Jv), a11 = dot3(Jv, Jv) + P->lm_lambda;
      double b0 = -dot3(Ju, r), b1 = -dot3(Jv, r);
      double det = a00 * a11 - a01 * a01;
      double du = (a11 * b0 - a01 * b1) / det;
      double dv = (a00 * b1 - a01 * b0) / det;
      last = sqrt(du * du + dv * dv);
#ifdef ORC_MUTANT_LM_SIGN
      u -= du;
      v -= dv;
#else
      u += du;
      v += dv;
#endif
      if (u < 0) u = 0;
      if (u > W - 1) u = W - 1;
      if (v < 0) v = 0;
      if (v > H - 1) v = H - 1;
    }
#ifdef ORC_MUTANT_ROUND_FLOOR
    int cu = (int)floor(u), cv = (int)floor(v);
#else
    int cu = (int)floor(u + 0.5), cv = (int)floor(v + 0.5);
#endif
    if (dg) {
      double fu = fabs(u - floor(u) - 0.5), fv = fabs(v - floor(v) - 0.5);
      dg[0] = u; dg[1] = v; dg[2] = last; dg[5] = fu < fv ? fu : fv;
    }
    /* coarse-to-fine refinement: maximum descriptor similarity in a window */
    const double* dq = D_qry + (int64_t)d * n;
    double best = -INFINITY;
    for (int lev = 0; lev < P->n_levels; ++lev) {
      int dil = P->win_dilation[lev], r = P->win_radius;
      double second = -INFINITY;
      int bu = cu, bv = cv;
      best = -INFINITY;
      for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
          int uu = cu + dx * dil, vv = cv + dy * dil;
          if (uu < 0 || uu >= W || vv < 0 || vv >= H) continue;
          double sc = desc_dot(dq, D_ref + (int64_t)d * ((int64_t)vv * W + uu), d);
          if (sc > best) {
            second = best;
            best = sc;
            bu = uu;
            bv = vv;
          } else if (sc > second) {
            second = sc;
          }
        }
      cu = bu;
      cv = bv;
      if (dg && lev < 2) dg[3 + lev] = best - second;
    }
    int64_t m = (int64_t)cv * W + cu;
    /* occlusion / outlier test: large 3D distance invalidates the match */
    const double* y = X_ref + 3 * m;
    double diff[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
    double ratio = norm3(diff) / nx;
    int ok = finite3(y) && (ratio <= P->max_rel_dist3d);
    if (dg) { dg[6] = ratio; dg[7] = 1.0; dg[8] = best; }
    idx_out[s] = ok ? (int32_t)m : -1;
    q_out[s] = ok ? sqrt(Q_ref[m] * Q_qry[n]) : 0.0;
  }
  free(R);
}

/* ------------------------------------------------------------------------ */
/* Supp. S1.2 (ray and distance Jacobians w.r.t. T_ij) and S1.4 (relative to  */
/* global pose via the adjoint).  The relative Jacobian is formed literally as */
/* (dr/dx) [I, -[x]x, x] so that its structure (zero scale column of the ray  */
/* rows, -[x]x/d rotation block) comes out of the arithmetic.                 */
/* Residual order (r = psi(T_ij X_j,n) - psi(X_i,m)) follows Supp. S1.2.       */
/* ------------------------------------------------------------------------ */
static int residual_jacobian_rel(const double Tij[8], const double Ad[49], const double Xj_n[3],
                                 const double Xi_m[3], double r[4], double J[56]) {
  double x[3];
  orc_sim3_act(Tij, Xj_n, x);
  double d = norm3(x), dy = norm3(Xi_m);
  if (!(finite3(x) && finite3(Xi_m) && d > 0.0 && dy > 0.0)) return 0;
  for (int c = 0; c < 3; ++c) r[c] = x[c] / d - Xi_m[c] / dy;
  r[3] = d - dy;
  /* dx/dtau = [I, -[x]x, x] (Eq. point_jac) */
  double Dx[21], S[9];
  skew(x, S);
  for (int rr = 0; rr < 3; ++rr) {
    for (int c = 0; c < 3; ++c) {
      Dx[7 * rr + c] = (rr == c) ? 1.0 : 0.0;
#ifdef ORC_MUTANT_JAC_ROT_SIGN
      Dx[7 * rr + 3 + c] = S[3 * rr + c];
#else
      Dx[7 * rr + 3 + c] = -S[3 * rr + c];
#endif
    }
    Dx[7 * rr + 6] = x[rr];
  }
  /* dr_psi/dx = (I - x x^T / d^2) / d (Eq. norm_jac);  dr_d/dx = x^T / d */
  double Dr[12];
  for (int rr = 0; rr < 3; ++rr)
    for (int c = 0; c < 3; ++c) Dr[3 * rr + c] = ((rr == c ? 1.0 : 0.0) - x[rr] * x[c] / (d * d)) / d;
  for (int c = 0; c < 3; ++c) Dr[9 + c] = x[c] / d;
  double Jrel[28];
  matmul(Dr, Dx, Jrel, 4, 3, 7);
  /* dT_ij/dT_i = -Ad_{T_i^-1}, dT_ij/dT_j = Ad_{T_i^-1} */
  double JA[28];
#ifdef ORC_MUTANT_ADJ_T
  double AdT[49];
  for (int a = 0; a < 7; ++a)
    for (int b = 0; b < 7; ++b) AdT[7 * a + b] = Ad[7 * b + a];
  matmul(Jrel, AdT, JA, 4, 7, 7);
#else
  matmul(Jrel, Ad, JA, 4, 7, 7);
#endif
  for (int rr = 0; rr < 4; ++rr)
    for (int c = 0; c < 7; ++c) {
      J[14 * rr + c] = -JA[7 * rr + c];
      J[14 * rr + 7 + c] = JA[7 * rr + c];
    }
  return 1;
}

int orc_residual_jacobian(const double Ti[8], const double Tj[8], const double Xj_n[3], const double Xi_m[3],
                          double r[4], double J[56]) {
  double Tii[8], Tij[8], Ad[49];
  orc_sim3_inv(Ti, Tii);
  orc_sim3_mul(Tii, Tj, Tij);
  orc_sim3_adjoint(Tii, Ad);
  return residual_jacobian_rel(Tij, Ad, Xj_n, Xi_m, r, J);
}

/* The other residual families, formed the same literal way: r and dr/dx of
 * the family, times dx/dtau = [I, -[x]x, x] (Eq. point_jac), times the
 * global map.  Point family (Supp. S1.1, Eq. track_point in backend
 * notation): r = T_ij X_j,n - X_i,m, dr/dx = I.  Pixel family with known
 * pinhole calibration (Sec. 3.6, Supp. S1.3): r = Pi(x) - p_m with
 * Pi(x) = (fx x/z + cx, fy y/z + cy) and p_m the reference pixel m, plus the
 * depth residual x_z - (X_i,m)_z that replaces the distance term.  A pixel
 * residual needs the point in front of the camera: z > 1e-3 |x|.  Returns
 * the number of rows, or 0 for a degenerate match. */
static int residual_jacobian_family(const orc_params* P, const double Tij[8], const double Ad[49],
                                    const double Xj_n[3], const double Xi_m[3], int32_t m, double r[4],
                                    double J[56]) {
  if (P->residual == ORC_RES_RAY) return residual_jacobian_rel(Tij, Ad, Xj_n, Xi_m, r, J) ? 4 : 0;
  double x[3];
  orc_sim3_act(Tij, Xj_n, x);
  if (!(finite3(x) && finite3(Xi_m) && norm3(x) > 0.0 && norm3(Xi_m) > 0.0)) return 0;
  double Dr[9];
  if (P->residual == ORC_RES_POINT) {
    for (int c = 0; c < 3; ++c) r[c] = x[c] - Xi_m[c];
    for (int k = 0; k < 9; ++k) Dr[k] = (k % 4 == 0) ? 1.0 : 0.0;
  } else if (P->residual == ORC_RES_PIXEL) {
    const double z = x[2];
    if (!(z > 1e-3 * norm3(x)) || P->img_w <= 0) return 0;
    const double u_m = (double)(m % P->img_w), v_m = (double)(m / P->img_w);
    r[0] = P->fx * x[0] / z + P->cx - u_m;
    r[1] = P->fy * x[1] / z + P->cy - v_m;
    r[2] = z - Xi_m[2];
    /* d Pi / dx = (1/z) [[fx, 0, -fx x/z], [0, fy, -fy y/z]] (Supp. S1.3); d z / dx = e_z^T */
    Dr[0] = P->fx / z; Dr[1] = 0.0; Dr[2] = -P->fx * x[0] / (z * z);
    Dr[3] = 0.0; Dr[4] = P->fy / z; Dr[5] = -P->fy * x[1] / (z * z);
    Dr[6] = 0.0; Dr[7] = 0.0; Dr[8] = 1.0;
  } else {
    return 0;
  }
  double Dx[21], S[9];
  skew(x, S);
  for (int rr = 0; rr < 3; ++rr) {
    for (int c = 0; c < 3; ++c) {
      Dx[7 * rr + c] = (rr == c) ? 1.0 : 0.0;
      Dx[7 * rr + 3 + c] = -S[3 * rr + c];
    }
    Dx[7 * rr + 6] = x[rr];
  }
  double Jrel[21], JA[21];
  matmul(Dr, Dx, Jrel, 3, 3, 7);
  matmul(Jrel, Ad, JA, 3, 7, 7);
  for (int rr = 0; rr < 3; ++rr)
    for (int c = 0; c < 7; ++c) {
      J[14 * rr + c] = -JA[7 * rr + c];
      J[14 * rr + 7 + c] = JA[7 * rr + c];
    }
  return 3;
}

int orc_residual_jacobian_p(const orc_params* P, const double Ti[8], const double Tj[8], const double Xj_n[3],
                            const double Xi_m[3], int32_t m, double r[4], double J[56]) {
  double Tii[8], Tij[8], Ad[49];
  orc_sim3_inv(Ti, Tii);
  orc_sim3_mul(Tii, Tj, Tij);
  orc_sim3_adjoint(Tii, Ad);
  return residual_jacobian_family(P, Tij, Ad, Xj_n, Xi_m, m, r, J);
}

/* Huber cost and IRLS weight of a whitened residual norm e */
static double huber_cost(double e, double delta) { return e <= delta ? 0.5 * e * e : delta * (e - 0.5 * delta); }
#ifdef ORC_MUTANT_HUBER_SQ
static double huber_weight(double e, double delta) { return e <= delta ? 1.0 : delta / (e * e); }
#else
static double huber_weight(double e, double delta) { return e <= delta ? 1.0 : delta / e; }
#endif

/* Eq. backend_ray for one edge with the weight w(q, sigma^2) = sigma^2 / q read
 * as the information q / sigma^2 on the squared residual, a Huber norm on the
 * ray residual and a separate one on the distance residual, and q <= q_min
 * excluded; accumulates J^T W J and J^T W r (Eq. gauss_newton). */
void orc_linearize_edge(const orc_params* P, const double Ti[8], const double Tj[8], int64_t n_pix,
                        const double* X_i, const double* X_j, const int32_t* idx, const double* q, double H14[196],
                        double g14[14], double* cost, int64_t* n_valid) {
  double Tii[8], Tij[8], Ad[49];
  orc_sim3_inv(Ti, Tii);
  orc_sim3_mul(Tii, Tj, Tij);
  orc_sim3_adjoint(Tii, Ad);
  memset(H14, 0, 196 * sizeof(double));
  memset(g14, 0, 14 * sizeof(double));
  double c = 0.0;
  int64_t nv = 0;
  for (int64_t n = 0; n < n_pix; ++n) {
    int32_t m = idx[n];
    if (m < 0 || !(q[n] > P->q_min)) continue;
    double r[4], J[56], w[4];
    const int rows = residual_jacobian_family(P, Tij, Ad, X_j + 3 * n, X_i + 3 * (int64_t)m, m, r, J);
    if (!rows) continue;
    if (P->residual == ORC_RES_RAY) {
      /* one Huber norm on the ray residual, one on the distance residual */
      double lr = q[n] / (P->sigma_ray * P->sigma_ray), ld = q[n] / (P->sigma_dist * P->sigma_dist);
      double er = sqrt(lr * dot3(r, r)), ed = sqrt(ld) * fabs(r[3]);
      w[0] = w[1] = w[2] = lr * huber_weight(er, P->huber_delta);
      w[3] = ld * huber_weight(ed, P->huber_delta);
      c += huber_cost(er, P->huber_delta) + huber_cost(ed, P->huber_delta);
    } else if (P->residual == ORC_RES_POINT) {
      /* one Huber norm on the 3D point residual */
      double lp = q[n] / (P->sigma_point * P->sigma_point);
      double ep = sqrt(lp * dot3(r, r));
      w[0] = w[1] = w[2] = lp * huber_weight(ep, P->huber_delta);
      c += huber_cost(ep, P->huber_delta);
    } else {
      /* one Huber norm on the 2D pixel residual, one on the depth residual */
      double lp = q[n] / (P->sigma_pixel * P->sigma_pixel), lz = q[n] / (P->sigma_depth * P->sigma_depth);
      double ep = sqrt(lp * (r[0] * r[0] + r[1] * r[1])), ez = sqrt(lz) * fabs(r[2]);
      w[0] = w[1] = lp * huber_weight(ep, P->huber_delta);
      w[2] = lz * huber_weight(ez, P->huber_delta);
      c += huber_cost(ep, P->huber_delta) + huber_cost(ez, P->huber_delta);
    }
    for (int a = 0; a < 14; ++a) {
      for (int b = 0; b < 14; ++b) {
        double s = 0.0;
        for (int k = 0; k < rows; ++k) s += J[14 * k + a] * w[k] * J[14 * k + b];
        H14[14 * a + b] += s;
      }
      double s = 0.0;
#ifdef ORC_MUTANT_DROP_DIST_GRAD
      for (int k = 0; k < (rows == 4 ? 3 : rows); ++k) s += J[14 * k + a] * w[k] * r[k];
#else
      for (int k = 0; k < rows; ++k) s += J[14 * k + a] * w[k] * r[k];
#endif
      g14[a] += s;
    }
    ++nv;
  }
  *cost = c;
  if (n_valid) *n_valid = nv;
}

/* Sec. 3.5: accumulate the 14 x 14 blocks into the 7N system, fix the first
 * 7-DoF pose (drop its rows and columns), Cholesky, solve
 * (J^T W J) tau = -J^T W r and apply T <- Exp(tau) o T (Eq. gauss_newton). */
int orc_gn_solve(int N, int E, const int32_t* edges, const double* H14, const double* g14, int gauge, double* T,
                 double* tau_out) {
  int n = 7 * N;
  double* A = (double*)calloc((size_t)n * n, sizeof(double));
  double* g = (double*)calloc((size_t)n, sizeof(double));
  for (int e = 0; e < E; ++e) {
    int pose[2] = {edges[2 * e], edges[2 * e + 1]};
    for (int a = 0; a < 14; ++a) {
      int ia = 7 * pose[a / 7] + a % 7;
      g[ia] += g14[14 * e + a];
      for (int b = 0; b < 14; ++b) {
        int ib = 7 * pose[b / 7] + b % 7;
        A[(size_t)ia * n + ib] += H14[196 * (size_t)e + 14 * a + b];
      }
    }
  }
  int m = 7 * (N - 1);
  int* keep = (int*)malloc(sizeof(int) * (m > 0 ? m : 1));
#ifdef ORC_MUTANT_GAUGE
  gauge = N - 1;  /* the last pose fixed instead of the first */
#endif
  for (int k = 0, c = 0; k < N; ++k)
    if (k != gauge)
      for (int a = 0; a < 7; ++a) keep[c++] = 7 * k + a;
  double* L = (double*)calloc((size_t)m * m, sizeof(double));
  int status = 0;
  for (int j = 0; j < m && !status; ++j) { /* Cholesky-Banachiewicz */
    for (int i = j; i < m; ++i) {
      double s = A[(size_t)keep[i] * n + keep[j]];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
      if (i == j) {
        /* a pivot that is not positive relative to its diagonal entry means the
         * reduced system is singular (e.g. a component not connected to the
         * fixed pose) or indefinite */
        double diag = A[(size_t)keep[j] * n + keep[j]];
        if (!isfinite(s) || !(s > 1e-12 * diag)) { status = 3; break; }
        L[(size_t)j * m + j] = sqrt(s);
      } else {
        L[(size_t)i * m + j] = s / L[(size_t)j * m + j];
      }
    }
  }
  if (!status) {
    double* y = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
    for (int i = 0; i < m; ++i) { /* L y = -g */
      double s = -g[keep[i]];
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * m + k] * y[k];
      y[i] = s / L[(size_t)i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) { /* L^T x = y */
      double s = y[i];
      for (int k = i + 1; k < m; ++k) s -= L[(size_t)k * m + i] * y[k];
      y[i] = s / L[(size_t)i * m + i];
    }
    for (int k = 0; k < 7 * N; ++k) tau_out[k] = 0.0;
    for (int i = 0; i < m; ++i) tau_out[keep[i]] = y[i];
    for (int k = 0; k < N; ++k)
      if (k != gauge) orc_sim3_retract(tau_out + 7 * k, T + 8 * k);
    free(y);
  }
  free(L);
  free(keep);
  free(g);
  free(A);
  return status;
}

int orc_gauss_newton(const orc_params* P, int N, int E, const int32_t* edges, const int64_t* kf_off,
                     const int64_t* e_off, const double* X_canon, const int32_t* idx, const double* q, int iters,
                     int gauge, double* T, double* cost_hist, int* iters_done) {
  double* H14 = (double*)malloc(sizeof(double) * 196 * (size_t)(E > 0 ? E : 1));
  double* g14 = (double*)malloc(sizeof(double) * 14 * (size_t)(E > 0 ? E : 1));
  double* ce = (double*)malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
  double* tau = (double*)malloc(sizeof(double) * 7 * (size_t)N);
  int status = 0, done = 0;
  for (int it = 0; it < iters; ++it) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int e = 0; e < E; ++e) {
      int i = edges[2 * e], j = edges[2 * e + 1];
      orc_linearize_edge(P, T + 8 * i, T + 8 * j, e_off[e + 1] - e_off[e], X_canon + 3 * kf_off[i],
                         X_canon + 3 * kf_off[j], idx + e_off[e], q + e_off[e], H14 + 196 * (size_t)e,
                         g14 + 14 * (size_t)e, ce + e, NULL);
    }
    double c = 0.0;
    for (int e = 0; e < E; ++e) c += ce[e];
    if (cost_hist) cost_hist[it] = c;
    status = orc_gn_solve(N, E, edges, H14, g14, gauge, T, tau);
    done = it + 1;
    if (status) break;
    double mx = 0.0;
    for (int k = 0; k < 7 * N; ++k) mx = fmax(mx, fabs(tau[k]));
    if (mx < P->conv_tol) break;
  }
  if (iters_done) *iters_done = done;
  free(tau);
  free(ce);
  free(g14);
  free(H14);
  return status;
}

/* Gradient of E_g (Eq. backend_ray with the Huber norm) with respect to the
 * canonical pointmaps and the match confidences, at fixed poses and matches:
 * d rho(e) / d r = w_h(e) lambda r, with r = psi(x) - psi(y),
 * dpsi(x)/dx = (I - u u^T) / |x|, x = s R X_j + t, and
 * d rho(e) / d q = w_h(e) e^2 / (2 q) since e^2 = q |r|^2 / sigma^2. */
void orc_cost_grad(const orc_params* P, int N, int E, const int32_t* edges, const int64_t* kf_off,
                   const int64_t* e_off, const double* T, const double* X_canon, const int32_t* idx, const double* q,
                   double* dX, double* dq, double* cost) {
  (void)N;
  double c = 0.0;
  for (int e = 0; e < E; ++e) {
    int i = edges[2 * e], j = edges[2 * e + 1];
    double Tii[8], Tij[8], Rm[9];
    orc_sim3_inv(T + 8 * i, Tii);
    orc_sim3_mul(Tii, T + 8 * j, Tij);
    quat_to_rot(Tij + 3, Rm);
    double s = Tij[7];
    const double* Xi = X_canon + 3 * kf_off[i];
    const double* Xj = X_canon + 3 * kf_off[j];
    double* dXi = dX + 3 * kf_off[i];
    double* dXj = dX + 3 * kf_off[j];
    int64_t np = e_off[e + 1] - e_off[e];
    for (int64_t n = 0; n < np; ++n) {
      int32_t m = idx[e_off[e] + n];
      double qq = q[e_off[e] + n];
      if (m < 0 || !(qq > P->q_min)) continue;
      double x[3], y[3] = {Xi[3 * m], Xi[3 * m + 1], Xi[3 * m + 2]};
      orc_sim3_act(Tij, Xj + 3 * n, x);
      double d = norm3(x), dy = norm3(y);
      if (!(finite3(x) && finite3(y) && d > 0.0 && dy > 0.0)) continue;
      double u[3] = {x[0] / d, x[1] / d, x[2] / d}, v[3] = {y[0] / dy, y[1] / dy, y[2] / dy};
      double r[3] = {u[0] - v[0], u[1] - v[1], u[2] - v[2]}, rd = d - dy;
      double lr = qq / (P->sigma_ray * P->sigma_ray), ld = qq / (P->sigma_dist * P->sigma_dist);
      double er = sqrt(lr * dot3(r, r)), ed = sqrt(ld) * fabs(rd);
      double wr = lr * huber_weight(er, P->huber_delta), wd = ld * huber_weight(ed, P->huber_delta);
      c += huber_cost(er, P->huber_delta) + huber_cost(ed, P->huber_delta);
      /* dE/dx and dE/dy */
      double ur = dot3(u, r), vr = dot3(v, r), gx[3], gy[3];
      for (int k = 0; k < 3; ++k) {
        gx[k] = wr * (r[k] - u[k] * ur) / d + wd * rd * u[k];
        gy[k] = -wr * (r[k] - v[k] * vr) / dy - wd * rd * v[k];
      }
      /* dE/dX_j = (s R)^T dE/dx */
      for (int k = 0; k < 3; ++k) dXj[3 * n + k] += s * (Rm[k] * gx[0] + Rm[3 + k] * gx[1] + Rm[6 + k] * gx[2]);
      for (int k = 0; k < 3; ++k) dXi[3 * (int64_t)m + k] += gy[k];
      dq[e_off[e] + n] += (huber_weight(er, P->huber_delta) * er * er + huber_weight(ed, P->huber_delta) * ed * ed) /
                          (2.0 * qq);
    }
  }
  if (cost) *cost = c;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of one Gauss-Newton step (project form; not in the paper).        */
/* tau = -H^-1 g (Eq. gauss_newton, gauge pose removed).  For L = a . tau,    */
/* dL = -b^T (dH tau + dg) with b = H^-1 a, i.e. dL/dtheta = -d phi/d theta   */
/* at fixed b and tau, phi = sum over matches of (J b)^T W (J tau + r), J the */
/* 4 x 14 global Jacobian.  Each match's phi depends on X_j[n], X_i[m], q[n]; */
/* its seven partial derivatives are taken by complex-step differentiation   */
/* (Squire & Trapp 1998): phi(v + i h e_k) with h = 1e-30, derivative =       */
/* Im / h, exact to rounding.  The complex evaluation below restates the      */
/* literal residual and Jacobian of residual_jacobian_rel.                    */
/* ------------------------------------------------------------------------ */
typedef double complex cplx;

static cplx huber_weight_c(cplx e, double delta) { return creal(e) <= delta ? 1.0 : delta / e; }

/* phi of one match with complex inputs xj (point in frame j), y (point X_i[m]), q */
static cplx match_phi_c(const orc_params* P, const double Tij[8], const double Ad[49], const double b14[14],
                        const double t14[14], const cplx xj[3], const cplx y[3], cplx q) {
  double R[9];
  quat_to_rot(Tij + 3, R);
  cplx x[3];
  for (int r = 0; r < 3; ++r) x[r] = Tij[7] * (R[3 * r] * xj[0] + R[3 * r + 1] * xj[1] + R[3 * r + 2] * xj[2]) + Tij[r];
  cplx d = csqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  cplx dy = csqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
  cplx r4[4];
  for (int c = 0; c < 3; ++c) r4[c] = x[c] / d - y[c] / dy;
  r4[3] = d - dy;
  /* dx/dtau = [I, -[x]x, x]; dr/dx = (I - x x^T/d^2)/d (ray), x^T/d (distance) */
  cplx Dx[21], Dr[12], J[28];
  cplx S[9] = {0, -x[2], x[1], x[2], 0, -x[0], -x[1], x[0], 0};
  for (int rr = 0; rr < 3; ++rr) {
    for (int c = 0; c < 3; ++c) {
      Dx[7 * rr + c] = (rr == c) ? 1.0 : 0.0;
      Dx[7 * rr + 3 + c] = -S[3 * rr + c];
      Dr[3 * rr + c] = ((rr == c ? 1.0 : 0.0) - x[rr] * x[c] / (d * d)) / d;
    }
    Dx[7 * rr + 6] = x[rr];
  }
  for (int c = 0; c < 3; ++c) Dr[9 + c] = x[c] / d;
  for (int rr = 0; rr < 4; ++rr)
    for (int c = 0; c < 7; ++c) {
      cplx acc = 0;
      for (int k = 0; k < 3; ++k) acc += Dr[3 * rr + k] * Dx[7 * k + c];
      J[7 * rr + c] = acc;
    }
  /* global Jacobian [-J Ad, J Ad] applied to b and tau */
  cplx Jb[4], Jt[4];
  for (int rr = 0; rr < 4; ++rr) {
    cplx sb = 0, st = 0;
    for (int c = 0; c < 7; ++c) {
      cplx ja = 0;
      for (int k = 0; k < 7; ++k) ja += J[7 * rr + k] * Ad[7 * k + c];
      sb += -ja * b14[c] + ja * b14[7 + c];
      st += -ja * t14[c] + ja * t14[7 + c];
    }
    Jb[rr] = sb;
    Jt[rr] = st;
  }
  cplx lr = q / (P->sigma_ray * P->sigma_ray), ld = q / (P->sigma_dist * P->sigma_dist);
  cplx er = csqrt(lr * (r4[0] * r4[0] + r4[1] * r4[1] + r4[2] * r4[2]));
  cplx ed = csqrt(ld * r4[3] * r4[3]);
  cplx wr = lr * huber_weight_c(er, P->huber_delta), wd = ld * huber_weight_c(ed, P->huber_delta);
  return wr * (Jb[0] * (Jt[0] + r4[0]) + Jb[1] * (Jt[1] + r4[1]) + Jb[2] * (Jt[2] + r4[2])) +
         wd * Jb[3] * (Jt[3] + r4[3]);
}

/* Solve the gauge-reduced dense system H x = rhs (Cholesky); returns 0 or 3. */
static int dense_spd_solve(int m, const double* A, const double* rhs, double* x) {
  double* L = (double*)calloc((size_t)m * m, sizeof(double));
  int st = 0;
  for (int j = 0; j < m && !st; ++j)
    for (int i = j; i < m; ++i) {
      double s = A[(size_t)i * m + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
      if (i == j) {
        if (!(s > 1e-12 * A[(size_t)j * m + j]) || !isfinite(s)) { st = 3; break; }
        L[(size_t)j * m + j] = sqrt(s);
      } else {
        L[(size_t)i * m + j] = s / L[(size_t)j * m + j];
      }
    }
  if (!st) {
    for (int i = 0; i < m; ++i) {
      double s = rhs[i];
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * m + k] * x[k];
      x[i] = s / L[(size_t)i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
      double s = x[i];
      for (int k = i + 1; k < m; ++k) s -= L[(size_t)k * m + i] * x[k];
      x[i] = s / L[(size_t)i * m + i];
    }
  }
  free(L);
  return st;
}

int orc_gn_step_grad(const orc_params* P, int N, int E, const int32_t* edges, const int64_t* kf_off,
                     const int64_t* e_off, const double* T, const double* X_canon, const int32_t* idx, const double* q,
                     const double* dL_dtau, double dL_dcost, double* dX, double* dq, double* tau_out) {
  /* linearise every edge and assemble the dense 7N system */
  int n = 7 * N, gauge = 0, m = 7 * (N - 1);
  double* H14 = (double*)malloc(sizeof(double) * 196 * (size_t)(E > 0 ? E : 1));
  double* g14 = (double*)malloc(sizeof(double) * 14 * (size_t)(E > 0 ? E : 1));
  double cost;
  for (int e = 0; e < E; ++e) {
    int i = edges[2 * e], j = edges[2 * e + 1];
    orc_linearize_edge(P, T + 8 * i, T + 8 * j, e_off[e + 1] - e_off[e], X_canon + 3 * kf_off[i],
                       X_canon + 3 * kf_off[j], idx + e_off[e], q + e_off[e], H14 + 196 * (size_t)e,
                       g14 + 14 * (size_t)e, &cost, NULL);
  }
  double* A = (double*)calloc((size_t)n * n, sizeof(double));
  double* g = (double*)calloc((size_t)n, sizeof(double));
  for (int e = 0; e < E; ++e) {
    int pose[2] = {edges[2 * e], edges[2 * e + 1]};
    for (int a = 0; a < 14; ++a) {
      int ia = 7 * pose[a / 7] + a % 7;
      g[ia] += g14[14 * e + a];
      for (int bb = 0; bb < 14; ++bb) A[(size_t)ia * n + 7 * pose[bb / 7] + bb % 7] += H14[196 * (size_t)e + 14 * a + bb];
    }
  }
  double* Ar = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * (m > 0 ? m : 1));
  double* rg = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
  double* ra = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
  double* tr = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
  double* br = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
  for (int i = 0; i < m; ++i) {
    rg[i] = -g[7 + i];
    ra[i] = dL_dtau ? dL_dtau[7 + i] : 0.0;
    for (int k = 0; k < m; ++k) Ar[(size_t)i * m + k] = A[(size_t)(7 + i) * n + 7 + k];
  }
  int st = dense_spd_solve(m, Ar, rg, tr);
  if (!st) st = dense_spd_solve(m, Ar, ra, br);
  double* tau = (double*)calloc((size_t)n, sizeof(double));
  double* b = (double*)calloc((size_t)n, sizeof(double));
  if (!st)
    for (int i = 0; i < m; ++i) {
      tau[7 + i] = tr[i];
      b[7 + i] = br[i];
    }
  if (tau_out) memcpy(tau_out, tau, sizeof(double) * n);
  (void)gauge;
  /* cost term */
  double c;
  orc_cost_grad(P, N, E, edges, kf_off, e_off, T, X_canon, idx, q, dX, dq, &c);
  if (dL_dcost != 1.0) {
    /* orc_cost_grad accumulated the unit-weight gradient: rescale it */
    for (int64_t k = 0; k < 3 * kf_off[N]; ++k) dX[k] *= dL_dcost;
    for (int64_t k = 0; k < e_off[E]; ++k) dq[k] *= dL_dcost;
  }
  /* step term by complex-step differentiation of phi */
  if (dL_dtau && !st) {
    const double h = 1e-30;
    for (int e = 0; e < E; ++e) {
      int i = edges[2 * e], j = edges[2 * e + 1];
      double Tii[8], Tij[8], Ad[49], b14[14], t14[14];
      orc_sim3_inv(T + 8 * i, Tii);
      orc_sim3_mul(Tii, T + 8 * j, Tij);
      orc_sim3_adjoint(Tii, Ad);
      for (int k = 0; k < 7; ++k) {
        b14[k] = b[7 * i + k];
        b14[7 + k] = b[7 * j + k];
        t14[k] = tau[7 * i + k];
        t14[7 + k] = tau[7 * j + k];
      }
      const double* Xi = X_canon + 3 * kf_off[i];
      const double* Xj = X_canon + 3 * kf_off[j];
      int64_t np = e_off[e + 1] - e_off[e];
      for (int64_t nn = 0; nn < np; ++nn) {
        int32_t mm = idx[e_off[e] + nn];
        double qq = q[e_off[e] + nn];
        if (mm < 0 || !(qq > P->q_min)) continue;
        const double* xj = Xj + 3 * nn;
        const double* y = Xi + 3 * (int64_t)mm;
        double xw[3];
        orc_sim3_act(Tij, xj, xw);
        if (!(finite3(xw) && finite3(y) && norm3(xw) > 0 && norm3(y) > 0)) continue;
        double grad[7];
        for (int k = 0; k < 7; ++k) {
          cplx xc[3] = {xj[0], xj[1], xj[2]}, yc[3] = {y[0], y[1], y[2]}, qc = qq;
          if (k < 3) xc[k] += _Complex_I * h;
          else if (k < 6) yc[k - 3] += _Complex_I * h;
          else qc += _Complex_I * h;
          grad[k] = cimag(match_phi_c(P, Tij, Ad, b14, t14, xc, yc, qc)) / h;
        }
        for (int k = 0; k < 3; ++k) {
          dX[3 * (kf_off[j] + nn) + k] -= grad[k];
          dX[3 * (kf_off[i] + mm) + k] -= grad[3 + k];
        }
        dq[e_off[e] + nn] -= grad[6];
      }
    }
  }
  free(b); free(tau); free(br); free(tr); free(ra); free(rg); free(Ar); free(g); free(A); free(g14); free(H14);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3 pointmap fusion: the keyframe's canonical pointmap and confidence */
/* are updated by a running weighted average with the new prediction of the  */
/* keyframe's points (made with the current frame) moved into the keyframe  */
/* frame by T_kf:  X~ <- (C~ X~ + C (T_kf X)) / (C~ + C),  C~ <- C~ + C.       */
/* Reading: a prediction with a non-finite or zero point, or a confidence    */
/* that is not positive, leaves the pixel unchanged.                         */
/* ------------------------------------------------------------------------ */
void orc_fuse(const double T_kf[8], int64_t n, double* X_canon, double* C_canon, const double* X_kf,
              const double* C_kf) {
  for (int64_t p = 0; p < n; ++p) {
    const double* x = X_kf + 3 * p;
    double c = C_kf[p];
    if (!(finite3(x) && norm3(x) > 0.0 && c > 0.0 && isfinite(c))) continue;
    double y[3];
    orc_sim3_act(T_kf, x, y);
    double cc = C_canon[p];
    for (int k = 0; k < 3; ++k) X_canon[3 * p + k] = (cc * X_canon[3 * p + k] + c * y[k]) / (cc + c);
    C_canon[p] = cc + c;
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.4 keyframe criterion counts for one edge's matches: the number of  */
/* valid matches and the number of distinct reference (keyframe) pixels they */
/* hit.  A new keyframe is added when either fraction falls below omega_k.  */
/* ------------------------------------------------------------------------ */
void orc_match_stats(int64_t n_qry, int64_t n_ref, const int32_t* idx, int64_t* n_valid, int64_t* n_unique) {
  unsigned char* seen = (unsigned char*)calloc((size_t)(n_ref > 0 ? n_ref : 1), 1);
  int64_t v = 0, u = 0;
  for (int64_t p = 0; p < n_qry; ++p) {
    int32_t m = idx[p];
    if (m < 0 || m >= n_ref) continue;
    ++v;
    if (!seen[m]) {
      seen[m] = 1;
      ++u;
    }
  }
  free(seen);
  *n_valid = v;
  *n_unique = u;
}

/* Sec. 3.6, first change for a known camera: the prediction contributes only
 * its depth; the point is rebuilt on the pixel's ray of the pinhole model. */
void orc_calib_backproject(int H, int W, double fx, double fy, double cx, double cy, double* X) {
  for (int64_t p = 0; p < (int64_t)H * W; ++p) {
    const double u = (double)(p % W), v = (double)(p / W), z = X[3 * p + 2];
    X[3 * p + 0] = z * (u - cx) / fx;
    X[3 * p + 1] = z * (v - cy) / fy;
    X[3 * p + 2] = z;
  }
}
