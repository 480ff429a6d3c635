/*
 * FP64 CPU oracle for the ray-error Sim(3) Gauss-Newton path of MASt3R-SLAM
 * (arXiv 2412.12392).  TEST INFRASTRUCTURE ONLY: tests, the smoke check and
 * the benchmark's CPU-baseline leg call it; the product path never does.
 *
 * Plain, slow, obviously correct: every function follows a passage of the
 * paper, in double precision, without blocking, fusion or reordering.  It
 * shares no code with the CUDA library.
 *
 * Pose layout: 8 doubles = translation t (3), unit quaternion q = (x, y, z, w)
 * (4), scale s (1); the pose maps a point X to s R(q) X + t (Eq. 1).
 * Tangent layout: tau = (rho (3), phi (3), sigma (1)), hat(tau) =
 * [[ [phi]x + sigma I, rho ], [0, 0]] and Exp(tau) = expm(hat(tau)).
 */
#ifndef MSLAM_ORACLE_H
#define MSLAM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double sigma_ray;      /* sigma_r of w(q, sigma^2), Sec. 3.3 */
  double sigma_dist;     /* sigma of the small-weight distance term */
  double huber_delta;    /* Huber threshold on the whitened residual norm */
  double q_min;          /* matches with q <= q_min are excluded (w = inf) */
  double lm_lambda;      /* Levenberg-Marquardt damping of the matching step */
  int lm_iters;          /* matching iterations (Sec. 3.2: 10 suffice) */
  int win_radius;        /* refinement window radius (candidates 2r+1 squared) */
  int n_levels;          /* coarse-to-fine levels of the refinement */
  int win_dilation[4];   /* candidate spacing per level, coarse first */
  double max_rel_dist3d; /* invalidate a match if |X_ref[m] - x| > this * |x| */
  double conv_tol;       /* GN stops once max|tau| < conv_tol */
  /* residual family of the Gauss-Newton cost */
  int residual;          /* 0: ray + distance (Eq. backend_ray); 1: 3D point (Eq. track_point);
                            2: pixel + depth with known pinhole calibration (Eq. backend_pixel) */
  double sigma_point;    /* sigma_p of the point error */
  double sigma_pixel;    /* sigma_Pi of the pixel error (pixels) */
  double sigma_depth;    /* sigma of the small-weight depth term of the pixel family */
  double fx, fy, cx, cy; /* pinhole calibration K of the pixel family (Supp. S1.3) */
  int img_w;             /* reference image width: pixel m sits at (m mod W, m div W) */
} orc_params;

#define ORC_RES_RAY 0
#define ORC_RES_POINT 1
#define ORC_RES_PIXEL 2

/* --- Sim(3), Eq. 1 -------------------------------------------------------- */
void orc_sim3_exp(const double tau[7], double T[8]);
void orc_sim3_log(const double T[8], double tau[7]);
void orc_sim3_mul(const double A[8], const double B[8], double C[8]);
void orc_sim3_inv(const double A[8], double Ai[8]);
void orc_sim3_act(const double T[8], const double x[3], double y[3]);
void orc_sim3_matrix(const double T[8], double M[16]);
void orc_sim3_adjoint(const double T[8], double Ad[49]);
void orc_sim3_retract(const double tau[7], double T[8]); /* T <- Exp(tau) o T */

/* --- ray normalisation, Sec. 3.1 ------------------------------------------ */
void orc_ray_image(const double* X, int64_t n, double* R);

/* --- projective matching, Sec. 3.2 (Eq. 2) plus feature refinement -------- */
/* Query pixels pix[0..n_pix) (or all H*W if pix == NULL).  Outputs idx (-1 =
 * invalid) and q; diag (9 doubles per pixel, may be NULL) = p*_u, p*_v, last
 * LM step norm, level margins (best - runner-up score) for levels 0 and 1,
 * distance of p* to the nearest rounding boundary, |X_ref[m]-x|/|x|,
 * validity before the 3D check, final best score. */
void orc_match(const orc_params* P, int H, int W, int d,
               const double* X_ref, const double* X_qry,
               const double* D_ref, const double* D_qry,
               const double* Q_ref, const double* Q_qry,
               const int32_t* init_idx,
               const int64_t* pix, int64_t n_pix,
               int32_t* idx_out, double* q_out, double* diag);

/* --- per-match residual and global Jacobian, Supp. S1.2 and S1.4 --------- */
/* r (4) = ray residual (3) and distance residual; J (4 x 14, row-major) =
 * derivative with respect to left perturbations of T_i (cols 0..6) and T_j
 * (cols 7..13).  Returns 0 if the match is degenerate. */
int orc_residual_jacobian(const double Ti[8], const double Tj[8], const double Xj_n[3],
                          const double Xi_m[3], double r[4], double J[56]);

/* Any residual family of P->residual: returns the number of residual rows
 * (4 ray, 3 point, 3 pixel) or 0 if the match is degenerate; m is the
 * reference pixel index (used by the pixel family). */
int orc_residual_jacobian_p(const orc_params* P, const double Ti[8], const double Tj[8], const double Xj_n[3],
                            const double Xi_m[3], int32_t m, double r[4], double J[56]);

/* --- per-edge linearisation (Eq. backend_ray and Eq. gauss_newton) -------- */
/* Edge (i, j): X_i is keyframe i's canonical pointmap (gathered at m), X_j
 * keyframe j's (streamed at n); idx[n] = m or -1, q[n] the match confidence.
 * H14 (14 x 14) = sum J^T W J, g14 = sum J^T W r, cost = sum of Huber costs. */
void orc_linearize_edge(const orc_params* P, const double Ti[8], const double Tj[8],
                        int64_t n_pix, const double* X_i, const double* X_j,
                        const int32_t* idx, const double* q,
                        double H14[196], double g14[14], double* cost, int64_t* n_valid);

/* --- Gauss-Newton solve with the first pose fixed (Sec. 3.5) -------------- */
/* Dense assembly of the 7N system from per-edge 14 x 14 blocks, removal of
 * pose `gauge`, Cholesky, substitution, T_k <- Exp(tau_k) o T_k.  Returns 0
 * on success, 3 if the system is not positive definite.  tau_out [N, 7]. */
int orc_gn_solve(int N, int E, const int32_t* edges, const double* H14, const double* g14,
                 int gauge, double* T, double* tau_out);

/* Full loop: iters x (linearise every edge, solve).  X_canon pool indexed by
 * kf_off, match pools indexed by e_off.  cost_hist [iters] may be NULL. */
int orc_gauss_newton(const orc_params* P, int N, int E, const int32_t* edges,
                     const int64_t* kf_off, const int64_t* e_off,
                     const double* X_canon, const int32_t* idx, const double* q,
                     int iters, int gauge, double* T, double* cost_hist, int* iters_done);

/* --- adjoint (gradient) of the weighted cost ------------------------------ */
/* dE/dX_canon for the cost of all edges at fixed poses, matches and q (Huber
 * weights differentiated), and dE/dq.  Accumulates into dX [pool, 3], dq. */
void orc_cost_grad(const orc_params* P, int N, int E, const int32_t* edges,
                   const int64_t* kf_off, const int64_t* e_off, const double* T,
                   const double* X_canon, const int32_t* idx, const double* q,
                   double* dX, double* dq, double* cost);

/* Gradient of L = dL_dcost * E_g + dL_dtau . tau, tau = -H^-1 g the Gauss-
 * Newton step at T with the first pose fixed, with respect to X_canon and q
 * (dX, dq overwritten).  The step term is differentiated by complex step.
 * tau_out [N, 7] may be NULL.  Returns 0, or 3 if H is not positive definite. */
int orc_gn_step_grad(const orc_params* P, int N, int E, const int32_t* edges, const int64_t* kf_off,
                     const int64_t* e_off, const double* T, const double* X_canon, const int32_t* idx, const double* q,
                     const double* dL_dtau, double dL_dcost, double* dX, double* dq, double* tau_out);

/* --- pointmap fusion, Sec. 3.3 -------------------------------------------- */
/* X_canon [n, 3] and C_canon [n] updated in place with the prediction X_kf
 * (keyframe points predicted with the current frame, in the frame's
 * coordinates) and its confidence C_kf, moved by T_kf (frame -> keyframe). */
void orc_fuse(const double T_kf[8], int64_t n, double* X_canon, double* C_canon, const double* X_kf,
              const double* C_kf);

/* --- known calibration, Sec. 3.6 ----------------------------------------- */
/* X [H*W, 3] in place: only the depth z of each point is kept and the point
 * is placed on its pixel's ray under the pinhole K,
 * X[p] = z ((u - cx) / fx, (v - cy) / fy, 1), (u, v) = (p mod W, p div W). */
void orc_calib_backproject(int H, int W, double fx, double fy, double cx, double cy, double* X);

/* --- keyframe criterion counts, Sec. 3.4 ---------------------------------- */
void orc_match_stats(int64_t n_qry, int64_t n_ref, const int32_t* idx, int64_t* n_valid, int64_t* n_unique);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
