// Shared definitions of the CUDA library: plan tables as laid out in device
// memory, parameter block, FP16/FP32 loads, FP64 Sim(3) device algebra and
// the host-side error plumbing.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mslam.h"

namespace mslam {

#ifndef MSLAM_LIN_TILE
#define MSLAM_LIN_TILE 8192
#endif
constexpr int kLinTile = MSLAM_LIN_TILE;  // default pixels per linearisation work tile
constexpr int kLinThreads = 256;     // threads per linearisation block
constexpr int kNumAcc = 30;          // accumulators of the ray family's relative 7x7 system
constexpr int kFamAcc = 37;          // accumulators of the point / pixel families (28 + 7 + 2)
constexpr int kAccStride = 40;       // floats per tile partial in the workspace
#ifndef MSLAM_MATCH_THREADS
#define MSLAM_MATCH_THREADS 256
#endif
constexpr int kMatchThreads = MSLAM_MATCH_THREADS;  // threads of a match block (default 32 x 8)
constexpr int kMatchBX = 32;
constexpr int kSolveThreads = 512;
constexpr int kLfRow = 12;          // floats per row of a block of the mixed-precision solve's FP32 factor
                                    // in shared memory (8 when the factor stays in the workspace)

// One directed edge as seen by the kernels.
struct DevEdge {
  int32_t i, j;         // reference keyframe, query keyframe
  int32_t H, W;         // image size (both keyframes)
  int64_t off_e;        // offset of the edge in the edge pools (pixels)
  int64_t off_i, off_j; // offsets of the keyframes in the keyframe pool
  int32_t graph;        // graph id
  int32_t tile_begin;   // linearisation tiles of this edge: [tile_begin, tile_end)
  int32_t tile_end;
  int32_t mblock_begin; // first match block of this edge (flat grid)
};

struct DevTile {
  int32_t edge;
  int32_t begin;  // pixel range within the edge
  int32_t end;
  int32_t pad;
};

// Per-graph symbolic factorisation (all indices local to the graph, arrays
// concatenated across graphs at the given offsets).
struct DevGraph {
  int32_t m;          // non-fixed poses = block rows of the reduced system
  int32_t n_blocks;   // 7x7 blocks of L: m diagonal blocks first, then off-diagonal
  int32_t gauge;      // fixed keyframe (global index)
  int32_t int_end;    // end of this graph's table integers (they start at off_pose)
  int32_t off_pose;   // -> pose_of_pos [m]: global keyframe at elimination position p
  int32_t off_col;    // -> col_ptr [m + 1] (into col_rows / col_blk, relative)
  int32_t off_colent; // -> col_rows, col_blk entries
  int32_t off_trip;   // -> trip_ptr [m + 1]
  int32_t off_tripent;// -> trips (3 ints each: target, src_row_block, src_col_block)
  int32_t off_asm;    // -> asm_ptr [n_blocks + 1]
  int32_t off_asment; // -> asm entries: edge * 4 + quadrant
  int32_t off_gasm;   // -> gasm_ptr [m + 1]
  int32_t off_gasment;// -> gasm entries: edge * 2 + side
  int32_t n_levels;   // levels of the elimination dependency schedule
  int32_t off_lev;    // -> lev_ptr [n_levels + 1] into lev_cols
  int32_t off_levcols;// -> positions ordered by level
  int32_t off_levtgt; // -> [n_levels + 1] into the per-level target-block list
  int32_t off_tgtlist;// -> target blocks of each level (diagonal, then column blocks, per column)
  int32_t off_tptr;   // -> tptr [n_blocks + 1] into pairs
  int32_t off_pairs;  // -> (row block, column block) source pairs of each target, in column order
  int32_t off_rsptr;  // -> rsptr [m + 1] into row structure
  int32_t off_rs;     // -> (column c, block L(p, c)) of each position p, in column order
  int32_t off_blkcol; // -> [n_blocks] column position of each block
  int32_t off_blkrow; // -> [n_blocks] row position of each block
  int32_t off_levupd; // -> [n_levels + 1] into the per-level list of targets that receive updates
  int32_t off_updlist;// -> those targets (a subset of the level's target list, same order)
  int32_t pad1;
  int64_t ws_off;     // offset (doubles) of this graph's numeric workspace
  int64_t ws_mixed;   // offset (doubles) of the mixed-precision solve's inputs: scaled FP32 factor
                      // [n_blocks][7][kLfRow or 8] floats in n_blocks * 7 * kLfRow, then S (7 m) and -g (7 m) in FP64
};

// Device view of a plan (pointers into the uploaded table blob).
struct PlanView {
  int32_t N, E, G, n_tiles, n_mblocks;
  int64_t P;  // pixels of the edge pools
  int32_t lin_tile;           // pixels per linearisation tile
  int32_t match_bx, match_by; // match block shape (match_bx * match_by = 256 threads)
  int32_t match_ppt;          // query pixels per match thread (rows match_by apart)
  uint32_t wait_polls;        // polls of a bounded device wait; 0 = give up at once, issuing no copy
  const DevEdge* edges;
  const DevTile* tiles;
  const DevGraph* graphs;
  const int32_t* ints;  // all int32 symbolic arrays of the graphs
};

// Parameters converted for the kernels.
struct KParams {
  float sigma_ray, sigma_dist, huber_delta, q_min, lm_lambda, max_rel_dist3d;
  int lm_iters, win_radius, n_levels;
  int win_dilation[4];
  double conv_tol;
};

inline KParams to_kparams(const mslam_params& p) {
  KParams k;
  k.sigma_ray = p.sigma_ray;
  k.sigma_dist = p.sigma_dist;
  k.huber_delta = p.huber_delta;
  k.q_min = p.q_min;
  k.lm_lambda = p.lm_lambda;
  k.max_rel_dist3d = p.max_rel_dist3d;
  k.lm_iters = p.lm_iters;
  k.win_radius = p.win_radius;
  k.n_levels = p.n_levels;
  for (int l = 0; l < 4; ++l) k.win_dilation[l] = p.win_dilation[l];
  k.conv_tol = p.conv_tol;
  return k;
}

// Hardware reciprocal square root approximation with denormal inputs
// flushed to zero (one MUFU instruction; the accuracy of rsqrtf for normal
// inputs).  For squared norms of points and whitened residuals, which are
// never denormal here.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------- loads
template <typename T> __device__ __forceinline__ float ldf(const T* p);
template <> __device__ __forceinline__ float ldf<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldf<__half>(const __half* p) {
  return __half2float(__ldg(reinterpret_cast<const __half*>(p)));
}
template <typename T> __device__ __forceinline__ void stf(T* p, float v);
template <> __device__ __forceinline__ void stf<float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void stf<__half>(__half* p, float v) { *p = __float2half_rn(v); }

template <typename T>
__device__ __forceinline__ float3 ld3(const T* base, int64_t pix) {
  const T* p = base + 3 * pix;
  return make_float3(ldf(p), ldf(p + 1), ldf(p + 2));
}

__device__ __forceinline__ bool finite3(float3 a) {
  return isfinite(a.x) && isfinite(a.y) && isfinite(a.z);
}

// ---------------------------------------------------------------- FP64 Sim(3)
// Pose: t (3), q = (x, y, z, w) (4), s (1); X -> s R(q) X + t.
struct Sim3d {
  double t[3];
  double q[4];
  double s;
};

__device__ __forceinline__ Sim3d load_pose(const double* T) {
  Sim3d a;
  for (int k = 0; k < 3; ++k) a.t[k] = T[k];
  for (int k = 0; k < 4; ++k) a.q[k] = T[3 + k];
  a.s = T[7];
  return a;
}

__device__ __forceinline__ void store_pose(const Sim3d& a, double* T) {
  for (int k = 0; k < 3; ++k) T[k] = a.t[k];
  for (int k = 0; k < 4; ++k) T[3 + k] = a.q[k];
  T[7] = a.s;
}

__device__ __forceinline__ void rot_of(const double q[4], double R[9]) {
  const double x = q[0], y = q[1], z = q[2], w = q[3];
  const double xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y,
               wz = w * z;
  R[0] = 1.0 - 2.0 * (yy + zz); R[1] = 2.0 * (xy - wz);       R[2] = 2.0 * (xz + wy);
  R[3] = 2.0 * (xy + wz);       R[4] = 1.0 - 2.0 * (xx + zz); R[5] = 2.0 * (yz - wx);
  R[6] = 2.0 * (xz - wy);       R[7] = 2.0 * (yz + wx);       R[8] = 1.0 - 2.0 * (xx + yy);
}

__device__ __forceinline__ void qmul(const double a[4], const double b[4], double c[4]) {
  c[3] = a[3] * b[3] - (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]);
  c[0] = a[3] * b[0] + b[3] * a[0] + (a[1] * b[2] - a[2] * b[1]);
  c[1] = a[3] * b[1] + b[3] * a[1] + (a[2] * b[0] - a[0] * b[2]);
  c[2] = a[3] * b[2] + b[3] * a[2] + (a[0] * b[1] - a[1] * b[0]);
}

__device__ __forceinline__ void qnormalise(double q[4]) {
  const double inv = 1.0 / sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) q[k] *= inv;
}

// a o b
__device__ __forceinline__ Sim3d compose(const Sim3d& a, const Sim3d& b) {
  Sim3d c;
  double R[9];
  rot_of(a.q, R);
  for (int r = 0; r < 3; ++r) c.t[r] = a.s * (R[3 * r] * b.t[0] + R[3 * r + 1] * b.t[1] + R[3 * r + 2] * b.t[2]) + a.t[r];
  qmul(a.q, b.q, c.q);
  qnormalise(c.q);
  c.s = a.s * b.s;
  return c;
}

__device__ __forceinline__ Sim3d inverse(const Sim3d& a) {
  Sim3d b;
  double R[9];
  rot_of(a.q, R);
  b.s = 1.0 / a.s;
  for (int r = 0; r < 3; ++r) b.t[r] = -b.s * (R[r] * a.t[0] + R[3 + r] * a.t[1] + R[6 + r] * a.t[2]);
  b.q[0] = -a.q[0]; b.q[1] = -a.q[1]; b.q[2] = -a.q[2]; b.q[3] = a.q[3];
  return b;
}

// Ad_T (7x7, row-major) for T Exp(tau) T^-1 = Exp(Ad_T tau), tau = (rho, phi, sigma):
// [[sR, [t]x R, -t], [0, R, 0], [0, 0, 1]].
__device__ __forceinline__ void adjoint_of(const Sim3d& a, double Ad[49]) {
  double R[9];
  rot_of(a.q, R);
  for (int k = 0; k < 49; ++k) Ad[k] = 0.0;
  const double* t = a.t;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      Ad[7 * r + c] = a.s * R[3 * r + c];
      Ad[7 * (3 + r) + 3 + c] = R[3 * r + c];
    }
  // [t]x R: row r of [t]x dotted with column c of R
  for (int c = 0; c < 3; ++c) {
    Ad[7 * 0 + 3 + c] = -t[2] * R[3 + c] + t[1] * R[6 + c];
    Ad[7 * 1 + 3 + c] = t[2] * R[c] - t[0] * R[6 + c];
    Ad[7 * 2 + 3 + c] = -t[1] * R[c] + t[0] * R[3 + c];
  }
  Ad[7 * 0 + 6] = -t[0];
  Ad[7 * 1 + 6] = -t[1];
  Ad[7 * 2 + 6] = -t[2];
  Ad[48] = 1.0;
}

// 1/k for k = 0..39 (entry 0 unused): the series below multiply by these
// instead of dividing (an FP64 division costs ~400 cycles on this GPU).
__device__ __constant__ const double kInvInt[40] = {
    0.0,       1.0,       1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,  1.0 / 7,  1.0 / 8,  1.0 / 9,
    1.0 / 10,  1.0 / 11,  1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17, 1.0 / 18, 1.0 / 19,
    1.0 / 20,  1.0 / 21,  1.0 / 22, 1.0 / 23, 1.0 / 24, 1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29,
    1.0 / 30,  1.0 / 31,  1.0 / 32, 1.0 / 33, 1.0 / 34, 1.0 / 35, 1.0 / 36, 1.0 / 37, 1.0 / 38, 1.0 / 39};

// m_n(s) = integral_0^1 x^n e^{s x} dx: the power series
// sum_k s^k / (k! (n + k + 1)) for |s| < 1 (stopped once the terms vanish),
// the upward recurrence m_n = (e^s - n m_{n-1}) / s otherwise.
__device__ __forceinline__ double moment_exp(int n, double s) {
  if (fabs(s) < 1.0) {
    double c = 1.0, acc = 0.0;
    for (int k = 0; k + n + 1 < 40 && k < 34; ++k) {
      acc = fma(c, kInvInt[n + k + 1], acc);
      c *= s * kInvInt[k + 1];
      if (fabs(c) < 1e-18) break;
    }
    return acc;
  }
  const double es = exp(s);
  double mval = expm1(s) / s;
  for (int k = 1; k <= n; ++k) mval = (es - k * mval) / s;
  return mval;
}

// Exp(tau) for tau = (rho, phi, sigma): R = exp([phi]x), s = e^sigma,
// t = V rho with V = int_0^1 e^{x sigma} R(x phi) dx = a I + b [phi]x + c [phi]x^2.
__device__ __forceinline__ Sim3d sim3_exp(const double tau[7]) {
  const double px = tau[3], py = tau[4], pz = tau[5], sg = tau[6];
  const double th2 = px * px + py * py + pz * pz, th = sqrt(th2);
  double a = moment_exp(0, sg), b, c;
  if (th < 1e-4) {
    b = moment_exp(1, sg) - th2 * moment_exp(3, sg) / 6.0;
    c = 0.5 * moment_exp(2, sg) - th2 * moment_exp(4, sg) / 24.0;
  } else {
    double sn, cs;
    sincos(th, &sn, &cs);
    const double es = exp(sg), den = sg * sg + th2;
    const double ic = ((es * cs - 1.0) * sg + es * th * sn) / den;  // int e^{sx} cos(th x)
    const double is = (es * sn * sg - (es * cs - 1.0) * th) / den;  // int e^{sx} sin(th x)
    b = is / th;
    c = (a - ic) / th2;
  }
  Sim3d e;
  const double h = (th < 1e-6) ? (0.5 - th2 / 48.0) : sin(0.5 * th) / th;
  e.q[0] = h * px; e.q[1] = h * py; e.q[2] = h * pz; e.q[3] = cos(0.5 * th);
  qnormalise(e.q);
  e.s = exp(sg);
  const double r0 = tau[0], r1 = tau[1], r2 = tau[2];
  // phi x rho and phi x (phi x rho)
  const double c0 = py * r2 - pz * r1, c1 = pz * r0 - px * r2, c2 = px * r1 - py * r0;
  const double d0 = py * c2 - pz * c1, d1 = pz * c0 - px * c2, d2 = px * c1 - py * c0;
  e.t[0] = a * r0 + b * c0 + c * d0;
  e.t[1] = a * r1 + b * c1 + c * d1;
  e.t[2] = a * r2 + b * c2 + c * d2;
  return e;
}

// Exp(tau) of sim3_exp split into independent pieces, so that different
// warps can evaluate them side by side: piece 0 sin and cos of theta, 1
// e^sigma, 2 the quaternion's half-angle terms, 3 the moment m_0, 4-7 the
// moments m_1, m_3, m_2, m_4 of the small-angle branch.  part[10] holds
// sn, cs, es, h, q3, m0, m1, m3, m2, m4.  The same formulas as sim3_exp on the
// same inputs, so the same values.
__device__ inline void sim3_exp_piece(const double* tau, int kind, double* part) {
  const double px = tau[3], py = tau[4], pz = tau[5], sg = tau[6];
  const double th2 = px * px + py * py + pz * pz, th = sqrt(th2);
  const bool small = th < 1e-4;
  if (kind == 0) {
    double sn = 0.0, cs = 0.0;
    if (!small) sincos(th, &sn, &cs);
    part[0] = sn;
    part[1] = cs;
  } else if (kind == 1) {
    part[2] = exp(sg);
  } else if (kind == 2) {
    part[3] = (th < 1e-6) ? (0.5 - th2 / 48.0) : sin(0.5 * th) / th;
    part[4] = cos(0.5 * th);
  } else if (kind == 3) {
    part[5] = moment_exp(0, sg);
  } else {
    const int n = kind == 4 ? 1 : kind == 5 ? 3 : kind == 6 ? 2 : 4;
    part[2 + kind] = small ? moment_exp(n, sg) : 0.0;
  }
}

__device__ inline Sim3d sim3_exp_parts(const double* tau, const double* part) {
  const double px = tau[3], py = tau[4], pz = tau[5], sg = tau[6];
  const double th2 = px * px + py * py + pz * pz, th = sqrt(th2);
  const double sn = part[0], cs = part[1], es = part[2], h = part[3], q3 = part[4], a = part[5];
  double b, c;
  if (th < 1e-4) {
    b = part[6] - th2 * part[7] / 6.0;
    c = 0.5 * part[8] - th2 * part[9] / 24.0;
  } else {
    const double den = sg * sg + th2;
    const double ic = ((es * cs - 1.0) * sg + es * th * sn) / den;
    const double is = (es * sn * sg - (es * cs - 1.0) * th) / den;
    b = is / th;
    c = (a - ic) / th2;
  }
  Sim3d e;
  e.q[0] = h * px;
  e.q[1] = h * py;
  e.q[2] = h * pz;
  e.q[3] = q3;
  qnormalise(e.q);
  e.s = es;
  const double r0 = tau[0], r1 = tau[1], r2 = tau[2];
  const double c0 = py * r2 - pz * r1, c1 = pz * r0 - px * r2, c2 = px * r1 - py * r0;
  const double d0 = py * c2 - pz * c1, d1 = pz * c0 - px * c2, d2 = px * c1 - py * c0;
  e.t[0] = a * r0 + b * c0 + c * d0;
  e.t[1] = a * r1 + b * c1 + c * d1;
  e.t[2] = a * r2 + b * c2 + c * d2;
  return e;
}

// 1/sqrt(d) in FP64 by Newton-Raphson iteration for the inverse square root,
// y <- y (3 - d y^2) / 2, seeded with the single-precision hardware estimate:
// two iterations take the ~23-bit seed past FP64 precision.  On this GPU a
// dependent FP64 operation costs ~64 cycles and FP64 sqrt + reciprocal
// ~1080, so the diagonal pivots of the factorisation use this (~8 dependent
// operations); outside the single-precision range it falls back to
// 1.0 / sqrt(d).
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double y = (double)rsqrtf((float)d);
  const double hd = 0.5 * d;
  y = y * fma(-hd * y, y, 1.5);
  y = y * fma(-hd * y, y, 1.5);
  return y;
}

// 1/x in FP64 by Newton's iteration for the reciprocal, y <- y (2 - x y),
// seeded with the single-precision reciprocal: two iterations take the
// ~23-bit seed past FP64 precision (an IEEE FP64 division is a long
// dependent chain on this GPU).  Outside the single-precision range it falls
// back to the division.
__device__ __forceinline__ double rcp_newton(double x) {
  if (!(fabs(x) > 1e-30 && fabs(x) < 1e30)) return 1.0 / x;
  double y = (double)(1.0f / (float)x);
  y = y * fma(-x, y, 2.0);
  y = y * fma(-x, y, 2.0);
  return y;
}

// Entry (r, c) of the rotation of the unit quaternion q = (v, w) stored at q
// (x, y, z, w): R = (w^2 - v.v) I + 2 v v^T + 2 w [v]x, one formula for every
// entry, so that the lanes of a warp evaluate different entries without
// diverging.
__device__ __forceinline__ double rot_entry4(double qx, double qy, double qz, double qw, int r, int c) {
  const bool diag = r == c;
  const int k = diag ? 0 : 3 - r - c;                     // the third axis
  const double sgn = (c == (r + 1) % 3) ? -1.0 : 1.0;     // [v]x (r, c) = sgn v_k
  const double vr = r == 0 ? qx : r == 1 ? qy : qz;
  const double vc = c == 0 ? qx : c == 1 ? qy : qz;
  const double vk = k == 0 ? qx : k == 1 ? qy : qz;
  const double base = diag ? fma(qw, qw, -(qx * qx + qy * qy + qz * qz)) : 0.0;
  const double cross = diag ? 0.0 : sgn * vk;
  return fma(2.0 * vr, vc, fma(2.0 * qw, cross, base));
}
__device__ __forceinline__ double rot_entry(const double* q, int r, int c) {
  return rot_entry4(q[0], q[1], q[2], q[3], r, c);
}

// ---------------------------------------------------------------- host errors
void set_error(const char* fmt, ...);
mslam_status cuda_check(cudaError_t e, const char* what);
bool check_plan_uploaded(const mslam_plan* plan);
PlanView plan_view(const mslam_plan* plan);
// Linearisation workspace: tile partials (256-byte aligned), then the
// per-edge relative poses (16 floats each).
inline size_t lin_partials_bytes(int n_tiles) {
  return ((sizeof(float) * kAccStride * (size_t)(n_tiles > 0 ? n_tiles : 1)) + 255) & ~size_t(255);
}
// Packed-match buffer size (records of every tile, then per-tile counts).
size_t pack_bytes(int n_tiles, int lin_tile, mslam_dtype dt);
// Persistent-grid size of the linearisation launches (0 = occupancy maximum).
int plan_lin_blocks_per_sm(const mslam_plan* plan);
int plan_lin_form(const mslam_plan* plan);  // 0 block-streamed, 1 register pipeline, 2 warp-streamed
int plan_solve_form(const mslam_plan* plan);  // 0 mixed precision, 1 FP64 only
int plan_match_form(const mslam_plan* plan);  // 0 per-query window, 1 tensor-core grouped, 2 staged window
int64_t plan_edge_off(const mslam_plan* plan, int e);  // edge-pool offset of edge e (e = E: the pool size)
int64_t plan_max_mixed_bytes(const mslam_plan* plan);  // shared memory of the mixed-precision solve
int64_t plan_max_mixed_bytes_nofactor(const mslam_plan* plan);  // the same without the FP32 factor
bool plan_tracking_form(const mslam_plan* plan);  // every graph: one fixed keyframe, one frame, one edge
int64_t plan_max_mixed_elems(const mslam_plan* plan);  // elements of its assembly kernel
int plan_max_unknown_blocks(const mslam_plan* plan);   // largest non-fixed pose count of a graph
int64_t plan_solve_ws_doubles(const mslam_plan* plan);    // FP64 solve workspace of all graphs (doubles)
int plan_max_image_dim(const mslam_plan* plan);  // largest H or W of the plan's keyframes
// Host-side per-edge ranges: linearisation tiles [t0, t1), match blocks [b0, b1).
void plan_edge_tiles(const mslam_plan* plan, int e, int* t0, int* t1);
void plan_edge_mblocks(const mslam_plan* plan, int e, int* b0, int* b1);
// Largest per-graph numeric solve workspace (doubles).
int64_t plan_max_graph_doubles(const mslam_plan* plan);

// Shared-memory barriers and bulk asynchronous copies (the copy engine
// writes shared memory and counts its bytes on an mbarrier).
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Per-thread asynchronous 16-byte copy global -> shared (L2 only), grouped by
// commit.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of `parity` to complete; false after `polls`
// non-blocking polls (the plan's wait limit, about a second by default).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t polls) {
  for (uint32_t it = 0; it < polls; ++it)
    if (mbar_test_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "{\n .reg .u64 g;\n cvta.to.global.u64 g, %1;\n"
      " cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [g], %2, [%3];\n}\n" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace mslam
