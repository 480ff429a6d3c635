// (a9) Adjoint of the ray-error cost and of one Gauss-Newton step
// (project form; the paper has no backward pass).
//
// Per matched pixel the residuals are recomputed from the inputs (no stored
// Jacobians).  For the cost term c_E * E_g:
//   d rho(e)/d r = w_h(e) lambda r,  dpsi(x)/dx = (I - u u^T)/|x|,
//   d r_d/dx = u^T,  x = s R X_j + t  =>  dE/dX_j = (s R)^T dE/dx,
//   dE/dX_i[m] = -(I - v v^T) w_r r/|y| - w_d r_d v,
//   dE/dq = (w_h(e_r) e_r^2 + w_h(e_d) e_d^2) / (2 q).
// For the step term a . tau with tau = -H^-1 g: with b = H^-1 a (same
// factorisation), dL = -b^T (dH tau + dg), i.e. the gradient of
// -phi(X, q), phi = sum_pixels (J b)^T W (J tau + r), evaluated per pixel by
// a hand-written reverse sweep over the pixel's computation.
// Gathered-side contributions are scattered with atomicAdd, so the result is
// reproducible only up to FP32 summation order.
#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace mslam {

struct BwdConst {
  float inv_sr2, inv_sd2, delta, q_min, c_cost;
  int with_step;
};

// Per edge, once per call (one thread per edge): T_ij as float s R and t,
// and the relative directions beta = Ad_{T_i^-1} (b_j - b_i) and theta
// likewise for tau, so that the per-pixel kernel needs no FP64.  32 floats
// per edge: s R (9), t (3), beta (7), theta (7), padding.
constexpr int kBwdEdgeFloats = 32;
__global__ void bwd_edge_kernel(PlanView pv, const double* __restrict__ T_wc, const double* __restrict__ stepvec,
                                int with_step, float* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= pv.E) return;
  const DevEdge ed = pv.edges[e];
  float* o = out + (size_t)e * kBwdEdgeFloats;
  const Sim3d Ti = load_pose(T_wc + 8 * ed.i), Tj = load_pose(T_wc + 8 * ed.j);
  const Sim3d Tii = inverse(Ti);
  const Sim3d Tij = compose(Tii, Tj);
  double R[9];
  rot_of(Tij.q, R);
  for (int k = 0; k < 9; ++k) o[k] = (float)(Tij.s * R[k]);
  for (int k = 0; k < 3; ++k) o[9 + k] = (float)Tij.t[k];
  for (int k = 12; k < kBwdEdgeFloats; ++k) o[k] = 0.0f;
  if (with_step) {
    double A[49];
    adjoint_of(Tii, A);
    const double* bvec = stepvec;
    const double* tvec = stepvec + 7 * (size_t)pv.N;
    for (int r = 0; r < 7; ++r) {
      double sb = 0.0, stt = 0.0;
      for (int c = 0; c < 7; ++c) {
        sb += A[7 * r + c] * (bvec[7 * ed.j + c] - bvec[7 * ed.i + c]);
        stt += A[7 * r + c] * (tvec[7 * ed.j + c] - tvec[7 * ed.i + c]);
      }
      o[12 + r] = (float)sb;
      o[19 + r] = (float)stt;
    }
  }
}

struct V3 {
  float x, y, z;
};
__device__ __forceinline__ V3 v3(float a, float b, float c) { return {a, b, c}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 scl(V3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ V3 axpy(float s, V3 a, V3 b) { return {fmaf(s, a.x, b.x), fmaf(s, a.y, b.y), fmaf(s, a.z, b.z)}; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Per-match gradient of f = c (rho(e_r) + rho(e_d)) - phi with respect to
// x = T_ij X_j[n] (3), y = X_i[m] (3) and q, by a hand-written reverse sweep
// over the forward computation of the ray and distance residuals, their
// IRLS weights and, for the step term, phi = w_r (J_psi beta).(J_psi theta + r)
// + w_d (J_d beta)(J_d theta + r_d) with J_psi v = ((I - u u^T) v_t + v_w x x)/d
// and J_d v = u.v_t + d v_s (Supp. S1.2).  Huber: h = min(1, delta/e) with
// dh/d(e^2) = -h / (2 e^2) above delta, d rho/d(e^2) = h / 2.  Returns false
// for a degenerate match (no contribution).
__device__ __forceinline__ bool match_grad(V3 x, V3 y, float q, const BwdConst& bc, const float* beta,
                                           const float* theta, V3& gx, V3& gy, float& gq) {
  const float d2 = dot(x, x), dy2 = dot(y, y);
  if (!(d2 > 0.0f && dy2 > 0.0f && d2 < INFINITY && dy2 < INFINITY)) return false;
  const float d = sqrtf(d2), dy = sqrtf(dy2);
  const float id = 1.0f / d, idy = 1.0f / dy;
  const V3 u = scl(x, id), v = scl(y, idy);
  const V3 r = v3(u.x - v.x, u.y - v.y, u.z - v.z);
  const float rd = d - dy;
  const float lr = q * bc.inv_sr2, ld = q * bc.inv_sd2;
  const float rr = dot(r, r), er2 = lr * rr;
  const float rd2 = rd * rd, ed2 = ld * rd2;
  const float d2l = bc.delta * bc.delta;
  const bool lin_r = er2 > d2l, lin_d = ed2 > d2l;
  const float hr = lin_r ? bc.delta * rsqrtf(er2) : 1.0f;
  const float hd = lin_d ? bc.delta * rsqrtf(ed2) : 1.0f;
  const float wr = lr * hr, wd = ld * hd;
  // adjoints (gradients of f) of the intermediate values
  V3 gu = v3(0.f, 0.f, 0.f), gr = v3(0.f, 0.f, 0.f);
  gx = v3(0.f, 0.f, 0.f);
  float gd = 0.0f, grd = 0.0f, gwr = 0.0f, gwd = 0.0f, gid = 0.0f;
  if (bc.with_step) {
    const V3 bt = v3(beta[0], beta[1], beta[2]), bw = v3(beta[3], beta[4], beta[5]);
    const V3 tt = v3(theta[0], theta[1], theta[2]), tw = v3(theta[3], theta[4], theta[5]);
    const float sb = dot(u, bt), st_ = dot(u, tt);
    const V3 Pb = add(axpy(-sb, u, bt), cross(bw, x)), Pt = add(axpy(-st_, u, tt), cross(tw, x));
    const V3 A = scl(Pb, id), B = add(scl(Pt, id), r);
    const float a = sb + d * beta[6], b = st_ + d * theta[6] + rd;
    const float AB = dot(A, B), ab = a * b;
    // phi enters f with coefficient -1
    gwr = -AB;
    gwd = -ab;
    const V3 gA = scl(B, -wr), gB = scl(A, -wr);
    const float ga = -wd * b, gb = -wd * a;
    gr = gB;   // B = J_psi theta + r
    grd = gb;  // b = J_d theta + r_d
    // J_psi beta = Pb id and J_psi theta = Pt id (adjoints gA, gB)
    gid += dot(gA, Pb) + dot(gB, Pt);
    const V3 gPb = scl(gA, id), gPt = scl(gB, id);
    // P = v_t - u (u.v_t) + v_w x x
    gu = axpy(-sb, gPb, axpy(-st_, gPt, gu));
    const float gsb = -dot(gPb, u), gst = -dot(gPt, u);
    gx = add(gx, add(cross(gPb, bw), cross(gPt, tw)));
    // s = u.v_t;  J_d v = u.v_t + d v_s (adjoints ga, gb)
    gu = axpy(gsb + ga, bt, axpy(gst + gb, tt, gu));
    gd += ga * beta[6] + gb * theta[6];
  }
  // weights w = lambda h and costs rho; d rho / d(e^2) = h / 2
  float ger2 = 0.5f * hr * bc.c_cost, ged2 = 0.5f * hd * bc.c_cost;
  const float glr0 = gwr * hr, gld0 = gwd * hd;
  const float ghr = gwr * lr, ghd = gwd * ld;
  if (lin_r) ger2 += ghr * (-0.5f * hr / er2);
  if (lin_d) ged2 += ghd * (-0.5f * hd / ed2);
  const float glr = glr0 + ger2 * rr, gld = gld0 + ged2 * rd2;
  gr = axpy(2.0f * ger2 * lr, r, gr);
  grd += 2.0f * ged2 * ld * rd;
  gq = glr * bc.inv_sr2 + gld * bc.inv_sd2;
  // r = u - v, r_d = d - dy
  gu = add(gu, gr);
  const V3 gv = scl(gr, -1.0f);
  gd += grd;
  const float gdy = -grd;
  // u = x id, id = 1/d, d = sqrt(x.x)
  gx = axpy(id, gu, gx);
  gid += dot(gu, x);
  gd += -gid * id * id;
  gx = axpy(gd * id, x, gx);
  // v = y idy, idy = 1/dy, dy = sqrt(y.y)
  gy = scl(gv, idy);
  const float gidy = dot(gv, y);
  const float gdyt = gdy - gidy * idy * idy;
  gy = axpy(gdyt * idy, y, gy);
  return true;
}

// kPose: also sum, per edge, the gradient with respect to a left
// perturbation xi of T_ij (x -> Exp(xi) x, dx/dxi = [I, -[x]x, x]):
// Xi_e = sum over the edge's matches of (g_x, x cross g_x, x . g_x), added
// into xi_out [E, 7] (FP64).
constexpr int kBwdU = 4;
template <typename T, bool kPose>
__global__ void __launch_bounds__(256) bwd_kernel(PlanView pv, BwdConst bc, const float* __restrict__ edge_data,
                                                  const T* __restrict__ X, const int32_t* __restrict__ idx,
                                                  const T* __restrict__ q, float* __restrict__ dX,
                                                  float* __restrict__ dq, double* __restrict__ xi_out) {
  __shared__ float s_xi[256 / 32][7];
  for (int tile = blockIdx.x; tile < pv.n_tiles; tile += gridDim.x) {
    float xi[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const DevTile tl = pv.tiles[tile];
    const DevEdge ed = pv.edges[tl.edge];
    const float* eg = edge_data + (size_t)tl.edge * kBwdEdgeFloats;
    float sR[9], st[3], sbeta[7], stheta[7];
#pragma unroll
    for (int k = 0; k < 9; ++k) sR[k] = __ldg(eg + k);
#pragma unroll
    for (int k = 0; k < 3; ++k) st[k] = __ldg(eg + 9 + k);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      sbeta[k] = __ldg(eg + 12 + k);
      stheta[k] = __ldg(eg + 19 + k);
    }
    // kBwdU pixels per thread and round: their loads (the match index, then
    // the confidence and both canonical points) are all issued before the
    // first pixel's reverse sweep
    for (int n0 = tl.begin + threadIdx.x; n0 < tl.end; n0 += blockDim.x * kBwdU) {
      int mv[kBwdU];
      float qv[kBwdU];
      float3 Xjv[kBwdU], yvv[kBwdU];
#pragma unroll
      for (int u = 0; u < kBwdU; ++u) {
        const int n = n0 + u * blockDim.x;
        mv[u] = n < tl.end ? idx[ed.off_e + n] : -1;
      }
#pragma unroll
      for (int u = 0; u < kBwdU; ++u) {
        const int n = n0 + u * blockDim.x;
        qv[u] = 0.0f;
        Xjv[u] = yvv[u] = make_float3(0.0f, 0.0f, 0.0f);
        if (mv[u] >= 0) {
          qv[u] = ldf(q + ed.off_e + n);
          Xjv[u] = ld3(X + 3 * ed.off_j, n);
          yvv[u] = ld3(X + 3 * ed.off_i, mv[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < kBwdU; ++u) {
        const int n = n0 + u * blockDim.x, m = mv[u];
        if (m < 0) continue;
        const float qq = qv[u];
        if (!(qq > bc.q_min)) continue;
        const float3 Xj = Xjv[u];
        const float3 yv = yvv[u];
        const V3 x = v3(sR[0] * Xj.x + sR[1] * Xj.y + sR[2] * Xj.z + st[0],
                        sR[3] * Xj.x + sR[4] * Xj.y + sR[5] * Xj.z + st[1],
                        sR[6] * Xj.x + sR[7] * Xj.y + sR[8] * Xj.z + st[2]);
        V3 gx, gy;
        float gq;
        if (!match_grad(x, v3(yv.x, yv.y, yv.z), qq, bc, sbeta, stheta, gx, gy, gq)) continue;
        // dL/dX_j = (s R)^T dL/dx
        float* dXj = dX + 3 * (ed.off_j + n);
        atomicAdd(dXj + 0, sR[0] * gx.x + sR[3] * gx.y + sR[6] * gx.z);
        atomicAdd(dXj + 1, sR[1] * gx.x + sR[4] * gx.y + sR[7] * gx.z);
        atomicAdd(dXj + 2, sR[2] * gx.x + sR[5] * gx.y + sR[8] * gx.z);
        float* dXi = dX + 3 * (ed.off_i + m);
        atomicAdd(dXi + 0, gy.x);
        atomicAdd(dXi + 1, gy.y);
        atomicAdd(dXi + 2, gy.z);
        dq[ed.off_e + n] = gq;
        if (kPose) {
          const V3 xg = cross(x, gx);
          xi[0] += gx.x;
          xi[1] += gx.y;
          xi[2] += gx.z;
          xi[3] += xg.x;
          xi[4] += xg.y;
          xi[5] += xg.z;
          xi[6] += dot(x, gx);
        }
      }
    }
    if (kPose) {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        float v = xi[k];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) s_xi[warp][k] = v;
      }
      __syncthreads();
      if (threadIdx.x < 7) {
        double t = 0.0;
        for (int w = 0; w < 256 / 32; ++w) t += (double)s_xi[w][threadIdx.x];
        atomicAdd(xi_out + 7 * (size_t)tl.edge + threadIdx.x, t);
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- poses
// Gradients with respect to the poses use the left perturbation
// T -> Exp(eta) T of each pose; at the C ABI they are given in the [N, 8]
// embedding (t, q, s) as the gradient G with J8^T G = dL/deta and no
// component along q (the quaternion's norm direction), J8 = d(t, q, s)/d eta:
//   dt = rho + phi x t + sigma t,  dq = (phi / 2, 0) (x) q,  ds = sigma s.
// Hence dL/deta = (G_t, t x G_t + Q^T G_q, t . G_t + s G_s) with
// Q = 1/2 [[q_w I - [q_v]x], [-q_v^T]], and back G = (g_rho,
// 4 Q (g_phi - t x g_rho), (g_sigma - t . g_rho) / s) ([2Q, q] is orthogonal).
__device__ void tangent_of_embedding(const Sim3d& T, const double* G, double g[7]) {
  const double* t = T.t;
  const double qx = T.q[0], qy = T.q[1], qz = T.q[2], qw = T.q[3];
  const double Gt0 = G[0], Gt1 = G[1], Gt2 = G[2];
  const double a = G[3], b = G[4], c = G[5], d = G[6];
  // Q^T G_q = 1/2 [(q_w I + [q_v]x) G_qv - q_v G_qw]
  const double qt0 = 0.5 * (qw * a + (qy * c - qz * b) - qx * d);
  const double qt1 = 0.5 * (qw * b + (qz * a - qx * c) - qy * d);
  const double qt2 = 0.5 * (qw * c + (qx * b - qy * a) - qz * d);
  g[0] = Gt0;
  g[1] = Gt1;
  g[2] = Gt2;
  g[3] = (t[1] * Gt2 - t[2] * Gt1) + qt0;
  g[4] = (t[2] * Gt0 - t[0] * Gt2) + qt1;
  g[5] = (t[0] * Gt1 - t[1] * Gt0) + qt2;
  g[6] = (t[0] * Gt0 + t[1] * Gt1 + t[2] * Gt2) + T.s * G[7];
}

__device__ void embedding_of_tangent(const Sim3d& T, const double g[7], double* G) {
  const double* t = T.t;
  const double qx = T.q[0], qy = T.q[1], qz = T.q[2], qw = T.q[3];
  // h = g_phi - t x g_rho
  const double h0 = g[3] - (t[1] * g[2] - t[2] * g[1]);
  const double h1 = g[4] - (t[2] * g[0] - t[0] * g[2]);
  const double h2 = g[5] - (t[0] * g[1] - t[1] * g[0]);
  // 4 Q h = 2 [(q_w I - [q_v]x) h; -q_v . h]
  G[0] = g[0];
  G[1] = g[1];
  G[2] = g[2];
  G[3] = 2.0 * (qw * h0 - (qy * h2 - qz * h1));
  G[4] = 2.0 * (qw * h1 - (qz * h0 - qx * h2));
  G[5] = 2.0 * (qw * h2 - (qx * h1 - qy * h0));
  G[6] = -2.0 * (qx * h0 + qy * h1 + qz * h2);
  G[7] = (g[6] - (t[0] * g[0] + t[1] * g[1] + t[2] * g[2])) / T.s;
}

// v^T ad(w) for the Lie bracket of sim(3), tau = (rho, phi, sigma):
// ad(w) = [[ [w_phi]x + w_sigma I, [w_rho]x, -w_rho ], [0, [w_phi]x, 0], [0, 0, 0]],
// so out = ad(w)^T v.
__device__ void ad_transpose_times(const double* w, const double* v, double out[7]) {
  const double r0 = w[0], r1 = w[1], r2 = w[2], p0 = w[3], p1 = w[4], p2 = w[5], sg = w[6];
  const double a0 = v[0], a1 = v[1], a2 = v[2], b0 = v[3], b1 = v[4], b2 = v[5];
  // ([w_phi]x)^T a = -w_phi x a = a x w_phi
  out[0] = (a1 * p2 - a2 * p1) + sg * a0;
  out[1] = (a2 * p0 - a0 * p2) + sg * a1;
  out[2] = (a0 * p1 - a1 * p0) + sg * a2;
  // ([w_rho]x)^T a + ([w_phi]x)^T b = a x w_rho + b x w_phi
  out[3] = (a1 * r2 - a2 * r1) + (b1 * p2 - b2 * p1);
  out[4] = (a2 * r0 - a0 * r2) + (b2 * p0 - b0 * p2);
  out[5] = (a0 * r1 - a1 * r0) + (b0 * p1 - b1 * p0);
  out[6] = -(r0 * a0 + r1 * a1 + r2 * a2);
}

// Per pose, before the solve for b: the updated pose T' = Exp(tau) T, its
// gradient dL/deta' from the embedding gradient G' (or zero), the right-hand
// side a = dL_dtau + J_l(tau)^T dL/deta' of the step term (J_l(tau) =
// sum_k ad(tau)^k / (k+1)! the left Jacobian, Exp(tau + d) = Exp(J_l d)
// Exp(tau)), and the direct part Ad_{Exp(tau)}^T dL/deta' of dL/deta
// (T' = Exp(tau) Exp(eta) T = Exp(Ad_{Exp(tau)} eta) T'), which starts the
// pose accumulator.
__global__ void bwd_pose_in_kernel(int N, const double* __restrict__ T_wc, const double* __restrict__ tau,
                                   const double* __restrict__ dL_dTnew, const double* __restrict__ dL_dtau,
                                   double* __restrict__ a_out, double* __restrict__ acc) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double tk[7], gn[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int c = 0; c < 7; ++c) tk[c] = tau[7 * k + c];
  if (dL_dTnew) {
    const Sim3d Tn = compose(sim3_exp(tk), load_pose(T_wc + 8 * k));
    tangent_of_embedding(Tn, dL_dTnew + 8 * k, gn);
  }
  // J_l(tau)^T gn = sum_k w_k, w_0 = gn, w_k = ad(tau)^T w_{k-1} / (k + 1)
  double a[7], w[7];
  for (int c = 0; c < 7; ++c) a[c] = w[c] = gn[c];
  for (int it = 1; it < 60; ++it) {
    double nw[7], nrm = 0.0, tot = 0.0;
    ad_transpose_times(tk, w, nw);
    const double f = 1.0 / (double)(it + 1);
    for (int c = 0; c < 7; ++c) {
      w[c] = nw[c] * f;
      a[c] += w[c];
      nrm = fmax(nrm, fabs(w[c]));
      tot = fmax(tot, fabs(a[c]));
    }
    if (nrm <= 1e-18 * tot || nrm == 0.0) break;
  }
  for (int c = 0; c < 7; ++c) a_out[7 * k + c] = a[c] + (dL_dtau ? dL_dtau[7 * k + c] : 0.0);
  double Ad[49];
  adjoint_of(sim3_exp(tk), Ad);
  for (int c = 0; c < 7; ++c) {
    double sum = 0.0;
    for (int r = 0; r < 7; ++r) sum += Ad[7 * r + c] * gn[r];
    acc[7 * k + c] = sum;
  }
}

// Per edge e = (i, j), after the per-match sweep: x = T_ij X_j depends on
// the poses through xi = Ad_{T_i^-1} (eta_j - eta_i), so dL/deta_j +=
// Ad^T Xi_e and dL/deta_i -= Ad^T Xi_e.  The step term phi also depends on
// T_i through Ad in beta = Ad (b_j - b_i) and theta = Ad (tau_j - tau_i)
// (Ad_{T_i^-1} -> Ad (I - ad(eta_i))); with sum dphi/dbeta = H_rel theta +
// g_rel, sum dphi/dtheta = H_rel beta and Ad^T H_rel Ad = H_jj, Ad^T g_rel =
// g_j (the edge's 14 x 14 block and gradient): dphi/deta_i =
// ad(db)^T (H_jj dtau + g_j) + ad(dtau)^T H_jj db, entering L with sign -1.
__global__ void bwd_pose_edge_kernel(PlanView pv, const double* __restrict__ T_wc, const double* __restrict__ bvec,
                                     const double* __restrict__ tvec, const float* __restrict__ H14,
                                     const float* __restrict__ g14, const double* __restrict__ xi,
                                     int with_step, double* __restrict__ acc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= pv.E) return;
  const DevEdge ed = pv.edges[e];
  double Ad[49];
  adjoint_of(inverse(load_pose(T_wc + 8 * ed.i)), Ad);
  double cj[7];
  for (int c = 0; c < 7; ++c) {
    double sum = 0.0;
    for (int r = 0; r < 7; ++r) sum += Ad[7 * r + c] * xi[7 * (size_t)e + r];
    cj[c] = sum;
  }
  double ei[7] = {0, 0, 0, 0, 0, 0, 0};
  if (with_step) {
    double db[7], dt[7], v1[7], v2[7], o1[7], o2[7];
    for (int c = 0; c < 7; ++c) {
      db[c] = bvec[7 * ed.j + c] - bvec[7 * ed.i + c];
      dt[c] = tvec[7 * ed.j + c] - tvec[7 * ed.i + c];
    }
    const float* Hb = H14 + 196 * (size_t)e;
    for (int r = 0; r < 7; ++r) {
      double s1 = (double)g14[14 * (size_t)e + 7 + r], s2 = 0.0;
      for (int c = 0; c < 7; ++c) {
        const double h = (double)Hb[14 * (7 + r) + 7 + c];
        s1 += h * dt[c];
        s2 += h * db[c];
      }
      v1[r] = s1;
      v2[r] = s2;
    }
    ad_transpose_times(db, v1, o1);
    ad_transpose_times(dt, v2, o2);
    for (int c = 0; c < 7; ++c) ei[c] = o1[c] + o2[c];
  }
  for (int c = 0; c < 7; ++c) {
    atomicAdd(acc + 7 * ed.j + c, cj[c]);
    atomicAdd(acc + 7 * ed.i + c, -cj[c] - ei[c]);
  }
}

// Per pose: the accumulated dL/deta in the [N, 8] embedding of T_wc.
__global__ void bwd_pose_out_kernel(int N, const double* __restrict__ T_wc, const double* __restrict__ acc,
                                    double* __restrict__ dL_dT) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  embedding_of_tangent(load_pose(T_wc + 8 * k), acc + 7 * k, dL_dT + 8 * k);
}

// b = H^-1 a for every graph using the factorisation (blocks and reciprocal
// pivots) that a preceding factor-only solve left in the workspace (one CTA
// per graph): forward and back substitution by elimination levels, one
// warp per column (as in the solve kernel).
__global__ void __launch_bounds__(kSolveThreads) bwd_rhs_kernel(PlanView pv, const double* __restrict__ a,
                                                                double* __restrict__ bout,
                                                                const int32_t* __restrict__ dev_status,
                                                                double* __restrict__ ws,
                                                                const int32_t* __restrict__ skip) {
  const int g = blockIdx.x;
  if (skip && skip[g]) return;  // solved by the mixed-precision kernel
  const DevGraph G = pv.graphs[g];
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
  const int m = G.m;
  if (tid < 7) bout[7 * G.gauge + tid] = 0.0;
  if (dev_status[g] > 1 || m == 0) return;
  const int32_t* I = pv.ints;
  const int32_t* pose_of_pos = I + G.off_pose;
  const int32_t* col_ptr = I + G.off_col;
  const int32_t* colent = I + G.off_colent;
  const int32_t* lev_ptr = I + G.off_lev;
  const int32_t* lev_cols = I + G.off_levcols;
  const int32_t* rsptr = I + G.off_rsptr;
  const int32_t* rs = I + G.off_rs;
  const double* L = ws + G.ws_off;
  double* rhs = ws + G.ws_off + (size_t)G.n_blocks * 49;
  const double* invd = rhs + 14 * (size_t)m;  // after the right-hand side and the assembled diagonal
  for (int t = tid; t < 7 * m; t += nth) rhs[t] = a[7 * __ldg(pose_of_pos + t / 7) + t % 7];
  __syncthreads();
  for (int l = 0; l < G.n_levels; ++l) {
    const int q0 = __ldg(lev_ptr + l), q1 = __ldg(lev_ptr + l + 1);
    for (int qi = q0 + warp; qi < q1; qi += nwarps) {
      const int p = __ldg(lev_cols + qi);
      double s = 0.0;
      if (lane < 7) {
        double ps[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int k = __ldg(rsptr + p); k < __ldg(rsptr + p + 1); ++k) {
          const double* Lpc = L + 49 * (size_t)__ldg(rs + 2 * k + 1) + 7 * lane;
          const double* yc = rhs + 7 * __ldg(rs + 2 * k);
#pragma unroll
          for (int kk = 0; kk < 7; ++kk) ps[kk] = fma(Lpc[kk], yc[kk], ps[kk]);
        }
        s = rhs[7 * p + lane] - (((ps[0] + ps[1]) + (ps[2] + ps[3])) + ((ps[4] + ps[5]) + ps[6]));
      }
      const double* D = L + 49 * (size_t)p;
      double out = 0.0;
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        const double yj = __shfl_sync(0xffffffffu, s, j) * invd[7 * p + j];
        if (lane == j) out = yj;
        if (lane > j && lane < 7) s = fma(-D[7 * lane + j], yj, s);
      }
      if (lane < 7) rhs[7 * p + lane] = out;
      __syncwarp();
    }
    __syncthreads();
  }
  for (int l = G.n_levels - 1; l >= 0; --l) {
    const int q0 = __ldg(lev_ptr + l), q1 = __ldg(lev_ptr + l + 1);
    for (int qi = q0 + warp; qi < q1; qi += nwarps) {
      const int p = __ldg(lev_cols + qi);
      const double* D = L + 49 * (size_t)p;
      double s = 0.0;
      if (lane < 7) {
        double ps[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int ent = __ldg(col_ptr + p); ent < __ldg(col_ptr + p + 1); ++ent) {
          const double* Lr = L + 49 * (size_t)__ldg(colent + 2 * ent + 1);
          const double* xr = rhs + 7 * __ldg(colent + 2 * ent);
#pragma unroll
          for (int k = 0; k < 7; ++k) ps[k] = fma(Lr[7 * k + lane], xr[k], ps[k]);
        }
        s = rhs[7 * p + lane] - (((ps[0] + ps[1]) + (ps[2] + ps[3])) + ((ps[4] + ps[5]) + ps[6]));
      }
      double xl = 0.0;
#pragma unroll
      for (int k = 6; k >= 0; --k) {
        const double xk = __shfl_sync(0xffffffffu, s, k) * invd[7 * p + k];
        if (lane == k) xl = xk;
        if (lane < k) s = fma(-D[7 * k + lane], xk, s);
      }
      if (lane < 7) rhs[7 * p + lane] = xl;
      __syncwarp();
    }
    __syncthreads();
  }
  for (int t = tid; t < 7 * m; t += nth) bout[7 * __ldg(pose_of_pos + t / 7) + t % 7] = rhs[t];
}

}  // namespace mslam

using namespace mslam;

extern mslam_status mslam_bwd_solve_tau(const mslam_plan* plan, const float* H_blocks, const float* g_blocks,
                                        double* tau, int32_t* dev_status, double* ws, cudaStream_t s,
                                        bool* mixed_used);
extern mslam_status mslam_bwd_solve_rhs(const mslam_plan* plan, const float* H_blocks, const float* g_blocks,
                                        const double* rhs, double* x, double* tau, int32_t* dev_status,
                                        double* ws, int32_t* handled2, cudaStream_t s);
// Both adjoint entry points: the cost and step terms with respect to X and q
// and, when dL_dT is given, the poses (with the retraction T' = Exp(tau) T
// and an upstream gradient dL_dTnew on T').
static mslam_status step_backward(const char* who, const mslam_params* p, const mslam_plan* plan, mslam_dtype dt,
                                  const double* T_wc, const void* X_canon, const int32_t* idx, const void* q,
                                  const float* H_blocks, const float* g_blocks, const double* dL_dTnew,
                                  const double* dL_dtau, double dL_dcost, float* dL_dX, float* dL_dq, double* dL_dT,
                                  int32_t* dev_status, void* workspace, size_t ws_bytes, void* stream) {
  if (!p || !check_plan_uploaded(plan)) {
    if (!p) set_error("params is NULL");
    return MSLAM_ERR_ARG;
  }
  if (dt != MSLAM_F32 && dt != MSLAM_F16) {
    set_error("unsupported dtype %d", (int)dt);
    return MSLAM_ERR_ARG;
  }
  if (p->residual != MSLAM_RES_RAY) {
    set_error("%s: the adjoint covers the ray-error cost only (residual = MSLAM_RES_RAY)", who);
    return MSLAM_ERR_ARG;
  }
  if (!T_wc || !X_canon || !idx || !q || !dL_dX || !dL_dq || !workspace) {
    set_error("%s: NULL device pointer", who);
    return MSLAM_ERR_ARG;
  }
  const bool with_step = dL_dtau || dL_dTnew;
  if ((with_step || dL_dT) && (!H_blocks || !g_blocks || !dev_status)) {
    set_error("%s: the step and pose terms need H_blocks, g_blocks and dev_status", who);
    return MSLAM_ERR_ARG;
  }
  if (ws_bytes < mslam_workspace_bytes(plan, MSLAM_OP_BACKWARD) || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    set_error("%s: workspace smaller than %zu bytes or not 256-byte aligned", who,
              mslam_workspace_bytes(plan, MSLAM_OP_BACKWARD));
    return MSLAM_ERR_ARG;
  }
  const PlanView pv = plan_view(plan);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mslam_status st = cuda_check(cudaMemsetAsync(dL_dX, 0, sizeof(float) * 3 * mslam_plan_kf_pixels(plan), s),
                               "gn_backward memset");
  if (st != MSLAM_OK) return st;
  st = cuda_check(cudaMemsetAsync(dL_dq, 0, sizeof(float) * mslam_plan_edge_pixels(plan), s), "gn_backward memset");
  if (st != MSLAM_OK) return st;
  if (dL_dT) {
    st = cuda_check(cudaMemsetAsync(dL_dT, 0, sizeof(double) * 8 * (size_t)pv.N, s), "gn_backward memset");
    if (st != MSLAM_OK) return st;
  }
  if (pv.E == 0) return MSLAM_OK;
  // workspace: the solve's, b and tau [N, 7] each, per-edge data (32 floats
  // per edge), then for the pose term a [N, 7], the pose accumulator [N, 7]
  // and Xi [E, 7] (FP64)
  double* ws = static_cast<double*>(workspace);
  const size_t solve_doubles = mslam_workspace_bytes(plan, MSLAM_OP_SOLVE) / sizeof(double);
  double* stepvec = ws + solve_doubles;  // [N,7] b then [N,7] tau
  double* bvec = stepvec;
  double* tvec = stepvec + 7 * (size_t)pv.N;
  float* edge_data = reinterpret_cast<float*>(stepvec + 14 * (size_t)pv.N);
  double* pose_ws = reinterpret_cast<double*>(reinterpret_cast<char*>(edge_data) +
                                              ((sizeof(float) * 32 * (size_t)std::max(pv.E, 1) + 255) & ~size_t(255)));
  double* a_tot = pose_ws;
  double* acc = pose_ws + 7 * (size_t)pv.N;
  double* xi = pose_ws + 14 * (size_t)pv.N;
  int32_t* handled2 = reinterpret_cast<int32_t*>(pose_ws + 14 * (size_t)pv.N + 7 * (size_t)std::max(pv.E, 1));
  bool mixed = false;
  if (with_step || dL_dT) {
    // tau = -H^-1 g without touching the poses (the FP32 factor with FP64
    // refinement where it applies, kept for b; the FP64 factor elsewhere)
    st = mslam_bwd_solve_tau(plan, H_blocks, g_blocks, tvec, dev_status, ws, s, &mixed);
    if (st != MSLAM_OK) return st;
  }
  if (dL_dT) {
    st = cuda_check(cudaMemsetAsync(xi, 0, sizeof(double) * 7 * (size_t)pv.E, s), "gn_backward memset");
    if (st != MSLAM_OK) return st;
    bwd_pose_in_kernel<<<(pv.N + 63) / 64, 64, 0, s>>>(pv.N, T_wc, tvec, dL_dTnew, dL_dtau, a_tot, acc);
  }
  if (with_step) {
    // b = H^-1 a with a = dL_dtau (+ the retraction's J_l^T dL/dT' with poses):
    // the kept FP32 factor with FP64 refinement, then the FP64 substitution
    // for the graphs it did not solve
    const double* a = dL_dT ? a_tot : dL_dtau;
    if (mixed) {
      st = mslam_bwd_solve_rhs(plan, H_blocks, g_blocks, a, bvec, tvec, dev_status, ws, handled2, s);
      if (st != MSLAM_OK) return st;
    }
    bwd_rhs_kernel<<<pv.G, kSolveThreads, 0, s>>>(pv, a, bvec, dev_status, ws, mixed ? handled2 : nullptr);
  }
  BwdConst bc;
  bc.inv_sr2 = 1.0f / (p->sigma_ray * p->sigma_ray);
  bc.inv_sd2 = 1.0f / (p->sigma_dist * p->sigma_dist);
  bc.delta = p->huber_delta;
  bc.q_min = p->q_min;
  bc.c_cost = (float)dL_dcost;
  bc.with_step = with_step ? 1 : 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  bwd_edge_kernel<<<(pv.E + 63) / 64, 64, 0, s>>>(pv, T_wc, stepvec, with_step ? 1 : 0, edge_data);
  const int grid = std::min(pv.n_tiles, std::max(1, sms) * 8);
  auto sweep = [&](auto kpose) {
    constexpr bool kP = decltype(kpose)::value;
    if (dt == MSLAM_F32)
      bwd_kernel<float, kP><<<grid, 256, 0, s>>>(pv, bc, edge_data, static_cast<const float*>(X_canon), idx,
                                                 static_cast<const float*>(q), dL_dX, dL_dq, xi);
    else
      bwd_kernel<__half, kP><<<grid, 256, 0, s>>>(pv, bc, edge_data, static_cast<const __half*>(X_canon), idx,
                                                  static_cast<const __half*>(q), dL_dX, dL_dq, xi);
  };
  if (dL_dT) {
    sweep(std::true_type{});
    bwd_pose_edge_kernel<<<(pv.E + 63) / 64, 64, 0, s>>>(pv, T_wc, bvec, tvec, H_blocks, g_blocks, xi,
                                                         with_step ? 1 : 0, acc);
    bwd_pose_out_kernel<<<(pv.N + 63) / 64, 64, 0, s>>>(pv.N, T_wc, acc, dL_dT);
  } else {
    sweep(std::false_type{});
  }
  return cuda_check(cudaGetLastError(), "gn_backward launch");
}

extern "C" mslam_status mslam_gn_backward(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt,
                                          const double* T_wc, const void* X_canon, const int32_t* idx,
                                          const void* q, const float* H_blocks, const float* g_blocks,
                                          const double* dL_dtau, double dL_dcost, float* dL_dX, float* dL_dq,
                                          int32_t* dev_status, void* workspace, size_t ws_bytes, void* stream) {
  return step_backward("gn_backward", p, plan, dt, T_wc, X_canon, idx, q, H_blocks, g_blocks, nullptr, dL_dtau,
                       dL_dcost, dL_dX, dL_dq, nullptr, dev_status, workspace, ws_bytes, stream);
}

extern "C" mslam_status mslam_gn_step_backward(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt,
                                               const double* T_wc, const void* X_canon, const int32_t* idx,
                                               const void* q, const float* H_blocks, const float* g_blocks,
                                               const double* dL_dTnew, const double* dL_dtau, double dL_dcost,
                                               float* dL_dX, float* dL_dq, double* dL_dT, int32_t* dev_status,
                                               void* workspace, size_t ws_bytes, void* stream) {
  if (!dL_dT) {
    set_error("gn_step_backward: dL_dT is NULL (use mslam_gn_backward without the pose term)");
    return MSLAM_ERR_ARG;
  }
  return step_backward("gn_step_backward", p, plan, dt, T_wc, X_canon, idx, q, H_blocks, g_blocks, dL_dTnew,
                       dL_dtau, dL_dcost, dL_dX, dL_dq, dL_dT, dev_status, workspace, ws_bytes, stream);
}
