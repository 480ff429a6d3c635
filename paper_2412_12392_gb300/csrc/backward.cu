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

template <typename T>
__global__ void __launch_bounds__(256) bwd_kernel(PlanView pv, BwdConst bc, const float* __restrict__ edge_data,
                                                  const T* __restrict__ X, const int32_t* __restrict__ idx,
                                                  const T* __restrict__ q, float* __restrict__ dX,
                                                  float* __restrict__ dq) {
  for (int tile = blockIdx.x; tile < pv.n_tiles; tile += gridDim.x) {
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
    for (int n = tl.begin + threadIdx.x; n < tl.end; n += blockDim.x) {
      const int m = idx[ed.off_e + n];
      if (m < 0) continue;
      const float qq = ldf(q + ed.off_e + n);
      if (!(qq > bc.q_min)) continue;
      const float3 Xj = ld3(X + 3 * ed.off_j, n);
      const float3 yv = ld3(X + 3 * ed.off_i, m);
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
    }
  }
}

// b = H^-1 a for every graph using the factorisation (blocks and reciprocal
// pivots) that a preceding factor-only solve left in the workspace (one CTA
// per graph): forward and back substitution by elimination levels, one
// warp per column (as in the solve kernel).
__global__ void __launch_bounds__(kSolveThreads) bwd_rhs_kernel(PlanView pv, const double* __restrict__ a,
                                                                double* __restrict__ bout,
                                                                const int32_t* __restrict__ dev_status,
                                                                double* __restrict__ ws) {
  const int g = blockIdx.x;
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

extern mslam_status mslam_factor_only(const mslam_plan* plan, const float* H_blocks, const float* g_blocks,
                                      double* tau, int32_t* dev_status, double* ws, cudaStream_t s);

extern "C" mslam_status mslam_gn_backward(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt,
                                          const double* T_wc, const void* X_canon, const int32_t* idx,
                                          const void* q, const float* H_blocks, const float* g_blocks,
                                          const double* dL_dtau, double dL_dcost, float* dL_dX, float* dL_dq,
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
    set_error("gn_backward: the adjoint covers the ray-error cost only (residual = MSLAM_RES_RAY)");
    return MSLAM_ERR_ARG;
  }
  if (!T_wc || !X_canon || !idx || !q || !dL_dX || !dL_dq || !workspace) {
    set_error("gn_backward: NULL device pointer");
    return MSLAM_ERR_ARG;
  }
  if (dL_dtau && (!H_blocks || !g_blocks || !dev_status)) {
    set_error("gn_backward: the step term needs H_blocks, g_blocks and dev_status");
    return MSLAM_ERR_ARG;
  }
  if (ws_bytes < mslam_workspace_bytes(plan, MSLAM_OP_BACKWARD) || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    set_error("gn_backward: workspace smaller than %zu bytes or not 256-byte aligned",
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
  if (pv.E == 0) return MSLAM_OK;
  double* ws = static_cast<double*>(workspace);
  const size_t solve_doubles = mslam_workspace_bytes(plan, MSLAM_OP_SOLVE) / sizeof(double);
  double* stepvec = ws + solve_doubles;  // [N,7] b then [N,7] tau
  if (dL_dtau) {
    // factor H (and compute tau) without touching the poses, then b = H^-1 a
    st = mslam_factor_only(plan, H_blocks, g_blocks, stepvec + 7 * (size_t)pv.N, dev_status, ws, s);
    if (st != MSLAM_OK) return st;
    bwd_rhs_kernel<<<pv.G, kSolveThreads, 0, s>>>(pv, dL_dtau, stepvec, dev_status, ws);
  }
  BwdConst bc;
  bc.inv_sr2 = 1.0f / (p->sigma_ray * p->sigma_ray);
  bc.inv_sd2 = 1.0f / (p->sigma_dist * p->sigma_dist);
  bc.delta = p->huber_delta;
  bc.q_min = p->q_min;
  bc.c_cost = (float)dL_dcost;
  bc.with_step = dL_dtau ? 1 : 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // per-edge data after the two pose vectors (b and tau)
  float* edge_data = reinterpret_cast<float*>(stepvec + 14 * (size_t)pv.N);
  bwd_edge_kernel<<<(pv.E + 63) / 64, 64, 0, s>>>(pv, T_wc, stepvec, dL_dtau ? 1 : 0, edge_data);
  const int grid = std::min(pv.n_tiles, std::max(1, sms) * 8);
  if (dt == MSLAM_F32)
    bwd_kernel<float><<<grid, 256, 0, s>>>(pv, bc, edge_data, static_cast<const float*>(X_canon), idx,
                                           static_cast<const float*>(q), dL_dX, dL_dq);
  else
    bwd_kernel<__half><<<grid, 256, 0, s>>>(pv, bc, edge_data, static_cast<const __half*>(X_canon), idx,
                                            static_cast<const __half*>(q), dL_dX, dL_dq);
  return cuda_check(cudaGetLastError(), "gn_backward launch");
}
