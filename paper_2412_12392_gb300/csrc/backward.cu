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
// forward-mode dual numbers over the pixel's seven inputs (x, y, q).
// Gathered-side contributions are scattered with atomicAdd, so the result is
// reproducible only up to FP32 summation order.
#include <algorithm>

#include "common.cuh"

namespace mslam {

struct BwdConst {
  float inv_sr2, inv_sd2, delta, q_min, c_cost;
  int with_step;
};

// value plus 7 tangents (x0, x1, x2, y0, y1, y2, q)
struct Dual {
  float v;
  float d[7];
};

__device__ __forceinline__ Dual dconst(float v) {
  Dual r;
  r.v = v;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = 0.0f;
  return r;
}
__device__ __forceinline__ Dual dvar(float v, int k) {
  Dual r = dconst(v);
  r.d[k] = 1.0f;
  return r;
}
__device__ __forceinline__ Dual operator+(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
__device__ __forceinline__ Dual operator-(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
__device__ __forceinline__ Dual operator*(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
__device__ __forceinline__ Dual operator*(float s, const Dual& a) {
  Dual r;
  r.v = s * a.v;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = s * a.d[k];
  return r;
}
__device__ __forceinline__ Dual dinv(const Dual& a) {
  Dual r;
  r.v = 1.0f / a.v;
  const float g = -r.v * r.v;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = g * a.d[k];
  return r;
}
__device__ __forceinline__ Dual dsqrt(const Dual& a) {
  Dual r;
  r.v = sqrtf(a.v);
  const float g = r.v > 0.0f ? 0.5f / r.v : 0.0f;
#pragma unroll
  for (int k = 0; k < 7; ++k) r.d[k] = g * a.d[k];
  return r;
}

// Huber IRLS weight lambda * w_h(e) with e = sqrt(lambda * s2) as a dual
__device__ __forceinline__ Dual irls_weight(const Dual& lambda, const Dual& s2, float delta) {
  const Dual e = dsqrt(lambda * s2);
  if (e.v <= delta) return lambda;
  return lambda * (delta * dinv(e));
}

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
      const float x0 = sR[0] * Xj.x + sR[1] * Xj.y + sR[2] * Xj.z + st[0];
      const float x1 = sR[3] * Xj.x + sR[4] * Xj.y + sR[5] * Xj.z + st[1];
      const float x2 = sR[6] * Xj.x + sR[7] * Xj.y + sR[8] * Xj.z + st[2];
      const Dual X0 = dvar(x0, 0), X1 = dvar(x1, 1), X2 = dvar(x2, 2);
      const Dual Y0 = dvar(yv.x, 3), Y1 = dvar(yv.y, 4), Y2 = dvar(yv.z, 5), Q = dvar(qq, 6);
      const Dual d2 = X0 * X0 + X1 * X1 + X2 * X2;
      const Dual dy2 = Y0 * Y0 + Y1 * Y1 + Y2 * Y2;
      if (!(d2.v > 0.0f && dy2.v > 0.0f && d2.v < INFINITY && dy2.v < INFINITY)) continue;
      const Dual d = dsqrt(d2), dy = dsqrt(dy2), id = dinv(d), idy = dinv(dy);
      const Dual u0 = X0 * id, u1 = X1 * id, u2 = X2 * id;
      const Dual r0 = u0 - Y0 * idy, r1 = u1 - Y1 * idy, r2 = u2 - Y2 * idy;
      const Dual rd = d - dy;
      const Dual lr = bc.inv_sr2 * Q, ld = bc.inv_sd2 * Q;
      const Dual rr = r0 * r0 + r1 * r1 + r2 * r2;
      const Dual wr = irls_weight(lr, rr, bc.delta);
      const Dual wd = irls_weight(ld, rd * rd, bc.delta);
      Dual f = dconst(0.0f);
      if (bc.c_cost != 0.0f) {
        // Huber cost rho(e) = e^2/2 (e <= delta) else delta (e - delta/2)
        const Dual er2 = lr * rr, ed2 = ld * (rd * rd);
        const Dual er = dsqrt(er2), edd = dsqrt(ed2);
        const Dual cr = er.v <= bc.delta ? 0.5f * er2 : bc.delta * (er - dconst(0.5f * bc.delta));
        const Dual cd = edd.v <= bc.delta ? 0.5f * ed2 : bc.delta * (edd - dconst(0.5f * bc.delta));
        f = f + bc.c_cost * (cr + cd);
      }
      if (bc.with_step) {
        // J_rel v = ((I - u u^T) v_t + v_w x x) / d (ray rows), u . v_t + d v_s (distance row)
        auto jray = [&](const float* vv, Dual out[3]) {
          const Dual ut = u0 * dconst(vv[0]) + u1 * dconst(vv[1]) + u2 * dconst(vv[2]);
          const Dual c0 = dconst(vv[4]) * X2 - dconst(vv[5]) * X1;
          const Dual c1 = dconst(vv[5]) * X0 - dconst(vv[3]) * X2;
          const Dual c2 = dconst(vv[3]) * X1 - dconst(vv[4]) * X0;
          out[0] = (dconst(vv[0]) - u0 * ut + c0) * id;
          out[1] = (dconst(vv[1]) - u1 * ut + c1) * id;
          out[2] = (dconst(vv[2]) - u2 * ut + c2) * id;
        };
        Dual jb[3], jt[3];
        jray(sbeta, jb);
        jray(stheta, jt);
        const Dual db = u0 * dconst(sbeta[0]) + u1 * dconst(sbeta[1]) + u2 * dconst(sbeta[2]) + d * dconst(sbeta[6]);
        const Dual dt_ = u0 * dconst(stheta[0]) + u1 * dconst(stheta[1]) + u2 * dconst(stheta[2]) +
                         d * dconst(stheta[6]);
        const Dual phi = wr * (jb[0] * (jt[0] + r0) + jb[1] * (jt[1] + r1) + jb[2] * (jt[2] + r2)) +
                         wd * (db * (dt_ + rd));
        f = f - phi;
      }
      // dL/dX_j = (s R)^T dL/dx
      float* dXj = dX + 3 * (ed.off_j + n);
      atomicAdd(dXj + 0, sR[0] * f.d[0] + sR[3] * f.d[1] + sR[6] * f.d[2]);
      atomicAdd(dXj + 1, sR[1] * f.d[0] + sR[4] * f.d[1] + sR[7] * f.d[2]);
      atomicAdd(dXj + 2, sR[2] * f.d[0] + sR[5] * f.d[1] + sR[8] * f.d[2]);
      float* dXi = dX + 3 * (ed.off_i + m);
      atomicAdd(dXi + 0, f.d[3]);
      atomicAdd(dXi + 1, f.d[4]);
      atomicAdd(dXi + 2, f.d[5]);
      dq[ed.off_e + n] = f.d[6];
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
