// (a6-a8) Gauss-Newton solve of Sec. 3.5 for every graph of a plan.
//
// One CTA per graph.  The 14x14 edge blocks are assembled in FP64 into the
// 7x7 blocks of the gauge-reduced system (first keyframe dropped), each
// block summed in edge order from a host-built list; a right-looking block
// Cholesky then runs in the plan's minimum-degree elimination order over the
// symbolic fill pattern (diagonal factor by one warp, column panel and the
// (target, row, column) update triples spread over the CTA); forward and
// back substitution give tau = -H^-1 g, and every non-fixed pose is retracted
// T <- Exp(tau) o T in FP64 (Eq. 1, Eq. gauss_newton).
#include <algorithm>

#include "common.cuh"

namespace mslam {

struct SolveConst {
  double conv_tol;
  int factor_only;  // 1: factor and write tau, never touch poses or the converged flag
};

__global__ void __launch_bounds__(kSolveThreads) solve_kernel(PlanView pv, SolveConst sc,
                                                              const float* __restrict__ H14,
                                                              const float* __restrict__ g14,
                                                              double* __restrict__ T_wc, double* __restrict__ tau_out,
                                                              int32_t* __restrict__ dev_status,
                                                              double* __restrict__ ws) {
  const int g = blockIdx.x;
  const DevGraph G = pv.graphs[g];
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int s_fail;
  __shared__ double s_y[7];
  __shared__ double s_max;
  __shared__ int s_nonfinite;
  // converged (1) or failed (> 1) earlier: no more updates; a factor-only
  // call still factors a converged graph
  if (dev_status[g] > (sc.factor_only ? 1 : 0)) return;
  const int m = G.m;
  if (tau_out) {
    // zero tau of this graph's fixed pose
    if (tid < 7) tau_out[7 * G.gauge + tid] = 0.0;
  }
  if (m == 0) {
    if (tid == 0 && !sc.factor_only) dev_status[g] = 1;
    return;
  }
  const int32_t* I = pv.ints;
  const int32_t* pose_of_pos = I + G.off_pose;
  const int32_t* col_ptr = I + G.off_col;
  const int32_t* colent = I + G.off_colent;
  const int32_t* trip_ptr = I + G.off_trip;
  const int32_t* trips = I + G.off_tripent;
  const int32_t* asm_ptr = I + G.off_asm;
  const int32_t* asment = I + G.off_asment;
  const int32_t* gasm_ptr = I + G.off_gasm;
  const int32_t* gasment = I + G.off_gasment;
  double* L = ws + G.ws_off;
  double* rhs = L + (size_t)G.n_blocks * 49;
  double* diag0 = rhs + 7 * (size_t)m;

  // ---- assembly (FP64, fixed order)
  for (int t = tid; t < G.n_blocks * 49; t += nth) {
    const int b = t / 49, e = t % 49, r = e / 7, c = e % 7;
    double s = 0.0;
    for (int k = asm_ptr[b]; k < asm_ptr[b + 1]; ++k) {
      const int code = asment[k], edge = code >> 2, quad = code & 3;
      const int r0 = (quad == 0 || quad == 2) ? 0 : 7;
      const int c0 = (quad == 0 || quad == 3) ? 0 : 7;
      s += (double)H14[(size_t)edge * 196 + (r0 + r) * 14 + c0 + c];
    }
    L[t] = s;
    if (b < m && r == c) diag0[7 * b + r] = s;
  }
  for (int t = tid; t < 7 * m; t += nth) {
    const int p = t / 7, a = t % 7;
    double s = 0.0;
    for (int k = gasm_ptr[p]; k < gasm_ptr[p + 1]; ++k) {
      const int code = gasment[k], edge = code >> 1, side = code & 1;
      s += (double)g14[(size_t)edge * 14 + 7 * side + a];
    }
    rhs[t] = -s;
  }
  if (tid == 0) {
    s_fail = 0;
    s_nonfinite = 0;
    s_max = 0.0;
  }
  __syncthreads();

  // ---- numeric factorisation, right-looking over block columns
  for (int p = 0; p < m; ++p) {
    double* D = L + 49 * (size_t)p;
    if (warp == 0) {
      for (int j = 0; j < 7; ++j) {
        if (lane == 0) {
          double d = D[7 * j + j];
          for (int k = 0; k < j; ++k) d -= D[7 * j + k] * D[7 * j + k];
          const double ref = diag0[7 * p + j];
          if (!(d > 1e-12 * ref) || !isfinite(d)) {
            s_fail = 1;
            d = 1.0;
          }
          D[7 * j + j] = sqrt(d);
        }
        __syncwarp();
        if (lane > j && lane < 7) {
          double v = D[7 * lane + j];
          for (int k = 0; k < j; ++k) v -= D[7 * lane + k] * D[7 * j + k];
          D[7 * lane + j] = v / D[7 * j + j];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (s_fail) break;
    // panel: L_rp = A_rp L_pp^-T, one thread per (block, row)
    const int c0 = col_ptr[p], c1 = col_ptr[p + 1];
    for (int w = tid; w < (c1 - c0) * 7; w += nth) {
      const int ent = c0 + w / 7, a = w % 7;
      double* row = L + 49 * (size_t)colent[2 * ent + 1] + 7 * a;
      double x[7];
      for (int k = 0; k < 7; ++k) {
        double v = row[k];
        for (int l = 0; l < k; ++l) v -= x[l] * D[7 * k + l];
        x[k] = v / D[7 * k + k];
      }
      for (int k = 0; k < 7; ++k) row[k] = x[k];
    }
    __syncthreads();
    // trailing update: A_t -= L_b L_a^T for each triple of this column
    const int t0 = trip_ptr[p], t1 = trip_ptr[p + 1];
    for (int w = tid; w < (t1 - t0) * 49; w += nth) {
      const int tr = t0 + w / 49, e = w % 49, r = e / 7, c = e % 7;
      const double* Lb = L + 49 * (size_t)trips[3 * tr + 1] + 7 * r;
      const double* La = L + 49 * (size_t)trips[3 * tr + 2] + 7 * c;
      double s = 0.0;
      for (int k = 0; k < 7; ++k) s += Lb[k] * La[k];
      L[49 * (size_t)trips[3 * tr] + e] -= s;
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) dev_status[g] = MSLAM_ERR_NOT_PD;
    return;
  }

  // ---- forward substitution L y = -g
  for (int p = 0; p < m; ++p) {
    const double* D = L + 49 * (size_t)p;
    if (tid == 0) {
      double* y = rhs + 7 * p;
      for (int k = 0; k < 7; ++k) {
        double v = y[k];
        for (int l = 0; l < k; ++l) v -= D[7 * k + l] * y[l];
        y[k] = v / D[7 * k + k];
        s_y[k] = y[k];
      }
    }
    __syncthreads();
    const int c0 = col_ptr[p], c1 = col_ptr[p + 1];
    for (int w = tid; w < (c1 - c0) * 7; w += nth) {
      const int ent = c0 + w / 7, a = w % 7;
      const double* row = L + 49 * (size_t)colent[2 * ent + 1] + 7 * a;
      double s = 0.0;
      for (int k = 0; k < 7; ++k) s += row[k] * s_y[k];
      rhs[7 * colent[2 * ent] + a] -= s;
    }
    __syncthreads();
  }
  // ---- back substitution L^T x = y
  for (int p = m - 1; p >= 0; --p) {
    const double* D = L + 49 * (size_t)p;
    const int c0 = col_ptr[p], c1 = col_ptr[p + 1];
    if (tid < 7) {
      double s = rhs[7 * p + tid];
      for (int ent = c0; ent < c1; ++ent) {
        const double* Lr = L + 49 * (size_t)colent[2 * ent + 1];
        const double* xr = rhs + 7 * colent[2 * ent];
        for (int k = 0; k < 7; ++k) s -= Lr[7 * k + tid] * xr[k];
      }
      s_y[tid] = s;
    }
    __syncthreads();
    if (tid == 0) {
      double x[7];
      for (int k = 6; k >= 0; --k) {
        double v = s_y[k];
        for (int l = k + 1; l < 7; ++l) v -= D[7 * l + k] * x[l];
        x[k] = v / D[7 * k + k];
      }
      for (int k = 0; k < 7; ++k) rhs[7 * p + k] = x[k];
    }
    __syncthreads();
  }
  // ---- step statistics, tau, retraction
  for (int t = tid; t < 7 * m; t += nth) {
    const double v = rhs[t];
    if (!isfinite(v)) atomicExch(&s_nonfinite, 1);
  }
  __syncthreads();
  if (s_nonfinite) {
    if (tid == 0) dev_status[g] = MSLAM_ERR_NONFINITE;
    return;
  }
  if (warp == 0) {
    double mx = 0.0;
    for (int t = lane; t < 7 * m; t += 32) mx = fmax(mx, fabs(rhs[t]));
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) s_max = mx;
  }
  for (int p = tid; p < m; p += nth) {
    const int k = pose_of_pos[p];
    double tau[7];
    for (int a = 0; a < 7; ++a) tau[a] = rhs[7 * p + a];
    if (tau_out)
      for (int a = 0; a < 7; ++a) tau_out[7 * k + a] = tau[a];
    if (sc.factor_only) continue;
    const Sim3d E = sim3_exp(tau);
    const Sim3d Tn = compose(E, load_pose(T_wc + 8 * k));
    store_pose(Tn, T_wc + 8 * k);
  }
  __syncthreads();
  if (tid == 0 && !sc.factor_only && s_max < sc.conv_tol) dev_status[g] = 1;
}

}  // namespace mslam

using namespace mslam;

extern "C" mslam_status mslam_gn_solve(const mslam_params* p, const mslam_plan* plan, const float* H_blocks,
                                       const float* g_blocks, double* T_wc, double* tau, int32_t* dev_status,
                                       void* workspace, size_t ws_bytes, void* stream) {
  if (!p || !check_plan_uploaded(plan)) {
    if (!p) set_error("params is NULL");
    return MSLAM_ERR_ARG;
  }
  if (!H_blocks || !g_blocks || !T_wc || !dev_status || !workspace) {
    set_error("gn_solve: NULL device pointer");
    return MSLAM_ERR_ARG;
  }
  if (ws_bytes < mslam_workspace_bytes(plan, MSLAM_OP_SOLVE) || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    set_error("gn_solve: workspace smaller than %zu bytes or not 256-byte aligned",
              mslam_workspace_bytes(plan, MSLAM_OP_SOLVE));
    return MSLAM_ERR_ARG;
  }
  const PlanView pv = plan_view(plan);
  SolveConst sc;
  sc.conv_tol = p->conv_tol;
  sc.factor_only = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  solve_kernel<<<pv.G, kSolveThreads, 0, s>>>(pv, sc, H_blocks, g_blocks, T_wc, tau, dev_status,
                                              static_cast<double*>(workspace));
  return cuda_check(cudaGetLastError(), "gn_solve launch");
}

// Factor every graph's system and write tau = -H^-1 g without updating poses
// (used by the adjoint, which needs the factorisation and the step).
mslam_status mslam_factor_only(const mslam_plan* plan, const float* H_blocks, const float* g_blocks, double* tau,
                               int32_t* dev_status, double* ws, cudaStream_t s) {
  const PlanView pv = plan_view(plan);
  SolveConst sc;
  sc.conv_tol = 0.0;
  sc.factor_only = 1;
  solve_kernel<<<pv.G, kSolveThreads, 0, s>>>(pv, sc, H_blocks, g_blocks, nullptr, tau, dev_status, ws);
  return cuda_check(cudaGetLastError(), "factor launch");
}
