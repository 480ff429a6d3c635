// (a6-a8) Gauss-Newton solve of Sec. 3.5 for every graph of a plan.
//
// One CTA per graph.  The 14x14 edge blocks are assembled in FP64 into the
// 7x7 blocks of the gauge-reduced system (first keyframe dropped), each
// block summed in edge order from a host-built list.  The block Cholesky is
// left-looking and scheduled by levels of the elimination dependencies in
// the plan's minimum-degree order (21 levels for the 63 columns of the
// 64-keyframe loop graph): per level, (A) every target block and right-hand
// side row of the level's columns gathers its updates from lower levels in a
// fixed order, (B) one warp per column factors the diagonal block (reciprocal
// pivots kept) and forward-substitutes y_p, (C) the column panels
// L_rp = A_rp L_pp^-T are formed.  Back substitution runs the levels in
// reverse, one warp per column, and every non-fixed pose is retracted
// T <- Exp(tau) o T in FP64 (Eq. 1, Eq. gauss_newton).  The numeric factor
// lives in shared memory when the graph fits (the 64-keyframe graph needs
// 151 KB), else in the caller's workspace.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace mslam {

struct SolveConst {
  double conv_tol;
  int factor_only;      // 1: factor and write tau, never touch poses or the converged flag
  int smem_doubles;     // dynamic shared memory available per CTA (doubles)
  const int32_t* skip;  // per graph: 1 = already solved by the mixed-precision kernel (may be NULL)
  // the mixed-precision kernel for the adjoint (never touches poses or the
  // converged flag): 0 = the forward step, 1 = x = tau = -H^-1 g into x_out
  // and the FP32 factor kept in the workspace, 2 = x = H^-1 rhs into x_out
  // with the kept factor, for the graphs whose handled_in flag is set
  int bwd_mode;
  const double* rhs;         // [N, 7] in pose order (mode 2)
  double* x_out;             // [N, 7] in pose order, zero for the fixed pose (modes 1, 2)
  const int32_t* handled_in; // per graph: 1 = mode 1 kept its factor (mode 2)
};

__global__ void __launch_bounds__(kSolveThreads) solve_kernel(PlanView pv, SolveConst sc,
                                                              const float* __restrict__ H14,
                                                              const float* __restrict__ g14,
                                                              double* __restrict__ T_wc, double* __restrict__ tau_out,
                                                              int32_t* __restrict__ dev_status,
                                                              double* __restrict__ ws) {
  extern __shared__ double smem[];
  const int g = blockIdx.x;
  const DevGraph G = pv.graphs[g];
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int s_fail;
  __shared__ double s_max;
  __shared__ int s_nonfinite;
  if (sc.skip && sc.skip[g]) return;
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
  const int32_t* asm_ptr = I + G.off_asm;
  const int32_t* asment = I + G.off_asment;
  const int32_t* gasm_ptr = I + G.off_gasm;
  const int32_t* gasment = I + G.off_gasment;
  const int64_t need = (int64_t)G.n_blocks * 49 + 21 * (int64_t)m;
  const bool in_smem = need <= sc.smem_doubles;
  double* gws = ws + G.ws_off;
  double* L = in_smem ? smem : gws;
  double* rhs = L + (size_t)G.n_blocks * 49;
  double* diag0 = rhs + 7 * (size_t)m;
  double* invd = diag0 + 7 * (size_t)m;

  // ---- assembly (FP64, fixed order)
  for (int t = tid; t < G.n_blocks * 49; t += nth) {
    const int b = t / 49, e = t % 49, r = e / 7, c = e % 7;
    double s = 0.0;
    const int k1 = __ldg(asm_ptr + b + 1);
    for (int k = __ldg(asm_ptr + b); k < k1; ++k) {
      const int code = __ldg(asment + k), edge = code >> 2, quad = code & 3;
      const int r0 = (quad == 0 || quad == 2) ? 0 : 7;
      const int c0 = (quad == 0 || quad == 3) ? 0 : 7;
      s += (double)__ldg(H14 + (size_t)edge * 196 + (r0 + r) * 14 + c0 + c);
    }
    L[t] = s;
    if (b < m && r == c) diag0[7 * b + r] = s;
  }
  for (int t = tid; t < 7 * m; t += nth) {
    const int p = t / 7, a = t % 7;
    double s = 0.0;
    const int k1 = __ldg(gasm_ptr + p + 1);
    for (int k = __ldg(gasm_ptr + p); k < k1; ++k) {
      const int code = __ldg(gasment + k), edge = code >> 1, side = code & 1;
      s += (double)__ldg(g14 + (size_t)edge * 14 + 7 * side + a);
    }
    rhs[t] = -s;
  }
  if (tid == 0) {
    s_fail = 0;
    s_nonfinite = 0;
    s_max = 0.0;
  }
  __syncthreads();

  // ---- numeric factorisation, left-looking, one elimination level at a time.
  // Level l holds columns whose dependencies all lie in lower levels; its
  // columns write disjoint blocks, so each phase runs over the whole level.
  const int32_t* lev_ptr = I + G.off_lev;
  const int32_t* lev_cols = I + G.off_levcols;
  const int32_t* levtgt = I + G.off_levtgt;
  const int32_t* tgtlist = I + G.off_tgtlist;
  const int32_t* tptr = I + G.off_tptr;
  const int32_t* pairs = I + G.off_pairs;
  const int32_t* rsptr = I + G.off_rsptr;
  const int32_t* rs = I + G.off_rs;
  const int32_t* blkcol = I + G.off_blkcol;
  const int nwarps = nth >> 5;
  for (int l = 0; l < G.n_levels; ++l) {
    const int q0 = __ldg(lev_ptr + l), q1 = __ldg(lev_ptr + l + 1);
    const int g0 = __ldg(levtgt + l), g1 = __ldg(levtgt + l + 1);
    // (A) updates from lower levels: A_t -= sum_c L_(r,c) L_(p,c)^T for every
    //     target block of the level, and rhs_p -= sum_c L_(p,c) y_c
    const int nA = (g1 - g0) * 49;
    for (int w = tid; w < nA + (q1 - q0) * 7; w += nth) {
      if (w < nA) {
        const int t = __ldg(tgtlist + g0 + w / 49), e = w % 49, r = e / 7, c = e % 7;
        const int k1 = __ldg(tptr + t + 1);
        double ps[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // independent chains (FP64 latency)
        for (int k = __ldg(tptr + t); k < k1; ++k) {
          const double* Lb = L + 49 * (size_t)__ldg(pairs + 2 * k) + 7 * r;
          const double* La = L + 49 * (size_t)__ldg(pairs + 2 * k + 1) + 7 * c;
#pragma unroll
          for (int kk = 0; kk < 7; ++kk) ps[kk] = fma(Lb[kk], La[kk], ps[kk]);
        }
        L[49 * (size_t)t + e] -= ((ps[0] + ps[1]) + (ps[2] + ps[3])) + ((ps[4] + ps[5]) + ps[6]);
      } else {
        const int ww = w - nA, p = __ldg(lev_cols + q0 + ww / 7), a = ww % 7;
        const int k1 = __ldg(rsptr + p + 1);
        double ps[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int k = __ldg(rsptr + p); k < k1; ++k) {
          const double* Lpc = L + 49 * (size_t)__ldg(rs + 2 * k + 1) + 7 * a;
          const double* yc = rhs + 7 * __ldg(rs + 2 * k);
#pragma unroll
          for (int kk = 0; kk < 7; ++kk) ps[kk] = fma(Lpc[kk], yc[kk], ps[kk]);
        }
        rhs[7 * p + a] -= ((ps[0] + ps[1]) + (ps[2] + ps[3])) + ((ps[4] + ps[5]) + ps[6]);
      }
    }
    __syncthreads();
    // (B) diagonal factor and y_p = L_pp^-1 rhs_p, one warp per column: lane
    //     i < 7 owns row i of the block and y_i; column-oriented inside the
    //     block, so each step is a few dependent FP64 operations.  All lanes
    //     execute every shuffle (full mask); lanes >= 7 carry dummies.
    for (int qi = q0 + warp; qi < q1; qi += nwarps) {
      const int p = __ldg(lev_cols + qi);
      double* D = L + 49 * (size_t)p;
      double* iv = invd + 7 * p;
      const bool mine = lane < 7;
      const int li = mine ? lane : 0;
      double row[7], yv = mine ? rhs[7 * p + li] : 0.0;
#pragma unroll
      for (int k = 0; k < 7; ++k) row[k] = D[7 * li + k];
      bool bad = false;
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        const double djj = __shfl_sync(0xffffffffu, row[j], j);  // A_jj after earlier steps
        const bool okj = (djj > 1e-12 * diag0[7 * p + j]) && isfinite(djj);
        bad |= !okj;
        const double ivj = rsqrt_newton(okj ? djj : 1.0);    // 1 / L_jj
        const double yj = __shfl_sync(0xffffffffu, yv, j) * ivj;
        // lane j: row[j] = A_jj / sqrt(A_jj) = L_jj; lanes > j: L_ij = A_ij / L_jj
        const double lij = (lane == j && !okj) ? 1.0 : row[j] * ivj;
        if (mine && lane >= j) row[j] = lij;
        if (lane == j) {
          iv[j] = ivj;
          yv = yj;
        } else if (mine && lane > j) {
          yv = fma(-lij, yj, yv);
        }
        // trailing update inside the block: A_ik -= L_ij L_kj for j < k <= i
#pragma unroll
        for (int k = j + 1; k < 7; ++k) {
          const double lkj = __shfl_sync(0xffffffffu, row[j], k);
          if (mine && lane >= k) row[k] = fma(-lij, lkj, row[k]);
        }
      }
      if (mine) {
#pragma unroll
        for (int k = 0; k < 7; ++k)
          if (k <= lane) D[7 * lane + k] = row[k];
        rhs[7 * p + lane] = yv;
      }
      if (bad && lane == 0) s_fail = 1;
      __syncwarp();
    }
    __syncthreads();
    if (s_fail) break;
    // (C) panel: L_rp = A_rp L_pp^-T for the column blocks of the level
    for (int w = tid; w < (g1 - g0) * 7; w += nth) {
      const int t = __ldg(tgtlist + g0 + w / 7), a = w % 7;
      if (t < m) continue;  // a diagonal block
      const int p = __ldg(blkcol + t);
      const double* D = L + 49 * (size_t)p;
      const double* iv = invd + 7 * p;
      double* row = L + 49 * (size_t)t + 7 * a;
      double x[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        double v = row[k];
        for (int l2 = 0; l2 < k; ++l2) v -= x[l2] * D[7 * k + l2];
        x[k] = v * iv[k];
      }
#pragma unroll
      for (int k = 0; k < 7; ++k) row[k] = x[k];
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) dev_status[g] = MSLAM_ERR_NOT_PD;
    return;
  }

  // ---- back substitution L^T x = y, levels in reverse (a column's rows all
  // lie in higher levels), one warp per column
  for (int l = G.n_levels - 1; l >= 0; --l) {
    const int q0 = __ldg(lev_ptr + l), q1 = __ldg(lev_ptr + l + 1);
    for (int qi = q0 + warp; qi < q1; qi += nwarps) {
      const int p = __ldg(lev_cols + qi);
      const double* D = L + 49 * (size_t)p;
      const int c0 = __ldg(col_ptr + p), c1 = __ldg(col_ptr + p + 1);
      double s = 0.0;
      if (lane < 7) {
        double ps[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // independent chains
        for (int ent = c0; ent < c1; ++ent) {
          const double* Lr = L + 49 * (size_t)__ldg(colent + 2 * ent + 1);
          const double* xr = rhs + 7 * __ldg(colent + 2 * ent);
#pragma unroll
          for (int k = 0; k < 7; ++k) ps[k] = fma(Lr[7 * k + lane], xr[k], ps[k]);
        }
        s = rhs[7 * p + lane] - (((ps[0] + ps[1]) + (ps[2] + ps[3])) + ((ps[4] + ps[5]) + ps[6]));
      }
      // L_pp^T x = s, column-oriented across lanes 0..6: x_k = s_k / L_kk,
      // then s_l -= L_kl x_k for l < k (a few dependent operations per k)
      const double* iv = invd + 7 * p;
      double xl = 0.0;
#pragma unroll
      for (int k = 6; k >= 0; --k) {
        const double xk = __shfl_sync(0xffffffffu, s, k) * iv[k];
        if (lane == k) xl = xk;
        if (lane < k) s = fma(-D[7 * k + lane], xk, s);
      }
      if (lane < 7) rhs[7 * p + lane] = xl;
      __syncwarp();
    }
    __syncthreads();
  }
  if (sc.factor_only && in_smem) {
    // the adjoint reuses the factor: leave it in the workspace
    for (size_t t = tid; t < (size_t)need; t += nth) gws[t] = L[t];
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
    const int k = __ldg(pose_of_pos + p);
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

// ---------------------------------------------------------------- cluster form
// The same factorisation spread over a thread-block cluster of kClusterSize
// CTAs (one cluster per graph).  Every CTA keeps a full replica of the
// factor, right-hand side, assembled diagonal and reciprocal pivots in its
// shared memory, so all reads are local; each value is computed by one
// thread of the cluster and written to all replicas through distributed
// shared memory, and a cluster barrier (release / acquire) separates the
// phases.  Control flow is uniform across the cluster: no CTA leaves early
// between barriers (a failed pivot only marks the status).
constexpr int kClusterSize = 2;  // measured fastest of 1, 2, 4, 8 on the 64-keyframe graph

__global__ void __launch_bounds__(kSolveThreads) solve_cluster_kernel(PlanView pv, SolveConst sc,
                                                                      const float* __restrict__ H14,
                                                                      const float* __restrict__ g14,
                                                                      double* __restrict__ T_wc,
                                                                      double* __restrict__ tau_out,
                                                                      int32_t* __restrict__ dev_status,
                                                                      double* __restrict__ ws) {
  namespace cg = cooperative_groups;
  extern __shared__ double smem[];
  __shared__ double* rbase[kClusterSize];
  __shared__ int* rfail[kClusterSize];
  __shared__ int s_fail;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int g = blockIdx.x / kClusterSize;
  const DevGraph G = pv.graphs[g];
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int ctid = rank * nth + tid, cnth = kClusterSize * nth;            // cluster-wide thread index
  const int nwarps = nth >> 5, cwarp = rank * nwarps + warp, cnwarps = kClusterSize * nwarps;
  // uniform across the cluster (all CTAs read the same flags and status)
  if (sc.skip && sc.skip[g]) return;
  if (dev_status[g] > (sc.factor_only ? 1 : 0)) return;
  const int m = G.m;
  if (m == 0) {
    if (rank == 0 && tid == 0 && !sc.factor_only) dev_status[g] = 1;
    if (rank == 0 && tau_out && tid < 7) tau_out[7 * G.gauge + tid] = 0.0;
    return;
  }
  if (tid < kClusterSize) {
    rbase[tid] = cl.map_shared_rank(smem, tid);
    rfail[tid] = cl.map_shared_rank(&s_fail, tid);
  }
  if (tid == 0) s_fail = 0;
  cl.sync();  // every CTA of the cluster is running and initialised
  const int32_t* I = pv.ints;
  const int32_t* pose_of_pos = I + G.off_pose;
  const int32_t* col_ptr = I + G.off_col;
  const int32_t* colent = I + G.off_colent;
  const int32_t* asm_ptr = I + G.off_asm;
  const int32_t* asment = I + G.off_asment;
  const int32_t* gasm_ptr = I + G.off_gasm;
  const int32_t* gasment = I + G.off_gasment;
  const int32_t* lev_ptr = I + G.off_lev;
  const int32_t* lev_cols = I + G.off_levcols;
  const int32_t* levtgt = I + G.off_levtgt;
  const int32_t* tgtlist = I + G.off_tgtlist;
  const int32_t* tptr = I + G.off_tptr;
  const int32_t* pairs = I + G.off_pairs;
  const int32_t* rsptr = I + G.off_rsptr;
  const int32_t* rs = I + G.off_rs;
  const int32_t* blkcol = I + G.off_blkcol;
  const size_t need = (size_t)G.n_blocks * 49 + 21 * (size_t)m;
  double* L = smem;
  const size_t off_rhs = (size_t)G.n_blocks * 49, off_d0 = off_rhs + 7 * (size_t)m, off_iv = off_d0 + 7 * (size_t)m;
  double* rhs = L + off_rhs;
  double* diag0 = L + off_d0;
  double* invd = L + off_iv;
  auto put = [&](size_t off, double v) {
#pragma unroll
    for (int r = 0; r < kClusterSize; ++r) rbase[r][off] = v;
  };

  // ---- assembly
  for (int t = ctid; t < G.n_blocks * 49; t += cnth) {
    const int b = t / 49, e = t % 49, r = e / 7, c = e % 7;
    double s = 0.0;
    const int k1 = __ldg(asm_ptr + b + 1);
    for (int k = __ldg(asm_ptr + b); k < k1; ++k) {
      const int code = __ldg(asment + k), edge = code >> 2, quad = code & 3;
      const int r0 = (quad == 0 || quad == 2) ? 0 : 7;
      const int c0 = (quad == 0 || quad == 3) ? 0 : 7;
      s += (double)__ldg(H14 + (size_t)edge * 196 + (r0 + r) * 14 + c0 + c);
    }
    put(t, s);
    if (b < m && r == c) put(off_d0 + 7 * b + r, s);
  }
  for (int t = ctid; t < 7 * m; t += cnth) {
    const int p = t / 7, a = t % 7;
    double s = 0.0;
    const int k1 = __ldg(gasm_ptr + p + 1);
    for (int k = __ldg(gasm_ptr + p); k < k1; ++k) {
      const int code = __ldg(gasment + k), edge = code >> 1, side = code & 1;
      s += (double)__ldg(g14 + (size_t)edge * 14 + 7 * side + a);
    }
    put(off_rhs + t, -s);
  }
  cl.sync();

  // ---- factorisation by levels
  for (int l = 0; l < G.n_levels; ++l) {
    const int q0 = __ldg(lev_ptr + l), q1 = __ldg(lev_ptr + l + 1);
    const int g0 = __ldg(levtgt + l), g1 = __ldg(levtgt + l + 1);
    const int nA = (g1 - g0) * 49;
    for (int w = ctid; w < nA + (q1 - q0) * 7; w += cnth) {
      if (w < nA) {
        const int t = __ldg(tgtlist + g0 + w / 49), e = w % 49, r = e / 7, c = e % 7;
        const int k1 = __ldg(tptr + t + 1);
        double ps[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int k = __ldg(tptr + t); k < k1; ++k) {
          const double* Lb = L + 49 * (size_t)__ldg(pairs + 2 * k) + 7 * r;
          const double* La = L + 49 * (size_t)__ldg(pairs + 2 * k + 1) + 7 * c;
#pragma unroll
          for (int kk = 0; kk < 7; ++kk) ps[kk] = fma(Lb[kk], La[kk], ps[kk]);
        }
        const size_t off = 49 * (size_t)t + e;
        put(off, L[off] - (((ps[0] + ps[1]) + (ps[2] + ps[3])) + ((ps[4] + ps[5]) + ps[6])));
      } else {
        const int ww = w - nA, p = __ldg(lev_cols + q0 + ww / 7), a = ww % 7;
        const int k1 = __ldg(rsptr + p + 1);
        double ps[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int k = __ldg(rsptr + p); k < k1; ++k) {
          const double* Lpc = L + 49 * (size_t)__ldg(rs + 2 * k + 1) + 7 * a;
          const double* yc = rhs + 7 * __ldg(rs + 2 * k);
#pragma unroll
          for (int kk = 0; kk < 7; ++kk) ps[kk] = fma(Lpc[kk], yc[kk], ps[kk]);
        }
        const size_t off = off_rhs + 7 * (size_t)p + a;
        put(off, L[off] - (((ps[0] + ps[1]) + (ps[2] + ps[3])) + ((ps[4] + ps[5]) + ps[6])));
      }
    }
    cl.sync();
    for (int qi = q0 + cwarp; qi < q1; qi += cnwarps) {
      const int p = __ldg(lev_cols + qi);
      const double* D = L + 49 * (size_t)p;
      const bool mine = lane < 7;
      const int li = mine ? lane : 0;
      double row[7], yv = mine ? rhs[7 * p + li] : 0.0;
#pragma unroll
      for (int k = 0; k < 7; ++k) row[k] = D[7 * li + k];
      bool bad = false;
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        const double djj = __shfl_sync(0xffffffffu, row[j], j);
        const bool okj = (djj > 1e-12 * diag0[7 * p + j]) && isfinite(djj);
        bad |= !okj;
        const double ivj = rsqrt_newton(okj ? djj : 1.0);
        const double yj = __shfl_sync(0xffffffffu, yv, j) * ivj;
        const double lij = (lane == j && !okj) ? 1.0 : row[j] * ivj;
        if (mine && lane >= j) row[j] = lij;
        if (lane == j) {
          put(off_iv + 7 * (size_t)p + j, ivj);
          yv = yj;
        } else if (mine && lane > j) {
          yv = fma(-lij, yj, yv);
        }
#pragma unroll
        for (int k = j + 1; k < 7; ++k) {
          const double lkj = __shfl_sync(0xffffffffu, row[j], k);
          if (mine && lane >= k) row[k] = fma(-lij, lkj, row[k]);
        }
      }
      if (mine) {
#pragma unroll
        for (int k = 0; k < 7; ++k)
          if (k <= lane) put(49 * (size_t)p + 7 * lane + k, row[k]);
        put(off_rhs + 7 * (size_t)p + lane, yv);
      }
      if (bad && lane == 0)
        for (int r = 0; r < kClusterSize; ++r) *rfail[r] = 1;
    }
    cl.sync();
    for (int w = ctid; w < (g1 - g0) * 7; w += cnth) {
      const int t = __ldg(tgtlist + g0 + w / 7), a = w % 7;
      if (t < m) continue;
      const int p = __ldg(blkcol + t);
      const double* D = L + 49 * (size_t)p;
      const double* iv = invd + 7 * p;
      const double* row = L + 49 * (size_t)t + 7 * a;
      double x[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        double v = row[k];
        for (int l2 = 0; l2 < k; ++l2) v -= x[l2] * D[7 * k + l2];
        x[k] = v * iv[k];
      }
#pragma unroll
      for (int k = 0; k < 7; ++k) put(49 * (size_t)t + 7 * a + k, x[k]);
    }
    cl.sync();
  }

  // ---- back substitution by levels (reverse)
  for (int l = G.n_levels - 1; l >= 0; --l) {
    const int q0 = __ldg(lev_ptr + l), q1 = __ldg(lev_ptr + l + 1);
    for (int qi = q0 + cwarp; qi < q1; qi += cnwarps) {
      const int p = __ldg(lev_cols + qi);
      const double* D = L + 49 * (size_t)p;
      const int c0 = __ldg(col_ptr + p), c1 = __ldg(col_ptr + p + 1);
      double s = 0.0;
      if (lane < 7) {
        double ps[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int ent = c0; ent < c1; ++ent) {
          const double* Lr = L + 49 * (size_t)__ldg(colent + 2 * ent + 1);
          const double* xr = rhs + 7 * __ldg(colent + 2 * ent);
#pragma unroll
          for (int k = 0; k < 7; ++k) ps[k] = fma(Lr[7 * k + lane], xr[k], ps[k]);
        }
        s = rhs[7 * p + lane] - (((ps[0] + ps[1]) + (ps[2] + ps[3])) + ((ps[4] + ps[5]) + ps[6]));
      }
      const double* iv = invd + 7 * p;
      double xl = 0.0;
#pragma unroll
      for (int k = 6; k >= 0; --k) {
        const double xk = __shfl_sync(0xffffffffu, s, k) * iv[k];
        if (lane == k) xl = xk;
        if (lane < k) s = fma(-D[7 * k + lane], xk, s);
      }
      if (lane < 7) put(off_rhs + 7 * (size_t)p + lane, xl);
      __syncwarp();
    }
    cl.sync();
  }
  // every replica now holds tau in rhs; the failure flag is the same in all CTAs
  const bool failed = s_fail != 0;
  if (sc.factor_only && rank == 0 && !failed) {
    for (size_t t = tid; t < need; t += nth) ws[G.ws_off + t] = L[t];  // the adjoint reuses the factor
  }
  if (failed) {
    if (rank == 0 && tid == 0) dev_status[g] = MSLAM_ERR_NOT_PD;
    cl.sync();  // keep every replica alive until all remote writes are done
    return;
  }
  // max |tau| and finiteness over the replica (the same in every CTA)
  __shared__ double s_wmax[kSolveThreads / 32];
  __shared__ int s_nf;
  if (tid == 0) s_nf = 0;
  __syncthreads();
  double mx = 0.0;
  for (int t = tid; t < 7 * m; t += nth) {
    const double v = rhs[t];
    if (!isfinite(v)) s_nf = 1;
    mx = fmax(mx, fabs(v));
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if (lane == 0) s_wmax[warp] = mx;
  __syncthreads();
  mx = 0.0;
  for (int w = 0; w < nwarps; ++w) mx = fmax(mx, s_wmax[w]);
  const bool nonfinite = s_nf != 0;
  if (tau_out && rank == 0 && tid < 7) tau_out[7 * G.gauge + tid] = 0.0;
  if (!nonfinite) {
    for (int p = ctid; p < m; p += cnth) {
      const int k = __ldg(pose_of_pos + p);
      double tau[7];
      for (int a = 0; a < 7; ++a) tau[a] = rhs[7 * p + a];
      if (tau_out)
        for (int a = 0; a < 7; ++a) tau_out[7 * k + a] = tau[a];
      if (sc.factor_only) continue;
      const Sim3d E = sim3_exp(tau);
      store_pose(compose(E, load_pose(T_wc + 8 * k)), T_wc + 8 * k);
    }
  }
  if (rank == 0 && tid == 0) {
    if (nonfinite) dev_status[g] = MSLAM_ERR_NONFINITE;
    else if (!sc.factor_only && mx < sc.conv_tol) dev_status[g] = 1;
  }
  cl.sync();  // no CTA exits while others may still read its shared memory
}

// ------------------------------------------------------- mixed-precision form
// The same system solved by a factorisation in FP32 and iterative refinement
// in FP64.  With D the assembled diagonal and S = D^-1/2, the scaled matrix
// S H S (unit diagonal) is factored in FP32 with the level schedule above;
// then x <- x + S (L L^T)^-1 S (b - H x), the residual b - H x formed in FP64
// from the assembled FP64 blocks, until the predicted next correction
// (the last correction times the observed contraction rate) is below 1e-9
// of |x|.  Each FP32 operation has a latency of a few cycles instead of about
// 64 for FP64 on this GPU, which shortens the solve's dependent chains; the
// refined solution is the FP64 solution of the same system.  A graph whose
// FP32 factorisation meets a pivot below 2^-20 of its unit diagonal, or
// whose refinement stalls, is left to the FP64 kernel (flag handled[g] = 0),
// which applies the exact not-positive-definite rule.
constexpr int kMixThreads = 512;
constexpr int kMixMaxIters = 10;
// FP32 factor block in shared memory: 7 rows of kLfRow floats (7 entries, then
// zeros), 48-byte rows: the seven rows of a block start in seven disjoint
// groups of four shared-memory banks, so a warp's 16-byte loads of different
// rows of one block take one wavefront.  A factor too large for shared memory
// stays in the workspace with 8-float rows (fewer bytes through L1 and L2);
// the workspace reserves kLfBlock floats per block for either form.
constexpr int kLfBlock = 7 * kLfRow;

// One element of an assembled block, summed in FP64 over its edge
// contributions in edge order (as in the FP64 kernel).
__device__ __forceinline__ double asm_sum(const float* __restrict__ H14, const int32_t* __restrict__ asm_ptr,
                                          const int32_t* __restrict__ asment, int b, int r, int c) {
  double s = 0.0;
  const int k1 = __ldg(asm_ptr + b + 1);
#pragma unroll 4
  for (int k = __ldg(asm_ptr + b); k < k1; ++k) {
    const int code = __ldg(asment + k), edge = code >> 2, quad = code & 3;
    const int r0 = (quad == 0 || quad == 2) ? 0 : 7;
    const int c0 = (quad == 0 || quad == 3) ? 0 : 7;
    s += (double)__ldg(H14 + (size_t)edge * 196 + (r0 + r) * 14 + c0 + c);
  }
  return s;
}

// Inputs of the mixed-precision solve, spread over many CTAs (the FP64 rate
// of a single SM would make this the solve's longest phase), one thread per
// element of the padded 7 x kLfRow blocks: every block element in FP64 (kept for
// the residuals) and the scaled FP32 factor input S H S (unit diagonal),
// with S = D^-1/2 from the assembled diagonal (each thread forms the two
// entries of S it needs); the padding threads of the diagonal blocks write
// S and -g for their unknown.  A diagonal entry that is not positive and
// finite gives S = NaN, which makes the solve decline the graph.
__device__ __forceinline__ double jacobi_scale(const float* __restrict__ H14, const int32_t* __restrict__ asm_ptr,
                                               const int32_t* __restrict__ asment, int p, int a) {
  const double d = asm_sum(H14, asm_ptr, asment, p, a, a);
  return (d > 0.0 && isfinite(d)) ? rsqrt_newton(d) : __longlong_as_double(0x7ff8000000000000LL);
}

__global__ void __launch_bounds__(64) solve_assemble_kernel(PlanView pv, const float* __restrict__ H14,
                                                            const float* __restrict__ g14,
                                                            const int32_t* __restrict__ dev_status,
                                                            double* __restrict__ ws, int max_status, int row) {
  const int g = blockIdx.y;
  const DevGraph G = pv.graphs[g];
  if (dev_status[g] > max_status || G.m == 0) return;  // the solve kernels skip these graphs too
  const int nb = G.n_blocks;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int blk = 7 * row;  // the mixed kernel's row stride for this plan
  if (t >= nb * blk) return;
  const int32_t* I = pv.ints;
  const int32_t* asm_ptr = I + G.off_asm;
  const int32_t* asment = I + G.off_asment;
  float* Lf = reinterpret_cast<float*>(ws + G.ws_mixed);
  const int b = t / blk, e = t % blk, r = e / row, c = e % row;
  if (c >= 7) {
    Lf[t] = 0.0f;
    if (c == 7 && b < G.m) {
      // diagonal block b = unknown block b: S and -g of unknown 7 b + r
      const int n7 = 7 * G.m, k = 7 * b + r;
      double* scl = ws + G.ws_mixed + (size_t)nb * (kLfBlock / 2);
      scl[k] = jacobi_scale(H14, asm_ptr, asment, b, r);
      const int32_t* gasm_ptr = I + G.off_gasm;
      const int32_t* gasment = I + G.off_gasment;
      double sg = 0.0;
      const int j1 = __ldg(gasm_ptr + b + 1);
#pragma unroll 4
      for (int j = __ldg(gasm_ptr + b); j < j1; ++j) {
        const int code = __ldg(gasment + j), edge = code >> 1, side = code & 1;
        sg += (double)__ldg(g14 + (size_t)edge * 14 + 7 * side + r);
      }
      scl[n7 + k] = -sg;
    }
    return;
  }
  const double h = asm_sum(H14, asm_ptr, asment, b, r, c);
  ws[G.ws_off + 49 * (size_t)b + 7 * r + c] = h;
  const int br = __ldg(I + G.off_blkrow + b), bc = __ldg(I + G.off_blkcol + b);
  const double sr = jacobi_scale(H14, asm_ptr, asment, br, r);
  const double sc = jacobi_scale(H14, asm_ptr, asment, bc, c);
  Lf[t] = (float)(h * sr * sc);
}

// Deterministic sum of the four 7-lane groups of a warp into lanes 0..6
// (lane a + 7 g holds group g's partial for row a).
__device__ __forceinline__ float sum_groups(float v) {
  const float v1 = __shfl_down_sync(0xffffffffu, v, 7);
  const float v2 = __shfl_down_sync(0xffffffffu, v, 14);
  const float v3 = __shfl_down_sync(0xffffffffu, v, 21);
  return (v + v1) + (v2 + v3);
}

__device__ __forceinline__ float dot8(const float* a, const float* b) {
  const float4 a0 = *reinterpret_cast<const float4*>(a), a1 = *reinterpret_cast<const float4*>(a + 4);
  const float4 b0 = *reinterpret_cast<const float4*>(b), b1 = *reinterpret_cast<const float4*>(b + 4);
  return ((a0.x * b0.x + a0.y * b0.y) + (a0.z * b0.z + a0.w * b0.w)) +
         ((a1.x * b1.x + a1.y * b1.y) + (a1.z * b1.z + a1.w * b1.w));
}

// kGlobalL: the FP32 factor stays in the workspace (L2-resident) where the
// assembly kernel wrote it and is factored in place, for graphs whose factor
// does not fit one SM's shared memory; everything else stays in shared memory.
template <bool kGlobalL>
__global__ void __launch_bounds__(kMixThreads) solve_mixed_kernel(PlanView pv, SolveConst sc,
                                                                  double* __restrict__ T_wc,
                                                                  double* __restrict__ tau_out,
                                                                  int32_t* __restrict__ dev_status,
                                                                  double* __restrict__ ws,
                                                                  int32_t* __restrict__ handled) {
  // the factor's row stride: 12 floats in shared memory (rows of a block in
  // disjoint bank groups), 8 in the workspace (fewer bytes through L2)
  constexpr int kRow = kGlobalL ? 8 : kLfRow;
  constexpr int kBlk = 7 * kRow;
  extern __shared__ double smem[];
  const int g = blockIdx.x;
  const DevGraph G = pv.graphs[g];
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
  __shared__ int s_fail, s_done, s_nonfinite;
  __shared__ double s_zmax, s_xmax, s_zprev, s_max;
  const int m = G.m, nb = G.n_blocks;
  const int bwd = sc.bwd_mode;
  if (dev_status[g] > (bwd ? 1 : 0) || m == 0 || (bwd == 2 && !sc.handled_in[g])) {
    // converged or failed earlier, or nothing to solve: the FP64 kernel
    // handles these cases exactly as before
    if (tid == 0) handled[g] = 0;
    return;
  }
  const int n7 = 7 * m;
  // shared memory: the padded FP32 factor, FP64 vectors, FP32 vectors, then
  // the graph's tables (all but the update triples), so that every dependent
  // lookup of the level schedule is a shared-memory access
  // scaled factor, FP32, 7 x kRow per block (16-byte aligned rows)
  float* Lf = kGlobalL ? reinterpret_cast<float*>(ws + G.ws_mixed) : reinterpret_cast<float*>(smem);
  double* scl = kGlobalL ? smem : reinterpret_cast<double*>(Lf + (size_t)nb * kBlk);  // S = D^-1/2
  double* xv = scl + n7;                        // solution
  double* bv = xv + n7;                         // right-hand side -g
  float* yv = reinterpret_cast<float*>(bv + n7);  // work vector
  float* ivf = yv + n7;                           // reciprocal pivots
  float* Linv = ivf + n7;                         // inverses of the diagonal factor blocks, 7 x 8 per column
  int* sI = reinterpret_cast<int*>(Linv + 8 * n7);
  const int seg1 = G.off_trip - G.off_pose, seg2 = G.int_end - G.off_lev;
  for (int t = tid; t < seg1; t += nth) sI[t] = __ldg(pv.ints + G.off_pose + t);
  for (int t = tid; t < seg2; t += nth) sI[seg1 + t] = __ldg(pv.ints + G.off_lev + t);
  {
    if (!kGlobalL) {
      const float4* src = reinterpret_cast<const float4*>(ws + G.ws_mixed);
      float4* dst = reinterpret_cast<float4*>(Lf);
      for (int t = tid; t < nb * (kBlk / 4); t += nth) dst[t] = src[t];
    }
    const double* sg = ws + G.ws_mixed + (size_t)nb * (kLfBlock / 2);
    for (int t = tid; t < n7; t += nth) {
      scl[t] = sg[t];
      bv[t] = bwd == 2 ? sc.rhs[7 * __ldg(pv.ints + G.off_pose + t / 7) + t % 7] : sg[n7 + t];
      xv[t] = 0.0;
    }
    // mode 2: the reciprocal pivots that mode 1 left in the -g slot
    if (bwd == 2)
      for (int t = tid; t < n7; t += nth) ivf[t] = reinterpret_cast<const float*>(sg + n7)[t];
  }
  const int32_t* pose_of_pos = sI;
  const int32_t* col_ptr = sI + (G.off_col - G.off_pose);
  const int32_t* colent = sI + (G.off_colent - G.off_pose);
  const int32_t* T2 = sI + seg1;  // second segment, starting at plan offset off_lev
  const int32_t* asm_ptr = T2 + (G.off_asm - G.off_lev);
  const int32_t* lev_ptr = T2;
  const int32_t* lev_cols = T2 + (G.off_levcols - G.off_lev);
  const int32_t* tptr = T2 + (G.off_tptr - G.off_lev);
  const int32_t* pairs = T2 + (G.off_pairs - G.off_lev);
  const int32_t* levupd = T2 + (G.off_levupd - G.off_lev);
  const int32_t* updlist = T2 + (G.off_updlist - G.off_lev);
  const int32_t* rsptr = T2 + (G.off_rsptr - G.off_lev);
  const int32_t* rs = T2 + (G.off_rs - G.off_lev);
  const double* H64 = ws + G.ws_off;  // assembled FP64 blocks (global, L2-resident)
  if (tid == 0) {
    s_fail = 0;
    s_done = 0;
    s_nonfinite = 0;
    s_zprev = 0.0;
  }
  __syncthreads();
  for (int t = tid; t < n7; t += nth)
    if (!isfinite(scl[t])) s_fail = 1;  // a diagonal entry that is not positive
  __syncthreads();
  if (s_fail) {
    if (tid == 0) handled[g] = 0;
    return;
  }

  // ---- FP32 factorisation of S H S by levels (mode 2 reuses mode 1's)
  for (int l = 0; l < (bwd == 2 ? 0 : G.n_levels); ++l) {
    const int q0 = lev_ptr[l], q1 = lev_ptr[l + 1];
    const int g0 = levupd[l], g1 = levupd[l + 1];  // targets of the level that receive updates
    for (int w = tid; w < (g1 - g0) * 49; w += nth) {
      const int t = updlist[g0 + w / 49], e = w % 49, r = e / 7, c = e % 7;
      const int k1 = tptr[t + 1];
      float s0 = 0.f, s1 = 0.f;
      int k = tptr[t];
      for (; k + 1 < k1; k += 2) {
        s0 += dot8(Lf + kBlk * (size_t)pairs[2 * k] + kRow * r,
                   Lf + kBlk * (size_t)pairs[2 * k + 1] + kRow * c);
        s1 += dot8(Lf + kBlk * (size_t)pairs[2 * k + 2] + kRow * r,
                   Lf + kBlk * (size_t)pairs[2 * k + 3] + kRow * c);
      }
      if (k < k1)
        s0 += dot8(Lf + kBlk * (size_t)pairs[2 * k] + kRow * r,
                   Lf + kBlk * (size_t)pairs[2 * k + 1] + kRow * c);
      Lf[kBlk * (size_t)t + kRow * r + c] -= s0 + s1;
    }
    if (g1 > g0) __syncthreads();
    for (int qi = q0 + warp; qi < q1; qi += nwarps) {
      const int p = lev_cols[qi];
      float* D = Lf + kBlk * (size_t)p;
      const bool mine = lane < 7;
      const int li = mine ? lane : 0;
      float row[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) row[k] = D[kRow * li + k];
      bool bad = false;
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        const float djj = __shfl_sync(0xffffffffu, row[j], j);
        const bool okj = djj > 9.5367431640625e-7f && djj < INFINITY;  // 2^-20 of the unit diagonal
        bad |= !okj;
        const float ivj = rsqrtf(okj ? djj : 1.0f);
        const float lij = (lane == j && !okj) ? 1.0f : row[j] * ivj;
        if (mine && lane >= j) row[j] = lij;
        if (lane == j) ivf[7 * p + j] = ivj;
#pragma unroll
        for (int k = j + 1; k < 7; ++k) {
          const float lkj = __shfl_sync(0xffffffffu, row[j], k);
          if (mine && lane >= k) row[k] = fmaf(-lij, lkj, row[k]);
        }
      }
      if (mine) {
#pragma unroll
        for (int k = 0; k < 7; ++k)
          if (k <= lane) D[kRow * lane + k] = row[k];
      }
      if (bad && lane == 0) s_fail = 1;
      __syncwarp();
      // the same warp forms its column's panel L_rp = A_rp L_pp^-T, one row
      // of a block below the diagonal per lane (no barrier in between)
      const float* iv = ivf + 7 * p;
      for (int ent = col_ptr[p] * 7 + lane; ent < col_ptr[p + 1] * 7; ent += 32) {
        float* prow = Lf + kBlk * (size_t)colent[2 * (ent / 7) + 1] + kRow * (ent % 7);
        float x[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) {
          float v = prow[k];
#pragma unroll
          for (int l2 = 0; l2 < k; ++l2) v = fmaf(-x[l2], D[kRow * k + l2], v);
          x[k] = v * iv[k];
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) prow[k] = x[k];
      }
      __syncwarp();
    }
    __syncthreads();
    if (s_fail) break;
  }
  if (s_fail) {
    if (tid == 0) handled[g] = 0;
    return;
  }
  if (bwd == 1) {
    // keep the factor for mode 2: the shared-memory factor back to the
    // workspace (where the assembly wrote its input) and the reciprocal
    // pivots in the -g slot (read above, no longer needed)
    double* sgw = ws + G.ws_mixed + (size_t)nb * (kLfBlock / 2);
    if (!kGlobalL) {
      float4* dst = reinterpret_cast<float4*>(ws + G.ws_mixed);
      const float4* src = reinterpret_cast<const float4*>(Lf);
      for (int t = tid; t < nb * (kBlk / 4); t += nth) dst[t] = src[t];
    }
    for (int t = tid; t < n7; t += nth) reinterpret_cast<float*>(sgw + n7)[t] = ivf[t];
  }

  // ---- explicit inverses of the diagonal factor blocks: thread (p, k)
  // solves L_pp x = e_k, so that each block step of the triangular solves
  // below is a 7 x 7 product (seven independent sums) instead of a chain of
  // seven dependent shuffles
  for (int t = tid; t < n7; t += nth) {
    const int p = t / 7, k = t % 7;
    const float* D = Lf + kBlk * (size_t)p;
    float x[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      float v = (j == k) ? 1.0f : 0.0f;
#pragma unroll
      for (int i = 0; i < j; ++i) v = (i >= k) ? fmaf(-D[kRow * j + i], x[i], v) : v;
      x[j] = (j >= k) ? v * ivf[7 * p + j] : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 7; ++j) Linv[56 * p + 8 * j + k] = x[j];
  }
  __syncthreads();

  // ---- iterative refinement
  for (int t = tid; t < n7; t += nth) yv[t] = (float)(scl[t] * bv[t]);
  __syncthreads();
  const int grp = lane / 7, ga = lane % 7;  // lanes 0..27: four groups of seven rows
  for (int it = 0; it < kMixMaxIters; ++it) {
    // forward substitution L y' = y, levels ascending, one warp per column;
    // the row gather is split over the four lane groups
    for (int l = 0; l < G.n_levels; ++l) {
      const int q0 = lev_ptr[l], q1 = lev_ptr[l + 1];
      for (int qi = q0 + warp; qi < q1; qi += nwarps) {
        const int p = lev_cols[qi];
        float part = 0.0f;
        if (lane < 28) {
          float ps[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          for (int k = rsptr[p] + grp; k < rsptr[p + 1]; k += 4) {
            const float* Lpc = Lf + kBlk * (size_t)rs[2 * k + 1] + kRow * ga;
            const float* yc = yv + 7 * rs[2 * k];
#pragma unroll
            for (int kk = 0; kk < 7; ++kk) ps[kk] = fmaf(Lpc[kk], yc[kk], ps[kk]);
          }
          part = ((ps[0] + ps[1]) + (ps[2] + ps[3])) + ((ps[4] + ps[5]) + ps[6]);
        }
        const float tot = sum_groups(part);
        const float s = (lane < 7) ? yv[7 * p + lane] - tot : 0.0f;
        // y_p = L_pp^-1 s
        const float* Li = Linv + 56 * p + 8 * (lane < 7 ? lane : 0);
        float out = 0.0f;
#pragma unroll
        for (int k = 0; k < 7; ++k) out = fmaf(Li[k], __shfl_sync(0xffffffffu, s, k), out);
        if (lane < 7) yv[7 * p + lane] = out;
        __syncwarp();
      }
      __syncthreads();
    }
    // back substitution L^T z = y', levels descending; the column gather is
    // split the same way
    for (int l = G.n_levels - 1; l >= 0; --l) {
      const int q0 = lev_ptr[l], q1 = lev_ptr[l + 1];
      for (int qi = q0 + warp; qi < q1; qi += nwarps) {
        const int p = lev_cols[qi];
        float part = 0.0f;
        if (lane < 28) {
          float ps[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          for (int ent = col_ptr[p] + grp; ent < col_ptr[p + 1]; ent += 4) {
            const float* Lr = Lf + kBlk * (size_t)colent[2 * ent + 1];
            const float* xr = yv + 7 * colent[2 * ent];
#pragma unroll
            for (int k = 0; k < 7; ++k) ps[k] = fmaf(Lr[kRow * k + ga], xr[k], ps[k]);
          }
          part = ((ps[0] + ps[1]) + (ps[2] + ps[3])) + ((ps[4] + ps[5]) + ps[6]);
        }
        const float tot = sum_groups(part);
        const float s = (lane < 7) ? yv[7 * p + lane] - tot : 0.0f;
        // z_p = L_pp^-T s
        const float* Li = Linv + 56 * p + (lane < 7 ? lane : 0);
        float xl = 0.0f;
#pragma unroll
        for (int k = 0; k < 7; ++k) xl = fmaf(Li[8 * k], __shfl_sync(0xffffffffu, s, k), xl);
        if (lane < 7) yv[7 * p + lane] = xl;
        __syncwarp();
      }
      __syncthreads();
    }
    // x += S z; the sizes of the correction and of x
    double zmax = 0.0, xmax = 0.0;
    for (int t = tid; t < n7; t += nth) {
      const double z = scl[t] * (double)yv[t];
      const double xn = xv[t] + z;
      xv[t] = xn;
      zmax = fmax(zmax, fabs(z));
      xmax = fmax(xmax, fabs(xn));
      if (!isfinite(z)) s_nonfinite = 1;
    }
    for (int off = 16; off > 0; off >>= 1) {
      zmax = fmax(zmax, __shfl_xor_sync(0xffffffffu, zmax, off));
      xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, off));
    }
    if (tid == 0) {
      s_zmax = 0.0;
      s_xmax = 0.0;
    }
    __syncthreads();
    if (lane == 0) {
      // non-negative doubles order like their bit patterns
      atomicMax(reinterpret_cast<unsigned long long*>(&s_zmax), (unsigned long long)__double_as_longlong(zmax));
      atomicMax(reinterpret_cast<unsigned long long*>(&s_xmax), (unsigned long long)__double_as_longlong(xmax));
    }
    __syncthreads();
    if (tid == 0) {
      const double zm = s_zmax, xm = s_xmax;
      if (s_nonfinite) {
        s_fail = 1;
      } else if (it > 0) {
        const double rho = s_zprev > 0.0 ? zm / s_zprev : 0.0;
        if (zm == 0.0 || rho * zm <= 1e-9 * xm) s_done = 1;
        else if (it > 1 && rho > 0.5) s_fail = 1;  // stalled: leave it to FP64
      } else if (zm == 0.0) {
        s_done = 1;  // b = 0
      }
      s_zprev = zm;
    }
    __syncthreads();
    if (s_done || s_fail) break;
    // residual b - H x in FP64 over the nonzero blocks of H, scaled into y
    for (int i = tid; i < n7; i += nth) {
      const int p = i / 7, a = i % 7;
      double ps[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      {
        const double* Hd = H64 + 49 * (size_t)p + 7 * a;
        const double* xp = xv + 7 * p;
#pragma unroll
        for (int kk = 0; kk < 7; ++kk) ps[kk] = fma(Hd[kk], xp[kk], ps[kk]);
      }
      for (int k = rsptr[p]; k < rsptr[p + 1]; ++k) {
        const int blk = rs[2 * k + 1];
        if (asm_ptr[blk] == asm_ptr[blk + 1]) continue;  // fill: zero in H
        const double* Hb = H64 + 49 * (size_t)blk + 7 * a;
        const double* xc = xv + 7 * rs[2 * k];
#pragma unroll
        for (int kk = 0; kk < 7; ++kk) ps[kk] = fma(Hb[kk], xc[kk], ps[kk]);
      }
      for (int ent = col_ptr[p]; ent < col_ptr[p + 1]; ++ent) {
        const int blk = colent[2 * ent + 1];
        if (asm_ptr[blk] == asm_ptr[blk + 1]) continue;
        const double* Hb = H64 + 49 * (size_t)blk + a;  // H_(p,r) = H_(r,p)^T
        const double* xr = xv + 7 * colent[2 * ent];
#pragma unroll
        for (int kk = 0; kk < 7; ++kk) ps[kk] = fma(Hb[7 * kk], xr[kk], ps[kk]);
      }
      const double r = bv[i] - (((ps[0] + ps[1]) + (ps[2] + ps[3])) + ((ps[4] + ps[5]) + ps[6]));
      yv[i] = (float)(scl[i] * r);
    }
    __syncthreads();
  }
  if (!s_done) {
    if (tid == 0) handled[g] = 0;
    return;
  }
  if (bwd) {
    // the adjoint's solves: x in pose order, nothing else changes
    for (int t = tid; t < n7; t += nth) sc.x_out[7 * (size_t)pose_of_pos[t / 7] + t % 7] = xv[t];
    if (tid < 7) sc.x_out[7 * (size_t)G.gauge + tid] = 0.0;
    if (tid == 0) handled[g] = 1;
    return;
  }

  // ---- step statistics, tau, retraction (as in the FP64 kernel)
  if (warp == 0) {
    double mx = 0.0;
    for (int t = lane; t < n7; t += 32) mx = fmax(mx, fabs(xv[t]));
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) s_max = mx;
  }
  if (tau_out && tid < 7) tau_out[7 * G.gauge + tid] = 0.0;
  // retraction T <- Exp(tau) o T: the transcendental pieces of every pose's
  // Exp are computed by different warps side by side (a warp runs one kind
  // of function for 32 poses), then combined per pose (sim3_exp_parts)
  {
    double* part = reinterpret_cast<double*>(Lf);  // 10 doubles per pose; the factor is no longer needed
    for (int w = warp; w < 8 * ((m + 31) / 32); w += nwarps) {
      const int kind = w & 7, p = (w >> 3) * 32 + lane;
      if (p < m) sim3_exp_piece(xv + 7 * p, kind, part + 10 * p);
    }
    __syncthreads();
    for (int p = tid; p < m; p += nth) {
      const int k = pose_of_pos[p];
      if (tau_out)
        for (int a = 0; a < 7; ++a) tau_out[7 * k + a] = xv[7 * p + a];
      const Sim3d E = sim3_exp_parts(xv + 7 * p, part + 10 * p);
      const Sim3d Tn = compose(E, load_pose(T_wc + 8 * k));
      store_pose(Tn, T_wc + 8 * k);
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (s_max < sc.conv_tol) dev_status[g] = 1;
    handled[g] = 1;
  }
}

// Dynamic shared memory for the solve: the largest graph's factor if it fits
// in the opt-in per-CTA limit, else none (all graphs then use the workspace).
static int smem_limit_bytes() {
  static int limit = -1;
  if (limit < 0) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    limit = std::max(0, optin - 2048);  // headroom for the static shared variables
    cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    cudaFuncSetAttribute(solve_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    cudaFuncSetAttribute(solve_mixed_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    cudaFuncSetAttribute(solve_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
  }
  return limit;
}

static int solve_smem_doubles(const mslam_plan* plan) {
  const int64_t need = plan_max_graph_doubles(plan);
  return (need * (int64_t)sizeof(double) <= smem_limit_bytes()) ? (int)need : 0;
}

// Whether one cluster of kClusterSize CTAs with this much shared memory can
// be resident (asked once per size, outside any stream capture).
static bool cluster_fits(int smem_bytes) {
  static int cached_bytes = -1;
  static bool cached_ok = false;
  if (smem_bytes == cached_bytes) return cached_ok;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterSize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(kClusterSize);
  cfg.blockDim = dim3(kSolveThreads);
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, solve_cluster_kernel, &cfg);
  cudaGetLastError();  // clear a refusal: the single-CTA form is used instead
  cached_bytes = smem_bytes;
  cached_ok = (e == cudaSuccess && n >= 1);
  return cached_ok;
}

// Shared memory of the mixed-precision solve if the plan's largest graph fits
// (0: use the FP64 kernels alone).
static int mixed_smem_bytes(const mslam_plan* plan, bool* global_factor = nullptr) {
  if (global_factor) *global_factor = false;
  if (plan_solve_form(plan) != 0) return 0;
  const int limit = smem_limit_bytes();
  const int64_t need = plan_max_mixed_bytes(plan);
  if (need > 0 && need <= limit) return (int)need;
  // the largest factor does not fit: every graph factors in the workspace
  const int64_t need2 = plan_max_mixed_bytes_nofactor(plan);
  if (need2 > 0 && need2 <= limit) {
    if (global_factor) *global_factor = true;
    return (int)need2;
  }
  return 0;
}

// The per-graph flags of the mixed-precision kernel, after the solve's FP64
// workspace.
static int32_t* solve_flags(const mslam_plan* plan, double* ws) {
  return reinterpret_cast<int32_t*>(reinterpret_cast<char*>(ws) +
                                    ((sizeof(double) * std::max<int64_t>(plan_solve_ws_doubles(plan), 1) + 255) &
                                     ~size_t(255)));
}

static mslam_status launch_solve(const PlanView& pv, SolveConst sc, const float* H, const float* g, double* T,
                                 double* tau, int32_t* st, double* ws, cudaStream_t s) {
  smem_limit_bytes();
  if (sc.smem_doubles > 0 && cluster_fits((int)(sizeof(double) * sc.smem_doubles))) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterSize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(pv.G * kClusterSize);
    cfg.blockDim = dim3(kSolveThreads);
    cfg.dynamicSmemBytes = sizeof(double) * sc.smem_doubles;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cuda_check(cudaLaunchKernelEx(&cfg, solve_cluster_kernel, pv, sc, H, g, T, tau, st, ws),
                      "gn_solve cluster launch");
  }
  solve_kernel<<<pv.G, kSolveThreads, sizeof(double) * sc.smem_doubles, s>>>(pv, sc, H, g, T, tau, st, ws);
  return cuda_check(cudaGetLastError(), "gn_solve launch");
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
  // with no edges the block arrays are empty and may be NULL
  if ((plan_view(plan).E > 0 && (!H_blocks || !g_blocks)) || !T_wc || !dev_status || !workspace) {
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
  sc.smem_doubles = solve_smem_doubles(plan);
  sc.skip = nullptr;
  sc.bwd_mode = 0;
  sc.rhs = nullptr;
  sc.x_out = nullptr;
  sc.handled_in = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* ws = static_cast<double*>(workspace);
  bool global_factor = false;
  const int mixed = mixed_smem_bytes(plan, &global_factor);
  if (mixed > 0 && pv.E > 0) {
    // FP32 factorisation + FP64 refinement first; graphs it declines (or
    // that need no solve) go through the FP64 kernel, which skips the rest
    int32_t* handled = solve_flags(plan, ws);
    const int elems = (int)plan_max_mixed_elems(plan);
    solve_assemble_kernel<<<dim3(std::max(1, (elems + 63) / 64), pv.G), 64, 0, s>>>(pv, H_blocks, g_blocks,
                                                                                     dev_status, ws, 0, global_factor ? 8 : kLfRow);
    if (global_factor)
      solve_mixed_kernel<true><<<pv.G, kMixThreads, mixed, s>>>(pv, sc, T_wc, tau, dev_status, ws, handled);
    else
      solve_mixed_kernel<false><<<pv.G, kMixThreads, mixed, s>>>(pv, sc, T_wc, tau, dev_status, ws, handled);
    mslam_status st = cuda_check(cudaGetLastError(), "gn_solve mixed launch");
    if (st != MSLAM_OK) return st;
    sc.skip = handled;
  }
  return launch_solve(pv, sc, H_blocks, g_blocks, T_wc, tau, dev_status, ws, s);
}

extern "C" int32_t mslam_gn_solve_launches(const mslam_plan* plan) {
  if (!plan) return 0;
  return (mixed_smem_bytes(plan) > 0 && plan_view(plan).E > 0) ? 3 : 1;
}

// Factor every graph's system and write tau = -H^-1 g without updating poses
// (used by the adjoint, which needs the factorisation and the step).
// The adjoint's first solve, tau = -H^-1 g for every graph (converged ones
// included), no pose touched: the mixed-precision kernel in mode 1 (its FP32
// factor kept in the workspace for the second solve) for the graphs it
// accepts, the FP64 factor-only solve for the others.  *mixed tells whether
// the mixed-precision kernel ran (its flags: the solve workspace's).
mslam_status mslam_bwd_solve_tau(const mslam_plan* plan, const float* H_blocks, const float* g_blocks, double* tau,
                                 int32_t* dev_status, double* ws, cudaStream_t s, bool* mixed_used) {
  const PlanView pv = plan_view(plan);
  SolveConst sc;
  sc.conv_tol = 0.0;
  sc.factor_only = 1;
  sc.smem_doubles = solve_smem_doubles(plan);
  sc.skip = nullptr;
  sc.bwd_mode = 0;
  sc.rhs = nullptr;
  sc.x_out = nullptr;
  sc.handled_in = nullptr;
  *mixed_used = false;
  bool global_factor = false;
  const int mixed = mixed_smem_bytes(plan, &global_factor);
  if (mixed > 0 && pv.E > 0) {
    int32_t* handled = solve_flags(plan, ws);
    const int elems = (int)plan_max_mixed_elems(plan);
    solve_assemble_kernel<<<dim3(std::max(1, (elems + 63) / 64), pv.G), 64, 0, s>>>(pv, H_blocks, g_blocks,
                                                                                     dev_status, ws, 1, global_factor ? 8 : kLfRow);
    SolveConst m1 = sc;
    m1.factor_only = 0;
    m1.bwd_mode = 1;
    m1.x_out = tau;
    if (global_factor)
      solve_mixed_kernel<true><<<pv.G, kMixThreads, mixed, s>>>(pv, m1, nullptr, nullptr, dev_status, ws, handled);
    else
      solve_mixed_kernel<false><<<pv.G, kMixThreads, mixed, s>>>(pv, m1, nullptr, nullptr, dev_status, ws, handled);
    mslam_status st = cuda_check(cudaGetLastError(), "gn_backward mixed launch");
    if (st != MSLAM_OK) return st;
    sc.skip = handled;
    *mixed_used = true;
  }
  return launch_solve(pv, sc, H_blocks, g_blocks, nullptr, tau, dev_status, ws, s);
}

// The adjoint's second solve after mslam_bwd_solve_tau used the
// mixed-precision kernel: x = H^-1 rhs by mode 2 with the kept factor
// (handled2[g] = 1 where it succeeded), then for every other graph the FP64
// factor-only solve again (its tau once more, and its FP64 factor for the
// caller's substitution, which skips the graphs flagged in handled2).
mslam_status mslam_bwd_solve_rhs(const mslam_plan* plan, const float* H_blocks, const float* g_blocks,
                                 const double* rhs, double* x, double* tau, int32_t* dev_status, double* ws,
                                 int32_t* handled2, cudaStream_t s) {
  const PlanView pv = plan_view(plan);
  bool global_factor = false;
  const int mixed = mixed_smem_bytes(plan, &global_factor);
  SolveConst sc;
  sc.conv_tol = 0.0;
  sc.factor_only = 0;
  sc.smem_doubles = solve_smem_doubles(plan);
  sc.skip = nullptr;
  sc.bwd_mode = 2;
  sc.rhs = rhs;
  sc.x_out = x;
  sc.handled_in = solve_flags(plan, ws);
  if (global_factor)
    solve_mixed_kernel<true><<<pv.G, kMixThreads, mixed, s>>>(pv, sc, nullptr, nullptr, dev_status, ws, handled2);
  else
    solve_mixed_kernel<false><<<pv.G, kMixThreads, mixed, s>>>(pv, sc, nullptr, nullptr, dev_status, ws, handled2);
  mslam_status st = cuda_check(cudaGetLastError(), "gn_backward mixed launch");
  if (st != MSLAM_OK) return st;
  SolveConst f;
  f.conv_tol = 0.0;
  f.factor_only = 1;
  f.smem_doubles = solve_smem_doubles(plan);
  f.skip = handled2;
  f.bwd_mode = 0;
  f.rhs = nullptr;
  f.x_out = nullptr;
  f.handled_in = nullptr;
  return launch_solve(pv, f, H_blocks, g_blocks, nullptr, tau, dev_status, ws, s);
}

