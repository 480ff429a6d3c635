// (a4-a5) Linearisation of the ray-error cost E_g (Eq. backend_ray) per edge.
//
// Per matched pixel n of edge (i, j): x = T_ij X_j[n], y = X_i[m],
// r = psi(x) - psi(y), r_d = |x| - |y| (Supp. S1.2), whitened by q / sigma^2
// with one Huber IRLS weight per residual group.  The relative Jacobian has
// the structure J_psi = [P/d, -[x]x/d, 0], J_d = [u^T, 0, d] (Supp. S1.2,
// P = I - u u^T, u = x/d), so J^T W J needs only 21 distinct sums:
//   H_tt = S1 I + S2,  H_tw = -[S3]x,  H_ts = S4,  H_ww = S5 I - S6,  H_ss = S7
// with S1 = sum w_r/d^2, S2 = sum (w_d - w_r/d^2) u u^T, S3 = sum w_r x/d^2,
// S4 = sum w_d x, S5 = sum w_r, S6 = sum w_r u u^T, S7 = sum w_d d^2, and
// J^T W r = [w_r (r - u (u.r))/d + w_d r_d u, w_r (x cross r)/d, w_d d r_d].
// Each tile of 4096 pixels reduces its 30 FP32 sums with a fixed tree (per
// thread, warp shuffles, shared memory) into its own workspace slot; a second
// kernel sums an edge's tiles in FP64 in tile order and maps the relative
// 7x7 system to the 14x14 block with Ad_{T_i^-1} (Supp. S1.4).  No atomics:
// the result is bitwise reproducible.
#include <algorithm>

#include "common.cuh"

namespace mslam {

struct RelPose {
  float R[9];  // s R of T_ij
  float t[3];
};

__device__ __forceinline__ void rel_pose_f32(const double* T_wc, int i, int j, RelPose* out) {
  const Sim3d Ti = load_pose(T_wc + 8 * i), Tj = load_pose(T_wc + 8 * j);
  const Sim3d Tij = compose(inverse(Ti), Tj);
  double R[9];
  rot_of(Tij.q, R);
  for (int k = 0; k < 9; ++k) out->R[k] = (float)(Tij.s * R[k]);
  for (int k = 0; k < 3; ++k) out->t[k] = (float)Tij.t[k];
}

__device__ __forceinline__ float huber_w(float e, float delta) { return e <= delta ? 1.0f : __fdividef(delta, e); }
__device__ __forceinline__ float huber_c(float e, float delta) {
  return e <= delta ? 0.5f * e * e : delta * (e - 0.5f * delta);
}

struct LinConst {
  float inv_sr2, inv_sd2, delta, q_min;
};

// Accumulate one match into acc[30].
__device__ __forceinline__ void accumulate(float acc[kNumAcc], const RelPose& P, float3 Xj, float3 y, float qq,
                                           const LinConst& c) {
  const float x0 = fmaf(P.R[0], Xj.x, fmaf(P.R[1], Xj.y, fmaf(P.R[2], Xj.z, P.t[0])));
  const float x1 = fmaf(P.R[3], Xj.x, fmaf(P.R[4], Xj.y, fmaf(P.R[5], Xj.z, P.t[1])));
  const float x2 = fmaf(P.R[6], Xj.x, fmaf(P.R[7], Xj.y, fmaf(P.R[8], Xj.z, P.t[2])));
  const float d2 = fmaf(x0, x0, fmaf(x1, x1, x2 * x2));
  const float dy2 = fmaf(y.x, y.x, fmaf(y.y, y.y, y.z * y.z));
  if (!(d2 > 0.0f && dy2 > 0.0f && d2 < INFINITY && dy2 < INFINITY)) return;
  const float d = sqrtf(d2), dy = sqrtf(dy2);
  const float id = 1.0f / d, idy = 1.0f / dy;
  const float u0 = x0 * id, u1 = x1 * id, u2 = x2 * id;
  const float r0 = u0 - y.x * idy, r1 = u1 - y.y * idy, r2 = u2 - y.z * idy;
  const float rd = d - dy;
  const float lr = qq * c.inv_sr2, ld = qq * c.inv_sd2;
  const float er = sqrtf(lr * fmaf(r0, r0, fmaf(r1, r1, r2 * r2)));
  const float ed = sqrtf(ld) * fabsf(rd);
  const float wr = lr * huber_w(er, c.delta), wd = ld * huber_w(ed, c.delta);
  const float A = wr * id * id;
  acc[0] += A;
  const float cc = wd - A;
  const float cu0 = cc * u0, cu1 = cc * u1, cu2 = cc * u2;
  acc[1] = fmaf(cu0, u0, acc[1]);
  acc[2] = fmaf(cu0, u1, acc[2]);
  acc[3] = fmaf(cu0, u2, acc[3]);
  acc[4] = fmaf(cu1, u1, acc[4]);
  acc[5] = fmaf(cu1, u2, acc[5]);
  acc[6] = fmaf(cu2, u2, acc[6]);
  acc[7] = fmaf(A, x0, acc[7]);
  acc[8] = fmaf(A, x1, acc[8]);
  acc[9] = fmaf(A, x2, acc[9]);
  acc[10] = fmaf(wd, x0, acc[10]);
  acc[11] = fmaf(wd, x1, acc[11]);
  acc[12] = fmaf(wd, x2, acc[12]);
  acc[13] += wr;
  const float wu0 = wr * u0, wu1 = wr * u1, wu2 = wr * u2;
  acc[14] = fmaf(wu0, u0, acc[14]);
  acc[15] = fmaf(wu0, u1, acc[15]);
  acc[16] = fmaf(wu0, u2, acc[16]);
  acc[17] = fmaf(wu1, u1, acc[17]);
  acc[18] = fmaf(wu1, u2, acc[18]);
  acc[19] = fmaf(wu2, u2, acc[19]);
  acc[20] = fmaf(wd, d2, acc[20]);
  const float ur = fmaf(u0, r0, fmaf(u1, r1, u2 * r2));
  const float ad = wr * id, wdr = wd * rd;
  acc[21] = fmaf(ad, fmaf(-u0, ur, r0), fmaf(wdr, u0, acc[21]));
  acc[22] = fmaf(ad, fmaf(-u1, ur, r1), fmaf(wdr, u1, acc[22]));
  acc[23] = fmaf(ad, fmaf(-u2, ur, r2), fmaf(wdr, u2, acc[23]));
  acc[24] = fmaf(ad, x1 * r2 - x2 * r1, acc[24]);
  acc[25] = fmaf(ad, x2 * r0 - x0 * r2, acc[25]);
  acc[26] = fmaf(ad, x0 * r1 - x1 * r0, acc[26]);
  acc[27] = fmaf(wdr, d, acc[27]);
  acc[28] += huber_c(er, c.delta) + huber_c(ed, c.delta);
  acc[29] += 1.0f;
}

constexpr int kUnroll = 4;

template <typename T>
__global__ void __launch_bounds__(kLinThreads) lin_tiles_kernel(PlanView pv, LinConst lc,
                                                                const double* __restrict__ T_wc,
                                                                const T* __restrict__ X,
                                                                const int32_t* __restrict__ idx,
                                                                const T* __restrict__ q,
                                                                float* __restrict__ partials, int tile_begin,
                                                                int tile_end) {
  __shared__ RelPose sP;
  __shared__ float red[kLinThreads / 32][kNumAcc];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int tile = tile_begin + blockIdx.x; tile < tile_end; tile += gridDim.x) {
    const DevTile tl = pv.tiles[tile];
    const DevEdge ed = pv.edges[tl.edge];
    if (tid == 0) rel_pose_f32(T_wc, ed.i, ed.j, &sP);
    __syncthreads();
    const RelPose P = sP;
    float acc[kNumAcc];
#pragma unroll
    for (int a = 0; a < kNumAcc; ++a) acc[a] = 0.0f;
    const int32_t* idx_e = idx + ed.off_e;
    const T* q_e = q + ed.off_e;
    const T* Xj = X + 3 * ed.off_j;
    const T* Xi = X + 3 * ed.off_i;
    for (int base = tl.begin + tid; base < tl.end; base += kUnroll * kLinThreads) {
      int mm[kUnroll];
      float qq[kUnroll];
      float3 xj[kUnroll], yy[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int n = base + u * kLinThreads;
        mm[u] = (n < tl.end) ? __ldg(idx_e + n) : -1;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int n = base + u * kLinThreads;
        qq[u] = 0.0f;
        if (mm[u] >= 0) {
          qq[u] = ldf(q_e + n);
          xj[u] = ld3(Xj, n);
          yy[u] = ld3(Xi, mm[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if (mm[u] >= 0 && qq[u] > lc.q_min) accumulate(acc, P, xj[u], yy[u], qq[u], lc);
    }
    // fixed-order tree: warp shuffles, then the 8 warp sums in order
#pragma unroll
    for (int a = 0; a < kNumAcc; ++a) {
      float v = acc[a];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][a] = v;
    }
    __syncthreads();
    if (tid < kNumAcc) {
      float s = red[0][tid];
#pragma unroll
      for (int w = 1; w < kLinThreads / 32; ++w) s += red[w][tid];
      partials[(size_t)tile * kAccStride + tid] = s;
    }
    __syncthreads();
  }
}

// One block per edge: FP64 sum of the edge's tile partials, then the 14x14.
__global__ void __launch_bounds__(64) lin_finalize_kernel(PlanView pv, const double* __restrict__ T_wc,
                                                          const float* __restrict__ partials,
                                                          float* __restrict__ H14, float* __restrict__ g14,
                                                          double* __restrict__ cost, int32_t* __restrict__ n_valid,
                                                          int e_begin) {
  const int e = e_begin + blockIdx.x;
  const DevEdge ed = pv.edges[e];
  __shared__ double S[kNumAcc];
  __shared__ double Hr[49], A[49], C[49], g[7];
  const int tid = threadIdx.x;
  if (tid < kNumAcc) {
    double s = 0.0;
    for (int t = ed.tile_begin; t < ed.tile_end; ++t) s += (double)partials[(size_t)t * kAccStride + tid];
    S[tid] = s;
  }
  if (tid == 32) {
    const Sim3d Ti = load_pose(T_wc + 8 * ed.i);
    adjoint_of(inverse(Ti), A);
  }
  __syncthreads();
  if (tid == 0) {
    for (int k = 0; k < 49; ++k) Hr[k] = 0.0;
    // H_tt = S1 I + S2
    const double s2[6] = {S[1], S[2], S[3], S[4], S[5], S[6]};
    const int sym[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        Hr[7 * a + b] = (a == b ? S[0] : 0.0) + s2[sym[a][b]];
        Hr[7 * (3 + a) + 3 + b] = (a == b ? S[13] : 0.0) - S[14 + sym[a][b]];
      }
    // H_tw = -[S3]x
    const double s3x = S[7], s3y = S[8], s3z = S[9];
    const double tw[9] = {0.0, s3z, -s3y, -s3z, 0.0, s3x, s3y, -s3x, 0.0};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        Hr[7 * a + 3 + b] = tw[3 * a + b];
        Hr[7 * (3 + b) + a] = tw[3 * a + b];
      }
    for (int a = 0; a < 3; ++a) {
      Hr[7 * a + 6] = S[10 + a];
      Hr[7 * 6 + a] = S[10 + a];
    }
    Hr[48] = S[20];
    for (int a = 0; a < 7; ++a) g[a] = S[21 + a];
    cost[e] = S[28];
    if (n_valid) n_valid[e] = (int32_t)S[29];
  }
  __syncthreads();
  // C = Hr A, then B = A^T C
  if (tid < 49) {
    const int r = tid / 7, c = tid % 7;
    double s = 0.0;
    for (int k = 0; k < 7; ++k) s += Hr[7 * r + k] * A[7 * k + c];
    C[tid] = s;
  }
  __syncthreads();
  if (tid < 49) {
    const int r = tid / 7, c = tid % 7;
    double s = 0.0;
    for (int k = 0; k < 7; ++k) s += A[7 * k + r] * C[7 * k + c];
    const float b = (float)s;
    float* Hb = H14 + (size_t)e * 196;
    Hb[14 * r + c] = b;
    Hb[14 * (7 + r) + 7 + c] = b;
    Hb[14 * r + 7 + c] = -b;
    Hb[14 * (7 + r) + c] = -b;
  }
  if (tid >= 49 && tid < 56) {
    const int r = tid - 49;
    double s = 0.0;
    for (int k = 0; k < 7; ++k) s += A[7 * k + r] * g[k];
    g14[(size_t)e * 14 + r] = (float)(-s);
    g14[(size_t)e * 14 + 7 + r] = (float)s;
  }
}

static int lin_grid_blocks() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, lin_tiles_kernel<float>, kLinThreads, 0);
    cached = std::max(1, sms) * std::max(1, per);
  }
  return cached;
}

}  // namespace mslam

using namespace mslam;

extern "C" mslam_status mslam_gn_linearize(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt,
                                           const double* T_wc, const void* X_canon, const int32_t* idx,
                                           const void* q, float* H_blocks, float* g_blocks, double* cost,
                                           int32_t* n_valid, void* workspace, size_t ws_bytes, uint32_t flags,
                                           void* stream) {
  if (!p || !check_plan_uploaded(plan)) {
    if (!p) set_error("params is NULL");
    return MSLAM_ERR_ARG;
  }
  if (dt != MSLAM_F32 && dt != MSLAM_F16) {
    set_error("unsupported dtype %d", (int)dt);
    return MSLAM_ERR_ARG;
  }
  if (!T_wc || !X_canon || !idx || !q || !H_blocks || !g_blocks || !cost || !workspace) {
    set_error("gn_linearize: NULL device pointer");
    return MSLAM_ERR_ARG;
  }
  if (ws_bytes < mslam_workspace_bytes(plan, MSLAM_OP_LINEARIZE) ||
      (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    set_error("gn_linearize: workspace smaller than %zu bytes or not 256-byte aligned",
              mslam_workspace_bytes(plan, MSLAM_OP_LINEARIZE));
    return MSLAM_ERR_ARG;
  }
  if (!(p->sigma_ray > 0.0f) || !(p->sigma_dist > 0.0f) || !(p->huber_delta > 0.0f)) {
    set_error("gn_linearize: sigma_ray, sigma_dist and huber_delta must be positive");
    return MSLAM_ERR_ARG;
  }
  const PlanView pv = plan_view(plan);
  if (pv.E == 0) return MSLAM_OK;
  LinConst lc;
  lc.inv_sr2 = 1.0f / (p->sigma_ray * p->sigma_ray);
  lc.inv_sd2 = 1.0f / (p->sigma_dist * p->sigma_dist);
  lc.delta = p->huber_delta;
  lc.q_min = p->q_min;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* partials = static_cast<float*>(workspace);
  if (flags & MSLAM_FLAG_PER_EDGE) {
    // plain form: a host loop of per-edge launches
    for (int e = 0; e < pv.E; ++e) {
      int t0, t1;
      plan_edge_tiles(plan, e, &t0, &t1);
      if (dt == MSLAM_F32)
        lin_tiles_kernel<float><<<t1 - t0, kLinThreads, 0, s>>>(pv, lc, T_wc, static_cast<const float*>(X_canon),
                                                               idx, static_cast<const float*>(q), partials, t0, t1);
      else
        lin_tiles_kernel<__half><<<t1 - t0, kLinThreads, 0, s>>>(pv, lc, T_wc,
                                                                static_cast<const __half*>(X_canon), idx,
                                                                static_cast<const __half*>(q), partials, t0, t1);
      lin_finalize_kernel<<<1, 64, 0, s>>>(pv, T_wc, partials, H_blocks, g_blocks, cost, n_valid, e);
    }
  } else {
    const int grid = std::min(pv.n_tiles, lin_grid_blocks());
    if (dt == MSLAM_F32)
      lin_tiles_kernel<float><<<grid, kLinThreads, 0, s>>>(pv, lc, T_wc, static_cast<const float*>(X_canon), idx,
                                                          static_cast<const float*>(q), partials, 0, pv.n_tiles);
    else
      lin_tiles_kernel<__half><<<grid, kLinThreads, 0, s>>>(pv, lc, T_wc, static_cast<const __half*>(X_canon),
                                                           idx, static_cast<const __half*>(q), partials, 0,
                                                           pv.n_tiles);
    lin_finalize_kernel<<<pv.E, 64, 0, s>>>(pv, T_wc, partials, H_blocks, g_blocks, cost, n_valid, 0);
  }
  return cuda_check(cudaGetLastError(), "gn_linearize launch");
}
