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
  float pad[4];
};

// T_ij = T_i^-1 T_j of every edge in FP64, stored as float s R and t: one
// thread per edge, once per linearisation (keeps FP64 out of the tile loop).
__global__ void rel_pose_kernel(PlanView pv, const double* __restrict__ T_wc, RelPose* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= pv.E) return;
  const DevEdge ed = pv.edges[e];
  const Sim3d Ti = load_pose(T_wc + 8 * ed.i), Tj = load_pose(T_wc + 8 * ed.j);
  const Sim3d Tij = compose(inverse(Ti), Tj);
  double R[9];
  rot_of(Tij.q, R);
  RelPose P;
  for (int k = 0; k < 9; ++k) P.R[k] = (float)(Tij.s * R[k]);
  for (int k = 0; k < 3; ++k) P.t[k] = (float)Tij.t[k];
  for (int k = 0; k < 4; ++k) P.pad[k] = 0.0f;
  out[e] = P;
}

__device__ __forceinline__ float huber_w(float e, float delta) { return e <= delta ? 1.0f : __fdividef(delta, e); }
__device__ __forceinline__ float huber_c(float e, float delta) {
  return e <= delta ? 0.5f * e * e : delta * (e - 0.5f * delta);
}

struct LinConst {
  float inv_sr2, inv_sd2, delta, delta2, q_min;
};

// Accumulate one match into acc[30].  Normalisation uses the hardware
// reciprocal square root (max error 2 ulp) and the Huber branch needs no
// square root in its quadratic region; the errors this adds are far below
// the FP32 rounding of the residual itself.
template <bool kCheckFinite>
__device__ __forceinline__ void accumulate(float acc[kNumAcc], const RelPose& P, float3 Xj, float3 y, float qq,
                                           const LinConst& c) {
  const float x0 = fmaf(P.R[0], Xj.x, fmaf(P.R[1], Xj.y, fmaf(P.R[2], Xj.z, P.t[0])));
  const float x1 = fmaf(P.R[3], Xj.x, fmaf(P.R[4], Xj.y, fmaf(P.R[5], Xj.z, P.t[1])));
  const float x2 = fmaf(P.R[6], Xj.x, fmaf(P.R[7], Xj.y, fmaf(P.R[8], Xj.z, P.t[2])));
  const float d2 = fmaf(x0, x0, fmaf(x1, x1, x2 * x2));
  const float dy2 = fmaf(y.x, y.x, fmaf(y.y, y.y, y.z * y.z));
  if (kCheckFinite) {
    if (!(d2 > 0.0f && dy2 > 0.0f && d2 < INFINITY && dy2 < INFINITY)) return;
  } else {
    if (!(d2 > 0.0f)) return;  // packed records are finite and non-zero already
  }
  const float id = rsqrtf(d2), idy = rsqrtf(dy2);
  const float d = d2 * id, dy = dy2 * idy;
  const float u0 = x0 * id, u1 = x1 * id, u2 = x2 * id;
  const float r0 = u0 - y.x * idy, r1 = u1 - y.y * idy, r2 = u2 - y.z * idy;
  const float rd = d - dy;
  const float lr = qq * c.inv_sr2, ld = qq * c.inv_sd2;
  const float er2 = lr * fmaf(r0, r0, fmaf(r1, r1, r2 * r2));
  const float ed2 = ld * rd * rd;
  // Huber: e <= delta -> weight 1, cost e^2/2; else weight delta/e, cost delta (e - delta/2)
  float wr = lr, wd = ld, cost = 0.5f * (er2 + ed2);
  if (er2 > c.delta2) {
    const float ir = rsqrtf(er2);
    wr = lr * c.delta * ir;
    cost += c.delta * (er2 * ir - 0.5f * c.delta) - 0.5f * er2;
  }
  if (ed2 > c.delta2) {
    const float ie = rsqrtf(ed2);
    wd = ld * c.delta * ie;
    cost += c.delta * (ed2 * ie - 0.5f * c.delta) - 0.5f * ed2;
  }
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
  acc[28] += cost;
  acc[29] += 1.0f;
}

#ifndef MSLAM_LIN_UNROLL
#define MSLAM_LIN_UNROLL 4
#endif
#ifndef MSLAM_LIN_MINBLOCKS
#define MSLAM_LIN_MINBLOCKS 2
#endif
constexpr int kUnroll = MSLAM_LIN_UNROLL;  // pixels per thread in flight

template <typename T>
__global__ void __launch_bounds__(kLinThreads, MSLAM_LIN_MINBLOCKS)
    lin_tiles_kernel(PlanView pv, LinConst lc, const RelPose* __restrict__ rel, const T* __restrict__ X,
                     const int32_t* __restrict__ idx, const T* __restrict__ q, float* __restrict__ partials,
                     int tile_begin, int tile_end) {
  __shared__ float red[kLinThreads / 32][kNumAcc];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int tile = tile_begin + blockIdx.x; tile < tile_end; tile += gridDim.x) {
    const DevTile tl = pv.tiles[tile];
    const DevEdge ed = pv.edges[tl.edge];
    RelPose P;
    {
      const float4* src = reinterpret_cast<const float4*>(rel + tl.edge);
      float4 a = __ldg(src), b = __ldg(src + 1), c = __ldg(src + 2);
      P.R[0] = a.x; P.R[1] = a.y; P.R[2] = a.z; P.R[3] = a.w;
      P.R[4] = b.x; P.R[5] = b.y; P.R[6] = b.z; P.R[7] = b.w;
      P.R[8] = c.x; P.t[0] = c.y; P.t[1] = c.z; P.t[2] = c.w;
    }
    float acc[kNumAcc];
#pragma unroll
    for (int a = 0; a < kNumAcc; ++a) acc[a] = 0.0f;
    const int32_t* idx_e = idx + ed.off_e;
    const T* q_e = q + ed.off_e;
    const T* Xj = X + 3 * ed.off_j;
    const T* Xi = X + 3 * ed.off_i;
    // software pipeline: the match indices of group g + 1 are loaded while the
    // gathers of group g are in flight, so each group costs one round trip
    int mnext[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int n = tl.begin + tid + u * kLinThreads;
      mnext[u] = (n < tl.end) ? __ldg(idx_e + n) : -1;
    }
    for (int base = tl.begin + tid; base < tl.end; base += kUnroll * kLinThreads) {
      int mm[kUnroll];
      float qq[kUnroll];
      float3 xj[kUnroll], yy[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int n = base + u * kLinThreads;
        mm[u] = mnext[u];
        qq[u] = 0.0f;
        if (mm[u] >= 0) {
          qq[u] = ldf(q_e + n);
          xj[u] = ld3(Xj, n);
          yy[u] = ld3(Xi, mm[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int n = base + (kUnroll + u) * kLinThreads;
        mnext[u] = (n < tl.end) ? __ldg(idx_e + n) : -1;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if (mm[u] >= 0 && qq[u] > lc.q_min) accumulate<true>(acc, P, xj[u], yy[u], qq[u], lc);
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

// ---------------------------------------------------------------- packed form
// The matches are fixed during the Gauss-Newton loop, so the gather of the
// canonical points at the matches is done once: mslam_gn_pack writes, for
// every tile, the matches that pass the q_min test as records in pixel order
// (deterministic) -- FP16: one 16-byte record {X_j[n], X_i[m], q, 0} in
// halves; FP32: two 16-byte float4 {X_j[n], X_i[m].x}, {X_i[m].yz, q, 0} --
// plus a per-tile count.  The packed linearisation then streams the records
// with coalesced 16-byte loads and no dependent loads.

#ifndef MSLAM_PACKED_MINBLOCKS
#define MSLAM_PACKED_MINBLOCKS 2
#endif
#ifndef MSLAM_PACKED_UNROLL
#define MSLAM_PACKED_UNROLL 4
#endif

template <typename T> struct PackRec;
template <> struct PackRec<__half> {
  static constexpr int kWords = 1;  // uint4 per record
  static __device__ __forceinline__ void store(uint4* dst, float3 xj, float3 y, float qq) {
    __half2 a = __floats2half2_rn(xj.x, xj.y), b = __floats2half2_rn(xj.z, y.x), c = __floats2half2_rn(y.y, y.z),
            d = __floats2half2_rn(qq, 0.0f);
    uint4 v;
    v.x = *reinterpret_cast<uint32_t*>(&a);
    v.y = *reinterpret_cast<uint32_t*>(&b);
    v.z = *reinterpret_cast<uint32_t*>(&c);
    v.w = *reinterpret_cast<uint32_t*>(&d);
    dst[0] = v;
  }
  static __device__ __forceinline__ void load(const uint4* src, float3& xj, float3& y, float& qq) {
    const uint4 v = __ldg(src);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    const float2 c = __half22float2(*reinterpret_cast<const __half2*>(&v.z));
    const float2 d = __half22float2(*reinterpret_cast<const __half2*>(&v.w));
    xj = make_float3(a.x, a.y, b.x);
    y = make_float3(b.y, c.x, c.y);
    qq = d.x;
  }
};
template <> struct PackRec<float> {
  static constexpr int kWords = 2;
  static __device__ __forceinline__ void store(uint4* dst, float3 xj, float3 y, float qq) {
    float4* d = reinterpret_cast<float4*>(dst);
    d[0] = make_float4(xj.x, xj.y, xj.z, y.x);
    d[1] = make_float4(y.y, y.z, qq, 0.0f);
  }
  static __device__ __forceinline__ void load(const uint4* src, float3& xj, float3& y, float& qq) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    const float4 a = __ldg(s4), b = __ldg(s4 + 1);
    xj = make_float3(a.x, a.y, a.z);
    y = make_float3(a.w, b.x, b.y);
    qq = b.z;
  }
};

// The storage values are copied bit for bit (FP16 -> float -> FP16 is exact).
template <typename T>
__global__ void __launch_bounds__(kLinThreads) pack_kernel(PlanView pv, float q_min, const T* __restrict__ X,
                                                           const int32_t* __restrict__ idx, const T* __restrict__ q,
                                                           uint4* __restrict__ recs, int32_t* __restrict__ counts) {
  __shared__ int warp_tot[kLinThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int W = PackRec<T>::kWords;
  for (int tile = blockIdx.x; tile < pv.n_tiles; tile += gridDim.x) {
    const DevTile tl = pv.tiles[tile];
    const DevEdge ed = pv.edges[tl.edge];
    const int32_t* idx_e = idx + ed.off_e;
    const T* q_e = q + ed.off_e;
    const T* Xj = X + 3 * ed.off_j;
    const T* Xi = X + 3 * ed.off_i;
    uint4* out = recs + (size_t)tile * pv.lin_tile * W;
    int base_count = 0;
    for (int base = tl.begin; base < tl.end; base += kLinThreads) {
      const int n = base + tid;
      int m = -1;
      float qq = 0.0f;
      if (n < tl.end) {
        m = __ldg(idx_e + n);
        if (m >= 0) qq = ldf(q_e + n);
      }
      bool valid = m >= 0 && qq > q_min;
      float3 xj = make_float3(0.f, 0.f, 0.f), y = xj;
      if (valid) {
        xj = ld3(Xj, n);
        y = ld3(Xi, m);
        // a degenerate point contributes nothing (as in the gathering form)
        const float a2 = xj.x * xj.x + xj.y * xj.y + xj.z * xj.z, b2 = y.x * y.x + y.y * y.y + y.z * y.z;
        valid = a2 > 0.0f && b2 > 0.0f && a2 < INFINITY && b2 < INFINITY;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, valid);
      const int rank = __popc(bal & ((1u << lane) - 1u));
      if (lane == 0) warp_tot[warp] = __popc(bal);
      __syncthreads();
      int off = base_count;
      for (int w = 0; w < warp; ++w) off += warp_tot[w];
      int tot = 0;
      for (int w = 0; w < kLinThreads / 32; ++w) tot += warp_tot[w];
      if (valid) PackRec<T>::store(out + (size_t)(off + rank) * W, xj, y, qq);
      base_count += tot;
      __syncthreads();
    }
    if (tid == 0) counts[tile] = base_count;
  }
}

template <typename T>
__global__ void __launch_bounds__(kLinThreads, MSLAM_PACKED_MINBLOCKS) lin_packed_kernel(PlanView pv, LinConst lc,
                                                                   const RelPose* __restrict__ rel,
                                                                   const uint4* __restrict__ recs,
                                                                   const int32_t* __restrict__ counts,
                                                                   float* __restrict__ partials, int tile_begin,
                                                                   int tile_end) {
  __shared__ float red[kLinThreads / 32][kNumAcc];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int W = PackRec<T>::kWords;
  constexpr int U = MSLAM_PACKED_UNROLL;
  for (int tile = tile_begin + blockIdx.x; tile < tile_end; tile += gridDim.x) {
    const DevTile tl = pv.tiles[tile];
    RelPose P;
    {
      const float4* src = reinterpret_cast<const float4*>(rel + tl.edge);
      float4 a = __ldg(src), b = __ldg(src + 1), c = __ldg(src + 2);
      P.R[0] = a.x; P.R[1] = a.y; P.R[2] = a.z; P.R[3] = a.w;
      P.R[4] = b.x; P.R[5] = b.y; P.R[6] = b.z; P.R[7] = b.w;
      P.R[8] = c.x; P.t[0] = c.y; P.t[1] = c.z; P.t[2] = c.w;
    }
    float acc[kNumAcc];
#pragma unroll
    for (int a = 0; a < kNumAcc; ++a) acc[a] = 0.0f;
    const int cnt = __ldg(counts + tile);
    const uint4* in = recs + (size_t)tile * pv.lin_tile * W;
    for (int r0 = tid; r0 < cnt; r0 += U * kLinThreads) {
      float3 xj[U], yy[U];
      float qq[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = r0 + u * kLinThreads;
        qq[u] = 0.0f;
        if (r < cnt) PackRec<T>::load(in + (size_t)r * W, xj[u], yy[u], qq[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (r0 + u * kLinThreads < cnt) accumulate<false>(acc, P, xj[u], yy[u], qq[u], lc);
    }
#pragma unroll
    for (int a = 0; a < kNumAcc; ++a) {
      float v = acc[a];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][a] = v;
    }
    __syncthreads();
    if (tid < kNumAcc) {
      float sum = red[0][tid];
#pragma unroll
      for (int w = 1; w < kLinThreads / 32; ++w) sum += red[w][tid];
      partials[(size_t)tile * kAccStride + tid] = sum;
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

// Blocks of a persistent linearisation launch: the plan's blocks per SM, or
// the occupancy maximum of the kernel.
template <typename K>
static int persistent_grid(const mslam_plan* plan, K kernel) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kLinThreads, 0);
  const int want = plan_lin_blocks_per_sm(plan);
  if (want > 0) per = std::min(std::max(per, 1), want);
  return std::max(1, sms) * std::max(1, per);
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
  if (plan_view(plan).E == 0) return MSLAM_OK;  // nothing to linearise; outputs are empty
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
  lc.delta2 = p->huber_delta * p->huber_delta;
  lc.q_min = p->q_min;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* partials = static_cast<float*>(workspace);
  RelPose* rel = reinterpret_cast<RelPose*>(static_cast<char*>(workspace) + lin_partials_bytes(pv.n_tiles));
  rel_pose_kernel<<<(pv.E + 127) / 128, 128, 0, s>>>(pv, T_wc, rel);
  if (flags & MSLAM_FLAG_PER_EDGE) {
    // plain form: a host loop of per-edge launches
    for (int e = 0; e < pv.E; ++e) {
      int t0, t1;
      plan_edge_tiles(plan, e, &t0, &t1);
      if (dt == MSLAM_F32)
        lin_tiles_kernel<float><<<t1 - t0, kLinThreads, 0, s>>>(pv, lc, rel, static_cast<const float*>(X_canon),
                                                               idx, static_cast<const float*>(q), partials, t0, t1);
      else
        lin_tiles_kernel<__half><<<t1 - t0, kLinThreads, 0, s>>>(pv, lc, rel,
                                                                static_cast<const __half*>(X_canon), idx,
                                                                static_cast<const __half*>(q), partials, t0, t1);
      lin_finalize_kernel<<<1, 64, 0, s>>>(pv, T_wc, partials, H_blocks, g_blocks, cost, n_valid, e);
    }
  } else {
    const int grid = std::min(pv.n_tiles, persistent_grid(plan, lin_tiles_kernel<float>));
    if (dt == MSLAM_F32)
      lin_tiles_kernel<float><<<grid, kLinThreads, 0, s>>>(pv, lc, rel, static_cast<const float*>(X_canon), idx,
                                                          static_cast<const float*>(q), partials, 0, pv.n_tiles);
    else
      lin_tiles_kernel<__half><<<grid, kLinThreads, 0, s>>>(pv, lc, rel, static_cast<const __half*>(X_canon),
                                                           idx, static_cast<const __half*>(q), partials, 0,
                                                           pv.n_tiles);
    lin_finalize_kernel<<<pv.E, 64, 0, s>>>(pv, T_wc, partials, H_blocks, g_blocks, cost, n_valid, 0);
  }
  return cuda_check(cudaGetLastError(), "gn_linearize launch");
}

static size_t pack_record_bytes(mslam_dtype dt) { return dt == MSLAM_F16 ? 16 : 32; }

namespace mslam {
size_t pack_bytes(int n_tiles, int lin_tile, mslam_dtype dt) {
  const size_t recs = ((size_t)(n_tiles > 0 ? n_tiles : 1) * lin_tile * pack_record_bytes(dt) + 255) & ~size_t(255);
  const size_t cnts = ((size_t)(n_tiles > 0 ? n_tiles : 1) * sizeof(int32_t) + 255) & ~size_t(255);
  return recs + cnts;
}
}  // namespace mslam

extern "C" mslam_status mslam_gn_pack(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt,
                                      const void* X_canon, const int32_t* idx, const void* q, void* packed,
                                      size_t packed_bytes, void* stream) {
  if (!p || !check_plan_uploaded(plan)) {
    if (!p) set_error("params is NULL");
    return MSLAM_ERR_ARG;
  }
  if (dt != MSLAM_F32 && dt != MSLAM_F16) {
    set_error("unsupported dtype %d", (int)dt);
    return MSLAM_ERR_ARG;
  }
  const PlanView pv = plan_view(plan);
  if (pv.E == 0) return MSLAM_OK;
  if (!X_canon || !idx || !q || !packed) {
    set_error("gn_pack: NULL device pointer");
    return MSLAM_ERR_ARG;
  }
  if (packed_bytes < pack_bytes(pv.n_tiles, pv.lin_tile, dt) || (reinterpret_cast<uintptr_t>(packed) & 255)) {
    set_error("gn_pack: packed buffer smaller than %zu bytes or not 256-byte aligned", pack_bytes(pv.n_tiles, pv.lin_tile, dt));
    return MSLAM_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint4* recs = static_cast<uint4*>(packed);
  int32_t* counts = reinterpret_cast<int32_t*>(static_cast<char*>(packed) + pack_bytes(pv.n_tiles, pv.lin_tile, dt) -
                                               (((size_t)pv.n_tiles * sizeof(int32_t) + 255) & ~size_t(255)));
  if (dt == MSLAM_F32)
    pack_kernel<float><<<pv.n_tiles, kLinThreads, 0, s>>>(pv, p->q_min, static_cast<const float*>(X_canon), idx,
                                                          static_cast<const float*>(q), recs, counts);
  else
    pack_kernel<__half><<<pv.n_tiles, kLinThreads, 0, s>>>(pv, p->q_min, static_cast<const __half*>(X_canon), idx,
                                                           static_cast<const __half*>(q), recs, counts);
  return cuda_check(cudaGetLastError(), "gn_pack launch");
}

extern "C" mslam_status mslam_gn_linearize_packed(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt,
                                                  const double* T_wc, const void* packed, size_t packed_bytes,
                                                  float* H_blocks, float* g_blocks, double* cost, int32_t* n_valid,
                                                  void* workspace, size_t ws_bytes, uint32_t flags, void* stream) {
  if (!p || !check_plan_uploaded(plan)) {
    if (!p) set_error("params is NULL");
    return MSLAM_ERR_ARG;
  }
  if (dt != MSLAM_F32 && dt != MSLAM_F16) {
    set_error("unsupported dtype %d", (int)dt);
    return MSLAM_ERR_ARG;
  }
  const PlanView pv = plan_view(plan);
  if (pv.E == 0) return MSLAM_OK;
  if (!T_wc || !packed || !H_blocks || !g_blocks || !cost || !workspace) {
    set_error("gn_linearize_packed: NULL device pointer");
    return MSLAM_ERR_ARG;
  }
  if (packed_bytes < pack_bytes(pv.n_tiles, pv.lin_tile, dt) || (reinterpret_cast<uintptr_t>(packed) & 255)) {
    set_error("gn_linearize_packed: packed buffer smaller than %zu bytes or not 256-byte aligned",
              pack_bytes(pv.n_tiles, pv.lin_tile, dt));
    return MSLAM_ERR_ARG;
  }
  if (ws_bytes < mslam_workspace_bytes(plan, MSLAM_OP_LINEARIZE) ||
      (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    set_error("gn_linearize_packed: workspace smaller than %zu bytes or not 256-byte aligned",
              mslam_workspace_bytes(plan, MSLAM_OP_LINEARIZE));
    return MSLAM_ERR_ARG;
  }
  if (!(p->sigma_ray > 0.0f) || !(p->sigma_dist > 0.0f) || !(p->huber_delta > 0.0f)) {
    set_error("gn_linearize_packed: sigma_ray, sigma_dist and huber_delta must be positive");
    return MSLAM_ERR_ARG;
  }
  LinConst lc;
  lc.inv_sr2 = 1.0f / (p->sigma_ray * p->sigma_ray);
  lc.inv_sd2 = 1.0f / (p->sigma_dist * p->sigma_dist);
  lc.delta = p->huber_delta;
  lc.delta2 = p->huber_delta * p->huber_delta;
  lc.q_min = p->q_min;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* partials = static_cast<float*>(workspace);
  RelPose* rel = reinterpret_cast<RelPose*>(static_cast<char*>(workspace) + lin_partials_bytes(pv.n_tiles));
  const uint4* recs = static_cast<const uint4*>(packed);
  const int32_t* counts = reinterpret_cast<const int32_t*>(
      static_cast<const char*>(packed) + pack_bytes(pv.n_tiles, pv.lin_tile, dt) -
      (((size_t)pv.n_tiles * sizeof(int32_t) + 255) & ~size_t(255)));
  rel_pose_kernel<<<(pv.E + 127) / 128, 128, 0, s>>>(pv, T_wc, rel);
  auto launch = [&](int grid, int t0, int t1) {
    if (dt == MSLAM_F32)
      lin_packed_kernel<float><<<grid, kLinThreads, 0, s>>>(pv, lc, rel, recs, counts, partials, t0, t1);
    else
      lin_packed_kernel<__half><<<grid, kLinThreads, 0, s>>>(pv, lc, rel, recs, counts, partials, t0, t1);
  };
  if (flags & MSLAM_FLAG_PER_EDGE) {
    for (int e = 0; e < pv.E; ++e) {
      int t0, t1;
      plan_edge_tiles(plan, e, &t0, &t1);
      launch(t1 - t0, t0, t1);
      lin_finalize_kernel<<<1, 64, 0, s>>>(pv, T_wc, partials, H_blocks, g_blocks, cost, n_valid, e);
    }
  } else {
    launch(std::min(pv.n_tiles, persistent_grid(plan, lin_packed_kernel<__half>)), 0, pv.n_tiles);
    lin_finalize_kernel<<<pv.E, 64, 0, s>>>(pv, T_wc, partials, H_blocks, g_blocks, cost, n_valid, 0);
  }
  return cuda_check(cudaGetLastError(), "gn_linearize_packed launch");
}
