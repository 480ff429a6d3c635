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
#include <cmath>
#include <mutex>
#include <type_traits>

#include "common.cuh"

namespace mslam {

struct RelPose {
  float R[9];  // s R of T_ij
  float t[3];
  float pad[4];
};

// T_ij = T_i^-1 T_j of every edge in FP64, stored as float s R and t: one
// thread per edge, once per linearisation (keeps FP64 out of the tile loop).
// It also clears the tile counter of the persistent launch that follows.
__global__ void rel_pose_kernel(PlanView pv, const double* __restrict__ T_wc, RelPose* __restrict__ out,
                                int* __restrict__ tile_ctr) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0 && tile_ctr) *tile_ctr = 0;
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
  float inv_s1, inv_s2;  // point: 1/sigma_p^2; pixel: 1/sigma_Pi^2 and 1/sigma_depth^2
  float fx, fy, cx, cy;  // pinhole K of the pixel family
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
  const float id = rsqrt_ftz(d2), idy = rsqrt_ftz(dy2);
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
    const float ir = rsqrt_ftz(er2);
    wr = lr * c.delta * ir;
    cost += c.delta * (er2 * ir - 0.5f * c.delta) - 0.5f * er2;
  }
  if (ed2 > c.delta2) {
    const float ie = rsqrt_ftz(ed2);
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

// ------------------------------------------------------------ other families
// Point (Eq. track_point, Supp. S1.1) and calibrated pixel + depth (Sec. 3.6,
// Eq. backend_pixel, Supp. S1.3) residuals: three rows J_k of the relative
// Jacobian (dr/dx)[I, -[x]x, x], each a 3-vector a and its rotation part
// x cross a, with weights w_k, accumulated as the 28 upper-triangle entries
// of sum w_k J_k^T J_k, the 7 entries of sum w_k J_k r_k, the cost and the
// count.  For the pixel family y = (u_m, v_m, depth of X_i[m]).
__device__ __forceinline__ void add_rows(float acc[kFamAcc], const float J[3][7], const float w[3], const float r[3]) {
  float wJ[3][7];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int a = 0; a < 7; ++a) wJ[k][a] = w[k] * J[k][a];
  int t = 0;
#pragma unroll
  for (int a = 0; a < 7; ++a)
#pragma unroll
    for (int b = a; b < 7; ++b, ++t) acc[t] = fmaf(wJ[0][a], J[0][b], fmaf(wJ[1][a], J[1][b], fmaf(wJ[2][a], J[2][b], acc[t])));
#pragma unroll
  for (int a = 0; a < 7; ++a) acc[28 + a] = fmaf(wJ[0][a], r[0], fmaf(wJ[1][a], r[1], fmaf(wJ[2][a], r[2], acc[28 + a])));
}

__device__ __forceinline__ void row_of(float J[7], float a0, float a1, float a2, float x0, float x1, float x2, float s) {
  J[0] = a0;
  J[1] = a1;
  J[2] = a2;
  J[3] = x1 * a2 - x2 * a1;  // x cross a
  J[4] = x2 * a0 - x0 * a2;
  J[5] = x0 * a1 - x1 * a0;
  J[6] = s;
}

__device__ __forceinline__ float huber_apply(float e2, float lam, const LinConst& c, float* cost) {
  // Huber on a whitened squared norm e2: returns the IRLS weight times lam
  if (e2 <= c.delta2) {
    *cost += 0.5f * e2;
    return lam;
  }
  const float ie = rsqrt_ftz(e2);
  *cost += c.delta * (e2 * ie - 0.5f * c.delta);
  return lam * c.delta * ie;
}

template <int kKind>
__device__ __forceinline__ void accumulate_family(float acc[kFamAcc], const RelPose& P, float3 Xj, float3 y, float qq,
                                                  const LinConst& c) {
  const float x0 = fmaf(P.R[0], Xj.x, fmaf(P.R[1], Xj.y, fmaf(P.R[2], Xj.z, P.t[0])));
  const float x1 = fmaf(P.R[3], Xj.x, fmaf(P.R[4], Xj.y, fmaf(P.R[5], Xj.z, P.t[1])));
  const float x2 = fmaf(P.R[6], Xj.x, fmaf(P.R[7], Xj.y, fmaf(P.R[8], Xj.z, P.t[2])));
  const float d2 = fmaf(x0, x0, fmaf(x1, x1, x2 * x2));
  if (!(d2 > 0.0f && d2 < INFINITY)) return;
  float J[3][7], r[3], w[3], cost = 0.0f;
  if (kKind == MSLAM_RES_POINT) {
    r[0] = x0 - y.x;
    r[1] = x1 - y.y;
    r[2] = x2 - y.z;
    const float lp = qq * c.inv_s1;
    w[0] = w[1] = w[2] = huber_apply(lp * fmaf(r[0], r[0], fmaf(r[1], r[1], r[2] * r[2])), lp, c, &cost);
    row_of(J[0], 1.0f, 0.0f, 0.0f, x0, x1, x2, x0);
    row_of(J[1], 0.0f, 1.0f, 0.0f, x0, x1, x2, x1);
    row_of(J[2], 0.0f, 0.0f, 1.0f, x0, x1, x2, x2);
  } else {
    if (!(x2 > 0.0f && x2 * x2 > 1e-6f * d2)) return;  // not in front of the camera
    const float iz = 1.0f / x2;
    const float a = c.fx * iz, b = c.fy * iz;
    r[0] = fmaf(a, x0, c.cx) - y.x;
    r[1] = fmaf(b, x1, c.cy) - y.y;
    r[2] = x2 - y.z;
    const float lp = qq * c.inv_s1, lz = qq * c.inv_s2;
    w[0] = w[1] = huber_apply(lp * fmaf(r[0], r[0], r[1] * r[1]), lp, c, &cost);
    w[2] = huber_apply(lz * r[2] * r[2], lz, c, &cost);
    // dPi/dx = (1/z) [[fx, 0, -fx x/z], [0, fy, -fy y/z]]; the scale column is zero
    row_of(J[0], a, 0.0f, -a * x0 * iz, x0, x1, x2, 0.0f);
    row_of(J[1], 0.0f, b, -b * x1 * iz, x0, x1, x2, 0.0f);
    row_of(J[2], 0.0f, 0.0f, 1.0f, x0, x1, x2, x2);
  }
  add_rows(acc, J, w, r);
  acc[35] += cost;
  acc[36] += 1.0f;
}

template <int kKind> struct FamilyAcc { static constexpr int N = kKind == MSLAM_RES_RAY ? kNumAcc : kFamAcc; };

template <int kKind, bool kCheckFinite>
__device__ __forceinline__ void accumulate_any(float* acc, const RelPose& P, float3 Xj, float3 y, float qq,
                                               const LinConst& c) {
  if constexpr (kKind == MSLAM_RES_RAY)
    accumulate<kCheckFinite>(acc, P, Xj, y, qq, c);
  else
    accumulate_family<kKind>(acc, P, Xj, y, qq, c);
}

// The reference-side value a family consumes: the ray and point families use
// X_i[m] (checked inside the ray accumulation, here for the point family);
// the pixel family uses the pixel of m and the depth of X_i[m].  Returns
// false for a degenerate (non-finite or zero) X_i[m].
template <int kKind>
__device__ __forceinline__ bool family_y(float3& y, int m, int W) {
  if constexpr (kKind == MSLAM_RES_RAY) {
    return true;
  } else {
    const float b2 = y.x * y.x + y.y * y.y + y.z * y.z;
    if (!(b2 > 0.0f && b2 < INFINITY)) return false;
    if (kKind == MSLAM_RES_PIXEL) y = make_float3((float)(m % W), (float)(m / W), y.z);
    return true;
  }
}

// Warp reduce-scatter of 32 values: after five butterfly rounds (one
// shuffle per kept value and round) lane L holds the warp's sum of value L.
__device__ __forceinline__ float warp_reduce_scatter(float v[32], int lane) {
#pragma unroll
  for (int round = 0; round < 5; ++round) {
    const int half = 16 >> round;
    const bool up = (lane & half) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = up ? v[i] : v[i + half];
      const float keep = up ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, half);
    }
  }
  return v[0];
}

// Fixed-order block reduction of NA accumulators into the tile's partial slot.
template <int NA>
__device__ __forceinline__ void reduce_store(const float* acc, float (*red)[kFamAcc], float* partials, int tile) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    float v = acc[a];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][a] = v;
  }
  __syncthreads();
  if (tid < NA) {
    float s = red[0][tid];
#pragma unroll
    for (int w = 1; w < kLinThreads / 32; ++w) s += red[w][tid];
    partials[(size_t)tile * kAccStride + tid] = s;
  }
  __syncthreads();
}

#ifndef MSLAM_LIN_UNROLL
#define MSLAM_LIN_UNROLL 4
#endif
#ifndef MSLAM_LIN_MINBLOCKS
#define MSLAM_LIN_MINBLOCKS 2
#endif
constexpr int kUnroll = MSLAM_LIN_UNROLL;  // pixels per thread in flight

// Next work tile of a launch: claimed from a counter (so that tiles of uneven
// match counts balance across the persistent blocks) or, without a counter,
// the static grid stride.  Every tile's partial is computed the same way
// whichever block takes it, so results do not depend on the schedule.
__device__ __forceinline__ int next_tile(int* s_tile, int* ctr, int tile_begin, int prev) {
  if (ctr) {
    __syncthreads();  // every thread has read the previous tile index
    if (threadIdx.x == 0) *s_tile = tile_begin + atomicAdd(ctr, 1);
    __syncthreads();
    return *s_tile;
  }
  return prev < 0 ? tile_begin + (int)blockIdx.x : prev + (int)gridDim.x;
}

template <typename T, int kKind>
__global__ void __launch_bounds__(kLinThreads, MSLAM_LIN_MINBLOCKS)
    lin_tiles_kernel(PlanView pv, LinConst lc, const RelPose* __restrict__ rel, const T* __restrict__ X,
                     const int32_t* __restrict__ idx, const T* __restrict__ q, float* __restrict__ partials,
                     int tile_begin, int tile_end, int* __restrict__ tile_ctr) {
  constexpr int NA = FamilyAcc<kKind>::N;
  __shared__ float red[kLinThreads / 32][kFamAcc];
  __shared__ int s_tile;
  const int tid = threadIdx.x;
  for (int tile = next_tile(&s_tile, tile_ctr, tile_begin, -1); tile < tile_end;
       tile = next_tile(&s_tile, tile_ctr, tile_begin, tile)) {
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
    float acc[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) acc[a] = 0.0f;
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
      // two-level (blocked) summation, as in lin_packed_kernel
      float bacc[NA];
#pragma unroll
      for (int a = 0; a < NA; ++a) bacc[a] = 0.0f;
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if (mm[u] >= 0 && qq[u] > lc.q_min && family_y<kKind>(yy[u], mm[u], ed.W))
          accumulate_any<kKind, true>(bacc, P, xj[u], yy[u], qq[u], lc);
#pragma unroll
      for (int a = 0; a < NA; ++a) acc[a] += bacc[a];
    }
    // fixed-order tree: warp shuffles, then the 8 warp sums in order
    reduce_store<NA>(acc, red, partials, tile);
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
// records a thread sums in FP32 before they join the warp's tree sum
constexpr int kFlushRecs = 16;

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
    unpack(__ldg(src), xj, y, qq);
  }
  static __device__ __forceinline__ void unpack(const uint4 v, float3& xj, float3& y, float& qq) {
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
// One 1024-thread block per tile keeps the tile's pixel order.  A round
// covers kPackSteps x 1024 pixels (pixel base + k 1024 + t for thread t and
// step k): first every thread tests its kPackSteps pixels (loads of several
// steps in flight) and each warp counts its valid pixels per step; then one
// warp per step scans that step's 32 warp counts and one thread adds up the
// step totals; then every thread writes its records (the valid pixels'
// values read again, from the caches) at its rank.  Three barriers per round
// instead of three per 1024 pixels; the records and their order are those of
// one compaction per 1024 pixels.
constexpr int kPackThreads = 1024;
constexpr int kPackSteps = 16;

// a pixel gives a record: matched, confident, both canonical points
// non-zero and finite (a degenerate point contributes nothing, as in the
// gathering form)
template <typename T>
__device__ __forceinline__ bool pack_valid(const int32_t* __restrict__ idx_e, const T* __restrict__ q_e,
                                           const T* __restrict__ Xj, const T* __restrict__ Xi, int n, float q_min) {
  const int m = __ldg(idx_e + n);
  if (m < 0 || !(ldf(q_e + n) > q_min)) return false;
  const float3 xj = ld3(Xj, n), y = ld3(Xi, m);
  const float a2 = xj.x * xj.x + xj.y * xj.y + xj.z * xj.z, b2 = y.x * y.x + y.y * y.y + y.z * y.z;
  return a2 > 0.0f && b2 > 0.0f && a2 < INFINITY && b2 < INFINITY;
}

template <typename T>
__global__ void __launch_bounds__(kPackThreads, 2) pack_kernel(PlanView pv, float q_min, int kind, const T* __restrict__ X,
                                                            const int32_t* __restrict__ idx, const T* __restrict__ q,
                                                            uint4* __restrict__ recs, int32_t* __restrict__ counts) {
  __shared__ int s_wcnt[kPackSteps][kPackThreads / 32];  // per step and warp: valid pixels, then their offset
  __shared__ int s_step[kPackSteps + 1];                 // per step: offset within the round
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lanes_below = (1u << lane) - 1u;
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
    for (int base = tl.begin; base < tl.end; base += kPackThreads * kPackSteps) {
      unsigned valid = 0;  // bit k: this thread's pixel of step k gives a record
#pragma unroll 4
      for (int k = 0; k < kPackSteps; ++k) {
        const int n = base + k * kPackThreads + tid;
        const bool v = n < tl.end && pack_valid(idx_e, q_e, Xj, Xi, n, q_min);
        const unsigned bal = __ballot_sync(0xffffffffu, v);
        if (lane == 0) s_wcnt[k][warp] = __popc(bal);
        valid |= (unsigned)v << k;
      }
      __syncthreads();
      if (warp < kPackSteps) {  // exclusive scan of step `warp`'s 32 warp counts
        const int c = s_wcnt[warp][lane];
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int o = __shfl_up_sync(0xffffffffu, incl, off);
          if (lane >= off) incl += o;
        }
        s_wcnt[warp][lane] = incl - c;
        if (lane == 31) s_step[warp + 1] = incl;
      }
      __syncthreads();
      if (tid == 0) {
        s_step[0] = 0;
#pragma unroll
        for (int k = 1; k <= kPackSteps; ++k) s_step[k] += s_step[k - 1];
      }
      __syncthreads();
#pragma unroll 4
      for (int k = 0; k < kPackSteps; ++k) {
        const bool v = (valid >> k) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, v);
        if (v) {
          const int n = base + k * kPackThreads + tid;
          const int m = __ldg(idx_e + n);
          const float3 xj = ld3(Xj, n);
          float3 y = ld3(Xi, m);
          // the pixel family stores the reference pixel of m and its depth
          if (kind == MSLAM_RES_PIXEL) y = make_float3((float)(m % ed.W), (float)(m / ed.W), y.z);
          const int slot = base_count + s_step[k] + s_wcnt[k][warp] + __popc(bal & lanes_below);
          PackRec<T>::store(out + (size_t)slot * W, xj, y, ldf(q_e + n));
        }
      }
      base_count += s_step[kPackSteps];
      __syncthreads();  // the next round rewrites the counts
    }
    if (tid == 0) counts[tile] = base_count;
  }
}

template <typename T, int kKind, bool kRing>
__global__ void __launch_bounds__(kLinThreads, MSLAM_PACKED_MINBLOCKS) lin_packed_kernel(PlanView pv, LinConst lc,
                                                                   const RelPose* __restrict__ rel,
                                                                   const uint4* __restrict__ recs,
                                                                   const int32_t* __restrict__ counts,
                                                                   float* __restrict__ partials, int tile_begin,
                                                                   int tile_end, int* __restrict__ tile_ctr) {
  constexpr int NA = FamilyAcc<kKind>::N;
  __shared__ float red[kLinThreads / 32][kFamAcc];
  __shared__ int s_tile;
  const int tid = threadIdx.x;
  constexpr int W = PackRec<T>::kWords;
  constexpr int U = MSLAM_PACKED_UNROLL;
  // kRing (plan option lin_form 3), FP16 records: each thread keeps its next
  // batch of U records in flight with asynchronous copies into its own slots
  // of a one-batch buffer in shared memory while it evaluates the current
  // batch, which it has read into registers first (no thread reads another's
  // slots, so no barrier guards them; 16 KB per block).  The sums are those
  // of the plain form, in the same order.
  constexpr bool kAsync = kRing && W == 1 && NA <= 32;
  __shared__ __align__(16) uint4 ring[kAsync ? U * kLinThreads : 1];
  for (int tile = next_tile(&s_tile, tile_ctr, tile_begin, -1); tile < tile_end;
       tile = next_tile(&s_tile, tile_ctr, tile_begin, tile)) {
    const DevTile tl = pv.tiles[tile];
    RelPose P;
    {
      const float4* src = reinterpret_cast<const float4*>(rel + tl.edge);
      float4 a = __ldg(src), b = __ldg(src + 1), c = __ldg(src + 2);
      P.R[0] = a.x; P.R[1] = a.y; P.R[2] = a.z; P.R[3] = a.w;
      P.R[4] = b.x; P.R[5] = b.y; P.R[6] = b.z; P.R[7] = b.w;
      P.R[8] = c.x; P.t[0] = c.y; P.t[1] = c.z; P.t[2] = c.w;
    }
    float acc[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) acc[a] = 0.0f;
    const int cnt = __ldg(counts + tile);
    const uint4* in = recs + (size_t)tile * pv.lin_tile * W;
    if constexpr (NA <= 32) {
      // Tree summation: a thread sums at most kFlushRecs records in FP32,
      // then the warp's sums are added by a reduce-scatter and lane L keeps
      // the running sum of value L over the tile; the 8 warp sums are added
      // in a fixed order (the loop runs warp-uniformly so that every lane
      // takes part in each reduce-scatter)
      const int lane = tid & 31, warp = tid >> 5;
      float wsum = 0.0f;
      int batches = 0;
      // copies of batch r0 into the thread's slots (none past the end)
      auto issue = [&](int r0) {
        if constexpr (kAsync) {
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int r = r0 + lane + u * kLinThreads;
            if (r < cnt) cp_async16(ring + u * kLinThreads + tid, in + r);
          }
          cp_async_commit();
        }
      };
      issue(tid - lane);
      for (int r0 = tid - lane; r0 < cnt; r0 += U * kLinThreads) {
        float3 xj[U], yy[U];
        float qq[U];
        if constexpr (kAsync) {
          cp_async_wait_all();  // this batch's copies have landed
#pragma unroll
          for (int u = 0; u < U; ++u) {
            qq[u] = 0.0f;
            if (r0 + lane + u * kLinThreads < cnt) PackRec<T>::unpack(ring[u * kLinThreads + tid], xj[u], yy[u], qq[u]);
          }
          // the slots' values are in registers (the unpacking consumed them):
          // the next batch may land there
          issue(r0 + U * kLinThreads);
        } else {
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int r = r0 + lane + u * kLinThreads;
            qq[u] = 0.0f;
            if (r < cnt) PackRec<T>::load(in + (size_t)r * W, xj[u], yy[u], qq[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (r0 + lane + u * kLinThreads < cnt) accumulate_any<kKind, false>(acc, P, xj[u], yy[u], qq[u], lc);
        if (++batches * U == kFlushRecs) {
          float v[32];
#pragma unroll
          for (int a = 0; a < 32; ++a) v[a] = a < NA ? acc[a] : 0.0f;
#pragma unroll
          for (int a = 0; a < NA; ++a) acc[a] = 0.0f;
          wsum += warp_reduce_scatter(v, lane);
          batches = 0;
        }
      }
      if constexpr (kAsync) cp_async_wait_all();  // nothing in flight when the next tile reuses the ring
      {
        float v[32];
#pragma unroll
        for (int a = 0; a < 32; ++a) v[a] = a < NA ? acc[a] : 0.0f;
        wsum += warp_reduce_scatter(v, lane);
      }
      if (lane < NA) red[warp][lane] = wsum;
      __syncthreads();
      if (tid < NA) {
        float sum = red[0][tid];
#pragma unroll
        for (int w2 = 1; w2 < kLinThreads / 32; ++w2) sum += red[w2][tid];
        partials[(size_t)tile * kAccStride + tid] = sum;
      }
      __syncthreads();
    } else {
      for (int r0 = tid; r0 < cnt; r0 += U * kLinThreads) {
        float3 xj[U], yy[U];
        float qq[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int r = r0 + u * kLinThreads;
          qq[u] = 0.0f;
          if (r < cnt) PackRec<T>::load(in + (size_t)r * W, xj[u], yy[u], qq[u]);
        }
        // two-level (blocked) summation: the U records of a batch are summed
        // on their own, then the batch sum is added to the running sums, so a
        // thread's FP32 sums grow in error like U + records / U, not records
        float bacc[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) bacc[a] = 0.0f;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (r0 + u * kLinThreads < cnt) accumulate_any<kKind, false>(bacc, P, xj[u], yy[u], qq[u], lc);
#pragma unroll
        for (int a = 0; a < NA; ++a) acc[a] += bacc[a];
      }
      reduce_store<NA>(acc, red, partials, tile);
    }
  }
}

// ---------------------------------------------------------- streamed form
// The packed FP16 records of the ray family streamed through shared memory.
// One persistent CTA per SM claims tiles from the tile counter; one thread
// copies each tile's 16-byte records ahead in 4096-record (64 KB) chunks
// with bulk asynchronous copies (TMA, completion counted on an mbarrier per
// stage), so loads need no registers and later chunks arrive while the
// current one is computed.  Every thread takes up to four pairs of records
// per chunk (records j and j + ceil(n/2) of an n-record chunk, consecutive
// 16-byte words across the warp),
// builds the half2 pairs (value of record a, value of record b) with byte
// permutes, and evaluates both records with paired FP32 instructions
// (__ffma2_rn / __fmul2_rn / __fadd2_rn, one instruction per two lanes of
// work), which halves the instruction count of the per-match arithmetic
// that bounds the unpaired kernel.  The Huber weight min(1, delta/e) and
// cost rho(e) = e^2 h (2 - h) / 2 with h that weight need no branch.  The
// tile's sums are reduced by a butterfly reduce-scatter (one shuffle per
// value and round) and a fixed-order sum over the warps.  Every paired
// operation rounds like its scalar form; results are deterministic and
// independent of the schedule.

constexpr int kStreamThreads = 512;
constexpr int kStreamStages = 3;
constexpr int kStreamPairsPerThread = 4;
constexpr int kStreamChunkRecs = 2 * kStreamThreads * kStreamPairsPerThread;  // 4096 records
constexpr int kStreamChunkBytes = kStreamChunkRecs * 16;                     // 64 KB per stage

// Paired FP32 arithmetic (one instruction for two lanes of work).
using f2 = float2;
__device__ __forceinline__ f2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ f2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }

// A bounded wait gave up: every tile partial of the launch becomes NaN and
// every graph the launch covers gets MSLAM_ERR_TIMEOUT (the solve skips it).
__device__ void mark_timeout(const PlanView& pv, float* partials, int32_t* status, int tile_begin, int tile_end,
                             int t0, int stride) {
  for (int t = tile_begin + t0; t < tile_end; t += stride) {
    partials[(size_t)t * kAccStride] = __int_as_float(0x7fc00000);
    if (status) status[pv.edges[pv.tiles[t].edge].graph] = MSLAM_ERR_TIMEOUT;
  }
}
// Huber weight factor h = min(1, delta / e) of a squared whitened norm, per lane.
__device__ __forceinline__ float huber_h(float e2, const LinConst& c) {
  return fminf(1.0f, c.delta * rsqrt_ftz(fmaxf(e2, c.delta2)));
}

// Two records (lanes a and b) of the ray family; mask = (1 or 0, 1 or 0)
// selects the lanes that hold a record with x != 0.
__device__ __forceinline__ void accumulate_pair(f2 acc[kNumAcc], const f2 Rp[12], f2 X0, f2 X1, f2 X2, f2 Y0, f2 Y1,
                                                f2 Y2, f2 Q, bool vb, const LinConst& c) {
  const f2 x0 = fma2(Rp[0], X0, fma2(Rp[1], X1, fma2(Rp[2], X2, Rp[9])));
  const f2 x1 = fma2(Rp[3], X0, fma2(Rp[4], X1, fma2(Rp[5], X2, Rp[10])));
  const f2 x2 = fma2(Rp[6], X0, fma2(Rp[7], X1, fma2(Rp[8], X2, Rp[11])));
  const f2 d2 = fma2(x0, x0, fma2(x1, x1, mul2(x2, x2)));
  const f2 dy2 = fma2(Y0, Y0, fma2(Y1, Y1, mul2(Y2, Y2)));
  // a lane without a record, or with x = 0, gets zero weights; its
  // arithmetic stays finite so that zero weights give exact zeros
  const bool va = d2.x > 0.0f;
  vb = vb && d2.y > 0.0f;
  const f2 mask = mk2(va ? 1.0f : 0.0f, vb ? 1.0f : 0.0f);
  const f2 id = mk2(rsqrt_ftz(va ? d2.x : 1.0f), rsqrt_ftz(vb ? d2.y : 1.0f));
  const f2 idy = mk2(rsqrt_ftz(va ? dy2.x : 1.0f), rsqrt_ftz(vb ? dy2.y : 1.0f));
  const f2 m1 = bc2(-1.0f);
  const f2 d = mul2(d2, id), dy = mul2(dy2, idy);
  const f2 u0 = mul2(x0, id), u1 = mul2(x1, id), u2 = mul2(x2, id);
  const f2 nidy = mul2(idy, m1);
  const f2 r0 = fma2(Y0, nidy, u0), r1 = fma2(Y1, nidy, u1), r2 = fma2(Y2, nidy, u2);
  const f2 rd = fma2(dy, m1, d);
  const f2 qm = mul2(Q, mask);
  const f2 lr = mul2(qm, bc2(c.inv_sr2)), ld = mul2(qm, bc2(c.inv_sd2));
  const f2 er2 = mul2(lr, fma2(r0, r0, fma2(r1, r1, mul2(r2, r2))));
  const f2 ed2 = mul2(ld, mul2(rd, rd));
  const f2 hr = mk2(huber_h(er2.x, c), huber_h(er2.y, c));
  const f2 hd = mk2(huber_h(ed2.x, c), huber_h(ed2.y, c));
  const f2 two = bc2(2.0f), half = bc2(0.5f);
  // rho = e^2 h (2 - h) / 2 in both Huber regions
  const f2 cost = fma2(mul2(half, er2), mul2(hr, fma2(hr, m1, two)), mul2(mul2(half, ed2), mul2(hd, fma2(hd, m1, two))));
  const f2 wr = mul2(lr, hr), wd = mul2(ld, hd);
  const f2 A = mul2(wr, mul2(id, id));
  acc[0] = add2(acc[0], A);
  const f2 cc = fma2(A, m1, wd);
  const f2 cu0 = mul2(cc, u0), cu1 = mul2(cc, u1), cu2 = mul2(cc, u2);
  acc[1] = fma2(cu0, u0, acc[1]);
  acc[2] = fma2(cu0, u1, acc[2]);
  acc[3] = fma2(cu0, u2, acc[3]);
  acc[4] = fma2(cu1, u1, acc[4]);
  acc[5] = fma2(cu1, u2, acc[5]);
  acc[6] = fma2(cu2, u2, acc[6]);
  acc[7] = fma2(A, x0, acc[7]);
  acc[8] = fma2(A, x1, acc[8]);
  acc[9] = fma2(A, x2, acc[9]);
  acc[10] = fma2(wd, x0, acc[10]);
  acc[11] = fma2(wd, x1, acc[11]);
  acc[12] = fma2(wd, x2, acc[12]);
  acc[13] = add2(acc[13], wr);
  const f2 wu0 = mul2(wr, u0), wu1 = mul2(wr, u1), wu2 = mul2(wr, u2);
  acc[14] = fma2(wu0, u0, acc[14]);
  acc[15] = fma2(wu0, u1, acc[15]);
  acc[16] = fma2(wu0, u2, acc[16]);
  acc[17] = fma2(wu1, u1, acc[17]);
  acc[18] = fma2(wu1, u2, acc[18]);
  acc[19] = fma2(wu2, u2, acc[19]);
  acc[20] = fma2(wd, d2, acc[20]);
  const f2 nur = mul2(fma2(u0, r0, fma2(u1, r1, mul2(u2, r2))), m1);
  const f2 ad = mul2(wr, id), wdr = mul2(wd, rd);
  acc[21] = fma2(ad, fma2(u0, nur, r0), fma2(wdr, u0, acc[21]));
  acc[22] = fma2(ad, fma2(u1, nur, r1), fma2(wdr, u1, acc[22]));
  acc[23] = fma2(ad, fma2(u2, nur, r2), fma2(wdr, u2, acc[23]));
  const f2 nx0 = mul2(x0, m1), nx1 = mul2(x1, m1), nx2 = mul2(x2, m1);
  acc[24] = fma2(ad, fma2(nx2, r1, mul2(x1, r2)), acc[24]);
  acc[25] = fma2(ad, fma2(nx0, r2, mul2(x2, r0)), acc[25]);
  acc[26] = fma2(ad, fma2(nx1, r0, mul2(x0, r1)), acc[26]);
  acc[27] = fma2(wdr, d, acc[27]);
  acc[28] = add2(acc[28], cost);
  acc[29] = add2(acc[29], mask);
}

__global__ void __launch_bounds__(kStreamThreads, 1)
    lin_stream_kernel(PlanView pv, LinConst lc, const RelPose* __restrict__ rel, const unsigned char* __restrict__ recs,
                      const int32_t* __restrict__ counts, float* __restrict__ partials, int tile_begin, int tile_end,
                      int* __restrict__ tile_ctr, int32_t* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char stage[];
  __shared__ __align__(8) uint64_t full[kStreamStages];
  __shared__ int m_tile[kStreamStages], m_np[kStreamStages], m_last[kStreamStages];
  __shared__ float red[kStreamThreads / 32][32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // producer state (thread 0): the tile being copied and its next pair
  int p_tile = -1, p_cnt = 0, p_off = 0;
  auto claim = [&]() {
    p_tile = tile_ctr ? tile_begin + atomicAdd(tile_ctr, 1) : (p_tile < 0 ? tile_begin + (int)blockIdx.x
                                                                          : p_tile + (int)gridDim.x);
    p_off = 0;
    p_cnt = p_tile < tile_end ? __ldg(counts + p_tile) : 0;
  };
  auto issue = [&](int slot) {
    if (pv.wait_polls == 0) return;  // wait limit "give up at once": no copy is issued
    if (p_tile >= tile_end) {  // end marker
      m_tile[slot] = -1;
      mbar_arrive(&full[slot]);
      return;
    }
    const int n = min(kStreamChunkRecs, p_cnt - p_off);
    m_tile[slot] = p_tile;
    m_np[slot] = n;
    m_last[slot] = (p_off + n >= p_cnt);
    if (n > 0) {
      mbar_arrive_tx(&full[slot], (uint32_t)(n * 16));
      bulk_g2s(stage + slot * kStreamChunkBytes, recs + ((size_t)p_tile * pv.lin_tile + p_off) * 16,
               (uint32_t)(n * 16), &full[slot]);
    } else {
      mbar_arrive(&full[slot]);
    }
    p_off += n;
    if (p_off >= p_cnt) claim();
  };
  if (tid == 0) {
    for (int sl = 0; sl < kStreamStages; ++sl) mbar_init(&full[sl], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    claim();
    for (int sl = 0; sl < kStreamStages; ++sl) issue(sl);
  }
  __syncthreads();

  f2 acc[kNumAcc];
#pragma unroll
  for (int a = 0; a < kNumAcc; ++a) acc[a] = mk2(0.0f, 0.0f);
  float wsum = 0.0f;  // lane L: this warp's running sum of value L over the tile's chunks
  int chunks = 0;     // chunks summed since the last reduce-scatter
  int cur_tile = -1;
  f2 Rp[12];
  bool aborted = false;
  for (int k = 0;; ++k) {
    const int slot = k % kStreamStages;
    const uint32_t parity = (uint32_t)((k / kStreamStages) & 1);
    const bool ok = mbar_wait_bounded(&full[slot], parity, pv.wait_polls);
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    const int tile = m_tile[slot];
    if (tile < 0) break;
    if (tile != cur_tile) {
      const float4* src = reinterpret_cast<const float4*>(rel + pv.tiles[tile].edge);
      const float4 a = __ldg(src), b = __ldg(src + 1), c4 = __ldg(src + 2);
      Rp[0] = bc2(a.x); Rp[1] = bc2(a.y); Rp[2] = bc2(a.z); Rp[3] = bc2(a.w);
      Rp[4] = bc2(b.x); Rp[5] = bc2(b.y); Rp[6] = bc2(b.z); Rp[7] = bc2(b.w);
      Rp[8] = bc2(c4.x); Rp[9] = bc2(c4.y); Rp[10] = bc2(c4.z); Rp[11] = bc2(c4.w);
      cur_tile = tile;
    }
    {
      // record layout (FP16): {X_j.x, X_j.y}, {X_j.z, y.x}, {y.y, y.z}, {q, 0}
      const int n = m_np[slot], h = (n + 1) >> 1;  // records j and j + h form pair j
      const uint4* rec = reinterpret_cast<const uint4*>(stage + slot * kStreamChunkBytes);
#pragma unroll
      for (int u = 0; u < kStreamPairsPerThread; ++u) {
        const int ra = tid + u * kStreamThreads, rb = ra + h;
        if (ra < h) {
          const bool vb = rb < n;
          const uint4 a = rec[ra], b = vb ? rec[rb] : make_uint4(0u, 0u, 0u, 0u);
          auto pr = [](uint32_t x, uint32_t y, uint32_t sel) {
            const uint32_t v = __byte_perm(x, y, sel);
            return __half22float2(*reinterpret_cast<const __half2*>(&v));
          };
          accumulate_pair(acc, Rp, pr(a.x, b.x, 0x5410), pr(a.x, b.x, 0x7632), pr(a.y, b.y, 0x5410),
                          pr(a.y, b.y, 0x7632), pr(a.z, b.z, 0x5410), pr(a.z, b.z, 0x7632), pr(a.w, b.w, 0x5410),
                          vb, lc);
        }
      }
    }
    if (++chunks == 2 || m_last[slot]) {
      // tree summation every two chunks: a thread's sums cover at most 16
      // records; the warp reduce-scatter adds them, and lane L keeps the
      // running sum of value L over the tile's chunks
      chunks = 0;
      float v[32];
#pragma unroll
      for (int a = 0; a < kNumAcc; ++a) {
        v[a] = acc[a].x + acc[a].y;
        acc[a] = mk2(0.0f, 0.0f);
      }
      v[30] = v[31] = 0.0f;
      wsum += warp_reduce_scatter(v, lane);
    }
    if (m_last[slot]) {
      // the tile is complete: the warps' sums in a fixed order into the
      // tile's partial slot
      red[warp][lane] = wsum;
      wsum = 0.0f;
      __syncthreads();
      if (tid < kNumAcc) {
        float sum = red[0][tid];
#pragma unroll
        for (int w = 1; w < kStreamThreads / 32; ++w) sum += red[w][tid];
        partials[(size_t)tile * kAccStride + tid] = sum;
      }
    }
    __syncthreads();  // every thread is done with this slot
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(slot);
    }
  }
  if (aborted) {
    // a copy did not complete in time: poison every tile's partial, report
    // the timeout per graph, and let in-flight copies land before the CTA's
    // shared memory is released (each stage's pending phase is waited for,
    // again with the bound)
    mark_timeout(pv, partials, status, tile_begin, tile_end, tid, kStreamThreads);
    if (tid == 0)
      for (int sl = 0; sl < kStreamStages; ++sl)
        mbar_wait_bounded(&full[sl], 0, pv.wait_polls), mbar_wait_bounded(&full[sl], 1, pv.wait_polls);
    __syncthreads();
  }
}

// ------------------------------------------------- per-warp streamed form
// The paired-FP32 evaluation of lin_stream_kernel with one pipeline per warp
// instead of one per block: every warp claims whole tiles from the tile
// counter, its lane 0 copies the tile's 16-byte records ahead into the
// warp's own ring of three 4 KB stages with bulk asynchronous copies
// (completion counted on one mbarrier per stage), and the warp reduces a
// finished tile by itself (reduce-scatter, then 30 lanes store the tile's
// partial).  No block-wide barrier is taken: warps drift apart, so loads,
// arithmetic and reductions of different warps overlap, and a stage is
// refilled as soon as its own warp has read it.  Tiles are smaller than in
// the block form (a warp takes a whole tile), which the plan's lin_tile sets.
constexpr int kWarpStreamThreads = 512;
constexpr int kWarpStreamWarps = kWarpStreamThreads / 32;
constexpr int kWarpStages = 3;
constexpr int kWarpStageRecs = 256;  // four pairs of records per lane
constexpr int kWarpStageBytes = kWarpStageRecs * 16;
constexpr size_t kWarpStreamSmem = (size_t)kWarpStreamWarps * kWarpStages * kWarpStageBytes;  // 192 KB

__global__ void __launch_bounds__(kWarpStreamThreads, 1)
    lin_warp_stream_kernel(PlanView pv, LinConst lc, const RelPose* __restrict__ rel,
                           const unsigned char* __restrict__ recs, const int32_t* __restrict__ counts,
                           float* __restrict__ partials, int tile_begin, int tile_end, int* __restrict__ tile_ctr,
                           int32_t* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char wstage[];
  __shared__ __align__(8) uint64_t full[kWarpStreamWarps][kWarpStages];
  __shared__ int m_tile[kWarpStreamWarps][kWarpStages], m_n[kWarpStreamWarps][kWarpStages],
      m_last[kWarpStreamWarps][kWarpStages];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* ring = wstage + (size_t)warp * kWarpStages * kWarpStageBytes;
  uint64_t* bars = full[warp];
  const int gwarp = (int)blockIdx.x * kWarpStreamWarps + warp, nwarps = (int)gridDim.x * kWarpStreamWarps;

  // producer state (lane 0): the tile being copied and its next record
  int p_tile = -1, p_cnt = 0, p_off = 0;
  auto claim = [&]() {
    p_tile = tile_ctr ? tile_begin + atomicAdd(tile_ctr, 1) : (p_tile < 0 ? tile_begin + gwarp : p_tile + nwarps);
    p_off = 0;
    p_cnt = p_tile < tile_end ? __ldg(counts + p_tile) : 0;
  };
  auto issue = [&](int slot) {
    if (pv.wait_polls == 0) return;  // wait limit "give up at once": no copy is issued
    if (p_tile >= tile_end) {  // end marker
      m_tile[warp][slot] = -1;
      mbar_arrive(&bars[slot]);
      return;
    }
    const int n = min(kWarpStageRecs, p_cnt - p_off);
    m_tile[warp][slot] = p_tile;
    m_n[warp][slot] = n;
    m_last[warp][slot] = (p_off + n >= p_cnt);
    if (n > 0) {
      mbar_arrive_tx(&bars[slot], (uint32_t)(n * 16));
      bulk_g2s(ring + slot * kWarpStageBytes, recs + ((size_t)p_tile * pv.lin_tile + p_off) * 16, (uint32_t)(n * 16),
               &bars[slot]);
    } else {
      mbar_arrive(&bars[slot]);
    }
    p_off += n;
    if (p_off >= p_cnt) claim();
  };
  if (lane == 0) {
    for (int sl = 0; sl < kWarpStages; ++sl) mbar_init(&bars[sl], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    claim();
    for (int sl = 0; sl < kWarpStages; ++sl) issue(sl);
  }
  __syncwarp();

  f2 acc[kNumAcc];
#pragma unroll
  for (int a = 0; a < kNumAcc; ++a) acc[a] = mk2(0.0f, 0.0f);
  float tsum = 0.0f;  // lane L: the running sum of value L over the tile's stages
  int stages = 0;     // stages summed since the last reduce-scatter
  int cur_tile = -1;
  // the relative pose of the current tile, pairs (v, v), in the warp's slot
  // of shared memory (read as broadcasts; keeps 24 registers free)
  __shared__ f2 rp_s[kWarpStreamWarps][12];
  f2* Rp = rp_s[warp];
  bool aborted = false;
  for (int k = 0;; ++k) {
    const int slot = k % kWarpStages;
    const uint32_t parity = (uint32_t)((k / kWarpStages) & 1);
    const bool ok = mbar_wait_bounded(&bars[slot], parity, pv.wait_polls);
    if (__any_sync(0xffffffffu, !ok)) {
      aborted = true;
      break;
    }
    const int tile = m_tile[warp][slot];
    if (tile < 0) break;
    if (tile != cur_tile) {
      const float4* src = reinterpret_cast<const float4*>(rel + pv.tiles[tile].edge);
      if (lane < 12) {  // the previous tile's reads ended at the last stage's __syncwarp
        const float4 v4 = __ldg(src + lane / 4);
        Rp[lane] = bc2((lane & 3) == 0 ? v4.x : (lane & 3) == 1 ? v4.y : (lane & 3) == 2 ? v4.z : v4.w);
      }
      __syncwarp();
      cur_tile = tile;
    }
    const int n = m_n[warp][slot], h = (n + 1) >> 1;  // records j and j + h form pair j
    const bool last = m_last[warp][slot] != 0;
    const uint4* rec = reinterpret_cast<const uint4*>(ring + slot * kWarpStageBytes);
    auto pair_at = [&](int ra, bool vb) {
      const uint4 a = rec[ra], b = vb ? rec[ra + h] : make_uint4(0u, 0u, 0u, 0u);
      auto pr = [](uint32_t x, uint32_t y, uint32_t sel) {
        const uint32_t v = __byte_perm(x, y, sel);
        return __half22float2(*reinterpret_cast<const __half2*>(&v));
      };
      accumulate_pair(acc, Rp, pr(a.x, b.x, 0x5410), pr(a.x, b.x, 0x7632), pr(a.y, b.y, 0x5410),
                      pr(a.y, b.y, 0x7632), pr(a.z, b.z, 0x5410), pr(a.z, b.z, 0x7632), pr(a.w, b.w, 0x5410), vb, lc);
    };
#pragma unroll
    for (int u = 0; u < kWarpStageRecs / 64; ++u) {
      const int ra = lane + 32 * u;
      if (ra < h) pair_at(ra, ra + h < n);
    }
    if (++stages == 2 || last) {
      // tree summation every two stages: a lane's sums cover at most 16
      // records; the reduce-scatter adds the warp's, and lane L keeps the
      // running sum of value L over the tile's stages
      stages = 0;
      float v[32];
#pragma unroll
      for (int a = 0; a < kNumAcc; ++a) {
        v[a] = acc[a].x + acc[a].y;
        acc[a] = mk2(0.0f, 0.0f);
      }
      v[30] = v[31] = 0.0f;
      tsum += warp_reduce_scatter(v, lane);
    }
    if (last) {
      // the tile is complete: lane a stores value a of the tile's partial
      if (lane < kNumAcc) partials[(size_t)tile * kAccStride + lane] = tsum;
      tsum = 0.0f;
    }
    __syncwarp();  // every lane is done with this stage
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(slot);
    }
  }
  if (aborted) {
    // a copy did not complete in time: poison every tile's partial, report
    // the timeout per graph, and let this warp's copies in flight land
    // before the block's shared memory is released
    mark_timeout(pv, partials, status, tile_begin, tile_end, lane, 32);
    if (lane == 0)
      for (int sl = 0; sl < kWarpStages; ++sl)
        mbar_wait_bounded(&bars[sl], 0, pv.wait_polls), mbar_wait_bounded(&bars[sl], 1, pv.wait_polls);
    __syncwarp();
  }
}

// The ray family's relative 7 x 7 system and gradient from its 30
// structured sums S (FP64): H_tt = S0 I + S[1..6], H_ww = S13 I - S[14..19],
// H_tw = -[S7..9]x, the scale column S[10..12] and S20, g = S[21..27].
__device__ void ray_relative_system(const double* S, double Hr[49], double g[7]) {
  for (int k = 0; k < 49; ++k) Hr[k] = 0.0;
  const double s2[6] = {S[1], S[2], S[3], S[4], S[5], S[6]};
  const int sym[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      Hr[7 * a + b] = (a == b ? S[0] : 0.0) + s2[sym[a][b]];
      Hr[7 * (3 + a) + 3 + b] = (a == b ? S[13] : 0.0) - S[14 + sym[a][b]];
    }
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
}

// One block per edge: FP64 sum of the edge's tile partials (four groups of
// threads take every fourth tile, then the groups' sums are added in a fixed
// order), then the 14x14.
constexpr int kFinalizeThreads = 256;
__global__ void __launch_bounds__(kFinalizeThreads) lin_finalize_kernel(PlanView pv, const double* __restrict__ T_wc,
                                                          const float* __restrict__ partials,
                                                          float* __restrict__ H14, float* __restrict__ g14,
                                                          double* __restrict__ cost, int32_t* __restrict__ n_valid,
                                                          int e_begin, int kind) {
  const int e = e_begin + blockIdx.x;
  const DevEdge ed = pv.edges[e];
  __shared__ double S[kFamAcc], Sg[kFinalizeThreads / 64][kFamAcc];
  __shared__ double Hr[49], A[49], C[49], g[7];
  const int tid = threadIdx.x;
  const int NA = kind == MSLAM_RES_RAY ? kNumAcc : kFamAcc;
  {
    const int a = tid & 63, grp = tid >> 6;
    if (a < NA) {
      double s = 0.0;
#pragma unroll 8
      for (int t = ed.tile_begin + grp; t < ed.tile_end; t += kFinalizeThreads / 64)
        s += (double)partials[(size_t)t * kAccStride + a];
      Sg[grp][a] = s;
    }
  }
  if (tid == 32) {
    const Sim3d Ti = load_pose(T_wc + 8 * ed.i);
    adjoint_of(inverse(Ti), A);
  }
  __syncthreads();
  if (tid < NA) S[tid] = (Sg[0][tid] + Sg[1][tid]) + (Sg[2][tid] + Sg[3][tid]);
  __syncthreads();
  if (tid == 0 && kind != MSLAM_RES_RAY) {
    // other families: the 28 upper-triangle sums, then g, cost and count
    int t = 0;
    for (int a = 0; a < 7; ++a)
      for (int b = a; b < 7; ++b, ++t) Hr[7 * a + b] = Hr[7 * b + a] = S[t];
    for (int a = 0; a < 7; ++a) g[a] = S[28 + a];
    cost[e] = S[35];
    if (n_valid) n_valid[e] = (int32_t)S[36];
  }
  if (tid == 0 && kind == MSLAM_RES_RAY) {
    ray_relative_system(S, Hr, g);
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

// ------------------------------------------------------------- tracking
// One Gauss-Newton iteration of tracking problems per launch, one block per
// tile: the block forms its edge's relative pose from T_wc, accumulates the
// tile's packed records (ray family) and stores the tile's sums; the block
// that completes an edge's last tile (a counter per edge, after a device
// fence) adds the edge's tile sums in tile order in FP64, maps the relative
// system to the frame's 7 x 7 with the adjoint of T_i^-1, solves it, retracts
// the frame's pose and resets the counter.  No block waits for another.
// A dependent FP64 operation takes tens of cycles on this GPU, so the FP64
// work of a launch is spread over lanes and warps: the entries of the
// relative pose, of the adjoint and of the relative 7 x 7 system are formed
// by different lanes, the pieces of Exp(tau) by different warps, and the
// 7 x 7 solve factors in FP32 with FP64 iterative refinement.

// Entry (r, c) of the ray family's relative 7 x 7 system from its 30 sums
// (the layout of ray_relative_system).
__device__ __forceinline__ double hr_entry(const double* S, int r, int c) {
  const bool rt = r < 3, ct = c < 3, rr = r >= 3 && r < 6, cr = c >= 3 && c < 6;
  if (rt && ct) {
    const int s = r == c ? (r == 0 ? 0 : r == 1 ? 3 : 5) : (r + c == 1 ? 1 : r + c == 2 ? 2 : 4);
    return (r == c ? S[0] : 0.0) + S[1 + s];
  }
  if (rr && cr) {
    const int a = r - 3, b = c - 3;
    const int s = a == b ? (a == 0 ? 0 : a == 1 ? 3 : 5) : (a + b == 1 ? 1 : a + b == 2 ? 2 : 4);
    return (a == b ? S[13] : 0.0) - S[14 + s];
  }
  // tw(a, b) for a < 3, b < 3 (the translation-rotation coupling)
  auto tw = [&](int a, int b) {
    if (a == b) return 0.0;
    const int k = 3 - a - b;
    const double v = S[7 + k];
    return (b == (a + 1) % 3) ? v : -v;  // tw = [[0, z, -y], [-z, 0, x], [y, -x, 0]]
  };
  if (rt && cr) return tw(r, c - 3);
  if (rr && ct) return tw(c, r - 3);
  if (rt && c == 6) return S[10 + r];
  if (r == 6 && ct) return S[10 + c];
  if (r == 6 && c == 6) return S[20];
  return 0.0;
}

// tau = -H7^-1 g7 by the 32 lanes of a warp (lanes 0..6 hold rows):
// Jacobi scaling s = diag(H7)^-1/2, FP32 Cholesky of s H7 s, then iterative
// refinement x <- x + s (L L^T)^-1 s (b - H7 x) with the residual in FP64,
// stopped when the predicted next correction (the last one times the
// observed contraction) is below 1e-9 of |x|, as in the mixed-precision
// graph solve.  Returns false in every lane (the caller then uses the FP64
// factorisation, which applies the exact not-positive-definite rule) when a
// diagonal entry is not positive, an FP32 pivot is not above 2^-20 of the
// unit diagonal, a value is not finite or the refinement stalls.  On success
// lanes 0..6 return their entry of tau in *tau.
constexpr int kTrackRefine = 8;
__device__ bool track_mixed_solve(const double* __restrict__ H7, const double* __restrict__ g7, int lane,
                                  double* tau) {
  constexpr unsigned kAll = 0xffffffffu;
  const bool row = lane < 7;
  const int i = row ? lane : 0;
  const double hii = H7[8 * i];
  if (!__all_sync(kAll, hii > 0.0 && hii < INFINITY)) return false;
  const double sc = rsqrt_newton(hii);
  float L[7], inv[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) L[k] = (float)(sc * H7[7 * i + k] * __shfl_sync(kAll, sc, k));
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const float djj = __shfl_sync(kAll, L[j], j);
    const bool okj = djj > 9.5367431640625e-7f && djj < INFINITY;  // 2^-20 of the unit diagonal
    ok = ok && okj;
    inv[j] = rsqrtf(okj ? djj : 1.0f);
    const float lij = L[j] * inv[j];
    if (lane >= j) L[j] = lij;
#pragma unroll
    for (int k = j + 1; k < 7; ++k) {
      const float lkj = __shfl_sync(kAll, L[j], k);
      if (lane >= k) L[k] = fmaf(-lij, lkj, L[k]);
    }
  }
  if (!ok) return false;  // the pivots are broadcast: the same decision in every lane
  // each lane also keeps its column of L (Lc[j] = L_ji, held by lane j)
  float Lc[7];
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    Lc[j] = 0.0f;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const float v = __shfl_sync(kAll, L[k], j);
      if (k == i) Lc[j] = v;
    }
  }
  // (L L^T)^-1 of the lanes' right-hand side entries
  auto solve = [&](float rhs) {
    float acc = rhs, y = 0.0f;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const float yj = __shfl_sync(kAll, acc, j) * inv[j];
      if (lane == j) y = yj;
      if (lane > j) acc = fmaf(-L[j], yj, acc);
    }
    float acc2 = y, z = 0.0f;
#pragma unroll
    for (int j = 6; j >= 0; --j) {
      const float zj = __shfl_sync(kAll, acc2, j) * inv[j];
      if (lane == j) z = zj;
      if (lane < j) acc2 = fmaf(-Lc[j], zj, acc2);
    }
    return z;
  };
  const double b = row ? -g7[i] : 0.0;
  double x = 0.0, r = b;
  float zprev = 0.0f;
  for (int it = 0; it < kTrackRefine; ++it) {
    const float z = solve((float)(sc * r));  // every lane takes part in the shuffles
    const double dx = row ? sc * (double)z : 0.0;
    x += dx;
    // the stopping test needs magnitudes only: FP32 maxima (FP64 instructions
    // occupy the SM's FP64 pipe for about 16 cycles each, whatever the lanes)
    float zm = fabsf((float)dx), xm = fabsf((float)x);
    // (fmaxf would pass over a NaN: every lane's entry is tested)
    if (__any_sync(kAll, !(zm < INFINITY && xm < INFINITY))) return false;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      zm = fmaxf(zm, __shfl_xor_sync(kAll, zm, off));
      xm = fmaxf(xm, __shfl_xor_sync(kAll, xm, off));
    }
    if (zm == 0.0f) break;
    if (it > 0) {  // contraction rho = zm / zprev (zprev > 0 here)
      if (zm * zm <= 1e-9f * xm * zprev) break;
      if (it > 1 && zm > 0.5f * zprev) return false;  // stalled
    }
    if (it == kTrackRefine - 1) return false;
    zprev = zm;
    // r = b - H7 x in FP64
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const double xk = __shfl_sync(kAll, x, k);
      if (k & 1) s1 = fma(H7[7 * i + k], xk, s1);
      else s0 = fma(H7[7 * i + k], xk, s0);
    }
    r = row ? b - (s0 + s1) : 0.0;
  }
  *tau = x;
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kLinThreads) track_kernel(PlanView pv, LinConst lc, double conv_tol,
                                                            double* __restrict__ T_wc,
                                                            const uint4* __restrict__ recs,
                                                            const int32_t* __restrict__ counts,
                                                            float* __restrict__ partials, int32_t* __restrict__ done,
                                                            int32_t* __restrict__ dev_status) {
  constexpr int kWarps = kLinThreads / 32;
  constexpr int kGroups = kWarps - 1;  // warps summing the tile partials in the finishing block
  __shared__ float red[kWarps][kFamAcc];
  __shared__ float sP[12];
  __shared__ int s_last, s_status, s_fb;
  __shared__ double S[kNumAcc], Hr[49], A[49], C[49], H7[49], g7[7];
  __shared__ double Sg[kGroups][kNumAcc];
  __shared__ double sR[18], s_inv, s_tp[3];  // R_i, R_j (row-major), 1 / s_i, t of T_i^-1
  __shared__ double s_tau[7], s_part[10], s_mx, s_Tk[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, tile = blockIdx.x;
  const DevTile tl = pv.tiles[tile];
  const DevEdge ed = pv.edges[tl.edge];
  const int g = ed.graph;
  // a converged or failed graph is skipped by all of its blocks (its status
  // changes only in the block that finishes the graph, after they all ran)
  if (__ldcg(dev_status + g) > 0) return;
  const double* Ti = T_wc + 8 * ed.i;
  const double* Tj = T_wc + 8 * ed.j;
  // T_ij = T_i^-1 T_j = (s_j / s_i R_i^T R_j, R_i^T (t_j - t_i) / s_i) in FP64
  // by lanes of warp 0: the entries of R_i, R_j and 1 / s_i, then the twelve
  // entries of s R and t of T_ij (no block of this launch changes a pose
  // before every block has read them here)
  if (warp == 0) {
    if (lane < 18) {
      const int e = lane % 9;
      sR[lane] = rot_entry((lane < 9 ? Ti : Tj) + 3, e / 3, e % 3);
    }
    if (lane == 18) s_inv = rcp_newton(Ti[7]);
    __syncwarp();
    if (lane < 9) {
      const int r = lane / 3, c = lane % 3;
      const double v = sR[r] * sR[9 + c] + sR[3 + r] * sR[12 + c] + sR[6 + r] * sR[15 + c];
      sP[lane] = (float)(Tj[7] * s_inv * v);
    } else if (lane < 12) {
      const int r = lane - 9;
      const double v = sR[r] * (Tj[0] - Ti[0]) + sR[3 + r] * (Tj[1] - Ti[1]) + sR[6 + r] * (Tj[2] - Ti[2]);
      sP[lane] = (float)(s_inv * v);
    }
  }
  __syncthreads();
  RelPose P;
  for (int k = 0; k < 9; ++k) P.R[k] = sP[k];
  for (int k = 0; k < 3; ++k) P.t[k] = sP[9 + k];
  float acc[kNumAcc];
#pragma unroll
  for (int a = 0; a < kNumAcc; ++a) acc[a] = 0.0f;
  constexpr int W = PackRec<T>::kWords;
  const int cnt = __ldg(counts + tile);
  const uint4* in = recs + (size_t)tile * pv.lin_tile * W;
  for (int r = tid; r < cnt; r += kLinThreads) {
    float3 xj, yy;
    float qq;
    PackRec<T>::load(in + (size_t)r * W, xj, yy, qq);
    accumulate<false>(acc, P, xj, yy, qq, lc);
  }
  reduce_store<kNumAcc>(acc, red, partials, tile);  // ends with a barrier
  if (tid == 0) {
    __threadfence();  // this tile's sums before the count
    s_last = atomicAdd(done + tl.edge, 1) == ed.tile_end - ed.tile_begin - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int gauge = pv.graphs[g].gauge;
  const int k_free = ed.i == gauge ? ed.j : ed.i;
  const double sgn = ed.i == gauge ? 1.0 : -1.0;  // g_j = Ad^T g_rel, g_i = -Ad^T g_rel
  if (warp < kGroups) {
    // seven warps take every seventh tile (loads of several tiles in flight),
    // then the groups' FP64 sums are added in a fixed order
    if (lane < kNumAcc) {
      double sum = 0.0;
#pragma unroll 4
      for (int t = ed.tile_begin + warp; t < ed.tile_end; t += kGroups)
        sum += (double)__ldcg(partials + (size_t)t * kAccStride + lane);
      Sg[warp][lane] = sum;
    }
  } else {
    // meanwhile the last warp forms Ad_{T_i^-1} =
    // [[s' R', [t']x R', -t'], [0, R', 0], [0, 0, 1]] with R' = R_i^T,
    // s' = 1 / s_i, t' = -s' R_i^T t_i (R_i and s' from the start of the block)
    if (lane < 3) s_tp[lane] = -s_inv * (sR[lane] * Ti[0] + sR[3 + lane] * Ti[1] + sR[6 + lane] * Ti[2]);
    if (lane >= 24) s_Tk[lane - 24] = __ldcg(T_wc + 8 * k_free + lane - 24);  // the pose to retract
    __syncwarp();
    for (int e = lane; e < 49; e += 32) {
      const int r = e / 7, c = e % 7;
      double v = 0.0;
      if (r < 3 && c < 3) {
        v = s_inv * sR[3 * c + r];
      } else if (r < 3 && c < 6) {
        const int cc = c - 3;  // row r of [t']x times column cc of R' (row cc of R_i)
        const double x0 = r == 0 ? 0.0 : r == 1 ? s_tp[2] : -s_tp[1];
        const double x1 = r == 0 ? -s_tp[2] : r == 1 ? 0.0 : s_tp[0];
        const double x2 = r == 0 ? s_tp[1] : r == 1 ? -s_tp[0] : 0.0;
        v = x0 * sR[3 * cc] + x1 * sR[3 * cc + 1] + x2 * sR[3 * cc + 2];
      } else if (r < 3) {
        v = -s_tp[r];
      } else if (r < 6 && c >= 3 && c < 6) {
        v = sR[3 * (c - 3) + (r - 3)];
      } else if (r == 6 && c == 6) {
        v = 1.0;
      }
      A[e] = v;
    }
  }
  __syncthreads();
  if (tid < kNumAcc) {
    double sum = 0.0;
    for (int w = 0; w < kGroups; ++w) sum += Sg[w][tid];
    S[tid] = sum;
  }
  __syncthreads();
  // the relative system Hr, C = Hr A, then H7 = A^T C and g7 = +-A^T g_rel
  // (entries in parallel lanes)
  if (tid < 49) Hr[tid] = hr_entry(S, tid / 7, tid % 7);
  __syncthreads();
  if (tid < 49) {
    const int r = tid / 7, c = tid % 7;
    double v = 0.0;
    for (int k = 0; k < 7; ++k) v += Hr[7 * r + k] * A[7 * k + c];
    C[tid] = v;
  }
  __syncthreads();
  if (tid < 49) {
    const int r = tid / 7, c = tid % 7;
    double v = 0.0;
    for (int k = 0; k < 7; ++k) v += A[7 * k + r] * C[7 * k + c];
    H7[tid] = v;
  }
  if (tid >= 64 && tid < 71) {
    const int r = tid - 64;
    double v = 0.0;
    for (int k = 0; k < 7; ++k) v += A[7 * k + r] * S[21 + k];
    g7[r] = sgn * v;
  }
  __syncthreads();
  if (warp == 0) {
    double t = 0.0;
    const bool ok = track_mixed_solve(H7, g7, lane, &t);
    if (ok) {
      double mx = lane < 7 ? fabs(t) : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      if (lane < 7) s_tau[lane] = t;
      if (lane == 0) {
        s_mx = mx;
        s_status = 0;
      }
    }
    if (lane == 0) s_fb = ok ? 0 : 1;
  }
  __syncthreads();
  if (s_fb && tid == 0) {
    // FP64 Cholesky H7 = L L^T (lower triangle in place), pivots checked
    // against the diagonal as in the FP64 solve, then tau = -H7^-1 g7
    // (reciprocal pivots from rsqrt_newton)
    double L[49], diag[7], tau[7], il[7];
    for (int k = 0; k < 49; ++k) L[k] = H7[k];
    for (int j = 0; j < 7; ++j) diag[j] = H7[8 * j];
    int status = 0;
    for (int j = 0; j < 7 && status == 0; ++j) {
      double d = L[8 * j];
      for (int k = 0; k < j; ++k) d -= L[7 * j + k] * L[7 * j + k];
      if (!(d > 1e-12 * diag[j]) || !isfinite(d)) {
        status = MSLAM_ERR_NOT_PD;
        break;
      }
      il[j] = rsqrt_newton(d);  // 1 / L_jj
      L[8 * j] = d * il[j];
      for (int i = j + 1; i < 7; ++i) {
        double v = L[7 * i + j];
        for (int k = 0; k < j; ++k) v -= L[7 * i + k] * L[7 * j + k];
        L[7 * i + j] = v * il[j];
      }
    }
    if (status == 0) {
      double y[7];
      for (int i = 0; i < 7; ++i) {
        double v = -g7[i];
        for (int k = 0; k < i; ++k) v -= L[7 * i + k] * y[k];
        y[i] = v * il[i];
      }
      for (int i = 6; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < 7; ++k) v -= L[7 * k + i] * tau[k];
        tau[i] = v * il[i];
      }
      double mx = 0.0;
      bool finite = true;
      for (int a = 0; a < 7; ++a) {
        finite = finite && isfinite(tau[a]);
        mx = fmax(mx, fabs(tau[a]));
        s_tau[a] = tau[a];
      }
      if (!finite) status = MSLAM_ERR_NONFINITE;
      s_mx = mx;
    }
    s_status = status;
  }
  __syncthreads();
  const int status0 = s_status;
  // Exp(tau): its transcendental pieces in different warps side by side
  if (status0 == 0 && lane == 0) sim3_exp_piece(s_tau, warp, s_part);
  __syncthreads();
  double* Tk = T_wc + 8 * k_free;
  if (status0 == 0) {
    // Exp(tau) = (t_E = V rho, q_E, s_E = e^sigma), V = a I + b [phi]x + c [phi]x^2
    // (the formulas of sim3_exp_parts, with Newton reciprocals), composed
    // with T_k: t = s_E R_E t_k + t_E by three lanes of warp 0 (each forms b,
    // c and q_E itself), q = q_E (x) q_k normalised by four lanes of warp 1,
    // s = s_E s_k by warp 2; no barrier between the pieces and the result
    const double px = s_tau[3], py = s_tau[4], pz = s_tau[5], sg = s_tau[6];
    const double th2 = px * px + py * py + pz * pz;
    // q_E, normalised: the half-angle terms of piece 2
    const double hq = s_part[3], q3 = s_part[4];
    if (warp == 0 && lane < 3) {
      const double iqn = rsqrt_newton(hq * hq * th2 + q3 * q3);
      const double a = s_part[5];
      double b, c;
      if (s_part[1] == 0.0) {  // the small-angle branch (piece 0 left sin and cos at 0)
        b = s_part[6] - th2 * s_part[7] * (1.0 / 6.0);
        c = 0.5 * s_part[8] - th2 * s_part[9] * (1.0 / 24.0);
      } else {
        const double ith = rsqrt_newton(th2), th = th2 * ith;
        const double sn = s_part[0], cs = s_part[1], es = s_part[2];
        const double iden = rcp_newton(sg * sg + th2);
        const double ic = ((es * cs - 1.0) * sg + es * th * sn) * iden;  // int e^{sx} cos(th x)
        const double is = (es * sn * sg - (es * cs - 1.0) * th) * iden;  // int e^{sx} sin(th x)
        b = is * ith;
        c = (a - ic) * (ith * ith);
      }
      const int r = lane;
      const double r0 = s_tau[0], r1 = s_tau[1], r2 = s_tau[2];
      // phi x rho and phi x (phi x rho)
      const double c0 = py * r2 - pz * r1, c1 = pz * r0 - px * r2, c2 = px * r1 - py * r0;
      const double d0 = py * c2 - pz * c1, d1 = pz * c0 - px * c2, d2 = px * c1 - py * c0;
      const double rr = r == 0 ? r0 : r == 1 ? r1 : r2;
      const double cr = r == 0 ? c0 : r == 1 ? c1 : c2;
      const double dr = r == 0 ? d0 : r == 1 ? d1 : d2;
      const double tE = a * rr + b * cr + c * dr;
      const double qx = hq * px * iqn, qy = hq * py * iqn, qz = hq * pz * iqn, qw = q3 * iqn;
      const double v = rot_entry4(qx, qy, qz, qw, r, 0) * s_Tk[0] + rot_entry4(qx, qy, qz, qw, r, 1) * s_Tk[1] +
                       rot_entry4(qx, qy, qz, qw, r, 2) * s_Tk[2];
      Tk[r] = s_part[2] * v + tE;
    }
    if (warp == 1 && lane < 4) {
      const double iqn = rsqrt_newton(hq * hq * th2 + q3 * q3);
      const double ax = hq * px * iqn, ay = hq * py * iqn, az = hq * pz * iqn, aw = q3 * iqn;
      const double bx = s_Tk[3], by = s_Tk[4], bz = s_Tk[5], bw = s_Tk[6];
      // (q_E (x) q_k)_lane
      double v;
      if (lane == 3) v = aw * bw - (ax * bx + ay * by + az * bz);
      else if (lane == 0) v = aw * bx + bw * ax + (ay * bz - az * by);
      else if (lane == 1) v = aw * by + bw * ay + (az * bx - ax * bz);
      else v = aw * bz + bw * az + (ax * by - ay * bx);
      double n2 = v * v;
      n2 += __shfl_xor_sync(0xfu, n2, 1);
      n2 += __shfl_xor_sync(0xfu, n2, 2);
      Tk[3 + lane] = v * rsqrt_newton(n2);
    }
    if (warp == 2 && lane == 0) Tk[7] = s_part[2] * s_Tk[7];
  }
  if (tid == 0) {
    int status = status0;
    if (status == 0 && s_mx < conv_tol) status = 1;
    if (status != 0) dev_status[g] = status;
    done[tl.edge] = 0;  // ready for the next iteration
  }
}

// The tile counter of the persistent launches: after the relative poses in
// the linearisation workspace.
static int* tile_counter(RelPose* rel, int E) {
  return reinterpret_cast<int*>(reinterpret_cast<char*>(rel) + ((sizeof(RelPose) * (size_t)std::max(E, 1) + 255) &
                                                                ~size_t(255)));
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

// The kernel of the packed linearisation for these parameters and plan:
// the FP16 ray family takes the block-streamed form (plan option lin_form
// 0) or the warp-streamed form (lin_form 2); lin_form 1, FP32 records and
// the other families take the register pipeline.
enum PackedForm { kFormRegs = 0, kFormBlockStream = 1, kFormWarpStream = 2, kFormRegsRing = 3 };
static PackedForm packed_form(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt) {
  if (p->residual != MSLAM_RES_RAY || dt != MSLAM_F16) return kFormRegs;
  const int f = plan_lin_form(plan);
  return f == 0 ? kFormBlockStream : f == 2 ? kFormWarpStream : f == 3 ? kFormRegsRing : kFormRegs;
}

// Opt a streamed kernel into its dynamic shared memory, once per device.
template <PackedForm kForm, typename K>
static mslam_status stream_kernel_setup(K kernel, size_t smem) {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  mslam_status st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (st != MSLAM_OK) return st;
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return MSLAM_OK;
  st = cuda_check(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                  "cudaFuncSetAttribute");
  if (st != MSLAM_OK) return st;
  if (dev >= 0 && dev < 64) done[dev] = true;
  return MSLAM_OK;
}

// Weights and constants of the residual family chosen in the parameters.
static mslam_status make_lin_const(const mslam_params* p, LinConst* lc, const char* who) {
  if (p->residual < MSLAM_RES_RAY || p->residual > MSLAM_RES_PIXEL) {
    set_error("%s: unknown residual family %d", who, (int)p->residual);
    return MSLAM_ERR_ARG;
  }
  bool ok = p->huber_delta > 0.0f;
  if (p->residual == MSLAM_RES_RAY) ok = ok && p->sigma_ray > 0.0f && p->sigma_dist > 0.0f;
  if (p->residual == MSLAM_RES_POINT) ok = ok && p->sigma_point > 0.0f;
  if (p->residual == MSLAM_RES_PIXEL)
    ok = ok && p->sigma_pixel > 0.0f && p->sigma_depth > 0.0f && p->fx > 0.0f && p->fy > 0.0f &&
         std::isfinite(p->fx) && std::isfinite(p->fy) && std::isfinite(p->cx) && std::isfinite(p->cy);
  if (!ok) {
    set_error("%s: the sigmas of the residual family and huber_delta must be positive (and fx, fy > 0 for the "
              "pixel family)", who);
    return MSLAM_ERR_ARG;
  }
  lc->inv_sr2 = 1.0f / (p->sigma_ray * p->sigma_ray);
  lc->inv_sd2 = 1.0f / (p->sigma_dist * p->sigma_dist);
  lc->delta = p->huber_delta;
  lc->delta2 = p->huber_delta * p->huber_delta;
  lc->q_min = p->q_min;
  lc->inv_s1 = p->residual == MSLAM_RES_POINT ? 1.0f / (p->sigma_point * p->sigma_point)
                                              : 1.0f / (p->sigma_pixel * p->sigma_pixel);
  lc->inv_s2 = 1.0f / (p->sigma_depth * p->sigma_depth);
  lc->fx = p->fx;
  lc->fy = p->fy;
  lc->cx = p->cx;
  lc->cy = p->cy;
  return MSLAM_OK;
}

// Calls f with the residual family as a compile-time constant.
template <typename F>
static void with_family(int kind, F&& f) {
  if (kind == MSLAM_RES_POINT)
    f(std::integral_constant<int, MSLAM_RES_POINT>{});
  else if (kind == MSLAM_RES_PIXEL)
    f(std::integral_constant<int, MSLAM_RES_PIXEL>{});
  else
    f(std::integral_constant<int, MSLAM_RES_RAY>{});
}

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
  LinConst lc;
  const mslam_status st = make_lin_const(p, &lc, "gn_linearize");
  if (st != MSLAM_OK) return st;
  const PlanView pv = plan_view(plan);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* partials = static_cast<float*>(workspace);
  RelPose* rel = reinterpret_cast<RelPose*>(static_cast<char*>(workspace) + lin_partials_bytes(pv.n_tiles));
  int* ctr = tile_counter(rel, pv.E);
  rel_pose_kernel<<<(pv.E + 127) / 128, 128, 0, s>>>(pv, T_wc, rel, ctr);
  with_family(p->residual, [&](auto K) {
    constexpr int kK = decltype(K)::value;
    auto launch = [&](int grid, int t0, int t1, int* c) {
      if (dt == MSLAM_F32)
        lin_tiles_kernel<float, kK><<<grid, kLinThreads, 0, s>>>(pv, lc, rel, static_cast<const float*>(X_canon),
                                                                idx, static_cast<const float*>(q), partials, t0, t1,
                                                                c);
      else
        lin_tiles_kernel<__half, kK><<<grid, kLinThreads, 0, s>>>(pv, lc, rel, static_cast<const __half*>(X_canon),
                                                                 idx, static_cast<const __half*>(q), partials, t0,
                                                                 t1, c);
    };
    if (flags & MSLAM_FLAG_PER_EDGE) {
      // plain form: a host loop of per-edge launches
      for (int e = 0; e < pv.E; ++e) {
        int t0, t1;
        plan_edge_tiles(plan, e, &t0, &t1);
        launch(t1 - t0, t0, t1, nullptr);
        lin_finalize_kernel<<<1, kFinalizeThreads, 0, s>>>(pv, T_wc, partials, H_blocks, g_blocks, cost, n_valid, e, kK);
      }
    } else {
      launch(std::min(pv.n_tiles, persistent_grid(plan, lin_tiles_kernel<float, kK>)), 0, pv.n_tiles, ctr);
      lin_finalize_kernel<<<pv.E, kFinalizeThreads, 0, s>>>(pv, T_wc, partials, H_blocks, g_blocks, cost, n_valid, 0, kK);
    }
  });
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
  if (p->residual < MSLAM_RES_RAY || p->residual > MSLAM_RES_PIXEL) {
    set_error("gn_pack: unknown residual family %d", (int)p->residual);
    return MSLAM_ERR_ARG;
  }
  if (p->residual == MSLAM_RES_PIXEL && dt == MSLAM_F16 && plan_max_image_dim(plan) > 2048) {
    set_error("gn_pack: FP16 records hold pixel coordinates exactly only up to 2048; use MSLAM_F32");
    return MSLAM_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint4* recs = static_cast<uint4*>(packed);
  int32_t* counts = reinterpret_cast<int32_t*>(static_cast<char*>(packed) + pack_bytes(pv.n_tiles, pv.lin_tile, dt) -
                                               (((size_t)pv.n_tiles * sizeof(int32_t) + 255) & ~size_t(255)));
  if (dt == MSLAM_F32)
    pack_kernel<float><<<pv.n_tiles, kPackThreads, 0, s>>>(pv, p->q_min, p->residual, static_cast<const float*>(X_canon), idx,
                                                          static_cast<const float*>(q), recs, counts);
  else
    pack_kernel<__half><<<pv.n_tiles, kPackThreads, 0, s>>>(pv, p->q_min, p->residual, static_cast<const __half*>(X_canon), idx,
                                                           static_cast<const __half*>(q), recs, counts);
  return cuda_check(cudaGetLastError(), "gn_pack launch");
}

extern "C" mslam_status mslam_gn_linearize_packed(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt,
                                                  const double* T_wc, const void* packed, size_t packed_bytes,
                                                  float* H_blocks, float* g_blocks, double* cost, int32_t* n_valid,
                                                  int32_t* dev_status, void* workspace, size_t ws_bytes,
                                                  uint32_t flags, void* stream) {
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
  LinConst lc;
  const mslam_status st = make_lin_const(p, &lc, "gn_linearize_packed");
  if (st != MSLAM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* partials = static_cast<float*>(workspace);
  RelPose* rel = reinterpret_cast<RelPose*>(static_cast<char*>(workspace) + lin_partials_bytes(pv.n_tiles));
  const uint4* recs = static_cast<const uint4*>(packed);
  const int32_t* counts = reinterpret_cast<const int32_t*>(
      static_cast<const char*>(packed) + pack_bytes(pv.n_tiles, pv.lin_tile, dt) -
      (((size_t)pv.n_tiles * sizeof(int32_t) + 255) & ~size_t(255)));
  int* ctr = tile_counter(rel, pv.E);
  rel_pose_kernel<<<(pv.E + 127) / 128, 128, 0, s>>>(pv, T_wc, rel, ctr);
  const size_t stream_smem = (size_t)kStreamStages * kStreamChunkBytes;
  const PackedForm form = packed_form(p, plan, dt);
  if (form == kFormBlockStream || form == kFormWarpStream) {
    mslam_status st2 = form == kFormBlockStream
                           ? stream_kernel_setup<kFormBlockStream>(lin_stream_kernel, stream_smem)
                           : stream_kernel_setup<kFormWarpStream>(lin_warp_stream_kernel, kWarpStreamSmem);
    if (st2 != MSLAM_OK) return st2;
  }
  const unsigned char* rec_bytes = static_cast<const unsigned char*>(packed);
  with_family(p->residual, [&](auto K) {
    constexpr int kK = decltype(K)::value;
    auto launch = [&](int grid, int t0, int t1, int* c) {
      // the FP16 ray family streams its records through shared memory
      if (kK == MSLAM_RES_RAY && form == kFormBlockStream) {
        lin_stream_kernel<<<grid, kStreamThreads, stream_smem, s>>>(pv, lc, rel, rec_bytes, counts, partials, t0, t1,
                                                                   c, dev_status);
        return;
      }
      if (kK == MSLAM_RES_RAY && form == kFormWarpStream) {
        // a warp takes a whole tile: without the counter, one warp per tile
        const int g = c ? grid : (t1 - t0 + kWarpStreamWarps - 1) / kWarpStreamWarps;
        lin_warp_stream_kernel<<<g, kWarpStreamThreads, kWarpStreamSmem, s>>>(pv, lc, rel, rec_bytes, counts,
                                                                             partials, t0, t1, c, dev_status);
        return;
      }
      if (dt == MSLAM_F32)
        lin_packed_kernel<float, kK, false><<<grid, kLinThreads, 0, s>>>(pv, lc, rel, recs, counts, partials, t0,
                                                                         t1, c);
      else if (form == kFormRegsRing)
        lin_packed_kernel<__half, kK, true><<<grid, kLinThreads, 0, s>>>(pv, lc, rel, recs, counts, partials, t0,
                                                                         t1, c);
      else
        lin_packed_kernel<__half, kK, false><<<grid, kLinThreads, 0, s>>>(pv, lc, rel, recs, counts, partials, t0,
                                                                          t1, c);
    };
    if (flags & MSLAM_FLAG_PER_EDGE) {
      for (int e = 0; e < pv.E; ++e) {
        int t0, t1;
        plan_edge_tiles(plan, e, &t0, &t1);
        launch(t1 - t0, t0, t1, nullptr);
        lin_finalize_kernel<<<1, kFinalizeThreads, 0, s>>>(pv, T_wc, partials, H_blocks, g_blocks, cost, n_valid, e, kK);
      }
    } else {
      int grid = form == kFormRegsRing ? persistent_grid(plan, lin_packed_kernel<__half, kK, true>)
                                       : persistent_grid(plan, lin_packed_kernel<__half, kK, false>);
      if (kK == MSLAM_RES_RAY && (form == kFormBlockStream || form == kFormWarpStream)) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = std::max(1, sms);  // one streaming CTA per SM
      }
      launch(std::min(pv.n_tiles, grid), 0, pv.n_tiles, ctr);
      lin_finalize_kernel<<<pv.E, kFinalizeThreads, 0, s>>>(pv, T_wc, partials, H_blocks, g_blocks, cost, n_valid, 0, kK);
    }
  });
  return cuda_check(cudaGetLastError(), "gn_linearize_packed launch");
}

extern "C" mslam_status mslam_gn_track(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt, double* T_wc,
                                       const void* packed, size_t packed_bytes, int32_t n_iters,
                                       int32_t* dev_status, void* workspace, size_t ws_bytes, void* stream) {
  if (!p || !check_plan_uploaded(plan)) {
    if (!p) set_error("params is NULL");
    return MSLAM_ERR_ARG;
  }
  if (dt != MSLAM_F32 && dt != MSLAM_F16) {
    set_error("unsupported dtype %d", (int)dt);
    return MSLAM_ERR_ARG;
  }
  if (!plan_tracking_form(plan)) {
    set_error("gn_track: every graph of the plan must be one keyframe and one frame joined by one edge");
    return MSLAM_ERR_ARG;
  }
  if (p->residual != MSLAM_RES_RAY) {
    set_error("gn_track: only the ray residual family (residual %d given)", (int)p->residual);
    return MSLAM_ERR_ARG;
  }
  if (n_iters < 0) {
    set_error("gn_track: n_iters %d < 0", (int)n_iters);
    return MSLAM_ERR_ARG;
  }
  if (!T_wc || !packed || !dev_status || !workspace) {
    set_error("gn_track: NULL device pointer");
    return MSLAM_ERR_ARG;
  }
  const PlanView pv = plan_view(plan);
  if (packed_bytes < pack_bytes(pv.n_tiles, pv.lin_tile, dt) || (reinterpret_cast<uintptr_t>(packed) & 255)) {
    set_error("gn_track: packed buffer smaller than %zu bytes or not 256-byte aligned",
              pack_bytes(pv.n_tiles, pv.lin_tile, dt));
    return MSLAM_ERR_ARG;
  }
  if (ws_bytes < mslam_workspace_bytes(plan, MSLAM_OP_TRACK) || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    set_error("gn_track: workspace smaller than %zu bytes or not 256-byte aligned",
              mslam_workspace_bytes(plan, MSLAM_OP_TRACK));
    return MSLAM_ERR_ARG;
  }
  LinConst lc;
  const mslam_status st = make_lin_const(p, &lc, "gn_track");
  if (st != MSLAM_OK) return st;
  if (n_iters == 0) return MSLAM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* partials = static_cast<float*>(workspace);
  int32_t* done = reinterpret_cast<int32_t*>(static_cast<char*>(workspace) + lin_partials_bytes(pv.n_tiles));
  const uint4* recs = static_cast<const uint4*>(packed);
  const int32_t* counts = reinterpret_cast<const int32_t*>(
      static_cast<const char*>(packed) + pack_bytes(pv.n_tiles, pv.lin_tile, dt) -
      (((size_t)pv.n_tiles * sizeof(int32_t) + 255) & ~size_t(255)));
  mslam_status st2 = cuda_check(cudaMemsetAsync(done, 0, sizeof(int32_t) * (size_t)pv.E, s), "gn_track memset");
  if (st2 != MSLAM_OK) return st2;
  for (int it = 0; it < n_iters; ++it) {
    if (dt == MSLAM_F32)
      track_kernel<float><<<pv.n_tiles, kLinThreads, 0, s>>>(pv, lc, p->conv_tol, T_wc, recs, counts, partials,
                                                             done, dev_status);
    else
      track_kernel<__half><<<pv.n_tiles, kLinThreads, 0, s>>>(pv, lc, p->conv_tol, T_wc, recs, counts, partials,
                                                              done, dev_status);
  }
  return cuda_check(cudaGetLastError(), "gn_track launch");
}
