// (a1-a3) Iterative projective matching with feature refinement, Sec. 3.2.
//
// One thread per query pixel, blocks of 256 query pixels (32 x 8 by default,
// a plan option) so that a
// block's bilinear taps and refinement windows fall in a compact region of
// the reference image (served from L1/L2).  Per pixel:
//   a1  the reference camera model psi(X_ref) is evaluated at the four
//       bilinear taps of every iteration (a zero or non-finite reference
//       point has the zero ray);
//   a2  lm_iters Levenberg-Marquardt steps on |R(p) - psi(x)|^2 (Eq. 2) with
//       the analytic 3x2 Jacobian of the bilinear cell and a closed-form 2x2
//       solve, p clamped to the image;
//   a3  rounding, coarse-to-fine descriptor window argmax (FP32 dot products
//       in index order), the 3D distance test and q = sqrt(Q_ref Q_qry).
#include <algorithm>
#include <climits>
#include <type_traits>

#include "common.cuh"

namespace mslam {

struct MatchConst {
  float lm_lambda, max_rel;
  int lm_iters, radius, n_levels;
  int dil[4];
};

template <typename T>
__device__ __forceinline__ float3 ray_at(const T* X, int64_t pix) {
  const float3 a = ld3(X, pix);
  const float n2 = fmaf(a.x, a.x, fmaf(a.y, a.y, a.z * a.z));
  if (!(n2 > 0.0f && n2 < INFINITY)) return make_float3(0.0f, 0.0f, 0.0f);
  const float inv = rsqrtf(n2);
  return make_float3(a.x * inv, a.y * inv, a.z * inv);
}

// Descriptors are stored chunk-planar: [d / C][P][C] with C = 16 bytes of
// elements (8 halves or 4 floats), P = pixels of the whole edge pool, so that
// a warp reading one chunk of 32 neighbouring pixels reads 512 contiguous
// bytes.  Dot products accumulate in FP32 in channel order.
template <typename T, int D> struct Desc;

template <int D> struct Desc<float, D> {
  using Q = float4;  // query descriptor kept as D / 4 float4
  static constexpr int NQ = D / 4;
  static __device__ __forceinline__ void load(const float* base, int64_t P, int64_t pix, Q* q) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < NQ; ++k) q[k] = __ldg(b + (int64_t)k * P + pix);
  }
  static __device__ __forceinline__ float dot(const float* base, int64_t P, int64_t pix, const Q* q) {
    const float4* b = reinterpret_cast<const float4*>(base);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const float4 v = __ldg(b + (int64_t)k * P + pix);
      s = fmaf(q[k].x, v.x, s);
      s = fmaf(q[k].y, v.y, s);
      s = fmaf(q[k].z, v.z, s);
      s = fmaf(q[k].w, v.w, s);
    }
    return s;
  }
};

// s += lo(a) lo(b); s += hi(a) hi(b) with the FP16 x FP16 -> FP32 fused
// multiply-add (the product of two halves is exact in FP32, so this equals
// converting both to float and using fmaf)
__device__ __forceinline__ void fma_h2(float& s, uint32_t a, uint32_t b) {
  asm("{\n\t.reg .b16 a0, a1, b0, b1;\n\t"
      "mov.b32 {a0, a1}, %1;\n\t"
      "mov.b32 {b0, b1}, %2;\n\t"
      "fma.rn.f32.f16 %0, a0, b0, %0;\n\t"
      "fma.rn.f32.f16 %0, a1, b1, %0;\n\t}"
      : "+f"(s)
      : "r"(a), "r"(b));
}

template <int D> struct Desc<__half, D> {
  using Q = uint4;  // query descriptor kept as D / 8 packed uint4 (8 halves each)
  static constexpr int NQ = D / 8;
  static __device__ __forceinline__ void load(const __half* base, int64_t P, int64_t pix, Q* q) {
    const uint4* b = reinterpret_cast<const uint4*>(base);
#pragma unroll
    for (int k = 0; k < NQ; ++k) q[k] = __ldg(b + (int64_t)k * P + pix);
  }
  static __device__ __forceinline__ float dot(const __half* base, int64_t P, int64_t pix, const Q* q) {
    const uint4* b = reinterpret_cast<const uint4*>(base);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const uint4 v = __ldg(b + (int64_t)k * P + pix);
      fma_h2(s, q[k].x, v.x);
      fma_h2(s, q[k].y, v.y);
      fma_h2(s, q[k].z, v.z);
      fma_h2(s, q[k].w, v.w);
    }
    return s;
  }
};

// a1 materialised: the unit rays psi(X_ref) of pool pixels [p0, p1) as
// float4 (x, y, z, 0), with ray_at's arithmetic (the zero ray for a zero or
// non-finite point), so that the LM taps read one 16-byte value each.
template <typename T>
__global__ void __launch_bounds__(256) ray4_kernel(const T* __restrict__ X, float4* __restrict__ R4, int64_t p0,
                                                   int64_t p1) {
  for (int64_t i = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p1; i += (int64_t)gridDim.x * blockDim.x) {
    const float3 r = ray_at(X, i);
    R4[i] = make_float4(r.x, r.y, r.z, 0.0f);
  }
}

// a2: lm_iters Levenberg-Marquardt steps of the ray error |R(p) - tg|^2
// (Eq. 2) from p = (pu, pv_), R bilinear in the unit rays of the cell
// (clamp(floor u, 0, W-2), clamp(floor v, 0, H-2)), p clamped to the image
// after each step.
// With R4_e != nullptr the unit rays come from the ray image [pixels] of
// float4 (x, y, z, 0) that ray4_kernel wrote with the same FP32 arithmetic
// as ray_at (one 16-byte load per tap, no normalisation per iteration).
// An iteration is a pure function of p: once a step leaves p unchanged (the
// update rounds away), every later step would too, so the loop stops there
// with exactly the p of all lm_iters steps.
template <typename T>
__device__ __forceinline__ float3 tap(const T* __restrict__ Xr_e, const float4* __restrict__ R4_e, int64_t pix) {
  if (R4_e) {
    const float4 r = __ldg(R4_e + pix);
    return make_float3(r.x, r.y, r.z);
  }
  return ray_at(Xr_e, pix);
}

template <typename T>
__device__ __forceinline__ void lm_iterate(const T* __restrict__ Xr_e, const float4* __restrict__ R4_e, int W, int H,
                                           float3 tg, const MatchConst& mc, float& pu, float& pv_) {
  const float lam = mc.lm_lambda;
  for (int it = 0; it < mc.lm_iters; ++it) {
    const float pu_in = pu, pv_in = pv_;
    const int u0 = min(max((int)floorf(pu), 0), W - 2);
    const int v0 = min(max((int)floorf(pv_), 0), H - 2);
    const float a = pu - (float)u0, b = pv_ - (float)v0;
    const int64_t t00 = (int64_t)v0 * W + u0;
    const float3 R00 = tap(Xr_e, R4_e, t00), R10 = tap(Xr_e, R4_e, t00 + 1);
    const float3 R01 = tap(Xr_e, R4_e, t00 + W), R11 = tap(Xr_e, R4_e, t00 + W + 1);
    // every product and sum is rounded where written (explicit fused
    // multiply-adds, no contraction left to the compiler), so that each form
    // of the kernel takes the same LM path for the same inputs
    const float ua = 1.0f - a, ub = 1.0f - b;
    const float3 Ju = make_float3(fmaf(ub, R10.x - R00.x, __fmul_rn(b, R11.x - R01.x)),
                                  fmaf(ub, R10.y - R00.y, __fmul_rn(b, R11.y - R01.y)),
                                  fmaf(ub, R10.z - R00.z, __fmul_rn(b, R11.z - R01.z)));
    const float3 Jv = make_float3(fmaf(ua, R01.x - R00.x, __fmul_rn(a, R11.x - R10.x)),
                                  fmaf(ua, R01.y - R00.y, __fmul_rn(a, R11.y - R10.y)),
                                  fmaf(ua, R01.z - R00.z, __fmul_rn(a, R11.z - R10.z)));
    const float w00 = __fmul_rn(ua, ub), w10 = __fmul_rn(a, ub), w01 = __fmul_rn(ua, b), w11 = __fmul_rn(a, b);
    const float rx = fmaf(w11, R11.x, fmaf(w01, R01.x, fmaf(w10, R10.x, fmaf(w00, R00.x, -tg.x))));
    const float ry = fmaf(w11, R11.y, fmaf(w01, R01.y, fmaf(w10, R10.y, fmaf(w00, R00.y, -tg.y))));
    const float rz = fmaf(w11, R11.z, fmaf(w01, R01.z, fmaf(w10, R10.z, fmaf(w00, R00.z, -tg.z))));
    const float a00 = fmaf(Ju.z, Ju.z, fmaf(Ju.y, Ju.y, fmaf(Ju.x, Ju.x, lam)));
    const float a01 = fmaf(Ju.z, Jv.z, fmaf(Ju.y, Jv.y, __fmul_rn(Ju.x, Jv.x)));
    const float a11 = fmaf(Jv.z, Jv.z, fmaf(Jv.y, Jv.y, fmaf(Jv.x, Jv.x, lam)));
    const float b0 = -fmaf(Ju.z, rz, fmaf(Ju.y, ry, __fmul_rn(Ju.x, rx)));
    const float b1 = -fmaf(Jv.z, rz, fmaf(Jv.y, ry, __fmul_rn(Jv.x, rx)));
    const float det = fmaf(a00, a11, -__fmul_rn(a01, a01));
    if (det > 0.0f) {
      pu = __fadd_rn(pu, __fdiv_rn(fmaf(a11, b0, -__fmul_rn(a01, b1)), det));
      pv_ = __fadd_rn(pv_, __fdiv_rn(fmaf(a00, b1, -__fmul_rn(a01, b0)), det));
    }
    // clamp (fmaxf/fminf also map a NaN to the image)
    pu = fminf(fmaxf(pu, 0.0f), (float)(W - 1));
    pv_ = fminf(fmaxf(pv_, 0.0f), (float)(H - 1));
    if (pu == pu_in && pv_ == pv_in) break;  // a fixed point: the remaining steps change nothing
  }
}

// kR > 0: the window radius as a compile-time constant (the default 3), so
// that each window row is unrolled with branch-free bounds (an out-of-image
// candidate reads a clamped pixel and scores -inf, which never wins, exactly
// as if it were skipped); kR = 0 takes the radius from the parameters.
// Keyframe-criterion counts (Sec. 3.4) taken in the matching epilogue: a
// valid match of edge e sets bit bit_off(e) + m of `bits` (its reference
// pixel) and adds to n_valid[e].  bit_off(e) = 32 ceil(e_off[e] / 32) + 32 e
// starts every edge on its own 32-bit word, so that calls on edge ranges
// never share a word.  bits == nullptr: no counts.
struct MatchStats {
  uint32_t* bits;
  int32_t* n_valid;
  int e_begin, e_end, block_base;  // the launch's edge range and first block (to find a block's edge)
};
__host__ __device__ __forceinline__ int64_t stats_bit_off(int64_t off_e, int e) {
  return ((off_e + 31) / 32) * 32 + 32 * (int64_t)e;
}
__device__ __forceinline__ int match_block_edge(const PlanView& pv, int gb, int e_begin, int e_end);
__device__ __forceinline__ void stats_epilogue(const PlanView& pv, const MatchStats& st, int64_t off_e, int m,
                                               bool ok) {
  if (!st.bits) return;
  const int e = match_block_edge(pv, st.block_base + blockIdx.x, st.e_begin, st.e_end);
  if (ok) {
    const int64_t b = stats_bit_off(off_e, e) + m;
    atomicOr(st.bits + (b >> 5), 1u << (b & 31));
  }
  const unsigned am = __activemask();
  const unsigned bal = __ballot_sync(am, ok);
  if ((threadIdx.x & 31) == __ffs(am) - 1 && bal) atomicAdd(st.n_valid + e, __popc(bal));
}

// Edge of match block gb: the last edge in [e_begin, e_end) whose first
// block <= gb.
__device__ __forceinline__ int match_block_edge(const PlanView& pv, int gb, int e_begin, int e_end) {
  int lo = e_begin, hi = e_end - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pv.edges[mid].mblock_begin <= gb) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The per-query matching (a1-a3) of query pixel (u, v) of edge ed.
template <typename T, int D, int kR>
__device__ __forceinline__ void match_query(const PlanView& pv, const MatchConst& mc, const DevEdge& ed, int u,
                                            int v, const MatchStats& st,
                                            const T* __restrict__ Xr, const T* __restrict__ Xq,
                                            const T* __restrict__ Dr, const T* __restrict__ Dq,
                                            const T* __restrict__ Qr, const T* __restrict__ Qq,
                                            const int32_t* __restrict__ init, int32_t* __restrict__ out_idx,
                                            T* __restrict__ out_q, const float4* __restrict__ R4) {
  const int W = ed.W, H = ed.H;
  if (u >= W || v >= H) return;
  const int64_t HW = (int64_t)H * W;
  const int n = v * W + u;
  const int64_t o = ed.off_e;
  const T* Xr_e = Xr + 3 * o;
  const float3 x = ld3(Xq + 3 * o, n);
  const float nx2 = fmaf(x.x, x.x, fmaf(x.y, x.y, x.z * x.z));
  if (!(finite3(x) && nx2 > 0.0f)) {
    out_idx[o + n] = -1;
    stf(out_q + o + n, 0.0f);
    return;
  }
  const float inx = rsqrtf(nx2);
  const float3 tg = make_float3(x.x * inx, x.y * inx, x.z * inx);
  int p0 = n;
  if (init) {
    const int32_t ii = init[o + n];
    if (ii >= 0 && ii < HW) p0 = ii;
  }
  float pu = (float)(p0 % W), pv_ = (float)(p0 / W);
  lm_iterate(Xr_e, R4 ? R4 + o : nullptr, W, H, tg, mc, pu, pv_);
  int cu = min((int)floorf(pu + 0.5f), W - 1), cv = min((int)floorf(pv_ + 0.5f), H - 1);
  // coarse-to-fine refinement: maximum descriptor similarity in a window
  typename Desc<T, D>::Q dq[Desc<T, D>::NQ];
  Desc<T, D>::load(Dq, pv.P, o + n, dq);
  const int r = mc.radius;
  for (int lev = 0; lev < mc.n_levels; ++lev) {
    const int dil = mc.dil[lev];
    float best = -INFINITY;
    int bu = cu, bv = cv;
    if (kR > 0) {
#pragma unroll 1
      for (int dy = -kR; dy <= kR; ++dy) {
        const int vv = cv + dy * dil;
        const bool vin = (unsigned)vv < (unsigned)H;
        const int64_t row = o + (int64_t)min(max(vv, 0), H - 1) * W;
#pragma unroll
        for (int dx = -kR; dx <= kR; ++dx) {
          const int uu = cu + dx * dil;
          const float s0 = Desc<T, D>::dot(Dr, pv.P, row + min(max(uu, 0), W - 1), dq);
          const float s = (vin && (unsigned)uu < (unsigned)W) ? s0 : -INFINITY;
          if (s > best) {
            best = s;
            bu = uu;
            bv = vv;
          }
        }
      }
      cu = bu;
      cv = bv;
      continue;
    }
    for (int dy = -r; dy <= r; ++dy) {
      const int vv = cv + dy * dil;
      if (vv < 0 || vv >= H) continue;
      for (int dx = -r; dx <= r; ++dx) {
        const int uu = cu + dx * dil;
        if (uu < 0 || uu >= W) continue;
        const float s = Desc<T, D>::dot(Dr, pv.P, o + (int64_t)vv * W + uu, dq);
        if (s > best) {
          best = s;
          bu = uu;
          bv = vv;
        }
      }
    }
    cu = bu;
    cv = bv;
  }
  const int m = cv * W + cu;
  const float3 y = ld3(Xr_e, m);
  const float dxv = y.x - x.x, dyv = y.y - x.y, dzv = y.z - x.z;
  const float dist = sqrtf(fmaf(dzv, dzv, fmaf(dyv, dyv, __fmul_rn(dxv, dxv))));
  const bool ok = finite3(y) && dist <= mc.max_rel * sqrtf(nx2);
  out_idx[o + n] = ok ? m : -1;
  stf(out_q + o + n, ok ? sqrtf(ldf(Qr + o + m) * ldf(Qq + o + n)) : 0.0f);
  stats_epilogue(pv, st, o, m, ok);
}

// A block covers match_bx x (match_by * match_ppt) query pixels: each thread
// takes match_ppt queries, match_by rows apart (plan option match_ppt).
template <typename T, int D, int kR, int kPPT>
__global__ void __launch_bounds__(kMatchThreads, 1024 / kMatchThreads) match_kernel(
    PlanView pv, MatchConst mc, const T* __restrict__ Xr, const T* __restrict__ Xq, const T* __restrict__ Dr,
    const T* __restrict__ Dq, const T* __restrict__ Qr, const T* __restrict__ Qq, const int32_t* __restrict__ init,
    int32_t* __restrict__ out_idx, T* __restrict__ out_q, int e_begin, int e_end, int block_base,
    const float4* __restrict__ R4, MatchStats st) {
  const int gb = block_base + blockIdx.x;
  const DevEdge ed = pv.edges[match_block_edge(pv, gb, e_begin, e_end)];
  const int local = gb - ed.mblock_begin;
  const int bx = pv.match_bx, by = pv.match_by;
  const int nbx = (ed.W + bx - 1) / bx;
  const int u = (local % nbx) * bx + (threadIdx.x % bx);
  const int v0 = (local / nbx) * (by * kPPT) + (threadIdx.x / bx);
#pragma unroll 1
  for (int k = 0; k < kPPT; ++k)
    match_query<T, D, kR>(pv, mc, ed, u, v0 + k * by, st, Xr, Xq, Dr, Dq, Qr, Qq, init, out_idx, out_q, R4);
}

// ------------------------------------------------------ staged window form
// The refinement windows scored from shared memory (plan option match_form
// 2; FP16 storage, window radius 3).  Per level, the block takes the
// bounding box of its active queries' windows (centre +- 3 dil, clipped to
// the image).  A box of at most kCap pixels is staged whole; a larger one
// (outlying centres) is cut to at most kBoxW x (kCap / kBoxW) pixels placed
// around the mean centre.  One warp copies the box row by row for every
// descriptor chunk with bulk asynchronous copies (the copy engine; the bytes
// are counted on an mbarrier, waited with the plan's bounded wait).  Every
// query whose window lies inside the box reads its candidates from shared
// memory, every other query from global memory, through one generic load
// whose address selects the space, so that no warp splits into two paths.
// A staged pixel crosses L1 once per block and level instead of once per
// window that contains it, and the eight lanes of a quarter-warp read
// consecutive box pixels (eight different 16-byte bank groups): four
// wavefronts per 16-byte load of a warp, where the scattered global loads
// of the per-query form take about eight.  The candidates, the FP32 dot
// products, their order and the first-maximum rule are those of
// match_kernel, so the matches are identical.  A wait that gives up (or a
// negative wait limit) leaves that level's queries on the global loads and
// stops staging in the block: the result does not change.
template <int D> struct StagedCfg {
  static constexpr int kChunks = D / 8;                   // 16-byte chunks of a descriptor
  static constexpr int kCap = 49152 / (16 * kChunks);     // box pixels in 48 KB of shared memory
  static constexpr int kBoxW = kCap / 32;                 // widest cut box
  static constexpr int kSmem = kCap * kChunks * 16;
};

template <int D, int kPPT>
__global__ void __launch_bounds__(kMatchThreads, 1024 / kMatchThreads) match_staged_kernel(
    PlanView pv, MatchConst mc, const __half* __restrict__ Xr, const __half* __restrict__ Xq,
    const __half* __restrict__ Dr, const __half* __restrict__ Dq, const __half* __restrict__ Qr,
    const __half* __restrict__ Qq, const int32_t* __restrict__ init, int32_t* __restrict__ out_idx,
    __half* __restrict__ out_q, int e_begin, int e_end, int block_base, const float4* __restrict__ R4,
    MatchStats st) {
  using Cfg = StagedCfg<D>;
  constexpr int NQ = Cfg::kChunks;
  constexpr int kWarps = kMatchThreads / 32;
  extern __shared__ __align__(128) uint4 s_desc[];  // [NQ][bh][bw] of the staged box
  __shared__ uint64_t s_bar;
  __shared__ int s_red[kWarps][7];  // per warp: min u, max u, min v, max v, count, sum u, sum v
  __shared__ int s_box[5];          // u0, v0, bw, bh, mode (0 no active query, 1 global only, 2 staged)
  __shared__ int s_dead;            // a wait gave up: no further staging in this block
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int gb = block_base + blockIdx.x;
  const DevEdge ed = pv.edges[match_block_edge(pv, gb, e_begin, e_end)];
  const int local = gb - ed.mblock_begin;
  const int bx = pv.match_bx, by = pv.match_by;
  const int W = ed.W, H = ed.H;
  const int nbx = (W + bx - 1) / bx;
  const int u = (local % nbx) * bx + (tid % bx);
  const int v0 = (local / nbx) * (by * kPPT) + (tid / bx);
  const int64_t o = ed.off_e, HW = (int64_t)H * W;
  const __half* Xr_e = Xr + 3 * o;
  const uint4* Dr4 = reinterpret_cast<const uint4*>(Dr);
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_dead = pv.wait_polls == 0;  // a negative wait limit: no copy is issued
  }
  __syncthreads();
  uint32_t phase = 0;
  bool pending = false;  // thread 0: a copy whose wait gave up may still be in flight
#pragma unroll 1
  for (int k = 0; k < kPPT; ++k) {
    const int v = v0 + k * by;
    const int n = v * W + u;
    bool act = u < W && v < H;
    float3 x = make_float3(0.0f, 0.0f, 0.0f);
    float nx2 = 0.0f;
    int cu = 0, cv = 0;
    uint4 dq[NQ];
    if (act) {
      x = ld3(Xq + 3 * o, n);
      nx2 = fmaf(x.x, x.x, fmaf(x.y, x.y, x.z * x.z));
      if (!(finite3(x) && nx2 > 0.0f)) {
        out_idx[o + n] = -1;
        stf(out_q + o + n, 0.0f);
        act = false;
      }
    }
    if (act) {
      const float inx = rsqrtf(nx2);
      const float3 tg = make_float3(x.x * inx, x.y * inx, x.z * inx);
      int p0 = n;
      if (init) {
        const int32_t ii = init[o + n];
        if (ii >= 0 && ii < HW) p0 = ii;
      }
      float pu = (float)(p0 % W), pv_ = (float)(p0 / W);
      lm_iterate(Xr_e, R4 ? R4 + o : nullptr, W, H, tg, mc, pu, pv_);
      cu = min((int)floorf(pu + 0.5f), W - 1);
      cv = min((int)floorf(pv_ + 0.5f), H - 1);
      const uint4* q4 = reinterpret_cast<const uint4*>(Dq);
#pragma unroll
      for (int c = 0; c < NQ; ++c) dq[c] = __ldg(q4 + (int64_t)c * pv.P + o + n);
    }
#pragma unroll 1
    for (int lev = 0; lev < mc.n_levels; ++lev) {
      const int dil = mc.dil[lev], marg = 3 * dil;
      // the block's bounding box of active centres
      const unsigned full = 0xffffffffu;
      const int r0 = __reduce_min_sync(full, act ? cu : INT_MAX);
      const int r1 = __reduce_max_sync(full, act ? cu : INT_MIN);
      const int r2 = __reduce_min_sync(full, act ? cv : INT_MAX);
      const int r3 = __reduce_max_sync(full, act ? cv : INT_MIN);
      const int r4 = __reduce_add_sync(full, act ? 1 : 0);
      const int r5 = __reduce_add_sync(full, act ? cu : 0);
      const int r6 = __reduce_add_sync(full, act ? cv : 0);
      if (lane == 0) {
        s_red[wid][0] = r0; s_red[wid][1] = r1; s_red[wid][2] = r2; s_red[wid][3] = r3;
        s_red[wid][4] = r4; s_red[wid][5] = r5; s_red[wid][6] = r6;
      }
      __syncthreads();
      if (tid == 0) {
        int umin = INT_MAX, umax = INT_MIN, vmin = INT_MAX, vmax = INT_MIN, cnt = 0, su = 0, sv = 0;
        for (int w = 0; w < kWarps; ++w) {
          umin = min(umin, s_red[w][0]); umax = max(umax, s_red[w][1]);
          vmin = min(vmin, s_red[w][2]); vmax = max(vmax, s_red[w][3]);
          cnt += s_red[w][4]; su += s_red[w][5]; sv += s_red[w][6];
        }
        int mode = cnt == 0 ? 0 : (s_dead ? 1 : 2), bu0 = 0, bv0 = 0, bw = 0, bh = 0;
        if (mode == 2) {
          bu0 = max(umin - marg, 0);
          bv0 = max(vmin - marg, 0);
          const int bu1 = min(umax + marg, W - 1), bv1 = min(vmax + marg, H - 1);
          bw = bu1 - bu0 + 1;
          bh = bv1 - bv0 + 1;
          if (bw * bh > Cfg::kCap) {  // outlying centres: the largest allowed box around the mean centre
            bw = min(bw, Cfg::kBoxW);
            bh = min(bh, Cfg::kCap / bw);
            bu0 = min(max(su / cnt - bw / 2, bu0), bu1 - bw + 1);
            bv0 = min(max(sv / cnt - bh / 2, bv0), bv1 - bh + 1);
          }
        }
        s_box[0] = bu0; s_box[1] = bv0; s_box[2] = bw; s_box[3] = bh; s_box[4] = mode;
      }
      __syncthreads();
      const int mode = s_box[4];
      if (mode == 0) continue;  // no active query in the block: nothing to score
      const int bu0 = s_box[0], bv0 = s_box[1], bw = s_box[2], bh = s_box[3];
      bool ok = false;
      if (mode == 2) {
        if (wid == 0) {
          // the box's earlier contents were read through the generic proxy (before the
          // barriers above); order those reads before the copy engine's writes
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          if (lane == 0) mbar_arrive_tx(&s_bar, (uint32_t)(NQ * bw * bh * 16));
          __syncwarp();
          for (int r = lane; r < NQ * bh; r += 32) {
            const int c = r / bh, row = r - c * bh;
            bulk_g2s(s_desc + (c * bh + row) * bw, Dr4 + (int64_t)c * pv.P + o + (int64_t)(bv0 + row) * W + bu0,
                     (uint32_t)(bw * 16), &s_bar);
          }
        }
        if (act || tid == 0) {
          ok = mbar_wait_bounded(&s_bar, phase, pv.wait_polls);
          if (!ok) {
            s_dead = 1;
            if (tid == 0) pending = true;
          }
        }
        phase ^= 1u;
      }
      if (!act) continue;
      // this query's window inside the box: shared memory, else global memory
      const bool inside = ok && max(cu - marg, 0) >= bu0 && min(cu + marg, W - 1) < bu0 + bw &&
                          max(cv - marg, 0) >= bv0 && min(cv + marg, H - 1) < bv0 + bh;
      // one base pointer per chunk; candidate offsets within the edge image or the box fit in 32 bits
      const uint4* cb[NQ];
#pragma unroll
      for (int c = 0; c < NQ; ++c)
        cb[c] = inside ? static_cast<const uint4*>(s_desc) + c * bw * bh : Dr4 + (int64_t)c * pv.P + o;
      const int ox = inside ? bu0 : 0, oy = inside ? bv0 : 0, rs = inside ? bw : W;
      float best = -INFINITY;
      int bu = cu, bv = cv;
#pragma unroll 1
      for (int dy = -3; dy <= 3; ++dy) {
        const int vv = cv + dy * dil;
        const bool vin = (unsigned)vv < (unsigned)H;
        const int row = (min(max(vv, 0), H - 1) - oy) * rs - ox;
#pragma unroll
        for (int dx = -3; dx <= 3; ++dx) {
          const int uu = cu + dx * dil;
          const int off = row + min(max(uu, 0), W - 1);
          float s0 = 0.0f;
#pragma unroll
          for (int c = 0; c < NQ; ++c) {
            const uint4 w4 = cb[c][off];
            fma_h2(s0, dq[c].x, w4.x);
            fma_h2(s0, dq[c].y, w4.y);
            fma_h2(s0, dq[c].z, w4.z);
            fma_h2(s0, dq[c].w, w4.w);
          }
          const float s = (vin && (unsigned)uu < (unsigned)W) ? s0 : -INFINITY;
          if (s > best) {
            best = s;
            bu = uu;
            bv = vv;
          }
        }
      }
      cu = bu;
      cv = bv;
    }
    if (act) {
      const int m = cv * W + cu;
      const float3 y = ld3(Xr_e, m);
      const float dxv = y.x - x.x, dyv = y.y - x.y, dzv = y.z - x.z;
      const float dist = sqrtf(fmaf(dzv, dzv, fmaf(dyv, dyv, __fmul_rn(dxv, dxv))));
      const bool good = finite3(y) && dist <= mc.max_rel * sqrtf(nx2);
      out_idx[o + n] = good ? m : -1;
      stf(out_q + o + n, good ? sqrtf(ldf(Qr + o + m) * ldf(Qq + o + n)) : 0.0f);
      stats_epilogue(pv, st, o, m, good);
    }
  }
  // a copy whose wait gave up must land before the block's shared memory is released
  if (tid == 0 && pending) mbar_wait_bounded(&s_bar, phase ^ 1u, pv.wait_polls);
}

// ----------------------------------------------- tensor-core window form
// The refinement windows scored on the tensor cores (plan option
// match_form 1; FP16 storage, window radius 3).  After the LM iterations
// every query of a warp holds its window centre (cu, cv).  Per level, the
// warp's queries are grouped by (cv, cu mod dil, cu div 8 dil): the members
// of a group share their window rows, their centres lie on one dilation
// grid, and (cu - min cu) / dil <= 7, so the seven window columns of every
// member fall in one run of 16 candidates base + dil a, a = 0..15, base =
// min cu - 3 dil.  For up to 8 members and each window row the warp computes
// the 16 x 8 score tile S[a][n] = <D_ref[candidate a], D_qry[member n]> with
// mma.sync m16n8k16 (+ m16n8k8 for the third 8-channel chunk at d = 24):
// FP16 products, exact in FP32, summed in FP32.  Each lane then keeps, for
// its two members, the best score of the candidates that lie in that
// member's window (|a - o_n| <= 3 with o_n = (cu_n - base) / dil) and inside
// the image, and the lanes holding a member are combined by the largest
// score with ties to the smaller row-major window index: the first maximum
// in (dy, dx) order, as in the per-query form.  Every window row of a group
// is read once for its up to 8 members (one 4-byte piece per lane and
// chunk) instead of once per member, and the dot products leave the FP32
// pipe.
__device__ __forceinline__ void mma_16816(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                          uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_1688(float c[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5}, {%6}, {%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(b0));
}

// One level of the grouped window scan for the calling warp (all 32 lanes).
// valid: this lane's query takes part; (cu, cv) its centre, updated in
// place; pix its pool pixel.  D32 = descriptors as 32-bit words of the
// chunk-planar layout: word ((k P + p) 4 + e / 2) holds elements e, e + 1 of
// chunk k of pixel p.
template <int D>
__device__ __forceinline__ void tc_window_level(const uint32_t* __restrict__ Dr32, const uint32_t* __restrict__ Dq32,
                                                int64_t P, int64_t o, int W, int H, int dil, bool valid, int64_t pix,
                                                int& cu, int& cv) {
  constexpr int NC = D / 8;  // 8-element chunks
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int key = valid ? cv * 65536 + (cu % dil) * 1024 + cu / (8 * dil) : -1;
  unsigned pending = __ballot_sync(FULL, valid);
  int ncu = cu, ncv = cv;
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const int lkey = __shfl_sync(FULL, key, leader);
    unsigned take = __ballot_sync(FULL, ((pending >> lane) & 1u) && key == lkey);
    // the first 8 members (lowest lanes); the rest wait for a later group
    if (__popc(take) > 8) take &= (1u << (__fns(take, 0, 9))) - 1u;
    pending &= ~take;
    const int k = __popc(take);
    // B operand: member g's descriptor (element pairs 2t, 2t + 1 of each chunk)
    const int mb = __fns(take, 0, (g < k ? g : 0) + 1);
    const int64_t pb = __shfl_sync(FULL, pix, mb);
    uint32_t b[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) b[c] = __ldg(Dq32 + ((int64_t)c * P + pb) * 4 + t);
    const int gcv = __shfl_sync(FULL, cv, leader);
    const int base = __reduce_min_sync(FULL, ((take >> lane) & 1u) ? cu : 0x7fffffff) - 3 * dil;
    // this lane's score columns: members 2t and 2t + 1
    const bool has0 = 2 * t < k, has1 = 2 * t + 1 < k;
    const int m0 = __fns(take, 0, (has0 ? 2 * t : 0) + 1), m1 = __fns(take, 0, (has1 ? 2 * t + 1 : 0) + 1);
    const int cu0 = __shfl_sync(FULL, cu, m0), cu1 = __shfl_sync(FULL, cu, m1);
    const int o0 = (cu0 - base) / dil, o1 = (cu1 - base) / dil;
    // this lane's candidate rows a = g and g + 8
    const int colA = base + dil * g, colB = base + dil * (g + 8);
    const bool okA = (unsigned)colA < (unsigned)W, okB = (unsigned)colB < (unsigned)W;
    const int dA0 = g - o0, dB0 = g + 8 - o0, dA1 = g - o1, dB1 = g + 8 - o1;
    const bool inA0 = has0 && okA && dA0 >= -3 && dA0 <= 3, inB0 = has0 && okB && dB0 >= -3 && dB0 <= 3;
    const bool inA1 = has1 && okA && dA1 >= -3 && dA1 <= 3, inB1 = has1 && okB && dB1 >= -3 && dB1 <= 3;
    const int cA = min(max(colA, 0), W - 1), cB = min(max(colB, 0), W - 1);
    float best0 = -INFINITY, best1 = -INFINITY;
    int code0 = 0x7fffffff, code1 = 0x7fffffff;  // row-major window index (dy + 3) 7 + dx + 3
#pragma unroll 1
    for (int dy = -3; dy <= 3; ++dy) {
      const int vv = gcv + dy * dil;
      if ((unsigned)vv >= (unsigned)H) continue;  // the same for the whole group
      const int64_t rowp = o + (int64_t)vv * W;
      const uint32_t* pA = Dr32 + (rowp + cA) * 4 + t;
      const uint32_t* pB = Dr32 + (rowp + cB) * 4 + t;
      const int64_t cs = P * 4;  // words between chunks
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      mma_16816(c, __ldg(pA), __ldg(pB), __ldg(pA + cs), __ldg(pB + cs), b[0], b[1]);
      if (NC == 3) mma_1688(c, __ldg(pA + 2 * cs), __ldg(pB + 2 * cs), b[NC - 1]);
      if (NC == 4) mma_16816(c, __ldg(pA + 2 * cs), __ldg(pB + 2 * cs), __ldg(pA + 3 * cs), __ldg(pB + 3 * cs), b[2],
                             b[NC - 1]);
      // c0 = (a = g, member 2t), c1 = (g, 2t + 1), c2 = (g + 8, 2t), c3 = (g + 8, 2t + 1);
      // at most one of a = g, g + 8 lies in a member's 7-wide window
      const int row = (dy + 3) * 7 + 3;
      if (inA0 && c[0] > best0) { best0 = c[0]; code0 = row + dA0; }
      if (inB0 && c[2] > best0) { best0 = c[2]; code0 = row + dB0; }
      if (inA1 && c[1] > best1) { best1 = c[1]; code1 = row + dA1; }
      if (inB1 && c[3] > best1) { best1 = c[3]; code1 = row + dB1; }
    }
    // combine the 8 lanes (g = 0..7) of each member column
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) {
      const float ob0 = __shfl_xor_sync(FULL, best0, off), ob1 = __shfl_xor_sync(FULL, best1, off);
      const int oc0 = __shfl_xor_sync(FULL, code0, off), oc1 = __shfl_xor_sync(FULL, code1, off);
      if (ob0 > best0 || (ob0 == best0 && oc0 < code0)) { best0 = ob0; code0 = oc0; }
      if (ob1 > best1 || (ob1 == best1 && oc1 < code1)) { best1 = ob1; code1 = oc1; }
    }
    // member n (the n-th lane of the group) reads its result from lane n / 2
    const int n_me = __popc(take & ((1u << lane) - 1u));
    const int src = (n_me >> 1) & 3;
    const int r0 = __shfl_sync(FULL, code0, src), r1 = __shfl_sync(FULL, code1, src);
    if ((take >> lane) & 1u) {
      const int code = (n_me & 1) ? r1 : r0;
      ncu = cu + dil * (code % 7 - 3);
      ncv = cv + dil * (code / 7 - 3);
    }
  }
  cu = ncu;
  cv = ncv;
}

template <int D>
__device__ __forceinline__ void match_tc_query(const PlanView& pv, const MatchConst& mc, const DevEdge& ed,
                                               int u, int v, const MatchStats& st, const __half* __restrict__ Xr, const __half* __restrict__ Xq,
                                               const __half* __restrict__ Dr, const __half* __restrict__ Dq,
                                               const __half* __restrict__ Qr, const __half* __restrict__ Qq,
                                               const int32_t* __restrict__ init, int32_t* __restrict__ out_idx,
                                               __half* __restrict__ out_q, const float4* __restrict__ R4) {
  const int W = ed.W, H = ed.H;
  const bool inside = u < W && v < H;
  const int64_t HW = (int64_t)H * W;
  const int n = inside ? v * W + u : 0;
  const int64_t o = ed.off_e;
  const __half* Xr_e = Xr + 3 * o;
  const float3 x = ld3(Xq + 3 * o, n);
  const float nx2 = fmaf(x.x, x.x, fmaf(x.y, x.y, x.z * x.z));
  const bool valid = inside && finite3(x) && nx2 > 0.0f;
  int cu = 0, cv = 0;
  if (valid) {
    const float inx = rsqrtf(nx2);
    const float3 tg = make_float3(x.x * inx, x.y * inx, x.z * inx);
    int p0 = n;
    if (init) {
      const int32_t ii = init[o + n];
      if (ii >= 0 && ii < HW) p0 = ii;
    }
    float pu = (float)(p0 % W), pv_ = (float)(p0 / W);
    lm_iterate(Xr_e, R4 ? R4 + o : nullptr, W, H, tg, mc, pu, pv_);
    cu = min((int)floorf(pu + 0.5f), W - 1);
    cv = min((int)floorf(pv_ + 0.5f), H - 1);
  }
  const uint32_t* Dr32 = reinterpret_cast<const uint32_t*>(Dr);
  const uint32_t* Dq32 = reinterpret_cast<const uint32_t*>(Dq);
  for (int lev = 0; lev < mc.n_levels; ++lev)
    tc_window_level<D>(Dr32, Dq32, pv.P, o, W, H, mc.dil[lev], valid, o + n, cu, cv);
  if (!inside) return;
  if (!valid) {
    out_idx[o + n] = -1;
    stf(out_q + o + n, 0.0f);
    return;
  }
  const int m = cv * W + cu;
  const float3 y = ld3(Xr_e, m);
  const float dxv = y.x - x.x, dyv = y.y - x.y, dzv = y.z - x.z;
  const float dist = sqrtf(fmaf(dzv, dzv, fmaf(dyv, dyv, __fmul_rn(dxv, dxv))));
  const bool ok = finite3(y) && dist <= mc.max_rel * sqrtf(nx2);
  out_idx[o + n] = ok ? m : -1;
  stf(out_q + o + n, ok ? sqrtf(ldf(Qr + o + m) * ldf(Qq + o + n)) : 0.0f);
  stats_epilogue(pv, st, o, m, ok);
}

// The matching kernel with the tensor-core window (FP16 storage, radius 3):
// the per-query part (a1, a2, the rounding, the 3D test and q) is that of
// match_kernel; every lane of a warp reaches the window levels, which are
// warp-collective.
template <int D>
__global__ void __launch_bounds__(kMatchThreads) match_tc_kernel(
    PlanView pv, MatchConst mc, const __half* __restrict__ Xr, const __half* __restrict__ Xq,
    const __half* __restrict__ Dr, const __half* __restrict__ Dq, const __half* __restrict__ Qr,
    const __half* __restrict__ Qq, const int32_t* __restrict__ init, int32_t* __restrict__ out_idx,
    __half* __restrict__ out_q, int e_begin, int e_end, int block_base, const float4* __restrict__ R4,
    MatchStats st) {
  const int gb = block_base + blockIdx.x;
  const DevEdge ed = pv.edges[match_block_edge(pv, gb, e_begin, e_end)];
  const int local = gb - ed.mblock_begin;
  const int bx = pv.match_bx, by = pv.match_by, bh = by * pv.match_ppt;
  const int nbx = (ed.W + bx - 1) / bx;
  const int u = (local % nbx) * bx + (threadIdx.x % bx);
  const int v0 = (local / nbx) * bh + (threadIdx.x / bx);
  for (int k = 0; k < pv.match_ppt; ++k)  // the same count in every lane: the window levels stay warp-collective
    match_tc_query<D>(pv, mc, ed, u, v0 + k * by, st, Xr, Xq, Dr, Dq, Qr, Qq, init, out_idx, out_q, R4);
}

template <typename T, int D>
static void launch_match(const PlanView& pv, const MatchConst& mc, const void* Xr, const void* Xq, const void* Dr,
                         const void* Dq, const void* Qr, const void* Qq, const int32_t* init, int32_t* out_idx,
                         void* out_q, int e0, int e1, int b0, int nblocks, int form, float4* R4, MatchStats st,
                         cudaStream_t s) {
  st.e_begin = e0;
  st.e_end = e1;
  st.block_base = b0;
  if constexpr (std::is_same<T, __half>::value) {
    if (form == 1 && mc.radius == 3) {
      match_tc_kernel<D><<<nblocks, kMatchThreads, 0, s>>>(
          pv, mc, static_cast<const __half*>(Xr), static_cast<const __half*>(Xq), static_cast<const __half*>(Dr),
          static_cast<const __half*>(Dq), static_cast<const __half*>(Qr), static_cast<const __half*>(Qq), init, out_idx,
          static_cast<__half*>(out_q), e0, e1, b0, R4, st);
      return;
    }
    if (form == 2 && mc.radius == 3) {
      auto ks = pv.match_ppt == 2 ? match_staged_kernel<D, 2> : match_staged_kernel<D, 1>;
      cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, StagedCfg<D>::kSmem);
      ks<<<nblocks, kMatchThreads, StagedCfg<D>::kSmem, s>>>(
          pv, mc, static_cast<const __half*>(Xr), static_cast<const __half*>(Xq), static_cast<const __half*>(Dr),
          static_cast<const __half*>(Dq), static_cast<const __half*>(Qr), static_cast<const __half*>(Qq), init, out_idx,
          static_cast<__half*>(out_q), e0, e1, b0, R4, st);
      return;
    }
  }
  auto k = mc.radius == 3 ? (pv.match_ppt == 2 ? match_kernel<T, D, 3, 2> : match_kernel<T, D, 3, 1>)
                           : (pv.match_ppt == 2 ? match_kernel<T, D, 0, 2> : match_kernel<T, D, 0, 1>);
  k<<<nblocks, kMatchThreads, 0, s>>>(pv, mc, static_cast<const T*>(Xr), static_cast<const T*>(Xq),
                                     static_cast<const T*>(Dr), static_cast<const T*>(Dq),
                                     static_cast<const T*>(Qr), static_cast<const T*>(Qq), init, out_idx,
                                     static_cast<T*>(out_q), e0, e1, b0, R4, st);
}

}  // namespace mslam

using namespace mslam;

namespace mslam {
// Distinct reference pixels of edges [e0, e0 + gridDim.x): popcount of each
// edge's word-aligned bit range of the fused epilogue's bitmap.
__global__ void __launch_bounds__(256) stats_count_fused_kernel(PlanView pv, const uint32_t* __restrict__ bits,
                                                                int32_t* __restrict__ n_unique, int e0) {
  const int e = e0 + blockIdx.x;
  const DevEdge ed = pv.edges[e];
  const int64_t b0 = stats_bit_off(ed.off_e, e), n = (int64_t)ed.H * ed.W;
  const int64_t w0 = b0 >> 5, nw = (n + 31) >> 5;
  int cnt = 0;
  for (int64_t k = threadIdx.x; k < nw; k += blockDim.x) {
    uint32_t v = bits[w0 + k];
    if (k == nw - 1 && (n & 31)) v &= (1u << (n & 31)) - 1u;
    cnt += __popc(v);
  }
  __shared__ int sw[8];
  for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < 8; ++w) t += sw[w];
    n_unique[e] = t;
  }
}
}  // namespace mslam

extern "C" mslam_status mslam_match(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt, int32_t d,
                                    const void* X_ref, const void* X_qry, const void* D_ref, const void* D_qry,
                                    const void* Q_ref, const void* Q_qry, const int32_t* init_idx, int32_t* idx_out,
                                    void* q_out, int32_t* n_valid, int32_t* n_unique, int32_t edge_begin,
                                    int32_t edge_end, void* workspace, size_t ws_bytes, uint32_t flags,
                                    void* stream) {
  if (!p || !check_plan_uploaded(plan)) {
    if (!p) set_error("params is NULL");
    return MSLAM_ERR_ARG;
  }
  if (dt != MSLAM_F32 && dt != MSLAM_F16) {
    set_error("unsupported dtype %d", (int)dt);
    return MSLAM_ERR_ARG;
  }
  if (d != 16 && d != 24 && d != 32) {
    set_error("descriptor dimension %d not supported (16, 24 or 32)", d);
    return MSLAM_ERR_ARG;
  }
  if (plan_view(plan).E == 0) return MSLAM_OK;  // no edges: empty pools, nothing to match
  if (!X_ref || !X_qry || !D_ref || !D_qry || !Q_ref || !Q_qry || !idx_out || !q_out) {
    set_error("match: NULL device pointer");
    return MSLAM_ERR_ARG;
  }
  const size_t esz = dt == MSLAM_F32 ? 4 : 2;
  auto mis = [&](const void* ptr, size_t al) { return (reinterpret_cast<uintptr_t>(ptr) % al) != 0; };
  if (mis(D_ref, 16) || mis(D_qry, 16) || mis(X_ref, esz) || mis(X_qry, esz) || mis(Q_ref, esz) ||
      mis(Q_qry, esz) || mis(q_out, esz) || mis(idx_out, 4) || (init_idx && mis(init_idx, 4))) {
    set_error("match: misaligned pointer (descriptors need 16-byte alignment)");
    return MSLAM_ERR_ARG;
  }
  if (p->lm_iters < 0 || p->lm_iters > 1000 || p->win_radius < 0 || p->win_radius > 32 || p->n_levels < 0 ||
      p->n_levels > 4 || !(p->lm_lambda >= 0.0f) || !(p->max_rel_dist3d >= 0.0f)) {
    set_error("match: parameter out of range");
    return MSLAM_ERR_ARG;
  }
  for (int l = 0; l < p->n_levels; ++l)
    if (p->win_dilation[l] < 1 || p->win_dilation[l] > 64) {
      set_error("match: win_dilation[%d] = %d out of range", l, p->win_dilation[l]);
      return MSLAM_ERR_ARG;
    }
  const PlanView pv = plan_view(plan);
  int e0 = edge_begin, e1 = edge_end;
  if (e0 < 0 && e1 < 0) {
    e0 = 0;
    e1 = pv.E;
  }
  if (e0 < 0 || e1 > pv.E || e0 > e1) {
    set_error("match: edge range [%d, %d) outside [0, %d)", e0, e1, pv.E);
    return MSLAM_ERR_ARG;
  }
  if (e0 == e1) return MSLAM_OK;
  MatchConst mc;
  mc.lm_lambda = p->lm_lambda;
  mc.max_rel = p->max_rel_dist3d;
  mc.lm_iters = p->lm_iters;
  mc.radius = p->win_radius;
  mc.n_levels = p->n_levels;
  for (int l = 0; l < 4; ++l) mc.dil[l] = p->win_dilation[l];
  if (workspace && (ws_bytes < mslam_workspace_bytes(plan, MSLAM_OP_MATCH) ||
                    (reinterpret_cast<uintptr_t>(workspace) & 255))) {
    set_error("match: workspace smaller than %zu bytes or not 256-byte aligned",
              mslam_workspace_bytes(plan, MSLAM_OP_MATCH));
    return MSLAM_ERR_ARG;
  }
  if ((n_valid != nullptr) != (n_unique != nullptr) || (n_valid && !workspace)) {
    set_error("match: the keyframe counts need both n_valid and n_unique and the workspace");
    return MSLAM_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int form = plan_match_form(plan);
  float4* R4 = static_cast<float4*>(workspace);
  MatchStats stats{nullptr, nullptr, 0, 0, 0};
  if (n_valid) {
    // the bitmap follows the ray image; clear the words and counts of edges [e0, e1)
    const int64_t P_all = plan_edge_off(plan, pv.E);
    stats.bits = reinterpret_cast<uint32_t*>(static_cast<char*>(workspace) + ((sizeof(float4) * (size_t)P_all + 255) &
                                                                              ~size_t(255)));
    stats.n_valid = n_valid;
    const int64_t w0 = stats_bit_off(plan_edge_off(plan, e0), e0) >> 5;
    const int64_t w1 = stats_bit_off(plan_edge_off(plan, e1), e1) >> 5;
    mslam_status st = cuda_check(cudaMemsetAsync(stats.bits + w0, 0, sizeof(uint32_t) * (size_t)(w1 - w0), s),
                                 "match memset");
    if (st == MSLAM_OK)
      st = cuda_check(cudaMemsetAsync(n_valid + e0, 0, sizeof(int32_t) * (size_t)(e1 - e0), s), "match memset");
    if (st != MSLAM_OK) return st;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto go = [&](int a, int b) {
    int b0, b1x, bt0, bt1;
    plan_edge_mblocks(plan, a, &b0, &bt0);
    plan_edge_mblocks(plan, b - 1, &bt1, &b1x);
    (void)bt0;
    (void)bt1;
    const int nb = b1x - b0;
    if (R4) {
      // a1: the unit rays of the reference pointmaps of edges [a, b)
      const int64_t p0 = plan_edge_off(plan, a), p1 = plan_edge_off(plan, b);
      const int grid = (int)std::min<int64_t>((p1 - p0 + 255) / 256, (int64_t)std::max(1, sms) * 16);
      if (dt == MSLAM_F32)
        ray4_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float*>(X_ref), R4, p0, p1);
      else
        ray4_kernel<__half><<<grid, 256, 0, s>>>(static_cast<const __half*>(X_ref), R4, p0, p1);
    }
#define MSLAM_MATCH_CASE(TT, DD)                                                                              \
  launch_match<TT, DD>(pv, mc, X_ref, X_qry, D_ref, D_qry, Q_ref, Q_qry, init_idx, idx_out, q_out, a, b, b0, nb, \
                       form, R4, stats, s)
    if (dt == MSLAM_F32) {
      if (d == 16) MSLAM_MATCH_CASE(float, 16);
      else if (d == 24) MSLAM_MATCH_CASE(float, 24);
      else MSLAM_MATCH_CASE(float, 32);
    } else {
      if (d == 16) MSLAM_MATCH_CASE(__half, 16);
      else if (d == 24) MSLAM_MATCH_CASE(__half, 24);
      else MSLAM_MATCH_CASE(__half, 32);
    }
#undef MSLAM_MATCH_CASE
  };
  if (flags & MSLAM_FLAG_PER_EDGE) {
    for (int e = e0; e < e1; ++e) go(e, e + 1);
  } else {
    go(e0, e1);
  }
  if (n_valid) stats_count_fused_kernel<<<e1 - e0, 256, 0, s>>>(pv, stats.bits, n_unique, e0);
  return cuda_check(cudaGetLastError(), "match launch");
}

// ---------------------------------------------------------------- Sec. 3.4 counts
namespace mslam {

// Mark every valid match's reference pixel in a pool-wide bitmap (bit
// e_off[e] + m) and count valid matches per edge (integer atomics: exact).
__global__ void __launch_bounds__(256) stats_mark_kernel(PlanView pv, const int32_t* __restrict__ idx,
                                                         uint32_t* __restrict__ bits, int32_t* __restrict__ n_valid) {
  __shared__ int s_cnt;
  for (int tile = blockIdx.x; tile < pv.n_tiles; tile += gridDim.x) {
    const DevTile tl = pv.tiles[tile];
    const DevEdge ed = pv.edges[tl.edge];
    const int HW = ed.H * ed.W;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    int cnt = 0;
    for (int n = tl.begin + threadIdx.x; n < tl.end; n += blockDim.x) {
      const int m = __ldg(idx + ed.off_e + n);
      if (m < 0 || m >= HW) continue;
      ++cnt;
      const int64_t b = ed.off_e + m;
      atomicOr(bits + (b >> 5), 1u << (b & 31));
    }
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(n_valid + tl.edge, s_cnt);
    __syncthreads();
  }
}

// Distinct reference pixels per edge: popcount of the edge's bit range.
__global__ void __launch_bounds__(256) stats_count_kernel(PlanView pv, const uint32_t* __restrict__ bits,
                                                          int32_t* __restrict__ n_unique) {
  const int e = blockIdx.x;
  const DevEdge ed = pv.edges[e];
  const int64_t b0 = ed.off_e, b1 = ed.off_e + (int64_t)ed.H * ed.W;  // [b0, b1)
  const int64_t w0 = b0 >> 5, w1 = (b1 - 1) >> 5;
  int cnt = 0;
  for (int64_t wd = w0 + threadIdx.x; wd <= w1; wd += blockDim.x) {
    uint32_t v = bits[wd];
    if (wd == w0) v &= ~0u << (b0 & 31);
    if (wd == w1 && ((b1 & 31) != 0)) v &= (1u << (b1 & 31)) - 1u;
    cnt += __popc(v);
  }
  __shared__ int s[8];
  for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < 8; ++w) t += s[w];
    n_unique[e] = t;
  }
}

}  // namespace mslam

extern "C" mslam_status mslam_match_stats(const mslam_plan* plan, const int32_t* idx, int32_t* n_valid,
                                          int32_t* n_unique, void* workspace, size_t ws_bytes, void* stream) {
  if (!check_plan_uploaded(plan)) return MSLAM_ERR_ARG;
  const PlanView pv = plan_view(plan);
  if (pv.E == 0) return MSLAM_OK;
  if (!idx || !n_valid || !n_unique || !workspace) {
    set_error("match_stats: NULL device pointer");
    return MSLAM_ERR_ARG;
  }
  const size_t need = mslam_workspace_bytes(plan, MSLAM_OP_STATS);
  if (ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    set_error("match_stats: workspace smaller than %zu bytes or not 256-byte aligned", need);
    return MSLAM_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mslam_status st = cuda_check(cudaMemsetAsync(workspace, 0, need, s), "match_stats memset");
  if (st != MSLAM_OK) return st;
  st = cuda_check(cudaMemsetAsync(n_valid, 0, sizeof(int32_t) * pv.E, s), "match_stats memset");
  if (st != MSLAM_OK) return st;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  stats_mark_kernel<<<std::min(pv.n_tiles, std::max(1, sms) * 8), 256, 0, s>>>(pv, idx,
                                                                             static_cast<uint32_t*>(workspace), n_valid);
  stats_count_kernel<<<pv.E, 256, 0, s>>>(pv, static_cast<const uint32_t*>(workspace), n_unique);
  return cuda_check(cudaGetLastError(), "match_stats launch");
}

extern "C" mslam_status mslam_keyframe_criterion(int32_t E, const int32_t* n_valid, const int32_t* n_unique,
                                                 const int64_t* n_query, double omega_k, int32_t* needed) {
  if (E < 0 || (E > 0 && (!n_valid || !n_unique || !n_query || !needed)) || !(omega_k >= 0.0 && omega_k <= 1.0)) {
    set_error("keyframe_criterion: E = %d, omega_k = %g (in [0, 1]) or a NULL host array", E, omega_k);
    return MSLAM_ERR_ARG;
  }
  for (int32_t e = 0; e < E; ++e) {
    const int64_t nq = n_query[e];
    if (nq <= 0) {
      needed[e] = 1;
      continue;
    }
    const double fv = (double)n_valid[e] / (double)nq, fu = (double)n_unique[e] / (double)nq;
    needed[e] = (fv < omega_k || fu < omega_k) ? 1 : 0;
  }
  return MSLAM_OK;
}

namespace mslam {
// One thread per (pixel, chunk): a 16-byte piece moves from [p][k] to [k][p];
// consecutive threads take consecutive pixels of one chunk, so the stores are
// coalesced and the loads read each pixel's descriptor once overall.
__global__ void __launch_bounds__(256) desc_chunk_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                         int64_t n_pix, int nc, int64_t stride) {
  const int64_t total = n_pix * nc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / n_pix, p = i - k * n_pix;
    dst[k * stride + p] = __ldg(src + p * nc + k);
  }
}
}  // namespace mslam

extern "C" mslam_status mslam_desc_to_chunked(mslam_dtype dt, int32_t d, int64_t n_pix, const void* src, void* dst,
                                              int64_t dst_pix_stride, void* stream) {
  if ((dt != MSLAM_F32 && dt != MSLAM_F16) || (d != 16 && d != 24 && d != 32) || n_pix < 0 ||
      dst_pix_stride < n_pix) {
    set_error("desc_to_chunked: dtype %d, d %d (16, 24 or 32), n_pix %lld, stride %lld", (int)dt, d,
              (long long)n_pix, (long long)dst_pix_stride);
    return MSLAM_ERR_ARG;
  }
  if (n_pix == 0) return MSLAM_OK;
  if (!src || !dst || (reinterpret_cast<uintptr_t>(src) & 15) || (reinterpret_cast<uintptr_t>(dst) & 15)) {
    set_error("desc_to_chunked: NULL or not 16-byte aligned buffer");
    return MSLAM_ERR_ARG;
  }
  const int nc = d * (dt == MSLAM_F32 ? 4 : 2) / 16;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n_pix * nc + 255) / 256;
  const int grid = (int)std::min<int64_t>(want, (int64_t)std::max(1, sms) * 16);
  desc_chunk_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const uint4*>(src),
                                                                         static_cast<uint4*>(dst), n_pix, nc,
                                                                         dst_pix_stride);
  return cuda_check(cudaGetLastError(), "desc_to_chunked launch");
}
