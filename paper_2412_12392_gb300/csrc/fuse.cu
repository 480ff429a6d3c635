// Per-pixel pointmap updates: fusion (Sec. 3.3) and the calibrated
// back-projection of Sec. 3.6.
//
// Pointmap fusion of Sec. 3.3 (a NEXT-stage kernel after tracking): the
// keyframe's canonical pointmap and confidence are updated per pixel by the
// running weighted average
//   X~ <- (C~ X~ + C (T_kf X)) / (C~ + C),   C~ <- C~ + C,
// with X the keyframe's points predicted together with the current frame (in
// the frame's coordinates) and T_kf = T_k^-1 T_f read from the device pose
// array, so the kernel can follow the tracking Gauss-Newton without a host
// round trip.  A prediction with a non-finite or zero point or a confidence
// that is not positive leaves its pixel unchanged.  HBM-bound: per pixel it
// reads X~, C~, X, C and writes X~, C~ (24 bytes in FP16, 48 in FP32).
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace mslam {

template <typename T>
__global__ void __launch_bounds__(256) fuse_kernel(const double* __restrict__ T_wc, int k, int f, int64_t n,
                                                   T* __restrict__ Xc, T* __restrict__ Cc, const T* __restrict__ Xkf,
                                                   const T* __restrict__ Ckf) {
  __shared__ float sR[9], st[3];
  if (threadIdx.x == 0) {
    const Sim3d Tk = load_pose(T_wc + 8 * k), Tf = load_pose(T_wc + 8 * f);
    const Sim3d Tkf = compose(inverse(Tk), Tf);
    double R[9];
    rot_of(Tkf.q, R);
    for (int a = 0; a < 9; ++a) sR[a] = (float)(Tkf.s * R[a]);
    for (int a = 0; a < 3; ++a) st[a] = (float)Tkf.t[a];
  }
  __syncthreads();
  float R[9], t[3];
#pragma unroll
  for (int a = 0; a < 9; ++a) R[a] = sR[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) t[a] = st[a];
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const float3 x = ld3(Xkf, p);
    const float c = ldf(Ckf + p);
    const float n2 = x.x * x.x + x.y * x.y + x.z * x.z;
    if (!(finite3(x) && n2 > 0.0f && c > 0.0f && c < INFINITY)) continue;
    const float y0 = fmaf(R[0], x.x, fmaf(R[1], x.y, fmaf(R[2], x.z, t[0])));
    const float y1 = fmaf(R[3], x.x, fmaf(R[4], x.y, fmaf(R[5], x.z, t[1])));
    const float y2 = fmaf(R[6], x.x, fmaf(R[7], x.y, fmaf(R[8], x.z, t[2])));
    const float cc = ldf(Cc + p);
    const float inv = 1.0f / (cc + c);
    const float3 xc = ld3(Xc, p);
    T* out = Xc + 3 * p;
    stf(out, (cc * xc.x + c * y0) * inv);
    stf(out + 1, (cc * xc.y + c * y1) * inv);
    stf(out + 2, (cc * xc.z + c * y2) * inv);
    stf(Cc + p, cc + c);
  }
}

// Known calibration (Sec. 3.6): only the depth of each predicted point is
// kept and the point is rebuilt on its pixel's pinhole ray,
// X[p] = z ((u - cx) / fx, (v - cy) / fy, 1), (u, v) = (p mod W, p div W).
template <typename T>
__global__ void __launch_bounds__(256) calib_backproject_kernel(int64_t n, int32_t H, int32_t W, float fx, float fy,
                                                                float cx, float cy, T* __restrict__ X) {
  const int64_t HW = (int64_t)H * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i % HW;
    const float u = (float)(p % W), v = (float)(p / W);
    const float z = ldf(X + 3 * i + 2);
    stf(X + 3 * i, z * (u - cx) / fx);
    stf(X + 3 * i + 1, z * (v - cy) / fy);
  }
}

// (a1) psi(X) = X / |X| per point, the zero ray for a zero or non-finite
// point (the same FP32 arithmetic as the match kernel's taps).
template <typename T>
__global__ void __launch_bounds__(256) ray_image_kernel(int64_t n, const T* X, T* R) {  // R may alias X
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float x = ldf(X + 3 * i), y = ldf(X + 3 * i + 1), z = ldf(X + 3 * i + 2);
    const float n2 = fmaf(x, x, fmaf(y, y, z * z));
    const bool ok = n2 > 0.0f && n2 < INFINITY;
    const float inv = ok ? rsqrtf(n2) : 0.0f;
    stf(R + 3 * i, ok ? x * inv : 0.0f);
    stf(R + 3 * i + 1, ok ? y * inv : 0.0f);
    stf(R + 3 * i + 2, ok ? z * inv : 0.0f);
  }
}

}  // namespace mslam

using namespace mslam;

extern "C" mslam_status mslam_ray_image(mslam_dtype dt, int64_t n_pix, const void* X, void* R, void* stream) {
  if (dt != MSLAM_F32 && dt != MSLAM_F16) {
    set_error("unsupported dtype %d", (int)dt);
    return MSLAM_ERR_ARG;
  }
  if (n_pix < 0) {
    set_error("ray_image: negative size %lld", (long long)n_pix);
    return MSLAM_ERR_ARG;
  }
  if (n_pix == 0) return MSLAM_OK;
  if (!X || !R) {
    set_error("ray_image: NULL device pointer");
    return MSLAM_ERR_ARG;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = std::min<int64_t>((n_pix + 255) / 256, (int64_t)std::max(1, sms) * 8);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dt == MSLAM_F32)
    ray_image_kernel<float><<<(int)blocks, 256, 0, s>>>(n_pix, static_cast<const float*>(X), static_cast<float*>(R));
  else
    ray_image_kernel<__half><<<(int)blocks, 256, 0, s>>>(n_pix, static_cast<const __half*>(X),
                                                         static_cast<__half*>(R));
  return cuda_check(cudaGetLastError(), "ray_image launch");
}

extern "C" mslam_status mslam_calib_backproject(mslam_dtype dt, int32_t n_images, int32_t H, int32_t W, float fx,
                                                float fy, float cx, float cy, void* X, void* stream) {
  if (dt != MSLAM_F32 && dt != MSLAM_F16) {
    set_error("unsupported dtype %d", (int)dt);
    return MSLAM_ERR_ARG;
  }
  if (n_images < 0 || H < 0 || W < 0 || !(fx > 0.0f) || !(fy > 0.0f) || !std::isfinite(fx) || !std::isfinite(fy) ||
      !std::isfinite(cx) || !std::isfinite(cy)) {
    set_error("calib_backproject: bad arguments (n_images %d, H %d, W %d, fx %g, fy %g)", n_images, H, W, fx, fy);
    return MSLAM_ERR_ARG;
  }
  const int64_t n = (int64_t)n_images * H * W;
  if (n == 0) return MSLAM_OK;
  if (!X) {
    set_error("calib_backproject: NULL device pointer");
    return MSLAM_ERR_ARG;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)std::max(1, sms) * 8);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dt == MSLAM_F32)
    calib_backproject_kernel<float><<<(int)blocks, 256, 0, s>>>(n, H, W, fx, fy, cx, cy, static_cast<float*>(X));
  else
    calib_backproject_kernel<__half><<<(int)blocks, 256, 0, s>>>(n, H, W, fx, fy, cx, cy, static_cast<__half*>(X));
  return cuda_check(cudaGetLastError(), "calib_backproject launch");
}

extern "C" mslam_status mslam_fuse(mslam_dtype dt, const double* T_wc, int32_t k, int32_t f, int64_t n_pix,
                                   void* X_canon_k, void* C_canon_k, const void* X_kf, const void* C_kf,
                                   void* stream) {
  if (dt != MSLAM_F32 && dt != MSLAM_F16) {
    set_error("unsupported dtype %d", (int)dt);
    return MSLAM_ERR_ARG;
  }
  if (n_pix < 0 || k < 0 || f < 0 || k == f) {
    set_error("fuse: bad arguments (n_pix %lld, k %d, f %d)", (long long)n_pix, k, f);
    return MSLAM_ERR_ARG;
  }
  if (n_pix == 0) return MSLAM_OK;
  if (!T_wc || !X_canon_k || !C_canon_k || !X_kf || !C_kf) {
    set_error("fuse: NULL device pointer");
    return MSLAM_ERR_ARG;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = std::min<int64_t>((n_pix + 255) / 256, (int64_t)std::max(1, sms) * 8);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dt == MSLAM_F32)
    fuse_kernel<float><<<(int)blocks, 256, 0, s>>>(T_wc, k, f, n_pix, static_cast<float*>(X_canon_k),
                                                   static_cast<float*>(C_canon_k), static_cast<const float*>(X_kf),
                                                   static_cast<const float*>(C_kf));
  else
    fuse_kernel<__half><<<(int)blocks, 256, 0, s>>>(T_wc, k, f, n_pix, static_cast<__half*>(X_canon_k),
                                                    static_cast<__half*>(C_canon_k), static_cast<const __half*>(X_kf),
                                                    static_cast<const __half*>(C_kf));
  return cuda_check(cudaGetLastError(), "fuse launch");
}
