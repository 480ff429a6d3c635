// mslam_gn_linearize_noalloc: the linearisation of mslam_gn_linearize with its
// scratch space in a fixed array owned by this library instead of a
// caller-provided workspace, for callers that cannot allocate device memory.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes, so
// every GPU that loads the library holds it until the process exits.  The
// entry point forwards to mslam_gn_linearize with that array as the
// workspace; it allocates nothing itself.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;  // 4 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_lin_scratch[kNoAllocScratchBytes];

// cuCtxGetCurrent, looked up once through the runtime (the library does not
// link the driver library directly).
typedef int (*CtxGetCurrentFn)(void**);

std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
void* g_scratch_ctx[kMaxDevices] = {};
CtxGetCurrentFn g_ctx_get = nullptr;
bool g_ctx_get_tried = false;

// Device address of the scratch array in the current device's current
// context.  The host-side name of the array is only a stand-in and must never
// be handed to a kernel.  The address is looked up (cudaGetSymbolAddress, with
// the device current) the first time a context of a device calls, and looked
// up again when the device's context has changed since (e.g. after
// cudaDeviceReset), so a destroyed context's address is never reused.
mslam_status scratch_address(void** out) {
  int dev = 0;
  mslam_status st = mslam::cuda_check(cudaGetDevice(&dev), "gn_linearize_noalloc: cudaGetDevice");
  if (st != MSLAM_OK) return st;
  if (dev < 0 || dev >= kMaxDevices) {
    mslam::set_error("gn_linearize_noalloc: device %d beyond the %d supported", dev, kMaxDevices);
    return MSLAM_ERR_RANGE;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_ctx_get_tried) {
    g_ctx_get_tried = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get = reinterpret_cast<CtxGetCurrentFn>(fn);
    else
      cudaGetLastError();  // clear: without the lookup every call resolves the address
  }
  // the current context (none yet if the runtime has not used this device)
  void* ctx = nullptr;
  const bool have_ctx = g_ctx_get && g_ctx_get(&ctx) == 0 && ctx;
  if (!g_scratch_ptr[dev] || !have_ctx || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;
    st = mslam::cuda_check(cudaGetSymbolAddress(&p, g_lin_scratch), "gn_linearize_noalloc: cudaGetSymbolAddress");
    if (st != MSLAM_OK) return st;
    // the lookup made the device's primary context current if it was not
    void* ctx_now = nullptr;
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = (g_ctx_get && g_ctx_get(&ctx_now) == 0) ? ctx_now : nullptr;
  }
  *out = g_scratch_ptr[dev];
  return MSLAM_OK;
}

}  // namespace

extern "C" mslam_status mslam_gn_linearize_noalloc(const mslam_params* p, const mslam_plan* plan, mslam_dtype dt,
                                                   const double* T_wc, const void* X_canon, const int32_t* idx,
                                                   const void* q, float* H_blocks, float* g_blocks, double* cost,
                                                   int32_t* n_valid, uint32_t flags, void* stream) {
  if (!plan) {
    mslam::set_error("gn_linearize_noalloc: plan is NULL");
    return MSLAM_ERR_ARG;
  }
  const size_t need = mslam_workspace_bytes(plan, MSLAM_OP_LINEARIZE);
  if (need > kNoAllocScratchBytes) {
    mslam::set_error(
        "gn_linearize_noalloc: this plan needs %zu bytes of scratch; the built-in scratch holds %zu bytes "
        "(about %zu linearisation tiles); use mslam_gn_linearize with a workspace",
        need, kNoAllocScratchBytes, kNoAllocScratchBytes / (sizeof(float) * mslam::kAccStride));
    return MSLAM_ERR_RANGE;
  }
  void* scratch = nullptr;
  const mslam_status st = scratch_address(&scratch);
  if (st != MSLAM_OK) return st;
  // Every partial sum and relative pose the linearisation reads is written
  // earlier in the same call, so the scratch needs no clearing between calls.
  return mslam_gn_linearize(p, plan, dt, T_wc, X_canon, idx, q, H_blocks, g_blocks, cost, n_valid, scratch,
                            kNoAllocScratchBytes, flags, stream);
}
