// rimg_icp_step_static: the association / Gauss-Newton step for callers that
// cannot allocate device memory.
//
// Some hosts of this library cannot call cudaMalloc at the point where they
// register scans: an embedded perception loop that forbids allocation after
// start-up, a plug-in running inside another framework's memory pool that
// hands it only the tensors it owns, or a real-time thread where an
// allocation could block on the driver.  rimg_icp_step needs a caller
// workspace for its per-block partial sums and per-pair completion counters;
// this entry point keeps that scratch in a fixed array inside the library
// instead, so the caller passes only inputs and outputs.
#include <mutex>

#include "rimg_internal.h"

namespace {

// The scratch every call of rimg_icp_step_static shares.  Each GPU that loads
// the library holds one copy until the process exits.
static __device__ __align__(256) unsigned char g_icp_scratch[RIMG_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_icp_scratch on the current device.  In host code the
// symbol name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached for the life of the
// process; a cudaDeviceReset would leave the cached address stale.
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return RIMG_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return RIMG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_icp_scratch);
    if (e != cudaSuccess || !p) return RIMG_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return RIMG_OK;
}

}  // namespace

extern "C" int rimg_icp_step_static(const rimg_sensor* src, const rimg_sensor* dst, int level, int n_pairs,
                                    const float* src_range_l, const float* dst_planes_l,
                                    const float* dst_range_l, double* pose, const rimg_params* p, int update,
                                    double* out29, int32_t* assoc, int* status, void* stream) {
  if (!src) return RIMG_ERR_INVALID_ARG;
  size_t need = 0;
  int rc = rimg_icp_workspace_bytes(src, n_pairs, &need);
  if (rc) return rc;
  if (need > (size_t)RIMG_STATIC_SCRATCH_BYTES) return RIMG_ERR_WORKSPACE;   // batch too large
  void* scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc) return rc;
  // rimg_icp_step zeroes the completion counters (the first bytes of the
  // scratch) on `stream` before its kernel, so leftovers of an earlier call
  // do not matter; the partial sums are fully rewritten by every call.
  return rimg_icp_step(src, dst, level, n_pairs, src_range_l, dst_planes_l, dst_range_l, pose, p, update,
                       out29, assoc, status, scratch, (size_t)RIMG_STATIC_SCRATCH_BYTES, stream);
}
