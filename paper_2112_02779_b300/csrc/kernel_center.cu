// Initial pose of the registration problem (Section 4.1): the rotation starts
// at the identity and the translation aligns the centres of the two point
// sets, t = mean(target points) - mean(source points), both sets being the
// valid pixels of a range image unprojected by Eq. 1-2.
//
// One 512-thread block per pair walks the source image, then the target
// image, four pixels (one float4 of ranges) at a time: the chunk's points are
// unprojected in FP32 from the separable tables and summed in FP32, and each
// chunk sum is added to FP64 running sums (so FP32 rounding stays within a
// chunk).  The block reduces the FP64 sums and integer counts by warp
// shuffles and shared memory; its first thread writes the pose.
#include "rimg_device.cuh"

namespace rimg {

namespace {

constexpr int kCenterThreads = 512;

// This thread's FP64 sums of the valid points of one level-l image and their
// count, over the four-pixel chunks tid, tid + 512, ...  (W_l is a multiple
// of four, so a chunk never crosses a row; the image is 16-byte aligned).
__device__ __forceinline__ void center_sums(const DevLevel& L, const float* __restrict__ img, double& sx, double& sy,
                                            double& sz, int& cnt) {
  const int cpr = L.W >> 2;
  const int nchunks = L.H * cpr;
  for (int c = threadIdx.x; c < nchunks; c += kCenterThreads) {
    const int v = c / cpr, u0 = (c - v * cpr) << 2;
    const float4 r4 = __ldg(reinterpret_cast<const float4*>(img) + c);
    const float rr[4] = {r4.x, r4.y, r4.z, r4.w};
    float fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!range_ok(rr[q])) continue;
      const float3 p = unproject_px(L, u0 + q, v, rr[q]);
      fx += p.x;
      fy += p.y;
      fz += p.z;
      ++cnt;
    }
    sx += (double)fx;
    sy += (double)fy;
    sz += (double)fz;
  }
}

// Block-wide sum of (x, y, z, count); the result is valid in thread 0.
__device__ __forceinline__ void block_sum4(double& x, double& y, double& z, int& n, double (*sh)[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
    z += __shfl_xor_sync(0xffffffffu, z, o);
    n += __shfl_xor_sync(0xffffffffu, n, o);
  }
  if (lane == 0) {
    sh[warp][0] = x;
    sh[warp][1] = y;
    sh[warp][2] = z;
    sh[warp][3] = (double)n;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    x = y = z = 0.0;
    double c = 0.0;
    for (int w = 0; w < kCenterThreads / 32; ++w) {
      x += sh[w][0];
      y += sh[w][1];
      z += sh[w][2];
      c += sh[w][3];
    }
    n = (int)c;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kCenterThreads) k_center(DevLevel S, DevLevel D, const float* __restrict__ src,
                                                           const float* __restrict__ dst, double* __restrict__ T_out,
                                                           int* __restrict__ status) {
  __shared__ double sh[kCenterThreads / 32][4];
  const int pair = blockIdx.x;
  double c[2][3];
  int cnt[2];
#pragma unroll
  for (int img = 0; img < 2; ++img) {
    const DevLevel& L = img ? D : S;
    const float* base = (img ? dst : src) + (long long)pair * L.H * L.W;
    double x = 0.0, y = 0.0, z = 0.0;
    int n = 0;
    center_sums(L, base, x, y, z, n);
    block_sum4(x, y, z, n, sh);
    c[img][0] = x;
    c[img][1] = y;
    c[img][2] = z;
    cnt[img] = n;
  }
  if (threadIdx.x == 0) {
    const bool ok = cnt[0] > 0 && cnt[1] > 0;
    double* T = T_out + (long long)pair * 16;
    for (int k = 0; k < 16; ++k) T[k] = (k % 5 == 0) ? 1.0 : 0.0;
    if (ok) {
      const double is = 1.0 / (double)cnt[0], id = 1.0 / (double)cnt[1];
      T[3] = c[1][0] * id - c[0][0] * is;
      T[7] = c[1][1] * id - c[0][1] * is;
      T[11] = c[1][2] * id - c[0][2] * is;
    } else if (status) {
      status[pair] |= RIMG_FLAG_DEGENERATE;
    }
  }
}

}  // namespace

cudaError_t launch_center(const DevLevel& S, const DevLevel& D, int n_pairs, const float* src, const float* dst,
                          double* T_out, int* status, cudaStream_t st) {
  if (n_pairs == 0) return cudaSuccess;
  k_center<<<n_pairs, kCenterThreads, 0, st>>>(S, D, src, dst, T_out, status);
  return cudaGetLastError();
}

}  // namespace rimg
