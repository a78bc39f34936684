// Point clouds without scan structure (Section 3.2, last paragraph): each
// point is projected by Pi (optionally after a rigid transform into the
// sensor frame) and the pixel keeps the smallest range.  Non-negative floats
// order like their bit patterns, so an integer atomicMin on the bits is an
// exact, order-independent minimum; the image starts at +inf (an invalid
// range under the library's rule) so untouched pixels stay invalid.
#include "rimg_device.cuh"
#include "rimg_internal.h"

namespace rimg {
namespace {

__global__ void k_fill_inf(float* __restrict__ img, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) img[i] = INFINITY;
}

template <bool R0>
__global__ void __launch_bounds__(256) k_points(DevLevel L, int max_points, const float* __restrict__ xyz,
                                               const int* __restrict__ counts, const double* __restrict__ T,
                                               int proj_iters, float* __restrict__ img) {
  __shared__ float P[12];
  const int c = blockIdx.y;
  if (threadIdx.x < 12)
    P[threadIdx.x] = T ? (float)T[(long long)c * 16 + threadIdx.x]
                       : ((threadIdx.x % 5 == 0) ? 1.f : 0.f);   // identity rows (R | t)
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = counts ? counts[c] : max_points;
  if (p >= min(n, max_points)) return;
  const float* q = xyz + ((long long)c * max_points + p) * 3;
  const float x = q[0], y = q[1], z = q[2];
  if (!(isfinite(x) && isfinite(y) && isfinite(z))) return;
  const float3 xs = make_float3(fmaf(P[0], x, fmaf(P[1], y, fmaf(P[2], z, P[3]))),
                                fmaf(P[4], x, fmaf(P[5], y, fmaf(P[6], z, P[7]))),
                                fmaf(P[8], x, fmaf(P[9], y, fmaf(P[10], z, P[11]))));
  int u, v;
  float r;
  if (!project_px<R0>(L, xs, proj_iters, u, v, r)) return;
  if (!(r > 0.f) || !isfinite(r)) return;
  int* dst = reinterpret_cast<int*>(img + ((long long)c * L.H + v) * L.W + u);
  atomicMin(dst, __float_as_int(r));
}

}  // namespace

cudaError_t launch_points(const DevLevel& L, int n_clouds, int max_points, const float* xyz, const int* counts,
                          const double* T, int proj_iters, float* img, cudaStream_t st) {
  const long long n_img = (long long)n_clouds * L.H * L.W;
  k_fill_inf<<<(unsigned)((n_img + 255) / 256), 256, 0, st>>>(img, n_img);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || max_points == 0) return e;
  dim3 grid((max_points + 255) / 256, n_clouds);
  if (L.r0 != 0.f)
    k_points<true><<<grid, 256, 0, st>>>(L, max_points, xyz, counts, T, proj_iters, img);
  else
    k_points<false><<<grid, 256, 0, st>>>(L, max_points, xyz, counts, T, proj_iters, img);
  return cudaGetLastError();
}

}  // namespace rimg
