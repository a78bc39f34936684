// Projective SDF integration (Section 4.2, Eq. 8-10) on a dense voxel grid.
//
// One thread per voxel: the voxel centre x is transformed into each scan's
// sensor frame (x_s = R_j x + t_j), projected by Pi (the same FP32 projection
// as the registration, rimg_device.cuh: Eq. 3-4 with the exact row argmin and
// the column recovery), and the scan's range at that pixel gives the signed
// distance along the ray d_j = Omega_j(u, v) - r (Eq. 9).  The thread sums
// the observations of all scans of the launch and merges them into the
// voxel's running least-squares mean (Eq. 10) with one division: the state
// is read and written once per launch, whatever the number of scans.
// Scan poses are staged into shared memory in tiles of kScanTile.
#include <stdint.h>

#include "rimg_device.cuh"
#include "rimg_internal.h"

namespace rimg {

namespace {

constexpr int kSdfThreads = 256;
constexpr int kScanTile = 32;

// FAST: the level's inverse table is exact, it has no azimuth offsets and its
// width is a power of two, so the projection takes its branch-free form (the
// field-of-view and range tests stay branches: they skip a scan's work).
template <bool R0, bool FAST>
__global__ void __launch_bounds__(kSdfThreads) k_sdf(DevLevel L, int n_scans, const float* __restrict__ ranges,
                                                    const double* __restrict__ poses, int nx, int ny, long long n_vox,
                                                    float ox, float oy, float oz, float voxel, float trunc,
                                                    int proj_iters, float* __restrict__ sdf,
                                                    float* __restrict__ weight) {
  __shared__ float4 P[kScanTile][3];   // rows of (R | t) in FP32
  const long long idx = (long long)blockIdx.x * kSdfThreads + threadIdx.x;
  const bool live = idx < n_vox;
  const long long plane = (long long)nx * ny;
  const int k = (int)(idx / plane);
  const long long rem = idx - (long long)k * plane;
  const int j = (int)(rem / nx), i = (int)(rem - (long long)j * nx);
  const float cx = fmaf(voxel, (float)i + 0.5f, ox);
  const float cy = fmaf(voxel, (float)j + 0.5f, oy);
  const float cz = fmaf(voxel, (float)k + 0.5f, oz);
  const long long img = (long long)L.H * L.W;
  float sum = 0.f, cnt = 0.f;
  for (int j0 = 0; j0 < n_scans; j0 += kScanTile) {
    const int nt = min(kScanTile, n_scans - j0);
    __syncthreads();
    for (int t = threadIdx.x; t < nt * 12; t += kSdfThreads)
      reinterpret_cast<float*>(&P[t / 12][0])[t % 12] = (float)poses[(long long)(j0 + t / 12) * 16 + t % 12];
    __syncthreads();
    if (!live) continue;
    for (int q = 0; q < nt; ++q) {
      const float4 a = P[q][0], b = P[q][1], c = P[q][2];
      const float3 xs = make_float3(fmaf(a.x, cx, fmaf(a.y, cy, fmaf(a.z, cz, a.w))),
                                    fmaf(b.x, cx, fmaf(b.y, cy, fmaf(b.z, cz, b.w))),
                                    fmaf(c.x, cx, fmaf(c.y, cy, fmaf(c.z, cz, c.w))));
      int u, v;
      float r;
      if (!project_px<R0, FAST>(L, xs, proj_iters, u, v, r)) continue;
      const float meas = __ldg(ranges + (long long)(j0 + q) * img + (long long)v * L.W + u);
      if (!range_ok(meas)) continue;
      float d = meas - r;
      if (trunc > 0.f) {
        if (d < -trunc) continue;   // hidden behind the measured surface
        d = fminf(d, trunc);
      }
      sum += d;
      cnt += 1.f;
    }
  }
  if (live && cnt > 0.f) {
    const float w0 = weight[idx];
    const float w1 = w0 + cnt;
    sdf[idx] = (fmaf(sdf[idx], w0, sum)) / w1;
    weight[idx] = w1;
  }
}

}  // namespace

cudaError_t launch_sdf(const DevLevel& L, int n_scans, const float* ranges, const double* poses, int nx, int ny,
                       int nz, float ox, float oy, float oz, float voxel, float trunc, int proj_iters, float* sdf,
                       float* weight, cudaStream_t st) {
  const long long n_vox = (long long)nx * ny * nz;
  if (n_vox == 0 || n_scans == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n_vox + kSdfThreads - 1) / kSdfThreads);
  const bool fast = L.bins_exact && !L.has_theta && L.W > 0 && (L.W & (L.W - 1)) == 0;
#define RIMG_SDF(R, F)                                                                                          \
  k_sdf<R, F><<<blocks, kSdfThreads, 0, st>>>(L, n_scans, ranges, poses, nx, ny, n_vox, ox, oy, oz, voxel, trunc, \
                                              proj_iters, sdf, weight)
  if (L.r0 != 0.f) {
    if (fast) RIMG_SDF(true, true); else RIMG_SDF(true, false);
  } else {
    if (fast) RIMG_SDF(false, true); else RIMG_SDF(false, false);
  }
#undef RIMG_SDF
  return cudaGetLastError();
}

}  // namespace rimg
