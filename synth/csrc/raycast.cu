// GPU ray caster for the synthetic scans (input generation only; holds none
// of the registration method's arithmetic).  It casts the same rays as
// synth.scenes.raycast -- one ray per pixel from a receiver on a cylinder of
// radius r0, azimuth 2 pi u / W + theta[v], elevation phi[v] -- against a
// ground plane z = 0 and vertical boxes and cylinders standing on it, in
// float32, so that large training sets of scan pairs can be generated on the
// device.  Range noise and pixel dropout come from a counter-based hash of
// (pair seed, scan of the pair, pixel) with a Box-Muller transform.
//
// Object records (8 floats): box      (0, cx, cy, cos yaw, sin yaw, hx, hy, h)
//                            cylinder (1, cx, cy, radius, h, 0, 0, 0)
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kThreads = 256;
constexpr int kPix = 4;          // pixels per thread
constexpr int kMaxObj = 512;

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// uniform in (0, 1]
__device__ __forceinline__ float unit(uint64_t h) { return ((float)(h >> 40) + 1.0f) * (1.0f / 16777216.0f); }

__device__ __forceinline__ float hit_box(const float* b, float ox, float oy, float oz, float dx, float dy, float dz) {
  const float c = b[3], s = b[4];
  const float px = ox - b[1], py = oy - b[2];
  const float lo[3] = {c * px + s * py, -s * px + c * py, oz};
  const float ld[3] = {c * dx + s * dy, -s * dx + c * dy, dz};
  const float lb[3] = {-b[5], -b[6], 0.f}, hb[3] = {b[5], b[6], b[7]};
  float tmin = -INFINITY, tmax = INFINITY;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float inv = 1.0f / ld[a];
    const float t1 = (lb[a] - lo[a]) * inv, t2 = (hb[a] - lo[a]) * inv;
    // fminf / fmaxf drop a NaN operand (0 * inf on a ray parallel to a slab face)
    tmin = fmaxf(tmin, fminf(t1, t2));
    tmax = fminf(tmax, fmaxf(t1, t2));
  }
  return (tmax >= tmin && tmin > 0.f) ? tmin : INFINITY;
}

__device__ __forceinline__ float hit_cyl(const float* q, float ox, float oy, float oz, float dx, float dy, float dz) {
  const float px = ox - q[1], py = oy - q[2], rr = q[3], h = q[4];
  const float a = dx * dx + dy * dy;
  const float b = 2.f * (px * dx + py * dy);
  const float c = px * px + py * py - rr * rr;
  const float disc = b * b - 4.f * a * c;
  float t = INFINITY;
  if (disc >= 0.f && a > 1e-14f) {
    // nearer root, in the cancellation-free form
    const float qq = -0.5f * (b + copysignf(sqrtf(disc), b));
    const float r1 = qq / a, r2 = qq != 0.f ? c / qq : INFINITY;
    const float ts = fminf(r1, r2);
    const float z = oz + ts * dz;
    if (ts > 0.f && z >= 0.f && z <= h) t = ts;
  }
  if (fabsf(dz) > 1e-12f) {
    const float tc = (h - oz) / dz;
    const float xc = px + tc * dx, yc = py + tc * dy;
    if (tc > 0.f && xc * xc + yc * yc <= rr * rr && tc < t) t = tc;
  }
  return t;
}

// grid: (pixel blocks, 2 * n_pairs); scan s = 2 * pair + k (k 0 target, 1 source)
__global__ void __launch_bounds__(kThreads) k_raycast(int H, int W, const float4* __restrict__ rows, float r0,
                                                      const float* __restrict__ objects, const int* __restrict__ n_obj,
                                                      int max_obj, const double* __restrict__ poses, float r_min,
                                                      float r_max, float sigma, float dropout,
                                                      const uint64_t* __restrict__ pair_seed, float* __restrict__ out,
                                                      int n_pairs) {
  __shared__ float so[kMaxObj * 8];
  __shared__ float pose[12];
  const int scan = blockIdx.y;
  const int pair = scan >> 1, k = scan & 1;
  const int no = min(n_obj[pair], max_obj);
  for (int i = threadIdx.x; i < no * 8; i += kThreads) so[i] = objects[(size_t)pair * max_obj * 8 + i];
  if (threadIdx.x < 12) pose[threadIdx.x] = (float)poses[(size_t)scan * 12 + threadIdx.x];
  __syncthreads();
  const float two_pi_over_w = 6.283185307179586f / W;
  float* dst = out + ((size_t)k * n_pairs + pair) * (size_t)H * W;
#pragma unroll 1
  for (int j = 0; j < kPix; ++j) {
    const int p = (blockIdx.x * kPix + j) * kThreads + threadIdx.x;
    if (p >= H * W) break;
    const int v = p / W, u = p % W;
    const float4 row = rows[v];   // cos phi, sin phi, theta, 0
    const float col_az = two_pi_over_w * u;
    float sa, ca, sc, cc;
    sincosf(col_az + row.z, &sa, &ca);
    sincosf(col_az, &sc, &cc);
    const float dsx = ca * row.x, dsy = sa * row.x, dsz = row.y;
    const float osx = r0 * cc, osy = r0 * sc;
    // world frame: o = R o_s + t, d = R d_s (pose rows: R row-major, then t)
    const float ox = pose[0] * osx + pose[1] * osy + pose[9];
    const float oy = pose[3] * osx + pose[4] * osy + pose[10];
    const float oz = pose[6] * osx + pose[7] * osy + pose[11];
    const float dx = pose[0] * dsx + pose[1] * dsy + pose[2] * dsz;
    const float dy = pose[3] * dsx + pose[4] * dsy + pose[5] * dsz;
    const float dz = pose[6] * dsx + pose[7] * dsy + pose[8] * dsz;
    float t = INFINITY;
    if (dz < -1e-12f) {
      const float tg = -oz / dz;
      if (tg > 0.f) t = tg;
    }
    for (int o = 0; o < no; ++o) {
      const float* q = so + 8 * o;
      const float th = q[0] == 0.f ? hit_box(q, ox, oy, oz, dx, dy, dz) : hit_cyl(q, ox, oy, oz, dx, dy, dz);
      t = fminf(t, th);
    }
    float r = (t >= r_min && t <= r_max) ? t : 0.f;
    if (sigma > 0.f || dropout > 0.f) {
      const uint64_t key = mix64(pair_seed[pair] ^ mix64(((uint64_t)k << 32) | (uint64_t)p));
      if (r > 0.f && sigma > 0.f) {
        const float u1 = unit(mix64(key + 1)), u2 = unit(mix64(key + 2));
        r += sigma * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
        if (!(r > 0.f)) r = 0.f;
      }
      if (dropout > 0.f && unit(mix64(key + 3)) <= dropout) r = 0.f;
    }
    dst[p] = r;
  }
}

}  // namespace

extern "C" {

// Ranges of n_pairs scan pairs: out [2][n_pairs][H][W] (index 0: the scan
// from poses[pair][0], the target; 1: from poses[pair][1], the source).
// rows: device float4 [H] (cos phi, sin phi, theta, 0); objects: device
// float [n_pairs][max_obj][8]; n_obj: device int [n_pairs]; poses: device
// float64 [n_pairs][2][12] (R row-major, t); pair_seed: device uint64
// [n_pairs], the key of each pair's noise.  Returns 0 or a CUDA error code.
int synth_raycast(int n_pairs, int H, int W, const void* rows, float r0, const float* objects, const int* n_obj,
                  int max_obj, const double* poses, float r_min, float r_max, float sigma, float dropout,
                  const uint64_t* pair_seed, float* out, void* stream) {
  if (n_pairs <= 0) return 0;
  if (H <= 0 || W <= 0 || max_obj < 0 || max_obj > kMaxObj || n_pairs > 32767) return -1;
  const int pix_blocks = (H * W + kThreads * kPix - 1) / (kThreads * kPix);
  dim3 grid(pix_blocks, 2 * n_pairs);
  k_raycast<<<grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      H, W, static_cast<const float4*>(rows), r0, objects, n_obj, max_obj, poses, r_min, r_max, sigma, dropout,
      pair_seed, out, n_pairs);
  return (int)cudaGetLastError();
}

}  // extern "C"
