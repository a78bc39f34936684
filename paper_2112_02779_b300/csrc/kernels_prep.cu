// Per-image preprocessing kernels: unprojection (Eq. 1-2), the strided
// pyramid (Section 4.1) and neighbour-cross-product normals (Section 4.1)
// with the target plane pyramid written by the same kernel.
#include "rimg_device.cuh"

namespace rimg {

// --------------------------------------------------------------------------
// Unprojection: one thread per pixel, three coalesced output planes.
__global__ void __launch_bounds__(256) k_unproject(DevLevel L, int n, const float* __restrict__ range,
                                                   float* __restrict__ xyz, uint8_t* __restrict__ mask) {
  const long long N = (long long)L.H * L.W;
  const long long total = N * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long img = i / N;
    const int pix = (int)(i - img * N);
    const int v = pix / L.W, u = pix - v * L.W;
    const float r = __ldcs(range + i);
    const bool ok = range_ok(r);
    const float3 p = unproject_px(L, u, v, ok ? r : 0.f);
    float* base = xyz + img * 3 * N + pix;
    __stcs(base, p.x);
    __stcs(base + N, p.y);
    __stcs(base + 2 * N, p.z);
    if (mask) mask[i] = ok ? 1 : 0;
  }
}

cudaError_t launch_unproject(const DevLevel& L, int n, const float* range, float* xyz,
                             uint8_t* mask, cudaStream_t st) {
  const long long total = (long long)L.H * L.W * n;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  long long blocks = (total + threads - 1) / threads;
  if (blocks > 148LL * 64) blocks = 148LL * 64;
  k_unproject<<<(unsigned)blocks, threads, 0, st>>>(L, n, range, xyz, mask);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Strided pyramid: one thread per level-1 pixel; it copies Omega_0(2u, 2v) to
// level 1 and, where its level-1 coordinates are even, to the coarser levels.
template <typename T>
struct PyrOut {
  T* p[RIMG_MAX_LEVELS];
};

template <typename T>
__global__ void __launch_bounds__(256) k_pyramid(int n, int H, int W, int levels, const T* __restrict__ in,
                                                 PyrOut<T> out) {
  const int H1 = H >> 1, W1 = W >> 1;
  const long long N1 = (long long)H1 * W1;
  const long long total = N1 * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long img = i / N1;
    const int pix = (int)(i - img * N1);
    const int v1 = pix / W1, u1 = pix - v1 * W1;
    const T val = in[img * (long long)H * W + (long long)(2 * v1) * W + 2 * u1];
    out.p[1][i] = val;
#pragma unroll
    for (int l = 2; l < RIMG_MAX_LEVELS; ++l) {
      const int m = (1 << (l - 1)) - 1;
      if (l >= levels || ((u1 & m) | (v1 & m))) break;
      const int Hl = H >> l, Wl = W >> l;
      out.p[l][img * (long long)Hl * Wl + (long long)(v1 >> (l - 1)) * Wl + (u1 >> (l - 1))] = val;
    }
  }
}

cudaError_t launch_pyramid(int n, int H, int W, int levels, int channels, const float* in,
                           float* const* out_levels, cudaStream_t st) {
  if (levels < 2 || n == 0) return cudaSuccess;
  const long long total = (long long)(H >> 1) * (W >> 1) * n;
  const int threads = 256;
  long long blocks = (total + threads - 1) / threads;
  if (blocks > 148LL * 64) blocks = 148LL * 64;
  if (channels == 1) {
    PyrOut<float> o{};
    for (int l = 1; l < levels; ++l) o.p[l] = out_levels[l];
    k_pyramid<float><<<(unsigned)blocks, threads, 0, st>>>(n, H, W, levels, in, o);
  } else {
    PyrOut<float4> o{};
    for (int l = 1; l < levels; ++l) o.p[l] = reinterpret_cast<float4*>(out_levels[l]);
    k_pyramid<float4><<<(unsigned)blocks, threads, 0, st>>>(n, H, W, levels,
                                                            reinterpret_cast<const float4*>(in), o);
  }
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Normals.  A 32 x 8 tile of output pixels per block; the block unprojects the
// (32+2) x (8+2) halo tile into shared memory once (u wraps, rows outside the
// image are invalid), then each thread forms the two central differences,
// their cross product and the validity tests, and writes the plane
// (n, n . P) to level 0 and, when its coordinates are multiples of 2^l, to
// level l (the strided normal pyramid).
constexpr int NT_X = 32, NT_Y = 8;
constexpr int NH_X = NT_X + 2, NH_Y = NT_Y + 2;

struct PlaneOut {
  float4* p[RIMG_MAX_LEVELS];
};

// The PCA variant (the eigen-decomposition alternative of Section 4.1): the
// window's points whose range passes the same jump test as the cross
// product's neighbours (at least kPcaMinPoints of the nine, centre included)
// give the scatter matrix C = sum (p - mean)(p - mean)^T; its eigenvalues come
// from the closed form for symmetric 3x3 matrices (trace / deviation /
// determinant, one acos and two cos), the normal from the largest cross
// product of two rows of C - lambda_0 I.  Invalid when lambda_1 <= 1e-4
// lambda_2 (collinear points).
// Plane (n, n . P) of pixel (u, v) to level 0 and, when its coordinates are
// multiples of 2^l, to level l; the optional mask gets the validity.
__device__ __forceinline__ void write_plane(const PlaneOut& out, uint8_t* mask0, int img, int H, int W, int u, int v,
                                            int levels, float4 plane, bool ok) {
  const long long N = (long long)H * W;
  out.p[0][img * N + (long long)v * W + u] = plane;
  if (mask0) mask0[img * N + (long long)v * W + u] = ok ? 1 : 0;
  // unrolled so the level pointers are read with constant indices (no local copy)
#pragma unroll
  for (int l = 1; l < RIMG_MAX_LEVELS; ++l) {
    const int m = (1 << l) - 1;
    if (l >= levels || ((u & m) | (v & m))) break;
    const int Hl = H >> l, Wl = W >> l;
    out.p[l][img * (long long)Hl * Wl + (long long)(v >> l) * Wl + (u >> l)] = plane;
  }
}

constexpr int kPcaMinPoints = 5;
constexpr float kPcaCollinear = 1e-4f;

__device__ __forceinline__ bool pca_normal(const float (&q)[9][3], const bool (&use)[9], float& nx, float& ny,
                                           float& nz) {
  float k = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    if (use[i]) { k += 1.f; mx += q[i][0]; my += q[i][1]; mz += q[i][2]; }
  if (k < (float)kPcaMinPoints) return false;
  const float ik = 1.f / k;
  mx *= ik; my *= ik; mz *= ik;
  float c00 = 0.f, c01 = 0.f, c02 = 0.f, c11 = 0.f, c12 = 0.f, c22 = 0.f;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    if (use[i]) {
      const float a = q[i][0] - mx, b = q[i][1] - my, c = q[i][2] - mz;
      c00 = fmaf(a, a, c00); c01 = fmaf(a, b, c01); c02 = fmaf(a, c, c02);
      c11 = fmaf(b, b, c11); c12 = fmaf(b, c, c12); c22 = fmaf(c, c, c22);
    }
  // scale to O(1) (the eigenvectors do not change)
  const float sc = fmaxf(fmaxf(fmaxf(fabsf(c00), fabsf(c11)), fmaxf(fabsf(c22), fabsf(c01))),
                         fmaxf(fabsf(c02), fabsf(c12)));
  if (!(sc > 0.f)) return false;
  const float is = 1.f / sc;
  c00 *= is; c01 *= is; c02 *= is; c11 *= is; c12 *= is; c22 *= is;
  const float qm = (c00 + c11 + c22) * (1.f / 3.f);
  const float b00 = c00 - qm, b11 = c11 - qm, b22 = c22 - qm;
  const float off = fmaf(c01, c01, fmaf(c02, c02, c12 * c12));
  const float p2 = fmaf(b00, b00, fmaf(b11, b11, fmaf(b22, b22, 2.f * off))) * (1.f / 6.f);
  if (!(p2 > 0.f)) return false;                     // isotropic: no preferred direction
  const float p = sqrtf(p2), ip = 1.f / p;
  // det((C - q I) / p) / 2
  const float d00 = b00 * ip, d11 = b11 * ip, d22 = b22 * ip, e01 = c01 * ip, e02 = c02 * ip, e12 = c12 * ip;
  const float det = d00 * fmaf(d11, d22, -e12 * e12) - e01 * fmaf(e01, d22, -e12 * e02) +
                    e02 * fmaf(e01, e12, -d11 * e02);
  const float hr = fminf(1.f, fmaxf(-1.f, 0.5f * det));
  const float phi = acosf(hr) * (1.f / 3.f);
  const float l2 = fmaf(2.f * p, cosf(phi), qm);
  const float l0 = fmaf(2.f * p, cosf(phi + 2.0943951023931953f), qm);
  const float l1 = 3.f * qm - l0 - l2;
  if (!(l1 > kPcaCollinear * l2)) return false;
  // null vector of C - l0 I: the longest cross product of two of its rows
  const float r0x = c00 - l0, r0y = c01, r0z = c02;
  const float r1x = c01, r1y = c11 - l0, r1z = c12;
  const float r2x = c02, r2y = c12, r2z = c22 - l0;
  const float ax = fmaf(r0y, r1z, -r0z * r1y), ay = fmaf(r0z, r1x, -r0x * r1z), az = fmaf(r0x, r1y, -r0y * r1x);
  const float bx = fmaf(r0y, r2z, -r0z * r2y), by = fmaf(r0z, r2x, -r0x * r2z), bz = fmaf(r0x, r2y, -r0y * r2x);
  const float cx = fmaf(r1y, r2z, -r1z * r2y), cy = fmaf(r1z, r2x, -r1x * r2z), cz = fmaf(r1x, r2y, -r1y * r2x);
  const float na = fmaf(ax, ax, fmaf(ay, ay, az * az));
  const float nb = fmaf(bx, bx, fmaf(by, by, bz * bz));
  const float nc = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
  float vx = ax, vy = ay, vz = az, vn = na;
  if (nb > vn) { vx = bx; vy = by; vz = bz; vn = nb; }
  if (nc > vn) { vx = cx; vy = cy; vz = cz; vn = nc; }
  if (!(vn > 0.f)) return false;
  const float inv = rsqrtf(vn);
  nx = vx * inv; ny = vy * inv; nz = vz * inv;
  return true;
}

template <bool PCA>
__global__ void __launch_bounds__(NT_X* NT_Y) k_normals(DevLevel L, int levels, int n, const float* __restrict__ range,
                                                        float rel_jump, PlaneOut out,
                                                        uint8_t* __restrict__ mask0) {
  __shared__ float4 sp[NH_Y][NH_X];   // point (x, y, z) and range (0: invalid) of each tile pixel
  const int img = blockIdx.z;
  const int u0 = blockIdx.x * NT_X - 1, v0 = blockIdx.y * NT_Y - 1;
  const int H = L.H, W = L.W;
  const float* rimg = range + (long long)img * H * W;
  const int tid = threadIdx.y * NT_X + threadIdx.x;
  auto stage = [&](int hy, int hx) {
    const int v = v0 + hy;
    // the halo wraps around the 360 degree image: u0 + hx lies in [-1, W + 32],
    // so one conditional step suffices unless the image is narrower than the tile
    int u = u0 + hx;
    u = (u < 0) ? u + W : u;
    u = (u >= W) ? u - W : u;
    if (u >= W) u %= W;
    const bool row_in = v >= 0 && v < H;
    const float r = row_in ? __ldg(rimg + (long long)v * W + u) : 0.f;
    const bool ok = row_in && range_ok(r);
    float3 p = make_float3(0.f, 0.f, 0.f);
    if (ok) p = unproject_px(L, u, v, r);
    sp[hy][hx] = make_float4(p.x, p.y, p.z, ok ? r : 0.f);
  };
  // each thread stages its own pixel, then 84 threads the ring around the tile
  // (top and bottom halo rows, left and right halo columns)
  stage(threadIdx.y + 1, threadIdx.x + 1);
  if (tid < 2 * NH_X + 2 * NT_Y) {
    int hy, hx;
    if (tid < NH_X) {
      hy = 0; hx = tid;
    } else if (tid < 2 * NH_X) {
      hy = NH_Y - 1; hx = tid - NH_X;
    } else {
      const int k = tid - 2 * NH_X;
      hy = 1 + (k >> 1); hx = (k & 1) ? NH_X - 1 : 0;
    }
    stage(hy, hx);
  }
  __syncthreads();
  const int u = blockIdx.x * NT_X + threadIdx.x;
  const int v = blockIdx.y * NT_Y + threadIdx.y;
  if (u >= W || v >= H) return;
  const int cx = threadIdx.x + 1, cy = threadIdx.y + 1;
  const float4 C = sp[cy][cx];
  const float rc = C.w;
  if (PCA) {
    float q[9][3];
    bool use[9];
    const float px = C.x, py = C.y, pz = C.z;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float4 Q = sp[cy + i / 3 - 1][cx + i % 3 - 1];
      use[i] = rc > 0.f && Q.w > 0.f && fmaf(rel_jump, rc, -fabsf(Q.w - rc)) >= 0.f;
      q[i][0] = Q.x - px;
      q[i][1] = Q.y - py;
      q[i][2] = Q.z - pz;
    }
    float nx = 0.f, ny = 0.f, nz = 0.f;
    bool ok = (v > 0) && (v < H - 1) && rc > 0.f && pca_normal(q, use, nx, ny, nz);
    float4 plane = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ok) {
      float d = fmaf(nx, px, fmaf(ny, py, nz * pz));
      if (d > 0.f) { nx = -nx; ny = -ny; nz = -nz; d = -d; }
      plane = make_float4(nx, ny, nz, d);
    }
    write_plane(out, mask0, img, H, W, u, v, levels, plane, ok);
    return;
  }
  const float4 Pl = sp[cy][cx - 1], Pr = sp[cy][cx + 1], Pu = sp[cy - 1][cx], Pd = sp[cy + 1][cx];
  const float rl = Pl.w, rr = Pr.w, ru = Pu.w, rd = Pd.w;
  // |r_nb - r_c| <= rel_jump * r_c decided exactly: the difference is exact
  // (Sterbenz) whenever the test can pass, and the sign of one fused
  // multiply-add is the sign of the exact value.
  bool ok = (v > 0) && (v < H - 1) && rc > 0.f && rl > 0.f && rr > 0.f && ru > 0.f && rd > 0.f;
  ok = ok && fmaf(rel_jump, rc, -fabsf(rl - rc)) >= 0.f && fmaf(rel_jump, rc, -fabsf(rr - rc)) >= 0.f &&
       fmaf(rel_jump, rc, -fabsf(ru - rc)) >= 0.f && fmaf(rel_jump, rc, -fabsf(rd - rc)) >= 0.f;
  const float ax = Pr.x - Pl.x, ay = Pr.y - Pl.y, az = Pr.z - Pl.z;
  const float bx = Pd.x - Pu.x, by = Pd.y - Pu.y, bz = Pd.z - Pu.z;
  float nx = fmaf(ay, bz, -az * by), ny = fmaf(az, bx, -ax * bz), nz = fmaf(ax, by, -ay * bx);
  const float c2 = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
  const float a2 = fmaf(ax, ax, fmaf(ay, ay, az * az));
  const float b2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
  ok = ok && (c2 > 1e-8f * a2 * b2);
  float4 plane = make_float4(0.f, 0.f, 0.f, 0.f);
  if (ok) {
    const float inv = rsqrtf(c2);
    nx *= inv; ny *= inv; nz *= inv;
    float d = fmaf(nx, C.x, fmaf(ny, C.y, nz * C.z));
    if (d > 0.f) { nx = -nx; ny = -ny; nz = -nz; d = -d; }
    plane = make_float4(nx, ny, nz, d);
  }
  write_plane(out, mask0, img, H, W, u, v, levels, plane, ok);
}

cudaError_t launch_normals(const rimg_sensor* s, int n, const float* range, float rel_jump, int method,
                           float* const* planes_levels, uint8_t* mask0, cudaStream_t st) {
  const DevLevel L = dev_level(s, 0);
  const long long N = (long long)L.H * L.W;
  for (int off = 0; off < n; off += 65535) {       // grid.z limit
    const int cnt = n - off < 65535 ? n - off : 65535;
    PlaneOut o{};
    for (int l = 0; l < s->levels; ++l)
      o.p[l] = reinterpret_cast<float4*>(planes_levels[l]) + (long long)off * (L.H >> l) * (L.W >> l);
    dim3 grid((L.W + NT_X - 1) / NT_X, (L.H + NT_Y - 1) / NT_Y, cnt);
    if (method == 1)
      k_normals<true><<<grid, dim3(NT_X, NT_Y), 0, st>>>(L, s->levels, cnt, range + off * N, rel_jump, o,
                                                         mask0 ? mask0 + off * N : nullptr);
    else
      k_normals<false><<<grid, dim3(NT_X, NT_Y), 0, st>>>(L, s->levels, cnt, range + off * N, rel_jump, o,
                                                          mask0 ? mask0 + off * N : nullptr);
  }
  return cudaGetLastError();
}

}  // namespace rimg
