// Per-image preprocessing kernels: unprojection (Eq. 1-2), the strided
// pyramid (Section 4.1) and neighbour-cross-product normals (Section 4.1)
// with the target plane pyramid written by the same kernel.
#include <algorithm>

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
// Normals.  Both kernels unproject a halo tile of the target image into
// shared memory once (u wraps around the 360 degree image, rows outside the
// image are invalid), form each pixel's normal from its neighbours there and
// write the plane (n, n . P) to level 0 and, when the pixel's coordinates are
// multiples of 2^l, to level l (the strided normal pyramid).  PCA variant: a
// 32 x 8 tile, one pixel per thread.
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

__global__ void __launch_bounds__(NT_X* NT_Y) k_normals_pca(DevLevel L, int levels, const float* __restrict__ range,
                                                            float rel_jump, PlaneOut out, uint8_t* __restrict__ mask0) {
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
}

// Cross-product normals, one warp per strip of 128 columns x NC_ROWS rows and
// four horizontally adjacent pixels per lane.  The warp walks down its strip
// with a rolling window of three unprojected rows held in registers (rows
// v - 1, v, v + 1), so every range row is loaded and unprojected once per
// strip, with the range loads issued two rows ahead of their use.  The left
// and right neighbours of a lane's group come from the adjacent lanes by
// shuffle; the strip's two edge columns are loaded by lanes 0 and 31.
// Columns wrap around the 360 degree image (W is a multiple of 4, so a group
// never straddles the wrap, and a lane past the image's last column holds
// the wrapped columns that the last active lane needs).  No shared memory
// and no barriers.  Per pixel the arithmetic is that of the one-pixel form
// (the same operations in the same order).
constexpr int NC_LANES_PX = 4;
constexpr int NC_W = 32 * NC_LANES_PX;   // strip width in pixels
#ifndef RIMG_NC_ROWS
#define RIMG_NC_ROWS 8
#endif
constexpr int NC_ROWS = RIMG_NC_ROWS;    // output rows per strip
constexpr int NC_WARPS = 4;              // warps per block

// Unprojection (Eq. 1-2) of one pixel from its row entry and column cos/sin;
// all zero when the pixel is invalid (rows outside the image arrive as range 0).
__device__ __forceinline__ float4 stage_point(const float4& rw, float cu, float su, float r0, float rq) {
  const bool ok = range_ok(rq);
  const float ct = fmaf(cu, rw.z, -su * rw.w);
  const float st = fmaf(su, rw.z, cu * rw.w);
  const float rc = rq * rw.x;
  return ok ? make_float4(fmaf(rc, ct, r0 * cu), fmaf(rc, st, r0 * su), rq * rw.y, rq)
            : make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ float4 shfl4(const float4& a, int src) {
  return make_float4(__shfl_sync(0xffffffffu, a.x, src), __shfl_sync(0xffffffffu, a.y, src),
                     __shfl_sync(0xffffffffu, a.z, src), __shfl_sync(0xffffffffu, a.w, src));
}

struct Row4 {
  float4 p[4];   // x, y, z, range of the lane's four pixels
};

__global__ void __launch_bounds__(32 * NC_WARPS, 4) k_normals_cross(DevLevel L, int levels, int n_img,
                                                                 const float* __restrict__ range, float rel_jump,
                                                                 PlaneOut out, uint8_t* __restrict__ mask0) {
  const int H = L.H, W = L.W;
  const long long N = (long long)H * W;
  const int lane = threadIdx.x & 31;
  const int segs = (W + NC_W - 1) / NC_W;
  const int per_img = segs * ((H + NC_ROWS - 1) / NC_ROWS);
  // strip index: < 2^31 for every accepted size (the launcher caps the images per launch)
  const int strip = blockIdx.x * NC_WARPS + (threadIdx.x >> 5);
  if (strip >= per_img * n_img) return;   // whole warps only
  const int img = strip / per_img;
  const int rem = strip - img * per_img;
  const int rb = rem / segs;
  const int c0 = (rem - rb * segs) * NC_W, v0 = rb * NC_ROWS;
  auto wrap = [&](int u) {
    if (u < 0) u += W;
    if (u >= W) u = (W >= NC_W) ? u - W : u % W;
    return u;
  };
  const float* rimg = range + img * N;
  const int u0 = c0 + NC_LANES_PX * lane;
  const int g = wrap(u0);
  const float4 cu = __ldg(reinterpret_cast<const float4*>(L.cos_u + g));
  const float4 su = __ldg(reinterpret_cast<const float4*>(L.sin_u + g));
  const bool edge = lane == 0 || lane == 31;
  const int ue = wrap(lane == 0 ? c0 - 1 : c0 + NC_W);   // the edge lanes' extra column
  const float cue = __ldg(L.cos_u + ue), sue = __ldg(L.sin_u + ue);
  auto load_row = [&](int vv) {
    return (vv >= 0 && vv < H) ? __ldg(reinterpret_cast<const float4*>(rimg + (long long)vv * W + g))
                               : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto load_edge = [&](int vv) { return (edge && vv >= 0 && vv < H) ? __ldg(rimg + (long long)vv * W + ue) : 0.f; };
  auto row_entry = [&](int vv) { return __ldg(L.rows + min(max(vv, 0), H - 1)); };
  auto unproject_row = [&](int vv, const float4& r4) {
    const float4 rw = row_entry(vv);
    Row4 R;
    R.p[0] = stage_point(rw, cu.x, su.x, L.r0, r4.x);
    R.p[1] = stage_point(rw, cu.y, su.y, L.r0, r4.y);
    R.p[2] = stage_point(rw, cu.z, su.z, L.r0, r4.z);
    R.p[3] = stage_point(rw, cu.w, su.w, L.r0, r4.w);
    return R;
  };
  const bool col_ok = u0 < W;
  const bool mask_aligned = (reinterpret_cast<uintptr_t>(mask0) & 3) == 0;

  Row4 Pu = unproject_row(v0 - 1, load_row(v0 - 1));
  Row4 Pc = unproject_row(v0, load_row(v0));
  float4 r_next = load_row(v0 + 1);          // range of row v + 1
  float4 r_next2 = load_row(v0 + 2);         // range of row v + 2
  float e_cur = load_edge(v0);               // edge range of row v
#pragma unroll
  for (int i = 0; i < NC_ROWS; ++i) {
    const int v = v0 + i;
    const Row4 Pd = unproject_row(v + 1, r_next);
    r_next = r_next2;
    r_next2 = load_row(v + 3);
    const float e_next = load_edge(v + 1);
    // left neighbour of pixel 0 and right neighbour of pixel 3 in row v
    float4 Pl = shfl4(Pc.p[3], (lane + 31) & 31);
    float4 Pr = shfl4(Pc.p[0], (lane + 1) & 31);
    if (edge) {
      const float4 p = stage_point(row_entry(v), cue, sue, L.r0, e_cur);
      if (lane == 0) Pl = p; else Pr = p;
    }
    if (v < H && col_ok) {
      const bool row_ok = (v > 0) && (v < H - 1);
      float4 plane[4];
      bool okq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 C = Pc.p[q];
        const float4 A = q == 0 ? Pl : Pc.p[q - 1];
        const float4 B = q == 3 ? Pr : Pc.p[q + 1];
        const float4 Up = Pu.p[q], Dn = Pd.p[q];
        const float rc = C.w, rl = A.w, rr = B.w, ru = Up.w, rd = Dn.w;
        bool ok = row_ok && rc > 0.f && rl > 0.f && rr > 0.f && ru > 0.f && rd > 0.f;
        ok = ok && fmaf(rel_jump, rc, -fabsf(rl - rc)) >= 0.f && fmaf(rel_jump, rc, -fabsf(rr - rc)) >= 0.f &&
             fmaf(rel_jump, rc, -fabsf(ru - rc)) >= 0.f && fmaf(rel_jump, rc, -fabsf(rd - rc)) >= 0.f;
        const float ax = B.x - A.x, ay = B.y - A.y, az = B.z - A.z;
        const float bx = Dn.x - Up.x, by = Dn.y - Up.y, bz = Dn.z - Up.z;
        float nx = fmaf(ay, bz, -az * by), ny = fmaf(az, bx, -ax * bz), nz = fmaf(ax, by, -ay * bx);
        const float c2 = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
        const float a2 = fmaf(ax, ax, fmaf(ay, ay, az * az));
        const float b2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
        ok = ok && (c2 > 1e-8f * a2 * b2);
        float4 pl = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ok) {
          const float inv = rsqrtf(c2);
          nx *= inv; ny *= inv; nz *= inv;
          float d = fmaf(nx, C.x, fmaf(ny, C.y, nz * C.z));
          if (d > 0.f) { nx = -nx; ny = -ny; nz = -nz; d = -d; }
          pl = make_float4(nx, ny, nz, d);
        }
        plane[q] = pl;
        okq[q] = ok;
      }
      const long long o0 = img * N + (long long)v * W + u0;
      float4* p0 = out.p[0] + o0;
#pragma unroll
      for (int q = 0; q < 4; ++q) p0[q] = plane[q];
      if (mask0) {
        const uchar4 m = make_uchar4(okq[0], okq[1], okq[2], okq[3]);
        if (mask_aligned) {
          *reinterpret_cast<uchar4*>(mask0 + o0) = m;
        } else {
          mask0[o0] = m.x; mask0[o0 + 1] = m.y; mask0[o0 + 2] = m.z; mask0[o0 + 3] = m.w;
        }
      }
      // the strided pyramid: level 1 takes pixels 0 and 2 of the group on
      // even rows, level l >= 2 pixel 0 where u0 and v are multiples of 2^l
      if (levels > 1 && (v & 1) == 0) {
        const int W1 = W >> 1;
        float4* p1 = out.p[1] + img * (long long)(H >> 1) * W1 + (long long)(v >> 1) * W1 + (u0 >> 1);
        p1[0] = plane[0];
        p1[1] = plane[2];
#pragma unroll
        for (int l = 2; l < RIMG_MAX_LEVELS; ++l) {
          const int m = (1 << l) - 1;
          if (l >= levels || ((u0 & m) | (v & m))) break;
          const int Hl = H >> l, Wl = W >> l;
          out.p[l][img * (long long)Hl * Wl + (long long)(v >> l) * Wl + (u0 >> l)] = plane[0];
        }
      }
    }
    Pu = Pc;
    Pc = Pd;
    e_cur = e_next;
  }
}

cudaError_t launch_normals(const rimg_sensor* s, int n, const float* range, float rel_jump, int method,
                           float* const* planes_levels, uint8_t* mask0, cudaStream_t st) {
  const DevLevel L = dev_level(s, 0);
  const long long N = (long long)L.H * L.W;
  // images per launch: the PCA grid's z limit; for the strip kernel, strip
  // indices below 2^31
  const long long per_img = (long long)((L.W + NC_W - 1) / NC_W) * ((L.H + NC_ROWS - 1) / NC_ROWS);
  const int chunk = (method == 1) ? 65535 : (int)std::max(1LL, std::min(65535LL, 2147483647LL / per_img));
  for (int off = 0; off < n; off += chunk) {
    const int cnt = n - off < chunk ? n - off : chunk;
    PlaneOut o{};
    for (int l = 0; l < s->levels; ++l)
      o.p[l] = reinterpret_cast<float4*>(planes_levels[l]) + (long long)off * (L.H >> l) * (L.W >> l);
    uint8_t* m = mask0 ? mask0 + off * N : nullptr;
    if (method == 1) {
      dim3 grid((L.W + NT_X - 1) / NT_X, (L.H + NT_Y - 1) / NT_Y, cnt);
      k_normals_pca<<<grid, dim3(NT_X, NT_Y), 0, st>>>(L, s->levels, range + off * N, rel_jump, o, m);
    } else {
      const unsigned blocks = (unsigned)((per_img * cnt + NC_WARPS - 1) / NC_WARPS);
      k_normals_cross<<<blocks, 32 * NC_WARPS, 0, st>>>(L, s->levels, cnt, range + off * N, rel_jump, o, m);
    }
  }
  return cudaGetLastError();
}

}  // namespace rimg
