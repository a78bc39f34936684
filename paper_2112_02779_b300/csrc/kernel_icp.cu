// The fused projective-association Gauss-Newton step (Section 4.1, Eq. 5-7):
// per source pixel unproject -> transform -> project -> gather the target
// plane -> residual, pseudo-Huber weight, Jacobian -> 29 reduced terms; warp
// shuffle, block and one-pass grid reduction (last-block-done counter, no
// spinning); the last block of each pair reduces in FP64, solves the 6x6
// system by Cholesky and composes the SE(3) update.
#include "rimg_device.cuh"

namespace rimg {

namespace {

// FP64 Cholesky solve of the 6x6 system H x = -g; false on a pivot
// <= 1e-12 * trace(H).
__device__ bool chol6_solve(const double (&Hm)[6][6], const double (&g)[6], double (&x)[6]) {
  double L[6][6];
  double tr = 0.0;
#pragma unroll
  for (int i = 0; i < 6; ++i) tr += Hm[i][i];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    double d = Hm[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 1e-12 * tr)) return false;
    const double ljj = sqrt(d);
    L[j][j] = ljj;
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      double s = Hm[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      L[i][j] = s / ljj;
    }
  }
  double y[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double s = -g[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
    y[i] = s / L[i][i];
  }
#pragma unroll
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
#pragma unroll
    for (int k = i + 1; k < 6; ++k) s -= L[k][i] * x[k];
    x[i] = s / L[i][i];
  }
  return true;
}

// T <- Exp(xi) T for xi = (omega, tau): Rodrigues rotation and the V matrix
// of SE(3), with second-order series below 1e-8 rad.
__device__ void se3_left_update(double* T, const double (&xi)[6]) {
  const double wx = xi[0], wy = xi[1], wz = xi[2];
  const double th2 = wx * wx + wy * wy + wz * wz;
  const double th = sqrt(th2);
  double A, B, C;
  if (th < 1e-8) {
    A = 1.0 - th2 / 6.0;
    B = 0.5 - th2 / 24.0;
    C = 1.0 / 6.0 - th2 / 120.0;
  } else {
    double s, c;
    sincos(th, &s, &c);
    A = s / th;
    B = (1.0 - c) / th2;
    C = (th - s) / (th2 * th);
  }
  const double K[3][3] = {{0.0, -wz, wy}, {wz, 0.0, -wx}, {-wy, wx, 0.0}};
  double K2[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) K2[i][j] = K[i][0] * K[0][j] + K[i][1] * K[1][j] + K[i][2] * K[2][j];
  double Ri[3][3], V[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double I = (i == j) ? 1.0 : 0.0;
      Ri[i][j] = I + A * K[i][j] + B * K2[i][j];
      V[i][j] = I + B * K[i][j] + C * K2[i][j];
    }
  double Tn[12];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Tn[i * 4 + j] = Ri[i][0] * T[0 * 4 + j] + Ri[i][1] * T[1 * 4 + j] + Ri[i][2] * T[2 * 4 + j];
    Tn[i * 4 + 3] = Ri[i][0] * T[3] + Ri[i][1] * T[7] + Ri[i][2] * T[11] +
                    (V[i][0] * xi[3] + V[i][1] * xi[4] + V[i][2] * xi[5]);
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) T[k] = Tn[k];
}

}  // namespace

// ---------------------------------------------------------------------------
// Packed FP32x2 arithmetic (two independent FP32 lanes per instruction).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, exactly rounded once (fma(b, -1, a))
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// 16-byte asynchronous global -> shared copy; with pred false nothing is read
// and the destination is filled with zeros.
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, bool pred) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int n = pred ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// The 29 reduced quantities live in 15 float2 accumulators (30 lanes):
// lane index f = 2 * pair + (0 for .x, 1 for .y).  kFlat maps the output
// order (21 upper-triangle J^T W J entries row-major, 6 J^T W e, sum w e^2,
// count) to lanes.
constexpr int kPairs = 15;
__constant__ int kFlat[kRed] = {0,  18, 2,  12, 4,  14,  // H00..H05
                                1,  13, 3,  15, 5,       // H11..H15
                                6,  19, 8,  16,          // H22..H25
                                7,  17, 9,               // H33..H35
                                10, 20,                  // H44, H45
                                11,                      // H55
                                22, 23, 24, 25, 26, 27,  // g0..g5
                                21, 28};                 // sum w e^2, count

// Point-to-plane terms of one association: residual e = n.x - d, IRLS weight,
// J = [x cross n, n]; adds w J J^T (upper triangle), w e J, w e^2 and the
// count into t.  A zero plane (no association) contributes exactly nothing.
__device__ __forceinline__ void accumulate_px(float2 (&t)[kPairs], float x, float y, float z, float4 pl,
                                              float inv_delta) {
  const float nx = pl.x, ny = pl.y, nz = pl.z;
  const float e = fmaf(nx, x, fmaf(ny, y, fmaf(nz, z, -pl.w)));
  float w = 1.f;
  if (inv_delta > 0.f) {
    const float q = e * inv_delta;
    w = rsqrtf(fmaf(q, q, 1.f));
  }
  const float J0 = fmaf(y, nz, -z * ny), J1 = fmaf(z, nx, -x * nz), J2 = fmaf(x, ny, -y * nx);
  const float2 J01 = f2(J0, J1), J23 = f2(J2, nx), J45 = f2(ny, nz);
  const float2 W2 = f2(w, w);
  const float2 U01 = mul2(W2, J01), U23 = mul2(W2, J23), U45 = mul2(W2, J45);
  const float2 E2 = f2(e, e);
  t[0] = fma2(U01, J01, t[0]);                         // H00 H11
  t[1] = fma2(U01, J23, t[1]);                         // H02 H13
  t[2] = fma2(U01, J45, t[2]);                         // H04 H15
  t[3] = fma2(U23, J23, t[3]);                         // H22 H33
  t[4] = fma2(U23, J45, t[4]);                         // H24 H35
  t[5] = fma2(U45, J45, t[5]);                         // H44 H55
  t[6] = fma2(U01, f2(nx, J2), t[6]);                  // H03 H12
  t[7] = fma2(U01, f2(nz, ny), t[7]);                  // H05 H14
  t[8] = fma2(U23, f2(nz, ny), t[8]);                  // H25 H34
  t[9] = fma2(f2(U01.x, U23.x), f2(J1, nx), t[9]);     // H01 H23
  t[10] = fma2(f2(U45.x, w * e), f2(nz, e), t[10]);    // H45, w e^2
  t[11] = fma2(U01, E2, t[11]);                        // g0 g1
  t[12] = fma2(U23, E2, t[12]);                        // g2 g3
  t[13] = fma2(U45, E2, t[13]);                        // g4 g5
  t[14].x += (nx != 0.f || ny != 0.f || nz != 0.f) ? 1.f : 0.f;
}

// Shared memory of one block (dynamic, > 48 KB).  Each thread owns column
// `tid` of the staging arrays: the gathered target planes of its in-flight
// chunks and their transformed source points (x, y, z, target index bits).
template <int THREADS>
struct IcpSmem {
  float4 planes[2][4][THREADS];
  float4 pts[2][4][THREADS];
  float red[THREADS / 32][2 * kPairs];     // per-warp sums
  double tot[32];
  float T[12];
  int last;
};

// Per-thread bookkeeping of one 4-pixel chunk between issuing its gathers and
// accumulating it (the points themselves wait in shared memory).
struct Chunk {
  long long off;
};

template <bool R0, bool GATE, bool ASSOC, bool KAHAN, int THREADS>
__global__ void __launch_bounds__(THREADS, 512 / THREADS) k_icp(IcpLaunch a) {
  extern __shared__ float4 smem_raw[];
  IcpSmem<THREADS>& sm = *reinterpret_cast<IcpSmem<THREADS>*>(smem_raw);
  const int tid = threadIdx.x;
  const int pair = blockIdx.x / a.bpp;
  const int blk = blockIdx.x - pair * a.bpp;
  if (tid < 12) sm.T[tid] = (float)a.pose[pair * 16 + tid];
  __syncthreads();
  const float R00 = sm.T[0], R01 = sm.T[1], R02 = sm.T[2], t0 = sm.T[3];
  const float R10 = sm.T[4], R11 = sm.T[5], R12 = sm.T[6], t1 = sm.T[7];
  const float R20 = sm.T[8], R21 = sm.T[9], R22 = sm.T[10], t2 = sm.T[11];

  const DevLevel& S = a.src;
  const DevLevel& D = a.dst;
  const int W = S.W, H = S.H;
  const long long Ns = (long long)H * W;
  const long long Nd = (long long)D.H * D.W;
  const float* src = a.src_range + pair * Ns;
  const float4* planes = a.dst_planes + pair * Nd;
  const float* drange = GATE ? a.dst_range + pair * Nd : nullptr;
  const float inv_delta = a.huber_delta > 0.f ? 1.f / a.huber_delta : 0.f;
  const float gate2 = a.max_corr_dist * a.max_corr_dist;

  float2 s[kPairs], c[kPairs];
#pragma unroll
  for (int i = 0; i < kPairs; ++i) { s[i] = f2(0.f, 0.f); c[i] = f2(0.f, 0.f); }

  const int cpr = W >> 2;                       // 4-pixel chunks per row
  const int v_begin = blk * a.rows_per_block;
  const int v_end = min(H, v_begin + a.rows_per_block);
  const int nchunks = max(0, v_end - v_begin) * cpr;
  int v = v_begin + tid / cpr;
  int cu = tid - (tid / cpr) * cpr;
  const int dv = THREADS / cpr, dcu = THREADS - dv * cpr;
  int ch = tid;

  // Stage A: unproject, transform and project the chunk at (v, cu); start
  // the asynchronous gathers of its target planes into staging buffer `buf`.
  auto issue = [&](Chunk& k, int buf) {
    const int u0 = cu << 2;
    k.off = (long long)v * W + u0;
    const float4 r4 = __ldcs(reinterpret_cast<const float4*>(src + k.off));
    const float rr[4] = {r4.x, r4.y, r4.z, r4.w};
    const float4 rw = __ldg(S.rows + v);
    const float4 cc = __ldg(reinterpret_cast<const float4*>(S.cos_u + u0));
    const float4 ss = __ldg(reinterpret_cast<const float4*>(S.sin_u + u0));
    const float cs[4] = {cc.x, cc.y, cc.z, cc.w}, sn[4] = {ss.x, ss.y, ss.z, ss.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool valid = range_ok(rr[q]);
      const float r = valid ? rr[q] : 0.f;
      const float ct = fmaf(cs[q], rw.z, -sn[q] * rw.w);
      const float st = fmaf(sn[q], rw.z, cs[q] * rw.w);
      const float rc = r * rw.x;
      const float px = R0 ? fmaf(rc, ct, S.r0 * cs[q]) : rc * ct;
      const float py = R0 ? fmaf(rc, st, S.r0 * sn[q]) : rc * st;
      const float pz = r * rw.y;
      const float X = fmaf(R00, px, fmaf(R01, py, fmaf(R02, pz, t0)));
      const float Y = fmaf(R10, px, fmaf(R11, py, fmaf(R12, pz, t1)));
      const float Z = fmaf(R20, px, fmaf(R21, py, fmaf(R22, pz, t2)));
      int uu, vv;
      const bool fov = project_px<R0>(D, make_float3(X, Y, Z), a.proj_iters, uu, vv);
      const bool ok = valid && fov;
      const int idx = ok ? vv * D.W + uu : -1;
      cp_async16_zfill(&sm.planes[buf][q][tid], planes + (ok ? idx : 0), ok);
      sm.pts[buf][q][tid] = make_float4(X, Y, Z, __int_as_float(idx));
    }
    cu += dcu;
    v += dv;
    if (cu >= cpr) { cu -= cpr; ++v; }
    ch += THREADS;
  };

  // Stage B: accumulate a chunk whose gathers have landed in buffer `buf`
  // into the plain FP32 chunk sums t; flush() adds t to the running sums with
  // Kahan compensation (once per two chunks, 8 pixels).
  float2 t[kPairs];
#pragma unroll
  for (int i = 0; i < kPairs; ++i) t[i] = f2(0.f, 0.f);
  auto flush = [&]() {
#pragma unroll
    for (int i = 0; i < kPairs; ++i) {
      if (KAHAN) {
        const float2 y = sub2(t[i], c[i]);
        const float2 tt = add2(s[i], y);
        c[i] = sub2(sub2(tt, s[i]), y);
        s[i] = tt;
      } else {
        s[i] = add2(s[i], t[i]);
      }
      t[i] = f2(0.f, 0.f);
    }
  };
  auto consume = [&](const Chunk& k, int buf) {
    int out_idx[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float4 pl = sm.planes[buf][q][tid];
      const float4 P = sm.pts[buf][q][tid];
      const int idx = __float_as_int(P.w);
      if (GATE) {
        bool keep = idx >= 0;
        if (keep) {
          const int vv = idx / D.W, uu = idx - vv * D.W;
          const float rq = __ldg(drange + idx);
          const float3 qq = unproject_px(D, uu, vv, range_ok(rq) ? rq : 0.f);
          const float dx = P.x - qq.x, dy = P.y - qq.y, dz = P.z - qq.z;
          keep = range_ok(rq) && (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= gate2);
        }
        if (!keep) pl = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      out_idx[q] = (pl.x != 0.f || pl.y != 0.f || pl.z != 0.f) ? idx : -1;
      accumulate_px(t, P.x, P.y, P.z, pl, inv_delta);
    }
    if (ASSOC) {
      int* ap = a.assoc + pair * Ns + k.off;
      *reinterpret_cast<int4*>(ap) = make_int4(out_idx[0], out_idx[1], out_idx[2], out_idx[3]);
    }
  };

  // Two chunks in flight per thread: issue chunk k+1's gathers, then
  // accumulate chunk k (each thread only reads its own staging slots, so no
  // block barrier is needed inside the loop).
  Chunk c0, c1;
  bool have0 = ch < nchunks;
  if (have0) issue(c0, 0);
  cp_async_commit();
  while (have0) {
    const bool have1 = ch < nchunks;
    if (have1) issue(c1, 1);
    cp_async_commit();
    cp_async_wait1();
    consume(c0, 0);
    if (!have1) break;
    have0 = ch < nchunks;
    if (have0) issue(c0, 0);
    cp_async_commit();
    cp_async_wait1();
    consume(c1, 1);
    flush();
  }
  flush();
  asm volatile("cp.async.wait_all;\n" ::: "memory");

  // thread sums -> warp tree -> block (FP32)
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int i = 0; i < kPairs; ++i) {
    float2 val = KAHAN ? sub2(s[i], c[i]) : s[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float2 other = f2(__shfl_xor_sync(0xffffffffu, val.x, o), __shfl_xor_sync(0xffffffffu, val.y, o));
      val = add2(val, other);
    }
    if (lane == 0) { sm.red[warp][2 * i] = val.x; sm.red[warp][2 * i + 1] = val.y; }
  }
  __syncthreads();
  if (a.bpp == 1) {
    // one block per pair: the block total is the pair total
    if (tid < kRed) {
      const int f = kFlat[tid];
      float acc = 0.f;
#pragma unroll
      for (int w = 0; w < THREADS / 32; ++w) acc += sm.red[w][f];
      sm.tot[tid] = (double)acc;
      if (a.out29) a.out29[pair * kRed + tid] = (double)acc;
    }
    __syncthreads();
  } else {
    if (tid < kRed) {
      const int f = kFlat[tid];
      float acc = 0.f;
#pragma unroll
      for (int w = 0; w < THREADS / 32; ++w) acc += sm.red[w][f];
      a.partials[((long long)pair * a.bpp + blk) * kRedStride + tid] = acc;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const unsigned prev = atomicAdd(a.counters + pair, 1u);
      sm.last = (prev == (unsigned)(a.bpp - 1));
    }
    __syncthreads();
    if (!sm.last) return;
    __threadfence();
    // last block of this pair: FP64 cross-block reduction in a fixed order
    if (tid < kRed) {
      double acc = 0.0;
      const float* pp = a.partials + (long long)pair * a.bpp * kRedStride + tid;
      for (int b = 0; b < a.bpp; ++b) acc += (double)__ldcg(pp + (long long)b * kRedStride);
      sm.tot[tid] = acc;
      if (a.out29) a.out29[pair * kRed + tid] = acc;
    }
    __syncthreads();
    if (tid == 0) a.counters[pair] = 0u;
  }
  if (tid == 0 && a.update) {
    double Hm[6][6], g[6], x[6];
    int q = 0;
    for (int i = 0; i < 6; ++i)
      for (int j = i; j < 6; ++j) { Hm[i][j] = sm.tot[q]; Hm[j][i] = sm.tot[q]; ++q; }
    for (int i = 0; i < 6; ++i) g[i] = sm.tot[21 + i];
    bool good = sm.tot[28] >= 6.0;
    if (good) good = chol6_solve(Hm, g, x);
    if (good) {
      double T[12];
      for (int k = 0; k < 12; ++k) T[k] = a.pose[pair * 16 + k];
      se3_left_update(T, x);
      for (int k = 0; k < 12; ++k) a.pose[pair * 16 + k] = T[k];
    } else if (a.status) {
      atomicOr(a.status + pair, RIMG_FLAG_DEGENERATE);
    }
  }
}

namespace {
int g_num_sms = 0;
int g_blocks_per_sm[2] = {0, 0};   // resident blocks per SM for 128- and 256-thread blocks

template <int T>
int occupancy() {
  constexpr size_t bytes = sizeof(IcpSmem<T>);
  cudaFuncSetAttribute(k_icp<false, false, false, true, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)bytes);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_icp<false, false, false, true, T>, T, bytes);
  return nb > 0 ? nb : 1;
}
}  // namespace

void icp_grid(int H, int W, int n_pairs, int* bpp, int* rows_per_block, int* threads) {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_blocks_per_sm[0] = occupancy<128>();
    g_blocks_per_sm[1] = occupancy<256>();
    g_num_sms = sms > 0 ? sms : 148;
  }
  // Aim at ~16 four-pixel chunks per thread: enough work to amortise a
  // block's reduction, few enough blocks per pair to keep the FP64
  // cross-block sum short.  Small levels use 128-thread blocks and one block
  // per pair (no grid-level counter at all).
  const long long cpp = (long long)H * (W / 4);
  const int T = (cpp <= 128 * 16) ? 128 : 256;
  long long b = cpp / ((long long)T * 16);
  if (b < 1) b = 1;
  // small batches: split each pair further until the grid fills the GPU
  const long long cap = (long long)g_num_sms * g_blocks_per_sm[T == 256 ? 1 : 0];
  while ((long long)n_pairs * b < cap && b < H) b = (2 * b < H) ? 2 * b : H;
  if (b > H) b = H;
  const int rpb = (int)((H + b - 1) / b);
  *rows_per_block = rpb;
  *bpp = (H + rpb - 1) / rpb;
  *threads = T;
}

template <bool R0, bool GATE, bool ASSOC, bool KAHAN, int T>
cudaError_t launch_icp_t(const IcpLaunch& a, long long blocks, cudaStream_t st) {
  constexpr size_t bytes = sizeof(IcpSmem<T>);
  static bool configured = false;   // per instantiation; the attribute is per function
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_icp<R0, GATE, ASSOC, KAHAN, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k_icp<R0, GATE, ASSOC, KAHAN, T><<<(unsigned)blocks, T, bytes, st>>>(a);
  return cudaGetLastError();
}

template <bool R0, bool GATE, bool ASSOC, bool KAHAN>
cudaError_t launch_icp_k(const IcpLaunch& a, long long blocks, cudaStream_t st) {
  return a.threads == 128 ? launch_icp_t<R0, GATE, ASSOC, KAHAN, 128>(a, blocks, st)
                          : launch_icp_t<R0, GATE, ASSOC, KAHAN, 256>(a, blocks, st);
}

cudaError_t launch_icp(const IcpLaunch& a, cudaStream_t st) {
  if (a.n_pairs == 0) return cudaSuccess;
  const long long blocks = (long long)a.n_pairs * a.bpp;
  const bool r0 = a.dst.r0 != 0.f || a.src.r0 != 0.f;
  const bool gate = a.max_corr_dist > 0.f;
  const bool assoc = a.assoc != nullptr;
  const bool kahan = a.kahan != 0;
#define RIMG_LAUNCH(R, G, A, K) return launch_icp_k<R, G, A, K>(a, blocks, st)
  if (r0) {
    if (gate) { if (assoc) { if (kahan) RIMG_LAUNCH(true, true, true, true); else RIMG_LAUNCH(true, true, true, false); }
                else { if (kahan) RIMG_LAUNCH(true, true, false, true); else RIMG_LAUNCH(true, true, false, false); } }
    else { if (assoc) { if (kahan) RIMG_LAUNCH(true, false, true, true); else RIMG_LAUNCH(true, false, true, false); }
           else { if (kahan) RIMG_LAUNCH(true, false, false, true); else RIMG_LAUNCH(true, false, false, false); } }
  } else {
    if (gate) { if (assoc) { if (kahan) RIMG_LAUNCH(false, true, true, true); else RIMG_LAUNCH(false, true, true, false); }
                else { if (kahan) RIMG_LAUNCH(false, true, false, true); else RIMG_LAUNCH(false, true, false, false); } }
    else { if (assoc) { if (kahan) RIMG_LAUNCH(false, false, true, true); else RIMG_LAUNCH(false, false, true, false); }
           else { if (kahan) RIMG_LAUNCH(false, false, false, true); else RIMG_LAUNCH(false, false, false, false); } }
  }
#undef RIMG_LAUNCH
}

}  // namespace rimg
