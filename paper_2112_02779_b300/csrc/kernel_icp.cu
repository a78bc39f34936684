// The fused projective-association Gauss-Newton step (Section 4.1, Eq. 5-7):
// per source pixel unproject -> transform -> project -> gather the target
// plane -> residual, pseudo-Huber weight, Jacobian -> 29 reduced terms; warp
// shuffle, block and one-pass grid reduction (last-block-done counter, no
// spinning); the last block of each pair reduces in FP64, solves the 6x6
// system by Cholesky and composes the SE(3) update.
#include "rimg_device.cuh"

namespace rimg {

namespace {

__device__ __forceinline__ void chunk_cols(const float2* cols, int u0, float2 (&c)[4]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(cols + u0));
  const float4 b = __ldg(reinterpret_cast<const float4*>(cols + u0 + 2));
  c[0] = make_float2(a.x, a.y);
  c[1] = make_float2(a.z, a.w);
  c[2] = make_float2(b.x, b.y);
  c[3] = make_float2(b.z, b.w);
}

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

template <bool R0, bool GATE, bool ASSOC, bool KAHAN>
__global__ void __launch_bounds__(kIcpThreads, 2) k_icp(IcpLaunch a) {
  __shared__ float sT[12];
  __shared__ float red[kIcpThreads / 32][kRedStride];
  __shared__ double tot[kRedStride];
  __shared__ int s_last;

  const int tid = threadIdx.x;
  const int pair = blockIdx.x / a.bpp;
  const int blk = blockIdx.x - pair * a.bpp;
  if (tid < 12) sT[tid] = (float)a.pose[pair * 16 + tid];
  __syncthreads();
  const float R00 = sT[0], R01 = sT[1], R02 = sT[2], t0 = sT[3];
  const float R10 = sT[4], R11 = sT[5], R12 = sT[6], t1 = sT[7];
  const float R20 = sT[8], R21 = sT[9], R22 = sT[10], t2 = sT[11];

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

  float s[kRed], c[kRed];
#pragma unroll
  for (int i = 0; i < kRed; ++i) { s[i] = 0.f; c[i] = 0.f; }

  const int cpr = W >> 2;                       // 4-pixel chunks per row
  const int v_begin = blk * a.rows_per_block;
  const int v_end = min(H, v_begin + a.rows_per_block);
  const int nchunks = max(0, v_end - v_begin) * cpr;
  int v = v_begin + tid / cpr;
  int cu = tid - (tid / cpr) * cpr;
  const int dv = kIcpThreads / cpr, dcu = kIcpThreads - dv * cpr;

  for (int ch = tid; ch < nchunks; ch += kIcpThreads) {
    const int u0 = cu << 2;
    const long long off = (long long)v * W + u0;
    const float4 r4 = __ldcs(reinterpret_cast<const float4*>(src + off));
    const float rr[4] = {r4.x, r4.y, r4.z, r4.w};
    const float4 rw = __ldg(S.rows + v);
    float2 cl[4];
    chunk_cols(S.cols, u0, cl);

    float3 X[4];
    int idx[4];
    bool ok[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool valid = range_ok(rr[k]);
      const float r = valid ? rr[k] : 0.f;
      const float ct = fmaf(cl[k].x, rw.z, -cl[k].y * rw.w);
      const float st = fmaf(cl[k].y, rw.z, cl[k].x * rw.w);
      const float rc = r * rw.x;
      const float px = fmaf(rc, ct, S.r0 * cl[k].x);
      const float py = fmaf(rc, st, S.r0 * cl[k].y);
      const float pz = r * rw.y;
      X[k] = make_float3(fmaf(R00, px, fmaf(R01, py, fmaf(R02, pz, t0))),
                         fmaf(R10, px, fmaf(R11, py, fmaf(R12, pz, t1))),
                         fmaf(R20, px, fmaf(R21, py, fmaf(R22, pz, t2))));
      int uu, vv;
      const bool fov = project_px<R0>(D, X[k], a.proj_iters, uu, vv);
      ok[k] = valid && fov;
      idx[k] = vv * D.W + uu;
    }
    float4 pl[4];
    float rq[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      pl[k] = ok[k] ? __ldg(planes + idx[k]) : make_float4(0.f, 0.f, 0.f, 0.f);
      if (GATE) rq[k] = ok[k] ? __ldg(drange + idx[k]) : 0.f;
    }

    float t[kRed];
#pragma unroll
    for (int i = 0; i < kRed; ++i) t[i] = 0.f;
    int out_idx[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float nx = pl[k].x, ny = pl[k].y, nz = pl[k].z;
      bool pv = ok[k] && (nx != 0.f || ny != 0.f || nz != 0.f);
      if (GATE) {
        const int vv = idx[k] / D.W, uu = idx[k] - vv * D.W;
        const float3 q = unproject_px(D, uu, vv, range_ok(rq[k]) ? rq[k] : 0.f);
        const float dx = X[k].x - q.x, dy = X[k].y - q.y, dz = X[k].z - q.z;
        pv = pv && range_ok(rq[k]) && (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= gate2);
      }
      out_idx[k] = pv ? idx[k] : -1;
      const float e0 = fmaf(nx, X[k].x, fmaf(ny, X[k].y, fmaf(nz, X[k].z, -pl[k].w)));
      float w = 1.f;
      if (inv_delta > 0.f) {
        const float z = e0 * inv_delta;
        w = rsqrtf(fmaf(z, z, 1.f));
      }
      w = pv ? w : 0.f;
      const float e = pv ? e0 : 0.f;
      const float J[6] = {fmaf(X[k].y, nz, -X[k].z * ny), fmaf(X[k].z, nx, -X[k].x * nz),
                          fmaf(X[k].x, ny, -X[k].y * nx), nx, ny, nz};
      float wJ[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) wJ[i] = w * J[i];
      int q = 0;
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j) { t[q] = fmaf(wJ[i], J[j], t[q]); ++q; }
#pragma unroll
      for (int i = 0; i < 6; ++i) t[21 + i] = fmaf(wJ[i], e, t[21 + i]);
      t[27] = fmaf(w * e, e, t[27]);
      t[28] += pv ? 1.f : 0.f;
    }
    if (ASSOC) {
      int* ap = a.assoc + pair * Ns + off;
      *reinterpret_cast<int4*>(ap) = make_int4(out_idx[0], out_idx[1], out_idx[2], out_idx[3]);
    }
#pragma unroll
    for (int i = 0; i < kRed; ++i) {
      if (KAHAN) {
        const float y = t[i] - c[i];
        const float tt = s[i] + y;
        c[i] = (tt - s[i]) - y;
        s[i] = tt;
      } else {
        s[i] += t[i];
      }
    }
    cu += dcu;
    v += dv;
    if (cu >= cpr) { cu -= cpr; ++v; }
  }

  // thread value -> warp tree -> block
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int i = 0; i < kRed; ++i) {
    float val = KAHAN ? (s[i] - c[i]) : s[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
    if (lane == 0) red[warp][i] = val;
  }
  __syncthreads();
  if (tid < kRed) {
    float acc = 0.f;
#pragma unroll
    for (int w = 0; w < kIcpThreads / 32; ++w) acc += red[w][tid];
    a.partials[((long long)pair * a.bpp + blk) * kRedStride + tid] = acc;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned prev = atomicAdd(a.counters + pair, 1u);
    s_last = (prev == (unsigned)(a.bpp - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // last block of this pair: FP64 cross-block reduction in a fixed order
  if (tid < kRed) {
    double acc = 0.0;
    const float* pp = a.partials + (long long)pair * a.bpp * kRedStride + tid;
    for (int b = 0; b < a.bpp; ++b) acc += (double)__ldcg(pp + (long long)b * kRedStride);
    tot[tid] = acc;
    if (a.out29) a.out29[pair * kRed + tid] = acc;
  }
  __syncthreads();
  if (tid == 0) {
    a.counters[pair] = 0u;
    if (a.update) {
      double Hm[6][6], g[6], x[6];
      int q = 0;
      for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) { Hm[i][j] = tot[q]; Hm[j][i] = tot[q]; ++q; }
      for (int i = 0; i < 6; ++i) g[i] = tot[21 + i];
      bool good = tot[28] >= 6.0;
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
}

namespace {
int g_blocks_per_sm = 0;
int g_num_sms = 0;
}

void icp_grid(int H, int W, int n_pairs, int* bpp, int* rows_per_block) {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_icp<false, false, false, true>, kIcpThreads, 0);
    g_blocks_per_sm = nb > 0 ? nb : 2;
  }
  const long long capacity = (long long)g_num_sms * g_blocks_per_sm;
  // enough blocks for ~8 resident waves, never more than one per row
  long long want = (8 * capacity + n_pairs - 1) / (n_pairs > 0 ? n_pairs : 1);
  if (want < 1) want = 1;
  if (want > H) want = H;
  int rpb = (int)((H + want - 1) / want);
  *rows_per_block = rpb;
  *bpp = (H + rpb - 1) / rpb;
  (void)W;
}

cudaError_t launch_icp(const IcpLaunch& a, cudaStream_t st) {
  if (a.n_pairs == 0) return cudaSuccess;
  const long long blocks = (long long)a.n_pairs * a.bpp;
  const bool r0 = a.dst.r0 != 0.f;
  const bool gate = a.max_corr_dist > 0.f;
  const bool assoc = a.assoc != nullptr;
  const bool kahan = a.kahan != 0;
#define RIMG_LAUNCH(R, G, A, K) k_icp<R, G, A, K><<<(unsigned)blocks, kIcpThreads, 0, st>>>(a)
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
  return cudaGetLastError();
}

}  // namespace rimg
