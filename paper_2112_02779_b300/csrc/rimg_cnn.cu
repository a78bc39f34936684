// Learned pose proposal: a small BF16 convolutional network that reads the
// coarsest pyramid level (Section 4.1) of a source and a target scan and
// regresses a 6-DoF initial pose for the multi-scale registration.  The paper
// stops at Gauss-Newton from a given initial pose and lists learned features
// on the range image as future work (Section 7); this network is an
// extension, and the registration stays its judge.
//
// Network (channels-last activations, one row per output pixel):
//   input  [n][8][128][2]  (source, target) ranges / 32, invalid -> 0
//   conv1..conv5: 3x3, stride 2, ReLU; rows zero-padded, columns wrapped
//   (360-degree azimuth); 2->32->64->64->128->128 channels,
//   8x128 -> 4x64 -> 2x32 -> 1x16 -> 1x8 -> 1x4
//   linear 512 -> 6: p = (omega / 0.25 rad, t / 3 m), T0 = [Exp(omega), t].
//
// Every contraction runs on the tcgen05 BF16 GEMM (kernel_gemm.cu) with FP32
// accumulation:
//   forward   Y_l   = relu(col(X_l) W_l^T + b_l)          M = pixels, K = 9 C_in
//   data grad dcol  = dZ_l W_l                           K = C_out
//   weight    dW_l  = dZ_l^T col(X_l), db_l = dZ_l^T 1    K = pixels (split-K)
// The GEMM wants both operands K-major, so the backward pass transposes dZ
// and the im2col matrix (the latter with an extra row of ones, which turns
// the bias gradient into one more output column).  Master weights and Adam
// moments are FP32; the GEMMs read BF16 shadows (and transposed shadows for
// the data gradient) that the optimizer rewrites after each update.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "rimg_internal.h"

namespace rimg {

namespace {

constexpr int kConv = 5;
constexpr int kFcIn = 512, kFcOut = 6;
constexpr int kInH = RIMG_CNN_IN_H, kInW = RIMG_CNN_IN_W;

struct ConvGeo {
  int Hi, Wi, Ci, Ho, Wo, Co, K, Kp, Cp;   // Kp = K rounded up to 64, Cp = C_out rounded up to 64
};

constexpr ConvGeo kGeo[kConv] = {
    {8, 128, 2, 4, 64, 32, 18, 64, 64},
    {4, 64, 32, 2, 32, 64, 288, 320, 64},
    {2, 32, 64, 1, 16, 64, 576, 576, 64},
    {1, 16, 64, 1, 8, 128, 576, 576, 128},
    {1, 8, 128, 1, 4, 128, 1152, 1152, 128},
};

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
inline size_t r64(size_t x) { return (x + 63) / 64 * 64; }

// Flat parameter layout: per conv W [Co][K] then b [Co]; then the linear W [6][512], b [6].
struct ParamLayout {
  size_t w[kConv + 1], b[kConv + 1], total;
};

ParamLayout param_layout() {
  ParamLayout p{};
  size_t o = 0;
  for (int l = 0; l < kConv; ++l) {
    p.w[l] = o;
    o += (size_t)kGeo[l].Co * kGeo[l].K;
    p.b[l] = o;
    o += kGeo[l].Co;
  }
  p.w[kConv] = o;
  o += (size_t)kFcOut * kFcIn;
  p.b[kConv] = o;
  o += kFcOut;
  p.total = o;
  return p;
}

// Model state: master parameters, Adam moments, BF16 shadows.
struct StateLayout {
  size_t master, m, v;
  size_t wbf[kConv + 1];   // [Co][Kp] (linear: [6][512])
  size_t wt[kConv + 1];    // [Kp][Cp] (linear: [512][64])
  size_t end;
};

StateLayout state_layout() {
  const ParamLayout P = param_layout();
  StateLayout s{};
  size_t o = 0;
  s.master = o; o = align_up(o + 4 * P.total);
  s.m = o; o = align_up(o + 4 * P.total);
  s.v = o; o = align_up(o + 4 * P.total);
  for (int l = 0; l < kConv; ++l) { s.wbf[l] = o; o = align_up(o + 2 * (size_t)kGeo[l].Co * kGeo[l].Kp); }
  s.wbf[kConv] = o; o = align_up(o + 2 * (size_t)kFcOut * kFcIn);
  for (int l = 0; l < kConv; ++l) { s.wt[l] = o; o = align_up(o + 2 * (size_t)kGeo[l].Kp * kGeo[l].Cp); }
  s.wt[kConv] = o; o = align_up(o + 2 * (size_t)kFcIn * 64);
  s.end = o;
  return s;
}

// Split count of the weight-gradient GEMM over K = M64 pixels: about four
// 64-wide K steps per split, at most 256 splits.
inline int wgrad_splits(size_t m64) { return (int)std::max<size_t>(1, std::min<size_t>(256, m64 / 256)); }

struct WsLayout {
  size_t x0;
  size_t col[kConv], y[kConv], act[kConv];
  size_t pred, dp, dpt, x6t, dx6;
  size_t dz[kConv], dzt[kConv], colt[kConv], dcol[kConv], dx[kConv];
  size_t part[kConv + 1];
  int splits[kConv + 1];
  size_t grad, loss, end;
};

WsLayout ws_layout(int n) {
  WsLayout w{};
  size_t o = 0;
  const size_t N = (size_t)n, n64 = r64(N);
  w.x0 = o; o = align_up(o + 2 * N * kInH * kInW * 2);
  for (int l = 0; l < kConv; ++l) {
    const ConvGeo& g = kGeo[l];
    const size_t M = N * g.Ho * g.Wo;
    w.col[l] = o; o = align_up(o + 2 * M * g.Kp);
    w.y[l] = o; o = align_up(o + 4 * M * g.Co);
    w.act[l] = o; o = align_up(o + 2 * M * g.Co);
  }
  w.pred = o; o = align_up(o + 4 * N * kFcOut);
  w.dp = o; o = align_up(o + 2 * N * 64);
  w.dpt = o; o = align_up(o + 2 * kFcOut * n64);
  w.x6t = o; o = align_up(o + 2 * (size_t)(kFcIn + 1) * n64);
  w.dx6 = o; o = align_up(o + 4 * N * kFcIn);
  for (int l = 0; l < kConv; ++l) {
    const ConvGeo& g = kGeo[l];
    const size_t M = N * g.Ho * g.Wo, M64 = r64(M);
    w.dz[l] = o; o = align_up(o + 2 * M * g.Cp);
    w.dzt[l] = o; o = align_up(o + 2 * (size_t)g.Co * M64);
    w.colt[l] = o; o = align_up(o + 2 * (size_t)(g.Kp + 1) * M64);
    w.dcol[l] = o; o = align_up(o + (l > 0 ? 4 * M * g.Kp : 0));
    w.dx[l] = o; o = align_up(o + (l > 0 ? 4 * N * g.Hi * g.Wi * g.Ci : 0));
    w.splits[l] = wgrad_splits(M64);
    w.part[l] = o; o = align_up(o + 4 * (size_t)w.splits[l] * g.Co * (g.Kp + 1));
  }
  w.splits[kConv] = wgrad_splits(n64);
  w.part[kConv] = o; o = align_up(o + 4 * (size_t)w.splits[kConv] * kFcOut * (kFcIn + 1));
  w.grad = o; o = align_up(o + 4 * param_layout().total);
  w.loss = o; o = align_up(o + sizeof(double));
  w.end = o;
  return w;
}

// ---------------------------------------------------------------------------
// Device helpers

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// Rotation vector -> R (Rodrigues), float64; second-order series below 1e-8 rad.
__device__ void so3_exp_d(const double w[3], double R[9]) {
  const double a2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double A, B;
  if (a2 < 1e-16) {
    A = 1.0;
    B = 0.5;
  } else {
    const double a = sqrt(a2);
    A = sin(a) / a;
    B = (1.0 - cos(a)) / a2;
  }
  const double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double kk = 0.0;
      for (int t = 0; t < 3; ++t) kk += K[3 * i + t] * K[3 * t + j];
      R[3 * i + j] = (i == j ? 1.0 : 0.0) + A * K[3 * i + j] + B * kk;
    }
}

// R -> rotation vector (angle in [0, pi]), float64.  The angle comes from
// atan2(|v|, (tr R - 1) / 2) with v the axial vector of (R - R^T) / 2; near pi
// the axis is taken from the symmetric part of R instead.
__device__ void so3_log_d(const double* T, double w[3]) {
  const double v0 = 0.5 * (T[9] - T[6]), v1 = 0.5 * (T[2] - T[8]), v2 = 0.5 * (T[4] - T[1]);
  const double c = 0.5 * (T[0] + T[5] + T[10] - 1.0);
  const double s = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
  const double a = atan2(s, c);
  if (c > -0.9) {
    const double f = s > 1e-12 ? a / s : 1.0 + a * a / 6.0;
    w[0] = f * v0; w[1] = f * v1; w[2] = f * v2;
    return;
  }
  // (R + R^T) / 2 - c I = (1 - c) k k^T
  const double S[9] = {T[0] - c, 0.5 * (T[1] + T[4]), 0.5 * (T[2] + T[8]),
                       0.5 * (T[4] + T[1]), T[5] - c, 0.5 * (T[6] + T[9]),
                       0.5 * (T[8] + T[2]), 0.5 * (T[9] + T[6]), T[10] - c};
  int j = 0;
  if (S[4] > S[0]) j = 1;
  if (S[8] > S[4 * j]) j = 2;
  const double d = sqrt(S[4 * j]);
  double k0 = S[j] / d, k1 = S[3 + j] / d, k2 = S[6 + j] / d;
  if (k0 * v0 + k1 * v1 + k2 * v2 < 0) { k0 = -k0; k1 = -k1; k2 = -k2; }
  const double kn = sqrt(k0 * k0 + k1 * k1 + k2 * k2);
  w[0] = a * k0 / kn; w[1] = a * k1 / kn; w[2] = a * k2 / kn;
}

// ---------------------------------------------------------------------------
// Kernels

// Coarsest-level input: pixel (v, u) of pair i reads (stride v, stride u) of
// the finest images (the strided pyramid keeps every 2^l-th row and column).
__global__ void k_cnn_input(int n, int H, int W, int stride, const float* __restrict__ src,
                            const float* __restrict__ dst, const int32_t* __restrict__ index,
                            __nv_bfloat162* __restrict__ x0) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * kInH * kInW) return;
  const int i = t / (kInH * kInW), r = t % (kInH * kInW);
  const int v = r / kInW, u = r % kInW;
  const size_t p = index ? (size_t)index[i] : (size_t)i;
  const size_t off = (p * H + (size_t)v * stride) * W + (size_t)u * stride;
  float a = src[off], b = dst[off];
  a = (isfinite(a) && a > 0.f) ? a * RIMG_CNN_RANGE_SCALE : 0.f;
  b = (isfinite(b) && b > 0.f) ? b * RIMG_CNN_RANGE_SCALE : 0.f;
  x0[t] = __floats2bfloat162_rn(a, b);
}

// im2col: row m = (i, ho, wo), column k = (kh * 3 + kw) * Ci + c, zero for
// rows outside the image and for k >= K (padding up to Kp).  Each thread
// writes 8 consecutive columns (16 bytes).
__global__ void k_im2col(int n, ConvGeo g, const uint16_t* __restrict__ x, uint16_t* __restrict__ col) {
  const int chunks = g.Kp / 8;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t M = (size_t)n * g.Ho * g.Wo;
  if (t >= M * chunks) return;
  const size_t m = t / chunks;
  const int k0 = (int)(t % chunks) * 8;
  const int wo = (int)(m % g.Wo), ho = (int)((m / g.Wo) % g.Ho);
  const size_t i = m / ((size_t)g.Wo * g.Ho);
  __align__(16) uint16_t out[8];
  if (g.Ci % 8 == 0) {
    // the 8 columns are 8 consecutive channels of one tap
    const int tap = k0 / g.Ci, c0 = k0 % g.Ci;
    const int kh = tap / 3, kw = tap % 3;
    const int hi = 2 * ho - 1 + kh, wi = (2 * wo - 1 + kw + g.Wi) % g.Wi;
    uint4 val = make_uint4(0, 0, 0, 0);
    if (k0 < g.K && hi >= 0 && hi < g.Hi)
      val = *reinterpret_cast<const uint4*>(x + ((i * g.Hi + hi) * g.Wi + wi) * g.Ci + c0);
    *reinterpret_cast<uint4*>(col + m * g.Kp + k0) = val;
    return;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int k = k0 + j;
    uint16_t v = 0;
    if (k < g.K) {
      const int tap = k / g.Ci, c = k % g.Ci;
      const int kh = tap / 3, kw = tap % 3;
      const int hi = 2 * ho - 1 + kh, wi = (2 * wo - 1 + kw + g.Wi) % g.Wi;
      if (hi >= 0 && hi < g.Hi) v = x[((i * g.Hi + hi) * g.Wi + wi) * g.Ci + c];
    }
    out[j] = v;
  }
  *reinterpret_cast<uint4*>(col + m * g.Kp + k0) = *reinterpret_cast<const uint4*>(out);
}

// out[c][r] = in[r][c] for r < R, c < C (BF16), zero for R <= r < Rp; with
// ones_row, out[C][r] = 1 for r < R (0 beyond).  32 x 32 tiles through shared
// memory; block (32, 8).
__global__ void k_transpose_bf16(int R, int C, const uint16_t* __restrict__ in, int ld_in, uint16_t* __restrict__ out,
                                 int Rp, int ones_row) {
  __shared__ uint16_t tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int j = ty; j < 32; j += 8) {
    const int r = r0 + j, c = c0 + tx;
    uint16_t v = 0;
    if (r < R && c < C) v = in[(size_t)r * ld_in + c];
    else if (ones_row && c == C && r < R) v = 0x3F80;   // BF16 1.0
    tile[j][tx] = v;
  }
  __syncthreads();
  const int Cout = C + (ones_row ? 1 : 0);
  for (int j = ty; j < 32; j += 8) {
    const int c = c0 + j, r = r0 + tx;
    if (c < Cout && r < Rp) out[(size_t)c * Rp + r] = tile[tx][j];
  }
}

// dZ = dY * (Y > 0) as BF16 [M][Cp] (columns Co..Cp-1 zero).
__global__ void k_relu_bwd(size_t M, int Co, int Cp, const float* __restrict__ dy, const float* __restrict__ y,
                           uint16_t* __restrict__ dz) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int chunks = Cp / 8;
  if (t >= M * chunks) return;
  const size_t m = t / chunks;
  const int c0 = (int)(t % chunks) * 8;
  __align__(16) uint16_t out[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = c0 + j;
    float v = 0.f;
    if (c < Co) {
      const size_t o = m * Co + c;
      v = y[o] > 0.f ? dy[o] : 0.f;
    }
    out[j] = bf16_bits(v);
  }
  *reinterpret_cast<uint4*>(dz + m * Cp + c0) = *reinterpret_cast<const uint4*>(out);
}

// Adjoint of im2col, as a gather: input element (i, hi, wi, c) sums the
// column entries of every output pixel whose window covers it (at most two
// taps per direction for a 3-wide stride-2 window), in a fixed order.
__global__ void k_col2im(int n, ConvGeo g, const float* __restrict__ dcol, float* __restrict__ dx) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)n * g.Hi * g.Wi * g.Ci;
  if (t >= total) return;
  const int c = (int)(t % g.Ci);
  const int wi = (int)((t / g.Ci) % g.Wi);
  const int hi = (int)((t / ((size_t)g.Ci * g.Wi)) % g.Hi);
  const size_t i = t / ((size_t)g.Ci * g.Wi * g.Hi);
  float acc = 0.f;
#pragma unroll
  for (int kh = 0; kh < 3; ++kh) {
    const int h2 = hi + 1 - kh;
    if (h2 < 0 || (h2 & 1)) continue;
    const int ho = h2 >> 1;
    if (ho >= g.Ho) continue;
#pragma unroll
    for (int kw = 0; kw < 3; ++kw) {
      const int w2 = (wi + 1 - kw + g.Wi) % g.Wi;
      if (w2 & 1) continue;
      const int wo = w2 >> 1;
      acc += dcol[((i * g.Ho + ho) * g.Wo + wo) * g.Kp + (kh * 3 + kw) * g.Ci + c];
    }
  }
  dx[t] = acc;
}

// Loss 1/(2n) sum |p - y|^2 with y = (Log R / 0.25, t / 3) of the label pose,
// and dL/dp = (p - y) / n as BF16 in both layouts the backward GEMMs read:
// dp [n][64] (columns 6..63 zero) and dp^T [6][n64] (columns n..n64-1 zero).
// One block; FP64 block reduction of the loss.
__global__ void k_cnn_loss(int n, int n64, const float* __restrict__ pred, const double* __restrict__ T_label,
                           const int32_t* __restrict__ index, double* __restrict__ loss, uint16_t* __restrict__ dp,
                           uint16_t* __restrict__ dpt) {
  __shared__ double red[32];
  double acc = 0.0;
  const double inv_n = 1.0 / n;
  for (int i = threadIdx.x; i < n64; i += blockDim.x) {
    if (i >= n) {
      for (int j = 0; j < kFcOut; ++j) dpt[(size_t)j * n64 + i] = 0;
      continue;
    }
    const double* T = T_label + 16 * (index ? (size_t)index[i] : (size_t)i);
    double w[3];
    so3_log_d(T, w);
    const double y[6] = {w[0] / RIMG_CNN_OMEGA_SCALE, w[1] / RIMG_CNN_OMEGA_SCALE, w[2] / RIMG_CNN_OMEGA_SCALE,
                         T[3] / RIMG_CNN_T_SCALE, T[7] / RIMG_CNN_T_SCALE, T[11] / RIMG_CNN_T_SCALE};
    for (int j = 0; j < kFcOut; ++j) {
      const double r = (double)pred[(size_t)i * kFcOut + j] - y[j];
      acc += r * r;
      const uint16_t b = bf16_bits((float)(r * inv_n));
      dp[(size_t)i * 64 + j] = b;
      dpt[(size_t)j * n64 + i] = b;
    }
    for (int j = kFcOut; j < 64; ++j) dp[(size_t)i * 64 + j] = 0;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    *loss = 0.5 * s * inv_n;
  }
}

// Parameter blocks for the gradient reduction and the optimizer.
struct Blocks {
  const float* part[kConv + 1];   // weight-gradient partials [S][Co][ld]
  int w_off[kConv + 1], b_off[kConv + 1], end[kConv + 1];
  int K[kConv + 1], Kp[kConv + 1], Cp[kConv + 1], ld[kConv + 1], S[kConv + 1], Co[kConv + 1];
  uint16_t* wbf[kConv + 1];
  uint16_t* wt[kConv + 1];
};

__device__ __forceinline__ int block_of(const Blocks& B, int g) {
  int l = 0;
#pragma unroll
  for (int k = 0; k < kConv; ++k) l += (g >= B.end[k]) ? 1 : 0;
  return l;
}

// grad[g] = sum over splits of the partial weight gradients (bias: the
// ones-row column, index ld - 1).
__global__ void k_grad_reduce(int P, Blocks B, float* __restrict__ grad) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= P) return;
  const int l = block_of(B, g);
  int c, k;
  if (g < B.b_off[l]) {
    c = (g - B.w_off[l]) / B.K[l];
    k = (g - B.w_off[l]) % B.K[l];
  } else {
    c = g - B.b_off[l];
    k = B.ld[l] - 1;
  }
  const size_t stride = (size_t)B.Co[l] * B.ld[l];
  const float* p = B.part[l] + (size_t)c * B.ld[l] + k;
  float s = 0.f;
  for (int z = 0; z < B.S[l]; ++z) s += p[z * stride];
  grad[g] = s;
}

__device__ __forceinline__ void write_shadow(const Blocks& B, int g, int l, float w) {
  if (g >= B.b_off[l]) return;   // biases are read in FP32 by the GEMM epilogue
  const int c = (g - B.w_off[l]) / B.K[l];
  const int k = (g - B.w_off[l]) % B.K[l];
  const uint16_t b = bf16_bits(w);
  B.wbf[l][(size_t)c * B.Kp[l] + k] = b;
  B.wt[l][(size_t)k * B.Cp[l] + c] = b;
}

// Adam step on the FP32 master parameters, then the BF16 shadows.
__global__ void k_adam(int P, Blocks B, const float* __restrict__ grad, float* __restrict__ w, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= P) return;
  const float gr = grad[g];
  const float mm = b1 * m[g] + (1.f - b1) * gr;
  const float vv = b2 * v[g] + (1.f - b2) * gr * gr;
  m[g] = mm;
  v[g] = vv;
  const float x = w[g] - lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
  w[g] = x;
  write_shadow(B, g, block_of(B, g), x);
}

// Shadows from the master parameters (after init / load); moments cleared.
__global__ void k_refresh(int P, Blocks B, const float* __restrict__ w, float* __restrict__ m, float* __restrict__ v) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= P) return;
  m[g] = 0.f;
  v[g] = 0.f;
  write_shadow(B, g, block_of(B, g), w[g]);
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// He-uniform weights U(-sqrt(6 / fan_in), +) for the convolutions, a small
// U(-0.1 sqrt(3 / 512), +) for the linear layer (initial proposals near the
// identity), zero biases.
__global__ void k_cnn_init(int P, Blocks B, uint64_t seed, float* __restrict__ w) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= P) return;
  const int l = block_of(B, g);
  float x = 0.f;
  if (g < B.b_off[l]) {
    const double u = (double)(splitmix64(seed * 0x100000001B3ull + (uint64_t)g) >> 11) * 0x1.0p-53;
    const double a = l < kConv ? sqrt(6.0 / B.K[l]) : 0.1 * sqrt(3.0 / B.K[l]);
    x = (float)((2.0 * u - 1.0) * a);
  }
  w[g] = x;
}

// T0 = [Exp(0.25 p[0:3]), 3 p[3:6]] in float64.
__global__ void k_pred_pose(int n, const float* __restrict__ pred, double* __restrict__ T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* p = pred + (size_t)i * kFcOut;
  const double w[3] = {RIMG_CNN_OMEGA_SCALE * (double)p[0], RIMG_CNN_OMEGA_SCALE * (double)p[1],
                       RIMG_CNN_OMEGA_SCALE * (double)p[2]};
  double R[9];
  so3_exp_d(w, R);
  double* o = T + 16 * (size_t)i;
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) o[4 * r + c] = R[3 * r + c];
    o[4 * r + 3] = RIMG_CNN_T_SCALE * (double)p[3 + r];
  }
  o[12] = 0.0; o[13] = 0.0; o[14] = 0.0; o[15] = 1.0;
}

// ---------------------------------------------------------------------------
// Host orchestration

inline unsigned blocks_for(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

Blocks make_blocks(unsigned char* state, const unsigned char* ws, const WsLayout* W) {
  const ParamLayout P = param_layout();
  const StateLayout S = state_layout();
  Blocks B{};
  for (int l = 0; l <= kConv; ++l) {
    const bool fc = l == kConv;
    B.w_off[l] = (int)P.w[l];
    B.b_off[l] = (int)P.b[l];
    B.end[l] = (int)(P.b[l] + (fc ? kFcOut : kGeo[l].Co));
    B.K[l] = fc ? kFcIn : kGeo[l].K;
    B.Kp[l] = fc ? kFcIn : kGeo[l].Kp;
    B.Cp[l] = fc ? 64 : kGeo[l].Cp;
    B.Co[l] = fc ? kFcOut : kGeo[l].Co;
    B.ld[l] = (fc ? kFcIn : kGeo[l].Kp) + 1;
    B.wbf[l] = reinterpret_cast<uint16_t*>(state + S.wbf[l]);
    B.wt[l] = reinterpret_cast<uint16_t*>(state + S.wt[l]);
    if (W) {
      B.part[l] = reinterpret_cast<const float*>(ws + W->part[l]);
      B.S[l] = W->splits[l];
    }
  }
  return B;
}

struct Net {
  const unsigned char* state;
  unsigned char* ws;
  WsLayout W;
  StateLayout S;
  ParamLayout P;
  int n;
  int* err;
  cudaStream_t st;
  template <class T>
  T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
  template <class T>
  const T* st_at(size_t off) const { return reinterpret_cast<const T*>(state + off); }
};

cudaError_t forward(const Net& N, int H, int W, int stride, const float* src, const float* dst, const int32_t* index) {
  const int n = N.n;
  k_cnn_input<<<blocks_for((size_t)n * kInH * kInW, 256), 256, 0, N.st>>>(
      n, H, W, stride, src, dst, index, N.at<__nv_bfloat162>(N.W.x0));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const uint16_t* x = N.at<uint16_t>(N.W.x0);
  const float* master = N.st_at<float>(N.S.master);
  for (int l = 0; l < kConv; ++l) {
    const ConvGeo& g = kGeo[l];
    const size_t M = (size_t)n * g.Ho * g.Wo;
    uint16_t* col = N.at<uint16_t>(N.W.col[l]);
    k_im2col<<<blocks_for(M * (g.Kp / 8), 256), 256, 0, N.st>>>(n, g, x, col);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_gemm_bf16((int)M, g.Co, g.Kp, col, g.Kp, N.st_at<uint16_t>(N.S.wbf[l]), g.Kp, N.at<float>(N.W.y[l]),
                         g.Co, N.at<uint16_t>(N.W.act[l]), master + N.P.b[l], 1, 1, N.err, N.st);
    if (e != cudaSuccess) return e;
    x = N.at<uint16_t>(N.W.act[l]);
  }
  // linear layer on the flattened (w, c) activations of conv5: [n][512]
  return launch_gemm_bf16(n, kFcOut, kFcIn, x, kFcIn, N.st_at<uint16_t>(N.S.wbf[kConv]), kFcIn,
                          N.at<float>(N.W.pred), kFcOut, nullptr, master + N.P.b[kConv], 0, 1, N.err, N.st);
}

cudaError_t backward(const Net& N, const double* T_label, const int32_t* index, double* loss, float* grad) {
  const int n = N.n;
  const int n64 = (int)r64(n);
  cudaError_t e;
  k_cnn_loss<<<1, 256, 0, N.st>>>(n, n64, N.at<float>(N.W.pred), T_label, index, loss, N.at<uint16_t>(N.W.dp),
                                  N.at<uint16_t>(N.W.dpt));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const dim3 tb(32, 8);
  // linear layer: dW = dp^T X6 (+ bias column), dX6 = dp W
  {
    const uint16_t* x6 = N.at<uint16_t>(N.W.act[kConv - 1]);
    uint16_t* x6t = N.at<uint16_t>(N.W.x6t);
    k_transpose_bf16<<<dim3(n64 / 32, (kFcIn + 1 + 31) / 32), tb, 0, N.st>>>(n, kFcIn, x6, kFcIn, x6t, n64, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_gemm_bf16(kFcOut, kFcIn + 1, n64, N.at<uint16_t>(N.W.dpt), n64, x6t, n64,
                         N.at<float>(N.W.part[kConv]), kFcIn + 1, nullptr, nullptr, 0, N.W.splits[kConv], N.err,
                         N.st);
    if (e != cudaSuccess) return e;
    e = launch_gemm_bf16(n, kFcIn, 64, N.at<uint16_t>(N.W.dp), 64, N.st_at<uint16_t>(N.S.wt[kConv]), 64,
                         N.at<float>(N.W.dx6), kFcIn, nullptr, nullptr, 0, 1, N.err, N.st);
    if (e != cudaSuccess) return e;
  }
  const float* dy = N.at<float>(N.W.dx6);
  for (int l = kConv - 1; l >= 0; --l) {
    const ConvGeo& g = kGeo[l];
    const size_t M = (size_t)n * g.Ho * g.Wo;
    const int M64 = (int)r64(M);
    uint16_t* dz = N.at<uint16_t>(N.W.dz[l]);
    uint16_t* dzt = N.at<uint16_t>(N.W.dzt[l]);
    uint16_t* colt = N.at<uint16_t>(N.W.colt[l]);
    k_relu_bwd<<<blocks_for(M * (g.Cp / 8), 256), 256, 0, N.st>>>(M, g.Co, g.Cp, dy, N.at<float>(N.W.y[l]), dz);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_transpose_bf16<<<dim3(M64 / 32, (g.Co + 31) / 32), tb, 0, N.st>>>((int)M, g.Co, dz, g.Cp, dzt, M64, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_transpose_bf16<<<dim3(M64 / 32, (g.Kp + 1 + 31) / 32), tb, 0, N.st>>>((int)M, g.Kp, N.at<uint16_t>(N.W.col[l]),
                                                                             g.Kp, colt, M64, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_gemm_bf16(g.Co, g.Kp + 1, M64, dzt, M64, colt, M64, N.at<float>(N.W.part[l]), g.Kp + 1, nullptr,
                         nullptr, 0, N.W.splits[l], N.err, N.st);
    if (e != cudaSuccess) return e;
    if (l == 0) break;
    float* dcol = N.at<float>(N.W.dcol[l]);
    e = launch_gemm_bf16((int)M, g.K, g.Cp, dz, g.Cp, N.st_at<uint16_t>(N.S.wt[l]), g.Cp, dcol, g.Kp, nullptr,
                         nullptr, 0, 1, N.err, N.st);
    if (e != cudaSuccess) return e;
    float* dx = N.at<float>(N.W.dx[l]);
    k_col2im<<<blocks_for((size_t)n * g.Hi * g.Wi * g.Ci, 256), 256, 0, N.st>>>(n, g, dcol, dx);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dy = dx;
  }
  Blocks B = make_blocks(const_cast<unsigned char*>(N.state), N.ws, &N.W);
  k_grad_reduce<<<blocks_for(N.P.total, 256), 256, 0, N.st>>>((int)N.P.total, B, grad);
  return cudaGetLastError();
}

int check_state(const void* state, size_t state_bytes) {
  if (!state) return RIMG_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(state) % kAlign || state_bytes < state_layout().end) return RIMG_ERR_WORKSPACE;
  return RIMG_OK;
}

int check_batch(int n, int H, int W, int stride, const float* src, const float* dst) {
  if (n < 0 || n > RIMG_CNN_MAX_BATCH || stride < 1) return RIMG_ERR_INVALID_ARG;
  if (n > 0 && (!src || !dst)) return RIMG_ERR_INVALID_ARG;
  if (H != kInH * stride || W != kInW * stride) return RIMG_ERR_SIZE;
  return RIMG_OK;
}

int check_ws(int n, const void* ws, size_t ws_bytes) {
  if (!ws) return RIMG_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % kAlign || ws_bytes < ws_layout(n).end) return RIMG_ERR_WORKSPACE;
  return RIMG_OK;
}

Net make_net(const void* state, int n, void* ws, int* err, void* stream) {
  Net N;
  N.state = static_cast<const unsigned char*>(state);
  N.ws = static_cast<unsigned char*>(ws);
  N.W = ws_layout(n);
  N.S = state_layout();
  N.P = param_layout();
  N.n = n;
  N.err = err;
  N.st = static_cast<cudaStream_t>(stream);
  return N;
}

#define RIMG_CNN_TRY(expr, where)                                   \
  do {                                                              \
    cudaError_t e_ = (expr);                                        \
    if (e_ != cudaSuccess) return record_cuda_error(e_, where);     \
  } while (0)

}  // namespace
}  // namespace rimg

using namespace rimg;

extern "C" {

int rimg_cnn_param_count(size_t* n_params) {
  if (!n_params) return RIMG_ERR_INVALID_ARG;
  *n_params = param_layout().total;
  return RIMG_OK;
}

int rimg_cnn_state_bytes(size_t* bytes) {
  if (!bytes) return RIMG_ERR_INVALID_ARG;
  *bytes = state_layout().end;
  return RIMG_OK;
}

int rimg_cnn_workspace_bytes(int n, size_t* bytes) {
  if (!bytes || n < 0 || n > RIMG_CNN_MAX_BATCH) return RIMG_ERR_INVALID_ARG;
  *bytes = ws_layout(std::max(n, 1)).end;
  return RIMG_OK;
}

int rimg_cnn_init(void* state, size_t state_bytes, uint64_t seed, void* stream) {
  int rc = check_state(state, state_bytes);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const StateLayout S = state_layout();
  const int P = (int)param_layout().total;
  unsigned char* s = static_cast<unsigned char*>(state);
  RIMG_CNN_TRY(cudaMemsetAsync(s + S.wbf[0], 0, S.end - S.wbf[0], st), "cnn init memset");
  Blocks B = make_blocks(s, nullptr, nullptr);
  float* w = reinterpret_cast<float*>(s + S.master);
  k_cnn_init<<<blocks_for(P, 256), 256, 0, st>>>(P, B, seed, w);
  RIMG_CNN_TRY(cudaGetLastError(), "cnn init kernel");
  k_refresh<<<blocks_for(P, 256), 256, 0, st>>>(P, B, w, reinterpret_cast<float*>(s + S.m),
                                                reinterpret_cast<float*>(s + S.v));
  RIMG_CNN_TRY(cudaGetLastError(), "cnn refresh kernel");
  return RIMG_OK;
}

int rimg_cnn_load(void* state, size_t state_bytes, const float* params, void* stream) {
  int rc = check_state(state, state_bytes);
  if (rc) return rc;
  if (!params) return RIMG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const StateLayout S = state_layout();
  const int P = (int)param_layout().total;
  unsigned char* s = static_cast<unsigned char*>(state);
  float* w = reinterpret_cast<float*>(s + S.master);
  if (params != w) RIMG_CNN_TRY(cudaMemcpyAsync(w, params, 4 * (size_t)P, cudaMemcpyDeviceToDevice, st), "cnn load");
  RIMG_CNN_TRY(cudaMemsetAsync(s + S.wbf[0], 0, S.end - S.wbf[0], st), "cnn load memset");
  Blocks B = make_blocks(s, nullptr, nullptr);
  k_refresh<<<blocks_for(P, 256), 256, 0, st>>>(P, B, w, reinterpret_cast<float*>(s + S.m),
                                                reinterpret_cast<float*>(s + S.v));
  RIMG_CNN_TRY(cudaGetLastError(), "cnn refresh kernel");
  return RIMG_OK;
}

int rimg_propose(const void* state, int n, int H, int W, int stride, const float* src_range, const float* dst_range,
                 const int32_t* index, float* pred, double* T_out, int* err, void* workspace, size_t workspace_bytes,
                 void* stream) {
  int rc = check_state(state, ~(size_t)0);
  if (rc) return rc;
  if ((rc = check_batch(n, H, W, stride, src_range, dst_range))) return rc;
  if (n == 0) return RIMG_OK;
  if ((rc = check_ws(n, workspace, workspace_bytes))) return rc;
  Net N = make_net(state, n, workspace, err, stream);
  RIMG_CNN_TRY(forward(N, H, W, stride, src_range, dst_range, index), "cnn forward");
  if (pred)
    RIMG_CNN_TRY(cudaMemcpyAsync(pred, N.at<float>(N.W.pred), 4 * (size_t)n * kFcOut, cudaMemcpyDeviceToDevice, N.st),
                 "cnn pred copy");
  if (T_out) {
    k_pred_pose<<<blocks_for(n, 128), 128, 0, N.st>>>(n, N.at<float>(N.W.pred), T_out);
    RIMG_CNN_TRY(cudaGetLastError(), "cnn pose kernel");
  }
  return RIMG_OK;
}

int rimg_cnn_grad(const void* state, int n, int H, int W, int stride, const float* src_range, const float* dst_range,
                  const int32_t* index, const double* T_label, double* loss, float* grad, float* pred, int* err,
                  void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_state(state, ~(size_t)0);
  if (rc) return rc;
  if ((rc = check_batch(n, H, W, stride, src_range, dst_range))) return rc;
  if (n == 0 || !T_label || !grad) return RIMG_ERR_INVALID_ARG;
  if ((rc = check_ws(n, workspace, workspace_bytes))) return rc;
  Net N = make_net(state, n, workspace, err, stream);
  RIMG_CNN_TRY(forward(N, H, W, stride, src_range, dst_range, index), "cnn forward");
  RIMG_CNN_TRY(backward(N, T_label, index, loss ? loss : N.at<double>(N.W.loss), grad), "cnn backward");
  if (pred)
    RIMG_CNN_TRY(cudaMemcpyAsync(pred, N.at<float>(N.W.pred), 4 * (size_t)n * kFcOut, cudaMemcpyDeviceToDevice, N.st),
                 "cnn pred copy");
  return RIMG_OK;
}

int rimg_cnn_train_step(void* state, size_t state_bytes, int n, int H, int W, int stride, const float* src_range,
                        const float* dst_range, const int32_t* index, const double* T_label, const rimg_adam* opt,
                        int step, double* loss, int* err, void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_state(state, state_bytes);
  if (rc) return rc;
  if ((rc = check_batch(n, H, W, stride, src_range, dst_range))) return rc;
  if (n == 0 || !T_label || !opt || step < 1) return RIMG_ERR_INVALID_ARG;
  if (!(opt->lr >= 0.f) || !(opt->beta1 >= 0.f && opt->beta1 < 1.f) || !(opt->beta2 >= 0.f && opt->beta2 < 1.f) ||
      !(opt->eps > 0.f))
    return RIMG_ERR_INVALID_ARG;
  if ((rc = check_ws(n, workspace, workspace_bytes))) return rc;
  Net N = make_net(state, n, workspace, err, stream);
  float* grad = N.at<float>(N.W.grad);
  RIMG_CNN_TRY(forward(N, H, W, stride, src_range, dst_range, index), "cnn forward");
  RIMG_CNN_TRY(backward(N, T_label, index, loss ? loss : N.at<double>(N.W.loss), grad), "cnn backward");
  unsigned char* s = static_cast<unsigned char*>(state);
  Blocks B = make_blocks(s, nullptr, nullptr);
  const int P = (int)N.P.total;
  const float bc1 = (float)(1.0 - std::pow((double)opt->beta1, step));
  const float bc2 = (float)(1.0 - std::pow((double)opt->beta2, step));
  k_adam<<<blocks_for(P, 256), 256, 0, N.st>>>(P, B, grad, reinterpret_cast<float*>(s + N.S.master),
                                               reinterpret_cast<float*>(s + N.S.m),
                                               reinterpret_cast<float*>(s + N.S.v), opt->lr, opt->beta1, opt->beta2,
                                               opt->eps, bc1, bc2);
  RIMG_CNN_TRY(cudaGetLastError(), "cnn adam kernel");
  return RIMG_OK;
}

}  // extern "C"
