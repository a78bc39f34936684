// The fused projective-association Gauss-Newton step (Section 4.1, Eq. 5-7):
// per source pixel unproject -> transform -> project -> gather the target
// plane -> residual, pseudo-Huber weight, Jacobian -> 29 reduced terms.  Each
// thread sums a few chunks plainly in FP32; a warp reduce-scatter then hands
// lane l the warp's component l, which it adds to its running sum with Kahan
// compensation; block and one-pass grid reduction follow (last-block-done
// counter, no spinning; the last block of a pair sums the block records in
// FP64).  k_solve then solves the 6x6 system in FP64 and composes the SE(3)
// update, one warp per pair.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include <cooperative_groups.h>

#include "rimg_device.cuh"

namespace rimg {

namespace {

// 1/d in FP64 by Newton-Raphson, x <- x (2 - d x), from the FP32 reciprocal:
// each step squares the relative error (~1e-7 -> ~1e-14 -> below 1 ulp), a
// short chain of multiply-adds instead of a full IEEE division.  d > 0 and
// within FP32 range here (pivots of a 6x6 normal-equation system).
__device__ __forceinline__ double recip_newton(double d) {
  double x = (double)__frcp_rn((float)d);
  x = x * fma(-d, x, 2.0);
  x = x * fma(-d, x, 2.0);
  return x;
}

constexpr unsigned kFullMask = 0xffffffffu;

// Index of H_ij (i <= j) in the reduced record: the 21 upper-triangle
// entries of J^T W J row-major (row i starts at i (11 - i) / 2).
__device__ __forceinline__ int upper_index(int i, int j) { return i * (11 - i) / 2 + j; }

// On this GPU every FP64 warp instruction occupies the sub-partition's FP64
// pipe for a fixed number of cycles whatever the number of active lanes, so
// the per-pair Gauss-Newton update is spread over the 32 lanes of one warp:
// one matrix entry per lane in the solve, one pose entry per lane in the
// update.  All lanes of the warp call these together with the same
// arguments; results are the same in every lane.

// 2^-e for the binary exponent e of x > 0: a power of two, so multiplying by
// it is exact (exponent field clamped to the normal range).
__device__ __forceinline__ double pow2_neg_exponent(double x) {
  const int E = min(max((__double2hiint(x) >> 20) & 0x7ff, 1), 2045);
  return __hiloint2double((2046 - E) << 20, 0);
}
// The significand of x > 0 as a number in [1, 2): x 2^-e, exactly.
__device__ __forceinline__ double significand_of(double x) {
  return __hiloint2double((__double2hiint(x) & 0x000fffff) | 0x3ff00000, __double2loint(x));
}

// Warp-cooperative FP64 solve of H x = -g (H from the packed upper triangle
// t[0..20], g = t[21..26]) by right-looking symmetric Gaussian elimination,
// i.e. LDL^T: lanes 0..20 hold the lower triangle (lane i (i + 1) / 2 + j for
// j <= i), lanes 21..26 the right-hand side.  Step k takes pivot d_k and
// replaces every entry below and right of it by (d_k a_ij - a_ik a_jk) 2^-e_k
// (e_k the exponent of d_k): the standard update a_ij - a_ik a_jk / d_k times
// s_k = d_k 2^-e_k in [1, 2), with no reciprocal on the step-to-step chain.
// The trailing block, right-hand side included, carries the product S_k of
// the earlier s, so the LDL^T pivot is d_k / S_k; each row of the final
// system U x = c (row k: column k of the stored lower triangle, pivot d_k,
// c_k) carries one common factor, which cancels in the column-oriented back
// substitution in lanes 21..26.  False if a pivot d_k / S_k <= 1e-12 trace(H).
__device__ bool warp_solve6(const double* t, int lane, double (&x)[6]) {
  int i, j;   // the lane's entry; j = 6 marks the right-hand side
  if (lane < 21) {
    i = 0;
    while ((i + 1) * (i + 2) / 2 <= lane) ++i;
    j = lane - i * (i + 1) / 2;
  } else {
    i = lane - 21;
    j = 6;
  }
  const bool rhs = lane >= 21 && lane < 27;
  const bool live = lane < 27;
  double v = 0.0;
  if (lane < 21) v = t[upper_index(j, i)];
  else if (rhs) v = -t[21 + i];
  const int base_a = live ? i * (i + 1) / 2 : 0;              // lane of entry (i, 0)
  const int base_b = (lane < 21) ? j * (j + 1) / 2 : 21;      // lane of (j, 0), or of c_0
  double dk = 1.0, sk = 1.0;                                  // lane k < 6: d_k and s_k
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double d = __shfl_sync(kFullMask, v, k * (k + 3) / 2);
    const double sc = pow2_neg_exponent(d);
    if (lane == k) {
      dk = d;
      sk = significand_of(d);
    }
    const double aik = __shfl_sync(kFullMask, v, (base_a + k) & 31);
    const double ajk = __shfl_sync(kFullMask, v, (base_b + k) & 31);
    if (live && i > k && j > k) v = fma(d, v, -(aik * ajk)) * sc;
  }
  // S_k = s_0 ... s_{k-1} in lane k (exclusive prefix product), then the pivot test
  double pre = sk;
#pragma unroll
  for (int off = 1; off < 8; off <<= 1) {
    const double o = __shfl_up_sync(kFullMask, pre, off);
    if (lane >= off) pre *= o;
  }
  double Sk = __shfl_up_sync(kFullMask, pre, 1);
  if (lane == 0) Sk = 1.0;
  double tr = 0.0;
#pragma unroll
  for (int q = 0; q < 6; ++q) tr += t[upper_index(q, q)];
  const bool bad = lane < 6 && !(dk > (1e-12 * tr) * Sk);
  if (__any_sync(kFullMask, bad)) return false;
  const double inv = recip_newton(dk);                        // 1 / d_k in lane k
#pragma unroll
  for (int k = 5; k >= 0; --k) {
    const double xk = __shfl_sync(kFullMask, v, 21 + k) * __shfl_sync(kFullMask, inv, k);
    x[k] = xk;
    const double u = __shfl_sync(kFullMask, v, (k * (k + 1) / 2 + (rhs ? i : 0)) & 31);
    if (rhs && i < k) v = fma(-u, xk, v);
  }
  return true;
}

__device__ __forceinline__ double pick3(int s, double a, double b, double c) { return s == 0 ? a : (s == 1 ? b : c); }

// Warp-cooperative T <- Exp(xi) T for xi = (omega, tau) and the 3x4 pose T
// (row-major; rewritten by lanes 0..11, one entry each; Tf, if given,
// receives its FP32 copy).  Rodrigues: R = I + A K + B K^2, V = I + B K + C K^2
// with K = [omega]_x, K^2 = omega omega^T - |omega|^2 I and A = sin(t)/t,
// B = (1 - cos t)/t^2, C = (t - sin t)/t^3.  For |omega| < 0.5 rad (every
// Gauss-Newton step in practice) lane s = 0, 1, 2 (mod 3) evaluates the
// Taylor series of A, B, C in t^2 to degree 6 (coefficients (-1)^n /
// (2n + 1 + s)!, truncation < 1e-16 relative), otherwise sincos.  Lane
// 4r + c forms row r of R times column c of T while lane 12 + r forms row r of
// V times tau, which lane 4r + 3 then adds to the new translation.
__device__ void warp_se3_update(double* T, const double (&xi)[6], int lane, float* Tf) {
  const double wx = xi[0], wy = xi[1], wz = xi[2];
  const double th2 = fma(wz, wz, fma(wy, wy, wx * wx));
  double A, B, C;
  if (th2 < 0.25) {
    const int s = lane % 3;
    double p = pick3(s, 1.0 / 6227020800.0, 1.0 / 87178291200.0, 1.0 / 1307674368000.0);
    p = fma(p, th2, pick3(s, -1.0 / 39916800.0, -1.0 / 479001600.0, -1.0 / 6227020800.0));
    p = fma(p, th2, pick3(s, 1.0 / 362880.0, 1.0 / 3628800.0, 1.0 / 39916800.0));
    p = fma(p, th2, pick3(s, -1.0 / 5040.0, -1.0 / 40320.0, -1.0 / 362880.0));
    p = fma(p, th2, pick3(s, 1.0 / 120.0, 1.0 / 720.0, 1.0 / 5040.0));
    p = fma(p, th2, pick3(s, -1.0 / 6.0, -1.0 / 24.0, -1.0 / 120.0));
    p = fma(p, th2, pick3(s, 1.0, 0.5, 1.0 / 6.0));
    A = __shfl_sync(kFullMask, p, 0);
    B = __shfl_sync(kFullMask, p, 1);
    C = __shfl_sync(kFullMask, p, 2);
  } else {
    const double th = sqrt(th2);
    double sn, cs;
    sincos(th, &sn, &cs);
    A = sn / th;
    B = (1.0 - cs) / th2;
    C = (th - sn) / (th2 * th);
  }
  const bool rot = lane < 12;
  const int r = rot ? lane >> 2 : (lane < 15 ? lane - 12 : 0), c = lane & 3;
  const double al = rot ? A : B, be = rot ? B : C;
  const double wr = pick3(r, wx, wy, wz);
  // row r of K: (0, -wz, wy), (wz, 0, -wx), (-wy, wx, 0)
  const double k0 = pick3(r, 0.0, wz, -wy), k1 = pick3(r, -wz, 0.0, wx), k2 = pick3(r, wy, -wx, 0.0);
  const double q0 = fma(wr, wx, r == 0 ? -th2 : 0.0);
  const double q1 = fma(wr, wy, r == 1 ? -th2 : 0.0);
  const double q2 = fma(wr, wz, r == 2 ? -th2 : 0.0);
  const double M0 = fma(al, k0, fma(be, q0, r == 0 ? 1.0 : 0.0));
  const double M1 = fma(al, k1, fma(be, q1, r == 1 ? 1.0 : 0.0));
  const double M2 = fma(al, k2, fma(be, q2, r == 2 ? 1.0 : 0.0));
  const double y0 = rot ? T[c] : xi[3], y1 = rot ? T[4 + c] : xi[4], y2 = rot ? T[8 + c] : xi[5];
  double acc = fma(M2, y2, fma(M1, y1, M0 * y0));
  const double vt = __shfl_sync(kFullMask, acc, 12 + r);
  if (rot && c == 3) acc += vt;
  __syncwarp();
  if (rot) {
    T[lane] = acc;
    if (Tf) Tf[lane] = (float)acc;
  }
  __syncwarp();
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
// lane index f = 2 * pair + (0 for .x, 1 for .y).  Pairs 0..11 are updated by
// packed FP32x2 FMAs whose operands are register pairs that arise without
// moves -- (a0, a1) and (a2, e) as computed, (nx, ny) as loaded -- plus the
// swaps (ny, nx) and (e, a2) and the broadcast (nz, nz); pairs 12 and 13 hold
// scalar FMAs, pair 14 the count.  kFlat maps the output order (21
// upper-triangle J^T W J entries row-major, 6 J^T W e, sum w e^2, count) to
// lanes.
constexpr int kPairs = 15;
__constant__ int kFlat[kRed] = {0,  24, 2,  4,  6,  18,  // H00..H05
                                1,  9,  7,  5,  19,      // H11..H15
                                10, 12, 14, 20,          // H22..H25
                                16, 25, 22,              // H33..H35
                                17, 23,                  // H44, H45
                                26,                      // H55
                                8,  3,  27, 15, 13, 21,  // g0..g5
                                11, 28};                 // sum w e^2, count

// Point-to-plane terms of one association: residual e = n.x - d, IRLS weight,
// J = [a, n] with a = x cross n; adds w J J^T (upper triangle), w e J, w e^2
// and the count into t.  A zero plane (no association) contributes exactly
// nothing.
__device__ __forceinline__ void accumulate_px(float2 (&t)[kPairs], float x, float y, float z, float4 pl,
                                              float inv_delta) {
  const float nx = pl.x, ny = pl.y, nz = pl.z;
  const float e = fmaf(nx, x, fmaf(ny, y, fmaf(nz, z, -pl.w)));
  // no branch, so that the four pixels of a chunk stay one block; without a
  // robust kernel inv_delta = 0, q = 0 and w = rsqrt(1) = 1 exactly
  const float q = e * inv_delta;
  const float w = rsqrtf(fmaf(q, q, 1.f));
  const float a0 = fmaf(y, nz, -z * ny), a1 = fmaf(z, nx, -x * nz), a2 = fmaf(x, ny, -y * nx);
  const float2 P1 = f2(a0, a1), P2 = f2(a2, e), N1 = f2(nx, ny);
  const float2 M1 = f2(ny, nx), S2 = f2(e, a2), Z2 = f2(nz, nz);
  const float2 W2 = f2(w, w);
  const float2 UP1 = mul2(W2, P1), UP2 = mul2(W2, P2), UN1 = mul2(W2, N1);
  t[0] = fma2(UP1, P1, t[0]);                          // H00 H11
  t[1] = fma2(UP1, P2, t[1]);                          // H02 g1
  t[2] = fma2(UP1, N1, t[2]);                          // H03 H14
  t[3] = fma2(UP1, M1, t[3]);                          // H04 H13
  t[4] = fma2(UP1, S2, t[4]);                          // g0 H12
  t[5] = fma2(UP2, P2, t[5]);                          // H22, w e^2
  t[6] = fma2(UP2, N1, t[6]);                          // H23 g4
  t[7] = fma2(UP2, M1, t[7]);                          // H24 g3
  t[8] = fma2(UN1, N1, t[8]);                          // H33 H44
  t[9] = fma2(UP1, Z2, t[9]);                          // H05 H15
  t[10] = fma2(UP2, Z2, t[10]);                        // H25 g5
  t[11] = fma2(UN1, Z2, t[11]);                        // H35 H45
  t[12].x = fmaf(UP1.x, a1, t[12].x);                  // H01
  t[12].y = fmaf(UN1.x, ny, t[12].y);                  // H34
  t[13].x = fmaf(w * nz, nz, t[13].x);                 // H55
  t[13].y = fmaf(UP2.x, e, t[13].y);                   // g2
  // an association counts when its plane is not the all-zero invalid plane
  // (stored as +0.f; a unit normal has a non-zero component)
  t[14].x += (__float_as_uint(nx) | __float_as_uint(ny) | __float_as_uint(nz)) ? 1.f : 0.f;
}

// Depth of the per-thread staging ring: a chunk's source ranges are fetched
// kRing chunks ahead of its projection, and its target planes are gathered
// kRing - 1 chunks ahead of its accumulation.
#ifndef RIMG_RING
#define RIMG_RING 2
#endif
constexpr int kRing = RIMG_RING;

// Shared memory of one block (dynamic).  Each thread owns column `tid` of the
// staging arrays: for each ring slot, the source ranges of one 4-pixel chunk
// and the gathered target planes.  The chunk's transformed points stay in
// registers.
template <int THREADS>
struct IcpSmem {
  float4 src[kRing][THREADS];
  float4 planes[kRing][4][THREADS];
  float4 T4[3];                            // pose rows (R | t) in FP32
  float red[THREADS / 32][2 * kPairs];     // per-warp sums
  double tot[32];
  int last;
};

// Per-row constants of the folded unprojection and transform (see issue in
// icp_block_terms), one table per block after its IcpSmem: for row v_begin + i
// of the block, entries 3i .. 3i + 2 hold A_v, B_v, C_v with the translation
// t_x, t_y, t_z in .w.  Blocks cover at most kMaxBlockRows rows.
constexpr int kMaxBlockRows = 1024;
template <int THREADS>
__host__ __device__ constexpr size_t row_table_offset() {
  return (sizeof(IcpSmem<THREADS>) + 15) & ~size_t(15);
}
template <int THREADS>
__host__ __device__ constexpr size_t icp_smem_bytes(int rows) {
  return row_table_offset<THREADS>() + sizeof(float4) * 3 * (size_t)rows;
}
template <int THREADS>
__device__ __forceinline__ float4* row_table(IcpSmem<THREADS>& sm) {
  return reinterpret_cast<float4*>(reinterpret_cast<char*>(&sm) + row_table_offset<THREADS>());
}

// Fills rows i = first, first + step, ... < nrows of the row table for rows
// [v_begin, v_begin + nrows) of level S at the FP32 pose rows T0, T1, T2
// (R | t).  With the row's cos/sin of elevation and azimuth offset and the
// rotation columns R0, R1, R2,
//   R p = r (cos u A + sin u B + C),  A = cos(phi) (cos(th) R0 + sin(th) R1),
//   B = cos(phi) (cos(th) R1 - sin(th) R0),  C = sin(phi) R2.
// The block is synchronised before the table is read.
__device__ __forceinline__ void fill_row_table(const DevLevel& S, float4* rt, float4 T0, float4 T1, float4 T2,
                                               int v_begin, int nrows, int first, int step) {
  for (int i = first; i < nrows; i += step) {
    const float4 rw = __ldg(S.rows + v_begin + i);
    const float q0 = rw.x * rw.z, q1 = rw.x * rw.w;
    rt[3 * i] = make_float4(fmaf(q0, T0.x, q1 * T0.y), fmaf(q0, T1.x, q1 * T1.y), fmaf(q0, T2.x, q1 * T2.y), T0.w);
    rt[3 * i + 1] = make_float4(fmaf(q0, T0.y, -q1 * T0.x), fmaf(q0, T1.y, -q1 * T1.x), fmaf(q0, T2.y, -q1 * T2.x),
                                T1.w);
    rt[3 * i + 2] = make_float4(rw.y * T0.z, rw.y * T1.z, rw.y * T2.z, T2.w);
  }
}

// The row table from the pose in sm.T4, by all threads of the block (the
// caller synchronised after writing sm.T4) or by one warp (lane = its lane,
// after the warp wrote sm.T4; step 32).
template <int THREADS>
__device__ __forceinline__ void icp_row_table(const DevLevel& S, IcpSmem<THREADS>& sm, int v_begin, int nrows,
                                              int first, int step) {
  fill_row_table(S, row_table(sm), sm.T4[0], sm.T4[1], sm.T4[2], v_begin, nrows, first, step);
}

// Chunks summed plainly per thread between two compensated warp steps.
#ifndef RIMG_WARP_FLUSH
#define RIMG_WARP_FLUSH 16
#endif
constexpr int kWarpFlush = RIMG_WARP_FLUSH;
static_assert(kWarpFlush >= 1, "at least one chunk between warp steps");

// Reduce-scatter of the 30 lanes of t (15 float2, padded to 16) across the
// warp: lane l receives the warp's sum of component l (component f is lane
// f % 2 of float2 f / 2).  Recursive halving: at offset o each lane keeps the
// half of its remaining values selected by bit o of its lane id and adds the
// partner's copy of that half.
__device__ __forceinline__ float warp_scatter_sum(const float2 (&t)[kPairs], int lane) {
  float2 v[16];
#pragma unroll
  for (int i = 0; i < kPairs; ++i) v[i] = t[i];
  v[15] = f2(0.f, 0.f);
#pragma unroll
  for (int half = 8; half >= 1; half >>= 1) {
    const bool hi = (lane & (2 * half)) != 0;      // offsets 16, 8, 4, 2
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const float2 keep = hi ? v[half + j] : v[j];
      const float2 send = hi ? v[j] : v[half + j];
      const float2 recv = f2(__shfl_xor_sync(0xffffffffu, send.x, 2 * half),
                             __shfl_xor_sync(0xffffffffu, send.y, 2 * half));
      v[j] = add2(keep, recv);
    }
  }
  const bool odd = lane & 1;
  const float keep = odd ? v[0].y : v[0].x;
  const float send = odd ? v[0].x : v[0].y;
  return keep + __shfl_xor_sync(0xffffffffu, send, 1);
}

#ifndef RIMG_ICP_THREADS_PER_SM
#define RIMG_ICP_THREADS_PER_SM 512
#endif
// One block's share of a step: the rows [v_begin, v_end) of pair `pair` at
// the pose in sm.T4, whose row table (icp_row_table) the caller has filled.
// On return (after a block barrier) sm.red[w][l] holds warp w's component l
// of the 29 sums (lane order, see kFlat).
// ROWSTRIDE 1: the thread stride is a whole number of rows (chunks per row
// divide THREADS), so a cursor advances by rows only; ROWSTRIDE 2: the
// stride is half a row (2 THREADS chunks per row), so a thread's chunks j
// sit at row v_begin + j / 2, column chunk tid + (j odd) THREADS -- the
// two-slot ring's slot is the parity, and no cursor is kept.  FAST: the target
// level's inverse table is exact, it has no azimuth offsets and its width is
// a power of two (the projection has no branch).
// The first two source-range fetches of icp_block_terms (chunks tid and
// tid + THREADS of rows [v_begin, v_end)), issued and committed as one
// cp.async group by a caller that has other latency to overlap them with
// (the pose load at the start of a block); icp_block_terms is then called
// with prefetched = true.
template <int THREADS>
__device__ __forceinline__ void icp_prefetch(const IcpLaunch& a, IcpSmem<THREADS>& sm, int pair, int v_begin,
                                             int v_end) {
  const int tid = threadIdx.x;
  const int W = a.src.W;
  const int cpr = W >> 2;
  const int nchunks = max(0, v_end - v_begin) * cpr;
  const float* src = a.src_range + pair * (long long)a.src.H * W;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int c = tid + j * THREADS;
    if (c < nchunks) {
      const int v = v_begin + c / cpr, cu = c - (c / cpr) * cpr;
      cp_async16_zfill(&sm.src[j][tid], src + (long long)v * W + (cu << 2), true);
    }
  }
  cp_async_commit();
}

template <bool R0, bool GATE, bool ASSOC, bool KAHAN, int THREADS, int ROWSTRIDE = 0, bool FAST = false>
__device__ __forceinline__ void icp_block_terms(const IcpLaunch& a, IcpSmem<THREADS>& sm, int pair, int v_begin,
                                                int v_end, bool prefetched = false) {
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
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
  const float4* rowtab = row_table(sm);

  float2 t[kPairs];
#pragma unroll
  for (int i = 0; i < kPairs; ++i) t[i] = f2(0.f, 0.f);
  // this lane's component of the warp's running sum, with its Kahan term
  float ks = 0.f, kc = 0.f;

  // This thread's chunks: the j-th is block chunk tid + j * THREADS of the
  // block's rows [v_begin, v_end).  Cursors walk (row, 4-pixel column) one
  // thread-stride at a time.
  const int cpr = W >> 2;
  const int nchunks = max(0, v_end - v_begin) * cpr;
  const int nmine = (tid < nchunks) ? (nchunks - 1 - tid) / THREADS + 1 : 0;
  // the warp's trip count: its first lane has the most chunks
  const int nwarp = __shfl_sync(0xffffffffu, nmine, 0);
  const int dv = THREADS / cpr, dcu = THREADS - dv * cpr;
  struct Cursor {
    int v, cu;
  };
  const Cursor start{v_begin + tid / cpr, tid - (tid / cpr) * cpr};
  constexpr bool HALF = ROWSTRIDE == 2;
  static_assert(!HALF || (!GATE && !ASSOC), "the half-row form has no association output and no gate");
  auto advance = [&](Cursor& k) {
    if (ROWSTRIDE == 1) {
      k.v += dv;
    } else {
      k.cu += dcu;
      k.v += dv;
      if (k.cu >= cpr) { k.cu -= cpr; ++k.v; }
    }
  };
  Cursor cf = start, ci = start, cc = start;   // fetch, issue, consume
  int vrow = v_begin;   // HALF: the row of the current even / odd step pair

  // the source ranges of the chunk two steps ahead (same slot)
  auto fetch_src = [&](int slot) {
    if (HALF) {
      cp_async16_zfill(&sm.src[slot][tid], src + (long long)(vrow + 1) * W + ((tid + slot * THREADS) << 2), true);
    } else {
      cp_async16_zfill(&sm.src[slot][tid], src + (long long)cf.v * W + (cf.cu << 2), true);
      advance(cf);
    }
  };

  struct Pts {
    float x[4], y[4], z[4];
    int idx[4];
  };

  // Unproject, transform and project the next chunk into P; start the
  // gathers of its target planes (zero-filled when the pixel has no
  // association).
  auto issue = [&](int slot, Pts& P) {
    int v, u0;
    if (HALF) {
      v = vrow;
      u0 = (tid + slot * THREADS) << 2;
    } else {
      v = ci.v;
      u0 = ci.cu << 2;
      advance(ci);
    }
    const float4 r4 = sm.src[slot][tid];
    const float rr[4] = {r4.x, r4.y, r4.z, r4.w};
    const float4 cc4 = __ldg(reinterpret_cast<const float4*>(S.cos_u + u0));
    const float4 ss4 = __ldg(reinterpret_cast<const float4*>(S.sin_u + u0));
    const float cs[4] = {cc4.x, cc4.y, cc4.z, cc4.w}, sn[4] = {ss4.x, ss4.y, ss4.z, ss4.w};
    // Unprojection and transform folded (icp_row_table): R p + t =
    // r (cs A + sn B + C) + t, plus r0 (cs R0 + sn R1) with a receiver offset.
    const float4* rt = rowtab + 3 * (v - v_begin);
    const float4 A = rt[0], B = rt[1], C = rt[2];
    int gidx[4];
    bool gok[4];
    const float4 T0 = sm.T4[0], T1 = sm.T4[1], T2 = sm.T4[2];   // read with a receiver offset only
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool valid = range_ok(rr[q]);
      const float r = valid ? rr[q] : 0.f;
      const float Dx = fmaf(cs[q], A.x, fmaf(sn[q], B.x, C.x));
      const float Dy = fmaf(cs[q], A.y, fmaf(sn[q], B.y, C.y));
      const float Dz = fmaf(cs[q], A.z, fmaf(sn[q], B.z, C.z));
      const float ox = R0 ? fmaf(S.r0 * cs[q], T0.x, fmaf(S.r0 * sn[q], T0.y, T0.w)) : A.w;
      const float oy = R0 ? fmaf(S.r0 * cs[q], T1.x, fmaf(S.r0 * sn[q], T1.y, T1.w)) : B.w;
      const float oz = R0 ? fmaf(S.r0 * cs[q], T2.x, fmaf(S.r0 * sn[q], T2.y, T2.w)) : C.w;
      const float X = fmaf(r, Dx, ox);
      const float Y = fmaf(r, Dy, oy);
      const float Z = fmaf(r, Dz, oz);
      int uu, vv;
      const bool fov = project_px<R0, FAST>(D, make_float3(X, Y, Z), a.proj_iters, uu, vv);
      const bool ok = valid && fov;
      const int idx = vv * D.W + uu;
      P.x[q] = X;
      P.y[q] = Y;
      P.z[q] = Z;
      P.idx[q] = ok ? idx : -1;    // read by the gate and the association output only
      gidx[q] = idx;               // a valid index whatever ok (project_px), read only when ok
      gok[q] = ok;
    }
    // The gathers after all four projections: each copy is an asm statement
    // that clobbers memory, so a copy between two projections would keep the
    // next pixel's table loads from moving above it.
#pragma unroll
    for (int q = 0; q < 4; ++q) cp_async16_zfill(&sm.planes[slot][q][tid], planes + gidx[q], gok[q]);
  };

  // The warp's plain sums since the last step, added to each lane's running
  // component with Kahan compensation (or plainly); t restarts at zero.
  auto warp_flush = [&]() {
    const float y0 = warp_scatter_sum(t, lane);
    if (KAHAN) {
      const float y = y0 - kc;
      const float tt = ks + y;
      kc = (tt - ks) - y;
      ks = tt;
    } else {
      ks += y0;
    }
#pragma unroll
    for (int i = 0; i < kPairs; ++i) t[i] = f2(0.f, 0.f);
  };

  // Accumulate a chunk in flight (its planes have landed) into t.
  auto consume = [&](int slot, const Pts& P) {
    int out_idx[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float4 pl = sm.planes[slot][q][tid];
      const int idx = P.idx[q];
      if (GATE) {
        bool keep = idx >= 0;
        if (keep) {
          const int vv = idx / D.W, uu = idx - vv * D.W;
          const float rq = __ldg(drange + idx);
          const float3 qq = unproject_px(D, uu, vv, range_ok(rq) ? rq : 0.f);
          const float dx = P.x[q] - qq.x, dy = P.y[q] - qq.y, dz = P.z[q] - qq.z;
          keep = range_ok(rq) && (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= gate2);
        }
        if (!keep) pl = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      out_idx[q] = (pl.x != 0.f || pl.y != 0.f || pl.z != 0.f) ? idx : -1;
      accumulate_px(t, P.x[q], P.y[q], P.z[q], pl, inv_delta);
    }
    if (ASSOC) {
      int* ap = a.assoc + pair * Ns + (long long)cc.v * W + (cc.cu << 2);
      *reinterpret_cast<int4*>(ap) = make_int4(out_idx[0], out_idx[1], out_idx[2], out_idx[3]);
      advance(cc);
    }
  };

  // Software pipeline over the warp's chunks (warp-uniform trip count; a lane
  // past its own last chunk only takes part in the warp steps) with a
  // two-slot ring: step i projects chunk i (ranges fetched two steps
  // earlier), starts its gathers and the range fetch of chunk i + 2 into the
  // same slot, commits one cp.async group, waits until at most one group is
  // pending (so group i - 1 has landed) and accumulates chunk i - 1.
  // Unrolled by two so slots are constants.
  static_assert(kRing == 2, "the pipeline below is written for a two-slot ring");
  Pts P0, P1;
  if (prefetched) {          // chunks 0 and 1 were fetched by icp_prefetch
    if (!HALF && nmine > 0) advance(cf);
    if (!HALF && nmine > 1) advance(cf);
  } else {
    if (HALF) {
      if (nmine > 0) cp_async16_zfill(&sm.src[0][tid], src + (long long)v_begin * W + (tid << 2), true);
      if (nmine > 1) cp_async16_zfill(&sm.src[1][tid], src + (long long)v_begin * W + ((tid + THREADS) << 2), true);
    } else {
      if (nmine > 0) fetch_src(0);
      if (nmine > 1) fetch_src(1);
    }
    cp_async_commit();
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  int i = 0;
  while (true) {
    // even step: slot 0 issues, slot 1 is consumed
    if (i < nmine) {
      issue(0, P0);
      if (i + 2 < nmine) fetch_src(0);
    }
    cp_async_commit();
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    if (i >= 1 && i - 1 < nmine) consume(1, P1);
    if (i >= 1 && (i % kWarpFlush) == 0) warp_flush();
    if (i >= nwarp) break;
    ++i;
    // odd step: slot 1 issues, slot 0 is consumed
    if (i < nmine) {
      issue(1, P1);
      if (i + 2 < nmine) fetch_src(1);
    }
    if (HALF) ++vrow;
    cp_async_commit();
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    if (i - 1 < nmine) consume(0, P0);
    if ((i % kWarpFlush) == 0) warp_flush();
    if (i >= nwarp) break;
    ++i;
  }
  // the last step flushed already when nwarp is a multiple of kWarpFlush
  // (nwarp = 0: nothing was summed)
  if ((nwarp % kWarpFlush) != 0) warp_flush();
  asm volatile("cp.async.wait_all;\n" ::: "memory");

  // lane l holds the warp's component l
  if (lane < 2 * kPairs) sm.red[warp][lane] = KAHAN ? ks - kc : ks;
  __syncthreads();
}

// Block's FP32 total of reduced quantity `tid` (output order) from the
// per-warp components.
template <int THREADS>
__device__ __forceinline__ float block_total(const IcpSmem<THREADS>& sm, int tid) {
  const int f = kFlat[tid];
  float acc = 0.f;
#pragma unroll
  for (int w = 0; w < THREADS / 32; ++w) acc += sm.red[w][f];
  return acc;
}

template <bool R0, bool GATE, bool ASSOC, bool KAHAN, int THREADS, int ROWSTRIDE = 0, bool FAST = false>
__global__ void __launch_bounds__(THREADS, RIMG_ICP_THREADS_PER_SM / THREADS) k_icp(IcpLaunch a) {
  extern __shared__ float4 smem_raw[];
  IcpSmem<THREADS>& sm = *reinterpret_cast<IcpSmem<THREADS>*>(smem_raw);
  const int tid = threadIdx.x;
  const int pair = blockIdx.x / a.bpp;
  const int blk = blockIdx.x - pair * a.bpp;
  const int v_begin = blk * a.rows_per_block;
  const int v_end = min(a.src.H, v_begin + a.rows_per_block);
  // the first source ranges are fetched while the pose is loaded
  icp_prefetch<THREADS>(a, sm, pair, v_begin, v_end);
  if (tid < 12) reinterpret_cast<float*>(sm.T4)[tid] = (float)a.pose[pair * 16 + tid];
  __syncthreads();
  // (filling the table straight from the pose in global memory, with one
  // barrier less, measured slower)
  icp_row_table(a.src, sm, v_begin, max(0, v_end - v_begin), tid, THREADS);
  __syncthreads();
  icp_block_terms<R0, GATE, ASSOC, KAHAN, THREADS, ROWSTRIDE, FAST>(a, sm, pair, v_begin, v_end, true);
  if (a.bpp == 1) {
    // one block per pair: the block total is the pair total
    if (tid < kRed) {
      const double v = (double)block_total(sm, tid);
      a.sums[pair * kRedStride + tid] = v;
      if (a.out29) a.out29[pair * kRed + tid] = v;
    }
  } else {
    if (tid < kRed) a.partials[((long long)pair * a.bpp + blk) * kRedStride + tid] = block_total(sm, tid);
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
      a.sums[pair * kRedStride + tid] = acc;
      if (a.out29) a.out29[pair * kRed + tid] = acc;
    }
    if (tid == 0) a.counters[pair] = 0u;
  }
}

// The Gauss-Newton update from a pair's FP64 sums t[0..28], by all 32 lanes
// of one warp: FP64 solve of the 6x6 system and T <- Exp(xi) T for the 3x4
// pose T (Tf: optional FP32 copy of the new pose).  rec, if given, receives
// |omega| (rad) and |tau| (m) of the step (to FP32 precision) and 1 if it was applied (0, 0, 0:
// fewer than 6 correspondences or a degenerate pivot, T unchanged).  Returns
// whether it was applied (the same in every lane).
__device__ __noinline__ bool warp_gn_update(const double* t, double* T, float* Tf, double* rec, int lane) {
  double x[6];
  bool good = t[28] >= 6.0;
  if (good) good = warp_solve6(t, lane, x);
  if (good) warp_se3_update(T, x, lane, Tf);
  if (rec && lane < 3) {
    double val = 0.0;
    if (good) {
      if (lane == 2) {
        val = 1.0;
      } else {
        const double p = lane ? x[3] : x[0], q = lane ? x[4] : x[1], r = lane ? x[5] : x[2];
        val = (double)sqrtf((float)fma(r, r, fma(q, q, p * p)));   // a diagnostic: FP32 root
      }
    }
    rec[lane] = val;
  }
  return good;
}

// The Gauss-Newton update of every pair from its FP64 sums: one warp per pair
// (four per block).  Kept out of k_icp so that no reduction block holds an
// SM slot through the FP64 chain.  The pair's record keeps the size of the
// step in its spare slots.
__global__ void __launch_bounds__(128) k_solve(int n_pairs, double* sums, double* pose, int* __restrict__ status) {
  const int pair = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (pair >= n_pairs) return;
  double* t = sums + (long long)pair * kRedStride;
  const bool ok = warp_gn_update(t, pose + (long long)pair * 16, nullptr, t + 29, lane);
  if (!ok && lane == 0 && status) status[pair] |= RIMG_FLAG_DEGENERATE;
}

// All iterations of one small level in one launch: one block per pair
// associates and reduces the pair's whole level, its first warp solves in
// FP64 and updates the pose in shared memory, and the block goes on with the
// next iteration -- the per-iteration launches (association + solve) of a
// level whose pair fits one block collapse into one.  Same arithmetic as
// k_icp with one block per pair followed by k_solve.  The pair's final sums
// and step record are left in a.sums (as after the last k_solve).
template <bool R0, bool GATE, bool KAHAN, int THREADS, int ROWSTRIDE = 0, bool FAST = false>
__global__ void __launch_bounds__(THREADS, RIMG_ICP_THREADS_PER_SM / THREADS) k_icp_iters(IcpLaunch a, int iters) {
  extern __shared__ float4 smem_raw[];
  IcpSmem<THREADS>& sm = *reinterpret_cast<IcpSmem<THREADS>*>(smem_raw);
  __shared__ double Tp[12];
  __shared__ int degenerate;
  const int tid = threadIdx.x;
  const int pair = blockIdx.x;
  if (tid < 12) {
    Tp[tid] = a.pose[pair * 16 + tid];
    reinterpret_cast<float*>(sm.T4)[tid] = (float)Tp[tid];
  }
  if (tid == 0) degenerate = 0;
  __syncthreads();
  icp_row_table(a.src, sm, 0, a.src.H, tid, THREADS);
  __syncthreads();
  for (int it = 0; it < iters; ++it) {
    icp_block_terms<R0, GATE, false, KAHAN, THREADS, ROWSTRIDE, FAST>(a, sm, pair, 0, a.src.H);
    if (tid < kRed) sm.tot[tid] = (double)block_total(sm, tid);
    __syncthreads();
    if (tid < 32) {
      const bool ok = warp_gn_update(sm.tot, Tp, reinterpret_cast<float*>(sm.T4), it == iters - 1 ? sm.tot + 29 : nullptr,
                                     tid);
      if (!ok && tid == 0) degenerate = 1;
      // the next iteration's row table, by the warp that updated the pose
      if (it + 1 < iters) {
        __syncwarp();
        icp_row_table(a.src, sm, 0, a.src.H, tid, 32);
      }
    }
    __syncthreads();
  }
  if (tid < 12) a.pose[pair * 16 + tid] = Tp[tid];
  if (iters > 0 && tid < kRedStride) a.sums[pair * kRedStride + tid] = sm.tot[tid];
  if (tid == 0 && degenerate && a.status) a.status[pair] |= RIMG_FLAG_DEGENERATE;
}

// All iterations of one small level in one launch, each pair on a cluster of
// C blocks (thread-block cluster, distributed shared memory): block r of the
// cluster takes rows [r * rpb, (r + 1) * rpb) of the pair (rpb = ceil(H / C)),
// the blocks' FP32 totals are exchanged through distributed shared memory
// after one cluster barrier per iteration, and every block sums them in FP64
// in rank order and runs the same FP64 update, so all blocks of a cluster
// carry the same pose without a second barrier.  Same arithmetic, in the same
// order, as k_icp with C blocks per pair (its last-block FP64 sum) followed by
// k_solve: poses and sums are bit-identical to that per-iteration schedule.
// The per-iteration latency of a pair (association, reduction, the update's
// FP64 chain) is spread over C SMs instead of one.  The block totals are
// double-buffered by iteration parity: a block writes buffer it % 2 again in
// iteration it + 2, after passing the barrier of iteration it + 1, which no
// block reaches before it has finished reading the buffers of iteration it.
// So one cluster barrier per iteration and one before exit (no block leaves
// while another may still read its shared memory) suffice; every block of a
// cluster runs the same number of iterations, so every barrier completes.
namespace cg = cooperative_groups;

template <bool R0, bool KAHAN, int THREADS, int ROWSTRIDE, bool FAST, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(THREADS, RIMG_ICP_THREADS_PER_SM / THREADS)
    k_icp_cluster(IcpLaunch a, int iters) {
  extern __shared__ float4 smem_raw[];
  IcpSmem<THREADS>& sm = *reinterpret_cast<IcpSmem<THREADS>*>(smem_raw);
  __shared__ double Tp[12];
  __shared__ float blk[2][32];
  __shared__ int degenerate;
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x;
  const int rank = (int)cluster.block_rank();
  const int pair = blockIdx.x / C;
  const int rpb = (a.src.H + C - 1) / C;
  const int v_begin = min(a.src.H, rank * rpb);
  const int v_end = min(a.src.H, v_begin + rpb);
  if (tid < 12) {
    Tp[tid] = a.pose[pair * 16 + tid];
    reinterpret_cast<float*>(sm.T4)[tid] = (float)Tp[tid];
  }
  if (tid == 0) degenerate = 0;
  __syncthreads();
  icp_row_table(a.src, sm, v_begin, v_end - v_begin, tid, THREADS);
  __syncthreads();
  for (int it = 0; it < iters; ++it) {
    icp_block_terms<R0, false, false, KAHAN, THREADS, ROWSTRIDE, FAST>(a, sm, pair, v_begin, v_end);
    float* mine = blk[it & 1];
    if (tid < kRed) mine[tid] = block_total(sm, tid);
    cluster.sync();
    if (tid < kRed) {
      double acc = 0.0;
#pragma unroll
      for (int r = 0; r < C; ++r) acc += (double)*cluster.map_shared_rank(mine + tid, r);
      sm.tot[tid] = acc;
    }
    __syncthreads();
    if (tid < 32) {
      const bool ok = warp_gn_update(sm.tot, Tp, reinterpret_cast<float*>(sm.T4), it == iters - 1 ? sm.tot + 29 : nullptr,
                                     tid);
      if (!ok && tid == 0) degenerate = 1;
      // the next iteration's row table, by the warp that updated the pose
      if (it + 1 < iters) {
        __syncwarp();
        icp_row_table(a.src, sm, v_begin, v_end - v_begin, tid, 32);
      }
    }
    __syncthreads();
  }
  cluster.sync();   // no block exits while another may still read its totals
  if (rank != 0) return;
  if (tid < 12) a.pose[pair * 16 + tid] = Tp[tid];
  if (iters > 0 && tid < kRedStride) a.sums[pair * kRedStride + tid] = sm.tot[tid];
  if (tid == 0 && degenerate && a.status) a.status[pair] |= RIMG_FLAG_DEGENERATE;
}

// ---------------------------------------------------------------------------
// Persistent work queue over the small levels of uneven batches.

// Copies one group descriptor (a kernel parameter) into device memory, so
// that the descriptor table is written inside the stream (and a captured
// graph carries it).
__global__ void k_put_group(QueueGroup g, QueueGroup* dst) {
  static_assert(sizeof(QueueGroup) % 4 == 0, "descriptor copied as words");
  const int* s = reinterpret_cast<const int*>(&g);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(QueueGroup) / 4); i += blockDim.x) d[i] = s[i];
}

// One block per item at a time: the block takes the next item from the
// counter, runs the item's pair through all its group's queued levels
// (association + reduction of the whole level, the FP64 update by the first
// warp, next iteration) and goes on to the next item.  Items are ordered by
// cost (the host lists the most expensive groups first).  No block waits for
// another; the last blocks to find the queue empty simply exit.
template <bool R0, bool KAHAN>
__global__ void __launch_bounds__(kQueueThreads, RIMG_ICP_THREADS_PER_SM / kQueueThreads)
    k_icp_queue(const QueueGroup* __restrict__ groups, int n_groups, int n_items, unsigned* counter) {
  constexpr int THREADS = kQueueThreads;
  constexpr int kDL = (int)(sizeof(DevLevel) / 4);
  static_assert(sizeof(DevLevel) % 4 == 0 && kDL <= 32, "a level view is copied by one warp");
  extern __shared__ float4 smem_raw[];
  IcpSmem<THREADS>& sm = *reinterpret_cast<IcpSmem<THREADS>*>(smem_raw);
  __shared__ IcpLaunch la;
  __shared__ double Tp[12];
  __shared__ int item_s, group_s, iters_s, degenerate;
  const int tid = threadIdx.x;
  while (true) {
    if (tid == 0) {
      const int it = (int)atomicAdd(counter, 1u);
      int g = 0;
      while (g + 1 < n_groups && it >= groups[g + 1].item0) ++g;
      item_s = it;
      group_s = g;
      degenerate = 0;
    }
    __syncthreads();
    const int item = item_s;
    if (item >= n_items) break;
    const QueueGroup* G = groups + group_s;
    const int pair = item - G->item0;
    if (tid < 12) {
      Tp[tid] = G->pose[(long long)pair * 16 + tid];
      reinterpret_cast<float*>(sm.T4)[tid] = (float)Tp[tid];
    }
    const int nl = G->n_lvl;
    bool ran = false;
    for (int k = 0; k < nl; ++k) {
      __syncthreads();                       // the previous level's readers of `la` are done
      const QueueLevel& QL = G->lvl[k];
      if (tid < kDL) {
        reinterpret_cast<int*>(&la.src)[tid] = reinterpret_cast<const int*>(&QL.src)[tid];
      } else if (tid >= 32 && tid < 32 + kDL) {
        reinterpret_cast<int*>(&la.dst)[tid - 32] = reinterpret_cast<const int*>(&QL.dst)[tid - 32];
      } else if (tid == 64) {
        la.src_range = QL.src_range;
        la.dst_planes = QL.planes;
        la.dst_range = nullptr;
        la.out29 = nullptr;
        la.assoc = nullptr;
        la.huber_delta = G->huber_delta;
        la.max_corr_dist = 0.f;
        la.proj_iters = G->proj_iters;
        la.kahan = KAHAN ? 1 : 0;
        la.n_pairs = G->n_pairs;
        iters_s = QL.iters;
      }
      __syncthreads();
      const int iters = iters_s;
      if (iters > 0) {
        icp_row_table(la.src, sm, 0, la.src.H, tid, THREADS);
        __syncthreads();
      }
      for (int it = 0; it < iters; ++it) {
        icp_block_terms<R0, false, false, KAHAN, THREADS, true, true>(la, sm, pair, 0, la.src.H);
        if (tid < kRed) sm.tot[tid] = (double)block_total<THREADS>(sm, tid);
        __syncthreads();
        if (tid < 32) {
          const bool last = (k == nl - 1) && (it == iters - 1);
          const bool ok = warp_gn_update(sm.tot, Tp, reinterpret_cast<float*>(sm.T4), last ? sm.tot + 29 : nullptr,
                                         tid);
          if (!ok && tid == 0) degenerate = 1;
          // the next iteration's row table, by the warp that updated the pose
          if (it + 1 < iters) {
            __syncwarp();
            icp_row_table(la.src, sm, 0, la.src.H, tid, 32);
          }
        }
        __syncthreads();
        ran = true;
      }
    }
    if (tid < 12) G->pose[(long long)pair * 16 + tid] = Tp[tid];
    if (ran && tid < kRedStride && G->sums) G->sums[(long long)pair * kRedStride + tid] = sm.tot[tid];
    if (tid == 0 && degenerate && G->status) G->status[pair] |= RIMG_FLAG_DEGENERATE;
    __syncthreads();                         // before item_s is overwritten
  }
}

bool queue_level_ok(int H, int W) {
  const int cpr = W / 4;
  return icp_iters_fits(H, W) && cpr > 0 && cpr <= kQueueThreads && kQueueThreads % cpr == 0;
}

namespace {
template <bool R0, bool KAHAN>
cudaError_t launch_queue_t(const QueueGroup* dev_groups, int n_groups, int n_items, unsigned* counter,
                           cudaStream_t st) {
  // every queued level fits one block (icp_iters_fits), so at most kMaxBlockRows rows
  constexpr size_t bytes = icp_smem_bytes<kQueueThreads>(kMaxBlockRows);
  static int grid_cap = 0;     // resident blocks on the device (per instantiation)
  if (grid_cap == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_icp_queue<R0, KAHAN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_icp_queue<R0, KAHAN>, kQueueThreads, bytes);
    grid_cap = std::max(1, sms) * std::max(1, occ);
  }
  const int grid = std::min(n_items, grid_cap);
  k_icp_queue<R0, KAHAN><<<grid, kQueueThreads, bytes, st>>>(dev_groups, n_groups, n_items, counter);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_icp_queue(const QueueGroup* host_groups, int n_groups, QueueGroup* dev_groups, unsigned* counter,
                             bool r0, bool kahan, cudaStream_t st) {
  int n_items = 0;
  for (int g = 0; g < n_groups; ++g) n_items += host_groups[g].n_pairs;
  if (n_items == 0) return cudaSuccess;
  for (int g = 0; g < n_groups; ++g) {
    k_put_group<<<1, 64, 0, st>>>(host_groups[g], dev_groups + g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (r0) return kahan ? launch_queue_t<true, true>(dev_groups, n_groups, n_items, counter, st)
                       : launch_queue_t<true, false>(dev_groups, n_groups, n_items, counter, st);
  return kahan ? launch_queue_t<false, true>(dev_groups, n_groups, n_items, counter, st)
               : launch_queue_t<false, false>(dev_groups, n_groups, n_items, counter, st);
}

cudaError_t launch_solve(int n_pairs, double* sums, double* pose, int* status, cudaStream_t st) {
  if (n_pairs == 0) return cudaSuccess;
  k_solve<<<(n_pairs + 3) / 4, 128, 0, st>>>(n_pairs, sums, pose, status);
  return cudaGetLastError();
}

namespace {
int g_num_sms = 0;
int g_blocks_per_sm[2] = {0, 0};   // resident blocks per SM for 128- and 256-thread blocks

template <int T>
int occupancy() {
  constexpr size_t bytes = icp_smem_bytes<T>(16);   // a typical block's row table
  cudaFuncSetAttribute(k_icp<false, false, false, true, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)icp_smem_bytes<T>(kMaxBlockRows));
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_icp<false, false, false, true, T>, T, bytes);
  return nb > 0 ? nb : 1;
}
}  // namespace

namespace {
// Launch shapes chosen by rimg_autotune, keyed by (level rows, columns, pairs).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, std::pair<int, int>> g_tune;
// Per-level schedule chosen by rimg_autotune: 1 = all iterations in one block
// per pair (k_icp_iters / the queue; levels that fit one block), 2, 4 or 8 =
// all iterations on a cluster of that many blocks per pair (k_icp_cluster),
// 0 = one multi-block association launch plus one solve per iteration.
std::map<std::tuple<int, int, int>, int> g_sched;
}  // namespace

void icp_tune_set(int H, int W, int n_pairs, int threads, int bpp) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[std::make_tuple(H, W, n_pairs)] = std::make_pair(threads, bpp);
}

void icp_tune_clear() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  g_sched.clear();
}

void icp_tune_erase(int H, int W, int n_pairs) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.erase(std::make_tuple(H, W, n_pairs));
}

void icp_sched_set(int H, int W, int n_pairs, int sched) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_sched[std::make_tuple(H, W, n_pairs)] = sched;
}

int icp_sched(int H, int W, int n_pairs) {
  const bool fits = icp_iters_fits(H, W);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_sched.find(std::make_tuple(H, W, n_pairs));
  if (it == g_sched.end()) return fits ? 1 : 0;
  // one block per pair only where the pair fits one block
  return (it->second == 1 && !fits) ? 0 : it->second;
}

int icp_tune_size() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int)(g_tune.size() + g_sched.size());
}

struct IcpTuneTable {
  std::map<std::tuple<int, int, int>, std::pair<int, int>> shapes;
  std::map<std::tuple<int, int, int>, int> sched;
};

void* icp_tune_save() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return new IcpTuneTable{g_tune, g_sched};
}

void icp_tune_restore(const void* saved) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const IcpTuneTable* t = static_cast<const IcpTuneTable*>(saved);
  g_tune = t->shapes;
  g_sched = t->sched;
}

void icp_tune_free(void* saved) { delete static_cast<IcpTuneTable*>(saved); }

void icp_grid(int H, int W, int n_pairs, int* bpp, int* rows_per_block, int* threads) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(H, W, n_pairs));
    if (it != g_tune.end()) {
      const int b = std::min(std::max(it->second.second, 1), H);
      const int rpb = (H + b - 1) / b;
      *rows_per_block = rpb;
      *bpp = (H + rpb - 1) / rpb;
      *threads = it->second.first;
      return;
    }
  }
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_blocks_per_sm[0] = occupancy<128>();
    g_blocks_per_sm[1] = occupancy<256>();
    g_num_sms = sms > 0 ? sms : 148;
  }
  // 128-thread blocks, aiming at ~32 four-pixel chunks per thread: enough
  // work to amortise a block's start and reduction, few enough blocks per
  // pair to keep the FP64 cross-block sum short (level 0 of 512 pairs of
  // 64 x 1024: 173.7 us against 192.9 us with 256-thread blocks of 16 chunks
  // per thread).
  const long long cpp = (long long)H * (W / 4);
  const int T = 128;
  long long b = cpp / ((long long)T * 32);
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

// Whether a thread stride of T chunks is a whole number of rows of the level.
inline bool row_stride(const IcpLaunch& a, int T) {
  const int cpr = a.src.W >> 2;
  return cpr > 0 && cpr <= T && T % cpr == 0;
}

// Whether a thread stride of T chunks is half a row of the level.
inline bool half_row(const IcpLaunch& a, int T) { return (a.src.W >> 2) == 2 * T; }

// Whether the target level's projection needs neither the boundary walk nor
// the azimuth offsets, and its columns wrap by a mask (power-of-two width).
inline bool fast_projection(const IcpLaunch& a) {
  return a.dst.bins_exact && !a.dst.has_theta && a.dst.W > 0 && (a.dst.W & (a.dst.W - 1)) == 0;
}

template <bool R0, bool GATE, bool ASSOC, bool KAHAN, int T, int ROWSTRIDE, bool FAST = false>
cudaError_t launch_icp_ts(const IcpLaunch& a, long long blocks, cudaStream_t st) {
  const size_t bytes = icp_smem_bytes<T>(a.rows_per_block);
  static bool configured = false;   // per instantiation; the attribute is per function
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_icp<R0, GATE, ASSOC, KAHAN, T, ROWSTRIDE, FAST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)icp_smem_bytes<T>(kMaxBlockRows));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k_icp<R0, GATE, ASSOC, KAHAN, T, ROWSTRIDE, FAST><<<(unsigned)blocks, T, bytes, st>>>(a);
  return cudaGetLastError();
}

// the row-stride and fast-projection forms only on the default path (no gate,
// no association output)
template <bool R0, bool GATE, bool ASSOC, bool KAHAN, int T>
cudaError_t launch_icp_t(const IcpLaunch& a, long long blocks, cudaStream_t st) {
  if constexpr (!GATE && !ASSOC) {
    const bool fast = fast_projection(a);
    if (row_stride(a, T)) {
      if (fast) return launch_icp_ts<R0, GATE, ASSOC, KAHAN, T, 1, true>(a, blocks, st);
      return launch_icp_ts<R0, GATE, ASSOC, KAHAN, T, 1>(a, blocks, st);
    }
    if (half_row(a, T)) {
      if (fast) return launch_icp_ts<R0, GATE, ASSOC, KAHAN, T, 2, true>(a, blocks, st);
      return launch_icp_ts<R0, GATE, ASSOC, KAHAN, T, 2>(a, blocks, st);
    }
    if (fast) return launch_icp_ts<R0, GATE, ASSOC, KAHAN, T, 0, true>(a, blocks, st);
  }
  return launch_icp_ts<R0, GATE, ASSOC, KAHAN, T, 0>(a, blocks, st);
}

template <bool R0, bool GATE, bool ASSOC, bool KAHAN>
cudaError_t launch_icp_k(const IcpLaunch& a, long long blocks, cudaStream_t st) {
  return a.threads == 128 ? launch_icp_t<R0, GATE, ASSOC, KAHAN, 128>(a, blocks, st)
                          : launch_icp_t<R0, GATE, ASSOC, KAHAN, 256>(a, blocks, st);
}

template <bool R0, bool GATE, bool KAHAN, int T, int ROWSTRIDE, bool FAST = false>
cudaError_t launch_icp_iters_ts(const IcpLaunch& a, int iters, cudaStream_t st) {
  const size_t bytes = icp_smem_bytes<T>(a.src.H);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_icp_iters<R0, GATE, KAHAN, T, ROWSTRIDE, FAST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)icp_smem_bytes<T>(kMaxBlockRows));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k_icp_iters<R0, GATE, KAHAN, T, ROWSTRIDE, FAST><<<(unsigned)a.n_pairs, T, bytes, st>>>(a, iters);
  return cudaGetLastError();
}

template <bool R0, bool GATE, bool KAHAN, int T>
cudaError_t launch_icp_iters_t(const IcpLaunch& a, int iters, cudaStream_t st) {
  if constexpr (!GATE) {
    if (row_stride(a, T)) {
      if (fast_projection(a)) return launch_icp_iters_ts<R0, GATE, KAHAN, T, true, true>(a, iters, st);
      return launch_icp_iters_ts<R0, GATE, KAHAN, T, true>(a, iters, st);
    }
  }
  return launch_icp_iters_ts<R0, GATE, KAHAN, T, false>(a, iters, st);
}

template <bool R0, bool GATE, bool KAHAN>
cudaError_t launch_icp_iters_k(const IcpLaunch& a, int iters, cudaStream_t st) {
  return launch_icp_iters_t<R0, GATE, KAHAN, 128>(a, iters, st);
}

bool icp_iters_fits(int H, int W) { return H <= kMaxBlockRows && (long long)H * (W / 4) <= kIcpItersMaxChunks; }

template <bool R0, bool KAHAN, int ROWSTRIDE, bool FAST, int C>
cudaError_t launch_icp_cluster_ts(const IcpLaunch& a, int iters, cudaStream_t st) {
  constexpr int T = 128;
  const size_t bytes = icp_smem_bytes<T>(a.rows_per_block);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_icp_cluster<R0, KAHAN, T, ROWSTRIDE, FAST, C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)icp_smem_bytes<T>(kMaxBlockRows));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k_icp_cluster<R0, KAHAN, T, ROWSTRIDE, FAST, C><<<(unsigned)((long long)a.n_pairs * C), T, bytes, st>>>(a, iters);
  return cudaGetLastError();
}

template <bool R0, bool KAHAN, int C>
cudaError_t launch_icp_cluster_c(const IcpLaunch& a, int iters, cudaStream_t st) {
  const bool fast = fast_projection(a);
  if (row_stride(a, 128))
    return fast ? launch_icp_cluster_ts<R0, KAHAN, 1, true, C>(a, iters, st)
                : launch_icp_cluster_ts<R0, KAHAN, 1, false, C>(a, iters, st);
  if (half_row(a, 128))
    return fast ? launch_icp_cluster_ts<R0, KAHAN, 2, true, C>(a, iters, st)
                : launch_icp_cluster_ts<R0, KAHAN, 2, false, C>(a, iters, st);
  return fast ? launch_icp_cluster_ts<R0, KAHAN, 0, true, C>(a, iters, st)
              : launch_icp_cluster_ts<R0, KAHAN, 0, false, C>(a, iters, st);
}

template <int C>
cudaError_t launch_icp_cluster_r(const IcpLaunch& a, int iters, cudaStream_t st) {
  const bool r0 = a.dst.r0 != 0.f || a.src.r0 != 0.f;
  const bool kahan = a.kahan != 0;
  if (r0) return kahan ? launch_icp_cluster_c<true, true, C>(a, iters, st) : launch_icp_cluster_c<true, false, C>(a, iters, st);
  return kahan ? launch_icp_cluster_c<false, true, C>(a, iters, st) : launch_icp_cluster_c<false, false, C>(a, iters, st);
}

cudaError_t launch_icp_cluster(IcpLaunch a, int iters, int cluster, cudaStream_t st) {
  if (a.n_pairs == 0 || iters == 0) return cudaSuccess;
  if ((cluster != 2 && cluster != 4 && cluster != 8) || a.max_corr_dist > 0.f || a.assoc)
    return cudaErrorInvalidValue;
  a.threads = 128;
  a.bpp = cluster;
  a.rows_per_block = (a.src.H + cluster - 1) / cluster;
  if (a.rows_per_block > kMaxBlockRows) return cudaErrorInvalidValue;
  if (cluster == 2) return launch_icp_cluster_r<2>(a, iters, st);
  return cluster == 4 ? launch_icp_cluster_r<4>(a, iters, st) : launch_icp_cluster_r<8>(a, iters, st);
}

cudaError_t launch_icp_iters(IcpLaunch a, int iters, cudaStream_t st) {
  if (a.n_pairs == 0 || iters == 0) return cudaSuccess;
  // 128-thread blocks: the level's blocks of concurrent sub-batches fit the
  // GPU in fewer waves than 256-thread ones (level 1 of 512 pairs of 64 x 1024
  // in four 128-pair sub-batches: 0.75 against 0.81 ms)
  a.threads = 128;
  a.bpp = 1;
  a.rows_per_block = a.src.H;
  const bool r0 = a.dst.r0 != 0.f || a.src.r0 != 0.f;
  const bool gate = a.max_corr_dist > 0.f;
  const bool kahan = a.kahan != 0;
  if (r0) {
    if (gate) return kahan ? launch_icp_iters_k<true, true, true>(a, iters, st) : launch_icp_iters_k<true, true, false>(a, iters, st);
    return kahan ? launch_icp_iters_k<true, false, true>(a, iters, st) : launch_icp_iters_k<true, false, false>(a, iters, st);
  }
  if (gate) return kahan ? launch_icp_iters_k<false, true, true>(a, iters, st) : launch_icp_iters_k<false, true, false>(a, iters, st);
  return kahan ? launch_icp_iters_k<false, false, true>(a, iters, st) : launch_icp_iters_k<false, false, false>(a, iters, st);
}

cudaError_t launch_icp(IcpLaunch a, cudaStream_t st) {
  if (a.n_pairs == 0) return cudaSuccess;
  if (a.rows_per_block > kMaxBlockRows) {   // the row table bounds a block's rows
    a.rows_per_block = kMaxBlockRows;
    a.bpp = (a.src.H + kMaxBlockRows - 1) / kMaxBlockRows;
  }
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
