// Device-side sensor model: unprojection (Eq. 1-2) and projection (Eq. 3-4
// plus the column recovery that reverts Eq. 2), FP32, table driven.
#pragma once

#include <cuda_runtime.h>
#include "rimg_internal.h"

namespace rimg {

// Eq. 1-2 at integer pixel (u, v) with range r, from the separable tables:
// cos/sin(theta) = cos/sin(col + theta_lut) by the angle-addition identities.
__device__ __forceinline__ float3 unproject_px(const DevLevel& L, int u, int v, float r) {
  const float4 rw = __ldg(L.rows + v);
  const float cu = __ldg(L.cos_u + u), su = __ldg(L.sin_u + u);
  const float ct = fmaf(cu, rw.z, -su * rw.w);
  const float st = fmaf(su, rw.z, cu * rw.w);
  const float rc = r * rw.x;
  return make_float3(fmaf(rc, ct, L.r0 * cu), fmaf(rc, st, L.r0 * su), r * rw.y);
}

// Eq. 4 in sin(elevation) space: the row whose elevation is nearest to that
// of a point with sin(elevation) = s.  Each bin of the inverse table holds at
// most one mid-elevation boundary (bins_exact), so one comparison with it
// picks the row below or above; the tie rule (exact ties go to the lower row
// index) is folded into the stored boundary.  For tables too uneven for that,
// the walk across the sorted boundaries (bounded by H) gives the same argmin.
// EXACT: the caller knows the table is exact (no walk, no branch).
template <bool EXACT = false>
__device__ __forceinline__ int row_from_sin(const DevLevel& L, float s) {
  int b = __float2int_rd((s - L.s_lo) * L.bin_scale);
  // clamp into the table; EXACT: one unsigned minimum (a negative bin, s
  // below the field of view, lands on the last bin -- its row is not used,
  // the caller's field-of-view test rejects the point)
  b = EXACT ? (int)min((unsigned)b, (unsigned)(L.n_bins - 1)) : min(max(b, 0), L.n_bins - 1);
  const int4 e = __ldg(L.bins + b);
  if (EXACT || L.bins_exact) return (s > __int_as_float(e.z)) ? e.y : e.x;   // tie rule folded into the boundary
  int j = e.w;
  if (L.tie_up) {
    for (int k = 0; k < L.H && j < L.H - 1 && s >= __ldg(L.bnd + j); ++k) ++j;
    for (int k = 0; k < L.H && j > 0 && s < __ldg(L.bnd + j - 1); ++k) --j;
  } else {
    for (int k = 0; k < L.H && j < L.H - 1 && s > __ldg(L.bnd + j); ++k) ++j;
    for (int k = 0; k < L.H && j > 0 && s <= __ldg(L.bnd + j - 1); ++k) --j;
  }
  return __ldg(L.rank2row + j);
}

// atan2(y, x) / (2 pi), in turns of a full circle, (-1/2, 1/2]: an odd
// polynomial of degree 15 for atan(t) / (2 pi) on t in [0, 1] and the octant
// symmetries atan(t) = pi/2 - atan(1/t), atan2(y, -x) = pi - atan2(y, x)
// (a quarter and a half turn).  The coefficients are those of a fit of
// atan(t) made here by iteratively re-weighted least squares on Chebyshev
// nodes (close to minimax; max error 3.7e-8 rad in exact arithmetic), divided
// by 2 pi and rounded to FP32; evaluated in FP32 the result is within about
// 3.7e-8 turns (2.3e-7 rad; the spacing of FP32 values near a quarter turn is
// 3e-8), i.e. 4e-5 columns of a 1024-wide image.  In turns, the column of a
// W-wide image is the turn count times W, exact for a power-of-two W.
__device__ __forceinline__ float atan2_turns(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  const float t = __fdividef(mn, mx);
  const float t2 = t * t;
  float p = -0.00064530195f;
  p = fmaf(p, t2, 0.0034795895f);
  p = fmaf(p, t2, -0.008898712f);
  p = fmaf(p, t2, 0.015346026f);
  p = fmaf(p, t2, -0.02213627f);
  p = fmaf(p, t2, 0.031745944f);
  p = fmaf(p, t2, -0.053046122f);
  p = fmaf(p, t2, 0.15915483f);
  float r = p * t;
  r = (ay > ax) ? 0.25f - r : r;
  r = (x < 0.f) ? 0.5f - r : r;
  return copysignf(r, y);
}

// round(turns * W) mod W for a power-of-two W = 2^k, by one FP32 addition:
// `magic` = 1.5 * 2^(23 - k) puts the sum in a binade whose spacing is
// exactly 1/W, so the addition itself rounds turns to the nearest multiple
// of 1/W (ties to even, like the conversion of the general form), and the
// low k bits of the sum's pattern are that multiple's count mod W (the sum is
// 2^(23 - k) (1 + 2^-1) + j / W, whose pattern ends in 2^22 + j, and 2^22 is
// a multiple of W).  |turns| <= 1/2, so the sum never leaves the binade; NaN
// gives column 0, as the conversion does.
__device__ __forceinline__ int col_from_turns_pow2(float turns, float magic, int W) {
  return __float_as_int(turns + magic) & (W - 1);
}

// Column from the continuous estimate u_c: u_c rounded to the nearest
// integer (floor(u_c + 1/2) except where u_c is exactly a half-integer, a tie;
// the same conversion as the branch-free form of project_px, so both forms
// decide alike) wrapped into [0, W).  Here |u_c| < W (atan2 in [-pi, pi] and
// |theta_lut| < pi), so one conditional add or subtract of W lands in [0, W);
// NaN converts to 0.
__device__ __forceinline__ int wrap_col(float uc, int W) {
  int u = __float2int_rn(uc);
  u = (u < 0) ? u + W : u;
  u = (u >= W) ? u - W : u;
  return u;
}

// Pi (Section 3.2) of point x into level L.  Returns true when the point lies
// inside the vertical field of view; (u, v) are always valid indices and r is
// the point's range from the receiver (|x - o| with the receiver offset o of
// the last fixed-point step).  FAST: the caller knows that L's inverse table
// is exact, that L has no azimuth offsets (theta_lut = 0) and that its width
// is a power of two, so the projection is one straight-line block and the
// column wraps by a mask: u_c rounded to the nearest integer (one conversion;
// it differs from floor(u_c + 1/2) only where u_c is exactly a half-integer,
// a tie) mod W, NaN -> 0.
template <bool R0, bool FAST = false>
__device__ __forceinline__ bool project_px(const DevLevel& L, float3 x, int proj_iters, int& u, int& v,
                                           float& r) {
  float s;
  if (!R0) {
    const float n2 = fmaf(x.x, x.x, fmaf(x.y, x.y, x.z * x.z));
    const float inv = rsqrtf(n2);
    s = x.z * inv;
    r = n2 * inv;
    v = row_from_sin<FAST>(L, s);
    const float turns = atan2_turns(x.y, x.x);
    if (FAST) {
      u = col_from_turns_pow2(turns, L.col_magic, L.W);
    } else {
      float uc = turns * L.wf;
      if (L.has_theta) uc -= __ldg(L.thu + v);
      u = wrap_col(uc, L.W);
    }
  } else {
    // receiver-offset fixed point on the column angle 2 pi u_c / W
    float turns = atan2_turns(x.y, x.x);
    float uc = turns * L.wf;
    s = 0.f;
    r = 0.f;
    v = 0;
    for (int k = 0; k < proj_iters; ++k) {
      float sa, ca;
      sincospif(uc * L.inv_w2, &sa, &ca);
      const float xp = fmaf(-L.r0, ca, x.x);
      const float yp = fmaf(-L.r0, sa, x.y);
      const float n2 = fmaf(xp, xp, fmaf(yp, yp, x.z * x.z));
      const float inv = rsqrtf(n2);
      s = x.z * inv;
      r = n2 * inv;
      v = row_from_sin<FAST>(L, s);
      turns = atan2_turns(yp, xp);
      uc = turns * L.wf;
      if (!FAST && L.has_theta) uc -= __ldg(L.thu + v);
    }
    u = FAST ? col_from_turns_pow2(turns, L.col_magic, L.W) : wrap_col(uc, L.W);
  }
  return (s >= L.s_lo) && (s <= L.s_hi);   // false for NaN
}

template <bool R0, bool FAST = false>
__device__ __forceinline__ bool project_px(const DevLevel& L, float3 x, int proj_iters, int& u, int& v) {
  float r;
  return project_px<R0, FAST>(L, x, proj_iters, u, v, r);
}

// 0 < r < inf, as one unsigned comparison on the bit pattern: the positive
// finite floats are exactly the patterns 1 .. 0x7f7fffff (NaN, +-inf, +-0 and
// negative values fall outside; checked over all 2^32 patterns).
__device__ __forceinline__ bool range_ok(float r) { return __float_as_uint(r) - 1u < 0x7f7fffffu; }

}  // namespace rimg
