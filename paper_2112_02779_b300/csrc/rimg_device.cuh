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
  const float2 cl = __ldg(L.cols + u);
  const float ct = fmaf(cl.x, rw.z, -cl.y * rw.w);
  const float st = fmaf(cl.y, rw.z, cl.x * rw.w);
  const float rc = r * rw.x;
  return make_float3(fmaf(rc, ct, L.r0 * cl.x), fmaf(rc, st, L.r0 * cl.y), r * rw.y);
}

// Eq. 4 in sin(elevation) space: the row whose elevation is nearest to that
// of a point with sin(elevation) = s.  The inverse table gives the rank at
// the bin's lower edge; walking across the (sorted) mid-elevation boundaries
// makes the result the exact argmin of the float tables.  Both walks are
// bounded by H.
__device__ __forceinline__ int row_from_sin(const DevLevel& L, float s) {
  int b = __float2int_rd((s - L.s_lo) * L.bin_scale);
  b = min(max(b, 0), L.n_bins - 1);
  int j = __ldg(L.bins + b);
  if (L.tie_up) {
    for (int k = 0; k < L.H && j < L.H - 1 && s >= __ldg(L.bnd + j); ++k) ++j;
    for (int k = 0; k < L.H && j > 0 && s < __ldg(L.bnd + j - 1); ++k) --j;
  } else {
    for (int k = 0; k < L.H && j < L.H - 1 && s > __ldg(L.bnd + j); ++k) ++j;
    for (int k = 0; k < L.H && j > 0 && s <= __ldg(L.bnd + j - 1); ++k) --j;
  }
  return __ldg(L.rank2row + j);
}

// Column from the continuous estimate u_c: floor(u_c + 1/2) wrapped into
// [0, W).  |u_c| < 2W always holds here (atan2 range plus |theta_lut| < pi).
__device__ __forceinline__ int wrap_col(float uc, int W) {
  int u = __float2int_rd(uc + 0.5f);
  u = (u < 0) ? u + W : u;
  u = (u >= W) ? u - W : u;
  return min(max(u, 0), W - 1);
}

// Pi (Section 3.2) of point x into level L.  Returns true when the point lies
// inside the vertical field of view; (u, v) are always valid indices.
template <bool R0>
__device__ __forceinline__ bool project_px(const DevLevel& L, float3 x, int proj_iters, int& u,
                                           int& v) {
  float s, uc;
  if (!R0) {
    const float n2 = fmaf(x.x, x.x, fmaf(x.y, x.y, x.z * x.z));
    s = x.z * rsqrtf(n2);
    v = row_from_sin(L, s);
    uc = fmaf(atan2f(x.y, x.x), L.w_over_2pi, -__ldg(L.thu + v));
  } else {
    // receiver-offset fixed point on the column angle 2 pi u_c / W
    uc = atan2f(x.y, x.x) * L.w_over_2pi;
    s = 0.f;
    v = 0;
    for (int k = 0; k < proj_iters; ++k) {
      float sa, ca;
      sincospif(uc * L.inv_w2, &sa, &ca);
      const float xp = fmaf(-L.r0, ca, x.x);
      const float yp = fmaf(-L.r0, sa, x.y);
      const float n2 = fmaf(xp, xp, fmaf(yp, yp, x.z * x.z));
      s = x.z * rsqrtf(n2);
      v = row_from_sin(L, s);
      uc = fmaf(atan2f(yp, xp), L.w_over_2pi, -__ldg(L.thu + v));
    }
  }
  u = wrap_col(uc, L.W);
  return (s >= L.s_lo) && (s <= L.s_hi);   // false for NaN
}

__device__ __forceinline__ bool range_ok(float r) { return r > 0.f && r < INFINITY; }

}  // namespace rimg
