// Host side of librimg: argument checking, sensor tables (step A1), workspace
// layouts, the multi-scale driver (step A9), the host-buffer variant and
// launch timing.  Every entry point is declared in include/rimg.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "rimg_internal.h"

namespace rimg {

namespace {

thread_local std::string g_last_error;

int cuda_fail(cudaError_t e, const char* where) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  g_last_error = buf;
  return RIMG_ERR_CUDA;
}

#define RIMG_CUDA(call)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
inline bool aligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) % kAlign) == 0; }

// Byte layout of one level's tables (see rimg_level).
struct LevelLayout {
  size_t rows, cols, thu, rank, bnd, bins, end;
  int n_bins;
};

LevelLayout level_layout(int Hl, int Wl, size_t start) {
  LevelLayout L{};
  L.n_bins = 64 * Hl;           // capacity; rimg_sensor_build uses as many as the table needs
  size_t o = align_up(start);
  L.rows = o; o = align_up(o + sizeof(float4) * Hl);
  L.cols = o; o = align_up(o + sizeof(float) * 2 * Wl);   // cos[W] then sin[W]
  L.thu = o; o = align_up(o + sizeof(float) * Hl);
  L.rank = o; o = align_up(o + sizeof(int) * Hl);
  L.bnd = o; o = align_up(o + sizeof(float) * std::max(1, Hl - 1));
  L.bins = o; o = align_up(o + sizeof(int4) * L.n_bins);
  L.end = o;
  return L;
}

int check_dims(int H, int W, int levels) {
  if (H <= 0 || W <= 0 || levels < 1 || levels > RIMG_MAX_LEVELS) return RIMG_ERR_INVALID_ARG;
  if ((H >> (levels - 1)) < 2) return RIMG_ERR_SIZE;
  if ((H % (1 << (levels - 1))) != 0) return RIMG_ERR_SIZE;
  if ((W % (4 << (levels - 1))) != 0) return RIMG_ERR_SIZE;
  return RIMG_OK;
}

int check_sensor(const rimg_sensor* s) {
  if (!s || !s->d_tables) return RIMG_ERR_INVALID_ARG;
  int rc = check_dims(s->H, s->W, s->levels);
  if (rc) return rc;
  for (int l = 0; l < s->levels; ++l)
    if (s->level[l].H != (s->H >> l) || s->level[l].W != (s->W >> l)) return RIMG_ERR_INVALID_ARG;
  return RIMG_OK;
}

int check_params(const rimg_params* p) {
  if (!p) return RIMG_ERR_INVALID_ARG;
  if (!std::isfinite(p->huber_delta) || !std::isfinite(p->max_corr_dist)) return RIMG_ERR_INVALID_ARG;
  if (!(p->normal_rel_jump >= 0.f && p->normal_rel_jump < 0.5f)) return RIMG_ERR_INVALID_ARG;
  if (p->proj_iters < 1 || p->proj_iters > 16) return RIMG_ERR_INVALID_ARG;
  if (p->streams < 1 || p->streams > 4) return RIMG_ERR_INVALID_ARG;
  if (p->normal_method != 0 && p->normal_method != 1) return RIMG_ERR_INVALID_ARG;
  return RIMG_OK;
}

// ---- launch timing ----
struct Prof {
  std::mutex mu;
  bool on = false;
  int cap = 0, n = 0;
  bool open = false;
  std::vector<cudaEvent_t> ev0, ev1;
  std::vector<int> kid, lvl, np;
} g_prof;

}  // namespace

void prof_before(cudaStream_t st, int kernel, int level, int n) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (!g_prof.on || g_prof.n >= g_prof.cap) return;
  const int i = g_prof.n;
  cudaEventRecord(g_prof.ev0[i], st);
  g_prof.kid[i] = kernel;
  g_prof.lvl[i] = level;
  g_prof.np[i] = n;
  g_prof.open = true;
}

void prof_after(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (!g_prof.on || !g_prof.open) return;
  cudaEventRecord(g_prof.ev1[g_prof.n], st);
  g_prof.open = false;
  ++g_prof.n;
}

DevLevel dev_level(const rimg_sensor* s, int l) {
  const rimg_level& L = s->level[l];
  const char* base = static_cast<const char*>(s->d_tables);
  DevLevel d;
  d.rows = reinterpret_cast<const float4*>(base + L.off_rows);
  d.cos_u = reinterpret_cast<const float*>(base + L.off_cols);
  d.sin_u = reinterpret_cast<const float*>(base + L.off_cols + sizeof(float) * L.W);
  d.thu = reinterpret_cast<const float*>(base + L.off_thu);
  d.rank2row = reinterpret_cast<const int*>(base + L.off_rank);
  d.bnd = reinterpret_cast<const float*>(base + L.off_bnd);
  d.bins = reinterpret_cast<const int4*>(base + L.off_bins);
  d.H = L.H;
  d.W = L.W;
  d.n_bins = L.n_bins;
  d.tie_up = L.tie_up;
  d.bins_exact = L.bins_exact;
  d.has_theta = L.has_theta;
  d.s_lo = L.s_lo;
  d.s_hi = L.s_hi;
  d.bin_scale = L.bin_scale;
  d.wf = (float)L.W;
  d.r0 = s->r0;
  d.inv_w2 = 2.0f / (float)L.W;
  d.col_magic = (float)(1.5 * 8388608.0 / (double)L.W);
  return d;
}

// ---- workspace layouts ----
namespace {

struct IcpWs {
  size_t counters, partials, sums, end;
};

IcpWs icp_ws(int H, int n_pairs, size_t start) {
  IcpWs w{};
  size_t o = align_up(start);
  w.counters = o; o = align_up(o + sizeof(unsigned) * (size_t)std::max(n_pairs, 1));
  w.sums = o; o = align_up(o + sizeof(double) * kRedStride * (size_t)std::max(n_pairs, 1));
  w.partials = o; o = align_up(o + sizeof(float) * kRedStride * (size_t)H * std::max(n_pairs, 1));
  w.end = o;
  return w;
}

struct RegWs {
  size_t src_lvl[RIMG_MAX_LEVELS];   // level >= 1 source ranges
  size_t dst_lvl[RIMG_MAX_LEVELS];   // level >= 1 target ranges (read by the distance gate)
  size_t planes[RIMG_MAX_LEVELS];    // target planes, all levels
  IcpWs icp;
  size_t end;
};

RegWs reg_ws(int H, int W, int n_pairs, int levels, size_t start) {
  RegWs r{};
  size_t o = align_up(start);
  const size_t n = (size_t)std::max(n_pairs, 0);
  for (int l = 0; l < levels; ++l) {
    const size_t Nl = (size_t)(H >> l) * (W >> l);
    if (l >= 1) {
      r.src_lvl[l] = o; o = align_up(o + sizeof(float) * Nl * n);
      r.dst_lvl[l] = o; o = align_up(o + sizeof(float) * Nl * n);
    }
    r.planes[l] = o; o = align_up(o + sizeof(float4) * Nl * n);
  }
  r.icp = icp_ws(H, n_pairs, o);
  r.end = r.icp.end;
  return r;
}

struct IcpScratch {
  unsigned* counters;   // [n_pairs], zero between launches
  double* sums;         // [n_pairs][32]
  float* partials;      // [n_pairs][H][32] (at most H blocks per pair)
};

IcpScratch icp_scratch(char* ws, const IcpWs& w, int H, int p0) {
  IcpScratch s;
  s.counters = reinterpret_cast<unsigned*>(ws + w.counters) + p0;
  s.sums = reinterpret_cast<double*>(ws + w.sums) + (size_t)p0 * kRedStride;
  s.partials = reinterpret_cast<float*>(ws + w.partials) + (size_t)p0 * H * kRedStride;
  return s;
}

int icp_launch(const rimg_sensor* src, const rimg_sensor* dst, int level, int n_pairs,
               const float* src_range_l, const float* dst_planes_l, const float* dst_range_l,
               double* pose, const rimg_params* p, int update, double* out29, int32_t* assoc,
               int* status, const IcpScratch& w, cudaStream_t st, int force_threads = 0, int force_bpp = 0) {
  if (p->max_corr_dist > 0.f && !dst_range_l) return RIMG_ERR_INVALID_ARG;
  IcpLaunch a{};
  a.src = dev_level(src, level);
  a.dst = dev_level(dst, level);
  a.n_pairs = n_pairs;
  a.src_range = src_range_l;
  a.dst_planes = reinterpret_cast<const float4*>(dst_planes_l);
  a.dst_range = dst_range_l;
  a.pose = pose;
  a.out29 = out29;
  a.assoc = assoc;
  a.status = status;
  a.partials = w.partials;
  a.counters = w.counters;
  a.sums = w.sums;
  a.huber_delta = p->huber_delta;
  a.max_corr_dist = p->max_corr_dist;
  a.proj_iters = p->proj_iters;
  a.kahan = p->kahan;
  a.update = update;
  icp_grid(a.src.H, a.src.W, n_pairs, &a.bpp, &a.rows_per_block, &a.threads);
  if (force_threads > 0) {   // the autotuner's candidates
    const int b = std::min(std::max(force_bpp, 1), a.src.H);
    a.rows_per_block = (a.src.H + b - 1) / b;
    a.bpp = (a.src.H + a.rows_per_block - 1) / a.rows_per_block;
    a.threads = force_threads;
  }
  prof_before(st, K_ICP, level, n_pairs);
  cudaError_t e = launch_icp(a, st);
  prof_after(st);
  if (e != cudaSuccess) return cuda_fail(e, "icp step kernel");
  if (update) {
    prof_before(st, K_SOLVE, level, n_pairs);
    e = launch_solve(n_pairs, a.sums, pose, status, st);
    prof_after(st);
    if (e != cudaSuccess) return cuda_fail(e, "solve kernel");
  }
  return RIMG_OK;
}

// All `iters` Gauss-Newton steps of a level in one launch: one block per
// pair (k_icp_iters), or with cluster = 2, 4 or 8 a thread-block cluster of
// that many blocks per pair (k_icp_cluster; not with the distance gate, which
// keeps one block per pair where the pair fits one and per-iteration launches
// elsewhere).
int icp_iters_launch(const rimg_sensor* src, const rimg_sensor* dst, int level, int n_pairs,
                     const float* src_range_l, const float* dst_planes_l, const float* dst_range_l, double* pose,
                     const rimg_params* p, int* status, const IcpScratch& w, int iters, cudaStream_t st,
                     int cluster = 1) {
  if (p->max_corr_dist > 0.f && !dst_range_l) return RIMG_ERR_INVALID_ARG;
  IcpLaunch a{};
  a.src = dev_level(src, level);
  a.dst = dev_level(dst, level);
  a.n_pairs = n_pairs;
  a.src_range = src_range_l;
  a.dst_planes = reinterpret_cast<const float4*>(dst_planes_l);
  a.dst_range = dst_range_l;
  a.pose = pose;
  a.status = status;
  a.partials = w.partials;
  a.counters = w.counters;
  a.sums = w.sums;
  a.huber_delta = p->huber_delta;
  a.max_corr_dist = p->max_corr_dist;
  a.proj_iters = p->proj_iters;
  a.kahan = p->kahan;
  a.update = 1;
  const bool on_cluster = cluster > 1 && p->max_corr_dist <= 0.f;
  if (!on_cluster && !icp_iters_fits(a.src.H, a.src.W)) {
    for (int it = 0; it < iters; ++it) {
      int rc = icp_launch(src, dst, level, n_pairs, src_range_l, dst_planes_l, dst_range_l, pose, p, 1, nullptr,
                          nullptr, status, w, st);
      if (rc) return rc;
    }
    return RIMG_OK;
  }
  prof_before(st, on_cluster ? K_ICP_CLUSTER : K_ICP_ITERS, level, n_pairs);
  cudaError_t e = on_cluster ? launch_icp_cluster(a, iters, cluster, st) : launch_icp_iters(a, iters, st);
  prof_after(st);
  if (e != cudaSuccess) return cuda_fail(e, "icp iterations kernel");
  return RIMG_OK;
}

// Per-level buffers of the pairs [p0, p0 + n) of a registration workspace.
struct SliceBufs {
  float* planes[RIMG_MAX_LEVELS];
  float* srcl[RIMG_MAX_LEVELS];
  float* dstl[RIMG_MAX_LEVELS];
};

SliceBufs slice_bufs(char* ws, const RegWs& R, int H, int W, int levels, int p0) {
  SliceBufs b{};
  for (int l = 0; l < levels; ++l) {
    const size_t Nl = (size_t)(H >> l) * (W >> l);
    b.planes[l] = reinterpret_cast<float*>(ws + R.planes[l]) + 4 * Nl * p0;
    if (l >= 1) {
      b.srcl[l] = reinterpret_cast<float*>(ws + R.src_lvl[l]) + Nl * p0;
      b.dstl[l] = reinterpret_cast<float*>(ws + R.dst_lvl[l]) + Nl * p0;
    }
  }
  return b;
}

// Normals + target plane pyramid and source (and, for the gate, target)
// range pyramids of n pairs whose ranges start at src_range / dst_range.
int prep_slice(const rimg_sensor* src, const rimg_sensor* dst, int n, const float* src_range, const float* dst_range,
               int levels, const rimg_params* p, const SliceBufs& b, cudaStream_t st) {
  const int H = src->H, W = src->W;
  float* planes[RIMG_MAX_LEVELS];
  float* srcl[RIMG_MAX_LEVELS];
  float* dstl[RIMG_MAX_LEVELS];
  for (int l = 0; l < RIMG_MAX_LEVELS; ++l) { planes[l] = b.planes[l]; srcl[l] = b.srcl[l]; dstl[l] = b.dstl[l]; }
  // rimg_normals writes every level of dst's table set; register may use fewer
  // levels than the sensor has, so build a view limited to `levels`.
  rimg_sensor dview = *dst;
  dview.levels = levels;
  prof_before(st, K_NORMALS, 0, n);
  cudaError_t e = launch_normals(&dview, n, dst_range, p->normal_rel_jump, p->normal_method, planes, nullptr, st);
  prof_after(st);
  if (e != cudaSuccess) return cuda_fail(e, "normals kernel");
  if (levels > 1) {
    prof_before(st, K_SRC_PYRAMID, 1, n);
    e = launch_pyramid(n, H, W, levels, 1, src_range, srcl, st);
    prof_after(st);
    if (e != cudaSuccess) return cuda_fail(e, "pyramid kernel");
    if (p->max_corr_dist > 0.f) {   // the distance gate reads the target ranges of every level
      prof_before(st, K_PYRAMID, 1, n);
      e = launch_pyramid(n, H, W, levels, 1, dst_range, dstl, st);
      prof_after(st);
      if (e != cudaSuccess) return cuda_fail(e, "pyramid kernel");
    }
  }
  return RIMG_OK;
}

// The pairs [p0, p0 + n) of a batch: status cleared, T_out initialised, the
// completion counters zeroed and the pyramids built, on one stream.
int slice_begin(const rimg_sensor* src, const rimg_sensor* dst, int p0, int n, const float* src_range,
                const float* dst_range, const double* T_init, double* T_out, int levels, const rimg_params* p,
                int* status, char* ws, const RegWs& R, cudaStream_t st) {
  const int H = src->H, W = src->W;
  const size_t N = (size_t)H * W;
  src_range += p0 * N;
  dst_range += p0 * N;
  T_init += 16 * (size_t)p0;
  T_out += 16 * (size_t)p0;
  if (status) RIMG_CUDA(cudaMemsetAsync(status + p0, 0, sizeof(int) * n, st));
  if (T_out != T_init)
    RIMG_CUDA(cudaMemcpyAsync(T_out, T_init, sizeof(double) * 16 * n, cudaMemcpyDeviceToDevice, st));
  const IcpScratch scr = icp_scratch(ws, R.icp, H, p0);
  RIMG_CUDA(cudaMemsetAsync(scr.counters, 0, sizeof(unsigned) * n, st));
  const SliceBufs b = slice_bufs(ws, R, H, W, levels, p0);
  return prep_slice(src, dst, n, src_range, dst_range, levels, p, b, st);
}

// Gauss-Newton steps of the schedule levels k >= k_first for the pairs
// [p0, p0 + n) (after slice_begin): a level whose pair fits one block runs all
// its iterations in one launch unless the autotuner chose per-iteration
// launches for it; other levels run one association and one solve launch per
// iteration.
int slice_levels(const rimg_sensor* src, const rimg_sensor* dst, int p0, int n, const float* src_range,
                 const float* dst_range, double* T_out, int levels, const int* iters, const rimg_params* p,
                 int* status, char* ws, const RegWs& R, int k_first, cudaStream_t st) {
  const int H = src->H, W = src->W;
  const size_t N = (size_t)H * W;
  src_range += p0 * N;
  dst_range += p0 * N;
  T_out += 16 * (size_t)p0;
  if (status) status += p0;
  const IcpScratch scr = icp_scratch(ws, R.icp, H, p0);
  const SliceBufs b = slice_bufs(ws, R, H, W, levels, p0);
  const bool gate = p->max_corr_dist > 0.f;
  for (int k = k_first; k < levels; ++k) {
    const int l = levels - 1 - k;
    const float* s_l = (l == 0) ? src_range : b.srcl[l];
    const float* d_l = gate ? ((l == 0) ? dst_range : b.dstl[l]) : nullptr;
    const int sched = icp_sched(H >> l, W >> l, n);
    if (iters[k] > 0 && sched >= 1) {
      int rc = icp_iters_launch(src, dst, l, n, s_l, b.planes[l], d_l, T_out, p, status, scr, iters[k], st, sched);
      if (rc) return rc;
      continue;
    }
    for (int it = 0; it < iters[k]; ++it) {
      int rc = icp_launch(src, dst, l, n, s_l, b.planes[l], d_l, T_out, p, 1, nullptr, nullptr, status, scr, st);
      if (rc) return rc;
    }
  }
  return RIMG_OK;
}

// Registration of the pairs [p0, p0 + n) of a batch on one stream; every
// buffer is addressed through the per-pair offsets of that range.
int register_slice(const rimg_sensor* src, const rimg_sensor* dst, int p0, int n, const float* src_range,
                   const float* dst_range, const double* T_init, double* T_out, int levels, const int* iters,
                   const rimg_params* p, int* status, char* ws, const RegWs& R, cudaStream_t st) {
  int rc = slice_begin(src, dst, p0, n, src_range, dst_range, T_init, T_out, levels, p, status, ws, R, st);
  if (rc) return rc;
  return slice_levels(src, dst, p0, n, src_range, dst_range, T_out, levels, iters, p, status, ws, R, 0, st);
}

// Internal streams for concurrent sub-batches, created once per device.
constexpr int kMaxSubStreams = 4;
struct SubStreams {
  std::mutex mu;
  int device = -1;
  cudaStream_t s[kMaxSubStreams] = {};
  cudaEvent_t fork = nullptr, join[kMaxSubStreams] = {};
} g_sub;

// Pairs are independent, so a batch splits into p->streams sub-batches that
// run concurrently on internal streams forked from (and joined back into)
// `st`: one sub-batch's FP64 solves, launch gaps and small coarse-level
// kernels overlap another's work.
// Whether the target's level l projects with the branch-free form (exact
// inverse table, no azimuth offsets, power-of-two width), which the queue
// kernel is built for.
bool fast_level(const rimg_sensor* dst, int l) {
  const rimg_level& L = dst->level[l];
  return L.bins_exact && !L.has_theta && L.W > 0 && (L.W & (L.W - 1)) == 0;
}

// The number of leading schedule levels (coarsest first) that can run in the
// persistent queue kernel: levels whose pair fits one block, with the
// branch-free projection, no distance gate, and the one-block schedule for
// every sub-batch size in `slice_sizes` (see rimg_autotune).
int queue_prefix_of(const rimg_sensor* src, const rimg_sensor* dst, int levels, const rimg_params* p,
                    const std::vector<int>& slice_sizes) {
  if (p->max_corr_dist > 0.f) return 0;
  int k = 0;
  for (; k < levels; ++k) {
    const int l = levels - 1 - k;
    const int Hl = src->H >> l, Wl = src->W >> l;
    if (!queue_level_ok(Hl, Wl) || !fast_level(dst, l)) break;
    bool fused = true;
    for (int n : slice_sizes) fused = fused && icp_sched(Hl, Wl, n) == 1;
    if (!fused) break;
  }
  return k;
}

int register_device(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs, const float* src_range,
                    const float* dst_range, const double* T_init, double* T_out, int levels,
                    const int* iters, const rimg_params* p, int* status, char* ws,
                    const RegWs& R, cudaStream_t st) {
  int S = std::min(std::max(p->streams, 1), kMaxSubStreams);
  if (n_pairs < 32 * S) S = std::max(1, n_pairs / 32);
  if (S <= 1) return register_slice(src, dst, 0, n_pairs, src_range, dst_range, T_init, T_out, levels, iters,
                                    p, status, ws, R, st);
  std::lock_guard<std::mutex> lk(g_sub.mu);
  int dev = 0;
  RIMG_CUDA(cudaGetDevice(&dev));
  if (g_sub.device != dev) {
    for (int i = 0; i < kMaxSubStreams; ++i) {
      RIMG_CUDA(cudaStreamCreateWithFlags(&g_sub.s[i], cudaStreamNonBlocking));
      RIMG_CUDA(cudaEventCreateWithFlags(&g_sub.join[i], cudaEventDisableTiming));
    }
    RIMG_CUDA(cudaEventCreateWithFlags(&g_sub.fork, cudaEventDisableTiming));
    g_sub.device = dev;
  }
  RIMG_CUDA(cudaEventRecord(g_sub.fork, st));
  int p0 = 0;
  for (int i = 0; i < S; ++i) {
    const int n = n_pairs / S + (i < n_pairs % S ? 1 : 0);
    RIMG_CUDA(cudaStreamWaitEvent(g_sub.s[i], g_sub.fork, 0));
    int rc = register_slice(src, dst, p0, n, src_range, dst_range, T_init, T_out, levels, iters, p, status, ws, R,
                            g_sub.s[i]);
    if (rc) return rc;
    RIMG_CUDA(cudaEventRecord(g_sub.join[i], g_sub.s[i]));
    RIMG_CUDA(cudaStreamWaitEvent(st, g_sub.join[i], 0));
    p0 += n;
  }
  return RIMG_OK;
}

// ---- groups of batches (uneven sizes) ----
struct GroupWs {
  std::vector<size_t> off;    // byte offset of each group's registration workspace
  std::vector<RegWs> reg;
  size_t queue = 0;           // QueueGroup[n_groups] for the persistent small-level kernel
  size_t queue_counters = 0;  // unsigned[4]: one item counter per kernel form (receiver offset x Kahan)
  size_t end = 0;
};

GroupWs groups_ws(int n_groups, const rimg_group* g) {
  GroupWs w;
  size_t o = 0;
  for (int i = 0; i < n_groups; ++i) {
    o = align_up(o);
    w.off.push_back(o);
    w.reg.push_back(reg_ws(g[i].src->H, g[i].src->W, g[i].n_pairs, g[i].levels, 0));
    o += w.reg.back().end;
  }
  w.queue = align_up(o);
  o = w.queue + sizeof(QueueGroup) * (size_t)std::max(n_groups, 1);
  w.queue_counters = align_up(o);
  o = w.queue_counters + 4 * sizeof(unsigned);
  w.end = align_up(o);
  return w;
}

// The queued prefix of a group (queue_prefix_of over its sub-batch sizes).
int queue_prefix(const rimg_group& g, const std::vector<int>& slice_sizes) {
  if (g.n_pairs == 0) return 0;
  return queue_prefix_of(g.src, g.dst, g.levels, g.params, slice_sizes);
}

struct Slice {
  int group, p0, n;
  double work;
};

// Slices of every group: each group splits into params->streams sub-batches
// of at least 32 pairs; largest work first.
std::vector<Slice> group_slices(int n_groups, const rimg_group* g) {
  std::vector<Slice> out;
  for (int i = 0; i < n_groups; ++i) {
    const int n = g[i].n_pairs;
    if (n == 0) continue;
    int S = std::min(std::max(g[i].params->streams, 1), 4);
    if (n < 32 * S) S = std::max(1, n / 32);
    int p0 = 0;
    for (int k = 0; k < S; ++k) {
      const int c = n / S + (k < n % S ? 1 : 0);
      int iters = 0;
      for (int l = 0; l < g[i].levels; ++l) iters += g[i].iters[l];
      out.push_back(Slice{i, p0, c, (double)c * g[i].src->H * g[i].src->W * iters});
      p0 += c;
    }
  }
  std::sort(out.begin(), out.end(), [](const Slice& a, const Slice& b) { return a.work > b.work; });
  return out;
}

constexpr int kGroupStreams = 8;
struct GroupStreams {
  std::mutex mu;
  int device = -1;
  cudaStream_t s[kGroupStreams] = {};
  cudaEvent_t fork = nullptr, join[kGroupStreams] = {};
} g_grp;

int check_register_args(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs, int levels,
                        const int* iters, const rimg_params* p) {
  int rc = check_sensor(src);
  if (rc) return rc;
  rc = check_sensor(dst);
  if (rc) return rc;
  if ((rc = check_params(p))) return rc;
  if (n_pairs < 0 || !iters) return RIMG_ERR_INVALID_ARG;
  if (src->H != dst->H || src->W != dst->W) return RIMG_ERR_MISMATCH;
  if (levels < 1 || levels > src->levels || levels > dst->levels) return RIMG_ERR_INVALID_ARG;
  for (int k = 0; k < levels; ++k)
    if (iters[k] < 0 || iters[k] > 100000) return RIMG_ERR_INVALID_ARG;
  return RIMG_OK;
}

// Host-buffer variant: a copy stream, a pool of compute streams and events,
// created once per device.
constexpr int kHostStreams = 4;
constexpr int kHostEvents = 64;
struct HostPipe {
  std::mutex mu;
  int device = -1;
  cudaStream_t copy = nullptr;
  cudaStream_t comp[kHostStreams] = {};
  cudaEvent_t start = nullptr;
  cudaEvent_t loaded[kHostEvents] = {};
  cudaEvent_t done[kHostStreams] = {};
} g_pipe;

struct HostWs {
  size_t src, dst, T, S;
  RegWs reg;
};

HostWs host_ws(int H, int W, int n_pairs, int levels) {
  HostWs h{};
  const size_t N = (size_t)H * W, n = (size_t)std::max(n_pairs, 1);
  size_t o = 0;
  h.src = o; o = align_up(o + sizeof(float) * N * n);
  h.dst = o; o = align_up(o + sizeof(float) * N * n);
  h.T = o; o = align_up(o + sizeof(double) * 16 * n);
  h.S = o; o = align_up(o + sizeof(int) * n);
  h.reg = reg_ws(H, W, n_pairs, levels, o);
  return h;
}
}  // namespace
}  // namespace rimg

using namespace rimg;

extern "C" {

int rimg_default_params(rimg_params* p) {
  if (!p) return RIMG_ERR_INVALID_ARG;
  p->huber_delta = 0.5f;
  p->max_corr_dist = 0.f;
  p->normal_rel_jump = 0.1f;
  p->proj_iters = 3;
  p->kahan = 1;
  p->streams = 2;
  p->normal_method = 0;
  return RIMG_OK;
}

const char* rimg_status_string(int code) {
  switch (code) {
    case RIMG_OK: return "ok";
    case RIMG_ERR_INVALID_ARG: return "invalid argument";
    case RIMG_ERR_LUT: return "elevation table not strictly monotone or out of range";
    case RIMG_ERR_SIZE: return "image size incompatible with the pyramid";
    case RIMG_ERR_WORKSPACE: return "workspace too small or misaligned";
    case RIMG_ERR_CUDA: return "CUDA error";
    case RIMG_ERR_MISMATCH: return "source and target sensors disagree";
    default: return "unknown status";
  }
}

const char* rimg_last_error(void) { return g_last_error.c_str(); }

int rimg_sensor_table_bytes(int H, int W, int levels, size_t* bytes) {
  if (!bytes) return RIMG_ERR_INVALID_ARG;
  int rc = check_dims(H, W, levels);
  if (rc) return rc;
  size_t o = 0;
  for (int l = 0; l < levels; ++l) o = level_layout(H >> l, W >> l, o).end;
  *bytes = o;
  return RIMG_OK;
}

int rimg_sensor_build(int H, int W, int levels, const double* phi_lut, const double* theta_lut,
                      double r0, void* d_tables, size_t table_bytes, rimg_sensor* out) {
  if (!phi_lut || !theta_lut || !d_tables || !out) return RIMG_ERR_INVALID_ARG;
  int rc = check_dims(H, W, levels);
  if (rc) return rc;
  if (!std::isfinite(r0) || r0 < 0.0) return RIMG_ERR_INVALID_ARG;
  if (!aligned(d_tables)) return RIMG_ERR_WORKSPACE;
  const double kHalfPi = 1.5707963267948966, kPi = 3.141592653589793;
  for (int v = 0; v < H; ++v) {
    if (!std::isfinite(phi_lut[v]) || std::fabs(phi_lut[v]) >= kHalfPi) return RIMG_ERR_LUT;
    if (!std::isfinite(theta_lut[v]) || std::fabs(theta_lut[v]) >= kPi) return RIMG_ERR_LUT;
  }
  const bool desc = H > 1 && phi_lut[1] < phi_lut[0];
  for (int v = 1; v < H; ++v) {
    if (desc ? !(phi_lut[v] < phi_lut[v - 1]) : !(phi_lut[v] > phi_lut[v - 1])) return RIMG_ERR_LUT;
  }
  size_t need = 0;
  rimg_sensor_table_bytes(H, W, levels, &need);
  if (table_bytes < need) return RIMG_ERR_WORKSPACE;

  rimg_sensor s{};
  s.H = H;
  s.W = W;
  s.levels = levels;
  s.r0 = (float)r0;
  s.d_tables = d_tables;
  s.table_bytes = need;
  std::vector<unsigned char> buf(need, 0);
  size_t o = 0;
  for (int l = 0; l < levels; ++l) {
    const int Hl = H >> l, Wl = W >> l;
    const LevelLayout L = level_layout(Hl, Wl, o);
    o = L.end;
    std::vector<double> ph(Hl), th(Hl);
    for (int v = 0; v < Hl; ++v) {
      ph[v] = phi_lut[v << l];
      th[v] = theta_lut[v << l];
    }
    float4* rows = reinterpret_cast<float4*>(buf.data() + L.rows);
    float* cosu = reinterpret_cast<float*>(buf.data() + L.cols);
    float* sinu = cosu + Wl;
    float* thu = reinterpret_cast<float*>(buf.data() + L.thu);
    int* rank = reinterpret_cast<int*>(buf.data() + L.rank);
    float* bnd = reinterpret_cast<float*>(buf.data() + L.bnd);
    int4* bins = reinterpret_cast<int4*>(buf.data() + L.bins);
    bool any_theta = false;
    for (int v = 0; v < Hl; ++v) {
      rows[v] = make_float4((float)std::cos(ph[v]), (float)std::sin(ph[v]), (float)std::cos(th[v]),
                            (float)std::sin(th[v]));
      thu[v] = (float)(th[v] * Wl / (2.0 * kPi));
      any_theta |= th[v] != 0.0;
    }
    for (int u = 0; u < Wl; ++u) {
      const double a = 2.0 * kPi * ((double)u / (double)Wl);
      cosu[u] = (float)std::cos(a);
      sinu[u] = (float)std::sin(a);
    }
    // rank j = j-th smallest elevation
    std::vector<int> order(Hl);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return ph[a] < ph[b]; });
    for (int j = 0; j < Hl; ++j) rank[j] = order[j];
    std::vector<double> asc(Hl);
    for (int j = 0; j < Hl; ++j) asc[j] = ph[order[j]];
    for (int j = 0; j + 1 < Hl; ++j) bnd[j] = (float)std::sin(0.5 * (asc[j] + asc[j + 1]));
    double lo = asc[0] - 0.5 * (asc[1] - asc[0]);
    double hi = asc[Hl - 1] + 0.5 * (asc[Hl - 1] - asc[Hl - 2]);
    lo = std::max(lo, -kHalfPi);
    hi = std::min(hi, kHalfPi);
    rimg_level& lv = s.level[l];
    lv.H = Hl;
    lv.W = Wl;
    lv.tie_up = desc ? 1 : 0;
    lv.has_theta = any_theta ? 1 : 0;
    lv.s_lo = (float)std::sin(lo);
    lv.s_hi = (float)std::sin(hi);
    lv.w_over_2pi = (float)((double)Wl / (2.0 * kPi));
    // Bins narrower than the smallest gap between row boundaries hold at most
    // one boundary each; then one comparison inside the bin decides the row.
    const double range = (double)lv.s_hi - (double)lv.s_lo;
    double min_gap = range;
    for (int j = 0; j + 2 < Hl; ++j) min_gap = std::min(min_gap, (double)bnd[j + 1] - (double)bnd[j]);
    long long nb = (min_gap > 0.0) ? (long long)std::ceil(range / min_gap) + 2 : (long long)L.n_bins;
    nb = std::max<long long>(nb, 2LL * Hl);
    nb = std::min<long long>(nb, (long long)L.n_bins);
    lv.n_bins = (int)nb;
    lv.bin_scale = (float)((double)nb / range);
    bool exact = true;
    for (int b = 0; b < lv.n_bins; ++b) {
      const double e0 = (double)lv.s_lo + (double)b / (double)lv.bin_scale;
      const double e1 = (double)lv.s_lo + (double)(b + 1) / (double)lv.bin_scale;
      int j = 0;   // rank at the lower edge (ties follow the device's comparison)
      while (j < Hl - 1 && (desc ? (double)bnd[j] <= e0 : (double)bnd[j] < e0)) ++j;
      int inside = 0;
      while (j + inside < Hl - 1 && (double)bnd[j + inside] < e1) ++inside;
      if (inside > 1) exact = false;
      float bb = (inside >= 1) ? bnd[j] : INFINITY;
      // the device tests s > bb; with tie_up a tie goes to the row above the
      // boundary, i.e. s >= bnd, which is s > (the largest float below bnd)
      if (desc && inside >= 1) bb = std::nextafter(bb, -INFINITY);
      int bits;
      std::memcpy(&bits, &bb, sizeof(bits));
      bins[b] = make_int4(rank[j], rank[std::min(j + 1, Hl - 1)], bits, j);
    }
    lv.bins_exact = exact ? 1 : 0;
    lv.off_rows = L.rows;
    lv.off_cols = L.cols;
    lv.off_thu = L.thu;
    lv.off_rank = L.rank;
    lv.off_bnd = L.bnd;
    lv.off_bins = L.bins;
  }
  RIMG_CUDA(cudaMemcpy(d_tables, buf.data(), need, cudaMemcpyHostToDevice));
  *out = s;
  return RIMG_OK;
}

int rimg_unproject(const rimg_sensor* s, int level, int n_images, const float* range, float* xyz,
                   uint8_t* mask, void* stream) {
  int rc = check_sensor(s);
  if (rc) return rc;
  if (level < 0 || level >= s->levels || n_images < 0) return RIMG_ERR_INVALID_ARG;
  if (n_images == 0) return RIMG_OK;
  if (!range || !xyz) return RIMG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_before(st, K_UNPROJECT, level, n_images);
  cudaError_t e = launch_unproject(dev_level(s, level), n_images, range, xyz, mask, st);
  prof_after(st);
  if (e != cudaSuccess) return cuda_fail(e, "unproject kernel");
  return RIMG_OK;
}

int rimg_center_init(const rimg_sensor* src, const rimg_sensor* dst, int level, int n_pairs, const float* src_range_l,
                     const float* dst_range_l, double* T_out, int* status, void* stream) {
  int rc = check_sensor(src);
  if (rc) return rc;
  if ((rc = check_sensor(dst))) return rc;
  if (level < 0 || level >= src->levels || level >= dst->levels || n_pairs < 0) return RIMG_ERR_INVALID_ARG;
  if (n_pairs == 0) return RIMG_OK;
  if (!src_range_l || !dst_range_l || !T_out) return RIMG_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(src_range_l) % 16) || (reinterpret_cast<uintptr_t>(dst_range_l) % 16) ||
      (reinterpret_cast<uintptr_t>(T_out) % 8))
    return RIMG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_center(dev_level(src, level), dev_level(dst, level), n_pairs, src_range_l, dst_range_l, T_out,
                                status, st);
  if (e != cudaSuccess) return cuda_fail(e, "centre kernel");
  return RIMG_OK;
}

int rimg_sdf_integrate(const rimg_sensor* s, int level, int n_scans, const float* range_l,
                       const double* T_world_to_sensor, const rimg_grid* grid, float trunc, float* sdf,
                       float* weight, const rimg_params* p, void* stream) {
  int rc = check_sensor(s);
  if (rc) return rc;
  if (level < 0 || level >= s->levels || n_scans < 0 || !grid) return RIMG_ERR_INVALID_ARG;
  if (grid->nx < 0 || grid->ny < 0 || grid->nz < 0) return RIMG_ERR_INVALID_ARG;
  if (!(grid->voxel > 0.f) || !std::isfinite(grid->voxel) || !std::isfinite(trunc)) return RIMG_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(grid->origin[a])) return RIMG_ERR_INVALID_ARG;
  if ((long long)grid->nx * grid->ny * grid->nz > ((long long)1 << 40)) return RIMG_ERR_SIZE;
  if (p && (rc = check_params(p))) return rc;
  const long long n_vox = (long long)grid->nx * grid->ny * grid->nz;
  if (n_scans == 0 || n_vox == 0) return RIMG_OK;
  if (!range_l || !T_world_to_sensor || !sdf || !weight) return RIMG_ERR_INVALID_ARG;
  rimg_params d;
  rimg_default_params(&d);
  const int iters = p ? p->proj_iters : d.proj_iters;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_before(st, K_SDF, level, n_scans);
  cudaError_t e = launch_sdf(dev_level(s, level), n_scans, range_l, T_world_to_sensor, grid->nx, grid->ny, grid->nz,
                             grid->origin[0], grid->origin[1], grid->origin[2], grid->voxel, trunc, iters, sdf,
                             weight, st);
  prof_after(st);
  if (e != cudaSuccess) return cuda_fail(e, "sdf kernel");
  return RIMG_OK;
}

int rimg_points_to_range(const rimg_sensor* s, int level, int n_clouds, int max_points, const float* xyz,
                         const int* counts, const double* T_cloud_to_sensor, float* range_l, const rimg_params* p,
                         void* stream) {
  int rc = check_sensor(s);
  if (rc) return rc;
  if (level < 0 || level >= s->levels || n_clouds < 0 || n_clouds > 65535 || max_points < 0)
    return RIMG_ERR_INVALID_ARG;
  if (p && (rc = check_params(p))) return rc;
  if (n_clouds == 0) return RIMG_OK;
  if (!range_l || (max_points > 0 && !xyz)) return RIMG_ERR_INVALID_ARG;
  rimg_params d;
  rimg_default_params(&d);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_before(st, K_POINTS, level, n_clouds);
  cudaError_t e = launch_points(dev_level(s, level), n_clouds, max_points, xyz, counts, T_cloud_to_sensor,
                                p ? p->proj_iters : d.proj_iters, range_l, st);
  prof_after(st);
  if (e != cudaSuccess) return cuda_fail(e, "points kernel");
  return RIMG_OK;
}

int rimg_pyramid(int n_images, int H, int W, int levels, int channels, const float* in,
                 float* const* out_levels, void* stream) {
  if (n_images < 0 || H <= 0 || W <= 0 || levels < 1 || levels > RIMG_MAX_LEVELS) return RIMG_ERR_INVALID_ARG;
  if (channels != 1 && channels != 4) return RIMG_ERR_INVALID_ARG;
  if ((H % (1 << (levels - 1))) || (W % (1 << (levels - 1)))) return RIMG_ERR_SIZE;
  if (n_images == 0 || levels == 1) return RIMG_OK;
  if (!in || !out_levels) return RIMG_ERR_INVALID_ARG;
  for (int l = 1; l < levels; ++l)
    if (!out_levels[l]) return RIMG_ERR_INVALID_ARG;
  if (channels == 4) {
    if (reinterpret_cast<uintptr_t>(in) % 16) return RIMG_ERR_INVALID_ARG;
    for (int l = 1; l < levels; ++l)
      if (reinterpret_cast<uintptr_t>(out_levels[l]) % 16) return RIMG_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_before(st, K_PYRAMID, 1, n_images);
  cudaError_t e = launch_pyramid(n_images, H, W, levels, channels, in, out_levels, st);
  prof_after(st);
  if (e != cudaSuccess) return cuda_fail(e, "pyramid kernel");
  return RIMG_OK;
}

int rimg_normals(const rimg_sensor* s, int n_images, const float* range, const rimg_params* p,
                 float* const* planes_levels, uint8_t* mask0, void* stream) {
  int rc = check_sensor(s);
  if (rc) return rc;
  if ((rc = check_params(p))) return rc;
  if (n_images < 0) return RIMG_ERR_INVALID_ARG;
  if (n_images == 0) return RIMG_OK;
  if (!range || !planes_levels || (reinterpret_cast<uintptr_t>(range) % 16)) return RIMG_ERR_INVALID_ARG;
  for (int l = 0; l < s->levels; ++l)
    if (!planes_levels[l] || (reinterpret_cast<uintptr_t>(planes_levels[l]) % 16)) return RIMG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_before(st, K_NORMALS, 0, n_images);
  cudaError_t e = launch_normals(s, n_images, range, p->normal_rel_jump, p->normal_method, planes_levels, mask0, st);
  prof_after(st);
  if (e != cudaSuccess) return cuda_fail(e, "normals kernel");
  return RIMG_OK;
}

int rimg_icp_workspace_bytes(const rimg_sensor* src, int n_pairs, size_t* bytes) {
  if (!bytes) return RIMG_ERR_INVALID_ARG;
  int rc = check_sensor(src);
  if (rc) return rc;
  if (n_pairs < 0) return RIMG_ERR_INVALID_ARG;
  *bytes = icp_ws(src->H, n_pairs, 0).end;
  return RIMG_OK;
}

int rimg_icp_step(const rimg_sensor* src, const rimg_sensor* dst, int level, int n_pairs,
                  const float* src_range_l, const float* dst_planes_l, const float* dst_range_l,
                  double* pose, const rimg_params* p, int update, double* out29, int32_t* assoc,
                  int* status, void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_sensor(src);
  if (rc) return rc;
  if ((rc = check_sensor(dst))) return rc;
  if ((rc = check_params(p))) return rc;
  if (src->levels != dst->levels) return RIMG_ERR_MISMATCH;
  if (level < 0 || level >= src->levels || n_pairs < 0) return RIMG_ERR_INVALID_ARG;
  if (n_pairs == 0) return RIMG_OK;
  if (!src_range_l || !dst_planes_l || !pose || !workspace) return RIMG_ERR_INVALID_ARG;
  if (p->max_corr_dist > 0.f && !dst_range_l) return RIMG_ERR_INVALID_ARG;
  const IcpWs w = icp_ws(src->H, n_pairs, 0);
  if (!aligned(workspace) || workspace_bytes < w.end) return RIMG_ERR_WORKSPACE;
  if ((reinterpret_cast<uintptr_t>(src_range_l) % 16) || (reinterpret_cast<uintptr_t>(dst_planes_l) % 16) ||
      (assoc && (reinterpret_cast<uintptr_t>(assoc) % 16)))
    return RIMG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  RIMG_CUDA(cudaMemsetAsync(ws + w.counters, 0, sizeof(unsigned) * n_pairs, st));
  return icp_launch(src, dst, level, n_pairs, src_range_l, dst_planes_l, dst_range_l, pose, p, update,
                    out29, assoc, status, icp_scratch(ws, w, src->H, 0), st);
}

int rimg_gn_update(int n_pairs, double* sums, double* pose, int* status, void* stream) {
  if (n_pairs < 0) return RIMG_ERR_INVALID_ARG;
  if (n_pairs == 0) return RIMG_OK;
  if (!sums || !pose) return RIMG_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(sums) % 8) || (reinterpret_cast<uintptr_t>(pose) % 8) ||
      (reinterpret_cast<uintptr_t>(status) % 4))
    return RIMG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  prof_before(st, K_SOLVE, 0, n_pairs);
  cudaError_t e = launch_solve(n_pairs, sums, pose, status, st);
  prof_after(st);
  if (e != cudaSuccess) return cuda_fail(e, "solve kernel");
  return RIMG_OK;
}

int rimg_register_workspace_bytes(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs, int levels,
                                  size_t* bytes) {
  if (!bytes) return RIMG_ERR_INVALID_ARG;
  int rc = check_sensor(src);
  if (rc) return rc;
  if ((rc = check_sensor(dst))) return rc;
  if (src->H != dst->H || src->W != dst->W) return RIMG_ERR_MISMATCH;
  if (n_pairs < 0 || levels < 1 || levels > src->levels || levels > dst->levels) return RIMG_ERR_INVALID_ARG;
  *bytes = reg_ws(src->H, src->W, n_pairs, levels, 0).end;
  return RIMG_OK;
}

int rimg_register(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs, const float* src_range,
                  const float* dst_range, const double* T_init, double* T_out, int levels, const int* iters,
                  const rimg_params* p, int* status, void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_register_args(src, dst, n_pairs, levels, iters, p);
  if (rc) return rc;
  if (n_pairs == 0) return RIMG_OK;
  if (!src_range || !dst_range || !T_init || !T_out || !workspace) return RIMG_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(src_range) % 16) || (reinterpret_cast<uintptr_t>(dst_range) % 16))
    return RIMG_ERR_INVALID_ARG;
  const RegWs R = reg_ws(src->H, src->W, n_pairs, levels, 0);
  if (!aligned(workspace) || workspace_bytes < R.end) return RIMG_ERR_WORKSPACE;
  return register_device(src, dst, n_pairs, src_range, dst_range, T_init, T_out, levels, iters, p, status,
                         static_cast<char*>(workspace), R, static_cast<cudaStream_t>(stream));
}

int rimg_register_last_sums(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs, int levels,
                            const void* workspace, size_t workspace_bytes, double* out32, void* stream) {
  int rc = check_sensor(src);
  if (rc) return rc;
  if ((rc = check_sensor(dst))) return rc;
  if (src->H != dst->H || src->W != dst->W) return RIMG_ERR_MISMATCH;
  if (n_pairs < 0 || levels < 1 || levels > src->levels || levels > dst->levels) return RIMG_ERR_INVALID_ARG;
  if (n_pairs == 0) return RIMG_OK;
  if (!out32 || !workspace) return RIMG_ERR_INVALID_ARG;
  const RegWs R = reg_ws(src->H, src->W, n_pairs, levels, 0);
  if (!aligned(workspace) || workspace_bytes < R.end) return RIMG_ERR_WORKSPACE;
  RIMG_CUDA(cudaMemcpyAsync(out32, static_cast<const char*>(workspace) + R.icp.sums,
                            sizeof(double) * kRedStride * (size_t)n_pairs, cudaMemcpyDeviceToDevice,
                            static_cast<cudaStream_t>(stream)));
  return RIMG_OK;
}

int rimg_register_host_workspace_bytes(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs, int levels,
                                       int chunk_pairs, size_t* bytes) {
  if (!bytes) return RIMG_ERR_INVALID_ARG;
  int rc = check_sensor(src);
  if (rc) return rc;
  if ((rc = check_sensor(dst))) return rc;
  if (src->H != dst->H || src->W != dst->W) return RIMG_ERR_MISMATCH;
  if (n_pairs < 0 || levels < 1 || levels > src->levels || levels > dst->levels) return RIMG_ERR_INVALID_ARG;
  (void)chunk_pairs;
  *bytes = host_ws(src->H, src->W, n_pairs, levels).reg.end;
  return RIMG_OK;
}

int rimg_register_host_async(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs,
                             const float* src_range_host, const float* dst_range_host, const double* T_init_host,
                             double* T_out_host, int levels, const int* iters, const rimg_params* p,
                             int* status_host, int chunk_pairs, void* workspace, size_t workspace_bytes,
                             void* stream) {
  int rc = check_register_args(src, dst, n_pairs, levels, iters, p);
  if (rc) return rc;
  if (n_pairs == 0) return RIMG_OK;
  if (!src_range_host || !dst_range_host || !T_init_host || !T_out_host || !workspace) return RIMG_ERR_INVALID_ARG;
  const HostWs hw = host_ws(src->H, src->W, n_pairs, levels);
  if (!aligned(workspace) || workspace_bytes < hw.reg.end) return RIMG_ERR_WORKSPACE;
  int chunk = (chunk_pairs <= 0 || chunk_pairs > n_pairs) ? n_pairs : chunk_pairs;
  if ((n_pairs + chunk - 1) / chunk > kHostEvents) chunk = (n_pairs + kHostEvents - 1) / kHostEvents;
  const size_t N = (size_t)src->H * src->W;
  char* ws = static_cast<char*>(workspace);
  float* d_src = reinterpret_cast<float*>(ws + hw.src);
  float* d_dst = reinterpret_cast<float*>(ws + hw.dst);
  double* dT = reinterpret_cast<double*>(ws + hw.T);
  int* dS = reinterpret_cast<int*>(ws + hw.S);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  std::lock_guard<std::mutex> lk(g_pipe.mu);
  int dev = 0;
  RIMG_CUDA(cudaGetDevice(&dev));
  if (g_pipe.device != dev) {
    RIMG_CUDA(cudaStreamCreateWithFlags(&g_pipe.copy, cudaStreamNonBlocking));
    for (int i = 0; i < kHostStreams; ++i) {
      RIMG_CUDA(cudaStreamCreateWithFlags(&g_pipe.comp[i], cudaStreamNonBlocking));
      RIMG_CUDA(cudaEventCreateWithFlags(&g_pipe.done[i], cudaEventDisableTiming));
    }
    for (int i = 0; i < kHostEvents; ++i)
      RIMG_CUDA(cudaEventCreateWithFlags(&g_pipe.loaded[i], cudaEventDisableTiming));
    RIMG_CUDA(cudaEventCreateWithFlags(&g_pipe.start, cudaEventDisableTiming));
    g_pipe.device = dev;
  }
  // Everything starts after the work already queued on `stream`.  The copy
  // stream uploads chunk after chunk; chunk k's registration runs on compute
  // stream k % 4 as soon as its own inputs have landed, so uploads overlap
  // registrations and registrations of successive chunks overlap each other.
  // Every chunk uses its own slice of the staging buffers and the workspace.
  RIMG_CUDA(cudaEventRecord(g_pipe.start, st));
  RIMG_CUDA(cudaStreamWaitEvent(g_pipe.copy, g_pipe.start, 0));
  for (int i = 0; i < kHostStreams; ++i) RIMG_CUDA(cudaStreamWaitEvent(g_pipe.comp[i], g_pipe.start, 0));
  RIMG_CUDA(cudaMemcpyAsync(dT, T_init_host, sizeof(double) * 16 * n_pairs, cudaMemcpyHostToDevice, g_pipe.copy));
  int k = 0;
  for (int off = 0; off < n_pairs; off += chunk, ++k) {
    const int cnt = std::min(chunk, n_pairs - off);
    RIMG_CUDA(cudaMemcpyAsync(d_src + N * off, src_range_host + N * off, sizeof(float) * N * cnt,
                              cudaMemcpyHostToDevice, g_pipe.copy));
    RIMG_CUDA(cudaMemcpyAsync(d_dst + N * off, dst_range_host + N * off, sizeof(float) * N * cnt,
                              cudaMemcpyHostToDevice, g_pipe.copy));
    RIMG_CUDA(cudaEventRecord(g_pipe.loaded[k], g_pipe.copy));
    cudaStream_t cs = g_pipe.comp[k % kHostStreams];
    RIMG_CUDA(cudaStreamWaitEvent(cs, g_pipe.loaded[k], 0));
    rc = register_slice(src, dst, off, cnt, d_src, d_dst, dT, dT, levels, iters, p, dS, ws, hw.reg, cs);
    if (rc) return rc;
    RIMG_CUDA(cudaMemcpyAsync(T_out_host + 16 * off, dT + 16 * off, sizeof(double) * 16 * cnt,
                              cudaMemcpyDeviceToHost, cs));
    if (status_host)
      RIMG_CUDA(cudaMemcpyAsync(status_host + off, dS + off, sizeof(int) * cnt, cudaMemcpyDeviceToHost, cs));
  }
  for (int i = 0; i < kHostStreams; ++i) {
    RIMG_CUDA(cudaEventRecord(g_pipe.done[i], g_pipe.comp[i]));
    RIMG_CUDA(cudaStreamWaitEvent(st, g_pipe.done[i], 0));
  }
  return RIMG_OK;
}

int rimg_register_host(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs, const float* src_range_host,
                       const float* dst_range_host, const double* T_init_host, double* T_out_host, int levels,
                       const int* iters, const rimg_params* p, int* status_host, int chunk_pairs, void* workspace,
                       size_t workspace_bytes, void* stream) {
  int rc = rimg_register_host_async(src, dst, n_pairs, src_range_host, dst_range_host, T_init_host, T_out_host,
                                    levels, iters, p, status_host, chunk_pairs, workspace, workspace_bytes, stream);
  if (rc) return rc;
  RIMG_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  return RIMG_OK;
}

int rimg_register_groups_workspace_bytes(int n_groups, const rimg_group* groups, size_t* bytes) {
  if (!bytes || n_groups < 0 || (n_groups > 0 && !groups)) return RIMG_ERR_INVALID_ARG;
  for (int i = 0; i < n_groups; ++i) {
    const rimg_group& g = groups[i];
    int rc = check_register_args(g.src, g.dst, g.n_pairs, g.levels, g.iters, g.params);
    if (rc) return rc;
  }
  *bytes = groups_ws(n_groups, groups).end;
  return RIMG_OK;
}

int rimg_register_groups(int n_groups, const rimg_group* groups, void* workspace, size_t workspace_bytes,
                         void* stream) {
  size_t need = 0;
  int rc = rimg_register_groups_workspace_bytes(n_groups, groups, &need);
  if (rc) return rc;
  for (int i = 0; i < n_groups; ++i) {
    const rimg_group& g = groups[i];
    if (g.n_pairs > 0 && (!g.src_range || !g.dst_range || !g.T_init || !g.T_out)) return RIMG_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(g.src_range) % 16) || (reinterpret_cast<uintptr_t>(g.dst_range) % 16))
      return RIMG_ERR_INVALID_ARG;
  }
  if (n_groups == 0) return RIMG_OK;
  if (!workspace || !aligned(workspace) || workspace_bytes < need) return RIMG_ERR_WORKSPACE;
  const GroupWs w = groups_ws(n_groups, groups);
  const std::vector<Slice> slices = group_slices(n_groups, groups);
  if (slices.empty()) return RIMG_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  std::lock_guard<std::mutex> lk(g_grp.mu);
  int dev = 0;
  RIMG_CUDA(cudaGetDevice(&dev));
  if (g_grp.device != dev) {
    for (int i = 0; i < kGroupStreams; ++i) {
      RIMG_CUDA(cudaStreamCreateWithFlags(&g_grp.s[i], cudaStreamNonBlocking));
      RIMG_CUDA(cudaEventCreateWithFlags(&g_grp.join[i], cudaEventDisableTiming));
    }
    RIMG_CUDA(cudaEventCreateWithFlags(&g_grp.fork, cudaEventDisableTiming));
    g_grp.device = dev;
  }
  // The leading small levels of eligible groups run in one persistent queue
  // launch per kernel form; every other level runs per sub-batch.
  std::vector<std::vector<int>> sizes(n_groups);
  for (const Slice& sl : slices) sizes[sl.group].push_back(sl.n);
  std::vector<int> prefix(n_groups, 0);
  bool any_queue = false;
  for (int i = 0; i < n_groups; ++i) {
    prefix[i] = queue_prefix(groups[i], sizes[i]);
    any_queue = any_queue || prefix[i] > 0;
  }
  // Longest-processing-time-first assignment of slices to internal streams;
  // slices of one group never share a workspace range, so all may overlap.
  const int nstreams = std::min<int>(kGroupStreams, (int)slices.size());
  std::vector<double> load(nstreams, 0.0);
  std::vector<std::vector<int>> assign(nstreams);
  for (int k = 0; k < (int)slices.size(); ++k) {
    const int best = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    assign[best].push_back(k);
    load[best] += slices[k].work;
  }
  // Phase 1: per sub-batch, either the whole registration or (groups with a
  // queued prefix) the set-up and pyramids only.
  RIMG_CUDA(cudaEventRecord(g_grp.fork, st));
  for (int i = 0; i < nstreams; ++i) {
    RIMG_CUDA(cudaStreamWaitEvent(g_grp.s[i], g_grp.fork, 0));
    for (int k : assign[i]) {
      const Slice& sl = slices[k];
      const rimg_group& g = groups[sl.group];
      char* gws = ws + w.off[sl.group];
      rc = prefix[sl.group] > 0
               ? slice_begin(g.src, g.dst, sl.p0, sl.n, g.src_range, g.dst_range, g.T_init, g.T_out, g.levels,
                             g.params, g.status, gws, w.reg[sl.group], g_grp.s[i])
               : register_slice(g.src, g.dst, sl.p0, sl.n, g.src_range, g.dst_range, g.T_init, g.T_out, g.levels,
                                g.iters, g.params, g.status, gws, w.reg[sl.group], g_grp.s[i]);
      if (rc) return rc;
    }
    RIMG_CUDA(cudaEventRecord(g_grp.join[i], g_grp.s[i]));
    RIMG_CUDA(cudaStreamWaitEvent(st, g_grp.join[i], 0));
  }
  if (!any_queue) return RIMG_OK;
  // Phase 2: the queued small levels of every eligible pair, one persistent
  // launch per kernel form (receiver offset, Kahan), most expensive groups
  // first.
  QueueGroup* dq = reinterpret_cast<QueueGroup*>(ws + w.queue);
  unsigned* counters = reinterpret_cast<unsigned*>(ws + w.queue_counters);
  int slot = 0;
  for (int form = 0; form < 4; ++form) {
    const bool r0 = (form & 1) != 0, kahan = (form & 2) != 0;
    std::vector<std::pair<double, int>> order;
    for (int i = 0; i < n_groups; ++i) {
      const rimg_group& g = groups[i];
      if (prefix[i] == 0) continue;
      const bool g_r0 = g.src->r0 != 0.f || g.dst->r0 != 0.f;
      if (g_r0 != r0 || (g.params->kahan != 0) != kahan) continue;
      double cost = 0.0;
      for (int k = 0; k < prefix[i]; ++k) {
        const int l = g.levels - 1 - k;
        cost += (double)(g.src->H >> l) * (g.src->W >> l) * g.iters[k];
      }
      order.push_back(std::make_pair(-cost, i));
    }
    if (order.empty()) continue;
    std::sort(order.begin(), order.end());
    std::vector<QueueGroup> hq(order.size());
    int item0 = 0;
    for (size_t q = 0; q < order.size(); ++q) {
      const int i = order[q].second;
      const rimg_group& g = groups[i];
      char* gws = ws + w.off[i];
      const RegWs& Rg = w.reg[i];
      const SliceBufs b = slice_bufs(gws, Rg, g.src->H, g.src->W, g.levels, 0);
      QueueGroup& Q = hq[q];
      Q = QueueGroup{};
      Q.n_lvl = prefix[i];
      for (int k = 0; k < prefix[i]; ++k) {
        const int l = g.levels - 1 - k;
        Q.lvl[k].src = dev_level(g.src, l);
        Q.lvl[k].dst = dev_level(g.dst, l);
        Q.lvl[k].src_range = (l == 0) ? g.src_range : b.srcl[l];
        Q.lvl[k].planes = reinterpret_cast<const float4*>(b.planes[l]);
        Q.lvl[k].iters = g.iters[k];
      }
      Q.n_pairs = g.n_pairs;
      Q.item0 = item0;
      item0 += g.n_pairs;
      Q.proj_iters = g.params->proj_iters;
      Q.huber_delta = g.params->huber_delta;
      Q.pose = g.T_out;
      Q.sums = icp_scratch(gws, Rg.icp, g.src->H, 0).sums;
      Q.status = g.status;
    }
    prof_before(st, K_ICP_QUEUE, -1, item0);
    cudaError_t e = launch_icp_queue(hq.data(), (int)hq.size(), dq + slot, counters + form, r0, kahan, st);
    prof_after(st);
    if (e != cudaSuccess) return cuda_fail(e, "queue kernel");
    slot += (int)hq.size();
  }
  // Phase 3: the remaining levels of the queued groups, per sub-batch.
  RIMG_CUDA(cudaEventRecord(g_grp.fork, st));
  for (int i = 0; i < nstreams; ++i) {
    bool used = false;
    for (int k : assign[i]) {
      const Slice& sl = slices[k];
      if (prefix[sl.group] == 0 || prefix[sl.group] >= groups[sl.group].levels) continue;
      if (!used) RIMG_CUDA(cudaStreamWaitEvent(g_grp.s[i], g_grp.fork, 0));
      used = true;
      const rimg_group& g = groups[sl.group];
      rc = slice_levels(g.src, g.dst, sl.p0, sl.n, g.src_range, g.dst_range, g.T_out, g.levels, g.iters, g.params,
                        g.status, ws + w.off[sl.group], w.reg[sl.group], prefix[sl.group], g_grp.s[i]);
      if (rc) return rc;
    }
    if (used) {
      RIMG_CUDA(cudaEventRecord(g_grp.join[i], g_grp.s[i]));
      RIMG_CUDA(cudaStreamWaitEvent(st, g_grp.join[i], 0));
    }
  }
  return RIMG_OK;
}

// The autotuner over the groups (see rimg_autotune), timing the whole
// registration through `call` (rimg_register_groups, or rimg_register for
// one group); ws holds each group's registration workspace at the offsets of
// groups_ws.
// Sub-batches up to this many pairs also time cluster schedules for the
// levels that do not fit one block (a latency gain where the batch leaves
// the GPU room; larger batches keep per-iteration launches there).
constexpr int kClusterTuneMaxPairs = 64;
// A cluster block's row table holds at most this many rows.
constexpr int kMaxRowsPerCluster = 1024;

int autotune_impl(int n_groups, const rimg_group* groups, char* ws, cudaStream_t st,
                  const std::function<int()>& call) {
  int rc = RIMG_OK;
  const GroupWs w = groups_ws(n_groups, groups);
  const std::vector<Slice> slices = group_slices(n_groups, groups);
  cudaEvent_t e0, e1;
  RIMG_CUDA(cudaEventCreate(&e0));
  RIMG_CUDA(cudaEventCreate(&e1));
  void* before = icp_tune_save();   // the table as this call found it
  int entries = 0;
  std::vector<std::tuple<int, int, int>> done;
  std::vector<std::tuple<int, int, int>> fitting;   // (H_l, W_l, pairs) of levels that fit one block
  // every shape's standalone time, per (H_l, W_l, pairs)
  std::map<std::tuple<int, int, int>, std::vector<std::tuple<float, int, int>>> shape_cands;
  for (const Slice& sl : slices) {
    const rimg_group& g = groups[sl.group];
    const int H = g.src->H, W = g.src->W;
    const size_t N = (size_t)H * W;
    // the shape depends on (level size, pairs per launch): tune each once
    if (std::find(done.begin(), done.end(), std::make_tuple(sl.group, sl.n, 0)) != done.end()) continue;
    done.push_back(std::make_tuple(sl.group, sl.n, 0));
    char* gws = ws + w.off[sl.group];
    const RegWs& R = w.reg[sl.group];
    const SliceBufs b = slice_bufs(gws, R, H, W, g.levels, sl.p0);
    const float* s0 = g.src_range + sl.p0 * N;
    rc = prep_slice(g.src, g.dst, sl.n, s0, g.dst_range + sl.p0 * N, g.levels, g.params, b, st);
    if (rc) return rc;
    double* pose = g.T_out + 16 * (size_t)sl.p0;
    RIMG_CUDA(cudaMemcpyAsync(pose, g.T_init + 16 * (size_t)sl.p0, sizeof(double) * 16 * sl.n,
                              cudaMemcpyDeviceToDevice, st));
    const IcpScratch scr = icp_scratch(gws, R.icp, H, sl.p0);
    RIMG_CUDA(cudaMemsetAsync(scr.counters, 0, sizeof(unsigned) * sl.n, st));
    const double* init0 = g.T_init + 16 * (size_t)sl.p0;
    auto restore_pose = [&]() {
      return cudaMemcpyAsync(pose, init0, sizeof(double) * 16 * sl.n, cudaMemcpyDeviceToDevice, st);
    };
    for (int l = 0; l < g.levels; ++l) {
      const int Hl = H >> l, Wl = W >> l;
      const int k = g.levels - 1 - l;     // schedule index of level l
      const float* sl_src = (l == 0) ? s0 : b.srcl[l];
      const float* sl_dst = g.params->max_corr_dist > 0.f ? ((l == 0) ? g.dst_range + sl.p0 * N : b.dstl[l])
                                                           : nullptr;
      float best = 1e30f;
      int best_t = 0, best_b = 0;
      for (int T : {128, 256}) {
        for (int bp = 1; bp <= Hl; bp *= 2) {
          if ((long long)Hl * (Wl / 4) < (long long)T / 4 * bp) continue;   // blocks with no work
          // the shortest of three runs of eight back-to-back launches (after one warm-up launch)
          float ms = 1e30f;
          rc = icp_launch(g.src, g.dst, l, sl.n, sl_src, b.planes[l], sl_dst, pose, g.params, 0, nullptr, nullptr,
                          nullptr, scr, st, T, bp);
          if (rc) return rc;
          for (int run = 0; run < 3; ++run) {
            RIMG_CUDA(cudaEventRecord(e0, st));
            for (int rep = 0; rep < 8; ++rep) {
              rc = icp_launch(g.src, g.dst, l, sl.n, sl_src, b.planes[l], sl_dst, pose, g.params, 0, nullptr,
                              nullptr, nullptr, scr, st, T, bp);
              if (rc) return rc;
            }
            RIMG_CUDA(cudaEventRecord(e1, st));
            RIMG_CUDA(cudaEventSynchronize(e1));
            float t = 0.f;
            RIMG_CUDA(cudaEventElapsedTime(&t, e0, e1));
            ms = std::min(ms, t);
          }
          if (ms < best) { best = ms; best_t = T; best_b = bp; }
          shape_cands[std::make_tuple(Hl, Wl, sl.n)].push_back(std::make_tuple(ms, T, bp));
        }
      }
      icp_tune_set(Hl, Wl, sl.n, best_t, best_b);
      ++entries;
      // levels whose schedule is timed in context: those that fit one block,
      // and in small sub-batches (clusters of blocks shorten a pair's
      // iteration chain where the GPU has room) every level
      if (g.iters[k] > 0 && (icp_iters_fits(Hl, Wl) || sl.n <= kClusterTuneMaxPairs)) {
        const auto key = std::make_tuple(Hl, Wl, sl.n);
        if (std::find(fitting.begin(), fitting.end(), key) == fitting.end()) fitting.push_back(key);
      }
    }
    RIMG_CUDA(restore_pose());
  }
  // Per-level schedules, measured in context: for every level that fits one
  // block (in every sub-batch size), the whole rimg_register_groups call is
  // timed with that level run both ways -- all iterations in one block per
  // pair (the persistent queue / one launch per level) and one association
  // launch plus one FP64 solve launch per iteration -- and the faster kept.
  // Timing the whole call keeps the concurrency of the other groups and
  // sub-batches, which a level timed alone would not show.
  auto time_call = [&](float* ms) -> int {   // the shortest of three runs of three calls
    int r = call();
    if (r) return r;
    *ms = 1e30f;
    for (int run = 0; run < 3; ++run) {
      RIMG_CUDA(cudaEventRecord(e0, st));
      for (int rep = 0; rep < 3; ++rep) {
        r = call();
        if (r) return r;
      }
      RIMG_CUDA(cudaEventRecord(e1, st));
      RIMG_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      RIMG_CUDA(cudaEventElapsedTime(&t, e0, e1));
      *ms = std::min(*ms, t);
    }
    return RIMG_OK;
  };
  for (const auto& key : fitting) {
    const int Hl = std::get<0>(key), Wl = std::get<1>(key), n = std::get<2>(key);
    // one block per pair (where the pair fits one), clusters of 2, 4 and 8
    // blocks per pair, per-iteration launches (ties keep the earlier candidate)
    const bool fits = icp_iters_fits(Hl, Wl);
    float best = 1e30f;
    int best_s = fits ? 1 : 0;
    for (int s : {1, 0, 2, 4, 8}) {
      if (s == 1 && !fits) continue;
      if (s > 1 && (Hl + s - 1) / s > kMaxRowsPerCluster) continue;
      float ms = 0.f;
      icp_sched_set(Hl, Wl, n, s);
      if ((rc = time_call(&ms))) return rc;
      if (ms < best) { best = ms; best_s = s; }
    }
    icp_sched_set(Hl, Wl, n, best_s);
    ++entries;
    // launch shapes stay only for levels that run as per-iteration launches
    if (best_s != 0) {
      icp_tune_erase(Hl, Wl, n);
      --entries;
    }
  }
  // Launch shapes of the levels that run as per-iteration launches, chosen in
  // context: the default shape and the three fastest shapes of the
  // standalone sweep, each timed over whole calls (the shape fastest alone is
  // not always the fastest beside the other sub-batches' launches).
  for (auto& kv : shape_cands) {
    const int Hl = std::get<0>(kv.first), Wl = std::get<1>(kv.first), n = std::get<2>(kv.first);
    if (icp_sched(Hl, Wl, n) != 0) continue;
    std::vector<std::tuple<float, int, int>> v = kv.second;
    std::sort(v.begin(), v.end());
    float best = 1e30f, ms = 0.f;
    int best_t = 0, best_b = 0;    // threads 0: the default shape (no entry)
    icp_tune_erase(Hl, Wl, n);
    if ((rc = time_call(&ms))) return rc;
    best = ms;
    for (size_t i = 0; i < v.size() && i < 3; ++i) {
      icp_tune_set(Hl, Wl, n, std::get<1>(v[i]), std::get<2>(v[i]));
      if ((rc = time_call(&ms))) return rc;
      if (ms < best) { best = ms; best_t = std::get<1>(v[i]); best_b = std::get<2>(v[i]); }
    }
    if (best_t) {
      icp_tune_set(Hl, Wl, n, best_t, best_b);
    } else {
      icp_tune_erase(Hl, Wl, n);
      --entries;
    }
  }
  // The tuned table against the table as this call found it, each timed in
  // context twice, alternately: the tuning stays only if it is faster (the
  // single decisions above are taken on noisy timings).
  {
    void* after = icp_tune_save();
    float t_after = 1e30f, t_before = 1e30f, t = 0.f;
    for (int r = 0; r < 2 && rc == RIMG_OK; ++r) {
      icp_tune_restore(after);
      if ((rc = time_call(&t)) == RIMG_OK) t_after = std::min(t_after, t);
      icp_tune_restore(before);
      if (rc == RIMG_OK && (rc = time_call(&t)) == RIMG_OK) t_before = std::min(t_before, t);
    }
    const bool keep = rc == RIMG_OK && t_after < t_before;
    icp_tune_restore(keep ? after : before);
    if (!keep) entries = 0;
    icp_tune_free(after);
  }
  icp_tune_free(before);
  if (rc) return rc;
  // T_out ends as a copy of T_init
  for (int i = 0; i < n_groups; ++i)
    if (groups[i].n_pairs > 0 && groups[i].T_out != groups[i].T_init)
      RIMG_CUDA(cudaMemcpyAsync(groups[i].T_out, groups[i].T_init, sizeof(double) * 16 * groups[i].n_pairs,
                                cudaMemcpyDeviceToDevice, st));
  RIMG_CUDA(cudaStreamSynchronize(st));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return entries;
}

int rimg_autotune(int n_groups, const rimg_group* groups, void* workspace, size_t workspace_bytes, void* stream) {
  size_t need = 0;
  int rc = rimg_register_groups_workspace_bytes(n_groups, groups, &need);
  if (rc) return rc;
  if (n_groups == 0) return 0;
  if (!workspace || !aligned(workspace) || workspace_bytes < need) return RIMG_ERR_WORKSPACE;
  return autotune_impl(n_groups, groups, static_cast<char*>(workspace), static_cast<cudaStream_t>(stream),
                       [&]() { return rimg_register_groups(n_groups, groups, workspace, workspace_bytes, stream); });
}

int rimg_autotune_register(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs, const float* src_range,
                           const float* dst_range, const double* T_init, double* T_out, int levels,
                           const int* iters, const rimg_params* p, void* workspace, size_t workspace_bytes,
                           void* stream) {
  int rc = check_register_args(src, dst, n_pairs, levels, iters, p);
  if (rc) return rc;
  if (n_pairs == 0) return 0;
  if (!src_range || !dst_range || !T_init || !T_out || !workspace) return RIMG_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(src_range) % 16) || (reinterpret_cast<uintptr_t>(dst_range) % 16))
    return RIMG_ERR_INVALID_ARG;
  const RegWs R = reg_ws(src->H, src->W, n_pairs, levels, 0);
  if (!aligned(workspace) || workspace_bytes < R.end) return RIMG_ERR_WORKSPACE;
  // one group whose registration workspace sits at offset 0, as rimg_register's
  const rimg_group g{src, dst, n_pairs, levels, iters, p, src_range, dst_range, T_init, T_out, nullptr};
  return autotune_impl(1, &g, static_cast<char*>(workspace), static_cast<cudaStream_t>(stream), [&]() {
    return rimg_register(src, dst, n_pairs, src_range, dst_range, T_init, T_out, levels, iters, p, nullptr,
                         workspace, workspace_bytes, stream);
  });
}

int rimg_autotune_clear(void) {
  icp_tune_clear();
  return RIMG_OK;
}

int rimg_autotune_set(int H_l, int W_l, int n_pairs, int threads, int blocks_per_pair, int schedule) {
  if (H_l <= 0 || W_l <= 0 || n_pairs <= 0 || schedule < -1 || schedule > 8 || schedule == 3 ||
      (schedule > 4 && schedule < 8))
    return RIMG_ERR_INVALID_ARG;
  if (threads != 0 && threads != 128 && threads != 256) return RIMG_ERR_INVALID_ARG;
  if (threads != 0 && (blocks_per_pair < 1 || blocks_per_pair > H_l)) return RIMG_ERR_INVALID_ARG;
  if (threads == 0)
    icp_tune_erase(H_l, W_l, n_pairs);
  else
    icp_tune_set(H_l, W_l, n_pairs, threads, blocks_per_pair);
  if (schedule >= 0) icp_sched_set(H_l, W_l, n_pairs, schedule);
  return RIMG_OK;
}

int rimg_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* C, int ldc,
                   void* C_bf16, const float* bias, int relu, int splits, int* err, void* stream) {
  if (M < 0 || N < 0 || K < 0 || splits < 1) return RIMG_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return RIMG_OK;
  if (K % 64 || lda < K || ldb < K || lda % 8 || ldb % 8 || ldc < N) return RIMG_ERR_SIZE;
  if (splits > 1 && (C_bf16 || bias || relu)) return RIMG_ERR_INVALID_ARG;
  if (splits > std::max(1, K / 64)) return RIMG_ERR_INVALID_ARG;
  if (!A || !B || !C) return RIMG_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(A) % 16) || (reinterpret_cast<uintptr_t>(B) % 16)) return RIMG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_gemm_bf16(M, N, K, A, lda, B, ldb, C, ldc, C_bf16, bias, relu, splits, err, st);
  if (e != cudaSuccess) return cuda_fail(e, "tcgen05 gemm kernel");
  return RIMG_OK;
}

int rimg_profile_begin(int max_launches) {
  if (max_launches < 0) return RIMG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  const int have = (int)g_prof.ev0.size();
  for (int i = have; i < max_launches; ++i) {
    cudaEvent_t a, b;
    RIMG_CUDA(cudaEventCreate(&a));
    RIMG_CUDA(cudaEventCreate(&b));
    g_prof.ev0.push_back(a);
    g_prof.ev1.push_back(b);
  }
  g_prof.kid.assign(std::max(have, max_launches), 0);
  g_prof.lvl.assign(std::max(have, max_launches), 0);
  g_prof.np.assign(std::max(have, max_launches), 0);
  g_prof.cap = max_launches;
  g_prof.n = 0;
  g_prof.open = false;
  g_prof.on = true;
  return RIMG_OK;
}

int rimg_profile_end(int cap, int* kernel_id, int* level, int* n_pairs, float* start_ms, float* ms) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.on = false;
  const int n = std::min(cap, g_prof.n);
  for (int i = 0; i < n; ++i) {
    RIMG_CUDA(cudaEventSynchronize(g_prof.ev1[i]));
    float t = 0.f, t0 = 0.f;
    RIMG_CUDA(cudaEventElapsedTime(&t, g_prof.ev0[i], g_prof.ev1[i]));
    RIMG_CUDA(cudaEventElapsedTime(&t0, g_prof.ev0[0], g_prof.ev0[i]));
    if (kernel_id) kernel_id[i] = g_prof.kid[i];
    if (level) level[i] = g_prof.lvl[i];
    if (n_pairs) n_pairs[i] = g_prof.np[i];
    if (start_ms) start_ms[i] = t0;
    if (ms) ms[i] = t;
  }
  g_prof.n = 0;
  return n;
}

}  // extern "C"

namespace rimg {
// Records a failed CUDA call for rimg_last_error (used by the other
// translation units' entry points).
int record_cuda_error(cudaError_t e, const char* where) { return cuda_fail(e, where); }
}  // namespace rimg
