// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/rimg.h"

namespace rimg {

// Device view of one pyramid level of a sensor's tables (built on the host
// from rimg_sensor and passed to kernels by value).
struct DevLevel {
  const float4* rows;     // [H] cos phi, sin phi, cos theta_lut, sin theta_lut
  const float* cos_u;     // [W] cos of 2 pi u / W
  const float* sin_u;     // [W] sin of 2 pi u / W
  const float* thu;       // [H] theta_lut * W / (2 pi)
  const int* rank2row;    // [H]
  const float* bnd;       // [H-1]
  const int4* bins;       // [n_bins] (row_lo, row_hi, boundary bits, rank at lower edge)
  int H, W, n_bins, tie_up, bins_exact, has_theta;
  float s_lo, s_hi, bin_scale, wf, r0, inv_w2;   // wf = W, inv_w2 = 2 / W
  float col_magic;        // 1.5 * 2^23 / W (the column rounding of a power-of-two W)
};

DevLevel dev_level(const rimg_sensor* s, int level);

enum KernelId { K_UNPROJECT = 0, K_PYRAMID = 1, K_NORMALS = 2, K_ICP = 3, K_SRC_PYRAMID = 4, K_SOLVE = 5, K_SDF = 6, K_POINTS = 7, K_ICP_ITERS = 8, K_ICP_QUEUE = 9, K_ICP_CLUSTER = 10 };

// Launch-timing hooks (no-ops unless rimg_profile_begin was called).
void prof_before(cudaStream_t st, int kernel, int level, int n);
void prof_after(cudaStream_t st);

// Launchers (return cudaGetLastError()).
cudaError_t launch_unproject(const DevLevel& L, int n, const float* range, float* xyz,
                             uint8_t* mask, cudaStream_t st);
cudaError_t launch_pyramid(int n, int H, int W, int levels, int channels, const float* in,
                           float* const* out_levels, cudaStream_t st);
cudaError_t launch_normals(const rimg_sensor* s, int n, const float* range, float rel_jump, int method,
                           float* const* planes_levels, uint8_t* mask0, cudaStream_t st);

struct IcpLaunch {
  DevLevel src, dst;
  int n_pairs;
  const float* src_range;
  const float4* dst_planes;
  const float* dst_range;
  double* pose;
  double* out29;
  int32_t* assoc;
  int* status;
  float* partials;          // [n_pairs][bpp][32]
  unsigned int* counters;   // [n_pairs]
  double* sums;             // [n_pairs][32] FP64 totals (input of the solve)
  float huber_delta, max_corr_dist;
  int proj_iters, kahan, update;
  int bpp, rows_per_block, threads;
};

// Blocks per pair and rows per block for a level (depends on the batch and
// the device's resident-block capacity).
void icp_grid(int H, int W, int n_pairs, int* bpp, int* rows_per_block, int* threads);
void icp_tune_set(int H, int W, int n_pairs, int threads, int bpp);
void icp_tune_clear();
void icp_tune_erase(int H, int W, int n_pairs);
// The schedule of a level (rimg_autotune's choice for (H, W, pairs)): 0 one
// association launch and one solve launch per iteration (the default for
// levels that do not fit one block), 1 all iterations in one block per pair
// (the default where the pair fits one block; taken only there), 2, 4 or 8
// all iterations on a cluster of that many blocks per pair.
void icp_sched_set(int H, int W, int n_pairs, int sched);
int icp_sched(int H, int W, int n_pairs);
int icp_tune_size();
// A copy of the whole table (shapes and schedules), put back by
// icp_tune_restore; icp_tune_free releases the copy.
void* icp_tune_save();
void icp_tune_restore(const void* saved);
void icp_tune_free(void* saved);
cudaError_t launch_icp(IcpLaunch a, cudaStream_t st);
cudaError_t launch_solve(int n_pairs, double* sums, double* pose, int* status, cudaStream_t st);
// All iterations of a level whose pair fits one block (H_l * W_l / 4 chunks
// <= kIcpItersMaxChunks, i.e. at most 32 chunks per thread of a 128-thread
// block) in one launch; a.pose is updated in place.
constexpr int kIcpItersMaxChunks = 4096;
bool icp_iters_fits(int H, int W);
cudaError_t launch_icp_iters(IcpLaunch a, int iters, cudaStream_t st);
// All iterations of a level with each pair on a thread-block cluster of
// `cluster` (2, 4 or 8) blocks of 128 threads (no gate, no association
// output); bit-identical to `cluster` blocks per pair in per-iteration
// launches.
cudaError_t launch_icp_cluster(IcpLaunch a, int iters, int cluster, cudaStream_t st);

cudaError_t launch_center(const DevLevel& S, const DevLevel& D, int n_pairs, const float* src, const float* dst,
                          double* T_out, int* status, cudaStream_t st);

// Persistent work queue over the small levels of uneven batches: every pair
// of every listed group is one item, processed by one block -- all the
// group's leading small levels (the coarsest, each fitting one block),
// coarse to fine, every iteration with its FP64 update.  Items are taken
// from an atomic counter; a block never waits for another.
struct QueueLevel {
  DevLevel src, dst;
  const float* src_range;     // level-l source ranges [n][H_l][W_l]
  const float4* planes;       // level-l target planes [n][H_l][W_l]
  int iters;
};
struct QueueGroup {
  QueueLevel lvl[RIMG_MAX_LEVELS];   // the leading small levels, coarse to fine
  int n_lvl;
  int n_pairs;
  int item0;                          // the group's pairs are items item0 .. item0 + n_pairs - 1
  int proj_iters;
  float huber_delta;
  double* pose;                       // [n][16], updated in place
  double* sums;                       // [n][32], the last step's sums and step record
  int* status;                        // [n] or null
};
#ifndef RIMG_QUEUE_THREADS
#define RIMG_QUEUE_THREADS 256
#endif
constexpr int kQueueThreads = RIMG_QUEUE_THREADS;
// Whether level (H, W) runs in the queue kernel: it fits one block and its
// chunks per row divide the block (row-stride cursors).
bool queue_level_ok(int H, int W);
// Writes the descriptors (device, `n_groups` entries) and launches the
// persistent kernel on `st`; counter: device, zeroed here first.
cudaError_t launch_icp_queue(const QueueGroup* host_groups, int n_groups, QueueGroup* dev_groups, unsigned* counter,
                             bool r0, bool kahan, cudaStream_t st);

cudaError_t launch_sdf(const DevLevel& L, int n_scans, const float* ranges, const double* poses, int nx, int ny,
                       int nz, float ox, float oy, float oz, float voxel, float trunc, int proj_iters, float* sdf,
                       float* weight, cudaStream_t st);

cudaError_t launch_points(const DevLevel& L, int n_clouds, int max_points, const float* xyz, const int* counts,
                          const double* T, int proj_iters, float* img, cudaStream_t st);

cudaError_t launch_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* C, int ldc,
                             void* Cbf, const float* bias, int relu, int splits, int* err, cudaStream_t st);

// Records a failed CUDA call for rimg_last_error; returns RIMG_ERR_CUDA.
int record_cuda_error(cudaError_t e, const char* where);

constexpr int kIcpThreads = 256;
constexpr int kRed = 29;          // reduced quantities per pair
constexpr int kRedStride = 32;    // floats per partial record

}  // namespace rimg
