// BF16 GEMM on the 5th-generation tensor cores (tcgen05): C[M x N] (FP32) =
// A[M x K] * B[N x K]^T with both operands K-major in global memory.  One CTA
// computes a 128 x NT tile (NT <= 256, a multiple of 16): its four warps stage
// 64-wide K slices of A and B into shared memory in the canonical
// no-swizzle layout (8-row x 16-byte core matrices), one elected thread issues
// tcgen05.mma (M=128, N=NT, K=16 per instruction) into a TMEM accumulator and
// commits to an mbarrier; the next K slice is staged while the tensor cores
// work (two buffers).  The epilogue reads TMEM with tcgen05.ld (each warp its
// 32 lanes = rows), adds an optional bias, applies an optional ReLU and writes
// FP32 (and optionally BF16) results.  gridDim.z > 1 splits K: split z writes
// its own partial C (C + z * M * ldc), summed by the caller.
//
// Waits on the mbarrier are bounded: after ~2^26 polls a CTA records an error
// code and skips its epilogue (the accumulator is still freed).
#include <cuda_bf16.h>
#include <stdint.h>

#include "rimg_internal.h"

namespace rimg {

namespace {

constexpr int kGemmThreads = 128;
constexpr int kTileM = 128;
constexpr int kTileK = 64;   // BF16 elements per staged K slice (8 core matrices)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (distance between core matrices along K), stride byte offset
// (distance between core matrices along M/N), descriptor version 1, no
// swizzle.  Addresses and offsets in 16-byte units.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor for kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (int i = 0; i < (1 << 26); ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g, bool pred) {
  const int n = pred ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(g), "r"(n) : "memory");
}

// Stage rows [row0, row0 + rows_tile) x K slice [k0, k0 + 64) of a K-major
// BF16 matrix (leading dimension ld elements) into the core-matrix layout:
// core (r / 8, kc) at byte offset ((r / 8) * 8 + kc) * 128, row r % 8 at +16 B.
// Rows >= nrows are zero-filled.
__device__ __forceinline__ void stage_tile(uint32_t sbase, const __nv_bfloat16* g, int ld, int nrows, int row0,
                                           int k0, int rows_tile, int tid) {
  const int chunks = rows_tile * (kTileK / 8);
  for (int c = tid; c < chunks; c += kGemmThreads) {
    const int r = c >> 3, kc = c & 7;
    const int gr = row0 + r;
    const bool ok = gr < nrows;
    const __nv_bfloat16* src = g + (size_t)(ok ? gr : 0) * ld + k0 + kc * 8;
    const uint32_t off = (uint32_t)(((r >> 3) * 8 + kc) * 128 + (r & 7) * 16);
    cp_async16(sbase + off, src, ok);
  }
}

template <int NT>
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_bf16_tn(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda,
                   const __nv_bfloat16* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                   __nv_bfloat16* __restrict__ Cbf, const float* __restrict__ bias, int relu, int k_per_split,
                   int* __restrict__ err) {
  constexpr int kTmemCols = NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256));
  constexpr uint32_t kABytes = kTileM * kTileK * 2;
  constexpr uint32_t kBBytes = NT * kTileK * 2;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA[2] = {smem, smem + kABytes};
  unsigned char* sB[2] = {smem + 2 * kABytes, smem + 2 * kABytes + kBBytes};
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_base;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * kTileM, n0 = blockIdx.y * NT;
  const int kb = blockIdx.z * k_per_split;
  const int ke = min(K, kb + k_per_split);
  const int KT = (ke - kb + kTileK - 1) / kTileK;
  if (gridDim.z > 1) C += (size_t)blockIdx.z * M * ldc;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "n"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = instr_desc_bf16(kTileM, NT);
  bool ok = true;

  for (int kt = 0; kt < KT; ++kt) {
    const int buf = kt & 1;
    if (kt >= 2) ok = ok && mbar_wait(&mbar[buf], ((kt - 2) >> 1) & 1);   // MMAs of tile kt-2 done
    stage_tile(smem_u32(sA[buf]), A, lda, M, m0, kb + kt * kTileK, kTileM, tid);
    stage_tile(smem_u32(sB[buf]), B, ldb, N, n0, kb + kt * kTileK, NT, tid);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a0 = smem_u32(sA[buf]), b0 = smem_u32(sB[buf]);
#pragma unroll
      for (int k = 0; k < kTileK / 16; ++k) {
        // K step of 16 = two core matrices along K (128 B apart); core
        // matrices along M / N are 8 * 128 B apart.
        const uint64_t da = smem_desc(a0 + k * 256, 128, 1024);
        const uint64_t db = smem_desc(b0 + k * 256, 128, 1024);
        const uint32_t acc = (kt > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&mbar[buf]))
                   : "memory");
    }
    __syncthreads();
  }
  if (KT > 0) ok = ok && mbar_wait(&mbar[(KT - 1) & 1], ((KT - 1) >> 1) & 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  if (!ok) {
    if (tid == 0 && err) atomicExch(err, 1);
  } else {
    // epilogue: warp w owns TMEM lanes (rows) 32 w .. 32 w + 31
    const int row = m0 + warp * 32 + (tid & 31);
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
            "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (KT == 0) {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0u;   // empty K range: the product is zero
      }
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (col < N) {
            float x = __uint_as_float(v[j]);
            if (bias) x += bias[col];
            if (relu) x = fmaxf(x, 0.f);
            C[(size_t)row * ldc + col] = x;
            if (Cbf) Cbf[(size_t)row * ldc + col] = __float2bfloat16_rn(x);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(kTmemCols) : "memory");
}

template <int NT>
cudaError_t launch_gemm_t(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
                          float* C, int ldc, __nv_bfloat16* Cbf, const float* bias, int relu, int splits, int* err,
                          cudaStream_t st) {
  const size_t smem = 2 * (size_t)(kTileM + NT) * kTileK * 2;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16_tn<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int kps = ((K + splits - 1) / splits + kTileK - 1) / kTileK * kTileK;
  dim3 grid((M + kTileM - 1) / kTileM, (N + NT - 1) / NT, splits);
  k_gemm_bf16_tn<NT><<<grid, kGemmThreads, smem, st>>>(M, N, K, A, lda, B, ldb, C, ldc, Cbf, bias, relu, kps, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* C, int ldc,
                             void* Cbf, const float* bias, int relu, int splits, int* err, cudaStream_t st) {
  const __nv_bfloat16* a = static_cast<const __nv_bfloat16*>(A);
  const __nv_bfloat16* b = static_cast<const __nv_bfloat16*>(B);
  __nv_bfloat16* cb = static_cast<__nv_bfloat16*>(Cbf);
  if (N <= 32) return launch_gemm_t<32>(M, N, K, a, lda, b, ldb, C, ldc, cb, bias, relu, splits, err, st);
  if (N <= 64) return launch_gemm_t<64>(M, N, K, a, lda, b, ldb, C, ldc, cb, bias, relu, splits, err, st);
  if (N <= 128) return launch_gemm_t<128>(M, N, K, a, lda, b, ldb, C, ldc, cb, bias, relu, splits, err, st);
  return launch_gemm_t<256>(M, N, K, a, lda, b, ldb, C, ldc, cb, bias, relu, splits, err, st);
}

}  // namespace rimg
