// Tensor-core GEMM for the learned preconditioner (5th-generation tensor cores):
//   C[M][N] = act( A1[M][K1] B1[N][K1]^T + A2[M][K2] B2[N][K2]^T + bias )
// with BF16 operands, FP32 accumulation in tensor memory (TMEM) and FP32 or BF16
// output. One CTA of 128 threads owns a 128-row tile and the whole N (<= 256):
//   thread 0 loads every K-slab of A and B with TMA (cp.async.bulk.tensor, 128-byte
//   swizzle) onto one mbarrier, issues the tcgen05.mma chain into TMEM and commits
//   it to a second mbarrier; the four warps then read their 32 TMEM lanes back
//   (tcgen05.ld), add the bias, apply ReLU and store their rows.
// Operands are K-major: rows of 64 BF16 (128 bytes) per K-slab, 8-row groups 1024
// bytes apart (the canonical 128-byte-swizzle layout). K1, K2 are multiples of 64.
// Every mbarrier wait is bounded (about a second of SM clock); on timeout the CTA
// records *err, skips the rest of its work, frees its TMEM and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ldg_tcgen05.cuh"

namespace ldg {

constexpr int TC_BM = 128;        // rows per CTA (MMA M)
constexpr int TC_BK = 64;         // K elements per slab (128 bytes of BF16)
constexpr int TC_SLAB_A = TC_BM * TC_BK * 2;   // bytes of one A slab

struct TcGemmArgs {
  int M, N, K1, K2;         // K2 = 0: one operand pair
  const float* bias;        // [N] or null
  int relu;
  void* C;                  // [M][ldc] FP32 or BF16
  int ldc;
  int out_bf16;
  int* err;                 // set to 1 when a wait times out
  const int* skip;          // optional: return at once when *skip != 0
};

__global__ void __launch_bounds__(128, 1) k_tc_gemm(const __grid_constant__ CUtensorMap ta1,
                                                    const __grid_constant__ CUtensorMap tb1,
                                                    const __grid_constant__ CUtensorMap ta2,
                                                    const __grid_constant__ CUtensorMap tb2, TcGemmArgs g) {
  if (g.skip && *g.skip) return;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  // the 128-byte swizzle is a function of the shared-memory address: align that to 1024
  unsigned char* smem = tc_smem_raw + ((1024u - (smem_u32(tc_smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int ok_s;
  __shared__ float bias_s[256];   // the bias, read once per CTA (the epilogue reads it per column)
  const int nk1 = g.K1 / TC_BK, nk2 = g.K2 / TC_BK, nk = nk1 + nk2;
  const int N = g.N;
  const int slab_b = N * TC_BK * 2;
  unsigned char* sA = smem;
  unsigned char* sB = smem + (size_t)nk * TC_SLAB_A;
  const uint32_t ncols = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TC_BM;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ok_s = 1;
  }
  for (int c = threadIdx.x; c < N; c += blockDim.x) bias_s[c] = g.bias ? g.bias[c] : 0.f;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar_tma, (uint32_t)(nk * (TC_SLAB_A + slab_b)));
    for (int kb = 0; kb < nk1; ++kb) {
      tma_load_2d(sA + (size_t)kb * TC_SLAB_A, &ta1, kb * TC_BK, m0, &bar_tma);
      tma_load_2d(sB + (size_t)kb * slab_b, &tb1, kb * TC_BK, 0, &bar_tma);
    }
    for (int kb = 0; kb < nk2; ++kb) {
      tma_load_2d(sA + (size_t)(nk1 + kb) * TC_SLAB_A, &ta2, kb * TC_BK, m0, &bar_tma);
      tma_load_2d(sB + (size_t)(nk1 + kb) * slab_b, &tb2, kb * TC_BK, 0, &bar_tma);
    }
    if (mbar_wait(&bar_tma, 0)) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t idesc = bf16_idesc(TC_BM, N);
      for (int kb = 0; kb < nk; ++kb)
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk) {
          const uint64_t ad = sw128_desc(sA + (size_t)kb * TC_SLAB_A + kk * 32);
          const uint64_t bd = sw128_desc(sB + (size_t)kb * slab_b + kk * 32);
          tc_mma(tmem, ad, bd, idesc, (kb | kk) != 0);
        }
      tc_commit(&bar_mma);
    } else {
      // the loads may still be landing in shared memory: give them a second bounded
      // wait before the CTA exits (no MMA was issued, so the tensor memory is idle)
      ok_s = 0;
      atomicExch(g.err, 1);
      (void)mbar_wait(&bar_tma, 0);
    }
  }
  __syncthreads();
  if (ok_s) {
    // every lane of a warp takes the same branch (tcgen05.ld is warp-collective)
    const bool mma_done = __all_sync(0xffffffffu, mbar_wait(&bar_mma, 0));
    if (!mma_done) {
      // a second bounded wait for the MMAs still writing the accumulator, so that the
      // tensor memory is not released under them
      atomicExch(g.err, 1);
      (void)mbar_wait(&bar_mma, 0);
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // the warp's 32 rows go through shared memory (the operand slabs, idle once the MMAs
      // are done): each lane writes its row there, then the warp stores whole rows, so that
      // every 32-byte sector of the output is written once and in full
      const int esz = g.out_bf16 ? 2 : 4;
      const int rowb = N * esz + 16;   // 16 bytes of padding staggers the rows over the banks
      unsigned char* stage = smem + (size_t)warp * 32 * rowb;
      const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tc_ld16(lane_addr + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float x = v[i] + bias_s[c0 + i];
          if (g.relu) x = fmaxf(x, 0.f);
          v[i] = x;
        }
        unsigned char* dst = stage + (size_t)lane * rowb + (size_t)c0 * esz;
        if (g.out_bf16) {
          uint32_t pk[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            pk[i] = *reinterpret_cast<uint32_t*>(&b2);
          }
          reinterpret_cast<uint4*>(dst)[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          reinterpret_cast<uint4*>(dst)[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            reinterpret_cast<float4*>(dst)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
      }
      __syncwarp();
      // rows of N * esz bytes (a multiple of 32) as 16-byte pieces, consecutive lanes on
      // consecutive pieces of a row
      const int pieces = N * esz / 16, total = 32 * pieces;
      unsigned char* gout = (unsigned char*)g.C;
      const size_t ldcb = (size_t)g.ldc * esz;
      for (int q = lane; q < total; q += 32) {
        const int r = q / pieces, pc = q - r * pieces;
        const int grow = m0 + warp * 32 + r;
        if (grow < g.M)
          *reinterpret_cast<uint4*>(gout + (size_t)grow * ldcb + (size_t)pc * 16) =
              *reinterpret_cast<const uint4*>(stage + (size_t)r * rowb + (size_t)pc * 16);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// dynamic shared memory of k_tc_gemm: the operand slabs, or the output staging of the
// epilogue if that is larger (+1 KB for the 1024-byte alignment)
inline size_t tc_gemm_smem(int N, int K1, int K2, int out_bf16) {
  const int nk = (K1 + K2) / TC_BK;
  const size_t slabs = (size_t)nk * (TC_SLAB_A + (size_t)N * TC_BK * 2);
  const size_t stage = (size_t)TC_BM * ((size_t)N * (out_bf16 ? 2 : 4) + 16);
  return (slabs > stage ? slabs : stage) + 1024;
}

// FP32 -> BF16, row-major with independent strides (rows x cols)
__global__ void k_to_bf16_2d(const float* __restrict__ src, int lds, __nv_bfloat16* __restrict__ dst, int ldd,
                             int64_t rows, int cols, const int* skip) {
  if (skip && *skip) return;
  const int64_t total = rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / cols;
    const int c = (int)(i - r * cols);
    dst[r * ldd + c] = __float2bfloat16(src[r * lds + c]);
  }
}

}  // namespace ldg
