// tt_umma.cu -- one 128 x N output tile through the tcgen05 tensor cores:
// C = A B^T with A [128][K], B [N][K] bfloat16 (row-major, K contiguous) and
// C [128][N] float.  The building block that the warm start's convolutions
// use, exposed on its own so that the descriptor and tensor-memory
// conventions can be checked against a plain product.
#include <cuda_bf16.h>

#include <cstdint>

#include "tt_internal.cuh"
#include "tt_umma.cuh"

using namespace tt;

namespace {

constexpr int kTileM = 128;
constexpr uint32_t kTmemCols = 256;          // >= any N this entry accepts
constexpr uint32_t kWaitTries = 1u << 22;

// Shared memory: A tile at 0, B tile, 32 KB spare, mbarrier, tensor-memory
// address.
__host__ __device__ inline uint32_t tile_b_offset(int K) { return kTileM * K * 2; }
__host__ __device__ inline uint32_t tile_mbar_offset(int N, int K)
{
    return (tile_b_offset(K) + N * K * 2 + 32768 + 15) & ~15u;
}

__global__ void __launch_bounds__(128, 1)
k_umma_tile(const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ B, float *__restrict__ C,
            int N, int K, int *__restrict__ status)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t b_off = tile_b_offset(K);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + tile_mbar_offset(N, K));
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);

    if (warp == 0) umma::tmem_alloc(tslot, kTmemCols);
    if (tid == 0) umma::mbar_init(mbar, 1);
    // operands into the K-major core-matrix layout: LBO = 128 B (next 8 K),
    // SBO = (K / 8) * 128 B (next 8 rows)
    const uint32_t lbo = 128, sbo = (uint32_t)(K / 8) * 128;
    for (int e = tid; e < kTileM * K; e += blockDim.x) {
        const int r = e / K, k = e % K;
        *reinterpret_cast<__nv_bfloat16 *>(smem + (r / 8) * sbo + (k / 8) * lbo + (r % 8) * 16 + (k % 8) * 2) = A[e];
    }
    for (int e = tid; e < N * K; e += blockDim.x) {
        const int r = e / K, k = e % K;
        *reinterpret_cast<__nv_bfloat16 *>(smem + b_off + (r / 8) * sbo + (k / 8) * lbo + (r % 8) * 16 + (k % 8) * 2) =
            B[e];
    }
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;

    if (tid == 0) {
        const uint32_t idesc = umma::idesc_bf16_f32(kTileM, N);
        const uint32_t sa = umma::smem_u32(smem), sb = umma::smem_u32(smem + b_off);
        for (int kk = 0; kk < K / 16; ++kk) {
            const uint64_t ad = umma::smem_desc(sa + kk * 2 * lbo, lbo, sbo);
            const uint64_t bd = umma::smem_desc(sb + kk * 2 * lbo, lbo, sbo);
            umma::mma_bf16(tmem, ad, bd, idesc, kk > 0 ? 1u : 0u);
        }
        umma::mma_commit(mbar);
    }
    const bool ok = umma::mbar_wait(mbar, 0, kWaitTries);
    umma::fence_after_sync();
    if (ok) {
        // warp w reads tensor-memory lanes 32 w .. 32 w + 31 = rows of C
        const int row = warp * 32 + lane;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            umma::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) C[row * N + c0 + i] = v[i];
        }
    } else if (tid == 0) {
        atomicExch(status, 1);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

extern "C" {

tt_status tt_umma_gemm_bf16(const void *A_dev, const void *B_dev, float *C_dev, int N, int K, int *status_dev,
                            void *stream)
{
    if (!A_dev || !B_dev || !C_dev || !status_dev) {
        set_error("tt_umma_gemm_bf16: null pointer");
        return TT_INVALID_ARG;
    }
    if (N < 16 || N > 256 || N % 16 != 0 || K < 16 || K > 256 || K % 16 != 0) {
        set_error("tt_umma_gemm_bf16: need N in 16..256 and K in 16..256, both multiples of 16");
        return TT_INVALID_ARG;
    }
    const size_t smem = tile_mbar_offset(N, K) + 64;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaFuncSetAttribute(k_umma_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(status_dev, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        k_umma_tile<<<1, 128, smem, s>>>((const __nv_bfloat16 *)A_dev, (const __nv_bfloat16 *)B_dev, C_dev, N, K,
                                         status_dev);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? TT_OK : cuda_fail(e, "tt_umma_gemm_bf16");
}

}  // extern "C"
