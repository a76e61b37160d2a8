// A single tensor-core tile, D = A B^T with A [128][K] and B [N][K] rounded to
// BF16 and FP32 accumulation in tensor memory: the primitive the BF16 distance
// tiles of the kNN search are built from, exposed for diagnostics.
#include "vb_internal.cuh"
#include "tc.cuh"

#include <cuda_bf16.h>

namespace vb {

__global__ void __launch_bounds__(128) tc_dot_tile_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                          int K, int N, float* D, DevReport* rep)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __nv_bfloat16* sa = (__nv_bfloat16*)smem;
    __nv_bfloat16* sb = sa + 128 * K;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int t = threadIdx.x, warp = t >> 5;
    for (int idx = t; idx < 128 * K; idx += 128) {
        const int row = idx / K, k = idx - (idx / K) * K;
        sa[tc::operand_offset(row, k, K) >> 1] = __float2bfloat16_rn(A[idx]);
    }
    for (int idx = t; idx < N * K; idx += 128) {
        const int row = idx / K, k = idx - (idx / K) * K;
        sb[tc::operand_offset(row, k, K) >> 1] = __float2bfloat16_rn(B[idx]);
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, 128);
    if (t == 0) tc::mbar_init(&bar, 1);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = tmem_base;
    if (t == 0) {
        const uint32_t sbo = (uint32_t)(K >> 3) * 128;
        for (int s = 0; s < K / 16; ++s) {
            const uint64_t ad = tc::smem_desc(tc::smem_addr(sa) + s * 256, 128, sbo);
            const uint64_t bd = tc::smem_desc(tc::smem_addr(sb) + s * 256, 128, sbo);
            tc::mma_bf16(tb, ad, bd, tc::idesc_bf16(128, N), s > 0 ? 1u : 0u);
        }
        tc::mma_commit(&bar);
    }
    const bool ok = tc::mbar_wait(&bar, 0);
    tc::fence_after_sync();
    if (!ok) {
        if (t == 0) report_error(rep, VB_ERR_TIMEOUT);
    } else {
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tb + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) D[t * N + c0 + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tb, 128);
}

}  // namespace vb

using namespace vb;

extern "C" vb_status vb_tc_dot_tile(vb_ctx* ctx, const float* a, const float* b, int32_t K, int32_t N, float* d)
{
    if (!ctx || !a || !b || !d || K < 16 || K > 128 || K % 16 || N < 32 || N > 128 || N % 32) return VB_ERR_ARG;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    const size_t sm = (size_t)(128 + N) * K * 2;
    static bool attr[16] = {};
    if (!attr[c->device & 15]) {
        if (cudaFuncSetAttribute(tc_dot_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 256 * 128 * 2) !=
            cudaSuccess)
            return VB_ERR_CUDA;
        attr[c->device & 15] = true;
    }
    tc_dot_tile_kernel<<<1, 128, sm, c->stream>>>(a, b, K, N, d, c->rep);
    c->launches += 1;
    return last_launch();
}
