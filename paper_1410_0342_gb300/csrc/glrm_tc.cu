// C entry point of the tcgen05 GEMM building block (glrm_tc.cuh).
#include "glrm_tc.cuh"

namespace {
static __device__ int g_tc_err;
}

extern "C" int glrm_tc_gemm_bf16(const void *A_dev, const void *B_dev, float *D_dev, int32_t M, int32_t N,
                                 int32_t K, void *stream)
{
    using namespace glrm;
    if (!A_dev || !B_dev || !D_dev) return GLRM_ERR_ARG;
    if (M <= 0 || N <= 0 || M % 128 || N % kTcNT || (K != 16 && K != 32 && K != 64 && K != 128)) return GLRM_ERR_RANGE;
    cudaStream_t st = (cudaStream_t)stream;
    int *err = nullptr;
    if (cudaGetSymbolAddress((void **)&err, g_tc_err) != cudaSuccess) return GLRM_ERR_CUDA;
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return GLRM_ERR_CUDA;
    // at least 57 KB of dynamic shared memory: at most 4 CTAs per SM, whose
    // 4 x 64 TMEM columns always fit in the SM's 512 (1 KB slack aligns the base)
    const size_t smem = std::max<size_t>((size_t)(128 + kTcNT) * kTcMaxK * 2 + 1024, 57 * 1024);
    if (cudaFuncSetAttribute(tc_gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return GLRM_ERR_CUDA;
    dim3 grid((unsigned)(M / 128), (unsigned)(N / kTcNT));
    tc_gemm_bf16_kernel<<<grid, 128, smem, st>>>((const __nv_bfloat16 *)A_dev, (const __nv_bfloat16 *)B_dev,
                                                 D_dev, M, N, K, err);
    if (cudaGetLastError() != cudaSuccess) return GLRM_ERR_CUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GLRM_ERR_CUDA;
    return h ? GLRM_ERR_TIMEOUT : GLRM_OK;
}
