// C entry point of the tcgen05 GEMM building block (glrm_tc.cuh), and two
// instrumentation entry points: the bounded-wait self-test and an FP32 FMA
// throughput probe (the denominator of the CUDA-core roofline).
#include "glrm_tc.cuh"

namespace {
static __device__ int g_tc_err;
static __device__ int g_wait_err;

// Self-test of the bounded wait used by every staged copy and tensor-core
// completion in the library: one thread waits, with the library's own
// mbar_wait_bounded and a caller-given attempt count, on an mbarrier phase.
// With `arm` the thread first arrives on the barrier itself, so the phase
// completes and the wait succeeds; without it nothing ever arrives, the wait
// runs out, and the kernel takes the library's expiry path: it raises the
// status flag and returns.  No copy or tensor-core operation is issued, so
// nothing is in flight when the wait gives up.
__global__ void wait_selftest_kernel(long limit, int arm, int *err)
{
    __shared__ uint64_t bar;
    glrm::mbar_init(&bar, 1);
    if (arm) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(glrm::smem_u32(&bar)) : "memory");
    if (!glrm::mbar_wait_bounded(&bar, 0, limit)) atomicOr(err, 1);
}

// FP32 FMA throughput: every thread runs 8 independent dependency chains of
// `iters` fmaf each (8 chains hide the FMA latency at full occupancy); the
// result is stored only when it is impossible (sink < 0 never holds for the
// values used), so the compiler keeps every FMA.
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, float b, float c, float *sink)
{
    float a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = 1.0f + 0.001f * (float)(threadIdx.x + q);
    for (int it = 0; it < iters; it += 16) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = fmaf(a[q], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += a[q];
    if (s < 0.f) sink[blockIdx.x] = s;
}
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

extern "C" int glrm_wait_selftest(int64_t attempts, int32_t arm, void *stream)
{
    if (attempts < 1) return GLRM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int *err = nullptr;
    if (cudaGetSymbolAddress((void **)&err, g_wait_err) != cudaSuccess) return GLRM_ERR_CUDA;
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return GLRM_ERR_CUDA;
    wait_selftest_kernel<<<1, 1, 0, st>>>((long)attempts, arm ? 1 : 0, err);
    if (cudaGetLastError() != cudaSuccess) return GLRM_ERR_CUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GLRM_ERR_CUDA;
    return h ? GLRM_ERR_TIMEOUT : GLRM_OK;
}

extern "C" int glrm_fma_peak(int32_t iters, double *tflops_host, int32_t *sms_host, void *stream)
{
    if (iters < 16 || iters % 16 || !tflops_host) return GLRM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel, 256, 0) != cudaSuccess)
        return GLRM_ERR_CUDA;
    const unsigned grid = (unsigned)(sms * std::max(per_sm, 1));
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GLRM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GLRM_ERR_CUDA;
    }
    int rc = GLRM_OK;
    const int reps = 5;
    fma_probe_kernel<<<grid, 256, 0, st>>>(iters, 0.9999f, 1e-4f, nullptr);  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) fma_probe_kernel<<<grid, 256, 0, st>>>(iters, 0.9999f, 1e-4f, nullptr);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
        rc = GLRM_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GLRM_OK) return rc;
    const double flops = 2.0 * 8.0 * (double)iters * 256.0 * (double)grid * reps;
    *tflops_host = flops / (ms * 1e-3) / 1e12;
    if (sms_host) *sms_host = sms;
    return GLRM_OK;
}
