// FP32 instantiation of the chunked sweep, objective, gradient, imputation
// and ALS engines and the BF16 form.  The staged (tiled) and masked
// half-steps are instantiated in their own translation units so that the
// library builds in parallel.
#include "glrm_als.cuh"
#include "glrm_bf16.cuh"

template struct glrm::Engine<float>;

namespace glrm {

static __global__ void fill_i32_kernel(int32_t *p, int64_t n, int32_t v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

cudaError_t bf16_half_step_entry(glrm_s *h, bool xstep) { return bf16_half_step(h, xstep); }

cudaError_t launch_fill_i32(int32_t *p, int64_t n, int32_t v, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    fill_i32_kernel<<<blocks_for(n, 256), 256, 0, st>>>(p, n, v);
    return cudaGetLastError();
}

}  // namespace glrm
