// FP32 instantiation of the chunked sweep, objective, gradient, imputation
// and ALS engines and the BF16 form.  The staged (tiled) and masked
// half-steps are instantiated in their own translation units so that the
// library builds in parallel.
#include "glrm_als.cuh"
#include "glrm_bf16.cuh"

template struct glrm::Engine<float>;

namespace glrm {
cudaError_t bf16_half_step_entry(glrm_s *h, bool xstep) { return bf16_half_step(h, xstep); }
cudaError_t launch_perm(const Orient &o, const Orient &other, cudaStream_t st)
{
    perm_kernel<<<blocks_for(o.nseg, 8), 256, 0, st>>>(o.nseg, o.ptr, o.idx, other.ptr, other.idx, o.perm);
    return cudaGetLastError();
}
}  // namespace glrm
