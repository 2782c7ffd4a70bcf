// FP32 masked-tile half-step, and the masked layout's set-up kernels.
#include "glrm_masked.cuh"

template cudaError_t glrm::Engine<float>::masked_half_step(glrm_s *h, bool xstep);

namespace glrm {
cudaError_t launch_mt_count(const Orient &o, int64_t nother, int32_t *cnt, cudaStream_t st)
{
    return mt_count(o, nother, cnt, st);
}
cudaError_t launch_mt_build(const Orient &o, int prec, cudaStream_t st)
{
    return prec == GLRM_FP64 ? mt_build<double>(o, st) : mt_build<float>(o, st);
}
}  // namespace glrm
