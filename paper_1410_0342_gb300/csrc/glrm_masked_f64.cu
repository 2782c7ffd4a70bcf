// FP64 masked-tile half-step.
#include "glrm_masked.cuh"

template cudaError_t glrm::Engine<double>::masked_half_step(glrm_s *h, bool xstep);
