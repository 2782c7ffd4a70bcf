// FP64 staged (fused / blocked) half-step.
#include "glrm_tiled.cuh"

template cudaError_t glrm::Engine<double>::tiled_half_step(glrm_s *h, bool xstep);
