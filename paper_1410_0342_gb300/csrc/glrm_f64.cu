// FP64 instantiation of the chunked sweep, objective, gradient, imputation
// and ALS engines (the staged and masked half-steps build in their own
// translation units; the BF16 form exists for FP32 models only).
#include "glrm_als.cuh"

template struct glrm::Engine<double>;
