// float instantiation of the stepper (see stepper_impl.cuh).
#include "stepper_impl.cuh"
#include "ragged.cuh"

namespace nsstab {

StepperBase* make_stepper_f32(const nsstab_config& cfg, int nsets, const double* Re, const double* D, int per_set,
                              cudaStream_t stream) {
    return new StepperImpl<float>(cfg, nsets, Re, D, per_set, stream);
}

RaggedBase* make_ragged_f32(cudaStream_t stream) { return new RaggedF32(stream); }

}  // namespace nsstab
