// double instantiation of the stepper (see stepper_impl.cuh).
#include "stepper_impl.cuh"

namespace nsstab {

StepperBase* make_stepper_f64(const nsstab_config& cfg, int nsets, const double* Re, const double* D, int per_set,
                              cudaStream_t stream) {
    return new StepperImpl<double>(cfg, nsets, Re, D, per_set, stream);
}

}  // namespace nsstab
