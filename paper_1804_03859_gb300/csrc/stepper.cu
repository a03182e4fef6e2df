// Stepper factory and configuration checks.  The stepper's kernels and host
// class are templates (stepper_impl.cuh) instantiated once per arithmetic in
// stepper_f64.cu (FP64), stepper_f32.cu (FP32) and stepper_df64.cu
// (double-float), compiled in parallel.
#include "stepper.cuh"

namespace nsstab {

StepperBase* make_stepper_f64(const nsstab_config&, int, const double*, const double*, int, cudaStream_t);
StepperBase* make_stepper_f32(const nsstab_config&, int, const double*, const double*, int, cudaStream_t);
StepperBase* make_stepper_df64(const nsstab_config&, int, const double*, const double*, int, cudaStream_t);

int validate_config(const nsstab_config& c) {
    auto bad = [](const char* m) {
        set_error(m);
        return NSSTAB_ERR_INVALID_ARG;
    };
    if (!is_pow2(c.nx) || !is_pow2(c.ny) || c.nx < 8 || c.ny < 8 || c.nx > 4096 || c.ny > 4096)
        return bad("nx and ny must be powers of two in [8, 4096]");
    if (!(c.Lx > 0) || !(c.Ly > 0) || !(c.dt > 0) || !(c.Re > 0)) return bad("Lx, Ly, dt and Re must be positive");
    if (c.cyl_D > 0 && !(c.eta > 0)) return bad("eta must be positive when the cylinder is enabled");
    if (c.cyl_D > 0 && !(c.mask_cells > 0)) return bad("mask_cells must be positive");
    if (c.sponge_sigma > 0 && !(c.sponge_frac > 0 && c.sponge_frac <= 1)) return bad("sponge_frac must be in (0, 1]");
    if (c.precision != 64 && c.precision != 32 && c.precision != 48)
        return bad("precision must be 64 (FP64), 32 (FP32) or 48 (double-float)");
    return NSSTAB_OK;
}

StepperBase* make_stepper(const nsstab_config& cfg, int nsets, const double* Re, const double* D, int per_set,
                          cudaStream_t stream) {
    if (cfg.precision == 32) return make_stepper_f32(cfg, nsets, Re, D, per_set, stream);
    if (cfg.precision == 48) return make_stepper_df64(cfg, nsets, Re, D, per_set, stream);
    return make_stepper_f64(cfg, nsets, Re, D, per_set, stream);
}

}  // namespace nsstab
