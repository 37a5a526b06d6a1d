// Sweep kernels: variable-coefficient acoustics (per-cell Z, c), double.
#include "sweep_dispatch.cuh"

namespace claw {
cudaError_t launch_sweep_acoustics_var_f64(const SweepLaunch& L) {
    using S = Acoustics<double, true>;
    const S::Params P{(double)0, (double)0, (double)0};
    return sweep_by_dir<S, double, true>(L, P, P, P);
}
}  // namespace claw
