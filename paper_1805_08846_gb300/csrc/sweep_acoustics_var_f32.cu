// Sweep kernels: variable-coefficient acoustics (per-cell Z, c), float.
#include "sweep_dispatch.cuh"

namespace claw {
cudaError_t launch_sweep_acoustics_var_f32(const SweepLaunch& L) {
    using S = Acoustics<float, true>;
    const S::Params P{(float)0, (float)0, (float)0};
    return sweep_by_dir<S, float, true>(L, P, P, P);
}
}  // namespace claw
