// Sweep kernels: constant-coefficient acoustics, float state and arithmetic.
#include "sweep_dispatch.cuh"

namespace claw {
cudaError_t launch_sweep_acoustics_f32(const SweepLaunch& L) {
    using S = Acoustics<float, false>;
    const S::Params P{(float)L.args.Z, (float)L.args.c, (float)(1.0 / (2.0 * L.args.Z))};
    return sweep_by_dir<S, float, true>(L, P, P, P);
}
}  // namespace claw
