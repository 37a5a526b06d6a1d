// Sweep kernels: constant-coefficient acoustics, double state and arithmetic.
#include "sweep_dispatch.cuh"

namespace claw {
cudaError_t launch_sweep_acoustics_f64(const SweepLaunch& L) {
    using S = Acoustics<double, false>;
    const S::Params P{(double)L.args.Z, (double)L.args.c, (double)(1.0 / (2.0 * L.args.Z))};
    return sweep_by_dir<S, double, true>(L, P, P, P);
}
}  // namespace claw
