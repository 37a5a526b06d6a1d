// Sweep kernels: shallow water over bathymetry with wetting and drying
// (hydrostatic reconstruction around HLLE), double, 2D only.
#include <math.h>

#include "sweep_dispatch.cuh"

namespace claw {
cudaError_t launch_sweep_shallow_water_dry_f64(const SweepLaunch& L) {
    using S = ShallowWaterDry<double>;
    const S::Params P{L.args.g, sqrt(L.args.g), 0.5 * L.args.g, L.args.dry_tol};
    return sweep_by_dir<S, double, false>(L, P, P, P);
}
}  // namespace claw
