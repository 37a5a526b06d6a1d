// Sweep kernels: shallow water over bathymetry (f-waves), double, 2D only.
#include <math.h>

#include "sweep_dispatch.cuh"

namespace claw {
cudaError_t launch_sweep_shallow_water_bathy_f64(const SweepLaunch& L) {
    using S = ShallowWaterBathy<double>;
    const S::Params P{(double)L.args.g, (double)sqrt(L.args.g), 0.5 * L.args.g};
    return sweep_by_dir<S, double, false>(L, P, P, P);
}
}  // namespace claw
