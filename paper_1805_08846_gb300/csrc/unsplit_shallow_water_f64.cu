// Unsplit update with transverse waves: shallow water (Roe + Harten-Hyman
// normal solver, Roe-average transverse solver), double.
#include <math.h>

#include "launch.h"
#include "unsplit.cuh"

namespace claw {
cudaError_t launch_unsplit_shallow_water_f64(const SweepLaunch& L) {
    using S = ShallowWater<double>;
    const S::Params P{L.args.g, sqrt(L.args.g), 0.5 * L.args.g};
    return unsplit_by_limiter<S, double>(L, P);
}
}  // namespace claw
