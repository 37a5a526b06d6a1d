// Unsplit update with transverse waves: shallow water (Roe + Harten-Hyman
// normal solver, Roe-average transverse solver), float.
#include <math.h>

#include "launch.h"
#include "unsplit.cuh"

namespace claw {
cudaError_t launch_unsplit_shallow_water_f32(const SweepLaunch& L) {
    using S = ShallowWater<float>;
    const S::Params P{(float)L.args.g, (float)sqrt(L.args.g), (float)(0.5 * L.args.g)};
    return unsplit_by_limiter<S, float>(L, P);
}
}  // namespace claw
