// Sweep kernels: shallow water (Roe + Harten-Hyman), float, 2D only.
#include <math.h>

#include "sweep_dispatch.cuh"

namespace claw {
cudaError_t launch_sweep_shallow_water_f32(const SweepLaunch& L) {
    using S = ShallowWater<float>;
    const S::Params P{(float)L.args.g, (float)sqrt(L.args.g)};
    return sweep_by_dir<S, float, false>(L, P);
}
}  // namespace claw
