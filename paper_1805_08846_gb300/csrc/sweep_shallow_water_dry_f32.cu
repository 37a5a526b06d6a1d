// Sweep kernels: shallow water over bathymetry with wetting and drying
// (hydrostatic reconstruction around HLLE), float, 2D only; one line per
// thread (the wet / dry decisions branch per cell).
#include <float.h>
#include <math.h>

#include "sweep_dispatch.cuh"

namespace claw {
cudaError_t launch_sweep_shallow_water_dry_f32(const SweepLaunch& L) {
    using S = ShallowWaterDry<float>;
    // a depth below the smallest normal float counts as dry in FP32 (the
    // solver's flush-to-zero SFU operations would read it as 0)
    const float tol = fmaxf((float)L.args.dry_tol, FLT_MIN);
    const S::Params P{(float)L.args.g, (float)sqrt(L.args.g), (float)(0.5 * L.args.g), tol};
    return sweep_by_dir<S, float, false>(L, P, P, P);
}
}  // namespace claw
