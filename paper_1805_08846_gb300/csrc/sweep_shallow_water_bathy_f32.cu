// Sweep kernels: shallow water over bathymetry (f-waves), float, 2D only.
// The sweeps march two lines per thread on packed FP32 pairs (f2); the
// speeds-only pass stays scalar.
#include <math.h>

#include "sweep_dispatch.cuh"

namespace claw {
cudaError_t launch_sweep_shallow_water_bathy_f32(const SweepLaunch& L) {
    using S = ShallowWaterBathy<float>;
    using S2 = ShallowWaterBathy<f2>;
    const float g = (float)L.args.g, sg = (float)sqrt(L.args.g), hg = (float)(0.5 * L.args.g);
    const S::Params P{g, sg, hg};
    const S2::Params P2{f2(g), f2(sg), f2(hg)};
    return sweep_by_dir<S, float, false, S2, S2>(L, P, P2, P2);
}
}  // namespace claw
