// Sweep kernels: shallow water (Roe + Harten-Hyman), float, 2D only.  The
// sweeps march two lines per thread on packed FP32 pairs (f2); the
// speeds-only pass stays scalar.
#include <math.h>

#include "sweep_dispatch.cuh"

namespace claw {
cudaError_t launch_sweep_shallow_water_f32(const SweepLaunch& L) {
    using S = ShallowWater<float>;
    using S2 = ShallowWater<f2>;
    const float g = (float)L.args.g, sg = (float)sqrt(L.args.g), hg = (float)(0.5 * L.args.g);
    const S::Params P{g, sg, hg};
    const S2::Params P2{f2(g), f2(sg), f2(hg)};
    return sweep_by_dir<S, float, false, S2, S2>(L, P, P2, P2);
}
}  // namespace claw
