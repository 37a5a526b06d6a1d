// Unsplit update with transverse waves: linear acoustics (constant and
// per-cell coefficients), float.
#include "launch.h"
#include "unsplit.cuh"

namespace claw {
cudaError_t launch_unsplit_acoustics_f32(const SweepLaunch& L) {
    if (L.system == kSysAcousticsVar) {
        using S = Acoustics<float, true>;
        const S::Params P{0.0f, 0.0f, 0.0f};
        return unsplit_by_limiter<S, float>(L, P);
    }
    using S = Acoustics<float, false>;
    const S::Params P{(float)L.args.Z, (float)L.args.c, (float)(1.0 / (2.0 * L.args.Z))};
    return unsplit_by_limiter<S, float>(L, P);
}
}  // namespace claw
