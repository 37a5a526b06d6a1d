// Unsplit update with transverse waves: linear acoustics (constant and
// per-cell coefficients), double.
#include "launch.h"
#include "unsplit.cuh"

namespace claw {
cudaError_t launch_unsplit_acoustics_f64(const SweepLaunch& L) {
    if (L.system == kSysAcousticsVar) {
        using S = Acoustics<double, true>;
        const S::Params P{0.0, 0.0, 0.0};
        return unsplit_by_limiter<S, double>(L, P);
    }
    using S = Acoustics<double, false>;
    const S::Params P{L.args.Z, L.args.c, 1.0 / (2.0 * L.args.Z)};
    return unsplit_by_limiter<S, double>(L, P);
}
}  // namespace claw
