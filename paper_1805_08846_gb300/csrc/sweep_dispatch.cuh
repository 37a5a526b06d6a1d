// Compile-time dispatch of the sweep kernel over limiter, direction and
// pass kind; each instantiation unit includes this for one (system, Real).
#pragma once
#include "launch.h"
#include "sweep.cuh"

namespace claw {

template <class Sys, class Real, int LIM, int DIR>
cudaError_t sweep_go(const SweepLaunch& L, const typename Sys::Params& P) {
    if (L.grid == 0) return cudaSuccess;
    using Cfg = StageCfg<Sys, Real, DIR>;
    static int resident = 0;   // CTAs of this kernel the whole GPU holds at once
    if (!resident) {
        cudaError_t e = cudaFuncSetAttribute(sweep_kernel<Sys, Real, LIM, DIR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<Sys, Real, LIM, DIR>, kLines,
                                                          Cfg::SMEM);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        resident = per_sm * sms > 0 ? per_sm * sms : 1;
    }
    unsigned grid = L.grid;
    if (L.args.persistent && grid > (unsigned)resident) grid = (unsigned)resident;
    sweep_kernel<Sys, Real, LIM, DIR><<<grid, kLines, Cfg::SMEM, L.stream>>>(L.args, P);
    return cudaGetLastError();
}

template <class Sys, class Real, int DIR>
cudaError_t speed_go(const SweepLaunch& L, const typename Sys::Params& P) {
    if (L.grid == 0) return cudaSuccess;
    speed_kernel<Sys, Real, DIR><<<L.grid, kLines, 0, L.stream>>>(L.args, P);
    return cudaGetLastError();
}

template <class Sys, class Real, int DIR>
cudaError_t sweep_by_limiter(const SweepLaunch& L, const typename Sys::Params& P) {
    if (L.speeds) return speed_go<Sys, Real, DIR>(L, P);
    switch (L.limiter) {
        case kLimNone: return sweep_go<Sys, Real, kLimNone, DIR>(L, P);
        case kLimMinmod: return sweep_go<Sys, Real, kLimMinmod, DIR>(L, P);
        default: return sweep_go<Sys, Real, kLimMC, DIR>(L, P);
    }
}

template <class Sys, class Real, bool HAS_Z>
cudaError_t sweep_by_dir(const SweepLaunch& L, const typename Sys::Params& P) {
    switch (L.dir) {
        case 0: return sweep_by_limiter<Sys, Real, 0>(L, P);
        case 1: return sweep_by_limiter<Sys, Real, 1>(L, P);
        default:
            if constexpr (HAS_Z) return sweep_by_limiter<Sys, Real, 2>(L, P);
            return cudaErrorInvalidValue;
    }
}

}  // namespace claw
