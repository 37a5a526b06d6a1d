// Compile-time dispatch of the sweep kernel over limiter, direction and
// pass kind; each instantiation unit includes this for one (system, Real).
#pragma once
#include "launch.h"
#include "sweep.cuh"

namespace claw {

template <class Sys, class Real, int LIM, int DIR, bool NARROW>
cudaError_t sweep_go_w(const SweepLaunch& L, const typename Sys::Params& P) {
    if (L.grid == 0) return cudaSuccess;
    using Cfg = StageCfg<Sys, Real, DIR, NARROW>;
    if (L.chunk_out || L.lines_out) {
        if (L.chunk_out) *L.chunk_out = Cfg::C;
        if (L.lines_out) *L.lines_out = Cfg::LINES;
        return cudaSuccess;
    }
    static int resident = 0;   // CTAs of this kernel the whole GPU holds at once
    if (!resident) {
        cudaError_t e = cudaFuncSetAttribute(sweep_kernel<Sys, Real, LIM, DIR, NARROW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        // all of L1 that can be shared memory: the resident CTA count is set
        // by the staging rings, not left to the driver's default split
        e = cudaFuncSetAttribute(sweep_kernel<Sys, Real, LIM, DIR, NARROW>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<Sys, Real, LIM, DIR, NARROW>, Cfg::NT,
                                                          Cfg::SMEM);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        resident = per_sm * sms > 0 ? per_sm * sms : 1;
    }
    if (L.resident_out) {
        *L.resident_out = resident;
        return cudaSuccess;
    }
    unsigned grid = L.grid;
    if (L.args.persistent && grid > (unsigned)resident) grid = (unsigned)resident;
    sweep_kernel<Sys, Real, LIM, DIR, NARROW><<<grid, Cfg::NT, Cfg::SMEM, L.stream>>>(L.args, P);
    return cudaGetLastError();
}

// The tile width: narrow (half the lines per tile) where the sweep offers it.
template <class Sys, class Real, int LIM, int DIR>
cudaError_t sweep_go(const SweepLaunch& L, const typename Sys::Params& P) {
    if constexpr (narrow_offered<Sys, DIR>()) {
        if (L.narrow) return sweep_go_w<Sys, Real, LIM, DIR, true>(L, P);
    }
    return sweep_go_w<Sys, Real, LIM, DIR, false>(L, P);
}

template <class Sys, class Real, int DIR>
cudaError_t speed_go(const SweepLaunch& L, const typename Sys::Params& P) {
    if (L.grid == 0) return cudaSuccess;
    speed_kernel<Sys, Real, DIR><<<L.grid, kLines, 0, L.stream>>>(L.args, P);
    return cudaGetLastError();
}

// Sys: the system of the speeds-only pass (scalar Real); SysX, SysT: the
// systems the x and the y, z sweeps compute with (Sys itself, or its
// two-line f2 form).
template <class Sys, class SysS, class Real, int DIR>
cudaError_t sweep_by_limiter(const SweepLaunch& L, const typename Sys::Params& P,
                             const typename SysS::Params& PS) {
    if (L.speeds) return speed_go<Sys, Real, DIR>(L, P);
    switch (L.limiter) {
        case kLimNone: return sweep_go<SysS, Real, kLimNone, DIR>(L, PS);
        case kLimMinmod: return sweep_go<SysS, Real, kLimMinmod, DIR>(L, PS);
        case kLimFirstOrder: return sweep_go<SysS, Real, kLimFirstOrder, DIR>(L, PS);
        default: return sweep_go<SysS, Real, kLimMC, DIR>(L, PS);
    }
}

template <class Sys, class Real, bool HAS_Z, class SysX = Sys, class SysT = Sys>
cudaError_t sweep_by_dir(const SweepLaunch& L, const typename Sys::Params& P,
                         const typename SysX::Params& PX, const typename SysT::Params& PT) {
    switch (L.dir) {
        case 0: return sweep_by_limiter<Sys, SysX, Real, 0>(L, P, PX);
        case 1: return sweep_by_limiter<Sys, SysT, Real, 1>(L, P, PT);
        default:
            if constexpr (HAS_Z) return sweep_by_limiter<Sys, SysT, Real, 2>(L, P, PT);
            return cudaErrorInvalidValue;
    }
}

}  // namespace claw
