// Host-side launchers of the library's kernels (defined in the .cu files).
#pragma once
#include <cuda_runtime.h>
#include "claw_types.cuh"

namespace claw {

enum : int {
    kSysAcoustics = 0,
    kSysAcousticsVar = 1,
    kSysShallowWater = 2,
    kSysShallowWaterBathy = 3,
    kSysShallowWaterDry = 4
};

struct SweepLaunch {
    SweepArgs args;
    int system;
    int limiter;
    int dir;
    int precision;   // 32 or 64
    bool speeds;     // speeds-only pass (CFL estimate), no update
    unsigned grid;   // CTAs (one per tile)
    cudaStream_t stream;
    int* resident_out;   // non-null: report the CTAs the GPU holds at once, launch nothing
    int* chunk_out;      // non-null: report the cells per staged chunk, launch nothing
    int* lines_out;      // non-null: report the lines per tile, launch nothing
    int narrow;          // 1: the narrow tile width (half the lines per tile), where offered
};

// Record the thread-local message claw_last_error() returns.
void set_last_error(const char* msg);

// Dispatch to the (system, precision) instantiation unit.
cudaError_t launch_sweep(const SweepLaunch& L);
cudaError_t launch_sweep_acoustics_f32(const SweepLaunch& L);
cudaError_t launch_sweep_acoustics_f64(const SweepLaunch& L);
cudaError_t launch_sweep_acoustics_var_f32(const SweepLaunch& L);
cudaError_t launch_sweep_acoustics_var_f64(const SweepLaunch& L);
cudaError_t launch_sweep_shallow_water_f32(const SweepLaunch& L);
cudaError_t launch_sweep_shallow_water_f64(const SweepLaunch& L);
cudaError_t launch_sweep_shallow_water_bathy_f32(const SweepLaunch& L);
cudaError_t launch_sweep_shallow_water_bathy_f64(const SweepLaunch& L);
cudaError_t launch_sweep_shallow_water_dry_f32(const SweepLaunch& L);
cudaError_t launch_sweep_shallow_water_dry_f64(const SweepLaunch& L);

// Unsplit update with transverse waves (2D acoustics and shallow water):
// one launch per step attempt over the strip tiles in args.tiles (TileDesc:
// line0 = first output column of a 28-column strip, [a, b) = rows), grid =
// CTAs of four one-warp tiles.  lines_out reports the output columns of a strip.
cudaError_t launch_unsplit(const SweepLaunch& L);
cudaError_t launch_unsplit_acoustics_f32(const SweepLaunch& L);
cudaError_t launch_unsplit_acoustics_f64(const SweepLaunch& L);
cudaError_t launch_unsplit_shallow_water_f32(const SweepLaunch& L);
cudaError_t launch_unsplit_shallow_water_f64(const SweepLaunch& L);

struct FinalSlots {
    int off[4];      // slot offset of each field's result after a full step
    int m;
};

// Step control (control.cu).
cudaError_t launch_arm(Control* ctl, int lo, int hi, int mode, long long nsteps, double t_final,
                       double fixed_dt, double cfl_desired, int* counters, cudaStream_t st);
cudaError_t launch_finish(Control* ctl, const InstDesc* inst, int lo, int hi, FinalSlots fs,
                          int* counters, cudaStream_t st);
cudaError_t launch_speed_reduce(Control* ctl, const InstDesc* inst, int lo, int hi, int set_dt,
                                cudaStream_t st);
cudaError_t launch_set_time(Control* ctl, int i, double t, double dt, long long nsteps,
                            cudaStream_t st);
cudaError_t launch_reset_status(Control* ctl, int i, cudaStream_t st);

// State conversion and reductions (control.cu); Real chosen by precision.
cudaError_t launch_convert_in(int precision, void* pool, const InstDesc& I, const Control* ctl,
                              const double* src, int m, cudaStream_t st);
cudaError_t launch_convert_out(int precision, const void* pool, const InstDesc& I,
                               const Control* ctl, double* dst, int m, cudaStream_t st);
cudaError_t launch_fill(int precision, void* pool, const InstDesc& I, int slot, int f, double v,
                        cudaStream_t st);
cudaError_t launch_aux(int precision, void* aux, const InstDesc& I, const double* rho,
                       const double* K, cudaStream_t st);
cudaError_t launch_aux_const(int precision, void* aux, const InstDesc& I, double rho, double K,
                             cudaStream_t st);
// One material plane (FP64 values, x fastest, no padding) into plane k.
cudaError_t launch_aux_plane(int precision, void* aux, const InstDesc& I, int k, const double* src,
                             cudaStream_t st);
// out: 8 doubles for the sums followed by room for 8 x kSumPartsMax partials.
constexpr int kSumPartsMax = 256;
cudaError_t launch_sums(int precision, const void* pool, const InstDesc& I, const Control* ctl,
                        int m, double* out, cudaStream_t st);

}  // namespace claw
