// Step control on the device (CUDACLAW Sec. 4.1: the speed reduction and
// the CFL kernel that keeps or reverts a step and sets the next one, Eq.
// CFL-condition), plus state conversion and conservation sums.
//
// A step attempt is: the sweeps (which read Control::dt_attempt and write the
// version slots after Control::cur), then finish_kernel, which forms
//   M = max_d (max|s^p|_d / dx_d)       (FP64, each max widened exactly)
// and keeps the attempt if dt_attempt * M <= cfl_max (rotating cur[] to the
// new slots, t += dt_attempt) or rejects it (cur[] unchanged, so the next
// attempt re-reads the same state), then proposes dt = cfl_desired / M and
// prepares the next attempt.  All of it lives on the device, so any number
// of attempts can be replayed from one CUDA graph without a host round trip.
#include <float.h>
#include "launch.h"

namespace claw {

__device__ __forceinline__ double next_dt(const Control& c, double M) {
    double dt = M > 0.0 ? c.cfl_desired / M : c.dt_max;
    return dt < c.dt_max ? dt : c.dt_max;
}

// Decide whether the next attempt runs and with which step.
__device__ __forceinline__ void prepare_attempt(Control& c) {
    c.last = 0;
    if (c.status) {
        c.active = 0;
        return;
    }
    const double dt = c.fixed_dt > 0.0 ? c.fixed_dt : c.dt;
    if (c.mode == kModeSteps) {
        c.active = c.nacc < c.target;
        c.dt_attempt = dt;
    } else if (c.mode == kModeTFinal) {
        c.active = c.t < c.t_final;
        double d = dt;
        if (d >= c.t_final - c.t) {
            d = c.t_final - c.t;
            c.last = 1;
        }
        c.dt_attempt = d;
    } else {
        c.active = 0;
    }
}

__global__ void arm_kernel(Control* ctl, int lo, int hi, int mode, long long nsteps,
                           double t_final, double fixed_dt, double cfl_desired, int* counters) {
    const int i = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (i == lo && counters)
        for (int k = 0; k < kMaxSweeps; ++k) counters[k] = 0;
    if (i >= hi) return;
    Control& c = ctl[i];
    if (cfl_desired > 0.0 && cfl_desired != c.cfl_desired) {
        c.cfl_desired = cfl_desired;
        c.dt = next_dt(c, c.M_last);
    }
    c.mode = mode;
    c.target = c.nacc + nsteps;
    c.t_final = t_final;
    c.fixed_dt = fixed_dt;
    c.streak = 0;
    c.smax[0] = c.smax[1] = c.smax[2] = 0ull;
    c.bad = 0u;
    c.cfl_peak = 0.0;
    prepare_attempt(c);
}

__global__ void finish_kernel(Control* ctl, const InstDesc* inst, int lo, int hi, FinalSlots fs,
                              int* counters) {
    const int i = lo + blockIdx.x * blockDim.x + threadIdx.x;
    // the sweeps of this attempt are done: rewind their tile schedules
    if (i == lo && counters)
        for (int k = 0; k < kMaxSweeps; ++k) counters[k] = 0;
    if (i >= hi) return;
    Control& c = ctl[i];
    if (!c.active) return;
    const InstDesc& I = inst[i];
    if (c.status) {   // a sweep latched a fault (e.g. a timed-out copy): keep nothing
        c.active = 0;
        return;
    }
    double M = 0.0;
    bool nonfinite = false;
    for (int d = 0; d < I.ndim; ++d) {
        const double md = __longlong_as_double((long long)c.smax[d]);
        c.smax[d] = 0ull;
        if (!(md <= DBL_MAX)) nonfinite = true;
        const double v = md / I.dx[d];
        if (v > M) M = v;
    }
    if (nonfinite || c.bad) {
        c.status |= kStatNonPhys;
        c.bad = 0u;
        c.active = 0;
        return;
    }
    const double cfl = c.dt_attempt * M;
    c.cfl_last = cfl;
    c.M_last = M;
    if (c.fixed_dt <= 0.0 && cfl > c.cfl_max) {
        c.nrej += 1;
        c.dt = next_dt(c, M);
        if (++c.streak > c.max_retries) {
            c.status |= kStatCfl;
            c.active = 0;
            return;
        }
    } else {
        c.streak = 0;
        if (cfl > c.cfl_peak) c.cfl_peak = cfl;
        for (int f = 0; f < fs.m; ++f) c.cur[f] = (c.cur[f] + fs.off[f]) % 3;
        c.t = c.last ? c.t_final : c.t + c.dt_attempt;
        c.nacc += 1;
        if (c.fixed_dt <= 0.0) c.dt = next_dt(c, M);
    }
    prepare_attempt(c);
}

// After a speeds-only pass: M from the per-direction maxima; optionally the
// next step cfl_desired / M (initial step of a new state).
__global__ void speed_reduce_kernel(Control* ctl, const InstDesc* inst, int lo, int hi, int set_dt) {
    const int i = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hi) return;
    Control& c = ctl[i];
    const InstDesc& I = inst[i];
    double M = 0.0;
    bool nonfinite = false;
    for (int d = 0; d < I.ndim; ++d) {
        const double md = __longlong_as_double((long long)c.smax[d]);
        c.smax[d] = 0ull;
        if (!(md <= DBL_MAX)) nonfinite = true;
        const double v = md / I.dx[d];
        if (v > M) M = v;
    }
    if (nonfinite) c.status |= kStatNonPhys;
    c.M_last = M;
    if (set_dt) c.dt = next_dt(c, M);
}

__global__ void set_time_kernel(Control* ctl, int i, double t, double dt, long long nsteps) {
    Control& c = ctl[i];
    c.t = t;
    c.nacc = nsteps;
    if (dt > 0.0) c.dt = dt;
}

__global__ void reset_status_kernel(Control* ctl, int i) {
    ctl[i].status = 0u;
    ctl[i].bad = 0u;
    ctl[i].streak = 0;
}

cudaError_t launch_arm(Control* ctl, int lo, int hi, int mode, long long nsteps, double t_final,
                       double fixed_dt, double cfl_desired, int* counters, cudaStream_t st) {
    const int n = hi - lo;
    if (n <= 0) return cudaSuccess;
    arm_kernel<<<(n + 127) / 128, 128, 0, st>>>(ctl, lo, hi, mode, nsteps, t_final, fixed_dt,
                                                cfl_desired, counters);
    return cudaGetLastError();
}

cudaError_t launch_finish(Control* ctl, const InstDesc* inst, int lo, int hi, FinalSlots fs,
                          int* counters, cudaStream_t st) {
    const int n = hi - lo;
    if (n <= 0) return cudaSuccess;
    finish_kernel<<<(n + 127) / 128, 128, 0, st>>>(ctl, inst, lo, hi, fs, counters);
    return cudaGetLastError();
}

cudaError_t launch_speed_reduce(Control* ctl, const InstDesc* inst, int lo, int hi, int set_dt,
                                cudaStream_t st) {
    const int n = hi - lo;
    if (n <= 0) return cudaSuccess;
    speed_reduce_kernel<<<(n + 127) / 128, 128, 0, st>>>(ctl, inst, lo, hi, set_dt);
    return cudaGetLastError();
}

cudaError_t launch_set_time(Control* ctl, int i, double t, double dt, long long nsteps,
                            cudaStream_t st) {
    set_time_kernel<<<1, 1, 0, st>>>(ctl, i, t, dt, nsteps);
    return cudaGetLastError();
}

cudaError_t launch_reset_status(Control* ctl, int i, cudaStream_t st) {
    reset_status_kernel<<<1, 1, 0, st>>>(ctl, i);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- conversion

// Dense FP64 q[f][z][y][x] <-> the pitched Real planes of slot cur[f].
template <class Real>
__global__ void convert_in_kernel(Real* pool, InstDesc I, const Control* ctl, const double* src,
                                  int m) {
    const long long nx = I.n[0];
    const long long ncell = nx * I.n[1] * I.n[2];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ncell;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long row = idx / nx, x = idx - row * nx;
        const long long o = row * I.pitch + x;
        for (int f = 0; f < m; ++f) {
            const int slot = ctl->cur[f];
            pool[I.offset + slot * I.vstride + f * I.fstride + o] = (Real)src[f * ncell + idx];
        }
    }
}

template <class Real>
__global__ void convert_out_kernel(const Real* pool, InstDesc I, const Control* ctl, double* dst,
                                   int m) {
    const long long nx = I.n[0];
    const long long ncell = nx * I.n[1] * I.n[2];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ncell;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long row = idx / nx, x = idx - row * nx;
        const long long o = row * I.pitch + x;
        for (int f = 0; f < m; ++f) {
            const int slot = ctl->cur[f];
            dst[f * ncell + idx] = (double)pool[I.offset + slot * I.vstride + f * I.fstride + o];
        }
    }
}

template <class Real>
__global__ void fill_kernel(Real* pool, InstDesc I, int slot, int f, double v) {
    const long long nx = I.n[0];
    const long long ncell = nx * I.n[1] * I.n[2];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ncell;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long row = idx / nx, x = idx - row * nx;
        pool[I.offset + slot * I.vstride + f * I.fstride + row * I.pitch + x] = (Real)v;
    }
}

// Per-cell impedance Z = rho c and speed c = sqrt(K / rho), formed in FP64.
template <class Real>
__global__ void aux_kernel(Real* aux, InstDesc I, const double* rho, const double* K) {
    const long long nx = I.n[0];
    const long long ncell = nx * I.n[1] * I.n[2];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ncell;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long row = idx / nx, x = idx - row * nx;
        const long long o = I.aux_offset + row * I.pitch + x;
        const double c = sqrt(K[idx] / rho[idx]);
        aux[o] = (Real)(rho[idx] * c);
        aux[o + I.fstride] = (Real)c;
    }
}

template <class Real>
__global__ void aux_plane_kernel(Real* aux, InstDesc I, int k, const double* src) {
    const long long nx = I.n[0];
    const long long ncell = nx * I.n[1] * I.n[2];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ncell;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long row = idx / nx, x = idx - row * nx;
        aux[I.aux_offset + k * I.fstride + row * I.pitch + x] = (Real)src[idx];
    }
}

template <class Real>
__global__ void aux_const_kernel(Real* aux, InstDesc I, double rho, double K) {
    const long long nx = I.n[0];
    const long long ncell = nx * I.n[1] * I.n[2];
    const double c = sqrt(K / rho);
    const double Z = rho * c;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ncell;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long row = idx / nx, x = idx - row * nx;
        const long long o = I.aux_offset + row * I.pitch + x;
        aux[o] = (Real)Z;
        aux[o + I.fstride] = (Real)c;
    }
}

// Deterministic FP64 field sums in two passes with a fixed shape: kSumParts
// CTAs per field each sum a fixed strided subset of the cells (every thread a
// fixed subsequence, then a fixed shared-memory tree) into a partial, and
// one CTA per field adds its partials in a fixed tree.  The same grid and
// state give the same bits on every call.
constexpr int kSumParts = 152;
constexpr int kSumThreads = 512;

template <class Real>
__global__ void __launch_bounds__(kSumThreads) sums_part_kernel(const Real* pool, InstDesc I, const Control* ctl,
                                                               double* partial) {
    __shared__ double part[kSumThreads];
    const int f = blockIdx.y;
    const long long nx = I.n[0];
    const long long ncell = nx * I.n[1] * I.n[2];
    const Real* q = pool + I.offset + ctl->cur[f] * I.vstride + f * I.fstride;
    double acc = 0.0;
    for (long long idx = (long long)blockIdx.x * kSumThreads + threadIdx.x; idx < ncell;
         idx += (long long)kSumParts * kSumThreads) {
        const long long row = idx / nx, x = idx - row * nx;
        acc += (double)q[row * I.pitch + x];
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kSumThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[f * kSumParts + blockIdx.x] = part[0];
}

__global__ void __launch_bounds__(256) sums_final_kernel(const double* partial, double* out) {
    __shared__ double part[256];
    const int f = blockIdx.x;
    part[threadIdx.x] = (int)threadIdx.x < kSumParts ? partial[f * kSumParts + threadIdx.x] : 0.0;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[f] = part[0];
}

static unsigned grid_for(const InstDesc& I) {
    const long long ncell = (long long)I.n[0] * I.n[1] * I.n[2];
    long long g = (ncell + 255) / 256;
    if (g > 152 * 64) g = 152 * 64;
    if (g < 1) g = 1;
    return (unsigned)g;
}

cudaError_t launch_convert_in(int precision, void* pool, const InstDesc& I, const Control* ctl,
                              const double* src, int m, cudaStream_t st) {
    if (precision == 64)
        convert_in_kernel<double><<<grid_for(I), 256, 0, st>>>((double*)pool, I, ctl, src, m);
    else
        convert_in_kernel<float><<<grid_for(I), 256, 0, st>>>((float*)pool, I, ctl, src, m);
    return cudaGetLastError();
}

cudaError_t launch_convert_out(int precision, const void* pool, const InstDesc& I,
                               const Control* ctl, double* dst, int m, cudaStream_t st) {
    if (precision == 64)
        convert_out_kernel<double><<<grid_for(I), 256, 0, st>>>((const double*)pool, I, ctl, dst, m);
    else
        convert_out_kernel<float><<<grid_for(I), 256, 0, st>>>((const float*)pool, I, ctl, dst, m);
    return cudaGetLastError();
}

cudaError_t launch_fill(int precision, void* pool, const InstDesc& I, int slot, int f, double v,
                        cudaStream_t st) {
    if (precision == 64)
        fill_kernel<double><<<grid_for(I), 256, 0, st>>>((double*)pool, I, slot, f, v);
    else
        fill_kernel<float><<<grid_for(I), 256, 0, st>>>((float*)pool, I, slot, f, v);
    return cudaGetLastError();
}

cudaError_t launch_aux(int precision, void* aux, const InstDesc& I, const double* rho,
                       const double* K, cudaStream_t st) {
    if (precision == 64)
        aux_kernel<double><<<grid_for(I), 256, 0, st>>>((double*)aux, I, rho, K);
    else
        aux_kernel<float><<<grid_for(I), 256, 0, st>>>((float*)aux, I, rho, K);
    return cudaGetLastError();
}

cudaError_t launch_aux_const(int precision, void* aux, const InstDesc& I, double rho, double K,
                             cudaStream_t st) {
    if (precision == 64)
        aux_const_kernel<double><<<grid_for(I), 256, 0, st>>>((double*)aux, I, rho, K);
    else
        aux_const_kernel<float><<<grid_for(I), 256, 0, st>>>((float*)aux, I, rho, K);
    return cudaGetLastError();
}

cudaError_t launch_aux_plane(int precision, void* aux, const InstDesc& I, int k, const double* src,
                             cudaStream_t st) {
    if (precision == 64)
        aux_plane_kernel<double><<<grid_for(I), 256, 0, st>>>((double*)aux, I, k, src);
    else
        aux_plane_kernel<float><<<grid_for(I), 256, 0, st>>>((float*)aux, I, k, src);
    return cudaGetLastError();
}

cudaError_t launch_sums(int precision, const void* pool, const InstDesc& I, const Control* ctl,
                        int m, double* out, cudaStream_t st) {
    static_assert(kSumParts <= 256, "the final pass adds at most 256 partials");
    double* partial = out + 8;   // the caller's buffer holds 8 sums, then 8 x kSumParts partials
    const dim3 grid(kSumParts, m);
    if (precision == 64)
        sums_part_kernel<double><<<grid, kSumThreads, 0, st>>>((const double*)pool, I, ctl, partial);
    else
        sums_part_kernel<float><<<grid, kSumThreads, 0, st>>>((const float*)pool, I, ctl, partial);
    sums_final_kernel<<<m, 256, 0, st>>>(partial, out);
    return cudaGetLastError();
}

}  // namespace claw
