// claw_max_speed_noalloc: the CFL speed pass over a caller-owned FP64 state,
// with its scratch in a file-scope device array instead of solver-owned
// memory, for callers that cannot allocate device memory.
//
// Scratch: g_speed_partials holds one partial maximum (the bits of a
// non-negative double) per CTA and direction.  Every CTA writes its slot
// before the reduce kernel reads it, so nothing needs clearing; the array
// keeps the last call's values.  Each device that loads the library has its
// own copy of the array, so calls on different devices never meet; two calls
// that overlap on the same device (on different streams) race on it.
#include <claw.h>

#include <float.h>
#include <math.h>
#include <mutex>

#include "launch.h"
#include "riemann.cuh"
#include "sweep.cuh"

namespace {

constexpr int kNaLines = 128;                    // lines per CTA
constexpr int kNaMaxCtasPerDir = 16384;          // => at most 2,097,152 lines per direction
constexpr int kNaScratchWords = 3 * kNaMaxCtasPerDir;   // 384 KiB

static __device__ __align__(256) unsigned long long g_speed_partials[kNaScratchWords];

struct NaGeom {
    int n[3];
    int ndim;
    int bc[6];
    double dx[3];
};

// Cell k (ghosts by the boundary rule) of a dense q[f][z][y][x] line.
template <class Sys, class Real>
__device__ __forceinline__ void na_load(typename Sys::Cell& cell, const double* q, long long ncell,
                                        long long base, long long stride, int k, int N, int d,
                                        int bc_lo, int bc_hi, const double* rho, const double* K,
                                        const typename Sys::Params& P) {
    bool flip;
    const int j = claw::map_cell(k, N, bc_lo, bc_hi, flip);
    const long long o = base + (long long)j * stride;
#pragma unroll
    for (int c = 0; c < Sys::NQ; ++c) cell.q[c] = (Real)q[Sys::field(d, c) * ncell + o];
    if (flip) cell.q[1] = -cell.q[1];
    if constexpr (Sys::NA > 0) {
        const double cc = sqrt(K[o] / rho[o]);
        cell.Z = (Real)(rho[o] * cc);
        cell.c = (Real)cc;
    }
    Sys::prepare(cell, P);
}

template <class Sys, int DIR>
__global__ void __launch_bounds__(kNaLines) na_speed_kernel(const double* q, const double* rho,
                                                            const double* K, NaGeom G,
                                                            typename Sys::Params P,
                                                            unsigned long long* partials) {
    using Real = double;
    const long long nx = G.n[0], ny = G.n[1], nz = G.n[2];
    const long long ncell = nx * ny * nz;
    const long long nlines = ncell / G.n[DIR];
    const long long line = (long long)blockIdx.x * kNaLines + threadIdx.x;
    unsigned long long m = 0ull;
    if (line < nlines) {
        long long base, stride;
        if (DIR == 0) {
            base = line * nx;
            stride = 1;
        } else if (DIR == 1) {
            const long long x = line % nx, z = line / nx;
            base = z * ny * nx + x;
            stride = nx;
        } else {
            base = line;               // (y, x) of the plane
            stride = nx * ny;
        }
        const int N = G.n[DIR];
        const int bl = G.bc[2 * DIR], bh = G.bc[2 * DIR + 1];
        typename Sys::Cell cl, cr;
        na_load<Sys, Real>(cl, q, ncell, base, stride, -1, N, DIR, bl, bh, rho, K, P);
        for (int k = 0; k <= N; ++k) {
            na_load<Sys, Real>(cr, q, ncell, base, stride, k, N, DIR, bl, bh, rho, K, P);
            Real s[Sys::NW];
            Sys::speeds(cl, cr, P, s);
#pragma unroll
            for (int p = 0; p < Sys::NW; ++p) m = max(m, claw::speed_bits(s[p]));
            cl = cr;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    __shared__ unsigned long long warp_max[kNaLines / 32];
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = warp_max[0];
        for (int w = 1; w < kNaLines / 32; ++w) b = warp_max[w] > b ? warp_max[w] : b;
        partials[DIR * kNaMaxCtasPerDir + blockIdx.x] = b;
    }
}

// M = max_d (max|s|_d / dx_d) from the partials: one CTA, each thread a
// strided subset of every direction's partials, then warp and CTA maxima
// (integer maxima of the bit patterns: exact, so the order does not matter).
constexpr int kNaReduceThreads = 512;

__global__ void __launch_bounds__(kNaReduceThreads) na_reduce_kernel(const unsigned long long* partials,
                                                                     NaGeom G, int nblk0, int nblk1,
                                                                     int nblk2, double* out) {
    const int nblk[3] = {nblk0, nblk1, nblk2};
    __shared__ unsigned long long warp_max[3][kNaReduceThreads / 32];
    for (int d = 0; d < G.ndim; ++d) {
        unsigned long long b = 0ull;
        for (int i = threadIdx.x; i < nblk[d]; i += kNaReduceThreads) {
            const unsigned long long v = partials[d * kNaMaxCtasPerDir + i];
            b = v > b ? v : b;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
            b = v > b ? v : b;
        }
        if ((threadIdx.x & 31) == 0) warp_max[d][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double M = 0.0;
    bool nonfinite = false;
    for (int d = 0; d < G.ndim; ++d) {
        unsigned long long b = 0ull;
        for (int w = 0; w < kNaReduceThreads / 32; ++w) b = warp_max[d][w] > b ? warp_max[d][w] : b;
        const double md = __longlong_as_double((long long)b);
        if (!(md <= DBL_MAX)) nonfinite = true;
        const double v = md / G.dx[d];
        if (v > M) M = v;
    }
    *out = nonfinite ? (double)NAN : M;
}

// Device address of the scratch array, looked up once per device.
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
unsigned long long* g_na_ptr[kNaMaxDevices] = {};

claw_status na_scratch(unsigned long long** out, const char** err) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
        *err = "claw_max_speed_noalloc: no usable current CUDA device";
        return CLAW_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_speed_partials);
        if (e != cudaSuccess || !p) {
            *err = "claw_max_speed_noalloc: cudaGetSymbolAddress of the scratch array failed";
            return CLAW_ECUDA;
        }
        g_na_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_na_ptr[dev];
    return CLAW_OK;
}

template <class Sys>
cudaError_t na_launch(const double* q, const double* rho, const double* K, const NaGeom& G,
                      const typename Sys::Params& P, unsigned long long* scratch, const int nblk[3],
                      double* out, cudaStream_t st) {
    na_speed_kernel<Sys, 0><<<nblk[0], kNaLines, 0, st>>>(q, rho, K, G, P, scratch);
    na_speed_kernel<Sys, 1><<<nblk[1], kNaLines, 0, st>>>(q, rho, K, G, P, scratch);
    if (G.ndim == 3) {
        if constexpr (Sys::NQ == 2) na_speed_kernel<Sys, 2><<<nblk[2], kNaLines, 0, st>>>(q, rho, K, G, P, scratch);
    }
    na_reduce_kernel<<<1, kNaReduceThreads, 0, st>>>(scratch, G, nblk[0], nblk[1], nblk[2], out);
    return cudaGetLastError();
}

claw_status na_fail(claw_status st, const char* msg) {
    claw::set_last_error(msg);
    return st;
}

}  // namespace

extern "C" claw_status claw_max_speed_noalloc(const claw_grid* grid, claw_system system,
                                              const claw_bc bc[6], const claw_params* params,
                                              const double* q, const double* rho, const double* K,
                                              double* out, void* cuda_stream) {
    if (!grid || !bc || !params || !q || !out)
        return na_fail(CLAW_EINVAL, "claw_max_speed_noalloc: NULL argument");
    if ((grid->ndim != 2 && grid->ndim != 3) || (system == CLAW_SHALLOW_WATER && grid->ndim != 2) ||
        system < CLAW_ACOUSTICS || system > CLAW_SHALLOW_WATER)
        return na_fail(CLAW_EINVAL, "claw_max_speed_noalloc: unsupported system / dimension");
    if (system == CLAW_ACOUSTICS_VAR && (!rho || !K))
        return na_fail(CLAW_EINVAL, "claw_max_speed_noalloc: CLAW_ACOUSTICS_VAR needs rho and K");
    NaGeom G{};
    G.ndim = grid->ndim;
    long long ncell = 1;
    for (int d = 0; d < 3; ++d) {
        G.n[d] = d < grid->ndim ? grid->n[d] : 1;
        G.dx[d] = d < grid->ndim ? grid->dx[d] : 1.0;
        if (d < grid->ndim && (G.n[d] < 2 || !(G.dx[d] > 0.0)))
            return na_fail(CLAW_EINVAL, "claw_max_speed_noalloc: need n[d] >= 2 and dx[d] > 0");
        ncell *= G.n[d];
    }
    for (int k = 0; k < 6; ++k) {
        G.bc[k] = k < 2 * grid->ndim ? (int)bc[k] : CLAW_BC_EXTRAP;
        if (G.bc[k] < CLAW_BC_PERIODIC || G.bc[k] > CLAW_BC_WALL)
            return na_fail(CLAW_EINVAL, "claw_max_speed_noalloc: unknown boundary kind");
    }
    int nblk[3] = {0, 0, 0};
    for (int d = 0; d < grid->ndim; ++d) {
        const long long lines = ncell / G.n[d];
        const long long b = (lines + kNaLines - 1) / kNaLines;
        if (b > kNaMaxCtasPerDir)
            return na_fail(CLAW_EBOUNDS, "claw_max_speed_noalloc: grid too large for the fixed "
                                         "scratch array (at most 2,097,152 lines per direction)");
        nblk[d] = (int)b;
    }
    unsigned long long* scratch = nullptr;
    const char* err = "";
    const claw_status st = na_scratch(&scratch, &err);
    if (st != CLAW_OK) return na_fail(st, err);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    cudaError_t e;
    if (system == CLAW_SHALLOW_WATER) {
        using S = claw::ShallowWater<double>;
        const S::Params P{params->g, sqrt(params->g), 0.5 * params->g};
        e = na_launch<S>(q, nullptr, nullptr, G, P, scratch, nblk, out, stream);
    } else if (system == CLAW_ACOUSTICS_VAR) {
        using S = claw::Acoustics<double, true>;
        const S::Params P{0.0, 0.0, 0.0};
        e = na_launch<S>(q, rho, K, G, P, scratch, nblk, out, stream);
    } else {
        using S = claw::Acoustics<double, false>;
        const double c = sqrt(params->K / params->rho);
        const double Z = params->rho * c;
        const S::Params P{Z, c, 1.0 / (2.0 * Z)};
        e = na_launch<S>(q, nullptr, nullptr, G, P, scratch, nblk, out, stream);
    }
    if (e != cudaSuccess) return na_fail(CLAW_ECUDA, "claw_max_speed_noalloc: kernel launch failed");
    return CLAW_OK;
}
