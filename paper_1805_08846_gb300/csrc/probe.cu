// Achievable arithmetic roof (CUDACLAW Sec. 7.1 measures its "achievable
// roof" with a multiply-add-only kernel): eight independent fused
// multiply-add chains per thread, enough CTAs to fill every SM, timed with
// CUDA events.  The FP64 path of the sweeps is bounded by this rate on GB300.
#include <claw.h>

#include "launch.h"

namespace {

template <class T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    const T sum = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (sum == (T)-12345) out[blockIdx.x] = sum;   // keeps the chains live
}

template <class T>
claw_status run_probe(double* flops, cudaStream_t st) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CLAW_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks) != cudaSuccess) return CLAW_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = (T)0.999999, b = (T)1e-7;
    int iters = sizeof(T) == 8 ? 4096 : 65536;
    fma_probe_kernel<T><<<blocks, threads, 0, st>>>(out, iters / 16, a, b);   // warm-up
    float ms = 0.f;
    for (int rep = 0; rep < 8; ++rep) {
        cudaEventRecord(e0, st);
        fma_probe_kernel<T><<<blocks, threads, 0, st>>>(out, iters, a, b);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 20.f) break;
        iters *= 2;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || ms <= 0.f) return CLAW_ECUDA;
    *flops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
    return CLAW_OK;
}

}  // namespace

extern "C" claw_status claw_probe_fma(int precision, double* flops_per_s, void* cuda_stream) {
    if (!flops_per_s || (precision != 32 && precision != 64)) {
        claw::set_last_error("claw_probe_fma: precision must be 32 or 64 and the output non-NULL");
        return CLAW_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const claw_status r = precision == 64 ? run_probe<double>(flops_per_s, st) : run_probe<float>(flops_per_s, st);
    if (r != CLAW_OK) claw::set_last_error("claw_probe_fma: CUDA failure");
    return r;
}
