"""The FP64 Newton reciprocal of the sweeps (`rcp_nr` in csrc/riemann.cuh:
two Newton-Raphson steps r <- r + r (1 - d r) from the hardware's approximate
reciprocal) against CUDA's correctly rounded 1.0 / d, on the GPU.

The FP64 sweeps take their limiter ratios and Roe-average reciprocals from
it, so the 1e-12 parity with the oracle rests on its accuracy.  The check
compiles a small program around the library's own header, runs it over
2^24 seeded normal d (every binade from 2^-1000 to 2^1000, plus powers of
two and the neighbours of 1) and asserts that every result is within 1 ulp
of 1.0 / d (measured: 0 ulp on all of them), and that d = 0 gives NaN (the
limiter's zero-wave case, harmless there).
"""
import os
import subprocess

import pytest

from paper_1805_08846_gb300 import build as B

pytestmark = pytest.mark.gpu

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1805_08846_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include <cmath>
#include "riemann.cuh"

__device__ unsigned long long g_ulps;
__device__ int g_bad;

__device__ double input(long long i) {
    unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 1805ull;
    z ^= z >> 31; z *= 0xBF58476D1CE4E5B9ull; z ^= z >> 27; z *= 0x94D049BB133111EBull; z ^= z >> 31;
    const int kind = (int)(i & 15);
    const int ex = (int)((z >> 52) % 2001) - 1000;
    if (kind == 0) return ldexp(1.0, ex);                                       // powers of two
    if (kind == 1) return __longlong_as_double(__double_as_longlong(1.0) + (long long)(z % 64) - 32);  // near 1
    return ldexp(1.0 + (double)(z & ((1ull << 52) - 1)) * 0x1p-52, ex);
}

__global__ void check(long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double d = input(i);
        const double r = claw::rcp_nr(d), q = 1.0 / d;
        long long du = __double_as_longlong(r) - __double_as_longlong(q);
        if (du < 0) du = -du;
        atomicMax(&g_ulps, (unsigned long long)du);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double z = claw::rcp_nr(0.0);
        if (z == z) atomicOr(&g_bad, 1);
    }
}

int main() {
    const long long n = 1ll << 24;
    check<<<152 * 4, 256>>>(n);
    if (cudaDeviceSynchronize() != cudaSuccess) { printf("cuda error\n"); return 2; }
    unsigned long long ulps = 0; int bad = 0;
    cudaMemcpyFromSymbol(&ulps, g_ulps, sizeof(ulps));
    cudaMemcpyFromSymbol(&bad, g_bad, sizeof(bad));
    printf("%llu %d %lld\n", ulps, bad, n);
    return 0;
}
"""


def test_newton_reciprocal_matches_the_correctly_rounded_one(tmp_path):
    src = tmp_path / "rcp64.cu"
    exe = tmp_path / "rcp64"
    src.write_text(PROGRAM)
    cmd = [B.nvcc(), B.ARCH, "-O3", "-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC,
           str(src), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    ulps, bad, n = (int(x) for x in out.stdout.split())
    assert n == 1 << 24
    assert ulps <= 1, ulps
    assert bad == 0
