// Value types of the sweep arithmetic: double, float, and f2 -- two FP32
// lanes (two grid lines marched by one thread) computed with the packed
// FP32x2 add / multiply / fused multiply-add of sm_100-family GPUs, one
// instruction for both lanes.  Comparisons give a mask per lane; branches
// test any(mask) and results are merged with sel().  The helpers below are
// overloaded for all three types so one solver source serves every path.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace claw {

struct f2 {
    float2 v;
    f2() = default;
    __host__ __device__ __forceinline__ f2(float a) : v(make_float2(a, a)) {}
    __host__ __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
    __host__ __device__ __forceinline__ explicit f2(float2 w) : v(w) {}
};
struct m2 {
    bool x, y;
};

__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
// a - b as b * (-1) + a: the product is exact, so this is the rounded difference
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
    return f2(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v));
}
__device__ __forceinline__ f2 operator-(f2 a) { return f2(__fmul2_rn(a.v, make_float2(-1.0f, -1.0f))); }
__device__ __forceinline__ f2& operator+=(f2& a, f2 b) { return a = a + b; }

__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }

__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ f2 vmin(f2 a, f2 b) { return f2(fminf(a.v.x, b.v.x), fminf(a.v.y, b.v.y)); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ f2 vmax(f2 a, f2 b) { return f2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y)); }
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ double vabs(double a) { return fabs(a); }
__device__ __forceinline__ f2 vabs(f2 a) { return f2(fabsf(a.v.x), fabsf(a.v.y)); }

// masks
__device__ __forceinline__ bool vlt(float a, float b) { return a < b; }
__device__ __forceinline__ bool vlt(double a, double b) { return a < b; }
__device__ __forceinline__ m2 vlt(f2 a, f2 b) { return {a.v.x < b.v.x, a.v.y < b.v.y}; }
__device__ __forceinline__ bool vgt(float a, float b) { return a > b; }
__device__ __forceinline__ bool vgt(double a, double b) { return a > b; }
__device__ __forceinline__ m2 vgt(f2 a, f2 b) { return {a.v.x > b.v.x, a.v.y > b.v.y}; }
__device__ __forceinline__ bool vle(float a, float b) { return a <= b; }
__device__ __forceinline__ bool vle(double a, double b) { return a <= b; }
__device__ __forceinline__ m2 vle(f2 a, f2 b) { return {a.v.x <= b.v.x, a.v.y <= b.v.y}; }
__device__ __forceinline__ m2 operator&(m2 a, m2 b) { return {a.x && b.x, a.y && b.y}; }
__device__ __forceinline__ m2 operator|(m2 a, m2 b) { return {a.x || b.x, a.y || b.y}; }
__device__ __forceinline__ m2 operator!(m2 a) { return {!a.x, !a.y}; }
__device__ __forceinline__ bool any(bool m) { return m; }
__device__ __forceinline__ bool any(m2 m) { return m.x || m.y; }
__device__ __forceinline__ float sel(bool m, float a, float b) { return m ? a : b; }
__device__ __forceinline__ double sel(bool m, double a, double b) { return m ? a : b; }
__device__ __forceinline__ f2 sel(m2 m, f2 a, f2 b) { return f2(m.x ? a.v.x : b.v.x, m.y ? a.v.y : b.v.y); }

// Lane access: lane k (0 or 1) of a value; scalars have lane 0 only.
__device__ __forceinline__ float lane_of(float a, int) { return a; }
__device__ __forceinline__ double lane_of(double a, int) { return a; }
__device__ __forceinline__ float lane_of(f2 a, int k) { return k ? a.v.y : a.v.x; }
__device__ __forceinline__ void set_lane(float& a, int, float x) { a = x; }
__device__ __forceinline__ void set_lane(double& a, int, double x) { a = x; }
__device__ __forceinline__ void set_lane(f2& a, int k, float x) {
    if (k) a.v.y = x;
    else a.v.x = x;
}
__device__ __forceinline__ bool lane_of(bool m, int) { return m; }
__device__ __forceinline__ bool lane_of(m2 m, int k) { return k ? m.y : m.x; }

// Lanes per value and the scalar type of a lane.
template <class V>
struct Lanes {
    static constexpr int N = 1;
    using Scalar = V;
};
template <>
struct Lanes<f2> {
    static constexpr int N = 2;
    using Scalar = float;
};

}  // namespace claw
