// Point-wise Riemann solvers as device functors (CUDACLAW Sec. 4.2: a
// solver is a scalar function of the two cell states beside one interface;
// the framework maps threads onto interfaces around it).  A new PDE system
// plugs in by providing one such struct:
//
//   Value   arithmetic type: double, float, or f2 (two lines per thread)
//   NQ      components of the reduced state a sweep touches; component 0 is
//           the scalar (p or h), 1 the velocity / momentum normal to the
//           sweep, 2.. transverse components that waves carry
//   NW      waves per interface;  NA  material values per cell
//   Cell    per-cell registers: q[NQ] plus whatever the solver precomputes
//           once per cell (it is shared by the cell's two interfaces)
//   field(d, c)        state field that reduced component c maps to
//   prepare(cell, P)   fill the precomputed part of a freshly loaded cell
//   solve(l, r, P, w)  waves w.W[p][c], speeds w.s[p], fluctuations
//                      w.amdq[c] (A-dQ), w.apdq[c] (A+dQ)
//   set_aux(cell, a)   store the cell's material values a[0..NA-1]
//   kFWave             true when solve() returns f-waves Z_p (the source
//                      folded in); the correction then weighs by sign(s_p)
//   nonphysical(q)     true for a state the method cannot continue from
//   zero(p, c)         true where component c of wave p is identically zero
//                      (products with it are skipped: IEEE rules forbid the
//                      compiler to drop x * 0 itself)
//
// Formulas the paper leaves to its textbook reference are the standard ones:
// linear acoustics with per-cell impedance, and Roe's linearisation for
// shallow water with the Harten-Hyman entropy fix.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "pair.cuh"

namespace claw {

template <class Real, int NQ, int NW>
struct Waves {
    Real W[NW][NQ];
    Real s[NW];
    Real amdq[NQ];
    Real apdq[NQ];
};

template <class Real>
__device__ __forceinline__ bool finite_(Real x) {
    return fabs(x) <= (Real)INFINITY && x == x;
}

// FP64 reciprocal by the Newton-Raphson iteration for 1/d,
//   e = 1 - d r,  r <- r + r e   (the relative error e squares each step),
// started from the hardware's approximate reciprocal (PTX rcp.approx.ftz.f64;
// measured on GB300 over 6.7e7 random normal d: relative error <= 9.9e-7
// before the steps, <= 9.9e-13 after one, and after two the correctly rounded
// 1/d on every one of them).  A subnormal d counts as 0 (an infinite start, a
// NaN result), as does d = 0: callers use it where d is a normal positive
// number or where a NaN ratio is harmless (the limiter ratio of a zero wave).
// Against the correctly rounded divide it took the 4096^2 FP64 shallow-water
// sweep from 5.63 to 4.27 ms and the 512^3 FP64 acoustics sweep from 18.8 to
// 17.2 ms.  (The same two steps for the reciprocal square root, from
// rsqrt.approx.ftz.f64, were slower than the library's rsqrt: 4.38 ms.)
__device__ __forceinline__ double rcp_nr(double d) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

// Division, reciprocal and square roots.  FP64 (the plain path) uses the
// correctly rounded divide (the rare entropy-fix ratios) and square root, the
// Newton reciprocal above and the double reciprocal square root (a few ulp)
// where a solver asks for one; the FP32 form uses the SFU approximations
// (reciprocal and reciprocal square root, a few ulp), far inside its
// 1e-4 / 1e-5 error budget and a fraction of the instruction count.
template <class Real>
struct Ops;
template <>
struct Ops<double> {
    __device__ __forceinline__ static double div(double a, double b) { return a / b; }
    __device__ __forceinline__ static double rcp(double x) { return rcp_nr(x); }
    __device__ __forceinline__ static double rsqrt(double x) { return ::rsqrt(x); }
    __device__ __forceinline__ static double sqrt_(double x) { return sqrt(x); }
};
// FP32 reciprocal and reciprocal square root: the SFU approximations with
// subnormal inputs and results flushed to zero (PTX rcp.approx.ftz.f32,
// rsqrt.approx.ftz.f32).  rsqrtf() and __fdividef() without flushing wrap the
// same SFU operations in range handling for subnormal operands; dropping it
// took the 4096^2 FP32 shallow-water sweeps from 139 / 125 to 113 / 100
// instructions per cell (x 0.128 -> 0.119 ms, y 0.0995 -> 0.089 ms).  A
// shallow-water depth below the smallest normal float (1.2e-38) then reads as
// 0: in the Roe solvers its speeds turn non-finite and the step control
// reports it as non-physical, which such a depth is; the wet/dry solver
// counts it as dry.
__device__ __forceinline__ float rcp_ftz(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <>
struct Ops<float> {
    __device__ __forceinline__ static float div(float a, float b) { return __fdividef(a, b); }
    __device__ __forceinline__ static float rcp(float x) { return rcp_ftz(x); }
    __device__ __forceinline__ static float rsqrt(float x) { return rsqrt_ftz(x); }
    // x > 0: x * rsqrt(x)
    __device__ __forceinline__ static float sqrt_(float x) { return x * rsqrt_ftz(x); }
};
template <>
struct Ops<f2> {
    __device__ __forceinline__ static f2 div(f2 a, f2 b) {
        return f2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y));
    }
    __device__ __forceinline__ static f2 rcp(f2 x) { return f2(rcp_ftz(x.v.x), rcp_ftz(x.v.y)); }
    __device__ __forceinline__ static f2 rsqrt(f2 x) { return f2(rsqrt_ftz(x.v.x), rsqrt_ftz(x.v.y)); }
    __device__ __forceinline__ static f2 sqrt_(f2 x) { return x * rsqrt(x); }
};

// ------------------------------------------------------------------------
// Linear acoustics, Sec. 3 Eq. acoustics with coefficients:
//   p_t + K div u = 0,  rho u_t + grad p = 0.
// Along a direction the normal system has speeds -c, +c (c = sqrt(K/rho))
// and eigenvectors (-Z, 1), (Z, 1) with impedance Z = rho c.  With
// different cells on the two sides the left-going wave takes the left
// cell's (Z, c) and the right-going wave the right cell's:
//   alpha1 = (-dp + Z_r du) / (Z_l + Z_r),  alpha2 = (dp + Z_l du) / (Z_l + Z_r).
// VAR = false: one (Z, c) for the whole grid (kernel parameters).
// ------------------------------------------------------------------------
template <class Real, bool VAR>
struct Acoustics {
    using Value = Real;
    static constexpr int NQ = 2;
    static constexpr int NW = 2;
    static constexpr int NA = VAR ? 2 : 0;
    struct Params {
        Real Z, c, inv2Z;
    };
    struct Cell {
        Real q[NQ];
        Real Z, c;
    };

    __device__ __forceinline__ static int field(int d, int comp) { return comp == 0 ? 0 : 1 + d; }
    __host__ __device__ static constexpr bool zero(int, int) { return false; }

    static constexpr bool kFWave = false;

    __device__ __forceinline__ static void set_aux(Cell& cell, const Real* a) {
        cell.Z = a[0];
        cell.c = a[1];
    }

    __device__ __forceinline__ static void prepare(Cell& cell, const Params& P) {
        if (!VAR) {
            cell.Z = P.Z;
            cell.c = P.c;
        }
    }

    __device__ __forceinline__ static void solve(const Cell& l, const Cell& r, const Params& P,
                                                 Waves<Real, NQ, NW>& w) {
        const Real dp = r.q[0] - l.q[0];
        const Real du = r.q[1] - l.q[1];
        const Real inv = VAR ? Ops<Real>::rcp(l.Z + r.Z) : P.inv2Z;
        const Real a1 = (r.Z * du - dp) * inv;
        const Real a2 = (dp + l.Z * du) * inv;
        w.W[0][0] = -a1 * l.Z;
        w.W[0][1] = a1;
        w.s[0] = -l.c;
        w.W[1][0] = a2 * r.Z;
        w.W[1][1] = a2;
        w.s[1] = r.c;
        // c > 0: the first wave always goes left, the second right.
        w.amdq[0] = w.s[0] * w.W[0][0];
        w.amdq[1] = w.s[0] * w.W[0][1];
        w.apdq[0] = w.s[1] * w.W[1][0];
        w.apdq[1] = w.s[1] * w.W[1][1];
    }

    // Interface speeds only (CFL pass).
    __device__ __forceinline__ static void speeds(const Cell& l, const Cell& r, const Params&,
                                                  Real s[NW]) {
        s[0] = -l.c;
        s[1] = r.c;
    }

    // max_p |s_p| of a solved interface.
    __device__ __forceinline__ static Real max_speed(const Waves<Real, NQ, NW>& w) {
        return fmax(-w.s[0], w.s[1]);
    }

    // A NaN / Inf pressure stops the run; a bad velocity reaches the
    // pressure at the next sweep along its direction.
    __device__ __forceinline__ static bool nonphysical(const Real q[NQ]) {
        return !(fabs(q[0]) <= (Real)3.0e38);
    }
    static constexpr bool kMinH = false;
};

// ------------------------------------------------------------------------
// Shallow water, Sec. 3 Eq. SW, reduced state (h, h u_n, h u_t).
// Roe averages h_bar = (h_l + h_r)/2, u_hat, v_hat weighted by sqrt(h),
// c_hat = sqrt(g h_bar); speeds u_hat -/+ c_hat and u_hat; eigenvectors
// r1 = (1, u_hat - c_hat, v_hat), r2 = (0, 0, 1), r3 = (1, u_hat + c_hat, v_hat).
// Harten-Hyman: a 1-wave with u_l - c_l < 0 < u_m - c_m at the middle
// state q_m = Q_l + W1 (a transonic rarefaction) is split with
// beta = (lam_m - s1) / (lam_m - lam_l) into beta lam_l W1 (left) and
// (1 - beta) lam_m W1 (right); the 3-wave mirrors this with
// q_m = Q_r - W3.  The sign test of lam_m is done without a square root:
// for h_m > 0, u_m - sqrt(g h_m) > 0  <=>  hu_m > 0 and hu_m^2 > g h_m^3;
// the four conditions of a transonic 1-wave (c_l - u_l, h_m, hu_m and
// hu_m^2 - g h_m^3 all positive) are one test, min(...) > 0, taken only
// where the rarely true last one holds (a supercritical middle state; in
// subcritical flow the whole test is one packed quantity and a compare).
// ------------------------------------------------------------------------
// The subsonic shortcut's test from sign bits alone, for every lane: s1 < 0
// (sign set), s3 > 0 (sign clear) and both middle-state tests hu^2 - g h^3
// negative (sign set).  A zero of either sign only ever sends a lane to the
// full solver, whose result is then the same; one AND of the bit patterns
// replaces six compares.
__device__ __forceinline__ bool subsonic_signs(float s1, float s3, float a, float b) {
    return (int)(__float_as_uint(s1) & ~__float_as_uint(s3) & __float_as_uint(a) & __float_as_uint(b)) < 0;
}
__device__ __forceinline__ bool subsonic_signs(double s1, double s3, double a, double b) {
    return (__double_as_longlong(s1) & ~__double_as_longlong(s3) & __double_as_longlong(a) &
            __double_as_longlong(b)) < 0;
}
__device__ __forceinline__ bool subsonic_signs(f2 s1, f2 s3, f2 a, f2 b) {
    const unsigned x = __float_as_uint(s1.v.x) & ~__float_as_uint(s3.v.x) & __float_as_uint(a.v.x) &
                       __float_as_uint(b.v.x);
    const unsigned y = __float_as_uint(s1.v.y) & ~__float_as_uint(s3.v.y) & __float_as_uint(a.v.y) &
                       __float_as_uint(b.v.y);
    return (int)(x & y) < 0;
}

template <class Real>   // double, float, or f2 (two lines)
struct ShallowWater {
    using Value = Real;
    static constexpr int NQ = 3;
    static constexpr int NW = 3;
    static constexpr int NA = 0;
    struct Params {
        Real g, sqrt_g, half_g;
    };
    struct Cell {
        Real q[NQ];
        Real u, v;   // velocities
        Real sqh;    // sqrt(h)
        Real c;      // sqrt(g h)
    };
    static constexpr bool kFWave = false;

    __device__ __forceinline__ static int field(int d, int comp) {
        return comp == 0 ? 0 : (comp == 1 ? 1 + d : 2 - d);
    }
    // the shear wave W2 = (0, 0, alpha2)
    __host__ __device__ static constexpr bool zero(int p, int c) { return p == 1 && c < 2; }
    __device__ __forceinline__ static void set_aux(Cell&, const Real*) {}

    // One reciprocal square root per cell gives sqrt(h) and 1/h, and one per
    // interface gives c_hat and 1/(2 c_hat), in every precision (FP64: the
    // double rsqrt, within a few ulp; measured 6.80 -> 6.09 ms per 4096^2
    // sweep against correctly rounded divides and square roots, parity with
    // the oracle unchanged at 1e-12).
    __device__ __forceinline__ static void prepare(Cell& cell, const Params& P) {
        const Real r = Ops<Real>::rsqrt(cell.q[0]);
        const Real rh = r * r;
        cell.sqh = cell.q[0] * r;
        cell.u = cell.q[1] * rh;
        cell.v = cell.q[2] * rh;
        cell.c = P.sqrt_g * cell.sqh;
    }

    // Roe averages; i2c = 1 / (2 c_hat), ni2c = -i2c.
    template <class C>
    __device__ __forceinline__ static void roe(const C& l, const C& r, const Params& P,
                                               Real& uh, Real& vh, Real& ch, Real& i2c, Real& ni2c) {
        const Real den = Ops<Real>::rcp(l.sqh + r.sqh);
        uh = vfma(l.sqh, l.u, r.sqh * r.u) * den;
        vh = vfma(l.sqh, l.v, r.sqh * r.v) * den;
        const Real gh = P.half_g * (l.q[0] + r.q[0]);   // 0.5 g exactly: g (0.5 s) = (0.5 g) s
        const Real rc = Ops<Real>::rsqrt(gh);
        ch = gh * rc;
        i2c = Real(0.5f) * rc;
        ni2c = Real(-0.5f) * rc;
    }

    __device__ __forceinline__ static void solve(const Cell& l, const Cell& r, const Params& P,
                                                 Waves<Real, NQ, NW>& w) {
        Real uh, vh, ch, i2c;
        solve(l, r, P, w, uh, vh, ch, i2c);
    }

    // The same, also returning the interface's Roe averages u_hat, v_hat,
    // c_hat and 1 / (2 c_hat) (the unsplit update's transverse solvers
    // reuse them).
    __device__ __forceinline__ static void solve(const Cell& l, const Cell& r, const Params& P,
                                                 Waves<Real, NQ, NW>& w, Real& uh, Real& vh, Real& ch,
                                                 Real& i2c) {
        Real ni2c;
        roe(l, r, P, uh, vh, ch, i2c, ni2c);
        // strengths with nd0 = -(h_r - h_l) so that no operand needs negating:
        //   a1 = (s3 d0 - d1) / 2c,  a2 = d2 - vh d0,  a3 = (d1 - s1 d0) / 2c
        const Real nd0 = l.q[0] - r.q[0];
        const Real d1 = r.q[1] - l.q[1];
        const Real d2 = r.q[2] - l.q[2];
        const Real s1 = uh - ch, s3 = uh + ch;
        const Real a1 = vfma(s3, nd0, d1) * ni2c;
        const Real a2 = vfma(vh, nd0, d2);
        const Real a3 = vfma(s1, nd0, d1) * i2c;
        w.s[0] = s1;
        w.s[1] = uh;
        w.s[2] = s3;
        w.W[0][0] = a1;
        w.W[0][1] = a1 * s1;
        w.W[0][2] = a1 * vh;
        w.W[1][0] = Real(0);
        w.W[1][1] = Real(0);
        w.W[1][2] = a2;
        w.W[2][0] = a3;
        w.W[2][1] = a3 * s3;
        w.W[2][2] = a3 * vh;

        const Real km2 = vmin(uh, Real(0)), kp2 = vmax(uh, Real(0));
        const Real ng = Real(0) - P.g;
        {
            // The whole warp subcritical at this interface (|u_hat| < c_hat,
            // so s1 < 0 < s3, and both middle states subcritical, so no
            // transonic wave): the 1-wave goes left and the 3-wave right, and
            // no split factor is needed (a warp vote keeps the branch uniform;
            // measured at 4096^2: x sweep 0.134 -> 0.128 ms, y 0.106 -> 0.100 ms).
            // The solver is called by every lane of a warp.
            const Real hm1 = l.q[0] + w.W[0][0], hum1 = l.q[1] + w.W[0][1];
            const Real hm3 = r.q[0] - w.W[2][0], hum3 = r.q[1] - w.W[2][1];
            const Real sup1 = vfma(hum1, hum1, (ng * hm1) * (hm1 * hm1));
            const Real sup3 = vfma(hum3, hum3, (ng * hm3) * (hm3 * hm3));
            const bool lane_sub = subsonic_signs(s1, s3, sup1, sup3);
            if (__all_sync(0xffffffffu, lane_sub)) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    w.amdq[c] = s1 * w.W[0][c];
                    w.apdq[c] = s3 * w.W[2][c];
                }
                w.amdq[2] = vfma(s1, w.W[0][2], km2 * w.W[1][2]);
                w.apdq[2] = vfma(s3, w.W[2][2], kp2 * w.W[1][2]);
                return;
            }
        }
        // Split factors: A-dQ = sum km_p W_p, A+dQ = sum kp_p W_p.
        Real km1 = vmin(s1, Real(0)), kp1 = vmax(s1, Real(0));
        Real km3 = vmin(s3, Real(0)), kp3 = vmax(s3, Real(0));

        // Transonic tests.  The middle state must be supercritical for either
        // wave to be transonic (hu_m^2 > g h_m^3), which subcritical flow never
        // is: that one packed quantity is tested first, the other three
        // conditions (as one minimum) only where it holds (measured at 4096^2:
        // x sweep 0.137 -> 0.132 ms, y 0.111 -> 0.108 ms, against testing the
        // minimum of all four everywhere)
        {
            const Real hm = l.q[0] + w.W[0][0];
            const Real hum = l.q[1] + w.W[0][1];
            const Real sup = vfma(hum, hum, (ng * hm) * (hm * hm));
            if (any(vgt(sup, Real(0)))) {
                const auto fix = vgt(vmin(vmin(l.c - l.u, hm), vmin(hum, sup)), Real(0));
                if (any(fix)) {
                    const Real lam_l = l.u - l.c;
                    const Real lam_m = Ops<Real>::div(hum, hm) - Ops<Real>::sqrt_(P.g * hm);
                    const Real beta = Ops<Real>::div(lam_m - s1, lam_m - lam_l);
                    km1 = sel(fix, beta * lam_l, km1);
                    kp1 = sel(fix, (Real(1) - beta) * lam_m, kp1);
                }
            }
        }
        {
            const Real hm = r.q[0] - w.W[2][0];
            const Real hum = r.q[1] - w.W[2][1];
            const Real sup = vfma(hum, hum, (ng * hm) * (hm * hm));
            if (any(vgt(sup, Real(0)))) {
                const auto fix = vgt(vmin(vmin(r.u + r.c, hm), vmin(Real(0) - hum, sup)), Real(0));
                if (any(fix)) {
                    const Real lam_r = r.u + r.c;
                    const Real lam_m = Ops<Real>::div(hum, hm) + Ops<Real>::sqrt_(P.g * hm);
                    const Real beta = Ops<Real>::div(lam_r - s3, lam_r - lam_m);
                    km3 = sel(fix, beta * lam_m, km3);
                    kp3 = sel(fix, (Real(1) - beta) * lam_r, kp3);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            w.amdq[c] = vfma(km1, w.W[0][c], km3 * w.W[2][c]);
            w.apdq[c] = vfma(kp1, w.W[0][c], kp3 * w.W[2][c]);
        }
        w.amdq[2] = vfma(km1, w.W[0][2], vfma(km2, w.W[1][2], km3 * w.W[2][2]));
        w.apdq[2] = vfma(kp1, w.W[0][2], vfma(kp2, w.W[1][2], kp3 * w.W[2][2]));
    }

    __device__ __forceinline__ static void speeds(const Cell& l, const Cell& r, const Params& P,
                                                  Real s[NW]) {
        Real uh, vh, ch, i2c, ni2c;
        roe(l, r, P, uh, vh, ch, i2c, ni2c);
        s[0] = uh - ch;
        s[1] = uh;
        s[2] = uh + ch;
    }

    // max_p |s_p| = max(|u_hat - c_hat|, |u_hat + c_hat|) (c_hat >= 0 bounds |u_hat|).
    __device__ __forceinline__ static Real max_speed(const Waves<Real, NQ, NW>& w) {
        return vmax(vabs(w.s[0]), vabs(w.s[2]));
    }

    // h <= 0 or NaN stops the run; a non-finite momentum makes the next
    // sweep's speeds non-finite, which the step control catches.
    __device__ __forceinline__ static auto nonphysical(const Real q[NQ]) {
        return !(vgt(q[0], Real(0)) & vle(q[0], Real(3.0e38)));
    }
    // Cheaper form for the sweep: fold h's bit pattern into a running
    // signed-integer minimum; a minimum <= 0 means some h <= 0 (a NaN h
    // makes the next sweep's speeds NaN, caught there).
    static constexpr bool kMinH = true;
};

// ------------------------------------------------------------------------
// Shallow water over a bottom elevation B (one material value per cell): the
// source (0, -g h B_x, -g h B_y) of the Clawpack base of Sec. 3 folded into
// the Riemann problem as f-waves (well-balanced):
//   delta = f(Q_r) - f(Q_l) - psi,  psi = (0, -g h_bar (B_r - B_l), 0),
//   delta_0 = d(hu),  delta_1 = d(hu u) + g h_bar (dh + dB),  delta_2 = d(hu v)
// (g (h_r^2 - h_l^2)/2 = g h_bar dh, so a lake at rest gives delta = 0
// exactly), split on the Roe eigenvectors: Z_p = beta_p r_p with
//   beta_1 = (s3 delta_0 - delta_1) / 2c,  beta_2 = delta_2 - v_hat delta_0,
//   beta_3 = (delta_1 - s1 delta_0) / 2c.
// A-dQ sums the Z_p with s_p < 0, A+dQ the others.  No entropy fix.  The
// negated differences below are exact negations, so the strengths need no
// negated operands.
// ------------------------------------------------------------------------
template <class Real>   // double, float, or f2 (two lines)
struct ShallowWaterBathy {
    using Value = Real;
    using SW = ShallowWater<Real>;
    static constexpr int NQ = 3;
    static constexpr int NW = 3;
    static constexpr int NA = 1;
    using Params = typename SW::Params;
    struct Cell {
        Real q[NQ];
        Real u, v, sqh, c;
        Real fu, fv;   // hu u, hu v (normal flux terms)
        Real B;        // bottom elevation
    };
    static constexpr bool kFWave = true;
    static constexpr bool kMinH = true;

    __device__ __forceinline__ static int field(int d, int comp) { return SW::field(d, comp); }
    __host__ __device__ static constexpr bool zero(int p, int c) { return p == 1 && c < 2; }
    __device__ __forceinline__ static void set_aux(Cell& cell, const Real* a) { cell.B = a[0]; }

    __device__ __forceinline__ static void prepare(Cell& cell, const Params& P) {
        const Real r = Ops<Real>::rsqrt(cell.q[0]);
        const Real rh = r * r;
        cell.sqh = cell.q[0] * r;
        cell.u = cell.q[1] * rh;
        cell.v = cell.q[2] * rh;
        cell.c = P.sqrt_g * cell.sqh;
        cell.fu = cell.q[1] * cell.u;
        cell.fv = cell.q[1] * cell.v;
    }

    __device__ __forceinline__ static void solve(const Cell& l, const Cell& r, const Params& P,
                                                 Waves<Real, NQ, NW>& w) {
        Real uh, vh, ch, i2c, ni2c;
        SW::roe(l, r, P, uh, vh, ch, i2c, ni2c);
        const Real s1 = uh - ch, s3 = uh + ch;
        const Real d0 = r.q[1] - l.q[1];
        const Real nd0 = l.q[1] - r.q[1];
        const Real d2 = r.fv - l.fv;
        // -delta_1 = (fu_l - fu_r) + g h_bar ((h_l - h_r) + (B_l - B_r))
        const Real ghb = P.half_g * (l.q[0] + r.q[0]);
        const Real nd1 = vfma(ghb, (l.q[0] - r.q[0]) + (l.B - r.B), l.fu - r.fu);
        const Real b1 = vfma(s3, d0, nd1) * i2c;
        const Real b2 = vfma(vh, nd0, d2);
        const Real b3 = vfma(s1, d0, nd1) * ni2c;
        w.s[0] = s1;
        w.s[1] = uh;
        w.s[2] = s3;
        w.W[0][0] = b1;
        w.W[0][1] = b1 * s1;
        w.W[0][2] = b1 * vh;
        w.W[1][0] = Real(0);
        w.W[1][1] = Real(0);
        w.W[1][2] = b2;
        w.W[2][0] = b3;
        w.W[2][1] = b3 * s3;
        w.W[2][2] = b3 * vh;
        const auto n0 = vlt(s1, Real(0)), n1 = vlt(uh, Real(0)), n2 = vlt(s3, Real(0));
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            Real am = Real(0), ap = Real(0);
            if (!zero(0, c)) {
                am = am + sel(n0, w.W[0][c], Real(0));
                ap = ap + sel(n0, Real(0), w.W[0][c]);
            }
            if (!zero(1, c)) {
                am = am + sel(n1, w.W[1][c], Real(0));
                ap = ap + sel(n1, Real(0), w.W[1][c]);
            }
            am = am + sel(n2, w.W[2][c], Real(0));
            ap = ap + sel(n2, Real(0), w.W[2][c]);
            w.amdq[c] = am;
            w.apdq[c] = ap;
        }
    }

    __device__ __forceinline__ static void speeds(const Cell& l, const Cell& r, const Params& P,
                                                  Real s[NW]) {
        Real uh, vh, ch, i2c, ni2c;
        SW::roe(l, r, P, uh, vh, ch, i2c, ni2c);
        s[0] = uh - ch;
        s[1] = uh;
        s[2] = uh + ch;
    }
    __device__ __forceinline__ static Real max_speed(const Waves<Real, NQ, NW>& w) { return SW::max_speed(w); }
    __device__ __forceinline__ static auto nonphysical(const Real q[NQ]) { return SW::nonphysical(q); }
};

// ------------------------------------------------------------------------
// Shallow water over a bottom elevation B with wetting and drying (the
// source of Sec. 3's Clawpack base; dry states are a reading of this
// library, the paper is silent on them): the hydrostatic reconstruction
// (Audusse et al. 2004) around the HLLE solver.  A cell is dry when
// h <= dry_tol: its velocities count as zero.  At an interface, with
// B* = max(B_l, B_r), the reconstructed depths h* = h + B - B* (0 when
// <= dry_tol: a dry side) and states q* = h* (1, u, v) define a flat-bottom
// problem solved by HLLE with Einfeldt's speeds,
//   s1 = min(lam_l^-, u_hat - c_hat),  s3 = max(lam_r^+, u_hat + c_hat),
//   lam_l^- = u_l - c_l* (wet) or u_r - 2 c_r* (dry l),
//   lam_r^+ = u_r + c_r* (wet) or u_l + 2 c_l* (dry r),
// (u -/+ 2c: the front of a rarefaction into a dry bed; Roe averages of the
// reconstructed states), waves W1 = (s3 dq* - df*)/(s3 - s1),
// W3 = (df* - s1 dq*)/(s3 - s1) (W1 + W3 = dq*, s1 W1 + s3 W3 = df*), a
// zero middle wave at u_hat, and fluctuations
//   A-dQ = sum_{s<0} s W + (h_l* - h_l)(u_l, u_l^2, u_l v_l),
//   A+dQ = sum_{s>=0} s W + (h_r - h_r*)(u_r, u_r^2, u_r v_r)
// (the reconstruction's hydrostatic pressure terms cancel exactly: mass
// telescopes, a lake at rest gives zero, the first-order update keeps
// h >= 0).  Where a reconstructed side is dry the waves are returned as zero:
// no second-order correction at the shoreline.  Scalar Real only (double,
// float): the wet / dry decisions are branches, not packed lanes.
// ------------------------------------------------------------------------
template <class Real>
struct ShallowWaterDry {
    using Value = Real;
    static constexpr int NQ = 3;
    static constexpr int NW = 3;
    static constexpr int NA = 1;
    struct Params {
        Real g, sqrt_g, half_g, dry_tol;
    };
    struct Cell {
        Real q[NQ];
        Real u, v;   // velocities, 0 in a dry cell
        Real B;      // bottom elevation
    };
    static constexpr bool kFWave = false;
    static constexpr bool kMinH = false;
    static constexpr bool kFast = !std::is_same<Real, double>::value;

    __device__ __forceinline__ static int field(int d, int comp) {
        return comp == 0 ? 0 : (comp == 1 ? 1 + d : 2 - d);
    }
    // the middle wave is identically zero
    __host__ __device__ static constexpr bool zero(int p, int) { return p == 1; }
    __device__ __forceinline__ static void set_aux(Cell& cell, const Real* a) { cell.B = a[0]; }

    __device__ __forceinline__ static void prepare(Cell& cell, const Params& P) {
        const bool wet = cell.q[0] > P.dry_tol;
        const Real rh = wet ? rcp_(cell.q[0]) : Real(0);
        cell.u = cell.q[1] * rh;
        cell.v = cell.q[2] * rh;
    }

    // 1/h and sqrt(h) of a wet depth.  FP64: the correctly rounded
    // reciprocal (with dry_tol = 0 a wet depth may be subnormal, which the
    // Newton reciprocal counts as 0).  FP32: the flush-to-zero SFU forms; the
    // FP32 launcher raises dry_tol to at least the smallest normal float, so
    // a wet depth is never subnormal there.
    __device__ __forceinline__ static Real rcp_(Real x) {
        if constexpr (kFast) return Ops<Real>::rcp(x);
        else return Real(1) / x;
    }
    __device__ __forceinline__ static Real sqrt_(Real x) {   // x > 0
        if constexpr (kFast) return Ops<Real>::sqrt_(x);
        else return sqrt(x);
    }

    __device__ __forceinline__ static Real gsqrt(Real gh) {
        if constexpr (kFast) return gh > Real(0) ? sqrt_(gh) : Real(0);
        else return sqrt(gh);
    }

    // Reconstructed depths and the HLLE speeds of an interface; false when
    // both reconstructed sides are dry (no waves, speeds 0).
    __device__ __forceinline__ static bool recon(const Cell& l, const Cell& r, const Params& P, Real& hl,
                                                 Real& hr, Real& s1, Real& uh, Real& s3) {
        const Real Bs = l.B > r.B ? l.B : r.B;
        hl = l.q[0] + l.B - Bs;
        hr = r.q[0] + r.B - Bs;
        if (!(hl > P.dry_tol)) hl = Real(0);
        if (!(hr > P.dry_tol)) hr = Real(0);
        const bool wl = hl > Real(0), wr = hr > Real(0);
        if (!wl && !wr) {
            s1 = uh = s3 = Real(0);
            return false;
        }
        Real sql, sqr, cl, cr, ch;
        if constexpr (kFast) {
            sql = wl ? sqrt_(hl) : Real(0);
            sqr = wr ? sqrt_(hr) : Real(0);
            cl = P.sqrt_g * sql;
            cr = P.sqrt_g * sqr;
            ch = gsqrt(P.half_g * (hl + hr));
        } else {
            sql = wl ? sqrt(hl) : Real(0);
            sqr = wr ? sqrt(hr) : Real(0);
            cl = wl ? sqrt(P.g * hl) : Real(0);
            cr = wr ? sqrt(P.g * hr) : Real(0);
            ch = sqrt(P.g * (Real(0.5) * (hl + hr)));
        }
        uh = (sql * l.u + sqr * r.u) * Ops<Real>::rcp(sql + sqr);
        const Real lm = wl ? l.u - cl : r.u - Real(2) * cr;
        const Real rp = wr ? r.u + cr : l.u + Real(2) * cl;
        s1 = fmin(uh - ch, lm);
        s3 = fmax(uh + ch, rp);
        return true;
    }

    __device__ __forceinline__ static void solve(const Cell& l, const Cell& r, const Params& P,
                                                 Waves<Real, NQ, NW>& w) {
        Real hl, hr, s1, uh, s3;
        const bool any_wet = recon(l, r, P, hl, hr, s1, uh, s3);
        // what the reconstruction removes from each cell's flux
        const Real kl = hl - l.q[0], kr = r.q[0] - hr;
        w.amdq[0] = kl * l.u;
        w.amdq[1] = kl * (l.u * l.u);
        w.amdq[2] = kl * (l.u * l.v);
        w.apdq[0] = kr * r.u;
        w.apdq[1] = kr * (r.u * r.u);
        w.apdq[2] = kr * (r.u * r.v);
        w.s[0] = s1;
        w.s[1] = uh;
        w.s[2] = s3;
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            w.W[0][c] = Real(0);
            w.W[1][c] = Real(0);
            w.W[2][c] = Real(0);
        }
        if (!any_wet) return;
        // reconstructed states (a dry side is all zero) and their fluxes
        const Real ql[3] = {hl, hl * l.u, hl * l.v};
        const Real qr[3] = {hr, hr * r.u, hr * r.v};
        const Real fl[3] = {ql[1], ql[1] * l.u + P.half_g * hl * hl, ql[1] * l.v};
        const Real fr[3] = {qr[1], qr[1] * r.u + P.half_g * hr * hr, qr[1] * r.v};
        // s3 - s1 >= 2 c_hat and sql + sqr >= sqrt(h) of a wet side: normal
        // numbers even for a subnormal depth, so the Newton reciprocal holds
        const Real inv = Ops<Real>::rcp(s3 - s1);
        const bool shore = !(hl > Real(0)) || !(hr > Real(0));
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            const Real dq = qr[c] - ql[c], df = fr[c] - fl[c];
            const Real W1 = (s3 * dq - df) * inv;
            const Real W3 = (df - s1 * dq) * inv;
            if (s1 < Real(0)) w.amdq[c] += s1 * W1;
            else w.apdq[c] += s1 * W1;
            if (s3 < Real(0)) w.amdq[c] += s3 * W3;
            else w.apdq[c] += s3 * W3;
            // no second-order correction at the shoreline
            w.W[0][c] = shore ? Real(0) : W1;
            w.W[2][c] = shore ? Real(0) : W3;
        }
    }

    __device__ __forceinline__ static void speeds(const Cell& l, const Cell& r, const Params& P,
                                                  Real s[NW]) {
        Real hl, hr;
        recon(l, r, P, hl, hr, s[0], s[1], s[2]);
    }

    // max_p |s_p| = max(|s1|, |s3|) (s1 <= u_hat <= s3).
    __device__ __forceinline__ static Real max_speed(const Waves<Real, NQ, NW>& w) {
        return fmax(fabs(w.s[0]), fabs(w.s[2]));
    }

    // h < 0 or NaN stops the run (h = 0 is a dry cell).
    __device__ __forceinline__ static bool nonphysical(const Real q[NQ]) {
        return !(q[0] >= Real(0) && q[0] <= Real(3.0e38));
    }
};

// ------------------------------------------------------------------------
// Wave limiters phi(theta) (Sec. 3, the wave limiter), theta the ratio of
// the upwind wave's projection to the wave's own norm.  fmin/fmax return the
// non-NaN operand, so a zero wave (theta = 0/0) still limits to zero.
// ------------------------------------------------------------------------
// kLimFirstOrder: no correction term at all (first-order upwind)
enum : int { kLimNone = 0, kLimMinmod = 1, kLimMC = 2, kLimFirstOrder = 3 };

template <int LIM, class Real>
__device__ __forceinline__ Real limiter_phi(Real theta) {
    if (LIM == kLimMinmod) return fmax(Real(0), fmin(Real(1), theta));
    if (LIM == kLimMC)
        return fmax(Real(0), fmin(fmin(Real(0.5) * (Real(1) + theta), Real(2)), Real(2) * theta));
    return Real(1);
}

// phi(num / den) for den >= 0.  FP32: a saturating multiply by the SFU
// reciprocal -- minmod is sat(theta); MC is 2 sat(min(theta, (1 + theta)/4)),
// the same function written around the clamp to [0, 1] (a NaN ratio of a
// zero wave saturates to 0).  FP64: num times the Newton reciprocal of den
// (within 2 ulp of the ratio; a zero wave gives NaN, as 0/0 does).
template <int LIM, class Real>
__device__ __forceinline__ Real limiter_ratio(Real num, Real den) {
    if constexpr (std::is_same<Real, f2>::value) {
        return f2(limiter_ratio<LIM, float>(num.v.x, den.v.x), limiter_ratio<LIM, float>(num.v.y, den.v.y));
    } else if constexpr (sizeof(Real) == 4) {
        const float theta = num * rcp_ftz(den);   // |W|^2 below 1.2e-38 reads as 0: a negligible wave
        if (LIM == kLimMinmod) return __saturatef(theta);
        if (LIM == kLimMC) return 2.0f * __saturatef(fminf(theta, 0.25f + 0.25f * theta));
        return 1.0f;
    } else {
        return limiter_phi<LIM, Real>(num * rcp_nr(den));
    }
}

}  // namespace claw
