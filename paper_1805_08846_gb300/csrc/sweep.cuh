// One directional sweep of the split wave-propagation update (CUDACLAW
// Sec. 3 Eq. LW-update, one half): along direction DIR every cell of every
// line gets
//   Q_i <- Q_i - nu (A+dQ_{i-1/2} + A-dQ_{i+1/2}) - nu (F_{i+1/2} - F_{i-1/2}),
//   F_{i-1/2} = 1/2 sum_p |s_p| (1 - nu |s_p|) phi(theta_p) W_p,
// with the ghost cells of the line filled from the boundary rules on the
// fly (the paper's separate BC stage, Sec. 4.1, fused in) and the largest
// |s_p| reduced into the instance's control block (Sec. 4.1, the block-local
// speed reduction; here a warp reduction and one atomic per warp).
//
// Work mapping (a GB300 design, not the paper's Fermi one): a CTA of kLines
// threads owns one tile -- kLines lines of one instance and a segment [a, b)
// along them -- and each thread marches along its own line with a sliding
// register window of cells and waves.  Every interface's Riemann problem is
// solved once per segment (plus three at the segment's ends), the limiter
// reads the neighbouring interfaces' waves from registers, and the update of
// a cell needs nothing from other threads, so there are no block barriers and
// no shared-memory wave arrays (the paper's Sec. 5.1/5.3 machinery).  Waves
// never reach global memory.  Lines along y or z are columns of adjacent x,
// so a warp's loads and stores of one step are one contiguous row segment.
#pragma once
#include "claw_types.cuh"
#include "riemann.cuh"

namespace claw {

enum : int { kBcPeriodic = 0, kBcExtrap = 1, kBcWall = 2 };

// Interior cell a ghost / interior position k of a line of N cells stands
// for, and whether the normal component changes sign (wall).
__device__ __forceinline__ int map_cell(int k, int N, int bc_lo, int bc_hi, bool& flip) {
    flip = false;
    if (k < 0) {
        if (bc_lo == kBcPeriodic) return k + N;
        if (bc_lo == kBcExtrap) return 0;
        flip = true;
        return -1 - k;
    }
    if (k >= N) {
        if (bc_hi == kBcPeriodic) return k - N;
        if (bc_hi == kBcExtrap) return N - 1;
        flip = true;
        return 2 * N - 1 - k;
    }
    return k;
}

__device__ __forceinline__ unsigned long long speed_bits(double s) {
    return (unsigned long long)__double_as_longlong(fabs(s));
}
__device__ __forceinline__ unsigned speed_bits(float s) { return __float_as_uint(fabsf(s)); }
__device__ __forceinline__ unsigned long long widen_bits(unsigned long long b) { return b; }
__device__ __forceinline__ unsigned long long widen_bits(unsigned b) {
    return (unsigned long long)__double_as_longlong((double)__uint_as_float(b));
}

template <class Real>
struct SpeedMax;
template <>
struct SpeedMax<double> {
    using T = unsigned long long;
};
template <>
struct SpeedMax<float> {
    using T = unsigned;
};

// Line geometry of thread `lane` in tile td: element offset of cell 0 of the
// line (relative to a field plane) and the stride between cells.
template <int DIR>
__device__ __forceinline__ bool line_geometry(const TileDesc& td, const InstDesc& I, int lane,
                                              long long& base, long long& stride) {
    if (DIR == 0) {
        const int r = td.line0 + lane;
        base = (long long)r * I.pitch;
        stride = 1;
        return r < I.n[1] * I.n[2];
    } else if (DIR == 1) {
        const int x = td.line0 + lane;
        base = (long long)td.other * I.n[1] * I.pitch + x;
        stride = I.pitch;
        return x < I.n[0];
    } else {
        const int x = td.line0 + lane;
        base = (long long)td.other * I.pitch + x;
        stride = (long long)I.n[1] * I.pitch;
        return x < I.n[0];
    }
}

template <class Sys, class Real, int LIM, int DIR, bool SPEEDS>
__global__ void __launch_bounds__(kLines) sweep_kernel(const SweepArgs A, const typename Sys::Params P) {
    using Cell = typename Sys::Cell;
    using W = Waves<Real, Sys::NQ, Sys::NW>;
    constexpr int NQ = Sys::NQ;
    constexpr int NW = Sys::NW;
    using SM = typename SpeedMax<Real>::T;

    const TileDesc td = A.tiles[blockIdx.x];
    if (td.inst < A.inst_lo || td.inst >= A.inst_hi) return;
    const InstDesc& I = A.inst[td.inst];
    Control* ctl = A.ctl + td.inst;
    if (!SPEEDS && *(volatile int*)&ctl->active == 0) return;

    const int lane = threadIdx.x;
    long long base, stride;
    const bool valid = line_geometry<DIR>(td, I, lane, base, stride);
    const int N = I.n[DIR];
    const int bc_lo = I.bc[2 * DIR], bc_hi = I.bc[2 * DIR + 1];

    const Real* pool = static_cast<const Real*>(A.pool);
    const Real* qin[NQ];
    Real* qout[NQ];
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        const int f = Sys::field(DIR, c);
        const int cur = ctl->cur[f];
        const int sin = SPEEDS ? cur : (cur + A.slots.in_off[f]) % 3;
        const int sout = (cur + A.slots.out_off[f]) % 3;
        qin[c] = pool + I.offset + sin * I.vstride + f * I.fstride + base;
        qout[c] = const_cast<Real*>(pool) + I.offset + sout * I.vstride + f * I.fstride + base;
    }
    const Real* aux = nullptr;
    if (Sys::NA > 0) aux = static_cast<const Real*>(A.aux) + I.aux_offset + base;
    const long long fstride = I.fstride;

    auto load = [&](int k, Cell& cell) {
        bool flip;
        const int j = map_cell(k, N, bc_lo, bc_hi, flip);
        const long long o = (long long)j * stride;
#pragma unroll
        for (int c = 0; c < NQ; ++c) cell.q[c] = __ldg(qin[c] + o);
        if (flip) cell.q[1] = -cell.q[1];
        if constexpr (Sys::NA > 0) {
            cell.Z = __ldg(aux + o);
            cell.c = __ldg(aux + fstride + o);
        }
        Sys::prepare(cell, P);
    };

    SM smax = 0;
    bool bad = false;

    if (valid) {
        const int a = td.a, b = td.b;
        if constexpr (SPEEDS) {
            // Speeds at interfaces a..b only (the CFL pass).
            Cell cl, cr;
            load(a - 1, cl);
            for (int Iif = a; Iif <= b; ++Iif) {
                load(Iif, cr);
                Real s[NW];
                Sys::speeds(cl, cr, P, s);
#pragma unroll
                for (int p = 0; p < NW; ++p) smax = max(smax, speed_bits(s[p]));
                cl = cr;
            }
        } else {
            const Real nu = (Real)(ctl->dt_attempt / I.dx[DIR]);
            Cell cA, cB;          // cells I-1 and I of the newest interface I
            W wA, wB, wC;         // waves at interfaces I-2, I-1, I
            Real F0[NQ];          // correction flux at interface I-2
            Real qkeep[NQ];       // kept state of cell I-2 (next to update)

            load(a - 2, cA);
            load(a - 1, cB);
            Sys::solve(cA, cB, P, wA);          // interface a-1
            cA = cB;
            load(a, cB);
            Sys::solve(cA, cB, P, wB);          // interface a
#pragma unroll
            for (int p = 0; p < NW; ++p) smax = max(smax, speed_bits(wB.s[p]));
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                qkeep[c] = cB.q[c];
                F0[c] = Real(0);
            }

#pragma unroll 2
            for (int Iif = a + 1; Iif <= b + 1; ++Iif) {
                cA = cB;
                load(Iif, cB);
                Sys::solve(cA, cB, P, wC);      // interface Iif
                if (Iif <= b) {
#pragma unroll
                    for (int p = 0; p < NW; ++p) smax = max(smax, speed_bits(wC.s[p]));
                }
                // Limited correction flux at interface Iif-1 (waves wB),
                // the upwind wave taken from Iif-2 (wA) or Iif (wC).
                Real F1[NQ];
#pragma unroll
                for (int c = 0; c < NQ; ++c) F1[c] = Real(0);
#pragma unroll
                for (int p = 0; p < NW; ++p) {
                    const Real sp = wB.s[p];
                    Real phi = Real(1);
                    if (LIM != kLimNone) {
                        Real num = Real(0), den = Real(0);
#pragma unroll
                        for (int c = 0; c < NQ; ++c) {
                            const Real up = sp > Real(0) ? wA.W[p][c] : wC.W[p][c];
                            num += up * wB.W[p][c];
                            den += wB.W[p][c] * wB.W[p][c];
                        }
                        phi = limiter_phi<LIM, Real>(num / den);
                    }
                    const Real as = fabs(sp);
                    const Real k = Real(0.5) * as * (Real(1) - nu * as) * phi;
#pragma unroll
                    for (int c = 0; c < NQ; ++c) F1[c] += k * wB.W[p][c];
                }
                // Update cell Iif-2 (its interfaces are Iif-2 and Iif-1).
                if (Iif >= a + 2) {
                    Real qn[NQ];
#pragma unroll
                    for (int c = 0; c < NQ; ++c) {
                        const Real first = wA.apdq[c] + wB.amdq[c];
                        const Real second = F1[c] - F0[c];
                        qn[c] = qkeep[c] - nu * first - nu * second;
                        qout[c][(long long)(Iif - 2) * stride] = qn[c];
                    }
                    bad |= Sys::nonphysical(qn);
                }
#pragma unroll
                for (int c = 0; c < NQ; ++c) {
                    qkeep[c] = cA.q[c];     // cell Iif-1, updated next iteration
                    F0[c] = F1[c];
                }
                wA = wB;
                wB = wC;
            }
        }
    }

    // Warp max of the speed bits (integer max keeps NaN above +Inf), one
    // atomic per warp into the instance's control block.
    unsigned long long m64 = widen_bits(smax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, m64, o);
        m64 = v > m64 ? v : m64;
    }
    const bool any_bad = __any_sync(0xffffffffu, bad);
    if ((lane & 31) == 0) {
        if (m64) atomicMax(&ctl->smax[DIR], m64);
        if (any_bad) atomicOr(&ctl->bad, 1u);
    }
}

}  // namespace claw
