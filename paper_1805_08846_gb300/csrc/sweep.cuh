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
// a cell needs nothing from other threads, so there are no shared wave
// arrays (the paper's Sec. 5.1/5.3 machinery).  Waves never reach global
// memory.
//
// Staging: the segment's cells arrive in chunks of C cells x kLines lines
// per field, copied by bulk-tensor (TMA) loads into a ring of STAGES shared
// memory buffers, several chunks ahead of the march, so the HBM stream is
// deep enough without any per-thread prefetch registers.  For the y and z
// sweeps a chunk is C rows of kLines consecutive x (one 512 B row per field
// for FP32) and results are stored directly (a warp writes 32 consecutive x).
// For the x sweep a chunk is 32 bytes of each of the tile's rows (32-byte
// swizzle); each result overwrites an input position of its stage that has
// been consumed, and a completed chunk leaves by a bulk-tensor store.  The two
// cells before and after the segment (ghosts at the domain edge) are read
// directly.
#pragma once
#include "claw_types.cuh"
#include "riemann.cuh"
#include "tma.cuh"

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

// Warp max of the speed bits (integer max keeps NaN above +Inf), one atomic
// per warp into the instance's control block; a non-physical flag likewise.
template <int DIR, class SM>
__device__ __forceinline__ void reduce_to_control(Control* ctl, SM smax, bool bad) {
    unsigned long long m64 = widen_bits(smax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, m64, o);
        m64 = v > m64 ? v : m64;
    }
    const bool any_bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        if (m64) atomicMax(&ctl->smax[DIR], m64);
        if (any_bad) atomicOr(&ctl->bad, 1u);
    }
}

// ------------------------------------------------------------------------
// Speeds-only pass (the CFL estimate of a new state): direct loads, no update.
// ------------------------------------------------------------------------
template <class Sys, class Real, int DIR>
__global__ void __launch_bounds__(kLines) speed_kernel(const SweepArgs A, const typename Sys::Params P) {
    using Cell = typename Sys::Cell;
    constexpr int NQ = Sys::NQ;
    using SM = typename SpeedMax<Real>::T;
    const TileDesc td = A.tiles[blockIdx.x];
    const InstDesc& I = A.inst[td.inst];
    Control* ctl = A.ctl + td.inst;
    long long base, stride;
    const bool valid = line_geometry<DIR>(td, I, threadIdx.x, base, stride) && (int)threadIdx.x < A.lines;
    const int N = I.n[DIR];
    const int bc_lo = I.bc[2 * DIR], bc_hi = I.bc[2 * DIR + 1];
    const Real* pool = static_cast<const Real*>(A.pool);
    const Real* qin[NQ];
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        const int f = Sys::field(DIR, c);
        qin[c] = pool + I.offset + ctl->cur[f] * I.vstride + f * I.fstride + base;
    }
    const Real* aux = nullptr;
    if (Sys::NA > 0) aux = static_cast<const Real*>(A.aux) + I.aux_offset + base;
    auto load = [&](int k, Cell& cell) {
        bool flip;
        const int j = map_cell(k, N, bc_lo, bc_hi, flip);
        const long long o = (long long)j * stride;
        const bool ok = cell_ok(base + o, I, ctl);
#pragma unroll
        for (int c = 0; c < NQ; ++c) cell.q[c] = ok ? __ldg(qin[c] + o) : Real(1);
        if (flip) cell.q[1] = -cell.q[1];
        if constexpr (Sys::NA > 0) {
            Real a[Sys::NA];
#pragma unroll
            for (int k = 0; k < Sys::NA; ++k) a[k] = ok ? __ldg(aux + k * I.fstride + o) : Real(1);
            Sys::set_aux(cell, a);
        }
        Sys::prepare(cell, P);
    };
    SM smax = 0;
    if (valid) {
        Cell cl, cr;
        load(td.a - 1, cl);
        for (int k = td.a; k <= td.b; ++k) {
            load(k, cr);
            Real s[Sys::NW];
            Sys::speeds(cl, cr, P, s);
#pragma unroll
            for (int p = 0; p < Sys::NW; ++p) smax = max(smax, speed_bits(s[p]));
            cl = cr;
        }
    }
    reduce_to_control<DIR>(ctl, smax, false);
}

// ------------------------------------------------------------------------
// The staged sweep.
// ------------------------------------------------------------------------
// A plane box holds 32 bytes' worth of cells (8 FP32 / 4 FP64) of 128
// lines, 4 KB: for the y, z sweeps C rows of 128 adjacent x, for the x sweep
// 32 bytes of each of 128 rows, kept with the 32-byte swizzle (the two
// 16-byte halves of a row swap places on bit 2 of the row), under which a
// warp's 16-byte reads of its own rows hit every bank once; the march reads
// one cell (4 bytes) per row, which meets 4-way conflicts (rows r, r+8,
// r+16, r+24 share banks; measured cheaper than reading 16-byte words).
// Tile widths a direction's sweep offers (the autotuner picks one): NARROW
// halves the lines per tile (fewer lanes past the edge of small or uneven
// grids, more tiles); the two-line x sweep has only its 64-row tiles.
template <class Sys, int DIR>
constexpr bool narrow_offered() {
    return !(Lanes<typename Sys::Value>::N == 2 && DIR == 0);
}

template <class Sys, class Real, int DIR, bool NARROW = false>
struct StageCfg {
    // lines per thread: 2 when the system computes on f2 (two FP32 lines)
    static constexpr int PK = Lanes<typename Sys::Value>::N;
    // lines per tile: 128, or 64 for the two-line x sweep (one-warp CTAs
    // whose three-stage ring is small enough for 11 CTAs per SM); a narrow
    // tile has half as many
    static constexpr int LINES = (PK == 2 && DIR == 0) ? kLines / 2 : (NARROW ? kLines / 2 : kLines);
    static constexpr int NT = LINES / PK;                       // threads per CTA
    static constexpr int NP = Sys::NQ + Sys::NA;               // planes per chunk
    static constexpr int C = 32 / (int)sizeof(Real);            // cells per chunk
    static constexpr int G = 16 / (int)sizeof(Real);            // cells per 16-byte half
    static constexpr int BOX = LINES * C * (int)sizeof(Real);    // bytes per plane box
    // y, z: two stages suffice for the two-line form (more CTAs fit); the x
    // sweep refills a stage only after the write-back of the chunk before
    // has read it, which needs three
    static constexpr int STAGES = (PK == 2 && DIR != 0) ? 2 : 3;
    // x sweep results leave through their input stages and bulk stores
    // (measured: direct stores from 32 rows per warp are 3x slower)
    static constexpr bool XWB = true;
    static_assert(DIR != 0 || !XWB || STAGES >= 3, "the x write-back ring needs three stages");
    static constexpr int STAGE_BYTES = NP * BOX;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 64;  // + alignment, barriers
    // register budget: 4 CTAs of 128 threads per SM for FP32 (measured best:
    // a 5-CTA budget forces worse schedules), 2 for FP64; 6 CTAs of 64
    // two-line threads for the packed y / z sweeps; 8 one-warp CTAs for the
    // packed x sweep, which its best segment lengths fill anyway (188
    // registers; measured against a 12-CTA budget at 166: 4096^2 x sweep
    // 0.1134 -> 0.1124 ms, the 256-grid ensemble's x sweep 0.746 -> 0.657 ms)
    // (the same per-SM budget for narrow tiles: twice as many CTAs)
    static constexpr int MIN_CTAS =
        (PK == 2 ? (DIR == 0 ? 8 : 6) : (sizeof(Real) == 4 ? 4 : 2)) * ((NARROW && !(PK == 2 && DIR == 0)) ? 2 : 1);
};

template <class Sys, class Real, int LIM, int DIR, bool NARROW>
__global__ void __launch_bounds__((StageCfg<Sys, Real, DIR, NARROW>::NT), (StageCfg<Sys, Real, DIR, NARROW>::MIN_CTAS))
    sweep_kernel(const SweepArgs A, const typename Sys::Params P) {
    using Cfg = StageCfg<Sys, Real, DIR, NARROW>;
    using V = typename Sys::Value;     // Real, or f2 for two lines per thread
    constexpr int PK = Cfg::PK;
    using Cell = typename Sys::Cell;
    using W = Waves<typename Sys::Value, Sys::NQ, Sys::NW>;
    constexpr int NQ = Sys::NQ;
    constexpr int NW = Sys::NW;
    constexpr int NA = Sys::NA;
    constexpr int NP = Cfg::NP;
    constexpr int C = Cfg::C;
    constexpr int STAGES = Cfg::STAGES;
    using SM = typename SpeedMax<Real>::T;

    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * Cfg::STAGE_BYTES);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(smem_addr(&bars[s]), 1);
        mbar_init_fence();
    }
    // Persistent schedule: each CTA takes the next tile of the (cost-ordered)
    // list until none is left; the staging ring and its barrier phases run on
    // across tiles (kbase = chunks this CTA has consumed so far).
    __shared__ int s_next;
    int kbase = 0;
    for (int iter = 0;; ++iter) {
    if (threadIdx.x == 0)
        s_next = A.persistent ? atomicAdd(A.tile_counter, 1) : (iter == 0 ? (int)blockIdx.x : A.ntiles);
    __syncthreads();
    const int tnext = s_next;
    __syncthreads();
    if (tnext >= A.ntiles) break;
    const TileDesc td = A.tiles[A.order ? A.order[tnext] : tnext];
    if (td.inst < A.inst_lo || td.inst >= A.inst_hi) continue;
    const InstDesc& I = A.inst[td.inst];
    Control* ctl = A.ctl + td.inst;
    if (*(volatile int*)&ctl->active == 0) continue;

    // Line slot k of this thread: the tile line it marches.  x sweep: rows t
    // and t + 64 (a warp reads 32 consecutive rows per access); y, z: the
    // adjacent lines 2t, 2t + 1 (one 8-byte access covers both).
    auto line_of = [](int k) { return DIR == 0 ? (int)threadIdx.x + k * Cfg::NT : (int)threadIdx.x * PK + k; };
    long long base[PK], stride = 0;
    bool valid[PK];
#pragma unroll
    for (int k = 0; k < PK; ++k) valid[k] = line_geometry<DIR>(td, I, line_of(k), base[k], stride);
    // y, z sweeps: a warp whose lines all lie past the grid edge (the last
    // tile of a line range that is not a multiple of the tile width: uneven
    // ensemble instances) skips the arithmetic and only keeps the CTA's
    // barriers; the x sweep's write-back has barriers inside the march, so
    // its warps always march (a harmless constant state past the edge)
    bool any_valid = false;
#pragma unroll
    for (int k = 0; k < PK; ++k) any_valid |= valid[k];
    const bool live = DIR == 0 || __any_sync(0xffffffffu, any_valid);
    const int N = I.n[DIR];
    const int bc_lo = I.bc[2 * DIR], bc_hi = I.bc[2 * DIR + 1];
    const int a = td.a, b = td.b;
    const int nchunks = (b - a + C - 1) / C;

    // Version slots: TMA plane index and field-plane pointers for each
    // component (a cell of line slot k sits at base[k] + i * stride).
    Real* pool = static_cast<Real*>(A.pool);
    int plane[NP], plane_out[NQ];
    const Real* qin[NQ];
    Real* qout[NQ];
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        const int f = Sys::field(DIR, c);
        const int cur = ctl->cur[f];
        const int sin = (cur + A.slots.in_off[f]) % 3;
        const int sout = (cur + A.slots.out_off[f]) % 3;
        plane[c] = sin * A.m + f;
        plane_out[c] = sout * A.m + f;
        qin[c] = pool + I.offset + sin * I.vstride + f * I.fstride;
        qout[c] = pool + I.offset + sout * I.vstride + f * I.fstride;
    }
#pragma unroll
    for (int k = 0; k < NA; ++k) plane[NQ + k] = k;
    const Real* aux = nullptr;
    if (NA > 0) aux = static_cast<const Real*>(A.aux) + I.aux_offset;
    const CUtensorMap* smap = &A.tma[td.inst].map[DIR];
    const CUtensorMap* amap = &A.tma[td.inst].map[3 + DIR];

    // Coordinates of a bulk copy of this tile at position pos along the
    // line (checked in debug builds only).
    auto coords_ok = [&](int pos) {
        const long long nl = DIR == 0 ? (long long)I.n[1] * I.n[2] : (long long)I.n[0];
        const long long no = DIR == 1 ? (long long)I.n[2] : (DIR == 2 ? (long long)I.n[1] : 1ll);
        return index_ok(pos, N, ctl) && index_ok(td.line0, nl, ctl) && index_ok(td.other, no, ctl);
    };
    // Thread 0 issues chunk k into stage (kbase + k) % STAGES.
    auto issue = [&](int k) {
        const int s = (kbase + k) % STAGES;
        const uint32_t bar = smem_addr(&bars[s]);
        mbar_arrive_expect_tx(bar, Cfg::STAGE_BYTES);
        const int pos = a + k * C;
        // a load is issued even when a check fails (its barrier expects the
        // bytes; the copy fills out-of-range cells), the failure is latched
        if constexpr (kDebugChecks) (void)coords_ok(pos);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const uint32_t dst = smem_addr(smem + s * Cfg::STAGE_BYTES + p * Cfg::BOX);
            const CUtensorMap* map = p < NQ ? smap : amap;
            if (DIR == 0) tma_load_3d(dst, map, bar, pos, td.line0, plane[p]);
            else if (DIR == 1) tma_load_4d(dst, map, bar, td.line0, pos, td.other, plane[p]);
            else tma_load_4d(dst, map, bar, td.line0, td.other, pos, plane[p]);
        }
    };
    if (threadIdx.x == 0) {
        for (int k = 0; k < STAGES && k < nchunks; ++k) issue(k);
    }

    // Direct load of cell k (ghost or interior) for the segment's ends.
    // (lines past the grid edge march a harmless constant state)
    auto load_direct = [&](int kc, Cell& cell) {
        bool flip;
        const int j = map_cell(kc, N, bc_lo, bc_hi, flip);
        V a[NA > 0 ? NA : 1];
#pragma unroll
        for (int k = 0; k < PK; ++k) {
            const long long o = base[k] + (long long)j * stride;
            const bool ok = valid[k] && cell_ok(o, I, ctl);
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                Real x = ok ? __ldg(qin[c] + o) : Real(1);
                if (c == 1 && flip) x = -x;
                set_lane(cell.q[c], k, x);
            }
#pragma unroll
            for (int m = 0; m < NA; ++m)
                set_lane(a[m], k, ok ? __ldg(aux + m * I.fstride + o) : Real(1));
        }
        if constexpr (NA > 0) Sys::set_aux(cell, a);
        Sys::prepare(cell, P);
    };

    const Real nu_s = (Real)(ctl->dt_attempt * A.dt_scale / I.dx[DIR]);
    const V nu = V(nu_s), nnu = V(-nu_s);
    SM smax = 0;
    bool bad = false;
    int hbits = 0x7fffffff;   // running minimum of h's (high) bit pattern

    // March state after interface I (between cells I-1 and I) is solved:
    //   prev   cell I (with its per-cell precomputation)
    //   wB     waves, speeds and fluctuations at interface I
    //   ssB    W_p . W_p at I;  dAB  W_p(I-1) . W_p(I)  (limiter ratios)
    //   apdqA  A+dQ at interface I-1
    //   F0     correction flux at interface I-1;  qkeep  state of cell I-1
    Cell prev;
    W wB;
    V ssB[NW], dAB[NW], apdqA[NQ], F0[NQ], qkeep[NQ];

    auto dot = [](const W& x, const W& y, int p) {
        V d = V(0);
        bool first = true;
#pragma unroll
        for (int c = 0; c < NQ; ++c)
            if (!Sys::zero(p, c)) {
                d = first ? x.W[p][c] * y.W[p][c] : vfma(x.W[p][c], y.W[p][c], d);
                first = false;
            }
        return d;
    };
    // Limited correction flux at interface I (waves wB, ratios from the
    // upwind side: I-1 when s > 0, else I+1).
    auto flux = [&](const V* d_up_left, const V* d_up_right, V* F) {
#pragma unroll
        for (int c = 0; c < NQ; ++c) F[c] = V(0);
        if (LIM == kLimFirstOrder) return;
#pragma unroll
        for (int p = 0; p < NW; ++p) {
            const V sp = wB.s[p];
            V phi = V(1);
            if (LIM != kLimNone) {
                const V num = sel(vgt(sp, V(0)), d_up_left[p], d_up_right[p]);
                phi = limiter_ratio<LIM, V>(num, ssB[p]);
            }
            const V as = vabs(sp);
            // 1/2 |s| (1 - nu |s|) phi; f-waves Z = s W: 1/2 sign(s) (1 - nu |s|) phi
            V k;
            if constexpr (Sys::kFWave)
                k = sel(vgt(sp, V(0)), V(0.5f), sel(vlt(sp, V(0)), V(-0.5f), V(0))) * vfma(nnu, as, V(1)) * phi;
            else
                k = V(0.5f) * as * vfma(nnu, as, V(1)) * phi;
#pragma unroll
            for (int c = 0; c < NQ; ++c)
                if (!Sys::zero(p, c)) F[c] = vfma(k, wB.W[p][c], F[c]);
        }
    };
    // Consume cell I+1: solve interface I+1, limit interface I, form the new
    // state qn of cell I-1.  SPEED: interface I+1 bounds an interior cell of
    // the segment.  UPDATE: cell I-1 belongs to the segment.
    auto step = [&](const Cell& cur, bool speed, bool update, V* qn) {
        W wC;
        Sys::solve(prev, cur, P, wC);
        if (speed) {
            const V ms = Sys::max_speed(wC);
#pragma unroll
            for (int k = 0; k < PK; ++k)
                if (valid[k]) smax = max(smax, speed_bits(lane_of(ms, k)));
        }
        V dBC[NW], ssC[NW];
#pragma unroll
        for (int p = 0; p < NW; ++p) {
            dBC[p] = dot(wB, wC, p);
            ssC[p] = dot(wC, wC, p);
        }
        V F1[NQ];
        flux(dAB, dBC, F1);
        if (update) {
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                const V first = apdqA[c] + wB.amdq[c];
                if (LIM == kLimFirstOrder) {
                    qn[c] = vfma(nnu, first, qkeep[c]);
                } else {
                    const V second = F1[c] - F0[c];
                    qn[c] = vfma(nnu, second, vfma(nnu, first, qkeep[c]));
                }
            }
            if constexpr (Sys::kMinH) {
#pragma unroll
                for (int k = 0; k < PK; ++k) {
                    const Real h = lane_of(qn[0], k);
                    int hb;
                    if constexpr (sizeof(Real) == 4) hb = __float_as_int(h);
                    else hb = (int)(__double_as_longlong(h) >> 32);
                    if (valid[k]) hbits = min(hbits, hb);
                }
            } else {
                const auto np = Sys::nonphysical(qn);
#pragma unroll
                for (int k = 0; k < PK; ++k) bad |= valid[k] && lane_of(np, k);
            }
        }
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            F0[c] = F1[c];
            apdqA[c] = wB.apdq[c];
            qkeep[c] = prev.q[c];
        }
#pragma unroll
        for (int p = 0; p < NW; ++p) {
            dAB[p] = dBC[p];
            ssB[p] = ssC[p];
        }
        wB = wC;
        prev = cur;
    };

    // Prologue (direct loads): cells a-2 .. a+1; interfaces a-1, a, a+1;
    // flux at a.  Needs b - a >= 2 (the tile builder guarantees it).
    if (live) {
        Cell c0, c1;
        W wX;
        load_direct(a - 2, c0);
        load_direct(a - 1, c1);
        Sys::solve(c0, c1, P, wX);                    // interface a-1
        load_direct(a, c0);
        Sys::solve(c1, c0, P, wB);                    // interface a
        {
            const V ms = Sys::max_speed(wB);
#pragma unroll
            for (int k = 0; k < PK; ++k)
                if (valid[k]) smax = max(smax, speed_bits(lane_of(ms, k)));
        }
#pragma unroll
        for (int p = 0; p < NW; ++p) {
            dAB[p] = dot(wX, wB, p);
            ssB[p] = dot(wB, wB, p);
        }
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            F0[c] = V(0);
            apdqA[c] = wX.apdq[c];
            qkeep[c] = c1.q[c];
        }
        prev = c0;                                     // cell a
        load_direct(a + 1, c1);
        V unused[NQ];
        step(c1, true, false, unused);                // interface a+1, flux at a
    }

    // y, z sweeps: the new state of cell i goes straight to global memory (a
    // warp writes 32 consecutive x, whole 128-byte lines).
    auto put_global = [&](int i, const V* qn) {
        if constexpr (PK == 2 && DIR != 0) {
            const long long o = base[0] + (long long)i * stride;   // even: 8-byte aligned
            if (valid[1]) {
                if (cell_ok(o, I, ctl) && cell_ok(o + 1, I, ctl)) {
#pragma unroll
                    for (int c = 0; c < NQ; ++c) *reinterpret_cast<float2*>(qout[c] + o) = qn[c].v;
                }
            } else if (valid[0] && cell_ok(o, I, ctl)) {
#pragma unroll
                for (int c = 0; c < NQ; ++c) qout[c][o] = qn[c].v.x;
            }
        } else {
#pragma unroll
            for (int k = 0; k < PK; ++k)
                if (valid[k] && cell_ok(base[k] + (long long)i * stride, I, ctl)) {
#pragma unroll
                    for (int c = 0; c < NQ; ++c) qout[c][base[k] + (long long)i * stride] = lane_of(qn[c], k);
                }
        }
    };
    constexpr int G = Cfg::G;

    // x sweep: results go back into the input stage they came from (each
    // result overwrites an input position already consumed) and leave by
    // bulk-tensor stores, so the staging buffers serve both ways (a warp's
    // direct stores would touch 32 rows).  Byte offset of chunk position jj
    // of line `lane` inside a plane box:
    // (the 32-byte swizzle of row r swaps its halves on bit 2 of r)
    auto pos_off = [&](int line, int jj) {
        return DIR == 0 ? line * 32 + 16 * ((jj / G) ^ ((line >> 2) & 1)) + (jj % G) * (int)sizeof(Real)
                        : (jj * Cfg::LINES + line) * (int)sizeof(Real);
    };
    auto stage_of = [&](int kk) { return smem + ((kbase + kk) % STAGES) * Cfg::STAGE_BYTES; };
    // result of the cell at position jj of the chunk held by stage st
    auto put_stage = [&](unsigned char* st, int jj, const V* qn) {
#pragma unroll
        for (int k = 0; k < PK; ++k) {
            unsigned char* sk = st + pos_off(line_of(k), jj);
#pragma unroll
            for (int c = 0; c < NQ; ++c) *reinterpret_cast<Real*>(sk + c * Cfg::BOX) = lane_of(qn[c], k);
        }
    };
    auto store_stage = [&](int kk) {       // thread 0
        const unsigned char* st = stage_of(kk);
        const int pos = a + kk * C;
        if (!coords_ok(pos)) {             // debug builds: skip a misplaced store
            bulk_commit();
            return;
        }
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            const uint32_t src = smem_addr(st + c * Cfg::BOX);
            if (DIR == 0) tma_store_3d(smap, src, pos, td.line0, plane_out[c]);
            else if (DIR == 1) tma_store_4d(smap, src, td.line0, pos, td.other, plane_out[c]);
            else tma_store_4d(smap, src, td.line0, td.other, pos, plane_out[c]);
        }
        bulk_commit();
    };
    int stored = 0;        // output chunks already written back

    bool ok = true;
    int kfail = nchunks;
    for (int k = 0; k < nchunks; ++k) {
        const int s = (kbase + k) % STAGES;
        const bool arrived = mbar_wait_bounded(smem_addr(&bars[s]), (uint32_t)(((kbase + k) / STAGES) & 1));
        unsigned char* const stage = smem + s * Cfg::STAGE_BYTES;
        // the stage of chunk k-1 (results of its last two cells land there)
        unsigned char* const stage_prev = smem + ((s + STAGES - 1) % STAGES) * Cfg::STAGE_BYTES;
        const int jlo = k == 0 ? 2 : 0;                // cells a, a+1 came directly
        const int jhi = min(C, b - (a + k * C));       // cells from b on come directly
        // Cells come straight from shared memory as they are marched over;
        // the stage is released once the whole chunk has been consumed.
        auto make_cell = [&](const V* vals, Cell& cur) {
#pragma unroll
            for (int c = 0; c < NQ; ++c) cur.q[c] = vals[c];
            if constexpr (NA > 0) Sys::set_aux(cur, vals + NQ);
            Sys::prepare(cur, P);
        };
        // One cell of line `lane` at a time.  x sweep: the result of cell
        // a + k*C + j - 2 overwrites an input position of this or the previous
        // chunk that has already been consumed.
#pragma unroll 4   // measured: 2 -> 4 takes 3% off the x sweep, 8 is slower
        for (int j = jlo; j < (live ? jhi : jlo); ++j) {
            V vals[NP];
            if constexpr (PK == 2 && DIR != 0) {
                const int off = pos_off(line_of(0), j);
#pragma unroll
                for (int p = 0; p < NP; ++p)
                    vals[p] = V(*reinterpret_cast<const float2*>(stage + p * Cfg::BOX + off));
            } else {
#pragma unroll
                for (int k = 0; k < PK; ++k) {
                    const int off = pos_off(line_of(k), j);
#pragma unroll
                    for (int p = 0; p < NP; ++p)
                        set_lane(vals[p], k, *reinterpret_cast<const Real*>(stage + p * Cfg::BOX + off));
                }
            }
            Cell cur;
            make_cell(vals, cur);
            V qn[NQ];
            step(cur, true, true, qn);
            if (DIR != 0 || !Cfg::XWB) {
                put_global(a + k * C + j - 2, qn);
                continue;
            }
            // cell a + k*C + j - 2: position j - 2 of chunk k, or j + C - 2
            // of chunk k - 1 (j < 2)
            put_stage(j >= 2 ? stage : stage_prev, (j + C - 2) & (C - 1), qn);
            if (j == 1) {
                // output chunk k-1 is complete in its stage: write it back; the
                // write-back issued one chunk ago has had time to read its
                // stage, which is refilled now
                fence_proxy_async_smem();
                __syncthreads();
                if (threadIdx.x == 0) {
                    store_stage(k - 1);
                    if (k >= 2) {
                        bulk_wait_read<1>();
                        if (k - 2 + STAGES < nchunks) issue(k - 2 + STAGES);
                    }
                }
                stored = k;
            }
        }
        // Every thread is done with stage s: it may be refilled.  The vote
        // makes a timed-out wait a uniform decision of the CTA (the chunk's
        // results then land in a version slot that is never kept).
        ok = __syncthreads_and(arrived) != 0;
        if (!ok) {
            kfail = k;
            break;
        }
        // stage s is consumed, refill it (an x sweep writing back through its
        // stages refills after the write-back)
        if ((DIR != 0 || !Cfg::XWB) && threadIdx.x == 0 && k + STAGES < nchunks) issue(k + STAGES);
    }

    if (!ok) {
        // A copy never arrived: record it, wait (bounded) for the copies still
        // in flight into this CTA's shared memory, and leave.
        if (threadIdx.x == 0) {
            atomicOr(&ctl->status, kStatTimeout);
            // chunks kfail .. kfail + STAGES - 1 were issued and not consumed
            for (int k = kfail; k < kfail + STAGES && k < nchunks; ++k)
                mbar_wait_bounded(smem_addr(&bars[(kbase + k) % STAGES]),
                                  (uint32_t)(((kbase + k) / STAGES) & 1));
            if (DIR == 0 && Cfg::XWB) bulk_wait_all();
        }
        return;
    }

    // Epilogue (direct loads): cells b, b+1; the last interface b+1 bounds no
    // interior cell of the segment.
    if (live) {
        Cell c1;
        V qn[NQ];
        load_direct(b, c1);
        step(c1, true, true, qn);
        if (DIR == 0 && Cfg::XWB) put_stage(stage_of((b - 2 - a) / C), (b - 2 - a) % C, qn); else put_global(b - 2, qn);
        load_direct(b + 1, c1);
        step(c1, false, true, qn);
        if (DIR == 0 && Cfg::XWB) put_stage(stage_of((b - 1 - a) / C), (b - 1 - a) % C, qn); else put_global(b - 1, qn);
    }
    if (DIR == 0 && Cfg::XWB) {
        // write back the output chunks still in their stages (a tail past b
        // is the grid edge: clipped); the next tile refills the stages, so the
        // reads must be done
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int ko = stored; ko < nchunks; ++ko) store_stage(ko);
            bulk_wait_read<0>();
        }
    }
    reduce_to_control<DIR>(ctl, smax, bad || hbits <= 0);
    kbase += nchunks;
    }  // tile loop
    if (DIR == 0 && Cfg::XWB && threadIdx.x == 0) bulk_wait_all();
}

}  // namespace claw
