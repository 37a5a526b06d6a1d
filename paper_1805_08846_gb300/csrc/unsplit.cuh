// The unsplit two-dimensional wave-propagation update with transverse waves
// (Sec. 3: Eq. LW-update without dimensional splitting, the other form the
// paper's Clawpack base offers).  Every Riemann problem of a step is solved
// from Q^n and each cell is updated once:
//   Q_ij <- Q_ij - nu_x (A+dQ_{i-1/2,j} + A-dQ_{i+1/2,j}) - nu_x (F_{i+1/2,j} - F_{i-1/2,j})
//               - nu_y (B+dQ_{i,j-1/2} + B-dQ_{i,j+1/2}) - nu_y (G_{i,j+1/2} - G_{i,j-1/2}).
// F (G) is the limited correction 1/2 sum_p |s_p| (1 - nu |s_p|) W~_p of an x
// (y) interface plus transverse parts: the x fluctuations entering a cell,
// modified by the corrections (A-dQ + cq from its right interface, A+dQ - cq
// from its left one), are split by a transverse solver into the part that
// crosses the cell's lower y interface and the part that crosses its upper
// one, G_{i,j-+1/2} -= nu_x / 2 B-+(.); the y fluctuations feed F the same
// way with x and y exchanged.
//
// Work mapping.  A warp owns a strip of 32 adjacent columns -- kStrip = 28
// output columns and two halo columns on each side -- and a segment [a, b)
// of rows, and marches down the rows with a register window.  Lane l holds
// column col = x0 - 2 + l; its cells arrive through a ring of rows in shared
// memory, copied asynchronously several rows ahead.  For each row R it reads
// cell (col, R), solves the
// x Riemann problem at interface col-1/2 (the left neighbour's cell arrives
// by shuffle) and the y problem at (col, R-1/2) between its previous and
// current cell.  Everything else needed from the neighbouring columns comes
// by shuffle: the upwind wave of the x limiter, the fluctuation and
// correction entering the cell from its right interface, that interface's
// transverse data, the up-going part of the left neighbour's y-transverse
// split and the right interface's flux.  Row R loaded completes row R-2.
// The transverse solvers are linear in the fluctuation for fixed cell
// states, so the two x fluctuations entering a cell are split as one sum
// (likewise along y).  No wave, fluctuation or flux reaches global memory.
#pragma once
#include "claw_types.cuh"
#include "riemann.cuh"
#include "sweep.cuh"

namespace claw {

constexpr int kStrip = 28;          // output columns of one warp's strip
constexpr int kUnsplitWarps = 4;    // warps (tiles) per CTA
// rows of a warp's shared-memory ring: kRing - 1 in flight ahead of its
// march (measured at 4096^2: 4 rows 0.423 ms, 8 rows 0.419 ms, 12 rows
// 0.430 ms, against 0.484 ms with direct loads two rows ahead)
constexpr int kRing = 8;

// Asynchronous global -> shared copies of one element (4 or 8 bytes), one
// commit group per row, and the wait for all but the newest N groups.
template <class Real>
__device__ __forceinline__ void cp_async_elem(Real* dst, const Real* src) {
    static_assert(sizeof(Real) == 4 || sizeof(Real) == 8, "4- or 8-byte elements");
    if constexpr (sizeof(Real) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ float shfl_idx(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double shfl_idx(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float shfl_dn(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_dn(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }

template <class Real>
__device__ __forceinline__ Real div_(Real a, Real b) {
    return Ops<Real>::div(a, b);
}

template <class Sys>
struct Unsplit;

// ------------------------------------------------------------------------
// Linear acoustics.  The x view of a cell is the solver's (p, u) with its
// (Z, c); v rides along.  Transverse split of a fluctuation a at a cell
// (textbook rule for a heterogeneous medium): the part going down moves at
// -c_d into the cell below, the part going up at +c_u into the cell above,
//   B-(a) = c_d al (Z_d, -1),  al = (-a_p + Z_c a_t) / (Z_d + Z_c),
//   B+(a) = c_u ar (Z_u,  1),  ar = ( a_p + Z_c a_t) / (Z_c + Z_u),
// in the transverse direction's view (p, its normal velocity).  An acoustic
// wave carries no transverse velocity, so a_t = 0 for every fluctuation
// (and correction) of a sweep and the a_t terms vanish.
// ------------------------------------------------------------------------
template <class Real, bool VAR>
struct Unsplit<Acoustics<Real, VAR>> {
    using S = Acoustics<Real, VAR>;
    using Cell = typename S::Cell;
    using Params = typename S::Params;
    static constexpr int NQ = 2;
    struct Full {
        Cell x;    // (p, u; Z, c)
        Real t;    // v
    };
    // Material of an interface's two cells (per-cell coefficients only).
    struct Tr {
        Real Zl, cl, Zr, cr;
    };

    __device__ __forceinline__ static void set(Full& f, const Real q[3], const Real* a, const Params& P) {
        f.x.q[0] = q[0];
        f.x.q[1] = q[1];
        f.t = q[2];
        if constexpr (VAR) S::set_aux(f.x, a);
        S::prepare(f.x, P);
    }
    __device__ __forceinline__ static void fields(const Full& f, Real q[3]) {
        q[0] = f.x.q[0];
        q[1] = f.x.q[1];
        q[2] = f.t;
    }
    __device__ __forceinline__ static Cell xview(const Full& f) { return f.x; }
    __device__ __forceinline__ static Cell yview(const Full& f) {
        Cell y = f.x;
        y.q[1] = f.t;
        return y;
    }
    __device__ __forceinline__ static Cell shfl_cell(const Cell& c, int src, const Params& P) {
        Cell o;
        o.q[0] = shfl_idx(c.q[0], src);
        o.q[1] = shfl_idx(c.q[1], src);
        if constexpr (VAR) {
            o.Z = shfl_idx(c.Z, src);
            o.c = shfl_idx(c.c, src);
        } else {
            S::prepare(o, P);
        }
        return o;
    }
    __device__ __forceinline__ static Tr shfl_tr_dn(const Tr& t) {
        Tr o{};
        if constexpr (VAR) {
            o.Zl = shfl_dn(t.Zl);
            o.cl = shfl_dn(t.cl);
            o.Zr = shfl_dn(t.Zr);
            o.cr = shfl_dn(t.cr);
        }
        return o;
    }
    __device__ __forceinline__ static void solve(const Cell& l, const Cell& r, const Params& P,
                                                 Waves<Real, 2, 2>& w, Tr& t) {
        S::solve(l, r, P, w);
        if constexpr (VAR) {
            t.Zl = l.Z;
            t.cl = l.c;
            t.Zr = r.Z;
            t.cr = r.c;
        }
    }
    // a: fluctuation in the sweep's view (p, normal velocity); lo / hi: the
    // cell's lower / upper transverse interfaces; bm, bp: transverse view.
    __device__ __forceinline__ static void transverse(const Real a[2], const Tr& lo, const Tr& hi,
                                                      const Params& P, Real bm[2], Real bp[2]) {
        Real Zd, cd, Zcl, Zu, cu, Zch;
        if constexpr (VAR) {
            Zd = lo.Zl;
            cd = lo.cl;
            Zcl = lo.Zr;
            Zu = hi.Zr;
            cu = hi.cr;
            Zch = hi.Zl;
        } else {
            Zd = Zcl = Zu = Zch = P.Z;
            cd = cu = P.c;
        }
        const Real al = div_(-a[0], Zd + Zcl);
        const Real ar = div_(a[0], Zch + Zu);
        const Real dl = cd * al, ur = cu * ar;
        bm[0] = dl * Zd;
        bm[1] = -dl;
        bp[0] = ur * Zu;
        bp[1] = ur;
    }
};

// ------------------------------------------------------------------------
// Shallow water.  The x view of a cell is the solver's (h, hu, hv) with its
// velocities, sqrt(h) and sqrt(g h); the y view swaps hu / hv and u / v.
// Transverse split of a fluctuation a at a cell: the Roe averages of the
// cell and its lower (upper) neighbour -- those of the transverse interface
// between them, which its own Riemann problem already formed -- decompose a
// on the eigenvectors of the transverse direction, (1, v~ - c~, u~),
// (0, 0, 1), (1, v~ + c~, u~) (transverse view: h, transverse momentum,
// sweep-normal momentum) with speeds v~ - c~, v~, v~ + c~; the lower part
// keeps the negative speeds, the upper part the positive ones:
//   B-(a) = sum_p min(lam_p, 0) beta_p r_p,  B+(a) = sum_p max(lam_p, 0) beta_p r_p.
// (No entropy fix in the transverse split.)
// ------------------------------------------------------------------------
template <class Real>
struct Unsplit<ShallowWater<Real>> {
    using S = ShallowWater<Real>;
    using Cell = typename S::Cell;
    using Params = typename S::Params;
    static constexpr int NQ = 3;
    struct Full {
        Cell x;
    };
    // Roe averages of an interface in its own view: normal velocity uh,
    // tangential velocity vh, celerity ch, and 1 / (2 ch).
    struct Tr {
        Real uh, vh, ch, i2c;
    };

    __device__ __forceinline__ static void set(Full& f, const Real q[3], const Real*, const Params& P) {
        f.x.q[0] = q[0];
        f.x.q[1] = q[1];
        f.x.q[2] = q[2];
        S::prepare(f.x, P);
    }
    __device__ __forceinline__ static void fields(const Full& f, Real q[3]) {
        q[0] = f.x.q[0];
        q[1] = f.x.q[1];
        q[2] = f.x.q[2];
    }
    __device__ __forceinline__ static Cell xview(const Full& f) { return f.x; }
    __device__ __forceinline__ static Cell yview(const Full& f) {
        Cell y;
        y.q[0] = f.x.q[0];
        y.q[1] = f.x.q[2];
        y.q[2] = f.x.q[1];
        y.u = f.x.v;
        y.v = f.x.u;
        y.sqh = f.x.sqh;
        y.c = f.x.c;
        return y;
    }
    __device__ __forceinline__ static Cell shfl_cell(const Cell& c, int src, const Params&) {
        Cell o;
        o.q[0] = shfl_idx(c.q[0], src);
        o.q[1] = shfl_idx(c.q[1], src);
        o.q[2] = shfl_idx(c.q[2], src);
        o.u = shfl_idx(c.u, src);
        o.v = shfl_idx(c.v, src);
        o.sqh = shfl_idx(c.sqh, src);
        o.c = shfl_idx(c.c, src);
        return o;
    }
    __device__ __forceinline__ static Tr shfl_tr_dn(const Tr& t) {
        return Tr{shfl_dn(t.uh), shfl_dn(t.vh), shfl_dn(t.ch), shfl_dn(t.i2c)};
    }
    __device__ __forceinline__ static void solve(const Cell& l, const Cell& r, const Params& P,
                                                 Waves<Real, 3, 3>& w, Tr& t) {
        S::solve(l, r, P, w, t.uh, t.vh, t.ch, t.i2c);
    }
    template <bool UP>
    __device__ __forceinline__ static void half(const Real a[3], const Tr& t, Real b[3]) {
        // the jump in the transverse view: (h, transverse momentum, sweep-normal momentum)
        const Real a0 = a[0], a1 = a[2], a2 = a[1];
        const Real s1 = t.uh - t.ch, s3 = t.uh + t.ch;
        const Real b1 = (s3 * a0 - a1) * t.i2c;
        const Real b2 = a2 - t.vh * a0;
        const Real b3 = (a1 - s1 * a0) * t.i2c;
        const Real k1 = UP ? vmax(s1, Real(0)) : vmin(s1, Real(0));
        const Real k2 = UP ? vmax(t.uh, Real(0)) : vmin(t.uh, Real(0));
        const Real k3 = UP ? vmax(s3, Real(0)) : vmin(s3, Real(0));
        const Real w1 = k1 * b1, w3 = k3 * b3;
        b[0] = w1 + w3;
        b[1] = w1 * s1 + w3 * s3;
        b[2] = (w1 + w3) * t.vh + k2 * b2;
    }
    __device__ __forceinline__ static void transverse(const Real a[3], const Tr& lo, const Tr& hi,
                                                      const Params&, Real bm[3], Real bp[3]) {
        half<false>(a, lo, bm);
        half<true>(a, hi, bp);
    }
};

// ------------------------------------------------------------------------
// The kernel: one warp per tile (a strip of columns x a segment of rows).
// ------------------------------------------------------------------------
template <class Sys, class Real, int LIM>
__global__ void __launch_bounds__(32 * kUnsplitWarps)
    unsplit_kernel(const SweepArgs A, const typename Sys::Params P) {
    using U = Unsplit<Sys>;
    using Cell = typename U::Cell;
    using Full = typename U::Full;
    using Tr = typename U::Tr;
    constexpr int NQ = Sys::NQ;
    constexpr int NW = Sys::NW;
    constexpr int NA = Sys::NA;
    using W = Waves<Real, NQ, NW>;
    using SM = typename SpeedMax<Real>::T;

    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.x * kUnsplitWarps + (int)(threadIdx.x >> 5);
    if (tile >= A.ntiles) return;                   // whole warp
    const TileDesc td = A.tiles[tile];
    if (td.inst < A.inst_lo || td.inst >= A.inst_hi) return;
    const InstDesc& I = A.inst[td.inst];
    Control* ctl = A.ctl + td.inst;
    if (*(volatile int*)&ctl->active == 0) return;

    // geometry in registers: the stores through qout below could otherwise
    // make the compiler reload these from the descriptor after every store
    const int nx = I.n[0], ny = I.n[1];
    const long long pitch = I.pitch, fstride = I.fstride;
    const int a = td.a, b = td.b;
    int col = td.line0 - 2 + lane;
    const bool out_lane = lane >= 2 && lane < 2 + kStrip && col < nx;
    // the x interface col-1/2 bounds an output cell of the strip
    const bool xif_lane = lane >= 2 && lane <= 2 + kStrip && col <= nx;
    col = min(col, nx + 1);                          // lanes past the ghosts repeat the last one
    bool flip_x;
    const int src_col = map_cell(col, nx, I.bc[0], I.bc[1], flip_x);
    const int bc_ylo = I.bc[2], bc_yhi = I.bc[3];

    Real* pool = static_cast<Real*>(A.pool);
    const Real* qin[3];
    Real* qout[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const int cur = ctl->cur[f];
        const int sin = (cur + A.slots.in_off[f]) % 3;
        const int sout = (cur + A.slots.out_off[f]) % 3;
        qin[f] = pool + I.offset + sin * I.vstride + f * I.fstride;
        qout[f] = pool + I.offset + sout * I.vstride + f * I.fstride;
    }
    const Real* aux = nullptr;
    if (NA > 0) aux = static_cast<const Real*>(A.aux) + I.aux_offset;

    // Field of component c of the x / y view.
    auto fx = [](int c) { return Sys::field(0, c); };
    auto fy = [](int c) { return Sys::field(1, c); };

    // Raw cell (col, R): the three fields (ghosts by the boundary rules, a
    // wall negating the normal momentum / velocity) and the material.
    struct Raw {
        Real q[3];
        Real m[NA > 0 ? NA : 1];
    };
    // Rows arrive through a ring of kRing rows in shared memory: each lane
    // copies its own column of a row (its three fields and the material)
    // asynchronously, kRing - 1 rows ahead of the march, and reads back only
    // what it copied itself.  A slot is refilled one row after it was read
    // (its values consumed by then), so no copy can overwrite a pending read.
    // (Direct loads two rows ahead left the warps waiting on global loads:
    // the top stall of this kernel.)
    constexpr int NPL = 3 + NA;
    __shared__ __align__(16) Real ring_all[kUnsplitWarps][kRing][NPL][32];
    Real (*ring)[NPL][32] = ring_all[threadIdx.x >> 5];
    auto slot_of = [&](int R) { return (R - (a - 2)) % kRing; };
    auto issue_row = [&](int R) {      // a - 2 <= R <= b + 1
        bool flip_y;
        const int sr = map_cell(R, ny, bc_ylo, bc_yhi, flip_y);
        const long long o = (long long)sr * pitch + src_col;
        Real (*dst)[32] = ring[slot_of(R)];
        if (cell_ok(o, I, ctl)) {
#pragma unroll
            for (int f = 0; f < 3; ++f) cp_async_elem(&dst[f][lane], qin[f] + o);
#pragma unroll
            for (int k = 0; k < NA; ++k) cp_async_elem(&dst[3 + k][lane], aux + k * fstride + o);
        } else {
#pragma unroll
            for (int f = 0; f < NPL; ++f) dst[f][lane] = Real(1);
        }
    };
    auto take_row = [&](int R, Raw& r) {
        bool flip_y;
        (void)map_cell(R, ny, bc_ylo, bc_yhi, flip_y);
        const Real (*src)[32] = ring[slot_of(R)];
#pragma unroll
        for (int f = 0; f < 3; ++f) r.q[f] = src[f][lane];
        if (flip_x) r.q[1] = -r.q[1];
        if (flip_y) r.q[2] = -r.q[2];
#pragma unroll
        for (int k = 0; k < NA; ++k) r.m[k] = src[3 + k][lane];
    };

    const double dt = ctl->dt_attempt * A.dt_scale;
    const Real nu_x = (Real)(dt / I.dx[0]), nu_y = (Real)(dt / I.dx[1]);
    const Real hnu_x = (Real)(0.5 * (dt / I.dx[0])), hnu_y = (Real)(0.5 * (dt / I.dx[1]));

    auto dot = [](const W& x, const W& y, int p) {
        Real d = Real(0);
        bool first = true;
#pragma unroll
        for (int c = 0; c < NQ; ++c)
            if (!Sys::zero(p, c)) {
                d = first ? x.W[p][c] * y.W[p][c] : vfma(x.W[p][c], y.W[p][c], d);
                first = false;
            }
        return d;
    };
    // Correction sum_p |s_p| (1 - nu |s_p|) phi_p W_p of waves w, the upwind
    // dot products given per wave.
    auto correction = [&](const W& w, const Real* up_left, const Real* up_right, const Real* self,
                          Real nu, Real* cq) {
#pragma unroll
        for (int c = 0; c < NQ; ++c) cq[c] = Real(0);
        if (LIM == kLimFirstOrder) return;
#pragma unroll
        for (int p = 0; p < NW; ++p) {
            const Real sp = w.s[p];
            Real phi = Real(1);
            if (LIM != kLimNone) phi = limiter_ratio<LIM, Real>(sp > Real(0) ? up_left[p] : up_right[p], self[p]);
            const Real as = fabs(sp);
            const Real k = as * vfma(-nu, as, Real(1)) * phi;
#pragma unroll
            for (int c = 0; c < NQ; ++c)
                if (!Sys::zero(p, c)) cq[c] = vfma(k, w.W[p][c], cq[c]);
        }
    };

    SM smax_x = 0, smax_y = 0;
    bool bad = false;
    int hbits = 0x7fffffff;

    // ---- march state (rows relative to the row R just loaded)
    Full prev;                       // cell (col, R-1)
    Real q2[3];                      // fields of cell (col, R-2)
    Real axf1[NQ], axf2[NQ];         // x fluctuations entering the cell, rows R-1, R-2
    Real axm1[NQ];                   // ... modified by the corrections, row R-1
    Real cqx1[NQ], cqx2[NQ];         // x correction at col-1/2, rows R-1, R-2
    Tr trx1, trx2;                   // x interface col-1/2 transverse data, rows R-1, R-2
    W wyp;                           // y interface R-1 (between rows R-2 and R-1)
    Real ssyp[NW], dleft[NW];        // its W.W and W(R-2).W(R-1)
    Tr tryp;                         // its transverse data
    Real apy2[NQ], cqy2[NQ];         // A+dQ and correction of y interface R-2
    Real G2[NQ];                     // G at y interface R-2
    Real bpx2[NQ];                   // up-going part of the x fluctuations of row R-2

    // rows a-2 .. a-2+kRing-2 in flight, one commit group each (empty past b+1)
#pragma unroll
    for (int k = 0; k < kRing - 1; ++k) {
        if (a - 2 + k <= b + 1) issue_row(a - 2 + k);
        cp_async_commit();
    }
    Raw n0;                          // row a-2
    cp_async_wait<kRing - 2>();
    take_row(a - 2, n0);
    {
        // Start as if row a-3 equalled row a-2: the values this produces
        // belong to rows before a and are never written.
        U::set(prev, n0.q, n0.m, P);
        U::fields(prev, q2);
        W w0;
        Tr t0;
        U::solve(U::xview(prev), U::xview(prev), P, w0, t0);
        trx1 = trx2 = t0;
        U::solve(U::yview(prev), U::yview(prev), P, wyp, tryp);
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            axf1[c] = axf2[c] = axm1[c] = cqx1[c] = cqx2[c] = Real(0);
            apy2[c] = cqy2[c] = G2[c] = bpx2[c] = Real(0);
        }
#pragma unroll
        for (int p = 0; p < NW; ++p) ssyp[p] = dleft[p] = Real(0);
    }

    const int src_l = (lane + 31) & 31, src_r = (lane + 1) & 31;
    // unrolled by two rows (measured at 4096^2: 0.526 -> 0.503 ms; three rows
    // need more registers than three CTAs per SM allow and run at 0.63 ms)
#pragma unroll 2
    for (int R = a - 2; R <= b + 1; ++R) {
        Full cur;
        {
            Raw rr;
            cp_async_wait<kRing - 2>();      // row R's group has landed
            take_row(R, rr);
            // the slot of row R-1, read last iteration, takes row R + kRing - 1
            if (R + kRing - 1 <= b + 1) issue_row(R + kRing - 1);
            cp_async_commit();
            U::set(cur, rr.q, rr.m, P);
        }

        // ---- x Riemann problem at interface col-1/2 of row R
        const Cell cx = U::xview(cur);
        const Cell lx = U::shfl_cell(cx, src_l, P);
        W wx;
        Tr trx;
        U::solve(lx, cx, P, wx, trx);
        if (xif_lane && R >= a && R < b) smax_x = max(smax_x, speed_bits(Sys::max_speed(wx)));
        // x limiter: the upwind wave is the left neighbour's (s > 0) or the right one's
        Real upx[NW], ssx[NW];
#pragma unroll
        for (int p = 0; p < NW; ++p) {
            const int src = wx.s[p] > Real(0) ? src_l : src_r;
            Real num = Real(0);
            bool first = true;
#pragma unroll
            for (int c = 0; c < NQ; ++c)
                if (!Sys::zero(p, c)) {
                    const Real wu = shfl_idx(wx.W[p][c], src);
                    num = first ? wu * wx.W[p][c] : vfma(wu, wx.W[p][c], num);
                    first = false;
                }
            upx[p] = num;
            ssx[p] = dot(wx, wx, p);
        }
        Real cqx[NQ];
        correction(wx, upx, upx, ssx, nu_x, cqx);
        // fluctuations entering cell (col, R) from its left (own) and right
        // (next lane's) x interfaces; modified by the corrections
        Real axf[NQ], axm[NQ];
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            const Real amr = shfl_dn(wx.amdq[c]);
            const Real cqr = shfl_dn(cqx[c]);
            axf[c] = wx.apdq[c] + amr;
            axm[c] = (wx.apdq[c] - cqx[c]) + (amr + cqr);
        }

        // ---- y Riemann problem at (col, R-1/2) and the limiter of R-3/2
        W wy;
        Tr trY;
        U::solve(U::yview(prev), U::yview(cur), P, wy, trY);
        if (out_lane && R >= a && R <= b) smax_y = max(smax_y, speed_bits(Sys::max_speed(wy)));
        Real dmid[NW], ssy[NW];
#pragma unroll
        for (int p = 0; p < NW; ++p) {
            dmid[p] = dot(wyp, wy, p);
            ssy[p] = dot(wy, wy, p);
        }
        Real cqy[NQ];                                     // correction at y interface R-1
        correction(wyp, dleft, dmid, ssyp, nu_y, cqy);
        // y fluctuations entering cell (col, R-2) from interfaces R-2 and R-1
        Real ayf[NQ], aym[NQ];
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            ayf[c] = apy2[c] + wyp.amdq[c];
            aym[c] = (apy2[c] - cqy2[c]) + (wyp.amdq[c] + cqy[c]);
        }

        // ---- x transverse at cell (col, R-1): G at y interface R-1
        Real bmx[NQ], bpx[NQ];                           // y view
        U::transverse(axm1, tryp, trY, P, bmx, bpx);
        Real Gn[NQ];
#pragma unroll
        for (int c = 0; c < NQ; ++c) Gn[c] = Real(0.5) * cqy[c] - hnu_x * (bmx[c] + bpx2[c]);

        // ---- y transverse at cell (col, R-2): F at x interface col-1/2 of row R-2
        const Tr trxr = U::shfl_tr_dn(trx2);
        Real bmy[NQ], bpy[NQ];                           // x view
        U::transverse(aym, trx2, trxr, P, bmy, bpy);
        Real Fl[NQ], Fr[NQ];
#pragma unroll
        for (int c = 0; c < NQ; ++c) Fl[c] = Real(0.5) * cqx2[c] - hnu_y * (bmy[c] + shfl_up1(bpy[c]));
#pragma unroll
        for (int c = 0; c < NQ; ++c) Fr[c] = shfl_dn(Fl[c]);

        // ---- update of cell (col, R-2)
        if (R - 2 >= a) {
            Real qn[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) qn[f] = q2[f];
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                const int f = fx(c);
                qn[f] = vfma(-nu_x, axf2[c], qn[f]);
                qn[f] = vfma(-nu_x, Fr[c] - Fl[c], qn[f]);
            }
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                const int f = fy(c);
                qn[f] = vfma(-nu_y, ayf[c], qn[f]);
                qn[f] = vfma(-nu_y, Gn[c] - G2[c], qn[f]);
            }
            if (out_lane && cell_ok((long long)(R - 2) * pitch + col, I, ctl)) {
                const long long o = (long long)(R - 2) * pitch + col;
#pragma unroll
                for (int f = 0; f < 3; ++f) qout[f][o] = qn[f];
                if constexpr (Sys::kMinH) {
                    int hb;
                    if constexpr (sizeof(Real) == 4) hb = __float_as_int(qn[0]);
                    else hb = (int)(__double_as_longlong(qn[0]) >> 32);
                    hbits = min(hbits, hb);
                } else {
                    bad |= Sys::nonphysical(qn);
                }
            }
        }

        // ---- shift the window
        U::fields(prev, q2);
        prev = cur;
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            axf2[c] = axf1[c];
            axf1[c] = axf[c];
            axm1[c] = axm[c];
            cqx2[c] = cqx1[c];
            cqx1[c] = cqx[c];
            apy2[c] = wyp.apdq[c];
            cqy2[c] = cqy[c];
            G2[c] = Gn[c];
            bpx2[c] = bpx[c];
        }
        trx2 = trx1;
        trx1 = trx;
#pragma unroll
        for (int p = 0; p < NW; ++p) {
            dleft[p] = dmid[p];
            ssyp[p] = ssy[p];
        }
        wyp = wy;
        tryp = trY;
    }
    reduce_to_control<0>(ctl, smax_x, bad || hbits <= 0);
    reduce_to_control<1>(ctl, smax_y, false);
}

template <class Sys, class Real, int LIM>
cudaError_t unsplit_go(const SweepLaunch& L, const typename Sys::Params& P) {
    if (L.lines_out) {
        *L.lines_out = kStrip;
        return cudaSuccess;
    }
    if (L.grid == 0) return cudaSuccess;
    unsplit_kernel<Sys, Real, LIM><<<L.grid, 32 * kUnsplitWarps, 0, L.stream>>>(L.args, P);
    return cudaGetLastError();
}

template <class Sys, class Real>
cudaError_t unsplit_by_limiter(const SweepLaunch& L, const typename Sys::Params& P) {
    switch (L.limiter) {
        case kLimNone: return unsplit_go<Sys, Real, kLimNone>(L, P);
        case kLimMinmod: return unsplit_go<Sys, Real, kLimMinmod>(L, P);
        case kLimFirstOrder: return unsplit_go<Sys, Real, kLimFirstOrder>(L, P);
        default: return unsplit_go<Sys, Real, kLimMC>(L, P);
    }
}

}  // namespace claw
