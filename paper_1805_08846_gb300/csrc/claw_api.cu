// Host side of the C ABI declared in include/claw.h: argument checks, device
// memory, tile lists, CUDA graphs of step attempts, and status reporting.
#include <claw.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "launch.h"

using namespace claw;

namespace {

thread_local std::string g_err;

claw_status fail(claw_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
claw_status fail(claw_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? CLAW_ENOMEM : CLAW_ECUDA,      \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define CKS(expr)                          \
    do {                                   \
        claw_status s_ = (expr);           \
        if (s_ != CLAW_OK) return s_;      \
    } while (0)

int slot_of_version(int v) { return v == 0 ? 0 : 1 + (v - 1) % 2; }

// Fields a sweep along d changes (the reduced state of the Riemann solver).
std::vector<int> touched_fields(int system, int d) {
    if (system == kSysShallowWater || system == kSysShallowWaterBathy || system == kSysShallowWaterDry)
        return {0, 1, 2};
    return {0, 1 + d};
}

bool is_sw(int system) {
    return system == CLAW_SHALLOW_WATER || system == CLAW_SHALLOW_WATER_BATHY || system == CLAW_SHALLOW_WATER_DRY;
}

// Systems with a bottom elevation (one material plane B).
bool has_bed(int system) { return system == CLAW_SHALLOW_WATER_BATHY || system == CLAW_SHALLOW_WATER_DRY; }

// Material planes per cell: (Z, c) for variable acoustics, B for bathymetry.
int aux_planes(int system) { return system == CLAW_ACOUSTICS_VAR ? 2 : (has_bed(system) ? 1 : 0); }

}  // namespace

struct claw_solver {
    int B = 0, ndim = 0, m = 0, mwaves = 0, system = 0, limiter = 0, precision = 64;
    size_t esize = 8;
    claw_params params{};
    int bc[6]{};
    std::vector<InstDesc> inst;
    InstDesc* d_inst = nullptr;
    TmaSet* d_tma = nullptr;
    Control* d_ctl = nullptr;
    Control* h_ctl = nullptr;  // pinned mirror for reads
    void* pool = nullptr;
    void* aux = nullptr;
    double* stage = nullptr;
    double* d_sums = nullptr;
    int* d_counters = nullptr;          // persistent tile schedule, one per sweep of a step
    int* d_order[3] = {nullptr, nullptr, nullptr};
    bool persistent = true;
    size_t stage_elems = 0;
    int seg[3] = {64, 64, 64};
    int tile_lines[3] = {kLines, kLines, kLines};   // lines per tile, from the sweep kernels
    int narrow[3] = {0, 0, 0};                       // narrow tile width per direction
    int tile_order[3] = {0, 0, 0};                   // CLAW_ORDER_* per direction
    std::vector<TileDesc> tiles[3];
    TileDesc* d_tiles[3] = {nullptr, nullptr, nullptr};
    std::vector<std::pair<int, int>> inst_tiles[3];  // [lo, hi) tile range per instance
    // The step's sweeps in order: direction, fraction of dt, version slots.
    int nseq = 0;
    int seq_dir[kMaxSweeps]{};
    double seq_frac[kMaxSweeps]{};
    SlotMap seq_slots[kMaxSweeps]{};
    FinalSlots fin{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::map<int, cudaGraphExec_t> graphs;
    double Z = 0, c = 0;
    // Unsplit update: one kernel per attempt over strip tiles (28 output
    // columns x a segment of seg[1] rows).
    bool unsplit = false;
    std::vector<TileDesc> utiles;
    TileDesc* d_utiles = nullptr;
    // claw_checkpoint: every field's kept version and the control blocks
    void* ckpt = nullptr;
    Control* ckpt_ctl = nullptr;
    std::vector<int> ckpt_cur;   // kept slot of each (instance, field) at the checkpoint
};

namespace {

claw_status check_grid(const claw_grid* g, int ndim_expect) {
    if (!g) return fail(CLAW_EINVAL, "grid is NULL");
    if (g->ndim != 2 && g->ndim != 3) return fail(CLAW_EINVAL, "ndim must be 2 or 3 (got %d)", g->ndim);
    if (ndim_expect && g->ndim != ndim_expect)
        return fail(CLAW_EINVAL, "all ensemble grids must share ndim");
    long long cells = 1;
    for (int d = 0; d < g->ndim; ++d) {
        if (g->n[d] < 2) return fail(CLAW_EINVAL, "n[%d] = %d: need at least 2 cells", d, g->n[d]);
        if (g->n[d] > (1 << 24)) return fail(CLAW_EBOUNDS, "n[%d] = %d too large", d, g->n[d]);
        if (!(g->dx[d] > 0.0)) return fail(CLAW_EINVAL, "dx[%d] must be > 0", d);
        cells *= g->n[d];
    }
    if (cells > (1ll << 34)) return fail(CLAW_EBOUNDS, "grid of %lld cells too large", cells);
    return CLAW_OK;
}

claw_status free_graphs(claw_solver* s) {
    for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
    s->graphs.clear();
    return CLAW_OK;
}

claw_status build_tiles(claw_solver* s) {
    free_graphs(s);
    for (int d = 0; d < s->ndim; ++d) {
        auto& T = s->tiles[d];
        T.clear();
        s->inst_tiles[d].assign(s->B, {0, 0});
        const int L = s->seg[d];
        for (int i = 0; i < s->B; ++i) {
            const InstDesc& I = s->inst[i];
            const int lo = (int)T.size();
            const int N = I.n[d];
            // Segments [a, b) of length L (a multiple of 8); a tail shorter
            // than 2 cells joins the segment before it (the sweep kernel needs
            // b - a >= 2); only the last segment of a line ends mid-chunk.
            std::vector<std::pair<int, int>> segs;
            for (int a = 0; a < N; a += L) segs.push_back({a, std::min(a + L, N)});
            if (segs.size() > 1 && segs.back().second - segs.back().first < 2) {
                segs[segs.size() - 2].second = N;
                segs.pop_back();
            }
            if (d == 0) {
                const int rows = I.n[1] * I.n[2];
                for (int r0 = 0; r0 < rows; r0 += s->tile_lines[0])
                    for (auto& sg : segs) T.push_back({i, r0, 0, sg.first, sg.second, {0, 0, 0}});
            } else {
                const int others = (d == 1) ? I.n[2] : I.n[1];
                for (int o = 0; o < others; ++o)
                    for (int x0 = 0; x0 < I.n[0]; x0 += s->tile_lines[d])
                        for (auto& sg : segs) T.push_back({i, x0, o, sg.first, sg.second, {0, 0, 0}});
            }
            s->inst_tiles[d][i] = {lo, (int)T.size()};
        }
        if (s->d_tiles[d]) cudaFree(s->d_tiles[d]);
        s->d_tiles[d] = nullptr;
        CK(cudaMalloc(&s->d_tiles[d], sizeof(TileDesc) * std::max<size_t>(T.size(), 1)));
        CK(cudaMemcpy(s->d_tiles[d], T.data(), sizeof(TileDesc) * T.size(), cudaMemcpyHostToDevice));
        // Visiting order of the persistent sweep: most cells first (longest
        // processing time first balances uneven instances), stable.
        std::vector<int> order(T.size());
        for (size_t t = 0; t < T.size(); ++t) order[t] = (int)t;
        auto cells = [&](const TileDesc& td) {
            const InstDesc& I = s->inst[td.inst];
            const int nl = d == 0 ? I.n[1] * I.n[2] : I.n[0];
            return (long long)std::min(s->tile_lines[d], nl - td.line0) * (td.b - td.a);
        };
        if (s->tile_order[d] == CLAW_ORDER_LARGEST_FIRST)
            std::stable_sort(order.begin(), order.end(),
                             [&](int x, int y) { return cells(T[x]) > cells(T[y]); });
        if (s->d_order[d]) cudaFree(s->d_order[d]);
        s->d_order[d] = nullptr;
        CK(cudaMalloc(&s->d_order[d], sizeof(int) * std::max<size_t>(order.size(), 1)));
        CK(cudaMemcpy(s->d_order[d], order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice));
    }
    if (s->unsplit) {
        // Strips of kStrip output columns x row segments of seg[1]; the
        // strips of one row segment are adjacent in the list, so the warps
        // of a CTA share their halo columns.
        auto& T = s->utiles;
        T.clear();
        int strip = 0;
        {
            SweepLaunch L{};
            L.system = s->system;
            L.limiter = s->limiter;
            L.precision = s->precision;
            L.lines_out = &strip;
            CK(launch_unsplit(L));
        }
        const int L = s->seg[1];
        for (int i = 0; i < s->B; ++i) {
            const InstDesc& I = s->inst[i];
            for (int a = 0; a < I.n[1]; a += L)
                for (int x0 = 0; x0 < I.n[0]; x0 += strip)
                    T.push_back({i, x0, 0, a, std::min(a + L, I.n[1]), {0, 0, 0}});
        }
        if (s->d_utiles) cudaFree(s->d_utiles);
        s->d_utiles = nullptr;
        CK(cudaMalloc(&s->d_utiles, sizeof(TileDesc) * std::max<size_t>(T.size(), 1)));
        CK(cudaMemcpy(s->d_utiles, T.data(), sizeof(TileDesc) * T.size(), cudaMemcpyHostToDevice));
    }
    return CLAW_OK;
}

// Arguments of a sweep along d; k is its place in the step's sequence (its
// version slots and dt fraction), -1 for passes that update nothing.
SweepArgs sweep_args(claw_solver* s, int d, int tile_lo, int tile_hi, int k = -1) {
    SweepArgs a{};
    a.tiles = s->d_tiles[d] + tile_lo;
    const bool whole = tile_lo == 0 && tile_hi == (int)s->tiles[d].size();
    a.order = whole ? s->d_order[d] : nullptr;
    a.tile_counter = s->d_counters + (k >= 0 ? k : 0);
    a.persistent = whole && s->persistent;
    a.ntiles = tile_hi - tile_lo;
    a.inst = s->d_inst;
    a.tma = s->d_tma;
    a.m = s->m;
    a.ctl = s->d_ctl;
    a.pool = s->pool;
    a.aux = s->aux;
    a.inst_lo = 0;
    a.inst_hi = s->B;
    if (k >= 0) a.slots = s->seq_slots[k];
    a.dt_scale = k >= 0 ? s->seq_frac[k] : 1.0;
    a.lines = s->tile_lines[d];
    a.Z = s->Z;
    a.c = s->c;
    a.g = s->params.g;
    a.dry_tol = s->params.dry_tol;
    return a;
}

claw_status launch_sweep_range(claw_solver* s, int d, int tile_lo, int tile_hi, bool speeds, int k = -1) {
    SweepLaunch L{};
    L.args = sweep_args(s, d, tile_lo, tile_hi, k);
    L.system = s->system;
    L.limiter = s->limiter;
    L.dir = d;
    L.precision = s->precision;
    L.speeds = speeds;
    L.grid = (unsigned)(tile_hi - tile_lo);
    L.stream = s->stream;
    L.narrow = s->narrow[d];
    CK(launch_sweep(L));
    return CLAW_OK;
}

// CTAs of direction d's sweep kernel the whole GPU holds at once.
claw_status resident_ctas(claw_solver* s, int d, int* out) {
    SweepLaunch L{};
    L.args = sweep_args(s, d, 0, (int)s->tiles[d].size());
    L.system = s->system;
    L.limiter = s->limiter;
    L.dir = d;
    L.precision = s->precision;
    L.grid = 1;
    L.stream = s->stream;
    L.resident_out = out;
    L.narrow = s->narrow[d];
    CK(launch_sweep(L));
    return CLAW_OK;
}

// Tiles direction d's sweep has with segments of length L (the tail merge
// of build_tiles aside).
long long tiles_for_segment(const claw_solver* s, int d, int L) {
    long long t = 0;
    for (int i = 0; i < s->B; ++i) {
        const InstDesc& I = s->inst[i];
        const int tl = s->tile_lines[d];
        const long long groups = d == 0 ? ((long long)I.n[1] * I.n[2] + tl - 1) / tl
                                        : (long long)(d == 1 ? I.n[2] : I.n[1]) * ((I.n[0] + tl - 1) / tl);
        t += groups * ((I.n[d] + L - 1) / L);
    }
    return t;
}

// The unsplit update of every instance (one kernel, four strip tiles per CTA).
claw_status launch_unsplit_step(claw_solver* s) {
    SweepLaunch L{};
    L.args = sweep_args(s, 0, 0, 0, 0);
    L.args.tiles = s->d_utiles;
    L.args.order = nullptr;
    L.args.persistent = 0;
    L.args.ntiles = (int)s->utiles.size();
    L.system = s->system;
    L.limiter = s->limiter;
    L.precision = s->precision;
    L.grid = (unsigned)((s->utiles.size() + 3) / 4);
    L.stream = s->stream;
    CK(launch_unsplit(L));
    return CLAW_OK;
}

// Sweep k of the step's sequence over every tile of its direction.
claw_status launch_seq_sweep(claw_solver* s, int k) {
    if (s->unsplit) return launch_unsplit_step(s);
    const int d = s->seq_dir[k];
    return launch_sweep_range(s, d, 0, (int)s->tiles[d].size(), false, k);
}

// One step attempt for every instance: the step's sweeps in order, then the
// step-control kernel.
claw_status enqueue_attempt(claw_solver* s) {
    for (int k = 0; k < s->nseq; ++k) CKS(launch_seq_sweep(s, k));
    CK(launch_finish(s->d_ctl, s->d_inst, 0, s->B, s->fin, s->d_counters, s->stream));
    return CLAW_OK;
}

claw_status get_graph(claw_solver* s, int K, cudaGraphExec_t* out) {
    auto it = s->graphs.find(K);
    if (it != s->graphs.end()) {
        *out = it->second;
        return CLAW_OK;
    }
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    claw_status st = CLAW_OK;
    for (int k = 0; k < K && st == CLAW_OK; ++k) st = enqueue_attempt(s);
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    if (st != CLAW_OK) return st;
    CK(e);
    cudaGraphExec_t ex;
    CK(cudaGraphInstantiate(&ex, g, 0));
    cudaGraphDestroy(g);
    s->graphs[K] = ex;
    *out = ex;
    return CLAW_OK;
}

claw_status read_ctl(claw_solver* s) {
    CK(cudaMemcpyAsync(s->h_ctl, s->d_ctl, sizeof(Control) * s->B, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return CLAW_OK;
}

claw_status status_of(unsigned bits) {
    if (bits & kStatNonPhys) return fail(CLAW_ENONPHYS, "non-finite state or h <= 0 detected on the device");
    if (bits & kStatCfl) return fail(CLAW_ECFL, "too many consecutive CFL rejections");
    if (bits & kStatTimeout) return fail(CLAW_ETIMEOUT, "a device-side wait timed out");
    if (bits & kStatBounds) return fail(CLAW_EBOUNDS, "device-side bounds check failed");
    return CLAW_OK;
}

claw_status latched_status(claw_solver* s, int lo, int hi) {
    unsigned bits = 0;
    for (int i = lo; i < hi; ++i) bits |= s->h_ctl[i].status;
    return status_of(bits);
}

// Replay graphs of step attempts until every instance reached its target
// (kModeSteps) or t_final (kModeTFinal), or latched a fault.
claw_status run_armed(claw_solver* s, int mode, long long nsteps) {
    long long budget;   // attempts, bounded
    int K;
    if (mode == kModeSteps) {
        long long remaining = nsteps;
        while (remaining > 0) {
            K = (int)std::min<long long>(remaining, 512);
            cudaGraphExec_t ex;
            CKS(get_graph(s, K, &ex));
            CK(cudaGraphLaunch(ex, s->stream));
            remaining -= K;
        }
        budget = 64 + 16ll * (s->params.max_retries + 1) * std::max<long long>(nsteps, 1);
        for (;;) {
            CKS(read_ctl(s));
            long long deficit = 0;
            for (int i = 0; i < s->B; ++i)
                if (!s->h_ctl[i].status && s->h_ctl[i].active)
                    deficit = std::max(deficit, s->h_ctl[i].target - s->h_ctl[i].nacc);
            if (deficit <= 0) break;
            if ((budget -= deficit) < 0) return fail(CLAW_ETIMEOUT, "step attempts exceeded their bound");
            K = (int)std::min<long long>(deficit, 512);
            cudaGraphExec_t ex;
            CKS(get_graph(s, K, &ex));
            CK(cudaGraphLaunch(ex, s->stream));
        }
    } else {
        budget = 1ll << 24;
        K = 16;
        for (;;) {
            cudaGraphExec_t ex;
            CKS(get_graph(s, K, &ex));
            CK(cudaGraphLaunch(ex, s->stream));
            CKS(read_ctl(s));
            bool any = false;
            for (int i = 0; i < s->B; ++i) any |= (!s->h_ctl[i].status && s->h_ctl[i].active);
            if (!any) break;
            if ((budget -= K) < 0) return fail(CLAW_ETIMEOUT, "step attempts exceeded their bound");
            K = std::min(K * 2, 256);
        }
    }
    return latched_status(s, 0, s->B);
}

// ---------------------------------------------------------------- TMA descriptors

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

claw_status encode(CUtensorMap* map, CUtensorMapDataType dt, int rank, void* base, const cuuint64_t* dims,
                   const cuuint64_t* strides, const cuuint32_t* box, CUtensorMapSwizzle swz,
                   CUtensorMapL2promotion promo = CU_TENSOR_MAP_L2_PROMOTION_L2_256B) {
    auto fn = encode_fn();
    if (!fn) return fail(CLAW_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = fn(map, dt, rank, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                          promo, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(CLAW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return CLAW_OK;
}

// State planes (3 slots x m fields) and material planes of instance i viewed
// for the x sweep (rows of the flattened (z, y) index) and the y / z sweeps.
claw_status encode_instance(claw_solver* s, int i, TmaSet& T) {
    memset(&T, 0, sizeof T);
    const InstDesc& I = s->inst[i];
    const CUtensorMapDataType dt = s->precision == 64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t es = s->esize;
    // x sweep boxes: the kernel's chunk of each row (32 bytes: swizzled) ×
    // its lines per tile; y / z boxes: lines per tile adjacent x × a chunk
    int chunk = 0;
    {
        SweepLaunch L{};
        L.system = s->system;
        L.limiter = s->limiter;
        L.dir = 0;
        L.precision = s->precision;
        L.grid = 1;
        L.chunk_out = &chunk;
        CK(launch_sweep(L));
    }
    const cuuint32_t cx = (cuuint32_t)chunk;
    const cuuint32_t lx = (cuuint32_t)s->tile_lines[0], ly = (cuuint32_t)s->tile_lines[1],
                     lz = (cuuint32_t)s->tile_lines[2];
    const CUtensorMapSwizzle xsw = cx * es == 32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE;
    const cuuint32_t ct = (cuuint32_t)(32 / es);   // cells per chunk along y / z (4 KB boxes)
    for (int kind = 0; kind < 2; ++kind) {
        if (kind == 1 && aux_planes(s->system) == 0) break;
        char* base = kind == 0 ? (char*)s->pool + I.offset * es : (char*)s->aux + I.aux_offset * es;
        const cuuint64_t planes = kind == 0 ? 3 * (cuuint64_t)s->m : (cuuint64_t)aux_planes(s->system);
        {
            const cuuint64_t dims[3] = {(cuuint64_t)I.n[0], (cuuint64_t)I.n[1] * I.n[2], planes};
            const cuuint64_t str[2] = {(cuuint64_t)I.pitch * es, (cuuint64_t)I.fstride * es};
            const cuuint32_t box[3] = {cx, lx, 1};
            // L2 promotion of 128 B: 256 B fetches whole neighbouring
            // segments' blocks that are evicted before those segments reach
            // them (measured: 1.24x the algorithmic bytes vs 1.03x, and the
            // 512^3 acoustics x sweep 0.76 -> 0.67 ms); 64 B is slower still
            CKS(encode(&T.map[3 * kind + 0], dt, 3, base, dims, str, box, xsw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B));
        }
        const cuuint64_t dims[4] = {(cuuint64_t)I.n[0], (cuuint64_t)I.n[1], (cuuint64_t)I.n[2], planes};
        const cuuint64_t str[3] = {(cuuint64_t)I.pitch * es, (cuuint64_t)I.n[1] * I.pitch * es,
                                   (cuuint64_t)I.fstride * es};
        {
            const cuuint32_t box[4] = {ly, ct, 1, 1};
            CKS(encode(&T.map[3 * kind + 1], dt, 4, base, dims, str, box, CU_TENSOR_MAP_SWIZZLE_NONE));
        }
        if (s->ndim == 3) {
            const cuuint32_t box[4] = {lz, 1, ct, 1};
            CKS(encode(&T.map[3 * kind + 2], dt, 4, base, dims, str, box, CU_TENSOR_MAP_SWIZZLE_NONE));
        }
    }
    return CLAW_OK;
}

// Lines per tile of direction d's sweep kernel at the solver's tile width
// (tile lists and bulk-tensor boxes follow it).
claw_status query_tile_lines(claw_solver* s, int d) {
    SweepLaunch L{};
    L.system = s->system;
    L.limiter = s->limiter;
    L.dir = d;
    L.precision = s->precision;
    L.grid = 1;
    L.narrow = s->narrow[d];
    L.lines_out = &s->tile_lines[d];
    CK(launch_sweep(L));
    return CLAW_OK;
}

// Lines per tile direction d's sweep would have at the given width.
claw_status tile_lines_for(claw_solver* s, int d, int narrow, int* out) {
    SweepLaunch L{};
    L.system = s->system;
    L.limiter = s->limiter;
    L.dir = d;
    L.precision = s->precision;
    L.grid = 1;
    L.narrow = narrow;
    L.lines_out = out;
    CK(launch_sweep(L));
    return CLAW_OK;
}

// Bulk-tensor descriptors of every instance (their boxes follow the tile
// widths) into the device copy.
claw_status encode_all(claw_solver* s) {
    std::vector<TmaSet> tma(s->B);
    for (int i = 0; i < s->B; ++i) CKS(encode_instance(s, i, tma[i]));
    CK(cudaMemcpy(s->d_tma, tma.data(), sizeof(TmaSet) * s->B, cudaMemcpyHostToDevice));
    return CLAW_OK;
}

claw_status speed_pass(claw_solver* s, int i, int set_dt) {
    for (int d = 0; d < s->ndim; ++d) {
        auto r = s->inst_tiles[d][i];
        CKS(launch_sweep_range(s, d, r.first, r.second, true));
    }
    CK(launch_speed_reduce(s->d_ctl, s->d_inst, i, i + 1, set_dt, s->stream));
    return CLAW_OK;
}

claw_status create_impl(int B, const claw_grid* grids, int m, int mwaves, claw_system system,
                        claw_limiter limiter, const claw_bc bc[6], const claw_params* params,
                        void* stream, claw_solver** out) {
    if (!out) return fail(CLAW_EINVAL, "out is NULL");
    *out = nullptr;
    if (B < 1) return fail(CLAW_EINVAL, "ensemble size must be >= 1 (got %d)", B);
    if (!grids || !bc || !params) return fail(CLAW_EINVAL, "NULL argument");
    if (system < CLAW_ACOUSTICS || system > CLAW_SHALLOW_WATER_DRY) return fail(CLAW_EINVAL, "unknown system %d", (int)system);
    if (limiter < CLAW_LIM_NONE || limiter > CLAW_LIM_FIRST_ORDER) return fail(CLAW_EINVAL, "unknown limiter %d", (int)limiter);
    const int ndim = grids[0].ndim;
    for (int i = 0; i < B; ++i) CKS(check_grid(&grids[i], ndim));
    if (is_sw(system) && ndim != 2) return fail(CLAW_EINVAL, "shallow water is 2D only");
    const int m_exp = is_sw(system) ? 3 : ndim + 1;
    const int mw_exp = is_sw(system) ? 3 : 2;
    if (m != m_exp || mwaves != mw_exp)
        return fail(CLAW_EINVAL, "(m, mwaves) = (%d, %d) does not match the system (expected (%d, %d))", m, mwaves, m_exp, mw_exp);
    for (int k = 0; k < 2 * ndim; ++k)
        if (bc[k] < CLAW_BC_PERIODIC || bc[k] > CLAW_BC_WALL) return fail(CLAW_EINVAL, "unknown bc[%d] = %d", k, (int)bc[k]);
    if (params->precision != 32 && params->precision != 64) return fail(CLAW_EINVAL, "precision must be 32 or 64");
    if (params->splitting != CLAW_SPLIT_GODUNOV && params->splitting != CLAW_SPLIT_STRANG &&
        params->splitting != CLAW_SPLIT_UNSPLIT)
        return fail(CLAW_EINVAL, "unknown splitting %d", params->splitting);
    if (params->splitting == CLAW_SPLIT_UNSPLIT && (ndim != 2 || has_bed(system)))
        return fail(CLAW_EINVAL, "the unsplit update covers 2D acoustics and shallow water without bathymetry");
    if (!(params->cfl_desired > 0.0) || !(params->cfl_max > 0.0)) return fail(CLAW_EINVAL, "cfl_desired and cfl_max must be > 0");
    if (!(params->dt_max > 0.0)) return fail(CLAW_EINVAL, "dt_max must be > 0");
    if (!is_sw(system) && (!(params->rho > 0.0) || !(params->K > 0.0)))
        return fail(CLAW_EINVAL, "rho and K must be > 0");
    if (is_sw(system) && !(params->g > 0.0)) return fail(CLAW_EINVAL, "g must be > 0");
    if (system == CLAW_SHALLOW_WATER_DRY && !(params->dry_tol >= 0.0))
        return fail(CLAW_EINVAL, "dry_tol must be >= 0");

    claw_solver* s = new claw_solver();
    s->B = B;
    s->ndim = ndim;
    s->m = m;
    s->mwaves = mwaves;
    s->system = system;
    s->limiter = limiter;
    s->precision = params->precision;
    s->esize = params->precision == 64 ? 8 : 4;
    s->params = *params;
    if (s->params.max_retries <= 0) s->params.max_retries = 8;
    for (int k = 0; k < 6; ++k) s->bc[k] = (k < 2 * ndim) ? bc[k] : CLAW_BC_EXTRAP;
    s->c = std::sqrt(params->K / params->rho);
    s->Z = params->rho * s->c;
    *out = s;   // from here on failures clean up through claw_destroy

    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        CK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
        s->own_stream = true;
    }

    // Storage layout.
    long long off = 0, aux_off = 0;
    size_t max_cells = 0;
    s->inst.resize(B);
    for (int i = 0; i < B; ++i) {
        InstDesc& I = s->inst[i];
        memset(&I, 0, sizeof I);
        I.ndim = ndim;
        for (int d = 0; d < 3; ++d) {
            I.n[d] = d < ndim ? grids[i].n[d] : 1;
            I.dx[d] = d < ndim ? grids[i].dx[d] : 1.0;
        }
        // Row pitch: a multiple of 32 elements (128 B FP32 rows), made an odd
        // multiple so that the rows an x-sweep box spans do not all start at
        // the same power-of-two stride (they would crowd a few HBM channels).
        I.pitch = (I.n[0] + 31) / 32 * 32;
        if ((I.pitch / 32) % 2 == 0) I.pitch += 32;
        I.fstride = (long long)I.n[2] * I.n[1] * I.pitch;
        I.vstride = (long long)m * I.fstride;
        I.offset = off;
        off += 3 * I.vstride;
        off = (off + 63) / 64 * 64;
        if (aux_planes(system) > 0) {
            I.aux_offset = aux_off;
            aux_off += aux_planes(system) * I.fstride;
            aux_off = (aux_off + 63) / 64 * 64;
        } else {
            I.aux_offset = -1;
        }
        for (int k = 0; k < 6; ++k) I.bc[k] = s->bc[k];
        max_cells = std::max(max_cells, (size_t)I.n[0] * I.n[1] * I.n[2]);
    }
    CK(cudaMalloc(&s->pool, (size_t)off * s->esize));
    CK(cudaMemsetAsync(s->pool, 0, (size_t)off * s->esize, s->stream));
    if (aux_off) {
        CK(cudaMalloc(&s->aux, (size_t)aux_off * s->esize));
        CK(cudaMemsetAsync(s->aux, 0, (size_t)aux_off * s->esize, s->stream));   // flat bottom
    }
    s->stage_elems = max_cells * m;
    CK(cudaMalloc(&s->stage, s->stage_elems * sizeof(double)));
    CK(cudaMalloc(&s->d_sums, 8 * (1 + kSumPartsMax) * sizeof(double)));   // sums, then partials
    CK(cudaMalloc(&s->d_counters, kMaxSweeps * sizeof(int)));
    CK(cudaMemsetAsync(s->d_counters, 0, kMaxSweeps * sizeof(int), s->stream));
    CK(cudaMalloc(&s->d_inst, sizeof(InstDesc) * B));
    CK(cudaMemcpyAsync(s->d_inst, s->inst.data(), sizeof(InstDesc) * B, cudaMemcpyHostToDevice, s->stream));
    // Lines per tile of each direction's sweep kernel (tile lists and
    // bulk-tensor boxes follow it).
    for (int d = 0; d < ndim; ++d) CKS(query_tile_lines(s, d));
    CK(cudaMalloc(&s->d_tma, sizeof(TmaSet) * B));
    CKS(encode_all(s));

    std::vector<Control> ctl(B);
    for (int i = 0; i < B; ++i) {
        Control& c = ctl[i];
        memset(&c, 0, sizeof c);
        c.cfl_desired = params->cfl_desired;
        c.cfl_max = params->cfl_max;
        c.dt_max = params->dt_max;
        c.max_retries = s->params.max_retries;
        c.mode = kModeIdle;
    }
    CK(cudaMalloc(&s->d_ctl, sizeof(Control) * B));
    CK(cudaMemcpyAsync(s->d_ctl, ctl.data(), sizeof(Control) * B, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMallocHost(&s->h_ctl, sizeof(Control) * B));

    // The step's sweep sequence (Godunov x, y(, z); Strang half steps
    // outside-in around a full step in the last direction) and each sweep's
    // version slots: a sweep reads a field's latest version of the step and
    // writes the next one; versions after Q^n alternate between slots 1 and
    // 2, so Q^n stays intact until the step is accepted.
    s->nseq = 0;
    s->unsplit = params->splitting == CLAW_SPLIT_UNSPLIT;
    if (s->unsplit) {
        // one update per step from Q^n: every field read from the kept
        // slot and written to the next one
        s->nseq = 1;
        s->seq_dir[0] = 0;
        s->seq_frac[0] = 1.0;
        memset(&s->seq_slots[0], 0, sizeof(SlotMap));
        for (int f = 0; f < m; ++f) s->seq_slots[0].out_off[f] = 1;
        s->fin.m = m;
        for (int f = 0; f < 4; ++f) s->fin.off[f] = f < m ? 1 : 0;
    } else if (params->splitting == CLAW_SPLIT_STRANG) {
        for (int d = 0; d < ndim - 1; ++d) { s->seq_dir[s->nseq] = d; s->seq_frac[s->nseq++] = 0.5; }
        s->seq_dir[s->nseq] = ndim - 1; s->seq_frac[s->nseq++] = 1.0;
        for (int d = ndim - 2; d >= 0; --d) { s->seq_dir[s->nseq] = d; s->seq_frac[s->nseq++] = 0.5; }
    } else {
        for (int d = 0; d < ndim; ++d) { s->seq_dir[s->nseq] = d; s->seq_frac[s->nseq++] = 1.0; }
    }
    int ver[4] = {0, 0, 0, 0};
    for (int k = 0; k < s->nseq && !s->unsplit; ++k) {
        memset(&s->seq_slots[k], 0, sizeof(SlotMap));
        for (int f : touched_fields(system, s->seq_dir[k])) {
            s->seq_slots[k].in_off[f] = (signed char)slot_of_version(ver[f]);
            s->seq_slots[k].out_off[f] = (signed char)slot_of_version(ver[f] + 1);
            ver[f] += 1;
        }
    }
    if (!s->unsplit) {
        s->fin.m = m;
        for (int f = 0; f < 4; ++f) s->fin.off[f] = slot_of_version(ver[f]);
    }

    CKS(build_tiles(s));
    // Initial state: zero (h = 1 for shallow water); material from params.
    for (int i = 0; i < B; ++i) {
        if (is_sw(system)) CK(launch_fill(s->precision, s->pool, s->inst[i], 0, 0, 1.0, s->stream));
        if (system == CLAW_ACOUSTICS_VAR)
            CK(launch_aux_const(s->precision, s->aux, s->inst[i], params->rho, params->K, s->stream));
        CKS(speed_pass(s, i, 1));
    }
    CK(cudaStreamSynchronize(s->stream));
    return CLAW_OK;
}

claw_status check_solver(claw_solver* s, int i = 0) {
    if (!s) return fail(CLAW_EINVAL, "solver is NULL");
    if (i < 0 || i >= s->B) return fail(CLAW_EINVAL, "instance %d out of range [0, %d)", i, s->B);
    return CLAW_OK;
}

// Device-side address of a pinned (page-locked, mapped) host buffer, or
// nullptr for pageable memory.  The conversion kernels read and write pinned
// host buffers directly over the host link (on a Grace-Blackwell part the
// coherent NVLink-C2C), fusing the copy with the precision conversion;
// pageable buffers go through the device stage with cudaMemcpyAsync.
const void* mapped_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // clear: an unknown pointer is pageable memory
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

claw_status set_q_impl(claw_solver* s, int i, const double* q, int on_device) {
    CKS(check_solver(s, i));
    if (!q) return fail(CLAW_EINVAL, "q is NULL");
    const InstDesc& I = s->inst[i];
    const size_t n = (size_t)I.n[0] * I.n[1] * I.n[2] * s->m;
    const double* src = q;
    if (!on_device) {
        src = static_cast<const double*>(mapped_host(q));
        if (!src) {
            CK(cudaMemcpyAsync(s->stage, q, n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
            src = s->stage;
        }
    }
    CK(launch_reset_status(s->d_ctl, i, s->stream));
    CK(launch_convert_in(s->precision, s->pool, I, s->d_ctl + i, src, s->m, s->stream));
    CKS(speed_pass(s, i, 1));
    if (!on_device) CK(cudaStreamSynchronize(s->stream));   // the host buffer may go away
    return CLAW_OK;
}

claw_status get_q_impl(claw_solver* s, int i, double* q, int on_device) {
    CKS(check_solver(s, i));
    if (!q) return fail(CLAW_EINVAL, "q is NULL");
    const InstDesc& I = s->inst[i];
    const size_t n = (size_t)I.n[0] * I.n[1] * I.n[2] * s->m;
    double* mapped = on_device ? nullptr : static_cast<double*>(const_cast<void*>(mapped_host(q)));
    double* dst = on_device ? q : (mapped ? mapped : s->stage);
    CK(launch_convert_out(s->precision, s->pool, I, s->d_ctl + i, dst, s->m, s->stream));
    if (!on_device && !mapped)
        CK(cudaMemcpyAsync(q, s->stage, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CKS(read_ctl(s));
    return latched_status(s, i, i + 1);
}

claw_status set_aux_impl(claw_solver* s, int i, const double* rho, const double* K, int on_device) {
    CKS(check_solver(s, i));
    if (s->system != CLAW_ACOUSTICS_VAR) return fail(CLAW_EINVAL, "claw_set_aux needs CLAW_ACOUSTICS_VAR");
    if (!rho || !K) return fail(CLAW_EINVAL, "rho or K is NULL");
    const InstDesc& I = s->inst[i];
    const size_t n = (size_t)I.n[0] * I.n[1] * I.n[2];
    const double *r = rho, *k = K;
    if (!on_device) {
        // the stage holds m >= 2 fields' worth of doubles
        CK(cudaMemcpyAsync(s->stage, rho, n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        CK(cudaMemcpyAsync(s->stage + n, K, n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        r = s->stage;
        k = s->stage + n;
    }
    CK(launch_aux(s->precision, s->aux, I, r, k, s->stream));
    CKS(speed_pass(s, i, 1));
    CK(cudaStreamSynchronize(s->stream));
    return CLAW_OK;
}

// Rows [y0, y0 + nrows) of every field of a 2D grid, FP64 (m, nrows, nx),
// into (in = true) or out of the kept state: the conversion kernels run on a
// descriptor whose origin is row y0 and whose height is nrows.
claw_status rows_impl(claw_solver* s, int y0, int nrows, double* buf, int on_device, bool in) {
    CKS(check_solver(s));
    if (!buf) return fail(CLAW_EINVAL, "rows buffer is NULL");
    if (s->ndim != 2 || s->B != 1) return fail(CLAW_EINVAL, "row access is for a single 2D grid");
    const InstDesc& I = s->inst[0];
    if (y0 < 0 || nrows < 1 || y0 > I.n[1] - nrows)
        return fail(CLAW_EBOUNDS, "rows [%d, %d) outside [0, %d)", y0, y0 + nrows, I.n[1]);
    InstDesc W = I;
    W.offset += (long long)y0 * I.pitch;
    W.n[1] = nrows;
    const size_t n = (size_t)I.n[0] * nrows * s->m;
    if (in) {
        const double* src = buf;
        if (!on_device) {
            CK(cudaMemcpyAsync(s->stage, buf, n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
            src = s->stage;
        }
        CK(launch_convert_in(s->precision, s->pool, W, s->d_ctl, src, s->m, s->stream));
        if (!on_device) CK(cudaStreamSynchronize(s->stream));   // the host buffer may go away
        return CLAW_OK;
    }
    double* dst = on_device ? buf : s->stage;
    CK(launch_convert_out(s->precision, s->pool, W, s->d_ctl, dst, s->m, s->stream));
    if (!on_device) CK(cudaMemcpyAsync(buf, s->stage, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CKS(read_ctl(s));
    return latched_status(s, 0, 1);
}

claw_status set_bathymetry_impl(claw_solver* s, int i, const double* B, int on_device) {
    CKS(check_solver(s, i));
    if (!has_bed(s->system))
        return fail(CLAW_EINVAL, "claw_set_bathymetry needs CLAW_SHALLOW_WATER_BATHY or CLAW_SHALLOW_WATER_DRY");
    if (!B) return fail(CLAW_EINVAL, "B is NULL");
    const InstDesc& I = s->inst[i];
    const size_t n = (size_t)I.n[0] * I.n[1] * I.n[2];
    const double* b = B;
    if (!on_device) {
        CK(cudaMemcpyAsync(s->stage, B, n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        b = s->stage;
    }
    CK(launch_aux_plane(s->precision, s->aux, I, 0, b, s->stream));
    // with wetting and drying the speeds depend on the bed (reconstruction)
    if (s->system == CLAW_SHALLOW_WATER_DRY) CKS(speed_pass(s, i, 1));
    CK(cudaStreamSynchronize(s->stream));
    return CLAW_OK;
}

}  // namespace

void claw::set_last_error(const char* msg) { g_err = msg; }

cudaError_t claw::launch_unsplit(const SweepLaunch& L) {
    if (L.system == kSysShallowWater)
        return L.precision == 64 ? launch_unsplit_shallow_water_f64(L) : launch_unsplit_shallow_water_f32(L);
    if (L.system == kSysAcoustics || L.system == kSysAcousticsVar)
        return L.precision == 64 ? launch_unsplit_acoustics_f64(L) : launch_unsplit_acoustics_f32(L);
    return cudaErrorInvalidValue;
}

cudaError_t claw::launch_sweep(const SweepLaunch& L) {
    switch (L.system) {
        case kSysAcoustics:
            return L.precision == 64 ? launch_sweep_acoustics_f64(L) : launch_sweep_acoustics_f32(L);
        case kSysAcousticsVar:
            return L.precision == 64 ? launch_sweep_acoustics_var_f64(L) : launch_sweep_acoustics_var_f32(L);
        case kSysShallowWaterBathy:
            return L.precision == 64 ? launch_sweep_shallow_water_bathy_f64(L)
                                     : launch_sweep_shallow_water_bathy_f32(L);
        case kSysShallowWaterDry:
            return L.precision == 64 ? launch_sweep_shallow_water_dry_f64(L)
                                     : launch_sweep_shallow_water_dry_f32(L);
        default:
            return L.precision == 64 ? launch_sweep_shallow_water_f64(L) : launch_sweep_shallow_water_f32(L);
    }
}

extern "C" {

const char* claw_last_error(void) { return g_err.c_str(); }

claw_status claw_create(const claw_grid* grid, int m, int mwaves, claw_system system,
                        claw_limiter limiter, const claw_bc bc[6], const claw_params* params,
                        void* cuda_stream, claw_solver** out) {
    claw_status st = create_impl(1, grid, m, mwaves, system, limiter, bc, params, cuda_stream, out);
    if (st != CLAW_OK && out && *out) {
        std::string keep = g_err;
        claw_destroy(*out);
        *out = nullptr;
        g_err = keep;
    }
    return st;
}

claw_status claw_ensemble_create(int B, const claw_grid* grids, claw_system system,
                                 claw_limiter limiter, const claw_bc bc[6],
                                 const claw_params* params, void* cuda_stream, claw_solver** out) {
    if (!grids) return fail(CLAW_EINVAL, "grids is NULL");
    if (B < 1) return fail(CLAW_EINVAL, "ensemble size must be >= 1 (got %d)", B);
    const int ndim = grids[0].ndim;
    const int m = is_sw(system) ? 3 : ndim + 1;
    const int mw = is_sw(system) ? 3 : 2;
    claw_status st = create_impl(B, grids, m, mw, system, limiter, bc, params, cuda_stream, out);
    if (st != CLAW_OK && out && *out) {
        std::string keep = g_err;
        claw_destroy(*out);
        *out = nullptr;
        g_err = keep;
    }
    return st;
}

void claw_destroy(claw_solver* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    free_graphs(s);
    for (int d = 0; d < 3; ++d) {
        if (s->d_tiles[d]) cudaFree(s->d_tiles[d]);
        if (s->d_order[d]) cudaFree(s->d_order[d]);
    }
    if (s->d_utiles) cudaFree(s->d_utiles);
    if (s->ckpt) cudaFree(s->ckpt);
    if (s->ckpt_ctl) cudaFree(s->ckpt_ctl);
    if (s->d_counters) cudaFree(s->d_counters);
    if (s->pool) cudaFree(s->pool);
    if (s->aux) cudaFree(s->aux);
    if (s->stage) cudaFree(s->stage);
    if (s->d_sums) cudaFree(s->d_sums);
    if (s->d_inst) cudaFree(s->d_inst);
    if (s->d_tma) cudaFree(s->d_tma);
    if (s->d_ctl) cudaFree(s->d_ctl);
    if (s->h_ctl) cudaFreeHost(s->h_ctl);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

claw_status claw_set_q(claw_solver* s, const double* q, int on_device) { return set_q_impl(s, 0, q, on_device); }
claw_status claw_get_q(claw_solver* s, double* q, int on_device) { return get_q_impl(s, 0, q, on_device); }
claw_status claw_set_aux(claw_solver* s, const double* rho, const double* K, int on_device) {
    return set_aux_impl(s, 0, rho, K, on_device);
}
claw_status claw_ensemble_set_q(claw_solver* s, int i, const double* q, int on_device) {
    return set_q_impl(s, i, q, on_device);
}
claw_status claw_ensemble_get_q(claw_solver* s, int i, double* q, int on_device) {
    return get_q_impl(s, i, q, on_device);
}
claw_status claw_ensemble_set_aux(claw_solver* s, int i, const double* rho, const double* K, int on_device) {
    return set_aux_impl(s, i, rho, K, on_device);
}
claw_status claw_set_bathymetry(claw_solver* s, const double* B, int on_device) {
    return set_bathymetry_impl(s, 0, B, on_device);
}
claw_status claw_ensemble_set_bathymetry(claw_solver* s, int i, const double* B, int on_device) {
    return set_bathymetry_impl(s, i, B, on_device);
}
int claw_ensemble_size(const claw_solver* s) { return s ? s->B : 0; }
claw_status claw_get_rows(claw_solver* s, int y0, int nrows, double* out, int on_device) {
    return rows_impl(s, y0, nrows, out, on_device, false);
}
claw_status claw_set_rows(claw_solver* s, int y0, int nrows, const double* rows, int on_device) {
    return rows_impl(s, y0, nrows, const_cast<double*>(rows), on_device, true);
}

claw_status claw_step(claw_solver* s, double dt, double* cfl_out) {
    CKS(check_solver(s));
    CK(launch_arm(s->d_ctl, 0, s->B, kModeSteps, 1, 0.0, dt > 0.0 ? dt : 0.0, 0.0, s->d_counters, s->stream));
    CKS(run_armed(s, kModeSteps, 1));
    if (cfl_out) *cfl_out = s->h_ctl[0].cfl_last;
    return CLAW_OK;
}

claw_status claw_run_fixed_steps(claw_solver* s, int nsteps, double dt, double* cfl_peak) {
    CKS(check_solver(s));
    if (nsteps < 0) return fail(CLAW_EINVAL, "nsteps < 0");
    if (!(dt > 0.0)) return fail(CLAW_EINVAL, "dt must be > 0");
    if (cfl_peak) *cfl_peak = 0.0;
    if (nsteps == 0) return CLAW_OK;
    CK(launch_arm(s->d_ctl, 0, s->B, kModeSteps, nsteps, 0.0, dt, 0.0, s->d_counters, s->stream));
    CKS(run_armed(s, kModeSteps, nsteps));
    if (cfl_peak)
        for (int i = 0; i < s->B; ++i) *cfl_peak = std::max(*cfl_peak, s->h_ctl[i].cfl_peak);
    return CLAW_OK;
}

// Element offset of (instance i, field f) inside the checkpoint buffer.
static long long ckpt_offset(const claw_solver* s, int i, int f) {
    long long off = 0;
    for (int j = 0; j < i; ++j) off += (long long)s->m * s->inst[j].fstride;
    return off + (long long)f * s->inst[i].fstride;
}

claw_status claw_checkpoint(claw_solver* s) {
    CKS(check_solver(s));
    if (!s->ckpt) {
        long long elems = 0;
        for (int i = 0; i < s->B; ++i) elems += (long long)s->m * s->inst[i].fstride;
        CK(cudaMalloc(&s->ckpt, (size_t)elems * s->esize));
        CK(cudaMalloc(&s->ckpt_ctl, sizeof(Control) * s->B));
    }
    CKS(read_ctl(s));                     // the kept slot of every field
    s->ckpt_cur.assign((size_t)s->B * s->m, 0);
    for (int i = 0; i < s->B; ++i)
        for (int f = 0; f < s->m; ++f) {
            const InstDesc& I = s->inst[i];
            const int slot = s->h_ctl[i].cur[f];
            s->ckpt_cur[(size_t)i * s->m + f] = slot;
            const char* src = (const char*)s->pool + (I.offset + slot * I.vstride + f * I.fstride) * s->esize;
            char* dst = (char*)s->ckpt + ckpt_offset(s, i, f) * s->esize;
            CK(cudaMemcpyAsync(dst, src, (size_t)I.fstride * s->esize, cudaMemcpyDeviceToDevice, s->stream));
        }
    CK(cudaMemcpyAsync(s->ckpt_ctl, s->d_ctl, sizeof(Control) * s->B, cudaMemcpyDeviceToDevice, s->stream));
    // the snapshot exists (and any failure of its copies is reported) when
    // the call returns
    CK(cudaStreamSynchronize(s->stream));
    return latched_status(s, 0, s->B);
}

claw_status claw_rollback(claw_solver* s) {
    CKS(check_solver(s));
    if (!s->ckpt || s->ckpt_cur.empty()) return fail(CLAW_EINVAL, "no checkpoint to roll back to");
    for (int i = 0; i < s->B; ++i)
        for (int f = 0; f < s->m; ++f) {
            const InstDesc& I = s->inst[i];
            const int slot = s->ckpt_cur[(size_t)i * s->m + f];
            char* dst = (char*)s->pool + (I.offset + slot * I.vstride + f * I.fstride) * s->esize;
            const char* src = (const char*)s->ckpt + ckpt_offset(s, i, f) * s->esize;
            CK(cudaMemcpyAsync(dst, src, (size_t)I.fstride * s->esize, cudaMemcpyDeviceToDevice, s->stream));
        }
    // the control blocks as they were: kept slots, clock, step counts, next step
    CK(cudaMemcpyAsync(s->d_ctl, s->ckpt_ctl, sizeof(Control) * s->B, cudaMemcpyDeviceToDevice, s->stream));
    CKS(read_ctl(s));
    return latched_status(s, 0, s->B);
}

claw_status claw_run_steps(claw_solver* s, int nsteps) {
    CKS(check_solver(s));
    if (nsteps < 0) return fail(CLAW_EINVAL, "nsteps < 0");
    if (nsteps == 0) return CLAW_OK;
    CK(launch_arm(s->d_ctl, 0, s->B, kModeSteps, nsteps, 0.0, 0.0, 0.0, s->d_counters, s->stream));
    return run_armed(s, kModeSteps, nsteps);
}

claw_status claw_ensemble_run_steps(claw_solver* s, int nsteps) { return claw_run_steps(s, nsteps); }

claw_status claw_advance(claw_solver* s, double t_final, double cfl_target, int* nsteps_out) {
    CKS(check_solver(s));
    CKS(read_ctl(s));
    const double t0 = s->h_ctl[0].t;
    const long long n0 = s->h_ctl[0].nacc;
    if (!(t_final >= t0)) return fail(CLAW_EINVAL, "t_final %.17g is before the current time %.17g", t_final, t0);
    CK(launch_arm(s->d_ctl, 0, s->B, kModeTFinal, 0, t_final, 0.0, cfl_target > 0.0 ? cfl_target : 0.0, s->d_counters, s->stream));
    claw_status st = run_armed(s, kModeTFinal, 0);
    if (nsteps_out) *nsteps_out = (int)(s->h_ctl[0].nacc - n0);
    return st;
}

claw_status claw_max_speed(claw_solver* s, double* smax_over_dx) {
    CKS(check_solver(s));
    if (!smax_over_dx) return fail(CLAW_EINVAL, "output is NULL");
    CKS(speed_pass(s, 0, 0));
    CKS(read_ctl(s));
    *smax_over_dx = s->h_ctl[0].M_last;
    return latched_status(s, 0, 1);
}

claw_status claw_ensemble_get_time(claw_solver* s, int i, double* t, double* dt, long* nsteps) {
    CKS(check_solver(s, i));
    CKS(read_ctl(s));
    if (t) *t = s->h_ctl[i].t;
    if (dt) *dt = s->h_ctl[i].dt;
    if (nsteps) *nsteps = (long)s->h_ctl[i].nacc;
    return latched_status(s, i, i + 1);
}

claw_status claw_get_time(claw_solver* s, double* t, double* dt, long* nsteps) {
    return claw_ensemble_get_time(s, 0, t, dt, nsteps);
}

claw_status claw_get_rejections(claw_solver* s, long* nrej) {
    CKS(check_solver(s));
    CKS(read_ctl(s));
    long tot = 0;
    for (int i = 0; i < s->B; ++i) tot += (long)s->h_ctl[i].nrej;
    if (nrej) *nrej = tot;
    return latched_status(s, 0, s->B);
}

claw_status claw_set_time(claw_solver* s, double t, double dt, long nsteps) {
    CKS(check_solver(s));
    if (nsteps < 0) return fail(CLAW_EINVAL, "nsteps < 0");
    CK(launch_set_time(s->d_ctl, 0, t, dt, nsteps, s->stream));
    if (!(dt > 0.0)) CKS(speed_pass(s, 0, 1));
    CK(cudaStreamSynchronize(s->stream));
    return CLAW_OK;
}

claw_status claw_conservation_sums(claw_solver* s, double* sums) {
    CKS(check_solver(s));
    if (!sums) return fail(CLAW_EINVAL, "sums is NULL");
    CK(launch_sums(s->precision, s->pool, s->inst[0], s->d_ctl, s->m, s->d_sums, s->stream));
    CK(cudaMemcpyAsync(sums, s->d_sums, sizeof(double) * s->m, cudaMemcpyDeviceToHost, s->stream));
    CKS(read_ctl(s));
    return latched_status(s, 0, 1);
}

claw_status claw_set_segment(claw_solver* s, int d, int seg_len) {
    CKS(check_solver(s));
    if (d < 0 || d >= s->ndim) return fail(CLAW_EINVAL, "direction %d out of range", d);
    if (seg_len < 4) return fail(CLAW_EINVAL, "segment length must be >= 4");
    CK(cudaStreamSynchronize(s->stream));
    // Segments are whole chunks (8 cells: 32 bytes of FP32, 2 chunks of
    // FP64): a chunk's results leave as one bulk store, so a segment may end
    // mid-chunk only at the grid edge, where the store is clipped.  For the
    // x sweep this also keeps chunk starts on the bulk copies' 16-byte boundary.
    s->seg[d] = (seg_len + 7) / 8 * 8;
    return build_tiles(s);
}

claw_status claw_set_tile_shape(claw_solver* s, int d, int lines, int seg_len, int order) {
    CKS(check_solver(s));
    if (d < 0 || d >= s->ndim) return fail(CLAW_EINVAL, "direction %d out of range", d);
    if (seg_len != 0 && seg_len < 4) return fail(CLAW_EINVAL, "segment length must be >= 4 (or 0: keep)");
    if (order < -1 || order > CLAW_ORDER_LIST) return fail(CLAW_EINVAL, "unknown tile order %d", order);
    int narrow = s->narrow[d];
    if (lines != 0) {
        int wide = 0, nar = 0;
        CKS(tile_lines_for(s, d, 0, &wide));
        CKS(tile_lines_for(s, d, 1, &nar));
        if (lines == wide) narrow = 0;
        else if (lines == nar) narrow = 1;
        else return fail(CLAW_EINVAL, "direction %d offers %d or %d lines per tile (got %d)", d, wide, nar, lines);
    }
    CK(cudaStreamSynchronize(s->stream));
    if (narrow != s->narrow[d]) {
        s->narrow[d] = narrow;
        CKS(query_tile_lines(s, d));
        CKS(encode_all(s));
    }
    if (seg_len != 0) s->seg[d] = (seg_len + 7) / 8 * 8;   // whole chunks, as claw_set_segment
    if (order >= 0) s->tile_order[d] = order;
    return build_tiles(s);
}

claw_status claw_get_tile_shape(claw_solver* s, int d, int* lines, int* seg_len, int* order) {
    CKS(check_solver(s));
    if (d < 0 || d >= s->ndim) return fail(CLAW_EINVAL, "direction %d out of range", d);
    if (lines) *lines = s->tile_lines[d];
    if (seg_len) *seg_len = s->seg[d];
    if (order) *order = s->tile_order[d];
    return CLAW_OK;
}

claw_status claw_autotune(claw_solver* s, int trial_steps, int seg_out[3]) {
    CKS(check_solver(s));
    if (trial_steps < 1) return fail(CLAW_EINVAL, "trial_steps must be >= 1");
    // Save the state pool and the control blocks; every trial runs from them.
    size_t pool_bytes = 0;
    for (int i = 0; i < s->B; ++i)
        pool_bytes = std::max(pool_bytes, (size_t)((s->inst[i].offset + 3 * s->inst[i].vstride) * s->esize));
    void* saved = nullptr;
    Control* saved_ctl = nullptr;
    CK(cudaMalloc(&saved, pool_bytes));
    CK(cudaMalloc(&saved_ctl, sizeof(Control) * s->B));
    CK(cudaMemcpyAsync(saved, s->pool, pool_bytes, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(saved_ctl, s->d_ctl, sizeof(Control) * s->B, cudaMemcpyDeviceToDevice, s->stream));
    auto restore = [&]() -> claw_status {
        CK(cudaMemcpyAsync(s->pool, saved, pool_bytes, cudaMemcpyDeviceToDevice, s->stream));
        CK(cudaMemcpyAsync(s->d_ctl, saved_ctl, sizeof(Control) * s->B, cudaMemcpyDeviceToDevice, s->stream));
        return CLAW_OK;
    };
    static const int cand_x[] = {16, 32, 48, 64, 96, 128, 192, 256, 512};
    static const int cand_t[] = {8, 16, 24, 32, 48, 64, 96, 128, 256};
    int best[3] = {s->seg[0], s->seg[1], s->seg[2]};
    claw_status st = CLAW_OK;
    if (s->unsplit) {
        // One kernel per step: the rows per strip tile (seg[1]) are the
        // only knob; its time is kernel_ms[0].
        static const int cand_u[] = {16, 24, 32, 48, 64, 96, 128, 192, 256};
        int maxN = 0;
        for (int i = 0; i < s->B; ++i) maxN = std::max(maxN, s->inst[i].n[1]);
        double best_ms = 1e30;
        for (int k = 0; k < 9 && st == CLAW_OK; ++k) {
            if (cand_u[k] > 2 * maxN && k > 0) break;
            st = claw_set_segment(s, 1, cand_u[k]);
            for (int rep = 0; rep < 2 && st == CLAW_OK; ++rep) {
                double ms[4], tot;
                long nl;
                st = claw_profile_steps(s, trial_steps, ms, &tot, &nl);
                if (st == CLAW_OK && ms[0] < best_ms) {
                    best_ms = ms[0];
                    best[1] = s->seg[1];
                }
                if (st == CLAW_OK) st = restore();
            }
        }
        if (st == CLAW_OK) st = claw_set_segment(s, 1, best[1]);
    }
    for (int d = 0; d < s->ndim && st == CLAW_OK && !s->unsplit; ++d) {
        int maxN = 0;
        for (int i = 0; i < s->B; ++i) maxN = std::max(maxN, s->inst[i].n[d]);
        // Tile widths the sweep offers (lines per tile), each searched over
        // segment lengths; then the tile order at the best shape.
        int widths[2] = {0, 0}, nw = 0;
        st = tile_lines_for(s, d, 0, &widths[nw++]);
        if (st == CLAW_OK) st = tile_lines_for(s, d, 1, &widths[nw]);
        if (st != CLAW_OK) break;
        if (widths[1] != widths[0]) ++nw;
        double best_ms = 1e30;
        int best_lines = s->tile_lines[d];
        for (int wi = 0; wi < nw && st == CLAW_OK; ++wi) {
            st = claw_set_tile_shape(s, d, widths[wi], 0, CLAW_ORDER_LARGEST_FIRST);
            if (st != CLAW_OK) break;
            // Fixed lengths, plus for w = 1..4 the shortest segment whose tiles
            // fill at most w waves of resident CTAs (a persistent sweep whose
            // tiles are few and even ends without a partial last wave).
            std::vector<int> cand(d == 0 ? cand_x : cand_t, (d == 0 ? cand_x : cand_t) + 9);
            int resident = 0;
            st = resident_ctas(s, d, &resident);
            if (st != CLAW_OK) break;
            for (int w = 1; w <= 4; ++w) {
                int lo = 8, hi = (maxN + 7) / 8 * 8;
                if (tiles_for_segment(s, d, hi) > (long long)w * resident) continue;
                while (lo < hi) {   // smallest multiple of 8 with few enough tiles
                    const int mid = (lo / 8 + hi / 8) / 2 * 8;
                    if (tiles_for_segment(s, d, mid) <= (long long)w * resident) hi = mid;
                    else lo = mid + 8;
                }
                cand.push_back(lo);
            }
            std::sort(cand.begin(), cand.end());
            cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
            double width_best = 1e30;
            int width_seg = s->seg[d];
            std::vector<int> tried;
            auto trial = [&](int L) -> claw_status {
                if (std::find(tried.begin(), tried.end(), L) != tried.end()) return CLAW_OK;
                tried.push_back(L);
                CKS(claw_set_segment(s, d, L));
                // best of two trials from the same state (the first also warms
                // caches and the new tile lists)
                for (int rep = 0; rep < 2; ++rep) {
                    double ms[4], tot;
                    long nl;
                    CKS(claw_profile_steps(s, trial_steps, ms, &tot, &nl));
                    if (ms[d] < width_best) {
                        width_best = ms[d];
                        width_seg = s->seg[d];
                    }
                    CKS(restore());
                }
                return CLAW_OK;
            };
            for (size_t k = 0; k < cand.size() && st == CLAW_OK; ++k) {
                if (cand[k] > 2 * maxN && k > 0) break;
                st = trial(cand[k]);
            }
            // Second pass: lengths that split the longest line into equal whole
            // chunks (k segments, no short tail), within a factor 1.5 of the
            // first pass's best.
            const int b0 = width_seg;
            for (int k = 1; k <= 256 && st == CLAW_OK; ++k) {
                const int L = ((maxN + k - 1) / k + 7) / 8 * 8;
                if (L < 8) break;
                if (2 * L > 3 * b0 || 3 * L < 2 * b0) continue;
                st = trial(L);
            }
            if (st == CLAW_OK && width_best < best_ms) {
                best_ms = width_best;
                best[d] = width_seg;
                best_lines = widths[wi];
            }
        }
        if (st == CLAW_OK) st = claw_set_tile_shape(s, d, best_lines, best[d], CLAW_ORDER_LARGEST_FIRST);
        // the tile list in its own order (instance, then row / column groups,
        // then segments) instead of largest first
        double list_ms = 1e30;
        if (st == CLAW_OK) st = claw_set_tile_shape(s, d, 0, 0, CLAW_ORDER_LIST);
        for (int rep = 0; rep < 2 && st == CLAW_OK; ++rep) {
            double ms[4], tot;
            long nl;
            st = claw_profile_steps(s, trial_steps, ms, &tot, &nl);
            if (st == CLAW_OK) st = restore();
            list_ms = std::min(list_ms, ms[d]);
        }
        if (st == CLAW_OK && list_ms >= best_ms) st = claw_set_tile_shape(s, d, 0, 0, CLAW_ORDER_LARGEST_FIRST);
    }
    cudaStreamSynchronize(s->stream);
    cudaFree(saved);
    cudaFree(saved_ctl);
    if (st != CLAW_OK) return st;
    if (seg_out)
        for (int d = 0; d < 3; ++d) seg_out[d] = s->seg[d];
    return CLAW_OK;
}

claw_status claw_profile_steps(claw_solver* s, int nsteps, double kernel_ms[4], double* total_ms,
                               long* launches) {
    CKS(check_solver(s));
    if (nsteps < 1) return fail(CLAW_EINVAL, "nsteps must be >= 1");
    const int nk = s->nseq + 1;
    std::vector<cudaEvent_t> ev((size_t)nsteps * nk * 2);
    for (auto& e : ev) CK(cudaEventCreate(&e));
    cudaEvent_t t0, t1;
    CK(cudaEventCreate(&t0));
    CK(cudaEventCreate(&t1));
    CK(launch_arm(s->d_ctl, 0, s->B, kModeSteps, nsteps, 0.0, 0.0, 0.0, s->d_counters, s->stream));
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    claw_status st = CLAW_OK;
    for (int k = 0; k < nsteps && st == CLAW_OK; ++k) {
        for (int j = 0; j <= s->nseq && st == CLAW_OK; ++j) {
            cudaEvent_t* e = &ev[((size_t)k * nk + j) * 2];
            // External records become event nodes of the graph (timestamps),
            // not just capture dependencies.
            cudaEventRecordWithFlags(e[0], s->stream, cudaEventRecordExternal);
            if (j < s->nseq) st = launch_seq_sweep(s, j);
            else if (launch_finish(s->d_ctl, s->d_inst, 0, s->B, s->fin, s->d_counters, s->stream) != cudaSuccess)
                st = fail(CLAW_ECUDA, "finish launch failed");
            cudaEventRecordWithFlags(e[1], s->stream, cudaEventRecordExternal);
        }
    }
    cudaError_t ce = cudaStreamEndCapture(s->stream, &g);
    if (st != CLAW_OK) return st;
    CK(ce);
    cudaGraphExec_t ex;
    CK(cudaGraphInstantiate(&ex, g, 0));
    cudaGraphDestroy(g);
    CK(cudaEventRecord(t0, s->stream));
    CK(cudaGraphLaunch(ex, s->stream));
    CK(cudaEventRecord(t1, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    double acc[4] = {0, 0, 0, 0};
    for (int k = 0; k < nsteps; ++k)
        for (int j = 0; j <= s->nseq; ++j) {
            float ms = 0.f;
            cudaEvent_t* e = &ev[((size_t)k * nk + j) * 2];
            CK(cudaEventElapsedTime(&ms, e[0], e[1]));
            acc[j < s->nseq ? s->seq_dir[j] : 3] += ms;
        }
    float tot = 0.f;
    CK(cudaEventElapsedTime(&tot, t0, t1));
    for (int d = 0; d < 4; ++d) kernel_ms[d] = acc[d] / nsteps;
    if (total_ms) *total_ms = tot;
    if (launches) *launches = (long)nsteps * nk;
    cudaGraphExecDestroy(ex);
    for (auto& e : ev) cudaEventDestroy(e);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    CKS(read_ctl(s));
    return latched_status(s, 0, s->B);
}

}  // extern "C"
