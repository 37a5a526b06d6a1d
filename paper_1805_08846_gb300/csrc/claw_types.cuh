// Device/host data structures shared by the sweep kernels, the step-control
// kernels and the host API of the wave-propagation library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace claw {

// Threads (one grid line each) per tile / CTA of a sweep.
constexpr int kLines = 128;
// sweeps per step at most (3D Strang: x y z y x); each has its own
// persistent tile counter
constexpr int kMaxSweeps = 5;

// Status bits latched on the device and reported by synchronising calls.
enum : unsigned {
    kStatNonPhys = 1u,   // NaN / Inf in the state or h <= 0
    kStatCfl = 2u,       // too many consecutive CFL rejections
    kStatTimeout = 4u,   // a bounded wait gave up
    kStatBounds = 8u,    // an index check failed
};

// Step-control modes (Control::mode).
enum : int { kModeIdle = 0, kModeSteps = 1, kModeTFinal = 2 };

// Geometry and storage of one instance (one grid).  State storage is three
// version slots of m field planes each: element (slot, f, z, y, x) lives at
//   offset + slot * vstride + f * fstride + (z * ny + y) * pitch + x.
struct InstDesc {
    int n[3];              // interior cells nx, ny, nz (nz = 1 in 2D)
    int pitch;             // row pitch in elements (multiple of 32)
    long long fstride;     // elements per field plane: nz * ny * pitch
    long long vstride;     // elements per version slot: m * fstride
    long long offset;      // element offset of slot 0, field 0 in the state pool
    long long aux_offset;  // element offset of the (Z, c) planes in the aux pool, or -1
    double dx[3];
    int bc[6];
    int ndim;
    int pad;
};

// Per-instance step control, resident on the device; only the step-control
// kernels write it (the sweeps read t, dt_attempt, cur[] and active, and
// accumulate smax / bad with atomics).
struct Control {
    double t;              // simulated time of the kept state
    double dt;             // proposal for the next step (cfl_desired / M)
    double t_final;        // target of kModeTFinal
    double dt_attempt;     // step size the sweeps of the current attempt use
    double fixed_dt;       // > 0: fixed step, no CFL control
    double cfl_last;       // Courant number of the last attempt
    double cfl_peak;       // largest Courant number of the steps kept since arming
    double cfl_desired;
    double cfl_max;
    double dt_max;
    double M_last;         // max_d(m_d / dx_d) of the last attempt or speed pass
    long long nacc;        // accepted steps
    long long nrej;        // rejected attempts
    long long target;      // kModeSteps: accept until nacc == target
    unsigned long long smax[3];  // bits of max|s| (as double) per direction
    int cur[4];            // version slot holding each field's kept state
    int mode;
    int active;            // the current attempt runs
    int last;              // the current attempt lands on t_final
    int streak;            // consecutive rejections
    int max_retries;
    unsigned status;       // latched kStat* bits
    unsigned bad;          // non-physical state seen in the current attempt
    int pad;
};

// Debug builds (-DCLAW_DEBUG, the library the CLAW_DEBUG=1 environment loads)
// check the kernels' direct global accesses, in place of a memory checker:
// an element offset o inside a field or material plane of instance I must
// name an interior cell (0 <= o < fstride and o mod pitch < nx), and a bulk
// copy's coordinates must lie in their ranges.  A failed check latches
// kStatBounds (CLAW_EBOUNDS at the next synchronising call) and the caller
// skips the access.  In release builds both checks are the constant true.
#ifdef CLAW_DEBUG
constexpr bool kDebugChecks = true;
#else
constexpr bool kDebugChecks = false;
#endif

__device__ __forceinline__ bool cell_ok(long long o, const InstDesc& I, Control* ctl) {
    if constexpr (kDebugChecks) {
        if (o < 0 || o >= I.fstride || o % I.pitch >= I.n[0]) {
            atomicOr(&ctl->status, kStatBounds);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ bool index_ok(long long i, long long n, Control* ctl) {
    if constexpr (kDebugChecks) {
        if (i < 0 || i >= n) {
            atomicOr(&ctl->status, kStatBounds);
            return false;
        }
    }
    return true;
}

// One tile of a sweep: kLines consecutive lines of one instance and the
// segment [a, b) of each line along the sweep direction.  For the x sweep the
// lines are rows r = line0 + t of the flattened (z, y) index; for the y (z)
// sweep they are columns x = line0 + t of plane z = other (row y = other).
struct TileDesc {
    int inst;
    int line0;
    int other;
    int a, b;
    int pad[3];
};

// Per-sweep description of which version slot each field is read from and
// written to, relative to the field's kept slot (Control::cur).
struct SlotMap {
    signed char in_off[4];
    signed char out_off[4];
};

// Bulk-tensor (TMA) descriptors of one instance: state planes viewed for the
// x, y and z sweeps, and the same three views of the (Z, c) material planes.
struct alignas(64) TmaSet {
    CUtensorMap map[6];
};

struct SweepArgs {
    const TileDesc* tiles;
    const int* order;      // tile visiting order (largest first), or null
    int* tile_counter;     // persistent schedule: next tile to take
    int persistent;
    const TmaSet* tma;
    const InstDesc* inst;
    Control* ctl;
    void* pool;            // state pool (float or double elements)
    const void* aux;       // aux pool: (Z, c) planes per instance
    int ntiles;
    int inst_lo, inst_hi;  // instances this launch may touch
    SlotMap slots;
    double dt_scale;   // this sweep's fraction of the step's dt (Strang: 1/2 or 1)
    int lines;         // lines per tile of this direction's tile list
    int m;                 // fields per state version (TMA plane = slot * m + field)
    double Z, c, g;        // constant acoustics impedance / speed; gravity
    double dry_tol;        // wetting and drying: a cell with h <= dry_tol is dry
};

}  // namespace claw
