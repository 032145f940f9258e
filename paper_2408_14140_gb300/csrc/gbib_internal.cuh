// Internal declarations of the GB300 multidirect-forcing IB library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"
#include "gbib.h"

namespace gbib {

// Cells per axis of one spreading tile (the unit owned by one CTA in the
// deterministic gather).  512 cells = one thread per cell.
constexpr int kTile = 8;
constexpr int kTileCells = kTile * kTile * kTile;
// Anchors (first stencil cell) that can touch a tile lie in
// [lo - 3, lo + kTile - 1]; rel = wrap(anchor - lo + 3) is in [0, kRow).
constexpr int kRow = kTile + 3;
constexpr int kRows = kRow * kRow;
// Largest candidate list one tile may gather from.
constexpr int kMaxCand = 4096;
// Bounded spin of device-side waits (iterations of ~100 ns sleeps).
constexpr long long kSpinLimit = 20LL * 1000 * 1000;

struct DevGrid {
    int n[3];
    double h, inv_h, inv_h3;
    double org[3];
};

// One case of a batch on the device: its grid, its fields and its particle
// range in the batch's flat particle arrays.
struct DevCase {
    DevGrid g;
    void *u;                // field of the case
    void *f;                // accumulated force field of the case (nullable)
    int p0, p1;             // particles [p0, p1)
    int tiles[3];           // 8^3 grid tiles per axis (global-tile binning)
    unsigned int tile_off;  // first global-tile slot of the case
    ib_phys phys;           // physical parameters (collision update only)
};

// Case table of a call: a device array of cases, or one case passed by value
// (single-case entry points, which stay capturable into CUDA graphs).
struct CaseTab {
    const DevCase *arr;  // nullptr: every particle belongs to `one`
    const int *pcase;    // [P] case of each particle (with arr)
    int ncases;
    long long ntiles;    // global 8^3 tiles over all cases
    DevCase one;
    __device__ __forceinline__ int case_of(int p) const { return arr ? pcase[p] : 0; }
    // by value: a reference could point at either the kernel parameter or
    // global memory, which forces the parameter into local memory
    __device__ __forceinline__ DevCase get(int c) const { return arr ? arr[c] : one; }
    __device__ __forceinline__ DevCase of_particle(int p) const { return arr ? arr[pcase[p]] : one; }
};

// Device-side error latch: first code wins.
struct DevStatus {
    int code;
    int detail;
};

__device__ __forceinline__ void raise_status(DevStatus *st, int code, int detail) {
    if (atomicCAS(&st->code, 0, code) == 0) st->detail = detail;
}

__host__ __device__ __forceinline__ int wrap_int(long long j, int n) {
    long long m = j % n;
    return (int)(m < 0 ? m + n : m);
}

// Add k (0 <= k < n) to a wrapped index without a modulo.
__device__ __forceinline__ int wrap_add(int j, int k, int n) {
    int v = j + k;
    return v >= n ? v - n : v;
}

// (c - j) mod n for c, j in [0, n).
__device__ __forceinline__ int wrap_diff(int c, int j, int n) {
    int d = c - j;
    return d < 0 ? d + n : d;
}

// Packed wrapped anchor: 21 bits per axis.
__host__ __device__ __forceinline__ uint64_t pack_anchor(int x, int y, int z) {
    return (uint64_t)x | ((uint64_t)y << 21) | ((uint64_t)z << 42);
}
__device__ __forceinline__ int anchor_x(uint64_t a) { return (int)(a & 0x1FFFFF); }
__device__ __forceinline__ int anchor_y(uint64_t a) { return (int)((a >> 21) & 0x1FFFFF); }
__device__ __forceinline__ int anchor_z(uint64_t a) { return (int)(a >> 42); }

template <int KER> struct Kernel;
template <> struct Kernel<IB_DELTA_ROMA3> { static constexpr int W = 3; };
template <> struct Kernel<IB_DELTA_PESKIN4> { static constexpr int W = 4; };

// One axis of the regularised delta kernel.  s is the position in units of
// h measured from the first cell centre; returns the first stencil cell
// (unwrapped) and the kernel weights of the W cells from there.  All
// stencil weights share one square root: for the three-point kernel with
// r = s - round(s) they are ((2 - 3r - q)/6, (1 + q)/3, (2 + 3r - q)/6),
// q = sqrt(1 - 3 r^2); for the four-point kernel with r = s - floor(s)
// they are ((3 - 2r - q)/8, (3 - 2r + q)/8, (1 + 2r + q)/8, (1 + 2r - q)/8),
// q = sqrt(1 + 4r - 4r^2).  These are the piecewise kernels of Roma et al.
// (1999) and Peskin (2002) evaluated at the W offsets of the stencil.
// s, the stencil cell and r are FP64 (r = s - b is exact); the weights are
// FP32 for FP32 fields.
template <int KER>
__device__ __forceinline__ long long axis_weights(double s, float w[4]) {
    if (KER == IB_DELTA_ROMA3) {
        double b = floor(s + 0.5);
        float r = (float)(s - b);
        float q = sqrtf(1.0f - 3.0f * r * r);
        w[0] = (2.0f - 3.0f * r - q) * (float)(1.0 / 6.0);
        w[1] = (1.0f + q) * (float)(1.0 / 3.0);
        w[2] = (2.0f + 3.0f * r - q) * (float)(1.0 / 6.0);
        w[3] = 0.0f;
        return (long long)b - 1;
    } else {
        double b = floor(s);
        float r = (float)(s - b);
        float q = sqrtf(1.0f + 4.0f * r - 4.0f * r * r);
        w[0] = (3.0f - 2.0f * r - q) * 0.125f;
        w[1] = (3.0f - 2.0f * r + q) * 0.125f;
        w[2] = (1.0f + 2.0f * r + q) * 0.125f;
        w[3] = (1.0f + 2.0f * r - q) * 0.125f;
        return (long long)b - 1;
    }
}

// The same weights for FP64 fields as double-float pairs (hi, lo), the form
// the pass kernels read (df.cuh), evaluated on the FP32 pipes: r split on the
// integer pipe, the products from the FMA remainder, the sums by TwoSum, the
// root by one Newton (Heron) step from the FP32 root, and the divisions by 3
// and 6 as products with the pairs of 1/3 and 1/6 (the divisions by 8 and
// the factors 2 and 4 are exact).  Each weight is within a few 2^-47 of the
// FP64 formula, which keeps only the first stencil cell's FP64 arithmetic.
template <int KER>
__device__ __forceinline__ long long axis_weights(double s, float2 w[4]) {
    if (KER == IB_DELTA_ROMA3) {
        const double b = floor(s + 0.5);
        const float2 r = df_split(s - b);
        const float2 r3 = df_mul(r, make_float2(3.0f, 0.0f));
        const float2 q = df_sqrt(df_add(make_float2(1.0f, 0.0f), df_neg(df_mul(r3, r))));
        constexpr float k6 = (float)(1.0 / 6.0), k3 = (float)(1.0 / 3.0);
        const float2 c6 = make_float2(k6, (float)(1.0 / 6.0 - (double)k6));
        const float2 c3 = make_float2(k3, (float)(1.0 / 3.0 - (double)k3));
        w[0] = df_mul(df_add(df_add(make_float2(2.0f, 0.0f), df_neg(r3)), df_neg(q)), c6);
        w[1] = df_mul(df_add(make_float2(1.0f, 0.0f), q), c3);
        w[2] = df_mul(df_add(df_add(make_float2(2.0f, 0.0f), r3), df_neg(q)), c6);
        w[3] = make_float2(0.0f, 0.0f);
        return (long long)b - 1;
    } else {
        const double b = floor(s);
        const float2 r = df_split(s - b);
        const float2 r2 = df_scale(r, 2.0f);
        // 1 + 4r - 4r^2 = 1 + 2 (2r) - (2r)^2
        const float2 q = df_sqrt(df_add(df_add(make_float2(1.0f, 0.0f), df_scale(r2, 2.0f)), df_neg(df_mul(r2, r2))));
        const float2 a = df_add(make_float2(3.0f, 0.0f), df_neg(r2)), c = df_add(make_float2(1.0f, 0.0f), r2);
        w[0] = df_scale(df_add(a, df_neg(q)), 0.125f);
        w[1] = df_scale(df_add(a, q), 0.125f);
        w[2] = df_scale(df_add(c, q), 0.125f);
        w[3] = df_scale(df_add(c, df_neg(q)), 0.125f);
        return (long long)b - 1;
    }
}

// x is finite: its exponent field is not all ones (an integer test, no FP64
// operation)
__device__ __forceinline__ bool finite_bits(double x) {
    return ((unsigned)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffu) != 0x7ffu;
}
__device__ __forceinline__ bool finite3(const double *v) {
    return finite_bits(v[0]) && finite_bits(v[1]) && finite_bits(v[2]);
}

}  // namespace gbib

// ---- host side ------------------------------------------------------------
#include <utility>
#include <vector>

struct ib_ctx {
    int device;
    int sm_count;
    void *ws;            // device workspace
    size_t ws_bytes;
    gbib::DevStatus *status;  // device error latch
    int timing;          // record phase events
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[IB_PHASE_COUNT];
    std::vector<cudaEvent_t> pool;
    // wavefront count of the last multidirect-forcing call (read back
    // asynchronously): how many wavefronts the next call enqueues as separate
    // kernels before the persistent kernel takes the rest
    int *h_nlev;         // pinned host word
    int nlev_hint;
    int pass_kernels;    // IB_PASSES_* of the sequential order
    int vol_split;       // CTAs per particle of the volume integrals (0: one resident wave)
    int spread_mode;     // IB_SPREAD_GATHER (deterministic) or IB_SPREAD_ATOMIC
    int gather_ctas;     // wavefront gather CTAs per SM (0: as many as fit)
    int gather_stage;    // candidates a gather CTA stages (0: the largest capacity)
    void *field_wait;    // cudaEvent_t waited on before the forcing passes (nullable)
    // a second stream and two events: the first interpolation of a forcing
    // call runs on it beside the slot-list kernels (fork and join)
    cudaStream_t fork_stream;
    cudaEvent_t fork_ev[4];  // call start, first interpolation, preparation, levels
    // pinned staging ring for the case tables of batch calls: a slot is
    // reused only after the copy that last read it has run (its event)
    static constexpr int kStageSlots = 4;
    void *stage_ptr[kStageSlots];
    size_t stage_cap[kStageSlots];
    cudaEvent_t stage_ev[kStageSlots];
    int stage_next;
};

// A batch's case table uploaded once (ib_batch_table_create): device memory
// owned by the table, so calls that take it stage nothing on the host.
struct ib_batch_table {
    int device;
    int P, ncases, prec;
    int has_phys;        // physical parameters given (needed by the collision update)
    void *mem;           // device: DevCase[ncases], then int pcase[P]
    size_t cap_cases, cap_p;  // capacity of mem
    void *stage;         // pinned host copy of the last update (read by its upload)
    size_t stage_cap;
    cudaEvent_t staged;  // the last update's upload has read `stage`
    gbib::CaseTab ct;
};

namespace gbib {

// Bump allocator over the context workspace (256-byte aligned chunks).
struct Arena {
    char *base;
    size_t cap, used;
    explicit Arena(ib_ctx *c) : base((char *)c->ws), cap(c->ws_bytes), used(0) {}
    template <typename T> T *take(size_t count) {
        size_t bytes = ((count * sizeof(T)) + 255) & ~(size_t)255;
        if (used + bytes > cap) {
            used += bytes;  // keep counting so the caller can report the need
            return nullptr;
        }
        T *p = (T *)(base + used);
        used += bytes;
        return p;
    }
    bool ok() const { return used <= cap; }
};

int set_error(int code, const char *fmt, ...);
// Record an out-of-workspace failure of `need` bytes and return IB_ERR_OOM.
int oom_error(size_t need, size_t have);
int check_launch(const char *what);
int validate_grid(const ib_grid *g, int need_prec);
DevGrid make_dev_grid(const ib_grid *g);
DevCase make_dev_case(const ib_grid *g, void *u, void *f, int p0, int p1);
// Case table of one case passed by value (no device memory, capturable).
CaseTab single_case(const ib_grid *g, void *u, void *f, int P);
// Case table in the workspace for `ncases` host cases, uploaded on stream `s`
// (a pageable copy: not capturable into a CUDA graph).  Returns an error status
// when the cases are invalid or the workspace is short.
int build_case_table(ib_ctx *ctx, struct Arena &ar, int ncases, const ib_case *cases, int P, int need_prec,
                     CaseTab &ct, cudaStream_t s, const ib_phys *phys = nullptr);
// Host side of a case table: validates the cases (grids, ranges partitioning
// [0, P), one precision when need_prec) and fills h and the global tile count.
int fill_case_table(int ncases, const ib_case *cases, int P, int need_prec, const ib_phys *phys,
                    std::vector<DevCase> &h, unsigned long long &ntiles);
// The table's CaseTab after checking it against the call (device, P).
int table_cases(const ib_batch_table *t, int P, CaseTab &ct);

// Records a CUDA event pair around a scope when the context times phases.
// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialization may start while the kernel before it in
// the stream still runs.  grid_dep_wait() returns once that predecessor grid
// has completed and its memory operations are visible to this grid;
// grid_dep_launch() allows the successor to start once every CTA of this grid
// has executed it (or exited).  Without the launch attribute both are no-ops.
// Every CTA of a kernel launched this way waits before it exits and triggers,
// if at all, only after its wait, so a grid that starts early has every grid
// but its predecessor complete: before its wait it may read anything the
// predecessor does not write.  The preparation kernels of a forcing call wait
// first thing (their launch and scheduling overlap the predecessor's tail);
// the level kernels load what they can before waiting.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Host side: launch with programmatic stream serialization.  The kernel must
// call grid_dep_wait() before it touches memory its predecessor may write.
// With pdl false it is an ordinary launch (after a wait on another stream's
// event, where the kernel's predecessor is not only the one in its stream).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args &&...args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args) {
    return launch_dep(true, kern, grid, block, smem, s, std::forward<Args>(args)...);
}

struct PhaseTimer {
    ib_ctx *ctx;
    int phase;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    PhaseTimer(ib_ctx *c, int ph, cudaStream_t st);
    void stop();
    ~PhaseTimer() { stop(); }
};

}  // namespace gbib
