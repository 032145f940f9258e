// Context, workspace, error reporting and the exclusive scan used by the
// binning stages.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "gbib_internal.cuh"

namespace gbib {

static thread_local char g_last_error[512] = "";
static thread_local size_t g_ws_need = 0;

int oom_error(size_t need, size_t have) {
    g_ws_need = need;
    return set_error(IB_ERR_OOM, "workspace too small: need %zu bytes (have %zu); call ib_ctx_reserve",
                     need, have);
}

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return code;
}

int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(IB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return IB_OK;
}

int validate_grid(const ib_grid *g, int need_prec) {
    if (!g) return set_error(IB_ERR_INVALID, "grid is NULL");
    for (int a = 0; a < 3; ++a)
        if (g->n[a] < 12 || g->n[a] >= (1 << 21))
            return set_error(IB_ERR_INVALID, "grid n[%d]=%d outside [12, 2^21)", a, g->n[a]);
    if (!(g->h > 0.0) || !isfinite(g->h))
        return set_error(IB_ERR_INVALID, "grid h must be finite and > 0");
    for (int a = 0; a < 3; ++a)
        if (!isfinite(g->origin[a])) return set_error(IB_ERR_INVALID, "grid origin not finite");
    if (need_prec && g->prec != IB_F64 && g->prec != IB_F32)
        return set_error(IB_ERR_INVALID, "grid prec must be IB_F64 or IB_F32");
    long long cells = (long long)g->n[0] * g->n[1] * g->n[2];
    if (cells > (1LL << 40)) return set_error(IB_ERR_INVALID, "grid too large");
    return IB_OK;
}

DevGrid make_dev_grid(const ib_grid *g) {
    DevGrid d;
    for (int a = 0; a < 3; ++a) {
        d.n[a] = g->n[a];
        d.org[a] = g->origin[a];
    }
    d.h = g->h;
    d.inv_h = 1.0 / g->h;
    d.inv_h3 = 1.0 / (g->h * g->h * g->h);
    return d;
}

DevCase make_dev_case(const ib_grid *g, void *u, void *f, int p0, int p1) {
    DevCase c;
    c.g = make_dev_grid(g);
    c.u = u;
    c.f = f;
    c.p0 = p0;
    c.p1 = p1;
    for (int a = 0; a < 3; ++a) c.tiles[a] = (g->n[a] + kTile - 1) / kTile;
    c.tile_off = 0;
    c.phys = ib_phys{};
    return c;
}

CaseTab single_case(const ib_grid *g, void *u, void *f, int P) {
    CaseTab ct;
    ct.arr = nullptr;
    ct.pcase = nullptr;
    ct.ncases = 1;
    ct.one = make_dev_case(g, u, f, 0, P);
    ct.ntiles = (long long)ct.one.tiles[0] * ct.one.tiles[1] * ct.one.tiles[2];
    return ct;
}

__global__ void k_case_of_particle(const DevCase *cases, int ncases, int *pcase) {
    for (int c = blockIdx.x; c < ncases; c += gridDim.x)
        for (int p = cases[c].p0 + threadIdx.x; p < cases[c].p1; p += blockDim.x) pcase[p] = c;
}

int fill_case_table(int ncases, const ib_case *cases, int P, int need_prec, const ib_phys *phys,
                    std::vector<DevCase> &h, unsigned long long &toff) {
    if (ncases < 1 || !cases) return set_error(IB_ERR_INVALID, "batch needs ncases >= 1 and a case array");
    int prec = cases[0].grid.prec;
    h.assign(ncases, DevCase{});
    toff = 0;
    for (int c = 0; c < ncases; ++c) {
        int rc = validate_grid(&cases[c].grid, need_prec);
        if (rc) return set_error(rc, "case %d: %s", c, ib_last_error());
        if (need_prec && cases[c].grid.prec != prec) return set_error(IB_ERR_INVALID, "case %d: mixed precisions", c);
        const int expect = c == 0 ? 0 : cases[c - 1].p_end;
        if (cases[c].p_begin != expect || cases[c].p_end < cases[c].p_begin)
            return set_error(IB_ERR_INVALID, "case %d: particle ranges must partition [0, P) in order", c);
        h[c] = make_dev_case(&cases[c].grid, cases[c].u, cases[c].f_out, cases[c].p_begin, cases[c].p_end);
        if (phys) h[c].phys = phys[c];
        h[c].tile_off = (unsigned int)toff;
        toff += (unsigned long long)h[c].tiles[0] * h[c].tiles[1] * h[c].tiles[2];
        if (toff > (1ull << 30)) return set_error(IB_ERR_UNSUPPORTED, "batch has too many grid tiles");
    }
    if (cases[ncases - 1].p_end != P) return set_error(IB_ERR_INVALID, "case ranges must end at P = %d", P);
    return IB_OK;
}

int build_case_table(ib_ctx *ctx, Arena &ar, int ncases, const ib_case *cases, int P, int need_prec,
                     CaseTab &ct, cudaStream_t s, const ib_phys *phys) {
    std::vector<DevCase> h;
    unsigned long long toff = 0;
    int rc = fill_case_table(ncases, cases, P, need_prec, phys, h, toff);
    if (rc) return rc;
    DevCase *d = ar.take<DevCase>(ncases);
    int *pcase = ar.take<int>(P > 0 ? P : 1);
    if (!ar.ok()) return oom_error(ar.used, ar.cap);
    // stage through a pinned slot so that the upload stays asynchronous
    const size_t bytes = sizeof(DevCase) * ncases;
    const int k = ctx->stage_next;
    ctx->stage_next = (k + 1) % ib_ctx::kStageSlots;
    if (ctx->stage_ev[k]) cudaEventSynchronize(ctx->stage_ev[k]);
    else if (cudaEventCreateWithFlags(&ctx->stage_ev[k], cudaEventDisableTiming) != cudaSuccess)
        return set_error(IB_ERR_CUDA, "case table event: %s", cudaGetErrorString(cudaGetLastError()));
    if (ctx->stage_cap[k] < bytes) {
        if (ctx->stage_ptr[k]) cudaFreeHost(ctx->stage_ptr[k]);
        ctx->stage_ptr[k] = nullptr;
        ctx->stage_cap[k] = 0;
        if (cudaHostAlloc(&ctx->stage_ptr[k], bytes, cudaHostAllocDefault) != cudaSuccess)
            return set_error(IB_ERR_CUDA, "case table staging: %s", cudaGetErrorString(cudaGetLastError()));
        ctx->stage_cap[k] = bytes;
    }
    memcpy(ctx->stage_ptr[k], h.data(), bytes);
    if (cudaMemcpyAsync(d, ctx->stage_ptr[k], bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return set_error(IB_ERR_CUDA, "case table upload: %s", cudaGetErrorString(cudaGetLastError()));
    cudaEventRecord(ctx->stage_ev[k], s);
    k_case_of_particle<<<ncases < 1024 ? ncases : 1024, 128, 0, s>>>(d, ncases, pcase);
    ct.arr = d;
    ct.pcase = pcase;
    ct.ncases = ncases;
    ct.ntiles = (long long)toff;
    ct.one = h[0];
    return check_launch("case table");
}

int table_cases(const ib_batch_table *t, int P, CaseTab &ct) {
    if (!t) return set_error(IB_ERR_INVALID, "table is NULL");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != t->device)
        return set_error(IB_ERR_INVALID, "table belongs to device %d, current device is %d", t->device, dev);
    if (P != t->P) return set_error(IB_ERR_INVALID, "table has P = %d particles, the call %d", t->P, P);
    ct = t->ct;
    return IB_OK;
}

}  // namespace gbib

// Validates the cases and uploads the table into t's memory on stream s,
// growing it first if needed (a synchronous reallocation); the host copy sits
// in t's pinned stage, reused once the previous upload from it has run.
static int table_upload(ib_batch_table *t, int ncases, const ib_case *cases, int P, const ib_phys *phys,
                        cudaStream_t s) {
    using namespace gbib;
    if (P < 0) return set_error(IB_ERR_INVALID, "P must be >= 0");
    for (int c = 0; c < ncases && cases; ++c) {
        if (!cases[c].u) return set_error(IB_ERR_INVALID, "case %d: NULL field", c);
        if (phys && (!(phys[c].eps_c > 0.0) || !(phys[c].d_c > 0.0)))
            return set_error(IB_ERR_INVALID, "case %d: eps_c and d_c must be > 0", c);
    }
    std::vector<DevCase> h;
    unsigned long long toff = 0;
    int rc = fill_case_table(ncases, cases, P, 1, phys, h, toff);
    if (rc) return rc;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || (t->mem && dev != t->device))
        return set_error(IB_ERR_INVALID, "table belongs to device %d, current device is %d", t->device, dev);
    if (!t->mem || (size_t)ncases > t->cap_cases || (size_t)(P > 0 ? P : 1) > t->cap_p) {
        // grow with headroom (rare: later updates of similar batches fit)
        const size_t cc = (size_t)ncases * 2 + 16, cp = (size_t)(P > 0 ? P : 1) * 2 + 64;
        const size_t cbytes = ((sizeof(DevCase) * cc + 255) / 256) * 256;
        void *mem = nullptr;
        if (cudaMalloc(&mem, cbytes + sizeof(int) * cp) != cudaSuccess)
            return set_error(IB_ERR_OOM, "case table: %s", cudaGetErrorString(cudaGetLastError()));
        if (t->mem) {
            cudaDeviceSynchronize();  // work queued on the old table has finished
            cudaFree(t->mem);
        }
        t->mem = mem;
        t->cap_cases = cc;
        t->cap_p = cp;
        t->device = dev;
    }
    const size_t cbytes = ((sizeof(DevCase) * t->cap_cases + 255) / 256) * 256;
    const size_t hb = sizeof(DevCase) * ncases, pb = sizeof(int) * (size_t)(P > 0 ? P : 1);
    if (t->staged) cudaEventSynchronize(t->staged);  // the previous upload has read the stage
    else if (cudaEventCreateWithFlags(&t->staged, cudaEventDisableTiming) != cudaSuccess)
        return set_error(IB_ERR_CUDA, "table event: %s", cudaGetErrorString(cudaGetLastError()));
    if (t->stage_cap < hb + pb) {
        if (t->stage) cudaFreeHost(t->stage);
        t->stage = nullptr;
        t->stage_cap = 0;
        if (cudaHostAlloc(&t->stage, hb + pb, cudaHostAllocDefault) != cudaSuccess)
            return set_error(IB_ERR_CUDA, "table staging: %s", cudaGetErrorString(cudaGetLastError()));
        t->stage_cap = hb + pb;
    }
    memcpy(t->stage, h.data(), hb);
    int *ps = (int *)((char *)t->stage + hb);
    for (int p = 0; p < P; ++p) ps[p] = 0;
    for (int c = 0; c < ncases; ++c)
        for (int p = cases[c].p_begin; p < cases[c].p_end; ++p) ps[p] = c;
    DevCase *d = (DevCase *)t->mem;
    int *dp = (int *)((char *)t->mem + cbytes);
    cudaError_t e = cudaMemcpyAsync(d, t->stage, hb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, ps, pb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(t->staged, s);
    if (e != cudaSuccess) return set_error(IB_ERR_CUDA, "case table upload: %s", cudaGetErrorString(e));
    t->P = P;
    t->ncases = ncases;
    t->prec = cases[0].grid.prec;
    t->has_phys = phys != nullptr;
    t->ct.arr = d;
    t->ct.pcase = dp;
    t->ct.ncases = ncases;
    t->ct.ntiles = (long long)toff;
    t->ct.one = h[0];
    return IB_OK;
}

extern "C" int ib_batch_table_create(ib_ctx *ctx, int ncases, const ib_case *cases, int P, const ib_phys *phys,
                                     ib_batch_table **out) {
    using namespace gbib;
    if (!ctx || !out) return set_error(IB_ERR_INVALID, "ctx or out is NULL");
    *out = nullptr;
    ib_batch_table *t = new (std::nothrow) ib_batch_table();
    if (!t) return set_error(IB_ERR_OOM, "table");
    // upload on a private non-blocking stream: the copy waits for nothing the
    // caller has queued (not even on the legacy default stream)
    cudaStream_t us = nullptr;
    if (cudaStreamCreateWithFlags(&us, cudaStreamNonBlocking) != cudaSuccess) {
        delete t;
        return set_error(IB_ERR_CUDA, "table stream: %s", cudaGetErrorString(cudaGetLastError()));
    }
    int rc = table_upload(t, ncases, cases, P, phys, us);
    if (rc == IB_OK && cudaStreamSynchronize(us) != cudaSuccess)
        rc = set_error(IB_ERR_CUDA, "case table upload: %s", cudaGetErrorString(cudaGetLastError()));
    cudaStreamDestroy(us);
    if (rc) {
        ib_batch_table_destroy(t);
        return rc;
    }
    *out = t;
    return IB_OK;
}

extern "C" int ib_batch_table_update(ib_batch_table *t, int ncases, const ib_case *cases, int P,
                                     const ib_phys *phys, void *stream) {
    using namespace gbib;
    if (!t) return set_error(IB_ERR_INVALID, "table is NULL");
    return table_upload(t, ncases, cases, P, phys, (cudaStream_t)stream);
}

extern "C" int ib_batch_table_destroy(ib_batch_table *t) {
    if (!t) return IB_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (t->mem && cur != t->device) cudaSetDevice(t->device);
    if (t->mem) cudaFree(t->mem);  // (cudaFree waits for the device's queued work first)
    if (t->staged) {
        cudaEventSynchronize(t->staged);
        cudaEventDestroy(t->staged);
    }
    if (t->stage) cudaFreeHost(t->stage);
    if (t->mem && cur >= 0 && cur != t->device) cudaSetDevice(cur);
    delete t;
    return IB_OK;
}

namespace gbib {

// A device word that nothing ever writes, and a bounded wait on it: the
// self-test of the failure path (ib_selftest_wait_timeout).  The wait has
// the shape of the library's others: poll, give up after a clock64 budget,
// raise IB_ERR_TIMEOUT in the context's status latch, return.
__device__ unsigned int g_never_set = 0u;

__global__ void k_selftest_wait(long long cycles, DevStatus *st) {
    if (threadIdx.x != 0) return;
    const long long t0 = clock64();
    while (*(volatile unsigned int *)&g_never_set == 0u) {
        if (clock64() - t0 > cycles) {
            raise_status(st, IB_ERR_TIMEOUT, -1);
            return;
        }
    }
}

static cudaEvent_t take_event(ib_ctx *c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

PhaseTimer::PhaseTimer(ib_ctx *c, int ph, cudaStream_t st) : ctx(c), phase(ph), s(st) {
    if (!ctx || !ctx->timing) return;
    a = take_event(ctx);
    b = take_event(ctx);
    if (a && b) cudaEventRecord(a, s);
}

void PhaseTimer::stop() {
    if (!ctx) return;
    if (ctx->timing && a && b) {
        cudaEventRecord(b, s);
        ctx->pending[phase].push_back({a, b});
    } else {
        if (a) ctx->pool.push_back(a);
        if (b) ctx->pool.push_back(b);
    }
    ctx = nullptr;
}

}  // namespace gbib

using namespace gbib;

extern "C" {

const char *ib_last_error(void) { return g_last_error; }

size_t ib_workspace_needed(void) { return g_ws_need; }

int ib_ctx_create(ib_ctx **ctx, size_t workspace_bytes) {
    if (!ctx) return set_error(IB_ERR_INVALID, "ctx out-pointer is NULL");
    *ctx = nullptr;
    ib_ctx *c = new ib_ctx();
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return set_error(IB_ERR_CUDA, "no CUDA device");
    }
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (workspace_bytes == 0) workspace_bytes = (size_t)64 << 20;
    c->ws_bytes = workspace_bytes;
    if (cudaMalloc(&c->ws, workspace_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return set_error(IB_ERR_OOM, "workspace of %zu bytes: cudaMalloc failed", workspace_bytes);
    }
    if (cudaMalloc(&c->status, sizeof(DevStatus)) != cudaSuccess ||
        cudaMemset(c->status, 0, sizeof(DevStatus)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->ws);
        delete c;
        return set_error(IB_ERR_CUDA, "status latch allocation failed");
    }
    if (cudaHostAlloc((void **)&c->h_nlev, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->status);
        cudaFree(c->ws);
        delete c;
        return set_error(IB_ERR_CUDA, "context host word allocation failed");
    }
    *c->h_nlev = 0;
    if (cudaStreamCreateWithFlags(&c->fork_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork_ev[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork_ev[2], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork_ev[3], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(c->h_nlev);
        cudaFree(c->status);
        cudaFree(c->ws);
        delete c;
        return set_error(IB_ERR_CUDA, "context stream/event creation failed");
    }
    c->pass_kernels = IB_PASSES_AUTO;
    c->vol_split = 0;  // automatic
    c->spread_mode = IB_SPREAD_GATHER;
    c->gather_ctas = 0;
    c->gather_stage = 0;
    c->field_wait = nullptr;
    for (int k = 0; k < ib_ctx::kStageSlots; ++k) {
        c->stage_ptr[k] = nullptr;
        c->stage_cap[k] = 0;
        c->stage_ev[k] = nullptr;
    }
    c->stage_next = 0;
    *ctx = c;
    return IB_OK;
}

int ib_ctx_reserve(ib_ctx *c, size_t bytes) {
    if (!c) return set_error(IB_ERR_INVALID, "ctx is NULL");
    if (bytes <= c->ws_bytes) return IB_OK;
    if (cudaDeviceSynchronize() != cudaSuccess)
        return set_error(IB_ERR_CUDA, "reserve: %s", cudaGetErrorString(cudaGetLastError()));
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(IB_ERR_OOM, "reserve: cudaMalloc(%zu) failed", bytes);
    }
    cudaFree(c->ws);
    c->ws = p;
    c->ws_bytes = bytes;
    return IB_OK;
}

int ib_ctx_set_timing(ib_ctx *c, int enable) {
    if (!c) return set_error(IB_ERR_INVALID, "ctx is NULL");
    c->timing = enable ? 1 : 0;
    return IB_OK;
}

int ib_ctx_set_pass_kernels(ib_ctx *c, int which) {
    if (!c) return set_error(IB_ERR_INVALID, "ctx is NULL");
    if (which != IB_PASSES_AUTO && which != IB_PASSES_WAVEFRONT && which != IB_PASSES_RESIDENT &&
        which != IB_PASSES_GROUPS)
        return set_error(IB_ERR_INVALID, "bad pass-kernel choice %d", which);
    c->pass_kernels = which;
    return IB_OK;
}

int ib_ctx_set_field_wait(ib_ctx *c, void *event) {
    if (!c) return set_error(IB_ERR_INVALID, "ctx is NULL");
    c->field_wait = event;
    return IB_OK;
}

int ib_selftest_wait_timeout(ib_ctx *c, long long cycles, void *stream) {
    if (!c) return set_error(IB_ERR_INVALID, "ctx is NULL");
    if (cycles < 1 || cycles > 4000000000LL)
        return set_error(IB_ERR_INVALID, "self-test wait of %lld cycles outside [1, 4e9]", cycles);
    k_selftest_wait<<<1, 32, 0, (cudaStream_t)stream>>>(cycles, c->status);
    return check_launch("self-test wait");
}

int ib_ctx_set_spread_mode(ib_ctx *c, int mode) {
    if (!c) return set_error(IB_ERR_INVALID, "ctx is NULL");
    if (mode != IB_SPREAD_GATHER && mode != IB_SPREAD_ATOMIC) return set_error(IB_ERR_INVALID, "spread mode %d", mode);
    c->spread_mode = mode;
    return IB_OK;
}

int ib_ctx_set_gather(ib_ctx *c, int ctas_per_sm, int stage) {
    if (!c) return set_error(IB_ERR_INVALID, "ctx is NULL");
    if (ctas_per_sm < 0 || ctas_per_sm > 32) return set_error(IB_ERR_INVALID, "gather CTAs per SM %d", ctas_per_sm);
    if (stage != 0 && (stage < 32 || stage > 256 || stage % 32))
        return set_error(IB_ERR_INVALID, "gather staging %d: 0 or a multiple of 32 in [32, 256]", stage);
    c->gather_ctas = ctas_per_sm;
    c->gather_stage = stage;
    return IB_OK;
}

int ib_ctx_set_volume_split(ib_ctx *c, int ctas_per_particle) {
    if (!c) return set_error(IB_ERR_INVALID, "ctx is NULL");
    if (ctas_per_particle < 0 || ctas_per_particle > 32)
        return set_error(IB_ERR_INVALID, "volume split %d outside [0, 32]", ctas_per_particle);
    c->vol_split = ctas_per_particle;
    return IB_OK;
}

int ib_ctx_read_timing(ib_ctx *c, int phase, double *ms_total, int *launches) {
    if (!c) return set_error(IB_ERR_INVALID, "ctx is NULL");
    if (phase < 0 || phase >= IB_PHASE_COUNT) return set_error(IB_ERR_INVALID, "bad phase");
    double tot = 0.0;
    int n = 0;
    for (auto &pr : c->pending[phase]) {
        if (cudaEventSynchronize(pr.second) != cudaSuccess)
            return set_error(IB_ERR_CUDA, "timing: %s", cudaGetErrorString(cudaGetLastError()));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, pr.first, pr.second);
        tot += ms;
        ++n;
        c->pool.push_back(pr.first);
        c->pool.push_back(pr.second);
    }
    c->pending[phase].clear();
    if (ms_total) *ms_total = tot;
    if (launches) *launches = n;
    return IB_OK;
}

int ib_ctx_destroy(ib_ctx *c) {
    if (!c) return IB_OK;
    cudaDeviceSynchronize();
    for (auto &v : c->pending)
        for (auto &pr : v) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    for (auto e : c->pool) cudaEventDestroy(e);
    cudaFreeHost(c->h_nlev);
    cudaStreamDestroy(c->fork_stream);
    for (auto e : c->fork_ev) cudaEventDestroy(e);
    for (int k = 0; k < ib_ctx::kStageSlots; ++k) {
        if (c->stage_ptr[k]) cudaFreeHost(c->stage_ptr[k]);
        if (c->stage_ev[k]) cudaEventDestroy(c->stage_ev[k]);
    }
    cudaFree(c->ws);
    cudaFree(c->status);
    delete c;
    return IB_OK;
}

int ib_ctx_status(ib_ctx *c, void *stream) {
    if (!c) return set_error(IB_ERR_INVALID, "ctx is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return set_error(IB_ERR_CUDA, "status: %s", cudaGetErrorString(cudaGetLastError()));
    DevStatus h;
    if (cudaMemcpy(&h, c->status, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_error(IB_ERR_CUDA, "status copy failed");
    if (h.code != 0) {
        cudaMemset(c->status, 0, sizeof(DevStatus));
        const char *what = h.code == IB_ERR_TIMEOUT      ? "a device-side wait gave up"
                           : h.code == IB_ERR_NONFINITE  ? "non-finite particle or marker input"
                           : h.code == IB_ERR_UNSUPPORTED ? "a bin exceeded its capacity"
                                                          : "device error";
        return set_error(h.code, "device status %d (%s), detail %d", h.code, what, h.detail);
    }
    return IB_OK;
}

int ib_ctx_sm_count(const ib_ctx *c) { return c ? c->sm_count : 0; }

}  // extern "C"
