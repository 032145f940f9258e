// Particle-group multidirect forcing: Algorithm 1 of arXiv 2408.14140
// (Sec. 3.1 Step 2) in the sequential particle order, one group of CTAs per
// particle, particles started as soon as the earlier particles they conflict
// with are done.
//
// The wavefront form runs a whole wavefront of non-conflicting particles per
// kernel and pays one kernel boundary per wavefront and pass.  Here a
// persistent cooperative launch is split into groups of kGroupCtas CTAs; a
// group takes particles in level-major rank order from a ticket counter and
// runs all Ns passes of one particle:
//   * interpolation: each CTA takes a contiguous share of the particle's
//     markers (U = J u, F += (U^d - U)/dt, A = (U^d - U) dV / h^3);
//   * a barrier over the group's CTAs;
//   * gather: each CTA takes a contiguous share of the particle's tiles,
//     stages all their candidates at once and adds their per-cell lists (the
//     same sums, in the same order, as the wavefront gather);
//   * a barrier over the group, then the next pass.
// A particle first waits (bounded) until every earlier particle it conflicts
// with has been published by all CTAs of its group.  Every wait is on a lower
// rank, which a running group already holds, and a cooperative launch keeps
// every CTA resident, so neither the waits nor the group barriers can
// deadlock.  All waits are bounded (IB_ERR_TIMEOUT).  Results are bitwise
// those of the wavefront form: every marker and cell does the same
// arithmetic in the same order.
#include "ib_device.cuh"

namespace gbib {

constexpr int kGroupCtas = 16;     // CTAs per particle
constexpr int kGroupThreads = 256;
// candidate records staged per CTA: all of a CTA's tiles at once (its share
// of a D = 24 sphere's tiles holds ~250 candidates, unevenly spread)
template <typename T> struct GroupStage;
template <> struct GroupStage<float> { static constexpr int N = 1024; };
template <> struct GroupStage<double> { static constexpr int N = 512; };
template <typename T>
constexpr size_t group_stage_bytes() {
    return (size_t)GroupStage<T>::N * 16 * sizeof(T);
}

// First of the items [0, n) that member r of C owns (contiguous chunks).
__device__ __forceinline__ int group_chunk(int r, int n, int C) { return (int)((long long)r * n / C); }

// Barrier over the G CTAs of one group: generation counter, bounded wait.
// The writers' fence before arriving and the acquire after the wait order
// every global-memory access of the group across it.
__device__ __forceinline__ bool group_sync(unsigned int *count, unsigned int *gen, unsigned int G, DevStatus *st) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int g0 = ld_acquire(gen);
        __threadfence();
        const unsigned int arrived = atomicAdd(count, 1u);
        int ok = 1;
        if (arrived == G - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const long long t0 = clock64();
            while (ld_acquire(gen) == g0) {
                if (clock64() - t0 > kSpinCycles) {
                    raise_status(st, IB_ERR_TIMEOUT, (int)blockIdx.x);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok;
}

// Waits until every conflicting earlier particle of p is published by all G
// CTAs of the group that ran it.  Thread 0 only; false after a timeout.
template <typename T>
__device__ bool group_wait_deps(const ResidentArgs<T> &a, int p, const DevCase &cd, unsigned int G) {
    const long long t0 = clock64();
    auto wait_one = [&](int q) {
        while (ld_acquire(a.done + q) < G)
            if (clock64() - t0 > kSpinCycles) {
                raise_status(a.st, IB_ERR_TIMEOUT, p);
                return false;
            }
        return true;
    };
    const int c = a.nbr_cnt[p];
    if (c >= 0) {
        for (int k = 0; k < c; ++k)
            if (!wait_one(a.nbr[(size_t)p * kMaxNbr + k])) return false;
    } else {
        // full conflict list: every earlier-level particle of the case (a
        // superset of the conflicts, all of lower rank)
        const int lp = a.level[p];
        for (int q = cd.p0; q < cd.p1; ++q)
            if (a.level[q] < lp && !wait_one(q)) return false;
    }
    return true;
}

template <typename T, int KER>
__global__ void __launch_bounds__(kGroupThreads) k_mdf_groups(ResidentArgs<T> a) {
    constexpr int KW = Kernel<KER>::W;
    constexpr unsigned int G = kGroupCtas;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sw = (T *)smem_raw;                        // [N][12]
    T *sA = sw + (size_t)GroupStage<T>::N * 12;   // [N][4]
    __shared__ int s_t;
    const int grp = blockIdx.x / G, r = blockIdx.x % G;
    unsigned int *gw = a.gwords + 4 * (size_t)grp;  // count, generation, ticket slot
    const double inv_dt = a.inv_dt;
    bool go_on = true;  // thread 0: no dependency wait has timed out
    for (;;) {
        // ---- next particle: the group's first CTA takes a ticket for all
        if (r == 0 && threadIdx.x == 0) atomicExch(gw + 2, atomicAdd(a.ticket, 1u));
        if (!group_sync(gw, gw + 1, G, a.st)) return;
        if (threadIdx.x == 0) s_t = (int)atomicAdd(gw + 2, 0u);
        __syncthreads();
        const int t = s_t;
        if (t >= a.P) return;
        const int p = a.by_rank[t];
        const DevCase cd = a.ct.of_particle(p);
        const DevGrid g = cd.g;
        const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
        const T *const u = (const T *)cd.u;
        if (threadIdx.x == 0 && go_on) go_on = group_wait_deps(a, p, cd, G);
        __syncthreads();
        // this CTA's markers and tiles of the particle
        const int rk = a.rank[p];
        const int c0 = (int)a.sl.flag_scan[(size_t)rk * kLocalSlots];
        const int nt = (int)a.sl.flag_scan[(size_t)(rk + 1) * kLocalSlots] - c0;
        const int k0 = group_chunk(r, nt, G), k1 = group_chunk(r + 1, nt, G);
        const int mb = a.mbase[p], nL = a.moff[p + 1] - a.moff[p];
        const int i0 = mb + group_chunk(r, nL, G), i1 = mb + group_chunk(r + 1, nL, G);
        for (int m = 0; m < a.Ns; ++m) {
            for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                const int l = a.mperm[i];
                T U[3];
                interp_marker<T, KW, true>(u, g, N, a.ms.anchor[l], a.ms.wts + 12 * (size_t)l, U);
                PassMarker<T> pm;
                pm.load(a.ms, a.dV, g.inv_h3, l);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T e = pm.err(c, U[c]);
                    a.F[3 * l + c] = PassMarker<T>::force(a.F[3 * l + c], e, inv_dt);
                    a.ms.A[4 * l + c] = pm.source(e);
                }
            }
            if (!group_sync(gw, gw + 1, G, a.st)) return;
            gather_tiles_lists<T, KW, true, GroupStage<T>::N>(a.ct, c0 + k0, k1 - k0, a.sl, a.ms.wts, a.ms.A,
                                                              inv_dt, sw, sA);
            // the last pass needs no group barrier: the particle is published
            // below, and the next ticket's barrier separates the tasks
            if (m + 1 < a.Ns && !group_sync(gw, gw + 1, G, a.st)) return;
        }
        // ---- publish: this CTA's stores precede its count on the particle
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(a.done + p, 1u);
        }
    }
}

template <typename T, int KER>
static int groups_capacity(ib_ctx *ctx, int *per_sm) {
    const size_t smem = group_stage_bytes<T>();
    void (*kern)(ResidentArgs<T>) = k_mdf_groups<T, KER>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, kGroupThreads, smem);
    if (e != cudaSuccess || *per_sm < 1) {
        *per_sm = 0;
        return set_error(IB_ERR_CUDA, "group kernel cannot be resident: %s", cudaGetErrorString(e));
    }
    return IB_OK;
}

template <typename T, int KER>
int mdf_groups_count(ib_ctx *ctx) {
    int per_sm = 0;
    if (groups_capacity<T, KER>(ctx, &per_sm)) return 0;
    return per_sm * ctx->sm_count / kGroupCtas;
}

template <typename T, int KER>
int launch_mdf_groups(ib_ctx *ctx, const ResidentArgs<T> &a, cudaStream_t s) {
    int per_sm = 0;
    int rc = groups_capacity<T, KER>(ctx, &per_sm);
    if (rc) return rc;
    const int groups_max = per_sm * ctx->sm_count / kGroupCtas;
    if (groups_max < 1) return set_error(IB_ERR_UNSUPPORTED, "device too small for a CTA group");
    const int groups = a.P < groups_max ? a.P : groups_max;
    void *args[] = {(void *)&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_mdf_groups<T, KER>, groups * kGroupCtas,
                                                kGroupThreads, args, group_stage_bytes<T>(), s);
    if (e != cudaSuccess) return set_error(IB_ERR_CUDA, "group kernel launch: %s", cudaGetErrorString(e));
    return IB_OK;
}

#define GBIB_GROUPS_INST(T, K)                                                           \
    template int launch_mdf_groups<T, K>(ib_ctx *, const ResidentArgs<T> &, cudaStream_t); \
    template int mdf_groups_count<T, K>(ib_ctx *);
GBIB_GROUPS_INST(float, IB_DELTA_ROMA3)
GBIB_GROUPS_INST(float, IB_DELTA_PESKIN4)
#undef GBIB_GROUPS_INST

}  // namespace gbib
