// Particle-resident multidirect forcing: Algorithm 1 of arXiv 2408.14140
// (Sec. 3.1 Step 2) in the sequential particle order, one particle per
// thread-block cluster.
//
// In the sequential order a particle runs all of its Ns passes on the field
// left by the particles before it whose stencils share cells with its own.
// Each pass touches only the particle's band, so the cluster keeps the band
// on chip for all passes:
//   * the particle's spreading tiles (8^3 cells of its stencil box) are split
//     over the cluster's CTAs; each CTA holds its tiles' u, their bin tables,
//     and the weights of every marker whose stencil reaches them in shared
//     memory;
//   * interpolation reads u through distributed shared memory (the taps of a
//     marker can fall in tiles of other CTAs); every CTA interpolates every
//     marker of its tiles' candidate lists, so the spread sources it gathers
//     are its own and nothing is exchanged through global memory; the marker
//     force F is accumulated by the one CTA that holds the marker's first
//     stencil cell;
//   * the gather adds each cell's sum in the tile's fixed (row, x offset,
//     marker) order, so every result is bitwise that of the wavefront
//     kernels;
//   * u leaves the chip once, after the last pass: only band cells are
//     stored, since cells of the tiles outside the band may belong to another
//     particle running at the same time.
// Particles are taken in level-major rank order from a ticket counter; a
// particle waits (bounded) until every earlier particle it conflicts with
// has been stored.  Any wait is on a lower rank, which a running cluster
// already holds, so the schedule cannot deadlock.  A particle whose tiles or
// candidates exceed the shared-memory capacity runs the same passes with u
// and the spread sources in global memory (slow path).
#include <cooperative_groups.h>

#include "ib_device.cuh"

namespace gbib {

namespace cg = cooperative_groups;

// Per-CTA capacity: resident tiles and staged candidate records.
template <typename T> struct Res;
template <> struct Res<float> { static constexpr int TM = 8, REC = 2048; };
template <> struct Res<double> { static constexpr int TM = 8, REC = 736; };
constexpr int kCluster = 8;      // CTAs per particle (portable cluster size)
constexpr int kMaxCluster = 16;

template <typename T>
constexpr size_t res_smem_bytes() {
    return (size_t)Res<T>::TM * 3 * kTileCells * sizeof(T) +  // u of the tiles
           (size_t)Res<T>::REC * 16 * sizeof(T) +             // weights [12] + source [4]
           (size_t)Res<T>::REC * 8 +                          // marker id, packed anchor
           (size_t)Res<T>::TM * kBins * 2;                    // bin tables
}

template <typename T>
struct ResSmem {
    T *u;            // [TM][3][512]
    T *w;            // [REC][12]
    T *A;            // [REC][4]
    int *id;         // [REC] marker of each record
    unsigned *anc;   // [REC] anchor relative to the box: x | y << 6 | z << 12 | primary << 18
    uint16_t *bins;  // [TM][kBins]
    __device__ explicit ResSmem(unsigned char *base) {
        u = (T *)base;
        w = u + (size_t)Res<T>::TM * 3 * kTileCells;
        A = w + (size_t)Res<T>::REC * 12;
        id = (int *)(A + (size_t)Res<T>::REC * 4);
        anc = (unsigned *)(id + Res<T>::REC);
        bins = (uint16_t *)(anc + Res<T>::REC);
    }
};

// First of the tiles [0, nt) that CTA r of C owns (contiguous chunks).
__device__ __forceinline__ int chunk_begin(int r, int nt, int C) { return (int)((long long)r * nt / C); }

// Barrier over the cluster that also orders global-memory traffic between
// its CTAs (slow path): the writers' fence, then an acquire on this SM
// before the loads that follow.
__device__ __forceinline__ void cluster_gpu_sync(cg::cluster_group &cl, const unsigned int *word) {
    __syncthreads();
    if (threadIdx.x == 0) __threadfence();
    cl.sync();
    if (threadIdx.x == 0) (void)ld_acquire(word);
    __syncthreads();
}

// Waits until every conflicting earlier particle of p has been stored.
// Thread 0 only; returns false after a timeout (status raised).
template <typename T>
__device__ bool wait_dependencies(const ResidentArgs<T> &a, int p, const DevCase &cd, unsigned C) {
    const long long t0 = clock64();
    auto wait_one = [&](int q) {
        while (ld_acquire(a.done + q) < C)
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
__global__ void __launch_bounds__(kBlock, 1) k_mdf_resident(ResidentArgs<T> a) {
    constexpr int KW = Kernel<KER>::W;
    constexpr int TM = Res<T>::TM, REC = Res<T>::REC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ResSmem<T> sm(smem_raw);
    __shared__ int s_map[kLocalSlots];  // local tile -> owner << 4 | slot; -1: not a tile of the particle
    __shared__ int4 s_lo[TM], s_dim[TM];
    __shared__ int s_off[TM + 1];
    __shared__ int s_ticket, s_fits;
    __shared__ const T *s_ru[kMaxCluster];  // every CTA's resident u, as seen from here
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int r = (int)cl.block_rank();
    const int tid = threadIdx.x;
    const int tx = tid & 7, ty = (tid >> 3) & 7, tz = tid >> 6;
    if (tid < C) s_ru[tid] = cl.map_shared_rank(sm.u, tid);
    const double inv_dt = a.inv_dt;
    bool go_on = true;  // thread 0: no wait has timed out
    for (;;) {
        // ---- next particle: rank 0 takes a ticket, every CTA reads it
        if (r == 0 && tid == 0) s_ticket = (int)atomicAdd(a.ticket, 1u);
        cl.sync();
        const int t = *cl.map_shared_rank(&s_ticket, 0);
        cl.sync();
        if (t >= a.P) break;
        const int p = a.by_rank[t];
        const DevCase cd = a.ct.of_particle(p);
        const DevGrid g = cd.g;
        const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
        T *const u = (T *)cd.u;
        T *const f_out = (T *)cd.f;
        if (tid == 0 && go_on) go_on = wait_dependencies(a, p, cd, (unsigned)C);
        // ---- the particle's tiles and this CTA's share
        const int rk = a.rank[p];
        const int c0 = (int)a.sl.flag_scan[(size_t)rk * kLocalSlots];
        const int nt = (int)a.sl.flag_scan[(size_t)(rk + 1) * kLocalSlots] - c0;
        const int k0 = chunk_begin(r, nt, C), nmine = chunk_begin(r + 1, nt, C) - k0;
        const int4 blo = a.box_lo[p];
        const int bx = wrap_int(blo.x, g.n[0]), by = wrap_int(blo.y, g.n[1]), bz = wrap_int(blo.z, g.n[2]);
        for (int k = tid; k < kLocalSlots; k += blockDim.x) s_map[k] = -1;
        if (tid == 0) {
            int tot = 0;
            const int nres = nmine < TM ? nmine : TM;
            for (int s = 0; s < nres; ++s) {
                const int cs = c0 + k0 + s;
                s_off[s] = tot;
                s_lo[s] = a.sl.geo_lo[cs];
                s_dim[s] = a.sl.geo_dim[cs];
                tot += a.sl.bins[(size_t)cs * kBins + kBins - 1];
            }
            s_off[nres] = tot;
            s_fits = nmine <= TM && tot <= REC;
        }
        __syncthreads();
        for (int k = tid; k < nt; k += blockDim.x) {
            const int lt = (int)a.sl.dense_of[c0 + k] - rk * kLocalSlots;
            int o = C - 1;
            while (chunk_begin(o, nt, C) > k) --o;
            s_map[lt] = (o << 4) | (k - chunk_begin(o, nt, C));
        }
        cl.sync();  // every CTA's capacity decision is set
        bool fast = true;
        for (int q = 0; q < C; ++q) fast = fast && *cl.map_shared_rank(&s_fits, q);

        if (fast) {
            // ---- stage u, bin tables and candidate records of the owned tiles
            for (int s = 0; s < nmine; ++s) {
                const int cs = c0 + k0 + s;
                const int4 lo = s_lo[s], dim = s_dim[s];
                if (tx < dim.x && ty < dim.y && tz < dim.z) {
                    const long long c = ((long long)wrap_add(lo.z, tz, g.n[2]) * g.n[1] +
                                         wrap_add(lo.y, ty, g.n[1])) * g.n[0] + wrap_add(lo.x, tx, g.n[0]);
#pragma unroll
                    for (int q = 0; q < 3; ++q) sm.u[(s * 3 + q) * kTileCells + tid] = u[q * N + c];
                }
                const uint16_t *bs = a.sl.bins + (size_t)cs * kBins;
                for (int i = tid; i < kBins; i += blockDim.x) sm.bins[s * kBins + i] = bs[i];
                const int lt = (int)a.sl.dense_of[cs] - rk * kLocalSlots;
                const int lx = lt & 7, ly = (lt >> 3) & 7, lz = lt >> 6;
                const int off = s_off[s], nc = s_off[s + 1] - off;
                const uint32_t *cand = a.sl.cand + dim.w;
                for (int i = tid; i < nc; i += blockDim.x) {
                    const int m = (int)cand[i];
                    sm.id[off + i] = m;
                    const T *wm = a.ms.wts + 12 * (size_t)m;
#pragma unroll
                    for (int q = 0; q < 3; ++q)
#pragma unroll
                        for (int j = 0; j < KW; ++j) sm.w[12 * (off + i) + 4 * q + j] = __ldg(wm + 4 * q + j);
                    const uint64_t an = a.ms.anchor[m];
                    const int rx = wrap_diff(anchor_x(an), bx, g.n[0]);
                    const int ry = wrap_diff(anchor_y(an), by, g.n[1]);
                    const int rz = wrap_diff(anchor_z(an), bz, g.n[2]);
                    const unsigned prim = (rx >> 3) == lx && (ry >> 3) == ly && (rz >> 3) == lz;
                    sm.anc[off + i] = (unsigned)rx | ((unsigned)ry << 6) | ((unsigned)rz << 12) | (prim << 18);
                }
            }
            cl.sync();  // staged u of every CTA is visible before the first interpolation
            const int ncand = s_off[nmine];
            unsigned hit = 0;
            for (int m = 0; m < a.Ns; ++m) {
                // interpolation of every candidate record: U = J u over the cluster's tiles
                for (int i = tid; i < ncand; i += blockDim.x) {
                    const unsigned pk = sm.anc[i];
                    const int rx = pk & 63, ry = (pk >> 6) & 63, rz = (pk >> 12) & 63;
                    const T *w = sm.w + 12 * i;
                    T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll 1
                    for (int kz = 0; kz < KW; ++kz) {
                        const int z = rz + kz;
#pragma unroll
                        for (int ky = 0; ky < KW; ++ky) {
                            const int y = ry + ky;
                            const int row = ((z >> 3) * kLocalTiles + (y >> 3)) * kLocalTiles;
                            const int crow = ((z & 7) * kTile + (y & 7)) * kTile;
                            const T wyz = w[8 + kz] * w[4 + ky];
#pragma unroll
                            for (int kx = 0; kx < KW; ++kx) {
                                const int x = rx + kx;
                                // every tap lies in a tile of the particle (the marker is a
                                // candidate of each tile its stencil touches); map >= 0
                                const int e = max(s_map[row + (x >> 3)], 0);
                                const T *src = s_ru[e >> 4] + (size_t)(e & 15) * 3 * kTileCells + crow + (x & 7);
                                const T wt = wyz * w[kx];
                                a0 += wt * src[0];
                                a1 += wt * src[kTileCells];
                                a2 += wt * src[2 * kTileCells];
                            }
                        }
                    }
                    const T U[3] = {a0, a1, a2};
                    const int l = sm.id[i];
                    PassMarker<T> pm;
                    pm.load(a.ms, a.dV, g.inv_h3, l);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const T e = pm.err(c, U[c]);
                        if (pk >> 18) a.F[3 * l + c] = PassMarker<T>::force(a.F[3 * l + c], e, inv_dt);
                        sm.A[4 * i + c] = pm.source(e);
                    }
                }
                cl.sync();  // all reads of u done before any tile is updated
                // gather into the owned tiles
#pragma unroll 1
                for (int s = 0; s < nmine; ++s) {
                    const int4 dim = s_dim[s];
                    const int off = s_off[s];
                    T acc[3];
                    if (tx < dim.x && ty < dim.y && tz < dim.z &&
                        gather_cell<T, KW, true, true>(tx, ty, tz, sm.bins + s * kBins, nullptr,
                                                       sm.w + 12 * (size_t)off, sm.A + 4 * (size_t)off, acc)) {
                        hit |= 1u << s;
#pragma unroll
                        for (int q = 0; q < 3; ++q) sm.u[(s * 3 + q) * kTileCells + tid] += acc[q];
                        if (f_out) {
                            const int4 lo = s_lo[s];
                            const long long c = ((long long)wrap_add(lo.z, tz, g.n[2]) * g.n[1] +
                                                 wrap_add(lo.y, ty, g.n[1])) * g.n[0] + wrap_add(lo.x, tx, g.n[0]);
#pragma unroll
                            for (int q = 0; q < 3; ++q) f_out[q * N + c] += (T)(acc[q] * inv_dt);
                        }
                    }
                }
                cl.sync();  // updated tiles visible to the next interpolation
            }
            // ---- store the band cells
            for (int s = 0; s < nmine; ++s)
                if ((hit >> s) & 1u) {
                    const int4 lo = s_lo[s];
                    const long long c = ((long long)wrap_add(lo.z, tz, g.n[2]) * g.n[1] +
                                         wrap_add(lo.y, ty, g.n[1])) * g.n[0] + wrap_add(lo.x, tx, g.n[0]);
#pragma unroll
                    for (int q = 0; q < 3; ++q) u[q * N + c] = sm.u[(s * 3 + q) * kTileCells + tid];
                }
        } else {
            // ---- slow path: the same passes through global memory
            const int mb = a.mbase[p], nL = a.moff[p + 1] - a.moff[p];
            const int ch = (nL + C - 1) / C;
            const int i0 = mb + r * ch, i1 = mb + min(nL, (r + 1) * ch);
            for (int m = 0; m < a.Ns; ++m) {
                for (int i = i0 + tid; i < i1; i += blockDim.x) {
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
                cluster_gpu_sync(cl, a.ticket);
#pragma unroll 1
                for (int k = k0; k < k0 + nmine; ++k) {
                    const int cs = c0 + k;
                    const int4 lo = a.sl.geo_lo[cs], dim = a.sl.geo_dim[cs];
                    T acc[3];
                    if (tx < dim.x && ty < dim.y && tz < dim.z &&
                        gather_cell<T, KW, false, true>(tx, ty, tz, a.sl.bins + (size_t)cs * kBins,
                                                        a.sl.cand + dim.w, a.ms.wts, a.ms.A, acc)) {
                        const long long c = ((long long)wrap_add(lo.z, tz, g.n[2]) * g.n[1] +
                                             wrap_add(lo.y, ty, g.n[1])) * g.n[0] + wrap_add(lo.x, tx, g.n[0]);
#pragma unroll
                        for (int q = 0; q < 3; ++q) u[q * N + c] += acc[q];
                        if (f_out)
#pragma unroll
                            for (int q = 0; q < 3; ++q) f_out[q * N + c] += (T)(acc[q] * inv_dt);
                    }
                }
                cluster_gpu_sync(cl, a.ticket);
            }
        }
        // ---- publish: this CTA's stores precede its count on the particle
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(a.done + p, 1u);
        }
    }
}

template <typename T, int KER>
int launch_mdf_resident(ib_ctx *ctx, const ResidentArgs<T> &a, cudaStream_t s) {
    const size_t smem = res_smem_bytes<T>();
    void (*kern)(ResidentArgs<T>) = k_mdf_resident<T, KER>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(IB_ERR_CUDA, "resident kernel attribute: %s", cudaGetErrorString(e));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(kCluster);
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, (const void *)kern, &cfg);
    if (e != cudaSuccess || ncl < 1)
        return set_error(IB_ERR_CUDA, "resident kernel cannot be resident: %s", cudaGetErrorString(e));
    const int nclusters = a.P < ncl ? a.P : ncl;
    cfg.gridDim = dim3(nclusters * kCluster);
    e = cudaLaunchKernelEx(&cfg, kern, a);
    if (e != cudaSuccess) return set_error(IB_ERR_CUDA, "resident kernel launch: %s", cudaGetErrorString(e));
    return IB_OK;
}

template int launch_mdf_resident<float, IB_DELTA_ROMA3>(ib_ctx *, const ResidentArgs<float> &, cudaStream_t);
template int launch_mdf_resident<float, IB_DELTA_PESKIN4>(ib_ctx *, const ResidentArgs<float> &, cudaStream_t);

}  // namespace gbib
