// Velocity interpolation, force spreading and Algorithm 1 (multidirect
// forcing) of arXiv 2408.14140, Sec. 3.1 Step 2.
//
// Data path on the device
// -----------------------
//  1. Marker preparation: position X_l = X_r + R_l, desired velocity
//     U^d_l = U_r + W_r x R_l (Eq. pr1), the first stencil cell ("anchor",
//     wrapped) and the per-axis kernel weights, computed once per call.
//  2. Binning: every marker is listed in each spreading tile (8^3 cells) its
//     stencil touches.  Tiles are global grid tiles (simultaneous order and
//     ib_spread) or tiles of each particle's own bounding box (sequential
//     order).  Each tile's list is sorted by (anchor row, marker index) once,
//     which fixes the summation order of every cell: spreading is a
//     deterministic gather over marker bins, with no floating-point atomics.
//  3. Passes: one persistent cooperative kernel runs, per wavefront of
//     non-conflicting particles and per forcing pass m, an interpolation
//     phase over markers (U, F += (U^d - U)/dt) and a gather phase over tiles
//     (u += S (U^d - U) dV / h^3, the increment of Algorithm 1's correction),
//     separated by grid-wide barriers with bounded waits.
//
// The correction is applied incrementally, u(m) = u(m-1) + dt S(F^m - F^{m-1}),
// which equals the paper's u(m) = u(0) + dt S F^m in exact arithmetic and
// needs no copy of u(0).
#include <float.h>

#include "ib_device.cuh"

namespace gbib {

// A marker's wrapped anchor and its per-axis weights in the pass storage
// form (FP32, or double-float pairs for FP64 fields).
template <typename T, int KER>
__device__ __forceinline__ uint64_t marker_weights(const DevGrid &g, const double X[3],
                                                   PS<T> w[12], long long first[3]) {
    int a[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double s = (X[d] - g.org[d]) * g.inv_h - 0.5;
        first[d] = axis_weights<KER>(s, w + 4 * d);
        a[d] = wrap_int(first[d], g.n[d]);
    }
    return pack_anchor(a[0], a[1], a[2]);
}

// ---------------------------------------------------------------------------
// ib_interpolate
// ---------------------------------------------------------------------------
template <typename T, int KER>
__global__ void __launch_bounds__(256) k_interpolate(DevGrid g, const T *__restrict__ u, int M,
                                                     const double *__restrict__ X,
                                                     double *__restrict__ U, DevStatus *st) {
    constexpr int KW = Kernel<KER>::W;
    long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < M; l += gridDim.x * blockDim.x) {
        double x[3] = {X[3 * l], X[3 * l + 1], X[3 * l + 2]};
        if (!finite3(x)) {
            raise_status(st, IB_ERR_NONFINITE, l);
            U[3 * l] = U[3 * l + 1] = U[3 * l + 2] = 0.0;
            continue;
        }
        PS<T> ws[12];
        long long first[3];
        uint64_t anc = marker_weights<T, KER>(g, x, ws, first);
        T o[3];
        interp_marker<T, KW>(u, g, N, anc, ws, o);
        U[3 * l] = (double)o[0];
        U[3 * l + 1] = (double)o[1];
        U[3 * l + 2] = (double)o[2];
    }
}

// ---------------------------------------------------------------------------
// marker preparation
// ---------------------------------------------------------------------------
// Standalone spreading: positions X given, source A = F dV / h^3.
template <typename T, int KER>
__global__ void k_prep_spread(DevGrid g, int M, const double *__restrict__ X,
                              const double *__restrict__ F, const double *__restrict__ dV,
                              MarkerState<T> ms, DevStatus *st) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < M; l += gridDim.x * blockDim.x) {
        double x[3] = {X[3 * l], X[3 * l + 1], X[3 * l + 2]};
        double f[3] = {F[3 * l], F[3 * l + 1], F[3 * l + 2]};
        double dv = dV[l];
        bool ok = finite3(x) && finite3(f) && isfinite(dv);
        if (!ok) {
            raise_status(st, IB_ERR_NONFINITE, l);
            x[0] = g.org[0];
            x[1] = g.org[1];
            x[2] = g.org[2];
            f[0] = f[1] = f[2] = 0.0;
            dv = 0.0;
        }
        PS<T> w[12];
        long long first[3];
        ms.anchor[l] = marker_weights<T, KER>(g, x, w, first);
#pragma unroll
        for (int k = 0; k < 12; ++k) ms.wts[12 * l + k] = w[k];
        double q = dv * g.inv_h3;
        ms.A[4 * l + 0] = to_store((T)(f[0] * q));
        ms.A[4 * l + 1] = to_store((T)(f[1] * q));
        ms.A[4 * l + 2] = to_store((T)(f[2] * q));
        ms.A[4 * l + 3] = to_store(T(0));
    }
}

// The marker radius of each particle, rho_p = max_l |R_l| (one CTA per
// particle; a marker with a non-finite input, or any marker of a particle
// with a non-finite state, counts as R_l = 0, as in the marker preparation,
// which reports it).  It reads only the call's inputs, so the conflict lists
// and the wavefront levels, which need rho, run on the context's second
// stream beside the marker preparation.  rho only widens the FP32 conflict
// test (whose margin is h/16), so it is formed in FP32 from the components'
// leading 24 bits (split on the integer pipe, each at most |R_l|) and then
// enlarged by a relative 2^-18, which keeps it an upper bound of max |R_l|
// above the FP32 roundings; no FP64 operation runs per marker.
constexpr int kRadiusThreads = 1024;  // a particle's ~2k markers: two loads in flight per thread
__global__ void __launch_bounds__(kRadiusThreads) k_marker_radius(int P, const double *__restrict__ Xr,
                                                       const double *__restrict__ Ur,
                                                       const double *__restrict__ Wr,
                                                       const int *__restrict__ moff, const double *__restrict__ R,
                                                       const double *__restrict__ dV, double *__restrict__ rho) {
    __shared__ float s_max[kRadiusThreads / 32];
    const int p = blockIdx.x;
    if (p >= P) return;
    const bool pok = finite3(Xr + 3 * p) && finite3(Ur + 3 * p) && finite3(Wr + 3 * p);
    float rmax = 0.0f;  // squared; the root is taken once below
    const int m1 = moff[p + 1];
#pragma unroll 4
    for (int l = moff[p] + threadIdx.x; l < m1; l += blockDim.x) {
        const double r[3] = {R[3 * l], R[3 * l + 1], R[3 * l + 2]};
        if (pok && finite3(r) && finite_bits(dV[l])) {
            const float x = df_split(r[0]).x, y = df_split(r[1]).x, z = df_split(r[2]).x;
            rmax = fmaxf(rmax, fmaf(z, z, fmaf(y, y, x * x)));
        }
    }
    for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = rmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) rmax = fmaxf(rmax, s_max[w]);
        rho[p] = (double)sqrtf(rmax) * (1.0 + 0x1p-18);
    }
}

// Per particle (kPrepSplit CTAs): marker positions, desired velocities,
// anchors, weights, and the particle's unwrapped stencil box.  Scratch of the
// cross-CTA reductions: per particle the stencil box bounds (lo starts at a
// huge value, hi at a very negative one: memset 0x7f / 0x80 bytes) and a
// completion count (0).
struct PrepScratch {
    long long *lo, *hi;          // [P][3]
    unsigned int *done;          // [P]
};
constexpr int kPrepSplit = 4;    // CTAs per particle

template <typename T, int KER>
__global__ void __launch_bounds__(256) k_prep_particles(
    CaseTab ct, int P, const double *__restrict__ Xr, const double *__restrict__ Ur,
    const double *__restrict__ Wr, const int *__restrict__ moff, const double *__restrict__ R,
    const double *__restrict__ dV, MarkerState<T> ms, double *__restrict__ F,
    int4 *__restrict__ box_lo, int4 *__restrict__ box_dim,
    int *__restrict__ part_of, PrepScratch ps, DevStatus *st) {
    constexpr int KW = Kernel<KER>::W;
    __shared__ long long s_lo[3], s_hi[3];
    __shared__ int s_last;
    const int p = blockIdx.x / kPrepSplit, part = blockIdx.x % kPrepSplit;
    if (p >= P) return;
    const DevGrid g = ct.of_particle(p).g;
    if (threadIdx.x < 3) {
        s_lo[threadIdx.x] = LLONG_MAX;
        s_hi[threadIdx.x] = LLONG_MIN;
    }
    __syncthreads();
    double xc[3] = {Xr[3 * p], Xr[3 * p + 1], Xr[3 * p + 2]};
    double uc[3] = {Ur[3 * p], Ur[3 * p + 1], Ur[3 * p + 2]};
    double wc[3] = {Wr[3 * p], Wr[3 * p + 1], Wr[3 * p + 2]};
    bool pok = finite3(xc) && finite3(uc) && finite3(wc);
    if (!pok && threadIdx.x == 0 && part == 0) raise_status(st, IB_ERR_NONFINITE, p);
    const int m0 = moff[p], m1 = moff[p + 1];
    const int nm = m1 - m0;
    const int l0 = m0 + (int)((long long)part * nm / kPrepSplit), l1 = m0 + (int)((long long)(part + 1) * nm / kPrepSplit);
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    for (int l = l0 + threadIdx.x; l < l1; l += blockDim.x) {
        double r[3] = {R[3 * l], R[3 * l + 1], R[3 * l + 2]};
        double dv = dV[l];
        if (!pok || !finite3(r) || !finite_bits(dv)) {
            raise_status(st, IB_ERR_NONFINITE, l);
            r[0] = r[1] = r[2] = 0.0;
        }
        double x[3] = {xc[0] + r[0], xc[1] + r[1], xc[2] + r[2]};
        if (!pok) x[0] = g.org[0], x[1] = g.org[1], x[2] = g.org[2];
        PS<T> w[12];
        long long first[3];
        ms.anchor[l] = marker_weights<T, KER>(g, x, w, first);
#pragma unroll
        for (int k = 0; k < 12; ++k) ms.wts[12 * l + k] = w[k];
        const double ud[3] = {uc[0] + (wc[1] * r[2] - wc[2] * r[1]), uc[1] + (wc[2] * r[0] - wc[0] * r[2]),
                              uc[2] + (wc[0] * r[1] - wc[1] * r[0])};
#pragma unroll
        for (int c = 0; c < 3; ++c) ms.Ud[3 * l + c] = ud[c];
        if (sizeof(T) == 4) {
            float4 h, o;
            h.x = (float)ud[0], h.y = (float)ud[1], h.z = (float)ud[2];
            h.w = (float)(dv * g.inv_h3);
            o.x = (float)(ud[0] - (double)h.x), o.y = (float)(ud[1] - (double)h.y);
            o.z = (float)(ud[2] - (double)h.z), o.w = 0.f;
            ((float4 *)(ms.Ud32 + 8 * (size_t)l))[0] = h;
            ((float4 *)(ms.Ud32 + 8 * (size_t)l))[1] = o;
        }
        F[3 * l] = F[3 * l + 1] = F[3 * l + 2] = 0.0;
        part_of[l] = p;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            lo[d] = min(lo[d], first[d]);
            hi[d] = max(hi[d], first[d] + KW - 1);
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        atomicMin(&s_lo[d], lo[d]);
        atomicMax(&s_hi[d], hi[d]);
    }
    __syncthreads();
    // combine the particle's CTAs; the last one to finish writes the results
    if (threadIdx.x == 0) {
        for (int d = 0; d < 3; ++d) {
            atomicMin(&ps.lo[3 * p + d], s_lo[d]);
            atomicMax(&ps.hi[3 * p + d], s_hi[d]);
        }
        __threadfence();
        s_last = atomicAdd(&ps.done[p], 1u) == kPrepSplit - 1;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_last) {
        long long blo[3], bhi[3];
        for (int d = 0; d < 3; ++d) {
            blo[d] = atomicAdd((unsigned long long *)&ps.lo[3 * p + d], 0ull);
            bhi[d] = atomicAdd((unsigned long long *)&ps.hi[3 * p + d], 0ull);
        }
        if (m1 > m0) {
            int dims[3];
            for (int d = 0; d < 3; ++d) dims[d] = (int)(bhi[d] - blo[d] + 1);
            box_lo[p] = make_int4(wrap_int(blo[0], g.n[0]), wrap_int(blo[1], g.n[1]), wrap_int(blo[2], g.n[2]), 0);
            box_dim[p] = make_int4(dims[0], dims[1], dims[2], 0);
            for (int d = 0; d < 3; ++d)
                if (dims[d] > kMaxBox || dims[d] > g.n[d]) raise_status(st, IB_ERR_UNSUPPORTED, p);
        } else {
            box_lo[p] = make_int4(0, 0, 0, 0);
            box_dim[p] = make_int4(0, 0, 0, 0);
        }
    }
}

// ---------------------------------------------------------------------------
// wavefront levels (sequential order).  One CTA.
// Particles p and q conflict when their marker stencils may share a cell:
// nearest-image centre distance < rho_p + rho_q + sqrt(3) * W * h.  level(p)
// = 1 + max level(q) over conflicting q < p; a level's particles have
// pairwise disjoint stencil supports, so running a level at once equals
// running its particles one after another.
// ---------------------------------------------------------------------------
struct LevelOut {
    int *level;       // [P]
    int *rank;        // [P] position of p in level-major order
    int *mbase;       // [P] first slot of p's markers in the level-major marker list
    int *lev_pbeg;    // [P+1] first level-major rank of each level
    int *lev_mbeg;    // [P+1] first level-major marker of each level
    int *nlev;        // [1]
};


// Conflict lists: for every p, the q < p whose stencils may share a cell
// (count -1 = more than kMaxNbr, scanned again when levels are assigned).
// The test runs in FP32 against a limit widened by h/16, far above FP32
// rounding of unit-scale positions, so no true conflict is ever missed (an
// extra conflict only serialises two particles).
__global__ void k_conflicts(CaseTab ct, int P, int KW, const double *__restrict__ Xr,
                            const double *__restrict__ rho, int *__restrict__ nbr_cnt,
                            int *__restrict__ nbr) {
    grid_dep_wait();
    // one warp per particle p; lanes test q = p0 + lane, p0 + 32 + lane, ...
    // and the hits are appended in ascending q (ballot order)
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < P; p += nw) {
        const DevCase cd = ct.of_particle(p);
        const DevGrid &g = cd.g;
        const float L[3] = {(float)(g.n[0] * g.h), (float)(g.n[1] * g.h), (float)(g.n[2] * g.h)};
        const float iL[3] = {1.0f / L[0], 1.0f / L[1], 1.0f / L[2]};
        const float halo = (float)(1.7320508075688772 * KW * g.h + 0.0625 * g.h);
        const float xp[3] = {(float)Xr[3 * p], (float)Xr[3 * p + 1], (float)Xr[3 * p + 2]};
        const float rp = (float)rho[p] + halo;
        int cnt = 0;
        for (int q0 = cd.p0; q0 < p; q0 += 32) {  // particles of other cases never conflict
            const int q = q0 + lane;
            bool hit = false;
            if (q < p) {
                float d2 = 0.0f;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float d = (float)Xr[3 * q + a] - xp[a];
                    d -= L[a] * rintf(d * iL[a]);
                    d2 += d * d;
                }
                const float lim = rp + (float)rho[q];
                hit = d2 < lim * lim;
            }
            const unsigned b = __ballot_sync(0xffffffffu, hit);
            const int pos = cnt + __popc(b & ((1u << lane) - 1u));
            if (hit && pos < kMaxNbr) nbr[(size_t)p * kMaxNbr + pos] = q;
            cnt += __popc(b);
        }
        if (lane == 0) nbr_cnt[p] = cnt <= kMaxNbr ? cnt : -1;
    }
}

// Levels by a sweep over each case's particles in index order (level(p)
// needs only the q < p of its own case; cases are independent and swept in
// parallel, one thread each), then a parallel counting sort of the particles
// by level and the level-major marker offsets.  The sweep's dependent reads
// stay on chip: levels in shared memory (up to kLevOnchipP particles) and the
// conflict lists too when they fit (kLevNbrP).  The order of particles inside
// a level is the order their atomic increments land in; it does not affect
// any result (a level's particles have disjoint stencil supports).
constexpr int kLevOnchipP = 8192;
constexpr int kLevNbrP = 1024;
constexpr size_t kLevSmem = (size_t)kLevOnchipP * 4 + (size_t)kLevNbrP * (2 + 2 * kMaxNbr);

// Exclusive scan of f(0..n-1) by one CTA (chunks of blockDim.x), calling
// out(i, prefix) for every i and returning the total (all threads).
template <typename F, typename O>
__device__ __forceinline__ int block_scan_chunked(int n, F f, O out) {
    __shared__ int s_w[32];
    __shared__ int s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < n ? f(i) : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        int wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += s_w[w];
        const int carry = s_carry;
        if (i < n) out(i, carry + wpre + x - v);
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < nw; ++w) t += s_w[w];
            s_carry = carry + t;
        }
        __syncthreads();
    }
    return s_carry;
}

constexpr int kLevSweeps = 64;  // parallel relaxation sweeps before the ordered sweep
// threads of the one k_levels CTA: 512 (24k registers) fit on an SM beside a
// marker-preparation CTA, so the levels need not wait for that kernel's tail
constexpr int kLevThreads = 512;

__global__ void __launch_bounds__(kLevThreads) k_levels(CaseTab ct, int P, int order, int KW,
                                                 const double *__restrict__ Xr,
                                                 const double *__restrict__ rho,
                                                 const int *__restrict__ moff,
                                                 const int *__restrict__ nbr_cnt,
                                                 const int *__restrict__ nbr, LevelOut lo,
                                                 int *__restrict__ by_rank, int *__restrict__ lev_cur) {
    grid_dep_wait();
    extern __shared__ __align__(16) unsigned char lsm[];
    __shared__ int s_nl;
    const bool lev_on = P <= kLevOnchipP;
    const bool nbr_on = P <= kLevNbrP && order == IB_ORDER_SEQUENTIAL;
    int *lev = lev_on ? (int *)lsm : lo.level;
    short *s_cnt = (short *)(lsm + (size_t)kLevOnchipP * 4);
    unsigned short *s_nbr = (unsigned short *)(s_cnt + kLevNbrP);
    if (threadIdx.x == 0) s_nl = 0;
    for (int i = threadIdx.x; i <= P; i += blockDim.x) {
        lo.lev_pbeg[i] = 0;
        lev_cur[i] = 0;
    }
    if (nbr_on)
        for (int p = threadIdx.x; p < P; p += blockDim.x) {
            const int c = nbr_cnt[p];
            s_cnt[p] = (short)c;
            for (int k = 0; k < c; ++k) s_nbr[p * kMaxNbr + k] = (unsigned short)nbr[(size_t)p * kMaxNbr + k];
        }
    __threadfence();  // the zeroed counters reach L2 before the atomics below
    __syncthreads();
    int mymax = 0;
    // ---- parallel levels: lev(p) = 1 + max lev(q) over conflicting q < p (0
    // without), the longest path to p in the conflict DAG, relaxed for all
    // particles at once until nothing changes.  Values only grow and never
    // pass the fixed point, so reading a neighbour's value mid-sweep is
    // harmless; a conflict chain of length c takes c + 1 sweeps.  Full
    // conflict lists, or chains longer than kLevSweeps, fall back to the
    // sweep in particle order below (which recomputes every level).
    __shared__ int s_flag;
    bool levels_done = false;
    if (order == IB_ORDER_SEQUENTIAL) {
        volatile int *vlev = lev;
        if (threadIdx.x == 0) s_flag = 0;
        __syncthreads();
        for (int p = threadIdx.x; p < P; p += blockDim.x) {
            if ((nbr_on ? s_cnt[p] : nbr_cnt[p]) < 0) s_flag = 1;
            vlev[p] = 0;
        }
        __syncthreads();
        const bool any_full = s_flag != 0;
        __syncthreads();
        for (int it = 0; !any_full && it < kLevSweeps; ++it) {
            if (threadIdx.x == 0) s_flag = 0;
            __syncthreads();
            for (int p = threadIdx.x; p < P; p += blockDim.x) {
                const int cn = nbr_on ? s_cnt[p] : nbr_cnt[p];
                int best = 0;
                for (int k = 0; k < cn; ++k)
                    best = max(best, vlev[nbr_on ? s_nbr[p * kMaxNbr + k] : nbr[(size_t)p * kMaxNbr + k]] + 1);
                if (best != vlev[p]) {
                    vlev[p] = best;
                    s_flag = 1;
                }
            }
            __syncthreads();
            const bool changed = s_flag != 0;
            __syncthreads();
            if (!changed) {
                levels_done = true;
                break;
            }
        }
        if (levels_done)
            for (int p = threadIdx.x; p < P; p += blockDim.x) mymax = max(mymax, vlev[p] + 1);
    }
    // ---- sweep in particle order, one thread per case
    const int ncases = ct.arr ? ct.ncases : 1;
    for (int c = threadIdx.x; !levels_done && c < ncases; c += blockDim.x) {
        const DevCase cd = ct.get(c);
        for (int p = cd.p0; p < cd.p1; ++p) {
            int best = 0;
            if (order == IB_ORDER_SEQUENTIAL) {
                const int cn = nbr_on ? s_cnt[p] : nbr_cnt[p];
                if (cn >= 0) {
                    for (int k = 0; k < cn; ++k)
                        best = max(best, lev[nbr_on ? s_nbr[p * kMaxNbr + k] : nbr[(size_t)p * kMaxNbr + k]] + 1);
                } else {
                    const DevGrid &g = cd.g;
                    const double L[3] = {g.n[0] * g.h, g.n[1] * g.h, g.n[2] * g.h};
                    const double iL[3] = {1.0 / L[0], 1.0 / L[1], 1.0 / L[2]};
                    const double halo = 1.7320508075688772 * KW * g.h;
                    for (int q = cd.p0; q < p; ++q) {
                        float d2 = 0.0f;
                        for (int a = 0; a < 3; ++a) {
                            float d = (float)Xr[3 * q + a] - (float)Xr[3 * p + a];
                            d -= (float)L[a] * rintf(d * (float)iL[a]);
                            d2 += d * d;
                        }
                        const float lim = (float)(rho[p] + rho[q] + halo + 0.0625 * g.h);
                        if (d2 < lim * lim) best = max(best, lev[q] + 1);
                    }
                }
            }
            lev[p] = best;
            mymax = max(mymax, best + 1);
        }
    }
    atomicMax(&s_nl, mymax);
    __syncthreads();
    const int nl = s_nl;
    // ---- counting sort by level
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        if (lev_on) lo.level[p] = lev[p];
        atomicAdd(&lo.lev_pbeg[lev[p]], 1);
    }
    __syncthreads();
    // counts -> exclusive offsets, in place (read through atomics: written by atomics above)
    block_scan_chunked(nl, [&](int l) { return atomicAdd(&lo.lev_pbeg[l], 0); },
                       [&](int l, int pre) { atomicExch(&lev_cur[l], pre); });
    __syncthreads();
    // (values shared through L2 are written and read with atomics throughout)
    for (int l = threadIdx.x; l < nl; l += blockDim.x) atomicExch(&lo.lev_pbeg[l], atomicAdd(&lev_cur[l], 0));
    if (threadIdx.x == 0) {
        lo.lev_pbeg[nl] = P;
        *lo.nlev = nl;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const int r = atomicAdd(&lev_cur[lev[p]], 1);
        lo.rank[p] = r;
        atomicExch(&by_rank[r], p);
    }
    __syncthreads();
    // ---- level-major marker offsets: exclusive scan of marker counts by rank
    const int M = block_scan_chunked(
        P, [&](int r) { const int p = atomicAdd(&by_rank[r], 0); return moff[p + 1] - moff[p]; },
        [&](int r, int pre) { atomicExch(&lo.mbase[atomicAdd(&by_rank[r], 0)], pre); });
    __syncthreads();
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
        const int r = atomicAdd(&lo.lev_pbeg[l], 0);
        lo.lev_mbeg[l] = atomicAdd(&lo.mbase[atomicAdd(&by_rank[r], 0)], 0);
    }
    if (threadIdx.x == 0) lo.lev_mbeg[nl] = M;
}

// ---------------------------------------------------------------------------
// slot counting and filling
// ---------------------------------------------------------------------------
// Tiles a marker's stencil touches along one axis: distinct tile indices of
// the KW cells from `first`.  Global tiles use wrapped cells; local tiles use
// cells relative to the particle box (no wrap, box <= grid).
template <int KW>
__device__ __forceinline__ int axis_tiles_global(int first, int n, int t[3], int c[3]) {
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < KW; ++k) {
        int cc = wrap_add(first, k, n);
        int tt = cc / kTile;
        int j = 0;
        while (j < cnt && t[j] != tt) ++j;
        if (j < cnt) ++c[j];
        else if (cnt < 3) {
            t[cnt] = tt;
            c[cnt++] = 1;
        }
    }
    return cnt;
}

template <int KW>
__device__ __forceinline__ int axis_tiles_local(long long first_rel, int t[3], int c[3]) {
    int a = (int)(first_rel / kTile), b = (int)((first_rel + KW - 1) / kTile);
    t[0] = a;
    if (b != a) {
        t[1] = b;
        c[0] = (int)((long long)(a + 1) * kTile - first_rel);
        c[1] = KW - c[0];
        return 2;
    }
    c[0] = KW;
    return 1;
}

struct SlotGeom {
    int mode;              // 0 global tiles (per case), 1 particle-local tiles
    const int *part_of;    // [M], nullptr: every marker in case 0
    const int *rank;       // [P]
    const int4 *box_lo;    // [P]
    const int4 *box_dim;   // [P]
};

// Enumerate the dense slots of marker l and call f(slot).
template <int KW, typename Fn>
__device__ __forceinline__ void for_marker_slots(const CaseTab &ct, const SlotGeom &sg, int l,
                                                 uint64_t anc, Fn f) {
    int tx[3], ty[3], tz[3], nx, ny, nz;
    int cx[3] = {0, 0, 0}, cy[3] = {0, 0, 0}, cz[3] = {0, 0, 0};  // stencil cells per axis tile
    uint32_t base = 0;
    const DevCase &cd = ct.get(sg.part_of ? ct.case_of(sg.part_of[l]) : 0);
    const DevGrid &g = cd.g;
    if (sg.mode == 0) {
        nx = axis_tiles_global<KW>(anchor_x(anc), g.n[0], tx, cx);
        ny = axis_tiles_global<KW>(anchor_y(anc), g.n[1], ty, cy);
        nz = axis_tiles_global<KW>(anchor_z(anc), g.n[2], tz, cz);
    } else {
        int p = sg.part_of[l];
        int4 blo = sg.box_lo[p];
        // relative first cell: (anchor - box_lo) mod n, < box dims
        // box_lo is wrapped by the preparation kernel: [0, n)
        long long rx = wrap_diff(anchor_x(anc), blo.x, g.n[0]);
        long long ry = wrap_diff(anchor_y(anc), blo.y, g.n[1]);
        long long rz = wrap_diff(anchor_z(anc), blo.z, g.n[2]);
        nx = axis_tiles_local<KW>(rx, tx, cx);
        ny = axis_tiles_local<KW>(ry, ty, cy);
        nz = axis_tiles_local<KW>(rz, tz, cz);
        // a box wider than kMaxBox is reported by the preparation kernel;
        // keep every slot id in range regardless
        if (tx[nx - 1] >= kLocalTiles || ty[ny - 1] >= kLocalTiles || tz[nz - 1] >= kLocalTiles) return;
        base = (uint32_t)sg.rank[p] * kLocalSlots;
    }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                uint32_t s;
                if (sg.mode == 0)
                    s = cd.tile_off + ((uint32_t)tz[k] * cd.tiles[1] + ty[j]) * cd.tiles[0] + tx[i];
                else
                    s = base + ((uint32_t)tz[k] * kLocalTiles + ty[j]) * kLocalTiles + tx[i];
                f(s, (uint32_t)(cx[i] * cy[j] * cz[k]));
            }
}

template <int KW>
__global__ void k_slot_count(CaseTab ct, int M, SlotGeom sg, const uint64_t *__restrict__ anchor,
                             uint32_t *__restrict__ count) {
    grid_dep_wait();
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < M; l += gridDim.x * blockDim.x)
        for_marker_slots<KW>(ct, sg, l, anchor[l], [&](uint32_t s, uint32_t) { atomicAdd(count + s, 1u); });
}

template <int KW>
__global__ void k_slot_fill(CaseTab ct, int M, SlotGeom sg, const uint64_t *__restrict__ anchor,
                            const uint32_t *__restrict__ start, uint32_t *__restrict__ cursor,
                            uint32_t *__restrict__ cand, uint32_t *__restrict__ pcnt) {
    grid_dep_wait();
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < M; l += gridDim.x * blockDim.x)
        for_marker_slots<KW>(ct, sg, l, anchor[l], [&](uint32_t s, uint32_t ncell) {
            uint32_t pos = start[s] + atomicAdd(cursor + s, 1u);
            cand[pos] = (uint32_t)l;
            if (pcnt) pcnt[pos] = ncell;
        });
}

// ---------------------------------------------------------------------------
// single-pass exclusive scans (decoupled look-back, Merrill & Garland 2016):
// each CTA takes the next tile of kLbTile elements from a ticket counter,
// publishes its tile sum, then -- walking back over the tiles before it
// until one has published its inclusive prefix -- its own inclusive prefix,
// and scans the tile from that base.  A tile waits only for tiles taken
// earlier by CTAs already running, so every wait ends; each is bounded all
// the same (IB_ERR_TIMEOUT).  Tile words pack a 2-bit state (0 none,
// 1 tile sum, 2 inclusive prefix) above a 62-bit value; the words and the
// ticket are zeroed before the call's kernel chain.
// ---------------------------------------------------------------------------
constexpr int kLbThreads = 256, kLbItems = 8, kLbTile = kLbThreads * kLbItems;
constexpr unsigned long long kLbVal = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive scan of one value per thread over the CTA (64-bit, fixed order).
__device__ __forceinline__ unsigned long long lb_block_scan(unsigned long long v, unsigned long long *total) {
    __shared__ unsigned long long s_w[kLbThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    unsigned long long wbase = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kLbThreads / 32; ++w) {
        if (w < warp) wbase += s_w[w];
        tot += s_w[w];
    }
    *total = tot;
    return wbase + x - v;
}

// The tile's exclusive base: warp 0 publishes the tile sum, then reads the
// words of the 32 tiles before it at once (lane l: tile - 1 - l), waiting for
// each to be published, and adds the sums up to the nearest inclusive prefix;
// without one it moves 32 tiles further back.  Positions before tile 0 count
// as an inclusive prefix of 0.  Every thread gets the base.  false: a wait
// gave up.
__device__ __forceinline__ bool lb_tile_base(int tile, unsigned long long tot, unsigned long long *tstat,
                                             DevStatus *st, unsigned long long &base) {
    __shared__ unsigned long long s_base;
    __shared__ int s_ok;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        unsigned long long pre = 0;
        bool ok = true;
        if (tile > 0) {
            if (lane == 0) st_release64(tstat + tile, (1ull << 62) | tot);
            for (int hi = tile - 1;; hi -= 32) {
                const int j = hi - lane;
                unsigned long long w = j >= 0 ? ld_acquire64(tstat + j) : (2ull << 62);
                if ((w >> 62) == 0) {
                    const long long t0 = clock64();
                    do {
                        if (clock64() - t0 > kSpinCycles) {
                            raise_status(st, IB_ERR_TIMEOUT, -2);
                            w = 2ull << 62;  // give up: stop here
                            ok = false;
                            break;
                        }
                        w = ld_acquire64(tstat + j);
                    } while ((w >> 62) == 0);
                }
                __syncwarp();
                const unsigned incl = __ballot_sync(0xffffffffu, (w >> 62) == 2);
                const int first = incl ? __ffs(incl) - 1 : 31;
                unsigned long long v = (lane <= first && j >= 0) ? (w & kLbVal) : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                pre += v;
                if (incl) break;
            }
            ok = __all_sync(0xffffffffu, ok);
        }
        if (lane == 0) {
            st_release64(tstat + tile, (2ull << 62) | ((pre + tot) & kLbVal));
            s_base = pre;
            s_ok = ok ? 1 : 0;
        }
    }
    __syncthreads();
    base = s_base;
    return s_ok != 0;
}

// The dense slots: start = exclusive scan of the counts, flag_scan =
// exclusive scan of (count > 0), and dense_of[flag_scan[i]] = i for every
// non-empty slot i -- one pass over the counts (the two sums packed in one
// 64-bit word: counts below, flags from bit 32).
__global__ void __launch_bounds__(kLbThreads) k_slot_scan(const uint32_t *__restrict__ count, int n,
                                                          uint32_t *__restrict__ start,
                                                          uint32_t *__restrict__ flag_scan,
                                                          uint32_t *__restrict__ dense_of,
                                                          unsigned long long *tstat, unsigned int *ticket,
                                                          DevStatus *st) {
    __shared__ int s_tile;
    grid_dep_wait();
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int i0 = tile * kLbTile + threadIdx.x * kLbItems;
    uint32_t c[kLbItems];
    unsigned long long sum = 0;
#pragma unroll
    for (int k = 0; k < kLbItems; ++k) {
        c[k] = i0 + k < n ? count[i0 + k] : 0u;
        sum += (unsigned long long)c[k] | ((unsigned long long)(c[k] != 0u) << 32);
    }
    unsigned long long tot, base;
    const unsigned long long ex = lb_block_scan(sum, &tot);
    if (!lb_tile_base(tile, tot, tstat, st, base)) return;
    unsigned long long run = base + ex;
#pragma unroll
    for (int k = 0; k < kLbItems; ++k) {
        const int i = i0 + k;
        if (i < n) {
            start[i] = (uint32_t)run;
            flag_scan[i] = (uint32_t)(run >> 32);
            if (c[k]) dense_of[run >> 32] = (uint32_t)i;
        }
        run += (unsigned long long)c[k] | ((unsigned long long)(c[k] != 0u) << 32);
    }
    if (i0 <= n && n < i0 + kLbItems) {  // the thread holding position n writes the totals
        start[n] = (uint32_t)run;
        flag_scan[n] = (uint32_t)(run >> 32);
    }
}

// out = exclusive scan of in[0, n'), n' = min(n, *n_dev); out[n'] = total.
// Tiles past n' return at once.
__global__ void __launch_bounds__(kLbThreads) k_scan_lb(const uint32_t *__restrict__ in, int n,
                                                        const uint32_t *__restrict__ n_dev,
                                                        uint32_t *__restrict__ out, unsigned long long *tstat,
                                                        unsigned int *ticket, DevStatus *st) {
    __shared__ int s_tile;
    grid_dep_wait();
    const int nn = min(n, (int)*n_dev);
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int tile = s_tile;
    if (tile * kLbTile > nn) return;  // no element, and not the tile of the total either
    const int i0 = tile * kLbTile + threadIdx.x * kLbItems;
    uint32_t v[kLbItems];
    unsigned long long sum = 0;
#pragma unroll
    for (int k = 0; k < kLbItems; ++k) {
        v[k] = i0 + k < nn ? in[i0 + k] : 0u;
        sum += v[k];
    }
    unsigned long long tot, base;
    const unsigned long long ex = lb_block_scan(sum, &tot);
    if (!lb_tile_base(tile, tot, tstat, st, base)) return;
    unsigned long long run = base + ex;
#pragma unroll
    for (int k = 0; k < kLbItems; ++k) {
        if (i0 + k < nn) out[i0 + k] = (uint32_t)run;
        run += v[k];
    }
    if (i0 <= nn && nn < i0 + kLbItems) out[nn] = (uint32_t)run;
}

__global__ void k_level_slots(int mode, const int *__restrict__ nlev_p, const int *__restrict__ lev_pbeg,
                              const uint32_t *__restrict__ fscan, int ndense, int *__restrict__ lev_sbeg) {
    grid_dep_wait();
    int nl = *nlev_p;
    for (int L = threadIdx.x; L <= nl; L += blockDim.x) {
        if (mode == 0) {
            lev_sbeg[L] = L == 0 ? 0 : (int)fscan[ndense];
        } else {
            long long d = (long long)lev_pbeg[L] * kLocalSlots;
            lev_sbeg[L] = (int)fscan[d < ndense ? d : ndense];
        }
    }
}

// Per wavefront, its tiles in decreasing number of band cells (a counting
// sort; equal sizes in any order).  The wavefront gather takes its tiles in
// this order, so when a wavefront has more tiles than resident CTAs the
// second round gets the smallest ones.  Only the launch order changes: every
// tile's sums are the same whichever CTA computes them.
__global__ void __launch_bounds__(512) k_level_tile_order(const int *__restrict__ nlev_p,
                                                           const int *__restrict__ lev_sbeg,
                                                           const int *__restrict__ nband, int *__restrict__ tperm) {
    grid_dep_wait();
    __shared__ int s_hist[kTileCells + 1];
    const int nl = *nlev_p;
    for (int L = blockIdx.x; L < nl; L += gridDim.x) {  // one CTA per wavefront
        const int s0 = lev_sbeg[L], s1 = lev_sbeg[L + 1];
        for (int k = threadIdx.x; k <= kTileCells; k += blockDim.x) s_hist[k] = 0;
        __syncthreads();
        for (int t = s0 + threadIdx.x; t < s1; t += blockDim.x)
            atomicAdd(&s_hist[kTileCells - min(max(nband[t], 0), kTileCells)], 1);
        __syncthreads();
        block_scan_chunked(kTileCells + 1, [&](int k) { return s_hist[k]; }, [&](int k, int pre) { s_hist[k] = pre; });
        __syncthreads();
        for (int t = s0 + threadIdx.x; t < s1; t += blockDim.x)
            tperm[s0 + atomicAdd(&s_hist[kTileCells - min(max(nband[t], 0), kTileCells)], 1)] = t;
        __syncthreads();
    }
}

// Level-major marker list: the markers of the particle of rank r follow
// those of the particles of lower rank, each particle's in index order (the
// Fibonacci lattice index already walks the sphere band by band in z; a
// spatial sort of each particle's markers measured slower end to end).
__global__ void k_marker_order(int P, const int *__restrict__ moff, const int *__restrict__ mbase,
                               int *__restrict__ mperm) {
    grid_dep_wait();
    for (int p = blockIdx.x; p < P; p += gridDim.x) {
        const int m0 = moff[p], n = moff[p + 1] - m0, base = mbase[p];
        for (int i = threadIdx.x; i < n; i += blockDim.x) mperm[base + i] = m0 + i;
    }
}

// ---------------------------------------------------------------------------
// per-slot sort by (row, marker) and row starts.  Tiles with at most
// kWarpSort candidates are sorted by one warp each (bitonic network in
// registers, the sorted keys then kept in a warp-private shared-memory
// region); larger tiles by a whole CTA (bitonic network in shared memory).
// ---------------------------------------------------------------------------
constexpr int kWarpSort = 256;

// Case of dense global-tile slot d: the last case whose tile_off <= d.
__device__ __forceinline__ int case_of_tile(const CaseTab &ct, uint32_t d) {
    if (!ct.arr) return 0;
    int a = 0, b = ct.ncases - 1;
    while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (ct.arr[mid].tile_off <= d) a = mid;
        else b = mid - 1;
    }
    return a;
}

__device__ __forceinline__ int slot_geometry(const CaseTab &ct, int mode, const SlotGeom &sg, const Slots &sl,
                                             const int *level, uint32_t d, uint32_t b, int lo[3], int dim[3],
                                             int &lev) {
    lev = 0;
    if (mode == 0) {
        const int c = case_of_tile(ct, d);
        const DevCase &cd = ct.get(c);
        const DevGrid &g = cd.g;
        d -= cd.tile_off;
        const int t[3] = {(int)(d % cd.tiles[0]), (int)((d / cd.tiles[0]) % cd.tiles[1]),
                          (int)(d / ((uint32_t)cd.tiles[0] * cd.tiles[1]))};
        for (int a = 0; a < 3; ++a) {
            lo[a] = t[a] * kTile;
            dim[a] = min(kTile, g.n[a] - lo[a]);
        }
        return c;
    } else {
        const int p = sg.part_of[sl.cand[b]];  // every candidate of a local tile has the same particle
        const DevGrid &g = ct.of_particle(p).g;
        const int lt = (int)(d % kLocalSlots);
        const int t[3] = {lt % kLocalTiles, (lt / kLocalTiles) % kLocalTiles, lt / (kLocalTiles * kLocalTiles)};
        const int4 blo = sg.box_lo[p], bd = sg.box_dim[p];
        const int bl[3] = {blo.x, blo.y, blo.z}, bdm[3] = {bd.x, bd.y, bd.z};
        for (int a = 0; a < 3; ++a) {
            lo[a] = wrap_int((long long)bl[a] + t[a] * kTile, g.n[a]);
            dim[a] = min(kTile, bdm[a] - t[a] * kTile);
        }
        lev = level[p];
        return ct.case_of(p);
    }
}

// v mod n for v in [-n, 2n)
__device__ __forceinline__ int wrap_once(int v, int n) {
    v += v < 0 ? n : 0;
    return v >= n ? v - n : v;
}

__device__ __forceinline__ unsigned long long slot_key(const DevGrid &g, const uint64_t *anchor, uint32_t m,
                                                       const int lo[3]) {
    const uint64_t anc = anchor[m];
    // anchor and lo lie in [0, n): one conditional add or subtract wraps
    const int rz = wrap_once(anchor_z(anc) - lo[2] + 3, g.n[2]);
    const int ry = wrap_once(anchor_y(anc) - lo[1] + 3, g.n[1]);
    const int v = wrap_once(anchor_x(anc) - lo[0] + 3, g.n[0]);
    const int bin = (rz < kRow && ry < kRow && v < kRow) ? (rz * kRow + ry) * kBinsPerRow + v
                                                         : kBins - 1;  // never read
    return ((unsigned long long)bin << 32) | m;
}

// Writes the sorted candidates, their x offsets and the row starts of slot cs
// from keys[0..nc) (sorted); `lane`/`nl` split the work over nl threads.
__device__ __forceinline__ void slot_emit(const DevGrid &g, const uint64_t *anchor, const unsigned long long *keys,
                                          int nc, uint32_t b, int cs, const int lo[3], const Slots &sl, int lane,
                                          int nl) {
    for (int i = lane; i < nc; i += nl) sl.cand[b + i] = (uint32_t)(keys[i] & 0xffffffffu);
    if (!sl.bins) return;
    uint16_t *bs = sl.bins + (size_t)cs * kBins;
    for (int r = lane; r < kBins; r += nl) {
        // first index whose bin >= r
        int a = 0, e = nc;
        while (a < e) {
            const int mid = (a + e) >> 1;
            if ((int)(keys[mid] >> 32) < r) a = mid + 1;
            else e = mid;
        }
        bs[r] = (uint16_t)(r == kBins - 1 ? nc : a);
    }
}

// Sorts 32 R keys held by one warp, element e = 32 r + lane in x[r], with a
// bitonic network in registers: partners in other lanes come by shuffle,
// partners in the same lane are compared directly.
template <int R>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&x)[R], int lane) {
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int jr = j >> 5;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if ((r & jr) == 0) {
                        const bool asc = ((32 * r + lane) & k) == 0;
                        const unsigned long long a = x[r], b = x[r | jr];
                        const bool sw = (a > b) == asc;
                        x[r] = sw ? b : a;
                        x[r | jr] = sw ? a : b;
                    }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const unsigned long long y = __shfl_xor_sync(0xffffffffu, x[r], j);
                    // the lower index of a pair keeps the minimum in an
                    // ascending block, the maximum in a descending one
                    const bool take_min = ((lane & j) == 0) == (((32 * r + lane) & k) == 0);
                    x[r] = take_min ? (y < x[r] ? y : x[r]) : (y > x[r] ? y : x[r]);
                }
            }
        }
}

// One warp: keys of a tile with nc <= 32 R candidates into wk[0, 32 R), sorted.
template <int R>
__device__ __forceinline__ void warp_sort_keys(const DevGrid &g, const uint64_t *anchor, const uint32_t *cand,
                                               int nc, const int lo[3], unsigned long long *wk, int lane) {
    unsigned long long x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = 32 * r + lane;
        x[r] = e < nc ? slot_key(g, anchor, cand[e], lo) : ~0ull;
    }
    warp_bitonic<R>(x, lane);
#pragma unroll
    for (int r = 0; r < R; ++r) wk[32 * r + lane] = x[r];
    __syncwarp();
}

__global__ void __launch_bounds__(kBlock) k_slot_sort(
    CaseTab ct, int mode, int ncompact_cap, const int *__restrict__ ncompact_p, SlotGeom sg,
    const uint32_t *__restrict__ dense_of, const uint32_t *__restrict__ start,
    const uint64_t *__restrict__ anchor, const int *__restrict__ level, Slots sl, DevStatus *st) {
    grid_dep_wait();
    __shared__ unsigned long long keys[kMaxCand];  // also kBlock/32 warp regions of kWarpSort
    const int ncompact = min(*ncompact_p, ncompact_cap);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // ---- phase 1: one warp per small tile
    unsigned long long *wk = keys + warp * kWarpSort;
    for (int cs = blockIdx.x * nwarp + warp; cs < ncompact; cs += gridDim.x * nwarp) {
        const uint32_t d = dense_of[cs];
        const uint32_t b = start[d];
        const int nc = (int)(start[d + 1] - b);
        if (nc > kWarpSort) continue;
        int lo[3], dim[3], lev;
        const int cse = slot_geometry(ct, mode, sg, sl, level, d, b, lo, dim, lev);
        const DevGrid &g = ct.get(cse).g;
        static_assert(kWarpSort == 256, "warp sorts cover 64, 128 or 256 keys");
        if (nc <= 64) warp_sort_keys<2>(g, anchor, sl.cand + b, nc, lo, wk, lane);
        else if (nc <= 128) warp_sort_keys<4>(g, anchor, sl.cand + b, nc, lo, wk, lane);
        else warp_sort_keys<8>(g, anchor, sl.cand + b, nc, lo, wk, lane);
        slot_emit(g, anchor, wk, nc, b, cs, lo, sl, lane, 32);
        if (lane == 0) {
            sl.geo_lo[cs] = make_int4(lo[0], lo[1], lo[2], lev);
            sl.geo_dim[cs] = make_int4(dim[0], dim[1], dim[2], (int)b);
            sl.geo_case[cs] = cse;
        }
        __syncwarp();
    }
    __syncthreads();
    // ---- phase 2: one CTA per large tile.  The CTA's tiles (cs = blockIdx.x
    // mod gridDim.x) are screened blockDim.x at a time, one load per thread,
    // and only the large ones are walked.
    __shared__ int s_big[kBlock];
    __shared__ int s_nbig;
    for (long long c0 = blockIdx.x; c0 < ncompact; c0 += (long long)gridDim.x * blockDim.x) {
        if (threadIdx.x == 0) s_nbig = 0;
        __syncthreads();
        const long long ct_cs = c0 + (long long)threadIdx.x * gridDim.x;
        if (ct_cs < ncompact) {
            const uint32_t d = dense_of[ct_cs];
            if ((int)(start[d + 1] - start[d]) > kWarpSort) s_big[atomicAdd(&s_nbig, 1)] = (int)ct_cs;
        }
        __syncthreads();
        const int nbig = s_nbig;
        for (int q = 0; q < nbig; ++q) {
            const int cs = s_big[q];
            const uint32_t d = dense_of[cs];
            const uint32_t b = start[d];
            const int nc = (int)(start[d + 1] - b);
            int lo[3], dim[3], lev;
            const int cse = slot_geometry(ct, mode, sg, sl, level, d, b, lo, dim, lev);
            const DevGrid &g = ct.get(cse).g;
            if (nc > kMaxCand) {
                // report, and leave an empty tile (no bins, no cells)
                if (sl.bins) {
                    uint16_t *bs = sl.bins + (size_t)cs * kBins;
                    for (int r = threadIdx.x; r < kBins; r += blockDim.x) bs[r] = 0;
                }
                if (threadIdx.x == 0) {
                    raise_status(st, IB_ERR_UNSUPPORTED, nc);
                    sl.geo_lo[cs] = make_int4(lo[0], lo[1], lo[2], lev);
                    sl.geo_dim[cs] = make_int4(0, 0, 0, (int)b);
                    sl.geo_case[cs] = cse;
                }
                __syncthreads();
                continue;
            }
            int np2 = 1;
            while (np2 < nc) np2 <<= 1;
            for (int i = threadIdx.x; i < np2; i += blockDim.x)
                keys[i] = i < nc ? slot_key(g, anchor, sl.cand[b + i], lo) : ~0ull;
            __syncthreads();
            for (int k = 2; k <= np2; k <<= 1)
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int i = threadIdx.x; i < np2; i += blockDim.x) {
                        const int ixj = i ^ j;
                        if (ixj > i) {
                            const unsigned long long x = keys[i], y = keys[ixj];
                            if ((x > y) == ((i & k) == 0)) {
                                keys[i] = y;
                                keys[ixj] = x;
                            }
                        }
                    }
                    __syncthreads();
                }
            slot_emit(g, anchor, keys, nc, b, cs, lo, sl, threadIdx.x, blockDim.x);
            if (threadIdx.x == 0) {
                sl.geo_lo[cs] = make_int4(lo[0], lo[1], lo[2], lev);
                sl.geo_dim[cs] = make_int4(dim[0], dim[1], dim[2], (int)b);
                sl.geo_case[cs] = cse;
            }
            __syncthreads();
        }
        __syncthreads();  // s_big and s_nbig are reused by the next screen
    }
}

// ---------------------------------------------------------------------------
// per-cell gather lists.  One CTA of 8 warps per compact tile (grid-stride).
// A cell's contributions are the candidates whose stencil covers it.  The
// bin walk of gather_cell visits a tile's bins in ascending (anchor z, y, x)
// order and a bin's candidates in index order -- in ascending candidate
// index, the order the tile's candidates are sorted in -- so listing every
// cell's candidates in ascending index reproduces its summation order.
// The (candidate, stencil cell) pairs are scattered by a stable counting sort
// on the cell: each warp counts the pairs of a contiguous range of candidates
// (one candidate per step, one lane per stencil offset, so the cells of a
// step are distinct), a scan over (cell, warp) gives every warp its base in
// every cell's list, and each warp then places its pairs candidate by
// candidate.
// ---------------------------------------------------------------------------
constexpr int kPairThreads = 256;
constexpr int kPairWarps = kPairThreads / 32;
static_assert(kTileCells == 2 * kPairThreads, "each thread of k_tile_pairs owns two cells");

template <typename T, int KW>
__global__ void __launch_bounds__(kPairThreads, 5) k_tile_pairs(CaseTab ct, int ncompact_cap,
                                                             const int *__restrict__ ncompact_p, Slots sl,
                                                             const uint64_t *__restrict__ anchor,
                                                             const PS<T> *__restrict__ wts) {
    PS<T> *const pwts = (PS<T> *)sl.pw;
    grid_dep_wait();
    constexpr int KW3 = KW * KW * KW;
    // per candidate: the in-tile stencil offsets per axis (bits 0-3 x, 4-7 y,
    // 8-11 z) and its first stencil cell relative to the tile, x + 8 y + 64 z
    // + 256, from bit 12
    __shared__ unsigned int s_anc[kMaxCand];
    __shared__ __align__(16) unsigned int s_cnt[kPairWarps][kTileCells];  // counts, then list cursors
    __shared__ int s_wp[kPairWarps], s_wb[kPairWarps];
    const int ncompact = min(*ncompact_p, ncompact_cap);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // this lane's stencil offsets k = lane + 32 q
    // (ox | oy << 2 | oz << 4, or ~0u past the stencil)
    constexpr int kSub = (KW3 + 31) / 32;
    unsigned kcode[kSub];
    int koff[kSub];  // the offset's cell step x + 8 y + 64 z
#pragma unroll
    for (int q = 0; q < kSub; ++q) {
        const int k = lane + 32 * q;
        kcode[q] = k < KW3 ? (unsigned)((k % KW) | (((k / KW) % KW) << 2) | ((k / (KW * KW)) << 4)) : ~0u;
        koff[q] = (k % KW) + kTile * ((k / KW) % KW) + kTile * kTile * (k / (KW * KW));
    }
    for (int cs = blockIdx.x; cs < ncompact; cs += gridDim.x) {
        const int4 lo = sl.geo_lo[cs], dim = sl.geo_dim[cs];
        const DevGrid g = ct.get(sl.geo_case[cs]).g;
        const int b = dim.w;
        const uint32_t dn = sl.dense_of[cs];
        int nc = (int)(sl.start[dn + 1] - sl.start[dn]);
        if (nc > kMaxCand) nc = 0;  // left empty by the sort (status raised there)
        int2 *band = sl.band + sl.poff[b];
        uint32_t *pairs = sl.pairs + sl.poff[b];
        PS<T> *pw = pwts ? pwts + sl.poff[b] : nullptr;
        for (int i = tid; i < nc; i += blockDim.x) {
            const uint64_t an = anchor[sl.cand[b + i]];
            int d[3] = {anchor_x(an) - lo.x + 3, anchor_y(an) - lo.y + 3, anchor_z(an) - lo.z + 3};
            const int dm[3] = {dim.x, dim.y, dim.z};
            unsigned code = 0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (d[q] < 0) d[q] += g.n[q];
                if (d[q] >= g.n[q]) d[q] -= g.n[q];
                d[q] = min(d[q], 15) - 3;  // a candidate's anchor lies within [-3, 8) of the tile
                unsigned mq = 0;
#pragma unroll
                for (int k = 0; k < KW; ++k) mq |= (d[q] + k >= 0 && d[q] + k < dm[q]) ? 1u << k : 0u;
                code |= mq << (4 * q);
            }
            s_anc[i] = code | (unsigned)(d[0] + kTile * d[1] + kTile * kTile * d[2] + 256) << 12;
        }
        for (int c = tid; c < kPairWarps * kTileCells / 4; c += blockDim.x)
            ((uint4 *)&s_cnt[0][0])[c] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        // Each warp walks a contiguous range of candidates, one candidate per
        // step, lane l taking the stencil offsets k = l + 32 q: the cells of
        // one step are distinct, so counts and list slots need no ranking.
        const int seg = (nc + kPairWarps - 1) / kPairWarps;
        const int i0 = min(nc, warp * seg), i1 = min(nc, i0 + seg);
        // cell of candidate i's stencil offset (lane, q), or -1
        auto cell_of = [&](unsigned pk, int q) {
            const unsigned o = kcode[q];
            const unsigned in = (pk >> (o & 3)) & (pk >> (4 + ((o >> 2) & 3))) & (pk >> (8 + ((o >> 4) & 3)));
            return (o != ~0u && (in & 1u)) ? (int)(pk >> 12) - 256 + koff[q] : -1;
        };
        for (int i = i0; i < i1; ++i) {
            const unsigned pk = s_anc[i];
#pragma unroll
            for (int q = 0; q < kSub; ++q) {
                const int c = cell_of(pk, q);
                if (c >= 0) atomicAdd(&s_cnt[warp][c], 1u);
            }
        }
        __syncthreads();
        // (cell, warp) scan: thread t owns cells 2t and 2t + 1
        int tot[2] = {0, 0}, pre[2][kPairWarps];
#pragma unroll
        for (int w = 0; w < kPairWarps; ++w) {
            const uint2 cw = ((const uint2 *)s_cnt[w])[tid];
            pre[0][w] = tot[0];
            pre[1][w] = tot[1];
            tot[0] += (int)cw.x;
            tot[1] += (int)cw.y;
        }
        int pv = tot[0] + tot[1], bv = (tot[0] > 0) + (tot[1] > 0);
        for (int o = 1; o < 32; o <<= 1) {
            const int yp = __shfl_up_sync(0xffffffffu, pv, o), yb = __shfl_up_sync(0xffffffffu, bv, o);
            if (lane >= o) pv += yp, bv += yb;
        }
        if (lane == 31) s_wp[warp] = pv, s_wb[warp] = bv;
        __syncthreads();
        int wp = 0, wb = 0;
        for (int w = 0; w < warp; ++w) wp += s_wp[w], wb += s_wb[w];
        const int cp0 = wp + pv - (tot[0] + tot[1]), cb0 = wb + bv - ((tot[0] > 0) + (tot[1] > 0));
        const int cbase[2] = {cp0, cp0 + tot[0]};
        if (tot[0] > 0) band[cb0] = make_int2((2 * tid) | (tot[0] << 16), cbase[0]);
        if (tot[1] > 0) band[cb0 + (tot[0] > 0)] = make_int2((2 * tid + 1) | (tot[1] << 16), cbase[1]);
        if (tid == blockDim.x - 1) {
            const int nbd = cb0 + (tot[0] > 0) + (tot[1] > 0);
            sl.nband[cs] = nbd;
            sl.tinfo[cs] = make_int4((int)sl.poff[b], (int)(sl.poff[b + nc] - sl.poff[b]), nbd, nc);
        }
#pragma unroll
        for (int w = 0; w < kPairWarps; ++w)
            ((uint2 *)s_cnt[w])[tid] = make_uint2((unsigned)(cbase[0] + pre[0][w]), (unsigned)(cbase[1] + pre[1][w]));
        __syncthreads();
        // placement in candidate order: a cell's list ascends in candidate
        // index (one step's cells are distinct; the warp barrier orders steps)
        for (int i = i0; i < i1; ++i) {
            const unsigned pk = s_anc[i];
#pragma unroll
            for (int q = 0; q < kSub; ++q) {
                const int c = cell_of(pk, q);
                if (c >= 0) pairs[atomicAdd(&s_cnt[warp][c], 1u)] = (unsigned)i | (kcode[q] << 16);
            }
            __syncwarp();
        }
        __syncthreads();
        // every pair's weight product, one pair per thread (the pair words
        // written above are visible to the whole CTA after the barrier), kPwU
        // pairs per thread at a time: the pair words, then the candidates'
        // marker indices, then their axis weights are each loaded together,
        // three dependent rounds of loads instead of three per pair
        if (pw) {
            const int np = (int)(sl.poff[b + nc] - sl.poff[b]);
            constexpr int kPwU = 4;
            for (int k0 = tid; k0 < np; k0 += kPwU * kPairThreads) {
                unsigned pk[kPwU];
                uint32_t mk[kPwU];
#pragma unroll
                for (int u = 0; u < kPwU; ++u) {
                    const int k = k0 + u * kPairThreads;
                    pk[u] = k < np ? pairs[k] : 0u;
                }
#pragma unroll
                for (int u = 0; u < kPwU; ++u) mk[u] = k0 + u * kPairThreads < np ? sl.cand[b + (pk[u] & 0xffff)] : 0u;
                PS<T> wx[kPwU], wy[kPwU], wz[kPwU];
#pragma unroll
                for (int u = 0; u < kPwU; ++u) {
                    const PS<T> *w = wts + 12 * (size_t)mk[u];
                    wx[u] = w[(pk[u] >> 16) & 3];
                    wy[u] = w[4 + ((pk[u] >> 18) & 3)];
                    wz[u] = w[8 + ((pk[u] >> 20) & 3)];
                }
#pragma unroll
                for (int u = 0; u < kPwU; ++u) {
                    const int k = k0 + u * kPairThreads;
                    if (k < np) pw[k] = pair_weight3(wx[u], wy[u], wz[u]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// gather of one tile: every cell sums w * A over the markers whose stencil
// covers it, rows in (z, y) order, markers in index order within a row.
// The tile's candidates (their per-axis weights, spread source and x offset)
// are first staged in shared memory with independent loads; the per-cell
// sums then read shared memory only.  Tiles with more than Stage<T>::N
// candidates read the same values from global memory instead.
// ---------------------------------------------------------------------------
// Spreading (ib_spread) over the tiles' per-cell lists: the case's u slot
// holds the field spread into, its f slot is null.
template <typename T, int KER>
__global__ void __launch_bounds__(256) k_spread_gather(CaseTab ct, const int *__restrict__ ncompact_p, Slots sl,
                                                       const PS<T> *__restrict__ wts, const PS<T> *__restrict__ A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PS<T> *sw = (PS<T> *)smem_raw;
    PS<T> *sA = sw + (size_t)TileStage<T>::N * 12;
    const int nc = *ncompact_p;
    for (int cs = blockIdx.x; cs < nc; cs += gridDim.x)
        gather_tile_lists<T, Kernel<KER>::W, false>(ct, cs, sl, wts, A, 0.0, sw, sA);
}

// Spreading (ib_spread) with warp-aggregated atomics: one lane per marker,
// weights formed on the fly, no binning.
template <typename T, int KER>
__global__ void __launch_bounds__(256) k_spread_atomic(DevGrid g, int M, const double *__restrict__ X,
                                                       const double *__restrict__ F, const double *__restrict__ dV,
                                                       T *__restrict__ f, DevStatus *st) {
    constexpr int KW = Kernel<KER>::W;
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    // warp-uniform loop: every lane takes part in the matching
    for (long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < M;
         base += nwarps * 32) {
        const long long l = base + lane;
        bool valid = l < M;
        double x[3] = {0, 0, 0}, fv[3] = {0, 0, 0}, dv = 0.0;
        if (valid) {
            x[0] = X[3 * l], x[1] = X[3 * l + 1], x[2] = X[3 * l + 2];
            fv[0] = F[3 * l], fv[1] = F[3 * l + 1], fv[2] = F[3 * l + 2];
            dv = dV[l];
            if (!(finite3(x) && finite3(fv) && isfinite(dv))) {
                raise_status(st, IB_ERR_NONFINITE, (int)l);
                valid = false;
            }
        }
        if (!valid) x[0] = g.org[0], x[1] = g.org[1], x[2] = g.org[2];
        PS<T> ws[12], A[3];
        long long first[3];
        const uint64_t anc = marker_weights<T, KER>(g, x, ws, first);
        const double q = dv * g.inv_h3;
#pragma unroll
        for (int c = 0; c < 3; ++c) A[c] = to_store((T)(fv[c] * q));
        scatter_marker<T, KW>(f, (T *)nullptr, g, N, anc, ws, A, valid, 0.0);
    }
}

// ---------------------------------------------------------------------------
// grid barrier with a bounded wait
// ---------------------------------------------------------------------------
struct Barrier {
    unsigned int *count;
    unsigned int *gen;
};


// Sense-free generation barrier over all CTAs of a cooperative launch.  The
// waiting thread polls the generation word without sleeping (a sleep's wake-up
// latency dominated the phases) and gives up after kSpinCycles SM cycles,
// raising IB_ERR_TIMEOUT; every CTA then returns.

__device__ __forceinline__ bool grid_sync(Barrier b, DevStatus *st) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        const unsigned int g0 = ld_acquire(b.gen);
        __threadfence();
        const unsigned int arrived = atomicAdd(b.count, 1u);
        int ok = 1;
        if (arrived == gridDim.x - 1) {
            atomicExch(b.count, 0u);
            __threadfence();
            atomicAdd(b.gen, 1u);
        } else {
            const long long t0 = clock64();
            while (ld_acquire(b.gen) == g0) {
                if (clock64() - t0 > kSpinCycles) {
                    raise_status(st, IB_ERR_TIMEOUT, (int)blockIdx.x);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok && (*(volatile int *)&st->code != IB_ERR_TIMEOUT);
    }
    __syncthreads();
    return s_ok;
}

// ---------------------------------------------------------------------------
// persistent multidirect-forcing passes (cooperative launch)
// ---------------------------------------------------------------------------
constexpr int kInterpThreads = 256;  // level interpolation CTA
constexpr int kGatherThreads = 256;  // level gather CTA (one tile at a time)

template <typename T>
struct PassArgs {
    CaseTab ct;        // cases: grid, u, accumulated force field (nullable)
    const int *part_of;  // [M] particle of each marker
    double *F;
    const double *dV;
    MarkerState<T> ms;
    Slots sl;
    const int *mperm;
    const int *lev_mbeg;
    const int *lev_sbeg;
    const int *tperm;  // per wavefront, its tiles largest first (wavefront gather order)
    const int *nlev;
    int Ns;
    int L0;  // first wavefront the persistent kernel processes
    int atomic;  // spread with warp-aggregated atomics instead of the tile gather
    int stage;   // candidates a gather CTA stages in shared memory (larger tiles read memory)
    double dt, inv_dt;  // inv_dt = 1 / dt, formed on the host
    Barrier bar;
    DevStatus *st;
};

// ---------------------------------------------------------------------------
// one wavefront pass as two ordinary kernels (the form CUDA-graph replay runs
// back to back): interpolation over the wavefront's markers, then a gather
// with one CTA per tile (grid-stride), many CTAs per SM hiding latency.
//
// Every level kernel but the first of a call is launched as a programmatic
// dependent of the one before it: it starts while its predecessor finishes,
// loads what the predecessor does not write (marker weights, anchors, desired
// velocities, forces; tile lists, candidate weights, the first band cell's
// field values), then waits for the predecessor and reads what it wrote (the
// field for an interpolation, the spread sources for a gather).  Every CTA
// waits before it exits, so a level kernel completes only after its
// predecessor.  An interpolation lets its gather start right after its own
// wait (the gather's CTAs stage their lists meanwhile); for FP32 fields a
// gather lets the next interpolation start only as its CTAs exit, so that
// interpolation's CTAs land on idle SMs (measured faster than an early start),
// and for FP64 fields once each of its CTAs has reached its last tile.
// ---------------------------------------------------------------------------
template <typename T, int KER>
__global__ void __launch_bounds__(kInterpThreads) k_interp_level(PassArgs<T> a, int L) {
    constexpr int KW = Kernel<KER>::W;
    // all 81 loads of a Roma-kernel marker in flight at once for FP32 fields
    constexpr bool kAll = KW == 3 && sizeof(T) == 4;
    const int nl = *a.nlev;
    const int m0 = L < nl ? a.lev_mbeg[L] : 0, m1 = L < nl ? a.lev_mbeg[L + 1] : 0;
    const int stride = gridDim.x * blockDim.x;
    int i = m0 + blockIdx.x * blockDim.x + threadIdx.x;
    // one marker's data but the field (loaded before the wait for the first)
    int l = 0;
    uint64_t anc = 0;
    PS<T> w[12];
    PassMarker<T> pm;
    double F[3];
    auto load = [&]() {
        l = a.mperm[i];
        anc = a.ms.anchor[l];
        if (kAll)
#pragma unroll
            for (int k = 0; k < 12; ++k) w[k] = __ldg(a.ms.wts + 12 * (size_t)l + k);
        pm.load(a.ms, a.dV, a.ct.of_particle(a.part_of[l]).g.inv_h3, l);
#pragma unroll
        for (int c = 0; c < 3; ++c) F[c] = a.F[3 * l + c];
    };
    if (i < m1) load();
    grid_dep_wait();
    grid_dep_launch();
    for (bool first = true; i < m1; i += stride, first = false) {
        if (!first) load();
        const DevCase cd = a.ct.of_particle(a.part_of[l]);
        const DevGrid &g = cd.g;
        const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
        T U[3];
        // the field was written by the predecessor: plain loads
        // (weights from registers when every tap is unrolled, else from memory)
        interp_marker<T, KW, true, kAll>((const T *)cd.u, g, N, anc, kAll ? w : a.ms.wts + 12 * (size_t)l, U);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T e = pm.err(c, U[c]);
            a.F[3 * l + c] = PassMarker<T>::force(F[c], e, a.inv_dt);
            a.ms.A[4 * l + c] = pm.source(e);
        }
    }
}

// FP64 fields: one thread per marker component, three per marker.  Each sums
// its component's taps in the order of interp_marker (planes z, rows y,
// columns x; the same double-float products and additions), so the result
// is bitwise the one-thread form's; three times the threads hide the latency
// of the double-float chains and of the field loads.
constexpr bool kInterpSplit = true;  // FP64 level interpolation by component
constexpr bool kInterpSplitAll = true;  // every tap of a component in flight at once

template <int KW, bool ALL>
__device__ __forceinline__ double interp_component(const double *__restrict__ uc, const DevGrid &g, uint64_t anc,
                                                   const float2 *w) {
    int ix[KW], iy[KW], iz[KW];
    const int ax = anchor_x(anc), ay = anchor_y(anc), az = anchor_z(anc);
#pragma unroll
    for (int k = 0; k < KW; ++k) {
        ix[k] = wrap_add(ax, k, g.n[0]);
        iy[k] = wrap_add(ay, k, g.n[1]);
        iz[k] = wrap_add(az, k, g.n[2]);
    }
    SumAcc<double> acc;
    auto plane = [&](int kz) {
        double v[KW][KW];
#pragma unroll
        for (int ky = 0; ky < KW; ++ky) {
            const long long row = ((long long)iz[kz] * g.n[1] + iy[ky]) * g.n[0];
#pragma unroll
            for (int kx = 0; kx < KW; ++kx) v[ky][kx] = uc[row + ix[kx]];
        }
#pragma unroll
        for (int ky = 0; ky < KW; ++ky) {
            const float2 wyz = df_mul(w[8 + kz], w[4 + ky]);
#pragma unroll
            for (int kx = 0; kx < KW; ++kx) acc.add(df_mul(wyz, w[kx]), df_split(v[ky][kx]));
        }
    };
    if (ALL) {
#pragma unroll
        for (int kz = 0; kz < KW; ++kz) plane(kz);
    } else {
#pragma unroll 1
        for (int kz = 0; kz < KW; ++kz) plane(kz);
    }
    return acc.value();
}

template <typename T, int KER>
__global__ void __launch_bounds__(kInterpThreads) k_interp_level_c3(PassArgs<T> a, int L) {
    static_assert(sizeof(T) == 8, "component split serves FP64 fields");
    constexpr int KW = Kernel<KER>::W;
    const int nl = *a.nlev;
    const int m0 = L < nl ? a.lev_mbeg[L] : 0, m1 = L < nl ? a.lev_mbeg[L + 1] : 0;
    const int n3 = 3 * (m1 - m0);
    const int stride = gridDim.x * blockDim.x;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    // one item's data but the field (loaded before the wait for the first)
    int l = 0, c = 0;
    uint64_t anc = 0;
    float2 w[12];
    double ud = 0.0, q = 0.0, F = 0.0;
    auto load = [&]() {
        l = a.mperm[m0 + t / 3];
        c = t % 3;
        anc = a.ms.anchor[l];
#pragma unroll
        for (int k = 0; k < 12; ++k) w[k] = __ldg(a.ms.wts + 12 * (size_t)l + k);
        ud = __ldg(a.ms.Ud + 3 * l + c);
        q = a.dV[l] * a.ct.of_particle(a.part_of[l]).g.inv_h3;
        F = a.F[3 * l + c];
    };
    if (t < n3) load();
    grid_dep_wait();
    grid_dep_launch();
    for (bool first = true; t < n3; t += stride, first = false) {
        if (!first) load();
        const DevCase cd = a.ct.of_particle(a.part_of[l]);
        const DevGrid &g = cd.g;
        const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
        const double U = interp_component<KW, kInterpSplitAll>((const double *)cd.u + c * N, g, anc, w);
        const double e = ud - U;
        a.F[3 * l + c] = fma(e, a.inv_dt, F);
        a.ms.A[4 * l + c] = to_store(e * q);
    }
}

// The wavefront gather, one CTA per tile (grid-stride), many CTAs per SM,
// over the tiles' per-cell lists (sums bitwise those of the bin walk).
//
// Before the wait (nothing here is written by the interpolation): the tile's
// pair words and pair weights (the weight products, formed once per call by
// k_tile_pairs) are staged in shared memory, and each thread loads the list
// heads and field values of its (at most two) band cells.  After the wait
// only the spread sources are loaded; the sums then run from shared memory
// and registers.  Each cell's pairs are added in list order with the same
// weight products as gather_tile_lists forms on the fly, so the sums are
// bitwise the same.
constexpr int kLevPairs = 3072;  // pairs staged per tile (more: read from memory)

constexpr int kLevHalf = kLevPairs / 2;  // a tile this small can be prefetched into half the buffer
constexpr int kLevBand = kTileCells;      // band records of a prefetched tile (at most one per cell)

// Shared memory of a level gather CTA staging `stage` candidates: their
// spread sources, the tile's pair words and pair weights (two halves), and
// two buffers of band records for prefetched tiles.
// FP32 fields only: there the staging round trips of a CTA's later tiles are
// on the critical path (prefetching measured 566 -> 553 us per step); the
// FP64 gather is bound by its double-float sums and measured no gain.
template <typename T>
constexpr bool kLevPrefetch = sizeof(T) == 4;

template <typename T>
size_t level_stage_bytes(int stage) {
    return (size_t)stage * 4 * sizeof(PS<T>) + (size_t)kLevPairs * (sizeof(uint32_t) + sizeof(PS<T>)) +
           (kLevPrefetch<T> ? (size_t)2 * kLevBand * sizeof(int2) : 0);
}

// Asynchronous global -> shared copies (cp.async, completed by
// cp_async_wait_all and made visible to the CTA by a barrier).
template <int B>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gmem), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Where a gather CTA's next tile stands: its lists prefetched into half
// `half` of the staging buffers (pre), or not.
struct GatherPipe {
    int half;
    bool pre;
};

// `wait` runs between the staging of what the interpolation does not write
// and the loads of the spread sources; false (a wait that gave up) leaves the
// tile untouched, CTA-uniformly.  Each pair's weight product comes from the
// per-pair weights k_tile_pairs formed (the value pair_weight gives).
// `pipe` says whether this tile's lists (pair words, pair weights, band
// records) were prefetched by the CTA's previous tile; on return it says the
// same of the next tile `cs_next` (-1: none), whose lists this tile
// prefetches into the other half while it works when both fit a half.
template <typename T, int KW, class Wait>
__device__ __forceinline__ bool gather_tile_level(const CaseTab &ct, int cs, const Slots &sl, const PS<T> *A_src,
                                                  double inv_dt, PS<T> *sA, uint32_t *sp_all, PS<T> *spw_all,
                                                  int2 *sband, int stage, Wait wait, GatherPipe &pipe,
                                                  int cs_next) {
    using S = PS<T>;
    // the tile's record, geometry and case: independent loads
    const int4 ti = sl.tinfo[cs];
    const int4 lo = sl.geo_lo[cs], dim = sl.geo_dim[cs];
    const DevCase cd = ct.get(sl.geo_case[cs]);
    const DevGrid &g = cd.g;
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    T *const u = (T *)cd.u;
    T *const f_out = (T *)cd.f;
    const uint32_t pb = (uint32_t)ti.x;
    const int np = ti.y, nb = ti.z, nc = ti.w;
    const uint32_t *cand = sl.cand + dim.w;
    const int2 *band = sl.band + pb;
    const uint32_t *pairs = sl.pairs + pb;
    const S *pwg = (const S *)sl.pw + pb;
    const bool pre = pipe.pre;
    const bool staged = nc <= stage, pstaged = pre || np <= kLevPairs;
    // this tile's lists: the prefetched half, or from the start of the buffer
    const int lbase = pre ? pipe.half * kLevHalf : 0;
    uint32_t *const sp = sp_all + lbase;
    S *const spw = spw_all + lbase;
    const int2 *const sb = sband + (pre ? pipe.half : 0) * kLevBand;
    if (pre) {
        cp_async_wait_all();
        __syncthreads();
    }
    // prefetch the next tile's lists into the other half when both tiles fit one
    pipe.pre = false;
    if (kLevPrefetch<T> && cs_next >= 0 && (pre || np <= kLevHalf)) {
        const int4 tn = sl.tinfo[cs_next];
        if (tn.y <= kLevHalf && tn.z <= kLevBand) {
            const int h = pre ? 1 - pipe.half : 1;
            const uint32_t *pn = sl.pairs + tn.x;
            const S *wn = (const S *)sl.pw + tn.x;
            const int2 *bn = sl.band + tn.x;
            for (int k = threadIdx.x; k < tn.y; k += blockDim.x) {
                cp_async<4>(sp_all + h * kLevHalf + k, pn + k);
                cp_async<(int)sizeof(S)>(spw_all + h * kLevHalf + k, wn + k);
            }
            for (int q = threadIdx.x; q < tn.z; q += blockDim.x) cp_async<8>(sband + h * kLevBand + q, bn + q);
            cp_async_commit();
            pipe.pre = true;
            pipe.half = h;
        }
    }
    auto cell_index = [&](int cell) {
        const int tx = cell & 7, ty = (cell >> 3) & 7, tz = cell >> 6;
        return ((long long)wrap_add(lo.z, tz, g.n[2]) * g.n[1] + wrap_add(lo.y, ty, g.n[1])) * g.n[0] +
               wrap_add(lo.x, tx, g.n[0]);
    };
    // ---- before the wait
    int2 e[2];
    long long c[2];
    T v[2][3];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int q = threadIdx.x + j * blockDim.x;
        e[j] = make_int2(0, 0);
        c[j] = 0;
        v[j][0] = v[j][1] = v[j][2] = T(0);
        if (q < nb) {
            e[j] = pre ? sb[q] : band[q];
            c[j] = cell_index(e[j].x & 0xffff);
            v[j][0] = u[c[j]];
            v[j][1] = u[N + c[j]];
            v[j][2] = u[2 * N + c[j]];
        }
    }
    if (pstaged && !pre)
        for (int k = threadIdx.x; k < np; k += blockDim.x) {
            sp[k] = __ldg(pairs + k);
            spw[k] = __ldg(pwg + k);
        }
    const uint32_t m0 = (staged && (int)threadIdx.x < nc) ? cand[threadIdx.x] : 0u;
    // ---- the interpolation's sources
    if (!wait()) return false;
    if (staged)
        for (int i = threadIdx.x; i < nc; i += blockDim.x) {
            const uint32_t m = i == (int)threadIdx.x ? m0 : cand[i];
#pragma unroll
            for (int q = 0; q < 3; ++q) sA[4 * i + q] = A_src[4 * (size_t)m + q];
        }
    __syncthreads();
    auto cell_sum = [&](int2 ee, T out[3]) {
        const int cnt = ee.x >> 16;
        SumAcc<T> acc[3];
        auto done = [&]() {
#pragma unroll
            for (int q = 0; q < 3; ++q) out[q] = acc[q].value();
        };
        if (staged && pstaged) {
            // batches of kSB pairs: every shared-memory load of a batch is
            // issued before its sums, which are added in list order
            constexpr int kSB = 4;
            for (int k0 = 0; k0 < cnt; k0 += kSB) {
                uint32_t pk[kSB];
                S wt[kSB], a[kSB][3];
#pragma unroll
                for (int j = 0; j < kSB; ++j) {
                    const bool in = k0 + j < cnt;
                    pk[j] = in ? sp[ee.y + k0 + j] : 0u;
                    wt[j] = in ? spw[ee.y + k0 + j] : S();
                }
#pragma unroll
                for (int j = 0; j < kSB; ++j) {
                    const S *Ai = sA + 4 * (pk[j] & 0xffff);
                    a[j][0] = Ai[0], a[j][1] = Ai[1], a[j][2] = Ai[2];
                }
#pragma unroll
                for (int j = 0; j < kSB; ++j)
                    if (k0 + j < cnt) {
                        acc[0].add(wt[j], a[j][0]);
                        acc[1].add(wt[j], a[j][1]);
                        acc[2].add(wt[j], a[j][2]);
                    }
            }
            done();
            return;
        }
        for (int k = 0; k < cnt; ++k) {
            const uint32_t pk = pstaged ? sp[ee.y + k] : __ldg(pairs + ee.y + k);
            const S wt = pstaged ? spw[ee.y + k] : __ldg(pwg + ee.y + k);
            const int i = pk & 0xffff;
            S a0, a1, a2;
            if (staged) {
                const S *Ai = sA + 4 * i;
                a0 = Ai[0], a1 = Ai[1], a2 = Ai[2];
            } else {
                const S *Ai = A_src + 4 * (size_t)cand[i];
                a0 = Ai[0], a1 = Ai[1], a2 = Ai[2];
            }
            acc[0].add(wt, a0);
            acc[1].add(wt, a1);
            acc[2].add(wt, a2);
        }
        done();
    };
    auto update = [&](long long cc, const T vv[3], const T acc[3]) {
#pragma unroll
        for (int q = 0; q < 3; ++q) u[q * N + cc] = vv[q] + acc[q];
        if (f_out)
#pragma unroll
            for (int q = 0; q < 3; ++q) f_out[q * N + cc] += (T)(acc[q] * inv_dt);
    };
#pragma unroll
    for (int j = 0; j < 2; ++j)
        if ((int)threadIdx.x + j * (int)blockDim.x < nb) {
            T acc[3];
            cell_sum(e[j], acc);
            update(c[j], v[j], acc);
        }
    // cells beyond two per thread (blocks smaller than half a tile)
    for (int q = threadIdx.x + 2 * blockDim.x; q < nb; q += blockDim.x) {
        const int2 ee = pre ? sb[q] : band[q];
        const long long cc = cell_index(ee.x & 0xffff);
        T acc[3];
        cell_sum(ee, acc);
        const T vv[3] = {u[cc], u[N + cc], u[2 * N + cc]};
        update(cc, vv, acc);
    }
    __syncthreads();
    return true;
}

template <typename T, int KER>
__global__ void __launch_bounds__(kGatherThreads, sizeof(T) == 4 ? 5 : 4) k_gather_level(PassArgs<T> a, int L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int stage = a.stage;                             // staged candidates per tile
    PS<T> *sA = (PS<T> *)smem_raw;                         // [stage][4]
    uint32_t *sp = (uint32_t *)(sA + (size_t)stage * 4);   // [kLevPairs]
    PS<T> *spw = (PS<T> *)(sp + kLevPairs);                // [kLevPairs]
    int2 *sband = (int2 *)(spw + kLevPairs);               // [2][kLevBand]
    const int nl = *a.nlev;
    const int s0 = L < nl ? a.lev_sbeg[L] : 0, s1 = L < nl ? a.lev_sbeg[L + 1] : 0;
    if (s0 + (int)blockIdx.x >= s1) {
        grid_dep_wait();
        return;
    }
    // Tiles come largest first.  FP64 sums are bound by FP64 issue, so their
    // rounds alternate direction (boustrophedon): the CTA with the largest tile
    // of one round takes the smallest of the next (measured 4 % faster per
    // step).  FP32 tiles are latency-bound and finish sooner in plain
    // grid-stride order (measured 0.5 %).  Either way, once a round's index
    // passes the end, every later round's does too.
    // (the wait inside returns at once after the first tile)
    constexpr bool kSnake = sizeof(T) == 8;
    const int G = gridDim.x, i = blockIdx.x, nt = s1 - s0;
    auto tile_of = [&](int r) { return (kSnake && (r & 1)) ? (r + 1) * G - 1 - i : r * G + i; };
    GatherPipe pipe{0, false};
    for (int r = 0;; ++r) {
        const int j = tile_of(r);
        if (j >= nt) break;
        const int jn = tile_of(r + 1);
        // FP64 fields: at its last tile the CTA lets the next interpolation be
        // scheduled, so its CTAs load their marker data while the last tiles
        // sum (measured 762 -> 739 us per step; FP32 fields, whose gather
        // ends sooner, measured 553 -> 567 us and keep the trigger at exit)
        if (sizeof(T) == 8 && jn >= nt) grid_dep_launch();
        gather_tile_level<T, Kernel<KER>::W>(
            a.ct, a.tperm[s0 + j], a.sl, a.ms.A, a.inv_dt, sA, sp, spw, sband, stage,
            [] {
                grid_dep_wait();
                return true;
            },
            pipe, jn < nt ? a.tperm[s0 + jn] : -1);
    }
    cp_async_wait_all();  // (a prefetch is only issued for a tile that follows)
}

// The atomic form of a wavefront's spreading (ib_ctx_set_spread_mode):
// every marker of the wavefront adds S A to the field with warp-aggregated
// atomics.  Its position data are loaded before the wait; the sources after.
template <typename T, int KER>
__global__ void __launch_bounds__(256) k_scatter_level(PassArgs<T> a, int L) {
    constexpr int KW = Kernel<KER>::W;
    const int nl = *a.nlev;
    const int m0 = L < nl ? a.lev_mbeg[L] : 0, m1 = L < nl ? a.lev_mbeg[L + 1] : 0;
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    bool waited = false;
    for (long long base = m0 + ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < m1;
         base += nwarps * 32) {
        const long long i = base + lane;
        const bool valid = i < m1;
        const int l = valid ? a.mperm[i] : a.mperm[m0];
        const uint64_t anc = a.ms.anchor[l];
        PS<T> w[12], A[3];
#pragma unroll
        for (int k = 0; k < 12; ++k) w[k] = __ldg(a.ms.wts + 12 * (size_t)l + k);
        const DevCase cd = a.ct.of_particle(a.part_of[l]);
        if (!waited) {
            grid_dep_wait();
            waited = true;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) A[c] = a.ms.A[4 * (size_t)l + c];
        const long long N = (long long)cd.g.n[0] * cd.g.n[1] * cd.g.n[2];
        scatter_marker<T, KW>((T *)cd.u, (T *)cd.f, cd.g, N, anc, w, A, valid, a.inv_dt);
    }
    if (!waited) grid_dep_wait();
}

template <typename T, int KER>
__global__ void __launch_bounds__(256) k_mdf_passes(PassArgs<T> a) {
    constexpr int KW = Kernel<KER>::W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PS<T> *sw = (PS<T> *)smem_raw;                      // [N][12]
    PS<T> *sA = sw + (size_t)TileStage<T>::N * 12;      // [N][4]
    const int nl = *a.nlev;
    const double inv_dt = a.inv_dt;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gsz = gridDim.x * blockDim.x;
    for (int L = a.L0; L < nl; ++L) {
        const int m0 = a.lev_mbeg[L], m1 = a.lev_mbeg[L + 1];
        const int s0 = a.lev_sbeg[L], s1 = a.lev_sbeg[L + 1];
        for (int m = 0; m < a.Ns; ++m) {
            // interpolation phase: U = J u, F += (U^d - U)/dt, A = (U^d - U) dV / h^3
            for (int i = m0 + gtid; i < m1; i += gsz) {
                const int l = a.mperm[i];
                const DevCase cd = a.ct.of_particle(a.part_of[l]);
                const DevGrid &g = cd.g;
                const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
                T U[3];
                interp_marker<T, KW, true>((const T *)cd.u, g, N, a.ms.anchor[l], a.ms.wts + 12 * (size_t)l, U);
                PassMarker<T> pm;
                pm.load(a.ms, a.dV, g.inv_h3, l);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T e = pm.err(c, U[c]);
                    a.F[3 * l + c] = PassMarker<T>::force(a.F[3 * l + c], e, inv_dt);
                    a.ms.A[4 * l + c] = pm.source(e);
                }
            }
            if (!grid_sync(a.bar, a.st)) return;
            if (a.atomic) {
                // atomic spreading of the wavefront's markers (warp-uniform loop)
                const int lane = threadIdx.x & 31;
                const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
                for (long long base = m0 + ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
                     base < m1; base += nwarps * 32) {
                    const long long i = base + lane;
                    const bool valid = i < m1;
                    const int l = valid ? a.mperm[i] : a.mperm[m0];
                    const DevCase cd = a.ct.of_particle(a.part_of[l]);
                    const long long N = (long long)cd.g.n[0] * cd.g.n[1] * cd.g.n[2];
                    PS<T> w[12], A[3];
#pragma unroll
                    for (int k = 0; k < 12; ++k) w[k] = a.ms.wts[12 * (size_t)l + k];
#pragma unroll
                    for (int c = 0; c < 3; ++c) A[c] = a.ms.A[4 * (size_t)l + c];
                    scatter_marker<T, KW>((T *)cd.u, (T *)cd.f, cd.g, N, a.ms.anchor[l], w, A, valid, inv_dt);
                }
            } else {
                // gather phase over the wavefront's tiles (their per-cell lists)
                for (int cs = s0 + blockIdx.x; cs < s1; cs += gridDim.x)
                    gather_tile_lists<T, KW, true>(a.ct, cs, a.sl, a.ms.wts, a.ms.A, inv_dt, sw, sA);
            }
            if (!grid_sync(a.bar, a.st)) return;
        }
    }
    // non-finite result check of the forces (cheap, once)
    for (int l = gtid; l < a.lev_mbeg[nl]; l += gsz) {
        int m = a.mperm[l];
        double fv[3] = {a.F[3 * m], a.F[3 * m + 1], a.F[3 * m + 2]};
        if (!finite3(fv)) raise_status(a.st, IB_ERR_NONFINITE, m);
    }
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
static int grid_blocks(long long work, int threads, int sm) {
    long long b = (work + threads - 1) / threads;
    long long cap = (long long)sm * 8;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

template <typename T>
static bool take_markers(Arena &ar, int M, MarkerState<T> &ms) {
    ms.anchor = ar.take<uint64_t>(M > 0 ? M : 1);
    ms.wts = ar.take<PS<T>>((size_t)12 * (M > 0 ? M : 1));
    ms.A = ar.take<PS<T>>((size_t)4 * (M > 0 ? M : 1));
    ms.Ud = ar.take<double>((size_t)3 * (M > 0 ? M : 1));
    ms.Ud32 = sizeof(T) == 4 ? ar.take<float>((size_t)8 * (M > 0 ? M : 1)) : nullptr;
    return ar.ok();
}

// Slot lists for `M` prepared markers over ndense dense slots, in two steps
// so that a call issues every memset before its kernel chain (the chain's
// kernels are programmatic dependents of one another; a memset in between
// would break it).
struct SlotScratch {
    size_t cand_cap;
    int ncompact_cap;
    int lb_tiles[2];              // look-back tiles of the slot scan and of the pair-count scan
    unsigned long long *lb_stat;  // [lb_tiles[0] + lb_tiles[1]] tile words
    unsigned int *lb_ticket;      // [2]
};

// Workspace of the slot lists, and the zeroing they need.
template <typename T, int KW>
static int slots_alloc(Arena &ar, int M, int ndense, int mode, Slots &sl, SlotScratch &sc, cudaStream_t s,
                       bool with_pairs, bool with_bins) {
    const size_t per = mode == 0 ? 27 : 8;
    sc.cand_cap = (size_t)M * per + 1;
    sc.ncompact_cap = (int)((size_t)M * per < (size_t)ndense ? (size_t)M * per : (size_t)ndense);
    if (sc.ncompact_cap < 1) sc.ncompact_cap = 1;
    const int ncap = sc.ncompact_cap;
    sl.count = ar.take<uint32_t>(ndense);
    sl.start = ar.take<uint32_t>(ndense + 1);
    sl.cursor = ar.take<uint32_t>(ndense);
    sl.flag_scan = ar.take<uint32_t>(ndense + 1);
    sc.lb_tiles[0] = ndense / kLbTile + 1;
    sc.lb_tiles[1] = with_pairs ? (int)(sc.cand_cap / kLbTile) + 1 : 0;
    sc.lb_stat = ar.take<unsigned long long>((size_t)sc.lb_tiles[0] + sc.lb_tiles[1]);
    sc.lb_ticket = ar.take<unsigned int>(2);
    sl.dense_of = ar.take<uint32_t>(ncap);
    sl.cand = ar.take<uint32_t>(sc.cand_cap);
    // bin tables: only the particle-resident form walks them
    sl.bins = with_bins ? ar.take<uint16_t>((size_t)ncap * kBins) : nullptr;
    sl.geo_lo = ar.take<int4>(ncap);
    sl.geo_dim = ar.take<int4>(ncap);
    sl.geo_case = ar.take<int>(ncap);
    constexpr int KW3 = KW * KW * KW;
    if (with_pairs) {
        // every stencil cell of every marker is one pair: KW^3 M in total
        sl.pcnt = ar.take<uint32_t>(sc.cand_cap);
        sl.poff = ar.take<uint32_t>(sc.cand_cap + 1);
        sl.band = ar.take<int2>((size_t)KW3 * M);
        sl.pairs = ar.take<uint32_t>((size_t)KW3 * M);
        sl.pw = ar.take<PS<T>>((size_t)KW3 * M);
        sl.nband = ar.take<int>(ncap);
        sl.tinfo = ar.take<int4>(ncap);
    } else {
        sl.pcnt = sl.poff = nullptr;
        sl.band = nullptr;
        sl.pairs = nullptr;
        sl.nband = nullptr;
        sl.tinfo = nullptr;
        sl.pw = nullptr;
    }
    if (!ar.ok())
        return oom_error(ar.used, ar.cap);
    cudaMemsetAsync(sl.count, 0, sizeof(uint32_t) * ndense, s);
    cudaMemsetAsync(sl.cursor, 0, sizeof(uint32_t) * ndense, s);
    cudaMemsetAsync(sc.lb_stat, 0, sizeof(unsigned long long) * (sc.lb_tiles[0] + sc.lb_tiles[1]), s);
    cudaMemsetAsync(sc.lb_ticket, 0, 2 * sizeof(unsigned int), s);
    return IB_OK;
}

// The kernel chain: count, scan, compact, fill, scan, sort, per-cell lists.
template <typename T, int KW>
static int slots_build(ib_ctx *ctx, const CaseTab &ct, int M, int ndense, SlotGeom sg, const uint64_t *anchor,
                       const PS<T> *wts, const int *level, Slots &sl, const SlotScratch &sc, int *&ncompact_dev,
                       cudaStream_t s, bool with_pairs, bool pdl_first = true) {
    const int nb = grid_blocks(M, 256, ctx->sm_count);
    launch_dep(pdl_first, k_slot_count<KW>, dim3(nb), dim3(256), 0, s, ct, M, sg, anchor, sl.count);
    launch_pdl(k_slot_scan, dim3(sc.lb_tiles[0]), dim3(kLbThreads), 0, s, (const uint32_t *)sl.count, ndense,
               sl.start, sl.flag_scan, sl.dense_of, sc.lb_stat, sc.lb_ticket, ctx->status);
    launch_pdl(k_slot_fill<KW>, dim3(nb), dim3(256), 0, s, ct, M, sg, anchor, (const uint32_t *)sl.start,
               sl.cursor, sl.cand, sl.pcnt);
    // the pair counts of the filled candidate positions [0, start[ndense])
    if (with_pairs)
        launch_pdl(k_scan_lb, dim3(sc.lb_tiles[1]), dim3(kLbThreads), 0, s, (const uint32_t *)sl.pcnt,
                   (int)sc.cand_cap, (const uint32_t *)(sl.start + ndense), sl.poff, sc.lb_stat + sc.lb_tiles[0],
                   sc.lb_ticket + 1, ctx->status);
    ncompact_dev = (int *)(sl.flag_scan + ndense);
    // one resident wave (a second wave would only repeat the screening)
    int sper = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sper, k_slot_sort, kBlock, 0);
    launch_pdl(k_slot_sort, dim3(ctx->sm_count * (sper > 0 ? sper : 1)), dim3(kBlock), 0, s, ct, sg.mode,
               sc.ncompact_cap, (const int *)ncompact_dev, sg, (const uint32_t *)sl.dense_of,
               (const uint32_t *)sl.start, anchor, level, sl, ctx->status);
    if (with_pairs) {
        // one resident wave
        int pper = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pper, k_tile_pairs<T, KW>, kPairThreads, 0);
        launch_pdl(k_tile_pairs<T, KW>, dim3(ctx->sm_count * (pper > 0 ? pper : 1)), dim3(kPairThreads), 0, s, ct,
                   sc.ncompact_cap, (const int *)ncompact_dev, sl, anchor, wts);
    }
    return check_launch("slot lists");
}

template <typename T, int KER>
static int run_interpolate(ib_ctx *ctx, const DevGrid &g, const void *u, int M, const double *X,
                           double *U, cudaStream_t s) {
    int nb = grid_blocks(M, 256, ctx->sm_count);
    PhaseTimer tm(ctx, IB_PHASE_INTERP, s);
    k_interpolate<T, KER><<<nb, 256, 0, s>>>(g, (const T *)u, M, X, U, ctx->status);
    return check_launch("ib_interpolate");
}

template <typename T, int KER>
static int run_spread(ib_ctx *ctx, const ib_grid *grid, int M, const double *X, const double *F,
                      const double *dV, void *f, cudaStream_t s) {
    constexpr int KW = Kernel<KER>::W;
    if (ctx->spread_mode == IB_SPREAD_ATOMIC) {
        PhaseTimer tm(ctx, IB_PHASE_SPREAD, s);
        const DevGrid g = make_dev_grid(grid);
        k_spread_atomic<T, KER><<<grid_blocks(M, 256, ctx->sm_count), 256, 0, s>>>(g, M, X, F, dV, (T *)f,
                                                                                 ctx->status);
        return check_launch("ib_spread");
    }
    Arena ar(ctx);
    MarkerState<T> ms;
    take_markers<T>(ar, M, ms);
    const CaseTab ct = single_case(grid, f, nullptr, 0);  // spread into the case's u slot
    const DevGrid &g = ct.one.g;
    SlotGeom sg{};
    sg.mode = 0;
    const long long ndense = ct.ntiles;
    if (ndense > (1LL << 30)) return set_error(IB_ERR_UNSUPPORTED, "grid has too many tiles");
    if (!ar.ok())
        return oom_error(ar.used, ar.cap);
    int nb = grid_blocks(M, 256, ctx->sm_count);
    Slots sl;
    SlotScratch sc;
    int *ncompact = nullptr;
    int rc = slots_alloc<T, KW>(ar, M, (int)ndense, sg.mode, sl, sc, s, true, false);
    if (rc) return rc;
    PhaseTimer tm(ctx, IB_PHASE_SPREAD, s);
    k_prep_spread<T, KER><<<nb, 256, 0, s>>>(g, M, X, F, dV, ms, ctx->status);
    rc = slots_build<T, KW>(ctx, ct, M, (int)ndense, sg, ms.anchor, (const PS<T> *)ms.wts, nullptr, sl, sc, ncompact, s,
                            true);
    if (rc) return rc;
    cudaFuncSetAttribute(k_spread_gather<T, KER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tile_stage_bytes<T>());
    k_spread_gather<T, KER><<<ctx->sm_count * 4, 256, tile_stage_bytes<T>(), s>>>(ct, ncompact, sl, ms.wts, ms.A);
    return check_launch("ib_spread");
}

template <typename T, int KER>
static int run_mdf(ib_ctx *ctx, Arena &ar, const CaseTab &ct, const ib_particles *pp, const ib_markers *mk,
                   int Ns, double dt, int order, double *F_out, cudaStream_t s) {
    constexpr int KW = Kernel<KER>::W;
    int P = pp->P, M = mk->M;
    MarkerState<T> ms;
    take_markers<T>(ar, M, ms);
    double *rho = ar.take<double>(P);
    int4 *box_lo = ar.take<int4>(P);
    int4 *box_dim = ar.take<int4>(P);
    int *part_of = ar.take<int>(M > 0 ? M : 1);
    PrepScratch prep_ps;
    prep_ps.lo = ar.take<long long>((size_t)3 * P);
    prep_ps.hi = ar.take<long long>((size_t)3 * P);
    prep_ps.done = ar.take<unsigned int>(P);
    LevelOut lo;
    lo.level = ar.take<int>(P);
    lo.rank = ar.take<int>(P);
    lo.mbase = ar.take<int>(P);
    lo.lev_pbeg = ar.take<int>(P + 1);
    lo.lev_mbeg = ar.take<int>(P + 1);
    lo.nlev = ar.take<int>(1);
    int *lev_work = ar.take<int>(P + 1);  // the particle of each rank
    int *lev_cur = ar.take<int>(P + 1);
    int *nbr_cnt = ar.take<int>(P);
    int *nbr = ar.take<int>((size_t)P * kMaxNbr);
    int *lev_sbeg = ar.take<int>(P + 1);
    int *mperm = ar.take<int>(M > 0 ? M : 1);
    unsigned int *sched = ar.take<unsigned int>(P + 1);  // done counters + ticket
    Barrier bar;
    bar.count = ar.take<unsigned int>(2);
    bar.gen = bar.count + 1;
    SlotGeom sg{};
    sg.mode = order == IB_ORDER_SEQUENTIAL ? 1 : 0;
    const long long ndense = sg.mode == 0 ? ct.ntiles : (long long)P * kLocalSlots;
    if (ndense > (1LL << 30)) return set_error(IB_ERR_UNSUPPORTED, "too many tiles");
    if (!ar.ok())
        return oom_error(ar.used, ar.cap);
    // the particle-resident and particle-group forms serve FP32 fields; FP64
    // fields always run the wavefront form (double-float pass sums)
    const int pass_kernels = sizeof(T) == 4 ? ctx->pass_kernels : IB_PASSES_WAVEFRONT;
    const bool resident = order == IB_ORDER_SEQUENTIAL && pass_kernels == IB_PASSES_RESIDENT;
    // atomic spreading (wavefront form): no tile lists at all
    const bool wavefront = order == IB_ORDER_SIMULTANEOUS || pass_kernels == IB_PASSES_AUTO ||
                           pass_kernels == IB_PASSES_WAVEFRONT;
    const bool atomic = wavefront && ctx->spread_mode == IB_SPREAD_ATOMIC;
    Slots sl{};
    SlotScratch sc{};
    int rc = IB_OK;
    int *tperm = nullptr;
    if (!atomic) {
        rc = slots_alloc<T, KW>(ar, M, (int)ndense, sg.mode, sl, sc, s, true, resident);
        if (rc) return rc;
        tperm = ar.take<int>(sc.ncompact_cap);
    }
    if (!ar.ok())
        return oom_error(ar.used, ar.cap);
    PassArgs<T> a;
    a.ct = ct;
    a.part_of = part_of;
    a.F = F_out;
    a.dV = mk->dV;
    a.ms = ms;
    a.sl = sl;
    a.mperm = mperm;
    a.lev_mbeg = lo.lev_mbeg;
    a.lev_sbeg = lev_sbeg;
    a.tperm = tperm;
    a.nlev = lo.nlev;
    a.Ns = Ns;
    a.dt = dt;
    a.inv_dt = 1.0 / dt;
    a.bar = bar;
    a.st = ctx->status;
    a.atomic = atomic ? 1 : 0;
    // staging capacity of the wavefront gather (a layout choice: the sums
    // are the same staged or not)
    a.stage = ctx->gather_stage > 0 && ctx->gather_stage < TileStage<T>::N ? ctx->gather_stage : TileStage<T>::N;
    // wavefronts enqueued as separate kernels: the count the last call on this
    // context copied to a pinned host word (read without synchronising: an
    // aligned 4-byte word is either the old or the new count; a short count
    // only leaves more wavefronts to the persistent kernel)
    ctx->nlev_hint = *(volatile int *)ctx->h_nlev;
    const int Lenq = ctx->nlev_hint < P ? ctx->nlev_hint : P;
    a.L0 = Lenq;
    // the level kernels' launch shapes; the first interpolation runs on the
    // context's second stream beside the slot-list kernels (it reads only the
    // field and the prepared markers), and the first gather joins it
    const bool level_path = !(sizeof(T) == 4 && order == IB_ORDER_SEQUENTIAL &&
                              (pass_kernels == IB_PASSES_RESIDENT || pass_kernels == IB_PASSES_GROUPS));
    const bool fork = level_path && Lenq >= 1;
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t ci = {};
    ci.gridDim = dim3(sizeof(T) == 8 && kInterpSplit ? grid_blocks(3LL * M, kInterpThreads, ctx->sm_count)
                                                     : grid_blocks(M, kInterpThreads, ctx->sm_count));
    ci.blockDim = dim3(kInterpThreads);
    ci.stream = s;
    ci.attrs = pdl;
    auto launch_interp = [&](int L, cudaStream_t st, bool dep) {
        ci.stream = st;
        ci.numAttrs = dep ? 1 : 0;
        if constexpr (sizeof(T) == 8 && kInterpSplit)
            cudaLaunchKernelEx(&ci, k_interp_level_c3<T, KER>, a, L);
        else
            cudaLaunchKernelEx(&ci, k_interp_level<T, KER>, a, L);
        ci.stream = s;
    };
    PhaseTimer tprep(ctx, IB_PHASE_MDF_PREP, s);
    // the marker radii, conflict lists, levels and level-major marker order
    // on the second stream, beside the marker preparation (after everything
    // already enqueued on the call's stream, whose earlier work may still use
    // this workspace)
    cudaStream_t fs = ctx->fork_stream;
    cudaEventRecord(ctx->fork_ev[0], s);
    cudaStreamWaitEvent(fs, ctx->fork_ev[0], 0);
    k_marker_radius<<<P, kRadiusThreads, 0, fs>>>(P, pp->Xr, pp->Ur, pp->Wr, pp->marker_offset, mk->R, mk->dV, rho);
    if (order == IB_ORDER_SEQUENTIAL)
        launch_pdl(k_conflicts, dim3(grid_blocks(32 * P, 256, ctx->sm_count)), dim3(256), 0, fs, ct, P, KW,
                   (const double *)pp->Xr, (const double *)rho, nbr_cnt, nbr);
    cudaFuncSetAttribute(k_levels, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLevSmem);
    launch_pdl(k_levels, dim3(1), dim3(kLevThreads), kLevSmem, fs, ct, P, order, KW, (const double *)pp->Xr,
               (const double *)rho, (const int *)pp->marker_offset, (const int *)nbr_cnt, (const int *)nbr, lo,
               lev_work, lev_cur);
    launch_pdl(k_marker_order, dim3(P < ctx->sm_count * 4 ? P : ctx->sm_count * 4), dim3(256), 0, fs, P,
               (const int *)pp->marker_offset, (const int *)lo.mbase, mperm);
    cudaEventRecord(ctx->fork_ev[3], fs);
    cudaMemsetAsync(bar.count, 0, 2 * sizeof(unsigned int), s);
    cudaMemsetAsync(prep_ps.lo, 0x7f, sizeof(long long) * 3 * P, s);
    cudaMemsetAsync(prep_ps.hi, 0x80, sizeof(long long) * 3 * P, s);
    cudaMemsetAsync(prep_ps.done, 0, sizeof(unsigned int) * P, s);
    k_prep_particles<T, KER><<<P * kPrepSplit, 256, 0, s>>>(ct, P, pp->Xr, pp->Ur, pp->Wr, pp->marker_offset, mk->R,
                                                 mk->dV, ms, F_out, box_lo, box_dim, part_of, prep_ps,
                                                 ctx->status);
    // the first interpolation (second stream) needs the prepared markers and
    // the marker order; the slot lists (this stream) need the levels' ranks
    cudaEventRecord(ctx->fork_ev[2], s);
    if (fork) {
        cudaStreamWaitEvent(fs, ctx->fork_ev[2], 0);
        if (ctx->field_wait) cudaStreamWaitEvent(fs, (cudaEvent_t)ctx->field_wait, 0);
        launch_interp(0, fs, false);
        cudaEventRecord(ctx->fork_ev[1], fs);
    }
    cudaStreamWaitEvent(s, ctx->fork_ev[3], 0);
    sg.part_of = part_of;
    sg.rank = lo.rank;
    sg.box_lo = box_lo;
    sg.box_dim = box_dim;
    int *ncompact = nullptr;
    if (!atomic) {
        rc = slots_build<T, KW>(ctx, ct, M, (int)ndense, sg, ms.anchor, (const PS<T> *)ms.wts, lo.level, sl, sc,
                                ncompact, s, true, false);
        if (rc) return rc;
        a.sl = sl;
    }
    if constexpr (sizeof(T) == 4) {
    if (order == IB_ORDER_SEQUENTIAL &&
        (pass_kernels == IB_PASSES_RESIDENT || pass_kernels == IB_PASSES_GROUPS)) {
        const bool groups = pass_kernels == IB_PASSES_GROUPS;
        const int ngroups = groups ? mdf_groups_count<T, KER>(ctx) : 0;
        if (groups && ngroups < 1) return set_error(IB_ERR_CUDA, "group kernel: no resident group");
        unsigned int *gwords = groups ? ar.take<unsigned int>((size_t)4 * ngroups) : nullptr;
        if (!ar.ok()) return oom_error(ar.used, ar.cap);
        // particle-resident passes: one cluster per particle, scheduled by rank
        ResidentArgs<T> ra;
        ra.ct = ct;
        ra.F = F_out;
        ra.dV = mk->dV;
        ra.ms = ms;
        ra.sl = sl;
        ra.mperm = mperm;
        ra.mbase = lo.mbase;
        ra.moff = pp->marker_offset;
        ra.by_rank = lev_work;  // k_levels leaves the particle of each rank there
        ra.rank = lo.rank;
        ra.level = lo.level;
        ra.box_lo = box_lo;
        ra.nbr_cnt = nbr_cnt;
        ra.nbr = nbr;
        ra.done = sched;
        ra.ticket = sched + P;
        ra.gwords = gwords;
        ra.P = P;
        ra.Ns = Ns;
        ra.dt = dt;
        ra.inv_dt = 1.0 / dt;
        ra.st = ctx->status;
        cudaMemsetAsync(sched, 0, sizeof(unsigned int) * (P + 1), s);
        if (groups) cudaMemsetAsync(gwords, 0, sizeof(unsigned int) * 4 * ngroups, s);
        tprep.stop();
        if (ctx->field_wait) cudaStreamWaitEvent(s, (cudaEvent_t)ctx->field_wait, 0);
        PhaseTimer tpass(ctx, IB_PHASE_MDF_PASSES, s);
        rc = groups ? launch_mdf_groups<T, KER>(ctx, ra, s) : launch_mdf_resident<T, KER>(ctx, ra, s);
        if (rc) return rc;
        tpass.stop();
        return check_launch("ib_multidirect_forcing");
    }
    }
    if (!atomic) {
        launch_pdl(k_level_slots, dim3(1), dim3(256), 0, s, sg.mode, (const int *)lo.nlev,
                   (const int *)lo.lev_pbeg, (const uint32_t *)sl.flag_scan, (int)ndense, lev_sbeg);
        launch_pdl(k_level_tile_order, dim3(P < 64 ? P : 64), dim3(512), 0, s, (const int *)lo.nlev,
                   (const int *)lev_sbeg, (const int *)sl.nband, tperm);
    }
    tprep.stop();
    // (the field is first read and written by the pass kernels below)
    if (ctx->field_wait) cudaStreamWaitEvent(s, (cudaEvent_t)ctx->field_wait, 0);
    // one timed phase: the wavefront kernels and the persistent remainder
    PhaseTimer tpass(ctx, IB_PHASE_MDF_PASSES, s);
    {
        const size_t gsm = level_stage_bytes<T>(a.stage);
        cudaFuncSetAttribute(k_gather_level<T, KER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
        // one resident wave of gather CTAs (grid-stride over the wavefront's tiles)
        int gper = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&gper, k_gather_level<T, KER>, kGatherThreads, gsm);
        if (gper < 1) gper = 1;
        if (ctx->gather_ctas > 0 && ctx->gather_ctas < gper) gper = ctx->gather_ctas;
        // every level kernel after the first is a programmatic dependent of
        // the one before it (see k_interp_level); the first gather instead
        // waits for the interpolation on the second stream
        cudaLaunchConfig_t cg = {};
        cg.gridDim = dim3(ctx->sm_count * gper);
        cg.blockDim = dim3(kGatherThreads);
        cg.dynamicSmemBytes = gsm;
        cg.stream = s;
        cg.attrs = pdl;
        // the atomic form: one lane per marker of the largest wavefront at most
        cudaLaunchConfig_t cs = cg;
        cs.gridDim = dim3(grid_blocks(M, 256, ctx->sm_count));
        cs.blockDim = dim3(256);
        cs.dynamicSmemBytes = 0;
        if (fork) cudaStreamWaitEvent(s, ctx->fork_ev[1], 0);
        for (int L = 0; L < Lenq; ++L)
            for (int m = 0; m < Ns; ++m) {
                const bool first = L == 0 && m == 0;
                if (!first || !fork) {
                    PhaseTimer ti(ctx, IB_PHASE_MDF_INTERP, s);
                    launch_interp(L, s, !first);
                }
                PhaseTimer tg(ctx, IB_PHASE_MDF_GATHER, s);
                cg.numAttrs = cs.numAttrs = first && fork ? 0 : 1;
                if (atomic)
                    cudaLaunchKernelEx(&cs, k_scatter_level<T, KER>, a, L);
                else
                    cudaLaunchKernelEx(&cg, k_gather_level<T, KER>, a, L);
            }
    }
    int per_sm = 0;
    const size_t smem = tile_stage_bytes<T>();
    cudaFuncSetAttribute(k_mdf_passes<T, KER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mdf_passes<T, KER>, 256, smem);
    if (per_sm < 1) return set_error(IB_ERR_CUDA, "mdf kernel cannot be resident");
    int nblocks = per_sm * ctx->sm_count;
    void *args[] = {&a};
    cudaError_t e =
        cudaLaunchCooperativeKernel((const void *)k_mdf_passes<T, KER>, nblocks, 256, args, smem, s);
    if (e != cudaSuccess) return set_error(IB_ERR_CUDA, "mdf launch: %s", cudaGetErrorString(e));
    tpass.stop();
    cudaMemcpyAsync(ctx->h_nlev, lo.nlev, sizeof(int), cudaMemcpyDeviceToHost, s);
    return check_launch("ib_multidirect_forcing");
}

}  // namespace gbib

using namespace gbib;

#define DISPATCH(prec, delta, FN, ...)                                                            \
    ((prec) == IB_F64 ? ((delta) == IB_DELTA_ROMA3 ? FN<double, IB_DELTA_ROMA3>(__VA_ARGS__)      \
                                                   : FN<double, IB_DELTA_PESKIN4>(__VA_ARGS__))   \
                      : ((delta) == IB_DELTA_ROMA3 ? FN<float, IB_DELTA_ROMA3>(__VA_ARGS__)       \
                                                   : FN<float, IB_DELTA_PESKIN4>(__VA_ARGS__)))

extern "C" {

int ib_interpolate(ib_ctx *ctx, const ib_grid *grid, const void *u, int M, const double *X, int delta,
                   double *U, void *stream) {
    if (!ctx) return set_error(IB_ERR_INVALID, "ctx is NULL");
    int rc = validate_grid(grid, 1);
    if (rc) return rc;
    if (delta != IB_DELTA_ROMA3 && delta != IB_DELTA_PESKIN4) return set_error(IB_ERR_INVALID, "bad delta");
    if (M < 0) return set_error(IB_ERR_INVALID, "M < 0");
    if (M == 0) return IB_OK;
    if (!u || !X || !U) return set_error(IB_ERR_INVALID, "NULL array");
    DevGrid g = make_dev_grid(grid);
    return DISPATCH(grid->prec, delta, run_interpolate, ctx, g, u, M, X, U, (cudaStream_t)stream);
}

int ib_spread(ib_ctx *ctx, const ib_grid *grid, int M, const double *X, const double *F, const double *dV,
              int delta, void *f, void *stream) {
    if (!ctx) return set_error(IB_ERR_INVALID, "ctx is NULL");
    int rc = validate_grid(grid, 1);
    if (rc) return rc;
    if (delta != IB_DELTA_ROMA3 && delta != IB_DELTA_PESKIN4) return set_error(IB_ERR_INVALID, "bad delta");
    if (M < 0) return set_error(IB_ERR_INVALID, "M < 0");
    if (M == 0) return IB_OK;
    if (!X || !F || !dV || !f) return set_error(IB_ERR_INVALID, "NULL array");
    return DISPATCH(grid->prec, delta, run_spread, ctx, grid, M, X, F, dV, f, (cudaStream_t)stream);
}

// Arguments shared by the single-case and batch forms; 1 = nothing to do.
static int check_mdf_args(ib_ctx *ctx, const ib_particles *parts, const ib_markers *marks, int Ns, double dt,
                          int delta, int order, const double *F_out) {
    if (!ctx) return set_error(IB_ERR_INVALID, "ctx is NULL");
    if (!parts || !marks) return set_error(IB_ERR_INVALID, "particles/markers NULL");
    if (delta != IB_DELTA_ROMA3 && delta != IB_DELTA_PESKIN4) return set_error(IB_ERR_INVALID, "bad delta");
    if (order != IB_ORDER_SEQUENTIAL && order != IB_ORDER_SIMULTANEOUS)
        return set_error(IB_ERR_INVALID, "bad order");
    if (Ns < 1) return set_error(IB_ERR_INVALID, "Ns must be >= 1");
    if (!(dt > 0.0) || !isfinite(dt)) return set_error(IB_ERR_INVALID, "dt must be finite and > 0");
    if (parts->P < 0 || marks->M < 0) return set_error(IB_ERR_INVALID, "negative P or M");
    if (parts->P == 0 || marks->M == 0) return 1;
    if (!parts->Xr || !parts->Ur || !parts->Wr || !parts->marker_offset || !marks->R || !marks->dV || !F_out)
        return set_error(IB_ERR_INVALID, "NULL array");
    return IB_OK;
}

int ib_multidirect_forcing(ib_ctx *ctx, const ib_grid *grid, void *u, const ib_particles *parts,
                           const ib_markers *marks, int Ns, double dt, int delta, int order, double *F_out,
                           void *f_out, void *stream) {
    int rc = check_mdf_args(ctx, parts, marks, Ns, dt, delta, order, F_out);
    if (rc) return rc == 1 ? IB_OK : rc;
    rc = validate_grid(grid, 1);
    if (rc) return rc;
    if (!u) return set_error(IB_ERR_INVALID, "NULL array");
    const CaseTab ct = single_case(grid, u, f_out, parts->P);
    Arena ar(ctx);
    return DISPATCH(grid->prec, delta, run_mdf, ctx, ar, ct, parts, marks, Ns, dt, order, F_out,
                    (cudaStream_t)stream);
}

int ib_batch_table_multidirect_forcing(ib_ctx *ctx, const ib_batch_table *table, const ib_particles *parts,
                                       const ib_markers *marks, int Ns, double dt, int delta, int order,
                                       double *F_out, void *stream) {
    int rc = check_mdf_args(ctx, parts, marks, Ns, dt, delta, order, F_out);
    if (rc) return rc == 1 ? IB_OK : rc;
    CaseTab ct;
    rc = table_cases(table, parts->P, ct);
    if (rc) return rc;
    Arena ar(ctx);
    return DISPATCH(table->prec, delta, run_mdf, ctx, ar, ct, parts, marks, Ns, dt, order, F_out,
                    (cudaStream_t)stream);
}

int ib_batch_multidirect_forcing(ib_ctx *ctx, int ncases, const ib_case *cases, const ib_particles *parts,
                                 const ib_markers *marks, int Ns, double dt, int delta, int order, double *F_out,
                                 void *stream) {
    int rc = check_mdf_args(ctx, parts, marks, Ns, dt, delta, order, F_out);
    if (rc) return rc == 1 ? IB_OK : rc;
    for (int c = 0; c < ncases && cases; ++c)
        if (!cases[c].u) return set_error(IB_ERR_INVALID, "case %d: NULL field", c);
    Arena ar(ctx);
    CaseTab ct;
    rc = build_case_table(ctx, ar, ncases, cases, parts->P, 1, ct, (cudaStream_t)stream);
    if (rc) return rc;
    return DISPATCH(cases[0].grid.prec, delta, run_mdf, ctx, ar, ct, parts, marks, Ns, dt, order, F_out,
                    (cudaStream_t)stream);
}

}  // extern "C"
