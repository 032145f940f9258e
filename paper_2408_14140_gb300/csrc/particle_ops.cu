// Per-particle reductions and updates around Algorithm 1 (arXiv 2408.14140):
//   * PVF volume integrals (Sec. 4.1, Eqs. level-set function / Heaviside;
//     the flow-unsteadiness terms of Eqs. particle1/particle2),
//   * marker force and torque (first terms of Eqs. particle1/particle2),
//   * repulsive-potential collision (Eq. DKT_model) + Newton-Euler update
//     (Eqs. particle1, particle2) + centroid update (Eq. pr2).
// All sums run in a fixed order (per-thread partials, then fixed warp, CTA
// and cross-CTA orders), so results are bitwise reproducible.  The volume
// integrals' per-cell sums are double-float (FP32 pipes, about 44 significant
// bits) in both field precisions; the force, torque, collision and update
// arithmetic is FP64.
#include <climits>
#include <mutex>
#include <new>

#include "df.cuh"
#include "gbib_internal.cuh"

namespace gbib {

constexpr double kPi = 3.14159265358979323846;

// Fixed-order sum of NV doubles over a CTA of NT threads (NT / 32 >= NV
// warps); result valid in thread 0.  The values go through shared memory and
// warp k sums quantity k (each lane NT / 32 entries, then a shuffle tree):
// NV (NT / 32 + 5) FP64 warp instructions, against NV * 5 per warp for a
// shuffle tree in every warp -- FP64 issue is scarce on this part.
template <int NV, int NT>
__device__ __forceinline__ void block_sum(double v[NV]) {
    static_assert(NT / 32 >= NV, "one warp per quantity");
    __shared__ double red[NV][NT];
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k][threadIdx.x] = v[k];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid < NV) {
        double x = 0.0;
#pragma unroll
        for (int m = 0; m < NT / 32; ++m) x += red[wid][lane + 32 * m];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[wid][0] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = red[k][0];
}

// ---------------------------------------------------------------------------
// volume integrals.  Grid = P * nsplit CTAs; CTA (p, s) walks a slab of
// cell planes of particle p's box.  Per plane it evaluates the level set
// phi = |x - X_r|/R - 1 once per node (only for nodes within 1.75 h of the
// surface: the corners of every cell whose centre lies within 0.8661 h of the
// surface), keeps two node planes in shared memory, and then visits, row by
// row, only the cells whose centre lies within R + 0.8661 h.  Cells whose
// centre lies deeper than R - 0.8661 h have all corners inside (alpha = 1);
// the others form alpha from their eight corner values.  The last CTA of a
// particle (completion counter) adds the nsplit partial sums in slab order.
// ---------------------------------------------------------------------------
constexpr int kVolSplit = 8;       // CTAs per particle of the allocation-free entry point
constexpr int kVolMaxSplit = 32;
constexpr int kVolThreads = 256;   // 8 warps
constexpr int kVolMaxBox = 40;     // cells per axis of one particle's box (tabulated path)
constexpr int kVolAx = kVolMaxBox + 1;
// two node planes of (max(-phi, 0), max(phi, 0)) pairs + per-row grid
// offsets + per-axis tables (cell offsets and node squares as float pairs,
// cell squares in FP32)
constexpr size_t kVolSmem = 2 * kVolAx * kVolAx * sizeof(double2) + kVolAx * sizeof(long long) +
                            6 * kVolAx * sizeof(float2) + 3 * kVolAx * sizeof(float);

// Double-float accumulation: a sum kept as the unevaluated pair hi + lo of two
// floats -- Knuth's TwoSum for the addition error and the fused multiply-add
// for the exact product error (Dekker 1971) -- about 44 significant bits on
// the FP32 pipes, which run 64 times faster than FP64 on GB300.  Used for the
// level set, alpha and the field sums of both field precisions; the per-CTA
// tables and the CTA reduction stay FP64.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ void df_add2(DF &a, float bh, float bl) {
    const float s = a.hi + bh;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (bh - bb);
    a.hi = s;
    a.lo += e + bl;
}
// a += (rh + rl) (wh + wl), keeping the product's rounding error and the
// first-order cross terms
__device__ __forceinline__ void df_add_prod(DF &a, float rh, float rl, float wh, float wl) {
    const float pr = rh * wh;
    const float pe = fmaf(rh, wh, -pr) + fmaf(rh, wl, rl * wh);
    df_add2(a, pr, pe);
}
// hi + lo of every lane added over the warp (fixed shuffle order); result in lane 0
__device__ __forceinline__ void df_warp_sum(DF &a) {
    for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_down_sync(0xffffffffu, a.hi, o), bl = __shfl_down_sync(0xffffffffu, a.lo, o);
        const float lo = a.lo;
        a.lo = 0.f;
        df_add2(a, bh, bl + lo);
    }
}
__device__ __forceinline__ float2 df_split_rn(double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}
// A field value as a float pair: an FP32 value exactly (lo = 0), an FP64 value
// split on the integer pipe (within 2^-47 of the double; no FP64 operation)
__device__ __forceinline__ float2 field_pair(float x) { return make_float2(x, 0.0f); }
__device__ __forceinline__ float2 field_pair(double x) { return df_split(x); }
// a + b, both double-float, renormalised (TwoSum on the high parts)
__device__ __forceinline__ DF df_sum(DF a, DF b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    const float l = e + (a.lo + b.lo);
    const float h = s + l;
    return DF{h, l - (h - s)};
}
// phi = sqrt(x2) * iR - 1 in double-float, x2 > 0: the square root by one
// Newton step from the FP32 reciprocal square root (Heron's iteration; the
// start's relative error below 2^-22 leaves about 2^-45), then the product
// with 1/R and the subtraction.
__device__ __forceinline__ DF df_phi(DF x2, float2 iR) {
    const float rs = rsqrtf(x2.hi);
    const float r = x2.hi * rs;
    const float p = r * r;
    const float pe = fmaf(r, r, -p);
    const float corr = (((x2.hi - p) - pe) + x2.lo) * (0.5f * rs);
    const float q = r * iR.x;
    const float qe = fmaf(r, iR.x, -q) + fmaf(r, iR.y, corr * iR.x);
    return df_sum(DF{q, qe}, DF{-1.0f, 0.0f});
}

// |x| from x^2 to within a few units of FP64 rounding: an FP32 square root
// refined by one Newton step in FP64 (s = s0 + (x2 - s0^2) / (2 s0), the
// classical Heron/Newton iteration; the FP32 start has relative error below
// 2^-22, so one step leaves an error below 2^-44 relative to the FP64 root).
// Cheaper than a full FP64 square root on parts whose FP64 rate is low.
__device__ __forceinline__ double norm_from_square(double x2) {
    const float sf = sqrtf((float)x2);
    if (!(sf > 0.0f)) return sqrt(x2);  // zero, or an FP32 under/overflow: exact path
    const double s0 = (double)sf;
    const double r = fma(-s0, s0, x2);
    return fma(r, (double)(0.5f / sf), s0);
}

// 1/x to within a few units of FP64 rounding: an FP32 reciprocal refined by
// one Newton step (r = r0 + r0 (1 - x r0)), for x in the FP32 normal range.
__device__ __forceinline__ double recip_refined(double x) {
    const double r0 = (double)(1.0f / (float)x);
    return fma(r0, fma(-x, r0, 1.0), r0);
}

// Exclusive scan of cnt[0..n) into pre[0..n] by warp 0 (n may exceed 32).
__device__ __forceinline__ void warp0_scan(const int *cnt, int *pre, int n) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    int carry = 0;
    for (int base = 0; base < n; base += 32) {
        const int v = base + lane < n ? cnt[base + lane] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (base + lane < n) pre[base + lane] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) pre[n] = carry;
}

// Row of flat index t: largest r with pre[r] <= t (pre ascending, pre[0] = 0).
__device__ __forceinline__ int find_row(const int *pre, int nrows, int t) {
    int a = 0, b = nrows - 1;
    while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (pre[mid] <= t) a = mid;
        else b = mid - 1;
    }
    return a;
}

// End of a volume-integral CTA: the fixed-order CTA sum of the 7 partial
// sums, scaled by h^3, is stored as slab `split` of particle p; the last slab
// of the particle to finish (completion counter) adds the nsplit slabs in
// order and writes the particle's integrals.
// s_acc: shared scratch of 7 * kVolThreads doubles (the kernel's dynamic shared
// memory, free again once the CTA's sums are done).
__device__ void volume_finish(double acc[7], double h, int p, int split, int nsplit, double *__restrict__ partial,
                              unsigned int *__restrict__ done, double *Iu, double *Irxu, double *vol, double *s_acc) {
    __shared__ int s_last;
    // fixed-order CTA sum of the 7 partials through shared memory: 7 warps,
    // one per quantity, each lane adding 8 entries then a shuffle tree (FP64
    // adds are scarce on this part: a shuffle tree over all 256 threads would
    // cost more FP64 work than a thin slab's cells)
    {
        __syncthreads();  // every thread is done with the shared memory reused here
#pragma unroll
        for (int k = 0; k < 7; ++k) s_acc[k * kVolThreads + threadIdx.x] = acc[k];
        __syncthreads();
        const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
        if (wq < 7) {
            double x = 0.0;
#pragma unroll
            for (int m = 0; m < kVolThreads / 32; ++m) x += s_acc[wq * kVolThreads + lane + 32 * m];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) s_acc[wq * kVolThreads] = x;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double h3 = h * h * h;
#pragma unroll
            for (int k = 0; k < 7; ++k) acc[k] = s_acc[k * kVolThreads] * h3;
        }
    }
    __shared__ double s_part[kVolMaxSplit * 7];
    if (threadIdx.x == 0) {
        double *dst = partial + ((size_t)p * nsplit + split) * 7;
        for (int k = 0; k < 7; ++k) dst[k] = acc[k];
        __threadfence();  // release: partials before the count
        s_last = atomicAdd(done + p, 1u) == (unsigned int)nsplit - 1;
        __threadfence();  // acquire: the count before the other partials
    }
    __syncthreads();
    if (s_last) {
        // the last CTA of the particle adds the partials in slab order
        for (int i = threadIdx.x; i < nsplit * 7; i += blockDim.x) s_part[i] = partial[(size_t)p * nsplit * 7 + i];
        __syncthreads();
    }
    if (s_last && threadIdx.x == 0) {
        double sum[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int sp = 0; sp < nsplit; ++sp)
            for (int k = 0; k < 7; ++k) sum[k] += s_part[sp * 7 + k];
        if (Iu)
            for (int a = 0; a < 3; ++a) Iu[3 * p + a] = sum[a];
        if (Irxu)
            for (int a = 0; a < 3; ++a) Irxu[3 * p + a] = sum[3 + a];
        if (vol) vol[p] = sum[6];
        done[p] = 0;  // ready for the next call
    }
}

// Most of this kernel's cost is GB300's low FP64 rate, and FP64 pipe time is
// charged per warp instruction whatever the number of active lanes.  So each
// plane is walked as flat lists that keep warps full and uniform:
//   * shell nodes (|x - X_r| within 1.75 h of the surface): phi in FP64;
//   * interior cells (centre deeper than R - 0.8661 h, shrunk by one cell,
//     all corners inside: alpha = 1): plain sums;
//   * boundary cells (the rest within R + 0.8661 h): alpha from the corners.
// Per-row index ranges come from FP32 square roots widened by a cell; every
// node and boundary cell is still tested exactly in FP64.
// A kept volume plan (particle_volume_integrals_keep / _plan): per particle,
// the cells each CTA visits plane by plane in its visiting order -- interior
// cells (alpha = 1) and boundary cells with their alpha, or a skip mark --
// so that a second call at the same particle positions sums another field
// over the same cells with the same alpha without evaluating a level set.
// Capacity `cap` entries per particle and list; a keeping CTA's slab starts
// at dims0 dims1 z0, and each plane's header gives its lists' counts and
// first entries.
struct PvfPlanDev {
    int cap;
    int4 *hdr;        // [P][kVolAx] per plane: interior and boundary counts, first entries
    unsigned *ient;   // [P][cap] interior cell i | j << 16
    unsigned *bent;   // [P][cap] boundary cell i | j << 16, or kPvfSkip
    float2 *balpha;   // [P][cap] boundary alpha as a float pair
    double *pos;      // [P][4] X_r and R the plan was kept for
};
constexpr unsigned kPvfSkip = 0x80000000u;

// MODE 0: plain; 1: also keep the plan (k_volume_plan sums from it).
template <typename T, int MODE = 0>
__global__ void __launch_bounds__(kVolThreads, 3) k_volume(CaseTab ct, int P, int nsplit,
                                                        const double *__restrict__ Xr,
                                                        const double *__restrict__ radius,
                                                        double *__restrict__ partial,
                                                        unsigned int *__restrict__ done, double *Iu,
                                                        double *Irxu, double *vol, DevStatus *st,
                                                        PvfPlanDev pl = PvfPlanDev{}) {
    extern __shared__ __align__(16) double s_vol[];
    // per-row work lists (rows <= kVolAx)
    __shared__ int r_na[kVolAx], r_nb[kVolAx], r_nc[2][kVolAx], r_ca[kVolAx], r_cb[kVolAx];
    __shared__ int r_ia[kVolAx], r_ib[kVolAx], r_ic[kVolAx];
    __shared__ int p_node[kVolAx + 1], p_int[kVolAx + 1], p_bnd[kVolAx + 1];
    __shared__ int c_node[kVolAx], c_int[kVolAx], c_bnd[kVolAx];
    const int p = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
    if (p >= P) return;
    const DevCase &cd = ct.of_particle(p);
    const DevGrid g = cd.g;
    const T *__restrict__ u = (const T *)cd.u;
    // the particle's scalars, formed once by thread 0 (FP64 is scarce here:
    // 256 threads each forming them cost more than a slab's cells)
    __shared__ double s_c[3], s_d[6];
    __shared__ float s_f[4];  // x of node 0 and of cell 0, 1/R as a float pair
    __shared__ int s_box[7];
    if (threadIdx.x == 0) {
        const double cc[3] = {Xr[3 * p], Xr[3 * p + 1], Xr[3 * p + 2]};
        const double R0 = radius[p];
        bool okk = finite3(cc) && isfinite(R0) && R0 > 0.0;
        if (!okk && split == 0) raise_status(st, IB_ERR_NONFINITE, p);
        int lo0[3] = {0, 0, 0}, dm0[3] = {0, 0, 0};
        if (okk) {
            for (int a = 0; a < 3; ++a) {
                long long l = (long long)floor((cc[a] - R0 - g.org[a]) * g.inv_h) - 1;
                long long hgh = (long long)floor((cc[a] + R0 - g.org[a]) * g.inv_h) + 1;
                lo0[a] = (int)l;
                dm0[a] = (int)(hgh - l + 1);
                if (dm0[a] > g.n[a] || l < INT_MIN / 2 || l > INT_MAX / 2) okk = false;
            }
            if (!okk && split == 0) raise_status(st, IB_ERR_UNSUPPORTED, p);
        }
        for (int a = 0; a < 3; ++a) {
            s_c[a] = cc[a];
            s_box[a] = lo0[a];
            s_box[3 + a] = dm0[a];
        }
        if constexpr (MODE != 0) {
            const bool tabbed = dm0[0] <= kVolMaxBox && dm0[1] <= kVolMaxBox && dm0[2] <= kVolMaxBox;
            if (okk && (!tabbed || (long long)dm0[0] * dm0[1] * dm0[2] > pl.cap)) {
                if (split == 0) raise_status(st, IB_ERR_UNSUPPORTED, p);
                okk = false;
            }
            if (split == 0) {
                pl.pos[4 * p] = cc[0], pl.pos[4 * p + 1] = cc[1], pl.pos[4 * p + 2] = cc[2];
                pl.pos[4 * p + 3] = R0;
            }
        }
        s_box[6] = okk;
        if (okk) {
            const double hh = g.h;
            const double rin = R0 - 0.8661 * hh, rout = R0 + 0.8661 * hh;
            const double sl = fmax(0.0, R0 - 1.75 * hh), sh = R0 + 1.75 * hh;
            s_d[0] = R0;
            s_d[1] = 1.0 / R0;
            s_d[2] = rin > 0 ? rin * rin : -1.0;
            s_d[3] = rout * rout;
            s_d[4] = sl * sl;
            s_d[5] = sh * sh;
            s_f[0] = (float)(g.org[0] + (double)lo0[0] * hh - cc[0]);
            s_f[1] = (float)(g.org[0] + ((double)lo0[0] + 0.5) * hh - cc[0]);
            const float2 ir = df_split_rn(s_d[1]);
            s_f[2] = ir.x;
            s_f[3] = ir.y;
        }
    }
    __syncthreads();
    const double c[3] = {s_c[0], s_c[1], s_c[2]};
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const bool ok = s_box[6] != 0;
    const int lo[3] = {s_box[0], s_box[1], s_box[2]}, dims[3] = {s_box[3], s_box[4], s_box[5]};
    const int t = (dims[2] + nsplit - 1) / nsplit;
    const int z0 = split * t, z1 = min(dims[2], z0 + t);
    if (ok && z0 < z1) {
        const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
        const double h = g.h, iR = s_d[1];
        const double rin2 = s_d[2], rout2 = s_d[3];
        const double sl2 = s_d[4], sh2 = s_d[5];
        const int lo0w = wrap_int(lo[0], g.n[0]);
        const bool tab = dims[0] <= kVolMaxBox && dims[1] <= kVolMaxBox && dims[2] <= kVolMaxBox;
        if (tab) {
            const int nx = dims[0] + 1, plane = nx * (dims[1] + 1);
            double2 *phi2 = (double2 *)s_vol;  // node planes: (max(-phi, 0), max(phi, 0))
            long long *row_off = (long long *)(phi2 + 2 * kVolAx * kVolAx);
            float2 *tbf = (float2 *)(row_off + kVolAx);  // cell offsets as float pairs
            float2 *tsq = tbf + 3 * kVolAx;               // node offset squares as float pairs
            float *tcf = (float *)(tsq + 3 * kVolAx);     // cell offset squares in FP32
            for (int a = 0; a < 3; ++a)
                for (int i = threadIdx.x; i <= dims[a]; i += blockDim.x) {
                    const double xc = g.org[a] + ((double)(lo[a] + i) + 0.5) * h - c[a];
                    const double xn = g.org[a] + (double)(lo[a] + i) * h - c[a];
                    tbf[a * kVolAx + i] = df_split_rn(xc);
                    tsq[a * kVolAx + i] = df_split_rn(xn * xn);
                    tcf[a * kVolAx + i] = (float)(xc * xc);
                }
            const float2 iRf = make_float2(s_f[2], s_f[3]);
            // FP32 centre tests with a relative margin far above their rounding;
            // cells in the margin take the corner formula, exact for them too
            const float rout2f = (float)rout2 * (1.0f + 1e-5f);
            const float rin2f = rin2 > 0 ? (float)rin2 * (1.0f - 1e-5f) : -1.0f;
            for (int j = threadIdx.x; j < dims[1]; j += blockDim.x)
                row_off[j] = (long long)wrap_int(lo[1] + j, g.n[1]) * g.n[0];
            __syncthreads();
            const float fih = (float)g.inv_h;
            // Index ranges of positions x_i = base + i h, i in [0, n), from FP32
            // bounds with a margin of kEps cells -- far above the FP32 error of
            // the bounds (< 1e-4 cells on grids up to 1024^3), so that every
            // exact member is listed (range_out: |x_i| <= w) or every listed
            // index is an exact member (range_in: |x_i| < w); empty when
            // first > last.  Exact FP64 tests decide the cells in the margin.
            constexpr float kEps = 1e-3f;
            auto range_out = [&](float base, float w, int n, int &first, int &last) {
                first = max(0, (int)ceilf((-w - base) * fih - kEps));
                last = min(n - 1, (int)floorf((w - base) * fih + kEps));
            };
            auto range_in = [&](float base, float w, int n, int &first, int &last) {
                first = max(0, (int)floorf((-w - base) * fih + kEps) + 1);
                last = min(n - 1, (int)ceilf((w - base) * fih - kEps) - 1);
            };
            const float xbf = s_f[0], xcbf = s_f[1];  // x of node 0 and of cell 0
            // FP32 fields: the per-row ranges from FP32 squares, the shell and
            // the cell bounds widened by a relative 1e-5 (the rows and cells
            // that matter lie 0.01 h inside the node shell and 8e-5 h inside
            // the cell bounds, far beyond the FP32 error of the squares)
            const float sh2f = (float)sh2 * (1.0f + 1e-5f), sl2f = (float)sl2 * (1.0f - 1e-5f);
            auto node_plane = [&](int kn, double2 *buf) {
                const int rows = dims[1] + 1;
                for (int j = threadIdx.x; j < rows; j += blockDim.x) {
                    bool in_shell, beyond_sl;
                    float wo, wi;
                    {
                        const float dyz = tsq[kVolAx + j].x + tsq[2 * kVolAx + kn].x;
                        in_shell = dyz < sh2f;
                        beyond_sl = sl2f > dyz;
                        wo = sqrtf(fmaxf(sh2f - dyz, 0.f));
                        wi = sqrtf(fmaxf(sl2f - dyz, 0.f));
                    }
                    int a0 = 0, n0 = 0, a1 = 0, n1 = 0;
                    if (in_shell) {
                        // nodes of the shell sl <= |x| <= sh: the outer range minus
                        // the nodes surely inside sl
                        int f, l, fi = 1, li = 0;
                        range_out(xbf, wo, nx, f, l);
                        if (beyond_sl) range_in(xbf, wi, nx, fi, li);
                        if (li >= fi && l >= f) {
                            a0 = f;
                            n0 = max(0, min(l, fi - 1) - f + 1);
                            a1 = max(li + 1, f);
                            n1 = max(0, l - a1 + 1);
                        } else {
                            a0 = f;
                            n0 = max(0, l - f + 1);
                        }
                    }
                    r_na[j] = a0, r_nc[0][j] = n0, r_nb[j] = a1, r_nc[1][j] = n1;
                    c_node[j] = n0 + n1;
                }
                __syncthreads();
                warp0_scan(c_node, p_node, rows);
                __syncthreads();
                const int tot = p_node[rows];
                for (int q = threadIdx.x; q < tot; q += blockDim.x) {
                    const int j = find_row(p_node, rows, q);
                    const int k = q - p_node[j];
                    const int i = k < r_nc[0][j] ? r_na[j] + k : r_nb[j] + (k - r_nc[0][j]);
                    // every listed node gets its level set value (nodes slightly
                    // outside the shell too: the values stay exact)
                    {
                        // double-float level set, stored as
                        // (max(-phi, 0), max(phi, 0)) float pairs
                        const DF x2 = df_sum(DF{tsq[i].x, tsq[i].y},
                                             df_sum(DF{tsq[kVolAx + j].x, tsq[kVolAx + j].y},
                                                    DF{tsq[2 * kVolAx + kn].x, tsq[2 * kVolAx + kn].y}));
                        const DF ph = x2.hi > 0.0f ? df_phi(x2, iRf) : DF{-1.0f, 0.0f};
                        ((float4 *)buf)[j * nx + i] = ph.hi < 0.0f ? make_float4(-ph.hi, -ph.lo, 0.f, 0.f)
                                                                   : make_float4(0.f, 0.f, ph.hi, ph.lo);
                    }
                }
            };
            node_plane(z0, phi2 + (z0 & 1) * plane);
            // the CTA's entries in the plan: from dims0 dims1 z0 on, plane by plane
            long long pi = (long long)p * pl.cap + (long long)dims[0] * dims[1] * z0, pb = pi;
            // per-thread double-float sums of w = alpha u, of the six products
            // ry w2, rz w1, rz w0, rx w2, rx w1, ry w0 (r x w = (ry w2 - rz w1,
            // rz w0 - rx w2, rx w1 - ry w0)) and of the boundary cells' alpha;
            // no FP64 operation per cell in either field precision
            long long nint_cells = 0;
            DF W[3] = {}, Pm[6] = {}, V = {};
            for (int kz = z0; kz < z1; ++kz) {
                node_plane(kz + 1, phi2 + ((kz + 1) & 1) * plane);
                // cell rows of plane kz: interior range and the boundary ranges around it
                for (int j = threadIdx.x; j < dims[1]; j += blockDim.x) {
                    bool in_out, in_in;
                    float wo, wi;
                    {
                        const float ryz2 = tcf[kVolAx + j] + tcf[2 * kVolAx + kz];
                        in_out = ryz2 <= rout2f;
                        in_in = ryz2 < rin2f;
                        wo = sqrtf(fmaxf(rout2f - ryz2, 0.f));
                        wi = sqrtf(fmaxf(rin2f - ryz2, 0.f));
                    }
                    int ia = 0, ib = -1, ja = 0, jb = -1;
                    if (in_out) {
                        range_out(xcbf, wo, dims[0], ia, ib);
                        if (in_in) range_in(xcbf, wi, dims[0], ja, jb);
                        ja = max(ja, ia);  // interior within the outer range
                        jb = min(jb, ib);
                    }
                    if (jb < ja) {
                        ja = ib + 1;  // no interior: one boundary interval [ia, ib]
                        jb = ib;
                    }
                    r_ia[j] = ia;
                    r_ib[j] = ib;
                    r_ic[j] = ja;  // interior [ja, jb] with jb stored implicitly by count
                    c_int[j] = jb >= ja ? jb - ja + 1 : 0;
                    r_ca[j] = max(0, min(ja - 1, ib) - ia + 1);   // left boundary [ia, ja-1]
                    r_cb[j] = jb >= ja ? max(0, ib - jb) : 0;      // right boundary [jb+1, ib]
                    c_bnd[j] = r_ca[j] + r_cb[j];
                }
                __syncthreads();
                warp0_scan(c_int, p_int, dims[1]);
                warp0_scan(c_bnd, p_bnd, dims[1]);
                __syncthreads();
                const int nint = p_int[dims[1]], nbnd = p_bnd[dims[1]];
                if (MODE == 1 && threadIdx.x == 0)
                    pl.hdr[p * kVolAx + kz] =
                        make_int4(nint, nbnd, (int)(pi - (long long)p * pl.cap), (int)(pb - (long long)p * pl.cap));
                const double2 *b0 = phi2 + (kz & 1) * plane, *b1 = phi2 + ((kz + 1) & 1) * plane;
                const float2 fz = tbf[2 * kVolAx + kz];
                const float rz2f = tcf[2 * kVolAx + kz];
                const long long plane_off = (long long)wrap_int(lo[2] + kz, g.n[2]) * g.n[1] * g.n[0];
                // interior cells: alpha = 1
                for (int q = threadIdx.x; q < nint; q += blockDim.x) {
                    const int j = find_row(p_int, dims[1], q);
                    const int i = r_ic[j] + (q - p_int[j]);
                    if (MODE == 1) pl.ient[pi + q] = (unsigned)i | ((unsigned)j << 16);
                    const long long cc = plane_off + row_off[j] + wrap_add(lo0w, i, g.n[0]);
                    const float2 fx = tbf[i], fy = tbf[kVolAx + j];
                    const float2 v0 = field_pair(u[cc]), v1 = field_pair(u[N + cc]), v2 = field_pair(u[2 * N + cc]);
                    df_add2(W[0], v0.x, v0.y);
                    df_add2(W[1], v1.x, v1.y);
                    df_add2(W[2], v2.x, v2.y);
                    df_add_prod(Pm[0], fy.x, fy.y, v2.x, v2.y);
                    df_add_prod(Pm[1], fz.x, fz.y, v1.x, v1.y);
                    df_add_prod(Pm[2], fz.x, fz.y, v0.x, v0.y);
                    df_add_prod(Pm[3], fx.x, fx.y, v2.x, v2.y);
                    df_add_prod(Pm[4], fx.x, fx.y, v1.x, v1.y);
                    df_add_prod(Pm[5], fy.x, fy.y, v0.x, v0.y);
                }
                nint_cells += (nint + (int)blockDim.x - 1 - (int)threadIdx.x) / (int)blockDim.x;
                // boundary cells: alpha = sum of max(-phi, 0) / sum |phi| over the corners
                for (int q = threadIdx.x; q < nbnd; q += blockDim.x) {
                    float2 a2 = make_float2(1.f, 0.f);
                    const int j = find_row(p_bnd, dims[1], q);
                    const int k = q - p_bnd[j];
                    const int i = k < r_ca[j] ? r_ia[j] + k : r_ic[j] + c_int[j] + (k - r_ca[j]);
                    if (MODE == 1) pl.bent[pb + q] = kPvfSkip;  // until the cell counts
                    {
                        // the cell's alpha in double-float (both field precisions)
                        const float d2f = tcf[i] + tcf[kVolAx + j] + rz2f;
                        if (d2f > rout2f) continue;
                        if (!(d2f < rin2f)) {
                            const int qn = j * nx + i;
                            const float4 *f0 = (const float4 *)b0, *f1 = (const float4 *)b1;
                            const float4 cn[8] = {f0[qn], f0[qn + 1], f0[qn + nx], f0[qn + nx + 1],
                                                  f1[qn], f1[qn + 1], f1[qn + nx], f1[qn + nx + 1]};
                            DF num = {0.f, 0.f}, neg = {0.f, 0.f};
#pragma unroll
                            for (int m = 0; m < 8; ++m) {
                                df_add2(num, cn[m].x, cn[m].y);
                                df_add2(neg, cn[m].z, cn[m].w);
                            }
                            num = df_sum(num, DF{0.f, 0.f});
                            neg = df_sum(neg, DF{0.f, 0.f});
                            if (num.hi == 0.0f && neg.hi > 0.0f) continue;  // alpha = 0
                            const DF den = df_sum(num, neg);
                            if (den.hi == 0.0f) {
                                a2 = make_float2(0.5f, 0.f);
                            } else if (neg.hi != 0.0f) {
                                if (den.hi < 1e-30f) {
                                    a2 = df_split_rn(((double)num.hi + num.lo) / ((double)den.hi + den.lo));
                                } else {
                                    // num / den: a quotient and one remainder correction
                                    const float rd = __frcp_rn(den.hi);
                                    const float q1 = num.hi * rd;
                                    const float pr = q1 * den.hi;
                                    const float pe = fmaf(q1, den.hi, -pr);
                                    const float rr = ((num.hi - pr) - pe) + fmaf(-q1, den.lo, num.lo);
                                    a2 = make_float2(q1, rr * rd);
                                }
                            }
                        }
                        if constexpr (MODE == 1) {
                            pl.bent[pb + q] = (unsigned)i | ((unsigned)j << 16);
                            pl.balpha[pb + q] = a2;
                        }
                        const long long cc = plane_off + row_off[j] + wrap_add(lo0w, i, g.n[0]);
                        df_add2(V, a2.x, a2.y);
                        const float2 fx = tbf[i], fy = tbf[kVolAx + j];
                        const float2 v[3] = {field_pair(u[cc]), field_pair(u[N + cc]), field_pair(u[2 * N + cc])};
                        float wh[3], wl[3];
#pragma unroll
                        for (int q3 = 0; q3 < 3; ++q3) {
                            // alpha u with the product's rounding error and the cross terms
                            wh[q3] = a2.x * v[q3].x;
                            wl[q3] = fmaf(a2.x, v[q3].x, -wh[q3]) + a2.y * v[q3].x;
                            if constexpr (sizeof(T) == 8) wl[q3] = fmaf(a2.x, v[q3].y, wl[q3]);
                            df_add2(W[q3], wh[q3], wl[q3]);
                        }
                        df_add_prod(Pm[0], fy.x, fy.y, wh[2], wl[2]);
                        df_add_prod(Pm[1], fz.x, fz.y, wh[1], wl[1]);
                        df_add_prod(Pm[2], fz.x, fz.y, wh[0], wl[0]);
                        df_add_prod(Pm[3], fx.x, fx.y, wh[2], wl[2]);
                        df_add_prod(Pm[4], fx.x, fx.y, wh[1], wl[1]);
                        df_add_prod(Pm[5], fy.x, fy.y, wh[0], wl[0]);
                    }
                }
                pi += nint;
                pb += nbnd;
                __syncthreads();
            }
            acc[6] += (double)nint_cells;
            // warp sums in double-float, then FP64 in lane 0 only
#pragma unroll
            for (int q = 0; q < 3; ++q) df_warp_sum(W[q]);
#pragma unroll
            for (int q = 0; q < 6; ++q) df_warp_sum(Pm[q]);
            df_warp_sum(V);
            if ((threadIdx.x & 31) == 0) {
                acc[6] += (double)V.hi + (double)V.lo;
                double pm[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) pm[q] = (double)Pm[q].hi + (double)Pm[q].lo;
#pragma unroll
                for (int q = 0; q < 3; ++q) acc[q] = (double)W[q].hi + (double)W[q].lo;
                acc[3] = pm[0] - pm[1];
                acc[4] = pm[2] - pm[3];
                acc[5] = pm[4] - pm[5];
            }
        } else {
            // boxes wider than kVolMaxBox: every cell of the slab, corners evaluated directly
            for (int kz = z0; kz < z1; ++kz) {
                const int k = lo[2] + kz;
                const double rz = g.org[2] + ((double)k + 0.5) * h - c[2];
                const long long plane_off = (long long)wrap_int(k, g.n[2]) * g.n[1];
                for (int q = threadIdx.x; q < dims[0] * dims[1]; q += blockDim.x) {
                    const int j = q / dims[0], i = q - j * dims[0];
                    const double rx = g.org[0] + ((double)(lo[0] + i) + 0.5) * h - c[0];
                    const double ry = g.org[1] + ((double)(lo[1] + j) + 0.5) * h - c[1];
                    const double d2 = rx * rx + ry * ry + rz * rz;
                    if (d2 > rout2) continue;
                    double al = 1.0;
                    if (!(d2 < rin2)) {
                        double num = 0.0, den = 0.0;
#pragma unroll
                        for (int m = 0; m < 8; ++m) {
                            const double x = g.org[0] + (double)(lo[0] + i + (m & 1)) * h - c[0];
                            const double y = g.org[1] + (double)(lo[1] + j + ((m >> 1) & 1)) * h - c[1];
                            const double z = g.org[2] + (double)(k + ((m >> 2) & 1)) * h - c[2];
                            const double ph = sqrt(x * x + y * y + z * z) * iR - 1.0;
                            if (-ph > 0.0) num += -ph;
                            den += fabs(ph);
                        }
                        al = den > 0.0 ? num / den : 0.5;
                        if (al == 0.0) continue;
                    }
                    const long long cc = (plane_off + wrap_int(lo[1] + j, g.n[1])) * g.n[0] + wrap_add(lo0w, i, g.n[0]);
                    const double u0 = (double)u[cc], u1 = (double)u[N + cc], u2 = (double)u[2 * N + cc];
                    acc[0] += al * u0;
                    acc[1] += al * u1;
                    acc[2] += al * u2;
                    acc[3] += al * (ry * u2 - rz * u1);
                    acc[4] += al * (rz * u0 - rx * u2);
                    acc[5] += al * (rx * u1 - ry * u0);
                    acc[6] += al;
                }
            }
        }
    }
    volume_finish(acc, g.h, p, split, nsplit, partial, done, Iu, Irxu, vol, s_vol);
}

// ---------------------------------------------------------------------------
// Volume integrals from a kept plan.  The particle's kept cells -- interior
// cells, and boundary cells with their double-float alpha -- are read as one
// list per particle (the planes' lists in plane order), split evenly over
// nsplit CTAs, each taking a contiguous range.  A thread sums its cells in
// double-float exactly as k_volume does per cell, kPlanUnroll cells at a
// time with their list entries and field values loaded together, so no chain
// of dependent loads runs plane by plane; then warp sums in double-float and
// the CTA's warp sums and the particle's CTA sums in FP64, in order.  The same
// cells, alpha and per-cell arithmetic as k_volume, in another summation
// order.
// ---------------------------------------------------------------------------
constexpr int kPlanUnroll = 4;
constexpr size_t kPlanSmem = 10 * (kVolThreads / 32) * sizeof(float2);  // the warps' sums

template <typename T>
__global__ void __launch_bounds__(kVolThreads, 2) k_volume_plan(CaseTab ct, int P, int nsplit,
                                                              const double *__restrict__ Xr,
                                                              const double *__restrict__ radius,
                                                              double *__restrict__ partial,
                                                              unsigned int *__restrict__ done, double *Iu,
                                                              double *Irxu, double *vol, DevStatus *st,
                                                              PvfPlanDev pl) {
    extern __shared__ __align__(16) double s_vol[];
    __shared__ float2 tbf[3 * kVolAx];  // cell-centre offsets from X_r as float pairs
    __shared__ long long row_off[kVolAx], plane_off[kVolAx];
    __shared__ int c_int[kVolAx], c_bnd[kVolAx], b_int[kVolAx], b_bnd[kVolAx];
    __shared__ int p_int[kVolAx + 1], p_bnd[kVolAx + 1];
    __shared__ double s_c[3];
    __shared__ int s_box[7];
    const int p = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
    if (p >= P) return;
    const DevCase &cd = ct.of_particle(p);
    const DevGrid g = cd.g;
    const T *__restrict__ u = (const T *)cd.u;
    // the plan's plane headers, loaded beside the particle's scalars (every
    // particle has kVolAx header slots; only the box's planes are read)
    for (int k = threadIdx.x; k < kVolAx; k += blockDim.x) {
        const int4 hc = pl.hdr[p * kVolAx + k];
        c_int[k] = hc.x;
        c_bnd[k] = hc.y;
        b_int[k] = hc.z;
        b_bnd[k] = hc.w;
    }
    if (threadIdx.x == 0) {
        // the particle's box as the keeping call formed it, once the plan is
        // known to be this particle's
        const double cc[3] = {Xr[3 * p], Xr[3 * p + 1], Xr[3 * p + 2]};
        const double R0 = radius[p];
        const double *q = pl.pos + 4 * p;
        bool okk = q[0] == cc[0] && q[1] == cc[1] && q[2] == cc[2] && q[3] == R0;
        if (!okk && split == 0) raise_status(st, IB_ERR_INVALID, p);  // not the plan's particle
        int lo0[3] = {0, 0, 0}, dm0[3] = {0, 0, 0};
        okk = okk && finite3(cc) && isfinite(R0) && R0 > 0.0;
        if (okk)
            for (int a = 0; a < 3; ++a) {
                const long long l = (long long)floor((cc[a] - R0 - g.org[a]) * g.inv_h) - 1;
                const long long hgh = (long long)floor((cc[a] + R0 - g.org[a]) * g.inv_h) + 1;
                lo0[a] = (int)l;
                dm0[a] = (int)(hgh - l + 1);
                // the keeping call kept only boxes of the tabulated size
                if (dm0[a] > g.n[a] || dm0[a] > kVolMaxBox || l < INT_MIN / 2 || l > INT_MAX / 2) okk = false;
            }
        if (okk && (long long)dm0[0] * dm0[1] * dm0[2] > pl.cap) okk = false;  // not kept (reported then)
        for (int a = 0; a < 3; ++a) {
            s_c[a] = cc[a];
            s_box[a] = lo0[a];
            s_box[3 + a] = dm0[a];
        }
        s_box[6] = okk;
    }
    __syncthreads();
    const bool ok = s_box[6] != 0;
    const int lo[3] = {s_box[0], s_box[1], s_box[2]}, dims[3] = {s_box[3], s_box[4], s_box[5]};
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    if (ok) {
        const double h = g.h;
        for (int a = 0; a < 3; ++a)
            for (int i = threadIdx.x; i <= dims[a]; i += blockDim.x)
                tbf[a * kVolAx + i] = df_split_rn(g.org[a] + ((double)(lo[a] + i) + 0.5) * h - s_c[a]);
        for (int j = threadIdx.x; j < dims[1]; j += blockDim.x)
            row_off[j] = (long long)wrap_int(lo[1] + j, g.n[1]) * g.n[0];
        for (int k = threadIdx.x; k < dims[2]; k += blockDim.x)
            plane_off[k] = (long long)wrap_int(lo[2] + k, g.n[2]) * g.n[1] * g.n[0];
    }
    __syncthreads();
    if (ok) {
        warp0_scan(c_int, p_int, dims[2]);
        warp0_scan(c_bnd, p_bnd, dims[2]);
    }
    __syncthreads();
    DF W[3] = {}, Pm[6] = {}, V = {};
    long long nint_cells = 0;
    if (ok) {
        const int lo0w = wrap_int(lo[0], g.n[0]);
        const long long base = (long long)p * pl.cap;
        const int NI = p_int[dims[2]], NB = p_bnd[dims[2]];
        // interior cells: alpha = 1
        const int i0 = (int)((long long)NI * split / nsplit), i1 = (int)((long long)NI * (split + 1) / nsplit);
        // a thread's entries ascend, so its plane only moves forward
        int kzc = i0 + (int)threadIdx.x < i1 ? find_row(p_int, dims[2], i0 + threadIdx.x) : 0;
        for (int e0 = i0 + threadIdx.x; e0 < i1; e0 += kPlanUnroll * blockDim.x) {
            long long cc[kPlanUnroll];
            int kz[kPlanUnroll];
            unsigned ent[kPlanUnroll];
#pragma unroll
            for (int t = 0; t < kPlanUnroll; ++t) {
                const int e = e0 + t * blockDim.x;
                if (e < i1)
                    while (p_int[kzc + 1] <= e) ++kzc;
                kz[t] = kzc;
                ent[t] = e < i1 ? pl.ient[base + b_int[kzc] + (e - p_int[kzc])] : 0u;
            }
            float2 v[kPlanUnroll][3];
#pragma unroll
            for (int t = 0; t < kPlanUnroll; ++t) {
                const int i = (int)(ent[t] & 0xffffu), j = (int)(ent[t] >> 16);
                cc[t] = plane_off[kz[t]] + row_off[j] + wrap_add(lo0w, i, g.n[0]);
                if (e0 + t * (int)blockDim.x < i1)
#pragma unroll
                    for (int c = 0; c < 3; ++c) v[t][c] = field_pair(u[c * N + cc[t]]);
            }
#pragma unroll
            for (int t = 0; t < kPlanUnroll; ++t) {
                if (e0 + t * (int)blockDim.x >= i1) break;
                const int i = (int)(ent[t] & 0xffffu), j = (int)(ent[t] >> 16);
                const float2 fx = tbf[i], fy = tbf[kVolAx + j], fz = tbf[2 * kVolAx + kz[t]];
                df_add2(W[0], v[t][0].x, v[t][0].y);
                df_add2(W[1], v[t][1].x, v[t][1].y);
                df_add2(W[2], v[t][2].x, v[t][2].y);
                df_add_prod(Pm[0], fy.x, fy.y, v[t][2].x, v[t][2].y);
                df_add_prod(Pm[1], fz.x, fz.y, v[t][1].x, v[t][1].y);
                df_add_prod(Pm[2], fz.x, fz.y, v[t][0].x, v[t][0].y);
                df_add_prod(Pm[3], fx.x, fx.y, v[t][2].x, v[t][2].y);
                df_add_prod(Pm[4], fx.x, fx.y, v[t][1].x, v[t][1].y);
                df_add_prod(Pm[5], fy.x, fy.y, v[t][0].x, v[t][0].y);
                ++nint_cells;
            }
        }
        // boundary cells: the kept alpha (entries of cells with alpha = 0 are marked)
        const int j0 = (int)((long long)NB * split / nsplit), j1 = (int)((long long)NB * (split + 1) / nsplit);
        int kzb = j0 + (int)threadIdx.x < j1 ? find_row(p_bnd, dims[2], j0 + threadIdx.x) : 0;
        for (int e0 = j0 + threadIdx.x; e0 < j1; e0 += kPlanUnroll * blockDim.x) {
            int kz[kPlanUnroll];
            unsigned ent[kPlanUnroll];
            float2 al[kPlanUnroll];
#pragma unroll
            for (int t = 0; t < kPlanUnroll; ++t) {
                const int e = e0 + t * blockDim.x;
                if (e < j1)
                    while (p_bnd[kzb + 1] <= e) ++kzb;
                kz[t] = kzb;
                const long long at = base + b_bnd[kz[t]] + (e - p_bnd[kz[t]]);
                ent[t] = e < j1 ? pl.bent[at] : kPvfSkip;
                al[t] = e < j1 ? pl.balpha[at] : make_float2(0.f, 0.f);
            }
            float2 v[kPlanUnroll][3];
#pragma unroll
            for (int t = 0; t < kPlanUnroll; ++t) {
                if (ent[t] == kPvfSkip) continue;
                const int i = (int)(ent[t] & 0xffffu), j = (int)(ent[t] >> 16);
                const long long cc = plane_off[kz[t]] + row_off[j] + wrap_add(lo0w, i, g.n[0]);
#pragma unroll
                for (int c = 0; c < 3; ++c) v[t][c] = field_pair(u[c * N + cc]);
            }
#pragma unroll
            for (int t = 0; t < kPlanUnroll; ++t) {
                if (ent[t] == kPvfSkip) continue;
                const float2 a2 = al[t];
                const int i = (int)(ent[t] & 0xffffu), j = (int)(ent[t] >> 16);
                df_add2(V, a2.x, a2.y);
                const float2 fx = tbf[i], fy = tbf[kVolAx + j], fz = tbf[2 * kVolAx + kz[t]];
                float wh[3], wl[3];
#pragma unroll
                for (int q3 = 0; q3 < 3; ++q3) {
                    wh[q3] = a2.x * v[t][q3].x;
                    wl[q3] = fmaf(a2.x, v[t][q3].x, -wh[q3]) + a2.y * v[t][q3].x;
                    if constexpr (sizeof(T) == 8) wl[q3] = fmaf(a2.x, v[t][q3].y, wl[q3]);
                    df_add2(W[q3], wh[q3], wl[q3]);
                }
                df_add_prod(Pm[0], fy.x, fy.y, wh[2], wl[2]);
                df_add_prod(Pm[1], fz.x, fz.y, wh[1], wl[1]);
                df_add_prod(Pm[2], fz.x, fz.y, wh[0], wl[0]);
                df_add_prod(Pm[3], fx.x, fx.y, wh[2], wl[2]);
                df_add_prod(Pm[4], fx.x, fx.y, wh[1], wl[1]);
                df_add_prod(Pm[5], fy.x, fy.y, wh[0], wl[0]);
            }
        }
    }
    // warp sums (double-float; the interior count exactly), the CTA's eight
    // warp sums in double-float too, one conversion to FP64 per quantity, and
    // the particle's nsplit CTA sums in FP64, in order (FP64 issue is scarce
    // on this part: no FP64 operation per warp)
#pragma unroll
    for (int q = 0; q < 3; ++q) df_warp_sum(W[q]);
#pragma unroll
    for (int q = 0; q < 6; ++q) df_warp_sum(Pm[q]);
    df_warp_sum(V);
    const unsigned ncell = __reduce_add_sync(0xffffffffu, (unsigned)nint_cells);
    float2 *s_w = (float2 *)s_vol;  // [warps][10] double-float warp sums
    __shared__ unsigned s_ncell[kVolThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) s_w[wid * 10 + q] = make_float2(W[q].hi, W[q].lo);
#pragma unroll
        for (int q = 0; q < 6; ++q) s_w[wid * 10 + 3 + q] = make_float2(Pm[q].hi, Pm[q].lo);
        s_w[wid * 10 + 9] = make_float2(V.hi, V.lo);
        s_ncell[wid] = ncell;
    }
    __syncthreads();
    __shared__ double s_q[10];
    if (threadIdx.x < 10) {
        const int k = threadIdx.x;
        DF x = {0.f, 0.f};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x = df_sum(x, DF{s_w[w * 10 + k].x, s_w[w * 10 + k].y});
        s_q[k] = df_to_double(make_float2(x.hi, x.lo));
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        const int k = threadIdx.x;
        double x;
        if (k < 3) {
            x = s_q[k];
        } else if (k < 6) {
            x = s_q[3 + 2 * (k - 3)] - s_q[4 + 2 * (k - 3)];  // (ry w2 - rz w1, rz w0 - rx w2, rx w1 - ry w0)
        } else {
            unsigned n = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) n += s_ncell[w];
            x = (double)n + s_q[9];
        }
        const double h3 = g.h * g.h * g.h;
        partial[((size_t)p * nsplit + split) * 7 + k] = x * h3;
        __threadfence();  // release: partials before the count
    }
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(done + p, 1u) == (unsigned int)nsplit - 1;
        __threadfence();  // acquire: the count before the other partials
    }
    __syncthreads();
    if (s_last && threadIdx.x < 7) {
        // the particle's last CTA adds the CTA sums in CTA order
        const int k = threadIdx.x;
        double x = 0.0;
        for (int sp = 0; sp < nsplit; ++sp) x += __ldcg(partial + ((size_t)p * nsplit + sp) * 7 + k);
        if (k < 3) {
            if (Iu) Iu[3 * p + k] = x;
        } else if (k < 6) {
            if (Irxu) Irxu[3 * p + k - 3] = x;
        } else if (vol) {
            vol[p] = x;
        }
        if (k == 0) done[p] = 0;  // ready for the next call
    }
}

// ---------------------------------------------------------------------------
// Volume integrals of axis-aligned ellipsoids (semi-axes a, b, c), through
// the level set of Eq. (level-set function of spheroidal geometries).  Grid =
// P * nsplit CTAs, CTA (p, s) walks a slab of cell planes of particle p's
// box: the level set is evaluated once per node into two rolling node planes
// in shared memory, and every cell of the plane forms alpha from its eight
// corners (cells with alpha = 0 are skipped).  Boxes wider than kEllAx - 1
// cells evaluate the corners per cell.  The same sums as the oracle, grouped
// per CTA then per slab.
// ---------------------------------------------------------------------------
constexpr int kEllAx = 65;
constexpr size_t kEllSmem = 2 * (size_t)kEllAx * kEllAx * sizeof(double);
static_assert(kEllSmem >= 7 * kVolThreads * sizeof(double) && kVolSmem >= 7 * kVolThreads * sizeof(double),
              "the CTA sum reuses the dynamic shared memory");

__device__ __forceinline__ double pvf_alpha8(const double ph[8]) {
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        num += fmax(-ph[m], 0.0);
        den += fabs(ph[m]);
    }
    return den > 0.0 ? num / den : 0.5;
}

template <typename T>
__global__ void __launch_bounds__(kVolThreads) k_volume_ellipsoid(CaseTab ct, int P, int nsplit,
                                                                  const double *__restrict__ Xr,
                                                                  const double *__restrict__ axes,
                                                                  double *__restrict__ partial,
                                                                  unsigned int *__restrict__ done, double *Iu,
                                                                  double *Irxu, double *vol, DevStatus *st) {
    extern __shared__ __align__(16) double s_phi[];
    const int p = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
    if (p >= P) return;
    const DevCase cd = ct.of_particle(p);
    const DevGrid g = cd.g;
    const T *__restrict__ u = (const T *)cd.u;
    const double c[3] = {Xr[3 * p], Xr[3 * p + 1], Xr[3 * p + 2]};
    const double ax[3] = {axes[3 * p], axes[3 * p + 1], axes[3 * p + 2]};
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    bool ok = finite3(c) && finite3(ax) && ax[0] > 0.0 && ax[1] > 0.0 && ax[2] > 0.0;
    if (!ok && threadIdx.x == 0 && split == 0) raise_status(st, IB_ERR_NONFINITE, p);
    int lo[3] = {0, 0, 0}, dims[3] = {0, 0, 0};
    if (ok) {
        for (int a = 0; a < 3; ++a) {
            const long long l = (long long)floor((c[a] - ax[a] - g.org[a]) * g.inv_h) - 1;
            const long long hg = (long long)floor((c[a] + ax[a] - g.org[a]) * g.inv_h) + 1;
            lo[a] = (int)l;
            dims[a] = (int)(hg - l + 1);
            if (dims[a] > g.n[a] || l < INT_MIN / 2 || l > INT_MAX / 2) ok = false;
        }
        if (!ok && threadIdx.x == 0 && split == 0) raise_status(st, IB_ERR_UNSUPPORTED, p);
    }
    const int t = (dims[2] + nsplit - 1) / nsplit;
    const int z0 = split * t, z1 = min(dims[2], z0 + t);
    if (ok && z0 < z1) {
        const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
        const double h = g.h;
        const double ia[3] = {1.0 / ax[0], 1.0 / ax[1], 1.0 / ax[2]};
        auto level = [&](int i, int j, int k) {  // node (lo + (i, j, k)): x_node = org + index h
            const double x = (g.org[0] + (double)(lo[0] + i) * h - c[0]) * ia[0];
            const double y = (g.org[1] + (double)(lo[1] + j) * h - c[1]) * ia[1];
            const double z = (g.org[2] + (double)(lo[2] + k) * h - c[2]) * ia[2];
            return sqrt(x * x + y * y + z * z) - 1.0;
        };
        auto add_cell = [&](int i, int j, int k, double al) {
            const long long cc = ((long long)wrap_int(lo[2] + k, g.n[2]) * g.n[1] + wrap_int(lo[1] + j, g.n[1])) *
                                     g.n[0] + wrap_int(lo[0] + i, g.n[0]);
            const double r[3] = {g.org[0] + ((double)(lo[0] + i) + 0.5) * h - c[0],
                                 g.org[1] + ((double)(lo[1] + j) + 0.5) * h - c[1],
                                 g.org[2] + ((double)(lo[2] + k) + 0.5) * h - c[2]};
            const double u0 = (double)u[cc], u1 = (double)u[N + cc], u2 = (double)u[2 * N + cc];
            acc[0] += al * u0;
            acc[1] += al * u1;
            acc[2] += al * u2;
            acc[3] += al * (r[1] * u2 - r[2] * u1);
            acc[4] += al * (r[2] * u0 - r[0] * u2);
            acc[5] += al * (r[0] * u1 - r[1] * u0);
            acc[6] += al;
        };
        const int nx = dims[0] + 1, ny = dims[1] + 1;
        if (nx <= kEllAx && ny <= kEllAx) {
            const int plane = nx * ny;
            auto node_plane = [&](int kn, double *buf) {
                for (int q = threadIdx.x; q < plane; q += blockDim.x) buf[q] = level(q % nx, q / nx, kn);
            };
            node_plane(z0, s_phi + (z0 & 1) * plane);
            for (int kz = z0; kz < z1; ++kz) {
                node_plane(kz + 1, s_phi + ((kz + 1) & 1) * plane);
                __syncthreads();
                const double *b0 = s_phi + (kz & 1) * plane, *b1 = s_phi + ((kz + 1) & 1) * plane;
                for (int q = threadIdx.x; q < dims[0] * dims[1]; q += blockDim.x) {
                    const int j = q / dims[0], i = q - j * dims[0];
                    const int qn = j * nx + i;
                    const double ph[8] = {b0[qn], b0[qn + 1], b0[qn + nx], b0[qn + nx + 1],
                                          b1[qn], b1[qn + 1], b1[qn + nx], b1[qn + nx + 1]};
                    const double al = pvf_alpha8(ph);
                    if (al != 0.0) add_cell(i, j, kz, al);
                }
                __syncthreads();
            }
        } else {
            for (int kz = z0; kz < z1; ++kz)
                for (int q = threadIdx.x; q < dims[0] * dims[1]; q += blockDim.x) {
                    const int j = q / dims[0], i = q - j * dims[0];
                    double ph[8];
#pragma unroll
                    for (int m = 0; m < 8; ++m) ph[m] = level(i + (m & 1), j + ((m >> 1) & 1), kz + ((m >> 2) & 1));
                    const double al = pvf_alpha8(ph);
                    if (al != 0.0) add_cell(i, j, kz, al);
                }
        }
    }
    volume_finish(acc, g.h, p, split, nsplit, partial, done, Iu, Irxu, vol, s_phi);
}

// Drag diagnostic of Eq. FD: F_D = F_ib + rho_f (Iu^{n+1} - Iu^n) / dt.
__global__ void k_drag(int P, const double *__restrict__ Fib, const double *__restrict__ Iu_new,
                       const double *__restrict__ Iu_old, double rho_f, double dt, double *__restrict__ FD) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 3 * P; q += gridDim.x * blockDim.x)
        FD[q] = Fib[q] + rho_f * (Iu_new[q] - Iu_old[q]) / dt;
}

// ---------------------------------------------------------------------------
// force and torque (Sec. 3.2.2): nsplit CTAs per particle, each summing a
// contiguous range of the particle's markers in FP64; with nsplit > 1 the
// particle's last CTA adds the CTAs' partial sums in CTA order (deterministic).
// FP64 issue (two operations per clock per SM) bounds these sums, so each
// particle's markers are spread over kFtSplit CTAs.  The split is a constant:
// a particle's sums do not depend on the other particles of the call (a
// request served alone equals the same request in a batch, bit for bit).
// ---------------------------------------------------------------------------
constexpr int kFtThreads = 256;
constexpr int kFtSplit = 4;
__global__ void __launch_bounds__(kFtThreads) k_force_torque(int P, int nsplit, const int *__restrict__ moff,
                                                             const double *__restrict__ R,
                                                             const double *__restrict__ dV,
                                                             const double *__restrict__ F, double rho_f,
                                                             double *__restrict__ partial,
                                                             unsigned int *__restrict__ done,
                                                             double *__restrict__ Fib, double *__restrict__ Tib) {
    const int p = blockIdx.x / nsplit, part = blockIdx.x % nsplit;
    if (p >= P) return;
    const int m0 = moff[p], nm = moff[p + 1] - m0;
    const int l0 = m0 + (int)((long long)part * nm / nsplit), l1 = m0 + (int)((long long)(part + 1) * nm / nsplit);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int l = l0 + threadIdx.x; l < l1; l += blockDim.x) {
        double gx = F[3 * l] * dV[l], gy = F[3 * l + 1] * dV[l], gz = F[3 * l + 2] * dV[l];
        double rx = R[3 * l], ry = R[3 * l + 1], rz = R[3 * l + 2];
        acc[0] += gx;
        acc[1] += gy;
        acc[2] += gz;
        acc[3] += ry * gz - rz * gy;
        acc[4] += rz * gx - rx * gz;
        acc[5] += rx * gy - ry * gx;
    }
    block_sum<6, kFtThreads>(acc);
    if (threadIdx.x != 0) return;
    if (nsplit > 1) {
        // the particle's last CTA adds the partial sums in CTA order
        double *dst = partial + ((size_t)p * nsplit + part) * 6;
        for (int a = 0; a < 6; ++a) dst[a] = acc[a];
        __threadfence();  // release: partials before the count
        const bool last = atomicAdd(done + p, 1u) == (unsigned int)nsplit - 1;
        __threadfence();  // acquire: the count before the other partials
        if (!last) return;
        for (int a = 0; a < 6; ++a) acc[a] = 0.0;
        for (int k = 0; k < nsplit; ++k)
            for (int a = 0; a < 6; ++a) acc[a] += __ldcg(partial + ((size_t)p * nsplit + k) * 6 + a);
    }
    for (int a = 0; a < 3; ++a) {
        Fib[3 * p + a] = -rho_f * acc[a];
        Tib[3 * p + a] = -rho_f * acc[3 + a];
    }
}

// ---------------------------------------------------------------------------
// collision + Newton-Euler: one thread per particle, pairs in index order
// ---------------------------------------------------------------------------
struct CollideArgs {
    int P;
    CaseTab ct;  // pairs are taken within a case, in the case's periodic box
    double *Xr, *Ur, *Wr;
    const double *radius, *rho_p;
    double dt, inv_dt;  // inv_dt = 1 / dt, formed on the host
    const double *Fib, *Tib, *Iu_new, *Iu_old, *Ir_new, *Ir_old;
    double *Fc_out;
    double *Xnew;  // [P][3] scratch: positions are read by every thread
};

// One warp per particle i; lane k takes j = k, k + 32, ...; the lane partial
// sums are combined by a fixed shuffle tree (deterministic).
__global__ void k_collide_forces(CollideArgs a, double *__restrict__ Fc) {
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= a.P) return;
    const DevCase &cd = a.ct.of_particle(i);
    const ib_phys &ph = cd.phys;
    const double L[3] = {cd.g.n[0] * cd.g.h, cd.g.n[1] * cd.g.h, cd.g.n[2] * cd.g.h};
    const double iL[3] = {1.0 / L[0], 1.0 / L[1], 1.0 / L[2]};
    const double xi[3] = {a.Xr[3 * i], a.Xr[3 * i + 1], a.Xr[3 * i + 2]};
    const double Ri = a.radius[i];
    const double mi = a.rho_p[i] * 4.0 / 3.0 * kPi * Ri * Ri * Ri;
    const double idc = 1.0 / ph.d_c;
    const double gscale = 0.5 * ph.g_coll / ph.eps_c;
    double f[3] = {0, 0, 0};
    for (int j = cd.p0 + lane; j < cd.p1; j += 32) {
        if (j == i) continue;
        double del[3], d2 = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double dd = a.Xr[3 * j + k] - xi[k];
            del[k] = dd - L[k] * rint(dd * iL[k]);
            d2 += del[k] * del[k];
        }
        const double Rj = a.radius[j];
        const double Dc = Ri + Rj + ph.d_c;
        if (d2 < Dc * Dc && d2 > 0.0) {
            const double d = sqrt(d2);
            const double mj = a.rho_p[j] * 4.0 / 3.0 * kPi * Rj * Rj * Rj;
            const double q = (d - Dc) * idc;
            const double coef = -((mi + mj) * gscale) * q * q / d;
#pragma unroll
            for (int k = 0; k < 3; ++k) f[k] += coef * del[k];
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        for (int o = 16; o > 0; o >>= 1) f[k] += __shfl_down_sync(0xffffffffu, f[k], o);
    if (lane == 0)
        for (int k = 0; k < 3; ++k) Fc[3 * i + k] = f[k];
}

__global__ void k_newton_euler(CollideArgs a, const double *__restrict__ Fc, DevStatus *st) {
    grid_dep_wait();  // a programmatic dependent of the collision forces
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.P) return;
    const DevCase &cd = a.ct.of_particle(p);
    const ib_phys &ph = cd.phys;
    double Rp = a.radius[p];
    double V = 4.0 / 3.0 * kPi * Rp * Rp * Rp;
    double m = a.rho_p[p] * V;
    double I = 0.4 * m * Rp * Rp;
    // FP64 divisions are long instruction sequences on a part with two FP64
    // operations per clock per SM: 1/dt comes from the host, dt/m and dt/I
    // are formed once
    const double dtm = a.dt / m, dtI = a.dt / I;
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
        double Un = a.Ur[3 * p + k];
        double rhs = a.Fib[3 * p + k] + ph.rho_f * (a.Iu_new[3 * p + k] - a.Iu_old[3 * p + k]) * a.inv_dt +
                     (a.rho_p[p] - ph.rho_f) * V * ph.g[k] + Fc[3 * p + k];
        double Unew = Un + dtm * rhs;
        double trq = a.Tib[3 * p + k] + ph.rho_f * (a.Ir_new[3 * p + k] - a.Ir_old[3 * p + k]) * a.inv_dt;
        double Wnew = a.Wr[3 * p + k] + dtI * trq;
        double Xnew = a.Xr[3 * p + k] + 0.5 * a.dt * (Unew + Un);
        ok = ok && isfinite(Unew) && isfinite(Wnew) && isfinite(Xnew);
        a.Ur[3 * p + k] = Unew;
        a.Wr[3 * p + k] = Wnew;
        a.Xr[3 * p + k] = Xnew;
        if (a.Fc_out) a.Fc_out[3 * p + k] = Fc[3 * p + k];
    }
    if (!ok) raise_status(st, IB_ERR_NONFINITE, p);
}

// CTAs per particle: the context's choice, or (0) as many as fill one resident
// wave of `kern` for P particles, within [1, kVolMaxSplit].
static int volume_split(ib_ctx *ctx, const void *kern, size_t smem, int P) {
    if (ctx->vol_split > 0) return ctx->vol_split;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kVolThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long n = (long long)per_sm * ctx->sm_count / (P > 0 ? P : 1);
    return (int)(n < 1 ? 1 : (n > kVolMaxSplit ? kVolMaxSplit : n));
}

template <typename T>
static int run_volume(ib_ctx *ctx, Arena &ar, const CaseTab &ct, const ib_particles *pp, double *Iu,
                      double *Irxu, double *vol, cudaStream_t s) {
    cudaFuncSetAttribute(k_volume<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVolSmem);
    const int nsplit = volume_split(ctx, (const void *)k_volume<T>, kVolSmem, pp->P);
    double *partial = ar.take<double>((size_t)pp->P * nsplit * 7);
    unsigned int *done = ar.take<unsigned int>(pp->P);
    if (!ar.ok())
        return oom_error(ar.used, ar.cap);
    PhaseTimer tm(ctx, IB_PHASE_VOLUME, s);
    cudaMemsetAsync(done, 0, sizeof(unsigned int) * pp->P, s);
    k_volume<T><<<pp->P * nsplit, kVolThreads, kVolSmem, s>>>(ct, pp->P, nsplit, pp->Xr, pp->radius, partial,
                                                               done, Iu, Irxu, vol, ctx->status);
    return check_launch("particle_volume_integrals");
}

// ---- allocation-free variant: scratch in a fixed device array -------------
// kVolSplit * 7 partial sums per particle for up to IB_STATIC_VOLUME_MAX_P
// particles (2048 * 8 * 7 doubles = 896 KiB).  Host code must not pass the
// array's name to a kernel (that is a host-side stand-in); the device address
// is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) double g_volume_scratch[(size_t)IB_STATIC_VOLUME_MAX_P * kVolSplit * 7];
static __device__ DevStatus g_volume_status;
// completion counters of the final reduction; zero at load, reset by each call
static __device__ unsigned int g_volume_done[IB_STATIC_VOLUME_MAX_P];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static double *g_scratch_ptr[kMaxDevices] = {};
static DevStatus *g_status_ptr[kMaxDevices] = {};
static unsigned int *g_done_ptr[kMaxDevices] = {};

static int static_scratch(double **scratch, DevStatus **status, unsigned int **done) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(IB_ERR_CUDA, "no current CUDA device");
    if (dev < 0 || dev >= kMaxDevices) return set_error(IB_ERR_UNSUPPORTED, "device id %d too large", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr, *q = nullptr, *r = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_volume_scratch);
        if (e != cudaSuccess) return set_error(IB_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        e = cudaGetSymbolAddress(&q, g_volume_status);
        if (e != cudaSuccess) return set_error(IB_ERR_CUDA, "cudaGetSymbolAddress(status): %s", cudaGetErrorString(e));
        e = cudaGetSymbolAddress(&r, g_volume_done);
        if (e != cudaSuccess) return set_error(IB_ERR_CUDA, "cudaGetSymbolAddress(done): %s", cudaGetErrorString(e));
        e = cudaFuncSetAttribute(k_volume<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVolSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_volume<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVolSmem);
        if (e != cudaSuccess) return set_error(IB_ERR_CUDA, "volume kernel attribute: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = (double *)p;
        g_status_ptr[dev] = (DevStatus *)q;
        g_done_ptr[dev] = (unsigned int *)r;
    }
    *scratch = g_scratch_ptr[dev];
    *status = g_status_ptr[dev];
    *done = g_done_ptr[dev];
    return IB_OK;
}

template <typename T>
static int run_volume_static(const CaseTab &ct, const ib_particles *pp, double *Iu,
                             double *Irxu, double *vol, cudaStream_t s) {
    double *partial = nullptr;
    DevStatus *st = nullptr;
    unsigned int *done = nullptr;
    int rc = static_scratch(&partial, &st, &done);
    if (rc) return rc;
    k_volume<T><<<pp->P * kVolSplit, kVolThreads, kVolSmem, s>>>(ct, pp->P, kVolSplit, pp->Xr, pp->radius,
                                                                 partial, done, Iu, Irxu, vol, st);
    return check_launch("particle_volume_integrals_static");
}

template <typename T, int MODE>
static int run_volume_plan(ib_ctx *ctx, Arena &ar, const CaseTab &ct, const ib_particles *pp, int nsplit,
                           const PvfPlanDev &pl, double *Iu, double *Irxu, double *vol, cudaStream_t s) {
    cudaFuncSetAttribute(k_volume<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVolSmem);
    double *partial = ar.take<double>((size_t)pp->P * nsplit * 7);
    unsigned int *done = ar.take<unsigned int>(pp->P);
    if (!ar.ok())
        return oom_error(ar.used, ar.cap);
    PhaseTimer tm(ctx, IB_PHASE_VOLUME, s);
    cudaMemsetAsync(done, 0, sizeof(unsigned int) * pp->P, s);
    k_volume<T, MODE><<<pp->P * nsplit, kVolThreads, kVolSmem, s>>>(ct, pp->P, nsplit, pp->Xr, pp->radius, partial,
                                                                    done, Iu, Irxu, vol, ctx->status, pl);
    return check_launch("particle_volume_integrals_keep");
}

template <typename T>
static int run_plan_sums(ib_ctx *ctx, Arena &ar, const CaseTab &ct, const ib_particles *pp, const PvfPlanDev &pl,
                         double *Iu, double *Irxu, double *vol, cudaStream_t s) {
    const int nsplit = volume_split(ctx, (const void *)k_volume_plan<T>, kPlanSmem, pp->P);
    double *partial = ar.take<double>((size_t)pp->P * nsplit * 7);
    unsigned int *done = ar.take<unsigned int>(pp->P);
    if (!ar.ok())
        return oom_error(ar.used, ar.cap);
    PhaseTimer tm(ctx, IB_PHASE_VOLUME, s);
    cudaMemsetAsync(done, 0, sizeof(unsigned int) * pp->P, s);
    k_volume_plan<T><<<pp->P * nsplit, kVolThreads, kPlanSmem, s>>>(ct, pp->P, nsplit, pp->Xr, pp->radius, partial,
                                                                    done, Iu, Irxu, vol, ctx->status, pl);
    return check_launch("particle_volume_integrals_plan");
}

}  // namespace gbib

using namespace gbib;

// The kept volume plan: device lists and the call it was kept for.
struct ib_pvf_plan {
    int device;
    int P, cap;
    int nsplit;     // CTAs per particle of the keeping call (0: not kept yet)
    ib_grid grid;   // the keeping call's grid
    void *mem;
    PvfPlanDev dev;
};

static bool same_grid(const ib_grid &a, const ib_grid &b) {
    return a.n[0] == b.n[0] && a.n[1] == b.n[1] && a.n[2] == b.n[2] && a.h == b.h && a.origin[0] == b.origin[0] &&
           a.origin[1] == b.origin[1] && a.origin[2] == b.origin[2] && a.prec == b.prec;
}

extern "C" {

int ib_pvf_plan_create(ib_ctx *ctx, int P, int max_box_cells, ib_pvf_plan **plan) {
    if (!ctx || !plan) return set_error(IB_ERR_INVALID, "NULL argument");
    *plan = nullptr;
    if (P < 1 || max_box_cells < 1 || max_box_cells > kVolMaxBox * kVolMaxBox * kVolMaxBox)
        return set_error(IB_ERR_INVALID, "bad plan size (P %d, max_box_cells %d)", P, max_box_cells);
    const size_t cap = (size_t)max_box_cells;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_hdr = up(sizeof(int4) * (size_t)P * kVolAx), b_ient = up(sizeof(unsigned) * P * cap),
                 b_bent = b_ient, b_alpha = up(sizeof(float2) * P * cap), b_pos = up(sizeof(double) * 4 * (size_t)P);
    ib_pvf_plan *pl = new (std::nothrow) ib_pvf_plan();
    if (!pl) return set_error(IB_ERR_OOM, "plan object");
    pl->device = ctx->device;
    pl->P = P;
    pl->cap = max_box_cells;
    pl->nsplit = 0;
    if (cudaMalloc(&pl->mem, b_hdr + b_ient + b_bent + b_alpha + b_pos) != cudaSuccess) {
        cudaGetLastError();
        delete pl;
        return set_error(IB_ERR_OOM, "plan of %zu bytes", b_hdr + b_ient + b_bent + b_alpha + b_pos);
    }
    char *m = (char *)pl->mem;
    pl->dev.cap = max_box_cells;
    pl->dev.hdr = (int4 *)m;
    pl->dev.ient = (unsigned *)(m + b_hdr);
    pl->dev.bent = (unsigned *)(m + b_hdr + b_ient);
    pl->dev.balpha = (float2 *)(m + b_hdr + b_ient + b_bent);
    pl->dev.pos = (double *)(m + b_hdr + b_ient + b_bent + b_alpha);
    *plan = pl;
    return IB_OK;
}

int ib_pvf_plan_destroy(ib_pvf_plan *plan) {
    if (!plan) return IB_OK;
    cudaDeviceSynchronize();
    cudaFree(plan->mem);
    delete plan;
    return IB_OK;
}

int particle_volume_integrals_keep(ib_ctx *ctx, const ib_grid *grid, const void *u, const ib_particles *parts,
                                   ib_pvf_plan *plan, double *Iu, double *Irxu, double *vol, void *stream) {
    if (!ctx || !plan) return set_error(IB_ERR_INVALID, "NULL argument");
    int rc = validate_grid(grid, 1);
    if (rc) return rc;
    if (!parts || parts->P < 0) return set_error(IB_ERR_INVALID, "bad particles");
    if (parts->P != plan->P) return set_error(IB_ERR_INVALID, "plan made for %d particles, not %d", plan->P, parts->P);
    if (!u || !parts->Xr || !parts->radius) return set_error(IB_ERR_INVALID, "NULL array");
    const CaseTab ct = single_case(grid, (void *)u, nullptr, parts->P);
    Arena ar(ctx);
    int nsplit;
    if (grid->prec == IB_F64) {
        cudaFuncSetAttribute(k_volume<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVolSmem);
        nsplit = volume_split(ctx, (const void *)k_volume<double, 1>, kVolSmem, parts->P);
    } else {
        cudaFuncSetAttribute(k_volume<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVolSmem);
        nsplit = volume_split(ctx, (const void *)k_volume<float, 1>, kVolSmem, parts->P);
    }
    plan->nsplit = nsplit;
    plan->grid = *grid;
    if (grid->prec == IB_F64)
        return run_volume_plan<double, 1>(ctx, ar, ct, parts, nsplit, plan->dev, Iu, Irxu, vol, (cudaStream_t)stream);
    return run_volume_plan<float, 1>(ctx, ar, ct, parts, nsplit, plan->dev, Iu, Irxu, vol, (cudaStream_t)stream);
}

int particle_volume_integrals_plan(ib_ctx *ctx, const ib_grid *grid, const void *u, const ib_particles *parts,
                                   const ib_pvf_plan *plan, double *Iu, double *Irxu, double *vol, void *stream) {
    if (!ctx || !plan) return set_error(IB_ERR_INVALID, "NULL argument");
    int rc = validate_grid(grid, 1);
    if (rc) return rc;
    if (!parts || parts->P != plan->P) return set_error(IB_ERR_INVALID, "plan made for %d particles", plan->P);
    if (plan->nsplit < 1) return set_error(IB_ERR_INVALID, "plan not kept yet");
    if (!same_grid(*grid, plan->grid)) return set_error(IB_ERR_INVALID, "grid differs from the plan's");
    if (!u || !parts->Xr || !parts->radius) return set_error(IB_ERR_INVALID, "NULL array");
    const CaseTab ct = single_case(grid, (void *)u, nullptr, parts->P);
    Arena ar(ctx);
    // any split: the plan holds each particle's cells
    if (grid->prec == IB_F64)
        return run_plan_sums<double>(ctx, ar, ct, parts, plan->dev, Iu, Irxu, vol, (cudaStream_t)stream);
    return run_plan_sums<float>(ctx, ar, ct, parts, plan->dev, Iu, Irxu, vol, (cudaStream_t)stream);
}

int particle_volume_integrals(ib_ctx *ctx, const ib_grid *grid, const void *u, const ib_particles *parts,
                              double *Iu, double *Irxu, double *vol, void *stream) {
    if (!ctx) return set_error(IB_ERR_INVALID, "ctx is NULL");
    int rc = validate_grid(grid, 1);
    if (rc) return rc;
    if (!parts || parts->P < 0) return set_error(IB_ERR_INVALID, "bad particles");
    if (parts->P == 0) return IB_OK;
    if (!u || !parts->Xr || !parts->radius) return set_error(IB_ERR_INVALID, "NULL array");
    if ((long long)parts->P * kVolMaxSplit > (1LL << 31) - 1) return set_error(IB_ERR_UNSUPPORTED, "too many particles");
    const CaseTab ct = single_case(grid, (void *)u, nullptr, parts->P);
    Arena ar(ctx);
    if (grid->prec == IB_F64)
        return run_volume<double>(ctx, ar, ct, parts, Iu, Irxu, vol, (cudaStream_t)stream);
    return run_volume<float>(ctx, ar, ct, parts, Iu, Irxu, vol, (cudaStream_t)stream);
}

int ib_batch_volume_integrals(ib_ctx *ctx, int ncases, const ib_case *cases, const ib_particles *parts,
                              double *Iu, double *Irxu, double *vol, void *stream) {
    if (!ctx) return set_error(IB_ERR_INVALID, "ctx is NULL");
    if (!parts || parts->P < 0) return set_error(IB_ERR_INVALID, "bad particles");
    if (parts->P == 0) return IB_OK;
    if (!parts->Xr || !parts->radius || !Iu || !Irxu || !vol) return set_error(IB_ERR_INVALID, "NULL array");
    for (int c = 0; c < ncases && cases; ++c)
        if (!cases[c].u) return set_error(IB_ERR_INVALID, "case %d: NULL field", c);
    if ((long long)parts->P * kVolMaxSplit > (1LL << 31) - 1) return set_error(IB_ERR_UNSUPPORTED, "too many particles");
    Arena ar(ctx);
    CaseTab ct;
    int rc = build_case_table(ctx, ar, ncases, cases, parts->P, 1, ct, (cudaStream_t)stream);
    if (rc) return rc;
    if (cases[0].grid.prec == IB_F64)
        return run_volume<double>(ctx, ar, ct, parts, Iu, Irxu, vol, (cudaStream_t)stream);
    return run_volume<float>(ctx, ar, ct, parts, Iu, Irxu, vol, (cudaStream_t)stream);
}

int particle_volume_integrals_static(const ib_grid *grid, const void *u, const ib_particles *parts,
                                     double *Iu, double *Irxu, double *vol, void *stream) {
    int rc = validate_grid(grid, 1);
    if (rc) return rc;
    if (!parts || parts->P < 0) return set_error(IB_ERR_INVALID, "bad particles");
    if (parts->P > IB_STATIC_VOLUME_MAX_P)
        return set_error(IB_ERR_INVALID, "particle_volume_integrals_static: P = %d exceeds the fixed maximum %d",
                         parts->P, IB_STATIC_VOLUME_MAX_P);
    if (parts->P == 0) return IB_OK;
    if (!u || !parts->Xr || !parts->radius) return set_error(IB_ERR_INVALID, "NULL array");
    const CaseTab ct = single_case(grid, (void *)u, nullptr, parts->P);
    if (grid->prec == IB_F64)
        return run_volume_static<double>(ct, parts, Iu, Irxu, vol, (cudaStream_t)stream);
    return run_volume_static<float>(ct, parts, Iu, Irxu, vol, (cudaStream_t)stream);
}

int particle_volume_integrals_ellipsoid(ib_ctx *ctx, const ib_grid *grid, const void *u, int P, const double *Xr,
                                        const double *axes, double *Iu, double *Irxu, double *vol, void *stream) {
    if (!ctx) return set_error(IB_ERR_INVALID, "ctx is NULL");
    int rc = validate_grid(grid, 1);
    if (rc) return rc;
    if (P < 0) return set_error(IB_ERR_INVALID, "P < 0");
    if (P == 0) return IB_OK;
    if (!u || !Xr || !axes || !Iu || !Irxu || !vol) return set_error(IB_ERR_INVALID, "NULL array");
    if ((long long)P * kVolMaxSplit > (1LL << 31) - 1) return set_error(IB_ERR_UNSUPPORTED, "too many particles");
    const CaseTab ct = single_case(grid, (void *)u, nullptr, P);
    Arena ar(ctx);
    const void *ek = grid->prec == IB_F64 ? (const void *)k_volume_ellipsoid<double> : (const void *)k_volume_ellipsoid<float>;
    cudaFuncSetAttribute(ek, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEllSmem);
    const int nsplit = volume_split(ctx, ek, kEllSmem, P);
    double *partial = ar.take<double>((size_t)P * nsplit * 7);
    unsigned int *done = ar.take<unsigned int>(P);
    if (!ar.ok()) return oom_error(ar.used, ar.cap);
    cudaStream_t s = (cudaStream_t)stream;
    PhaseTimer tm(ctx, IB_PHASE_VOLUME, s);
    cudaMemsetAsync(done, 0, sizeof(unsigned int) * P, s);
    if (grid->prec == IB_F64) {
        cudaFuncSetAttribute(k_volume_ellipsoid<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEllSmem);
        k_volume_ellipsoid<double><<<P * nsplit, kVolThreads, kEllSmem, s>>>(ct, P, nsplit, Xr, axes, partial, done,
                                                                             Iu, Irxu, vol, ctx->status);
    } else {
        cudaFuncSetAttribute(k_volume_ellipsoid<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEllSmem);
        k_volume_ellipsoid<float><<<P * nsplit, kVolThreads, kEllSmem, s>>>(ct, P, nsplit, Xr, axes, partial, done,
                                                                            Iu, Irxu, vol, ctx->status);
    }
    return check_launch("particle_volume_integrals_ellipsoid");
}

int particle_drag_force(ib_ctx *ctx, int P, const double *F_ib, const double *Iu_new, const double *Iu_old,
                        double rho_f, double dt, double *F_D, void *stream) {
    if (!ctx) return set_error(IB_ERR_INVALID, "ctx is NULL");
    if (P < 0) return set_error(IB_ERR_INVALID, "P < 0");
    if (!(dt > 0.0) || !isfinite(dt) || !isfinite(rho_f)) return set_error(IB_ERR_INVALID, "dt or rho_f invalid");
    if (P == 0) return IB_OK;
    if (!F_ib || !Iu_new || !Iu_old || !F_D) return set_error(IB_ERR_INVALID, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (3 * P + 255) / 256;
    k_drag<<<nb < 1024 ? nb : 1024, 256, 0, s>>>(P, F_ib, Iu_new, Iu_old, rho_f, dt, F_D);
    return check_launch("particle_drag_force");
}

int particle_force_torque(ib_ctx *ctx, const ib_particles *parts, const ib_markers *marks, const double *F,
                          double rho_f, double *F_ib, double *T_ib, void *stream) {
    if (!ctx) return set_error(IB_ERR_INVALID, "ctx is NULL");
    if (!parts || !marks || parts->P < 0 || marks->M < 0) return set_error(IB_ERR_INVALID, "bad arguments");
    if (!isfinite(rho_f)) return set_error(IB_ERR_INVALID, "rho_f not finite");
    if (parts->P == 0) return IB_OK;
    if (!parts->marker_offset || !F_ib || !T_ib || (marks->M > 0 && (!marks->R || !marks->dV || !F)))
        return set_error(IB_ERR_INVALID, "NULL array");
    const int P = parts->P, nsplit = kFtSplit;
    cudaStream_t s = (cudaStream_t)stream;
    Arena ar(ctx);
    double *partial = nsplit > 1 ? ar.take<double>((size_t)P * nsplit * 6) : nullptr;
    unsigned int *done = nsplit > 1 ? ar.take<unsigned int>(P) : nullptr;
    if (!ar.ok())
        return oom_error(ar.used, ar.cap);
    PhaseTimer tm(ctx, IB_PHASE_FORCE, s);
    if (done) cudaMemsetAsync(done, 0, sizeof(unsigned int) * P, s);
    k_force_torque<<<P * nsplit, kFtThreads, 0, s>>>(P, nsplit, parts->marker_offset, marks->R, marks->dV, F, rho_f,
                                                   partial, done, F_ib, T_ib);
    return check_launch("particle_force_torque");
}

// Arguments shared by the single-case and batch forms; 1 = nothing to do.
static int check_collide_args(ib_ctx *ctx, const ib_particles *parts, const ib_phys *phys, double dt,
                              const double *F_ib, const double *T_ib, const double *Iu_new, const double *Iu_old,
                              const double *Irxu_new, const double *Irxu_old) {
    if (!ctx) return set_error(IB_ERR_INVALID, "ctx is NULL");
    if (!parts || !phys || parts->P < 0) return set_error(IB_ERR_INVALID, "bad arguments");
    if (!(dt > 0.0) || !isfinite(dt)) return set_error(IB_ERR_INVALID, "dt must be finite and > 0");
    if (!(phys->eps_c > 0.0) || !(phys->d_c > 0.0)) return set_error(IB_ERR_INVALID, "eps_c and d_c must be > 0");
    if (parts->P == 0) return 1;
    if (!parts->Xr || !parts->Ur || !parts->Wr || !parts->radius || !parts->rho_p || !F_ib || !T_ib ||
        !Iu_new || !Iu_old || !Irxu_new || !Irxu_old)
        return set_error(IB_ERR_INVALID, "NULL array");
    return IB_OK;
}

static int run_collide(ib_ctx *ctx, Arena &ar, const CaseTab &ct, ib_particles *parts,
                       double dt, const double *F_ib, const double *T_ib, const double *Iu_new,
                       const double *Iu_old, const double *Irxu_new, const double *Irxu_old, double *Fc_out,
                       cudaStream_t s) {
    double *Fc = ar.take<double>((size_t)3 * parts->P);
    if (!ar.ok())
        return oom_error(ar.used, ar.cap);
    CollideArgs a;
    a.P = parts->P;
    a.ct = ct;
    a.Xr = parts->Xr;
    a.Ur = parts->Ur;
    a.Wr = parts->Wr;
    a.radius = parts->radius;
    a.rho_p = parts->rho_p;
    a.dt = dt;
    a.inv_dt = 1.0 / dt;
    a.Fib = F_ib;
    a.Tib = T_ib;
    a.Iu_new = Iu_new;
    a.Iu_old = Iu_old;
    a.Ir_new = Irxu_new;
    a.Ir_old = Irxu_old;
    a.Fc_out = Fc_out;
    a.Xnew = nullptr;
    // one warp per CTA: both kernels are FP64-issue bound (two operations per
    // clock per SM), so the particles' warps are spread over as many SMs
    PhaseTimer tm(ctx, IB_PHASE_COLLIDE, s);
    k_collide_forces<<<parts->P, 32, 0, s>>>(a, Fc);
    launch_pdl(k_newton_euler, dim3((parts->P + 31) / 32), dim3(32), 0, s, a, (const double *)Fc, ctx->status);
    return check_launch("particle_collide_update");
}

int particle_collide_update(ib_ctx *ctx, ib_particles *parts, const ib_grid *grid, const ib_phys *phys,
                            double dt, const double *F_ib, const double *T_ib, const double *Iu_new,
                            const double *Iu_old, const double *Irxu_new, const double *Irxu_old,
                            double *Fc_out, void *stream) {
    int rc = check_collide_args(ctx, parts, phys, dt, F_ib, T_ib, Iu_new, Iu_old, Irxu_new, Irxu_old);
    if (rc) return rc == 1 ? IB_OK : rc;
    rc = validate_grid(grid, 0);
    if (rc) return rc;
    CaseTab ct = single_case(grid, nullptr, nullptr, parts->P);
    ct.one.phys = *phys;
    Arena ar(ctx);
    return run_collide(ctx, ar, ct, parts, dt, F_ib, T_ib, Iu_new, Iu_old, Irxu_new, Irxu_old, Fc_out,
                       (cudaStream_t)stream);
}

int ib_batch_table_volume_integrals(ib_ctx *ctx, const ib_batch_table *table, const ib_particles *parts,
                                    double *Iu, double *Irxu, double *vol, void *stream) {
    if (!ctx) return set_error(IB_ERR_INVALID, "ctx is NULL");
    if (!parts || parts->P < 0) return set_error(IB_ERR_INVALID, "bad particles");
    CaseTab ct;
    int rc = table_cases(table, parts->P, ct);
    if (rc) return rc;
    if (parts->P == 0) return IB_OK;
    if (!parts->Xr || !parts->radius || !Iu || !Irxu || !vol) return set_error(IB_ERR_INVALID, "NULL array");
    if ((long long)parts->P * kVolMaxSplit > (1LL << 31) - 1) return set_error(IB_ERR_UNSUPPORTED, "too many particles");
    Arena ar(ctx);
    if (table->prec == IB_F64) return run_volume<double>(ctx, ar, ct, parts, Iu, Irxu, vol, (cudaStream_t)stream);
    return run_volume<float>(ctx, ar, ct, parts, Iu, Irxu, vol, (cudaStream_t)stream);
}

int ib_batch_table_collide_update(ib_ctx *ctx, const ib_batch_table *table, ib_particles *parts, double dt,
                                  const double *F_ib, const double *T_ib, const double *Iu_new,
                                  const double *Iu_old, const double *Irxu_new, const double *Irxu_old,
                                  double *Fc_out, void *stream) {
    if (table && !table->has_phys) return set_error(IB_ERR_INVALID, "the table was created without physical parameters");
    const ib_phys *ph = table ? &table->ct.one.phys : nullptr;
    int rc = check_collide_args(ctx, parts, ph, dt, F_ib, T_ib, Iu_new, Iu_old, Irxu_new, Irxu_old);
    if (rc) return rc == 1 ? IB_OK : rc;
    CaseTab ct;
    rc = table_cases(table, parts->P, ct);
    if (rc) return rc;
    Arena ar(ctx);
    return run_collide(ctx, ar, ct, parts, dt, F_ib, T_ib, Iu_new, Iu_old, Irxu_new, Irxu_old, Fc_out,
                       (cudaStream_t)stream);
}

int ib_batch_collide_update(ib_ctx *ctx, int ncases, const ib_case *cases, ib_particles *parts,
                            const ib_phys *phys, double dt, const double *F_ib, const double *T_ib,
                            const double *Iu_new, const double *Iu_old, const double *Irxu_new,
                            const double *Irxu_old, double *Fc_out, void *stream) {
    int rc = check_collide_args(ctx, parts, phys, dt, F_ib, T_ib, Iu_new, Iu_old, Irxu_new, Irxu_old);
    if (rc) return rc == 1 ? IB_OK : rc;
    Arena ar(ctx);
    CaseTab ct;
    for (int c = 0; c < ncases && cases; ++c)
        if (!(phys[c].eps_c > 0.0) || !(phys[c].d_c > 0.0))
            return set_error(IB_ERR_INVALID, "case %d: eps_c and d_c must be > 0", c);
    rc = build_case_table(ctx, ar, ncases, cases, parts->P, 0, ct, (cudaStream_t)stream, phys);
    if (rc) return rc;
    return run_collide(ctx, ar, ct, parts, dt, F_ib, T_ib, Iu_new, Iu_old, Irxu_new, Irxu_old, Fc_out,
                       (cudaStream_t)stream);
}

}  // extern "C"
