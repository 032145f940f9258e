// Device-side pieces shared by the forcing kernels of arXiv 2408.14140,
// Sec. 3.1 Step 2 (Algorithm 1): per-marker state, spreading-tile records,
// one marker's interpolation and one cell's deterministic gather.
#pragma once

#include "df.cuh"
#include "gbib_internal.cuh"

namespace gbib {

// Storage of the per-marker kernel weights and spread sources of a pass:
// the field type for FP32 fields; a double-float pair (hi, lo) for FP64
// fields, whose pass sums run on the FP32 pipes (df.cuh).  Both are the size
// of the field type.
template <typename T> struct PassStore { using type = T; };
template <> struct PassStore<double> { using type = float2; };
template <typename T> using PS = typename PassStore<T>::type;

__device__ __forceinline__ float to_store(float v) { return v; }
__device__ __forceinline__ float2 to_store(double v) { return df_split(v); }

// Product of a pair's three axis weights (w[0..3] x, w[4..7] y, w[8..11] z).
__device__ __forceinline__ float pair_weight(const float *w, int ox, int oy, int oz) {
    return w[ox] * w[4 + oy] * w[8 + oz];
}
__device__ __forceinline__ float2 pair_weight(const float2 *w, int ox, int oy, int oz) {
    return df_mul(df_mul(w[ox], w[4 + oy]), w[8 + oz]);
}

__device__ __forceinline__ float pair_weight3(float wx, float wy, float wz) { return wx * wy * wz; }
__device__ __forceinline__ float2 pair_weight3(float2 wx, float2 wy, float2 wz) {
    return df_mul(df_mul(wx, wy), wz);
}

// Running sum of weight x source products of one cell or marker component.
template <typename T> struct SumAcc;
template <> struct SumAcc<float> {
    float v = 0.0f;
    __device__ __forceinline__ void add(float w, float a) { v += w * a; }
    __device__ __forceinline__ float value() const { return v; }
};
template <> struct SumAcc<double> {
    DFAcc v;
    __device__ __forceinline__ void add(float2 w, float2 a) { v.add_prod(w, a); }
    __device__ __forceinline__ double value() const { return v.value(); }
};

constexpr int kBlock = 512;          // threads per CTA (one per tile cell)
constexpr int kLocalTiles = 8;       // local tiles per axis of a particle box
constexpr int kLocalSlots = kLocalTiles * kLocalTiles * kLocalTiles;
constexpr int kMaxBox = kLocalTiles * kTile;  // 64 cells
// A tile's candidates are sorted by (anchor row, x offset, marker).  Bin
// (row, v), v = x offset + 3 in [0, 10], holds the markers whose first stencil
// cell is at row `row` and x offset v - 3 from the tile; kBins[row * 12 + v]
// is the bin's first candidate and [row * 12 + 11] the row's end, so a cell
// reads exactly the KW^3 bins of its stencil.
constexpr int kBinsPerRow = 12;
// Conflict-list entries kept per particle (more: the list is marked full).
constexpr int kMaxNbr = 48;
// Bounded device-side waits give up after this many SM cycles (~2 s).
constexpr long long kSpinCycles = 4LL * 1000 * 1000 * 1000;  // ~2 s at 2 GHz

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

constexpr int kBins = kRows * kBinsPerRow + 1;

// Per-marker state kept in the workspace for one call.
template <typename T>
struct MarkerState {
    uint64_t *anchor;  // [M] wrapped first stencil cell
    PS<T> *wts;        // [M][12] per-axis weights (x 0..3, y 4..7, z 8..11)
    PS<T> *A;          // [M][4] spread source of the current pass
    double *Ud;        // [M][3] desired velocity
    // FP32 fields only: [M][8] the desired velocity as float pairs, hi
    // (0..2) + lo (4..6), and dV / h^3 (3)
    float *Ud32;
};

// One marker's update in one pass of Algorithm 1, given its interpolated
// velocity U: with the velocity error e = U^d - U, the force F += e / dt
// and the spread source A = e dV / h^3 (the field correction is S A).
// FP64 fields: all in FP64, the source stored as a float pair.  FP32 fields:
// U^d is held as an unevaluated float
// pair hi + lo and e = (hi - U) + lo is formed in FP32, which is within a unit
// roundoff of e (the precision of the interpolated U itself); only the force
// sum stays in FP64.  GB300 runs FP64 at a small fraction of its FP32 rate,
// so this keeps a pass to six FP64 instructions per marker.
template <typename T>
struct PassMarker {
    T hi[3], lo[3], q;
    __device__ __forceinline__ void load(const MarkerState<T> &ms, const double *dV, double inv_h3, int l) {
        if constexpr (sizeof(T) == 8) {
#pragma unroll
            for (int c = 0; c < 3; ++c) hi[c] = __ldg(ms.Ud + 3 * l + c);
            q = dV[l] * inv_h3;
        } else {
            const float4 a = __ldg((const float4 *)(ms.Ud32 + 8 * (size_t)l));
            const float4 b = __ldg((const float4 *)(ms.Ud32 + 8 * (size_t)l) + 1);
            hi[0] = a.x, hi[1] = a.y, hi[2] = a.z, q = a.w;
            lo[0] = b.x, lo[1] = b.y, lo[2] = b.z;
        }
    }
    // velocity error of component c
    __device__ __forceinline__ T err(int c, T U) const {
        if constexpr (sizeof(T) == 8)
            return hi[c] - U;
        else
            return (hi[c] - U) + lo[c];
    }
    // F + e / dt (one FP64 fused multiply-add)
    __device__ __forceinline__ static double force(double F, T e, double inv_dt) {
        return fma((double)e, inv_dt, F);
    }
    __device__ __forceinline__ PS<T> source(T e) const { return to_store(e * q); }
};

// Slot (spreading tile) records.
struct Slots {
    uint32_t *count;   // [ndense] candidates per dense slot
    uint32_t *start;   // [ndense+1] exclusive scan of count
    uint32_t *cursor;  // [ndense] fill cursors
    uint32_t *flag_scan;  // [ndense+1] compact index of non-empty slots
    uint32_t *dense_of;   // [ncompact_max] dense id of each compact slot
    uint32_t *cand;    // [total candidates] marker ids, sorted per slot
    uint16_t *bins;    // [ncompact_max][kBins] bin starts, relative (see kBins)
    int4 *geo_lo;      // [ncompact_max] tile first cell (wrapped), w = level
    int4 *geo_dim;     // [ncompact_max] tile dims, w = first candidate
    int *geo_case;     // [ncompact_max] case of the tile
    // per-cell gather lists (built once per call, see k_tile_pairs).  A
    // candidate contributes one pair per stencil cell inside its tile;
    // poff[i] is the exclusive prefix of those counts over candidate
    // positions, so tile cs with first candidate b owns pairs
    // [poff[b], poff[b + nc]) -- KW^3 M in total.  band[poff[b] + q] =
    // {cell | count << 16, first pair relative to poff[b]} for its q-th band
    // cell (cells in index order), and pairs[poff[b] + k] = candidate | ox << 16
    // | oy << 18 | oz << 20, each cell's pairs in ascending candidate order
    // (the gather order).
    uint32_t *pcnt;    // [cand_cap] in-tile stencil cells of each candidate
    uint32_t *poff;    // [cand_cap + 1] exclusive scan of pcnt
    int2 *band;
    uint32_t *pairs;
    int *nband;        // [ncompact_max] band cells of the tile
    // [ncompact_max] the tile's list record {first pair poff[b], pairs,
    // band cells, candidates}, one load for the wavefront gather
    int4 *tinfo;
    // [KW^3 M] per pair, its weight product pair_weight(w, ox, oy, oz) in the
    // pass-sum type PS<T> (parallel to pairs; nullable)
    void *pw;
};

// ---------------------------------------------------------------------------
// interpolation of one marker from precomputed weights
// ---------------------------------------------------------------------------
// Loads of data that other CTAs of the persistent kernel write between grid
// barriers (COH) are ordinary weak loads: the barrier is a GPU-scope
// release/acquire pattern, so by the PTX memory model every write before it
// is visible to every load after it.  (The read-only path, ld.global.nc, is
// not coherent with writes made during the kernel and is used only for data
// that no kernel writes meanwhile.)  ld.global.cg forms are avoided here:
// they were issued one at a time, serialising ~80 L2 round trips per marker.
template <bool COH, typename T>
__device__ __forceinline__ T ld(const T *p) {
    if (COH) return *p;
    return __ldg(p);
}

// ALL: every tap's loads issued at once (the z loop unrolled too); the sums
// are the same, in the same order.  FP64 fields: every tap value is split
// into a float pair and the products and their sum run in double-float
// arithmetic (df.cuh), in the same tap order (z, y, x).
template <typename T, int KW, bool COH = false, bool ALL = false>
__device__ __forceinline__ void interp_marker(const T *__restrict__ u, const DevGrid &g,
                                              long long N, uint64_t anc,
                                              const PS<T> *__restrict__ w, T out[3]) {
    int ix[KW], iy[KW], iz[KW];
    int ax = anchor_x(anc), ay = anchor_y(anc), az = anchor_z(anc);
#pragma unroll
    for (int k = 0; k < KW; ++k) {
        ix[k] = wrap_add(ax, k, g.n[0]);
        iy[k] = wrap_add(ay, k, g.n[1]);
        iz[k] = wrap_add(az, k, g.n[2]);
    }
    if constexpr (sizeof(T) == 8) {
        SumAcc<double> a0, a1, a2;
        auto plane = [&](int kz) {
#pragma unroll
            for (int ky = 0; ky < KW; ++ky) {
                long long row = ((long long)iz[kz] * g.n[1] + iy[ky]) * g.n[0];
                const float2 wyz = df_mul(w[8 + kz], w[4 + ky]);
                double v[KW][3];
#pragma unroll
                for (int kx = 0; kx < KW; ++kx) {
                    long long c = row + ix[kx];
                    v[kx][0] = ld<COH>(u + c);
                    v[kx][1] = ld<COH>(u + N + c);
                    v[kx][2] = ld<COH>(u + 2 * N + c);
                }
#pragma unroll
                for (int kx = 0; kx < KW; ++kx) {
                    const float2 wt = df_mul(wyz, w[kx]);
                    a0.add(wt, df_split(v[kx][0]));
                    a1.add(wt, df_split(v[kx][1]));
                    a2.add(wt, df_split(v[kx][2]));
                }
            }
        };
#pragma unroll 1
        for (int kz = 0; kz < KW; ++kz) plane(kz);
        out[0] = a0.value();
        out[1] = a1.value();
        out[2] = a2.value();
    } else {
        T a0 = 0, a1 = 0, a2 = 0;
        auto plane = [&](int kz) {
#pragma unroll
            for (int ky = 0; ky < KW; ++ky) {
                long long row = ((long long)iz[kz] * g.n[1] + iy[ky]) * g.n[0];
                T wyz = w[8 + kz] * w[4 + ky];
#pragma unroll
                for (int kx = 0; kx < KW; ++kx) {
                    long long c = row + ix[kx];
                    T wt = wyz * w[kx];
                    a0 += wt * ld<COH>(u + c);
                    a1 += wt * ld<COH>(u + N + c);
                    a2 += wt * ld<COH>(u + 2 * N + c);
                }
            }
        };
        if (ALL) {
#pragma unroll
            for (int kz = 0; kz < KW; ++kz) plane(kz);
        } else {
#pragma unroll 1
            for (int kz = 0; kz < KW; ++kz) plane(kz);
        }
        out[0] = a0;
        out[1] = a1;
        out[2] = a2;
    }
}

// Atomic spreading of one marker: u += w_c A at its KW^3 stencil cells (and
// f_out += w_c A / dt when given), combined first across the lanes of the warp
// that target the same cell, so each distinct cell takes one atomic addition
// per warp and component.  Every lane of the warp must call it together
// (lanes with valid = false take part in the matching only).  FP64 fields:
// the products run in double-float and each contribution is rounded to
// double once before the lane sums.
template <typename T, int KW>
__device__ __forceinline__ void scatter_marker(T *u, T *f_out, const DevGrid &g, long long N, uint64_t anc,
                                               const PS<T> *w, const PS<T> *A, bool valid, double inv_dt) {
    const int lane = threadIdx.x & 31;
    int ix[KW], iy[KW], iz[KW];
    const int ax = anchor_x(anc), ay = anchor_y(anc), az = anchor_z(anc);
#pragma unroll
    for (int k = 0; k < KW; ++k) {
        ix[k] = wrap_add(ax, k, g.n[0]);
        iy[k] = wrap_add(ay, k, g.n[1]);
        iz[k] = wrap_add(az, k, g.n[2]);
    }
#pragma unroll 1
    for (int kz = 0; kz < KW; ++kz)
#pragma unroll
        for (int ky = 0; ky < KW; ++ky)
#pragma unroll
            for (int kx = 0; kx < KW; ++kx) {
                const long long c = ((long long)iz[kz] * g.n[1] + iy[ky]) * g.n[0] + ix[kx];
                T v[3];
                if constexpr (sizeof(T) == 8) {
                    const float2 wt = pair_weight(w, kx, ky, kz);
#pragma unroll
                    for (int q = 0; q < 3; ++q) v[q] = valid ? df_to_double(df_mul(wt, A[q])) : 0.0;
                } else {
                    const T wt = pair_weight(w, kx, ky, kz);
#pragma unroll
                    for (int q = 0; q < 3; ++q) v[q] = valid ? wt * A[q] : T(0);
                }
                const unsigned long long key = valid ? (unsigned long long)c : ~0ull - (unsigned)lane;
                const unsigned grp = __match_any_sync(0xffffffffu, key);
                T sum[3] = {T(0), T(0), T(0)};
                for (unsigned m = grp; m; m &= m - 1) {
                    const int src = __ffs(m) - 1;
#pragma unroll
                    for (int q = 0; q < 3; ++q) sum[q] += __shfl_sync(grp, v[q], src);
                }
                if (valid && lane == __ffs(grp) - 1) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) atomicAdd(u + q * N + c, sum[q]);
                    if (f_out)
#pragma unroll
                        for (int q = 0; q < 3; ++q) atomicAdd(f_out + q * N + c, (T)(sum[q] * inv_dt));
                }
            }
}

template <typename T, int KW, bool STAGED, bool COH>
__device__ __forceinline__ bool gather_cell(int tx, int ty, int tz, const uint16_t *bins, const uint32_t *cand,
                                            const T *w_src, const T *A_src, T acc[3]) {
    bool hit = false;
    acc[0] = acc[1] = acc[2] = T(0);
#pragma unroll 1
    for (int dz = 0; dz < KW; ++dz) {
        const int rz = tz + 3 - (KW - 1) + dz, oz = KW - 1 - dz;
#pragma unroll 1
        for (int dy = 0; dy < KW; ++dy) {
            const int ry = ty + 3 - (KW - 1) + dy, oy = KW - 1 - dy;
            const uint16_t *rb = bins + (rz * kRow + ry) * kBinsPerRow + tx + 3 - (KW - 1);
            int e[KW + 1];
#pragma unroll
            for (int dx = 0; dx <= KW; ++dx) e[dx] = rb[dx];
#pragma unroll
            for (int dx = 0; dx < KW; ++dx) {
                const int ox = KW - 1 - dx;
                for (int i = e[dx]; i < e[dx + 1]; ++i) {
                    const size_t k = STAGED ? (size_t)i : (size_t)cand[i];
                    const T *w = w_src + 12 * k;
                    const T *A = A_src + 4 * k;
                    T wt, a0, a1, a2;
                    if (STAGED) {
                        wt = w[ox] * w[4 + oy] * w[8 + oz];
                        a0 = A[0], a1 = A[1], a2 = A[2];
                    } else {
                        wt = __ldg(w + ox) * __ldg(w + 4 + oy) * __ldg(w + 8 + oz);
                        a0 = ld<COH>(A), a1 = ld<COH>(A + 1), a2 = ld<COH>(A + 2);
                    }
                    acc[0] += wt * a0;
                    acc[1] += wt * a1;
                    acc[2] += wt * a2;
                    hit = true;
                }
            }
        }
    }
    return hit;
}

}  // namespace gbib

namespace gbib {

// Candidates of one tile staged in shared memory by the list gathers.
template <typename T> struct TileStage;
template <> struct TileStage<float> { static constexpr int N = 256; };
template <> struct TileStage<double> { static constexpr int N = 192; };

template <typename T>
constexpr size_t tile_stage_bytes() {
    return (size_t)TileStage<T>::N * 16 * sizeof(T);
}

// One tile (compact slot cs) of a gather phase over its per-cell lists: the
// tile's candidate weights and sources are staged in shared memory (sw
// [N][12], sA [N][4]) when they fit, then each thread takes band cells and
// adds their pairs in list order (ascending candidate), u += S A and, when the
// case has a force field, f += S A / dt.  COH: the sources were written during
// this kernel (plain loads after an acquire) rather than by an earlier one.
// Ends with a CTA barrier.
template <typename T, int KW, bool COH>
__device__ __forceinline__ void gather_tile_lists(const CaseTab &ct, int cs, const Slots &sl, const PS<T> *wts,
                                                  const PS<T> *A_src, double inv_dt, PS<T> *sw, PS<T> *sA) {
    using S = PS<T>;
    const DevCase cd = ct.get(sl.geo_case[cs]);
    const DevGrid &g = cd.g;
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    T *const u = (T *)cd.u;
    T *const f_out = (T *)cd.f;
    const int4 lo = sl.geo_lo[cs], dim = sl.geo_dim[cs];
    const uint32_t d = sl.dense_of[cs];
    const int nc = (int)(sl.start[d + 1] - sl.start[d]);
    const int nb = sl.nband[cs];
    const uint32_t *cand = sl.cand + dim.w;
    const int2 *band = sl.band + sl.poff[dim.w];
    const uint32_t *pairs = sl.pairs + sl.poff[dim.w];
    const bool staged = nc <= TileStage<T>::N;
    auto cell_index = [&](int cell) {
        const int tx = cell & 7, ty = (cell >> 3) & 7, tz = cell >> 6;
        return ((long long)wrap_add(lo.z, tz, g.n[2]) * g.n[1] + wrap_add(lo.y, ty, g.n[1])) * g.n[0] +
               wrap_add(lo.x, tx, g.n[0]);
    };
    // this thread's first band cell, its list head and its u values are
    // loaded before the staging barrier (none of them changes meanwhile: a
    // band cell is updated by its own thread only)
    // (and the first batch of its pairs)
    constexpr int kPB = 8;  // pairs loaded per batch, all in flight at once
    const int q0 = threadIdx.x;
    int2 e0 = make_int2(0, 0);
    long long c0 = 0;
    T v0[3] = {T(0), T(0), T(0)};
    uint32_t pb0[kPB];
    if (q0 < nb) {
        e0 = band[q0];
        c0 = cell_index(e0.x & 0xffff);
        v0[0] = u[c0];
        v0[1] = u[N + c0];
        v0[2] = u[2 * N + c0];
#pragma unroll
        for (int j = 0; j < kPB; ++j) pb0[j] = j < (e0.x >> 16) ? pairs[e0.y + j] : 0u;
    }
    if (staged) {
        // weights first (written before this phase), then the sources
        const uint32_t m0 = threadIdx.x < nc ? cand[threadIdx.x] : 0u;
        for (int i = threadIdx.x; i < nc; i += blockDim.x) {
            const uint32_t m = i == (int)threadIdx.x ? m0 : cand[i];
            const S *wm = wts + 12 * (size_t)m;
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int j = 0; j < KW; ++j) sw[12 * i + 4 * q + j] = __ldg(wm + 4 * q + j);
        }
        for (int i = threadIdx.x; i < nc; i += blockDim.x) {
            const uint32_t m = i == (int)threadIdx.x ? m0 : cand[i];
#pragma unroll
            for (int q = 0; q < 3; ++q) sA[4 * i + q] = ld<COH>(A_src + 4 * (size_t)m + q);
        }
        __syncthreads();
    }
    for (int q = q0; q < nb; q += blockDim.x) {
        const bool first = q == q0;
        const int2 e = first ? e0 : band[q];
        const int cnt = e.x >> 16;
        const uint32_t *pr = pairs + e.y;
        SumAcc<T> acc0, acc1, acc2;
        for (int k0 = 0; k0 < cnt; k0 += kPB) {
            uint32_t pk[kPB];
#pragma unroll
            for (int j = 0; j < kPB; ++j)
                pk[j] = (first && k0 == 0) ? pb0[j] : (k0 + j < cnt ? pr[k0 + j] : 0u);
#pragma unroll
            for (int j = 0; j < kPB; ++j) {
                if (k0 + j >= cnt) break;
                const int i = pk[j] & 0xffff, ox = (pk[j] >> 16) & 3, oy = (pk[j] >> 18) & 3,
                          oz = (pk[j] >> 20) & 3;
                S wt, a0, a1, a2;
                if (staged) {
                    const S *w = sw + 12 * i;
                    const S *Ai = sA + 4 * i;
                    wt = pair_weight(w, ox, oy, oz);
                    a0 = Ai[0], a1 = Ai[1], a2 = Ai[2];
                } else {
                    const size_t m = cand[i];
                    const S *w = wts + 12 * m;
                    const S *Ai = A_src + 4 * m;
                    wt = pair_weight3(__ldg(w + ox), __ldg(w + 4 + oy), __ldg(w + 8 + oz));
                    a0 = ld<COH>(Ai), a1 = ld<COH>(Ai + 1), a2 = ld<COH>(Ai + 2);
                }
                acc0.add(wt, a0);
                acc1.add(wt, a1);
                acc2.add(wt, a2);
            }
        }
        const long long c = first ? c0 : cell_index(e.x & 0xffff);
        const T u0 = first ? v0[0] : u[c], u1 = first ? v0[1] : u[N + c], u2 = first ? v0[2] : u[2 * N + c];
        const T s0 = acc0.value(), s1 = acc1.value(), s2 = acc2.value();
        u[c] = u0 + s0;
        u[N + c] = u1 + s1;
        u[2 * N + c] = u2 + s2;
        if (f_out) {
            f_out[c] += (T)(s0 * inv_dt);
            f_out[N + c] += (T)(s1 * inv_dt);
            f_out[2 * N + c] += (T)(s2 * inv_dt);
        }
    }
    __syncthreads();
}

// Several consecutive tiles [cs0, cs0 + nt) of one case gathered together:
// the candidates of all of them are staged at once when they fit (CAP
// records in sw/sA; single tiles need TileStage<T>::N), and the
// band cells of all of them form one flat loop (one staging round trip and
// one barrier for the lot).  Falls back to one tile at a time otherwise.
// Sums are those of gather_tile_lists.  Ends with a CTA barrier.
constexpr int kMultiTiles = 8;

template <typename T, int KW, bool COH, int CAP>
__device__ __forceinline__ void gather_tiles_lists(const CaseTab &ct, int cs0, int nt, const Slots &sl,
                                                   const T *wts, const T *A_src, double inv_dt, T *sw, T *sA) {
    __shared__ int s_coff[kMultiTiles + 1], s_boff[kMultiTiles + 1];
    if (nt <= 0) return;
    if (nt > kMultiTiles) {
        for (int k = 0; k < nt; ++k) gather_tile_lists<T, KW, COH>(ct, cs0 + k, sl, wts, A_src, inv_dt, sw, sA);
        return;
    }
    if (threadIdx.x == 0) {
        int co = 0, bo = 0;
        for (int k = 0; k < nt; ++k) {
            const uint32_t d = sl.dense_of[cs0 + k];
            s_coff[k] = co;
            s_boff[k] = bo;
            co += (int)(sl.start[d + 1] - sl.start[d]);
            bo += sl.nband[cs0 + k];
        }
        s_coff[nt] = co;
        s_boff[nt] = bo;
    }
    __syncthreads();
    if (s_coff[nt] > CAP) {
        for (int k = 0; k < nt; ++k) gather_tile_lists<T, KW, COH>(ct, cs0 + k, sl, wts, A_src, inv_dt, sw, sA);
        return;
    }
    const DevCase cd = ct.get(sl.geo_case[cs0]);
    const DevGrid &g = cd.g;
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    T *const u = (T *)cd.u;
    T *const f_out = (T *)cd.f;
    // stage every candidate of the tiles (tile k's at offset s_coff[k])
    const int ctot = s_coff[nt];
    for (int j = threadIdx.x; j < ctot; j += blockDim.x) {
        int k = 0;
        while (k + 1 < nt && s_coff[k + 1] <= j) ++k;
        const uint32_t m = sl.cand[sl.geo_dim[cs0 + k].w + (j - s_coff[k])];
        const T *wm = wts + 12 * (size_t)m;
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int jj = 0; jj < KW; ++jj) sw[12 * j + 4 * q + jj] = __ldg(wm + 4 * q + jj);
#pragma unroll
        for (int q = 0; q < 3; ++q) sA[4 * j + q] = ld<COH>(A_src + 4 * (size_t)m + q);
    }
    __syncthreads();
    const int btot = s_boff[nt];
    for (int qq = threadIdx.x; qq < btot; qq += blockDim.x) {
        int k = 0;
        while (k + 1 < nt && s_boff[k + 1] <= qq) ++k;
        const int cs = cs0 + k;
        const int4 lo = sl.geo_lo[cs];
        const int b = sl.geo_dim[cs].w;
        const size_t pb = sl.poff[b];
        const int2 e = sl.band[pb + (qq - s_boff[k])];
        const int cell = e.x & 0xffff, cnt = e.x >> 16;
        const uint32_t *pr = sl.pairs + pb + e.y;
        const T *swk = sw + 12 * (size_t)s_coff[k];
        const T *sAk = sA + 4 * (size_t)s_coff[k];
        T acc0 = 0, acc1 = 0, acc2 = 0;
        for (int kk = 0; kk < cnt; ++kk) {
            const uint32_t pk = pr[kk];
            const int i = pk & 0xffff, ox = (pk >> 16) & 3, oy = (pk >> 18) & 3, oz = (pk >> 20) & 3;
            const T *w = swk + 12 * i;
            const T *Ai = sAk + 4 * i;
            const T wt = w[ox] * w[4 + oy] * w[8 + oz];
            acc0 += wt * Ai[0];
            acc1 += wt * Ai[1];
            acc2 += wt * Ai[2];
        }
        const int tx = cell & 7, ty = (cell >> 3) & 7, tz = cell >> 6;
        const long long c = ((long long)wrap_add(lo.z, tz, g.n[2]) * g.n[1] + wrap_add(lo.y, ty, g.n[1])) * g.n[0] +
                            wrap_add(lo.x, tx, g.n[0]);
        u[c] += acc0;
        u[N + c] += acc1;
        u[2 * N + c] += acc2;
        if (f_out) {
            f_out[c] += (T)(acc0 * inv_dt);
            f_out[N + c] += (T)(acc1 * inv_dt);
            f_out[2 * N + c] += (T)(acc2 * inv_dt);
        }
    }
    __syncthreads();
}

// Arguments of the particle-resident pass kernel (sequential order): the
// outputs of the preparation kernels plus the scheduling words.
template <typename T>
struct ResidentArgs {
    CaseTab ct;
    double *F;              // [M][3] marker forces (zeroed by the preparation)
    const double *dV;       // [M]
    MarkerState<T> ms;
    Slots sl;               // particle-local tiles, compact and sorted
    const int *mperm;       // markers level-major, each particle's in index order
    const int *mbase;       // [P] first position of a particle's markers in mperm
    const int *moff;        // [P+1]
    const int *by_rank;     // [P] particle of each rank (level-major order)
    const int *rank;        // [P]
    const int *level;       // [P]
    const int4 *box_lo;     // [P] first cell of the particle's stencil box
    const int *nbr_cnt;     // [P] conflicts with q < p (-1: list full)
    const int *nbr;         // [P][kMaxNbr]
    unsigned int *done;     // [P] CTAs that finished each particle (zeroed)
    unsigned int *ticket;   // next rank to take (zeroed)
    unsigned int *gwords;   // [4 * groups] group barrier words and ticket slot (zeroed; group form)
    int P, Ns;
    double dt, inv_dt;  // inv_dt = 1 / dt, formed on the host
    DevStatus *st;
};

// Enqueues the particle-resident passes on `s` (mdf_resident.cu).
template <typename T, int KER>
int launch_mdf_resident(ib_ctx *ctx, const ResidentArgs<T> &a, cudaStream_t s);

// Enqueues the particle-group passes on `s` (mdf_groups.cu); `gwords` must
// hold 4 * mdf_groups_count(ctx) words, zeroed.
template <typename T, int KER>
int launch_mdf_groups(ib_ctx *ctx, const ResidentArgs<T> &a, cudaStream_t s);
template <typename T, int KER>
int mdf_groups_count(ib_ctx *ctx);

}  // namespace gbib
