// The fluid step around the IB forcing on one uniform periodic level
// (arXiv 2408.14140, Sec. 3.1): Step 1, the momentum predictor (Eq. 31), and
// Step 3, the level projection (Eqs. ns_lp1-ns_lp3).
//
// Grid (semi-staggered, Sec. 3.1): velocity at cell centres, [3][n2][n1][n0]
// (x fastest); pressure at nodes, [n2][n1][n0], node (i, j, k) the lower
// corner of cell (i, j, k).
//   G p  (cells)  = along x, (1/4h) sum over the cell's four x-edges of p(i+1) - p(i)
//   D V  (nodes)  = the negative adjoint of G, so the projection's Laplacian is D G
//   L_c u (cells) = 7-point Laplacian per component
// The implicit solves -- (I - nu dt/2 L_c) for Crank-Nicolson viscosity and
// D G for the pressure -- are diagonal in Fourier space on a periodic grid
// and are done exactly with a radix-2 FFT along each axis (Stockham
// autosort in shared memory, one CTA per group of lines), so every grid axis
// must be a power of two.  Convection div(u u)^{n+1/2} is a second-order
// Godunov edge extrapolation: per face, states from both neighbours by a
// Taylor step along monotonized-central limited slopes, the normal velocity
// from the Burgers Riemann solution of the two normal states, the state
// upwinded by it, and the flux difference over the cell.
#include "gbib_internal.cuh"

namespace gbib {

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

__device__ __forceinline__ void sincos_pi(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincos_pi(double x, double *s, double *c) { sincospi(x, s, c); }

constexpr int kFftThreads = 256;
constexpr int kFftPoints = 2048;  // points of one CTA (lines x length)

// Lines of one CTA along `axis`.
__host__ __device__ inline int fft_lines(int N, int axis, int n0) {
    int L = kFftPoints / N;
    L = L < 1 ? 1 : (L > 8 ? 8 : L);
    if (axis > 0 && L > n0) L = n0;
    return L;
}

// One radix-2 Stockham FFT of length N = 2^logN along `axis` for L lines per
// CTA: stage t combines x[q + s p] and x[q + s (p + m)] (s = 2^t,
// m = N / 2^(t+1)) into y[q + 2 s p] = a + b and y[q + s (2p + 1)] = (a - b) w^p
// with w = exp(-+ 2 pi i s / N).  inverse: conjugate twiddles, no scaling.
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_fft_axis(typename Cx<T>::type *data, int n0, int n1, int n2,
                                                          int axis, int logN, int inverse) {
    using C = typename Cx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = 1 << logN;
    const int L = fft_lines(N, axis, n0);
    C *buf0 = (C *)smem_raw;
    C *buf1 = buf0 + (size_t)L * N;
    C *tw = buf1 + (size_t)L * N;
    const long long stride = axis == 0 ? 1 : (axis == 1 ? (long long)n0 : (long long)n0 * n1);
    const long long nlines = (long long)n0 * n1 * n2 / N;
    for (int k = threadIdx.x; k < N / 2; k += blockDim.x) {
        T s, c;
        sincos_pi((T)(2 * k) / (T)N, &s, &c);
        tw[k] = C{c, inverse ? s : -s};
    }
    for (long long l0 = (long long)blockIdx.x * L; l0 < nlines; l0 += (long long)gridDim.x * L) {
        // base offset of line l0 + l
        auto base = [&](long long l) -> long long {
            if (axis == 0) return l * n0;
            if (axis == 1) return (l / n0) * (long long)n0 * n1 + l % n0;
            return l;  // axis 2: l = y n0 + x
        };
        __syncthreads();
        for (int t = threadIdx.x; t < L * N; t += blockDim.x) {
            // axis 0: consecutive threads walk one line; else consecutive lines (adjacent x)
            const int l = axis == 0 ? t / N : t % L, j = axis == 0 ? t % N : t / L;
            buf0[l * N + j] = data[base(l0 + l) + j * stride];
        }
        __syncthreads();
        C *x = buf0, *y = buf1;
        for (int st = 0; st < logN; ++st) {
            const int s = 1 << st, m = N >> (st + 1);
            for (int t = threadIdx.x; t < L * (N / 2); t += blockDim.x) {
                const int l = t / (N / 2), bfl = t % (N / 2);
                const int p = bfl / s, q = bfl % s;
                const C a = x[l * N + q + s * p], b = x[l * N + q + s * (p + m)];
                y[l * N + q + 2 * s * p] = cadd(a, b);
                y[l * N + q + s * (2 * p + 1)] = cmul(csub(a, b), tw[p * s]);
            }
            __syncthreads();
            C *tmp = x;
            x = y;
            y = tmp;
        }
        for (int t = threadIdx.x; t < L * N; t += blockDim.x) {
            const int l = axis == 0 ? t / N : t % L, j = axis == 0 ? t % N : t / L;
            data[base(l0 + l) + j * stride] = x[l * N + j];
        }
    }
}

// theta_a = 2 pi k_a / n_a of FFT index i (frequencies above n/2 are negative)
template <typename T>
__device__ __forceinline__ T half_theta_pi(int i, int n) {
    // theta / 2 / pi = k / n, with k in (-n/2, n/2]
    const int k = i <= n / 2 ? i : i - n;
    return (T)k / (T)n;
}

// Multiplies the spectrum by the inverse of the operator's symbol and by
// 1 / (n0 n1 n2) (the inverse FFT is unscaled).
//   kind 0: (I - coef L_c)^-1, L_c symbol -(4/h^2) sum sin^2(theta/2)
//   kind 1: coef (D G)^-1, D G symbol -(4/h^2) sum_a sin^2 prod_b cos^2, 0 on its null modes
template <typename T>
__global__ void k_symbol(typename Cx<T>::type *data, int n0, int n1, int n2, int kind, double coef, double h) {
    const long long N = (long long)n0 * n1 * n2;
    const T inv_n = (T)(1.0 / (double)N);
    const T c4 = (T)(4.0 / (h * h));
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % n0), j = (int)((idx / n0) % n1), k = (int)(idx / ((long long)n0 * n1));
        T sx, cx, sy, cy, sz, cz;
        sincos_pi(half_theta_pi<T>(i, n0), &sx, &cx);
        sincos_pi(half_theta_pi<T>(j, n1), &sy, &cy);
        sincos_pi(half_theta_pi<T>(k, n2), &sz, &cz);
        sx *= sx, cx *= cx, sy *= sy, cy *= cy, sz *= sz, cz *= cz;
        T f;
        if (kind == 0) {
            f = inv_n / ((T)1 + (T)coef * c4 * (sx + sy + sz));
        } else {
            const T lam = -c4 * (sx * cy * cz + sy * cx * cz + sz * cx * cy);
            f = fabs(lam) <= (T)1e-13 * (T)3 * c4 ? (T)0 : (T)coef * inv_n / lam;
        }
        data[idx].x *= f;
        data[idx].y *= f;
    }
}

template <typename T>
__device__ __forceinline__ T mc_slope(T um, T u0, T up) {
    const T a = u0 - um, b = up - u0;
    const T mag = fmin(fmin((T)2 * fabs(a), (T)2 * fabs(b)), (T)0.5 * fabs(a + b));
    return a * b > (T)0 ? copysign(mag, a + b) : (T)0;
}

// Flux of all three components through the face between cells i and i+1
// along axis a, from the cells i-1 .. i+2 (v[0..3][c]).
template <typename T>
__device__ __forceinline__ void face_flux(const T v[4][3], int a, T dt, T h, T flux[3]) {
    T left[3], right[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T sl = mc_slope(v[0][c], v[1][c], v[2][c]);
        const T sr = mc_slope(v[1][c], v[2][c], v[3][c]);
        left[c] = v[1][c] + ((T)0.5 - dt * v[1][a] / ((T)2 * h)) * sl;
        right[c] = v[2][c] - ((T)0.5 + dt * v[2][a] / ((T)2 * h)) * sr;
    }
    const T lv = left[a], rv = right[a];
    const T un = (lv > (T)0 && lv + rv > (T)0) ? lv : ((rv < (T)0 && lv + rv < (T)0) ? rv : (T)0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T s = un > (T)0 ? left[c] : (un < (T)0 ? right[c] : (T)0.5 * (left[c] + right[c]));
        flux[c] = un * s;
    }
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Right-hand side of the predictor at every cell,
//   u^n + dt (-div(u u) - G p / rho + (nu / 2) L_c u^n + g),
// packed for the spectral solve: (x, y) components as one complex field, z
// as the real part of another (the symbol is real and even, so the two
// real fields of one complex field stay separate).
template <typename T>
__global__ void k_predictor_rhs(DevGrid g, const T *__restrict__ u, const T *__restrict__ p, double rho_f, double nu,
                                double gx, double gy, double gz, double dt, typename Cx<T>::type *c0,
                                typename Cx<T>::type *c1) {
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    const long long N = (long long)n0 * n1 * n2;
    const T h = (T)g.h, tdt = (T)dt;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % n0), j = (int)((idx / n0) % n1), k = (int)(idx / ((long long)n0 * n1));
        auto cell = [&](int di, int dj, int dk) {
            return ((long long)wrapi(k + dk, n2) * n1 + wrapi(j + dj, n1)) * n0 + wrapi(i + di, n0);
        };
        T conv[3] = {0, 0, 0}, lap[3] = {0, 0, 0};
        T u0[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) u0[c] = u[c * N + idx];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            T v[5][3];  // cells -2 .. +2 along a
#pragma unroll
            for (int o = 0; o < 5; ++o) {
                const long long cc = cell(a == 0 ? o - 2 : 0, a == 1 ? o - 2 : 0, a == 2 ? o - 2 : 0);
#pragma unroll
                for (int c = 0; c < 3; ++c) v[o][c] = o == 2 ? u0[c] : u[c * N + cc];
            }
            T fm[3], fp[3];
            face_flux<T>(*(const T(*)[4][3])&v[0], a, tdt, h, fm);  // face i - 1/2 (cells i-2 .. i+1)
            face_flux<T>(*(const T(*)[4][3])&v[1], a, tdt, h, fp);  // face i + 1/2 (cells i-1 .. i+2)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                conv[c] += (fp[c] - fm[c]) / h;
                lap[c] += (v[3][c] - (T)2 * v[2][c] + v[1][c]) / (h * h);
            }
        }
        // G p at the cell: node (i, j, k) is the cell's lower corner
        T pc[2][2][2];
#pragma unroll
        for (int dk = 0; dk < 2; ++dk)
#pragma unroll
            for (int dj = 0; dj < 2; ++dj)
#pragma unroll
                for (int di = 0; di < 2; ++di) pc[dk][dj][di] = p[cell(di, dj, dk)];
        const T q = (T)0.25 / h;
        T gp[3];
        {
            T d00 = pc[0][0][1] - pc[0][0][0], d10 = pc[0][1][1] - pc[0][1][0];
            T d01 = pc[1][0][1] - pc[1][0][0], d11 = pc[1][1][1] - pc[1][1][0];
            gp[0] = q * (d00 + d10 + d01 + d11);
            d00 = pc[0][1][0] - pc[0][0][0], d10 = pc[0][1][1] - pc[0][0][1];
            d01 = pc[1][1][0] - pc[1][0][0], d11 = pc[1][1][1] - pc[1][0][1];
            gp[1] = q * (d00 + d10 + d01 + d11);
            d00 = pc[1][0][0] - pc[0][0][0], d10 = pc[1][0][1] - pc[0][0][1];
            d01 = pc[1][1][0] - pc[0][1][0], d11 = pc[1][1][1] - pc[0][1][1];
            gp[2] = q * (d00 + d10 + d01 + d11);
        }
        const T gv[3] = {(T)gx, (T)gy, (T)gz};
        T r[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            r[c] = u0[c] + tdt * (-conv[c] - gp[c] / (T)rho_f + (T)(0.5 * nu) * lap[c] + gv[c]);
        c0[idx] = typename Cx<T>::type{r[0], r[1]};
        c1[idx] = typename Cx<T>::type{r[2], (T)0};
    }
}

template <typename T>
__global__ void k_unpack_velocity(long long N, const typename Cx<T>::type *c0, const typename Cx<T>::type *c1,
                                  T *u) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        u[idx] = c0[idx].x;
        u[N + idx] = c0[idx].y;
        u[2 * N + idx] = c1[idx].x;
    }
}

// G of a nodal field at cell (i, j, k), component a.
template <typename T, typename F>
__device__ __forceinline__ void grad_at_cell(F nodal, T h, T out[3]) {
    T pc[2][2][2];
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj)
#pragma unroll
            for (int di = 0; di < 2; ++di) pc[dk][dj][di] = nodal(di, dj, dk);
    const T q = (T)0.25 / h;
    out[0] = q * ((pc[0][0][1] - pc[0][0][0]) + (pc[0][1][1] - pc[0][1][0]) + (pc[1][0][1] - pc[1][0][0]) +
                  (pc[1][1][1] - pc[1][1][0]));
    out[1] = q * ((pc[0][1][0] - pc[0][0][0]) + (pc[0][1][1] - pc[0][0][1]) + (pc[1][1][0] - pc[1][0][0]) +
                  (pc[1][1][1] - pc[1][0][1]));
    out[2] = q * ((pc[1][0][0] - pc[0][0][0]) + (pc[1][0][1] - pc[0][0][1]) + (pc[1][1][0] - pc[0][1][0]) +
                  (pc[1][1][1] - pc[0][1][1]));
}

// D V at every node, V = u*/dt + G p_old / rho_f (Eq. ns_lp1) formed at the
// eight cells around the node; the result is the real part of the spectrum
// buffer.
template <typename T>
__global__ void k_projection_div(DevGrid g, const T *__restrict__ u, const T *__restrict__ p, double rho_f, double dt,
                                 typename Cx<T>::type *c) {
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    const long long N = (long long)n0 * n1 * n2;
    const T h = (T)g.h, idt = (T)(1.0 / dt), irho = (T)(1.0 / rho_f);
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % n0), j = (int)((idx / n0) % n1), k = (int)(idx / ((long long)n0 * n1));
        // the cells around node (i, j, k): (i-1|i, j-1|j, k-1|k)
        T V[2][2][2][3];
#pragma unroll
        for (int ck = 0; ck < 2; ++ck)
#pragma unroll
            for (int cj = 0; cj < 2; ++cj)
#pragma unroll
                for (int ci = 0; ci < 2; ++ci) {
                    const int ii = wrapi(i - 1 + ci, n0), jj = wrapi(j - 1 + cj, n1), kk = wrapi(k - 1 + ck, n2);
                    const long long cidx = ((long long)kk * n1 + jj) * n0 + ii;
                    T gp[3];
                    grad_at_cell<T>([&](int di, int dj, int dk) {
                        return p[((long long)wrapi(kk + dk, n2) * n1 + wrapi(jj + dj, n1)) * n0 + wrapi(ii + di, n0)];
                    }, h, gp);
#pragma unroll
                    for (int a = 0; a < 3; ++a) V[ck][cj][ci][a] = u[a * N + cidx] * idt + gp[a] * irho;
                }
        const T q = (T)0.25 / h;
        T d = q * ((V[1][1][1][0] - V[1][1][0][0]) + (V[0][1][1][0] - V[0][1][0][0]) +
                   (V[1][0][1][0] - V[1][0][0][0]) + (V[0][0][1][0] - V[0][0][0][0]));
        d += q * ((V[1][1][1][1] - V[1][0][1][1]) + (V[0][1][1][1] - V[0][0][1][1]) +
                  (V[1][1][0][1] - V[1][0][0][1]) + (V[0][1][0][1] - V[0][0][0][1]));
        d += q * ((V[1][1][1][2] - V[0][1][1][2]) + (V[1][0][1][2] - V[0][0][1][2]) +
                  (V[1][1][0][2] - V[0][1][0][2]) + (V[1][0][0][2] - V[0][0][0][2]));
        c[idx] = typename Cx<T>::type{d, (T)0};
    }
}

// u^{n+1} = dt (V - G p_new / rho_f) = u* + (dt / rho_f) G (p_old - p_new)
// (Eq. ns_lp3), p_new the real part of the solved buffer.
template <typename T>
__global__ void k_projection_update(DevGrid g, T *__restrict__ u, const T *__restrict__ p,
                                    const typename Cx<T>::type *__restrict__ c, double rho_f, double dt) {
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    const long long N = (long long)n0 * n1 * n2;
    const T h = (T)g.h, s = (T)(dt / rho_f);
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % n0), j = (int)((idx / n0) % n1), k = (int)(idx / ((long long)n0 * n1));
        auto node = [&](int di, int dj, int dk) {
            return ((long long)wrapi(k + dk, n2) * n1 + wrapi(j + dj, n1)) * n0 + wrapi(i + di, n0);
        };
        T go[3], gn[3];
        grad_at_cell<T>([&](int di, int dj, int dk) { return p[node(di, dj, dk)]; }, h, go);
        grad_at_cell<T>([&](int di, int dj, int dk) { return c[node(di, dj, dk)].x; }, h, gn);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const T V = u[a * N + idx] / (T)dt + go[a] / (T)rho_f;
            u[a * N + idx] = (T)dt * (V - gn[a] / (T)rho_f);
        }
        (void)s;
    }
}

template <typename T>
__global__ void k_take_pressure(long long N, const typename Cx<T>::type *c, T *p) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x)
        p[idx] = c[idx].x;
}

static int ilog2_exact(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return (1 << l) == n ? l : -1;
}

static int check_fluid_grid(const ib_grid *grid) {
    int rc = validate_grid(grid, 1);
    if (rc) return rc;
    for (int a = 0; a < 3; ++a) {
        const int l = ilog2_exact(grid->n[a]);
        if (l < 4 || l > 10)
            return set_error(IB_ERR_UNSUPPORTED, "fluid step: n[%d] = %d must be a power of two in [16, 1024]", a,
                             grid->n[a]);
    }
    return IB_OK;
}

// 3D FFT (forward or inverse, unscaled) of a complex field in place.
template <typename T>
static int fft3(ib_ctx *ctx, typename Cx<T>::type *c, const int n[3], int inverse, cudaStream_t s) {
    using C = typename Cx<T>::type;
    for (int axis = 0; axis < 3; ++axis) {
        const int N = n[axis], logN = ilog2_exact(N);
        const int L = fft_lines(N, axis, n[0]);
        const size_t smem = ((size_t)2 * L * N + N / 2) * sizeof(C);
        cudaFuncSetAttribute(k_fft_axis<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const long long nlines = (long long)n[0] * n[1] * n[2] / N;
        long long blocks = (nlines + L - 1) / L;
        const long long cap = (long long)ctx->sm_count * 16;
        if (blocks > cap) blocks = cap;
        k_fft_axis<T><<<(int)blocks, kFftThreads, smem, s>>>(c, n[0], n[1], n[2], axis, logN, inverse);
    }
    return check_launch("fft");
}

static int elem_blocks(long long n, int sm) {
    long long b = (n + 255) / 256, cap = (long long)sm * 16;
    return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

template <typename T>
static int run_predictor(ib_ctx *ctx, const ib_grid *grid, const void *u, const void *p, double rho_f, double mu,
                         const double g[3], double dt, void *u_star, cudaStream_t s) {
    using C = typename Cx<T>::type;
    const DevGrid dg = make_dev_grid(grid);
    const long long N = (long long)grid->n[0] * grid->n[1] * grid->n[2];
    Arena ar(ctx);
    C *c0 = ar.take<C>(N), *c1 = ar.take<C>(N);
    if (!ar.ok()) return oom_error(ar.used, ar.cap);
    const int nb = elem_blocks(N, ctx->sm_count);
    const double nu = mu / rho_f;
    PhaseTimer tm(ctx, IB_PHASE_FLUID_PREDICTOR, s);
    k_predictor_rhs<T><<<nb, 256, 0, s>>>(dg, (const T *)u, (const T *)p, rho_f, nu, g[0], g[1], g[2], dt, c0, c1);
    for (C *c : {c0, c1}) {
        int rc = fft3<T>(ctx, c, grid->n, 0, s);
        if (rc) return rc;
        k_symbol<T><<<nb, 256, 0, s>>>(c, grid->n[0], grid->n[1], grid->n[2], 0, 0.5 * nu * dt, grid->h);
        rc = fft3<T>(ctx, c, grid->n, 1, s);
        if (rc) return rc;
    }
    k_unpack_velocity<T><<<nb, 256, 0, s>>>(N, c0, c1, (T *)u_star);
    return check_launch("fluid_predictor");
}

template <typename T>
static int run_projection(ib_ctx *ctx, const ib_grid *grid, void *u, void *p, double rho_f, double dt,
                          cudaStream_t s) {
    using C = typename Cx<T>::type;
    const DevGrid dg = make_dev_grid(grid);
    const long long N = (long long)grid->n[0] * grid->n[1] * grid->n[2];
    Arena ar(ctx);
    C *c = ar.take<C>(N);
    if (!ar.ok()) return oom_error(ar.used, ar.cap);
    const int nb = elem_blocks(N, ctx->sm_count);
    PhaseTimer tm(ctx, IB_PHASE_FLUID_PROJECTION, s);
    k_projection_div<T><<<nb, 256, 0, s>>>(dg, (const T *)u, (const T *)p, rho_f, dt, c);
    int rc = fft3<T>(ctx, c, grid->n, 0, s);
    if (rc) return rc;
    // p_new = rho_f (D G)^-1 D V   (Eq. ns_lp2 with L p = div((1/rho_f) grad p))
    k_symbol<T><<<nb, 256, 0, s>>>(c, grid->n[0], grid->n[1], grid->n[2], 1, rho_f, grid->h);
    rc = fft3<T>(ctx, c, grid->n, 1, s);
    if (rc) return rc;
    k_projection_update<T><<<nb, 256, 0, s>>>(dg, (T *)u, (const T *)p, c, rho_f, dt);
    k_take_pressure<T><<<nb, 256, 0, s>>>(N, c, (T *)p);
    return check_launch("level_projection");
}

}  // namespace gbib

using namespace gbib;

extern "C" {

int fluid_predictor(ib_ctx *ctx, const ib_grid *grid, const void *u, const void *p, double rho_f, double mu,
                    const double *g, double dt, void *u_star, void *stream) {
    if (!ctx) return set_error(IB_ERR_INVALID, "ctx is NULL");
    int rc = check_fluid_grid(grid);
    if (rc) return rc;
    if (!u || !p || !u_star || !g) return set_error(IB_ERR_INVALID, "NULL array");
    if (!(rho_f > 0.0) || !(mu >= 0.0) || !isfinite(mu) || !(dt > 0.0) || !isfinite(dt) || !isfinite(g[0]) ||
        !isfinite(g[1]) || !isfinite(g[2]))
        return set_error(IB_ERR_INVALID, "rho_f > 0, mu >= 0, dt > 0 and g must be finite");
    if (grid->prec == IB_F64)
        return run_predictor<double>(ctx, grid, u, p, rho_f, mu, g, dt, u_star, (cudaStream_t)stream);
    return run_predictor<float>(ctx, grid, u, p, rho_f, mu, g, dt, u_star, (cudaStream_t)stream);
}

int level_projection(ib_ctx *ctx, const ib_grid *grid, void *u, void *p, double rho_f, double dt, void *stream) {
    if (!ctx) return set_error(IB_ERR_INVALID, "ctx is NULL");
    int rc = check_fluid_grid(grid);
    if (rc) return rc;
    if (!u || !p) return set_error(IB_ERR_INVALID, "NULL array");
    if (!(rho_f > 0.0) || !(dt > 0.0) || !isfinite(dt)) return set_error(IB_ERR_INVALID, "rho_f > 0 and dt > 0");
    if (grid->prec == IB_F64) return run_projection<double>(ctx, grid, u, p, rho_f, dt, (cudaStream_t)stream);
    return run_projection<float>(ctx, grid, u, p, rho_f, dt, (cudaStream_t)stream);
}

}  // extern "C"
