/*
 * ib_oracle.c -- plain, slow FP64 CPU oracle for the multidirect-forcing
 * immersed-boundary step of Zeng et al., "IAMReX" (arXiv 2408.14140).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; it is written directly from
 * the paper's equations with no blocking, fusion or reordering beyond what
 * those equations state, so that each function can be checked against the
 * paper by eye.
 *
 * Conventions (shared by definition of the problem, not by code):
 *   grid      n[3] cells, uniform spacing h, origin org[3]; cell (i,j,k) has
 *             centre org + (i+1/2, j+1/2, k+1/2) h, nodes sit at org + (i,j,k) h.
 *             The domain is periodic with period n[a]*h on every axis.
 *   fields    structure of arrays u[c][k][j][i], c = 0..2, x fastest.
 *   vectors   [count][3] row-major.
 *
 * Readings of points on which the paper is silent are marked "Reading:".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_ROMA3 0
#define OR_PESKIN4 1
#define OR_SEQUENTIAL 0
#define OR_SIMULTANEOUS 1

/* ------------------------------------------------------------------------ */
/* Regularised delta kernel, Sec. 2 (delta(x) = prod_i delta(x_i)) and
 * Sec. 3.1 Step 2 ("three-point or four-point delta function").
 * Reading: the three-point kernel is the one of Roma, Peskin & Berger (1999),
 * the four-point kernel the one of Peskin (2002); r is in cell units.        */
/* ------------------------------------------------------------------------ */
static double phi_roma3(double r)
{
    double a = fabs(r);
    if (a <= 0.5)
        return (1.0 + sqrt(1.0 - 3.0 * a * a)) / 3.0;
    if (a <= 1.5) {
        double t = 1.0 - a;
        return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * t * t)) / 6.0;
    }
    return 0.0;
}

static double phi_peskin4(double r)
{
    double a = fabs(r);
    if (a <= 1.0)
        return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    if (a <= 2.0)
        return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
    return 0.0;
}

double or_phi(int kernel, double r)
{
    return kernel == OR_PESKIN4 ? phi_peskin4(r) : phi_roma3(r);
}

/* Number of cells per axis in the kernel's support and the first of them.
 * s is the marker position in cell-index units measured from the first cell
 * centre, s = (X - org)/h - 1/2, so cell j sits at distance r = s - j.
 * Roma:   |r| < 3/2  ->  j in round(s) + {-1, 0, 1}
 * Peskin: |r| < 2    ->  j in floor(s) + {-1, 0, 1, 2}                      */
static int stencil_width(int kernel) { return kernel == OR_PESKIN4 ? 4 : 3; }

static long stencil_first(int kernel, double s)
{
    if (kernel == OR_PESKIN4)
        return (long)floor(s) - 1;
    return (long)floor(s + 0.5) - 1;
}

static long wrap(long j, long n)
{
    long m = j % n;
    return m < 0 ? m + n : m;
}

static long cell_index(const int n[3], long i, long j, long k)
{
    return (wrap(k, n[2]) * n[1] + wrap(j, n[1])) * n[0] + wrap(i, n[0]);
}

/* ------------------------------------------------------------------------ */
/* Velocity interpolation J, Eq. (u)/(vi) and Algorithm 1 (interpolation
 * step): U(X_l) = sum_ijk u(x_ijk) delta_h(x_ijk - X_l) h^3.  The h^3 cancels
 * the h^-3 of delta_h, leaving the product of the three 1-D kernels.        */
/* ------------------------------------------------------------------------ */
static void interp_one(const int n[3], double h, const double org[3],
                       const double *u, const double X[3], int kernel,
                       double U[3])
{
    long N = (long)n[0] * n[1] * n[2];
    int w = stencil_width(kernel);
    double s[3];
    long j0[3];
    for (int a = 0; a < 3; ++a) {
        s[a] = (X[a] - org[a]) / h - 0.5;
        j0[a] = stencil_first(kernel, s[a]);
    }
    U[0] = U[1] = U[2] = 0.0;
    for (int dk = 0; dk < w; ++dk)
        for (int dj = 0; dj < w; ++dj)
            for (int di = 0; di < w; ++di) {
                long i = j0[0] + di, j = j0[1] + dj, k = j0[2] + dk;
                double wt = or_phi(kernel, s[0] - (double)i) *
                            or_phi(kernel, s[1] - (double)j) *
                            or_phi(kernel, s[2] - (double)k);
                long c = cell_index(n, i, j, k);
                U[0] += u[c] * wt;
                U[1] += u[N + c] * wt;
                U[2] += u[2 * N + c] * wt;
            }
}

void or_interpolate(const int n[3], double h, const double org[3],
                    const double *u, long M, const double *X, int kernel,
                    double *U)
{
#pragma omp parallel for schedule(static)
    for (long l = 0; l < M; ++l)
        interp_one(n, h, org, u, X + 3 * l, kernel, U + 3 * l);
}

/* ------------------------------------------------------------------------ */
/* Force spreading S, Eq. (f)/(fs) and Algorithm 1 (spreading step):
 * f(x_ijk) += sum_l F_l delta_h(x_ijk - X_l) dV_l, delta_h = h^-3 prod phi.
 * Markers are visited in index order; f is accumulated, not overwritten.    */
/* ------------------------------------------------------------------------ */
void or_spread(const int n[3], double h, const double org[3], long M,
               const double *X, const double *F, const double *dV, int kernel,
               double *f)
{
    long N = (long)n[0] * n[1] * n[2];
    int w = stencil_width(kernel);
    double inv_h3 = 1.0 / (h * h * h);
    for (long l = 0; l < M; ++l) {
        double s[3];
        long j0[3];
        for (int a = 0; a < 3; ++a) {
            s[a] = (X[3 * l + a] - org[a]) / h - 0.5;
            j0[a] = stencil_first(kernel, s[a]);
        }
        double q = dV[l] * inv_h3;
        for (int dk = 0; dk < w; ++dk)
            for (int dj = 0; dj < w; ++dj)
                for (int di = 0; di < w; ++di) {
                    long i = j0[0] + di, j = j0[1] + dj, k = j0[2] + dk;
                    double wt = or_phi(kernel, s[0] - (double)i) *
                                or_phi(kernel, s[1] - (double)j) *
                                or_phi(kernel, s[2] - (double)k);
                    long c = cell_index(n, i, j, k);
                    f[c] += F[3 * l + 0] * q * wt;
                    f[N + c] += F[3 * l + 1] * q * wt;
                    f[2 * N + c] += F[3 * l + 2] * q * wt;
                }
    }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (multidirect forcing) for one set of markers, in the paper's
 * cumulative form:
 *   u(0) = u~*;  F^0 = 0 (Reading: the paper does not state F^0);
 *   for m = 1..Ns:
 *     U^{m-1} = J u(m-1)
 *     F^m     = F^{m-1} + (U^d - U^{m-1}) / dt
 *     f^m     = S F^m
 *     u(m)    = u(0) + dt f^m
 * Only cells inside the markers' kernel supports change (f^m = 0 elsewhere);
 * the oracle therefore keeps u(0) and f^m on the list of touched cells.
 * X[l], Ud[l] are the set's marker positions and desired velocities.         */
/* ------------------------------------------------------------------------ */
typedef struct {
    long *stamp;   /* [N] slot of a cell in the touched list, or -1 */
    long *cells;   /* touched cell indices                         */
    double *u0;    /* [3][cap] u(0) on touched cells               */
    double *fT;    /* [3][cap] f^m on touched cells                */
    long cap;
} touched_t;

static int run_marker_set(const int n[3], double h, const double org[3],
                          double *u, long m0, long m1, const double *X,
                          const double *Ud, const double *dV, int Ns, double dt,
                          int kernel, double *F, double *f_out, touched_t *T)
{
    long N = (long)n[0] * n[1] * n[2];
    int w = stencil_width(kernel);
    long w3 = (long)w * w * w;
    long cnt = 0;
    long need = (m1 - m0) * w3;
    if (need > T->cap) {
        long cap = need;
        long *cells = (long *)realloc(T->cells, sizeof(long) * cap);
        double *u0 = (double *)realloc(T->u0, sizeof(double) * 3 * cap);
        double *fT = (double *)realloc(T->fT, sizeof(double) * 3 * cap);
        if (!cells || !u0 || !fT)
            return -1;
        T->cells = cells; T->u0 = u0; T->fT = fT; T->cap = cap;
    }
    /* collect the touched cells (union of the kernel supports) */
    for (long l = m0; l < m1; ++l) {
        long j0[3];
        for (int a = 0; a < 3; ++a)
            j0[a] = stencil_first(kernel, (X[3 * l + a] - org[a]) / h - 0.5);
        for (int dk = 0; dk < w; ++dk)
            for (int dj = 0; dj < w; ++dj)
                for (int di = 0; di < w; ++di) {
                    long c = cell_index(n, j0[0] + di, j0[1] + dj, j0[2] + dk);
                    if (T->stamp[c] < 0) {
                        T->stamp[c] = cnt;
                        T->cells[cnt++] = c;
                    }
                }
    }
    long cap = T->cap;
    for (long t = 0; t < cnt; ++t)
        for (int a = 0; a < 3; ++a)
            T->u0[a * cap + t] = u[a * N + T->cells[t]];

    for (long l = m0; l < m1; ++l)
        F[3 * l] = F[3 * l + 1] = F[3 * l + 2] = 0.0;

    double inv_h3 = 1.0 / (h * h * h);
    for (int m = 1; m <= Ns; ++m) {
        /* interpolate U^{m-1} = J u(m-1) and update F^m */
        for (long l = m0; l < m1; ++l) {
            double U[3];
            interp_one(n, h, org, u, X + 3 * l, kernel, U);
            for (int a = 0; a < 3; ++a)
                F[3 * l + a] += (Ud[3 * l + a] - U[a]) / dt;
        }
        /* f^m = S F^m on the touched cells */
        for (long t = 0; t < cnt; ++t)
            T->fT[t] = T->fT[cap + t] = T->fT[2 * cap + t] = 0.0;
        for (long l = m0; l < m1; ++l) {
            double s[3];
            long j0[3];
            for (int a = 0; a < 3; ++a) {
                s[a] = (X[3 * l + a] - org[a]) / h - 0.5;
                j0[a] = stencil_first(kernel, s[a]);
            }
            double q = dV[l] * inv_h3;
            for (int dk = 0; dk < w; ++dk)
                for (int dj = 0; dj < w; ++dj)
                    for (int di = 0; di < w; ++di) {
                        long i = j0[0] + di, j = j0[1] + dj, k = j0[2] + dk;
                        double wt = or_phi(kernel, s[0] - (double)i) *
                                    or_phi(kernel, s[1] - (double)j) *
                                    or_phi(kernel, s[2] - (double)k);
                        long t = T->stamp[cell_index(n, i, j, k)];
                        for (int a = 0; a < 3; ++a)
                            T->fT[a * cap + t] += F[3 * l + a] * q * wt;
                    }
        }
        /* u(m) = u(0) + dt f^m */
        for (long t = 0; t < cnt; ++t)
            for (int a = 0; a < 3; ++a)
                u[a * N + T->cells[t]] = T->u0[a * cap + t] + dt * T->fT[a * cap + t];
    }
    for (long t = 0; t < cnt; ++t) {
        if (f_out)
            for (int a = 0; a < 3; ++a)
                f_out[a * N + T->cells[t]] += T->fT[a * cap + t];
        T->stamp[T->cells[t]] = -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One multidirect-forcing call over P rigid particles.
 *   X_l   = X_r + R_l                                   (Eq. pr1, R_l def.)
 *   U^d_l = U_r + W_r x R_l                             (Eq. pr1)
 * order == OR_SEQUENTIAL: particles enter the Ns loop one after another in
 *   index order, each starting from the field left by the previous ones
 *   (Sec. 3.1: "each particle goes into 1 to Ns loop sequentially").
 * order == OR_SIMULTANEOUS: all markers share one Ns loop (variant).
 * F_out[M][3] receives each marker's final F^{Ns}; f_out (nullable) is
 * accumulated with the Eulerian force of every particle's final pass.
 * Returns 0, or -1 on allocation failure.                                   */
/* ------------------------------------------------------------------------ */
int or_multidirect(const int n[3], double h, const double org[3], double *u,
                   int P, const double *Xr, const double *Ur, const double *Wr,
                   const long *moff, const double *R, const double *dV, int Ns,
                   double dt, int kernel, int order, double *F_out,
                   double *f_out)
{
    long N = (long)n[0] * n[1] * n[2];
    long M = moff[P];
    double *X = (double *)malloc(sizeof(double) * 3 * (M > 0 ? M : 1));
    double *Ud = (double *)malloc(sizeof(double) * 3 * (M > 0 ? M : 1));
    touched_t T = {0};
    T.stamp = (long *)malloc(sizeof(long) * N);
    int rc = 0;
    if (!X || !Ud || !T.stamp) {
        rc = -1;
        goto done;
    }
    for (long c = 0; c < N; ++c)
        T.stamp[c] = -1;
    for (int p = 0; p < P; ++p)
        for (long l = moff[p]; l < moff[p + 1]; ++l) {
            const double *r = R + 3 * l;
            const double *W = Wr + 3 * p;
            for (int a = 0; a < 3; ++a)
                X[3 * l + a] = Xr[3 * p + a] + r[a];
            Ud[3 * l + 0] = Ur[3 * p + 0] + (W[1] * r[2] - W[2] * r[1]);
            Ud[3 * l + 1] = Ur[3 * p + 1] + (W[2] * r[0] - W[0] * r[2]);
            Ud[3 * l + 2] = Ur[3 * p + 2] + (W[0] * r[1] - W[1] * r[0]);
        }
    if (order == OR_SIMULTANEOUS) {
        rc = run_marker_set(n, h, org, u, 0, M, X, Ud, dV, Ns, dt, kernel,
                            F_out, f_out, &T);
    } else {
        for (int p = 0; p < P && rc == 0; ++p)
            rc = run_marker_set(n, h, org, u, moff[p], moff[p + 1], X, Ud, dV,
                                Ns, dt, kernel, F_out, f_out, &T);
    }
done:
    free(X);
    free(Ud);
    free(T.stamp);
    free(T.cells);
    free(T.u0);
    free(T.fT);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Particle volume fraction from the level set, Eq. (level-set function) and
 * Eq. (Heaviside): alpha = sum_m -phi_m H(-phi_m) / sum_m |phi_m| over the 8
 * corners (nodes) of a cell; H(x) = 1 for x > 0, else 0.
 * Reading: alpha = 1/2 when every corner has phi = 0 (0/0, measure zero).   */
/* ------------------------------------------------------------------------ */
static double pvf_alpha(const double phi[8])
{
    double num = 0.0, den = 0.0;
    for (int m = 0; m < 8; ++m) {
        if (-phi[m] > 0.0)
            num += -phi[m];
        den += fabs(phi[m]);
    }
    return den > 0.0 ? num / den : 0.5;
}

/* Ellipsoid level set, Eq. (level-set function of spheroidal geometries).
 * Reading: the printed x_{i,j,k} in the y and z terms stands for y and z.   */
static double level_set_ellipsoid(double x, double y, double z,
                                  const double c[3], const double ax[3])
{
    double a = (x - c[0]) / ax[0], b = (y - c[1]) / ax[1], d = (z - c[2]) / ax[2];
    return sqrt(a * a + b * b + d * d) - 1.0;
}

/* Volume sum_cells alpha h^3 of an ellipsoid on a (non-periodic) box of
 * n[3] cells -- the quantity of the sphere / ellipsoid PVF tables (Sec. 4.1). */
double or_pvf_ellipsoid_volume(const int n[3], double h, const double org[3],
                               const double centre[3], const double axes[3])
{
    double vol = 0.0;
    for (long k = 0; k < n[2]; ++k)
        for (long j = 0; j < n[1]; ++j)
            for (long i = 0; i < n[0]; ++i) {
                double phi[8];
                for (int m = 0; m < 8; ++m) {
                    double x = org[0] + (double)(i + (m & 1)) * h;
                    double y = org[1] + (double)(j + ((m >> 1) & 1)) * h;
                    double z = org[2] + (double)(k + ((m >> 2) & 1)) * h;
                    phi[m] = level_set_ellipsoid(x, y, z, centre, axes);
                }
                vol += pvf_alpha(phi) * h * h * h;
            }
    return vol;
}

/* ------------------------------------------------------------------------ */
/* Volume integrals of a particle through its PVF (Sec. 3.2.2 "flow
 * unsteadiness" terms, Sec. 4.1):
 *   Iu   = sum_c alpha_c u_c h^3
 *   Irxu = sum_c alpha_c (x_c - X_r) x u_c h^3
 *   vol  = sum_c alpha_c h^3
 * with alpha from the level set of an axis-aligned ellipsoid of semi-axes
 * (a, b, c) centred at X_r, Eq. (level-set function of spheroidal
 * geometries); a sphere is a = b = c = R.  Cells are visited around the
 * particle centre without wrapping, so x_c - X_r is already the nearest
 * periodic image; only the field index wraps.                              */
/* ------------------------------------------------------------------------ */
static void volume_integrals_one(const int n[3], double h, const double org[3], const double *u,
                                 const double c[3], const double axes[3], double *Iu, double *Irxu,
                                 double *vol)
{
    long N = (long)n[0] * n[1] * n[2];
    long lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = (long)floor((c[a] - axes[a] - org[a]) / h) - 1;
        hi[a] = (long)floor((c[a] + axes[a] - org[a]) / h) + 1;
    }
    double su[3] = {0, 0, 0}, sw[3] = {0, 0, 0}, sv = 0.0;
    double h3 = h * h * h;
    for (long k = lo[2]; k <= hi[2]; ++k)
        for (long j = lo[1]; j <= hi[1]; ++j)
            for (long i = lo[0]; i <= hi[0]; ++i) {
                double phi[8];
                for (int m = 0; m < 8; ++m) {
                    double x = org[0] + (double)(i + (m & 1)) * h;
                    double y = org[1] + (double)(j + ((m >> 1) & 1)) * h;
                    double z = org[2] + (double)(k + ((m >> 2) & 1)) * h;
                    phi[m] = level_set_ellipsoid(x, y, z, c, axes);
                }
                double al = pvf_alpha(phi);
                if (al == 0.0)
                    continue;
                long cc = cell_index(n, i, j, k);
                double uc[3] = {u[cc], u[N + cc], u[2 * N + cc]};
                double r[3] = {org[0] + ((double)i + 0.5) * h - c[0],
                               org[1] + ((double)j + 0.5) * h - c[1],
                               org[2] + ((double)k + 0.5) * h - c[2]};
                double wv = al * h3;
                su[0] += wv * uc[0];
                su[1] += wv * uc[1];
                su[2] += wv * uc[2];
                sw[0] += wv * (r[1] * uc[2] - r[2] * uc[1]);
                sw[1] += wv * (r[2] * uc[0] - r[0] * uc[2]);
                sw[2] += wv * (r[0] * uc[1] - r[1] * uc[0]);
                sv += wv;
            }
    for (int a = 0; a < 3; ++a) {
        Iu[a] = su[a];
        Irxu[a] = sw[a];
    }
    *vol = sv;
}

void or_volume_integrals(const int n[3], double h, const double org[3],
                         const double *u, int P, const double *Xr,
                         const double *radius, double *Iu, double *Irxu,
                         double *vol)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
        double axes[3] = {radius[p], radius[p], radius[p]};
        volume_integrals_one(n, h, org, u, Xr + 3 * p, axes, Iu + 3 * p, Irxu + 3 * p, vol + p);
    }
}

/* The same for ellipsoids: axes[P][3] = (a, b, c) of each particle. */
void or_volume_integrals_ellipsoid(const int n[3], double h, const double org[3],
                                   const double *u, int P, const double *Xr,
                                   const double *axes, double *Iu, double *Irxu,
                                   double *vol)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p)
        volume_integrals_one(n, h, org, u, Xr + 3 * p, axes + 3 * p, Iu + 3 * p, Irxu + 3 * p, vol + p);
}

/* ------------------------------------------------------------------------ */
/* Drag diagnostic, Eq. (FD): the marker-force sum plus the rate of change of
 * the velocity integral over the particle volume,
 *   F_D = -rho_f sum_l F_l dV_l + rho_f d/dt int_Vp u dV
 *       = F_ib + rho_f (Iu^{n+1} - Iu^n) / dt,
 * the time derivative taken as the difference of the PVF integrals.        */
/* ------------------------------------------------------------------------ */
void or_drag_force(int P, const double *Fib, const double *Iu_new, const double *Iu_old,
                   double rho_f, double dt, double *FD)
{
    for (long q = 0; q < 3L * P; ++q)
        FD[q] = Fib[q] + rho_f * (Iu_new[q] - Iu_old[q]) / dt;
}

/* ------------------------------------------------------------------------ */
/* Hydrodynamic force and torque on each particle, the first right-hand-side
 * terms of Eqs. (particle1) and (particle2):
 *   F_ib = -rho_f sum_l F_l dV_l,   T_ib = -rho_f sum_l R_l x F_l dV_l.
 * Sums are compensated (Kahan) and run in marker index order.               */
/* ------------------------------------------------------------------------ */
static void kahan_add(double *s, double *c, double x)
{
    double y = x - *c;
    double t = *s + y;
    *c = (t - *s) - y;
    *s = t;
}

void or_force_torque(int P, const long *moff, const double *R,
                     const double *dV, const double *F, double rho_f,
                     double *Fib, double *Tib)
{
    for (int p = 0; p < P; ++p) {
        double sf[3] = {0, 0, 0}, cf[3] = {0, 0, 0};
        double st[3] = {0, 0, 0}, ct[3] = {0, 0, 0};
        for (long l = moff[p]; l < moff[p + 1]; ++l) {
            const double *r = R + 3 * l;
            double g[3] = {F[3 * l] * dV[l], F[3 * l + 1] * dV[l], F[3 * l + 2] * dV[l]};
            double t[3] = {r[1] * g[2] - r[2] * g[1], r[2] * g[0] - r[0] * g[2],
                           r[0] * g[1] - r[1] * g[0]};
            for (int a = 0; a < 3; ++a) {
                kahan_add(&sf[a], &cf[a], g[a]);
                kahan_add(&st[a], &ct[a], t[a]);
            }
        }
        for (int a = 0; a < 3; ++a) {
            Fib[3 * p + a] = -rho_f * sf[a];
            Tib[3 * p + a] = -rho_f * st[a];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Repulsive-potential collision force, Eq. (DKT_model), and the Newton-Euler
 * update, Eqs. (particle1), (particle2) and (pr2).
 *   delta_ij = X_j - X_i (nearest periodic image), d = |delta_ij|,
 *   D_c = R_i + R_j + d_c; for d < D_c:
 *     F_c,ij = -(m ||g|| / eps_c) ((d - D_c)/d_c)^2 delta_ij / d.
 * Readings: delta_ij points from i to j (the force is then repulsive);
 *   m = (m_i + m_j)/2 so that F_c,ij = -F_c,ji; ||g|| is phys g_coll; a pair
 *   at d = 0 has no direction and gets no force; T_c = 0 (central force).
 * Newton-Euler (Reading of "second-order mid-point", Sec. 3.2.2):
 *   U^{n+1} = U^n + dt/(rho_p V_p) [F_ib + rho_f (Iu^{n+1} - Iu^n)/dt
 *                                   + (rho_p - rho_f) V_p g + F_c]
 *   W^{n+1} = W^n + dt/I_p [T_ib + rho_f (Irxu^{n+1} - Irxu^n)/dt + T_c]
 *   X^{n+1} = X^n + dt/2 (U^{n+1} + U^n)                    (Eq. pr2)
 * with V_p = 4/3 pi R^3 and I_p = 2/5 rho_p V_p R^2 (solid sphere).
 * phys = {rho_f, g0, g1, g2, g_coll, eps_c, d_c}.  Fc_out is nullable.      */
/* ------------------------------------------------------------------------ */
void or_collide_update(int P, double *Xr, double *Ur, double *Wr,
                       const double *radius, const double *rho_p,
                       const int n[3], double h, const double *phys, double dt,
                       const double *Fib, const double *Tib,
                       const double *Iu_new, const double *Iu_old,
                       const double *Irxu_new, const double *Irxu_old,
                       double *Fc_out)
{
    const double PI = 3.14159265358979323846;
    double rho_f = phys[0], g[3] = {phys[1], phys[2], phys[3]};
    double g_coll = phys[4], eps_c = phys[5], d_c = phys[6];
    double L[3] = {n[0] * h, n[1] * h, n[2] * h};
    double *Fc = (double *)calloc((size_t)3 * (P > 0 ? P : 1), sizeof(double));
    if (!Fc)
        return;
    for (int i = 0; i < P; ++i) {
        double mi = rho_p[i] * 4.0 / 3.0 * PI * radius[i] * radius[i] * radius[i];
        for (int j = 0; j < P; ++j) {
            if (j == i)
                continue;
            double mj = rho_p[j] * 4.0 / 3.0 * PI * radius[j] * radius[j] * radius[j];
            double del[3];
            for (int a = 0; a < 3; ++a) {
                double dd = Xr[3 * j + a] - Xr[3 * i + a];
                del[a] = dd - L[a] * nearbyint(dd / L[a]);
            }
            double d = sqrt(del[0] * del[0] + del[1] * del[1] + del[2] * del[2]);
            double Dc = radius[i] + radius[j] + d_c;
            if (d < Dc && d > 0.0) {
                double q = (d - Dc) / d_c;
                double coef = -(0.5 * (mi + mj) * g_coll / eps_c) * q * q / d;
                for (int a = 0; a < 3; ++a)
                    Fc[3 * i + a] += coef * del[a];
            }
        }
    }
    for (int p = 0; p < P; ++p) {
        double Rp = radius[p];
        double V = 4.0 / 3.0 * PI * Rp * Rp * Rp;
        double m = rho_p[p] * V;
        double I = 0.4 * m * Rp * Rp;
        for (int a = 0; a < 3; ++a) {
            double Un = Ur[3 * p + a];
            double rhs = Fib[3 * p + a] +
                         rho_f * (Iu_new[3 * p + a] - Iu_old[3 * p + a]) / dt +
                         (rho_p[p] - rho_f) * V * g[a] + Fc[3 * p + a];
            double Unew = Un + dt / m * rhs;
            double trq = Tib[3 * p + a] +
                         rho_f * (Irxu_new[3 * p + a] - Irxu_old[3 * p + a]) / dt;
            Wr[3 * p + a] += dt / I * trq;
            Ur[3 * p + a] = Unew;
            Xr[3 * p + a] += 0.5 * dt * (Unew + Un);
            if (Fc_out)
                Fc_out[3 * p + a] = Fc[3 * p + a];
        }
    }
    free(Fc);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0)
        omp_set_num_threads(t);
#else
    (void)t;
#endif
}
