/*
 * FP64 CPU oracle for the demagnetising field of a finite-difference mesh.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code with the CUDA path and is deliberately plain and slow: every step is
 * the textbook definition, written so it can be checked against the paper by
 * eye.
 *
 * Contents (paper: "Boris Computational Spintronics", arXiv 2008.02478):
 *   - Newell f and g auxiliary functions and the 27-point cell-averaged
 *     demagnetising tensor (Table 1 "Demagnetizing Field": N from Newell et
 *     al., Ref. [50]; the formulas themselves are not printed in the paper and
 *     are restated here from the published Newell-Williams-Dunlop result).
 *   - A far-field asymptotic form of the same tensor (box-averaged dipole,
 *     second order in the cell size), used beyond a switch radius.
 *   - The demagnetising field H(r0) = -sum_r N(r - r0) M(r) (Table 1; Eq. 4 for
 *     one mesh) as (i) an O(N^2) direct sum and (ii) the convolution theorem
 *     with zero padding to twice the mesh size (Section 7), using this file's
 *     own mixed-radix FFT.
 *
 * Layout of every field: SoA [3][nz][ny][nx], x fastest.  Tensor tables:
 * [6][nz][ny][nx] for displacements (i dx, j dy, k dz), 0 <= i < nx etc., in
 * component order xx, yy, zz, xy, xz, yz.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Newell auxiliary functions                                                */
/* ------------------------------------------------------------------------ */

/* f(x,y,z): even in each argument.  A term whose polynomial prefactor is zero
 * is taken as zero (the 0*inf and 0/0 limits of the closed form). */
double orc_newell_f(double x, double y, double z)
{
    x = fabs(x); y = fabs(y); z = fabs(z);
    double x2 = x * x, y2 = y * y, z2 = z * z;
    double R = sqrt(x2 + y2 + z2);
    if (R == 0.0) return 0.0;
    double s = 0.0, p;
    p = 0.5 * y * (z2 - x2);
    if (p != 0.0) s += p * asinh(y / sqrt(x2 + z2));
    p = 0.5 * z * (y2 - x2);
    if (p != 0.0) s += p * asinh(z / sqrt(x2 + y2));
    p = x * y * z;
    if (p != 0.0) s -= p * atan(y * z / (x * R));
    s += (2.0 * x2 - y2 - z2) * R / 6.0;
    return s;
}

/* g(x,y,z): odd in x and in y, even in z. */
double orc_newell_g(double x, double y, double z)
{
    double sgn = ((x < 0) ? -1.0 : 1.0) * ((y < 0) ? -1.0 : 1.0);
    x = fabs(x); y = fabs(y); z = fabs(z);
    double x2 = x * x, y2 = y * y, z2 = z * z;
    double R = sqrt(x2 + y2 + z2);
    if (R == 0.0) return 0.0;
    double s = 0.0, p;
    p = x * y * z;
    if (p != 0.0) s += p * asinh(z / sqrt(x2 + y2));
    p = y * (3.0 * z2 - y2) / 6.0;
    if (p != 0.0) s += p * asinh(x / sqrt(y2 + z2));
    p = x * (3.0 * z2 - x2) / 6.0;
    if (p != 0.0) s += p * asinh(y / sqrt(x2 + z2));
    p = z * z2 / 6.0;
    if (p != 0.0) s -= p * atan(x * y / (z * R));
    p = 0.5 * z * y2;
    if (p != 0.0) s -= p * atan(x * z / (y * R));
    p = 0.5 * z * x2;
    if (p != 0.0) s -= p * atan(y * z / (x * R));
    s -= x * y * R / 3.0;
    return sgn * s;
}

/* Weighted 27-point sum sum_e w(e) F(X + ex a, Y + ey b, Z + ez c) with
 * w = prod w1, w1(0) = 2, w1(+-1) = -1, divided by 4 pi a b c. */
static double stencil27(double (*F)(double, double, double),
                        double X, double Y, double Z, double a, double b, double c)
{
    double s = 0.0;
    for (int ex = -1; ex <= 1; ex++)
        for (int ey = -1; ey <= 1; ey++)
            for (int ez = -1; ez <= 1; ez++) {
                double w = (ex ? -1.0 : 2.0) * (ey ? -1.0 : 2.0) * (ez ? -1.0 : 2.0);
                s += w * F(X + ex * a, Y + ey * b, Z + ez * c);
            }
    return s / (4.0 * ORC_PI * a * b * c);
}

/* Exact cell-averaged tensor between two cells of size (dx,dy,dz) whose
 * centres are separated by (X,Y,Z).  out = {xx, yy, zz, xy, xz, yz}. */
void orc_newell_exact(double X, double Y, double Z, double dx, double dy, double dz, double* out)
{
    out[0] = stencil27(orc_newell_f, X, Y, Z, dx, dy, dz);
    out[1] = stencil27(orc_newell_f, Y, X, Z, dy, dx, dz);
    out[2] = stencil27(orc_newell_f, Z, Y, X, dz, dy, dx);
    out[3] = stencil27(orc_newell_g, X, Y, Z, dx, dy, dz);
    out[4] = stencil27(orc_newell_g, X, Z, Y, dx, dz, dy);
    out[5] = stencil27(orc_newell_g, Y, Z, X, dy, dz, dx);
}

/* Far field: N_ij = -(V/4pi) [D_ij + sum_k (h_k^2/12) d_k^2 D_ij] with
 * D_ij = d_i d_j (1/r) = (3 x_i x_j - r^2 delta_ij)/r^5.  The second-order term
 * is the average of the Taylor expansion of D over the difference of two
 * points drawn uniformly from the source and target boxes (variance h_k^2/6
 * per axis).  Derivatives of D are written out below from
 *   d_k d_k D_ij = d_i d_j d_k d_k (1/r)
 * using the general formula for the fourth derivative of 1/r:
 *   d_i d_j d_k d_l (1/r) = 105 x_i x_j x_k x_l / r^9
 *      - 15 (x_i x_j d_kl + x_i x_k d_jl + x_i x_l d_jk + x_j x_k d_il
 *            + x_j x_l d_ik + x_k x_l d_ij) / r^7
 *      + 3 (d_ij d_kl + d_ik d_jl + d_il d_jk) / r^5. */
static double d4inv(const double* x, double r, int i, int j, int k, int l)
{
#define DL(a, b) ((a) == (b) ? 1.0 : 0.0)
    double r2 = r * r, r5 = r2 * r2 * r, r7 = r5 * r2, r9 = r7 * r2;
    double t = 105.0 * x[i] * x[j] * x[k] * x[l] / r9;
    t -= 15.0 * (x[i] * x[j] * DL(k, l) + x[i] * x[k] * DL(j, l) + x[i] * x[l] * DL(j, k) +
                 x[j] * x[k] * DL(i, l) + x[j] * x[l] * DL(i, k) + x[k] * x[l] * DL(i, j)) / r7;
    t += 3.0 * (DL(i, j) * DL(k, l) + DL(i, k) * DL(j, l) + DL(i, l) * DL(j, k)) / r5;
    return t;
#undef DL
}

void orc_newell_asymptotic(double X, double Y, double Z, double dx, double dy, double dz, double* out)
{
    double x[3] = {X, Y, Z};
    double h[3] = {dx, dy, dz};
    double r = sqrt(X * X + Y * Y + Z * Z);
    double r2 = r * r, r5 = r2 * r2 * r;
    double V = dx * dy * dz;
    static const int ci[6] = {0, 1, 2, 0, 0, 1};
    static const int cj[6] = {0, 1, 2, 1, 2, 2};
    for (int c = 0; c < 6; c++) {
        int i = ci[c], j = cj[c];
        double D = (3.0 * x[i] * x[j] - (i == j ? r2 : 0.0)) / r5;
        double corr = 0.0;
        for (int k = 0; k < 3; k++) corr += h[k] * h[k] / 12.0 * d4inv(x, r, i, j, k, k);
        out[c] = -V / (4.0 * ORC_PI) * (D + corr);
    }
}

/* Tensor table for the displacement octant 0<=i<nx, 0<=j<ny, 0<=k<nz:
 * exact formula when |r| <= rs * max(dx,dy,dz), asymptotic beyond. */
void orc_tensor_table(int nx, int ny, int nz, double dx, double dy, double dz, double rs, double* out)
{
    size_t n = (size_t)nx * ny * nz;
    double hmax = fmax(dx, fmax(dy, dz));
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                double X = i * dx, Y = j * dy, Z = k * dz, v[6];
                double r = sqrt(X * X + Y * Y + Z * Z);
                if (r <= rs * hmax)
                    orc_newell_exact(X, Y, Z, dx, dy, dz, v);
                else
                    orc_newell_asymptotic(X, Y, Z, dx, dy, dz, v);
                size_t idx = ((size_t)k * ny + j) * nx + i;
                for (int c = 0; c < 6; c++) out[c * n + idx] = v[c];
            }
}

/* Periodic boundary conditions by multiple images (Section 4, extending
 * Eq. 4): the field at a cell of the computational mesh includes the
 * sources in the images of the mesh displaced by whole periods
 * (a nx dx, b ny dy, c nz dz), |a| <= kx, |b| <= ky, |c| <= kz.  For a
 * displacement d between two mesh cells the kernel is therefore the sum of
 * the cell tensor over the images, N(d + (a Lx, b Ly, c Lz)); the table keeps
 * the octant form because the image set is symmetric. */
void orc_tensor_table_pbc(int nx, int ny, int nz, double dx, double dy, double dz, double rs, int kx, int ky, int kz,
                          double* out)
{
    size_t n = (size_t)nx * ny * nz;
    double hmax = fmax(dx, fmax(dy, dz));
    double Lx = nx * dx, Ly = ny * dy, Lz = nz * dz;
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                double acc[6] = {0, 0, 0, 0, 0, 0};
                for (int c = -kz; c <= kz; c++)
                    for (int b = -ky; b <= ky; b++)
                        for (int a = -kx; a <= kx; a++) {
                            double X = i * dx + a * Lx, Y = j * dy + b * Ly, Z = k * dz + c * Lz, v[6];
                            double r = sqrt(X * X + Y * Y + Z * Z);
                            if (r <= rs * hmax)
                                orc_newell_exact(X, Y, Z, dx, dy, dz, v);
                            else
                                orc_newell_asymptotic(X, Y, Z, dx, dy, dz, v);
                            for (int q = 0; q < 6; q++) acc[q] += v[q];
                        }
                size_t idx = ((size_t)k * ny + j) * nx + i;
                for (int q = 0; q < 6; q++) out[q * n + idx] = acc[q];
            }
}

/* ------------------------------------------------------------------------ */
/* Oersted kernel (Table 1: H(r0) = sum_r K(r - r0) J_C(r); the formulas of   */
/* its Ref. [63] are not in the paper and are derived here)                  */
/* ------------------------------------------------------------------------ */
/* For a uniform current density J in a source cell, Biot-Savart averaged over
 * a target cell at centre displacement D (target - source) gives
 *   H = J x g(D),  g(D) = -(1/(4 pi V)) grad_D P(D),
 *   P(D) = int_target int_source dr dr' / |r - r'|.
 * The demagnetising tensor of the same two cells is N_ij = -(1/(4 pi V))
 * d_i d_j P = d_i g_j, so g_k is an antiderivative of N_kk along axis k and
 * g -> 0 far away:
 *   g_k(D) = g_k(D + (t_e - D_k) e_k) - int_{D_k}^{t_e} N_kk(D + (t - D_k) e_k) dt,
 * with the end point t_e in the far zone, where
 *   g_k = -(V/4 pi) d_k [1/r + sum_m (h_m^2/12) d_m^2 (1/r)]
 * (the gradient of the box-averaged potential whose Hessian is the far form
 * of N).  The integral runs over intervals that end on multiples of h_k
 * (where N has its kinks), 16-point Gauss-Legendre rules each. */
static void gl16(double* xs, double* ws)
{
    /* nodes and weights on [-1, 1] by Newton iteration on P_16 */
    const int n = 16;
    for (int i = 0; i < n; i++) {
        double x = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; k++) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double dp = n * (x * p1 - p0) / (x * x - 1.0);
        xs[i] = x;
        ws[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

static void oersted_far(const double* x, const double* h, double V, double* g)
{
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2], r = sqrt(r2);
    double r3 = r2 * r, r5 = r3 * r2, r7 = r5 * r2;
    for (int k = 0; k < 3; k++) {
        double s = -x[k] / r3;
        for (int m = 0; m < 3; m++)
            s += h[m] * h[m] / 12.0 *
                 ((6.0 * x[m] * (m == k ? 1.0 : 0.0) - 2.0 * x[k]) / r5 - 5.0 * x[k] * (3.0 * x[m] * x[m] - r2) / r7);
        g[k] = -V / (4.0 * ORC_PI) * s;
    }
}

/* N_kk at a point, exact form */
static double nkk_exact(int k, const double* x, const double* h)
{
    double v[6];
    orc_newell_exact(x[0], x[1], x[2], h[0], h[1], h[2], v);
    return v[k];
}

/* g(D) at an arbitrary displacement; rs: far zone beyond rs * max cell size */
void orc_oersted_g(double X, double Y, double Z, double dx, double dy, double dz, double rs, double* g)
{
    double h[3] = {dx, dy, dz}, D[3] = {X, Y, Z};
    double hmax = fmax(dx, fmax(dy, dz)), V = dx * dy * dz;
    double r = sqrt(X * X + Y * Y + Z * Z);
    if (r > rs * hmax) {
        oersted_far(D, h, V, g);
        return;
    }
    double xs[16], ws[16];
    gl16(xs, ws);
    for (int k = 0; k < 3; k++) {
        /* integrate along +k from |D_k| (g_k is odd in D_k) */
        double s = D[k] < 0 ? -1.0 : 1.0;
        double p[3] = {D[0], D[1], D[2]};
        p[k] = fabs(D[k]);
        double t = p[k], acc = 0.0;
        for (;;) {
            double q[3] = {p[0], p[1], p[2]};
            q[k] = t;
            double rq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
            if (rq > rs * hmax) break;
            /* intervals end on multiples of h_k, where N has its kinks */
            double b = (floor(t / h[k] * (1.0 + 1e-14)) + 1.0) * h[k];
            double a = t, half = 0.5 * (b - a), mid = 0.5 * (a + b);
            for (int i = 0; i < 16; i++) {
                q[k] = mid + half * xs[i];
                acc += ws[i] * half * nkk_exact(k, q, h);
            }
            t = b;
        }
        double e[3] = {p[0], p[1], p[2]}, ge[3];
        e[k] = t;
        oersted_far(e, h, V, ge);
        g[k] = s * (ge[k] - acc);
    }
}

/* octant table [3][nz][ny][nx] of g at (i dx, j dy, k dz) */
void orc_oersted_table(int nx, int ny, int nz, double dx, double dy, double dz, double rs, double* out)
{
    size_t n = (size_t)nx * ny * nz;
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                double g[3];
                orc_oersted_g(i * dx, j * dy, k * dz, dx, dy, dz, rs, g);
                size_t idx = ((size_t)k * ny + j) * nx + i;
                for (int c = 0; c < 3; c++) out[c * n + idx] = g[c];
            }
}

/* Direct sum H(r0) = sum_r J(r) x g(r0 - r): g_k is odd in its own axis and
 * even in the other two, so a signed displacement reads the octant table
 * with the sign of its k-th coordinate. */
void orc_oersted_direct(int nx, int ny, int nz, const double* G, const double* J, double* H)
{
    size_t n = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 16)
    for (long t = 0; t < (long)n; t++) {
        int ti = (int)(t % nx), tj = (int)((t / nx) % ny), tk = (int)(t / ((size_t)nx * ny));
        double hx = 0, hy = 0, hz = 0;
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    int di = ti - i, dj = tj - j, dk = tk - k;
                    size_t idx = ((size_t)abs(dk) * ny + abs(dj)) * nx + abs(di);
                    double gx = (di < 0 ? -1.0 : 1.0) * G[idx];
                    double gy = (dj < 0 ? -1.0 : 1.0) * G[n + idx];
                    double gz = (dk < 0 ? -1.0 : 1.0) * G[2 * n + idx];
                    size_t s = ((size_t)k * ny + j) * nx + i;
                    double jx = J[s], jy = J[n + s], jz = J[2 * n + s];
                    hx += jy * gz - jz * gy;
                    hy += jz * gx - jx * gz;
                    hz += jx * gy - jy * gx;
                }
        H[t] = hx;
        H[n + t] = hy;
        H[2 * n + t] = hz;
    }
}

/* Tensor entry for a signed displacement (i,j,k) from the octant table:
 * diagonal components are even in every axis; N_xy is odd in x and y, N_xz odd
 * in x and z, N_yz odd in y and z. */
static void tensor_signed(const double* T, int nx, int ny, int nz, int i, int j, int k, double* v)
{
    size_t n = (size_t)nx * ny * nz;
    size_t idx = ((size_t)abs(k) * ny + abs(j)) * nx + abs(i);
    double sx = i < 0 ? -1.0 : 1.0, sy = j < 0 ? -1.0 : 1.0, sz = k < 0 ? -1.0 : 1.0;
    v[0] = T[idx];
    v[1] = T[n + idx];
    v[2] = T[2 * n + idx];
    v[3] = sx * sy * T[3 * n + idx];
    v[4] = sx * sz * T[4 * n + idx];
    v[5] = sy * sz * T[5 * n + idx];
}

/* ------------------------------------------------------------------------ */
/* Direct sum H(r0) = -sum_r N(r - r0) M(r)                                  */
/* ------------------------------------------------------------------------ */

static void direct_one(const double* T, int nx, int ny, int nz, const double* M, size_t t, double* h)
{
    size_t n = (size_t)nx * ny * nz;
    int ti = (int)(t % nx), tj = (int)((t / nx) % ny), tk = (int)(t / ((size_t)nx * ny));
    double hx = 0, hy = 0, hz = 0;
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                double v[6];
                tensor_signed(T, nx, ny, nz, i - ti, j - tj, k - tk, v);
                size_t s = ((size_t)k * ny + j) * nx + i;
                double mx = M[s], my = M[n + s], mz = M[2 * n + s];
                hx -= v[0] * mx + v[3] * my + v[4] * mz;
                hy -= v[3] * mx + v[1] * my + v[5] * mz;
                hz -= v[4] * mx + v[5] * my + v[2] * mz;
            }
    h[0] = hx; h[1] = hy; h[2] = hz;
}

void orc_demag_direct(int nx, int ny, int nz, const double* T, const double* M, double* H)
{
    size_t n = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 16)
    for (long t = 0; t < (long)n; t++) {
        double h[3];
        direct_one(T, nx, ny, nz, M, (size_t)t, h);
        H[t] = h[0]; H[n + t] = h[1]; H[2 * n + t] = h[2];
    }
}

/* Direct sum at a list of target cells; H is [ns][3]. */
void orc_demag_direct_at(int nx, int ny, int nz, const double* T, const double* M,
                         int ns, const int64_t* cells, double* H)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < ns; s++) direct_one(T, nx, ny, nz, M, (size_t)cells[s], H + 3 * s);
}

/* ------------------------------------------------------------------------ */
/* Mixed-radix FFT (any length), FP64                                        */
/* ------------------------------------------------------------------------ */
/* X[k] = sum_j x[j] exp(sign * 2 pi i j k / n).  Recursive decimation in time
 * by the smallest prime factor p of n: the p interleaved subsequences are
 * transformed, then combined with X[k + q n/p] = sum_r W^{r(k + q n/p)} Y_r[k].
 * W^e is read from a table tw[e] = exp(sign 2 pi i e / n_top) at stride
 * n_top / n. */

static int smallest_factor(int n)
{
    for (int p = 2; p * p <= n; p++)
        if (n % p == 0) return p;
    return n;
}

static void fft_rec(const double complex* in, int istride, double complex* out, int n,
                    const double complex* tw, int ntop, double complex* scratch)
{
    if (n == 1) { out[0] = in[0]; return; }
    int p = smallest_factor(n), m = n / p, step = ntop / n;
    for (int r = 0; r < p; r++)
        fft_rec(in + (size_t)r * istride, istride * p, out + (size_t)r * m, m, tw, ntop, scratch + n);
    for (int k = 0; k < m; k++)
        for (int q = 0; q < p; q++) {
            int kk = k + q * m;
            double complex acc = 0.0;
            for (int r = 0; r < p; r++) {
                long e = ((long)r * kk) % n;
                acc += out[(size_t)r * m + k] * tw[e * step];
            }
            scratch[kk] = acc;
        }
    memcpy(out, scratch, sizeof(double complex) * n);
}

/* scratch needs 2n entries. */
static void fft1d(double complex* line, int n, const double complex* tw, double complex* tmp,
                  double complex* scratch)
{
    if (n == 1) return;
    fft_rec(line, 1, tmp, n, tw, n, scratch);
    memcpy(line, tmp, sizeof(double complex) * n);
}

static double complex* twiddles(int n, int sign)
{
    double complex* tw = malloc(sizeof(double complex) * n);
    for (int e = 0; e < n; e++) {
        double a = 2.0 * ORC_PI * e / n;
        tw[e] = cos(a) + I * (sign * sin(a));
    }
    return tw;
}

/* In-place 3D FFT of a[n2][n1][n0] (n0 fastest), one axis at a time. */
void orc_fft3d(double complex* a, int n0, int n1, int n2, int sign)
{
    int dims[3] = {n0, n1, n2};
    size_t strides[3] = {1, (size_t)n0, (size_t)n0 * n1};
    for (int ax = 0; ax < 3; ax++) {
        int n = dims[ax];
        if (n == 1) continue;
        double complex* tw = twiddles(n, sign);
        size_t st = strides[ax];
        size_t nlines = (size_t)n0 * n1 * n2 / n;
#pragma omp parallel
        {
            double complex* line = malloc(sizeof(double complex) * n);
            double complex* tmp = malloc(sizeof(double complex) * n);
            double complex* scr = malloc(sizeof(double complex) * 2 * n);
#pragma omp for schedule(static)
            for (long L = 0; L < (long)nlines; L++) {
                /* line L: all index combinations of the two other axes */
                size_t base;
                if (ax == 0) base = (size_t)L * n0;
                else if (ax == 1) base = ((size_t)L / n0) * n0 * n1 + ((size_t)L % n0);
                else base = (size_t)L;
                for (int j = 0; j < n; j++) line[j] = a[base + j * st];
                fft1d(line, n, tw, tmp, scr);
                for (int j = 0; j < n; j++) a[base + j * st] = line[j];
            }
            free(line); free(tmp); free(scr);
        }
        free(tw);
    }
}

/* 1D transform of a single line (used by the oracle's own pin tests). */
void orc_fft1d(double complex* a, int n, int sign)
{
    double complex* tw = twiddles(n, sign);
    double complex* tmp = malloc(sizeof(double complex) * n);
    double complex* scr = malloc(sizeof(double complex) * 2 * n);
    fft1d(a, n, tw, tmp, scr);
    free(tw); free(tmp); free(scr);
}

/* ------------------------------------------------------------------------ */
/* Convolution-theorem demag (Section 7): pad each axis of length n > 1 to    */
/* 2n, transform M and the padded tensor, multiply, transform back, crop.     */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz, px, py, pz;
    double complex* K[6]; /* FFT of the padded tensor components */
} orc_plan;

static int padlen(int n) { return n > 1 ? 2 * n : 1; }

/* Signed displacement stored at padded index idx of a length-P axis for a mesh
 * of n cells: idx < n -> idx; idx > P - n -> idx - P; otherwise no displacement. */
static int pad_disp(int idx, int n, int P, int* ok)
{
    if (idx < n) { *ok = 1; return idx; }
    if (idx > P - n) { *ok = 1; return idx - P; }
    *ok = 0;
    return 0;
}

void* orc_demag_plan(int nx, int ny, int nz, const double* T)
{
    orc_plan* p = calloc(1, sizeof(orc_plan));
    p->nx = nx; p->ny = ny; p->nz = nz;
    p->px = padlen(nx); p->py = padlen(ny); p->pz = padlen(nz);
    size_t P = (size_t)p->px * p->py * p->pz;
    for (int c = 0; c < 6; c++) {
        p->K[c] = calloc(P, sizeof(double complex));
        if (!p->K[c]) return NULL;
    }
    for (int K = 0; K < p->pz; K++)
        for (int J = 0; J < p->py; J++)
            for (int Ii = 0; Ii < p->px; Ii++) {
                int okx, oky, okz;
                int i = pad_disp(Ii, nx, p->px, &okx);
                int j = pad_disp(J, ny, p->py, &oky);
                int k = pad_disp(K, nz, p->pz, &okz);
                if (!(okx && oky && okz)) continue;
                double v[6];
                tensor_signed(T, nx, ny, nz, i, j, k, v);
                size_t idx = ((size_t)K * p->py + J) * p->px + Ii;
                for (int c = 0; c < 6; c++) p->K[c][idx] = v[c];
            }
    for (int c = 0; c < 6; c++) orc_fft3d(p->K[c], p->px, p->py, p->pz, -1);
    return p;
}

void orc_demag_plan_free(void* vp)
{
    orc_plan* p = vp;
    if (!p) return;
    for (int c = 0; c < 6; c++) free(p->K[c]);
    free(p);
}

/* Copy out the kernel spectrum (complex, [6][pz][py][px], interleaved re/im). */
void orc_demag_plan_spectrum(void* vp, double* out)
{
    orc_plan* p = vp;
    size_t P = (size_t)p->px * p->py * p->pz;
    for (int c = 0; c < 6; c++) memcpy(out + 2 * c * P, p->K[c], sizeof(double complex) * P);
}

void orc_demag_plan_dims(void* vp, int* out)
{
    orc_plan* p = vp;
    out[0] = p->px; out[1] = p->py; out[2] = p->pz;
}

/* H = -N * M by the convolution theorem.  Returns 0 on success. */
int orc_demag_fft(void* vp, const double* M, double* H)
{
    orc_plan* p = vp;
    int nx = p->nx, ny = p->ny, nz = p->nz;
    size_t n = (size_t)nx * ny * nz;
    size_t P = (size_t)p->px * p->py * p->pz;
    double complex* Mh[3];
    for (int c = 0; c < 3; c++) {
        Mh[c] = calloc(P, sizeof(double complex));
        if (!Mh[c]) return -1;
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++)
                    Mh[c][((size_t)k * p->py + j) * p->px + i] = M[c * n + ((size_t)k * ny + j) * nx + i];
        orc_fft3d(Mh[c], p->px, p->py, p->pz, -1);
    }
    /* H^ = -K^ M^ with K symmetric: rows (xx xy xz), (xy yy yz), (xz yz zz) */
#pragma omp parallel for schedule(static)
    for (long q = 0; q < (long)P; q++) {
        double complex mx = Mh[0][q], my = Mh[1][q], mz = Mh[2][q];
        double complex kxx = p->K[0][q], kyy = p->K[1][q], kzz = p->K[2][q];
        double complex kxy = p->K[3][q], kxz = p->K[4][q], kyz = p->K[5][q];
        Mh[0][q] = -(kxx * mx + kxy * my + kxz * mz);
        Mh[1][q] = -(kxy * mx + kyy * my + kyz * mz);
        Mh[2][q] = -(kxz * mx + kyz * my + kzz * mz);
    }
    for (int c = 0; c < 3; c++) {
        orc_fft3d(Mh[c], p->px, p->py, p->pz, +1);
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++)
                    H[c * n + ((size_t)k * ny + j) * nx + i] =
                        creal(Mh[c][((size_t)k * p->py + j) * p->px + i]) / (double)P;
        free(Mh[c]);
    }
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the parallel loops that follow (n >= 1); timing only */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Multi-mesh (Eq. 4): cells of different z thickness                        */
/* ------------------------------------------------------------------------ */
/* Generalised stencil for a target box of z size a and a source box of z size
 * b (equal in-plane sizes hx, hy).  Per axis the double integral over the two
 * boxes of a function whose second antiderivative is F is
 *   F(z + s) - F(z + d) - F(z - d) + F(z - s),  s = (a + b)/2, d = (a - b)/2,
 * which is F(z+h) - 2F(z) + F(z-h) for a = b: the Newell weights (2, -1, -1)
 * are minus this.  The tensor is normalised by 1/(4 pi hx hy a) (target
 * volume). */
typedef struct {
    int n;
    double off[4], w[4];
} orc_axis_stencil;

static orc_axis_stencil stencil_equal(double h)
{
    orc_axis_stencil s = {3, {-h, 0.0, h, 0}, {-1.0, 2.0, -1.0, 0}};
    return s;
}

static orc_axis_stencil stencil_pair(double a, double b)
{
    double s = 0.5 * (a + b), d = 0.5 * (a - b);
    orc_axis_stencil st = {4, {-s, -d, d, s}, {1.0, -1.0, -1.0, 1.0}};
    /* minus the double integral: -[F(z+s) - F(z+d) - F(z-d) + F(z-s)] */
    for (int i = 0; i < 4; i++) st.w[i] = -st.w[i];
    return st;
}

static double stencil3(double (*F)(double, double, double), double X, double Y, double Z,
                       const orc_axis_stencil* s1, const orc_axis_stencil* s2, const orc_axis_stencil* s3)
{
    double acc = 0.0;
    for (int i = 0; i < s1->n; i++)
        for (int j = 0; j < s2->n; j++)
            for (int k = 0; k < s3->n; k++)
                acc += s1->w[i] * s2->w[j] * s3->w[k] * F(X + s1->off[i], Y + s2->off[j], Z + s3->off[k]);
    return acc;
}

/* Exact pair tensor at centre separation (X,Y,Z), target z size a, source z
 * size b.  out = {xx, yy, zz, xy, xz, yz}. */
void orc_newell_pair_exact(double X, double Y, double Z, double hx, double hy, double a, double b, double* out)
{
    orc_axis_stencil sx = stencil_equal(hx), sy = stencil_equal(hy), sz = stencil_pair(a, b);
    double norm = 1.0 / (4.0 * ORC_PI * hx * hy * a);
    out[0] = norm * stencil3(orc_newell_f, X, Y, Z, &sx, &sy, &sz);
    out[1] = norm * stencil3(orc_newell_f, Y, X, Z, &sy, &sx, &sz);
    out[2] = norm * stencil3(orc_newell_f, Z, Y, X, &sz, &sy, &sx);
    out[3] = norm * stencil3(orc_newell_g, X, Y, Z, &sx, &sy, &sz);
    out[4] = norm * stencil3(orc_newell_g, X, Z, Y, &sx, &sz, &sy);
    out[5] = norm * stencil3(orc_newell_g, Y, Z, X, &sy, &sz, &sx);
}

/* Far field of the pair tensor: box-averaged dipole expansion with the
 * variance of the difference of two uniform points per axis, hx^2/6, hy^2/6
 * and (a^2 + b^2)/12, and the source volume hx hy b. */
void orc_newell_pair_asymptotic(double X, double Y, double Z, double hx, double hy, double a, double b, double* out)
{
    double x[3] = {X, Y, Z};
    double var[3] = {hx * hx / 6.0, hy * hy / 6.0, (a * a + b * b) / 12.0};
    double r = sqrt(X * X + Y * Y + Z * Z);
    double r2 = r * r, r5 = r2 * r2 * r;
    double Vs = hx * hy * b;
    static const int ci[6] = {0, 1, 2, 0, 0, 1};
    static const int cj[6] = {0, 1, 2, 1, 2, 2};
    for (int c = 0; c < 6; c++) {
        int i = ci[c], j = cj[c];
        double D = (3.0 * x[i] * x[j] - (i == j ? r2 : 0.0)) / r5;
        double corr = 0.0;
        for (int k = 0; k < 3; k++) corr += 0.5 * var[k] * d4inv(x, r, i, j, k, k);
        out[c] = -Vs / (4.0 * ORC_PI) * (D + corr);
    }
}

/* Pair tensor with the far-field switch at rs times the largest cell size. */
void orc_newell_pair(double X, double Y, double Z, double hx, double hy, double a, double b, double rs, double* out)
{
    double hmax = fmax(fmax(hx, hy), fmax(a, b));
    if (sqrt(X * X + Y * Y + Z * Z) <= rs * hmax) orc_newell_pair_exact(X, Y, Z, hx, hy, a, b, out);
    else orc_newell_pair_asymptotic(X, Y, Z, hx, hy, a, b, out);
}

/* Direct sum of Eq. 4 over a stack of layers sharing the in-plane cell
 * (hx, hy).  Layer l: nxyz[3l..3l+2] cells, z size hz[l], in-plane offset
 * (ox[l], oy[l]) in cells, bottom face at zb[l]; fields of all layers are
 * concatenated, each SoA [3][nz][ny][nx].  H at the cells listed in `cells`
 * (global cell index into the concatenation) -> H[3 * s + c]. */
void orc_multilayer_direct_at(int nl, const int* nxyz, const double* hz, const int* ox, const int* oy,
                              const double* zb, double hx, double hy, double rs, const double* M, int ns,
                              const int64_t* cells, double* H)
{
    long off[64];
    long tot = 0;
    for (int l = 0; l < nl; l++) {
        off[l] = tot;
        tot += 3L * nxyz[3 * l] * nxyz[3 * l + 1] * nxyz[3 * l + 2];
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < ns; s++) {
        /* locate the target cell */
        long g = cells[s], base = 0;
        int tl = 0;
        for (int l = 0; l < nl; l++) {
            long n = (long)nxyz[3 * l] * nxyz[3 * l + 1] * nxyz[3 * l + 2];
            if (g < base + n) { tl = l; break; }
            base += n;
        }
        long loc = g - base;
        int tnx = nxyz[3 * tl], tny = nxyz[3 * tl + 1];
        int ti = (int)(loc % tnx), tj = (int)((loc / tnx) % tny), tk = (int)(loc / ((long)tnx * tny));
        double tx = (ox[tl] + ti + 0.5) * hx, ty = (oy[tl] + tj + 0.5) * hy, tz = zb[tl] + (tk + 0.5) * hz[tl];
        double h3[3] = {0, 0, 0};
        for (int l = 0; l < nl; l++) {
            int nx = nxyz[3 * l], ny = nxyz[3 * l + 1], nz = nxyz[3 * l + 2];
            long n = (long)nx * ny * nz;
            const double* Ml = M + off[l];
            for (int k = 0; k < nz; k++)
                for (int j = 0; j < ny; j++)
                    for (int i = 0; i < nx; i++) {
                        double sx = (ox[l] + i + 0.5) * hx, sy = (oy[l] + j + 0.5) * hy, sz = zb[l] + (k + 0.5) * hz[l];
                        double v[6];
                        orc_newell_pair(tx - sx, ty - sy, tz - sz, hx, hy, hz[tl], hz[l], rs, v);
                        long c = ((long)k * ny + j) * nx + i;
                        double mx = Ml[c], my = Ml[n + c], mz = Ml[2 * n + c];
                        h3[0] -= v[0] * mx + v[3] * my + v[4] * mz;
                        h3[1] -= v[3] * mx + v[1] * my + v[5] * mz;
                        h3[2] -= v[4] * mx + v[5] * my + v[2] * mz;
                    }
        }
        H[3 * s] = h3[0];
        H[3 * s + 1] = h3[1];
        H[3 * s + 2] = h3[2];
    }
}
