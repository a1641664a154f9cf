// FP64 precompute of the demagnetising-tensor spectrum (Table 1, "N computed
// using formulas in Ref. [50]": Newell, Williams and Dunlop).
//
// 1. newell_octant_kernel: the cell-averaged tensor for every displacement
//    (i dx, j dy, k dz), 0 <= i < nx etc. (summed over the periodic images of
//    a periodic mesh).  Within rs * max(dx,dy,dz) the exact
//    closed form: N_xx = (1/(4 pi V)) sum over the 27 shifts of prod_axis w(e)
//    f(...), w(0) = 2, w(+-1) = -1, with Newell's f (xx, yy, zz by permuting
//    the arguments) and g (xy, xz, yz).  Beyond it the box-averaged dipole
//    expansion N_ij = -(V/4 pi)[D_ij + (1/12) sum_k h_k^2 d_k^2 D_ij],
//    D_ij = d_i d_j (1/r), which is the Taylor expansion of the point-dipole
//    kernel averaged over the source and target boxes (the FP64 closed form
//    loses ~(r/h)^6 eps to cancellation far from the cell).
// 2. Three axis passes: each extends the octant line to the padded length
//    with the component's parity (xx, yy, zz even in every axis; xy odd in x
//    and y; xz odd in x and z; yz odd in y and z), transforms it with the
//    shared-memory FFT in FP64, and keeps the first P/2 + 1 bins.
// 3. finalize: the spectrum is real (even or odd-odd symmetric sequences);
//    store -Re / (px py pz) as rows [kx][ky] of kz * 6 + component (row
//    length padded to a multiple of 4 with zeros) in FP32 or FP64.
#include "boris_internal.cuh"
#include "newell_fg.cuh"

namespace boris {

// Exact tensor: all six components from one sweep over the 27 shifts.
__device__ void newell_exact_dev(double X, double Y, double Z, double dx, double dy, double dz, double out[6])
{
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int a = -1; a <= 1; a++) {
        const double wa = a == 0 ? 2.0 : -1.0;
        const double x = X + a * dx;
        for (int b = -1; b <= 1; b++) {
            const double wb = b == 0 ? 2.0 : -1.0;
            const double y = Y + b * dy;
            for (int c = -1; c <= 1; c++) {
                const double w = wa * wb * (c == 0 ? 2.0 : -1.0);
                const double z = Z + c * dz;
                s[0] += w * newell_f_dev(x, y, z);
                s[1] += w * newell_f_dev(y, x, z);
                s[2] += w * newell_f_dev(z, y, x);
                s[3] += w * newell_g_dev(x, y, z);
                s[4] += w * newell_g_dev(x, z, y);
                s[5] += w * newell_g_dev(y, z, x);
            }
        }
    }
    const double inv = 1.0 / (4.0 * 3.14159265358979323846 * dx * dy * dz);
    for (int i = 0; i < 6; i++) out[i] = s[i] * inv;
}

// Box-averaged dipole expansion to second order in the cell size.  With
// S2 = sum_k h_k^2 x_k^2 and Hs = sum_k h_k^2,
//   sum_k h_k^2 d_k^2 D_ij = 105 x_i x_j S2 / r^9
//       - 15 [x_i x_j (Hs + 2 h_i^2 + 2 h_j^2) + delta_ij S2] / r^7
//       + 3 delta_ij (Hs + 2 h_i^2) / r^5.
__device__ void newell_far_dev(double X, double Y, double Z, double dx, double dy, double dz, double out[6])
{
    const double x[3] = {X, Y, Z};
    const double h2[3] = {dx * dx, dy * dy, dz * dz};
    const double r2 = X * X + Y * Y + Z * Z;
    const double r = sqrt(r2);
    const double ir2 = 1.0 / r2;
    const double ir5 = ir2 * ir2 / r;
    const double ir7 = ir5 * ir2, ir9 = ir7 * ir2;
    const double S2 = h2[0] * X * X + h2[1] * Y * Y + h2[2] * Z * Z;
    const double Hs = h2[0] + h2[1] + h2[2];
    const double pre = -(dx * dy * dz) / (4.0 * 3.14159265358979323846);
    const int I[6] = {0, 1, 2, 0, 0, 1}, J[6] = {0, 1, 2, 1, 2, 2};
    for (int c = 0; c < 6; c++) {
        const int i = I[c], j = J[c];
        const double xij = x[i] * x[j];
        const double d = (i == j) ? 1.0 : 0.0;
        const double D = (3.0 * xij - d * r2) * ir5;
        const double corr = 105.0 * xij * S2 * ir9 -
                            15.0 * (xij * (Hs + 2.0 * h2[i] + 2.0 * h2[j]) + d * S2) * ir7 +
                            3.0 * d * (Hs + 2.0 * h2[i]) * ir5;
        out[c] = pre * (D + corr / 12.0);
    }
}

// Cell-averaged tensor at displacement (i dx, j dy, k dz), summed over the
// periodic images (i dx + a nx dx, j dy + b ny dy, k dz + c nz dz) with
// |a| <= kx, |b| <= ky, |c| <= kz (multiple-images method, Section 4; no
// images: kx = ky = kz = 0).  The image set is symmetric, so the sum keeps
// the parities of the octant form.
__global__ void newell_octant_kernel(int nx, int ny, int nz, double dx, double dy, double dz, double rs, int kx,
                                     int ky, int kz, double* __restrict__ T)
{
    const size_t n = (size_t)nx * ny * nz;
    const double hmax = fmax(dx, fmax(dy, dz));
    const double Lx = nx * dx, Ly = ny * dy, Lz = nz * dz;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % nx);
        const int j = (int)((idx / nx) % ny);
        const int k = (int)(idx / ((size_t)nx * ny));
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (int c = -kz; c <= kz; c++)
            for (int b = -ky; b <= ky; b++)
                for (int a = -kx; a <= kx; a++) {
                    const double X = i * dx + a * Lx, Y = j * dy + b * Ly, Z = k * dz + c * Lz;
                    double v[6];
                    if (sqrt(X * X + Y * Y + Z * Z) <= rs * hmax) newell_exact_dev(X, Y, Z, dx, dy, dz, v);
                    else newell_far_dev(X, Y, Z, dx, dy, dz, v);
                    for (int q = 0; q < 6; q++) acc[q] += v[q];
                }
        for (int q = 0; q < 6; q++) T[q * n + idx] = acc[q];
    }
}

// Parity of component c along axis a: -1 for the odd (off-diagonal) axes.
__device__ __forceinline__ double comp_parity(int c, int a)
{
    // c: 0 xx, 1 yy, 2 zz, 3 xy, 4 xz, 5 yz
    if (c == 3) return (a == 0 || a == 1) ? -1.0 : 1.0;
    if (c == 4) return (a == 0 || a == 2) ? -1.0 : 1.0;
    if (c == 5) return (a == 1 || a == 2) ? -1.0 : 1.0;
    return 1.0;
}

// One axis pass.  Input: [6][d2][d1][d0] (real if in_real, else complex) with
// the transformed axis of length n (octant); output: same with that axis of
// length P/2 + 1.  NL lines per CTA, each extended to length P in shared
// memory with the component's parity.
// pmode 0: the six demagnetising-tensor components (comp_parity); pmode 1:
// the three Oersted components, component c odd along axis c only.
__global__ void __launch_bounds__(256) axis_pass_kernel(const void* __restrict__ in, bool in_real,
                                                        double2* __restrict__ out, int axis, int d0, int d1,
                                                        int d2, int n, int P, int lgP, int NL,
                                                        const double2* __restrict__ tw, int lglmax, int ncomp,
                                                        int pmode)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);  // [NL][P]
    const int dims[3] = {d0, d1, d2};
    int od[3] = {d0, d1, d2};
    const int kh = P / 2 + 1;
    od[axis] = kh;
    // line = (c, the two other coordinates)
    const int oa = axis == 0 ? 1 : 0, ob = axis == 2 ? 1 : 2;
    const long nlines_total = (long)ncomp * dims[oa] * dims[ob];
    const long line0 = (long)blockIdx.x * NL;
    auto in_index = [&](int c, int u, int v, int e) -> size_t {
        int co[3];
        co[axis] = e;
        co[oa] = u;
        co[ob] = v;
        return (size_t)c * d0 * d1 * d2 + ((size_t)co[2] * d1 + co[1]) * d0 + co[0];
    };
    auto out_index = [&](int c, int u, int v, int e) -> size_t {
        int co[3];
        co[axis] = e;
        co[oa] = u;
        co[ob] = v;
        return (size_t)c * od[0] * od[1] * od[2] + ((size_t)co[2] * od[1] + co[1]) * od[0] + co[0];
    };
    auto decode = [&](long line, int& c, int& u, int& v) {
        u = (int)(line % dims[oa]);
        long rest = line / dims[oa];
        v = (int)(rest % dims[ob]);
        c = (int)(rest / dims[ob]);
    };
    for (int i = threadIdx.x; i < NL * P; i += blockDim.x) {
        const int l = i / P, e = i % P;
        const long line = line0 + l;
        double2 val = make_double2(0.0, 0.0);
        if (line < nlines_total) {
            int c, u, v;
            decode(line, c, u, v);
            int src = -1;
            double s = 1.0;
            if (e < n) src = e;
            else if (e > P - n) {
                src = P - e;
                s = pmode ? (c == axis ? -1.0 : 1.0) : comp_parity(c % 6, axis);
            }
            if (src >= 0) {
                const size_t ii = in_index(c, u, v, src);
                if (in_real) val = make_double2(s * reinterpret_cast<const double*>(in)[ii], 0.0);
                else {
                    const double2 t = reinterpret_cast<const double2*>(in)[ii];
                    val = make_double2(s * t.x, s * t.y);
                }
            }
        }
        buf[i] = val;
    }
    __syncthreads();
    if (lgP > 0) {
        Lines ln{NL, NL, P, 0, 1, false};
        fft_dif(buf, ln, lgP, 0, tw, lglmax - lgP);
    }
    for (int i = threadIdx.x; i < NL * kh; i += blockDim.x) {
        const int l = i / kh, k = i % kh;
        const long line = line0 + l;
        if (line >= nlines_total) continue;
        int c, u, v;
        decode(line, c, u, v);
        out[out_index(c, u, v, k)] = buf[l * P + bitrev(k, lgP)];
    }
}

template <typename T>
__global__ void finalize_kernel(const double2* __restrict__ S, T* __restrict__ K, int nkx, int kyh, int kzh, int krow,
                                double scale)
{
    const size_t n = (size_t)nkx * kyh * kzh;
    const size_t total = (size_t)nkx * kyh * krow;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const int o = (int)(idx % krow);
        const size_t row = idx / krow;  // = kx * kyh + ky
        const int ky = (int)(row % kyh);
        const int kx = (int)(row / kyh);
        T val = T(0);  // row padding
        if (o < kzh * 6) {
            const int kz = o / 6, c = o % 6;
            const double v = S[(size_t)c * n + ((size_t)kz * kyh + ky) * nkx + kx].x;
            val = (T)(-v * scale);
        }
        K[idx] = val;
    }
}

void host_twiddles(int n, double2* out)
{
    const double twopi = 6.283185307179586476925286766559;
    for (int e = 0; e < n; e++) {
        const double a = twopi * (double)e / (double)n;
        out[e] = make_double2(std::cos(a), -std::sin(a));
    }
}

cudaError_t newell_octant(int nx, int ny, int nz, double dx, double dy, double dz, double rs, double* T,
                          cudaStream_t st, const int* images)
{
    const size_t n = (size_t)nx * ny * nz;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 64) blocks = 152 * 64;
    const int kx = images ? images[0] : 0, ky = images ? images[1] : 0, kz = images ? images[2] : 0;
    newell_octant_kernel<<<blocks, 256, 0, st>>>(nx, ny, nz, dx, dy, dz, rs, kx, ky, kz, T);
    return cudaGetLastError();
}

cudaError_t run_axis_n(const void* in, bool in_real, double2* out, int axis, int d0, int d1, int d2, int n, int P,
                       int ncomp, const double2* tw, int lglmax, cudaStream_t st, int pmode)
{
    const int lgP = ilog2(P);
    int NL = 4096 / P;
    if (NL < 1) NL = 1;
    if (NL > 32) NL = 32;
    const size_t smem = (size_t)NL * P * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(axis_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int dims[3] = {d0, d1, d2};
    const int oa = axis == 0 ? 1 : 0, ob = axis == 2 ? 1 : 2;
    const long nlines = (long)ncomp * dims[oa] * dims[ob];
    const long blocks = (nlines + NL - 1) / NL;
    axis_pass_kernel<<<(unsigned)blocks, 256, smem, st>>>(in, in_real, out, axis, d0, d1, d2, n, P, lgP, NL, tw,
                                                           lglmax, ncomp, pmode);
    return cudaGetLastError();
}

static cudaError_t run_axis(const void* in, bool in_real, double2* out, int axis, int d0, int d1, int d2, int n,
                            int P, const double2* tw, int lglmax, cudaStream_t st)
{
    return run_axis_n(in, in_real, out, axis, d0, d1, d2, n, P, 6, tw, lglmax, st, 0);
}

cudaError_t build_kernel_spectrum(const Geometry& g, double dx, double dy, double dz, double rs, void* K_out,
                                  bool k_is_f64, const double2* tw64, cudaStream_t st, const int* images)
{
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    double* T = nullptr;
    double2 *A = nullptr, *B = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&T, 6 * n * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const size_t a_elems = 6 * (size_t)g.nkx * g.ny * g.nz;
    const size_t b_elems = 6 * (size_t)g.nkx * g.kyh * g.nz;
    const size_t c_elems = 6 * (size_t)g.nkx * g.kyh * g.kzh;
    do {
        if ((e = newell_octant(g.nx, g.ny, g.nz, dx, dy, dz, rs, T, st, images)) != cudaSuccess) break;
        if ((e = cudaMallocAsync((void**)&A, a_elems * sizeof(double2), st)) != cudaSuccess) break;
        if ((e = run_axis(T, true, A, 0, g.nx, g.ny, g.nz, g.nx, g.px, tw64, g.lglmax, st)) != cudaSuccess) break;
        cudaFreeAsync(T, st);
        T = nullptr;
        if ((e = cudaMallocAsync((void**)&B, b_elems * sizeof(double2), st)) != cudaSuccess) break;
        if ((e = run_axis(A, false, B, 1, g.nkx, g.ny, g.nz, g.ny, g.py, tw64, g.lglmax, st)) != cudaSuccess) break;
        cudaFreeAsync(A, st);
        A = nullptr;
        if ((e = cudaMallocAsync((void**)&A, c_elems * sizeof(double2), st)) != cudaSuccess) break;
        if ((e = run_axis(B, false, A, 2, g.nkx, g.kyh, g.nz, g.nz, g.pz, tw64, g.lglmax, st)) != cudaSuccess) break;
        const double scale = 1.0 / ((double)g.px * g.py * g.pz);
        const size_t tot = (size_t)g.nkx * g.kyh * g.krow;
        int blocks = (int)((tot + 255) / 256);
        if (blocks > 152 * 64) blocks = 152 * 64;
        if (k_is_f64) finalize_kernel<double><<<blocks, 256, 0, st>>>(A, (double*)K_out, g.nkx, g.kyh, g.kzh, g.krow, scale);
        else finalize_kernel<float><<<blocks, 256, 0, st>>>(A, (float*)K_out, g.nkx, g.kyh, g.kzh, g.krow, scale);
        e = cudaGetLastError();
    } while (0);
    if (T) cudaFreeAsync(T, st);
    if (A) cudaFreeAsync(A, st);
    if (B) cudaFreeAsync(B, st);
    return e;
}

// ---------------------------------------------------------------------------
// Oersted kernel (Table 1, "K computed using formulas in Ref. [63]", which
// the paper does not reproduce).  For a uniform current density J in a source
// cell, the Biot-Savart field averaged over a target cell at centre
// displacement D is H = J x g(D), g = -(1/(4 pi V)) grad_D P(D), P the
// two-cell Coulomb integral of 1/|r - r'|.  The demagnetising tensor of the
// same pair is N_ij = d_i g_j, so g_k is the antiderivative of N_kk along axis
// k that vanishes far away:
//   g_k(D) = gfar_k(D_e) - int_{D_k}^{t_e} N_kk dt,
// integrated with 16-point Gauss-Legendre rules on whole cells (the kinks of
// N lie on multiples of h_k) up to the first end point t_e beyond
// rs max(h), where the far form (the gradient of the box-averaged potential
// 1/r + sum_m h_m^2/12 d_m^2 (1/r)) takes over.  FP64.
// ---------------------------------------------------------------------------
struct GL16 {
    double x[16], w[16];
};

// N_kk by Newell's 27-point stencil of f with k's argument first
__device__ double newell_kk_dev(int k, double X, double Y, double Z, double dx, double dy, double dz)
{
    double s = 0.0;
    for (int a = -1; a <= 1; a++) {
        const double wa = a == 0 ? 2.0 : -1.0;
        const double x = X + a * dx;
        for (int b = -1; b <= 1; b++) {
            const double wb = b == 0 ? 2.0 : -1.0;
            const double y = Y + b * dy;
            for (int c = -1; c <= 1; c++) {
                const double w = wa * wb * (c == 0 ? 2.0 : -1.0);
                const double z = Z + c * dz;
                s += w * (k == 0 ? newell_f_dev(x, y, z) : k == 1 ? newell_f_dev(y, x, z) : newell_f_dev(z, y, x));
            }
        }
    }
    return s / (4.0 * 3.14159265358979323846 * dx * dy * dz);
}

__device__ double oersted_far_dev(int k, const double x[3], const double h[3], double V)
{
    const double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    const double r = sqrt(r2);
    const double ir3 = 1.0 / (r2 * r), ir5 = ir3 / r2, ir7 = ir5 / r2;
    double s = -x[k] * ir3;  // d_k (1/r)
    for (int m = 0; m < 3; m++) {
        // d_k d_m^2 (1/r) = (6 x_m delta_km - 2 x_k)/r^5 - 5 x_k (3 x_m^2 - r^2)/r^7
        const double d3 = (6.0 * x[m] * (m == k ? 1.0 : 0.0) - 2.0 * x[k]) * ir5 - 5.0 * x[k] * (3.0 * x[m] * x[m] - r2) * ir7;
        s += h[m] * h[m] * (1.0 / 12.0) * d3;
    }
    return -V / (4.0 * 3.14159265358979323846) * s;
}

// thread per (component, octant displacement): G[c][k][j][i] = g_c(i dx, j dy, k dz)
__global__ void oersted_octant_kernel(int nx, int ny, int nz, double dx, double dy, double dz, double rs, GL16 gl,
                                      double* __restrict__ G)
{
    const size_t n = (size_t)nx * ny * nz;
    const double h[3] = {dx, dy, dz};
    const double hmax = fmax(dx, fmax(dy, dz)), V = dx * dy * dz, rlim = rs * hmax;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < 3 * n; t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        const size_t idx = t - (size_t)c * n;
        const int i = (int)(idx % nx), j = (int)((idx / nx) % ny), k = (int)(idx / ((size_t)nx * ny));
        double p[3] = {i * dx, j * dy, k * dz};
        double val;
        if (sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) > rlim) {
            val = oersted_far_dev(c, p, h, V);
        } else {
            double acc = 0.0;
            double tpos = p[c];
            for (;;) {
                double q[3] = {p[0], p[1], p[2]};
                q[c] = tpos;
                if (sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]) > rlim) break;
                const double half = 0.5 * h[c], mid = tpos + half;
                for (int g = 0; g < 16; g++) {
                    q[c] = mid + half * gl.x[g];
                    acc += gl.w[g] * half * newell_kk_dev(c, q[0], q[1], q[2], dx, dy, dz);
                }
                tpos += h[c];
            }
            double e[3] = {p[0], p[1], p[2]};
            e[c] = tpos;
            val = oersted_far_dev(c, e, h, V) - acc;
        }
        G[t] = val;
    }
}

// KO[kx][ky'][kz'][4] = (Im gx, Im gy, Im gz, 0) / (px py pz): each spectrum is
// imaginary (one odd axis), so the convolution is H^ = i (J^ x KO).
__global__ void oersted_finalize_kernel(const double2* __restrict__ S, float* __restrict__ KO, int nkx, int kyh, int kzh,
                                        double scale)
{
    const size_t n = (size_t)nkx * kyh * kzh;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < 4 * n; idx += (size_t)gridDim.x * blockDim.x) {
        const int o = (int)(idx % 4);
        const size_t cell = idx / 4;  // (kx * kyh + ky) * kzh + kz
        const int kz = (int)(cell % kzh);
        const size_t row = cell / kzh;
        const int ky = (int)(row % kyh), kx = (int)(row / kyh);
        float v = 0.f;
        if (o < 3) v = (float)(S[(size_t)o * n + ((size_t)kz * kyh + ky) * nkx + kx].y * scale);
        KO[idx] = v;
    }
}

cudaError_t build_oersted_spectrum(const Geometry& g, double dx, double dy, double dz, double rs, float* KO,
                                   const double2* tw64, cudaStream_t st)
{
    GL16 gl;
    const int nn = 16;
    for (int i = 0; i < nn; i++) {  // Legendre nodes by Newton iteration, FP64
        double x = std::cos(3.14159265358979323846 * (i + 0.75) / (nn + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= nn; k++) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = nn * (x * p1 - p0) / (x * x - 1.0);
            const double step = p1 / dp;
            x -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= nn; k++) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = nn * (x * p1 - p0) / (x * x - 1.0);
        gl.x[i] = x;
        gl.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    double* T = nullptr;
    double2 *A = nullptr, *B = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&T, 3 * n * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const size_t a_elems = 3 * (size_t)g.nkx * g.ny * g.nz;
    const size_t b_elems = 3 * (size_t)g.nkx * g.kyh * g.nz;
    const size_t c_elems = 3 * (size_t)g.nkx * g.kyh * g.kzh;
    do {
        int blocks = (int)((3 * n + 127) / 128);
        if (blocks > 152 * 64) blocks = 152 * 64;
        oersted_octant_kernel<<<blocks, 128, 0, st>>>(g.nx, g.ny, g.nz, dx, dy, dz, rs, gl, T);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaMallocAsync((void**)&A, a_elems * sizeof(double2), st)) != cudaSuccess) break;
        if ((e = run_axis_n(T, true, A, 0, g.nx, g.ny, g.nz, g.nx, g.px, 3, tw64, g.lglmax, st, 1)) != cudaSuccess) break;
        cudaFreeAsync(T, st);
        T = nullptr;
        if ((e = cudaMallocAsync((void**)&B, b_elems * sizeof(double2), st)) != cudaSuccess) break;
        if ((e = run_axis_n(A, false, B, 1, g.nkx, g.ny, g.nz, g.ny, g.py, 3, tw64, g.lglmax, st, 1)) != cudaSuccess) break;
        cudaFreeAsync(A, st);
        A = nullptr;
        if ((e = cudaMallocAsync((void**)&A, c_elems * sizeof(double2), st)) != cudaSuccess) break;
        if ((e = run_axis_n(B, false, A, 2, g.nkx, g.kyh, g.nz, g.nz, g.pz, 3, tw64, g.lglmax, st, 1)) != cudaSuccess) break;
        const double scale = 1.0 / ((double)g.px * g.py * g.pz);
        const size_t tot = 4 * (size_t)g.nkx * g.kyh * g.kzh;
        int fb = (int)((tot + 255) / 256);
        if (fb > 152 * 64) fb = 152 * 64;
        oersted_finalize_kernel<<<fb, 256, 0, st>>>(A, KO, g.nkx, g.kyh, g.kzh, scale);
        e = cudaGetLastError();
    } while (0);
    if (T) cudaFreeAsync(T, st);
    if (A) cudaFreeAsync(A, st);
    if (B) cudaFreeAsync(B, st);
    return e;
}

}  // namespace boris
