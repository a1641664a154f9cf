// Multi-mesh demagnetising field (Eq. 4) for a stack of layers that share the
// in-plane cell (hx, hy): each layer has its own z cell size, in-plane offset
// and z position.
//
// All layers are embedded in one common in-plane frame (NX x NY cells), so
// every z plane of every layer is a plane of one batched transform: the x and
// y transforms of the single-mesh path run once over all Z = sum nz planes.
// In transform space the inter-mesh sum of Eq. 4 becomes, per (kx, ky),
//   Hh(p) = sum_q N^(kx, ky; p, q) Mh(q)
// with N^ the 2D spectrum of the inter-mesh tensor between the cells of plane
// p (z size a) and plane q (z size b) at z offset dz = z_p - z_q.  The two-box
// stencil below is the same for (a, b) and (b, a), and only the volume of the
// target box normalises it, so a N_ab = b N_ba at every displacement (the
// reciprocity of Eq. 4's tensor): the plan stores Nt = a N_ab once per
// (min(a, b), max(a, b), |dz|) and the sum divides by the target's a.  dz < 0
// flips the xz and yz components (odd in z).  The tensor itself is Newell's construction with the z stencil of two
// boxes of unequal height, F(z + s) - F(z + d) - F(z - d) + F(z - s),
// s = (a + b)/2, d = (a - b)/2, normalised by the target volume; beyond 40
// cell sizes the box-averaged dipole expansion with per-axis variances
// hx^2/6, hy^2/6, (a^2 + b^2)/12 and the source volume.
#include <algorithm>

#include "boris_internal.cuh"
#include "bulk_async.cuh"
#include "multilayer.cuh"
#include "newell_fg.cuh"

namespace boris {

// Stencil of one axis: n taps at offsets off with weights w.
struct Taps {
    int n;
    double off[4], w[4];
};
__device__ __forceinline__ Taps taps_equal(double h) { return Taps{3, {-h, 0.0, h, 0.0}, {-1.0, 2.0, -1.0, 0.0}}; }
__device__ __forceinline__ Taps taps_pair(double a, double b)
{
    const double s = 0.5 * (a + b), d = 0.5 * (a - b);
    return Taps{4, {-s, -d, d, s}, {-1.0, 1.0, 1.0, -1.0}};
}

template <bool G>
__device__ double pair_sum(double X, double Y, double Z, const Taps& t1, const Taps& t2, const Taps& t3)
{
    double acc = 0.0;
    for (int i = 0; i < t1.n; i++)
        for (int j = 0; j < t2.n; j++)
            for (int k = 0; k < t3.n; k++) {
                const double w = t1.w[i] * t2.w[j] * t3.w[k];
                const double x = X + t1.off[i], y = Y + t2.off[j], z = Z + t3.off[k];
                acc += w * (G ? newell_g_dev(x, y, z) : newell_f_dev(x, y, z));
            }
    return acc;
}

__device__ void pair_tensor(double X, double Y, double Z, double hx, double hy, double a, double b, double rs,
                            double out[6])
{
    const double hmax = fmax(fmax(hx, hy), fmax(a, b));
    const double r2 = X * X + Y * Y + Z * Z;
    if (sqrt(r2) <= rs * hmax) {
        const Taps tx = taps_equal(hx), ty = taps_equal(hy), tz = taps_pair(a, b);
        const double norm = 1.0 / (4.0 * 3.14159265358979323846 * hx * hy * a);
        out[0] = norm * pair_sum<false>(X, Y, Z, tx, ty, tz);
        out[1] = norm * pair_sum<false>(Y, X, Z, ty, tx, tz);
        out[2] = norm * pair_sum<false>(Z, Y, X, tz, ty, tx);
        out[3] = norm * pair_sum<true>(X, Y, Z, tx, ty, tz);
        out[4] = norm * pair_sum<true>(X, Z, Y, tx, tz, ty);
        out[5] = norm * pair_sum<true>(Y, Z, X, ty, tz, tx);
        return;
    }
    // sum_k var_k/2 d_k^2 D_ij with var = (hx^2/6, hy^2/6, (a^2+b^2)/12):
    // with S2 = sum_k c_k x_k^2, Cs = sum_k c_k (c_k = var_k/2):
    //   105 x_i x_j S2/r^9 - 15 [x_i x_j (Cs + 2 c_i + 2 c_j) + delta_ij S2]/r^7 + 3 delta_ij (Cs + 2 c_i)/r^5
    const double x[3] = {X, Y, Z};
    const double c[3] = {hx * hx / 12.0, hy * hy / 12.0, (a * a + b * b) / 24.0};
    const double r = sqrt(r2), ir2 = 1.0 / r2, ir5 = ir2 * ir2 / r, ir7 = ir5 * ir2, ir9 = ir7 * ir2;
    const double S2 = c[0] * X * X + c[1] * Y * Y + c[2] * Z * Z, Cs = c[0] + c[1] + c[2];
    const double pre = -(hx * hy * b) / (4.0 * 3.14159265358979323846);
    const int I[6] = {0, 1, 2, 0, 0, 1}, J[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; k++) {
        const int i = I[k], j = J[k];
        const double xij = x[i] * x[j], d = i == j ? 1.0 : 0.0;
        const double D = (3.0 * xij - d * r2) * ir5;
        const double corr = 105.0 * xij * S2 * ir9 - 15.0 * (xij * (Cs + 2.0 * c[i] + 2.0 * c[j]) + d * S2) * ir7 +
                            3.0 * d * (Cs + 2.0 * c[i]) * ir5;
        out[k] = pre * (D + corr);
    }
}

// In-plane tables of nu unique (a, b, |dz|) entries, a N_ab (the reciprocal
// form, symmetric in a and b): T[u][6][NY][NX].
__global__ void ml_tensor_kernel(int nu, const double* __restrict__ ua, const double* __restrict__ ub,
                                 const double* __restrict__ udz, int NX, int NY, double hx, double hy, double rs,
                                 double* __restrict__ T)
{
    const size_t plane = (size_t)NX * NY;
    const size_t n = (size_t)nu * plane;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int u = (int)(idx / plane);
        const size_t cell = idx % plane;
        const int i = (int)(cell % NX), j = (int)(cell / NX);
        double v[6];
        pair_tensor(i * hx, j * hy, udz[u], hx, hy, ua[u], ub[u], rs, v);
        for (int c = 0; c < 6; c++) T[((size_t)u * 6 + c) * plane + cell] = ua[u] * v[c];
    }
}

// 2D spectra [6 nu][kyh][nkx] (complex) -> K[u][kx][c][kyp] (component-major,
// ky' fastest, rows padded to kyp = kyh rounded up to 32 with zeros) with the
// real part of xx, yy, zz, xy and the imaginary part of xz, yz (odd in exactly
// one in-plane axis), scaled by -1/(px py).
__global__ void ml_finalize_kernel(const double2* __restrict__ S, float* __restrict__ K, int nu, int nkx, int kyh,
                                   int kyp, double scale)
{
    const size_t per = (size_t)nkx * kyh;
    const size_t total = (size_t)nu * nkx * 6 * kyp;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const int ky = (int)(idx % kyp);
        size_t rest = idx / kyp;
        const int c = (int)(rest % 6);
        rest /= 6;
        const int kx = (int)(rest % nkx);
        const int u = (int)(rest / nkx);
        float v = 0.f;
        if (ky < kyh) {
            const double2 s = S[((size_t)u * 6 + c) * per + (size_t)ky * nkx + kx];
            v = (float)(-(c < 4 ? s.x : s.y) * scale);
        }
        K[idx] = v;
    }
}

// Embed the concatenated layer fields (scaled by Ms) into the frame [3][Z][NY][NX].
__global__ void ml_embed_kernel(MLTable t, const float* __restrict__ M, const float* __restrict__ ms_map, float ms,
                                float* __restrict__ F)
{
    const size_t fplane = (size_t)t.NX * t.NY;
    const size_t total = 3 * (size_t)t.Z * fplane;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(idx % t.NX);
        const int y = (int)((idx / t.NX) % t.NY);
        const int p = (int)((idx / fplane) % t.Z);
        const int c = (int)(idx / (fplane * t.Z));
        const int l = t.plane_layer[p], q = p - t.plane0[l];
        const int lx = x - t.ox[l], ly = y - t.oy[l];
        float v = 0.f;
        if (lx >= 0 && lx < t.nx[l] && ly >= 0 && ly < t.ny[l]) {
            const size_t n = (size_t)t.nx[l] * t.ny[l] * t.nz[l];
            const size_t cell = ((size_t)q * t.ny[l] + ly) * t.nx[l] + lx;
            v = M[t.off[l] + c * n + cell] * (ms_map ? ms_map[t.off[l] / 3 + cell] : ms);
        }
        F[idx] = v;
    }
}

// Extract the layers' cells of the frame field into the concatenated layout.
__global__ void ml_extract_kernel(MLTable t, const float* __restrict__ F, float* __restrict__ H)
{
    const size_t total = t.total3;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < t.nl && idx >= t.off[l + 1]) l++;
        const size_t local = idx - t.off[l];
        const size_t n = (size_t)t.nx[l] * t.ny[l] * t.nz[l];
        const int c = (int)(local / n);
        const size_t cell = local % n;
        const int lx = (int)(cell % t.nx[l]), ly = (int)((cell / t.nx[l]) % t.ny[l]), q = (int)(cell / ((size_t)t.nx[l] * t.ny[l]));
        const int p = t.plane0[l] + q;
        H[idx] = F[(((size_t)c * t.Z + p) * t.NY + ly + t.oy[l]) * t.NX + lx + t.ox[l]];
    }
}

// Inter-plane sum in transform space (Eq. 4 moved to transform space).  CTA:
// 32 consecutive folded rows ky' = 32 t + lane of one kx; each thread serves
// column ky = ky' and its mirror py - ky' (which read the same spectrum row,
// with xy and yz negated), so every spectrum entry is loaded once per kx.
// Warp w accumulates the target planes p = w, w + 8, ...  Y layout
// [kx][c][p][ky]; K[u][kx][c][kyp] (one coalesced 128-byte load per component);
// pairs[p * Z + q] = u (>= 0) with bit 30 set when z_p < z_q (xz and yz change
// sign).
template <int PMAX>
__global__ void __launch_bounds__(256) ml_mix_kernel(Geometry g, int Z, float2* __restrict__ Y,
                                                     const float* __restrict__ K, int kyp, const int* __restrict__ pairs,
                                                     const float* __restrict__ inv_hz)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* Ms = reinterpret_cast<float2*>(smem_raw);  // [Z][3][2][32]: column ky', mirror
    int* pr = reinterpret_cast<int*>(Ms + (size_t)Z * 3 * 64);
    const int kx = blockIdx.y, kf0 = blockIdx.x * 32, py = g.py;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int kf = kf0 + lane;
    const bool onA = kf <= py / 2;                 // column ky = kf
    const bool onB = kf > 0 && kf < py / 2;        // mirror column py - kf
    float2* base = Y + (size_t)kx * 3 * Z * py;
    for (int i = threadIdx.x; i < Z * Z; i += 256) pr[i] = pairs[i];
    for (int i = threadIdx.x; i < 3 * Z * 64; i += 256) {
        const int col = i & 31, half = (i >> 5) & 1, line = i >> 6;  // line = c * Z + p
        const int c = line / Z, p = line % Z;
        const int f = kf0 + col;
        const bool ok = half ? (f > 0 && f < py / 2) : (f <= py / 2);
        const int ky = half ? py - f : f;
        Ms[((p * 3 + c) * 2 + half) * 32 + col] = ok ? base[(size_t)line * py + ky] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const size_t ustride = (size_t)g.nkx * 6 * kyp;
    const float* Kc = K + (size_t)kx * 6 * kyp + (onA ? kf : 0);
    float2 acc[PMAX][2][3];
#pragma unroll
    for (int j = 0; j < PMAX; j++)
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc[j][h][c] = make_float2(0.f, 0.f);
    for (int q = 0; q < Z; q++) {
        float2 mv[2][3];
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int c = 0; c < 3; c++) mv[h][c] = Ms[((q * 3 + c) * 2 + h) * 32 + lane];
#pragma unroll
        for (int j = 0; j < PMAX; j++) {
            const int p = warp + 8 * j;
            if (p < Z) {
                const int code = pr[p * Z + q];
                const int u = code & 0x3fffffff;
                const float sz = (code >> 30) & 1 ? -1.f : 1.f;
                const float* k = Kc + (size_t)u * ustride;
                const float kxx = k[0], kyy = k[kyp], kzz = k[2 * kyp], kxy0 = k[3 * kyp];
                const float kxz = sz * k[4 * kyp], kyz0 = sz * k[5 * kyp];  // imaginary parts: i kxz, i kyz
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const float kxy = h ? -kxy0 : kxy0, kyz = h ? -kyz0 : kyz0;  // mirror: ky odd entries flip
                    const float2 mx = mv[h][0], my = mv[h][1], mz = mv[h][2];
                    acc[j][h][0].x += kxx * mx.x + kxy * my.x - kxz * mz.y;
                    acc[j][h][0].y += kxx * mx.y + kxy * my.y + kxz * mz.x;
                    acc[j][h][1].x += kxy * mx.x + kyy * my.x - kyz * mz.y;
                    acc[j][h][1].y += kxy * mx.y + kyy * my.y + kyz * mz.x;
                    acc[j][h][2].x += -kxz * mx.y - kyz * my.y + kzz * mz.x;
                    acc[j][h][2].y += kxz * mx.x + kyz * my.x + kzz * mz.y;
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < PMAX; j++) {
        const int p = warp + 8 * j;
        if (p < Z) {
            const float ia = inv_hz[p];  // the spectra hold a N: divide by the target's a
#pragma unroll
            for (int c = 0; c < 3; c++) {
                if (onA) base[(size_t)(c * Z + p) * py + kf] = make_float2(acc[j][0][c].x * ia, acc[j][0][c].y * ia);
                if (onB)
                    base[(size_t)(c * Z + p) * py + (py - kf)] = make_float2(acc[j][1][c].x * ia, acc[j][1][c].y * ia);
            }
        }
    }
}

// The same sum with the spectrum rows staged asynchronously: for each source
// plane q every warp copies the 6 x 128-byte rows of its own targets'
// spectra (the CTA's 32 columns) into its shared-memory buffer by cp.async
// one source ahead (two buffers), so the loads overlap the previous source's
// arithmetic and only warp-level synchronisation is needed (Z <= 64).

template <int PMAX>
__global__ void __launch_bounds__(256, 2) ml_mix_staged_kernel(Geometry g, int Z, float2* __restrict__ Y,
                                                               const float* __restrict__ K, int kyp,
                                                               const int* __restrict__ pairs,
                                                               const float* __restrict__ inv_hz)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // per warp: [2][nt][6][32] rows of its own nt targets p = warp + 8 j (Z
    // targets over the eight warps: Z x 2 x 6 x 32 floats in all)
    const int nt = (Z - warp + 7) / 8;
    int before = 0;
    for (int v = 0; v < warp; v++) before += (Z - v + 7) / 8;
    float* Kw = reinterpret_cast<float*>(smem_raw) + (size_t)before * 2 * 6 * 32;
    float2* Ms = reinterpret_cast<float2*>(reinterpret_cast<float*>(smem_raw) + (size_t)Z * 2 * 6 * 32);
    int* pr = reinterpret_cast<int*>(Ms + (size_t)Z * 3 * 64);
    const int kx = blockIdx.y, kf0 = blockIdx.x * 32, py = g.py;
    const int kf = kf0 + lane;
    const bool onA = kf <= py / 2;
    const bool onB = kf > 0 && kf < py / 2;
    float2* base = Y + (size_t)kx * 3 * Z * py;
    const size_t ustride = (size_t)g.nkx * 6 * kyp;
    // lane's share of a target's six 128-byte rows: 16-byte part lane & 7 of
    // components lane >> 3 and (lane >> 3) + 4 (the latter for lanes 0..15)
    const int part = lane & 7, c0 = lane >> 3;
    const float* Kx = K + (size_t)kx * 6 * kyp + kf0 + part * 4;
    for (int i = threadIdx.x; i < Z * Z; i += 256) pr[i] = pairs[i];
    __syncthreads();
    auto stage = [&](int q, int b) {
#pragma unroll
        for (int j = 0; j < PMAX; j++) {
            const int p = warp + 8 * j;
            if (p < Z) {
                const float* src = Kx + (size_t)(pr[p * Z + q] & 0x3fffffff) * ustride;
                float* dst = Kw + ((size_t)(b * nt + j) * 6) * 32 + part * 4;
                cp_async16(dst + c0 * 32, src + (size_t)c0 * kyp);
                if (c0 < 2) cp_async16(dst + (c0 + 4) * 32, src + (size_t)(c0 + 4) * kyp);
            }
        }
        cp_async_commit();
    };
    stage(0, 0);
    for (int i = threadIdx.x; i < 3 * Z * 64; i += 256) {
        const int col = i & 31, half = (i >> 5) & 1, line = i >> 6;  // line = c * Z + p
        const int c = line / Z, p = line % Z;
        const int f = kf0 + col;
        const bool ok = half ? (f > 0 && f < py / 2) : (f <= py / 2);
        const int ky = half ? py - f : f;
        Ms[((p * 3 + c) * 2 + half) * 32 + col] = ok ? base[(size_t)line * py + ky] : make_float2(0.f, 0.f);
    }
    __syncthreads();  // the columns are in shared memory
    float2 acc[PMAX][2][3];
#pragma unroll
    for (int j = 0; j < PMAX; j++)
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc[j][h][c] = make_float2(0.f, 0.f);
    for (int q = 0; q < Z; q++) {
        if (q + 1 < Z) {
            stage(q + 1, (q + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();  // every lane's copies of source q are visible to the warp
        const float* kb = Kw + (size_t)(q & 1) * nt * 6 * 32 + lane;
        float2 mv[2][3];
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int c = 0; c < 3; c++) mv[h][c] = Ms[((q * 3 + c) * 2 + h) * 32 + lane];
#pragma unroll
        for (int j = 0; j < PMAX; j++) {
            const int p = warp + 8 * j;
            if (p < Z) {
                const float sz = (pr[p * Z + q] >> 30) & 1 ? -1.f : 1.f;
                const float* k = kb + j * 6 * 32;
                const float kxx = k[0], kyy = k[32], kzz = k[64], kxy0 = k[96];
                const float kxz = sz * k[128], kyz0 = sz * k[160];  // imaginary parts: i kxz, i kyz
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const float kxy = h ? -kxy0 : kxy0, kyz = h ? -kyz0 : kyz0;  // mirror: ky odd entries flip
                    const float2 mx = mv[h][0], my = mv[h][1], mz = mv[h][2];
                    acc[j][h][0].x += kxx * mx.x + kxy * my.x - kxz * mz.y;
                    acc[j][h][0].y += kxx * mx.y + kxy * my.y + kxz * mz.x;
                    acc[j][h][1].x += kxy * mx.x + kyy * my.x - kyz * mz.y;
                    acc[j][h][1].y += kxy * mx.y + kyy * my.y + kyz * mz.x;
                    acc[j][h][2].x += -kxz * mx.y - kyz * my.y + kzz * mz.x;
                    acc[j][h][2].y += kxz * mx.x + kyz * my.x + kzz * mz.y;
                }
            }
        }
        __syncwarp();  // buffer q & 1 is free for source q + 2
    }
#pragma unroll
    for (int j = 0; j < PMAX; j++) {
        const int p = warp + 8 * j;
        if (p < Z) {
            const float ia = inv_hz[p];  // the spectra hold a N: divide by the target's a
#pragma unroll
            for (int c = 0; c < 3; c++) {
                if (onA) base[(size_t)(c * Z + p) * py + kf] = make_float2(acc[j][0][c].x * ia, acc[j][0][c].y * ia);
                if (onB)
                    base[(size_t)(c * Z + p) * py + (py - kf)] = make_float2(acc[j][1][c].x * ia, acc[j][1][c].y * ia);
            }
        }
    }
}

// The inter-plane sum as one persistent launch over all work items (kx,
// 32-column tile of folded ky'), tiles of one kx consecutive.  Per item: the
// Z planes' 32 columns and their mirrors go to shared memory (the mirror's
// M_y negated, see below); then for each source plane q every warp stages, by
// cp.async one source ahead, the 6 x 128-byte spectrum rows of its own
// targets p = warp + 8 j, whose offsets (in 128-byte units, the kz sign in
// bit 31) come precomputed in pcode; the 3 x 3 products run as packed FP32x2
// multiply-adds on (Re, Im) pairs.  The mirror column ky -> py - ky flips the
// ky-odd entries xy and yz; with M_y negated in the mirror the same entries
// give the mirror's H_x, H_z and -H_y, so both columns share one set of
// entry pairs.  The source loop is compiled for the warp's exact target count
// (the counts of the warps differ by at most one), so it has no per-target
// branches.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <int NT, int PM>
__device__ __forceinline__ void ml_v2_sum(int Z, int warp, int lane, const float* __restrict__ Kx, int kyp, float* Kw,
                                          const float2* Ms, const unsigned* pc, float2 (&acc)[PM][2][3])
{
    // the NT targets' 6 rows x 8 sixteen-byte pieces of source q into buffer b:
    // lane (c0 = lane / 8, part = lane mod 8) copies piece part of rows c0 and,
    // for c0 < 2, c0 + 4 of each target
    const int part = lane & 7, c0 = lane >> 3;
    const int so0 = c0 * kyp + part * 4, so1 = (c0 + 4) * kyp + part * 4;
    const int do0 = c0 * 32 + part * 4, do1 = (c0 + 4) * 32 + part * 4;
    // the kz signs of the staged source: bit j = bit 31 of target j's code
    unsigned sgm = 0, sgm_next = 0;
    auto stage = [&](int q, int b, unsigned& sgbits) {
        float* dstb = Kw + (size_t)b * NT * 6 * 32;
        sgbits = 0;
#pragma unroll
        for (int j = 0; j < NT; j++) {
            const unsigned code = pc[(warp + 8 * j) * Z + q];
            sgbits |= (code >> 31) << j;
            const float* src = Kx + (size_t)(code & 0x7fffffffu) * 32;
            cp_async16(dstb + j * 6 * 32 + do0, src + so0);
            if (c0 < 2) cp_async16(dstb + j * 6 * 32 + do1, src + so1);
        }
        cp_async_commit();
    };
    stage(0, 0, sgm);
    for (int q = 0; q < Z; q++) {
        if (q + 1 < Z) {
            stage(q + 1, (q + 1) & 1, sgm_next);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();  // every lane's copies of source q are visible to the warp
        const float* kb = Kw + (size_t)(q & 1) * NT * 6 * 32 + lane;
        // source columns m and i m (i times, for the imaginary xz and yz entries)
        float2 m[2][3], im[2][3];
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                m[h][c] = Ms[((q * 3 + c) * 2 + h) * 32 + lane];
                im[h][c] = make_float2(-m[h][c].y, m[h][c].x);
            }
#pragma unroll
        for (int j = 0; j < NT; j++) {
            const float* k = kb + j * 6 * 32;
            // the kz-odd entries change sign for a source above the target
            const unsigned sg = ((sgm >> j) & 1u) << 31;
            const float2 bxx = f2(k[0]), byy = f2(k[32]), bzz = f2(k[64]), bxy = f2(k[96]);
            const float2 bxz = f2(__uint_as_float(__float_as_uint(k[128]) ^ sg));
            const float2 byz = f2(__uint_as_float(__float_as_uint(k[160]) ^ sg));
#pragma unroll
            for (int h = 0; h < 2; h++) {
                acc[j][h][0] = ffma2(bxx, m[h][0], ffma2(bxy, m[h][1], ffma2(bxz, im[h][2], acc[j][h][0])));
                acc[j][h][1] = ffma2(bxy, m[h][0], ffma2(byy, m[h][1], ffma2(byz, im[h][2], acc[j][h][1])));
                acc[j][h][2] = ffma2(bxz, im[h][0], ffma2(byz, im[h][1], ffma2(bzz, m[h][2], acc[j][h][2])));
            }
        }
        __syncwarp();  // buffer q & 1 is free for source q + 2
        sgm = sgm_next;
    }
}

template <int PMAX>
__global__ void __launch_bounds__(256, 2) ml_mix_v2_kernel(Geometry g, int Z, float2* __restrict__ Y,
                                                           const float* __restrict__ K, int kyp,
                                                           const unsigned* __restrict__ pcode,
                                                           const float* __restrict__ inv_hz, int ntile, int nwork)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nt = (Z - warp + 7) / 8;
    int before = 0;
    for (int v = 0; v < warp; v++) before += (Z - v + 7) / 8;
    float* Kw = reinterpret_cast<float*>(smem_raw) + (size_t)before * 2 * 6 * 32;
    float2* Ms = reinterpret_cast<float2*>(reinterpret_cast<float*>(smem_raw) + (size_t)Z * 2 * 6 * 32);
    unsigned* pc = reinterpret_cast<unsigned*>(Ms + (size_t)Z * 3 * 64);
    float* ih = reinterpret_cast<float*>(pc + (size_t)Z * Z);
    const int py = g.py;
    for (int i = threadIdx.x; i < Z * Z; i += 256) pc[i] = pcode[i];
    for (int i = threadIdx.x; i < Z; i += 256) ih[i] = inv_hz[i];
    __syncthreads();
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int kx = w / ntile, kf0 = (w - kx * ntile) * 32;
        const int kf = kf0 + lane;
        const bool onA = kf <= py / 2;
        const bool onB = kf > 0 && kf < py / 2;
        float2* base = Y + (size_t)kx * 3 * Z * py;
        const float* Kx = K + (size_t)kx * 6 * kyp + kf0;
        for (int i = threadIdx.x; i < 3 * Z * 64; i += 256) {
            const int col = i & 31, half = (i >> 5) & 1, line = i >> 6;  // line = c * Z + p
            const int c = line / Z, p = line - c * Z;
            const int f = kf0 + col;
            const bool ok = half ? (f > 0 && f < py / 2) : (f <= py / 2);
            const int ky = half ? py - f : f;
            float2 v = ok ? base[(size_t)line * py + ky] : make_float2(0.f, 0.f);
            if (half && c == 1) v = make_float2(-v.x, -v.y);  // the mirror's M_y, negated
            Ms[((p * 3 + c) * 2 + half) * 32 + col] = v;
        }
        __syncthreads();  // the columns are in shared memory
        float2 acc[PMAX][2][3];
#pragma unroll
        for (int j = 0; j < PMAX; j++)
#pragma unroll
            for (int h = 0; h < 2; h++)
#pragma unroll
                for (int c = 0; c < 3; c++) acc[j][h][c] = make_float2(0.f, 0.f);
        if (nt == PMAX) ml_v2_sum<PMAX, PMAX>(Z, warp, lane, Kx, kyp, Kw, Ms, pc, acc);
        else if (nt == PMAX - 1) ml_v2_sum<(PMAX > 1 ? PMAX - 1 : 0), PMAX>(Z, warp, lane, Kx, kyp, Kw, Ms, pc, acc);
#pragma unroll
        for (int j = 0; j < PMAX; j++) {
            const int p = warp + 8 * j;
            if (p < Z) {
                const float ia = ih[p];  // the spectra hold a N: divide by the target's a
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    if (onA) base[(size_t)(c * Z + p) * py + kf] = __fmul2_rn(acc[j][0][c], f2(ia));
                    if (onB) base[(size_t)(c * Z + p) * py + (py - kf)] = __fmul2_rn(acc[j][1][c], f2(c == 1 ? -ia : ia));
                }
            }
        }
        __syncthreads();  // the column stage is reused by the next item
    }
}

cudaError_t ml_build_spectra(const MLHost& h, const Geometry& g, float* K, const double2* tw64, cudaStream_t st)
{
    const int nu = (int)h.ua.size();
    const int NX = g.nx, NY = g.ny;
    // process the unique entries in batches that keep the FP64 staging modest
    const size_t plane = (size_t)NX * NY;
    int batch = (int)std::max<size_t>(1, ((size_t)1 << 31) / (plane * 6 * sizeof(double) * 3));
    if (batch > nu) batch = nu;
    double *ua = nullptr, *ub = nullptr, *udz = nullptr, *T = nullptr;
    double2 *A = nullptr, *B = nullptr;
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaMallocAsync((void**)&ua, nu * sizeof(double), st)) != cudaSuccess) break;
        if ((e = cudaMallocAsync((void**)&ub, nu * sizeof(double), st)) != cudaSuccess) break;
        if ((e = cudaMallocAsync((void**)&udz, nu * sizeof(double), st)) != cudaSuccess) break;
        cudaMemcpyAsync(ua, h.ua.data(), nu * sizeof(double), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(ub, h.ub.data(), nu * sizeof(double), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(udz, h.udz.data(), nu * sizeof(double), cudaMemcpyHostToDevice, st);
        if ((e = cudaMallocAsync((void**)&T, (size_t)batch * 6 * plane * sizeof(double), st)) != cudaSuccess) break;
        if ((e = cudaMallocAsync((void**)&A, (size_t)batch * 6 * g.nkx * NY * sizeof(double2), st)) != cudaSuccess) break;
        if ((e = cudaMallocAsync((void**)&B, (size_t)batch * 6 * g.nkx * g.kyh * sizeof(double2), st)) != cudaSuccess) break;
        for (int u0 = 0; u0 < nu && e == cudaSuccess; u0 += batch) {
            const int nb = std::min(batch, nu - u0);
            const size_t tot = (size_t)nb * plane;
            int blocks = (int)std::min<size_t>((tot + 255) / 256, 152 * 64);
            ml_tensor_kernel<<<blocks, 256, 0, st>>>(nb, ua + u0, ub + u0, udz + u0, NX, NY, h.hx, h.hy, 40.0, T);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            // x then y transform of the parity-extended in-plane tables
            if ((e = run_axis_n(T, true, A, 0, NX, NY, 1, NX, g.px, 6 * nb, tw64, g.lglmax, st)) != cudaSuccess) break;
            if ((e = run_axis_n(A, false, B, 1, g.nkx, NY, 1, NY, g.py, 6 * nb, tw64, g.lglmax, st)) != cudaSuccess) break;
            const size_t kt = (size_t)nb * g.nkx * g.kyh * 6;
            blocks = (int)std::min<size_t>((kt + 255) / 256, 152 * 64);
            const int kyp = ml_kyp(g);
            const size_t kt2 = (size_t)nb * g.nkx * 6 * kyp;
            blocks = (int)std::min<size_t>((kt2 + 255) / 256, 152 * 64);
            ml_finalize_kernel<<<blocks, 256, 0, st>>>(B, K + (size_t)u0 * g.nkx * 6 * kyp, nb, g.nkx, g.kyh, kyp,
                                                       1.0 / ((double)g.px * g.py));
            e = cudaGetLastError();
        }
    } while (0);
    if (ua) cudaFreeAsync(ua, st);
    if (ub) cudaFreeAsync(ub, st);
    if (udz) cudaFreeAsync(udz, st);
    if (T) cudaFreeAsync(T, st);
    if (A) cudaFreeAsync(A, st);
    if (B) cudaFreeAsync(B, st);
    return e;
}

static int grid_n(size_t n)
{
    size_t b = (n + 255) / 256;
    return (int)std::max<size_t>(1, std::min<size_t>(b, 152 * 32));
}

cudaError_t ml_embed(const MLTable& t, const float* M, const float* ms_map, float ms, float* F, cudaStream_t st)
{
    ml_embed_kernel<<<grid_n(3 * (size_t)t.Z * t.NX * t.NY), 256, 0, st>>>(t, M, ms_map, ms, F);
    return cudaGetLastError();
}

cudaError_t ml_extract(const MLTable& t, const float* F, float* H, cudaStream_t st)
{
    ml_extract_kernel<<<grid_n(t.total3), 256, 0, st>>>(t, F, H);
    return cudaGetLastError();
}

int ml_kyp(const Geometry& g) { return (g.kyh + 31) / 32 * 32; }



size_t ml_mix_v2_smem(int Z)
{
    return (size_t)Z * 2 * 6 * 32 * sizeof(float) + (size_t)Z * 3 * 64 * sizeof(float2) +
           (size_t)Z * Z * sizeof(unsigned) + (size_t)Z * sizeof(float);
}

cudaError_t ml_mix(const Geometry& g, int Z, float2* Y, const float* K, const int* pairs, const unsigned* pcode,
                   const float* inv_hz, int variant, int nsm, cudaStream_t st)
{
    const dim3 grid(g.py / 64 + 1, g.nkx);  // folded rows 0 .. py/2
    const int pmax = (Z + 7) / 8;
    const int kyp = ml_kyp(g);
    cudaError_t e;
    if (variant >= 2) {
        // persistent: (variant - 1) CTAs per SM over all (kx, tile) items
        const size_t smem = ml_mix_v2_smem(Z);
        const int ntile = g.py / 64 + 1, nwork = ntile * g.nkx;
        const int G = std::min(nwork, (variant - 1) * nsm);
#define ML_V2(P)                                                                                             \
    e = cudaFuncSetAttribute(ml_mix_v2_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);   \
    if (e != cudaSuccess) return e;                                                                          \
    ml_mix_v2_kernel<P><<<G, 256, smem, st>>>(g, Z, Y, K, kyp, pcode, inv_hz, ntile, nwork);                 \
    return cudaGetLastError();
        if (pmax <= 1) { ML_V2(1) }
        if (pmax <= 2) { ML_V2(2) }
        if (pmax <= 3) { ML_V2(3) }
        if (pmax <= 4) { ML_V2(4) }
        if (pmax <= 5) { ML_V2(5) }
        if (pmax <= 6) { ML_V2(6) }
        if (pmax <= 8) { ML_V2(8) }
#undef ML_V2
        return cudaErrorInvalidValue;
    }
    const size_t smem_s = (size_t)Z * 2 * 6 * 32 * sizeof(float) + (size_t)Z * 3 * 64 * sizeof(float2) +
                          (size_t)Z * Z * sizeof(int);
    const bool staged = variant == 1;
    const size_t smem = staged ? smem_s : (size_t)Z * 3 * 64 * sizeof(float2) + (size_t)Z * Z * sizeof(int);
#define ML_MIX(P)                                                                                              \
    if (staged) {                                                                                              \
        e = cudaFuncSetAttribute(ml_mix_staged_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                        \
        ml_mix_staged_kernel<P><<<grid, 256, smem, st>>>(g, Z, Y, K, kyp, pairs, inv_hz);                      \
    } else {                                                                                                   \
        e = cudaFuncSetAttribute(ml_mix_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
        if (e != cudaSuccess) return e;                                                                        \
        ml_mix_kernel<P><<<grid, 256, smem, st>>>(g, Z, Y, K, kyp, pairs, inv_hz);                             \
    }                                                                                                          \
    return cudaGetLastError();
    if (pmax <= 1) { ML_MIX(1) }
    if (pmax <= 2) { ML_MIX(2) }
    if (pmax <= 3) { ML_MIX(3) }
    if (pmax <= 4) { ML_MIX(4) }
    if (pmax <= 5) { ML_MIX(5) }
    if (pmax <= 6) { ML_MIX(6) }
    if (pmax <= 8) { ML_MIX(8) }
#undef ML_MIX
    return cudaErrorInvalidValue;
}

}  // namespace boris
