// Per-cell effective field and Landau-Lifshitz right-hand side (Eq. 1 in LL
// form; Table 1 exchange with Neumann boundaries, uniaxial anisotropy,
// applied field), shared by the stage kernels and the fused inverse-x-
// transform + stage kernel.
#pragma once
#include "llg_kernels.cuh"

namespace boris {

// k = -g' [m x H + alpha m x (m x H)] from the cell's m, its Laplacian
// sum_j w_j (m_j - m), H_d, Ms and Ku.
template <typename T>
__device__ __forceinline__ void rhs_local(const LLGArgs<T>& a, const T m[3], const T lap[3], const T hd[3], T Ms, T Ku,
                                          T k[3])
{
    const T inv = T(1) / (T(MU0_D) * Ms);
    const T cex = T(2) * a.A * inv;
    const T me = m[0] * a.e[0] + m[1] * a.e[1] + m[2] * a.e[2];
    const T can = T(2) * Ku * inv * me;
    T H[3];
#pragma unroll
    for (int c = 0; c < 3; c++) H[c] = hd[c] + cex * lap[c] + can * a.e[c] + a.Hext[c];
    const T mxH[3] = {m[1] * H[2] - m[2] * H[1], m[2] * H[0] - m[0] * H[2], m[0] * H[1] - m[1] * H[0]};
    const T mmH[3] = {m[1] * mxH[2] - m[2] * mxH[1], m[2] * mxH[0] - m[0] * mxH[2], m[0] * mxH[1] - m[1] * mxH[0]};
#pragma unroll
    for (int c = 0; c < 3; c++) k[c] = -a.gp * (mxH[c] + a.alpha * mmH[c]);
}

// ---------------------------------------------------------------------------
// Further Table 1 terms (boris_field_terms): second-order uniaxial and cubic
// anisotropy (local), bulk or interfacial DMI with the non-homogeneous
// Neumann boundary condition dm/dn = (D/2A) u x m (u = n for bulk, z x n for
// interfacial DMI, n the outward normal).  A neighbour outside the mesh is
// the ghost m + h (D/2A) u x m; the exchange Laplacian and the central DMI
// differences both use it (without DMI the ghost is m: homogeneous Neumann).
// TC is the arithmetic type (T for the stage kernels, double for energies).
// ---------------------------------------------------------------------------
template <typename TC, typename T>
__device__ __forceinline__ void nb_or_ghost(const LLGArgs<T>& a, const T* __restrict__ ms, bool inside, size_t j,
                                            int axis, int sgn, const TC m[3], TC out[3])
{
    const size_t n = a.ncell;
    if (inside) {
        out[0] = (TC)ms[j];
        out[1] = (TC)ms[n + j];
        out[2] = (TC)ms[2 * n + j];
        return;
    }
    out[0] = m[0];
    out[1] = m[1];
    out[2] = m[2];
    if (a.dmi == 0) return;
    int ua;
    TC us;
    if (a.dmi == 1) {
        ua = axis;
        us = (TC)sgn;
    } else {
        if (axis == 2) return;  // z x z = 0
        ua = axis == 0 ? 1 : 0;  // z x x = y, z x y = -x
        us = axis == 0 ? (TC)sgn : (TC)(-sgn);
    }
    const TC h = axis == 0 ? (TC)a.hx : axis == 1 ? (TC)a.hy : (TC)a.hz;
    const TC f = h * (TC)a.kD * us;
    if (ua == 0) {  // x x m = (0, -mz, my)
        out[1] -= f * m[2];
        out[2] += f * m[1];
    } else if (ua == 1) {  // y x m = (mz, 0, -mx)
        out[0] += f * m[2];
        out[2] -= f * m[0];
    } else {  // z x m = (-my, mx, 0)
        out[0] -= f * m[1];
        out[1] += f * m[0];
    }
}

// Exchange Laplacian sum_axes (m_+ + m_- - 2m)/h^2 and the DMI vector w with
// H_dmi = (2D/(mu0 Ms)) w: bulk w = -curl m, interfacial w = (-dmz/dx,
// -dmz/dy, dmx/dx + dmy/dy), derivatives (m_+ - m_-)/(2h).
template <typename TC, typename T>
__device__ __forceinline__ void ext_exchange_dmi(const LLGArgs<T>& a, const T* __restrict__ ms, size_t i, int x, int y,
                                                 int z, const TC m[3], TC lap[3], TC w[3])
{
    const size_t sy = a.nx, sz = (size_t)a.nx * a.ny;
    const bool px = a.pbc & 1, py = a.pbc & 2, pz = a.pbc & 4;
    TC xm[3], xp[3], ym[3], yp[3], zm[3], zp[3];
    // a periodic axis wraps to the cell on the opposite face
    nb_or_ghost<TC>(a, ms, x > 0 || px, x > 0 ? i - 1 : i + (a.nx - 1), 0, -1, m, xm);
    nb_or_ghost<TC>(a, ms, x < a.nx - 1 || px, x < a.nx - 1 ? i + 1 : i - (a.nx - 1), 0, 1, m, xp);
    nb_or_ghost<TC>(a, ms, y > 0 || py, y > 0 ? i - sy : i + (a.ny - 1) * sy, 1, -1, m, ym);
    nb_or_ghost<TC>(a, ms, y < a.ny - 1 || py, y < a.ny - 1 ? i + sy : i - (a.ny - 1) * sy, 1, 1, m, yp);
    nb_or_ghost<TC>(a, ms, z > 0 || pz, z > 0 ? i - sz : i + (a.nz - 1) * sz, 2, -1, m, zm);
    nb_or_ghost<TC>(a, ms, z < a.nz - 1 || pz, z < a.nz - 1 ? i + sz : i - (a.nz - 1) * sz, 2, 1, m, zp);
#pragma unroll
    for (int c = 0; c < 3; c++)
        lap[c] = (xp[c] + xm[c] - TC(2) * m[c]) * (TC)a.ihx2 + (yp[c] + ym[c] - TC(2) * m[c]) * (TC)a.ihy2 +
                 (zp[c] + zm[c] - TC(2) * m[c]) * (TC)a.ihz2;
    w[0] = w[1] = w[2] = TC(0);
    if (a.dmi == 0) return;
    TC dx[3], dy[3], dz[3];
    const TC ix = TC(0.5) / (TC)a.hx, iy = TC(0.5) / (TC)a.hy, iz = TC(0.5) / (TC)a.hz;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        dx[c] = (xp[c] - xm[c]) * ix;
        dy[c] = (yp[c] - ym[c]) * iy;
        dz[c] = (zp[c] - zm[c]) * iz;
    }
    if (a.dmi == 1) {
        w[0] = -(dy[2] - dz[1]);
        w[1] = -(dz[0] - dx[2]);
        w[2] = -(dx[1] - dy[0]);
    } else {
        w[0] = -dx[2];
        w[1] = -dy[2];
        w[2] = dx[0] + dy[1];
    }
}

// Local further terms added to H: (4 K2/(mu0 Ms)) (1 - (m.e)^2)(m.e) e and the
// cubic field -(2 Kc1/(mu0 Ms)) [e1 a(b^2 + c^2) + ...] - (2 Kc2/(mu0 Ms)) [e1 a b^2 c^2 + ...].
template <typename TC, typename T>
__device__ __forceinline__ void ext_local_field(const LLGArgs<T>& a, const TC m[3], TC Ms, TC H[3])
{
    const TC inv = TC(1) / (TC(MU0_D) * Ms);
    if (a.K2 != T(0)) {
        const TC me = m[0] * (TC)a.e[0] + m[1] * (TC)a.e[1] + m[2] * (TC)a.e[2];
        const TC f = TC(4) * (TC)a.K2 * inv * (TC(1) - me * me) * me;
#pragma unroll
        for (int c = 0; c < 3; c++) H[c] += f * (TC)a.e[c];
    }
    if (a.Kc1 != T(0) || a.Kc2 != T(0)) {
        const TC p = m[0] * (TC)a.c1[0] + m[1] * (TC)a.c1[1] + m[2] * (TC)a.c1[2];
        const TC q = m[0] * (TC)a.c2[0] + m[1] * (TC)a.c2[1] + m[2] * (TC)a.c2[2];
        const TC r = m[0] * (TC)a.c3[0] + m[1] * (TC)a.c3[1] + m[2] * (TC)a.c3[2];
        const TC f1 = -TC(2) * (TC)a.Kc1 * inv, f2 = -TC(2) * (TC)a.Kc2 * inv;
        const TC g1 = f1 * p * (q * q + r * r) + f2 * p * q * q * r * r;
        const TC g2 = f1 * q * (p * p + r * r) + f2 * p * p * q * r * r;
        const TC g3 = f1 * r * (p * p + q * q) + f2 * p * p * q * q * r;
#pragma unroll
        for (int c = 0; c < 3; c++) H[c] += g1 * (TC)a.c1[c] + g2 * (TC)a.c2[c] + g3 * (TC)a.c3[c];
    }
}

// Energy densities of the local further terms: K2 (1 - (m.e)^2)^2 and the cubic density.
template <typename TC, typename T>
__device__ __forceinline__ TC ext_local_energy(const LLGArgs<T>& a, const TC m[3])
{
    const TC me = m[0] * (TC)a.e[0] + m[1] * (TC)a.e[1] + m[2] * (TC)a.e[2];
    const TC p = m[0] * (TC)a.c1[0] + m[1] * (TC)a.c1[1] + m[2] * (TC)a.c1[2];
    const TC q = m[0] * (TC)a.c2[0] + m[1] * (TC)a.c2[1] + m[2] * (TC)a.c2[2];
    const TC r = m[0] * (TC)a.c3[0] + m[1] * (TC)a.c3[1] + m[2] * (TC)a.c3[2];
    const TC u = TC(1) - me * me;
    return (TC)a.K2 * u * u + (TC)a.Kc1 * (p * p * q * q + p * p * r * r + q * q * r * r) +
           (TC)a.Kc2 * p * p * q * q * r * r;
}

// ---------------------------------------------------------------------------
// Thermal field: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) from its
// published definition - ten rounds of (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^
// k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)), the key bumped by the Weyl
// constants between rounds - and Box-Muller normals from its four words.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(unsigned int c[4], unsigned int k0, unsigned int k1)
{
    constexpr unsigned int M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const unsigned int hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
        const unsigned int hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
        const unsigned int n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

// three standard normals of cell i at the plan's current step
template <typename T>
__device__ __forceinline__ void thermal_normals(const LLGArgs<T>& a, size_t i, T g[3])
{
    const unsigned long long s = *a.step;
    unsigned int c[4] = {(unsigned int)i, (unsigned int)s, (unsigned int)(s >> 32), 0u};
    philox4x32_10(c, a.seed_lo, a.seed_hi);
    T u[4];
#pragma unroll
    for (int j = 0; j < 4; j++) u[j] = ((T)c[j] + T(0.5)) * T(2.3283064365386963e-10);  // 2^-32
    const T ra = sqrt(T(-2) * log(u[0])), rb = sqrt(T(-2) * log(u[2]));
    T s1, c1, s3, c3;
    if constexpr (sizeof(T) == 4) {
        sincospif(2.f * u[1], &s1, &c1);
        sincospif(2.f * u[3], &s3, &c3);
    } else {
        sincospi(2.0 * u[1], &s1, &c1);
        sincospi(2.0 * u[3], &s3, &c3);
    }
    (void)s3;
    g[0] = ra * c1;
    g[1] = ra * s1;
    g[2] = rb * c3;
}

// k = -g' [m x H + alpha m x (m x H)] for a given total field H.
template <typename T>
__device__ __forceinline__ void rhs_from_field(const LLGArgs<T>& a, const T m[3], const T H[3], T k[3])
{
    const T mxH[3] = {m[1] * H[2] - m[2] * H[1], m[2] * H[0] - m[0] * H[2], m[0] * H[1] - m[1] * H[0]};
    const T mmH[3] = {m[1] * mxH[2] - m[2] * mxH[1], m[2] * mxH[0] - m[0] * mxH[2], m[0] * mxH[1] - m[1] * mxH[0]};
#pragma unroll
    for (int c = 0; c < 3; c++) k[c] = -a.gp * (mxH[c] + a.alpha * mmH[c]);
}

// m = ms[i]; k = -g' [m x H + alpha m x (m x H)], H = hd + exchange + anisotropy + Hext
// (+ the further terms when a.extra is set).
template <typename T>
__device__ __forceinline__ void cell_rhs(const LLGArgs<T>& a, const T* __restrict__ ms, const T hd[3], size_t i, int x,
                                         int y, int z, T m[3], T k[3])
{
    const size_t n = a.ncell;
    m[0] = ms[i];
    m[1] = ms[n + i];
    m[2] = ms[2 * n + i];
    if (a.extra) {
        T lap[3], w[3];
        ext_exchange_dmi<T>(a, ms, i, x, y, z, m, lap, w);
        const T Ms = a.ms_map ? a.ms_map[i] : a.Ms;
        const T Ku = a.ku_map ? a.ku_map[i] : a.Ku;
        const T inv = T(1) / (T(MU0_D) * Ms);
        const T cex = T(2) * a.A * inv, cd = T(2) * a.D * inv;
        const T me = m[0] * a.e[0] + m[1] * a.e[1] + m[2] * a.e[2];
        const T can = T(2) * Ku * inv * me;
        T H[3];
#pragma unroll
        for (int c = 0; c < 3; c++) H[c] = hd[c] + cex * lap[c] + cd * w[c] + can * a.e[c] + a.Hext[c];
        ext_local_field<T>(a, m, Ms, H);
        if (a.hadd) {
#pragma unroll
            for (int c = 0; c < 3; c++) H[c] += a.hadd[c * n + i];
        }
        if (a.th_s0 > T(0)) {
            T g[3];
            thermal_normals(a, i, g);
            const T sg = a.th_s0 / sqrt(Ms);
#pragma unroll
            for (int c = 0; c < 3; c++) H[c] += sg * g[c];
        }
        rhs_from_field(a, m, H, k);
        return;
    }
    T lap[3] = {T(0), T(0), T(0)};
    auto nb = [&](size_t j, T w) {
        lap[0] += w * (ms[j] - m[0]);
        lap[1] += w * (ms[n + j] - m[1]);
        lap[2] += w * (ms[2 * n + j] - m[2]);
    };
    const size_t sy = a.nx, sz = (size_t)a.nx * a.ny;
    // a missing neighbour is the cell itself (homogeneous Neumann), or the
    // cell on the opposite face along a periodic axis
    if (x > 0) nb(i - 1, a.ihx2);
    else if (a.pbc & 1) nb(i + (a.nx - 1), a.ihx2);
    if (x < a.nx - 1) nb(i + 1, a.ihx2);
    else if (a.pbc & 1) nb(i - (a.nx - 1), a.ihx2);
    if (y > 0) nb(i - sy, a.ihy2);
    else if (a.pbc & 2) nb(i + (a.ny - 1) * sy, a.ihy2);
    if (y < a.ny - 1) nb(i + sy, a.ihy2);
    else if (a.pbc & 2) nb(i - (a.ny - 1) * sy, a.ihy2);
    if (z > 0) nb(i - sz, a.ihz2);
    else if (a.pbc & 4) nb(i + (a.nz - 1) * sz, a.ihz2);
    if (z < a.nz - 1) nb(i + sz, a.ihz2);
    else if (a.pbc & 4) nb(i - (a.nz - 1) * sz, a.ihz2);
    const T Ms = a.ms_map ? a.ms_map[i] : a.Ms;
    const T Ku = a.ku_map ? a.ku_map[i] : a.Ku;
    rhs_local(a, m, lap, hd, Ms, Ku, k);
}

template <typename T>
__device__ __forceinline__ void field_and_rhs(const LLGArgs<T>& a, const T* __restrict__ ms, const T* __restrict__ Hd,
                                              size_t i, int x, int y, int z, T m[3], T k[3])
{
    const size_t n = a.ncell;
    const T hd[3] = {Hd[i], Hd[n + i], Hd[2 * n + i]};
    cell_rhs(a, ms, hd, i, x, y, z, m, k);
}

// RK4 stage combine for cell i (stage s in 0..3; m = stage state, k = its rate).
template <typename T>
__device__ __forceinline__ void rk4_combine(const LLGArgs<T>& a, int s, size_t i, const T m[3], const T k[3],
                                            T* __restrict__ m0, T* __restrict__ acc, T* __restrict__ mnext)
{
    const size_t n = a.ncell;
    if (s == 0) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            acc[c * n + i] = k[c];
            mnext[c * n + i] = m[c] + T(0.5) * a.dt * k[c];
        }
    } else if (s < 3) {
        const T cdt = s == 1 ? T(0.5) * a.dt : a.dt;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            acc[c * n + i] += T(2) * k[c];
            mnext[c * n + i] = m0[c * n + i] + cdt * k[c];
        }
    } else {
        T v[3];
#pragma unroll
        for (int c = 0; c < 3; c++) v[c] = m0[c * n + i] + a.dt * (T(1) / T(6)) * (acc[c * n + i] + k[c]);
        const T inv = T(1) / sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
        for (int c = 0; c < 3; c++) m0[c * n + i] = v[c] * inv;
    }
}

}  // namespace boris
