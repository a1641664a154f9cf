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

// m = ms[i]; k = -g' [m x H + alpha m x (m x H)], H = hd + exchange + anisotropy + Hext.
template <typename T>
__device__ __forceinline__ void cell_rhs(const LLGArgs<T>& a, const T* __restrict__ ms, const T hd[3], size_t i, int x,
                                         int y, int z, T m[3], T k[3])
{
    const size_t n = a.ncell;
    m[0] = ms[i];
    m[1] = ms[n + i];
    m[2] = ms[2 * n + i];
    T lap[3] = {T(0), T(0), T(0)};
    auto nb = [&](size_t j, T w) {
        lap[0] += w * (ms[j] - m[0]);
        lap[1] += w * (ms[n + j] - m[1]);
        lap[2] += w * (ms[2 * n + j] - m[2]);
    };
    const size_t sy = a.nx, sz = (size_t)a.nx * a.ny;
    if (x > 0) nb(i - 1, a.ihx2);
    if (x < a.nx - 1) nb(i + 1, a.ihx2);
    if (y > 0) nb(i - sy, a.ihy2);
    if (y < a.ny - 1) nb(i + sy, a.ihy2);
    if (z > 0) nb(i - sz, a.ihz2);
    if (z < a.nz - 1) nb(i + sz, a.ihz2);
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
