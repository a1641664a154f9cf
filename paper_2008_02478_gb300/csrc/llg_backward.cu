// Discrete adjoint of one RK4 step of the LLG equation (the paper has no
// adjoint; this serves gradients of a loss on the final state with respect to
// the initial state and the per-cell Ms and Ku maps).
//
// Forward (recomputed): m1 = m, k_s = f(m_s), m2 = m + dt/2 k1, m3 = m + dt/2 k2,
// m4 = m + dt k3, v = m + dt/6 (k1 + 2k2 + 2k3 + k4), m_out = v/|v|, with
// f(m) = -g' [a + alpha m x a], a = m x H(m), H = Hd(Ms m) + c lap m
// + (2Ku/(mu0 Ms))(m.e)e + Hext, c = 2A/(mu0 Ms).
// Backward: gv = (g - m_out (m_out.g))/|v|; gk_s = w_s dt gv; for s = 4..1 the
// VJP of f at m_s gives gm_s, added to g_m and to gk_{s-1} (times the stage
// coefficient).  The VJP of f splits into a per-cell part (cross products)
// and the field transpose: the demagnetising operator is self-adjoint, so its
// transpose is one more demag application; the Neumann Laplacian is
// symmetric, so its transpose is itself.
#include "boris_internal.cuh"
#include "llg_kernels.cuh"

namespace boris {

template <typename T>
__device__ __forceinline__ void lap_at(const T* __restrict__ f, size_t n, size_t i, int x, int y, int z,
                                       const LLGArgs<T>& a, T out[3])
{
    const T fc[3] = {f[i], f[n + i], f[2 * n + i]};
    out[0] = out[1] = out[2] = T(0);
    auto nb = [&](size_t j, T w) {
        out[0] += w * (f[j] - fc[0]);
        out[1] += w * (f[n + j] - fc[1]);
        out[2] += w * (f[2 * n + j] - fc[2]);
    };
    const size_t sy = a.nx, sz = (size_t)a.nx * a.ny;
    if (x > 0) nb(i - 1, a.ihx2);
    if (x < a.nx - 1) nb(i + 1, a.ihx2);
    if (y > 0) nb(i - sy, a.ihy2);
    if (y < a.ny - 1) nb(i + sy, a.ihy2);
    if (z > 0) nb(i - sz, a.ihz2);
    if (z < a.nz - 1) nb(i + sz, a.ihz2);
}

// Forward stage of the recompute: stores the stage state's effective field H_s
// and k_s, and the next stage state.  s in 0..3; ms = m_s; Hd = demag of Ms m_s.
template <typename T>
__global__ void __launch_bounds__(256) fwd_stage_kernel(LLGArgs<T> a, int s, const T* __restrict__ ms,
                                                        const T* __restrict__ Hd, const T* __restrict__ m0,
                                                        T* __restrict__ Hs, T* __restrict__ ks,
                                                        T* __restrict__ mnext)
{
    const size_t n = a.ncell;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % a.nx), y = (int)((i / a.nx) % a.ny), z = (int)(i / ((size_t)a.nx * a.ny));
        const T m[3] = {ms[i], ms[n + i], ms[2 * n + i]};
        T lap[3];
        lap_at(ms, n, i, x, y, z, a, lap);
        const T Ms = a.ms_map ? a.ms_map[i] : a.Ms;
        const T Ku = a.ku_map ? a.ku_map[i] : a.Ku;
        const T inv = T(1) / (T(MU0_D) * Ms);
        const T me = m[0] * a.e[0] + m[1] * a.e[1] + m[2] * a.e[2];
        T H[3];
#pragma unroll
        for (int c = 0; c < 3; c++)
            H[c] = Hd[c * n + i] + T(2) * a.A * inv * lap[c] + T(2) * Ku * inv * me * a.e[c] + a.Hext[c];
        const T A_[3] = {m[1] * H[2] - m[2] * H[1], m[2] * H[0] - m[0] * H[2], m[0] * H[1] - m[1] * H[0]};
        const T B_[3] = {m[1] * A_[2] - m[2] * A_[1], m[2] * A_[0] - m[0] * A_[2], m[0] * A_[1] - m[1] * A_[0]};
        const T cdt = s == 2 ? a.dt : T(0.5) * a.dt;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const T k = -a.gp * (A_[c] + a.alpha * B_[c]);
            Hs[c * n + i] = H[c];
            ks[c * n + i] = k;
            if (s < 3) mnext[c * n + i] = m0[c * n + i] + cdt * k;
        }
    }
}

// Start of the backward pass: v from the stored stage derivatives, then
// gv = (g - m_out (m_out.g))/|v|; g_m = gv; gk_s = w_s dt gv for the four stages.
template <typename T>
__global__ void __launch_bounds__(256) bwd_start_kernel(LLGArgs<T> a, const T* __restrict__ m0,
                                                        const T* __restrict__ k1, const T* __restrict__ k2,
                                                        const T* __restrict__ k3, const T* __restrict__ k4,
                                                        const T* __restrict__ gout, T* __restrict__ gm,
                                                        T* __restrict__ gk)  // gk: 4 x 3n
{
    const size_t n = a.ncell;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        T v[3], g[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const size_t j = c * n + i;
            v[c] = m0[j] + a.dt / T(6) * (k1[j] + T(2) * k2[j] + T(2) * k3[j] + k4[j]);
            g[c] = gout[j];
        }
        const T nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const T mo[3] = {v[0] / nv, v[1] / nv, v[2] / nv};
        const T mg = mo[0] * g[0] + mo[1] * g[1] + mo[2] * g[2];
        const T w[4] = {a.dt / T(6), a.dt / T(3), a.dt / T(3), a.dt / T(6)};
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const T gv = (g[c] - mo[c] * mg) / nv;
            gm[c * n + i] = gv;
#pragma unroll
            for (int s = 0; s < 4; s++) gk[(size_t)s * 3 * n + c * n + i] = w[s] * gv;
        }
    }
}

// Per-cell part of the VJP of f at stage state m_s: from gk, writes
// gH = ga x m (ga = -g' gk + (-g' alpha gk) x m) and the local gm part
// a x gB + H x ga.
template <typename T>
__global__ void __launch_bounds__(256) bwd_local_kernel(LLGArgs<T> a, const T* __restrict__ ms,
                                                        const T* __restrict__ Hs, const T* __restrict__ gk,
                                                        T* __restrict__ gH, T* __restrict__ gml)
{
    const size_t n = a.ncell;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const T m[3] = {ms[i], ms[n + i], ms[2 * n + i]};
        const T H[3] = {Hs[i], Hs[n + i], Hs[2 * n + i]};
        const T g[3] = {gk[i], gk[n + i], gk[2 * n + i]};
        const T A_[3] = {m[1] * H[2] - m[2] * H[1], m[2] * H[0] - m[0] * H[2], m[0] * H[1] - m[1] * H[0]};
        const T gA[3] = {-a.gp * g[0], -a.gp * g[1], -a.gp * g[2]};
        const T gB[3] = {gA[0] * a.alpha, gA[1] * a.alpha, gA[2] * a.alpha};
        // b = m x a: d/dm = a x gB, d/da = gB x m
        const T ga[3] = {gA[0] + gB[1] * m[2] - gB[2] * m[1], gA[1] + gB[2] * m[0] - gB[0] * m[2],
                         gA[2] + gB[0] * m[1] - gB[1] * m[0]};
        const T gm1[3] = {A_[1] * gB[2] - A_[2] * gB[1], A_[2] * gB[0] - A_[0] * gB[2], A_[0] * gB[1] - A_[1] * gB[0]};
        // a = m x H: d/dm = H x ga, d/dH = ga x m
        const T gm2[3] = {H[1] * ga[2] - H[2] * ga[1], H[2] * ga[0] - H[0] * ga[2], H[0] * ga[1] - H[1] * ga[0]};
        const T gh[3] = {ga[1] * m[2] - ga[2] * m[1], ga[2] * m[0] - ga[0] * m[2], ga[0] * m[1] - ga[1] * m[0]};
#pragma unroll
        for (int c = 0; c < 3; c++) {
            gH[c * n + i] = gh[c];
            gml[c * n + i] = gm1[c] + gm2[c];
        }
    }
}

// Field transpose at stage state m_s: gm_s = gml + Ms D(gH) + L(c gH)
// + (2Ku/(mu0 Ms))(gH.e)e; accumulates gm_s into g_m and coef * gm_s into the
// previous stage's gk, and the Ms / Ku gradients.  DgH = demag of gH.
template <typename T>
__global__ void __launch_bounds__(256) bwd_field_kernel(LLGArgs<T> a, const T* __restrict__ ms,
                                                        const T* __restrict__ gH, const T* __restrict__ DgH,
                                                        const T* __restrict__ gml, T* __restrict__ gm,
                                                        T* __restrict__ gk_prev, T coef, T* __restrict__ gMs,
                                                        T* __restrict__ gKu)
{
    const size_t n = a.ncell;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % a.nx), y = (int)((i / a.nx) % a.ny), z = (int)(i / ((size_t)a.nx * a.ny));
        const T m[3] = {ms[i], ms[n + i], ms[2 * n + i]};
        const T g[3] = {gH[i], gH[n + i], gH[2 * n + i]};
        const T Ms = a.ms_map ? a.ms_map[i] : a.Ms;
        const T Ku = a.ku_map ? a.ku_map[i] : a.Ku;
        const T inv = T(1) / (T(MU0_D) * Ms);
        // L(c gH) at i: sum_j w (c_j gH_j - c_i gH_i)
        T lcg[3] = {T(0), T(0), T(0)};
        const T ci = T(2) * a.A * inv;
        auto nb = [&](size_t j, T w) {
            const T Msj = a.ms_map ? a.ms_map[j] : a.Ms;
            const T cj = T(2) * a.A / (T(MU0_D) * Msj);
            lcg[0] += w * (cj * gH[j] - ci * g[0]);
            lcg[1] += w * (cj * gH[n + j] - ci * g[1]);
            lcg[2] += w * (cj * gH[2 * n + j] - ci * g[2]);
        };
        const size_t sy = a.nx, sz = (size_t)a.nx * a.ny;
        if (x > 0) nb(i - 1, a.ihx2);
        if (x < a.nx - 1) nb(i + 1, a.ihx2);
        if (y > 0) nb(i - sy, a.ihy2);
        if (y < a.ny - 1) nb(i + sy, a.ihy2);
        if (z > 0) nb(i - sz, a.ihz2);
        if (z < a.nz - 1) nb(i + sz, a.ihz2);
        T lm[3];
        lap_at(ms, n, i, x, y, z, a, lm);
        const T me = m[0] * a.e[0] + m[1] * a.e[1] + m[2] * a.e[2];
        const T ge = g[0] * a.e[0] + g[1] * a.e[1] + g[2] * a.e[2];
        const T D[3] = {DgH[i], DgH[n + i], DgH[2 * n + i]};
        T gms = m[0] * D[0] + m[1] * D[1] + m[2] * D[2];
        gms -= (ci / Ms) * (g[0] * lm[0] + g[1] * lm[1] + g[2] * lm[2]);
        gms -= T(2) * Ku * inv / Ms * me * ge;
        const T gku = T(2) * inv * me * ge;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const size_t j = c * n + i;
            const T v = gml[j] + Ms * D[c] + lcg[c] + T(2) * Ku * inv * ge * a.e[c];
            gm[j] += v;
            if (gk_prev) gk_prev[j] += coef * v;
        }
        if (gMs) gMs[i] += gms;
        if (gKu) gKu[i] += gku;
    }
}

static int grid_for_n(size_t n)
{
    size_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b > 0 ? b : 1);
}

template <typename T>
cudaError_t launch_fwd_stage(const LLGArgs<T>& a, int s, const T* ms, const T* Hd, const T* m0, T* Hs, T* ks,
                             T* mnext, cudaStream_t st)
{
    fwd_stage_kernel<T><<<grid_for_n(a.ncell), 256, 0, st>>>(a, s, ms, Hd, m0, Hs, ks, mnext);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_bwd_start(const LLGArgs<T>& a, const T* m0, const T* k1, const T* k2, const T* k3, const T* k4,
                             const T* gout, T* gm, T* gk, cudaStream_t st)
{
    bwd_start_kernel<T><<<grid_for_n(a.ncell), 256, 0, st>>>(a, m0, k1, k2, k3, k4, gout, gm, gk);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_bwd_local(const LLGArgs<T>& a, const T* ms, const T* Hs, const T* gk, T* gH, T* gml,
                             cudaStream_t st)
{
    bwd_local_kernel<T><<<grid_for_n(a.ncell), 256, 0, st>>>(a, ms, Hs, gk, gH, gml);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_bwd_field(const LLGArgs<T>& a, const T* ms, const T* gH, const T* DgH, const T* gml, T* gm,
                             T* gk_prev, T coef, T* gMs, T* gKu, cudaStream_t st)
{
    bwd_field_kernel<T><<<grid_for_n(a.ncell), 256, 0, st>>>(a, ms, gH, DgH, gml, gm, gk_prev, coef, gMs, gKu);
    return cudaGetLastError();
}

#define BWD_INST(T)                                                                                              \
    template cudaError_t launch_fwd_stage<T>(const LLGArgs<T>&, int, const T*, const T*, const T*, T*, T*, T*,    \
                                             cudaStream_t);                                                      \
    template cudaError_t launch_bwd_start<T>(const LLGArgs<T>&, const T*, const T*, const T*, const T*, const T*, \
                                             const T*, T*, T*, cudaStream_t);                                    \
    template cudaError_t launch_bwd_local<T>(const LLGArgs<T>&, const T*, const T*, const T*, T*, T*,             \
                                             cudaStream_t);                                                      \
    template cudaError_t launch_bwd_field<T>(const LLGArgs<T>&, const T*, const T*, const T*, const T*, T*, T*, T, \
                                             T*, T*, cudaStream_t);
BWD_INST(float)
BWD_INST(double)

}  // namespace boris
