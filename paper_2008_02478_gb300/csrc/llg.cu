// Fused effective-field + LLG right-hand side + Runge-Kutta stage kernels.
//
// Per cell (Eq. 1 in Landau-Lifshitz form, fields of Table 1):
//   H = Hd + (2A/(mu0 Ms)) lap(m) + (2Ku/(mu0 Ms)) (m.e) e + Hext,
//   lap(m) = sum over axes and existing neighbours j of (m_j - m)/h^2
//            (homogeneous Neumann boundary: a missing neighbour equals m),
//   k = -gamma/(1+alpha^2) [m x H + alpha m x (m x H)].
// RK4 (Section 2; four field evaluations per step, Section 7): the stage
// kernel consumes Hd of the current stage state, accumulates sum w_s k_s and
// writes the next stage state m0 + c dt k; the fourth stage writes
// normalise(m0 + dt/6 (k1 + 2k2 + 2k3 + k4)) over m0 in place.
// RKF45 (Fehlberg): the same field evaluation, with the stage combinations of
// the Fehlberg tableau and the embedded error max |m5 - m4|.
#include "boris_internal.cuh"
#include "llg_kernels.cuh"
#include "llg_cell.cuh"
#include "multilayer.cuh"

namespace boris {

// Runge-Kutta-Fehlberg 4(5) coefficients (Fehlberg's published tableau):
// stage s state = m0 + dt sum_j A[s][j] k_j; 4th/5th order weights B4, B5.
__constant__ double RKF_A[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 4, 0, 0, 0, 0},
    {3.0 / 32, 9.0 / 32, 0, 0, 0},
    {1932.0 / 2197, -7200.0 / 2197, 7296.0 / 2197, 0, 0},
    {439.0 / 216, -8.0, 3680.0 / 513, -845.0 / 4104, 0},
    {-8.0 / 27, 2.0, -3544.0 / 2565, 1859.0 / 4104, -11.0 / 40},
};
__constant__ double RKF_B4[6] = {25.0 / 216, 0.0, 1408.0 / 2565, 2197.0 / 4104, -1.0 / 5, 0.0};
__constant__ double RKF_B5[6] = {16.0 / 135, 0.0, 6656.0 / 12825, 28561.0 / 56430, -9.0 / 50, 2.0 / 55};

// stage s in 0..3; ms = stage state (m0 itself for s = 0).
template <typename T>
__global__ void __launch_bounds__(256) rk4_stage_kernel(LLGArgs<T> a, int s, const T* __restrict__ ms,
                                                        const T* __restrict__ Hd, T* __restrict__ m0,
                                                        T* __restrict__ acc, T* __restrict__ mnext)
{
    const size_t n = a.ncell;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % a.nx);
        const int y = (int)((i / a.nx) % a.ny);
        const int z = (int)(i / ((size_t)a.nx * a.ny));
        T m[3], k[3];
        field_and_rhs(a, ms, Hd, i, x, y, z, m, k);
        rk4_combine(a, s, i, m, k, m0, acc, mnext);
    }
}

// FP32 RK4 stage over quads of four consecutive x cells (nx % 4 == 0): one
// 16-byte load per component and neighbour direction instead of four scalar
// loads, so each thread keeps several times more bytes in flight.  The x
// neighbours of the quad's end cells come from scalar loads that hit the
// lines the adjacent quads bring in.
__device__ __forceinline__ float q_get(const float4& v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }
__device__ __forceinline__ void q_set(float4& v, int j, float f)
{
    if (j == 0) v.x = f;
    else if (j == 1) v.y = f;
    else if (j == 2) v.z = f;
    else v.w = f;
}
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, const float4& v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void lap_add(float4& L, const float4& u, const float4& v, float w)
{
    L.x += w * (u.x - v.x);
    L.y += w * (u.y - v.y);
    L.z += w * (u.z - v.z);
    L.w += w * (u.w - v.w);
}

// WRAP: some axis is periodic (neighbours wrap around the mesh); the open-mesh
// instantiation keeps the conditional loads.
template <bool WRAP>
__global__ void __launch_bounds__(256, 4) rk4_stage_quad_kernel(LLGArgs<float> a, int s, const float* __restrict__ ms,
                                                             const float* __restrict__ Hd, float* __restrict__ m0,
                                                             float* __restrict__ acc, float* __restrict__ mnext)
{
    const size_t n = a.ncell, nq = n >> 2;
    const int nxq = a.nx >> 2;
    const size_t sy = a.nx, sz = (size_t)a.nx * a.ny;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nq; q += (size_t)gridDim.x * blockDim.x) {
        const size_t row = q / nxq;
        const int x0 = (int)(q - row * nxq) * 4;
        const int y = (int)(row % a.ny), z = (int)(row / a.ny);
        const size_t i = q * 4;
        const bool wy = WRAP && (a.pbc & 2), wz = WRAP && (a.pbc & 4);
        const ptrdiff_t oym = y > 0 ? -(ptrdiff_t)sy : wy ? (ptrdiff_t)((a.ny - 1) * sy) : 0;
        const ptrdiff_t oyp = y < a.ny - 1 ? (ptrdiff_t)sy : wy ? -(ptrdiff_t)((a.ny - 1) * sy) : 0;
        const ptrdiff_t ozm = z > 0 ? -(ptrdiff_t)sz : wz ? (ptrdiff_t)((a.nz - 1) * sz) : 0;
        const ptrdiff_t ozp = z < a.nz - 1 ? (ptrdiff_t)sz : wz ? -(ptrdiff_t)((a.nz - 1) * sz) : 0;
        float4 mv[3], L[3], hv[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float* b = ms + c * n + i;
            const float4 v = ld4(b);
            mv[c] = v;
            hv[c] = ld4(Hd + c * n + i);
            // x: inner differences of the quad plus the two outer neighbours
            // (a missing neighbour equals the cell: zero difference; along a
            // periodic axis the neighbour wraps to the opposite face)
            const bool wx = WRAP && (a.pbc & 1);
            const float xl = x0 > 0 ? b[-1] : wx ? b[a.nx - 1] : v.x;
            const float xr = x0 + 4 < a.nx ? b[4] : wx ? b[4 - a.nx] : v.w;
            float4 Lc;
            Lc.x = a.ihx2 * ((xl - v.x) + (v.y - v.x));
            Lc.y = a.ihx2 * ((v.x - v.y) + (v.z - v.y));
            Lc.z = a.ihx2 * ((v.y - v.z) + (v.w - v.z));
            Lc.w = a.ihx2 * ((v.z - v.w) + (xr - v.w));
            if (WRAP) {
                // y and z neighbours as offsets: a missing one is the cell itself
                // (offset 0, zero difference), so all four loads issue unconditionally
                lap_add(Lc, ld4(b + oym), v, a.ihy2);
                lap_add(Lc, ld4(b + oyp), v, a.ihy2);
                lap_add(Lc, ld4(b + ozm), v, a.ihz2);
                lap_add(Lc, ld4(b + ozp), v, a.ihz2);
            } else {
                if (y > 0) lap_add(Lc, ld4(b - sy), v, a.ihy2);
                if (y < a.ny - 1) lap_add(Lc, ld4(b + sy), v, a.ihy2);
                if (z > 0) lap_add(Lc, ld4(b - sz), v, a.ihz2);
                if (z < a.nz - 1) lap_add(Lc, ld4(b + sz), v, a.ihz2);
            }
            L[c] = Lc;
        }
        const float4 Msv = a.ms_map ? ld4(a.ms_map + i) : make_float4(a.Ms, a.Ms, a.Ms, a.Ms);
        const float4 Kuv = a.ku_map ? ld4(a.ku_map + i) : make_float4(a.Ku, a.Ku, a.Ku, a.Ku);
        float4 kv[3];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const float m[3] = {q_get(mv[0], j), q_get(mv[1], j), q_get(mv[2], j)};
            const float lap[3] = {q_get(L[0], j), q_get(L[1], j), q_get(L[2], j)};
            const float hd[3] = {q_get(hv[0], j), q_get(hv[1], j), q_get(hv[2], j)};
            float k[3];
            rhs_local(a, m, lap, hd, q_get(Msv, j), q_get(Kuv, j), k);
#pragma unroll
            for (int c = 0; c < 3; c++) q_set(kv[c], j, k[c]);
        }
        if (s == 0) {
            const float h = 0.5f * a.dt;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                st4(acc + c * n + i, kv[c]);
                const float4 v = mv[c], k = kv[c];
                st4(mnext + c * n + i, make_float4(v.x + h * k.x, v.y + h * k.y, v.z + h * k.z, v.w + h * k.w));
            }
        } else if (s < 3) {
            const float h = s == 1 ? 0.5f * a.dt : a.dt;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                float4 ac = ld4(acc + c * n + i);
                const float4 b = ld4(m0 + c * n + i), k = kv[c];
                ac.x += 2.f * k.x;
                ac.y += 2.f * k.y;
                ac.z += 2.f * k.z;
                ac.w += 2.f * k.w;
                st4(acc + c * n + i, ac);
                st4(mnext + c * n + i, make_float4(b.x + h * k.x, b.y + h * k.y, b.z + h * k.z, b.w + h * k.w));
            }
        } else {
            float4 nv[3];
            const float h = a.dt * (1.f / 6.f);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float4 ac = ld4(acc + c * n + i), b = ld4(m0 + c * n + i), k = kv[c];
                nv[c] = make_float4(b.x + h * (ac.x + k.x), b.y + h * (ac.y + k.y), b.z + h * (ac.z + k.z),
                                    b.w + h * (ac.w + k.w));
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float vx = q_get(nv[0], j), vy = q_get(nv[1], j), vz = q_get(nv[2], j);
                const float inv = 1.f / sqrtf(vx * vx + vy * vy + vz * vz);
#pragma unroll
                for (int c = 0; c < 3; c++) q_set(nv[c], j, q_get(nv[c], j) * inv);
            }
#pragma unroll
            for (int c = 0; c < 3; c++) st4(m0 + c * n + i, nv[c]);
        }
    }
}

// RKF45 stage s in 0..5: k_s = f(ms); for s < 5 writes the next stage state
// mnext = m0 + dt sum_{j<=s} a_{s+1,j} k_j; for s = 5 writes the normalised
// 4th-order solution into mnext and folds max |m5 - m4| into *err.
template <typename T>
__global__ void __launch_bounds__(256) rkf45_stage_kernel(LLGArgs<T> a, int s, const T* __restrict__ ms,
                                                          const T* __restrict__ Hd, const T* __restrict__ m0,
                                                          T* __restrict__ kbuf, T* __restrict__ mnext,
                                                          unsigned long long* __restrict__ err_bits)
{
    const size_t n = a.ncell;
    const T dt = a.dt_dev ? (T)*a.dt_dev : a.dt;
    double local_err = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % a.nx);
        const int y = (int)((i / a.nx) % a.ny);
        const int z = (int)(i / ((size_t)a.nx * a.ny));
        T m[3], k[3];
        field_and_rhs(a, ms, Hd, i, x, y, z, m, k);
#pragma unroll
        for (int c = 0; c < 3; c++) kbuf[((size_t)s * 3 + c) * n + i] = k[c];
        if (s < 5) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                T v = m0[c * n + i];
                for (int j = 0; j < s; j++) v += dt * T(RKF_A[s + 1][j]) * kbuf[((size_t)j * 3 + c) * n + i];
                v += dt * T(RKF_A[s + 1][s]) * k[c];
                mnext[c * n + i] = v;
            }
        } else {
            T v4[3];
            double e2 = 0.0;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                T s4 = T(0);
                double d = 0.0;  // m5 - m4 = dt sum_j (b5_j - b4_j) k_j, accumulated in FP64
                for (int j = 0; j < 6; j++) {
                    const T kj = j == 5 ? k[c] : kbuf[((size_t)j * 3 + c) * n + i];
                    s4 += T(RKF_B4[j]) * kj;
                    d += (RKF_B5[j] - RKF_B4[j]) * (double)kj;
                }
                v4[c] = m0[c * n + i] + dt * s4;
                d *= (double)dt;
                e2 += d * d;
            }
            local_err = fmax(local_err, sqrt(e2));
            const T inv = T(1) / sqrt(v4[0] * v4[0] + v4[1] * v4[1] + v4[2] * v4[2]);
#pragma unroll
            for (int c = 0; c < 3; c++) mnext[c * n + i] = v4[c] * inv;
        }
    }
    if (s == 5) {
        // non-negative doubles order like their bit patterns read as unsigned integers
        for (int o = 16; o > 0; o >>= 1) local_err = fmax(local_err, __shfl_xor_sync(0xffffffffu, local_err, o));
        if ((threadIdx.x & 31) == 0) atomicMax(err_bits, (unsigned long long)__double_as_longlong(local_err));
    }
}

__global__ void rkf45_set_dt_kernel(RKFControl* c, double dt, int reset)
{
    c->dt = dt;
    if (reset) {
        c->t = 0.0;
        c->trials = 0ull;
        c->accepted_steps = 0ull;
        c->failed_steps = 0ull;
    }
}

__global__ void rkf45_begin_kernel(RKFControl* c)
{
    c->attempts = 0u;
    c->accepted = 0;
    c->err_bits = 0ull;
}

__global__ void rkf45_control_kernel(RKFControl* c, double tol, double dt_min, double dt_max, int* status,
                                     cudaGraphConditionalHandle loop)
{
    const double err = __longlong_as_double((long long)c->err_bits);
    const double h = c->dt;
    const double fac = err == 0.0 ? 2.0 : fmin(2.0, fmax(0.2, 0.9 * pow(tol / err, 0.2)));
    const double hn = fmin(dt_max, fmax(dt_min, h * fac));
    const bool acc = err <= tol || h <= dt_min;
    const unsigned int tries = c->attempts + 1u;
    c->attempts = tries;
    c->err = err;
    c->trials += 1ull;
    c->err_bits = 0ull;
    c->dt = hn;
    if (acc) {
        c->accepted = 1;
        c->dt_used = h;
        c->t += h;
        c->accepted_steps += 1ull;
    } else if (tries >= RKF_MAX_TRIALS) {
        c->failed_steps += 1ull;
        if (status) atomicCAS(status, 0, -6);  // BORIS_ERR_STEP_CONTROL
    }
    // repeat the trial only while it is rejected and trials remain: the loop
    // ends after at most RKF_MAX_TRIALS passes whatever the error is
    cudaGraphSetConditional(loop, (!acc && tries < RKF_MAX_TRIALS) ? 1u : 0u);
}

template <typename T>
__global__ void rkf45_accept_kernel(const RKFControl* __restrict__ c, const T* __restrict__ trial, T* __restrict__ m,
                                    size_t n)
{
    if (!c->accepted) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m[i] = trial[i];
}

// FP64 energies: E_demag, E_exchange, E_anisotropy, E_Zeeman, E_DMI.
template <typename T>
__global__ void __launch_bounds__(256) energy_kernel(LLGArgs<T> a, const T* __restrict__ m, const T* __restrict__ Hd,
                                                     double* __restrict__ out)
{
    const size_t n = a.ncell;
    double e[5] = {0, 0, 0, 0, 0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % a.nx);
        const int y = (int)((i / a.nx) % a.ny);
        const int z = (int)(i / ((size_t)a.nx * a.ny));
        const double mc[3] = {(double)m[i], (double)m[n + i], (double)m[2 * n + i]};
        double lap[3], w[3];
        // neighbours (or boundary ghosts) in FP64; without DMI the ghost is the cell itself
        ext_exchange_dmi<double>(a, m, i, x, y, z, mc, lap, w);
        const double Ms = a.ms_map ? (double)a.ms_map[i] : (double)a.Ms;
        const double Ku = a.ku_map ? (double)a.ku_map[i] : (double)a.Ku;
        const double me = mc[0] * a.e[0] + mc[1] * a.e[1] + mc[2] * a.e[2];
        double mHd = 0, mHz = 0, mlap = 0, mw = 0;
        for (int c = 0; c < 3; c++) {
            mHd += mc[c] * (double)Hd[c * n + i];
            mHz += mc[c] * ((double)a.Hext[c] + (a.hadd ? (double)a.hadd[c * n + i] : 0.0));
            mlap += mc[c] * lap[c];
            mw += mc[c] * w[c];
        }
        // -(mu0 Ms/2) m.Hex with Hex = (2A/(mu0 Ms)) lap m  ->  -A m.lap m; likewise -D m.w
        e[0] += -0.5 * MU0_D * Ms * mHd;
        e[1] += -(double)a.A * mlap;
        e[2] += Ku * (1.0 - me * me) + (a.extra ? ext_local_energy<double>(a, mc) : 0.0);
        e[3] += -MU0_D * Ms * mHz;
        e[4] += -(double)a.D * mw;
    }
    __shared__ double red[5][8];
    for (int c = 0; c < 5; c++) {
        double v = e[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += red[threadIdx.x][w];
        atomicAdd(out + threadIdx.x, v * a.V);
    }
}

// ---------------------------------------------------------------------------
// Multi-mesh RK4 stage: one launch over all layers' cells (fields concatenated
// in layer order, each SoA [3][nz][ny][nx]); exchange couples neighbours
// inside a layer only (Table 1 exchange with Neumann boundaries per mesh).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void ml_field_and_rhs(const LLGArgs<T>& a, const MLTable& t, const T* __restrict__ ms,
                                                 const T* __restrict__ Hd, size_t idx, size_t vi[3], T m[3], T k[3])
{
    int l = 0;
    while (l + 1 < t.nl && idx >= t.off[l + 1] / 3) l++;
    const size_t base = t.off[l], cell = idx - base / 3;
    const int nx = t.nx[l], ny = t.ny[l], nz = t.nz[l];
    const size_t n = (size_t)nx * ny * nz;
    const int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((size_t)nx * ny));
    for (int c = 0; c < 3; c++) vi[c] = base + c * n + cell;
    m[0] = ms[vi[0]];
    m[1] = ms[vi[1]];
    m[2] = ms[vi[2]];
    T lap[3] = {T(0), T(0), T(0)};
    auto nb = [&](size_t j, T w) {
        lap[0] += w * (ms[vi[0] + j - cell] - m[0]);
        lap[1] += w * (ms[vi[1] + j - cell] - m[1]);
        lap[2] += w * (ms[vi[2] + j - cell] - m[2]);
    };
    const T ihz2 = T(1) / (T(t.hz[l]) * T(t.hz[l]));
    const size_t sy = nx, sz = (size_t)nx * ny;
    if (x > 0) nb(cell - 1, a.ihx2);
    if (x < nx - 1) nb(cell + 1, a.ihx2);
    if (y > 0) nb(cell - sy, a.ihy2);
    if (y < ny - 1) nb(cell + sy, a.ihy2);
    if (z > 0) nb(cell - sz, ihz2);
    if (z < nz - 1) nb(cell + sz, ihz2);
    const T Ms = a.ms_map ? a.ms_map[idx] : a.Ms;
    const T Ku = a.ku_map ? a.ku_map[idx] : a.Ku;
    const T inv = T(1) / (T(MU0_D) * Ms);
    const T cex = T(2) * a.A * inv;
    const T me = m[0] * a.e[0] + m[1] * a.e[1] + m[2] * a.e[2];
    const T can = T(2) * Ku * inv * me;
    T H[3];
#pragma unroll
    for (int c = 0; c < 3; c++) H[c] = Hd[vi[c]] + cex * lap[c] + can * a.e[c] + a.Hext[c];
    if (a.extra) {
        ext_local_field<T>(a, m, Ms, H);
        // surface exchange (Eq. 5): the top plane of layer l with the bottom
        // plane of layer l + 1 where they overlap in-plane, and the reverse;
        // Delta = this cell's z size
        if (a.J1 != T(0) || a.J2 != T(0)) {
            const T cs = inv / T(t.hz[l]);
            auto couple = [&](int lj, int zj) {
                const int xj = x + t.ox[l] - t.ox[lj], yj = y + t.oy[l] - t.oy[lj];
                if (xj < 0 || xj >= t.nx[lj] || yj < 0 || yj >= t.ny[lj]) return;
                const size_t nj = (size_t)t.nx[lj] * t.ny[lj] * t.nz[lj];
                const size_t cj = ((size_t)zj * t.ny[lj] + yj) * t.nx[lj] + xj;
                const T mj[3] = {ms[t.off[lj] + cj], ms[t.off[lj] + nj + cj], ms[t.off[lj] + 2 * nj + cj]};
                const T d = m[0] * mj[0] + m[1] * mj[1] + m[2] * mj[2];
                const T f = cs * (a.J1 + T(2) * a.J2 * d);
#pragma unroll
                for (int c = 0; c < 3; c++) H[c] += f * mj[c];
            };
            if (z == nz - 1 && l + 1 < t.nl) couple(l + 1, 0);
            if (z == 0 && l > 0) couple(l - 1, t.nz[l - 1] - 1);
        }
    }
    const T mxH[3] = {m[1] * H[2] - m[2] * H[1], m[2] * H[0] - m[0] * H[2], m[0] * H[1] - m[1] * H[0]};
    const T mmH[3] = {m[1] * mxH[2] - m[2] * mxH[1], m[2] * mxH[0] - m[0] * mxH[2], m[0] * mxH[1] - m[1] * mxH[0]};
#pragma unroll
    for (int c = 0; c < 3; c++) k[c] = -a.gp * (mxH[c] + a.alpha * mmH[c]);
}

__global__ void __launch_bounds__(256) rk4_stage_ml_kernel(LLGArgs<float> a, MLTable t, int s,
                                                           const float* __restrict__ ms, const float* __restrict__ Hd,
                                                           float* __restrict__ m0, float* __restrict__ acc,
                                                           float* __restrict__ mnext)
{
    const size_t n = a.ncell;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        size_t vi[3];
        float m[3], k[3];
        ml_field_and_rhs(a, t, ms, Hd, i, vi, m, k);
        if (s == 0) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                acc[vi[c]] = k[c];
                mnext[vi[c]] = m[c] + 0.5f * a.dt * k[c];
            }
        } else if (s < 3) {
            const float cdt = s == 1 ? 0.5f * a.dt : a.dt;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                acc[vi[c]] += 2.f * k[c];
                mnext[vi[c]] = m0[vi[c]] + cdt * k[c];
            }
        } else {
            float v[3];
#pragma unroll
            for (int c = 0; c < 3; c++) v[c] = m0[vi[c]] + a.dt * (1.f / 6.f) * (acc[vi[c]] + k[c]);
            const float inv = rsqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
            for (int c = 0; c < 3; c++) m0[vi[c]] = v[c] * inv;
        }
    }
}

cudaError_t launch_rk4_stage_ml(const LLGArgs<float>& a, const MLTable& t, int s, const float* ms, const float* Hd,
                                float* m0, float* acc, float* mnext, cudaStream_t st)
{
    size_t b = (a.ncell + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    rk4_stage_ml_kernel<<<(int)(b > 0 ? b : 1), 256, 0, st>>>(a, t, s, ms, Hd, m0, acc, mnext);
    return cudaGetLastError();
}

static int grid_for_words(int n)
{
    const int b = (n + 255) / 256;
    return b < 152 * 8 ? b : 152 * 8;
}

__global__ void thermal_advance_kernel(unsigned long long* step) { *step += 1ull; }
__global__ void thermal_set_kernel(unsigned long long* step, unsigned long long v) { *step = v; }

cudaError_t launch_thermal_advance(unsigned long long* step, cudaStream_t st)
{
    thermal_advance_kernel<<<1, 1, 0, st>>>(step);
    return cudaGetLastError();
}

cudaError_t launch_thermal_set(unsigned long long* step, unsigned long long v, cudaStream_t st)
{
    thermal_set_kernel<<<1, 1, 0, st>>>(step, v);
    return cudaGetLastError();
}

// The stage kernels' generator on caller-given counters and keys: ctr [n][4],
// key [n][2], out [n][4] 32-bit words.
__global__ void philox_words_kernel(const unsigned int* __restrict__ ctr, const unsigned int* __restrict__ key,
                                    unsigned int* __restrict__ out, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned int c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
        philox4x32_10(c, key[2 * i], key[2 * i + 1]);
#pragma unroll
        for (int j = 0; j < 4; j++) out[4 * i + j] = c[j];
    }
}

cudaError_t launch_philox_words(const unsigned int* ctr, const unsigned int* key, unsigned int* out, int n,
                                cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    philox_words_kernel<<<grid_for_words(n), 256, 0, st>>>(ctr, key, out, n);
    return cudaGetLastError();
}

static int grid_for(size_t n)
{
    size_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b > 0 ? b : 1);
}

template <typename T>
cudaError_t launch_rk4_stage(const LLGArgs<T>& a, int s, const T* ms, const T* Hd, T* m0, T* acc, T* mnext,
                             cudaStream_t st)
{
    if constexpr (sizeof(T) == 4) {
        if (a.nx % 4 == 0 && !a.extra) {
            if (a.pbc) rk4_stage_quad_kernel<true><<<grid_for(a.ncell / 4), 256, 0, st>>>(a, s, ms, Hd, m0, acc, mnext);
            else rk4_stage_quad_kernel<false><<<grid_for(a.ncell / 4), 256, 0, st>>>(a, s, ms, Hd, m0, acc, mnext);
            return cudaGetLastError();
        }
    }
    rk4_stage_kernel<T><<<grid_for(a.ncell), 256, 0, st>>>(a, s, ms, Hd, m0, acc, mnext);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rkf45_stage(const LLGArgs<T>& a, int s, const T* ms, const T* Hd, const T* m0, T* kbuf, T* mnext,
                               unsigned long long* err_bits, cudaStream_t st)
{
    rkf45_stage_kernel<T><<<grid_for(a.ncell), 256, 0, st>>>(a, s, ms, Hd, m0, kbuf, mnext, err_bits);
    return cudaGetLastError();
}

cudaError_t launch_rkf45_set_dt(RKFControl* c, double dt, bool reset_counters, cudaStream_t st)
{
    rkf45_set_dt_kernel<<<1, 1, 0, st>>>(c, dt, reset_counters ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_rkf45_begin(RKFControl* c, cudaStream_t st)
{
    rkf45_begin_kernel<<<1, 1, 0, st>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_rkf45_control(RKFControl* c, double tol, double dt_min, double dt_max, int* status,
                                 cudaGraphConditionalHandle loop, cudaStream_t st)
{
    rkf45_control_kernel<<<1, 1, 0, st>>>(c, tol, dt_min, dt_max, status, loop);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rkf45_accept(const RKFControl* c, const T* trial, T* m, size_t n, cudaStream_t st)
{
    rkf45_accept_kernel<T><<<grid_for(n), 256, 0, st>>>(c, trial, m, n);
    return cudaGetLastError();
}
template cudaError_t launch_rkf45_accept<float>(const RKFControl*, const float*, float*, size_t, cudaStream_t);
template cudaError_t launch_rkf45_accept<double>(const RKFControl*, const double*, double*, size_t, cudaStream_t);

template <typename T>
cudaError_t launch_energy(const LLGArgs<T>& a, const T* m, const T* Hd, double* out, cudaStream_t st)
{
    energy_kernel<T><<<grid_for(a.ncell), 256, 0, st>>>(a, m, Hd, out);
    return cudaGetLastError();
}

template cudaError_t launch_rk4_stage<float>(const LLGArgs<float>&, int, const float*, const float*, float*, float*,
                                             float*, cudaStream_t);
template cudaError_t launch_rk4_stage<double>(const LLGArgs<double>&, int, const double*, const double*, double*,
                                              double*, double*, cudaStream_t);
template cudaError_t launch_rkf45_stage<float>(const LLGArgs<float>&, int, const float*, const float*, const float*,
                                               float*, float*, unsigned long long*, cudaStream_t);
template cudaError_t launch_rkf45_stage<double>(const LLGArgs<double>&, int, const double*, const double*,
                                                const double*, double*, double*, unsigned long long*, cudaStream_t);
template cudaError_t launch_energy<float>(const LLGArgs<float>&, const float*, const float*, double*, cudaStream_t);
template cudaError_t launch_energy<double>(const LLGArgs<double>&, const double*, const double*, double*,
                                           cudaStream_t);

}  // namespace boris
