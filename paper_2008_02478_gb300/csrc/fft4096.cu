// Transforms of length 4096 (meshes of 1025..2048 cells along the axis), built
// on the warp-held length-1024 transform of warp_fft.cuh (w = exp(-2 pi i /
// 4096) below).
//
// y forward of a complex line of ny <= 2048 values zero-padded to 4096, split
// by output residue r = k mod 4 (one warp each):
//   Y[4k + r] = FFT_1024( w^(r m) (x[m] + (-i)^r x[m + 1024]) )[k].
// y inverse cropped to n < 2048: with u_r = IFFT_1024(Y[4k + r]) and
// v_r[m] = w^(-r m) u_r[m],
//   x[m] = v_0 + v_1 + v_2 + v_3,   x[m + 1024] = (v_0 - v_2) + i (v_1 - v_3),
// the four residues summed through shared memory.
//
// x real-to-complex of a real row of nx <= 2048 samples: the half-length
// sequence z[n] = x[2n] + i x[2n+1] (n < 1024, zero above) has the length-2048
// transform Z[2k] = FFT_1024(z)[k], Z[2k+1] = FFT_1024(z[n] w_2048^n)[k] (two
// warps), and X[k] = E[k] + w^k O[k] (k = 0..2048) with E[k] = (Z[k] +
// conj Z[2048-k]) / 2, O[k] = (Z[k] - conj Z[2048-k]) / (2i).
// x complex-to-real (unscaled, DC and Nyquist bins taken as real): Z'[k] =
// X[k] + conj X[2048-k] + i (X[k] - conj X[2048-k]) w^-k, z = IFFT_2048(Z')
// cropped to n < 1024 as IFFT_1024(Z'_even)[n] + w_2048^-n IFFT_1024(Z'_odd)[n],
// and x[2n] = Re z[n], x[2n+1] = Im z[n].
#include <type_traits>

#include "boris_internal.cuh"
#include "warp_fft.cuh"

namespace boris {

namespace {

constexpr int TWR = 1024;    // the row twiddle table only (no slot layout here)
constexpr int R1025 = 1025;  // per-warp region stride (complex)
// y passes: region stride 1028 (4 mod 16), so the interleaved view
// q[(j & 3) R1028 + (j >> 2)] of 16 consecutive j falls in 16 distinct bank pairs
constexpr int R1028 = 1028;
constexpr int XROWS = 4;     // x passes: rows per CTA (two warps each)
constexpr int YLINES = 2;    // y passes: lines per CTA (four warps each)

// Twiddles w^(32 e + lane') are formed as w_128^e (a literal or a 128-entry
// shared table) times a per-lane value read once from the plan's table.

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    y_fwd_4096_kernel(Geometry g, const typename Cx<T>::t* __restrict__ X, typename Cx<T>::t* __restrict__ Y,
                      const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* w128s = tws + TWR;  // w^(32 e) = w_128^e
    C* reg = w128s + 128;  // [8 warps][R1028]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lines = 3 * g.nz, ny = g.ny;
    const int kx = blockIdx.y, line = blockIdx.x * YLINES + (warp >> 2), r = warp & 3;
    const int sh = g.lglmax - 12;
    load_tw1024(tws, tw_g, g.lmax);
    if (threadIdx.x < 128) w128s[threadIdx.x] = tw_g[(32 * threadIdx.x) << sh];
    __syncthreads();
    const bool act = line < lines;
    C* mine = reg + warp * R1028;
    if (act) {
        const C* src = X + ((size_t)kx * lines + line) * ny;
        const C wlr = tw_g[(r * lane) << sh];  // w^(r lane)
        // (-i)^r = (cr, ci)
        const T cr = r == 0 ? T(1) : r == 2 ? T(-1) : T(0);
        const T ci = r == 1 ? T(-1) : r == 3 ? T(1) : T(0);
        C v[32];
#pragma unroll
        for (int a = 0; a < 32; a++) {
            const int m = 32 * a + lane;
            const C lo = m < ny ? src[m] : C{T(0), T(0)};
            const C hi = m + 1024 < ny ? src[m + 1024] : C{T(0), T(0)};
            const C s{lo.x + cr * hi.x - ci * hi.y, lo.y + cr * hi.y + ci * hi.x};
            v[a] = c_mul(s, c_mul(w128s[(r * a) & 127], wlr));
        }
        warp_fft1024_fwd(v, mine, tws);
#pragma unroll
        for (int pos = 0; pos < 32; pos++) mine[lane + 32 * brev5(pos)] = v[pos];  // Y[4 k + r] at k
    }
    __syncthreads();  // all four residues of every line in shared memory
    if (!act) return;
    // warp r stores Y[j], j = 1024 r .. 1024 r + 1023, in 256-byte rows
    const C* q = reg + (warp & ~3) * R1028;
    C* dst = Y + ((size_t)kx * lines + line) * 4096;
#pragma unroll 8
    for (int i = 0; i < 32; i++) {
        const int j = 1024 * r + 32 * i + lane;
        dst[j] = q[(j & 3) * R1028 + (j >> 2)];
    }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    y_inv_4096_kernel(Geometry g, const typename Cx<T>::t* __restrict__ Y, typename Cx<T>::t* __restrict__ X,
                      const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* w128s = tws + TWR;
    C* reg = w128s + 128;  // [8 warps][R1028]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lines = 3 * g.nz, ny = g.ny;
    const int kx = blockIdx.y, line = blockIdx.x * YLINES + (warp >> 2), r = warp & 3;
    const int sh = g.lglmax - 12;
    load_tw1024(tws, tw_g, g.lmax);
    if (threadIdx.x < 128) w128s[threadIdx.x] = tw_g[(32 * threadIdx.x) << sh];
    const bool act = line < lines;
    C* q = reg + (warp & ~3) * R1028;  // the line's four regions
    if (act) {
        // warp r loads Y[j], j = 1024 r .. 1024 r + 1023, in 256-byte rows; residue
        // j & 3 goes to region j & 3 at j >> 2
        const C* src = Y + ((size_t)kx * lines + line) * 4096;
#pragma unroll 8
        for (int i = 0; i < 32; i++) {
            const int j = 1024 * r + 32 * i + lane;
            q[(j & 3) * R1028 + (j >> 2)] = src[j];
        }
    }
    __syncthreads();  // twiddles and every line's residues staged
    C* mine = reg + warp * R1028;
    C v[32];
    if (act) {
#pragma unroll
        for (int d = 0; d < 32; d++) v[brev5(d)] = mine[lane + 32 * d];
        __syncwarp();
        warp_fft1024_inv(v, mine, tws);
        const C wlr = tw_g[(r * lane) << sh];
#pragma unroll
        for (int a = 0; a < 32; a++) mine[32 * a + lane] = c_mulc(v[a], c_mul(w128s[(r * a) & 127], wlr));
    }
    __syncthreads();  // all four residues of every line published
    if (!act) return;
    C* dst = X + ((size_t)kx * lines + line) * ny;
    // warp r stores m = 256 r + 32 i + lane and m + 1024
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int m = 256 * r + 32 * i + lane;
        const C v0 = q[m], v1 = q[R1028 + m], v2 = q[2 * R1028 + m], v3 = q[3 * R1028 + m];
        const C s02 = c_add(v0, v2), d02 = c_sub(v0, v2), s13 = c_add(v1, v3), d13 = c_sub(v1, v3);
        if (m < ny) dst[m] = c_add(s02, s13);
        if (m + 1024 < ny) dst[m + 1024] = C{d02.x - d13.y, d02.y + d13.x};
    }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    x_r2c_4096_kernel(Geometry g, const T* __restrict__ M, const T* __restrict__ ms_map, T ms_scale,
                      typename Cx<T>::t* __restrict__ X, const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* wq = tws + TWR;  // w^(32 q) = w_128^q, q <= 64
    C* wr = wq + 72;    // w^e, e < 32
    C* reg = wr + 32;   // [8 warps][R1025]: warp 2 t + p holds Z[2 k + p] of row t at k
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0 = blockIdx.x * XROWS, z = blockIdx.y, c = blockIdx.z;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int sh = g.lglmax - 12;
    load_tw1024(tws, tw_g, g.lmax);
    if (threadIdx.x < 65) wq[threadIdx.x] = tw_g[(32 * threadIdx.x) << sh];
    if (threadIdx.x < 32) wr[threadIdx.x] = tw_g[threadIdx.x << sh];
    __syncthreads();
    const int t = warp >> 1, par = warp & 1;
    const int y = y0 + t;
    const bool oky = y < ny;
    const size_t ncell = (size_t)nx * ny * nz;
    const T* row = M + c * ncell + ((size_t)z * ny + y) * nx;
    const T* mrow = ms_map ? ms_map + ((size_t)z * ny + y) * nx : nullptr;
    const C wl2 = tw_g[(2 * lane) << sh];  // w_2048^lane
    C v[32];
#pragma unroll
    for (int a = 0; a < 32; a++) {
        const int i0 = 2 * (32 * a + lane), i1 = i0 + 1;  // z[n] = x[2n] + i x[2n+1], n < 1024
        const bool in0 = oky && i0 < nx, in1 = oky && i1 < nx;
        T x0 = in0 ? row[i0] : T(0), x1 = in1 ? row[i1] : T(0);
        if (mrow) {
            x0 *= in0 ? mrow[i0] : T(0);
            x1 *= in1 ? mrow[i1] : T(0);
        } else {
            x0 *= ms_scale;
            x1 *= ms_scale;
        }
        v[a] = C{x0, x1};
        if (par) v[a] = c_mul(v[a], a == 0 ? wl2 : c_mul(w128lit<C>(2 * a), wl2));  // z[n] w_2048^n
    }
    C* mine = reg + warp * R1025;
    warp_fft1024_fwd(v, mine, tws);
#pragma unroll
    for (int pos = 0; pos < 32; pos++) mine[lane + 32 * brev5(pos)] = v[pos];
    __syncthreads();
    // X[k][c][z][y0 + t], k = 0..2048: 4 consecutive y per k
    for (int i = threadIdx.x; i < 2049 * XROWS; i += blockDim.x) {
        const int tt = i & (XROWS - 1), k = i >> 2;
        const int yy = y0 + tt;
        if (yy >= ny) continue;
        const C* Zr = reg + 2 * tt * R1025;  // Z[j] at Zr[(j & 1) R1025 + (j >> 1)]
        const int j1 = k & 2047, j2 = (2048 - k) & 2047;
        const C zk = Zr[(j1 & 1) * R1025 + (j1 >> 1)], zm = Zr[(j2 & 1) * R1025 + (j2 >> 1)];
        const C E{T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y)};
        const C O{T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x)};
        const C w = c_mul(wq[k >> 5], wr[k & 31]);
        X[(((size_t)k * 3 + c) * nz + z) * ny + yy] = c_add(E, c_mul(w, O));
    }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    x_c2r_4096_kernel(Geometry g, const typename Cx<T>::t* __restrict__ X, T* __restrict__ H,
                      const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    // the 2049 x 4 half-spectrum block, row t's even bins at S[2t][k/2] and odd
    // bins at S[2t + 1][k/2] (stride R1025); afterwards the warps' regions
    C* S = tws + TWR;
    C* reg = S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0 = blockIdx.x * XROWS, z = blockIdx.y, c = blockIdx.z;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int sh = g.lglmax - 12;
    load_tw1024(tws, tw_g, g.lmax);
    const size_t plane = (size_t)3 * nz * ny;
    const size_t col0 = ((size_t)c * nz + z) * ny + y0;
    staged_loop<256, C>(
        2049 * XROWS,
        [&](int i) {
            const int k = i >> 2, t = i & (XROWS - 1);
            return y0 + t < ny ? X[(size_t)k * plane + col0 + t] : C{T(0), T(0)};
        },
        [&](int i, C a) {
            const int k = i >> 2, t = i & (XROWS - 1);
            S[(2 * t + (k & 1)) * R1025 + (k >> 1)] = a;
        });
    __syncthreads();
    const int t = warp >> 1, par = warp & 1;
    const C* Se = S + 2 * t * R1025;  // even bins of row t
    const C* Sp = Se + par * R1025;   // this warp's parity
    const C wk = tw_g[(2 * lane + par) << sh];  // w^(2 lane + par)
    C v[32];
#pragma unroll
    for (int d = 0; d < 32; d++) {
        const int kk = lane + 32 * d;  // k = 2 kk + par, 2048 - k = 2 (1024 - kk - par) + par
        C Xk = Sp[kk];
        C Xm = Sp[1024 - kk - par];
        if (d == 0 && lane == 0 && par == 0) {  // DC and Nyquist bins of a real signal are real
            Xk.y = T(0);
            Xm.y = T(0);
        }
        const C E{Xk.x + Xm.x, Xk.y - Xm.y};
        const C O = c_mulc(C{Xk.x - Xm.x, Xk.y + Xm.y}, d == 0 ? wk : c_mul(w128lit<C>(2 * d), wk));
        v[brev5(d)] = C{E.x - O.y, E.y + O.x};
    }
    __syncthreads();  // the block is consumed: its bytes become the transpose regions
    C* mine = reg + warp * R1025;
    warp_fft1024_inv(v, mine, tws);
    if (par) {
        const C wl2 = tw_g[(2 * lane) << sh];  // w_2048^lane
#pragma unroll
        for (int a = 0; a < 32; a++) v[a] = c_mulc(v[a], a == 0 ? wl2 : c_mul(w128lit<C>(2 * a), wl2));
    }
#pragma unroll
    for (int a = 0; a < 32; a++) mine[32 * a + lane] = v[a];
    __syncthreads();  // both halves of every row published
    const int y = y0 + t;
    if (y >= ny) return;
    const C* other = reg + (warp ^ 1) * R1025;
    const size_t ncell = (size_t)nx * ny * nz;
    T* row = H + c * ncell + ((size_t)z * ny + y) * nx;
    // the even warp stores n < 512, the odd one 512 <= n < 1024 (x[2n], x[2n+1])
    auto store = [&](auto first) {
#pragma unroll
        for (int a = first; a < first + 16; a++) {
            const int n = 32 * a + lane;
            const C s = c_add(v[a], other[n]);
            if (2 * n < nx) row[2 * n] = s.x;
            if (2 * n + 1 < nx) row[2 * n + 1] = s.y;
        }
    };
    if (par) store(std::integral_constant<int, 16>{});
    else store(std::integral_constant<int, 0>{});
}

template <typename T>
size_t smem_y_4096()
{
    return ((size_t)TWR + 128 + 8 * (size_t)R1028) * sizeof(typename Cx<T>::t);
}
template <typename T>
size_t smem_x_r2c_4096()
{
    return ((size_t)TWR + 104 + 8 * (size_t)R1025) * sizeof(typename Cx<T>::t);
}
template <typename T>
size_t smem_x_c2r_4096()
{
    return ((size_t)TWR + 8 * (size_t)R1025) * sizeof(typename Cx<T>::t);
}

}  // namespace

template <typename T>
bool x4096_ok(const Geometry& g, int max_smem)
{
    return g.px == 4096 && g.nx <= 2048 && g.lglmax >= 12 && smem_x_r2c_4096<T>() <= (size_t)max_smem &&
           smem_x_c2r_4096<T>() <= (size_t)max_smem;
}
template <typename T>
bool y4096_ok(const Geometry& g, int max_smem)
{
    return g.py == 4096 && g.ny <= 2048 && g.lglmax >= 12 && smem_y_4096<T>() <= (size_t)max_smem;
}

template <typename T>
cudaError_t launch_x_r2c_4096(const Geometry& g, const T* M, const T* ms_map, T ms_scale, typename Cx<T>::t* X,
                              const typename Cx<T>::t* tw, cudaStream_t st)
{
    const size_t smem = smem_x_r2c_4096<T>();
    cudaError_t e = cudaFuncSetAttribute(x_r2c_4096_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    x_r2c_4096_kernel<T><<<dim3((g.ny + XROWS - 1) / XROWS, g.nz, 3), 256, smem, st>>>(g, M, ms_map, ms_scale, X, tw);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_x_c2r_4096(const Geometry& g, const typename Cx<T>::t* X, T* H, const typename Cx<T>::t* tw,
                              cudaStream_t st)
{
    const size_t smem = smem_x_c2r_4096<T>();
    cudaError_t e = cudaFuncSetAttribute(x_c2r_4096_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    x_c2r_4096_kernel<T><<<dim3((g.ny + XROWS - 1) / XROWS, g.nz, 3), 256, smem, st>>>(g, X, H, tw);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_y_4096(const Geometry& g, typename Cx<T>::t* X, typename Cx<T>::t* Y, const typename Cx<T>::t* tw,
                          cudaStream_t st, bool forward)
{
    const size_t smem = smem_y_4096<T>();
    const dim3 grid((3 * g.nz + YLINES - 1) / YLINES, g.nkx);
    if (forward) {
        cudaError_t e = cudaFuncSetAttribute(y_fwd_4096_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        y_fwd_4096_kernel<T><<<grid, 256, smem, st>>>(g, X, Y, tw);
    } else {
        cudaError_t e = cudaFuncSetAttribute(y_inv_4096_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        y_inv_4096_kernel<T><<<grid, 256, smem, st>>>(g, Y, X, tw);
    }
    return cudaGetLastError();
}

#define FFT4096_INST(T)                                                                                           \
    template bool x4096_ok<T>(const Geometry&, int);                                                             \
    template bool y4096_ok<T>(const Geometry&, int);                                                             \
    template cudaError_t launch_x_r2c_4096<T>(const Geometry&, const T*, const T*, T, Cx<T>::t*, const Cx<T>::t*, \
                                              cudaStream_t);                                                     \
    template cudaError_t launch_x_c2r_4096<T>(const Geometry&, const Cx<T>::t*, T*, const Cx<T>::t*, cudaStream_t); \
    template cudaError_t launch_y_4096<T>(const Geometry&, Cx<T>::t*, Cx<T>::t*, const Cx<T>::t*, cudaStream_t, bool);
FFT4096_INST(float)
FFT4096_INST(double)

}  // namespace boris
