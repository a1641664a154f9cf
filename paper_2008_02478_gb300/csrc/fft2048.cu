// Transforms of length 2048 (meshes of 513..1024 cells along the axis), built
// on the warp-held length-1024 transform of warp_fft.cuh (w = exp(-2 pi i /
// 2048) below).
//
// x real-to-complex: one real row of nx <= 1024 samples, zero-padded to 2048,
// per warp, as the half-length sequence z[n] = x[2n] + i x[2n+1] (n < 1024).
// With Z = FFT_1024(z), E[k] = (Z[k] + conj Z[1024-k]) / 2 and
// O[k] = (Z[k] - conj Z[1024-k]) / (2i) are the transforms of the even and
// odd samples, and X[k] = E[k] + w^k O[k] for k = 0..1024.
//
// x complex-to-real (unscaled inverse, DC and Nyquist bins taken as real):
// E'[k] = X[k] + conj X[1024-k], O'[k] = (X[k] - conj X[1024-k]) w^-k and
// z = IFFT_1024(E' + i O') give x[2n] = Re z[n], x[2n+1] = Im z[n].
//
// y forward of a complex line of ny <= 1024 values zero-padded to 2048: the
// even outputs are FFT_1024(x), the odd ones FFT_1024(x[n] w^n); one warp each.
//
// y inverse cropped to n < 1024: x[n] = IFFT_1024(Y_even)[n] + w^-n
// IFFT_1024(Y_odd)[n]; one warp each, the two halves summed through shared
// memory.
//
// The twiddle w^(32 a + lane) of a compile-time a is w_128^(2a) (a literal)
// times the lane's w^lane (one register).
#include <type_traits>

#include "boris_internal.cuh"
#include "warp_fft.cuh"

namespace boris {

namespace {

constexpr int R1025 = 1025;  // per-warp region stride (complex)
// y passes: region stride 1032 (8 mod 16), so the interleaved view
// q[(j & 1) R1032 + (j >> 1)] of 16 consecutive j falls in 16 distinct bank pairs
constexpr int R1032 = 1032;
constexpr int XROWS = 8;     // x passes: rows per CTA (one per warp)
constexpr int YLINES = 4;    // y passes: lines per CTA (two warps each)

template <typename C>
__device__ __forceinline__ C w2048_at(int a, C wl)  // w^(32 a + lane), a < 64 known at compile time
{
    return a == 0 ? wl : c_mul(w128lit<C>(2 * a), wl);
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    x_r2c_2048_kernel(Geometry g, const T* __restrict__ M, const T* __restrict__ ms_map, T ms_scale,
                      typename Cx<T>::t* __restrict__ X, const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* wq = tws + TW1024_SLOTS;  // w^(32 q), q <= 32
    C* wr = wq + 40;             // w^r, r < 32
    C* reg = wr + 32;            // [XROWS][R1025]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0 = blockIdx.x * XROWS, z = blockIdx.y, c = blockIdx.z;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int sh = g.lglmax - 11;
    load_tw1024(tws, tw_g, g.lmax);
    if (threadIdx.x < 33) wq[threadIdx.x] = tw_g[(32 * threadIdx.x) << sh];
    if (threadIdx.x < 32) wr[threadIdx.x] = tw_g[threadIdx.x << sh];
    __syncthreads();
    const int y = y0 + warp;
    const bool oky = y < ny;
    const size_t ncell = (size_t)nx * ny * nz;
    const T* row = M + c * ncell + ((size_t)z * ny + y) * nx;
    const T* mrow = ms_map ? ms_map + ((size_t)z * ny + y) * nx : nullptr;
    C v[32];
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int i0 = 2 * (32 * a + lane), i1 = i0 + 1;  // samples 2n, 2n + 1 (n < 512: 2n + 1 < 1024)
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
    }
#pragma unroll
    for (int a = 16; a < 32; a++) v[a] = C{T(0), T(0)};
    C* mine = reg + warp * R1025;
    warp_fft1024_fwd(v, mine, tws);
#pragma unroll
    for (int pos = 0; pos < 32; pos++) mine[lane + 32 * brev5(pos)] = v[pos];
    __syncthreads();
    // X[k][c][z][y0 + t], k = 0..1024: 8 consecutive y per k
    for (int i = threadIdx.x; i < 1025 * XROWS; i += blockDim.x) {
        const int t = i & (XROWS - 1), k = i >> 3;
        const int yy = y0 + t;
        if (yy >= ny) continue;
        const C* line = reg + t * R1025;
        const C zk = line[k & 1023], zm = line[(1024 - k) & 1023];
        const C E{T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y)};
        const C O{T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x)};
        const C w = c_mul(wq[k >> 5], wr[k & 31]);
        X[(((size_t)k * 3 + c) * nz + z) * ny + yy] = c_add(E, c_mul(w, O));
    }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    x_c2r_2048_kernel(Geometry g, const typename Cx<T>::t* __restrict__ X, T* __restrict__ H,
                      const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    // the 1025 x 8 half-spectrum block: row k holds column t at t ^ ((k >> 1) & 7),
    // so 16 consecutive rows of one column fall in 16 distinct bank pairs;
    // afterwards the same bytes are the warps' transpose regions
    C* S = tws + TW1024_SLOTS;
    C* reg = S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0 = blockIdx.x * XROWS, z = blockIdx.y, c = blockIdx.z;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    load_tw1024(tws, tw_g, g.lmax);
    const size_t plane = (size_t)3 * nz * ny;
    const size_t col0 = ((size_t)c * nz + z) * ny + y0;
    staged_loop<256, C>(
        1025 * XROWS,
        [&](int i) {
            const int k = i >> 3, t = i & (XROWS - 1);
            return y0 + t < ny ? X[(size_t)k * plane + col0 + t] : C{T(0), T(0)};
        },
        [&](int i, C a) {
            const int k = i >> 3, t = i & (XROWS - 1);
            S[k * XROWS + (t ^ ((k >> 1) & 7))] = a;
        });
    __syncthreads();
    const C wl = tw_g[lane << (g.lglmax - 11)];
    const int t = warp;
    C v[32];
#pragma unroll
    for (int d = 0; d < 32; d++) {
        const int k = lane + 32 * d, km = 1024 - k;
        C Xk = S[k * XROWS + (t ^ ((k >> 1) & 7))];
        C Xm = S[km * XROWS + (t ^ ((km >> 1) & 7))];
        if (d == 0 && lane == 0) {  // DC and Nyquist bins of a real signal are real
            Xk.y = T(0);
            Xm.y = T(0);
        }
        const C E{Xk.x + Xm.x, Xk.y - Xm.y};
        const C O = c_mulc(C{Xk.x - Xm.x, Xk.y + Xm.y}, w2048_at(d, wl));
        v[brev5(d)] = C{E.x - O.y, E.y + O.x};
    }
    __syncthreads();  // the block is consumed: its bytes become the transpose regions
    warp_fft1024_inv(v, reg + warp * R1025, tws);
    const int y = y0 + warp;
    if (y >= ny) return;
    const size_t ncell = (size_t)nx * ny * nz;
    T* row = H + c * ncell + ((size_t)z * ny + y) * nx;
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int i0 = 2 * (32 * a + lane);
        if (i0 < nx) row[i0] = v[a].x;
        if (i0 + 1 < nx) row[i0 + 1] = v[a].y;
    }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    y_fwd_2048_kernel(Geometry g, const typename Cx<T>::t* __restrict__ X, typename Cx<T>::t* __restrict__ Y,
                      const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* reg = tws + TW1024_SLOTS;  // [8 warps][R1032]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lines = 3 * g.nz, ny = g.ny;
    const int kx = blockIdx.y, line = blockIdx.x * YLINES + (warp >> 1), par = warp & 1;
    load_tw1024(tws, tw_g, g.lmax);
    __syncthreads();
    const bool act = line < lines;
    C* mine = reg + warp * R1032;
    if (act) {
        const C* src = X + ((size_t)kx * lines + line) * ny;
        C v[32];
#pragma unroll
        for (int a = 0; a < 32; a++) {
            const int y = 32 * a + lane;
            v[a] = y < ny ? src[y] : C{T(0), T(0)};
        }
        if (par) {
            const C wl = tw_g[lane << (g.lglmax - 11)];
#pragma unroll
            for (int a = 0; a < 32; a++) v[a] = c_mul(v[a], w2048_at(a, wl));
        }
        warp_fft1024_fwd(v, mine, tws);
#pragma unroll
        for (int pos = 0; pos < 32; pos++) mine[lane + 32 * brev5(pos)] = v[pos];  // Y[2 k + par] at k
    }
    __syncthreads();  // both halves of every line in shared memory
    if (!act) return;
    // warp par stores Y[j], j = 1024 par .. 1024 par + 1023, in 256-byte rows
    const C* q = reg + (warp & ~1) * R1032;
    C* dst = Y + ((size_t)kx * lines + line) * 2048;
#pragma unroll 8
    for (int i = 0; i < 32; i++) {
        const int j = 1024 * par + 32 * i + lane;
        dst[j] = q[(j & 1) * R1032 + (j >> 1)];
    }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    y_inv_2048_kernel(Geometry g, const typename Cx<T>::t* __restrict__ Y, typename Cx<T>::t* __restrict__ X,
                      const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* reg = tws + TW1024_SLOTS;  // [8 warps][R1032]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lines = 3 * g.nz, ny = g.ny;
    const int kx = blockIdx.y, line = blockIdx.x * YLINES + (warp >> 1), par = warp & 1;
    load_tw1024(tws, tw_g, g.lmax);
    const bool act = line < lines;
    C* q = reg + (warp & ~1) * R1032;  // the line's two regions
    if (act) {
        // warp par loads Y[j], j = 1024 par .. 1024 par + 1023, in 256-byte rows;
        // parity j & 1 goes to region j & 1 at j >> 1
        const C* src = Y + ((size_t)kx * lines + line) * 2048;
#pragma unroll 8
        for (int i = 0; i < 32; i++) {
            const int j = 1024 * par + 32 * i + lane;
            q[(j & 1) * R1032 + (j >> 1)] = src[j];
        }
    }
    __syncthreads();  // twiddles and both halves of every line staged
    C* mine = reg + warp * R1032;
    C v[32];
    if (act) {
#pragma unroll
        for (int d = 0; d < 32; d++) v[brev5(d)] = mine[lane + 32 * d];
        __syncwarp();
        warp_fft1024_inv(v, mine, tws);
        if (par) {
            const C wl = tw_g[lane << (g.lglmax - 11)];
#pragma unroll
            for (int a = 0; a < 32; a++) v[a] = c_mulc(v[a], w2048_at(a, wl));
        }
#pragma unroll
        for (int a = 0; a < 32; a++) mine[32 * a + lane] = v[a];
    }
    __syncthreads();  // both halves of every line published
    if (!act) return;
    const C* other = reg + (warp ^ 1) * R1032;
    C* dst = X + ((size_t)kx * lines + line) * ny;
    // the even warp stores n < 512, the odd one 512 <= n < 1024
    auto store = [&](auto first) {
#pragma unroll
        for (int a = first; a < first + 16; a++) {
            const int n = 32 * a + lane;
            if (n < ny) dst[n] = c_add(v[a], other[n]);
        }
    };
    if (par) store(std::integral_constant<int, 16>{});
    else store(std::integral_constant<int, 0>{});
}

template <typename T>
size_t smem_x_r2c_2048()
{
    return ((size_t)TW1024_SLOTS + 72 + (size_t)XROWS * R1025) * sizeof(typename Cx<T>::t);
}
template <typename T>
size_t smem_x_c2r_2048()
{
    return ((size_t)TW1024_SLOTS + (size_t)1025 * XROWS) * sizeof(typename Cx<T>::t);
}
template <typename T>
size_t smem_y_2048()
{
    return ((size_t)TW1024_SLOTS + 8 * (size_t)R1032) * sizeof(typename Cx<T>::t);
}

}  // namespace

template <typename T>
bool x2048_ok(const Geometry& g, int max_smem)
{
    return g.px == 2048 && g.nx <= 1024 && g.lglmax >= 11 && smem_x_r2c_2048<T>() <= (size_t)max_smem &&
           smem_x_c2r_2048<T>() <= (size_t)max_smem;
}
template <typename T>
bool y2048_ok(const Geometry& g, int max_smem)
{
    return g.py == 2048 && g.ny <= 1024 && g.lglmax >= 11 && smem_y_2048<T>() <= (size_t)max_smem;
}

template <typename T>
cudaError_t launch_x_r2c_2048(const Geometry& g, const T* M, const T* ms_map, T ms_scale, typename Cx<T>::t* X,
                              const typename Cx<T>::t* tw, cudaStream_t st)
{
    const size_t smem = smem_x_r2c_2048<T>();
    cudaError_t e = cudaFuncSetAttribute(x_r2c_2048_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    x_r2c_2048_kernel<T><<<dim3((g.ny + XROWS - 1) / XROWS, g.nz, 3), 256, smem, st>>>(g, M, ms_map, ms_scale, X, tw);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_x_c2r_2048(const Geometry& g, const typename Cx<T>::t* X, T* H, const typename Cx<T>::t* tw,
                              cudaStream_t st)
{
    const size_t smem = smem_x_c2r_2048<T>();
    cudaError_t e = cudaFuncSetAttribute(x_c2r_2048_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    x_c2r_2048_kernel<T><<<dim3((g.ny + XROWS - 1) / XROWS, g.nz, 3), 256, smem, st>>>(g, X, H, tw);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_y_2048(const Geometry& g, typename Cx<T>::t* X, typename Cx<T>::t* Y, const typename Cx<T>::t* tw,
                          cudaStream_t st, bool forward)
{
    const size_t smem = smem_y_2048<T>();
    const dim3 grid((3 * g.nz + YLINES - 1) / YLINES, g.nkx);
    if (forward) {
        cudaError_t e = cudaFuncSetAttribute(y_fwd_2048_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        y_fwd_2048_kernel<T><<<grid, 256, smem, st>>>(g, X, Y, tw);
    } else {
        cudaError_t e = cudaFuncSetAttribute(y_inv_2048_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        y_inv_2048_kernel<T><<<grid, 256, smem, st>>>(g, Y, X, tw);
    }
    return cudaGetLastError();
}

#define FFT2048_INST(T)                                                                                           \
    template bool x2048_ok<T>(const Geometry&, int);                                                             \
    template bool y2048_ok<T>(const Geometry&, int);                                                             \
    template cudaError_t launch_x_r2c_2048<T>(const Geometry&, const T*, const T*, T, Cx<T>::t*, const Cx<T>::t*, \
                                              cudaStream_t);                                                     \
    template cudaError_t launch_x_c2r_2048<T>(const Geometry&, const Cx<T>::t*, T*, const Cx<T>::t*, cudaStream_t); \
    template cudaError_t launch_y_2048<T>(const Geometry&, Cx<T>::t*, Cx<T>::t*, const Cx<T>::t*, cudaStream_t, bool);
FFT2048_INST(float)
FFT2048_INST(double)

}  // namespace boris
