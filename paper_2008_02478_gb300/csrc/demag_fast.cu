// Warp-per-line kernels for transform length 1024 (meshes of 257..512 cells
// along the axis): the x real-to-complex and complex-to-real passes and the
// y forward / inverse passes of the split schedule.  Each warp owns one
// (packed) line in registers (warp_fft.cuh); global loads and stores are
// 32 consecutive elements per instruction.
#include "boris_internal.cuh"
#include "warp_fft.cuh"

namespace boris {

constexpr int REG1025 = 1025;  // per-warp region stride (complex): one pad element spreads the regions over banks

// x real-to-complex, px = 1024: 16 rows (c, z, y0..y0+15) per CTA; warp w packs
// row w (real part) and row w + 8 (imaginary part) into one complex line.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) x_r2c_1024_kernel(Geometry g, const T* __restrict__ M,
                                                         const T* __restrict__ ms_map, T ms_scale,
                                                         typename Cx<T>::t* __restrict__ X,
                                                         const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* reg = tws + TW1024_SLOTS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0 = blockIdx.x * 16, z = blockIdx.y, c = blockIdx.z;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    load_tw1024(tws, tw_g, g.lglmax - 10);
    __syncthreads();
    const size_t ncell = (size_t)nx * ny * nz;
    const int ya = y0 + warp, yb = y0 + warp + 8;
    const T* ra = M + c * ncell + ((size_t)z * ny + ya) * nx;
    const T* rb = M + c * ncell + ((size_t)z * ny + yb) * nx;
    const T* ma = ms_map ? ms_map + ((size_t)z * ny + ya) * nx : nullptr;
    const T* mb = ms_map ? ms_map + ((size_t)z * ny + yb) * nx : nullptr;
    C v[32];
    const bool oka = ya < ny, okb = yb < ny;
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int x = 32 * a + lane;
        const bool in = x < nx;
        v[a] = C{(in && oka) ? ra[x] : T(0), (in && okb) ? rb[x] : T(0)};
    }
    if (ms_map) {
#pragma unroll
        for (int a = 0; a < 16; a++) {
            const int x = 32 * a + lane;
            const bool in = x < nx;
            v[a].x *= (in && oka) ? ma[x] : T(0);
            v[a].y *= (in && okb) ? mb[x] : T(0);
        }
    } else {
#pragma unroll
        for (int a = 0; a < 16; a++) {
            v[a].x *= ms_scale;
            v[a].y *= ms_scale;
        }
    }
#pragma unroll
    for (int a = 16; a < 32; a++) v[a] = C{T(0), T(0)};
    C* mine = reg + warp * REG1025;
    warp_fft1024_fwd(v, mine, tws);
#pragma unroll
    for (int pos = 0; pos < 32; pos++) mine[lane + 32 * brev5(pos)] = v[pos];
    __syncthreads();
    // unpack: A_k = (Z_k + conj Z_{N-k})/2 (row w), B_k = (Z_k - conj Z_{N-k})/(2i) (row w + 8)
    for (int i = threadIdx.x; i < 513 * 16; i += 256) {
        const int t = i & 15, kx = i >> 4;
        const int y = y0 + t;
        if (y >= ny) continue;
        const C* line = reg + (t & 7) * REG1025;
        const C zk = line[kx], zm = line[(1024 - kx) & 1023];
        C out;
        if (t < 8) out = C{T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y)};
        else out = C{T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x)};
        X[(((size_t)kx * 3 + c) * nz + z) * ny + y] = out;
    }
}

// x complex-to-real, px = 1024: warp w rebuilds Z = A + i B from the half
// spectra of rows w and w + 8 and transforms back.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) x_c2r_1024_kernel(Geometry g, const typename Cx<T>::t* __restrict__ X,
                                                         T* __restrict__ H,
                                                         const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* reg = tws + TW1024_SLOTS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0 = blockIdx.x * 16, z = blockIdx.y, c = blockIdx.z;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    load_tw1024(tws, tw_g, g.lglmax - 10);
    __syncthreads();
    const int ya = y0 + warp, yb = y0 + warp + 8;
    // stage the 513 x 16 half-spectrum block with coalesced 128-byte rows;
    // row kx holds column t at t ^ (kx & 15), so lanes walking kx read
    // distinct banks without padding (which would cost the third CTA per SM)
    C* S = reg;
    staged_loop<256, C>(513 * 16, [&](int i) {
        const int kx = i >> 4, t = i & 15;
        return y0 + t < ny ? X[(((size_t)kx * 3 + c) * nz + z) * ny + y0 + t] : C{T(0), T(0)};
    }, [&](int i, C a) { S[(i >> 4) * 16 + ((i & 15) ^ ((i >> 4) & 15))] = a; });
    __syncthreads();
    C v[32];
#pragma unroll
    for (int d = 0; d < 32; d++) {
        const int k = lane + 32 * d;
        const bool upper = k > 512;
        const int kx = upper ? 1024 - k : k;
        C A = S[kx * 16 + (warp ^ (kx & 15))], B = S[kx * 16 + ((warp + 8) ^ (kx & 15))];
        if (kx == 0 || kx == 512) {
            A.y = T(0);  // DC and Nyquist bins of a real signal are real
            B.y = T(0);
        }
        if (upper) {
            A.y = -A.y;
            B.y = -B.y;
        }
        v[brev5(d)] = C{A.x - B.y, A.y + B.x};
    }
    __syncthreads();  // the staging area becomes the warps' transpose tiles
    warp_fft1024_inv(v, reg + warp * REG1025, tws);
    const size_t ncell = (size_t)nx * ny * nz;
    T* ha = H + c * ncell + ((size_t)z * ny + ya) * nx;
    T* hb = H + c * ncell + ((size_t)z * ny + yb) * nx;
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int x = 32 * a + lane;
        if (x < nx) {
            if (ya < ny) ha[x] = v[a].x;
            if (yb < ny) hb[x] = v[a].y;
        }
    }
}

// y forward, py = 1024: X[kx][line][y] -> Y[kx][line][ky], one line per warp.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) y_fwd_1024_kernel(Geometry g, const typename Cx<T>::t* __restrict__ X,
                                                         typename Cx<T>::t* __restrict__ Y,
                                                         const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* reg = tws + TW1024_SLOTS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lines = 3 * g.nz, ny = g.ny;
    const int kx = blockIdx.y, line = blockIdx.x * 8 + warp;
    load_tw1024(tws, tw_g, g.lglmax - 10);
    __syncthreads();
    if (line >= lines) return;
    const C* src = X + ((size_t)kx * lines + line) * ny;
    C v[32];
#pragma unroll
    for (int a = 0; a < 32; a++) {
        const int y = 32 * a + lane;
        v[a] = (a < 16 && y < ny) ? src[y] : C{T(0), T(0)};
    }
    warp_fft1024_fwd(v, reg + warp * REG1025, tws);
    C* dst = Y + ((size_t)kx * lines + line) * 1024;
#pragma unroll
    for (int pos = 0; pos < 32; pos++) dst[lane + 32 * brev5(pos)] = v[pos];
}

// y inverse, py = 1024: Y[kx][line][ky] -> X[kx][line][y], cropped to ny.
template <typename T>
__global__ void __launch_bounds__(256) y_inv_1024_kernel(Geometry g, const typename Cx<T>::t* __restrict__ Y,
                                                         typename Cx<T>::t* __restrict__ X,
                                                         const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* reg = tws + TW1024_SLOTS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lines = 3 * g.nz, ny = g.ny;
    const int kx = blockIdx.y, line = blockIdx.x * 8 + warp;
    load_tw1024(tws, tw_g, g.lglmax - 10);
    __syncthreads();
    if (line >= lines) return;
    const C* src = Y + ((size_t)kx * lines + line) * 1024;
    C v[32];
#pragma unroll
    for (int d = 0; d < 32; d++) v[brev5(d)] = src[lane + 32 * d];
    warp_fft1024_inv(v, reg + warp * REG1025, tws);
    C* dst = X + ((size_t)kx * lines + line) * ny;
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int y = 32 * a + lane;
        if (y < ny) dst[y] = v[a];
    }
}

template <typename T>
static size_t smem_1024()
{
    // per-warp regions, also used as the 513 x 16 staging block of x_c2r
    // (74.4 KB in FP32 with the twiddles: three CTAs per SM)
    const size_t regions = 8 * (size_t)REG1025 > 513 * 16 ? 8 * (size_t)REG1025 : 513 * 16;
    return ((size_t)TW1024_SLOTS + regions) * sizeof(typename Cx<T>::t);
}

template <typename T>
bool x1024_ok(const Geometry& g, int max_smem)
{
    return g.px == 1024 && g.nx <= 512 && smem_1024<T>() <= (size_t)max_smem;
}
template <typename T>
bool y1024_ok(const Geometry& g, int max_smem)
{
    return g.py == 1024 && g.ny <= 512 && smem_1024<T>() <= (size_t)max_smem;
}

template <typename T>
cudaError_t launch_x_r2c_1024(const Geometry& g, const T* M, const T* ms_map, T ms_scale, typename Cx<T>::t* X,
                              const typename Cx<T>::t* tw, cudaStream_t st)
{
    const size_t smem = smem_1024<T>();
    cudaError_t e = cudaFuncSetAttribute(x_r2c_1024_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    x_r2c_1024_kernel<T><<<dim3((g.ny + 15) / 16, g.nz, 3), 256, smem, st>>>(g, M, ms_map, ms_scale, X, tw);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_x_c2r_1024(const Geometry& g, const typename Cx<T>::t* X, T* H, const typename Cx<T>::t* tw,
                              cudaStream_t st)
{
    const size_t smem = smem_1024<T>();
    cudaError_t e = cudaFuncSetAttribute(x_c2r_1024_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    x_c2r_1024_kernel<T><<<dim3((g.ny + 15) / 16, g.nz, 3), 256, smem, st>>>(g, X, H, tw);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_y_1024(const Geometry& g, typename Cx<T>::t* X, typename Cx<T>::t* Y, const typename Cx<T>::t* tw,
                          cudaStream_t st, bool forward)
{
    const size_t smem = smem_1024<T>();
    const dim3 grid((3 * g.nz + 7) / 8, g.nkx);
    if (forward) {
        cudaError_t e = cudaFuncSetAttribute(y_fwd_1024_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        y_fwd_1024_kernel<T><<<grid, 256, smem, st>>>(g, X, Y, tw);
    } else {
        cudaError_t e = cudaFuncSetAttribute(y_inv_1024_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        y_inv_1024_kernel<T><<<grid, 256, smem, st>>>(g, Y, X, tw);
    }
    return cudaGetLastError();
}

cudaError_t upload_twiddles_fast() { return upload_small_twiddles_here(); }

#define FAST_INST(T)                                                                                              \
    template bool x1024_ok<T>(const Geometry&, int);                                                             \
    template bool y1024_ok<T>(const Geometry&, int);                                                             \
    template cudaError_t launch_x_r2c_1024<T>(const Geometry&, const T*, const T*, T, Cx<T>::t*, const Cx<T>::t*, \
                                              cudaStream_t);                                                     \
    template cudaError_t launch_x_c2r_1024<T>(const Geometry&, const Cx<T>::t*, T*, const Cx<T>::t*, cudaStream_t); \
    template cudaError_t launch_y_1024<T>(const Geometry&, Cx<T>::t*, Cx<T>::t*, const Cx<T>::t*, cudaStream_t, bool);
FAST_INST(float)
FAST_INST(double)

}  // namespace boris
