// Transforms of length 512 (meshes of 129..256 cells along the axis): two
// lines per warp through the warp-held length-1024 transform of warp_fft.cuh.
//
// With u[2n + p] = l_p[n] (p = 0, 1; n < 512) and U = FFT_1024(u),
//   L_0[k] = (U[k] + U[k + 512]) / 2,   L_1[k] = (U[k] - U[k + 512]) w^-k / 2
// (w = exp(-2 pi i / 1024), k < 512) are the two lines' length-512
// transforms; U[k + 512] sits in the same lane as U[k], at register position
// pos ^ 1.  The inverse forms U[k] = L_0[k] + w^k L_1[k], U[k + 512] =
// L_0[k] - w^k L_1[k] and halves IFFT_1024(U) (unscaled transforms throughout).
//
// x passes: a complex line packs two real rows (real and imaginary parts), so
// a warp carries four rows and a CTA of eight warps 32 rows; the real
// spectra are untangled as A_k = (Z_k + conj Z_{512-k}) / 2 and
// B_k = (Z_k - conj Z_{512-k}) / (2i), k = 0..256, and packed back as
// Z_k = A_k + i B_k (A, B Hermitian) for the inverse.
// y passes: two complex lines per warp, 16 lines per CTA.
#include "boris_internal.cuh"
#include "warp_fft.cuh"

namespace boris {

namespace {

constexpr int R1025 = 1025;  // per-warp region stride (complex)

// w^(lane + 32 c) = w^lane w_32^c; w^lane is row 1 of the twiddle table
template <typename C>
__device__ __forceinline__ C w1024_at(int c, C wl)
{
    return c == 0 ? wl : c_mul(w128lit<C>(4 * c), wl);
}

// U (forward output, v[pos] = U[lane + 32 brev5(pos)]) -> L0, L1 at k = lane + 32 brev5(2q)
template <typename C, typename T>
__device__ __forceinline__ void split_pair(const C (&v)[32], C (&L0)[16], C (&L1)[16], C wl)
{
#pragma unroll
    for (int q = 0; q < 16; q++) {
        const C a = v[2 * q], b = v[2 * q + 1];  // U[k], U[k + 512]
        L0[q] = C{T(0.5) * (a.x + b.x), T(0.5) * (a.y + b.y)};
        L1[q] = c_mulc(C{T(0.5) * (a.x - b.x), T(0.5) * (a.y - b.y)}, w1024_at(brev5(2 * q), wl));
    }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    y_fwd_512_kernel(Geometry g, const typename Cx<T>::t* __restrict__ X, typename Cx<T>::t* __restrict__ Y,
                     const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* reg = tws + TW1024_SLOTS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lines = 3 * g.nz, ny = g.ny;
    const int kx = blockIdx.y, l0 = blockIdx.x * 16 + 2 * warp;
    load_tw1024(tws, tw_g, g.lmax);
    __syncthreads();
    if (l0 >= lines) return;
    const int p = lane & 1;
    const bool okl = l0 + p < lines;
    const C* src = X + ((size_t)kx * lines + l0 + p) * ny;
    C v[32];
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int n = 16 * a + (lane >> 1);  // u[32 a + lane] = l_p[n]
        v[a] = okl && n < ny ? src[n] : C{T(0), T(0)};
    }
#pragma unroll
    for (int a = 16; a < 32; a++) v[a] = C{T(0), T(0)};
    warp_fft1024_fwd(v, reg + warp * R1025, tws);
    C L0[16], L1[16];
    split_pair<C, T>(v, L0, L1, tws[32 + lane]);
    C* d0 = Y + ((size_t)kx * lines + l0) * 512;
    const bool has1 = l0 + 1 < lines;
#pragma unroll
    for (int q = 0; q < 16; q++) {
        const int k = lane + 32 * brev5(2 * q);
        d0[k] = L0[q];
        if (has1) d0[512 + k] = L1[q];
    }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    y_inv_512_kernel(Geometry g, const typename Cx<T>::t* __restrict__ Y, typename Cx<T>::t* __restrict__ X,
                     const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* reg = tws + TW1024_SLOTS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lines = 3 * g.nz, ny = g.ny;
    const int kx = blockIdx.y, l0 = blockIdx.x * 16 + 2 * warp;
    load_tw1024(tws, tw_g, g.lmax);
    __syncthreads();
    if (l0 >= lines) return;
    const bool has1 = l0 + 1 < lines;
    const C* s0 = Y + ((size_t)kx * lines + l0) * 512;
    const C wl = tws[32 + lane];
    C v[32];
#pragma unroll
    for (int d = 0; d < 16; d++) {
        const int k = lane + 32 * d;
        const C a = s0[k];
        const C b = has1 ? c_mul(s0[512 + k], w1024_at(d, wl)) : C{T(0), T(0)};
        v[brev5(d)] = c_add(a, b);      // U[k]
        v[brev5(d) ^ 1] = c_sub(a, b);  // U[k + 512]
    }
    warp_fft1024_inv(v, reg + warp * R1025, tws);
    // v[a] = 2 l_p[n], p = lane & 1, n = 16 a + lane / 2
    const int p = lane & 1;
    if (p && !has1) return;
    C* dst = X + ((size_t)kx * lines + l0 + p) * ny;
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int n = 16 * a + (lane >> 1);
        if (n < ny) dst[n] = C{T(0.5) * v[a].x, T(0.5) * v[a].y};
    }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    x_r2c_512_kernel(Geometry g, const T* __restrict__ M, const T* __restrict__ ms_map, T ms_scale,
                     typename Cx<T>::t* __restrict__ X, const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* reg = tws + TW1024_SLOTS;  // warp w: L_0 at [0, 512), L_1 at [512, 1024)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0 = blockIdx.x * 32, z = blockIdx.y, c = blockIdx.z;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    load_tw1024(tws, tw_g, g.lmax);
    __syncthreads();
    // line p of warp w packs rows y0 + w + 16 p (real part) and y0 + w + 16 p + 8 (imaginary part)
    const int p = lane & 1;
    const int ya = y0 + warp + 16 * p, yb = ya + 8;
    const size_t ncell = (size_t)nx * ny * nz;
    const T* ra = M + c * ncell + ((size_t)z * ny + ya) * nx;
    const T* rb = M + c * ncell + ((size_t)z * ny + yb) * nx;
    const T* ma = ms_map ? ms_map + ((size_t)z * ny + ya) * nx : nullptr;
    const T* mb = ms_map ? ms_map + ((size_t)z * ny + yb) * nx : nullptr;
    const bool oka = ya < ny, okb = yb < ny;
    C v[32];
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int n = 16 * a + (lane >> 1);
        const bool in = n < nx;
        T xa = (in && oka) ? ra[n] : T(0), xb = (in && okb) ? rb[n] : T(0);
        if (ms_map) {
            xa *= (in && oka) ? ma[n] : T(0);
            xb *= (in && okb) ? mb[n] : T(0);
        } else {
            xa *= ms_scale;
            xb *= ms_scale;
        }
        v[a] = C{xa, xb};
    }
#pragma unroll
    for (int a = 16; a < 32; a++) v[a] = C{T(0), T(0)};
    C* mine = reg + warp * R1025;
    warp_fft1024_fwd(v, mine, tws);
    {
        C L0[16], L1[16];
        split_pair<C, T>(v, L0, L1, tws[32 + lane]);
#pragma unroll
        for (int q = 0; q < 16; q++) {
            const int k = lane + 32 * brev5(2 * q);
            mine[k] = L0[q];
            mine[512 + k] = L1[q];
        }
    }
    __syncthreads();
    // X[kx][c][z][y0 + t], kx = 0..256: 32 consecutive y per kx
    for (int i = threadIdx.x; i < 257 * 32; i += blockDim.x) {
        const int t = i & 31, k = i >> 5;
        const int yy = y0 + t;
        if (yy >= ny) continue;
        const C* line = reg + (t & 7) * R1025 + 512 * ((t >> 4) & 1);
        const C zk = line[k & 511], zm = line[(512 - k) & 511];
        C out;
        if ((t & 8) == 0) out = C{T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y)};
        else out = C{T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x)};
        X[(((size_t)k * 3 + c) * nz + z) * ny + yy] = out;
    }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    x_c2r_512_kernel(Geometry g, const typename Cx<T>::t* __restrict__ X, T* __restrict__ H,
                     const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    // the 257 x 32 half-spectrum block, row kx holding column t at t ^ (kx & 31);
    // afterwards the warps' transpose regions
    C* S = tws + TW1024_SLOTS;
    C* reg = S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0 = blockIdx.x * 32, z = blockIdx.y, c = blockIdx.z;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    load_tw1024(tws, tw_g, g.lmax);
    const size_t plane = (size_t)3 * nz * ny;
    const size_t col0 = ((size_t)c * nz + z) * ny + y0;
    staged_loop<256, C>(
        257 * 32,
        [&](int i) {
            const int k = i >> 5, t = i & 31;
            return y0 + t < ny ? X[(size_t)k * plane + col0 + t] : C{T(0), T(0)};
        },
        [&](int i, C a) {
            const int k = i >> 5, t = i & 31;
            S[k * 32 + (t ^ (k & 31))] = a;
        });
    __syncthreads();
    // the spectrum of row t at bin k < 512 (Hermitian above 256; DC and Nyquist real)
    auto spec = [&](int t, int k) {
        C a = k <= 256 ? S[k * 32 + (t ^ (k & 31))] : S[(512 - k) * 32 + (t ^ ((512 - k) & 31))];
        if (k > 256) a.y = -a.y;
        if (k == 0 || k == 256) a.y = T(0);
        return a;
    };
    const C wl = tws[32 + lane];
    C v[32];
#pragma unroll
    for (int d = 0; d < 16; d++) {
        const int k = lane + 32 * d;
        C Lp[2];
#pragma unroll
        for (int p = 0; p < 2; p++) {  // Z_p = A + i B, rows warp + 16 p and warp + 16 p + 8
            const C A = spec(warp + 16 * p, k), B = spec(warp + 16 * p + 8, k);
            Lp[p] = C{A.x - B.y, A.y + B.x};
        }
        const C b = c_mul(Lp[1], w1024_at(d, wl));
        v[brev5(d)] = c_add(Lp[0], b);
        v[brev5(d) ^ 1] = c_sub(Lp[0], b);
    }
    __syncthreads();  // the block is consumed: its bytes become the transpose regions
    warp_fft1024_inv(v, reg + warp * R1025, tws);
    // v[a] = 2 z_p[n], p = lane & 1, n = 16 a + lane / 2: Re -> row warp + 16 p, Im -> row warp + 16 p + 8
    const int p = lane & 1;
    const int ya = y0 + warp + 16 * p, yb = ya + 8;
    const size_t ncell = (size_t)nx * ny * nz;
    T* ha = H + c * ncell + ((size_t)z * ny + ya) * nx;
    T* hb = H + c * ncell + ((size_t)z * ny + yb) * nx;
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int n = 16 * a + (lane >> 1);
        if (n < nx) {
            if (ya < ny) ha[n] = T(0.5) * v[a].x;
            if (yb < ny) hb[n] = T(0.5) * v[a].y;
        }
    }
}

template <typename T>
size_t smem_512()
{
    const size_t body = (size_t)8 * R1025 > (size_t)257 * 32 ? (size_t)8 * R1025 : (size_t)257 * 32;
    return ((size_t)TW1024_SLOTS + body) * sizeof(typename Cx<T>::t);
}

}  // namespace

template <typename T>
bool x512_ok(const Geometry& g, int max_smem)
{
    return g.px == 512 && g.nx <= 256 && smem_512<T>() <= (size_t)max_smem;
}
template <typename T>
bool y512_ok(const Geometry& g, int max_smem)
{
    return g.py == 512 && g.ny <= 256 && smem_512<T>() <= (size_t)max_smem;
}

template <typename T>
cudaError_t launch_x_r2c_512(const Geometry& g, const T* M, const T* ms_map, T ms_scale, typename Cx<T>::t* X,
                             const typename Cx<T>::t* tw, cudaStream_t st)
{
    const size_t smem = smem_512<T>();
    cudaError_t e = cudaFuncSetAttribute(x_r2c_512_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    x_r2c_512_kernel<T><<<dim3((g.ny + 31) / 32, g.nz, 3), 256, smem, st>>>(g, M, ms_map, ms_scale, X, tw);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_x_c2r_512(const Geometry& g, const typename Cx<T>::t* X, T* H, const typename Cx<T>::t* tw,
                             cudaStream_t st)
{
    const size_t smem = smem_512<T>();
    cudaError_t e = cudaFuncSetAttribute(x_c2r_512_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    x_c2r_512_kernel<T><<<dim3((g.ny + 31) / 32, g.nz, 3), 256, smem, st>>>(g, X, H, tw);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_y_512(const Geometry& g, typename Cx<T>::t* X, typename Cx<T>::t* Y, const typename Cx<T>::t* tw,
                         cudaStream_t st, bool forward)
{
    const size_t smem = smem_512<T>();
    const dim3 grid((3 * g.nz + 15) / 16, g.nkx);
    if (forward) {
        cudaError_t e = cudaFuncSetAttribute(y_fwd_512_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        y_fwd_512_kernel<T><<<grid, 256, smem, st>>>(g, X, Y, tw);
    } else {
        cudaError_t e = cudaFuncSetAttribute(y_inv_512_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        y_inv_512_kernel<T><<<grid, 256, smem, st>>>(g, Y, X, tw);
    }
    return cudaGetLastError();
}

#define FFT512_INST(T)                                                                                           \
    template bool x512_ok<T>(const Geometry&, int);                                                             \
    template bool y512_ok<T>(const Geometry&, int);                                                             \
    template cudaError_t launch_x_r2c_512<T>(const Geometry&, const T*, const T*, T, Cx<T>::t*, const Cx<T>::t*, \
                                             cudaStream_t);                                                     \
    template cudaError_t launch_x_c2r_512<T>(const Geometry&, const Cx<T>::t*, T*, const Cx<T>::t*, cudaStream_t); \
    template cudaError_t launch_y_512<T>(const Geometry&, Cx<T>::t*, Cx<T>::t*, const Cx<T>::t*, cudaStream_t, bool);
FFT512_INST(float)
FFT512_INST(double)

}  // namespace boris
