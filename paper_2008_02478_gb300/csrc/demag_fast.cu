// Warp-per-line kernels for transform length 1024 (meshes of 257..512 cells
// along the axis): the x real-to-complex and complex-to-real passes and the
// y forward / inverse passes of the split schedule.  Each warp owns one
// (packed) line in registers (warp_fft.cuh); global loads and stores are
// 32 consecutive elements per instruction.
#include <cstdint>
#include <cstdlib>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "boris_internal.cuh"
#include "bulk_async.cuh"
#include "warp_fft.cuh"

namespace boris {

constexpr int REG1025 = 1025;  // per-warp region stride (complex): one pad element spreads the regions over banks

// x real-to-complex, px = 1024: 16 rows (c, z, y0..y0+15) per CTA; warp w packs
// row w (real part) and row w + 8 (imaginary part) into one complex line.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) x_r2c_1024_kernel(Geometry g, const T* __restrict__ M,
                                                         const T* __restrict__ ms_map, T ms_scale,
                                                         typename Cx<T>::t* __restrict__ X,
                                                         const typename Cx<T>::t* __restrict__ tw_g,
                                                         unsigned* __restrict__ absmax)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* reg = tws + TW1024_SLOTS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0 = blockIdx.x * 16, z = blockIdx.y, c = blockIdx.z;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    load_tw1024(tws, tw_g, g.lmax);
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
    if (absmax) {
        // the largest |Ms M| this warp loaded (one atomic per warp; the bits of
        // non-negative floats order like the floats)
        float mx = 0.f;
#pragma unroll
        for (int a = 0; a < 16; a++) mx = fmaxf(mx, fmaxf(fabsf((float)v[a].x), fabsf((float)v[a].y)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomicMax(absmax, __float_as_uint(mx));
    }
#pragma unroll
    for (int a = 16; a < 32; a++) v[a] = C{T(0), T(0)};
    C* mine = reg + warp * REG1025;
    warp_fft1024_fwd<C, true>(v, mine, tws);
#pragma unroll
    for (int pos = 0; pos < 32; pos++) mine[lane + 32 * brev5(pos)] = v[pos];
    __syncthreads();
    // unpack: A_k = (Z_k + conj Z_{N-k})/2 (row w), B_k = (Z_k - conj Z_{N-k})/(2i) (row w + 8).
    // A thread keeps its row t = tid mod 16 and walks kx = tid / 16 + 16 j, so
    // its shared and global addresses advance by fixed strides.
    {
        const int t = threadIdx.x & 15, kx0 = threadIdx.x >> 4;
        const int y = y0 + t;
        if (y < ny) {
            const C* line = reg + (t & 7) * REG1025;
            const size_t xstride = (size_t)3 * nz * ny;  // one kx step in X
            C* dst = X + ((size_t)kx0 * 3 + c) * nz * ny + (size_t)z * ny + y;
            const bool lo = t < 8;
            // kx = 0 (with N - kx = 1024 -> 0) is the only index whose mirror wraps
            const C* lk = line + kx0;
            const C* lm = line + (1024 - kx0);
            if (kx0 == 0) lm = line;
#pragma unroll 4
            for (int kx = kx0; kx < 513; kx += 16) {
                const C zk = *lk, zm = *lm;
                // row w: (Re zk + Re zm, Im zk - Im zm) / 2; row w + 8: (Im zk + Im zm, Re zm - Re zk) / 2
                const T a0 = lo ? zk.x : zk.y, a1 = lo ? zm.x : zm.y;
                const T b0 = lo ? zk.y : zm.x, b1 = lo ? zm.y : zk.x;
                *dst = C{T(0.5) * (a0 + a1), T(0.5) * (b0 - b1)};
                dst += 16 * xstride;
                lk += 16;
                lm = (kx == 0) ? line + (1024 - 16) : lm - 16;
            }
        }
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
    load_tw1024(tws, tw_g, g.lmax);
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

// x complex-to-real, px = 1024, FP32, with the 513 x 16 half-spectrum block
// of the CTA fetched by tensor copies: rows kx < 512 as four 128-row boxes
// with the 128-byte swizzle (16-byte chunk c of row kx lands at chunk
// c ^ (kx & 7)), so the whole block is in flight at once and the column reads
// below spread over the banks; row 512 by plain loads.  The wait for the
// copies is bounded; when it gives up, the CTA latches BORIS_ERR_TIMEOUT in
// *status and returns.
constexpr size_t XC2R_TMA_SMEM = 1024 + 512 * 128 + 128 + (size_t)TW1024_SLOTS * sizeof(float2) + 16;

__global__ void __launch_bounds__(256, 3) x_c2r_1024_tma_kernel(const __grid_constant__ CUtensorMap xmap, Geometry g,
                                                                 const float2* __restrict__ X, float* __restrict__ H,
                                                                 const float2* __restrict__ tw_g, int* status,
                                                                 unsigned long long limit_ns)
{
    extern __shared__ unsigned char smem_raw[];
    // aligned to 1024 bytes by an offset from the shared array itself, so that the
    // compiler keeps every access derived from base in the shared state space
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    float2* S = reinterpret_cast<float2*>(base);               // rows kx < 512, swizzled
    float2* R512 = reinterpret_cast<float2*>(base + 512 * 128);  // row kx = 512
    float2* tws = reinterpret_cast<float2*>(base + 512 * 128 + 128);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + 512 * 128 + 128 + TW1024_SLOTS * sizeof(float2));
    float2* reg = S;  // per-warp transpose regions once the block is consumed
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0 = blockIdx.x * 16, z = blockIdx.y, c = blockIdx.z;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int x0 = (c * nz + z) * ny + y0;  // column of the block in the [kx][(c, z, y)] view of X
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(bar, 512 * 128);
        for (int i = 0; i < 4; i++) tma_load_2d(S + i * 128 * 16, &xmap, x0, i * 128, bar);
    }
    load_tw1024(tws, tw_g, g.lmax);
    if (warp == 0 && lane < 16) {
        const size_t plane = (size_t)3 * nz * ny;
        R512[lane] = y0 + lane < ny ? X[512 * plane + x0 + lane] : float2{0.f, 0.f};
    }
    __syncthreads();  // barrier initialised, twiddles and row 512 staged
    const bool ok = mbar_wait_bounded(bar, 0, limit_ns);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicCAS(status, 0, -5);  // BORIS_ERR_TIMEOUT
        return;
    }
    const int ya = y0 + warp, yb = y0 + warp + 8;
    // element (kx, t) sits at kx 16 + 2 ((t >> 1) ^ (kx & 7)) + (t & 1); for
    // k = lane + 32 d the row is kx = k (d < 16, kx & 7 = lane & 7) or
    // 1024 - k (d > 16, kx & 7 = -lane & 7), so each half reads at fixed
    // per-thread offsets plus a compile-time 512 d
    const int wa = warp >> 1, wb = (warp + 8) >> 1, wl = warp & 1;
    const float2* loA = S + lane * 16 + 2 * (wa ^ (lane & 7)) + wl;
    const float2* loB = S + lane * 16 + 2 * (wb ^ (lane & 7)) + wl;
    const float2* hiA = S + (1024 - lane) * 16 + 2 * (wa ^ (-lane & 7)) + wl;
    const float2* hiB = S + (1024 - lane) * 16 + 2 * (wb ^ (-lane & 7)) + wl;
    float2 v[32];
#pragma unroll
    for (int d = 0; d < 32; d++) {
        float2 A, B;
        if (d < 16) {
            A = loA[512 * d];
            B = loB[512 * d];
            if (d == 0 && lane == 0) {
                A.y = 0.f;  // DC bin of a real signal is real
                B.y = 0.f;
            }
        } else if (d > 16) {
            A = hiA[-512 * d];
            B = hiB[-512 * d];
            A.y = -A.y;
            B.y = -B.y;
        } else if (lane == 0) {
            A = float2{R512[warp].x, 0.f};  // Nyquist bin, real
            B = float2{R512[warp + 8].x, 0.f};
        } else {
            A = hiA[-512 * d];  // k = 512 + lane: kx = 512 - lane
            B = hiB[-512 * d];
            A.y = -A.y;
            B.y = -B.y;
        }
        v[brev5(d)] = float2{A.x - B.y, A.y + B.x};
    }
    __syncthreads();  // the staging block becomes the warps' transpose tiles
    warp_fft1024_inv(v, reg + warp * REG1025, tws);
    const size_t ncell = (size_t)nx * ny * nz;
    float* ha = H + c * ncell + ((size_t)z * ny + ya) * nx;
    float* hb = H + c * ncell + ((size_t)z * ny + yb) * nx;
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int x = 32 * a + lane;
        if (x < nx) {
            if (ya < ny) ha[x] = v[a].x;
            if (yb < ny) hb[x] = v[a].y;
        }
    }
}

// X as a 2D array of 8-byte elements: nkx rows of 3 nz ny columns; boxes of
// 16 columns x 128 rows, 128-byte swizzle
static cudaError_t xc2r_map(const Geometry& g, const float2* X, CUtensorMap* map)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)3 * g.nz * g.ny, (cuuint64_t)g.nkx};
    const cuuint64_t strides[1] = {(cuuint64_t)3 * g.nz * g.ny * sizeof(float2)};
    const cuuint32_t box[2] = {16, 128};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<float2*>(X), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// the tensor-copy form needs 16-byte aligned block columns and row pitch (ny even)
bool x_c2r_tma_ok(const Geometry& g, int max_smem)
{
    return g.px == 1024 && g.nx <= 512 && g.ny % 2 == 0 && XC2R_TMA_SMEM <= (size_t)max_smem;
}

cudaError_t launch_x_c2r_1024_tma(const Geometry& g, const float2* X, float* H, const float2* tw, int* status,
                                  unsigned long long limit_ns, cudaStream_t st)
{
    CUtensorMap map;
    cudaError_t e = xc2r_map(g, X, &map);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(x_c2r_1024_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XC2R_TMA_SMEM);
    if (e != cudaSuccess) return e;
    x_c2r_1024_tma_kernel<<<dim3((g.ny + 15) / 16, g.nz, 3), 256, XC2R_TMA_SMEM, st>>>(map, g, X, H, tw, status,
                                                                                       limit_ns);
    return cudaGetLastError();
}

// y forward, py = 1024: X[kx][line][y] -> Y[kx][line][ky], one line per warp.
// Two CTAs per SM (93 registers): 0.099 ms at 512 x 512 x 32 against 0.107 ms
// with three (80 registers) - fewer lines in flight, and more loads in flight
// per line; the x passes and the 16-bit y passes measured slower with two.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) y_fwd_1024_kernel(Geometry g, const typename Cx<T>::t* __restrict__ X,
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
    load_tw1024(tws, tw_g, g.lmax);
    __syncthreads();
    if (line >= lines) return;
    const C* src = X + ((size_t)kx * lines + line) * ny;
    C v[32];
#pragma unroll
    for (int a = 0; a < 32; a++) {
        const int y = 32 * a + lane;
        v[a] = (a < 16 && y < ny) ? src[y] : C{T(0), T(0)};
    }
    warp_fft1024_fwd<C, true>(v, reg + warp * REG1025, tws);
    C* dst = Y + ((size_t)kx * lines + line) * 1024;
#pragma unroll
    for (int pos = 0; pos < 32; pos++) dst[lane + 32 * brev5(pos)] = v[pos];
}

// y inverse, py = 1024: Y[kx][line][ky] -> X[kx][line][y], cropped to ny.
// Its twiddles use the padded-index table layout (measured 0.105 ms against
// 0.127-0.129 ms with the row-per-c layout at 512 x 512 x 32; the persistent
// 16-bit inverse below is the other way round).
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
    load_tw1024_slots(tws, tw_g, g.lglmax - 10);
    __syncthreads();
    if (line >= lines) return;
    const C* src = Y + ((size_t)kx * lines + line) * 1024;
    C v[32];
#pragma unroll
    for (int d = 0; d < 32; d++) v[brev5(d)] = src[lane + 32 * d];
    warp_fft1024_inv<C, false>(v, reg + warp * REG1025, tws);
    C* dst = X + ((size_t)kx * lines + line) * ny;
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int y = 32 * a + lane;
        if (y < ny) dst[y] = v[a];
    }
}

// The same y passes on the 16-bit spectrum of the mixed-precision split schedule
// (BF16, line-contiguous layout [kx][c][part][z][ky], see zconv_tc6.cu): each
// (part, z) line of a kx plane is py consecutive values, so a warp moves 32
// consecutive ky (64 bytes) per instruction.
__device__ __forceinline__ size_t y16_index(int kx, int c, int part, int z, int ky, int nz, int py)
{
    return ((((size_t)kx * 3 + c) * 2 + part) * nz + z) * (size_t)py + ky;
}

// Power-of-two scale s of an FP16 spectrum: s nx ny nz max|M| < 2^14, so that
// the spectrum (at most nx ny max|M| after the x and y transforms), its z
// transform and the kernel products stay inside FP16's range.
__device__ __forceinline__ float y16_scale_exp(const Geometry& g, const unsigned* absmax, int* e)
{
    const float bound = __uint_as_float(*absmax) * ((float)g.nx * (float)g.ny * (float)g.nz);
    *e = 0;
    if (!(bound > 0.f) || !isfinite(bound)) return 1.f;
    frexpf(bound, e);  // bound = f 2^e, 0.5 <= f < 1
    return ldexpf(1.f, 14 - *e);
}

template <bool H16>
__device__ __forceinline__ unsigned short to16(float v)
{
    if constexpr (H16) return __half_as_ushort(__float2half_rn(v));
    else return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
template <bool H16>
__device__ __forceinline__ float from16(unsigned short v)
{
    if constexpr (H16) return __half2float(__ushort_as_half(v));
    else return __bfloat162float(__ushort_as_bfloat16(v));
}

// H16: FP16 values scaled by s (y16_scale_exp), else BF16 unscaled
template <bool H16>
__global__ void __launch_bounds__(256, 3) y_fwd_1024_b16_kernel(Geometry g, const float2* __restrict__ X,
                                                                unsigned short* __restrict__ Y16,
                                                                const float2* __restrict__ tw_g,
                                                                const unsigned* __restrict__ absmax)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tws = reinterpret_cast<float2*>(smem_raw);
    float2* reg = tws + TW1024_SLOTS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lines = 3 * g.nz, ny = g.ny, nz = g.nz;
    const int kx = blockIdx.y, line = blockIdx.x * 8 + warp;
    load_tw1024(tws, tw_g, g.lmax);
    __syncthreads();
    if (line >= lines) return;
    const int c = line / nz, z = line - c * nz;
    const float2* src = X + ((size_t)kx * lines + line) * ny;
    float2 v[32];
#pragma unroll
    for (int a = 0; a < 32; a++) {
        const int y = 32 * a + lane;
        v[a] = (a < 16 && y < ny) ? src[y] : float2{0.f, 0.f};
    }
    warp_fft1024_fwd<float2, true>(v, reg + warp * REG1025, tws);
    float s = 1.f;
    if constexpr (H16) {
        int e;
        s = y16_scale_exp(g, absmax, &e);
    }
    // v[pos] = Y[ky], ky = lane + 32 brev5(pos)
    unsigned short* re = Y16 + y16_index(kx, c, 0, z, lane, nz, 1024);
    unsigned short* im = Y16 + y16_index(kx, c, 1, z, lane, nz, 1024);
#pragma unroll
    for (int pos = 0; pos < 32; pos++) {
        re[32 * brev5(pos)] = to16<H16>(H16 ? v[pos].x * s : v[pos].x);
        im[32 * brev5(pos)] = to16<H16>(H16 ? v[pos].y * s : v[pos].y);
    }
}

// H16: the FP16 result of the z stage carries px py pz s / 128 (see zconv_tc6.cu)
template <bool H16>
__global__ void __launch_bounds__(256) y_inv_1024_b16_kernel(Geometry g, const unsigned short* __restrict__ Y16,
                                                             float2* __restrict__ X, const float2* __restrict__ tw_g,
                                                             const unsigned* __restrict__ absmax)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tws = reinterpret_cast<float2*>(smem_raw);
    float2* reg = tws + TW1024_SLOTS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lines = 3 * g.nz, ny = g.ny, nz = g.nz;
    const int kx = blockIdx.y, line = blockIdx.x * 8 + warp;
    load_tw1024_slots(tws, tw_g, g.lglmax - 10);
    __syncthreads();
    if (line >= lines) return;
    const int c = line / nz, z = line - c * nz;
    const unsigned short* re = Y16 + y16_index(kx, c, 0, z, lane, nz, 1024);
    const unsigned short* im = Y16 + y16_index(kx, c, 1, z, lane, nz, 1024);
    float u = 1.f;
    if constexpr (H16) {
        int e;
        y16_scale_exp(g, absmax, &e);
        u = ldexpf(128.f / ((float)g.px * (float)g.py * (float)g.pz), e - 14);  // 128 / (px py pz s)
    }
    float2 v[32];
#pragma unroll
    for (int d = 0; d < 32; d++) {
        const float a = from16<H16>(re[32 * d]), b = from16<H16>(im[32 * d]);
        v[brev5(d)] = H16 ? float2{a * u, b * u} : float2{a, b};
    }
    warp_fft1024_inv<float2, false>(v, reg + warp * REG1025, tws);
    float2* dst = X + ((size_t)kx * lines + line) * ny;
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int y = 32 * a + lane;
        if (y < ny) dst[y] = v[a];
    }
}

// Persistent form of the 16-bit y passes (spectrum in BF16 or scaled FP16).
// Each warp walks the lines gl = kx * 3 nz + line, from its global warp index
// in steps of the grid's warp count, and stages the next line's input in its
// own transpose tile by 16-byte asynchronous copies as soon as the tile is
// free (right after the transpose), so that the loads overlap the second
// register transform and the stores of the current line.  Needs even ny
// (16-byte line starts) and 16-byte aligned arrays.  (The FP32 passes gain
// nothing from it: they run at 0.85-0.89 of HBM bandwidth as they are.)
constexpr int REGP = 1056;  // per-warp tile of the persistent form: 32 rows of 33 (16-byte aligned tiles)
constexpr int YP_CTAS = 3;  // resident CTAs per SM (76.3 KB of shared memory, 80 registers)
constexpr size_t YP_SMEM = ((size_t)TW1024_SLOTS + 8 * (size_t)REGP) * sizeof(float2);

template <bool H16>
__global__ void __launch_bounds__(256, YP_CTAS) y_fwd_1024_persist_kernel(Geometry g, const float2* __restrict__ X,
                                                                          unsigned short* __restrict__ Y16,
                                                                          const float2* __restrict__ tw_g,
                                                                          const unsigned* __restrict__ absmax,
                                                                          int total)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tws = reinterpret_cast<float2*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* tile = tws + TW1024_SLOTS + warp * REGP;
    const int lines = 3 * g.nz, ny = g.ny, nz = g.nz;
    const int stride = gridDim.x * 8;
    int gl = blockIdx.x * 8 + warp;
    auto stage = [&](int l) {
        const float2* src = X + (size_t)l * ny;
        for (int i = lane; 2 * i < ny; i += 32) cp_async16(tile + 2 * i, src + 2 * i);
        cp_async_commit();
    };
    if (gl < total) stage(gl);  // the first line lands while the twiddles load
    load_tw1024(tws, tw_g, g.lmax);
    __syncthreads();
    float s = 1.f;
    if constexpr (H16) {
        int e;
        s = y16_scale_exp(g, absmax, &e);
    }
    for (; gl < total; gl += stride) {
        cp_async_wait<0>();
        __syncwarp();
        float2 v[32];
#pragma unroll
        for (int a = 0; a < 32; a++) {
            const int y = 32 * a + lane;
            v[a] = (a < 16 && y < ny) ? tile[y] : float2{0.f, 0.f};
        }
        __syncwarp();  // the staged line is in registers: the transpose may overwrite it
        warp_fft1024_fwd_a<float2, true, 33>(v, tile, tws);
        if (gl + stride < total) stage(gl + stride);
        warp_fft1024_fwd_b(v);
        // v[pos] = Y[ky], ky = lane + 32 brev5(pos)
        const int kx = gl / lines, line = gl - kx * lines;
        const int c = line / nz, z = line - c * nz;
        unsigned short* re = Y16 + y16_index(kx, c, 0, z, lane, nz, 1024);
        unsigned short* im = re + (size_t)nz * 1024;
#pragma unroll
        for (int pos = 0; pos < 32; pos++) {
            re[32 * brev5(pos)] = to16<H16>(H16 ? v[pos].x * s : v[pos].x);
            im[32 * brev5(pos)] = to16<H16>(H16 ? v[pos].y * s : v[pos].y);
        }
    }
}

template <bool H16>
__global__ void __launch_bounds__(256, YP_CTAS) y_inv_1024_persist_kernel(Geometry g,
                                                                          const unsigned short* __restrict__ Y16,
                                                                          float2* __restrict__ X,
                                                                          const float2* __restrict__ tw_g,
                                                                          const unsigned* __restrict__ absmax,
                                                                          int total)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tws = reinterpret_cast<float2*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* tile = tws + TW1024_SLOTS + warp * REGP;
    const int lines = 3 * g.nz, ny = g.ny, nz = g.nz;
    const int stride = gridDim.x * 8;
    int gl = blockIdx.x * 8 + warp;
    auto stage = [&](int l) {  // the real and imaginary 1024-value lines, 2 KB each
        const int kx = l / lines, line = l - kx * lines;
        const int c = line / nz, z = line - c * nz;
        const unsigned short* re = Y16 + y16_index(kx, c, 0, z, 0, nz, 1024);
        const unsigned short* im = re + (size_t)nz * 1024;
        unsigned short* t16 = reinterpret_cast<unsigned short*>(tile);
#pragma unroll
        for (int i = lane; i < 128; i += 32) {
            cp_async16(t16 + 8 * i, re + 8 * i);
            cp_async16(t16 + 1024 + 8 * i, im + 8 * i);
        }
        cp_async_commit();
    };
    if (gl < total) stage(gl);
    load_tw1024(tws, tw_g, g.lmax);  // row table: constant offsets, no bank conflicts (0.086 -> 0.074 ms)
    __syncthreads();
    float u = 1.f;
    if constexpr (H16) {
        int e;
        y16_scale_exp(g, absmax, &e);
        u = ldexpf(128.f / ((float)g.px * (float)g.py * (float)g.pz), e - 14);  // 128 / (px py pz s)
    }
    for (; gl < total; gl += stride) {
        cp_async_wait<0>();
        __syncwarp();
        float2 v[32];
        const unsigned short* t16 = reinterpret_cast<const unsigned short*>(tile);
#pragma unroll
        for (int d = 0; d < 32; d++) {
            const float a = from16<H16>(t16[lane + 32 * d]), b = from16<H16>(t16[1024 + lane + 32 * d]);
            v[brev5(d)] = H16 ? float2{a * u, b * u} : float2{a, b};
        }
        __syncwarp();
        warp_fft1024_inv_a<float2, true, 33>(v, tile, tws);
        if (gl + stride < total) stage(gl + stride);
        warp_fft1024_inv_b(v);
        float2* dst = X + (size_t)gl * ny;
#pragma unroll
        for (int a = 0; a < 16; a++) {
            const int y = 32 * a + lane;
            if (y < ny) dst[y] = v[a];
        }
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
                              const typename Cx<T>::t* tw, cudaStream_t st, unsigned* absmax)
{
    const size_t smem = smem_1024<T>();
    cudaError_t e = cudaFuncSetAttribute(x_r2c_1024_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    x_r2c_1024_kernel<T><<<dim3((g.ny + 15) / 16, g.nz, 3), 256, smem, st>>>(g, M, ms_map, ms_scale, X, tw, absmax);
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
// The persistent 16-bit y passes apply to even ny and 16-byte aligned arrays;
// BORIS_Y_PERSIST=0 selects the one-line-per-warp grid instead.
static bool y_persist_ok(const Geometry& g, const void* a, const void* b)
{
    const char* env = getenv("BORIS_Y_PERSIST");
    if (env && atoi(env) == 0) return false;
    return g.ny % 2 == 0 && ((uintptr_t)a & 15) == 0 && ((uintptr_t)b & 15) == 0;
}

template <bool H16>
static cudaError_t launch_y16_persist(const Geometry& g, float2* X, unsigned short* Y16, const float2* tw,
                                      cudaStream_t st, bool forward, const unsigned* absmax)
{
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const void* fn = forward ? (const void*)y_fwd_1024_persist_kernel<H16> : (const void*)y_inv_1024_persist_kernel<H16>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)YP_SMEM);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, YP_SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // every CTA resident at once: the grid is the resident count, or fewer when there are fewer lines
    const int total = g.nkx * 3 * g.nz;
    const int grid = (total + 7) / 8 < per_sm * nsm ? (total + 7) / 8 : per_sm * nsm;
    if (forward)
        y_fwd_1024_persist_kernel<H16><<<grid, 256, YP_SMEM, st>>>(g, X, Y16, tw, absmax, total);
    else
        y_inv_1024_persist_kernel<H16><<<grid, 256, YP_SMEM, st>>>(g, Y16, X, tw, absmax, total);
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

// max |Ms M| over the field (SoA [3][nz][ny][nx], Ms per cell from ms_map or
// the scalar ms) raised into *out, for the FP16 spectrum scale where the x pass
// is not the length-1024 one (which finds it while loading)
__global__ void absmax_kernel(const float* __restrict__ M, const float* __restrict__ ms_map, float ms, size_t ncell,
                              unsigned* __restrict__ out)
{
    float mx = 0.f;
    const size_t n3 = 3 * ncell;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x)
        mx = fmaxf(mx, fabsf(M[i] * (ms_map ? ms_map[i % ncell] : ms)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));
}

cudaError_t launch_absmax(const Geometry& g, const float* M, const float* ms_map, float ms, unsigned* out, int nsm,
                          cudaStream_t st)
{
    absmax_kernel<<<4 * nsm, 256, 0, st>>>(M, ms_map, ms, (size_t)g.nx * g.ny * g.nz, out);
    return cudaGetLastError();
}

template <bool H16>
static cudaError_t launch_y16(const Geometry& g, float2* X, void* Y16, const float2* tw, cudaStream_t st,
                              bool forward, const unsigned* absmax)
{
    if (y_persist_ok(g, X, Y16))
        return launch_y16_persist<H16>(g, X, (unsigned short*)Y16, tw, st, forward, absmax);
    const size_t smem = smem_1024<float>();
    const dim3 grid((3 * g.nz + 7) / 8, g.nkx);
    if (forward) {
        cudaError_t e =
            cudaFuncSetAttribute(y_fwd_1024_b16_kernel<H16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        y_fwd_1024_b16_kernel<H16><<<grid, 256, smem, st>>>(g, X, (unsigned short*)Y16, tw, absmax);
    } else {
        cudaError_t e =
            cudaFuncSetAttribute(y_inv_1024_b16_kernel<H16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        y_inv_1024_b16_kernel<H16><<<grid, 256, smem, st>>>(g, (const unsigned short*)Y16, X, tw, absmax);
    }
    return cudaGetLastError();
}

cudaError_t launch_y_1024_b16(const Geometry& g, float2* X, void* Y16, const float2* tw, cudaStream_t st,
                              bool forward, bool fp16, const unsigned* absmax)
{
    if (fp16) {
        if (!absmax) return cudaErrorInvalidValue;
        return launch_y16<true>(g, X, Y16, tw, st, forward, absmax);
    }
    return launch_y16<false>(g, X, Y16, tw, st, forward, nullptr);
}

cudaError_t upload_twiddles_fast() { return upload_small_twiddles_here(); }

#define FAST_INST(T)                                                                                              \
    template bool x1024_ok<T>(const Geometry&, int);                                                             \
    template bool y1024_ok<T>(const Geometry&, int);                                                             \
    template cudaError_t launch_x_r2c_1024<T>(const Geometry&, const T*, const T*, T, Cx<T>::t*, const Cx<T>::t*, \
                                              cudaStream_t, unsigned*);                                          \
    template cudaError_t launch_x_c2r_1024<T>(const Geometry&, const Cx<T>::t*, T*, const Cx<T>::t*, cudaStream_t); \
    template cudaError_t launch_y_1024<T>(const Geometry&, Cx<T>::t*, Cx<T>::t*, const Cx<T>::t*, cudaStream_t, bool);
FAST_INST(float)
FAST_INST(double)

}  // namespace boris
