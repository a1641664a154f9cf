// Mixed-precision z stage on the tensor cores (FP16 or BF16 operands, FP32
// accumulation): the zero-padded length-64 z transform of the pipelined
// convolution (Section 7) recast as two dense real matrix products per tile
// of QC ky columns of one kx plane (the paper has no mixed-precision path;
// this is the reduced-precision variant of the split schedule's z_conv).
//
// With n = (component, column) and the data D[z][n] (z < nz <= 32, complex):
//   forward  Mh[kz][n] = sum_z exp(-2 pi i kz z / 64) D[z][n],   kz < 64
//   multiply Hh[kz][n] = sum_d N_cd(kx, ky, kz) Mh[kz][(d, column)]
//   inverse  Hz[z][n]  = sum_kz exp(+2 pi i kz z / 64) Hh[kz][n],  z < nz
// In real form the forward product is A1 (128 x 64) . [Re D; Im D] (64 x N)
// with A1 = [[C, S], [-S, C]] (C = cos, S = sin of 2 pi kz z / 64), and the
// inverse A2 (64 x 128) . [Re Hh; Im Hh] (128 x N) with A2 = [[C, -S], [S, C]].
// Each operand column n is scaled by its largest magnitude before the cast
// to 16 bits (a per-slab scale, one per (kx, ky, component)) and the products
// are scaled back in FP32.  mma.sync m16n8k16 (row.col) keeps every fragment
// in registers; warp w owns M tiles {w, w + 4} of the forward product - the
// real and imaginary rows of the same 16 wavenumbers - and therefore holds
// all three components of its columns for the kernel multiply.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "boris_internal.cuh"

namespace boris {

namespace {
constexpr int TQC = 16;           // ky columns per CTA
constexpr int TN = 3 * TQC;       // operand columns (component, column)
constexpr int TNT = TN / 8;       // n tiles of 8
constexpr int K1 = 64;            // forward contraction: Re and Im of z < 32
constexpr int K1S = K1 + 8;       // row stride (16-bit units) of the forward operand
constexpr int K2 = 128;           // inverse contraction: Re and Im of kz < 64
constexpr int K2S = K2 + 8;
constexpr int ZMAX = 32;
constexpr int ZS = ZMAX + 1;      // staging stride per column (odd: no bank conflicts)

template <typename H> struct Pack;
template <> struct Pack<__half> {
    static __device__ __forceinline__ unsigned two(float a, float b)
    {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<unsigned*>(&h);
    }
    static __device__ __forceinline__ __half one(float a) { return __float2half_rn(a); }
};
template <> struct Pack<__nv_bfloat16> {
    static __device__ __forceinline__ unsigned two(float a, float b)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<unsigned*>(&h);
    }
    static __device__ __forceinline__ __nv_bfloat16 one(float a) { return __float2bfloat16_rn(a); }
};

template <typename H>
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    if constexpr (sizeof(H) == 2 && std::is_same<H, __half>::value) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// cos and sin of 2 pi e / 64 from the twiddle table w64[e] = exp(-2 pi i e / 64)
__device__ __forceinline__ float cos64(const float2* w, int e) { return w[e & 63].x; }
__device__ __forceinline__ float sin64(const float2* w, int e) { return -w[e & 63].y; }

// Forward operand A1[r][k]: r = part * 64 + kz, k = kpart * 32 + z.
__device__ __forceinline__ float a1_at(const float2* w, int r, int k)
{
    const int part = r >> 6, kz = r & 63, kpart = k >> 5, z = k & 31;
    const int e = kz * z;
    if (part == kpart) return cos64(w, e);
    return part == 0 ? sin64(w, e) : -sin64(w, e);
}
// Inverse operand A2[r][k]: r = part * 32 + z, k = kpart * 64 + kz.
__device__ __forceinline__ float a2_at(const float2* w, int r, int k)
{
    const int part = r >> 5, z = r & 31, kpart = k >> 6, kz = k & 63;
    const int e = kz * z;
    if (part == kpart) return cos64(w, e);
    return part == 0 ? -sin64(w, e) : sin64(w, e);
}

// A fragment of m16n8k16 (row-major 16 x 16 tile at (r0, k0)) built by f(r, k).
template <typename H, typename F>
__device__ __forceinline__ void a_frag(unsigned (&a)[4], int r0, int k0, F f)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    a[0] = Pack<H>::two(f(r0 + g, k0 + 2 * t), f(r0 + g, k0 + 2 * t + 1));
    a[1] = Pack<H>::two(f(r0 + g + 8, k0 + 2 * t), f(r0 + g + 8, k0 + 2 * t + 1));
    a[2] = Pack<H>::two(f(r0 + g, k0 + 2 * t + 8), f(r0 + g, k0 + 2 * t + 9));
    a[3] = Pack<H>::two(f(r0 + g + 8, k0 + 2 * t + 8), f(r0 + g + 8, k0 + 2 * t + 9));
}
}  // namespace

template <typename H>
__global__ void __launch_bounds__(128) z_conv_tc_kernel(Geometry g, float2* __restrict__ Y, const float* __restrict__ K,
                                                        const float2* __restrict__ tw_g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nz = g.nz, lines = 3 * nz, py = g.py;
    const int kx = blockIdx.y, ky0 = blockIdx.x * TQC;
    const int ncol = min(TQC, py - ky0);
    const int KS = g.krow + 1;
    float2* w64 = reinterpret_cast<float2*>(smem_raw);            // [64]
    float* cmax1 = reinterpret_cast<float*>(w64 + 64);             // [TN]
    float* cmax2 = cmax1 + TN;                                     // [TN]
    float2* stage = reinterpret_cast<float2*>(cmax2 + TN);         // [TN][ZS] (in) / [3][nz][TQC] (out)
    H* D1 = reinterpret_cast<H*>(stage + TN * ZS);                 // [TN][K1S]
    H* D2 = D1 + TN * K1S;                                         // [TN][K2S]
    float* Ks = reinterpret_cast<float*>(D2 + TN * K2S);           // [TQC][KS]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, gq = lane >> 2, tq = lane & 3;
    const int shz = g.lglmax - 6;
    for (int i = tid; i < 64; i += 128) w64[i] = tw_g[i << shz];
    for (int i = tid; i < 2 * TN; i += 128) cmax1[i] = 0.f;  // cmax1 and cmax2
    for (int i = tid; i < TN * ZS; i += 128) stage[i] = make_float2(0.f, 0.f);
    __syncthreads();
    // ---- stage the columns Y[kx][c][z][ky0 + col] and the kernel rows -------
    const float2* ysrc = Y + (size_t)kx * lines * py + ky0;
    staged_loop<128, float2>(lines * TQC, [&](int i) {
        const int line = i / TQC, col = i % TQC;
        return col < ncol ? ysrc[(size_t)line * py + col] : make_float2(0.f, 0.f);
    }, [&](int i, float2 v) {
        const int line = i / TQC, col = i % TQC;
        const int n = (line / nz) * TQC + col;
        stage[n * ZS + line % nz] = v;
        atomicMax(reinterpret_cast<unsigned*>(cmax1 + n), __float_as_uint(fmaxf(fabsf(v.x), fabsf(v.y))));
    });
    const float* Kx = K + (size_t)kx * g.kyh * g.krow;
    const int vrow = g.krow / 4;
    staged_loop<128, float4>(ncol * vrow, [&](int i) {
        const int col = i / vrow, o = i % vrow;
        const int ky = ky0 + col;
        const int kyf = ky > py / 2 ? py - ky : ky;
        return reinterpret_cast<const float4*>(Kx + (size_t)kyf * g.krow)[o];
    }, [&](int i, float4 v) {
        float* d = Ks + (i / vrow) * KS + (i % vrow) * 4;
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    });
    for (int i = ncol * g.krow + tid; i < TQC * g.krow; i += 128) Ks[(i / g.krow) * KS + i % g.krow] = 0.f;
    __syncthreads();
    // ---- scaled 16-bit forward operand D1[n][k]: k < 32 Re z, k >= 32 Im z --
    for (int i = tid; i < TN * ZMAX / 2; i += 128) {
        const int n = i / (ZMAX / 2), z2 = 2 * (i % (ZMAX / 2));
        const float s = cmax1[n] > 0.f ? 1.f / cmax1[n] : 0.f;
        const float2 a = stage[n * ZS + z2], b = stage[n * ZS + z2 + 1];
        *reinterpret_cast<unsigned*>(D1 + n * K1S + z2) = Pack<H>::two(a.x * s, b.x * s);
        *reinterpret_cast<unsigned*>(D1 + n * K1S + 32 + z2) = Pack<H>::two(a.y * s, b.y * s);
    }
    __syncthreads();
    // ---- forward product: warp w, M tiles w (Re rows) and w + 4 (Im rows) ---
    float acc[2][TNT][4];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int nt = 0; nt < TNT; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) acc[m][nt][e] = 0.f;
#pragma unroll
    for (int kt = 0; kt < K1 / 16; kt++) {
        unsigned a0[4], a1[4];
        a_frag<H>(a0, 16 * warp, 16 * kt, [&](int r, int k) { return a1_at(w64, r, k); });
        a_frag<H>(a1, 64 + 16 * warp, 16 * kt, [&](int r, int k) { return a1_at(w64, r, k); });
#pragma unroll
        for (int nt = 0; nt < TNT; nt++) {
            const H* bp = D1 + (nt * 8 + gq) * K1S + 16 * kt + 2 * tq;
            const unsigned b0 = *reinterpret_cast<const unsigned*>(bp);
            const unsigned b1 = *reinterpret_cast<const unsigned*>(bp + 8);
            mma16816<H>(acc[0][nt], a0, b0, b1);
            mma16816<H>(acc[1][nt], a1, b0, b1);
        }
    }
    // ---- kernel multiply in registers --------------------------------------
    // accumulator element e of n tile nt: row kz = 16 warp + gq + 8 (e >> 1),
    // column n = 8 nt + 2 tq + (e & 1); n tiles 2c, 2c + 1 hold component c.
    const int pz = 64;
    float lmax[TNT][2];
#pragma unroll
    for (int nt = 0; nt < TNT; nt++) lmax[nt][0] = lmax[nt][1] = 0.f;
#pragma unroll
    for (int half = 0; half < 2; half++) {      // columns 8 half + 2 tq + j
#pragma unroll
        for (int hi = 0; hi < 2; hi++) {        // row gq or gq + 8
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const int e = 2 * hi + j;
                const int kz = 16 * warp + gq + 8 * hi;
                const int col = 8 * half + 2 * tq + j;
                float mre[3], mim[3];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const int nt = 2 * c + half;
                    const float s = cmax1[8 * nt + 2 * tq + j];
                    mre[c] = acc[0][nt][e] * s;
                    mim[c] = acc[1][nt][e] * s;
                }
                const int ky = ky0 + col;
                const bool fy = ky > py / 2, fz = kz > pz / 2;
                const int kzf = fz ? pz - kz : kz;
                const float* kr = Ks + col * KS + kzf * 6;
                const float sxy = fy ? -1.f : 1.f, sxz = fz ? -1.f : 1.f;
                const float kxx = kr[0], kyy = kr[1], kzz = kr[2];
                const float kxy = sxy * kr[3], kxz = sxz * kr[4], kyz = sxy * sxz * kr[5];
                const float hre[3] = {kxx * mre[0] + kxy * mre[1] + kxz * mre[2],
                                      kxy * mre[0] + kyy * mre[1] + kyz * mre[2],
                                      kxz * mre[0] + kyz * mre[1] + kzz * mre[2]};
                const float him[3] = {kxx * mim[0] + kxy * mim[1] + kxz * mim[2],
                                      kxy * mim[0] + kyy * mim[1] + kyz * mim[2],
                                      kxz * mim[0] + kyz * mim[1] + kzz * mim[2]};
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const int nt = 2 * c + half;
                    acc[0][nt][e] = hre[c];
                    acc[1][nt][e] = him[c];
                    lmax[nt][j] = fmaxf(lmax[nt][j], fmaxf(fabsf(hre[c]), fabsf(him[c])));
                }
            }
        }
    }
#pragma unroll
    for (int nt = 0; nt < TNT; nt++)
#pragma unroll
        for (int j = 0; j < 2; j++) atomicMax(reinterpret_cast<unsigned*>(cmax2 + 8 * nt + 2 * tq + j), __float_as_uint(lmax[nt][j]));
    __syncthreads();
    // ---- scaled 16-bit inverse operand D2[n][k]: k < 64 Re kz, k >= 64 Im kz -
#pragma unroll
    for (int nt = 0; nt < TNT; nt++)
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int n = 8 * nt + 2 * tq + (e & 1);
            const int kz = 16 * warp + gq + 8 * (e >> 1);
            const float s = cmax2[n] > 0.f ? 1.f / cmax2[n] : 0.f;
            D2[n * K2S + kz] = Pack<H>::one(acc[0][nt][e] * s);
            D2[n * K2S + 64 + kz] = Pack<H>::one(acc[1][nt][e] * s);
        }
    __syncthreads();
    // ---- inverse product: warp w, M tiles (w & 1) (Re z) and 2 + (w & 1) (Im z),
    //      n tiles 3 (w >> 1) .. 3 (w >> 1) + 2
    float o[2][3][4];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int q = 0; q < 3; q++)
#pragma unroll
            for (int e = 0; e < 4; e++) o[m][q][e] = 0.f;
    const int mt = warp & 1, nt0 = 3 * (warp >> 1);
#pragma unroll
    for (int kt = 0; kt < K2 / 16; kt++) {
        unsigned a0[4], a1[4];
        a_frag<H>(a0, 16 * mt, 16 * kt, [&](int r, int k) { return a2_at(w64, r, k); });
        a_frag<H>(a1, 32 + 16 * mt, 16 * kt, [&](int r, int k) { return a2_at(w64, r, k); });
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const H* bp = D2 + ((nt0 + q) * 8 + gq) * K2S + 16 * kt + 2 * tq;
            const unsigned b0 = *reinterpret_cast<const unsigned*>(bp);
            const unsigned b1 = *reinterpret_cast<const unsigned*>(bp + 8);
            mma16816<H>(o[0][q], a0, b0, b1);
            mma16816<H>(o[1][q], a1, b0, b1);
        }
    }
    // ---- unscale, stage as [line][col], store coalesced ------------------------
    float2* out = stage;  // [3 nz][TQC]
#pragma unroll
    for (int q = 0; q < 3; q++)
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int n = 8 * (nt0 + q) + 2 * tq + (e & 1);
            const int z = 16 * mt + gq + 8 * (e >> 1);
            const float s = cmax2[n];
            if (z < nz) out[((n / TQC) * nz + z) * TQC + n % TQC] = make_float2(o[0][q][e] * s, o[1][q][e] * s);
        }
    __syncthreads();
    float2* ydst = Y + (size_t)kx * lines * py + ky0;
    for (int i = tid; i < lines * TQC; i += 128) {
        const int line = i / TQC, col = i % TQC;
        if (col < ncol) ydst[(size_t)line * py + col] = out[i];
    }
}

static size_t zconv_tc_smem(const Geometry& g)
{
    return 64 * sizeof(float2) + 2 * TN * sizeof(float) + (size_t)TN * ZS * sizeof(float2) +
           (size_t)TN * (K1S + K2S) * 2 + (size_t)TQC * (g.krow + 1) * sizeof(float);
}

bool zconv_tc_supported(const Geometry& g) { return g.pz == 64 && g.nz <= ZMAX && g.nz >= 17; }

cudaError_t launch_zconv_tc(const Geometry& g, float2* Y, const float* K, const float2* tw, bool bf16, cudaStream_t st)
{
    const size_t smem = zconv_tc_smem(g);
    const dim3 grid((g.py + TQC - 1) / TQC, g.nkx);
    cudaError_t e;
    if (bf16) {
        e = cudaFuncSetAttribute(z_conv_tc_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        z_conv_tc_kernel<__nv_bfloat16><<<grid, 128, smem, st>>>(g, Y, K, tw);
    } else {
        e = cudaFuncSetAttribute(z_conv_tc_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        z_conv_tc_kernel<__half><<<grid, 128, smem, st>>>(g, Y, K, tw);
    }
    return cudaGetLastError();
}

}  // namespace boris
