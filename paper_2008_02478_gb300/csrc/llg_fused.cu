// The inverse x transform of the demagnetising convolution fused with the RK4
// stage (FP32, transform length px = 1024, so nx in 257..512).
//
// One CTA owns the FY rows y0..y0+FY-1 of plane z for all three components:
// it stages their x half spectra (513 bins x 3 FY rows) in shared memory,
// runs 3 FY / 2 packed inverse transforms (two real rows per complex line,
// one line per warp, warp_fft.cuh), keeps the resulting H_d rows in shared
// memory and applies the RK4 stage (Section 2; per-cell fields of Table 1,
// Eq. 1 in Landau-Lifshitz form) to its FY x nx cells.  H_d never travels
// through HBM: per stage this saves writing and re-reading 24 bytes a cell.
#include "boris_internal.cuh"
#include "llg_cell.cuh"
#include "llg_kernels.cuh"
#include "warp_fft.cuh"

namespace boris {

namespace {

constexpr int FY = 8;           // rows per component and CTA
constexpr int FR = 3 * FY;      // rows per CTA (component-major: r = c FY + t)
constexpr int FL = FR / 2;      // packed lines = warps
constexpr int FT = 32 * FL;     // threads
constexpr int FS = FR + 1;      // staging stride in complex (odd: lanes walking kx hit distinct banks)
constexpr int FREG = 1025;      // per-warp transpose tile stride (complex)
constexpr int HROW = 512;       // H_d row stride in shared memory (floats)
constexpr int FREGIONS = 513 * FS > FL * FREG ? 513 * FS : FL * FREG;
static_assert(FR * HROW <= 2 * FREGIONS, "H_d rows must fit in the staging area");

constexpr size_t fused_smem() { return ((size_t)TW1024_SLOTS + FREGIONS) * sizeof(float2); }

__global__ void __launch_bounds__(FT, 2)
    x_c2r_rk4_kernel(Geometry g, const float2* __restrict__ X, const float2* __restrict__ tw_g, LLGArgs<float> a,
                     int s, const float* __restrict__ ms, float* __restrict__ m0, float* __restrict__ acc,
                     float* __restrict__ mnext)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tws = reinterpret_cast<float2*>(smem_raw);
    float2* reg = tws + TW1024_SLOTS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0 = blockIdx.x * FY, z = blockIdx.y;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    load_tw1024(tws, tw_g, g.lmax);
    // stage S[kx][c FY + t] = X[kx][c][z][y0 + t]: each group of FY
    // consecutive threads reads one FY-element run of a spectrum column
    float2* S = reg;
    staged_loop<FT, float2>(3 * 513 * FY, [&](int i) {
        const int t = i % FY, q = i / FY;
        const int c = q / 513, kx = q - c * 513;
        return y0 + t < ny ? X[(((size_t)kx * 3 + c) * nz + z) * ny + y0 + t] : float2{0.f, 0.f};
    }, [&](int i, float2 v) {
        const int t = i % FY, q = i / FY;
        const int c = q / 513, kx = q - c * 513;
        S[kx * FS + c * FY + t] = v;
    });
    __syncthreads();
    // line w carries row w (real part) and row w + FL (imaginary part):
    // Z_k = A_k + i B_k with A, B the Hermitian half spectra of the two rows
    float2 v[32];
#pragma unroll
    for (int d = 0; d < 32; d++) {
        const int k = lane + 32 * d;
        const bool upper = k > 512;
        const int kx = upper ? 1024 - k : k;
        float2 A = S[kx * FS + warp], B = S[kx * FS + warp + FL];
        if (kx == 0 || kx == 512) {  // DC and Nyquist bins of a real signal are real
            A.y = 0.f;
            B.y = 0.f;
        }
        if (upper) {
            A.y = -A.y;
            B.y = -B.y;
        }
        v[brev5(d)] = float2{A.x - B.y, A.y + B.x};
    }
    __syncthreads();  // the staging area becomes the warps' transpose tiles
    warp_fft1024_inv(v, reg + warp * FREG, tws);
    __syncthreads();  // and then the H_d rows
    float* Hs = reinterpret_cast<float*>(reg);
#pragma unroll
    for (int q = 0; q < 16; q++) {
        const int x = 32 * q + lane;
        Hs[warp * HROW + x] = v[q].x;
        Hs[(warp + FL) * HROW + x] = v[q].y;
    }
    __syncthreads();
    const int rows = ny - y0 < FY ? ny - y0 : FY;
    for (int j = threadIdx.x; j < rows * nx; j += FT) {
        const int t = j / nx, x = j - t * nx;
        const int y = y0 + t;
        const size_t i = ((size_t)z * ny + y) * nx + x;
        const float hd[3] = {Hs[t * HROW + x], Hs[(FY + t) * HROW + x], Hs[(2 * FY + t) * HROW + x]};
        float m[3], k[3];
        cell_rhs(a, ms, hd, i, x, y, z, m, k);
        rk4_combine(a, s, i, m, k, m0, acc, mnext);
    }
}

}  // namespace

bool x_c2r_rk4_ok(const Geometry& g, int max_smem)
{
    return g.px == 1024 && g.nx <= 512 && fused_smem() <= (size_t)max_smem;
}

cudaError_t launch_x_c2r_rk4(const Geometry& g, const float2* X, const float2* tw, const LLGArgs<float>& a, int s,
                             const float* ms, float* m0, float* acc, float* mnext, cudaStream_t st)
{
    const size_t smem = fused_smem();
    cudaError_t e = cudaFuncSetAttribute(x_c2r_rk4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    x_c2r_rk4_kernel<<<dim3((g.ny + FY - 1) / FY, g.nz), FT, smem, st>>>(g, X, tw, a, s, ms, m0, acc, mnext);
    return cudaGetLastError();
}

}  // namespace boris
