// Mixed-precision z stage on the fifth-generation tensor cores (tcgen05 with
// accumulators in tensor memory): the zero-padded length-64 z transform of
// the pipelined convolution (Section 7) and its inverse as two dense real
// matrix products per tile, FP16 or BF16 operands, FP32 accumulation (the
// paper has no mixed-precision path; this is the reduced-precision variant of
// the split schedule's z convolution).
//
// A tile is 32 consecutive ky columns of one kx plane; operand column
// n = c * 32 + col (component c, column col), N = 96.  With the tile's data
// D[z][n] (z < nz <= 32, complex):
//   forward  Mh (128 x 96) = A1 (128 x 64) . [Re D; Im D]
//            rows 0..63 Re Mh[kz], rows 64..127 Im Mh[kz];
//            A1 = [[C, S], [-S, C]], C = cos, S = sin of 2 pi kz z / 64
//   multiply H[kz][(c, col)] = sum_d N_cd(kx, ky, kz) Mh[kz][(d, col)]; the
//            kernel spectrum is real, so the real and imaginary rows are
//            multiplied independently by the same 3 x 3 matrix
//   inverse  Hz (64 x 96) = A2 (64 x 128) . [Re H; Im H]
//            rows 0..31 Re Hz[z], rows 32..63 Im Hz[z]; A2 = [[C, -S], [S, C]]
// Scaling: each forward operand column is divided by its largest magnitude
// over z before the 16-bit cast, each inverse operand column by its largest
// magnitude over kz (a per-column slab scale, FP32), and both are undone in
// FP32 after the products.
//
// One CTA (8 warps, two CTAs per SM, persistent over tiles): the tile and the
// kernel block arrive by 2D tensor copies (the blocked kernel-spectrum copy of
// the residue-split z convolution) one tile ahead; the threads build the
// scaled 16-bit operand in shared memory; one thread issues the tcgen05.mma
// instructions (M = 128, N = 96, K = 16 each) into 96 tensor-memory columns
// and commits them to an mbarrier; every thread then reads its accumulator
// row (tensor-memory lane) with tcgen05.ld, so the 3 x 3 multiply needs no
// exchange between threads.  The inverse product reuses the same columns.
// Outputs go through shared memory and leave as 256-byte rows.
//
// Operand layout in shared memory (16-bit, K-major, no swizzle): element
// (row, k) at (row / 8) SBO + (k / 8) LBO + (row % 8) 16 + (k % 8) 2 bytes,
// i.e. 8 x 8 core matrices of 128 contiguous bytes.  The data operands use
// LBO = 160 / 144 so that the threads' stores fall in distinct banks.
//
// Every mbarrier wait is bounded (device timer); when one gives up, the CTA
// latches BORIS_ERR_TIMEOUT in *status, waits (bounded) for the copies and
// products it still has in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "boris_internal.cuh"
#include "bulk_async.cuh"

namespace boris {

namespace {

constexpr int Q5 = 32;              // ky columns per tile
constexpr int N5 = 96;              // operand columns: 3 components x 32
constexpr int T5 = 256;             // threads per CTA
constexpr int HZ5 = 32;             // z cells held (pz = 64)
constexpr int KBW5 = 34;            // blocked kernel row: ky' = 32 b .. 32 b + 32, one pad
constexpr int KROWS5 = (HZ5 + 1) * 3;
constexpr uint32_t TMEM_COLS = 128;  // power of two >= 96
constexpr int STATUS_TIMEOUT5 = -5;  // BORIS_ERR_TIMEOUT

constexpr uint32_t A1_LBO = 128, A1_SBO = 1024;  // 128 rows x 64 k
constexpr uint32_t A2_LBO = 128, A2_SBO = 2048;  // 64 rows x 128 k
constexpr uint32_t D1_LBO = 160, D1_SBO = 1280;  // 96 rows x 64 k
constexpr uint32_t D2_LBO = 144, D2_SBO = 2304;  // 96 rows x 128 k
constexpr int OUT_ROW = 65;                      // floats per (c, z) row of the output stage

// shared memory (bytes).  A2 comes first: an M = 128 product reads 128 rows,
// and rows 64..127 of A2's view fall on A1 (finite values, outputs ignored).
constexpr size_t OFF_A2 = 0;
constexpr size_t OFF_A1 = 16384;
constexpr size_t OFF_STAGE = 32768;                                          // [c][z][col] float2
constexpr size_t OFF_KST = OFF_STAGE + (size_t)3 * HZ5 * Q5 * 8;              // kernel block
constexpr size_t OFF_D = (OFF_KST + (size_t)KROWS5 * KBW5 * 8 + 127) / 128 * 128;  // D1, D2, output stage
constexpr size_t D_BYTES = (size_t)(N5 / 8) * D2_SBO;
constexpr size_t OFF_S1 = OFF_D + D_BYTES;  // [col][4] forward column scales (sign of ky fold in .y)
constexpr size_t OFF_S2 = OFF_S1 + Q5 * 16;  // [col][4] inverse column maxima (float bits)
constexpr size_t OFF_BAR = OFF_S2 + Q5 * 16;
constexpr size_t OFF_TSLOT = OFF_BAR + 3 * 8;
constexpr size_t SMEM5 = OFF_TSLOT + 16;
static_assert((size_t)(N5 / 8) * D1_SBO <= D_BYTES, "D1 fits the operand region");
static_assert((size_t)3 * HZ5 * OUT_ROW * 4 <= D_BYTES, "output stage fits the operand region");
static_assert(OFF_KST % 128 == 0 && OFF_STAGE % 128 == 0, "tensor-copy destinations");
static_assert(2 * (SMEM5 + 1024) <= 233472, "two CTAs per SM");

template <typename H> struct Cvt16;
template <> struct Cvt16<__half> {
    static constexpr uint32_t fmt = 0;
    static __device__ __forceinline__ uint32_t two(float a, float b)
    {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
    static __device__ __forceinline__ unsigned short one(float a) { return __half_as_ushort(__float2half_rn(a)); }
};
template <> struct Cvt16<__nv_bfloat16> {
    static constexpr uint32_t fmt = 1;
    static __device__ __forceinline__ uint32_t two(float a, float b)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
    static __device__ __forceinline__ unsigned short one(float a)
    {
        return __bfloat16_as_ushort(__float2bfloat16_rn(a));
    }
};

// shared-memory matrix descriptor: start, leading (k) and stride (row group)
// byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(const void* p, uint32_t lbo, uint32_t sbo)
{
    const uint32_t a = smem_u32(p);
    return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void umma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// the mbarrier's next phase completes when this thread's issued products have
__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// columns taddr + 16 c + j (c < 3 at stride 32, j < 16) of this thread's lane;
// the wait sits in the same statement so no use of v can move above it
__device__ __forceinline__ void tmem_ld48(uint32_t taddr, float (&v)[3][16])
{
    uint32_t r[48];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%48];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%49];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47}, [%50];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
        : "r"(taddr), "r"(taddr + 32), "r"(taddr + 64)
        : "memory");
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int j = 0; j < 16; j++) v[c][j] = __uint_as_float(r[16 * c + j]);
}

// cos and sin of 2 pi e / 64 from the plan's twiddles exp(-2 pi i e / lmax)
__device__ __forceinline__ float2 cs64(const float2* __restrict__ tw, int shz, int e)
{
    const float2 w = tw[(e & 63) << shz];
    return make_float2(w.x, -w.y);
}
// A1[m][k]: m = part * 64 + kz, k = kpart * 32 + z
__device__ __forceinline__ float a1_val(const float2* __restrict__ tw, int shz, int m, int k)
{
    const int part = m >> 6, kpart = k >> 5;
    const float2 cs = cs64(tw, shz, (m & 63) * (k & 31));
    return part == kpart ? cs.x : (part == 0 ? cs.y : -cs.y);
}
// A2[m][k]: m = part * 32 + z, k = kpart * 64 + kz
__device__ __forceinline__ float a2_val(const float2* __restrict__ tw, int shz, int m, int k)
{
    const int part = m >> 5, kpart = k >> 6;
    const float2 cs = cs64(tw, shz, (k & 63) * (m & 31));
    return part == kpart ? cs.x : (part == 0 ? -cs.y : cs.y);
}

__device__ __forceinline__ uint32_t op_off(int row, int k, uint32_t lbo, uint32_t sbo)
{
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * lbo + (uint32_t)(row & 7) * 16 + (uint32_t)(k & 7) * 2;
}

__device__ __forceinline__ float inv_max(uint32_t bits)
{
    const float m = __uint_as_float(bits);
    return m > 0.f ? 1.f / m : 0.f;
}

template <typename H>
__global__ void __launch_bounds__(T5, 2)
    z_conv_tc5_kernel(const __grid_constant__ CUtensorMap ymap, const __grid_constant__ CUtensorMap kmap, Geometry g,
                      int nkb, float2* __restrict__ Y, const float2* __restrict__ tw_g, int* __restrict__ status,
                      uint32_t extra_tx, unsigned long long limit_ns)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* A2 = smem_raw + OFF_A2;
    unsigned char* A1 = smem_raw + OFF_A1;
    float2* stage = reinterpret_cast<float2*>(smem_raw + OFF_STAGE);
    float2* kst = reinterpret_cast<float2*>(smem_raw + OFF_KST);
    unsigned char* Dm = smem_raw + OFF_D;
    float* S1 = reinterpret_cast<float*>(smem_raw + OFF_S1);
    uint32_t* S2 = reinterpret_cast<uint32_t*>(smem_raw + OFF_S2);
    uint64_t* fullY = reinterpret_cast<uint64_t*>(smem_raw + OFF_BAR);
    uint64_t* fullK = fullY + 1;
    uint64_t* mmab = fullY + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_raw + OFF_TSLOT);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nz = g.nz, lines = 3 * nz, py = g.py;
    const int nty = py / Q5, ntiles = g.nkx * nty, G = gridDim.x;
    const uint32_t ybytes = (uint32_t)lines * Q5 * sizeof(float2);
    constexpr uint32_t kbytes = (uint32_t)KROWS5 * KBW5 * sizeof(float2);
    // kind::f16, FP32 accumulator, A and B of type H, both K-major, N = 96, M = 128
    constexpr uint32_t IDESC = (1u << 4) | (Cvt16<H>::fmt << 7) | (Cvt16<H>::fmt << 10) |
                               ((uint32_t)(N5 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the DFT operands, once per CTA
    const int shz = g.lglmax - 6;
    for (int i = tid; i < 128 * 32; i += T5) {
        const int m = i >> 5, k = (i & 31) * 2;
        *reinterpret_cast<uint32_t*>(A1 + op_off(m, k, A1_LBO, A1_SBO)) =
            Cvt16<H>::two(a1_val(tw_g, shz, m, k), a1_val(tw_g, shz, m, k + 1));
    }
    for (int i = tid; i < 64 * 64; i += T5) {
        const int m = i >> 6, k = (i & 63) * 2;
        *reinterpret_cast<uint32_t*>(A2 + op_off(m, k, A2_LBO, A2_SBO)) =
            Cvt16<H>::two(a2_val(tw_g, shz, m, k), a2_val(tw_g, shz, m, k + 1));
    }
    if (tid == 0) {
        mbar_init(fullY, 1);
        mbar_init(fullK, 1);
        mbar_init(mmab, 1);
        fence_mbar_init();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;

    auto load_y = [&](int t, uint32_t extra) {
        const int kx = t / nty, ky0 = (t - kx * nty) * Q5;
        mbar_arrive_expect_tx(fullY, ybytes + extra);
        for (int c = 0; c < 3; c++) tma_load_2d(stage + c * HZ5 * Q5, &ymap, ky0, kx * lines + c * nz, fullY);
    };
    // the kernel block of tile t: b = ky0 / 32 below the fold, (py - ky0 - 31) / 32 above it
    auto load_k = [&](int t) {
        const int kx = t / nty, ky0 = (t - kx * nty) * Q5;
        const int b = ky0 >= py / 2 ? (py - ky0 - (Q5 - 1)) / 32 : ky0 / 32;
        mbar_arrive_expect_tx(fullK, kbytes);
        tma_load_2d(kst, &kmap, 0, (kx * nkb + b) * KROWS5, fullK);
    };
    // copies and product groups issued by thread 0 (for the drain after a timeout)
    int ny_issued = 0, nk_issued = 0, nm_issued = 0;
    if (tid == 0 && (int)blockIdx.x < ntiles) {
        load_y(blockIdx.x, extra_tx);
        load_k(blockIdx.x);
        ny_issued = nk_issued = 1;
    }

    // this thread's accumulator row (tensor-memory lane) and its columns
    const int q = warp & 3, wg = warp >> 2;
    const int r = 32 * q + lane;
    const int kz = r & 63;
    const int kzf = kz <= HZ5 ? kz : 64 - kz;
    const float sz = kz > HZ5 ? -1.f : 1.f;  // xz and yz are odd in kz
    const uint32_t trow = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * wg);
    float* outs = reinterpret_cast<float*>(Dm);

    bool failed = false;
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += G, k++) {
        const int kx = t / nty, ky0 = (t - kx * nty) * Q5;
        const bool more = t + G < ntiles;
        const bool fy = ky0 >= py / 2;  // ky beyond the fold: xy and yz change sign
        {
            const bool ok = mbar_wait_bounded(fullY, k & 1, limit_ns);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
        }
        // scaled 16-bit forward operand D1[n][k]: k < 32 Re z, k >= 32 Im z;
        // thread pair (2 n, 2 n + 1) takes z < 16 and z >= 16 of column n
        if (tid < 2 * N5) {
            const int n = tid >> 1, zh = tid & 1, c = n >> 5, col = n & 31;
            const float2* src = stage + (c * HZ5 + 16 * zh) * Q5 + col;
            float2 a[16];
            float mx = 0.f;
#pragma unroll
            for (int i = 0; i < 16; i++) {
                a[i] = 16 * zh + i < nz ? src[i * Q5] : make_float2(0.f, 0.f);
                mx = fmaxf(mx, fmaxf(fabsf(a[i].x), fabsf(a[i].y)));
            }
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
            const float s = mx > 0.f ? 1.f / mx : 0.f;
            unsigned char* row = Dm + (n >> 3) * D1_SBO + (n & 7) * 16;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                uint4 re, im;
                re.x = Cvt16<H>::two(a[8 * h + 0].x * s, a[8 * h + 1].x * s);
                re.y = Cvt16<H>::two(a[8 * h + 2].x * s, a[8 * h + 3].x * s);
                re.z = Cvt16<H>::two(a[8 * h + 4].x * s, a[8 * h + 5].x * s);
                re.w = Cvt16<H>::two(a[8 * h + 6].x * s, a[8 * h + 7].x * s);
                im.x = Cvt16<H>::two(a[8 * h + 0].y * s, a[8 * h + 1].y * s);
                im.y = Cvt16<H>::two(a[8 * h + 2].y * s, a[8 * h + 3].y * s);
                im.z = Cvt16<H>::two(a[8 * h + 4].y * s, a[8 * h + 5].y * s);
                im.w = Cvt16<H>::two(a[8 * h + 6].y * s, a[8 * h + 7].y * s);
                *reinterpret_cast<uint4*>(row + (2 * zh + h) * D1_LBO) = re;
                *reinterpret_cast<uint4*>(row + (4 + 2 * zh + h) * D1_LBO) = im;
            }
            // the y component carries the sign of the ky fold (see the multiply)
            if (zh == 0) S1[col * 4 + c] = (c == 1 && fy) ? -mx : mx;
        }
        if (tid < 4 * Q5) S2[tid] = 0u;
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            if (more) {
                fence_proxy_async_smem();
                load_y(t + G, 0);
                ny_issued++;
            }
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 4; ks++)
                umma_f16(tbase, sdesc(A1 + ks * 2 * A1_LBO, A1_LBO, A1_SBO), sdesc(Dm + ks * 2 * D1_LBO, D1_LBO, D1_SBO),
                         IDESC, ks > 0);
            umma_commit(mmab);
            nm_issued++;
        }
        {
            const bool ok = mbar_wait_bounded(fullK, k & 1, limit_ns) && mbar_wait_bounded(mmab, 0, limit_ns);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
        }
        tc_fence_after();
        float h[3][16];
        tmem_ld48(trow, h);
        // kernel multiply at (kz, ky) for this row's 16 columns.  With
        // M1' = s_y M1 (in the y column scale) and M2' = s_z M2:
        //   H0 = xx M0 + xy' M1' + xz' M2',  s_y H1 = xy' M0 + yy M1' + yz' M2',
        //   s_z H2 = xz' M0 + yz' M1' + zz M2'   (primes: the stored octant values)
        {
            const float2* kp = kst + kzf * 3 * KBW5;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int col = 16 * wg + j;
                const int e = fy ? 32 - col : col;
                const float4 s = *reinterpret_cast<const float4*>(S1 + col * 4);
                const float m0 = h[0][j] * s.x, m1 = h[1][j] * s.y, m2 = h[2][j] * (s.z * sz);
                const float2 p0 = kp[e], p1 = kp[KBW5 + e], p2 = kp[2 * KBW5 + e];
                h[0][j] = p0.x * m0 + p1.y * m1 + p2.x * m2;
                h[1][j] = p1.y * m0 + p0.y * m1 + p2.y * m2;
                h[2][j] = p2.x * m0 + p2.y * m1 + p1.x * m2;
            }
        }
        // largest magnitude of each operand column over the 128 rows
        {
            uint32_t sel0 = 0, sel1 = 0;
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int i = 16 * c + j;
                    const uint32_t u = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(h[c][j])));
                    if (lane == (i & 31)) {
                        if (i < 32) sel0 = u;
                        else sel1 = u;
                    }
                }
            atomicMax(S2 + (16 * wg + (lane & 15)) * 4 + (lane >> 4), sel0);
            if (lane < 16) atomicMax(S2 + (16 * wg + lane) * 4 + 2, sel1);
        }
        tc_fence_before();
        __syncthreads();
        if (tid == 0 && more) {
            fence_proxy_async_smem();
            load_k(t + G);
            nk_issued++;
        }
        // scaled 16-bit inverse operand D2[n][k = r]; s_z H2 is turned back into H2 here
        {
            unsigned short* base = reinterpret_cast<unsigned short*>(Dm + (r >> 3) * D2_LBO + (r & 7) * 2);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int col = 16 * wg + j;
                const uint4 mb = *reinterpret_cast<const uint4*>(S2 + col * 4);
                const float i0 = inv_max(mb.x), i1 = inv_max(mb.y), i2 = inv_max(mb.z) * sz;
                const int n0 = col, n1 = 32 + col, n2 = 64 + col;
                base[((n0 >> 3) * D2_SBO + (n0 & 7) * 16) / 2] = Cvt16<H>::one(h[0][j] * i0);
                base[((n1 >> 3) * D2_SBO + (n1 & 7) * 16) / 2] = Cvt16<H>::one(h[1][j] * i1);
                base[((n2 >> 3) * D2_SBO + (n2 & 7) * 16) / 2] = Cvt16<H>::one(h[2][j] * i2);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 8; ks++)
                umma_f16(tbase, sdesc(A2 + ks * 2 * A2_LBO, A2_LBO, A2_SBO), sdesc(Dm + ks * 2 * D2_LBO, D2_LBO, D2_SBO),
                         IDESC, ks > 0);
            umma_commit(mmab);
            nm_issued++;
        }
        {
            const bool ok = mbar_wait_bounded(mmab, 1, limit_ns);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
        }
        tc_fence_after();
        // rows r < 64: Re (r < 32) and Im (r >= 32) of z = r mod 32; the y
        // component takes back the sign of the ky fold
        if (q < 2) {
            float o[3][16];
            tmem_ld48(trow, o);
            const int z = r & 31, part = r >> 5;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int col = 16 * wg + j;
                const uint4 mb = *reinterpret_cast<const uint4*>(S2 + col * 4);
                const float s1 = fy ? -__uint_as_float(mb.y) : __uint_as_float(mb.y);
                outs[(0 * HZ5 + z) * OUT_ROW + 2 * col + part] = o[0][j] * __uint_as_float(mb.x);
                outs[(1 * HZ5 + z) * OUT_ROW + 2 * col + part] = o[1][j] * s1;
                outs[(2 * HZ5 + z) * OUT_ROW + 2 * col + part] = o[2][j] * __uint_as_float(mb.z);
            }
        }
        tc_fence_before();
        __syncthreads();
        {
            float2* dst = Y + (size_t)kx * lines * py + ky0;
            for (int i = tid; i < lines * Q5; i += T5) {
                const int line = i >> 5, col = i & 31;
                const int c = line / nz, z = line - c * nz;
                const float* src = outs + (c * HZ5 + z) * OUT_ROW + 2 * col;
                dst[(size_t)line * py + col] = make_float2(src[0], src[1]);
            }
        }
        // the output stage is rewritten only after the next tile's first barrier
    }
    if (failed && tid == 0) {
        atomicCAS(status, 0, STATUS_TIMEOUT5);
        // let the copies and products still in flight land (bounded)
        if (ny_issued > 0) mbar_wait_bounded(fullY, (ny_issued - 1) & 1, limit_ns);
        if (nk_issued > 0) mbar_wait_bounded(fullK, (nk_issued - 1) & 1, limit_ns);
        if (nm_issued > 0) mbar_wait_bounded(mmab, (nm_issued - 1) & 1, limit_ns);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
    }
}

template <typename H>
cudaError_t launch5(const CUtensorMap& ymap, const CUtensorMap& kmap, const Geometry& g, float2* Y, const float2* tw,
                    int* status, uint32_t extra_tx, unsigned long long limit_ns, int nsm, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(z_conv_tc5_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM5);
    if (e != cudaSuccess) return e;
    const int ntiles = g.nkx * (g.py / Q5);
    const int grid = std::min(ntiles, 2 * nsm);
    z_conv_tc5_kernel<H><<<grid, T5, SMEM5, st>>>(ymap, kmap, g, zconv_res_nkb(g), Y, tw, status, extra_tx, limit_ns);
    return cudaGetLastError();
}

}  // namespace

bool zconv_tc5_supported(const Geometry& g, int max_smem)
{
    // pz = 64 (17 <= nz <= 32); py >= 64 so that a tile lies wholly on one side
    // of the ky fold; the blocked kernel copy of the residue-split stage
    return g.pz == 2 * HZ5 && g.nz >= 17 && g.nz <= HZ5 && g.py >= 2 * Q5 && g.py % Q5 == 0 &&
           g.krow == ((HZ5 + 1) * 6 + 3) / 4 * 4 && SMEM5 <= (size_t)max_smem && g.lglmax >= 6;
}

cudaError_t launch_zconv_tc5(const void* ymap_p, const void* kmap_p, const Geometry& g, float2* Y, const float2* tw,
                             bool bf16, int* status, uint32_t extra_tx, unsigned long long limit_ns, int nsm,
                             cudaStream_t st)
{
    const CUtensorMap& ymap = *reinterpret_cast<const CUtensorMap*>(ymap_p);
    const CUtensorMap& kmap = *reinterpret_cast<const CUtensorMap*>(kmap_p);
    return bf16 ? launch5<__nv_bfloat16>(ymap, kmap, g, Y, tw, status, extra_tx, limit_ns, nsm, st)
                : launch5<__half>(ymap, kmap, g, Y, tw, status, extra_tx, limit_ns, nsm, st);
}

}  // namespace boris
