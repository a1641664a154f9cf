// Mixed-precision z stage on the fifth-generation tensor cores (tcgen05 with
// accumulators in tensor memory): the zero-padded length-64 z transform of
// the pipelined convolution (Section 7) and its inverse as two dense real
// matrix products per tile, FP16 or BF16 operands, FP32 accumulation (the
// paper has no mixed-precision path; this is the reduced-precision variant of
// the split schedule's z convolution).
//
// A tile is 16 consecutive ky columns of one kx plane; operand column
// n = c * 16 + col (component c, column col), N = 48.  With the tile's data
// D[z][n] (z < nz <= 32, complex):
//   forward  Mh (128 x 48) = A1 (128 x 64) . [Re D; Im D]
//            rows 0..63 Re Mh[kz], rows 64..127 Im Mh[kz];
//            A1 = [[C, S], [-S, C]], C = cos, S = sin of 2 pi kz z / 64
//   multiply H[kz][(c, col)] = sum_d N_cd(kx, ky, kz) Mh[kz][(d, col)]; the
//            kernel spectrum is real, so the real and imaginary rows are
//            multiplied independently by the same 3 x 3 matrix
//   inverse  Hz (64 x 48) = A2 (64 x 128) . [Re H; Im H]
//            rows 0..31 Re Hz[z], rows 32..63 Im Hz[z]; A2 = [[C, -S], [S, C]]
//            = A1 transposed, so the inverse reads A1's storage as an MN-major
//            operand
// Scaling: each forward operand column is multiplied by the power of two that
// brings its largest magnitude over z into [1, 2) before the 16-bit cast, each
// inverse operand column likewise for its largest magnitude over kz (a per-
// column slab scale, exact), and both are undone in FP32 after the products.
//
// One CTA (4 warps, 55 KB of shared memory, four CTAs per SM, persistent over
// tiles): the tile and its kernel rows arrive by 2D tensor copies (the blocked
// kernel-spectrum copy of the residue-split z convolution) one tile ahead; the
// threads build the scaled 16-bit operand in shared memory; one thread issues
// the tcgen05.mma instructions (M = 128, N = 48, K = 16 each) into 48 tensor-
// memory columns and commits them to an mbarrier; every thread then reads its
// accumulator row (tensor-memory lane) with tcgen05.ld, so the 3 x 3 multiply
// needs no exchange between threads.  The inverse product reuses the same
// columns.  Outputs go through shared memory and leave as 128-byte rows.
//
// Operand layout in shared memory (16-bit, no swizzle, 8 x 8 core matrices of
// 128 contiguous bytes): K-major element (row, k) at (row / 8) SBO + (k / 8)
// LBO + (row % 8) 16 + (k % 8) 2 bytes (A1 and the forward data operand,
// whose LBO = 160 spreads the threads' 16-byte stores over the banks); A2 is
// the MN-major view of A1 (element (m, k) of A2 is element (k, m) of A1); the
// inverse data operand is MN-major, element (n, k) at (n / 8) SBO + (k / 8) LBO
// + (k % 8) 16 + (n % 8) 2, so a thread writes its row's 8 consecutive n as one
// 16-byte store.
//
// Accumulator rows are permuted: row m (and m + 64) holds kz = kz_of(m), which
// puts into each half-warp eight kernel rows kz' with distinct kz' mod 8 (each
// read by the two lanes of kz and 64 - kz), so the kernel-row loads are free of
// bank conflicts.  Scales are powers of two (exact, no divisions).
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

constexpr int Q5 = 16;               // ky columns per tile
constexpr int N5 = 48;               // operand columns: 3 components x 16
constexpr int T5 = 128;              // threads per CTA (one per accumulator row)
constexpr int HZ5 = 32;              // z cells held (pz = 64)
constexpr int KBW5 = 18;             // kernel-row box: 18 of the blocked copy's 34 entries per row
constexpr int KBW2 = 34;             // entries per row of the blocked copy (ky' = 32 b .. 32 b + 32, one pad)
constexpr int KROWS5 = (HZ5 + 1) * 3;
constexpr uint32_t TMEM_COLS = 64;   // power of two >= 48
constexpr int STATUS_TIMEOUT5 = -5;  // BORIS_ERR_TIMEOUT

constexpr uint32_t A1_LBO = 128, A1_SBO = 1024;  // K-major, 128 rows x 64 k
constexpr uint32_t A2_LBO = 1024, A2_SBO = 128;  // MN-major view of A1: 64 (x 128) rows x 128 k
constexpr uint32_t D1_LBO = 160, D1_SBO = 1280;  // K-major, 48 rows x 64 k
constexpr uint32_t D2_LBO = 128, D2_SBO = 2048;  // MN-major, 48 n x 128 k
constexpr int OUT_ROW = 2 * Q5 + 1;               // floats per (c, z) row of the output stage

// shared memory (bytes).  An M = 128 product through the A2 view reads rows
// 64..127 from A1's other elements and up to 1 KB past A1 (finite data in the
// stage; those output rows are ignored).
constexpr size_t OFF_A1 = 0;
constexpr size_t OFF_STAGE = 16384;                                            // [c][z][col] float2
constexpr size_t OFF_KST = OFF_STAGE + (size_t)3 * HZ5 * Q5 * 8;                // kernel rows [kz' 3 + p][18]
constexpr size_t OFF_D = (OFF_KST + (size_t)KROWS5 * KBW5 * 8 + 127) / 128 * 128;  // D1, D2, output stage
constexpr size_t D1_BYTES = (size_t)(N5 / 8) * D1_SBO, D2_BYTES = (size_t)(N5 / 8) * D2_SBO;
constexpr size_t OUT_BYTES = (size_t)3 * HZ5 * OUT_ROW * 4;
constexpr size_t D_BYTES = OUT_BYTES > D2_BYTES ? OUT_BYTES : D2_BYTES;
constexpr size_t OFF_S1 = OFF_D + D_BYTES;   // [col][4] forward column scales (sign of ky fold in .y)
constexpr size_t OFF_S2 = OFF_S1 + Q5 * 16;  // [col][4] inverse column maxima (float bits)
constexpr size_t OFF_BAR = OFF_S2 + Q5 * 16;
constexpr size_t OFF_TSLOT = OFF_BAR + 3 * 8;
constexpr size_t SMEM5 = OFF_TSLOT + 16;
static_assert(D1_BYTES <= D_BYTES, "operands fit");
static_assert(OFF_KST % 128 == 0 && OFF_STAGE % 128 == 0, "tensor-copy destinations");
static_assert(16384 + 1024 <= OFF_D, "the A2 view's ignored rows stay inside the allocation");
static_assert(4 * (SMEM5 + 1024) <= 233472, "four CTAs per SM");

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

// columns taddr + 16 c + j (c < 3, j < 16) of this thread's lane;
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
        : "r"(taddr), "r"(taddr + 16), "r"(taddr + 32)
        : "memory");
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int j = 0; j < 16; j++) v[c][j] = __uint_as_float(r[16 * c + j]);
}

// kz held by accumulator row m (mod 64): groups of 16 rows take kz' = 8 j + 1 .. 8 j + 8
// with both signs (j < 3), and kz' = 25 .. 32 with 33 .. 39 and 0 (j = 3)
__device__ __forceinline__ int kz_of(int m)
{
    const int j = m >> 4, i = m & 15;
    if (j < 3) return i < 8 ? 8 * j + 1 + i : 63 - 8 * j - (i - 8);
    return i < 8 ? 25 + i : (i < 15 ? 47 - i : 0);
}

// 2^(e - 127) for the exponent field e of a non-negative float (0 below the
// normal range), and 2^(127 - e): exact scales that bring |x| into [1, 2)
__device__ __forceinline__ float pow2_of(uint32_t bits) { return __uint_as_float(bits & 0x7f800000u); }
__device__ __forceinline__ float inv_pow2_of(uint32_t bits)
{
    return __uint_as_float((254u - ((bits >> 23) & 0xffu)) << 23);
}

// largest |x| over the warp
__device__ __forceinline__ float warp_max_abs(float x)
{
    float r;
    asm volatile("redux.sync.max.abs.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(x));
    return r;
}

// mbarrier wait that lets the hardware suspend the thread (up to 20 us per
// try) instead of spinning; false after limit_ns of device time
__device__ __forceinline__ bool mbar_wait_hint(uint64_t* bar, uint32_t parity, uint64_t limit_ns)
{
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 24); it++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// A1[m][k]: m = part * 64 + (row of kz), k = kpart * 32 + z; cs[e] = (cos, sin) of 2 pi e / 64
__device__ __forceinline__ float a1_val(const float2* cs64, int m, int k)
{
    const int part = m >> 6, kpart = k >> 5;
    const float2 cs = cs64[(kz_of(m & 63) * (k & 31)) & 63];
    return part == kpart ? cs.x : (part == 0 ? cs.y : -cs.y);
}
__device__ __forceinline__ uint32_t op_off(int row, int k, uint32_t lbo, uint32_t sbo)
{
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * lbo + (uint32_t)(row & 7) * 16 + (uint32_t)(k & 7) * 2;
}


template <typename H>
__global__ void __launch_bounds__(T5, 4)
    z_conv_tc5_kernel(const __grid_constant__ CUtensorMap ymap, const __grid_constant__ CUtensorMap kmap, Geometry g,
                      int nkb, float2* __restrict__ Y, const float2* __restrict__ tw_g, int* __restrict__ status,
                      uint32_t extra_tx, unsigned long long limit_ns)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
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
    // kind::f16, FP32 accumulator, A and B of type H, N = 48, M = 128; forward:
    // both K-major; inverse: both MN-major (bits 15 and 16)
    constexpr uint32_t IDESC = (1u << 4) | (Cvt16<H>::fmt << 7) | (Cvt16<H>::fmt << 10) |
                               ((uint32_t)(N5 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    constexpr uint32_t IDESC_MN = IDESC | (1u << 15) | (1u << 16);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the DFT operand, once per CTA, from (cos, sin) of 2 pi e / 64 staged in
    // the (still unused) operand region; the plan's twiddles are exp(-2 pi i e / lmax)
    {
        float2* cs64 = reinterpret_cast<float2*>(Dm);
        const int shz = g.lglmax - 6;
        if (tid < 64) {
            const float2 w = tw_g[tid << shz];
            cs64[tid] = make_float2(w.x, -w.y);
        }
        __syncthreads();
        for (int i = tid; i < 128 * 32; i += T5) {
            const int m = i >> 5, k = (i & 31) * 2;
            *reinterpret_cast<uint32_t*>(A1 + op_off(m, k, A1_LBO, A1_SBO)) =
                Cvt16<H>::two(a1_val(cs64, m, k), a1_val(cs64, m, k + 1));
        }
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
    // kernel rows of tile t: block b of the blocked copy and 18 of its 34
    // entries from x0, with k32 = ky0 rounded down to a multiple of 32.  Below
    // the fold column col reads entry (ky0 mod 32) + col of block k32 / 32;
    // above it entry 32 - (ky0 mod 32) - col of block (py - k32) / 32 - 1.
    auto load_k = [&](int t) {
        const int kx = t / nty, ky0 = (t - kx * nty) * Q5, k32 = ky0 & ~31;
        const bool up = ky0 >= py / 2;
        const int b = up ? (py - k32) / 32 - 1 : k32 / 32;
        const int x0 = up ? 16 - (ky0 & 16) : (ky0 & 16);
        mbar_arrive_expect_tx(fullK, kbytes);
        tma_load_2d(kst, &kmap, x0, (kx * nkb + b) * KROWS5, fullK);
    };
    // copies and product groups issued by thread 0 (for the drain after a timeout)
    int ny_issued = 0, nk_issued = 0, nm_issued = 0;
    if (tid == 0 && (int)blockIdx.x < ntiles) {
        load_y(blockIdx.x, extra_tx);
        load_k(blockIdx.x);
        ny_issued = nk_issued = 1;
    }

    // this thread's accumulator row (tensor-memory lane)
    const int r = tid;
    const int kz = kz_of(r & 63);
    const int kzf = kz <= HZ5 ? kz : 64 - kz;
    const float sz = kz > HZ5 ? -1.f : 1.f;  // xz and yz are odd in kz
    const uint32_t trow = tbase + ((uint32_t)(32 * warp) << 16);
    float* outs = reinterpret_cast<float*>(Dm);

    bool failed = false;
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += G, k++) {
        const int kx = t / nty, ky0 = (t - kx * nty) * Q5;
        const bool more = t + G < ntiles;
        const bool fy = ky0 >= py / 2;  // ky beyond the fold: xy and yz change sign
        {
            const bool ok = mbar_wait_hint(fullY, k & 1, limit_ns);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
        }
        // scaled 16-bit forward operand D1[n][k]: k < 32 Re z, k >= 32 Im z;
        // thread pair (2 n, 2 n + 1) takes z < 16 and z >= 16 of column n
        if (tid < 2 * N5) {
            const int n = tid >> 1, zh = tid & 1, c = n >> 4, col = n & 15;
            const float2* src = stage + (c * HZ5 + 16 * zh) * Q5 + col;
            float2 a[16];
            float mx = 0.f;
#pragma unroll
            for (int i = 0; i < 16; i++) {
                a[i] = 16 * zh + i < nz ? src[i * Q5] : make_float2(0.f, 0.f);
                mx = fmaxf(mx, fmaxf(fabsf(a[i].x), fabsf(a[i].y)));
            }
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
            const float s = inv_pow2_of(__float_as_uint(mx));
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
            if (zh == 0) {
                const float p2 = pow2_of(__float_as_uint(mx));
                S1[col * 4 + c] = (c == 1 && fy) ? -p2 : p2;
            }
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
            const bool ok = mbar_wait_hint(fullK, k & 1, limit_ns) && mbar_wait_hint(mmab, 0, limit_ns);
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
                const int e = fy ? 16 - j : j;
                const float4 s = *reinterpret_cast<const float4*>(S1 + j * 4);
                const float m0 = h[0][j] * s.x, m1 = h[1][j] * s.y, m2 = h[2][j] * (s.z * sz);
                const float2 p0 = kp[e], p1 = kp[KBW5 + e], p2 = kp[2 * KBW5 + e];
                h[0][j] = p0.x * m0 + p1.y * m1 + p2.x * m2;
                h[1][j] = p1.y * m0 + p0.y * m1 + p2.y * m2;
                h[2][j] = p2.x * m0 + p2.y * m1 + p1.x * m2;
            }
        }
        // largest magnitude of each operand column over the 128 rows
        {
            float sel0 = 0.f, sel1 = 0.f;
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int i = 16 * c + j;
                    const float u = warp_max_abs(h[c][j]);
                    if (lane == (i & 31)) {
                        if (i < 32) sel0 = u;
                        else sel1 = u;
                    }
                }
            atomicMax(S2 + (lane & 15) * 4 + (lane >> 4), __float_as_uint(sel0));
            if (lane < 16) atomicMax(S2 + lane * 4 + 2, __float_as_uint(sel1));
        }
        tc_fence_before();
        __syncthreads();
        if (tid == 0 && more) {
            fence_proxy_async_smem();
            load_k(t + G);
            nk_issued++;
        }
        // scaled 16-bit inverse operand D2[n][k = r] (MN-major: the row's 8
        // consecutive n per 16-byte store); s_z H2 is turned back into H2 here
        {
            unsigned char* base = Dm + (r >> 3) * D2_LBO + (r & 7) * 16;
#pragma unroll
            for (int hh = 0; hh < 2; hh++) {
                float v[3][8];
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    const int col = 8 * hh + e;
                    const uint4 mb = *reinterpret_cast<const uint4*>(S2 + col * 4);
                    v[0][e] = h[0][col] * inv_pow2_of(mb.x);
                    v[1][e] = h[1][col] * inv_pow2_of(mb.y);
                    v[2][e] = h[2][col] * (inv_pow2_of(mb.z) * sz);
                }
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    uint4 w;
                    w.x = Cvt16<H>::two(v[c][0], v[c][1]);
                    w.y = Cvt16<H>::two(v[c][2], v[c][3]);
                    w.z = Cvt16<H>::two(v[c][4], v[c][5]);
                    w.w = Cvt16<H>::two(v[c][6], v[c][7]);
                    *reinterpret_cast<uint4*>(base + (2 * c + hh) * D2_SBO) = w;
                }
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 8; ks++)
                umma_f16(tbase, sdesc(A1 + ks * 2 * A2_LBO, A2_LBO, A2_SBO), sdesc(Dm + ks * 2 * D2_LBO, D2_LBO, D2_SBO),
                         IDESC_MN, ks > 0);
            umma_commit(mmab);
            nm_issued++;
        }
        {
            const bool ok = mbar_wait_hint(mmab, 1, limit_ns);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
        }
        tc_fence_after();
        // rows r < 64: Re (r < 32) and Im (r >= 32) of z = r mod 32; the y
        // component takes back the sign of the ky fold
        if (warp < 2) {
            float o[3][16];
            tmem_ld48(trow, o);
            const int z = r & 31, part = r >> 5;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const uint4 mb = *reinterpret_cast<const uint4*>(S2 + j * 4);
                const float s1 = fy ? -pow2_of(mb.y) : pow2_of(mb.y);
                outs[(0 * HZ5 + z) * OUT_ROW + 2 * j + part] = o[0][j] * pow2_of(mb.x);
                outs[(1 * HZ5 + z) * OUT_ROW + 2 * j + part] = o[1][j] * s1;
                outs[(2 * HZ5 + z) * OUT_ROW + 2 * j + part] = o[2][j] * pow2_of(mb.z);
            }
        }
        tc_fence_before();
        __syncthreads();
        {
            float2* dst = Y + (size_t)kx * lines * py + ky0;
#pragma unroll
            for (int c = 0; c < 3; c++)
                for (int i = tid; i < nz * Q5; i += T5) {
                    const int z = i >> 4, col = i & 15;
                    const float* src = outs + (c * HZ5 + z) * OUT_ROW + 2 * col;
                    dst[(size_t)(c * nz + z) * py + col] = make_float2(src[0], src[1]);
                }
        }
        // the output stage is rewritten only after the next tile's first barrier
    }
    if (failed && tid == 0) {
        atomicCAS(status, 0, STATUS_TIMEOUT5);
        // let the copies and products still in flight land (bounded)
        if (ny_issued > 0) mbar_wait_hint(fullY, (ny_issued - 1) & 1, limit_ns);
        if (nk_issued > 0) mbar_wait_hint(fullK, (nk_issued - 1) & 1, limit_ns);
        if (nm_issued > 0) mbar_wait_hint(mmab, (nm_issued - 1) & 1, limit_ns);
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
    const int grid = std::min(ntiles, 4 * nsm);
    z_conv_tc5_kernel<H><<<grid, T5, SMEM5, st>>>(ymap, kmap, g, zconv_res_nkb(g), Y, tw, status, extra_tx, limit_ns);
    return cudaGetLastError();
}

}  // namespace

bool zconv_tc5_supported(const Geometry& g, int max_smem)
{
    // pz = 64 (17 <= nz <= 32); py >= 64 so that the ky fold falls on a block
    // boundary of the blocked kernel copy (that of the residue-split stage)
    return g.pz == 2 * HZ5 && g.nz >= 17 && g.nz <= HZ5 && g.py >= 64 && g.py % 32 == 0 &&
           g.krow == ((HZ5 + 1) * 6 + 3) / 4 * 4 && SMEM5 <= (size_t)max_smem && g.lglmax >= 6;
}

// Y[kx][c][z][ky] as rows (kx, c, z) of py complex values, boxes of 16 x nz;
// the blocked kernel copy as rows of 34 entries, boxes of 18 x 3 (HZ + 1)
cudaError_t zconv_tc5_maps(const Geometry& g, float2* Y, float2* K2, void* ymap, void* kmap)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint32_t es[2] = {1, 1};
    {
        const cuuint64_t dims[2] = {(cuuint64_t)g.py, (cuuint64_t)g.nkx * 3 * g.nz};
        const cuuint64_t strides[1] = {(cuuint64_t)g.py * sizeof(float2)};
        const cuuint32_t box[2] = {(cuuint32_t)Q5, (cuuint32_t)g.nz};
        const CUresult r = enc(reinterpret_cast<CUtensorMap*>(ymap), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, Y, dims,
                               strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t rows = (cuuint64_t)g.nkx * zconv_res_nkb(g) * g.kzh * 3;
        const cuuint64_t dims[2] = {(cuuint64_t)KBW2, rows};
        const cuuint64_t strides[1] = {(cuuint64_t)KBW2 * sizeof(float2)};
        const cuuint32_t box[2] = {(cuuint32_t)KBW5, (cuuint32_t)KROWS5};
        const CUresult r = enc(reinterpret_cast<CUtensorMap*>(kmap), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, K2, dims,
                               strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
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
