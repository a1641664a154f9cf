// Mixed-precision z stage with 16-bit storage of the padded y-z spectrum: the
// zero-padded length-64 z transform of the pipelined convolution (Section 7)
// and its inverse as dense products on the tcgen05 tensor cores, BF16 or
// FP16 operands, FP32 accumulation in tensor memory (the paper has FP32 and
// FP64 only; this is the reduced-precision variant of the split schedule).
// BF16 spectra are stored as they are; FP16 spectra carry a power-of-two scale
// s (chosen by the y forward pass from max |Ms M|), which the multiply and the
// DFTs preserve, and the output is multiplied by 1/128 instead of 1/(px py pz)
// (the y inverse pass undoes both).
//
// Layout of the 16-bit spectrum Y16 (written by the y forward pass, read by
// the y inverse): [kx][c][part][z][ky], part 0 = Re, 1 = Im, each (part, z)
// line of a kx plane py consecutive values.  A 5D tensor-copy view of it -
// (ky mod 64, z, part, ky / 64, (kx, c)) with the ky / 64 dimension at a stride
// of 128 bytes, boxes of (64, 32, 2, 2, 1), the 128-byte swizzle - lands in
// shared memory as the MN-major operand of a 128-row product: element (m = ky
// in the tile, k = 32 part + z) in the 128-byte row (m / 64) 64 + k at byte
// 2 (m mod 64), its 16-byte chunk index XOR-ed with k mod 8.  z >= nz is
// filled with zeros by the copy (the zero padding of the z transform).
//
// A tile is 128 ky columns of one kx plane.  Per component c:
//   forward  D_c (128 x 128) = A_c (128 x 64) . F (64 x 128): the data are the
//            A operand (rows = ky columns), F the DFT matrix,
//            n = 64 q + kz (q: Re / Im of X^(kz)), k = 32 p + z (p: Re / Im of
//            x(z)), F = [[C, S], [-S, C]] with C, S = cos, sin(2 pi kz z / 64)
//   multiply H_c(kz) = sum_d N_cd(kx, ky, kz) M_d(kz): thread t owns
//            accumulator row t (one ky column) for all three components and
//            all kz, so the 3 x 3 product needs no exchange between threads;
//            the kernel spectrum is real, Re and Im are multiplied alike
//   inverse  out_c^T (64 x 128) = F^T (64 x 128) . H_c^T (128 x 128): F^T is
//            F's storage read as an MN-major operand (M = 64 rows (part, z):
//            row m of the result lands in tensor-memory lane 32 (m / 16) +
//            m mod 16), the products H_c the K-major B operand (rows = ky
//            columns); the rows (part, z < nz) are read back by half-warp
//            loads (16 lanes, two column runs) and stored as 32-byte pieces
// The kernel spectrum arrives as FP16 pairs (xx, yy), (zz, xy), (xz, yz) of
// the octant scaled by px py pz (the fold of the normalisation is undone on
// the output).  Everything runs in one persistent CTA per SM: sixteen compute
// warps and one warp whose first thread issues the tensor copies and the
// products.  The four compute warps of a tensor-memory lane quarter split the
// kz range of the multiply (sixteen kz each, so that the fold signs are fixed
// per warp and tile) and the ky columns of the output (32 each);
// tensor-memory loads are issued in groups with one wait each.  Tensor memory
// holds four regions of 128 columns; the forward products of a tile take
// three of them and its inverse products the free one and two that the
// multiply has consumed, so the next tile's forward products go into each
// region as soon as the current tile's rows there have been read (mbarrier
// arrivals of the compute warps), while those rows are being stored.  The
// next tile's data are copied in once the forward products are done, its
// kernel rows once the multiply is done.
//
// Every mbarrier wait is bounded (device timer); when one gives up the CTA
// latches BORIS_ERR_TIMEOUT in *status, waits (bounded) for its copies and
// products in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "boris_internal.cuh"
#include "tcgen05.cuh"

namespace boris {

namespace {

constexpr int NCW6 = 16;                // compute warps: four per tensor-memory lane quarter
constexpr int T6 = 32 * (NCW6 + 1);     // and one warp that issues the copies and products
constexpr int MT = 128;       // ky columns per tile
constexpr int HZ6 = 32;       // z cells held (pz = 64)
constexpr int KZH6 = HZ6 + 1;  // kz' rows of the kernel octant
constexpr int KW6 = 136;      // kernel-spectrum box width (ky' entries, 16-byte multiple)
constexpr uint32_t TMEM6 = 512;
constexpr int STATUS_TIMEOUT6 = -5;

constexpr uint32_t F_LBO = 128, F_SBO = 1024;    // F: K-major, 128 n x 64 k
constexpr uint32_t FI_LBO = 1024, FI_SBO = 128;  // F^T as an MN-major operand: 64 rows x 128 k
// data: MN-major with the 128-byte swizzle, 128 m x 64 k (tensor copy): atoms of
// 64 m (128 bytes) x 8 k; LBO = stride between the two 64-m atom columns,
// SBO = stride between groups of 8 k
constexpr uint32_t AF_LBO = 8192, AF_SBO = 1024;
constexpr uint32_t AI_LBO = 128, AI_SBO = 2048;  // products: K-major, 128 m x 128 k

constexpr size_t F_BYTES = 128 * 64 * 2;
constexpr size_t AF_COMP = (size_t)MT * 64 * 2;   // 16 KB per component
constexpr size_t AI_COMP = (size_t)MT * 128 * 2;  // 32 KB per component
constexpr size_t K_BYTES = (size_t)KZH6 * 3 * KW6 * 4;
constexpr size_t OFF_F = 0;
constexpr size_t OFF_AF = OFF_F + F_BYTES;
constexpr size_t OFF_AI = OFF_AF + 3 * AF_COMP;
constexpr size_t OFF_K = OFF_AI + 3 * AI_COMP;
constexpr size_t OFF_BAR = (OFF_K + K_BYTES + 15) / 16 * 16;
constexpr size_t OFF_TSLOT = OFF_BAR + 9 * 8;
constexpr size_t SMEM6 = OFF_TSLOT + 16 + 1024;  // + alignment of the base to 1024 bytes
static_assert(SMEM6 <= 232448, "one CTA per SM");
static_assert(OFF_AF % 1024 == 0 && OFF_AI % 1024 == 0 && OFF_K % 128 == 0, "operand and copy alignment");

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}
// the operand format: FP16 (H16) or BF16
template <bool H16>
__device__ __forceinline__ uint32_t pack16(float a, float b)
{
    if constexpr (H16) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        return pack_bf16(a, b);
    }
}

// The kernel multiply of one chunk of eight kz for accumulator row `row`
// (kernel entry ke of the staged rows): the forward products of the three
// components from tensor memory (row addresses t0, t1, t2), H_c = sum_d N_cd M_d with the fold signs
// known at compile time (UP: above the ky fold, xy and yz odd in ky; NEGZ:
// kz > 32, xz and yz odd in kz, whose kz = 32 entries vanish), BF16 products
// to the K-major inverse operand (k = kz for Re, 64 + kz for Im).
template <bool UP, bool NEGZ, bool H16>
__device__ __forceinline__ void tc6_multiply_chunk(int j, uint32_t t0, uint32_t t1, uint32_t t2,
                                                   const __half2* __restrict__ kst, int ke, unsigned char* AI, int row)
{
    const int kz0 = 8 * j;
    // this chunk's kernel pairs first: their shared-memory latency then
    // overlaps that of the tensor-memory loads below
    __half2 kq[8][3];
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const int kz = kz0 + e;
        const int kzp = kz <= HZ6 ? kz : 64 - kz;
        const __half2* kp = kst + (kzp * 3) * KW6 + ke;
        kq[e][0] = kp[0];
        kq[e][1] = kp[KW6];
        kq[e][2] = kp[2 * KW6];
    }
    float v6[6][8];
    {
        const uint32_t a[6] = {t0 + kz0, t0 + 64 + kz0, t1 + kz0, t1 + 64 + kz0, t2 + kz0, t2 + 64 + kz0};
        tc::ld8x6(a, v6);
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float hr[8], hi[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const float2 p0 = __half22float2(kq[e][0]), p1 = __half22float2(kq[e][1]), p2 = __half22float2(kq[e][2]);
            const float xx = p0.x, yy = p0.y, zz = p1.x;
            const float xy = UP ? -p1.y : p1.y, xz = NEGZ ? -p2.x : p2.x, yz = (UP != NEGZ) ? -p2.y : p2.y;
            const float n0 = c == 0 ? xx : c == 1 ? xy : xz;
            const float n1 = c == 0 ? xy : c == 1 ? yy : yz;
            const float n2 = c == 0 ? xz : c == 1 ? yz : zz;
            hr[e] = n0 * v6[0][e] + n1 * v6[2][e] + n2 * v6[4][e];
            hi[e] = n0 * v6[1][e] + n1 * v6[3][e] + n2 * v6[5][e];
        }
        // row `row`, k = kz (Re) and 64 + kz (Im): one 16-byte store each
        unsigned char* arow = AI + c * AI_COMP + (row >> 3) * AI_SBO + (row & 7) * 16;
        uint4 wr, wi;
        wr.x = pack16<H16>(hr[0], hr[1]);
        wr.y = pack16<H16>(hr[2], hr[3]);
        wr.z = pack16<H16>(hr[4], hr[5]);
        wr.w = pack16<H16>(hr[6], hr[7]);
        wi.x = pack16<H16>(hi[0], hi[1]);
        wi.y = pack16<H16>(hi[2], hi[3]);
        wi.z = pack16<H16>(hi[4], hi[5]);
        wi.w = pack16<H16>(hi[6], hi[7]);
        *reinterpret_cast<uint4*>(arow + j * AI_LBO) = wr;
        *reinterpret_cast<uint4*>(arow + (8 + j) * AI_LBO) = wi;
    }
}

template <bool H16>
__global__ void __launch_bounds__(T6, 1)
    z_conv_tc6_kernel(const __grid_constant__ CUtensorMap ymap, const __grid_constant__ CUtensorMap kmap, Geometry g,
                      unsigned short* __restrict__ Y16, const float2* __restrict__ tw_g, float out_scale,
                      int* __restrict__ status, uint32_t extra_tx, unsigned long long limit_ns)
{
    extern __shared__ unsigned char smem_raw[];
    // aligned to 1024 bytes by an offset from the shared array itself, so that the
    // compiler keeps every access derived from base in the shared state space
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* F = base + OFF_F;
    unsigned char* AF = base + OFF_AF;
    unsigned char* AI = base + OFF_AI;
    const __half2* kst = reinterpret_cast<const __half2*>(base + OFF_K);
    uint64_t* fullA = reinterpret_cast<uint64_t*>(base + OFF_BAR);
    uint64_t* fullK = fullA + 1;
    uint64_t* fwdb = fullA + 2;  // forward products of a tile (tcgen05.commit)
    uint64_t* mulb = fullA + 3;  // kernel multiply of a tile done (one arrival per compute warp)
    uint64_t* invb = fullA + 4;  // inverse products of component c: invb[c] (tcgen05.commit)
    uint64_t* outb = fullA + 7;  // result rows of component c (c < 2) read from tensor memory
    uint32_t* tslot = reinterpret_cast<uint32_t*>(base + OFF_TSLOT);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lq = warp & 3, wp = warp >> 2;  // tensor-memory lane quarter, work part (0..3)
    const int row = 32 * lq + lane;           // accumulator row of the multiply (ky column in the tile)
    const int py = g.py;
    const int nty = py / MT, ntiles = g.nkx * nty, G = gridDim.x;
    constexpr uint32_t abytes = 3 * (uint32_t)AF_COMP;
    constexpr uint32_t kbytes = (uint32_t)K_BYTES;
    constexpr uint32_t FMT = H16 ? 0 : 1;                                    // FP16 or BF16 operands
    constexpr uint32_t IDESC_F = tc::idesc_f16(FMT, true, false, 128, 128);  // data MN-major, F K-major
    constexpr uint32_t IDESC_I = tc::idesc_f16(FMT, true, false, 64, 128);   // F^T MN-major, products K-major

    if (warp == 0) tc::alloc(tslot, TMEM6);
    // the forward DFT matrix F, once per CTA; the plan's twiddles are exp(-2 pi i e / lmax)
    {
        float2* cs64 = reinterpret_cast<float2*>(AI);  // scratch: AI is written only later
        const int shz = g.lglmax - 6;
        if (tid < 64) {
            const float2 w = tw_g[tid << shz];
            cs64[tid] = make_float2(w.x, -w.y);
        }
        __syncthreads();
        for (int i = tid; i < 128 * 32; i += T6) {
            const int n = i >> 5, k = (i & 31) * 2;  // two consecutive k of row n
            const int q = n >> 6, kz = n & 63;
            float v[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int kk = k + h, p = kk >> 5, z = kk & 31;
                const float2 cs = cs64[(kz * z) & 63];
                v[h] = q == p ? cs.x : (q == 0 ? cs.y : -cs.y);
            }
            *reinterpret_cast<uint32_t*>(F + (n >> 3) * F_SBO + (k >> 3) * F_LBO + (n & 7) * 16 + (k & 7) * 2) =
                pack16<H16>(v[0], v[1]);
        }
    }
    if (tid == 0) {
        mbar_init(fullA, 1);
        mbar_init(fullK, 1);
        mbar_init(fwdb, 1);
        mbar_init(mulb, NCW6);
        for (int c = 0; c < 3; c++) mbar_init(invb + c, 1);
        for (int c = 0; c < 2; c++) mbar_init(outb + c, NCW6);
        fence_mbar_init();
    }
    fence_proxy_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tslot;

    // extra: bytes the first copy also waits for (a test hook that makes the wait run out)
    auto load_a = [&](int t, uint32_t extra) {
        const int kx = t / nty, ky0 = (t - kx * nty) * MT;
        mbar_arrive_expect_tx(fullA, abytes + extra);
        for (int c = 0; c < 3; c++) tc::tma_load_5d(AF + c * AF_COMP, &ymap, 0, 0, 0, ky0 / 64, kx * 3 + c, fullA);
    };
    // kernel rows of tile t: ky' = ky below the fold, py - ky above it (a box
    // starting 128 entries below py - ky0, so that ky' = x + 128 - t)
    auto load_k = [&](int t) {
        const int kx = t / nty, ky0 = (t - kx * nty) * MT;
        const int x = ky0 < py / 2 ? ky0 : py - ky0 - MT;
        mbar_arrive_expect_tx(fullK, kbytes);
        tc::tma_load_3d(base + OFF_K, &kmap, x, 0, kx, fullK);
    };
    // Tensor memory holds four 128-column regions.  Tile number it (of this CTA)
    // has its forward products of component c in region (r + c) mod 4, r = 2 it
    // mod 4, and its inverse products in regions (r + 3, r, r + 1) mod 4: the
    // region the multiply frees last (r + 2) and the one its inverse leaves free
    // take the next tile's forward products of components 0 and 1, so those run
    // while the current tile's results are read and stored.
    const bool producer = warp == NCW6;
    bool failed = false;
    int na = 0, nk = 0, nf = 0, ni = 0;  // copies and product groups the producer issued
    if (producer) {
        if (lane == 0) {
            auto fwd = [&](int region, int c) {
#pragma unroll
                for (int ks = 0; ks < 4; ks++)
                    tc::mma_f16(tbase + region * 128,
                                tc::sdesc_sw128(AF + c * AF_COMP + ks * 2 * AF_SBO, AF_LBO, AF_SBO),
                                tc::sdesc(F + ks * 2 * F_LBO, F_LBO, F_SBO), IDESC_F, ks > 0);
            };
            if ((int)blockIdx.x < ntiles) {
                load_a(blockIdx.x, extra_tx);
                load_k(blockIdx.x);
                na = nk = 1;
                if (!tc::wait(fullA, 0, limit_ns)) {
                    failed = true;
                } else {
                    tc::fence_after();
                    for (int c = 0; c < 3; c++) fwd(c, c);
                    tc::commit(fwdb);
                    nf = 1;
                }
            }
            int it = 0;
            for (int t = blockIdx.x; t < ntiles && !failed; t += G, it++) {
                const int r = (2 * it) & 3;
                const bool more = t + G < ntiles;
                // the forward products are done: the data operand is free
                if (!tc::wait(fwdb, it & 1, limit_ns)) {
                    failed = true;
                    break;
                }
                if (more) {
                    load_a(t + G, 0);
                    na++;
                }
                // the multiply is done: products in shared memory, forward regions read,
                // kernel rows consumed
                if (!tc::wait(mulb, it & 1, limit_ns)) {
                    failed = true;
                    break;
                }
                if (more) {
                    load_k(t + G);
                    nk++;
                }
                tc::fence_after();
                for (int c = 0; c < 3; c++) {
                    const int region = c == 0 ? (r + 3) & 3 : c == 1 ? r : (r + 1) & 3;
#pragma unroll
                    for (int ks = 0; ks < 8; ks++)
                        tc::mma_f16(tbase + region * 128, tc::sdesc(F + ks * 2 * FI_LBO, FI_LBO, FI_SBO),
                                    tc::sdesc(AI + c * AI_COMP + ks * 2 * AI_LBO, AI_LBO, AI_SBO), IDESC_I, ks > 0);
                    tc::commit(invb + c);
                }
                ni++;
                if (!more) continue;
                // the next tile's forward products, each into a region as soon as it is free
                if (!tc::wait(fullA, (it + 1) & 1, limit_ns)) {
                    failed = true;
                    break;
                }
                tc::fence_after();
                fwd((r + 2) & 3, 0);
                if (!tc::wait(outb, it & 1, limit_ns)) {
                    failed = true;
                    break;
                }
                tc::fence_after();
                fwd((r + 3) & 3, 1);
                if (!tc::wait(outb + 1, it & 1, limit_ns)) {
                    failed = true;
                    break;
                }
                tc::fence_after();
                fwd(r, 2);
                tc::commit(fwdb);
                nf++;
            }
        }
    } else {
        const uint32_t trow = tbase + ((uint32_t)(32 * lq) << 16);
        int it = 0;
        for (int t = blockIdx.x; t < ntiles; t += G, it++) {
            const int kx = t / nty, ky0 = (t - kx * nty) * MT;
            const int r = (2 * it) & 3;
            const bool up = ky0 >= py / 2;  // above the ky fold: xy and yz change sign
            const int ke = up ? MT - row : row;
            {
                const bool ok = tc::wait(fwdb, it & 1, limit_ns) && tc::wait(fullK, it & 1, limit_ns);
                if (__any_sync(0xffffffffu, !ok)) {
                    failed = true;
                    break;
                }
            }
            tc::fence_after();
            // kernel multiply: this warp's part of the kz range, two chunks of
            // eight (parts 2 and 3 lie above kz = 32)
            {
                const uint32_t t0 = trow + 128 * r, t1 = trow + 128 * ((r + 1) & 3), t2 = trow + 128 * ((r + 2) & 3);
                const bool nz_ = wp >= 2;
#pragma unroll 1
                for (int j = 2 * wp; j < 2 * wp + 2; j++) {
                    if (up) {
                        if (nz_) tc6_multiply_chunk<true, true, H16>(j, t0, t1, t2, kst, ke, AI, row);
                        else tc6_multiply_chunk<true, false, H16>(j, t0, t1, t2, kst, ke, AI, row);
                    } else {
                        if (nz_) tc6_multiply_chunk<false, true, H16>(j, t0, t1, t2, kst, ke, AI, row);
                        else tc6_multiply_chunk<false, false, H16>(j, t0, t1, t2, kst, ke, AI, row);
                    }
                }
            }
            fence_proxy_async_smem();
            tc::fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(mulb);
            // outputs: result row m = 16 lq + (lane mod 16) (part = m / 32, z = m mod 32)
            // sits in lane 32 lq + m mod 16; warp part wp stores the tile's ky
            // 32 wp .. 32 wp + 31 of it, each half-warp sixteen consecutive ky (one
            // 32-byte store per thread, 64 contiguous bytes per row and instruction)
            const int m = 16 * lq + (lane & 15), part = m >> 5, z = m & 31;
            const bool keep = z < g.nz;
            const int kyo = 32 * wp + 16 * (lane >> 4);
#pragma unroll 1
            for (int c = 0; c < 3; c++) {
                {
                    // the products of component c
                    const bool ok = tc::wait(invb + c, it & 1, limit_ns);
                    if (__any_sync(0xffffffffu, !ok)) {
                        failed = true;
                        break;
                    }
                }
                tc::fence_after();
                const int region = c == 0 ? (r + 3) & 3 : c == 1 ? r : (r + 1) & 3;
                float v[16];
                tc::ld16x2_16(trow + 128 * region + 32 * wp, v);
                if (c < 2) {
                    // this warp's rows of component c are read: the region may be reused
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(outb + c);
                }
                if (keep) {
                    unsigned short* dst =
                        Y16 + ((((size_t)kx * 3 + c) * 2 + part) * g.nz + z) * (size_t)py + ky0 + kyo;
                    uint32_t w[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) w[q] = pack16<H16>(v[2 * q] * out_scale, v[2 * q + 1] * out_scale);
                    tc::st_global_v8(dst, w);
                }
            }
            if (failed) break;
        }
    }

    // every wait above is bounded, so all warps arrive here; after a timeout the
    // producer drains what it issued before the tensor memory is freed
    tc::fence_before();
    failed = __syncthreads_or(failed);
    if (failed && producer && lane == 0) {
        atomicCAS(status, 0, STATUS_TIMEOUT6);
        if (na > 0) tc::wait(fullA, (na - 1) & 1, limit_ns);
        if (nk > 0) tc::wait(fullK, (nk - 1) & 1, limit_ns);
        if (nf > 0) tc::wait(fwdb, (nf - 1) & 1, limit_ns);
        for (int c = 0; c < 3 && ni > 0; c++) tc::wait(invb + c, (ni - 1) & 1, limit_ns);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::dealloc(tbase, TMEM6);
    }
}

// K16 [kx][kz'][pair][ky'] of FP16 pairs (xx, yy), (zz, xy), (xz, yz) from the
// octant K [kx][ky'][kz' 6 + comp], scaled by s; rows padded to kyp16 entries
__global__ void k16_build_kernel(Geometry g, const float* __restrict__ K, __half2* __restrict__ K16, int kyp16, float s)
{
    const size_t total = (size_t)g.nkx * g.kzh * 3 * kyp16;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int kyp = (int)(i % kyp16);
        size_t r = i / kyp16;
        const int pair = (int)(r % 3);
        r /= 3;
        const int kzp = (int)(r % g.kzh);
        const int kx = (int)(r / g.kzh);
        float a = 0.f, b = 0.f;
        if (kyp < g.kyh) {
            const float* row = K + ((size_t)kx * g.kyh + kyp) * g.krow + kzp * 6 + 2 * pair;
            a = row[0] * s;
            b = row[1] * s;
        }
        K16[i] = __floats2half2_rn(a, b);
    }
}

}  // namespace

bool zconv_tc6_supported(const Geometry& g, int max_smem)
{
    // pz = 64 (17 <= nz <= 32), whole 128-column tiles on both sides of the ky fold
    return g.pz == 2 * HZ6 && g.nz >= 17 && g.nz <= HZ6 && g.py >= 2 * MT && g.py % MT == 0 && g.kzh == KZH6 &&
           SMEM6 <= (size_t)max_smem && g.lglmax >= 6;
}

int zconv_tc6_kyp16(const Geometry& g) { return g.py / 2 + 8; }
size_t zconv_tc6_y16_bytes(const Geometry& g) { return (size_t)g.nkx * 3 * 2 * g.nz * g.py * 2; }
size_t zconv_tc6_k16_bytes(const Geometry& g) { return (size_t)g.nkx * g.kzh * 3 * zconv_tc6_kyp16(g) * 4; }

cudaError_t zconv_tc6_build_k16(const Geometry& g, const float* K, void* K16, cudaStream_t st)
{
    const size_t total = (size_t)g.nkx * g.kzh * 3 * zconv_tc6_kyp16(g);
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 32);
    const float s = (float)((double)g.px * g.py * g.pz);
    k16_build_kernel<<<blocks, 256, 0, st>>>(g, K, (__half2*)K16, zconv_tc6_kyp16(g), s);
    return cudaGetLastError();
}

// Y16 [kx][c][part][z][ky] as the 5D tensor (ky%8, z, part, ky/8, kx c), boxes of
// (8, 32, 2, 16, 1); K16 as (ky', kz' pair, kx) of 32-bit pairs, boxes of (136, 99, 1)
cudaError_t zconv_tc6_maps(const Geometry& g, void* Y16, void* K16, void* ymap, void* kmap, bool fp16)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    {
        const cuuint64_t dims[5] = {64, (cuuint64_t)g.nz, 2, (cuuint64_t)g.py / 64, (cuuint64_t)g.nkx * 3};
        const cuuint64_t strides[4] = {(cuuint64_t)g.py * 2, (cuuint64_t)g.nz * g.py * 2, 128,
                                       (cuuint64_t)2 * g.nz * g.py * 2};
        const cuuint32_t box[5] = {64, (cuuint32_t)HZ6, 2, (cuuint32_t)MT / 64, 1};
        const cuuint32_t es[5] = {1, 1, 1, 1, 1};
        const CUresult r = enc(reinterpret_cast<CUtensorMap*>(ymap),
                               fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, Y16, dims,
                               strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    {
        const int kyp16 = zconv_tc6_kyp16(g);
        const cuuint64_t dims[3] = {(cuuint64_t)kyp16, (cuuint64_t)g.kzh * 3, (cuuint64_t)g.nkx};
        const cuuint64_t strides[2] = {(cuuint64_t)kyp16 * 4, (cuuint64_t)kyp16 * 4 * g.kzh * 3};
        const cuuint32_t box[3] = {(cuuint32_t)KW6, (cuuint32_t)(g.kzh * 3), 1};
        const cuuint32_t es[3] = {1, 1, 1};
        const CUresult r = enc(reinterpret_cast<CUtensorMap*>(kmap), CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, K16, dims,
                               strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t launch_zconv_tc6(const void* ymap_p, const void* kmap_p, const Geometry& g, void* Y16, const float2* tw,
                             int* status, uint32_t extra_tx, unsigned long long limit_ns, int nsm, cudaStream_t st,
                             bool fp16)
{
    const CUtensorMap& ymap = *reinterpret_cast<const CUtensorMap*>(ymap_p);
    const CUtensorMap& kmap = *reinterpret_cast<const CUtensorMap*>(kmap_p);
    const int ntiles = g.nkx * (g.py / MT);
    const int grid = std::min(ntiles, nsm);
    // BF16: the output carries the true scale (the kernel pairs' px py pz undone);
    // FP16: 1/128 keeps the length-64 inverse sums of products below 2^15, and
    // the y inverse pass divides by px py pz s / 128
    if (fp16) {
        cudaError_t e =
            cudaFuncSetAttribute(z_conv_tc6_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM6);
        if (e != cudaSuccess) return e;
        z_conv_tc6_kernel<true><<<grid, T6, SMEM6, st>>>(ymap, kmap, g, (unsigned short*)Y16, tw, 1.f / 128.f, status,
                                                         extra_tx, limit_ns);
    } else {
        cudaError_t e =
            cudaFuncSetAttribute(z_conv_tc6_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM6);
        if (e != cudaSuccess) return e;
        const float out_scale = (float)(1.0 / ((double)g.px * g.py * g.pz));
        z_conv_tc6_kernel<false><<<grid, T6, SMEM6, st>>>(ymap, kmap, g, (unsigned short*)Y16, tw, out_scale, status,
                                                          extra_tx, limit_ns);
    }
    return cudaGetLastError();
}

}  // namespace boris
