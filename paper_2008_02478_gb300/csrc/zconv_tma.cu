// z convolution of the split y-z schedule (Section 7: z transform, point-by-
// point kernel multiply, inverse z transform), FP32, as a persistent pipeline
// fed by the bulk-copy engine.
//
// Work unit: a tile of 32 consecutive ky columns of one kx plane, i.e. for
// each of the 3 nz lines (c, z) of Y[kx][c][z][ky] one 256-byte run.  Each
// CTA walks tiles blockIdx.x, + gridDim.x, ... and keeps one or two tile
// stages in shared memory.  A tile arrives as three 2D tensor copies (one
// 32 x nz box per component, completing on an mbarrier) and leaves the same
// way from its stage; with two stages the copy engine fills one while the
// threads compute the other.
// The kernel-spectrum rows of the tile are staged by the threads into a
// row-padded block (odd stride: the per-column reads hit distinct banks)
// after an L2 prefetch issued one tile earlier.
//
// Thread (column, component c, z parity h), six warps: as in the one-tile
// kernel, the zero-padded length-2 HZ z transform is computed as two
// length-HZ transforms (even outputs from x, odd outputs from x w^z), the
// 3 x 3 symmetric kernel multiply mixes the components of one parity through
// shared memory, and the inverse recombines the parities.
//
// Every mbarrier wait is bounded (device timer); when one gives up, the CTA
// latches BORIS_ERR_TIMEOUT in *status, waits (bounded) for its other copies
// in flight and returns.
#include <cudaTypedefs.h>

#include <mutex>

#include "boris_internal.cuh"
#include "bulk_async.cuh"

namespace boris {

namespace {

constexpr int TQ = 32;         // ky columns per tile: one 256-byte run per line
constexpr int TTHREADS = 192;  // (column, component, parity)
constexpr int STATUS_TIMEOUT = -5;  // BORIS_ERR_TIMEOUT

template <int HZ, int NS>
struct TmaLayout {
    static constexpr int KROW = ((HZ + 1) * 6 + 3) / 4 * 4;  // kernel row (kz' x 6 entries, padded to 16 bytes)
    static constexpr int KS = KROW + 1;                      // staged row stride (odd)
    static constexpr size_t stage = (size_t)3 * HZ * TQ * sizeof(float2);  // rows c HZ + z, 32 columns
    static constexpr size_t ks = ((size_t)TQ * KS * sizeof(float) + 15) / 16 * 16;
    static constexpr size_t total = (NS + 1) * stage + ks + 16;  // NS stages, odd-parity area, kernel rows, barriers
};

__device__ __forceinline__ int sym_entry(int i, int j) { return i == j ? i : (i + j == 1 ? 3 : (i + j == 2 ? 4 : 5)); }

// Point-by-point multiply of one parity's spectrum (Section 7): v[pos] holds
// component c at kz = 2 brev(pos) + H; m1, m2 point at the other two
// components' rows; k0..k2 at the column's kernel entries (c,c), (c,c1),
// (c,c2) of the octant row kz' = |kz| folded; s*n / s*f the entries' signs
// below / above the folding point.
template <int HZ, int H>
__device__ __forceinline__ void tma_multiply(float2 (&v)[HZ], const float* k0, const float* k1, const float* k2,
                                             const float2* m1, const float2* m2, float s1n, float s1f, float s2n,
                                             float s2f)
{
    constexpr int LGH = HZ == 2 ? 1 : HZ == 4 ? 2 : HZ == 8 ? 3 : HZ == 16 ? 4 : 5;
#pragma unroll
    for (int pos = 0; pos < HZ; pos++) {
        const int kz = 2 * (int)(__brev((unsigned)pos) >> (32 - LGH)) + H;  // compile-time
        const bool fz = kz > HZ;
        const int kzf = fz ? 2 * HZ - kz : kz;
        const float w0 = k0[kzf * 6];
        const float w1 = k1[kzf * 6] * (fz ? s1f : s1n);
        const float w2 = k2[kzf * 6] * (fz ? s2f : s2n);
        const float2 a = m1[pos * TQ], b = m2[pos * TQ];
        const float2 own = v[pos];
        v[pos] = float2{w0 * own.x + w1 * a.x + w2 * b.x, w0 * own.y + w1 * a.y + w2 * b.y};
    }
}

// NS tile stages per CTA (1: the next tile is fetched after the current one
// is stored, other CTAs on the SM hide the wait; 2: fetched while the current
// one is computed); MINB CTAs per SM for the register budget.
template <int HZ, int NS, int MINB>
__global__ void __launch_bounds__(TTHREADS, MINB)
    z_conv_tma_kernel(const __grid_constant__ CUtensorMap ymap, Geometry g, const float* __restrict__ K,
                      int* __restrict__ status, uint32_t extra_tx, unsigned long long limit_ns)
{
    using L = TmaLayout<HZ, NS>;
    constexpr int KROW = L::KROW, KS = L::KS;
    constexpr int SE = 3 * HZ * TQ;  // stage size in float2
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* stages = reinterpret_cast<float2*>(smem_raw);
    float2* odd = stages + NS * SE;
    float* Ks = reinterpret_cast<float*>(odd + SE);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (NS + 1) * L::stage + L::ks);

    const int nz = g.nz, lines = 3 * nz, py = g.py;
    const int nty = py / TQ;
    const int ntiles = g.nkx * nty;
    const int G = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ybytes = (uint32_t)lines * TQ * sizeof(float2);

    // thread 0: arm stage s for tile t and copy its three component boxes
    // (rows kx 3 nz + c nz .. + nz - 1, columns ky0 .. ky0 + 31) to rows c HZ ..
    auto issue_load = [&](int t, int s, uint32_t extra) {
        const int kx = t / nty, ky0 = (t - kx * nty) * TQ;
        mbar_arrive_expect_tx(&full[s], ybytes + extra);
        float2* dst = stages + s * SE;
        for (int c = 0; c < 3; c++) tma_load_2d(dst + c * HZ * TQ, &ymap, ky0, kx * lines + c * nz, &full[s]);
    };
    // first row of the kernel octant that tile (kx, ky0) reads: ky' = ky0 + col
    // below py/2, else py - ky0 - col (32 consecutive rows either way)
    auto krow0 = [&](int ky0) { return ky0 < py / 2 ? ky0 : py - ky0 - (TQ - 1); };

    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; i++) mbar_init(&full[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; i++)
            if ((int)blockIdx.x + i * G < ntiles) issue_load(blockIdx.x + i * G, i, i == 0 ? extra_tx : 0);
    }
    if (threadIdx.x == 32 && (int)blockIdx.x < ntiles) {
        const int t = blockIdx.x, kx = t / nty, ky0 = (t - kx * nty) * TQ;
        prefetch_l2(K + ((size_t)kx * g.kyh + krow0(ky0)) * KROW, TQ * KROW * sizeof(float));
    }

    // thread role
    const int col = lane, c = warp % 3, h = warp / 3;
    const int c1 = c == 0 ? 1 : 0, c2 = c == 2 ? 1 : 2;
    const int e0 = c, e1 = sym_entry(c, c1), e2 = sym_entry(c, c2);
    // signs of the folded octant entries: xy and yz are odd in ky, xz and yz
    // odd in kz; e1 is odd in kz only for c = 2 (xz), e2 always (xz or yz)
    const float* k0 = Ks + col * KS + e0;
    const float* k1 = Ks + col * KS + e1;
    const float* k2 = Ks + col * KS + e2;

    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += G, k++) {
        const int s = NS == 1 ? 0 : k % NS;
        const int kx = t / nty, ky0 = (t - kx * nty) * TQ;
        if (threadIdx.x == 32 && t + G < ntiles) {
            const int tn = t + G, kxn = tn / nty, kyn = (tn - kxn * nty) * TQ;
            prefetch_l2(K + ((size_t)kxn * g.kyh + krow0(kyn)) * KROW, TQ * KROW * sizeof(float));
        }
        // kernel rows of the tile's 32 columns
        {
            const float* Kx = K + (size_t)kx * g.kyh * KROW;
            constexpr int vrow = KROW / 4;
            staged_loop<TTHREADS, float4>(TQ * vrow, [&](int i) {
                const int cc = i / vrow, o = i - cc * vrow;
                const int ky = ky0 + cc;
                const int kyf = ky > py / 2 ? py - ky : ky;
                return reinterpret_cast<const float4*>(Kx + (size_t)kyf * KROW)[o];
            }, [&](int i, float4 v4) {
                const int cc = i / vrow, o = i - cc * vrow;
                float* d = Ks + cc * KS + o * 4;
                d[0] = v4.x;
                d[1] = v4.y;
                d[2] = v4.z;
                d[3] = v4.w;
            });
        }
        const bool ok = mbar_wait_bounded(&full[s], (k / NS) & 1, limit_ns);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicCAS(status, 0, STATUS_TIMEOUT);
                // the other stages' copies, if issued, land before the CTA leaves
                for (int i = 1; i < NS; i++)
                    if (t + i * G < ntiles) mbar_wait_bounded(&full[(k + i) % NS], ((k + i) / NS) & 1, limit_ns);
            }
            if (threadIdx.x == 0) bulk_wait0();
            return;
        }
        float2* A = stages + s * SE;
        // forward: even outputs from x, odd outputs from x w_(2HZ)^z
        float2 v[HZ];
#pragma unroll
        for (int z = 0; z < HZ; z++) {
            float2 x = z < nz ? A[(c * HZ + z) * TQ + col] : float2{0.f, 0.f};
            if (h) x = c_mul(x, w128lit<float2>(z * (64 / HZ)));
            v[z] = x;
        }
        reg_fft<HZ, -1>(v);
        __syncthreads();  // every input row read
        float2* spec = h ? odd : A;  // [c][pos][col] of this parity
#pragma unroll
        for (int pos = 0; pos < HZ; pos++) spec[(c * HZ + pos) * TQ + col] = v[pos];
        __syncthreads();
        {
            const bool fy = ky0 + col > py / 2;
            const float a1 = (fy && (e1 == 3 || e1 == 5)) ? -1.f : 1.f;
            const float a2 = (fy && (e2 == 3 || e2 == 5)) ? -1.f : 1.f;
            const float s1f = c == 2 ? -a1 : a1;
            const float2* m1 = spec + c1 * HZ * TQ + col;
            const float2* m2 = spec + c2 * HZ * TQ + col;
            if (h) tma_multiply<HZ, 1>(v, k0, k1, k2, m1, m2, a1, s1f, a2, -a2);
            else tma_multiply<HZ, 0>(v, k0, k1, k2, m1, m2, a1, s1f, a2, -a2);
        }
        reg_fft<HZ, 1>(v);
        __syncthreads();  // spectra consumed
        // out[z] = even[z] + w^(-z) odd[z] for z < nz, the two parities
        // splitting the work: the odd thread hands over z < HZ/2, the even
        // thread z >= HZ/2, and each finishes the other half
        constexpr int HH = HZ / 2;
        float2* x = odd + c * HZ * TQ + col;
        if (h) {
#pragma unroll
            for (int z = 0; z < HH; z++)
                if (z < nz) x[z * TQ] = c_mulc(v[z], w128lit<float2>(z * (64 / HZ)));
        } else {
#pragma unroll
            for (int z = HH; z < HZ; z++)
                if (z < nz) x[z * TQ] = v[z];
        }
        __syncthreads();
        float2* o = A + c * HZ * TQ + col;
        if (h) {
#pragma unroll
            for (int z = HH; z < HZ; z++)
                if (z < nz) o[z * TQ] = c_add(x[z * TQ], c_mulc(v[z], w128lit<float2>(z * (64 / HZ))));
        } else {
#pragma unroll
            for (int z = 0; z < HH; z++)
                if (z < nz) o[z * TQ] = c_add(v[z], x[z * TQ]);
        }
        fence_proxy_async_smem();  // the rows just written are read by the bulk stores
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int cc = 0; cc < 3; cc++) tma_store_2d(&ymap, ky0, kx * lines + cc * nz, A + cc * HZ * TQ);
            bulk_commit();
            bulk_wait_read0();
            if (t + NS * G < ntiles) issue_load(t + NS * G, s, 0);
        }
    }
    if (threadIdx.x == 0) bulk_wait0();
}

template <int HZ, int NS, int MINB>
cudaError_t launch_v(const CUtensorMap& ymap, const Geometry& g, const float* K, int* status, uint32_t extra_tx,
                     unsigned long long limit_ns, int nsm, cudaStream_t st)
{
    const size_t smem = TmaLayout<HZ, NS>::total;
    auto kern = z_conv_tma_kernel<HZ, NS, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int ntiles = g.nkx * (g.py / TQ);
    const int grid = ntiles < MINB * nsm ? ntiles : MINB * nsm;
    kern<<<grid, TTHREADS, smem, st>>>(ymap, g, K, status, extra_tx, limit_ns);
    return cudaGetLastError();
}

template <int HZ>
cudaError_t launch_hz(const CUtensorMap& ymap, const Geometry& g, const float* K, int* status, uint32_t extra_tx,
                      unsigned long long limit_ns, int nsm, int variant, cudaStream_t st)
{
    if (variant == 2) return launch_v<HZ, 2, 2>(ymap, g, K, status, extra_tx, limit_ns, nsm, st);
    return launch_v<HZ, 1, 3>(ymap, g, K, status, extra_tx, limit_ns, nsm, st);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn_once()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

size_t tma_smem(int hz, int variant)
{
    const bool two = variant == 2;
    switch (hz) {
    case 2: return two ? TmaLayout<2, 2>::total : TmaLayout<2, 1>::total;
    case 4: return two ? TmaLayout<4, 2>::total : TmaLayout<4, 1>::total;
    case 8: return two ? TmaLayout<8, 2>::total : TmaLayout<8, 1>::total;
    case 16: return two ? TmaLayout<16, 2>::total : TmaLayout<16, 1>::total;
    case 32: return two ? TmaLayout<32, 2>::total : TmaLayout<32, 1>::total;
    default: return 0;
    }
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return encode_fn_once(); }

bool zconv_tma_supported(const Geometry& g, int max_smem, int variant)
{
    const int hz = g.pz / 2;
    const size_t smem = tma_smem(hz, variant);
    // py >= 64: py / 2 is a multiple of 32, so every tile reads 32 consecutive octant rows
    return smem > 0 && g.py >= 2 * TQ && g.py % TQ == 0 && g.nz <= hz && smem <= (size_t)max_smem &&
           g.krow == ((hz + 1) * 6 + 3) / 4 * 4;
}

cudaError_t zconv_tma_map(const Geometry& g, float2* Y, void* map)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    // Y[kx][c][z][ky] as a 2D array of complex (8-byte) elements: rows
    // (kx, c, z), py columns; boxes of 32 columns x nz rows
    const cuuint64_t dims[2] = {(cuuint64_t)g.py, (cuuint64_t)g.nkx * 3 * g.nz};
    const cuuint64_t strides[1] = {(cuuint64_t)g.py * sizeof(float2)};
    const cuuint32_t box[2] = {(cuuint32_t)TQ, (cuuint32_t)g.nz};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, Y, dims, strides, box,
                           es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_zconv_tma(const void* map, const Geometry& g, const float* K, int* status, uint32_t extra_tx,
                             unsigned long long limit_ns, int nsm, int variant, cudaStream_t st)
{
    const CUtensorMap& ymap = *reinterpret_cast<const CUtensorMap*>(map);
    switch (g.pz / 2) {
    case 2: return launch_hz<2>(ymap, g, K, status, extra_tx, limit_ns, nsm, variant, st);
    case 4: return launch_hz<4>(ymap, g, K, status, extra_tx, limit_ns, nsm, variant, st);
    case 8: return launch_hz<8>(ymap, g, K, status, extra_tx, limit_ns, nsm, variant, st);
    case 16: return launch_hz<16>(ymap, g, K, status, extra_tx, limit_ns, nsm, variant, st);
    case 32: return launch_hz<32>(ymap, g, K, status, extra_tx, limit_ns, nsm, variant, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace boris
