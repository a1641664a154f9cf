// z convolution of the split y-z schedule (Section 7: z transform, point-by-
// point kernel multiply, inverse z transform), FP32, with the zero-padded
// length-P (P = 2 HZ) z transform split by output residue kz mod 4.
//
// For input x[z], z < HZ, and L = P / 4, the outputs kz = 4 j + r are
//   X[4 j + r] = sum_{z' < L} w_L^(z' j) y_r[z'],
//   y_r[z'] = w_P^(z' r) (x[z'] + (-i)^r x[z' + L]),
// i.e. one length-L transform per residue r.  The inverse, cropped to z < HZ,
//   out[z'] = sum_r v_r[z'],  out[z' + L] = sum_r i^r v_r[z'],
//   v_r[z'] = w_P^(-z' r) u_r[z'],  u_r = unscaled inverse length-L transform,
// recombines the residues.
//
// Work unit: a tile of 32 consecutive ky columns of one kx plane.  Warp r of
// a CTA owns residue r for the tile's 32 columns (lane = column) and holds
// the three components' length-L spectra in registers, so the 3 x 3 kernel
// multiply at kz = 4 j + r needs no exchange between threads.  A tile arrives
// by three 2D tensor copies (one 32 x nz box per component) into a stage that
// is refilled with the next tile as soon as every thread has read it; the
// recombination goes through a small per-component scratch and the results
// are stored straight to global memory (coalesced 256-byte rows).
//
// The kernel spectrum is read in a blocked copy K2 [kx][b][kz'][pair][34]
// (pairs (xx,yy), (zz,xy), (xz,yz); entry (b, e) is ky' = 32 b + e for
// e <= 32, e = 33 is padding), so that the 32 columns of any tile - ky' =
// ky0 + col below the ky fold, py - ky0 - col above it - lie in one block:
// a tile's kernel rows are one 2D tensor copy (34 x 3 (HZ + 1) entries),
// issued one tile ahead into a kernel stage.
//
// Two shared-memory plans: SEPARATE (kernel stage, scratch and input stage
// apart, the next tile's kernel rows fetched right after the multiply; three
// CTAs per SM) and shared (the scratch overlays the kernel stage, which is
// refilled after the recombination; four CTAs per SM).
//
// Every mbarrier wait is bounded (device timer); when one gives up, the CTA
// latches BORIS_ERR_TIMEOUT in *status, waits (bounded) for its other copy in
// flight and returns.
#include <cudaTypedefs.h>

#include "boris_internal.cuh"
#include "bulk_async.cuh"

namespace boris {

namespace {

constexpr int RQ = 32;              // ky columns per tile
constexpr int RTHREADS = 128;       // 4 residue warps
constexpr int KBW = 34;             // entries per K2 block row (ky' = 32 b .. 32 b + 32, one pad)
constexpr int STATUS_TIMEOUT = -5;  // BORIS_ERR_TIMEOUT

// NP: kernel pairs per kz' (3 for the symmetric demagnetising tensor, 2 for
// the Oersted vector: (Gx, Gy), (Gz, 0))
template <int HZ, bool SEPARATE, int NP = 3>
struct ResLayout {
    static constexpr int L = HZ / 2;
    static constexpr int KROWS = (HZ + 1) * NP;
    static constexpr size_t stage = (size_t)3 * HZ * RQ * sizeof(float2);      // rows c HZ + z, 32 columns
    static constexpr size_t kstage = (size_t)KROWS * KBW * sizeof(float2);    // rows kz' 3 + pair
    static constexpr size_t scratch = (size_t)L * 4 * RQ * sizeof(float2);    // [z'][r][column]
    static_assert(SEPARATE || scratch <= kstage, "scratch overlays the kernel stage");
    static constexpr size_t kstage_off = stage;
    static constexpr size_t scratch_off = SEPARATE ? stage + (kstage + 127) / 128 * 128 : stage;
    static constexpr size_t bar_off = (SEPARATE ? scratch_off + scratch : stage + kstage + 15) / 16 * 16;
    // per residue r: L entries w_P^(z r), L entries w_P^(z r) (-i)^r
    static constexpr size_t tw_off = bar_off + 16;
    static constexpr size_t total = tw_off + (size_t)4 * 2 * L * sizeof(float2);
};

constexpr int lg2c(int v) { return v <= 1 ? 0 : 1 + lg2c(v / 2); }
// bit reversal of the lg low bits; a plain loop, so that an unrolled caller's
// constant argument folds to a constant (no call, no run-time branches on it)
__host__ __device__ __forceinline__ constexpr int brevc(int v, int lg)
{
    int r = 0;
    for (int i = 0; i < lg; i++) r |= ((v >> i) & 1) << (lg - 1 - i);
    return r;
}

__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 w)  // acc + a w
{
    return float2{acc.x + a.x * w.x - a.y * w.y, acc.y + a.x * w.y + a.y * w.x};
}

// One component's residues (v = v_r of this thread) through the scratch
// [z'][r][column]; thread (column, r) writes out[z'] and out[z' + L] for
// z' = r, r + 4, ... (rows of py complex values, cropped to nz).
template <int L, bool FULL>
__device__ __forceinline__ void recombine(const float2 (&v)[L], float2* scr, float2* out, int r, int col, int nz,
                                          int py)
{
#pragma unroll
    for (int z = 0; z < L; z++) scr[(z * 4 + r) * RQ + col] = v[z];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < (L + 3) / 4; i++) {
        const int z = r + 4 * i;
        if (L % 4 == 0 || z < L) {  // r < 4: always true when 4 divides L
            const float2 a0 = scr[(z * 4 + 0) * RQ + col], a1 = scr[(z * 4 + 1) * RQ + col];
            const float2 a2 = scr[(z * 4 + 2) * RQ + col], a3 = scr[(z * 4 + 3) * RQ + col];
            const float2 s02 = c_add(a0, a2), d02 = c_sub(a0, a2);
            const float2 s13 = c_add(a1, a3), d13 = c_sub(a1, a3);
            if (FULL || z < nz) out[(size_t)z * py] = c_add(s02, s13);
            if (FULL || z + L < nz) out[(size_t)(z + L) * py] = float2{d02.x - d13.y, d02.y + d13.x};  // d02 + i d13
        }
    }
    __syncthreads();
}

// The 3 x 3 demagnetising multiply of one thread's L accumulator positions
// (kz = 4 brev(pos) + r): kernel row kz' = kz up to the z Nyquist index HZ,
// else P - kz with xz and yz negated; FY (the tile lies above the ky fold)
// negates xy and yz.  Both signs are compile-time constants here, and the
// products of the real entries with the complex components run as packed
// FP32x2 multiply-adds.
template <int L, int LGL, int HZ, int NP, bool FY>
__device__ __forceinline__ void res_multiply(float2 (&v0)[L], float2 (&v1)[L], float2 (&v2)[L], const float2* Kup,
                                             const float2* Kdn, int r)
{
    constexpr int P = 2 * HZ;
#pragma unroll
    for (int pos = 0; pos < L; pos++) {
        const int j = brevc(pos, LGL);
        const float2* kp;
        float sz;
        if (4 * j < HZ) {
            kp = Kup + 4 * j * NP * KBW;
            sz = 1.f;
        } else if (4 * j > HZ) {
            kp = Kdn + (P - 4 * j) * NP * KBW;
            sz = -1.f;
        } else {
            kp = Kdn + HZ * NP * KBW;  // kz = HZ + r: the Nyquist row for r = 0
            sz = r == 0 ? 1.f : -1.f;
        }
        const float2 m0 = v0[pos], m1 = v1[pos], m2 = v2[pos];
        const float2 p0 = kp[0], p1 = kp[KBW], p2 = kp[2 * KBW];
        const float sy = FY ? -1.f : 1.f;
        const float2 xx = make_float2(p0.x, p0.x), yy = make_float2(p0.y, p0.y), zz = make_float2(p1.x, p1.x);
        const float xys = p1.y * sy, xzs = p2.x * sz, yzs = p2.y * (sy * sz);
        const float2 xy = make_float2(xys, xys), xz = make_float2(xzs, xzs), yz = make_float2(yzs, yzs);
        v0[pos] = __ffma2_rn(xz, m2, __ffma2_rn(xy, m1, __fmul2_rn(xx, m0)));
        v1[pos] = __ffma2_rn(yz, m2, __ffma2_rn(yy, m1, __fmul2_rn(xy, m0)));
        v2[pos] = __ffma2_rn(zz, m2, __ffma2_rn(yz, m1, __fmul2_rn(xz, m0)));
    }
}

// FULL: nz == HZ (no cropped rows: no predicates on the loads and stores).
// CURL: the Oersted multiply H^ = i (J^ x G) instead of the symmetric 3 x 3
// demagnetising multiply.
template <int HZ, int MINB, bool FULL, bool SEPARATE, bool CURL = false>
__global__ void __launch_bounds__(RTHREADS, MINB)
    z_conv_res_kernel(const __grid_constant__ CUtensorMap ymap, const __grid_constant__ CUtensorMap kmap, Geometry g,
                      int nkb, float2* __restrict__ Y, int* __restrict__ status, uint32_t extra_tx,
                      unsigned long long limit_ns)
{
    constexpr int NP = CURL ? 2 : 3;
    using Lay = ResLayout<HZ, SEPARATE, NP>;
    constexpr int L = Lay::L, LGL = lg2c(L), P = 2 * HZ, S = 128 / P, KROWS = Lay::KROWS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* stage = reinterpret_cast<float2*>(smem_raw);
    float2* kst = reinterpret_cast<float2*>(smem_raw + Lay::kstage_off);
    float2* scr = reinterpret_cast<float2*>(smem_raw + Lay::scratch_off);
    uint64_t* fullY = reinterpret_cast<uint64_t*>(smem_raw + Lay::bar_off);
    uint64_t* fullK = fullY + 1;

    const int nz = FULL ? HZ : g.nz, lines = 3 * nz, py = g.py;
    const int nty = py / RQ;
    const int ntiles = g.nkx * nty;
    const int G = gridDim.x;
    const int r = threadIdx.x >> 5, col = threadIdx.x & 31;
    const uint32_t ybytes = (uint32_t)lines * RQ * sizeof(float2);
    constexpr uint32_t kbytes = (uint32_t)KROWS * KBW * sizeof(float2);

    auto load_y = [&](int t, uint32_t extra) {
        const int kx = t / nty, ky0 = (t - kx * nty) * RQ;
        mbar_arrive_expect_tx(fullY, ybytes + extra);
        for (int c = 0; c < 3; c++) tma_load_2d(stage + c * HZ * RQ, &ymap, ky0, kx * lines + c * nz, fullY);
    };
    // the kernel block of tile t: b = ky0 / 32 below the fold, (py - ky0 - 31) / 32 above it
    auto load_k = [&](int t) {
        const int kx = t / nty, ky0 = (t - kx * nty) * RQ;
        const int b = ky0 >= py / 2 ? (py - ky0 - (RQ - 1)) / 32 : ky0 / 32;
        mbar_arrive_expect_tx(fullK, kbytes);
        tma_load_2d(kst, &kmap, 0, (kx * nkb + b) * KROWS, fullK);
    };

    // the warp's twiddle rows at compile-time offsets (no index arithmetic per use)
    float2* twr = reinterpret_cast<float2*>(smem_raw + Lay::tw_off);
    for (int i = threadIdx.x; i < 4 * 2 * L; i += RTHREADS) {
        const int rr = i / (2 * L), k = i - rr * 2 * L, z = k % L;
        twr[i] = c_w128f[(S * z * rr + (k >= L ? 32 * rr : 0)) & 127];
    }
    const float2* twa = twr + r * 2 * L;  // w_P^(z r)
    const float2* twb = twa + L;          // w_P^(z r) (-i)^r
    if (threadIdx.x == 0) {
        mbar_init(fullY, 1);
        mbar_init(fullK, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) {
        load_y(blockIdx.x, extra_tx);
        load_k(blockIdx.x);
    }

    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += G, k++) {
        const int kx = t / nty, ky0 = (t - kx * nty) * RQ;
        const bool more = t + G < ntiles;
        {
            const bool ok = mbar_wait_bounded(fullY, k & 1, limit_ns);
            if (__syncthreads_or(!ok)) {
                // the kernel rows of this tile are in flight: let them land first
                if (threadIdx.x == 0) {
                    atomicCAS(status, 0, STATUS_TIMEOUT);
                    mbar_wait_bounded(fullK, k & 1, limit_ns);
                }
                return;
            }
        }
        // fold and twiddle: v_c[z'] = y_r[z'] of component c
        float2 v0[L], v1[L], v2[L];
        {
            const float2* A = stage + col;
#pragma unroll
            for (int z = 0; z < L; z++) {
                const float2 ta = twa[z];
                const float2 tb = twb[z];
                const bool lo = FULL || z < nz, hi = FULL || z + L < nz;
                const float2 f0{0.f, 0.f};
                const float2 a0 = lo ? A[(0 * HZ + z) * RQ] : f0, b0 = hi ? A[(0 * HZ + z + L) * RQ] : f0;
                const float2 a1 = lo ? A[(1 * HZ + z) * RQ] : f0, b1 = hi ? A[(1 * HZ + z + L) * RQ] : f0;
                const float2 a2 = lo ? A[(2 * HZ + z) * RQ] : f0, b2 = hi ? A[(2 * HZ + z + L) * RQ] : f0;
                v0[z] = cfma(c_mul(a0, ta), b0, tb);
                v1[z] = cfma(c_mul(a1, ta), b1, tb);
                v2[z] = cfma(c_mul(a2, ta), b2, tb);
            }
        }
        __syncthreads();  // the input stage is consumed: refill it with the next tile
        if (threadIdx.x == 0 && more) {
            fence_proxy_async_smem();
            load_y(t + G, 0);
        }
        reg_fft<L, -1>(v0);
        reg_fft<L, -1>(v1);
        reg_fft<L, -1>(v2);
        {
            const bool ok = mbar_wait_bounded(fullK, k & 1, limit_ns);
            if (__syncthreads_or(!ok)) {
                // the next tile's input is in flight: let it land first
                if (threadIdx.x == 0) {
                    atomicCAS(status, 0, STATUS_TIMEOUT);
                    if (more) mbar_wait_bounded(fullY, (k + 1) & 1, limit_ns);
                }
                return;
            }
        }
        // v_c[pos] = component c at kz = 4 brev(pos) + r.  Kernel row kz' = kz
        // up to the z Nyquist index HZ, else P - kz with xz and yz negated;
        // ky beyond py / 2 reads ky' = py - ky with xy and yz negated.
        {
            const bool fy = ky0 >= py / 2;
            const float2* Kc = kst + (fy ? 32 - col : col);
            const float2* Kup = Kc + r * NP * KBW;  // rows 4 j + r
            const float2* Kdn = Kc - r * NP * KBW;  // rows P - 4 j - r
            if (!CURL) {
                if (fy) res_multiply<L, LGL, HZ, NP, true>(v0, v1, v2, Kup, Kdn, r);
                else res_multiply<L, LGL, HZ, NP, false>(v0, v1, v2, Kup, Kdn, r);
            } else {
                const float sy = fy ? -1.f : 1.f;
#pragma unroll
                for (int pos = 0; pos < L; pos++) {
                    const int j = brevc(pos, LGL);
                    const float2* kp;
                    float sz;
                    if (4 * j < HZ) {
                        kp = Kup + 4 * j * NP * KBW;
                        sz = 1.f;
                    } else if (4 * j > HZ) {
                        kp = Kdn + (P - 4 * j) * NP * KBW;
                        sz = -1.f;
                    } else {
                        kp = Kdn + HZ * NP * KBW;  // kz = HZ + r: the Nyquist row for r = 0
                        sz = r == 0 ? 1.f : -1.f;
                    }
                    const float2 m0 = v0[pos], m1 = v1[pos], m2 = v2[pos];
                    // Gx odd in kx only, Gy odd in ky, Gz odd in kz; H^ = i (J^ x G)
                    const float2 p0 = kp[0], p1 = kp[KBW];
                    const float gx = p0.x, gy = p0.y * sy, gz = p1.x * sz;
                    const float2 c0{m1.x * gz - m2.x * gy, m1.y * gz - m2.y * gy};
                    const float2 c1{m2.x * gx - m0.x * gz, m2.y * gx - m0.y * gz};
                    const float2 c2{m0.x * gy - m1.x * gx, m0.y * gy - m1.y * gx};
                    v0[pos] = float2{-c0.y, c0.x};
                    v1[pos] = float2{-c1.y, c1.x};
                    v2[pos] = float2{-c2.y, c2.x};
                }
            }
        }
        if (SEPARATE) {
            __syncthreads();  // the kernel stage is consumed: fetch the next tile's rows
            if (threadIdx.x == 0 && more) {
                fence_proxy_async_smem();
                load_k(t + G);
            }
        }
        reg_fft<L, 1>(v0);
        reg_fft<L, 1>(v1);
        reg_fft<L, 1>(v2);
#pragma unroll
        for (int z = 0; z < L; z++) {
            const float2 w = twa[z];
            v0[z] = c_mulc(v0[z], w);
            v1[z] = c_mulc(v1[z], w);
            v2[z] = c_mulc(v2[z], w);
        }
        // recombine the residues, one component at a time; without SEPARATE
        // the scratch overlays the kernel stage, so every thread must be past
        // its multiply first, and the scratch is published to the async proxy
        // before the next kernel rows are copied over it
        float2* out = Y + ((size_t)kx * 3 * nz) * py + ky0 + col;
        if (!SEPARATE) __syncthreads();
        recombine<L, FULL>(v0, scr, out, r, col, nz, py);
        recombine<L, FULL>(v1, scr, out + (size_t)nz * py, r, col, nz, py);
        recombine<L, FULL>(v2, scr, out + (size_t)2 * nz * py, r, col, nz, py);
        if (!SEPARATE && more) {
            fence_proxy_async_smem();
            __syncthreads();
            if (threadIdx.x == 0) load_k(t + G);
        }
    }
}

template <int HZ, int MINB, bool SEPARATE>
cudaError_t launch_hz(const CUtensorMap& ymap, const CUtensorMap& kmap, const Geometry& g, int nkb, float2* Y,
                      int* status, uint32_t extra_tx, unsigned long long limit_ns, int nsm, cudaStream_t st)
{
    const size_t smem = ResLayout<HZ, SEPARATE>::total;
    auto kern = g.nz == HZ ? z_conv_res_kernel<HZ, MINB, true, SEPARATE> : z_conv_res_kernel<HZ, MINB, false, SEPARATE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int ntiles = g.nkx * (g.py / RQ);
    const int grid = ntiles < MINB * nsm ? ntiles : MINB * nsm;
    kern<<<grid, RTHREADS, smem, st>>>(ymap, kmap, g, nkb, Y, status, extra_tx, limit_ns);
    return cudaGetLastError();
}

template <bool SEPARATE>
size_t res_smem(int hz)
{
    switch (hz) {
    case 4: return ResLayout<4, SEPARATE>::total;
    case 8: return ResLayout<8, SEPARATE>::total;
    case 16: return ResLayout<16, SEPARATE>::total;
    case 32: return ResLayout<32, SEPARATE>::total;
    default: return 0;
    }
}

// K2[kx][b][kz'][p][e] = (K[kx][ky'][kz' 6 + 2p], K[kx][ky'][kz' 6 + 2p + 1]) with
// ky' = 32 b + e (e <= 32); zero for e = 33 and ky' >= kyh
__global__ void k2_build_kernel(Geometry g, const float* __restrict__ K, float2* __restrict__ K2, int nkb)
{
    const size_t total = (size_t)g.nkx * nkb * g.kzh * 3 * KBW;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(i % KBW);
        size_t rest = i / KBW;
        const int p = (int)(rest % 3);
        rest /= 3;
        const int kz = (int)(rest % g.kzh);
        rest /= g.kzh;
        const int b = (int)(rest % nkb);
        const size_t kx = rest / nkb;
        const int ky = b * 32 + e;
        K2[i] = (e <= 32 && ky < g.kyh)
                    ? *reinterpret_cast<const float2*>(K + (kx * g.kyh + ky) * g.krow + kz * 6 + 2 * p)
                    : float2{0.f, 0.f};
    }
}

// K2c[kx][b][kz'][p][e] from KO[kx][ky'][kz'][4]: p = 0 (Gx, Gy), p = 1 (Gz, 0);
// ky' = 32 b + e (e <= 32); zero for e = 33 and ky' >= kyh
__global__ void k2_curl_build_kernel(Geometry g, const float* __restrict__ KO, float2* __restrict__ K2, int nkb)
{
    const size_t total = (size_t)g.nkx * nkb * g.kzh * 2 * KBW;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(i % KBW);
        size_t rest = i / KBW;
        const int p = (int)(rest % 2);
        rest /= 2;
        const int kz = (int)(rest % g.kzh);
        rest /= g.kzh;
        const int b = (int)(rest % nkb);
        const size_t kx = rest / nkb;
        const int ky = b * 32 + e;
        float2 v{0.f, 0.f};
        if (e <= 32 && ky < g.kyh) {
            const float* q = KO + ((kx * g.kyh + ky) * g.kzh + kz) * 4;
            v = p == 0 ? float2{q[0], q[1]} : float2{q[2], 0.f};
        }
        K2[i] = v;
    }
}

// pz = 1: H^(kx, ky) = i (J^ x G) on Y[kx][c][0][ky] in place; Gy odd in ky
__global__ void curl_point_kernel(Geometry g, float2* __restrict__ Y, const float* __restrict__ KO)
{
    const size_t total = (size_t)g.nkx * g.py;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int ky = (int)(t % g.py);
        const size_t kx = t / g.py;
        const bool fy = ky > g.py / 2;
        const int kyf = fy ? g.py - ky : ky;
        const float* q = KO + (kx * g.kyh + kyf) * g.kzh * 4;
        const float gx = q[0], gy = fy ? -q[1] : q[1], gz = q[2];
        float2* y0 = Y + (kx * 3 + 0) * g.py + ky;
        float2* y1 = Y + (kx * 3 + 1) * g.py + ky;
        float2* y2 = Y + (kx * 3 + 2) * g.py + ky;
        const float2 m0 = *y0, m1 = *y1, m2 = *y2;
        const float2 c0{m1.x * gz - m2.x * gy, m1.y * gz - m2.y * gy};
        const float2 c1{m2.x * gx - m0.x * gz, m2.y * gx - m0.y * gz};
        const float2 c2{m0.x * gy - m1.x * gx, m0.y * gy - m1.y * gx};
        *y0 = float2{-c0.y, c0.x};
        *y1 = float2{-c1.y, c1.x};
        *y2 = float2{-c2.y, c2.x};
    }
}

template <int HZ>
cudaError_t launch_curl_hz(const CUtensorMap& ymap, const CUtensorMap& kmap, const Geometry& g, int nkb, float2* Y,
                           int* status, unsigned long long limit_ns, int nsm, cudaStream_t st)
{
    constexpr int MINB = 3;
    const size_t smem = ResLayout<HZ, true, 2>::total;
    auto kern = g.nz == HZ ? z_conv_res_kernel<HZ, MINB, true, true, true> : z_conv_res_kernel<HZ, MINB, false, true, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int ntiles = g.nkx * (g.py / RQ);
    const int grid = ntiles < MINB * nsm ? ntiles : MINB * nsm;
    kern<<<grid, RTHREADS, smem, st>>>(ymap, kmap, g, nkb, Y, status, 0u, limit_ns);
    return cudaGetLastError();
}

}  // namespace

// ky' blocks per kx plane of K2: tiles start at block ky0 / 32 (below the
// fold) or (py - ky0 - 31) / 32 (above it), both below py / 64
int zconv_res_nkb(const Geometry& g) { return g.py / 64; }

size_t zconv_res_k2_bytes(const Geometry& g)
{
    return (size_t)g.nkx * zconv_res_nkb(g) * g.kzh * 3 * KBW * sizeof(float2);
}

bool zconv_res_supported(const Geometry& g, int max_smem)
{
    const int hz = g.pz / 2;
    const size_t smem = res_smem<true>(hz);
    // py >= 64: py / 2 is a multiple of 32, so a tile lies wholly on one side of the ky fold;
    // the kernel block's 3 (HZ + 1) <= 99 rows fit a tensor-copy box (<= 256 rows)
    return smem > 0 && g.py >= 2 * RQ && g.py % RQ == 0 && g.nz <= hz && smem <= (size_t)max_smem &&
           g.krow == ((hz + 1) * 6 + 3) / 4 * 4;
}

cudaError_t zconv_res_build_k2(const Geometry& g, const float* K, float2* K2, cudaStream_t st)
{
    k2_build_kernel<<<1024, 256, 0, st>>>(g, K, K2, zconv_res_nkb(g));
    return cudaGetLastError();
}

// K2 as a 2D array of 8-byte elements: rows (kx, b, kz', p), 34 columns
// (272-byte rows); boxes of 34 x 3 (HZ + 1)
cudaError_t zconv_res_kmap(const Geometry& g, float2* K2, void* map)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t rows = (cuuint64_t)g.nkx * zconv_res_nkb(g) * g.kzh * 3;
    const cuuint64_t dims[2] = {(cuuint64_t)KBW, rows};
    const cuuint64_t strides[1] = {(cuuint64_t)KBW * sizeof(float2)};
    const cuuint32_t box[2] = {(cuuint32_t)KBW, (cuuint32_t)(g.kzh * 3)};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, K2, dims, strides,
                           box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_zconv_res(const void* ymap_p, const void* kmap_p, const Geometry& g, float2* Y, int* status,
                             uint32_t extra_tx, unsigned long long limit_ns, int nsm, int ctas_per_sm, cudaStream_t st)
{
    const CUtensorMap& ymap = *reinterpret_cast<const CUtensorMap*>(ymap_p);
    const CUtensorMap& kmap = *reinterpret_cast<const CUtensorMap*>(kmap_p);
    const int nkb = zconv_res_nkb(g);
#define RES_CASE(HZ)                                                                                                   \
    case HZ:                                                                                                           \
        return ctas_per_sm == 3                                                                                        \
                   ? launch_hz<HZ, 3, true>(ymap, kmap, g, nkb, Y, status, extra_tx, limit_ns, nsm, st)                \
                   : launch_hz<HZ, 4, false>(ymap, kmap, g, nkb, Y, status, extra_tx, limit_ns, nsm, st);
    switch (g.pz / 2) {
        RES_CASE(4)
        RES_CASE(8)
        RES_CASE(16)
        RES_CASE(32)
    default: return cudaErrorInvalidValue;
    }
#undef RES_CASE
}

bool zconv_res_curl_supported(const Geometry& g, int max_smem)
{
    const int hz = g.pz / 2;
    size_t smem = 0;
    switch (hz) {
    case 4: smem = ResLayout<4, true, 2>::total; break;
    case 8: smem = ResLayout<8, true, 2>::total; break;
    case 16: smem = ResLayout<16, true, 2>::total; break;
    case 32: smem = ResLayout<32, true, 2>::total; break;
    default: return false;
    }
    return g.py >= 2 * RQ && g.py % RQ == 0 && g.nz <= hz && smem <= (size_t)max_smem;
}

size_t zconv_res_k2_curl_bytes(const Geometry& g)
{
    return (size_t)g.nkx * zconv_res_nkb(g) * g.kzh * 2 * KBW * sizeof(float2);
}

cudaError_t zconv_res_build_k2_curl(const Geometry& g, const float* KO, float2* K2, cudaStream_t st)
{
    k2_curl_build_kernel<<<1024, 256, 0, st>>>(g, KO, K2, zconv_res_nkb(g));
    return cudaGetLastError();
}

cudaError_t zconv_res_kmap_curl(const Geometry& g, float2* K2, void* map)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t rows = (cuuint64_t)g.nkx * zconv_res_nkb(g) * g.kzh * 2;
    const cuuint64_t dims[2] = {(cuuint64_t)KBW, rows};
    const cuuint64_t strides[1] = {(cuuint64_t)KBW * sizeof(float2)};
    const cuuint32_t box[2] = {(cuuint32_t)KBW, (cuuint32_t)(g.kzh * 2)};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, K2, dims, strides,
                           box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_zconv_res_curl(const void* ymap_p, const void* kmap_p, const Geometry& g, float2* Y, int* status,
                                  unsigned long long limit_ns, int nsm, cudaStream_t st)
{
    const CUtensorMap& ymap = *reinterpret_cast<const CUtensorMap*>(ymap_p);
    const CUtensorMap& kmap = *reinterpret_cast<const CUtensorMap*>(kmap_p);
    const int nkb = zconv_res_nkb(g);
    switch (g.pz / 2) {
    case 4: return launch_curl_hz<4>(ymap, kmap, g, nkb, Y, status, limit_ns, nsm, st);
    case 8: return launch_curl_hz<8>(ymap, kmap, g, nkb, Y, status, limit_ns, nsm, st);
    case 16: return launch_curl_hz<16>(ymap, kmap, g, nkb, Y, status, limit_ns, nsm, st);
    case 32: return launch_curl_hz<32>(ymap, kmap, g, nkb, Y, status, limit_ns, nsm, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_curl_point(const Geometry& g, float2* Y, const float* KO, cudaStream_t st)
{
    size_t b = ((size_t)g.nkx * g.py + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    curl_point_kernel<<<(int)(b ? b : 1), 256, 0, st>>>(g, Y, KO);
    return cudaGetLastError();
}

cudaError_t upload_twiddles_res() { return upload_small_twiddles_here(); }

}  // namespace boris
