// Split schedule of the y-z part of the convolution (Section 7): three
// cluster-free kernels that each keep many CTAs resident per SM.
//
//   y_fwd  : per (kx, group of G lines (c, z)): zero-padded length-py y
//            transform of each line (natural in, DIF, bit-reversed in shared
//            memory), written column-major to Y[kx][ky][c][z] so every
//            (kx, ky) column of 3 nz values is contiguous.
//   z_conv : the pipelined convolution of Section 7 (z transform, point-by-
//            point kernel multiply, inverse z transform in one launch for all
//            three components), one thread per (column, component, z-parity)
//            with the half-length z transform in registers; columns of one
//            kx plane are processed QC at a time.
//   y_inv  : inverse y transform of each line (DIT from bit-reversed order),
//            cropped to ny, written back to X[kx][c][z][y].
// Compared with the fused pass this moves the padded spectrum (2x the
// unpadded one) through HBM twice, but needs no cross-CTA exchange.
#include "boris_internal.cuh"

namespace boris {

constexpr int YG = 8;  // lines per CTA in the y kernels
template <typename T>
__global__ void __launch_bounds__(256) y_fwd_kernel(Geometry g, const typename Cx<T>::t* __restrict__ X,
                                                    typename Cx<T>::t* __restrict__ Y,
                                                    const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int py = g.py, ny = g.ny, nz = g.nz, lines = 3 * nz;
    const int LP = py + 2;  // padded line stride (bank spread for line-parallel passes)
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + py;  // [YG][LP]
    const int kx = blockIdx.y, l0 = blockIdx.x * YG;
    const int nl = min(YG, lines - l0);
    const int shy = g.lglmax - g.lgy;
    for (int i = threadIdx.x; i < py; i += blockDim.x) tw[i] = tw_g[i << shy];
    const C* src = X + ((size_t)kx * lines + l0) * ny;
    if (py == 1) {
        for (int l = threadIdx.x; l < nl; l += blockDim.x) buf[l * LP] = src[(size_t)l * ny];
    } else {
        // pruned first DIF stage: entries y >= ny (>= py/2) are zero
        const int half = py >> 1;
        __syncthreads();
        for (int i = threadIdx.x; i < nl * (half - ny); i += blockDim.x) {
            const int l = i / (half - ny), o = ny + i % (half - ny);
            buf[l * LP + o] = C{T(0), T(0)};
            buf[l * LP + o + half] = C{T(0), T(0)};
        }
        // the nl source lines are contiguous: nl * ny complex values
        staged_loop<256, C>(nl * ny, [&](int i) { return src[i]; }, [&](int i, C a) {
            const int l = i / ny, o = i % ny;
            buf[l * LP + o] = a;
            buf[l * LP + o + half] = c_mul(a, tw[o]);
        });
    }
    __syncthreads();
    if (py > 1) {
        Lines ln{nl, nl, LP, 0, 1, true};
        fft_dif(buf, ln, g.lgy, 1, tw, 0);
    }
    // Y[kx][ky][line]: consecutive threads take consecutive lines of one ky
    C* dst = Y + (size_t)kx * py * lines + l0;
    for (int i = threadIdx.x; i < py * nl; i += blockDim.x) {
        const int l = i % nl, ky = i / nl;
        dst[(size_t)ky * lines + l] = buf[l * LP + bitrev(ky, g.lgy)];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) y_inv_kernel(Geometry g, const typename Cx<T>::t* __restrict__ Y,
                                                    typename Cx<T>::t* __restrict__ X,
                                                    const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int py = g.py, ny = g.ny, nz = g.nz, lines = 3 * nz;
    const int LP = py + 2;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + py;
    const int kx = blockIdx.y, l0 = blockIdx.x * YG;
    const int nl = min(YG, lines - l0);
    const int shy = g.lglmax - g.lgy;
    for (int i = threadIdx.x; i < py; i += blockDim.x) tw[i] = tw_g[i << shy];
    const C* src = Y + (size_t)kx * py * lines + l0;
    staged_loop<256, C>(py * nl, [&](int i) { return src[(size_t)(i / nl) * lines + i % nl]; }, [&](int i, C a) {
        buf[(i % nl) * LP + bitrev(i / nl, g.lgy)] = a;
    });
    __syncthreads();
    if (py > 1) {
        Lines ln{nl, nl, LP, 0, 1, true};
        fft_dit(buf, ln, g.lgy, 0, tw, 0);
    }
    C* dst = X + ((size_t)kx * lines + l0) * ny;
    for (int i = threadIdx.x; i < nl * ny; i += blockDim.x) {
        const int l = i / ny, y = i % ny;
        dst[(size_t)l * ny + y] = buf[l * LP + y];
    }
}

// ---------------------------------------------------------------------------
// z_conv: QC columns (kx, ky..ky+QC) per CTA; thread (col, c, h) with c and h
// uniform across each warp (QC = 32), so the component row of the kernel and
// the z parity are compile-time inside the per-warp body.
// ---------------------------------------------------------------------------
constexpr int QC = 32;

// Phases of the per-warp work; (CP, HP) = (component, z parity) of the warp.
// The kernel runs each phase through a warp-uniform switch and places the
// block barriers between phases, outside the per-warp code.
template <typename T, int HZ, int CP, int HP>
__device__ __forceinline__ void zc_forward(const Geometry& g, int col, typename Cx<T>::t* tile, int CS,
                                           typename Cx<T>::t (&v)[HZ])
{
    using C = typename Cx<T>::t;
    const C* mine = tile + col * CS + CP * HZ;
#pragma unroll
    for (int z = 0; z < HZ; z++) {
        C x = z < g.nz ? mine[z] : C{T(0), T(0)};
        if (HP) x = c_mul(x, cw128<C>(z * (64 / HZ)));
        v[z] = x;
    }
    reg_fft<HZ, -1>(v);
}

template <typename T, int HZ, int CP, int HP>
__device__ __forceinline__ void zc_store_spec(int col, typename Cx<T>::t* tile, typename Cx<T>::t* odd, int CS,
                                              typename Cx<T>::t (&v)[HZ])
{
    typename Cx<T>::t* spec = HP ? odd : tile;  // spectrum of this parity: [col][c][pos]
#pragma unroll
    for (int pos = 0; pos < HZ; pos++) spec[col * CS + CP * HZ + pos] = v[pos];
}

template <typename T, int HZ, int CP, int HP>
__device__ __forceinline__ void zc_multiply_inverse(const Geometry& g, int col, int ky0, const typename Cx<T>::t* tile,
                                                    const typename Cx<T>::t* odd, const T* Ks, int CS, int KS,
                                                    typename Cx<T>::t (&v)[HZ])
{
    using C = typename Cx<T>::t;
    const C* spec = HP ? odd : tile;
    const int pz = 2 * HZ;
    const int ky = ky0 + col;
    const bool fy = ky > g.py / 2;
    const T sy = fy ? T(-1) : T(1);
    const T* kr = Ks + col * KS;
    constexpr int i0 = CP == 0 ? 0 : CP == 1 ? 3 : 4;  // row c: (xx xy xz) (xy yy yz) (xz yz zz)
    constexpr int i1 = CP == 0 ? 3 : CP == 1 ? 1 : 5;
    constexpr int i2 = CP == 0 ? 4 : CP == 1 ? 5 : 2;
    constexpr int LGH = HZ == 2 ? 1 : HZ == 4 ? 2 : HZ == 8 ? 3 : HZ == 16 ? 4 : 5;
#pragma unroll
    for (int pos = 0; pos < HZ; pos++) {
        const int kz = 2 * (int)((__brev((unsigned)pos) >> (32 - LGH))) + HP;
        const bool fz = kz > pz / 2;
        const int kzf = fz ? pz - kz : kz;
        const T sz = fz ? T(-1) : T(1);
        // component signs: xy odd in ky; xz odd in kz; yz odd in both
        auto sgn = [&](int idx) -> T { return idx == 3 ? sy : idx == 4 ? sz : idx == 5 ? sy * sz : T(1); };
        const T k0 = kr[kzf * 6 + i0] * sgn(i0);
        const T k1 = kr[kzf * 6 + i1] * sgn(i1);
        const T k2 = kr[kzf * 6 + i2] * sgn(i2);
        const C* s = spec + col * CS + pos;
        const C m0 = CP == 0 ? v[pos] : s[0];
        const C m1 = CP == 1 ? v[pos] : s[HZ];
        const C m2 = CP == 2 ? v[pos] : s[2 * HZ];
        v[pos] = C{k0 * m0.x + k1 * m1.x + k2 * m2.x, k0 * m0.y + k1 * m1.y + k2 * m2.y};
    }
    reg_fft<HZ, 1>(v);
}

template <typename T, int HZ, int CP, int HP>
__device__ __forceinline__ void zc_odd_store(int col, typename Cx<T>::t* odd, int CS, typename Cx<T>::t (&v)[HZ])
{
    if (HP) {
#pragma unroll
        for (int z = 0; z < HZ; z++) odd[col * CS + CP * HZ + z] = c_mulc(v[z], cw128<typename Cx<T>::t>(z * (64 / HZ)));
    }
}

template <typename T, int HZ, int CP, int HP>
__device__ __forceinline__ void zc_combine(int col, typename Cx<T>::t* tile, const typename Cx<T>::t* odd, int CS,
                                           typename Cx<T>::t (&v)[HZ])
{
    if (!HP) {
#pragma unroll
        for (int z = 0; z < HZ; z++) tile[col * CS + CP * HZ + z] = c_add(v[z], odd[col * CS + CP * HZ + z]);
    }
}

#define ZC_DISPATCH(CALL)                    \
    switch (warp) {                          \
    case 0: CALL(0, 0); break;               \
    case 1: CALL(1, 0); break;               \
    case 2: CALL(2, 0); break;               \
    case 3: CALL(0, 1); break;               \
    case 4: CALL(1, 1); break;               \
    default: CALL(2, 1); break;              \
    }

template <typename T, int HZ>
__global__ void __launch_bounds__(QC * 6) z_conv_kernel(Geometry g, typename Cx<T>::t* __restrict__ Y,
                                                        const T* __restrict__ K)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nz = g.nz, lines = 3 * nz, py = g.py;
    const int kx = blockIdx.y, ky0 = blockIdx.x * QC;
    const int ncol = min(QC, py - ky0);
    const int CS = 3 * HZ + 1;  // column stride (odd: bank spread)
    const int KS = g.krow + 1;
    C* tile = reinterpret_cast<C*>(smem_raw);     // [QC][CS]
    C* odd = tile + QC * CS;                      // [QC][CS]
    T* Ks = reinterpret_cast<T*>(odd + QC * CS);  // [QC][KS]
    C* col0 = Y + ((size_t)kx * py + ky0) * lines;
    // stage the columns (contiguous in Y) and their kernel rows; the columns
    // of a ragged last tile are zero and never written back
    auto tpos = [&](int i) {
        const int col = i / lines, r = i % lines;
        return col * CS + (r / nz) * HZ + r % nz;
    };
    staged_loop<QC * 6, C>(ncol * lines, [&](int i) { return col0[i]; }, [&](int i, C a) { tile[tpos(i)] = a; });
    for (int i = ncol * lines + threadIdx.x; i < QC * lines; i += blockDim.x) tile[tpos(i)] = C{T(0), T(0)};
    // kernel rows: krow floats (a multiple of 4: 16-byte vectors)
    const T* Kx = K + (size_t)kx * g.kyh * g.krow;
    const int vrow = g.krow * (int)sizeof(T) / 16;  // 16-byte vectors per row
    staged_loop<QC * 6, float4>(ncol * vrow, [&](int i) {
        const int col = i / vrow, o = i % vrow;
        const int ky = ky0 + col;
        const int kyf = ky > py / 2 ? py - ky : ky;
        return reinterpret_cast<const float4*>(Kx + (size_t)kyf * g.krow)[o];
    }, [&](int i, float4 v4) {
        const int col = i / vrow, o = i % vrow;
        const T* e = reinterpret_cast<const T*>(&v4);
        constexpr int PER = 16 / sizeof(T);
#pragma unroll
        for (int k = 0; k < PER; k++) Ks[col * KS + o * PER + k] = e[k];
    });
    for (int i = ncol * g.krow + threadIdx.x; i < QC * g.krow; i += blockDim.x)
        Ks[(i / g.krow) * KS + i % g.krow] = T(0);
    __syncthreads();
    const int warp = threadIdx.x >> 5, col = threadIdx.x & 31;
    C v[HZ];
#define ZC1(CP, HP) zc_forward<T, HZ, CP, HP>(g, col, tile, CS, v)
    ZC_DISPATCH(ZC1)
    __syncthreads();
#define ZC2(CP, HP) zc_store_spec<T, HZ, CP, HP>(col, tile, odd, CS, v)
    ZC_DISPATCH(ZC2)
    __syncthreads();
#define ZC3(CP, HP) zc_multiply_inverse<T, HZ, CP, HP>(g, col, ky0, tile, odd, Ks, CS, KS, v)
    ZC_DISPATCH(ZC3)
    __syncthreads();
#define ZC4(CP, HP) zc_odd_store<T, HZ, CP, HP>(col, odd, CS, v)
    ZC_DISPATCH(ZC4)
    __syncthreads();
#define ZC5(CP, HP) zc_combine<T, HZ, CP, HP>(col, tile, odd, CS, v)
    ZC_DISPATCH(ZC5)
    __syncthreads();
#undef ZC1
#undef ZC2
#undef ZC3
#undef ZC4
#undef ZC5
    for (int i = threadIdx.x; i < ncol * lines; i += blockDim.x) {
        const int col = i / lines, r = i % lines;
        const int c = r / nz, z = r % nz;
        col0[i] = tile[col * CS + c * HZ + z];
    }
}

// 2D mode (pz = 1): the multiply alone, one thread per column.
template <typename T>
__global__ void __launch_bounds__(256) z_mult_kernel(Geometry g, typename Cx<T>::t* __restrict__ Y,
                                                     const T* __restrict__ K)
{
    using C = typename Cx<T>::t;
    const int py = g.py;
    const size_t ncol = (size_t)g.nkx * py;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ncol; i += (size_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i / py), ky = (int)(i % py);
        const bool fy = ky > py / 2;
        const T* k = K + ((size_t)kx * g.kyh + (fy ? py - ky : ky)) * g.krow;
        const T kxx = k[0], kyy = k[1], kzz = k[2];
        const T kxy = fy ? -k[3] : k[3], kxz = k[4], kyz = fy ? -k[5] : k[5];
        C* col = Y + i * 3;
        const C a = col[0], b = col[1], c = col[2];
        col[0] = C{kxx * a.x + kxy * b.x + kxz * c.x, kxx * a.y + kxy * b.y + kxz * c.y};
        col[1] = C{kxy * a.x + kyy * b.x + kyz * c.x, kxy * a.y + kyy * b.y + kyz * c.y};
        col[2] = C{kxz * a.x + kyz * b.x + kzz * c.x, kxz * a.y + kyz * b.y + kzz * c.y};
    }
}

template <typename T>
size_t split_y_smem(const Geometry& g)
{
    return ((size_t)g.py + (size_t)YG * (g.py + 2)) * sizeof(typename Cx<T>::t);
}

template <typename T>
size_t split_z_smem(const Geometry& g)
{
    const int hz = g.pz / 2;
    return (2 * (size_t)QC * (3 * hz + 1)) * sizeof(typename Cx<T>::t) + (size_t)QC * (g.krow + 1) * sizeof(T);
}

template <typename T>
bool split_supported(const Geometry& g, int max_smem)
{
    const int hz = g.pz / 2;
    if (!(g.pz == 1 || (hz >= 2 && hz <= 32))) return false;
    if (split_y_smem<T>(g) > (size_t)max_smem) return false;
    if (g.pz > 1 && split_z_smem<T>(g) > (size_t)max_smem) return false;
    return true;
}

template <typename T, int HZ>
static cudaError_t launch_zconv_hz(const Geometry& g, typename Cx<T>::t* Y, const T* K, cudaStream_t st)
{
    const size_t smem = split_z_smem<T>(g);
    cudaError_t e = cudaFuncSetAttribute(z_conv_kernel<T, HZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.py + QC - 1) / QC, g.nkx);
    z_conv_kernel<T, HZ><<<grid, QC * 6, smem, st>>>(g, Y, K);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_split(const Geometry& g, typename Cx<T>::t* X, typename Cx<T>::t* Y, const T* K,
                         const typename Cx<T>::t* tw, cudaStream_t st, int part)
{
    const size_t ys = split_y_smem<T>(g);
    const int lines = 3 * g.nz;
    dim3 ygrid((lines + YG - 1) / YG, g.nkx);
    cudaError_t e = cudaSuccess;
    if (part == 0) {
        e = cudaFuncSetAttribute(y_fwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ys);
        if (e != cudaSuccess) return e;
        y_fwd_kernel<T><<<ygrid, 256, ys, st>>>(g, X, Y, tw);
        return cudaGetLastError();
    }
    if (part == 1) {
        if (g.pz == 1) {
            size_t n = (size_t)g.nkx * g.py;
            int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
            z_mult_kernel<T><<<blocks, 256, 0, st>>>(g, Y, K);
            return cudaGetLastError();
        }
        switch (g.pz / 2) {
        case 2: return launch_zconv_hz<T, 2>(g, Y, K, st);
        case 4: return launch_zconv_hz<T, 4>(g, Y, K, st);
        case 8: return launch_zconv_hz<T, 8>(g, Y, K, st);
        case 16: return launch_zconv_hz<T, 16>(g, Y, K, st);
        case 32: return launch_zconv_hz<T, 32>(g, Y, K, st);
        default: return cudaErrorInvalidValue;
        }
    }
    e = cudaFuncSetAttribute(y_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ys);
    if (e != cudaSuccess) return e;
    y_inv_kernel<T><<<ygrid, 256, ys, st>>>(g, Y, X, tw);
    return cudaGetLastError();
}

cudaError_t upload_twiddles_split() { return upload_small_twiddles_here(); }

template bool split_supported<float>(const Geometry&, int);
template bool split_supported<double>(const Geometry&, int);
template cudaError_t launch_split<float>(const Geometry&, float2*, float2*, const float*, const float2*, cudaStream_t,
                                         int);
template cudaError_t launch_split<double>(const Geometry&, double2*, double2*, const double*, const double2*,
                                          cudaStream_t, int);

}  // namespace boris
