// Split schedule of the y-z part of the convolution (Section 7): three
// cluster-free kernels that each keep many CTAs resident per SM.
//
//   y_fwd  : per (kx, group of G lines (c, z)): zero-padded length-py y
//            transform of each line (natural in, DIF, bit-reversed in shared
//            memory), written to Y[kx][c][z][ky] (ky fastest).
//   z_conv : the pipelined convolution of Section 7 (z transform, point-by-
//            point kernel multiply, inverse z transform in one launch for all
//            three components), one thread per (column, component, z-parity)
//            with the half-length z transform in registers; QC consecutive
//            ky columns of one kx plane per CTA (32 consecutive ky per line
//            load and store).
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
    // Y[kx][line][ky]
    C* dst = Y + ((size_t)kx * lines + l0) * py;
    for (int i = threadIdx.x; i < py * nl; i += blockDim.x) {
        const int l = i / py, ky = i % py;
        dst[(size_t)l * py + ky] = buf[l * LP + bitrev(ky, g.lgy)];
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
    const C* src = Y + ((size_t)kx * lines + l0) * py;
    staged_loop<256, C>(py * nl, [&](int i) { return src[i]; }, [&](int i, C a) {
        buf[(i / py) * LP + bitrev(i % py, g.lgy)] = a;
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

// Per-thread work of z_conv.  The component c is a runtime value (its kernel
// row, the rows of the other two components and the sign pattern are
// precomputed per thread); only the z parity HP is a template parameter, so
// the kernel has two code paths.  The phases are separated by block
// barriers placed in the kernel itself.
template <typename T>
struct ZcThread {
    int col, c, o1, o2;  // column, component, row offsets of the other two components
    const T* k0;         // kernel row entries of (c, c), (c, other1), (c, other2)
    const T* k1;
    const T* k2;
    T a0, a1, a2;        // sign of each entry under ky -> -ky (xy, yz odd in ky)
    T b0, b1, b2;        // sign of each entry under kz -> -kz (xz, yz odd in kz)
};

template <typename T, int HZ, int HP>
__device__ __forceinline__ void zc_forward(const Geometry& g, const ZcThread<T>& t, typename Cx<T>::t* tile, int CS,
                                           typename Cx<T>::t (&v)[HZ])
{
    using C = typename Cx<T>::t;
    const C* mine = tile + t.col * CS + t.c * HZ;
#pragma unroll
    for (int z = 0; z < HZ; z++) {
        C x = z < g.nz ? mine[z] : C{T(0), T(0)};
        if (HP) x = c_mul(x, w128lit<C>(z * (64 / HZ)));
        v[z] = x;
    }
    reg_fft<HZ, -1>(v);
}

template <typename T, int HZ, int HP>
__device__ __forceinline__ void zc_multiply_inverse(const ZcThread<T>& t, const typename Cx<T>::t* spec, int CS,
                                                    typename Cx<T>::t (&v)[HZ])
{
    using C = typename Cx<T>::t;
    constexpr int PZ = 2 * HZ;
    constexpr int LGH = HZ == 2 ? 1 : HZ == 4 ? 2 : HZ == 8 ? 3 : HZ == 16 ? 4 : 5;
    const C* s = spec + t.col * CS;
#pragma unroll
    for (int pos = 0; pos < HZ; pos++) {
        const int kz = 2 * (int)((__brev((unsigned)pos) >> (32 - LGH))) + HP;  // compile-time
        const bool fz = kz > PZ / 2;
        const int kzf = fz ? PZ - kz : kz;
        const T w0 = t.k0[kzf * 6] * t.a0 * (fz ? t.b0 : T(1));
        const T w1 = t.k1[kzf * 6] * t.a1 * (fz ? t.b1 : T(1));
        const T w2 = t.k2[kzf * 6] * t.a2 * (fz ? t.b2 : T(1));
        const C m1 = s[t.o1 + pos], m2 = s[t.o2 + pos];
        const C own = v[pos];
        v[pos] = C{w0 * own.x + w1 * m1.x + w2 * m2.x, w0 * own.y + w1 * m1.y + w2 * m2.y};
    }
    reg_fft<HZ, 1>(v);
}

template <typename T, int HZ, int MINB>
__global__ void __launch_bounds__(QC * 6, MINB) z_conv_kernel(Geometry g, typename Cx<T>::t* __restrict__ Y,
                                                              const T* __restrict__ K)
{
    constexpr int KROW = ((HZ + 1) * 6 + 3) / 4 * 4;  // kernel row length (g.krow for pz = 2 HZ)
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nz = g.nz, lines = 3 * nz, py = g.py;
    const int kx = blockIdx.y, ky0 = blockIdx.x * QC;
    const int ncol = min(QC, py - ky0);
    const int CS = 3 * HZ + 1;  // column stride (odd: bank spread)
    constexpr int KS = KROW + 1;
    C* tile = reinterpret_cast<C*>(smem_raw);     // [QC][CS]
    C* odd = tile + QC * CS;                      // [QC][CS]
    T* Ks = reinterpret_cast<T*>(odd + QC * CS);  // [QC][KS]
    // stage the QC columns: Y[kx][line][ky0 + col] (32 consecutive ky per line)
    const C* ysrc = Y + (size_t)kx * lines * py + ky0;
    // line = c * nz + z sits at row c * HZ + z of a column
    const bool full = nz == HZ;  // then the row is the line index itself
    auto row_of = [&](int line) { return full ? line : (line / nz) * HZ + line % nz; };
    staged_loop<QC * 6, C>(lines * QC, [&](int i) {
        const int line = i / QC, col = i % QC;
        return col < ncol ? ysrc[(size_t)line * py + col] : C{T(0), T(0)};
    }, [&](int i, C a) {
        const int line = i / QC, col = i % QC;
        tile[col * CS + row_of(line)] = a;
    });
    // kernel rows: KROW values (a multiple of 4: 16-byte vectors)
    const T* Kx = K + (size_t)kx * g.kyh * KROW;
    constexpr int vrow = KROW * (int)sizeof(T) / 16;
    staged_loop<QC * 6, float4>(ncol * vrow, [&](int i) {
        const int col = i / vrow, o = i % vrow;
        const int ky = ky0 + col;
        const int kyf = ky > py / 2 ? py - ky : ky;
        return reinterpret_cast<const float4*>(Kx + (size_t)kyf * KROW)[o];
    }, [&](int i, float4 v4) {
        const int col = i / vrow, o = i % vrow;
        const T* e = reinterpret_cast<const T*>(&v4);
        constexpr int PER = 16 / sizeof(T);
#pragma unroll
        for (int k = 0; k < PER; k++) Ks[col * KS + o * PER + k] = e[k];
    });
    for (int i = ncol * KROW + threadIdx.x; i < QC * KROW; i += blockDim.x) Ks[(i / KROW) * KS + i % KROW] = T(0);
    __syncthreads();
    // thread = (col, c, h): warp w takes component w % 3 and z parity w / 3
    const int warp = threadIdx.x >> 5;
    ZcThread<T> t;
    t.col = threadIdx.x & 31;
    t.c = warp % 3;
    const int h = warp / 3;
    const int c1 = t.c == 0 ? 1 : 0, c2 = t.c == 2 ? 1 : 2;
    t.o1 = c1 * HZ;
    t.o2 = c2 * HZ;
    // entry (i, j) of the symmetric kernel in the (xx yy zz xy xz yz) order
    auto comp = [](int i, int j) { return i == j ? i : (i + j == 1 ? 3 : (i + j == 2 ? 4 : 5)); };
    const int e0 = comp(t.c, t.c), e1 = comp(t.c, c1), e2 = comp(t.c, c2);
    const T* kr = Ks + t.col * KS;
    t.k0 = kr + e0;
    t.k1 = kr + e1;
    t.k2 = kr + e2;
    const bool fy = ky0 + t.col > py / 2;
    auto sgn_y = [&](int e) { return (fy && (e == 3 || e == 5)) ? T(-1) : T(1); };
    auto sgn_z = [](int e) { return (e == 4 || e == 5) ? T(-1) : T(1); };
    t.a0 = sgn_y(e0); t.a1 = sgn_y(e1); t.a2 = sgn_y(e2);
    t.b0 = sgn_z(e0); t.b1 = sgn_z(e1); t.b2 = sgn_z(e2);
    C v[HZ];
    if (h) zc_forward<T, HZ, 1>(g, t, tile, CS, v);
    else zc_forward<T, HZ, 0>(g, t, tile, CS, v);
    __syncthreads();
    C* spec = h ? odd : tile;  // spectrum of this parity: [col][c][pos]
#pragma unroll
    for (int pos = 0; pos < HZ; pos++) spec[t.col * CS + t.c * HZ + pos] = v[pos];
    __syncthreads();
    if (h) zc_multiply_inverse<T, HZ, 1>(t, spec, CS, v);
    else zc_multiply_inverse<T, HZ, 0>(t, spec, CS, v);
    __syncthreads();
    if (h) {
#pragma unroll
        for (int z = 0; z < HZ; z++) odd[t.col * CS + t.c * HZ + z] = c_mulc(v[z], w128lit<C>(z * (64 / HZ)));
    }
    __syncthreads();
    if (!h) {
#pragma unroll
        for (int z = 0; z < HZ; z++) tile[t.col * CS + t.c * HZ + z] = c_add(v[z], odd[t.col * CS + t.c * HZ + z]);
    }
    __syncthreads();
    C* ydst = Y + (size_t)kx * lines * py + ky0;
    for (int i = threadIdx.x; i < lines * QC; i += blockDim.x) {
        const int line = i / QC, col = i % QC;
        if (col < ncol) ydst[(size_t)line * py + col] = tile[col * CS + row_of(line)];
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
        // Y[kx][c][ky] (nz = 1)
        C* col = Y + (size_t)kx * 3 * py + ky;
        const C a = col[0], b = col[py], c = col[2 * py];
        col[0] = C{kxx * a.x + kxy * b.x + kxz * c.x, kxx * a.y + kxy * b.y + kxz * c.y};
        col[py] = C{kxy * a.x + kyy * b.x + kyz * c.x, kxy * a.y + kyy * b.y + kyz * c.y};
        col[2 * py] = C{kxz * a.x + kyz * b.x + kzz * c.x, kxz * a.y + kyz * b.y + kzz * c.y};
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
    // the y passes: warp-held transforms of length 1024 / 2048 / 4096, else shared-memory passes
    const bool ywarp = y512_ok<T>(g, max_smem) || y1024_ok<T>(g, max_smem) || y2048_ok<T>(g, max_smem) ||
                       y4096_ok<T>(g, max_smem);
    if (!ywarp && split_y_smem<T>(g) > (size_t)max_smem) return false;
    if (g.pz > 1 && split_z_smem<T>(g) > (size_t)max_smem) return false;
    return true;
}

template <typename T, int HZ, int MINB>
static cudaError_t launch_zconv_hz(const Geometry& g, typename Cx<T>::t* Y, const T* K, cudaStream_t st)
{
    const size_t smem = split_z_smem<T>(g);
    cudaError_t e =
        cudaFuncSetAttribute(z_conv_kernel<T, HZ, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.py + QC - 1) / QC, g.nkx);
    z_conv_kernel<T, HZ, MINB><<<grid, QC * 6, smem, st>>>(g, Y, K);
    return cudaGetLastError();
}

template <typename T, int HZ>
static cudaError_t launch_zconv_occ(const Geometry& g, typename Cx<T>::t* Y, const T* K, cudaStream_t st, int occ)
{
    // occ: CTAs per SM the register budget is fitted to (FP64 always 1)
    if (sizeof(T) == 8) return launch_zconv_hz<T, HZ, 1>(g, Y, K, st);
    if (occ == 3) return launch_zconv_hz<T, HZ, 3>(g, Y, K, st);
    return launch_zconv_hz<T, HZ, 2>(g, Y, K, st);
}

template <typename T>
cudaError_t launch_split(const Geometry& g, typename Cx<T>::t* X, typename Cx<T>::t* Y, const T* K,
                         const typename Cx<T>::t* tw, cudaStream_t st, int part, int occ)
{
    const size_t ys = split_y_smem<T>(g);
    const int lines = 3 * g.nz;
    dim3 ygrid((lines + YG - 1) / YG, g.nkx);
    cudaError_t e = cudaSuccess;
    if (part != 1 && y1024_ok<T>(g, 227 * 1024)) return launch_y_1024<T>(g, X, Y, tw, st, part == 0);
    if (part != 1 && y512_ok<T>(g, 227 * 1024)) return launch_y_512<T>(g, X, Y, tw, st, part == 0);
    if (part != 1 && y2048_ok<T>(g, 227 * 1024)) return launch_y_2048<T>(g, X, Y, tw, st, part == 0);
    if (part != 1 && y4096_ok<T>(g, 227 * 1024)) return launch_y_4096<T>(g, X, Y, tw, st, part == 0);
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
        case 2: return launch_zconv_occ<T, 2>(g, Y, K, st, occ);
        case 4: return launch_zconv_occ<T, 4>(g, Y, K, st, occ);
        case 8: return launch_zconv_occ<T, 8>(g, Y, K, st, occ);
        case 16: return launch_zconv_occ<T, 16>(g, Y, K, st, occ);
        case 32: return launch_zconv_occ<T, 32>(g, Y, K, st, occ);
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
                                         int, int);
template cudaError_t launch_split<double>(const Geometry&, double2*, double2*, const double*, const double2*,
                                          cudaStream_t, int, int);

}  // namespace boris
