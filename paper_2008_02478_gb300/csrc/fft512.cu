// Transforms of length N = 1024 / P (P = 2: N = 512, meshes of 129..256 cells
// along the axis; P = 4: N = 256, 65..128 cells): P lines per warp through
// the warp-held length-1024 transform of warp_fft.cuh.
//
// With u[P n + p] = l_p[n] (p < P, n < N) and U = FFT_1024(u),
//   U[k + N j] = sum_p w_P^(p j) w^(p k) L_p[k]     (w = exp(-2 pi i / 1024)),
// so for each k < N the P values U[k + N j] - all in one lane, at register
// positions brev5(c + (32 / P) j) for k = lane + 32 c - give the lines'
// transforms by a length-P inverse DFT:
//   L_p[k] = w^(-p k) (1 / P) sum_j U[k + N j] w_P^(-p j).
// The inverse runs the same steps backwards (forward length-P DFT of
// w^(p k) L_p[k], IFFT_1024, scale 1 / P); transforms are unscaled.
//
// x passes: a complex line packs two real rows (real and imaginary parts), so
// a warp carries 2 P rows and a CTA of eight warps 16 P rows; the real
// spectra are untangled as A_k = (Z_k + conj Z_{N-k}) / 2 and
// B_k = (Z_k - conj Z_{N-k}) / (2i), k = 0..N/2, and packed back as
// Z_k = A_k + i B_k (A, B Hermitian) for the inverse.
// y passes: P complex lines per warp, 8 P lines per CTA.
#include "boris_internal.cuh"
#include "warp_fft.cuh"

namespace boris {

namespace {

constexpr int R1025 = 1025;  // per-warp region stride (complex)

template <int P>
struct Short {
    static constexpr int N = 1024 / P;  // line length
    static constexpr int CN = 32 / P;   // k = lane + 32 c, c < CN
    static constexpr int LGP = P == 2 ? 1 : 2;
    static constexpr int ROWS = 16 * P;  // x passes: real rows per CTA
};

// w_P^m (compile-time m) as a literal
template <int P, typename C>
__device__ __forceinline__ C wP(int m)
{
    return w128lit<C>(((128 / P) * m) & 127);
}

// v (forward output, v[pos] = U[lane + 32 brev5(pos)]) -> L[p][c] = L_p[lane + 32 c]
template <int P, typename C, typename T>
__device__ __forceinline__ void untangle(const C (&v)[32], C (&L)[P][32 / P], const C* tws)
{
    constexpr int CN = 32 / P;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < CN; c++) {
        C U[P];
#pragma unroll
        for (int j = 0; j < P; j++) U[j] = v[brev5(c + CN * j)];
#pragma unroll
        for (int p = 0; p < P; p++) {
            C s = U[0];
#pragma unroll
            for (int j = 1; j < P; j++) s = c_add(s, (p * j) % P == 0 ? U[j] : c_mulc(U[j], wP<P, C>((p * j) % P)));
            if (p > 0) s = c_mulc(s, c_mul(w128lit<C>((4 * p * c) & 127), tws[32 * p + lane]));  // w^(p k)
            L[p][c] = C{s.x * (T(1) / P), s.y * (T(1) / P)};
        }
    }
}

// L[p][c] = L_p[lane + 32 c] -> v in the inverse transform's input order
template <int P, typename C>
__device__ __forceinline__ void tangle(const C (&L)[P][32 / P], C (&v)[32], const C* tws)
{
    constexpr int CN = 32 / P;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < CN; c++) {
        C t[P];
#pragma unroll
        for (int p = 0; p < P; p++)
            t[p] = p == 0 ? L[0][c] : c_mul(L[p][c], c_mul(w128lit<C>((4 * p * c) & 127), tws[32 * p + lane]));
#pragma unroll
        for (int j = 0; j < P; j++) {
            C s = t[0];
#pragma unroll
            for (int p = 1; p < P; p++) s = c_add(s, (p * j) % P == 0 ? t[p] : c_mul(t[p], wP<P, C>((p * j) % P)));
            v[brev5(c + CN * j)] = s;
        }
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    y_fwd_short_kernel(Geometry g, const typename Cx<T>::t* __restrict__ X, typename Cx<T>::t* __restrict__ Y,
                       const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    using S = Short<P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* reg = tws + TW1024_SLOTS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lines = 3 * g.nz, ny = g.ny;
    const int kx = blockIdx.y, l0 = blockIdx.x * 8 * P + P * warp;
    load_tw1024(tws, tw_g, g.lmax);
    __syncthreads();
    if (l0 >= lines) return;
    const int p = lane & (P - 1);
    const bool okl = l0 + p < lines;
    const C* src = X + ((size_t)kx * lines + l0 + p) * ny;
    C v[32];
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int n = S::CN * a + (lane >> S::LGP);  // u[32 a + lane] = l_p[n]
        v[a] = okl && n < ny ? src[n] : C{T(0), T(0)};
    }
#pragma unroll
    for (int a = 16; a < 32; a++) v[a] = C{T(0), T(0)};
    warp_fft1024_fwd(v, reg + warp * R1025, tws);
    C L[P][S::CN];
    untangle<P, C, T>(v, L, tws);
    C* d0 = Y + ((size_t)kx * lines + l0) * S::N;
#pragma unroll
    for (int q = 0; q < P; q++) {
        if (l0 + q >= lines) break;
#pragma unroll
        for (int c = 0; c < S::CN; c++) d0[q * S::N + lane + 32 * c] = L[q][c];
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    y_inv_short_kernel(Geometry g, const typename Cx<T>::t* __restrict__ Y, typename Cx<T>::t* __restrict__ X,
                       const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    using S = Short<P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* reg = tws + TW1024_SLOTS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lines = 3 * g.nz, ny = g.ny;
    const int kx = blockIdx.y, l0 = blockIdx.x * 8 * P + P * warp;
    load_tw1024(tws, tw_g, g.lmax);
    __syncthreads();
    if (l0 >= lines) return;
    const C* s0 = Y + ((size_t)kx * lines + l0) * S::N;
    C L[P][S::CN];
#pragma unroll
    for (int q = 0; q < P; q++) {
        const bool ok = l0 + q < lines;
#pragma unroll
        for (int c = 0; c < S::CN; c++) L[q][c] = ok ? s0[q * S::N + lane + 32 * c] : C{T(0), T(0)};
    }
    C v[32];
    tangle<P, C>(L, v, tws);
    warp_fft1024_inv(v, reg + warp * R1025, tws);
    // v[a] = P l_p[n], p = lane mod P, n = (32 / P) a + lane / P
    const int p = lane & (P - 1);
    if (l0 + p >= lines) return;
    C* dst = X + ((size_t)kx * lines + l0 + p) * ny;
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int n = S::CN * a + (lane >> S::LGP);
        if (n < ny) dst[n] = C{v[a].x * (T(1) / P), v[a].y * (T(1) / P)};
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    x_r2c_short_kernel(Geometry g, const T* __restrict__ M, const T* __restrict__ ms_map, T ms_scale,
                       typename Cx<T>::t* __restrict__ X, const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    using S = Short<P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    C* reg = tws + TW1024_SLOTS;  // warp w: line p at [N p, N p + N)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0 = blockIdx.x * S::ROWS, z = blockIdx.y, c = blockIdx.z;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    load_tw1024(tws, tw_g, g.lmax);
    __syncthreads();
    // line p of warp w packs rows y0 + w + 16 p (real part) and y0 + w + 16 p + 8 (imaginary part)
    const int p = lane & (P - 1);
    const int ya = y0 + warp + 16 * p, yb = ya + 8;
    const size_t ncell = (size_t)nx * ny * nz;
    const T* ra = M + c * ncell + ((size_t)z * ny + ya) * nx;
    const T* rb = M + c * ncell + ((size_t)z * ny + yb) * nx;
    const T* ma = ms_map ? ms_map + ((size_t)z * ny + ya) * nx : nullptr;
    const T* mb = ms_map ? ms_map + ((size_t)z * ny + yb) * nx : nullptr;
    const bool oka = ya < ny, okb = yb < ny;
    C v[32];
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int n = S::CN * a + (lane >> S::LGP);
        const bool in = n < nx;
        T xa = (in && oka) ? ra[n] : T(0), xb = (in && okb) ? rb[n] : T(0);
        if (ms_map) {
            xa *= (in && oka) ? ma[n] : T(0);
            xb *= (in && okb) ? mb[n] : T(0);
        } else {
            xa *= ms_scale;
            xb *= ms_scale;
        }
        v[a] = C{xa, xb};
    }
#pragma unroll
    for (int a = 16; a < 32; a++) v[a] = C{T(0), T(0)};
    C* mine = reg + warp * R1025;
    warp_fft1024_fwd(v, mine, tws);
    {
        C L[P][S::CN];
        untangle<P, C, T>(v, L, tws);
#pragma unroll
        for (int q = 0; q < P; q++)
#pragma unroll
            for (int cc = 0; cc < S::CN; cc++) mine[S::N * q + lane + 32 * cc] = L[q][cc];
    }
    __syncthreads();
    // X[kx][c][z][y0 + t], kx = 0..N/2: 16 P consecutive y per kx
    for (int i = threadIdx.x; i < (S::N / 2 + 1) * S::ROWS; i += blockDim.x) {
        const int t = i & (S::ROWS - 1), k = i / S::ROWS;
        const int yy = y0 + t;
        if (yy >= ny) continue;
        const C* line = reg + (t & 7) * R1025 + S::N * (t >> 4);
        const C zk = line[k & (S::N - 1)], zm = line[(S::N - k) & (S::N - 1)];
        C out;
        if ((t & 8) == 0) out = C{T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y)};
        else out = C{T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x)};
        X[(((size_t)k * 3 + c) * nz + z) * ny + yy] = out;
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    x_c2r_short_kernel(Geometry g, const typename Cx<T>::t* __restrict__ X, T* __restrict__ H,
                       const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    using S = Short<P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tws = reinterpret_cast<C*>(smem_raw);
    // the (N/2 + 1) x 16 P half-spectrum block, row kx holding column t at
    // t ^ (kx & (16 P - 1)); afterwards the warps' transpose regions
    C* Sb = tws + TW1024_SLOTS;
    C* reg = Sb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y0 = blockIdx.x * S::ROWS, z = blockIdx.y, c = blockIdx.z;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    load_tw1024(tws, tw_g, g.lmax);
    const size_t plane = (size_t)3 * nz * ny;
    const size_t col0 = ((size_t)c * nz + z) * ny + y0;
    staged_loop<256, C>(
        (S::N / 2 + 1) * S::ROWS,
        [&](int i) {
            const int k = i / S::ROWS, t = i & (S::ROWS - 1);
            return y0 + t < ny ? X[(size_t)k * plane + col0 + t] : C{T(0), T(0)};
        },
        [&](int i, C a) {
            const int k = i / S::ROWS, t = i & (S::ROWS - 1);
            Sb[k * S::ROWS + (t ^ (k & (S::ROWS - 1)))] = a;
        });
    __syncthreads();
    // the spectrum of row t at bin k < N (Hermitian above N/2; DC and Nyquist real)
    auto spec = [&](int t, int k) {
        const int kk = k <= S::N / 2 ? k : S::N - k;
        C a = Sb[kk * S::ROWS + (t ^ (kk & (S::ROWS - 1)))];
        if (k > S::N / 2) a.y = -a.y;
        if (k == 0 || k == S::N / 2) a.y = T(0);
        return a;
    };
    C L[P][S::CN];
#pragma unroll
    for (int cc = 0; cc < S::CN; cc++) {
        const int k = lane + 32 * cc;
#pragma unroll
        for (int q = 0; q < P; q++) {  // Z_q = A + i B, rows warp + 16 q and warp + 16 q + 8
            const C A = spec(warp + 16 * q, k), B = spec(warp + 16 * q + 8, k);
            L[q][cc] = C{A.x - B.y, A.y + B.x};
        }
    }
    C v[32];
    tangle<P, C>(L, v, tws);
    __syncthreads();  // the block is consumed: its bytes become the transpose regions
    warp_fft1024_inv(v, reg + warp * R1025, tws);
    // v[a] = P z_p[n], p = lane mod P, n = (32 / P) a + lane / P:
    // Re -> row warp + 16 p, Im -> row warp + 16 p + 8
    const int p = lane & (P - 1);
    const int ya = y0 + warp + 16 * p, yb = ya + 8;
    const size_t ncell = (size_t)nx * ny * nz;
    T* ha = H + c * ncell + ((size_t)z * ny + ya) * nx;
    T* hb = H + c * ncell + ((size_t)z * ny + yb) * nx;
#pragma unroll
    for (int a = 0; a < 16; a++) {
        const int n = S::CN * a + (lane >> S::LGP);
        if (n < nx) {
            if (ya < ny) ha[n] = v[a].x * (T(1) / P);
            if (yb < ny) hb[n] = v[a].y * (T(1) / P);
        }
    }
}

template <typename T, int P>
size_t smem_short()
{
    const size_t blk = (size_t)(Short<P>::N / 2 + 1) * Short<P>::ROWS;
    const size_t body = (size_t)8 * R1025 > blk ? (size_t)8 * R1025 : blk;
    return ((size_t)TW1024_SLOTS + body) * sizeof(typename Cx<T>::t);
}

// P for the padded length L (0: none)
constexpr int short_p(int L) { return L == 512 ? 2 : L == 256 ? 4 : 0; }

template <typename T, int P>
cudaError_t launch_x_r2c_p(const Geometry& g, const T* M, const T* ms_map, T ms_scale, typename Cx<T>::t* X,
                           const typename Cx<T>::t* tw, cudaStream_t st)
{
    const size_t smem = smem_short<T, P>();
    cudaError_t e =
        cudaFuncSetAttribute(x_r2c_short_kernel<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    x_r2c_short_kernel<T, P><<<dim3((g.ny + Short<P>::ROWS - 1) / Short<P>::ROWS, g.nz, 3), 256, smem, st>>>(
        g, M, ms_map, ms_scale, X, tw);
    return cudaGetLastError();
}
template <typename T, int P>
cudaError_t launch_x_c2r_p(const Geometry& g, const typename Cx<T>::t* X, T* H, const typename Cx<T>::t* tw,
                           cudaStream_t st)
{
    const size_t smem = smem_short<T, P>();
    cudaError_t e =
        cudaFuncSetAttribute(x_c2r_short_kernel<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    x_c2r_short_kernel<T, P><<<dim3((g.ny + Short<P>::ROWS - 1) / Short<P>::ROWS, g.nz, 3), 256, smem, st>>>(
        g, X, H, tw);
    return cudaGetLastError();
}
template <typename T, int P>
cudaError_t launch_y_p(const Geometry& g, typename Cx<T>::t* X, typename Cx<T>::t* Y, const typename Cx<T>::t* tw,
                       cudaStream_t st, bool forward)
{
    const size_t smem = smem_short<T, P>();
    const dim3 grid((3 * g.nz + 8 * P - 1) / (8 * P), g.nkx);
    if (forward) {
        cudaError_t e =
            cudaFuncSetAttribute(y_fwd_short_kernel<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        y_fwd_short_kernel<T, P><<<grid, 256, smem, st>>>(g, X, Y, tw);
    } else {
        cudaError_t e =
            cudaFuncSetAttribute(y_inv_short_kernel<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        y_inv_short_kernel<T, P><<<grid, 256, smem, st>>>(g, Y, X, tw);
    }
    return cudaGetLastError();
}

}  // namespace

template <typename T>
bool x512_ok(const Geometry& g, int max_smem)
{
    const int P = short_p(g.px);
    if (P == 2) return g.nx <= 256 && smem_short<T, 2>() <= (size_t)max_smem;
    if (P == 4) return g.nx <= 128 && smem_short<T, 4>() <= (size_t)max_smem;
    return false;
}
template <typename T>
bool y512_ok(const Geometry& g, int max_smem)
{
    const int P = short_p(g.py);
    if (P == 2) return g.ny <= 256 && smem_short<T, 2>() <= (size_t)max_smem;
    if (P == 4) return g.ny <= 128 && smem_short<T, 4>() <= (size_t)max_smem;
    return false;
}

template <typename T>
cudaError_t launch_x_r2c_512(const Geometry& g, const T* M, const T* ms_map, T ms_scale, typename Cx<T>::t* X,
                             const typename Cx<T>::t* tw, cudaStream_t st)
{
    return short_p(g.px) == 2 ? launch_x_r2c_p<T, 2>(g, M, ms_map, ms_scale, X, tw, st)
                              : launch_x_r2c_p<T, 4>(g, M, ms_map, ms_scale, X, tw, st);
}
template <typename T>
cudaError_t launch_x_c2r_512(const Geometry& g, const typename Cx<T>::t* X, T* H, const typename Cx<T>::t* tw,
                             cudaStream_t st)
{
    return short_p(g.px) == 2 ? launch_x_c2r_p<T, 2>(g, X, H, tw, st) : launch_x_c2r_p<T, 4>(g, X, H, tw, st);
}
template <typename T>
cudaError_t launch_y_512(const Geometry& g, typename Cx<T>::t* X, typename Cx<T>::t* Y, const typename Cx<T>::t* tw,
                         cudaStream_t st, bool forward)
{
    return short_p(g.py) == 2 ? launch_y_p<T, 2>(g, X, Y, tw, st, forward) : launch_y_p<T, 4>(g, X, Y, tw, st, forward);
}

#define FFT512_INST(T)                                                                                           \
    template bool x512_ok<T>(const Geometry&, int);                                                             \
    template bool y512_ok<T>(const Geometry&, int);                                                             \
    template cudaError_t launch_x_r2c_512<T>(const Geometry&, const T*, const T*, T, Cx<T>::t*, const Cx<T>::t*, \
                                             cudaStream_t);                                                     \
    template cudaError_t launch_x_c2r_512<T>(const Geometry&, const Cx<T>::t*, T*, const Cx<T>::t*, cudaStream_t); \
    template cudaError_t launch_y_512<T>(const Geometry&, Cx<T>::t*, Cx<T>::t*, const Cx<T>::t*, cudaStream_t, bool);
FFT512_INST(float)
FFT512_INST(double)

}  // namespace boris
