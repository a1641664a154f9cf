// Demagnetising field H = -N * M by the convolution theorem (Section 7).
//
// Three kernels per evaluation, all data resident in HBM between them:
//   x_r2c   : zero-padded real-to-complex transform along x of M = Ms m, two
//             real rows packed per complex line; writes the spectrum X in the
//             plane-major layout [kx][c][z][y] so each kx plane is contiguous.
//   yz_conv : one thread-block cluster per kx plane.  CTA r of the cluster owns
//             the ky = r (mod C) residue class: a cross-CTA radix-C butterfly
//             (through distributed shared memory) splits the zero-padded
//             length-py y transform into C independent length-py/C transforms,
//             then each CTA runs its y transforms, the zero-padded z transform,
//             the point-by-point multiply with the real kernel spectrum (the
//             pipelined convolution of Section 7, generalised to the y axis),
//             the inverse z and y transforms, and the inverse cross-CTA
//             butterfly writes the plane back in place.
//   x_c2r   : complex-to-real inverse transform along x, cropped to nx.
// The 1/(px py pz) normalisation and the minus sign of H = -N * M are folded
// into the kernel spectrum, so no extra scaling pass exists.
#include <cooperative_groups.h>

#include "boris_internal.cuh"

namespace cg = cooperative_groups;

namespace boris {

// ---------------------------------------------------------------------------
// x_r2c
// ---------------------------------------------------------------------------
template <typename T, int TY>
__global__ void __launch_bounds__(256) x_r2c_kernel(Geometry g, const T* __restrict__ M,
                                                    const T* __restrict__ ms_map, T ms_scale,
                                                    typename Cx<T>::t* __restrict__ X,
                                                    const typename Cx<T>::t* __restrict__ tw)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);  // [TY/2][px]
    constexpr int HL = TY / 2;
    const int y0 = blockIdx.x * TY, z = blockIdx.y, c = blockIdx.z;
    const int px = g.px, nx = g.nx, ny = g.ny, nz = g.nz;
    const size_t ncell = (size_t)nx * ny * nz;
    const T* Mc = M + c * ncell;

    auto val = [&](int row, int x) -> T {
        const int y = y0 + row;
        if (y >= ny || x >= nx) return T(0);
        const size_t cell = ((size_t)z * ny + y) * nx + x;
        T v = Mc[cell];
        return ms_map ? v * ms_map[cell] : v * ms_scale;
    };

    if (px == 1) {
        for (int t = threadIdx.x; t < HL; t += blockDim.x) buf[t] = C{val(t, 0), val(t + HL, 0)};
    } else {
        // pruned first DIF stage: the upper half of every padded line is zero;
        // row t of the tile goes to the real part of line t % HL (t < HL) or
        // its imaginary part (t >= HL)
        const int half = px >> 1;
        const int sh = g.lglmax - g.lgx;
        const int nrow = min(TY, ny - y0);
        for (int i = threadIdx.x; i < HL * half; i += blockDim.x) buf[(i / half) * px + i % half] = C{T(0), T(0)};
        __syncthreads();
        const T* base = Mc + ((size_t)z * ny + y0) * nx;  // nrow contiguous rows
        const T* mbase = ms_map ? ms_map + ((size_t)z * ny + y0) * nx : nullptr;
        staged_loop<256, T>(nrow * nx, [&](int i) { return mbase ? base[i] * mbase[i] : base[i] * ms_scale; },
                            [&](int i, T v) {
                                const int row = i / nx, x = i % nx;
                                T* slot = reinterpret_cast<T*>(&buf[(row % HL) * px + x]) + (row >= HL ? 1 : 0);
                                *slot = v;
                            });
        __syncthreads();
        for (int i = threadIdx.x; i < HL * half; i += blockDim.x) {
            const int t = i / half, o = i % half;
            buf[t * px + o + half] = c_mul(buf[t * px + o], tw[o << sh]);
        }
    }
    __syncthreads();
    if (px > 1) {
        Lines ln{HL, HL, px, 0, 1, false};
        fft_dif(buf, ln, g.lgx, 1, tw, g.lglmax - g.lgx);
    }
    // unpack the two real spectra and store [kx][c][z][y]
    const int nkx = g.nkx;
    for (int i = threadIdx.x; i < nkx * TY; i += blockDim.x) {
        const int row = i % TY, kx = i / TY;
        const int y = y0 + row;
        if (y >= ny) continue;
        const int t = row % HL;
        const C zk = buf[t * px + bitrev(kx, g.lgx)];
        const C zm = buf[t * px + bitrev((px - kx) & (px - 1), g.lgx)];
        C out;
        if (row < HL) out = C{T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y)};
        else out = C{T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x)};
        X[(((size_t)kx * 3 + c) * nz + z) * ny + y] = out;
    }
}

// ---------------------------------------------------------------------------
// x_c2r
// ---------------------------------------------------------------------------
template <typename T, int TY>
__global__ void __launch_bounds__(256) x_c2r_kernel(Geometry g, const typename Cx<T>::t* __restrict__ X,
                                                    T* __restrict__ H,
                                                    const typename Cx<T>::t* __restrict__ tw)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);  // [TY/2][px]
    constexpr int HL = TY / 2;
    const int y0 = blockIdx.x * TY, z = blockIdx.y, c = blockIdx.z;
    const int px = g.px, nx = g.nx, ny = g.ny, nz = g.nz;
    const int nkx = g.nkx;
    struct AB {
        C a, b;
    };
    staged_loop<256, AB>(nkx * HL, [&](int i) {
        const int t = i % HL, kx = i / HL;
        const int ya = y0 + t, yb = y0 + t + HL;
        const size_t rowbase = ((size_t)kx * 3 + c) * nz + z;
        AB r;
        r.a = ya < ny ? X[rowbase * ny + ya] : C{T(0), T(0)};
        r.b = yb < ny ? X[rowbase * ny + yb] : C{T(0), T(0)};
        return r;
    }, [&](int i, AB r) {
        const int t = i % HL, kx = i / HL;
        const C A = r.a, B = r.b;
        const int km = (px - kx) & (px - 1);
        if (kx == 0 || kx == km) {
            // DC and Nyquist bins of a real signal are real
            buf[t * px + bitrev(kx, g.lgx)] = C{A.x, B.x};
        } else {
            buf[t * px + bitrev(kx, g.lgx)] = C{A.x - B.y, A.y + B.x};
            buf[t * px + bitrev(km, g.lgx)] = C{A.x + B.y, B.x - A.y};
        }
    });
    __syncthreads();
    if (px > 1) {
        Lines ln{HL, HL, px, 0, 1, false};
        fft_dit(buf, ln, g.lgx, 0, tw, g.lglmax - g.lgx);
    }
    const size_t ncell = (size_t)nx * ny * nz;
    T* Hc = H + c * ncell;
    for (int i = threadIdx.x; i < TY * nx; i += blockDim.x) {
        const int row = i / nx, x = i % nx;
        const int y = y0 + row;
        if (y >= ny) continue;
        const C v = buf[(row % HL) * px + x];
        Hc[((size_t)z * ny + y) * nx + x] = row < HL ? v.x : v.y;
    }
}

// ---------------------------------------------------------------------------
// In-register radix-2 DIF of length CC (natural in, bit-reversed out);
// DIR = -1 uses w = exp(-2 pi i e/CC), DIR = +1 the conjugate.
// ---------------------------------------------------------------------------
template <int CC, int DIR, typename C>
__device__ __forceinline__ void reg_dif(C* v, const C* __restrict__ tw, int lglmax)
{
    constexpr int LG = CC == 1 ? 0 : CC == 2 ? 1 : CC == 4 ? 2 : CC == 8 ? 3 : CC == 16 ? 4 : 5;
#pragma unroll
    for (int t = 0; t < LG; t++) {
        const int half = CC >> (t + 1);
#pragma unroll
        for (int j = 0; j < CC; j++) {
            if ((j & half) == 0) {
                const int e = (j & (2 * half - 1)) << t;
                const C w = tw[e << (lglmax - LG)];
                const C a = v[j], b = v[j + half];
                v[j] = c_add(a, b);
                v[j + half] = DIR < 0 ? c_mul(c_sub(a, b), w) : c_mulc(c_sub(a, b), w);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// yz_conv
// ---------------------------------------------------------------------------
template <typename T, int CC>
__global__ void __launch_bounds__(256) yz_conv_kernel(Geometry g, int Qc, typename Cx<T>::t* __restrict__ X,
                                                      const T* __restrict__ K,
                                                      const typename Cx<T>::t* __restrict__ tw)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int LGC = CC == 1 ? 0 : CC == 2 ? 1 : CC == 4 ? 2 : CC == 8 ? 3 : 4;
    const int r = CC == 1 ? 0 : (int)cg::this_cluster().block_rank();
    const int kx = blockIdx.y;
    const int ny = g.ny, nz = g.nz, py = g.py, pz = g.pz;
    const int lgL = g.lgy - LGC;
    const int L = 1 << lgL;
    const int lglmax = g.lglmax;
    C* data = reinterpret_cast<C*>(smem_raw);  // [3][nz][L]
    C* work = data + 3 * nz * L;               // [3][pz][Qc]
    C* plane = X + (size_t)kx * 3 * nz * ny;   // [3][nz][ny]
    const int nitems = 3 * nz * L;

    // ---- 1: forward cross-CTA radix-CC butterfly --------------------------
    // u_r[n] = w_py^(n r) * sum_p x[n + p L] w_CC^(p r), scattered to CTA r.
    {
        const int chunk = (nitems + CC - 1) / CC;
        const int i0 = r * chunk, i1 = min(nitems, i0 + chunk);
        for (int it = i0 + (int)threadIdx.x; it < i1; it += blockDim.x) {
            const int n = it % L, line = it / L;  // line = c * nz + z
            const C* src = plane + (size_t)line * ny;
            C v[CC];
#pragma unroll
            for (int p = 0; p < CC; p++) {
                const int y = n + p * L;
                v[p] = y < ny ? src[y] : C{T(0), T(0)};
            }
            reg_dif<CC, -1>(v, tw, lglmax);
#pragma unroll
            for (int j = 0; j < CC; j++) {
                const int rr = CC == 1 ? 0 : (int)(__brev((unsigned)j) >> (32 - LGC));
                const C u = c_mul(v[j], tw[(n * rr) << (lglmax - g.lgy)]);
                if (CC == 1) {
                    data[it] = u;
                } else {
                    C* dst = cg::this_cluster().map_shared_rank(data, rr);
                    dst[it] = u;
                }
            }
        }
    }
    if (CC == 1) __syncthreads();
    else cg::this_cluster().sync();

    // ---- 2: y transforms of length L (DIF, bit-reversed positions) ---------
    Lines yl{3 * nz, 3 * nz, L, 0, 1, false};
    if (lgL > 0) fft_dif(data, yl, lgL, 0, tw, lglmax - lgL);

    // ---- 3: z stage and kernel multiply, Qc columns at a time ---------------
    const int kyh = g.kyh;
    const T* Kx = K + (size_t)kx * kyh * g.krow;
    auto kernel_at = [&](int ky, int kz, T k[6]) {
        const bool fy = ky > py / 2, fz = kz > pz / 2;
        const int kyf = fy ? py - ky : ky, kzf = fz ? pz - kz : kz;
        const T* kp = Kx + (size_t)kyf * g.krow + kzf * 6;
#pragma unroll
        for (int i = 0; i < 6; i++) k[i] = kp[i];
        if (fy) { k[3] = -k[3]; k[5] = -k[5]; }
        if (fz) { k[4] = -k[4]; k[5] = -k[5]; }
    };
    auto mult = [&](const T k[6], C& a, C& b, C& c) {
        const C hx{k[0] * a.x + k[3] * b.x + k[4] * c.x, k[0] * a.y + k[3] * b.y + k[4] * c.y};
        const C hy{k[3] * a.x + k[1] * b.x + k[5] * c.x, k[3] * a.y + k[1] * b.y + k[5] * c.y};
        const C hz{k[4] * a.x + k[5] * b.x + k[2] * c.x, k[4] * a.y + k[5] * b.y + k[2] * c.y};
        a = hx; b = hy; c = hz;
    };
    if (pz == 1) {
        for (int q = threadIdx.x; q < L; q += blockDim.x) {
            const int ky = r + CC * bitrev(q, lgL);
            T k[6];
            kernel_at(ky, 0, k);
            C a = data[q], b = data[L + q], c = data[2 * L + q];
            mult(k, a, b, c);
            data[q] = a; data[L + q] = b; data[2 * L + q] = c;
        }
        __syncthreads();
    } else {
        const int hz = pz >> 1;
        const int shz = lglmax - g.lgz;
        for (int q0 = 0; q0 < L; q0 += Qc) {
            const int Qn = min(Qc, L - q0);
            // pruned first z stage: rows z >= nz are zero
            for (int i = threadIdx.x; i < 3 * hz * Qn; i += blockDim.x) {
                const int qq = i % Qn, rest = i / Qn, zz = rest % hz, c = rest / hz;
                const C a = zz < nz ? data[(c * nz + zz) * L + q0 + qq] : C{T(0), T(0)};
                work[(c * pz + zz) * Qc + qq] = a;
                work[(c * pz + zz + hz) * Qc + qq] = c_mul(a, tw[zz << shz]);
            }
            __syncthreads();
            Lines zl{3 * Qn, Qn, 1, pz * Qc, Qc, true};
            fft_dif(work, zl, g.lgz, 1, tw, shz);
            for (int i = threadIdx.x; i < pz * Qn; i += blockDim.x) {
                const int qq = i % Qn, pos = i / Qn;
                const int ky = r + CC * bitrev(q0 + qq, lgL);
                const int kz = bitrev(pos, g.lgz);
                T k[6];
                kernel_at(ky, kz, k);
                C* w0 = work + pos * Qc + qq;
                C a = w0[0], b = w0[pz * Qc], c = w0[2 * pz * Qc];
                mult(k, a, b, c);
                w0[0] = a; w0[pz * Qc] = b; w0[2 * pz * Qc] = c;
            }
            __syncthreads();
            fft_dit(work, zl, g.lgz, 1, tw, shz);
            // pruned last z stage: keep rows z < nz
            for (int i = threadIdx.x; i < 3 * nz * Qn; i += blockDim.x) {
                const int qq = i % Qn, rest = i / Qn, zz = rest % nz, c = rest / nz;
                const C a = work[(c * pz + zz) * Qc + qq];
                const C b = work[(c * pz + zz + hz) * Qc + qq];
                data[(c * nz + zz) * L + q0 + qq] = c_add(a, c_mulc(b, tw[zz << shz]));
            }
            __syncthreads();
        }
    }

    // ---- 4: inverse y transforms of length L (DIT, natural order out) -------
    if (lgL > 0) fft_dit(data, yl, lgL, 0, tw, lglmax - lgL);
    if (CC == 1) __syncthreads();
    else cg::this_cluster().sync();

    // ---- 5: inverse cross-CTA butterfly, written back in place --------------
    // y[n + p L] = sum_r w_CC^(-p r) conj(w_py^(n r)) v_r[n]
    {
        const int chunk = (nitems + CC - 1) / CC;
        const int i0 = r * chunk, i1 = min(nitems, i0 + chunk);
        for (int it = i0 + (int)threadIdx.x; it < i1; it += blockDim.x) {
            const int n = it % L, line = it / L;
            C v[CC];
#pragma unroll
            for (int rr = 0; rr < CC; rr++) {
                C u;
                if (CC == 1) u = data[it];
                else u = cg::this_cluster().map_shared_rank(data, rr)[it];
                v[rr] = c_mulc(u, tw[(n * rr) << (lglmax - g.lgy)]);
            }
            reg_dif<CC, 1>(v, tw, lglmax);
            C* dst = plane + (size_t)line * ny;
#pragma unroll
            for (int j = 0; j < CC; j++) {
                const int p = CC == 1 ? 0 : (int)(__brev((unsigned)j) >> (32 - LGC));
                const int y = n + p * L;
                if (y < ny) dst[y] = v[j];
            }
        }
    }
    if (CC > 1) cg::this_cluster().sync();
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <typename T>
static int xrow_tile(const Geometry& g)
{
    // rows per CTA: keep (TY/2) * px complex within 64 KB
    const size_t line = (size_t)g.px * sizeof(typename Cx<T>::t);
    if (line * 8 <= 65536) return 16;
    if (line * 4 <= 65536) return 8;
    return 4;
}

template <typename T, int TY>
static cudaError_t launch_r2c_ty(const Geometry& g, const T* M, const T* ms_map, T ms_scale,
                                 typename Cx<T>::t* X, const typename Cx<T>::t* tw, cudaStream_t st)
{
    const size_t smem = (size_t)(TY / 2) * g.px * sizeof(typename Cx<T>::t);
    cudaError_t e = cudaFuncSetAttribute(x_r2c_kernel<T, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.ny + TY - 1) / TY, g.nz, 3);
    x_r2c_kernel<T, TY><<<grid, 256, smem, st>>>(g, M, ms_map, ms_scale, X, tw);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_x_r2c(const Geometry& g, const T* M, const T* ms_map, T ms_scale,
                         typename Cx<T>::t* X, const typename Cx<T>::t* tw, cudaStream_t st, unsigned* absmax)
{
    if (x1024_ok<T>(g, 227 * 1024)) return launch_x_r2c_1024<T>(g, M, ms_map, ms_scale, X, tw, st, absmax);
    if (absmax) return cudaErrorInvalidValue;
    if (x512_ok<T>(g, 227 * 1024)) return launch_x_r2c_512<T>(g, M, ms_map, ms_scale, X, tw, st);
    if (x2048_ok<T>(g, 227 * 1024)) return launch_x_r2c_2048<T>(g, M, ms_map, ms_scale, X, tw, st);
    if (x4096_ok<T>(g, 227 * 1024)) return launch_x_r2c_4096<T>(g, M, ms_map, ms_scale, X, tw, st);
    switch (xrow_tile<T>(g)) {
    case 16: return launch_r2c_ty<T, 16>(g, M, ms_map, ms_scale, X, tw, st);
    case 8: return launch_r2c_ty<T, 8>(g, M, ms_map, ms_scale, X, tw, st);
    default: return launch_r2c_ty<T, 4>(g, M, ms_map, ms_scale, X, tw, st);
    }
}

template <typename T, int TY>
static cudaError_t launch_c2r_ty(const Geometry& g, const typename Cx<T>::t* X, T* H,
                                 const typename Cx<T>::t* tw, cudaStream_t st)
{
    const size_t smem = (size_t)(TY / 2) * g.px * sizeof(typename Cx<T>::t);
    cudaError_t e = cudaFuncSetAttribute(x_c2r_kernel<T, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.ny + TY - 1) / TY, g.nz, 3);
    x_c2r_kernel<T, TY><<<grid, 256, smem, st>>>(g, X, H, tw);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_x_c2r(const Geometry& g, const typename Cx<T>::t* X, T* H,
                         const typename Cx<T>::t* tw, cudaStream_t st, int* status, unsigned long long limit_ns)
{
    if constexpr (sizeof(T) == 4) {
        if (status && x_c2r_tma_ok(g, 227 * 1024)) return launch_x_c2r_1024_tma(g, X, H, tw, status, limit_ns, st);
    }
    if (x1024_ok<T>(g, 227 * 1024)) return launch_x_c2r_1024<T>(g, X, H, tw, st);
    if (x512_ok<T>(g, 227 * 1024)) return launch_x_c2r_512<T>(g, X, H, tw, st);
    if (x2048_ok<T>(g, 227 * 1024)) return launch_x_c2r_2048<T>(g, X, H, tw, st);
    if (x4096_ok<T>(g, 227 * 1024)) return launch_x_c2r_4096<T>(g, X, H, tw, st);
    switch (xrow_tile<T>(g)) {
    case 16: return launch_c2r_ty<T, 16>(g, X, H, tw, st);
    case 8: return launch_c2r_ty<T, 8>(g, X, H, tw, st);
    default: return launch_c2r_ty<T, 4>(g, X, H, tw, st);
    }
}

template <typename T>
static size_t yz_smem(const Geometry& g, int C, int Qc)
{
    const size_t cs = sizeof(typename Cx<T>::t);
    const size_t L = (size_t)g.py / C;
    size_t s = 3 * (size_t)g.nz * L * cs;
    if (g.pz > 1) s += 3 * (size_t)g.pz * Qc * cs;
    return s;
}

template <typename T>
void yz_candidates(const Geometry& g, int max_smem, YZSchedule* out, int* n)
{
    int k = 0;
    const size_t cs = sizeof(typename Cx<T>::t);
    // register z stage: HZ = pz/2 in {0, 2, ..., 32}; L = py/C; 6L threads when pz > 1
    const int hz = g.pz / 2;
    const bool hz_ok = g.pz == 1 || (hz >= 2 && hz <= 32);
    if (hz_ok) {
        const int rows = hz > 0 ? hz : 1;
        for (int C : {1, 8, 16}) {
            if (C > g.py) continue;
            const int L = g.py / C;
            for (int NT : {384, 768}) {
                if (sizeof(T) == 8 && NT > 384) continue;
                if (g.pz > 1 && 6 * L > NT) continue;
                if (g.pz == 1 && NT == 768) continue;
                const size_t smem = ((size_t)g.lmax + 2 * 3 * (size_t)rows * (L + 1)) * cs;
                if (smem > (size_t)max_smem) continue;
                out[k++] = YZSchedule{1, C, 0, NT, smem};
            }
        }
    }
    // shared-memory z stage: any nz
    const int cmax = g.py < 16 ? g.py : 16;
    for (int C = 1; C <= cmax; C *= 2) {
        const int L = g.py / C;
        const int Qc = L < 16 ? L : 16;
        const size_t smem = yz_smem<T>(g, C, Qc);
        if (smem <= (size_t)max_smem) out[k++] = YZSchedule{0, C, Qc, 256, smem};
    }
    *n = k;
}

template <typename T>
bool choose_yz_schedule(const Geometry& g, int max_smem, YZSchedule* out)
{
    YZSchedule c[16];
    int n = 0;
    yz_candidates<T>(g, max_smem, c, &n);
    if (n == 0) return false;
    *out = c[0];
    return true;
}

template <typename T, int CC>
static cudaError_t set_attr_cc(const YZSchedule& sc)
{
    cudaError_t e = cudaFuncSetAttribute(yz_conv_kernel<T, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc.smem);
    if (e != cudaSuccess) return e;
    if (CC > 8) e = cudaFuncSetAttribute(yz_conv_kernel<T, CC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <typename T, int CC>
static cudaError_t launch_yz_cc(const Geometry& g, const YZSchedule& sc, typename Cx<T>::t* X, const T* K,
                                const typename Cx<T>::t* tw, cudaStream_t st)
{
    // the attributes are per function: set them for this launch's shared memory
    cudaError_t e = set_attr_cc<T, CC>(sc);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CC, g.nkx, 1);
    cfg.blockDim = dim3(sc.threads, 1, 1);
    cfg.dynamicSmemBytes = sc.smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CC;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, yz_conv_kernel<T, CC>, g, sc.Qc, X, K, tw);
}

template <typename T>
cudaError_t yz_set_attributes(const YZSchedule& sc)
{
    if (sc.kind != 0) return cudaSuccess;  // set at each launch
    switch (sc.C) {
    case 1: return set_attr_cc<T, 1>(sc);
    case 2: return set_attr_cc<T, 2>(sc);
    case 4: return set_attr_cc<T, 4>(sc);
    case 8: return set_attr_cc<T, 8>(sc);
    case 16: return set_attr_cc<T, 16>(sc);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_yz_conv(const Geometry& g, const YZSchedule& sc, typename Cx<T>::t* X, const T* K,
                           const typename Cx<T>::t* tw, cudaStream_t st)
{
    if (sc.kind == 1) return launch_yz_reg<T>(g, sc, X, K, tw, st);
    switch (sc.C) {
    case 1: return launch_yz_cc<T, 1>(g, sc, X, K, tw, st);
    case 2: return launch_yz_cc<T, 2>(g, sc, X, K, tw, st);
    case 4: return launch_yz_cc<T, 4>(g, sc, X, K, tw, st);
    case 8: return launch_yz_cc<T, 8>(g, sc, X, K, tw, st);
    case 16: return launch_yz_cc<T, 16>(g, sc, X, K, tw, st);
    default: return cudaErrorInvalidValue;
    }
}

#define BORIS_INST(T)                                                                                         \
    template cudaError_t launch_x_r2c<T>(const Geometry&, const T*, const T*, T, Cx<T>::t*, const Cx<T>::t*, \
                                         cudaStream_t, unsigned*);                                            \
    template cudaError_t launch_yz_conv<T>(const Geometry&, const YZSchedule&, Cx<T>::t*, const T*,           \
                                           const Cx<T>::t*, cudaStream_t);                                    \
    template cudaError_t launch_x_c2r<T>(const Geometry&, const Cx<T>::t*, T*, const Cx<T>::t*, cudaStream_t, int*, \
                                         unsigned long long);                                                  \
    template bool choose_yz_schedule<T>(const Geometry&, int, YZSchedule*);                                   \
    template void yz_candidates<T>(const Geometry&, int, YZSchedule*, int*);                                  \
    template cudaError_t yz_set_attributes<T>(const YZSchedule&);
BORIS_INST(float)
BORIS_INST(double)

}  // namespace boris
