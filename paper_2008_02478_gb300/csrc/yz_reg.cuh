// Fused y-z spectral pass with the z stage in registers (templated kernel,
// instantiated per precision in yz_reg_f32.cu / yz_reg_f64.cu).
#pragma once
#include <cooperative_groups.h>

#include "boris_internal.cuh"

namespace cg = cooperative_groups;

namespace boris {

// ---------------------------------------------------------------------------
// yz_conv_reg: the same fused y-z pass with the z stage in registers.
//
// CTA r of a CC-CTA cluster owns the L = py/CC wavenumbers ky = r (mod CC) of
// one kx plane; shared memory holds the twiddle table and the plane slice
// [3][HZ][L + 1] (one pad element per line keeps line-parallel accesses free
// of bank conflicts) plus an equal second buffer.  The padded length-pz z
// transform of a column splits into its even and odd wavenumbers, two
// length-HZ = pz/2 transforms of x[z] and x[z] w_pz^z; thread (q, c, h) holds
// column q, component c, parity h in HZ registers, transforms it with
// compile-time twiddles, multiplies by row c of the kernel, transforms back,
// and the two parities are summed through shared memory.
// ---------------------------------------------------------------------------
template <typename T, int CC, int HZ, int NT>
__global__ void __launch_bounds__(NT) yz_conv_reg_kernel(Geometry g, typename Cx<T>::t* __restrict__ X,
                                                         const T* __restrict__ K,
                                                         const typename Cx<T>::t* __restrict__ tw_g)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int LGC = CC == 1 ? 0 : CC == 2 ? 1 : CC == 4 ? 2 : CC == 8 ? 3 : 4;
    constexpr int ROWS = HZ > 0 ? HZ : 1;  // rows per component in the slice
    const int r = CC == 1 ? 0 : (int)cg::this_cluster().block_rank();
    const int kx = blockIdx.y;
    const int ny = g.ny, nz = g.nz, py = g.py, pz = g.pz;
    const int lgL = g.lgy - LGC;
    const int L = 1 << lgL, LP = L + 1;
    const int lmax = g.lmax;
    C* tw = reinterpret_cast<C*>(smem_raw);  // [lmax]
    C* data = tw + lmax;                      // [3][ROWS][LP]
    C* extra = data + 3 * ROWS * LP;          // [3][ROWS][LP]
    C* plane = X + (size_t)kx * 3 * nz * ny;  // [3][nz][ny]
    const int tid = threadIdx.x;
    for (int i = tid; i < lmax; i += NT) tw[i] = tw_g[i];
    if (CC == 1) __syncthreads();
    else cg::this_cluster().sync();

    const int nitems = 3 * nz * L;
    const int chunk = (nitems + CC - 1) / CC;
    const int i0 = r * chunk, i1 = min(nitems, i0 + chunk);
    const int shy = g.lglmax - g.lgy;
    // ---- 1: forward cross-CTA radix-CC butterfly (natural order) ----------
    for (int it = i0 + tid; it < i1; it += NT) {
        const int n = it % L, line = it / L;  // line = c * nz + z
        const C* src = plane + (size_t)line * ny;
        C v[CC];
#pragma unroll
        for (int p = 0; p < CC; p++) {
            const int y = n + p * L;
            v[p] = y < ny ? src[y] : C{T(0), T(0)};
        }
        if (CC > 1) reg_fft<CC, -1>(v);
        const int row = (line / nz) * ROWS + (line % nz);
#pragma unroll
        for (int j = 0; j < CC; j++) {
            const int rr = CC == 1 ? 0 : (int)(__brev((unsigned)j) >> (32 - LGC));
            const C u = c_mul(v[j], tw[(n * rr) << shy]);
            if (CC == 1) data[row * LP + n] = u;
            else cg::this_cluster().map_shared_rank(data, rr)[row * LP + n] = u;
        }
    }
    if (CC == 1) __syncthreads();
    else cg::this_cluster().sync();

    // ---- 2: y transforms (DIF, bit-reversed positions) ---------------------
    Lines yl{3 * nz, nz, LP, ROWS * LP, 1, true};
    if (lgL > 0) fft_dif(data, yl, lgL, 0, tw, g.lglmax - lgL);

    // ---- 3: z stage in registers and kernel multiply ------------------------
    const int kyh = g.kyh, kzh = g.kzh;
    const T* Kx = K + (size_t)kx * kyh * g.krow;
    if constexpr (HZ == 0) {
        // 2D mode: one row per component, multiply only
        for (int q = tid; q < L; q += NT) {
            const int ky = r + CC * bitrev(q, lgL);
            const bool fy = ky > py / 2;
            const C* kp = reinterpret_cast<const C*>(Kx + (size_t)(fy ? py - ky : ky) * g.krow);
            const C k01 = kp[0], k23 = kp[1], k45 = kp[2];  // (xx,yy) (zz,xy) (xz,yz)
            const T kxx = k01.x, kyy = k01.y, kzz = k23.x;
            const T kxy = fy ? -k23.y : k23.y, kxz = k45.x, kyz = fy ? -k45.y : k45.y;
            const C a = data[q], b = data[LP + q], c = data[2 * LP + q];
            data[q] = C{kxx * a.x + kxy * b.x + kxz * c.x, kxx * a.y + kxy * b.y + kxz * c.y};
            data[LP + q] = C{kxy * a.x + kyy * b.x + kyz * c.x, kxy * a.y + kyy * b.y + kyz * c.y};
            data[2 * LP + q] = C{kxz * a.x + kyz * b.x + kzz * c.x, kxz * a.y + kyz * b.y + kzz * c.y};
        }
        __syncthreads();
    } else {
        constexpr int LGH = HZ == 1 ? 0 : HZ == 2 ? 1 : HZ == 4 ? 2 : HZ == 8 ? 3 : HZ == 16 ? 4 : HZ == 32 ? 5 : 6;
        const bool active = tid < 6 * L;
        const int q = tid % L;
        const int c = (tid / L) % 3;
        const int h = tid / (3 * L);
        C v[HZ];
        if (active) {
#pragma unroll
            for (int z = 0; z < HZ; z++) {
                C x = z < nz ? data[(c * ROWS + z) * LP + q] : C{T(0), T(0)};
                // x[z] w_pz^(h z), w_pz^z = w_128^(z * 128/pz)
                if (h) x = c_mul(x, cw128<C>(z * (64 / HZ)));
                v[z] = x;
            }
            reg_fft<HZ, -1>(v);
        }
        __syncthreads();
        C* buf = h ? extra : data;
        if (active) {
#pragma unroll
            for (int pos = 0; pos < HZ; pos++) buf[(c * ROWS + pos) * LP + q] = v[pos];
        }
        __syncthreads();
        if (active) {
            const int ky = r + CC * bitrev(q, lgL);
            const bool fy = ky > py / 2;
            const T* Kr = Kx + (size_t)(fy ? py - ky : ky) * g.krow;
            // row c of the symmetric kernel: (xx xy xz) (xy yy yz) (xz yz zz)
            const int i0c = c == 0 ? 0 : c == 1 ? 3 : 4;
            const int i1c = c == 0 ? 3 : c == 1 ? 1 : 5;
            const int i2c = c == 0 ? 4 : c == 1 ? 5 : 2;
            const int c1 = c == 0 ? 1 : 0, c2 = c == 2 ? 1 : 2;  // the other two components
#pragma unroll
            for (int pos = 0; pos < HZ; pos++) {
                const int kz = 2 * (LGH == 0 ? 0 : (int)(__brev((unsigned)pos) >> (32 - LGH))) + h;
                const bool fz = kz > pz / 2;
                const T* kp = Kr + (size_t)(fz ? pz - kz : kz) * 6;
                // sign flips: xy odd in ky; xz odd in kz; yz odd in both
                const T s3 = fy ? T(-1) : T(1), s4 = fz ? T(-1) : T(1), s5 = s3 * s4;
                auto kval = [&](int idx) -> T {
                    const T v0 = kp[idx];
                    return idx == 3 ? s3 * v0 : idx == 4 ? s4 * v0 : idx == 5 ? s5 * v0 : v0;
                };
                const T kc[3] = {kval(i0c), kval(i1c), kval(i2c)};
                const C m1 = buf[(c1 * ROWS + pos) * LP + q];
                const C m2 = buf[(c2 * ROWS + pos) * LP + q];
                const C own = v[pos];
                // H_c = k_c0 m_0 + k_c1 m_1 + k_c2 m_2 with own = m_c
                T wown, w1, w2;
                if (c == 0) { wown = kc[0]; w1 = kc[1]; w2 = kc[2]; }
                else if (c == 1) { wown = kc[1]; w1 = kc[0]; w2 = kc[2]; }
                else { wown = kc[2]; w1 = kc[0]; w2 = kc[1]; }
                v[pos] = C{wown * own.x + w1 * m1.x + w2 * m2.x, wown * own.y + w1 * m1.y + w2 * m2.y};
            }
            reg_fft<HZ, 1>(v);
        }
        __syncthreads();
        if (active && h) {
#pragma unroll
            for (int z = 0; z < HZ; z++)
                if (z < nz) extra[(c * ROWS + z) * LP + q] = c_mulc(v[z], cw128<C>(z * (64 / HZ)));
        }
        __syncthreads();
        if (active && !h) {
#pragma unroll
            for (int z = 0; z < HZ; z++)
                if (z < nz) data[(c * ROWS + z) * LP + q] = c_add(v[z], extra[(c * ROWS + z) * LP + q]);
        }
        __syncthreads();
    }

    // ---- 4: inverse y transforms (DIT, natural order out) -------------------
    if (lgL > 0) fft_dit(data, yl, lgL, 0, tw, g.lglmax - lgL);
    if (CC == 1) __syncthreads();
    else cg::this_cluster().sync();

    // ---- 5: inverse cross-CTA butterfly, written back in place --------------
    for (int it = i0 + tid; it < i1; it += NT) {
        const int n = it % L, line = it / L;
        const int row = (line / nz) * ROWS + (line % nz);
        // the inverse length-CC transform runs as a DIT: rank rr's value goes to
        // register bitrev(rr), and the output comes out in natural order of p
        C v[CC];
#pragma unroll
        for (int j = 0; j < CC; j++) {
            const int rr = CC == 1 ? 0 : (int)(__brev((unsigned)j) >> (32 - LGC));
            const C u = CC == 1 ? data[row * LP + n] : cg::this_cluster().map_shared_rank(data, rr)[row * LP + n];
            v[j] = c_mulc(u, tw[(n * rr) << shy]);
        }
        if (CC > 1) reg_fft<CC, 1>(v);
        C* dst = plane + (size_t)line * ny;
#pragma unroll
        for (int j = 0; j < CC; j++) {
            const int y = n + j * L;
            if (y < ny) dst[y] = v[j];
        }
    }
    if (CC > 1) cg::this_cluster().sync();
}


template <typename T, int CC, int HZ, int NT>
cudaError_t launch_yz_reg_t(const Geometry& g, size_t smem, typename Cx<T>::t* X, const T* K,
                            const typename Cx<T>::t* tw, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(yz_conv_reg_kernel<T, CC, HZ, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (CC > 8) {
        e = cudaFuncSetAttribute(yz_conv_reg_kernel<T, CC, HZ, NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CC, g.nkx, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CC;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, yz_conv_reg_kernel<T, CC, HZ, NT>, g, X, K, tw);
}

template <typename T, int CC, int NT>
cudaError_t launch_yz_reg_hz(const Geometry& g, size_t smem, typename Cx<T>::t* X, const T* K,
                             const typename Cx<T>::t* tw, cudaStream_t st)
{
    switch (g.pz / 2) {
    case 0: return launch_yz_reg_t<T, CC, 0, NT>(g, smem, X, K, tw, st);
    case 2: return launch_yz_reg_t<T, CC, 2, NT>(g, smem, X, K, tw, st);
    case 4: return launch_yz_reg_t<T, CC, 4, NT>(g, smem, X, K, tw, st);
    case 8: return launch_yz_reg_t<T, CC, 8, NT>(g, smem, X, K, tw, st);
    case 16: return launch_yz_reg_t<T, CC, 16, NT>(g, smem, X, K, tw, st);
    case 32: return launch_yz_reg_t<T, CC, 32, NT>(g, smem, X, K, tw, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace boris
