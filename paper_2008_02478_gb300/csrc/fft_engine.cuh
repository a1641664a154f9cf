// Shared-memory radix-2^K FFT passes for power-of-two lengths.
//
// The convolution theorem of Section 7 (forward transforms, point-by-point
// multiply, inverse transforms) is built here from in-place decimation-in-
// frequency (DIF) passes, which take natural-order input to bit-reversed output,
// and decimation-in-time (DIT) passes with conjugated twiddles, which take the
// bit-reversed spectrum back to natural order.  Because the kernel multiply is
// point-by-point, the spectrum never needs to be reordered.
//
// A pass groups K consecutive radix-2 stages: each thread loads 2^K elements
// of one line into registers, runs the K butterfly stages there, and writes
// them back, so a length-L transform costs ceil(log2 L / K) shared-memory
// round trips.  Twiddles come from a table tw[e] = exp(-2 pi i e / Lmax)
// computed on the host in FP64; a length-L transform reads it at stride
// Lmax / L.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "twiddle128.h"

namespace boris {

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

template <typename C> __device__ __forceinline__ C c_add(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C c_sub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
// FP32: the complex sum and difference as one packed FP32x2 instruction each
// (sm_100 and later), rounded like the two scalar operations.
template <> __device__ __forceinline__ float2 c_add<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 c_sub<float2>(float2 a, float2 b)
{
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
template <typename C> __device__ __forceinline__ C c_mul(C a, C b)
{
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C c_mulc(C a, C b)
{
    return C{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename C, typename T> __device__ __forceinline__ C c_scale(C a, T s) { return C{a.x * s, a.y * s}; }


__device__ __forceinline__ int bitrev(int v, int lg) { return lg == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - lg)); }

// Geometry of a batch of lines in shared memory: element e of line l lives at
// buf[(l / lsplit) * lstride_hi + (l % lsplit) * lstride_lo + e * estride].
// Two-level line indexing covers both "lines contiguous" layouts (z-lines of a
// [c][z][q] tile) and "elements contiguous" layouts (y-lines of [c][z][n]).
struct Lines {
    int nlines;
    int lsplit;
    int lstride_lo;
    int lstride_hi;
    int estride;
    bool lines_fast;  // consecutive threads take consecutive lines (else consecutive groups)
    __device__ __forceinline__ int base(int l) const { return (l / lsplit) * lstride_hi + (l % lsplit) * lstride_lo; }
};

// K radix-2 stages starting at stage s0 of a length 2^lgL transform.
// DIR = -1: DIF with twiddles w^e; DIR = +1: DIT (stages in reverse order) with conj(w^e).
template <int K, int DIR, typename C>
__device__ __forceinline__ void fft_pass(C* __restrict__ buf, const Lines& ln, int lgL, int s0,
                                         const C* __restrict__ tw, int twshift)
{
    constexpr int R = 1 << K;
    const int L = 1 << lgL;
    const int S = (L >> s0) >> K;  // stride between the elements of one group
    const int gpl = L >> K;        // groups per line
    const int total = ln.nlines * gpl;
    for (int g = threadIdx.x; g < total; g += blockDim.x) {
        int line, gi;
        if (ln.lines_fast) {
            line = g % ln.nlines;
            gi = g / ln.nlines;
        } else {
            line = g / gpl;
            gi = g % gpl;
        }
        const int o = gi % S;
        const int b = gi / S;
        const int e0 = b * (S << K) + o;
        C* p = buf + ln.base(line);
        C v[R];
#pragma unroll
        for (int j = 0; j < R; j++) v[j] = p[(e0 + j * S) * ln.estride];
        if (DIR < 0) {
#pragma unroll
            for (int t = 0; t < K; t++) {
                const int half = R >> (t + 1);
                const int s = s0 + t;
#pragma unroll
                for (int j = 0; j < R; j++) {
                    if ((j & half) == 0) {
                        const int off = o + (j & ((R >> t) - 1)) * S;
                        const C w = tw[(off << s) << twshift];
                        const C a = v[j], c = v[j + half];
                        v[j] = c_add(a, c);
                        v[j + half] = c_mul(c_sub(a, c), w);
                    }
                }
            }
        } else {
#pragma unroll
            for (int t = K - 1; t >= 0; t--) {
                const int half = R >> (t + 1);
                const int s = s0 + t;
#pragma unroll
                for (int j = 0; j < R; j++) {
                    if ((j & half) == 0) {
                        const int off = o + (j & ((R >> t) - 1)) * S;
                        const C w = tw[(off << s) << twshift];
                        const C a = v[j];
                        const C c = c_mulc(v[j + half], w);
                        v[j] = c_add(a, c);
                        v[j + half] = c_sub(a, c);
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < R; j++) p[(e0 + j * S) * ln.estride] = v[j];
    }
}

// All DIF stages from s_begin (natural order in, bit-reversed out), radix-8 passes.
template <typename C>
__device__ void fft_dif(C* buf, const Lines& ln, int lgL, int s_begin, const C* tw, int twshift)
{
    int s = s_begin;
    while (s < lgL) {
        const int k = lgL - s;
        if (k >= 3) {
            fft_pass<3, -1>(buf, ln, lgL, s, tw, twshift);
            s += 3;
        } else if (k == 2) {
            fft_pass<2, -1>(buf, ln, lgL, s, tw, twshift);
            s += 2;
        } else {
            fft_pass<1, -1>(buf, ln, lgL, s, tw, twshift);
            s += 1;
        }
        __syncthreads();
    }
}

// All DIT stages down to s_end (bit-reversed in, natural order out, unscaled).
// The grouping mirrors fft_dif so the two are exact inverses up to the factor L.
template <typename C>
__device__ void fft_dit(C* buf, const Lines& ln, int lgL, int s_end, const C* tw, int twshift)
{
    // replay the DIF grouping (passes of 3 stages from s_end, a shorter last one) in reverse
    const int npass = (lgL - s_end + 2) / 3;
    for (int i = npass - 1; i >= 0; i--) {
        const int st = s_end + 3 * i;
        const int k = lgL - st >= 3 ? 3 : lgL - st;
        if (k == 3) fft_pass<3, 1>(buf, ln, lgL, st, tw, twshift);
        else if (k == 2) fft_pass<2, 1>(buf, ln, lgL, st, tw, twshift);
        else fft_pass<1, 1>(buf, ln, lgL, st, tw, twshift);
        __syncthreads();
    }
}

constexpr int UNR = 8;  // independent global loads in flight per thread in staging loops

// Staging loops: every thread issues UNR independent loads before it uses any
// of them, so enough bytes are in flight per SM to cover HBM latency.
// f(i) loads element i; g(i, v) consumes it.
template <int NT, typename V, typename Load, typename Use>
__device__ __forceinline__ void staged_loop(int n, Load f, Use g)
{
    for (int b = threadIdx.x; b < n; b += NT * UNR) {
        V r[UNR];
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            const int i = b + u * NT;
            if (i < n) r[u] = f(i);
        }
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            const int i = b + u * NT;
            if (i < n) g(i, r[u]);
        }
    }
}

// exp(-2 pi i e / 128), e in [0, 128): the twiddles of every in-register
// transform of length <= 128, read with compile-time indices (a constant-cache
// broadcast).  Each translation unit that uses them holds its own copy and
// fills it from host FP64 cos/sin with upload_small_twiddles_here().
static __constant__ float2 c_w128f[128];
static __constant__ double2 c_w128d[128];
template <typename C> __device__ __forceinline__ C cw128(int e);
template <> __device__ __forceinline__ float2 cw128<float2>(int e) { return c_w128f[e]; }
template <> __device__ __forceinline__ double2 cw128<double2>(int e) { return c_w128d[e]; }

// w_128^e from the literal table, for indices known at compile time (the
// values then fold into the multiply instructions).
template <typename C> __device__ __forceinline__ C w128lit(int e);
template <> __device__ __forceinline__ float2 w128lit<float2>(int e)
{
    return make_float2((float)w128_re(e), (float)w128_im(e));
}
template <> __device__ __forceinline__ double2 w128lit<double2>(int e) { return make_double2(w128_re(e), w128_im(e)); }

// v * w_128^e for a compile-time e (exact for e = 0 and e = 32, i.e. 1 and -i).
template <int DIR, typename C>
__device__ __forceinline__ C twiddle128(C v, int e)
{
    if (e == 0) return v;
    if (e == 32) return DIR < 0 ? C{v.y, -v.x} : C{-v.y, v.x};
    const C w = w128lit<C>(e);
    return DIR < 0 ? c_mul(v, w) : c_mulc(v, w);
}

constexpr int reg_fft_lg(int n) { return n <= 1 ? 0 : 1 + reg_fft_lg(n / 2); }

// In-register transform of length N <= 128 (power of two), fully unrolled,
// radix 4 (one radix-2 stage where log2 N is odd): a radix-4 butterfly does
// the work of two radix-2 stages with three twiddle multiplies instead of
// four, the fourth being the free rotation by -i (or +i).  Same output order
// as the radix-2 form.
// DIR = -1: DIF, natural order in, bit-reversed out, w = exp(-2 pi i/N); a
//   block of length s = 4q maps (x0, x1, x2, x3) = v[j + {0, q, 2q, 3q}] to
//   v[j] = a0 + a2, v[j + q] = (a0 - a2) w_s^(2j), v[j + 2q] = (a1 + a3) w_s^j,
//   v[j + 3q] = (a1 - a3) w_s^(3j), with a0 = x0 + x2, a1 = x0 - x2,
//   a2 = x1 + x3, a3 = -i (x1 - x3).  ZHI: v[N/2 .. N-1] are zero on entry
//   (x2 = x3 = 0 in the first stage).
// DIR = +1: DIT with conjugate twiddles, bit-reversed in, natural out
//   (unscaled inverse); t0 = x0, t1 = x1 w_s^(-2j), t2 = x2 w_s^(-j),
//   t3 = x3 w_s^(-3j) give v[j] = t0 + t1 + t2 + t3, v[j + 2q] = t0 + t1 - t2 - t3,
//   v[j + q] = (t0 - t1) + i (t2 - t3), v[j + 3q] = (t0 - t1) - i (t2 - t3).
template <int N, int DIR, typename C, bool ZHI = false>
__device__ __forceinline__ void reg_fft(C* v)
{
    constexpr int LG = reg_fft_lg(N);
    if (DIR < 0) {
#pragma unroll
        for (int s = N; s >= 4; s /= 4) {
            const int q = s / 4, u = 128 / s;  // w_s^k = w_128^(k u)
            const bool zero_hi = ZHI && s == N;
#pragma unroll
            for (int b = 0; b < N; b += s) {
#pragma unroll
                for (int j = 0; j < q; j++) {
                    C* p = v + b + j;
                    C a0, a1, a2, t;
                    if (zero_hi) {
                        a0 = p[0];
                        a1 = p[0];
                        a2 = p[q];
                        t = p[q];
                    } else {
                        a0 = c_add(p[0], p[2 * q]);
                        a1 = c_sub(p[0], p[2 * q]);
                        a2 = c_add(p[q], p[3 * q]);
                        t = c_sub(p[q], p[3 * q]);
                    }
                    const C a3{t.y, -t.x};  // -i t
                    p[0] = c_add(a0, a2);
                    p[q] = twiddle128<-1>(c_sub(a0, a2), (2 * j * u) & 127);
                    p[2 * q] = twiddle128<-1>(c_add(a1, a3), (j * u) & 127);
                    p[3 * q] = twiddle128<-1>(c_sub(a1, a3), (3 * j * u) & 127);
                }
            }
        }
        if (LG & 1) {
#pragma unroll
            for (int b = 0; b < N; b += 2) {
                const C a = v[b];
                if (ZHI && N == 2) {
                    v[b + 1] = a;
                } else {
                    const C c = v[b + 1];
                    v[b] = c_add(a, c);
                    v[b + 1] = c_sub(a, c);
                }
            }
        }
    } else {
        if (LG & 1) {
#pragma unroll
            for (int b = 0; b < N; b += 2) {
                const C a = v[b], c = v[b + 1];
                v[b] = c_add(a, c);
                v[b + 1] = c_sub(a, c);
            }
        }
#pragma unroll
        for (int q = (LG & 1) ? 2 : 1; 4 * q <= N; q *= 4) {
            const int s = 4 * q, u = 128 / s;
#pragma unroll
            for (int b = 0; b < N; b += s) {
#pragma unroll
                for (int j = 0; j < q; j++) {
                    C* p = v + b + j;
                    const C t0 = p[0];
                    const C t1 = twiddle128<1>(p[q], (2 * j * u) & 127);
                    const C t2 = twiddle128<1>(p[2 * q], (j * u) & 127);
                    const C t3 = twiddle128<1>(p[3 * q], (3 * j * u) & 127);
                    const C A0 = c_add(t0, t1), A1 = c_sub(t0, t1), B0 = c_add(t2, t3), B1 = c_sub(t2, t3);
                    const C iB1{-B1.y, B1.x};  // i (t2 - t3)
                    p[0] = c_add(A0, B0);
                    p[2 * q] = c_sub(A0, B0);
                    p[q] = c_add(A1, iB1);
                    p[3 * q] = c_sub(A1, iB1);
                }
            }
        }
    }
}

static inline cudaError_t upload_small_twiddles_here()
{
    float2 f[128];
    double2 d[128];
    for (int e = 0; e < 128; e++) {
        const double a = 6.283185307179586476925286766559 * e / 128.0;
        d[e] = make_double2(std::cos(a), -std::sin(a));
        f[e] = make_float2((float)d[e].x, (float)d[e].y);
    }
    cudaError_t err = cudaMemcpyToSymbol(c_w128f, f, sizeof(f));
    if (err != cudaSuccess) return err;
    return cudaMemcpyToSymbol(c_w128d, d, sizeof(d));
}

}  // namespace boris
