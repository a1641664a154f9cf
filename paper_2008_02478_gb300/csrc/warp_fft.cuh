// Length-1024 transforms held by one warp: lane b keeps the 32 values
// x[32 a + b] in registers (four-step decomposition 1024 = 32 x 32).
//
//   X[c + 32 d] = sum_b w_32^(b d) w_1024^(b c) sum_a x[32 a + b] w_32^(a c)
//
// Forward: a length-32 transform over a in registers, the twiddle
// w_1024^(b c) (shared-memory table), a transpose through a per-warp 32 x 32
// shared tile (column index XOR-swizzled with the row, so both the row-wise
// writes and the column-wise reads are free of bank conflicts), and a
// length-32 transform over b.  The inverse runs the same steps backwards with
// conjugate twiddles.  No block-wide barrier is involved: one warp owns the
// whole line.
#pragma once
#include "fft_engine.cuh"

namespace boris {

__device__ __forceinline__ constexpr int brev5(int v)
{
    return ((v & 1) << 4) | ((v & 2) << 2) | (v & 4) | ((v & 8) >> 2) | ((v & 16) >> 4);
}

// Twiddle tables in shared memory (TW1024_SLOTS entries reserved for either):
//  * rows: w_1024^(c b) at c * 32 + b (c, b < 32), so the lookup of one c by
//    the 32 lanes (b = lane) reads one contiguous row.  The plan keeps the
//    same table in global memory right after its length-lmax twiddles, so
//    filling the shared copy is a contiguous read.
//  * slots: w_1024^e at e + (e >> 4), filled from the plan's length-lmax
//    table at stride lmax / 1024.
constexpr int TW1024_SLOTS = 1024 + 64;

template <typename C>
__device__ __forceinline__ void load_tw1024(C* tws, const C* __restrict__ tw_g, int lmax)
{
    const C* src = tw_g + lmax;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) tws[i] = src[i];
}
__device__ __forceinline__ int tw1024_slot(int e) { return e + (e >> 4); }
template <typename C>
__device__ __forceinline__ void load_tw1024_slots(C* tws, const C* __restrict__ tw_g, int shift)
{
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) tws[tw1024_slot(e)] = tw_g[e << shift];
}

// Forward.  In: v[a] = x[32 a + lane].  Out: v[pos] = X[lane + 32 brev5(pos)].
// In two parts: _a ends with the transpose (the tile is free again on return),
// _b is the second register transform.  ZHI: x[n] = 0 for n >= 512 (the
// zero-padded upper half; v[16..31] are then not read).  TS: the tile layout,
// 0 = 32 x 32 with the column XOR-swizzled by the row (1024 entries), 33 =
// rows of 33 entries (1056 entries: constant offsets, no swizzle arithmetic);
// both keep the row writes and the column reads free of bank conflicts.
template <int TS>
__device__ __forceinline__ int tile_at(int row, int col)
{
    return TS == 33 ? row * 33 + col : row * 32 + (col ^ row);
}

template <typename C, bool ZHI = false, int TS = 0>
__device__ __forceinline__ void warp_fft1024_fwd_a(C (&v)[32], C* tile, const C* tws)
{
    const int lane = threadIdx.x & 31;
    reg_fft<32, -1, C, ZHI>(v);
#pragma unroll
    for (int pos = 0; pos < 32; pos++) {
        const int c = brev5(pos);
        const C t = c_mul(v[pos], tws[c * 32 + lane]);
        tile[tile_at<TS>(c, lane)] = t;  // row c, column lane
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < 32; b++) v[b] = tile[tile_at<TS>(lane, b)];  // row lane, column b
    __syncwarp();
}
template <typename C>
__device__ __forceinline__ void warp_fft1024_fwd_b(C (&v)[32])
{
    reg_fft<32, -1>(v);
}
template <typename C, bool ZHI = false>
__device__ __forceinline__ void warp_fft1024_fwd(C (&v)[32], C* tile, const C* tws)
{
    warp_fft1024_fwd_a<C, ZHI>(v, tile, tws);
    warp_fft1024_fwd_b(v);
}

// Inverse (unscaled).  In: v[brev5(d)] = Z[lane + 32 d].  Out: v[a] = z[32 a + lane].
// ROWTAB: tws holds the row table, else the slot table.  Split like the
// forward transform (_a ends with the transpose); TS as there.
template <typename C, bool ROWTAB = true, int TS = 0>
__device__ __forceinline__ void warp_fft1024_inv_a(C (&v)[32], C* tile, const C* tws)
{
    const int lane = threadIdx.x & 31;
    reg_fft<32, 1>(v);  // v[b] = sum_d Z[lane + 32 d] w_32^(-b d)
#pragma unroll
    for (int b = 0; b < 32; b++) {
        const C t = c_mulc(v[b], ROWTAB ? tws[b * 32 + lane] : tws[tw1024_slot(lane * b)]);
        tile[tile_at<TS>(b, lane)] = t;  // row b, column c = lane
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 32; c++) v[brev5(c)] = tile[tile_at<TS>(lane, c)];  // row b = lane, column c
    __syncwarp();
}
template <typename C>
__device__ __forceinline__ void warp_fft1024_inv_b(C (&v)[32])
{
    reg_fft<32, 1>(v);
}
template <typename C, bool ROWTAB = true>
__device__ __forceinline__ void warp_fft1024_inv(C (&v)[32], C* tile, const C* tws)
{
    warp_fft1024_inv_a<C, ROWTAB>(v, tile, tws);
    warp_fft1024_inv_b(v);
}

}  // namespace boris
