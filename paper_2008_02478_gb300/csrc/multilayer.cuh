// Multi-mesh (layer stack) tables shared by the plan code and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "boris_internal.cuh"

namespace boris {

constexpr int ML_MAX_LAYERS = 16;
constexpr int ML_MAX_PLANES = 256;

// Passed by value to the embed / extract / LLG kernels.
struct MLTable {
    int nl, Z, NX, NY;
    int nx[ML_MAX_LAYERS], ny[ML_MAX_LAYERS], nz[ML_MAX_LAYERS];
    int ox[ML_MAX_LAYERS], oy[ML_MAX_LAYERS];
    int plane0[ML_MAX_LAYERS];            // first frame plane of each layer
    size_t off[ML_MAX_LAYERS + 1];        // offset of each layer in the concatenated vector field
    size_t total3;                        // 3 x total cells
    float hz[ML_MAX_LAYERS];              // z cell size (for the exchange stencil)
    float ms[ML_MAX_LAYERS];              // unused by the demag kernels
    unsigned char plane_layer[ML_MAX_PLANES];
};

// Host-side description of the unique inter-plane spectra.
struct MLHost {
    double hx, hy;
    std::vector<double> ua, ub, udz;  // target z size, source z size, |dz| of each unique spectrum
    std::vector<int> pairs;           // [p * Z + q]: unique index, bit 30 set when z_p < z_q
};

cudaError_t run_axis_n(const void* in, bool in_real, double2* out, int axis, int d0, int d1, int d2, int n, int P,
                       int ncomp, const double2* tw, int lglmax, cudaStream_t st, int pmode = 0);
cudaError_t ml_build_spectra(const MLHost& h, const Geometry& g, float* K, const double2* tw64, cudaStream_t st);
cudaError_t ml_embed(const MLTable& t, const float* M, const float* ms_map, float ms, float* F, cudaStream_t st);
cudaError_t ml_extract(const MLTable& t, const float* F, float* H, cudaStream_t st);
// The inter-plane sum in transform space.  variant 0: one CTA per (kx, tile),
// spectrum rows read by the threads; 1: the same with the rows staged by
// cp.async; v >= 2: one persistent launch of (v - 1) CTAs per SM over all
// (kx, tile) items, precomputed row offsets, packed FP32x2 products.  pairs:
// [p Z + q] unique index (bit 30: z_p < z_q); pcode: the same as the row
// offset u nkx 6 kyp / 32 with the sign in bit 31; inv_hz[p] = 1 / (z size of
// plane p) (the spectra hold a N_ab).
cudaError_t ml_mix(const Geometry& g, int Z, float2* Y, const float* K, const int* pairs, const unsigned* pcode,
                   const float* inv_hz, int variant, int nsm, cudaStream_t st);
size_t ml_mix_v2_smem(int Z);
// row pitch of the multi-mesh spectra K[u][kx][c][kyp]
int ml_kyp(const Geometry& g);

}  // namespace boris
