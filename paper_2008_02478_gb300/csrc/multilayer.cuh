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
cudaError_t ml_mix(const Geometry& g, int Z, float2* Y, const float* K, const int* pairs, cudaStream_t st);
// row pitch of the multi-mesh spectra K[u][kx][c][kyp]
int ml_kyp(const Geometry& g);

}  // namespace boris
