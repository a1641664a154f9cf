// Internal declarations shared by the CUDA translation units of libboris.
#pragma once
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/boris.h"
#include "fft_engine.cuh"

namespace boris {

// Padded transform length along one axis: the smallest power of two that is
// >= 2n - 1, so the circular convolution of the zero-padded data equals the
// linear convolution (Section 7 pads by doubling; for n a power of two the two
// agree, and any length >= 2n - 1 gives the same result).  n = 1 needs none.
inline int padded_len(int n)
{
    if (n <= 1) return 1;
    int p = 1;
    while (p < 2 * n - 1) p <<= 1;
    return p;
}
inline int ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) l++;
    return l;
}

// Geometry of one demag problem on the device.
struct Geometry {
    int nx, ny, nz;       // mesh
    int px, py, pz;       // padded transform lengths
    int lgx, lgy, lgz;
    int nkx;              // px/2 + 1 spectral planes kept by the real transform
    int kyh, kzh;         // py/2 + 1, pz/2 + 1 (octant extent of the kernel spectrum)
    int krow;             // floats per (kx, ky') row of the kernel spectrum: kzh * 6 rounded
                          // up to a multiple of 4 (16-byte rows; the pad is zero)
    int lmax, lglmax;     // twiddle table length
};

// Launch schedule of the fused y-z spectral pass.
struct YZSchedule {
    int kind;     // 0: fused, z stage through shared-memory passes; 1: fused, z stage in
                  // registers; 2: split into y-forward, z-convolution and y-inverse kernels
    int C;        // kinds 0/1: CTAs per cluster (one cluster per kx plane; ky residues mod C);
                  // kind 2: CTAs per SM targeted by the z-convolution's register budget
    int Qc;       // z-columns processed per chunk of the z stage
    int threads;  // threads per CTA
    size_t smem;  // dynamic shared memory per CTA (bytes)
};

// Kernel launchers (demag.cu); T = float or double.
// absmax (optional, length-1024 x transforms only): raised to max |Ms M| over
// the field (as the bits of a non-negative float) for the FP16 spectrum scale
template <typename T>
cudaError_t launch_x_r2c(const Geometry& g, const T* M, const T* ms_map, T ms_scale,
                         typename Cx<T>::t* X, const typename Cx<T>::t* tw, cudaStream_t st,
                         unsigned* absmax = nullptr);
template <typename T>
cudaError_t launch_yz_conv(const Geometry& g, const YZSchedule& sc, typename Cx<T>::t* X,
                           const T* K, const typename Cx<T>::t* tw, cudaStream_t st);
// with a status word (FP32 plans) the tensor-copy form of the length-1024
// pass may run; its bounded wait latches BORIS_ERR_TIMEOUT there
template <typename T>
cudaError_t launch_x_c2r(const Geometry& g, const typename Cx<T>::t* X, T* H,
                         const typename Cx<T>::t* tw, cudaStream_t st, int* status = nullptr,
                         unsigned long long limit_ns = 1000000000ull);
template <typename T>
cudaError_t launch_yz_reg(const Geometry& g, const YZSchedule& sc, typename Cx<T>::t* X, const T* K,
                          const typename Cx<T>::t* tw, cudaStream_t st);
template <>
cudaError_t launch_yz_reg<float>(const Geometry& g, const YZSchedule& sc, float2* X, const float* K, const float2* tw,
                                 cudaStream_t st);
template <>
cudaError_t launch_yz_reg<double>(const Geometry& g, const YZSchedule& sc, double2* X, const double* K,
                                  const double2* tw, cudaStream_t st);
// Split schedule (demag_split.cu): part 0 = y forward X -> Y, part 1 = z
// transform + multiply + inverse z on Y, part 2 = y inverse Y -> X, with the
// padded spectrum Y laid out [kx][c][z][ky] (ky fastest).
template <typename T>
bool split_supported(const Geometry& g, int max_smem);
// occ: CTAs per SM that the z-convolution's register budget targets (2 or 3).
template <typename T>
cudaError_t launch_split(const Geometry& g, typename Cx<T>::t* X, typename Cx<T>::t* Y, const T* K,
                         const typename Cx<T>::t* tw, cudaStream_t st, int part, int occ);
cudaError_t upload_twiddles_split();
// Warp-per-line kernels for transform length 1024 (demag_fast.cu).
template <typename T>
bool x1024_ok(const Geometry& g, int max_smem);
template <typename T>
bool y1024_ok(const Geometry& g, int max_smem);
template <typename T>
cudaError_t launch_x_r2c_1024(const Geometry& g, const T* M, const T* ms_map, T ms_scale, typename Cx<T>::t* X,
                              const typename Cx<T>::t* tw, cudaStream_t st, unsigned* absmax = nullptr);
template <typename T>
cudaError_t launch_x_c2r_1024(const Geometry& g, const typename Cx<T>::t* X, T* H, const typename Cx<T>::t* tw,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_y_1024(const Geometry& g, typename Cx<T>::t* X, typename Cx<T>::t* Y, const typename Cx<T>::t* tw,
                          cudaStream_t st, bool forward);
cudaError_t upload_twiddles_fast();
// y passes of length 1024 on the 16-bit spectrum of the mixed-precision split
// schedule (layout [kx][c][part][z][ky]); BF16, or with fp16 FP16 scaled by the
// power of two s with s nx ny nz max|M| < 2^14 (max|M| from absmax)
cudaError_t launch_y_1024_b16(const Geometry& g, float2* X, void* Y16, const float2* tw, cudaStream_t st,
                              bool forward, bool fp16 = false, const unsigned* absmax = nullptr);
// max |Ms M| raised into *out (a non-negative float's bits; *out zeroed before)
cudaError_t launch_absmax(const Geometry& g, const float* M, const float* ms_map, float ms, unsigned* out, int nsm,
                          cudaStream_t st);
// Mixed-precision z stage with the spectrum stored in 16 bits (zconv_tc6.cu):
// pz = 64, py >= 256 in 128-column tiles; reads the FP16 kernel pairs K16
bool zconv_tc6_supported(const Geometry& g, int max_smem);
int zconv_tc6_kyp16(const Geometry& g);
size_t zconv_tc6_y16_bytes(const Geometry& g);
size_t zconv_tc6_k16_bytes(const Geometry& g);
cudaError_t zconv_tc6_build_k16(const Geometry& g, const float* K, void* K16, cudaStream_t st);
cudaError_t zconv_tc6_maps(const Geometry& g, void* Y16, void* K16, void* ymap, void* kmap, bool fp16 = false);
cudaError_t launch_zconv_tc6(const void* ymap, const void* kmap, const Geometry& g, void* Y16, const float2* tw,
                             int* status, uint32_t extra_tx, unsigned long long limit_ns, int nsm, cudaStream_t st,
                             bool fp16 = false);
// Length-512 passes (meshes of 129..256 cells along the axis), two lines per
// warp through the length-1024 warp transform (fft512.cu).
template <typename T>
bool x512_ok(const Geometry& g, int max_smem);
template <typename T>
bool y512_ok(const Geometry& g, int max_smem);
template <typename T>
cudaError_t launch_x_r2c_512(const Geometry& g, const T* M, const T* ms_map, T ms_scale, typename Cx<T>::t* X,
                             const typename Cx<T>::t* tw, cudaStream_t st);
template <typename T>
cudaError_t launch_x_c2r_512(const Geometry& g, const typename Cx<T>::t* X, T* H, const typename Cx<T>::t* tw,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_y_512(const Geometry& g, typename Cx<T>::t* X, typename Cx<T>::t* Y, const typename Cx<T>::t* tw,
                         cudaStream_t st, bool forward);
// Length-2048 passes (meshes of 513..1024 cells along the axis) from the
// warp-held length-1024 transform (fft2048.cu).
template <typename T>
bool x2048_ok(const Geometry& g, int max_smem);
template <typename T>
bool y2048_ok(const Geometry& g, int max_smem);
template <typename T>
cudaError_t launch_x_r2c_2048(const Geometry& g, const T* M, const T* ms_map, T ms_scale, typename Cx<T>::t* X,
                              const typename Cx<T>::t* tw, cudaStream_t st);
template <typename T>
cudaError_t launch_x_c2r_2048(const Geometry& g, const typename Cx<T>::t* X, T* H, const typename Cx<T>::t* tw,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_y_2048(const Geometry& g, typename Cx<T>::t* X, typename Cx<T>::t* Y, const typename Cx<T>::t* tw,
                          cudaStream_t st, bool forward);
// Length-4096 passes (meshes of 1025..2048 cells along the axis), fft4096.cu.
template <typename T>
bool x4096_ok(const Geometry& g, int max_smem);
template <typename T>
bool y4096_ok(const Geometry& g, int max_smem);
template <typename T>
cudaError_t launch_x_r2c_4096(const Geometry& g, const T* M, const T* ms_map, T ms_scale, typename Cx<T>::t* X,
                              const typename Cx<T>::t* tw, cudaStream_t st);
template <typename T>
cudaError_t launch_x_c2r_4096(const Geometry& g, const typename Cx<T>::t* X, T* H, const typename Cx<T>::t* tw,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_y_4096(const Geometry& g, typename Cx<T>::t* X, typename Cx<T>::t* Y, const typename Cx<T>::t* tw,
                          cudaStream_t st, bool forward);
// FP32 x complex-to-real (px = 1024, ny even) with the half-spectrum block
// fetched by tensor copies; a wait that gives up latches BORIS_ERR_TIMEOUT in *status
bool x_c2r_tma_ok(const Geometry& g, int max_smem);
cudaError_t launch_x_c2r_1024_tma(const Geometry& g, const float2* X, float* H, const float2* tw, int* status,
                                  unsigned long long limit_ns, cudaStream_t st);
// Tensor-core (FP16 / BF16) z stage of the split schedule (zconv_tc.cu), pz = 64.
bool zconv_tc_supported(const Geometry& g);
// bulk-copy pipelined z convolution of the split schedule (FP32; zconv_tma.cu);
// variant 1: one tile stage, three CTAs per SM; 2: two stages, two CTAs per SM
bool zconv_tma_supported(const Geometry& g, int max_smem, int variant);
// encodes the tensor map of Y (128 bytes at map) the kernel copies tiles with
cudaError_t zconv_tma_map(const Geometry& g, float2* Y, void* map);
cudaError_t launch_zconv_tma(const void* map, const Geometry& g, const float* K, int* status, uint32_t extra_tx,
                             unsigned long long limit_ns, int nsm, int variant, cudaStream_t st);
// residue-split z convolution of the split schedule (FP32; zconv_res.cu):
// reads the kernel spectrum in the blocked copy K2 [kx][ky'/32][kz'][pair][ky' mod 32]
// that zconv_res_build_k2 makes from K
bool zconv_res_supported(const Geometry& g, int max_smem);
int zconv_res_nkb(const Geometry& g);
size_t zconv_res_k2_bytes(const Geometry& g);
cudaError_t zconv_res_build_k2(const Geometry& g, const float* K, float2* K2, cudaStream_t st);
// encodes the tensor map of K2 (128 bytes at map)
cudaError_t zconv_res_kmap(const Geometry& g, float2* K2, void* map);
// ctas_per_sm 3: separate kernel stage and scratch; 4: the scratch overlays the kernel stage
cudaError_t launch_zconv_res(const void* ymap, const void* kmap, const Geometry& g, float2* Y, int* status,
                             uint32_t extra_tx, unsigned long long limit_ns, int nsm, int ctas_per_sm, cudaStream_t st);
// cuTensorMapEncodeTiled from the driver (nullptr if unavailable)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();
cudaError_t upload_twiddles_res();
cudaError_t launch_zconv_tc(const Geometry& g, float2* Y, const float* K, const float2* tw, bool bf16, cudaStream_t st);
// Tensor-core z stage on tcgen05 (zconv_tc5.cu): pz = 64, 17 <= nz <= 32, py >= 64; reads the
// blocked kernel copy K2 (kmap) and the tiles of Y (ymap) by tensor copies
bool zconv_tc5_supported(const Geometry& g, int max_smem);
// encodes the stage's tensor maps of Y and of the blocked kernel copy K2 (128 bytes each)
cudaError_t zconv_tc5_maps(const Geometry& g, float2* Y, float2* K2, void* ymap, void* kmap);
cudaError_t launch_zconv_tc5(const void* ymap, const void* kmap, const Geometry& g, float2* Y, const float2* tw,
                             bool bf16, int* status, uint32_t extra_tx, unsigned long long limit_ns, int nsm,
                             cudaStream_t st);
cudaError_t upload_twiddles_yz_f32();
cudaError_t upload_twiddles_yz_f64();
// Candidate schedules of the fused y-z pass that fit this geometry.
template <typename T>
void yz_candidates(const Geometry& g, int max_smem, YZSchedule* out, int* n);
template <typename T>
bool choose_yz_schedule(const Geometry& g, int max_smem, YZSchedule* out);
template <typename T>
cudaError_t yz_set_attributes(const YZSchedule& sc);

// Newell tensor precompute (newell.cu): writes the kernel spectrum K in the
// layout [kx][ky'][krow] with (kz', component) at kz' * 6 + component (octant,
// FP32 or FP64), already scaled by
// -1/(px py pz) so that the inverse transforms yield H = -N * M.
// images (optional, per axis): periodic images on each side summed into the
// tensor (multiple-images method); NULL or 0 for a non-periodic axis.
cudaError_t build_kernel_spectrum(const Geometry& g, double dx, double dy, double dz, double rs,
                                  void* K_out, bool k_is_f64, const double2* tw64, cudaStream_t st,
                                  const int* images = nullptr);
// Exact/asymptotic tensor on the displacement octant, FP64 [6][nz][ny][nx] (for tests).
cudaError_t newell_octant(int nx, int ny, int nz, double dx, double dy, double dz, double rs,
                          double* T, cudaStream_t st, const int* images = nullptr);

// Oersted kernel spectrum (newell.cu): KO[kx][ky'][kz'][4] = (Gx, Gy, Gz, 0),
// the imaginary parts of the padded g spectra scaled by 1/(px py pz), so that
// the field of a current density J is H^ = i (J^ x KO) (Gx odd in kx; Gy odd in
// ky; Gz odd in kz).
cudaError_t build_oersted_spectrum(const Geometry& g, double dx, double dy, double dz, double rs, float* KO,
                                   const double2* tw64, cudaStream_t st);
// Oersted multiply stages (zconv_res.cu): the residue-split z convolution with
// the curl multiply (pz >= 8; its kernel rows in the blocked copy with two
// pairs per kz', built by zconv_res_build_k2_curl), and the pointwise multiply
// for pz = 1.
bool zconv_res_curl_supported(const Geometry& g, int max_smem);
size_t zconv_res_k2_curl_bytes(const Geometry& g);
cudaError_t zconv_res_build_k2_curl(const Geometry& g, const float* KO, float2* K2, cudaStream_t st);
cudaError_t zconv_res_kmap_curl(const Geometry& g, float2* K2, void* map);
cudaError_t launch_zconv_res_curl(const void* ymap, const void* kmap, const Geometry& g, float2* Y, int* status,
                                  unsigned long long limit_ns, int nsm, cudaStream_t st);
cudaError_t launch_curl_point(const Geometry& g, float2* Y, const float* KO, cudaStream_t st);

// Twiddle table exp(-2 pi i e / n), e in [0, n), on the host in FP64.
void host_twiddles(int n, double2* out);

// Read-only view of a plan's geometry, schedule and kernel spectrum (capi.cu).
struct PlanView {
    Geometry g;
    YZSchedule yz;
    bool f64;
    cudaStream_t stream;
    int device;
    const void* K;
    const void* tw;
    bool ml;       // multi-mesh plan
    bool oersted;  // Oersted plan: its spectrum is the curl kernel, not the demag tensor
};
// Number of kernel classes timed by the plan's profiler.
constexpr int NPROF = 9;
bool plan_view(boris_plan p, PlanView* v);

// Thread-local last error message (capi.cu).
void set_error(const std::string& msg);

}  // namespace boris
