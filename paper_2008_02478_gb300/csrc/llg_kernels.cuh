// Arguments and launchers of the LLG kernels (llg.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace boris {

constexpr double MU0_D = 1.25663706143591729539e-6;  // 4 pi 1e-7

// Per-launch constants of the effective field and the step.
template <typename T>
struct LLGArgs {
    int nx, ny, nz;
    size_t ncell;
    T ihx2, ihy2, ihz2;  // 1/h^2 per axis
    T Ms, Ku, A;         // uniform values (used when the map is NULL)
    const T* ms_map;
    const T* ku_map;
    T e[3];
    T Hext[3];
    T gp;     // gamma / (1 + alpha^2)
    T alpha;
    T dt;
    double V;  // cell volume (energies)
    // further Table 1 terms (boris_field_terms); extra = 0 when none is set
    int extra;
    T K2;               // uniaxial second order along e
    T Kc1, Kc2;         // cubic anisotropy
    T c1[3], c2[3], c3[3];
    int dmi;            // 0 none, 1 bulk, 2 interfacial
    T D;                // DMI constant
    T kD;               // D / (2A): boundary slope of the non-homogeneous Neumann condition
    T hx, hy, hz;       // cell sizes (central differences, boundary ghosts)
    T J1, J2;           // surface exchange between consecutive multi-mesh layers (Eq. 5)
    int pbc;            // periodic axes (bit 0 x, 1 y, 2 z): stencil neighbours wrap around
    // thermal field: sigma_i = th_s0 / sqrt(Ms_i) (0: off); Philox key and step counter
    T th_s0;
    unsigned int seed_lo, seed_hi;
    const unsigned long long* step;
    const T* hadd;      // additive field map [3][nz][ny][nx] (e.g. an Oersted field) or NULL
    // RKF45 trial steps read their step size here (device memory, set by the
    // step controller) when non-NULL, else use dt
    const double* dt_dev;
};

// Device-side RKF45 step control (Section 2: 4th order with an embedded 5th
// order error estimate).  One trial = six stages; after it a one-thread
// controller kernel reads the FP64 error max |m5 - m4| (err_bits: the bit
// pattern of a non-negative double, which orders like the value), accepts
// when err <= tol or dt <= dt_min, sets the next step
// dt clip(0.9 (tol/err)^(1/5), 0.2, 2) within [dt_min, dt_max], and decides
// whether the trial loop of the captured step graph repeats.
struct RKFControl {
    double dt;                     // step of the next trial
    double dt_used;                // the step that was accepted
    double err;                    // error of the last trial
    double t;                      // sum of accepted steps
    unsigned long long err_bits;   // running max over cells of the trial in flight
    unsigned int attempts;         // trials of the current step
    int accepted;                  // the current step was accepted
    unsigned long long trials;     // all trials since the last reset of the counters
    unsigned long long accepted_steps;
    unsigned long long failed_steps;  // steps that ran out of trials
};
constexpr unsigned int RKF_MAX_TRIALS = 16;
// the next step to try
cudaError_t launch_rkf45_set_dt(RKFControl* c, double dt, bool reset_counters, cudaStream_t st);
// start of a step: no trial yet, error max cleared
cudaError_t launch_rkf45_begin(RKFControl* c, cudaStream_t st);
// after a trial; sets the trial loop's condition (1: repeat) and latches
// BORIS_ERR_STEP_CONTROL in *status when RKF_MAX_TRIALS trials were rejected
cudaError_t launch_rkf45_control(RKFControl* c, double tol, double dt_min, double dt_max, int* status,
                                 cudaGraphConditionalHandle loop, cudaStream_t st);
// end of a step: m = trial when the step was accepted (else m is unchanged)
template <typename T>
cudaError_t launch_rkf45_accept(const RKFControl* c, const T* trial, T* m, size_t n, cudaStream_t st);
// advances the thermal field's step counter by one (after an RK4 step) / sets it
cudaError_t launch_thermal_advance(unsigned long long* step, cudaStream_t st);
cudaError_t launch_thermal_set(unsigned long long* step, unsigned long long v, cudaStream_t st);
cudaError_t launch_philox_words(const unsigned int* ctr, const unsigned int* key, unsigned int* out, int n,
                                cudaStream_t st);

template <typename T>
cudaError_t launch_rk4_stage(const LLGArgs<T>& a, int s, const T* ms, const T* Hd, T* m0, T* acc, T* mnext,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_rkf45_stage(const LLGArgs<T>& a, int s, const T* ms, const T* Hd, const T* m0, T* kbuf, T* mnext,
                               unsigned long long* err_bits, cudaStream_t st);
template <typename T>
cudaError_t launch_fwd_stage(const LLGArgs<T>& a, int s, const T* ms, const T* Hd, const T* m0, T* Hs, T* ks,
                             T* mnext, cudaStream_t st);
template <typename T>
cudaError_t launch_bwd_start(const LLGArgs<T>& a, const T* m0, const T* k1, const T* k2, const T* k3, const T* k4,
                             const T* gout, T* gm, T* gk, cudaStream_t st);
template <typename T>
cudaError_t launch_bwd_local(const LLGArgs<T>& a, const T* ms, const T* Hs, const T* gk, T* gH, T* gml,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_bwd_field(const LLGArgs<T>& a, const T* ms, const T* gH, const T* DgH, const T* gml, T* gm,
                             T* gk_prev, T coef, T* gMs, T* gKu, cudaStream_t st);
struct MLTable;
cudaError_t launch_rk4_stage_ml(const LLGArgs<float>& a, const MLTable& t, int s, const float* ms, const float* Hd,
                                float* m0, float* acc, float* mnext, cudaStream_t st);
struct Geometry;
// inverse x transform + RK4 stage in one kernel (FP32, px = 1024; llg_fused.cu)
bool x_c2r_rk4_ok(const Geometry& g, int max_smem);
cudaError_t launch_x_c2r_rk4(const Geometry& g, const float2* X, const float2* tw, const LLGArgs<float>& a, int s,
                             const float* ms, float* m0, float* acc, float* mnext, cudaStream_t st);
// out[0..4]: demag, exchange, anisotropy, Zeeman, DMI energies (J), accumulated
template <typename T>
cudaError_t launch_energy(const LLGArgs<T>& a, const T* m, const T* Hd, double* out, cudaStream_t st);

}  // namespace boris
