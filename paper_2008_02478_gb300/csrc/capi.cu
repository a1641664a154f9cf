// C ABI of libboris (declared in include/boris.h): plans, workspaces,
// status codes and the host-side orchestration of the demag and LLG kernels.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>

#include "boris_internal.cuh"
#include "llg_kernels.cuh"
#include "multilayer.cuh"

using namespace boris;

namespace boris {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
}  // namespace boris

struct boris_plan_s {
    Geometry g;
    double dx, dy, dz;
    unsigned flags;
    bool f64;
    int tc = 0;  // 0: FP32 z stage; 1: FP16 tensor cores; 2: BF16 tensor cores
    bool tc5 = false;  // tensor-core z stage on tcgen05 (else the mma.sync form)
    // BF16 and FP16 plans: the padded y-z spectrum stored in 16 bits (Y16), the z
    // stage on tcgen05 with the data as the 128-row operand, FP16 kernel pairs
    // (K16); FP16 plans scale the spectrum by a power of two from max |Ms M|,
    // which the x pass raises in absmax
    bool tc6 = false;
    unsigned* d_absmax = nullptr;
    void* Y16 = nullptr;
    void* K16 = nullptr;
    alignas(64) unsigned char ymap16[128] = {};
    alignas(64) unsigned char kmap16[128] = {};
    cudaStream_t stream;
    int device;
    YZSchedule yz;
    // FP32 RK4 stages fuse the inverse x transform with the stage (px = 1024)
    bool fuse_rk4 = false;
    // further field terms (boris_set_field_terms) and a counter that keys the CUDA graph
    boris_field_terms terms = {};
    bool has_terms = false;
    // periodic axes (multiple-images kernel, wrapping stencil): bit 0 x, 1 y, 2 z
    int pbc = 0;
    int images[3] = {0, 0, 0};
    // thermal field step counter (device), allocated with the first thermal terms
    unsigned long long* d_step = nullptr;
    // Oersted plan (boris_oersted_plan): K holds the spectrum KO [kx][ky'][kz'][4],
    // K2 its blocked copy for the residue-split z stage (pz > 1), kmap that copy's tensor map
    bool oersted = false;
    long long terms_version = 0;
    // device status word latched by bounded device-side waits (boris_sync_status)
    int* d_status = nullptr;
    int nsm = 0;
    uint32_t wait_extra_tx = 0;              // test hook: bytes that never arrive
    unsigned long long wait_limit_ns = 1000000000ull;
    // tensor map of Y for the bulk-copy z convolution (encoded on first use)
    alignas(64) unsigned char ymap[128] = {};
    bool ymap_ready = false;
    // kernel spectrum [kx][ky'][kz'][6] in the plan precision
    void* K = nullptr;
    // its column-major copy for the residue-split z convolution (kept only
    // when that schedule is chosen)
    void* K2 = nullptr;
    size_t k2_bytes = 0;
    alignas(64) unsigned char kmap[128] = {};  // its tensor map
    // twiddles exp(-2 pi i e / lmax) in the plan precision and in FP64
    void* tw = nullptr;
    double2* tw64 = nullptr;
    // spectral workspace [kx][c][z][y]
    void* X = nullptr;
    // column-major padded spectrum [kx][ky][c][z] of the split schedule
    void* Y = nullptr;
    // LLG workspace (allocated on first use)
    void* Hd = nullptr;
    void* msa = nullptr;
    void* msb = nullptr;
    void* acc = nullptr;
    void* kbuf = nullptr;   // RKF45: 6 stage derivatives
    void* mtrial = nullptr; // RKF45: trial solution
    // RKF45 step control on the device, its pinned host mirror, and the CUDA
    // graph of one step (trial loop as a conditional WHILE node), keyed by
    // the state pointer, the parameters and the field terms
    RKFControl* d_rkf = nullptr;
    RKFControl* h_rkf = nullptr;
    cudaGraphExec_t rkf_exec = nullptr;
    void* rkf_m = nullptr;
    boris_llg_params rkf_prm = {};
    long long rkf_terms_version = -1;
    long long rkf_trial_launches = 0;  // kernel launches of one trial
    double* energy = nullptr;
    void* m_dev_e2e = nullptr;
    // CUDA graph of one RK4 step (boris_llg_run_graph), keyed by its arguments
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    float* g_m = nullptr;
    boris_llg_params g_prm = {};
    double g_dt = 0.0;
    long long g_terms_version = -1;
    long long g_launches = 0;  // kernel launches inside one captured step
    // multi-mesh plans (boris_multimesh_plan)
    bool ml = false;
    MLTable mlt;
    double ml_zb[ML_MAX_LAYERS] = {};  // z of each layer's lower face (m)
    void* Kml = nullptr;    // unique inter-plane spectra [u][kx][c][kyp]
    int* d_pairs = nullptr; // [Z * Z]
    unsigned* d_pcode = nullptr;  // [Z * Z] spectrum row offsets / 32, kz sign in bit 31
    float* d_invhz = nullptr;     // [Z] 1 / z size of each plane
    int ml_variant = 1;           // inter-plane sum kernel (ml_mix), chosen by timing at plan time
    float* Mf = nullptr;    // frame fields [3][Z][NY][NX]
    float* Hf = nullptr;
    int ml_unique = 0;
    // adjoint workspace: stage states m2..m4, stage fields, stage derivatives,
    // stage cotangents, and three scratch fields
    void* bw = nullptr;
    size_t bytes = 0;
    // optional per-kernel CUDA-event timing (boris_profile_enable)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
    long long launches = 0;  // kernels launched by the library on this plan
};

namespace {

#define CUDA_TRY(expr)                                                                             \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e != cudaSuccess) {                                                                   \
            set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));                         \
            return _e == cudaErrorMemoryAllocation ? BORIS_ERR_OOM : BORIS_ERR_CUDA;               \
        }                                                                                          \
    } while (0)

int fail(int code, const std::string& msg)
{
    set_error(msg);
    return code;
}

int dev_alloc(boris_plan p, void** ptr, size_t bytes)
{
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? BORIS_ERR_OOM : BORIS_ERR_CUDA,
                    std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    p->bytes += bytes;
    return BORIS_OK;
}

bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

// The plan's twiddle tables, FP64 (tw64) and in the plan precision (tw):
// entries e < lmax are exp(-2 pi i e / lmax); the 1024 entries after them are
// exp(-2 pi i c b / 1024) at c * 32 + b (c, b < 32), the row-per-c table the
// length-1024 warp transforms copy to shared memory.
int upload_plan_twiddles(boris_plan p, const Geometry& g, bool f64)
{
    const int n = g.lmax + 1024;
    std::vector<double2> tw(n);
    host_twiddles(g.lmax, tw.data());
    const double twopi = 6.283185307179586476925286766559;
    for (int i = 0; i < 1024; i++) {
        const double a = twopi * (double)((i >> 5) * (i & 31)) / 1024.0;
        tw[g.lmax + i] = make_double2(std::cos(a), -std::sin(a));
    }
    int rc;
    if ((rc = dev_alloc(p, (void**)&p->tw64, n * sizeof(double2)))) return rc;
    if (cudaMemcpy(p->tw64, tw.data(), n * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(BORIS_ERR_CUDA, "twiddle upload");
    if (f64) {
        p->tw = p->tw64;
        return BORIS_OK;
    }
    std::vector<float2> twf(n);
    for (int i = 0; i < n; i++) twf[i] = make_float2((float)tw[i].x, (float)tw[i].y);
    if ((rc = dev_alloc(p, &p->tw, n * sizeof(float2)))) return rc;
    if (cudaMemcpy(p->tw, twf.data(), n * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(BORIS_ERR_CUDA, "twiddle upload");
    return BORIS_OK;
}

size_t ncell(const boris_plan p)
{
    if (p->ml) return p->mlt.total3 / 3;
    return (size_t)p->g.nx * p->g.ny * p->g.nz;
}

cudaEvent_t take_event(boris_plan p)
{
    if (p->ev_pool.empty()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    cudaEvent_t e = p->ev_pool.back();
    p->ev_pool.pop_back();
    return e;
}

// Runs one kernel launcher; with profiling on, brackets it with CUDA events on
// the plan's stream and files the pair under kernel class `kind`.
template <typename F>
cudaError_t timed(boris_plan p, int kind, F&& launch)
{
    p->launches++;
    if (!p->prof) return launch();
    cudaEvent_t a = take_event(p), b = take_event(p);
    if (a) cudaEventRecord(a, p->stream);
    cudaError_t e = launch();
    if (b) cudaEventRecord(b, p->stream);
    if (a && b) p->ev_used.push_back({kind, {a, b}});
    return e;
}

template <typename T>
cudaError_t yz_stage(boris_plan p, const YZSchedule& sc)
{
    using C = typename Cx<T>::t;
    if (sc.kind == 2 && p->tc6) {
        const bool h16 = p->tc == 1;
        cudaError_t e = timed(p, 5, [&] {
            return launch_y_1024_b16(p->g, (float2*)p->X, p->Y16, (const float2*)p->tw, p->stream, true, h16,
                                     p->d_absmax);
        });
        if (e == cudaSuccess)
            e = timed(p, 6, [&] {
                return launch_zconv_tc6(p->ymap16, p->kmap16, p->g, p->Y16, (const float2*)p->tw, p->d_status,
                                        p->wait_extra_tx, p->wait_limit_ns, p->nsm, p->stream, h16);
            });
        if (e == cudaSuccess)
            e = timed(p, 7, [&] {
                return launch_y_1024_b16(p->g, (float2*)p->X, p->Y16, (const float2*)p->tw, p->stream, false, h16,
                                         p->d_absmax);
            });
        return e;
    }
    if (sc.kind == 2) {
        cudaError_t e = cudaSuccess;
        for (int part = 0; part < 3 && e == cudaSuccess; part++)
            e = timed(p, 5 + part, [&] {
                if (part == 1 && p->tc && p->tc5)
                    return launch_zconv_tc5(p->ymap, p->kmap, p->g, (float2*)p->Y, (const float2*)p->tw, p->tc == 2,
                                            p->d_status, p->wait_extra_tx, p->wait_limit_ns, p->nsm, p->stream);
                if (part == 1 && p->tc)
                    return launch_zconv_tc(p->g, (float2*)p->Y, (const float*)p->K, (const float2*)p->tw, p->tc == 2,
                                           p->stream);
                if (part == 1 && sc.Qc == 3) {
                    if (!p->ymap_ready) {
                        cudaError_t me = zconv_tma_map(p->g, (float2*)p->Y, p->ymap);
                        if (me != cudaSuccess) return me;
                        p->ymap_ready = true;
                    }
                    return launch_zconv_res(p->ymap, p->kmap, p->g, (float2*)p->Y, p->d_status, p->wait_extra_tx,
                                            p->wait_limit_ns, p->nsm, sc.C, p->stream);
                }
                if (part == 1 && sc.Qc >= 1) {
                    if (!p->ymap_ready) {
                        cudaError_t me = zconv_tma_map(p->g, (float2*)p->Y, p->ymap);
                        if (me != cudaSuccess) return me;
                        p->ymap_ready = true;
                    }
                    return launch_zconv_tma(p->ymap, p->g, (const float*)p->K, p->d_status, p->wait_extra_tx,
                                            p->wait_limit_ns, p->nsm, sc.Qc, p->stream);
                }
                return launch_split<T>(p->g, (C*)p->X, (C*)p->Y, (const T*)p->K, (const C*)p->tw, p->stream, part,
                                       sc.C);
            });
        return e;
    }
    return timed(p, 1, [&] { return launch_yz_conv<T>(p->g, sc, (C*)p->X, (const T*)p->K, (const C*)p->tw, p->stream); });
}

int ml_demag_apply(boris_plan p, const float* M, const float* ms_map, float ms_scale, float* H)
{
    float2* X = (float2*)p->X;
    float2* Yb = (float2*)p->Y;
    const float2* tw = (const float2*)p->tw;
    CUDA_TRY(timed(p, 4, [&] { return ml_embed(p->mlt, M, ms_map, ms_scale, p->Mf, p->stream); }));
    CUDA_TRY(timed(p, 0, [&] { return launch_x_r2c<float>(p->g, p->Mf, nullptr, 1.0f, X, tw, p->stream); }));
    CUDA_TRY(timed(p, 5, [&] { return launch_split<float>(p->g, X, Yb, nullptr, tw, p->stream, 0, 2); }));
    CUDA_TRY(timed(p, 6, [&] {
        return ml_mix(p->g, p->mlt.Z, Yb, (const float*)p->Kml, p->d_pairs, p->d_pcode, p->d_invhz, p->ml_variant,
                      p->nsm, p->stream);
    }));
    CUDA_TRY(timed(p, 7, [&] { return launch_split<float>(p->g, X, Yb, nullptr, tw, p->stream, 2, 2); }));
    CUDA_TRY(timed(p, 2, [&] { return launch_x_c2r<float>(p->g, X, p->Hf, tw, p->stream, p->d_status, p->wait_limit_ns); }));
    CUDA_TRY(timed(p, 4, [&] { return ml_extract(p->mlt, p->Hf, H, p->stream); }));
    return BORIS_OK;
}

// Forward x transform and y-z convolution: X holds the x half spectrum of H_d.
template <typename T>
int demag_to_spectrum_t(boris_plan p, const T* M, const T* ms_map, T ms_scale)
{
    using C = typename Cx<T>::t;
    // FP16 spectrum: the x pass also finds max |Ms M| for the y passes' scale
    unsigned* absmax = nullptr;
    if constexpr (sizeof(T) == 4) {
        if (p->tc6 && p->tc == 1) {
            absmax = p->d_absmax;
            CUDA_TRY(cudaMemsetAsync(absmax, 0, sizeof(unsigned), p->stream));
            if (!x1024_ok<float>(p->g, 227 * 1024)) {
                CUDA_TRY(timed(p, 4, [&] {
                    return launch_absmax(p->g, (const float*)M, (const float*)ms_map, (float)ms_scale, absmax, p->nsm,
                                         p->stream);
                }));
                absmax = nullptr;
            }
        }
    }
    CUDA_TRY(timed(p, 0, [&] {
        return launch_x_r2c<T>(p->g, M, ms_map, ms_scale, (C*)p->X, (const C*)p->tw, p->stream, absmax);
    }));
    CUDA_TRY(yz_stage<T>(p, p->yz));
    return BORIS_OK;
}

template <typename T>
int demag_apply_t(boris_plan p, const T* M, const T* ms_map, T ms_scale, T* H)
{
    using C = typename Cx<T>::t;
    if (p->oersted) return fail(BORIS_ERR_INVALID_ARG, "an Oersted plan serves boris_oersted_apply only");
    if constexpr (sizeof(T) == 4) {
        if (p->ml) return ml_demag_apply(p, M, ms_map, ms_scale, H);
    }
    int rc = demag_to_spectrum_t<T>(p, M, ms_map, ms_scale);
    if (rc) return rc;
    CUDA_TRY(timed(p, 2, [&] {
        return launch_x_c2r<T>(p->g, (const C*)p->X, H, (const C*)p->tw, p->stream, p->d_status, p->wait_limit_ns);
    }));
    return BORIS_OK;
}

template <typename T>
int check_params(boris_plan p, const boris_llg_params* prm, LLGArgs<T>* a, double dt)
{
    if (!prm) return fail(BORIS_ERR_INVALID_ARG, "params is NULL");
    if (!(prm->A >= 0) || !(prm->alpha >= 0) || !(prm->gamma > 0))
        return fail(BORIS_ERR_INVALID_ARG, "need A >= 0, alpha >= 0, gamma > 0");
    if (!prm->Ms_map && !(prm->Ms > 0)) return fail(BORIS_ERR_INVALID_ARG, "need Ms > 0 or an Ms map");
    if ((prm->Ms_map && !aligned16(prm->Ms_map)) || (prm->Ku_map && !aligned16(prm->Ku_map)))
        return fail(BORIS_ERR_INVALID_ARG, "maps must be 16-byte aligned");
    const Geometry& g = p->g;
    a->nx = g.nx;
    a->ny = g.ny;
    a->nz = g.nz;
    a->ncell = ncell(p);
    a->ihx2 = (T)(1.0 / (p->dx * p->dx));
    a->ihy2 = (T)(1.0 / (p->dy * p->dy));
    a->ihz2 = (T)(1.0 / (p->dz * p->dz));
    a->Ms = (T)prm->Ms;
    a->Ku = (T)prm->Ku;
    a->A = (T)prm->A;
    a->ms_map = (const T*)prm->Ms_map;
    a->ku_map = (const T*)prm->Ku_map;
    for (int c = 0; c < 3; c++) {
        a->e[c] = (T)prm->easy[c];
        a->Hext[c] = (T)prm->Hext[c];
    }
    a->gp = (T)(prm->gamma / (1.0 + prm->alpha * prm->alpha));
    a->alpha = (T)prm->alpha;
    a->dt = (T)dt;
    a->V = p->dx * p->dy * p->dz;
    const boris_field_terms& t = p->terms;
    a->extra = p->has_terms ? 1 : 0;
    a->K2 = (T)t.K2;
    a->Kc1 = (T)t.Kc1;
    a->Kc2 = (T)t.Kc2;
    const double e3[3] = {t.cubic_e1[1] * t.cubic_e2[2] - t.cubic_e1[2] * t.cubic_e2[1],
                          t.cubic_e1[2] * t.cubic_e2[0] - t.cubic_e1[0] * t.cubic_e2[2],
                          t.cubic_e1[0] * t.cubic_e2[1] - t.cubic_e1[1] * t.cubic_e2[0]};
    for (int c = 0; c < 3; c++) {
        a->c1[c] = (T)t.cubic_e1[c];
        a->c2[c] = (T)t.cubic_e2[c];
        a->c3[c] = (T)e3[c];
    }
    a->dmi = p->has_terms ? t.dmi : 0;
    a->D = (T)(a->dmi ? t.D : 0.0);
    if (a->dmi && !(prm->A > 0)) return fail(BORIS_ERR_INVALID_ARG, "DMI needs A > 0 (boundary slope D/2A)");
    a->kD = (T)(a->dmi ? t.D / (2.0 * prm->A) : 0.0);
    a->hx = (T)p->dx;
    a->hy = (T)p->dy;
    a->hz = (T)p->dz;
    a->J1 = (T)t.J1;
    a->J2 = (T)t.J2;
    a->pbc = p->pbc;
    const double kB = 1.380649e-23;
    a->th_s0 = (T)((p->has_terms && t.temperature > 0 && dt > 0)
                       ? std::sqrt(2.0 * prm->alpha * kB * t.temperature / (prm->gamma * MU0_D * a->V * dt))
                       : 0.0);
    a->seed_lo = (unsigned int)(t.seed & 0xffffffffull);
    a->seed_hi = (unsigned int)(t.seed >> 32);
    a->step = p->d_step;
    a->hadd = p->has_terms ? (const T*)t.H_add : nullptr;
    a->dt_dev = nullptr;
    if (a->th_s0 > 0 && !p->d_step) return fail(BORIS_ERR_INVALID_ARG, "thermal step counter missing");
    if (a->th_s0 > 0) a->extra = 1;
    return BORIS_OK;
}

template <typename T>
int ensure_llg_workspace(boris_plan p, bool rkf)
{
    const size_t vb = 3 * ncell(p) * sizeof(T);
    int rc;
    if (!p->Hd && (rc = dev_alloc(p, &p->Hd, vb))) return rc;
    if (!p->msa && (rc = dev_alloc(p, &p->msa, vb))) return rc;
    if (!p->msb && (rc = dev_alloc(p, &p->msb, vb))) return rc;
    if (!p->acc && (rc = dev_alloc(p, &p->acc, vb))) return rc;
    if (rkf) {
        if (!p->kbuf && (rc = dev_alloc(p, &p->kbuf, 6 * vb))) return rc;
        if (!p->mtrial && (rc = dev_alloc(p, &p->mtrial, vb))) return rc;
        if (!p->d_rkf) {
            if ((rc = dev_alloc(p, (void**)&p->d_rkf, sizeof(RKFControl)))) return rc;
            CUDA_TRY(cudaMemsetAsync(p->d_rkf, 0, sizeof(RKFControl), p->stream));
        }
        if (!p->h_rkf) CUDA_TRY(cudaMallocHost((void**)&p->h_rkf, sizeof(RKFControl)));
    }
    return BORIS_OK;
}

template <typename T>
int rk4_step_t(boris_plan p, T* m, const LLGArgs<T>& a)
{
    T* ms_map = (T*)a.ms_map;
    const T ms_scale = a.Ms;
    T* Hd = (T*)p->Hd;
    T* acc = (T*)p->acc;
    T* sa = (T*)p->msa;
    T* sb = (T*)p->msb;
    // stage states: m0 -> sa -> sb -> sa
    const T* in[4] = {m, sa, sb, sa};
    T* out[4] = {sa, sb, sa, nullptr};
    for (int s = 0; s < 4; s++) {
        if constexpr (sizeof(T) == 4) {
            if (p->fuse_rk4 && !a.extra && !a.pbc) {
                int rc = demag_to_spectrum_t<T>(p, in[s], ms_map, ms_scale);
                if (rc) return rc;
                CUDA_TRY(timed(p, 8, [&] {
                    return launch_x_c2r_rk4(p->g, (const float2*)p->X, (const float2*)p->tw, a, s, in[s], m, acc,
                                            out[s], p->stream);
                }));
                continue;
            }
        }
        int rc = demag_apply_t<T>(p, in[s], ms_map, ms_scale, Hd);
        if (rc) return rc;
        if constexpr (sizeof(T) == 4) {
            if (p->ml) {
                CUDA_TRY(timed(p, 3, [&] {
                    return launch_rk4_stage_ml(a, p->mlt, s, in[s], Hd, m, acc, out[s], p->stream);
                }));
                continue;
            }
        }
        CUDA_TRY(timed(p, 3, [&] { return launch_rk4_stage<T>(a, s, in[s], Hd, m, acc, out[s], p->stream); }));
    }
    if (a.th_s0 > T(0)) CUDA_TRY(timed(p, 4, [&] { return launch_thermal_advance(p->d_step, p->stream); }));
    return BORIS_OK;
}

// One RKF45 trial (six stages of Fehlberg's tableau) from m into mtrial at the
// step size held on the device; the embedded error max goes to d_rkf->err_bits.
template <typename T>
int rkf45_trial_t(boris_plan p, const T* m, LLGArgs<T> a)
{
    a.dt_dev = &p->d_rkf->dt;
    T* ms_map = (T*)a.ms_map;
    T* Hd = (T*)p->Hd;
    T* sa = (T*)p->msa;
    T* sb = (T*)p->msb;
    T* kb = (T*)p->kbuf;
    // stage states alternate m -> sa -> sb -> sa -> sb -> sa -> (trial)
    const T* in[6] = {m, sa, sb, sa, sb, sa};
    T* out[6] = {sa, sb, sa, sb, sa, (T*)p->mtrial};
    for (int s = 0; s < 6; s++) {
        int rc = demag_apply_t<T>(p, in[s], ms_map, a.Ms, Hd);
        if (rc) return rc;
        CUDA_TRY(timed(p, 3, [&] {
            return launch_rkf45_stage<T>(a, s, in[s], Hd, m, kb, out[s], &p->d_rkf->err_bits, p->stream);
        }));
    }
    return BORIS_OK;
}

// The CUDA graph of one RKF45 step: begin (no trial yet) -> WHILE(trial,
// controller) -> accept (m = trial if accepted).  The controller ends the loop
// when a trial is accepted or RKF_MAX_TRIALS were rejected, so one launch of
// the graph never runs more than RKF_MAX_TRIALS trials and needs no host
// decision.
template <typename T>
int rkf45_graph_t(boris_plan p, T* m, const boris_llg_params* prm, const LLGArgs<T>& a)
{
    const bool same = p->rkf_exec && p->rkf_m == (void*)m && p->rkf_terms_version == p->terms_version &&
                      std::memcmp(&p->rkf_prm, prm, sizeof(*prm)) == 0;
    if (same) return BORIS_OK;
    if (p->rkf_exec) {
        cudaGraphExecDestroy(p->rkf_exec);
        p->rkf_exec = nullptr;
    }
    if (!p->gstream) CUDA_TRY(cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaStream_t user = p->stream;
    const bool prof = p->prof;
    const long long before = p->launches;
    p->stream = p->gstream;  // the caller's stream may be the legacy default stream, which cannot be captured
    p->prof = false;
    int rc = BORIS_OK;
    cudaError_t e = cudaSuccess;
    cudaGraphNode_t begin = nullptr, loop = nullptr;
    size_t nn = 0;
    cudaGraphConditionalHandle cond = 0;
    auto capture_into = [&](cudaGraph_t target, const cudaGraphNode_t* dep, size_t ndep, auto&& body) -> cudaError_t {
        cudaError_t ce = cudaStreamBeginCaptureToGraph(p->gstream, target, dep, nullptr, ndep,
                                                       cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) return ce;
        body();
        cudaGraph_t out = nullptr;
        cudaError_t ce2 = cudaStreamEndCapture(p->gstream, &out);
        return ce2;
    };
    // 1. begin
    e = capture_into(g, nullptr, 0, [&] {
        cudaError_t le = launch_rkf45_begin(p->d_rkf, p->gstream);
        if (le != cudaSuccess) rc = fail(BORIS_ERR_CUDA, std::string("rkf45 begin: ") + cudaGetErrorString(le));
    });
    if (e == cudaSuccess && rc == BORIS_OK) e = cudaGraphGetNodes(g, nullptr, &nn);
    if (e == cudaSuccess && rc == BORIS_OK && nn == 1) e = cudaGraphGetNodes(g, &begin, &nn);
    // 2. the trial loop
    if (e == cudaSuccess && rc == BORIS_OK) e = cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault);
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess && rc == BORIS_OK) {
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&loop, g, &begin, nullptr, 1, &np);
        if (e == cudaSuccess) body = np.conditional.phGraph_out[0];
    }
    long long trial_launches = 0;
    if (e == cudaSuccess && rc == BORIS_OK) {
        const long long b0 = p->launches;
        e = capture_into(body, nullptr, 0, [&] {
            rc = rkf45_trial_t<T>(p, m, a);
            if (rc == BORIS_OK) {
                cudaError_t le = launch_rkf45_control(p->d_rkf, prm->tol, prm->dt_min, prm->dt_max, p->d_status, cond,
                                                      p->gstream);
                if (le != cudaSuccess) rc = fail(BORIS_ERR_CUDA, std::string("rkf45 control: ") + cudaGetErrorString(le));
                p->launches++;
            }
        });
        trial_launches = p->launches - b0;
    }
    // 3. accept
    if (e == cudaSuccess && rc == BORIS_OK) {
        e = capture_into(g, &loop, 1, [&] {
            cudaError_t le = launch_rkf45_accept<T>(p->d_rkf, (const T*)p->mtrial, m, 3 * ncell(p), p->gstream);
            if (le != cudaSuccess) rc = fail(BORIS_ERR_CUDA, std::string("rkf45 accept: ") + cudaGetErrorString(le));
        });
    }
    p->stream = user;
    p->prof = prof;
    p->launches = before;
    if (rc == BORIS_OK && e != cudaSuccess) rc = fail(BORIS_ERR_CUDA, std::string("RKF45 step graph: ") + cudaGetErrorString(e));
    if (rc == BORIS_OK) {
        e = cudaGraphInstantiate(&p->rkf_exec, g, 0);
        if (e != cudaSuccess) {
            p->rkf_exec = nullptr;
            rc = fail(BORIS_ERR_CUDA, std::string("RKF45 graph instantiate: ") + cudaGetErrorString(e));
        }
    }
    cudaGraphDestroy(g);
    if (rc != BORIS_OK) {
        cudaGetLastError();
        return rc;
    }
    p->rkf_m = (void*)m;
    p->rkf_prm = *prm;
    p->rkf_terms_version = p->terms_version;
    p->rkf_trial_launches = trial_launches;
    return BORIS_OK;
}

// nsteps accepted RKF45 steps from *dt (device-side control; graph launches
// only), then one copy of the controller state to the host and one
// synchronisation.  *dt receives the controller's next step.
template <typename T>
int rkf45_run_t(boris_plan p, T* m, const boris_llg_params* prm, double* dt, int nsteps, double* t_elapsed)
{
    if (!(*dt > 0) || !std::isfinite(*dt)) return fail(BORIS_ERR_INVALID_ARG, "dt must be > 0");
    if (!(prm->tol > 0) || !(prm->dt_min > 0) || !(prm->dt_max >= prm->dt_min))
        return fail(BORIS_ERR_INVALID_ARG, "RKF45 needs tol > 0 and 0 < dt_min <= dt_max");
    LLGArgs<T> a;
    int rc = check_params<T>(p, prm, &a, 1.0);
    if (rc) return rc;
    if ((rc = rkf45_graph_t<T>(p, m, prm, a))) return rc;
    CUDA_TRY(launch_rkf45_set_dt(p->d_rkf, *dt, true, p->stream));
    for (int i = 0; i < nsteps; i++) CUDA_TRY(cudaGraphLaunch(p->rkf_exec, p->stream));
    CUDA_TRY(cudaMemcpyAsync(p->h_rkf, p->d_rkf, sizeof(RKFControl), cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    const RKFControl& c = *p->h_rkf;
    p->launches += 1 + (long long)nsteps * 2 + (long long)c.trials * p->rkf_trial_launches;
    *dt = c.dt;
    if (t_elapsed) *t_elapsed = c.t;
    if (c.failed_steps > 0)
        return fail(BORIS_ERR_STEP_CONTROL, "RKF45: " + std::to_string(c.failed_steps) + " step(s) rejected " +
                                                std::to_string(RKF_MAX_TRIALS) + " trials in a row");
    return BORIS_OK;
}

template <typename T>
int llg_step_t(boris_plan p, T* m, const boris_llg_params* prm, double* dt)
{
    if (!p || !m || !dt) return fail(BORIS_ERR_INVALID_ARG, "NULL argument");
    if (!aligned16(m)) return fail(BORIS_ERR_INVALID_ARG, "m must be 16-byte aligned");
    if (!prm) return fail(BORIS_ERR_INVALID_ARG, "params is NULL");
    int rc = ensure_llg_workspace<T>(p, prm->method == BORIS_RKF45);
    if (rc) return rc;
    if (prm->method == BORIS_RK4) {
        if (!(*dt > 0) || !std::isfinite(*dt)) return fail(BORIS_ERR_INVALID_ARG, "dt must be > 0");
        LLGArgs<T> a;
        if ((rc = check_params<T>(p, prm, &a, *dt))) return rc;
        return rk4_step_t<T>(p, m, a);
    }
    if (prm->method == BORIS_RKF45) {
        if (p->ml) return fail(BORIS_ERR_INVALID_ARG, "multi-mesh plans step with RK4");
        if (p->has_terms && p->terms.temperature > 0)
            return fail(BORIS_ERR_INVALID_ARG, "the thermal field steps with RK4 (fixed dt)");
        return rkf45_run_t<T>(p, m, prm, dt, 1, nullptr);
    }
    return fail(BORIS_ERR_INVALID_ARG, "unknown method");
}

template <typename T>
int llg_backward_t(boris_plan p, const T* m_in, const boris_llg_params* prm, double dt, const T* g_out, T* g_in,
                   T* g_Ms, T* g_Ku)
{
    if (!p || !m_in || !prm || !g_out || !g_in) return fail(BORIS_ERR_INVALID_ARG, "NULL argument");
    if (!aligned16(m_in) || !aligned16(g_out) || !aligned16(g_in) || (g_Ms && !aligned16(g_Ms)) ||
        (g_Ku && !aligned16(g_Ku)))
        return fail(BORIS_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
    if (prm->method != BORIS_RK4) return fail(BORIS_ERR_INVALID_ARG, "the adjoint is of the RK4 step");
    if (p->ml) return fail(BORIS_ERR_INVALID_ARG, "the adjoint serves single-mesh plans");
    if (p->has_terms) return fail(BORIS_ERR_INVALID_ARG, "the adjoint covers the base field terms; clear the further terms");
    if (p->pbc) return fail(BORIS_ERR_INVALID_ARG, "the adjoint serves non-periodic meshes");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(BORIS_ERR_INVALID_ARG, "dt must be > 0");
    int rc = ensure_llg_workspace<T>(p, false);
    if (rc) return rc;
    LLGArgs<T> a;
    if ((rc = check_params<T>(p, prm, &a, dt))) return rc;
    const size_t n3 = 3 * ncell(p);
    if (!p->bw && (rc = dev_alloc(p, &p->bw, 18 * n3 * sizeof(T)))) return rc;
    T* w = (T*)p->bw;
    T* mst[4] = {(T*)m_in, w, w + n3, w + 2 * n3};
    T* Hs = w + 3 * n3;   // 4 x n3
    T* ks = w + 7 * n3;   // 4 x n3
    T* gk = w + 11 * n3;  // 4 x n3
    T* gH = w + 15 * n3;
    T* DgH = w + 16 * n3;
    T* gml = w + 17 * n3;
    T* Hd = (T*)p->Hd;
    const T* ms_map = (const T*)prm->Ms_map;
    for (int s = 0; s < 4; s++) {
        if ((rc = demag_apply_t<T>(p, mst[s], ms_map, a.Ms, Hd))) return rc;
        CUDA_TRY(timed(p, 3, [&] {
            return launch_fwd_stage<T>(a, s, mst[s], Hd, m_in, Hs + s * n3, ks + s * n3, s < 3 ? mst[s + 1] : nullptr,
                                       p->stream);
        }));
    }
    CUDA_TRY(timed(p, 3, [&] {
        return launch_bwd_start<T>(a, m_in, ks, ks + n3, ks + 2 * n3, ks + 3 * n3, g_out, g_in, gk, p->stream);
    }));
    const T back[4] = {T(0), T(0.5 * dt), T(0.5 * dt), T(dt)};
    for (int s = 3; s >= 0; s--) {
        CUDA_TRY(timed(p, 3, [&] { return launch_bwd_local<T>(a, mst[s], Hs + s * n3, gk + s * n3, gH, gml, p->stream); }));
        if ((rc = demag_apply_t<T>(p, gH, nullptr, T(1), DgH))) return rc;
        CUDA_TRY(timed(p, 3, [&] {
            return launch_bwd_field<T>(a, mst[s], gH, DgH, gml, g_in, s > 0 ? gk + (s - 1) * n3 : nullptr, back[s],
                                       g_Ms, g_Ku, p->stream);
        }));
    }
    return BORIS_OK;
}

// Plan-time autotuner of the fused y-z pass: every candidate schedule that fits
// the geometry runs on the (zeroed) spectral workspace, timed with CUDA events
// on the plan's stream; the fastest is kept.
int autotune_yz(boris_plan p, const YZSchedule* cand, int ncand)
{
    const size_t xbytes = (size_t)p->g.nkx * 3 * p->g.nz * p->g.ny * 2 * (p->f64 ? sizeof(double) : sizeof(float));
    CUDA_TRY(cudaMemsetAsync(p->X, 0, xbytes, p->stream));
    cudaEvent_t a, b;
    CUDA_TRY(cudaEventCreate(&a));
    CUDA_TRY(cudaEventCreate(&b));
    float best = 1e30f;
    int besti = 0;
    for (int i = 0; i < ncand; i++) {
        cudaError_t e = cudaSuccess;
        auto run = [&]() { e = p->f64 ? yz_stage<double>(p, cand[i]) : yz_stage<float>(p, cand[i]); };
        run();
        if (e != cudaSuccess) {
            cudaGetLastError();  // a candidate the device cannot launch is skipped
            continue;
        }
        cudaEventRecord(a, p->stream);
        for (int r = 0; r < 3 && e == cudaSuccess; r++) run();
        cudaEventRecord(b, p->stream);
        if (cudaEventSynchronize(b) != cudaSuccess || e != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) {
            best = ms;
            besti = i;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    p->yz = cand[besti];
    return BORIS_OK;
}

}  // namespace

namespace boris {
// Read-only view of a plan for entry points defined in other files.
bool plan_view(boris_plan p, PlanView* v)
{
    if (!p) return false;
    v->g = p->g;
    v->yz = p->yz;
    v->f64 = p->f64;
    v->stream = p->stream;
    v->device = p->device;
    v->K = p->K;
    v->tw = p->tw;
    v->ml = p->ml;
    v->oersted = p->oersted;
    return true;
}
}  // namespace boris

extern "C" {

const char* boris_last_error(void) { return g_last_error.c_str(); }

static int plan_create(int nx, int ny, int nz, double dx, double dy, double dz, unsigned flags, void* cuda_stream,
                       boris_plan* out, const int* images);

int boris_demag_plan(int nx, int ny, int nz, double dx, double dy, double dz, unsigned flags, void* cuda_stream,
                     boris_plan* out)
{
    return plan_create(nx, ny, nz, dx, dy, dz, flags, cuda_stream, out, nullptr);
}

int boris_demag_plan_pbc(int nx, int ny, int nz, double dx, double dy, double dz, const int images[3], unsigned flags,
                         void* cuda_stream, boris_plan* out)
{
    if (!images) return fail(BORIS_ERR_INVALID_ARG, "images is NULL");
    for (int a = 0; a < 3; a++)
        if (images[a] < 0 || images[a] > 1000) return fail(BORIS_ERR_INVALID_ARG, "images per axis must be 0..1000");
    return plan_create(nx, ny, nz, dx, dy, dz, flags, cuda_stream, out, images);
}

static int plan_create(int nx, int ny, int nz, double dx, double dy, double dz, unsigned flags, void* cuda_stream,
                       boris_plan* out, const int* images)
{
    if (!out) return fail(BORIS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(BORIS_ERR_INVALID_ARG, "mesh sizes must be >= 1");
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dz))
        return fail(BORIS_ERR_INVALID_ARG, "cell sizes must be finite and > 0");
    if (flags & ~(BORIS_FLAG_F64 | BORIS_FLAG_FP16_TC | BORIS_FLAG_BF16_TC)) return fail(BORIS_ERR_INVALID_ARG, "unknown flags");
    const int tc = (flags & BORIS_FLAG_FP16_TC) ? 1 : (flags & BORIS_FLAG_BF16_TC) ? 2 : 0;
    if (tc && (flags & BORIS_FLAG_F64)) return fail(BORIS_ERR_INVALID_ARG, "tensor-core z stage is an FP32-plan option");
    if ((flags & BORIS_FLAG_FP16_TC) && (flags & BORIS_FLAG_BF16_TC))
        return fail(BORIS_ERR_INVALID_ARG, "choose FP16 or BF16 tensor cores, not both");
    Geometry g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.px = padded_len(nx);
    g.py = padded_len(ny);
    g.pz = padded_len(nz);
    if (g.px > 4096 || g.py > 4096 || g.pz > 4096)
        return fail(BORIS_ERR_UNSUPPORTED_SIZE, "padded transform length above 4096");
    g.lgx = ilog2(g.px);
    g.lgy = ilog2(g.py);
    g.lgz = ilog2(g.pz);
    g.nkx = g.px / 2 + 1;
    g.kyh = g.py / 2 + 1;
    g.kzh = g.pz / 2 + 1;
    g.krow = (g.kzh * 6 + 3) / 4 * 4;
    g.lmax = std::max(g.px, std::max(g.py, std::max(g.pz, 32)));
    g.lglmax = ilog2(g.lmax);
    if ((size_t)3 * nx * ny * nz > (size_t)1 << 31) return fail(BORIS_ERR_UNSUPPORTED_SIZE, "mesh too large");

    boris_plan p = new (std::nothrow) boris_plan_s();
    if (!p) return fail(BORIS_ERR_OOM, "host allocation");
    p->g = g;
    p->dx = dx;
    p->dy = dy;
    p->dz = dz;
    p->flags = flags;
    p->f64 = (flags & BORIS_FLAG_F64) != 0;
    p->tc = tc;
    for (int a = 0; a < 3; a++) {
        p->images[a] = images ? images[a] : 0;
        if (p->images[a] > 0) p->pbc |= 1 << a;
    }
    p->stream = (cudaStream_t)cuda_stream;
    int rc = BORIS_OK;
    auto bail = [&](int code) {
        boris_plan_destroy(p);
        return code;
    };
    if (cudaGetDevice(&p->device) != cudaSuccess) return bail(fail(BORIS_ERR_CUDA, "no CUDA device"));
    cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device);
    if ((rc = dev_alloc(p, (void**)&p->d_status, sizeof(int)))) return bail(rc);
    if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return bail(fail(BORIS_ERR_CUDA, "status word"));
    if (const char* tw = std::getenv("BORIS_TEST_WAIT_TIMEOUT"); tw && std::atoi(tw) == 1) {
        // test hook: the first bulk-copy wait of each CTA expects 16 bytes that
        // never arrive and gives up after 2 ms
        p->wait_extra_tx = 16;
        p->wait_limit_ns = 2000000ull;
    }
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    YZSchedule cand[20];
    int ncand = 0;
    if (p->f64) yz_candidates<double>(g, max_smem, cand, &ncand);
    else yz_candidates<float>(g, max_smem, cand, &ncand);
    const bool split_ok = p->f64 ? split_supported<double>(g, max_smem) : split_supported<float>(g, max_smem);
    if (split_ok && ncand < 14) {
        cand[ncand++] = YZSchedule{2, 2, 0, 0, 0};
        if (!p->f64) cand[ncand++] = YZSchedule{2, 3, 0, 0, 0};
        // Qc = 1 / 2 on a split schedule: the bulk-copy pipelined z convolution
        // with one tile stage and 3 CTAs per SM / two stages and 2 CTAs per SM
        for (int v = 1; v <= 2; v++)
            if (!p->f64 && zconv_tma_supported(g, max_smem, v)) cand[ncand++] = YZSchedule{2, v == 1 ? 3 : 2, v, 0, 0};
        // Qc = 3: the residue-split z convolution, register budgets for 4 and 3 CTAs per SM
        if (!p->f64 && zconv_res_supported(g, max_smem)) {
            cand[ncand++] = YZSchedule{2, 4, 3, 0, 0};
            cand[ncand++] = YZSchedule{2, 3, 3, 0, 0};
        }
    }
    if (tc) {
        // the tensor-core z stage runs inside the split schedule only
        if (!split_ok || !zconv_tc_supported(g))
            return bail(fail(BORIS_ERR_UNSUPPORTED_SIZE, "tensor-core z stage needs pz = 64 (17 <= nz <= 32)"));
        cand[0] = YZSchedule{2, 2, 0, 0, 0};
        ncand = 1;
        // tcgen05 form where the tile layout allows it; BORIS_TC_MMASYNC=1 keeps
        // the mma.sync form (for comparisons)
        const char* ms = std::getenv("BORIS_TC_MMASYNC");
        p->tc5 = zconv_tc5_supported(g, max_smem) && !(ms && std::atoi(ms) == 1);
        // tensor-core plans store the padded spectrum in their 16-bit format where
        // the length-1024 x and y passes and the 128-column tiles apply
        // (BORIS_TC_STORE16=0 keeps the FP32 spectrum with the tcgen05 stage of
        // 16-column tiles)
        const char* s16 = std::getenv("BORIS_TC_STORE16");
        p->tc6 = p->tc5 && zconv_tc6_supported(g, max_smem) && y1024_ok<float>(g, max_smem) &&
                 !(s16 && std::atoi(s16) == 0);
    }
    if (ncand == 0) return bail(fail(BORIS_ERR_UNSUPPORTED_SIZE, "y-z plane does not fit the cluster shared memory"));
    // optional override for tests and sweeps: BORIS_YZ_KIND / BORIS_YZ_CLUSTER / BORIS_YZ_THREADS / BORIS_YZ_QC
    {
        const char* sk = std::getenv("BORIS_YZ_KIND");
        const char* sc = std::getenv("BORIS_YZ_CLUSTER");
        const char* st = std::getenv("BORIS_YZ_THREADS");
        const char* sq = std::getenv("BORIS_YZ_QC");
        const char* sp = std::getenv("BORIS_YZ_TMA");
        if (sk || sc || st || sp) {
            int m = 0;
            for (int i = 0; i < ncand; i++) {
                if (sk && cand[i].kind != std::atoi(sk)) continue;
                if (sc && cand[i].C != std::atoi(sc)) continue;
                if (st && cand[i].threads != std::atoi(st)) continue;
                if (sp && (cand[i].kind != 2 || cand[i].Qc != std::atoi(sp))) continue;
                cand[m++] = cand[i];
            }
            if (m == 0) return bail(fail(BORIS_ERR_UNSUPPORTED_SIZE, "no y-z schedule matches the override"));
            ncand = m;
        }
        if (sq) {
            for (int i = 0; i < ncand; i++) {
                if (cand[i].kind != 0) continue;
                const int L = g.py / cand[i].C;
                cand[i].Qc = std::max(1, std::min(L, std::atoi(sq)));
                const size_t cs = p->f64 ? sizeof(double2) : sizeof(float2);
                cand[i].smem = 3 * (size_t)g.nz * L * cs + (g.pz > 1 ? 3 * (size_t)g.pz * cand[i].Qc * cs : 0);
            }
        }
    }
    p->yz = cand[0];
    {
        // BORIS_FUSE_STAGE=1 runs the inverse x transform and the RK4 stage as
        // one kernel (off by default: two CTAs per SM hide less latency than
        // the separate kernels do)
        const char* sf = std::getenv("BORIS_FUSE_STAGE");
        p->fuse_rk4 = !p->f64 && x_c2r_rk4_ok(g, max_smem) && sf && std::atoi(sf) == 1;
    }
    cudaError_t ce = p->f64 ? upload_twiddles_yz_f64() : upload_twiddles_yz_f32();
    if (ce == cudaSuccess) ce = upload_twiddles_split();
    if (ce == cudaSuccess) ce = upload_twiddles_fast();
    if (ce == cudaSuccess) ce = upload_twiddles_res();
    if (ce != cudaSuccess) return bail(fail(BORIS_ERR_CUDA, std::string("twiddle constants: ") + cudaGetErrorString(ce)));
    ce = p->f64 ? yz_set_attributes<double>(p->yz) : yz_set_attributes<float>(p->yz);
    if (ce != cudaSuccess) return bail(fail(BORIS_ERR_CUDA, std::string("yz attributes: ") + cudaGetErrorString(ce)));

    // twiddles
    if ((rc = upload_plan_twiddles(p, g, p->f64))) return bail(rc);
    // kernel spectrum
    const size_t kelems = (size_t)g.nkx * g.kyh * g.krow;
    const size_t esz = p->f64 ? sizeof(double) : sizeof(float);
    if ((rc = dev_alloc(p, &p->K, kelems * esz))) return bail(rc);
    const double rs = 40.0;
    ce = build_kernel_spectrum(g, dx, dy, dz, rs, p->K, p->f64, p->tw64, p->stream, p->images);
    if (ce != cudaSuccess) return bail(fail(BORIS_ERR_CUDA, std::string("kernel spectrum: ") + cudaGetErrorString(ce)));
    // spectral workspace
    const size_t xelems = (size_t)g.nkx * 3 * g.nz * g.ny;
    if ((rc = dev_alloc(p, &p->X, xelems * 2 * esz))) return bail(rc);
    bool want_y = false;
    for (int i = 0; i < ncand; i++) want_y |= cand[i].kind == 2;
    if (want_y) {
        const size_t yelems = (size_t)g.nkx * g.py * 3 * g.nz;
        if (dev_alloc(p, &p->Y, yelems * 2 * esz) != BORIS_OK) {
            // no room for the split schedule: drop it
            cudaGetLastError();
            int m = 0;
            for (int i = 0; i < ncand; i++)
                if (cand[i].kind != 2) cand[m++] = cand[i];
            ncand = m;
            if (ncand == 0) return bail(fail(BORIS_ERR_OOM, "no memory for the y-z workspace"));
            p->yz = cand[0];
        }
    }
    bool want_k2 = false;
    for (int i = 0; i < ncand; i++) want_k2 |= cand[i].kind == 2 && cand[i].Qc == 3;
    want_k2 |= p->tc5;
    if (want_k2) {
        if (dev_alloc(p, &p->K2, zconv_res_k2_bytes(g)) == BORIS_OK) {
            p->k2_bytes = zconv_res_k2_bytes(g);
            if ((ce = zconv_res_build_k2(g, (const float*)p->K, (float2*)p->K2, p->stream)) != cudaSuccess ||
                (ce = p->tc5 ? zconv_tc5_maps(g, (float2*)p->Y, (float2*)p->K2, p->ymap, p->kmap)
                             : zconv_res_kmap(g, (float2*)p->K2, p->kmap)) != cudaSuccess)
                return bail(fail(BORIS_ERR_CUDA, std::string("kernel spectrum copy: ") + cudaGetErrorString(ce)));
            if (p->tc5) p->ymap_ready = true;
        } else {
            // no room for the column-major copy: drop the schedules that read it
            cudaGetLastError();
            p->tc5 = false;
            int m = 0;
            for (int i = 0; i < ncand; i++)
                if (!(cand[i].kind == 2 && cand[i].Qc == 3)) cand[m++] = cand[i];
            ncand = m;
            if (ncand == 0) return bail(fail(BORIS_ERR_OOM, "no memory for the kernel spectrum copy"));
            p->yz = cand[0];
        }
    }
    if (p->tc6) {
        if ((rc = dev_alloc(p, &p->Y16, zconv_tc6_y16_bytes(g)))) return bail(rc);
        if ((rc = dev_alloc(p, &p->K16, zconv_tc6_k16_bytes(g)))) return bail(rc);
        if (p->tc == 1 && (rc = dev_alloc(p, (void**)&p->d_absmax, 16))) return bail(rc);
        if ((ce = zconv_tc6_build_k16(g, (const float*)p->K, p->K16, p->stream)) != cudaSuccess ||
            (ce = zconv_tc6_maps(g, p->Y16, p->K16, p->ymap16, p->kmap16, p->tc == 1)) != cudaSuccess)
            return bail(fail(BORIS_ERR_CUDA, std::string("16-bit spectrum set-up: ") + cudaGetErrorString(ce)));
    }
    if ((ce = cudaStreamSynchronize(p->stream)) != cudaSuccess)
        return bail(fail(BORIS_ERR_CUDA, std::string("plan build: ") + cudaGetErrorString(ce)));
    if (ncand > 1 && (rc = autotune_yz(p, cand, ncand))) return bail(rc);
    if (p->K2 && !(p->yz.kind == 2 && p->yz.Qc == 3) && !p->tc5) {
        cudaFree(p->K2);
        p->K2 = nullptr;
        p->bytes -= p->k2_bytes;
        p->k2_bytes = 0;
    }
    *out = p;
    return BORIS_OK;
}

int boris_oersted_plan(int nx, int ny, int nz, double dx, double dy, double dz, void* cuda_stream, boris_plan* out)
{
    if (!out) return fail(BORIS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(BORIS_ERR_INVALID_ARG, "mesh sizes must be >= 1");
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dz))
        return fail(BORIS_ERR_INVALID_ARG, "cell sizes must be finite and > 0");
    Geometry g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.px = padded_len(nx);
    g.py = padded_len(ny);
    g.pz = padded_len(nz);
    if (g.px > 4096 || g.py > 4096 || g.pz > 4096)
        return fail(BORIS_ERR_UNSUPPORTED_SIZE, "padded transform length above 4096");
    g.lgx = ilog2(g.px);
    g.lgy = ilog2(g.py);
    g.lgz = ilog2(g.pz);
    g.nkx = g.px / 2 + 1;
    g.kyh = g.py / 2 + 1;
    g.kzh = g.pz / 2 + 1;
    g.krow = (g.kzh * 6 + 3) / 4 * 4;
    g.lmax = std::max(g.px, std::max(g.py, std::max(g.pz, 32)));
    g.lglmax = ilog2(g.lmax);
    if ((size_t)3 * nx * ny * nz > (size_t)1 << 31) return fail(BORIS_ERR_UNSUPPORTED_SIZE, "mesh too large");
    boris_plan p = new (std::nothrow) boris_plan_s();
    if (!p) return fail(BORIS_ERR_OOM, "host allocation");
    p->g = g;
    p->dx = dx;
    p->dy = dy;
    p->dz = dz;
    p->oersted = true;
    p->stream = (cudaStream_t)cuda_stream;
    p->yz = YZSchedule{2, 3, 3, 0, 0};
    auto bail = [&](int code) {
        boris_plan_destroy(p);
        return code;
    };
    int rc;
    if (cudaGetDevice(&p->device) != cudaSuccess) return bail(fail(BORIS_ERR_CUDA, "no CUDA device"));
    cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device);
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    if (!split_supported<float>(g, max_smem) || !(g.pz == 1 || zconv_res_curl_supported(g, max_smem)))
        return bail(fail(BORIS_ERR_UNSUPPORTED_SIZE,
                         "Oersted plans need nz = 1 or 3 <= nz <= 32 with ny >= 33 (padded y >= 64)"));
    if ((rc = dev_alloc(p, (void**)&p->d_status, sizeof(int)))) return bail(rc);
    if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return bail(fail(BORIS_ERR_CUDA, "status word"));
    cudaError_t ce = upload_twiddles_split();
    if (ce == cudaSuccess) ce = upload_twiddles_fast();
    if (ce == cudaSuccess) ce = upload_twiddles_res();
    if (ce != cudaSuccess) return bail(fail(BORIS_ERR_CUDA, std::string("twiddle constants: ") + cudaGetErrorString(ce)));
    if ((rc = upload_plan_twiddles(p, g, false))) return bail(rc);
    if ((rc = dev_alloc(p, &p->K, (size_t)g.nkx * g.kyh * g.kzh * 4 * sizeof(float)))) return bail(rc);
    ce = build_oersted_spectrum(g, dx, dy, dz, 40.0, (float*)p->K, p->tw64, p->stream);
    if (ce != cudaSuccess) return bail(fail(BORIS_ERR_CUDA, std::string("Oersted spectrum: ") + cudaGetErrorString(ce)));
    if ((rc = dev_alloc(p, &p->X, (size_t)g.nkx * 3 * g.nz * g.ny * sizeof(float2)))) return bail(rc);
    if ((rc = dev_alloc(p, &p->Y, (size_t)g.nkx * g.py * 3 * g.nz * sizeof(float2)))) return bail(rc);
    if (g.pz > 1) {
        if ((rc = dev_alloc(p, &p->K2, zconv_res_k2_curl_bytes(g)))) return bail(rc);
        p->k2_bytes = zconv_res_k2_curl_bytes(g);
        if ((ce = zconv_res_build_k2_curl(g, (const float*)p->K, (float2*)p->K2, p->stream)) != cudaSuccess ||
            (ce = zconv_res_kmap_curl(g, (float2*)p->K2, p->kmap)) != cudaSuccess ||
            (ce = zconv_tma_map(g, (float2*)p->Y, p->ymap)) != cudaSuccess)
            return bail(fail(BORIS_ERR_CUDA, std::string("Oersted spectrum copy: ") + cudaGetErrorString(ce)));
        p->ymap_ready = true;
    }
    if ((ce = cudaStreamSynchronize(p->stream)) != cudaSuccess)
        return bail(fail(BORIS_ERR_CUDA, std::string("plan build: ") + cudaGetErrorString(ce)));
    *out = p;
    return BORIS_OK;
}

int boris_oersted_apply(boris_plan p, const float* J, float* H)
{
    if (!p || !J || !H) return fail(BORIS_ERR_INVALID_ARG, "NULL argument");
    if (!p->oersted) return fail(BORIS_ERR_INVALID_ARG, "not an Oersted plan (boris_oersted_plan)");
    if (!aligned16(J) || !aligned16(H)) return fail(BORIS_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
    if ((const void*)J == (const void*)H) return fail(BORIS_ERR_INVALID_ARG, "J and H may not alias");
    const Geometry& g = p->g;
    float2* X = (float2*)p->X;
    float2* Y = (float2*)p->Y;
    const float2* tw = (const float2*)p->tw;
    CUDA_TRY(timed(p, 0, [&] { return launch_x_r2c<float>(g, J, nullptr, 1.0f, X, tw, p->stream); }));
    CUDA_TRY(timed(p, 5, [&] { return launch_split<float>(g, X, Y, nullptr, tw, p->stream, 0, 2); }));
    CUDA_TRY(timed(p, 6, [&] {
        if (g.pz == 1) return launch_curl_point(g, Y, (const float*)p->K, p->stream);
        return launch_zconv_res_curl(p->ymap, p->kmap, g, Y, p->d_status, p->wait_limit_ns, p->nsm, p->stream);
    }));
    CUDA_TRY(timed(p, 7, [&] { return launch_split<float>(g, X, Y, nullptr, tw, p->stream, 2, 2); }));
    CUDA_TRY(timed(p, 2, [&] {
        return launch_x_c2r<float>(g, X, H, tw, p->stream, p->d_status, p->wait_limit_ns);
    }));
    return BORIS_OK;
}

int boris_multimesh_plan(int n_layers, const int* nxyz, const double* hxyz, const double* origin, unsigned flags,
                         void* cuda_stream, boris_plan* out)
{
    if (!out) return fail(BORIS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_layers < 1 || n_layers > ML_MAX_LAYERS || !nxyz || !hxyz || !origin)
        return fail(BORIS_ERR_INVALID_ARG, "need 1..16 layers and their sizes, cells and origins");
    if (flags != BORIS_FLAG_F32) return fail(BORIS_ERR_INVALID_ARG, "multi-mesh plans are FP32");
    const double hx = hxyz[0], hy = hxyz[1];
    double x0 = origin[0], y0 = origin[1];
    int Z = 0;
    for (int l = 0; l < n_layers; l++) {
        if (nxyz[3 * l] < 1 || nxyz[3 * l + 1] < 1 || nxyz[3 * l + 2] < 1)
            return fail(BORIS_ERR_INVALID_ARG, "layer sizes must be >= 1");
        if (!(hxyz[3 * l + 2] > 0) || std::fabs(hxyz[3 * l] - hx) > 1e-9 * hx || std::fabs(hxyz[3 * l + 1] - hy) > 1e-9 * hy)
            return fail(BORIS_ERR_INVALID_ARG, "all layers must share the in-plane cell size (hx, hy)");
        x0 = std::min(x0, origin[3 * l]);
        y0 = std::min(y0, origin[3 * l + 1]);
        Z += nxyz[3 * l + 2];
    }
    if (!(hx > 0) || !(hy > 0)) return fail(BORIS_ERR_INVALID_ARG, "cell sizes must be > 0");
    if (Z > ML_MAX_PLANES) return fail(BORIS_ERR_UNSUPPORTED_SIZE, "more than 256 z planes in the stack");
    MLTable t = {};
    t.nl = n_layers;
    t.Z = Z;
    std::vector<double> zc(Z), hzp(Z);
    size_t off = 0;
    int p0 = 0;
    for (int l = 0; l < n_layers; l++) {
        const double fx = (origin[3 * l] - x0) / hx, fy = (origin[3 * l + 1] - y0) / hy;
        const int ox = (int)std::lround(fx), oy = (int)std::lround(fy);
        if (std::fabs(fx - ox) > 1e-6 || std::fabs(fy - oy) > 1e-6)
            return fail(BORIS_ERR_INVALID_ARG, "in-plane layer offsets must be whole cells");
        t.nx[l] = nxyz[3 * l];
        t.ny[l] = nxyz[3 * l + 1];
        t.nz[l] = nxyz[3 * l + 2];
        t.ox[l] = ox;
        t.oy[l] = oy;
        t.hz[l] = (float)hxyz[3 * l + 2];
        t.plane0[l] = p0;
        t.off[l] = off;
        off += 3 * (size_t)t.nx[l] * t.ny[l] * t.nz[l];
        t.NX = std::max(t.NX, ox + t.nx[l]);
        t.NY = std::max(t.NY, oy + t.ny[l]);
        for (int q = 0; q < t.nz[l]; q++) {
            zc[p0 + q] = origin[3 * l + 2] + (q + 0.5) * hxyz[3 * l + 2];
            hzp[p0 + q] = hxyz[3 * l + 2];
            t.plane_layer[p0 + q] = (unsigned char)l;
        }
        p0 += t.nz[l];
    }
    t.off[n_layers] = off;
    t.total3 = off;
    // unique inter-plane spectra: a N_ab keyed by (min(a, b), max(a, b), |dz|)
    // (a N_ab = b N_ba: the stencil of two boxes is symmetric in a and b)
    MLHost h;
    h.hx = hx;
    h.hy = hy;
    h.pairs.resize((size_t)Z * Z);
    std::map<std::tuple<long long, long long, long long>, int> uniq;
    const double qz = 1e-6 * *std::min_element(hzp.begin(), hzp.end());
    for (int pp = 0; pp < Z; pp++)
        for (int q = 0; q < Z; q++) {
            const double dz = zc[pp] - zc[q];
            const double lo = std::min(hzp[pp], hzp[q]), hi = std::max(hzp[pp], hzp[q]);
            auto key = std::make_tuple(std::llround(lo / qz), std::llround(hi / qz), std::llround(std::fabs(dz) / qz));
            auto it = uniq.find(key);
            int u;
            if (it == uniq.end()) {
                u = (int)h.ua.size();
                uniq[key] = u;
                h.ua.push_back(lo);
                h.ub.push_back(hi);
                h.udz.push_back(std::fabs(dz));
            } else {
                u = it->second;
            }
            h.pairs[(size_t)pp * Z + q] = u | (dz < 0 ? (1 << 30) : 0);
        }
    Geometry g;
    g.nx = t.NX;
    g.ny = t.NY;
    g.nz = Z;
    g.px = padded_len(t.NX);
    g.py = padded_len(t.NY);
    g.pz = 1;
    if (g.px > 4096 || g.py > 4096) return fail(BORIS_ERR_UNSUPPORTED_SIZE, "padded transform length above 4096");
    g.lgx = ilog2(g.px);
    g.lgy = ilog2(g.py);
    g.lgz = 0;
    g.nkx = g.px / 2 + 1;
    g.kyh = g.py / 2 + 1;
    g.kzh = 1;
    g.krow = 8;
    g.lmax = std::max(g.px, std::max(g.py, 64));
    g.lglmax = ilog2(g.lmax);

    boris_plan p = new (std::nothrow) boris_plan_s();
    if (!p) return fail(BORIS_ERR_OOM, "host allocation");
    auto bail = [&](int code) {
        boris_plan_destroy(p);
        return code;
    };
    p->g = g;
    p->dx = hx;
    p->dy = hy;
    p->dz = hxyz[2];
    p->flags = flags;
    p->stream = (cudaStream_t)cuda_stream;
    p->ml = true;
    p->mlt = t;
    for (int l = 0; l < n_layers; l++) p->ml_zb[l] = origin[3 * l + 2];
    p->ml_unique = (int)h.ua.size();
    p->yz = YZSchedule{2, 2, 0, 0, 0};
    int rc;
    if (cudaGetDevice(&p->device) != cudaSuccess) return bail(fail(BORIS_ERR_CUDA, "no CUDA device"));
    cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device);
    if ((rc = dev_alloc(p, (void**)&p->d_status, sizeof(int)))) return bail(rc);
    if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return bail(fail(BORIS_ERR_CUDA, "status word"));
    if (const char* tw = std::getenv("BORIS_TEST_WAIT_TIMEOUT"); tw && std::atoi(tw) == 1) {
        // test hook: the first bulk-copy wait of each CTA expects 16 bytes that
        // never arrive and gives up after 2 ms
        p->wait_extra_tx = 16;
        p->wait_limit_ns = 2000000ull;
    }
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    if (!split_supported<float>(g, max_smem)) return bail(fail(BORIS_ERR_UNSUPPORTED_SIZE, "frame too large"));
    cudaError_t ce = upload_twiddles_split();
    if (ce == cudaSuccess) ce = upload_twiddles_fast();
    if (ce == cudaSuccess) ce = upload_twiddles_res();
    if (ce != cudaSuccess) return bail(fail(BORIS_ERR_CUDA, "twiddle constants"));
    if ((rc = upload_plan_twiddles(p, g, false))) return bail(rc);
    const size_t kbytes = (size_t)p->ml_unique * g.nkx * 6 * ml_kyp(g) * sizeof(float);
    if ((rc = dev_alloc(p, &p->Kml, kbytes))) return bail(rc);
    if ((rc = dev_alloc(p, (void**)&p->d_pairs, h.pairs.size() * sizeof(int)))) return bail(rc);
    cudaMemcpy(p->d_pairs, h.pairs.data(), h.pairs.size() * sizeof(int), cudaMemcpyHostToDevice);
    ce = ml_build_spectra(h, g, (float*)p->Kml, p->tw64, p->stream);
    if (ce != cudaSuccess) return bail(fail(BORIS_ERR_CUDA, std::string("inter-mesh spectra: ") + cudaGetErrorString(ce)));
    const size_t frame = 3 * (size_t)Z * t.NY * t.NX;
    if ((rc = dev_alloc(p, (void**)&p->Mf, frame * sizeof(float)))) return bail(rc);
    if ((rc = dev_alloc(p, (void**)&p->Hf, frame * sizeof(float)))) return bail(rc);
    if ((rc = dev_alloc(p, &p->X, (size_t)g.nkx * 3 * Z * g.ny * sizeof(float2)))) return bail(rc);
    if ((rc = dev_alloc(p, &p->Y, (size_t)g.nkx * g.py * 3 * Z * sizeof(float2)))) return bail(rc);
    // the persistent inter-plane sum reads 32-bit row offsets (128-byte units)
    {
        const size_t ustride32 = (size_t)g.nkx * 6 * ml_kyp(g) / 32;
        const bool fits = (size_t)p->ml_unique * ustride32 < ((size_t)1 << 31);
        std::vector<unsigned> pcode((size_t)Z * Z);
        std::vector<float> invhz(Z);
        for (size_t i = 0; i < pcode.size(); i++) {
            const int code = h.pairs[i];
            pcode[i] = (unsigned)((size_t)(code & 0x3fffffff) * ustride32) | ((code >> 30) & 1 ? 0x80000000u : 0u);
        }
        for (int i = 0; i < Z; i++) invhz[i] = (float)(1.0 / hzp[i]);
        if ((rc = dev_alloc(p, (void**)&p->d_pcode, pcode.size() * sizeof(unsigned)))) return bail(rc);
        if ((rc = dev_alloc(p, (void**)&p->d_invhz, invhz.size() * sizeof(float)))) return bail(rc);
        cudaMemcpy(p->d_pcode, pcode.data(), pcode.size() * sizeof(unsigned), cudaMemcpyHostToDevice);
        cudaMemcpy(p->d_invhz, invhz.data(), invhz.size() * sizeof(float), cudaMemcpyHostToDevice);
        if ((ce = cudaStreamSynchronize(p->stream)) != cudaSuccess)
            return bail(fail(BORIS_ERR_CUDA, std::string("plan build: ") + cudaGetErrorString(ce)));
        // multi-mesh autotuner: time each inter-plane sum kernel that fits on the
        // (zeroed) padded spectrum and keep the fastest; BORIS_ML_MIX forces one
        std::vector<int> vars = {0, 1};
        if (fits && ml_mix_v2_smem(Z) <= (size_t)max_smem) {
            vars.push_back(2);
            if (2 * (ml_mix_v2_smem(Z) + 1024) <= 233472) vars.push_back(3);
        }
        const size_t staged = (size_t)Z * 2 * 6 * 32 * 4 + (size_t)Z * 3 * 64 * 8 + (size_t)Z * Z * 4;
        if (staged > (size_t)max_smem) vars.erase(std::remove(vars.begin(), vars.end(), 1), vars.end());
        if (const char* sv = std::getenv("BORIS_ML_MIX")) {
            const int want = std::atoi(sv);
            if (std::find(vars.begin(), vars.end(), want) == vars.end())
                return bail(fail(BORIS_ERR_UNSUPPORTED_SIZE, "the requested inter-plane sum kernel does not fit"));
            vars = {want};
        }
        CUDA_TRY(cudaMemsetAsync(p->Y, 0, (size_t)g.nkx * g.py * 3 * Z * sizeof(float2), p->stream));
        cudaEvent_t a, b;
        CUDA_TRY(cudaEventCreate(&a));
        CUDA_TRY(cudaEventCreate(&b));
        float best = 1e30f;
        p->ml_variant = vars[0];
        for (int v : vars) {
            if (vars.size() == 1) break;
            cudaError_t e = ml_mix(g, Z, (float2*)p->Y, (const float*)p->Kml, p->d_pairs, p->d_pcode, p->d_invhz, v,
                                   p->nsm, p->stream);
            if (e != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cudaEventRecord(a, p->stream);
            for (int r = 0; r < 3 && e == cudaSuccess; r++)
                e = ml_mix(g, Z, (float2*)p->Y, (const float*)p->Kml, p->d_pairs, p->d_pcode, p->d_invhz, v, p->nsm,
                           p->stream);
            cudaEventRecord(b, p->stream);
            if (cudaEventSynchronize(b) != cudaSuccess || e != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (ms < best) {
                best = ms;
                p->ml_variant = v;
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        p->yz.Qc = p->ml_variant;
    }
    if ((ce = cudaStreamSynchronize(p->stream)) != cudaSuccess)
        return bail(fail(BORIS_ERR_CUDA, std::string("plan build: ") + cudaGetErrorString(ce)));
    *out = p;
    return BORIS_OK;
}

int boris_plan_multimesh_info(boris_plan p, int out[4])
{
    if (!p || !out) return fail(BORIS_ERR_INVALID_ARG, "NULL argument");
    if (!p->ml) return fail(BORIS_ERR_INVALID_ARG, "not a multi-mesh plan");
    out[0] = p->mlt.Z;
    out[1] = p->ml_unique;
    out[2] = p->mlt.NX;
    out[3] = p->mlt.NY;
    return BORIS_OK;
}

int boris_demag_apply(boris_plan p, const float* M, float* Hd)
{
    if (!p || !M || !Hd) return fail(BORIS_ERR_INVALID_ARG, "NULL argument");
    if (p->f64) return fail(BORIS_ERR_INVALID_ARG, "FP64 plan: use boris_demag_apply_f64");
    if (!aligned16(M) || !aligned16(Hd)) return fail(BORIS_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
    if ((const void*)M == (const void*)Hd) return fail(BORIS_ERR_INVALID_ARG, "M and Hd may not alias");
    return demag_apply_t<float>(p, M, nullptr, 1.0f, Hd);
}

int boris_demag_apply_f64(boris_plan p, const double* M, double* Hd)
{
    if (!p || !M || !Hd) return fail(BORIS_ERR_INVALID_ARG, "NULL argument");
    if (!p->f64) return fail(BORIS_ERR_INVALID_ARG, "FP32 plan: use boris_demag_apply");
    if (!aligned16(M) || !aligned16(Hd)) return fail(BORIS_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
    if ((const void*)M == (const void*)Hd) return fail(BORIS_ERR_INVALID_ARG, "M and Hd may not alias");
    return demag_apply_t<double>(p, M, nullptr, 1.0, Hd);
}

int boris_demag_adjoint(boris_plan p, const float* gHd, float* gM)
{
    // the operator M -> -N * M is symmetric: its adjoint is itself
    return boris_demag_apply(p, gHd, gM);
}

int boris_llg_step(boris_plan p, float* m, const boris_llg_params* prm, double* dt)
{
    if (p && p->f64) return fail(BORIS_ERR_INVALID_ARG, "FP64 plan: use boris_llg_step_f64");
    return llg_step_t<float>(p, m, prm, dt);
}

int boris_llg_step_f64(boris_plan p, double* m, const boris_llg_params* prm, double* dt)
{
    if (p && !p->f64) return fail(BORIS_ERR_INVALID_ARG, "FP32 plan: use boris_llg_step");
    return llg_step_t<double>(p, m, prm, dt);
}

int boris_llg_step_backward(boris_plan p, const float* m_in, const boris_llg_params* prm, double dt,
                            const float* g_m_out, float* g_m_in, float* g_Ms, float* g_Ku)
{
    if (p && p->f64) return fail(BORIS_ERR_INVALID_ARG, "FP64 plan: use boris_llg_step_backward_f64");
    return llg_backward_t<float>(p, m_in, prm, dt, g_m_out, g_m_in, g_Ms, g_Ku);
}

int boris_llg_step_backward_f64(boris_plan p, const double* m_in, const boris_llg_params* prm, double dt,
                                const double* g_m_out, double* g_m_in, double* g_Ms, double* g_Ku)
{
    if (p && !p->f64) return fail(BORIS_ERR_INVALID_ARG, "FP32 plan: use boris_llg_step_backward");
    return llg_backward_t<double>(p, m_in, prm, dt, g_m_out, g_m_in, g_Ms, g_Ku);
}

int boris_llg_run_graph(boris_plan p, float* m, const boris_llg_params* prm, double dt, int nsteps)
{
    if (!p || !m || !prm) return fail(BORIS_ERR_INVALID_ARG, "NULL argument");
    if (p->f64) return fail(BORIS_ERR_INVALID_ARG, "FP64 plan");
    if (prm->method != BORIS_RK4 || nsteps < 0 || !(dt > 0)) return fail(BORIS_ERR_INVALID_ARG, "RK4, nsteps >= 0, dt > 0");
    if (!aligned16(m)) return fail(BORIS_ERR_INVALID_ARG, "m must be 16-byte aligned");
    int rc = ensure_llg_workspace<float>(p, false);
    if (rc) return rc;
    const bool same = p->gexec && p->g_m == m && p->g_dt == dt && p->g_terms_version == p->terms_version &&
                      std::memcmp(&p->g_prm, prm, sizeof(*prm)) == 0;
    if (!same) {
        if (p->gexec) {
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
        if (!p->gstream) CUDA_TRY(cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking));
        LLGArgs<float> a;
        if ((rc = check_params<float>(p, prm, &a, dt))) return rc;
        // capture one step on the plan's private stream (the caller's stream may
        // be the legacy default stream, which cannot be captured)
        CUDA_TRY(cudaStreamSynchronize(p->stream));
        cudaStream_t user = p->stream;
        const bool prof = p->prof;
        p->stream = p->gstream;
        p->prof = false;
        cudaGraph_t graph = nullptr;
        const long long before = p->launches;
        cudaError_t e = cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = rk4_step_t<float>(p, m, a);
            p->g_launches = p->launches - before;
            p->launches = before;
            cudaError_t e2 = cudaStreamEndCapture(p->gstream, &graph);
            if (rc == BORIS_OK && e2 != cudaSuccess) {
                rc = fail(BORIS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e2));
            }
        } else {
            rc = fail(BORIS_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
        }
        p->stream = user;
        p->prof = prof;
        if (rc != BORIS_OK) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return rc;
        }
        e = cudaGraphInstantiate(&p->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            p->gexec = nullptr;
            return fail(BORIS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        p->g_m = m;
        p->g_dt = dt;
        p->g_prm = *prm;
        p->g_terms_version = p->terms_version;
    }
    for (int i = 0; i < nsteps; i++) {
        CUDA_TRY(cudaGraphLaunch(p->gexec, p->stream));
        p->launches += p->g_launches;
    }
    return BORIS_OK;
}

int boris_llg_run_rkf45(boris_plan p, float* m, const boris_llg_params* prm, double* dt, int nsteps, double* t_elapsed)
{
    if (!p || !m || !prm || !dt) return fail(BORIS_ERR_INVALID_ARG, "NULL argument");
    if (p->f64) return fail(BORIS_ERR_INVALID_ARG, "FP64 plan: use boris_llg_step_f64");
    if (p->oersted) return fail(BORIS_ERR_INVALID_ARG, "an Oersted plan serves boris_oersted_apply only");
    if (prm->method != BORIS_RKF45 || nsteps < 0) return fail(BORIS_ERR_INVALID_ARG, "RKF45 with nsteps >= 0");
    if (p->ml) return fail(BORIS_ERR_INVALID_ARG, "multi-mesh plans step with RK4");
    if (p->has_terms && p->terms.temperature > 0)
        return fail(BORIS_ERR_INVALID_ARG, "the thermal field steps with RK4 (fixed dt)");
    if (!aligned16(m)) return fail(BORIS_ERR_INVALID_ARG, "m must be 16-byte aligned");
    int rc = ensure_llg_workspace<float>(p, true);
    if (rc) return rc;
    return rkf45_run_t<float>(p, m, prm, dt, nsteps, t_elapsed);
}

int boris_llg_run_host(boris_plan p, float* m_host, const boris_llg_params* prm, double dt, int nsteps)
{
    if (!p || !m_host || !prm) return fail(BORIS_ERR_INVALID_ARG, "NULL argument");
    if (p->f64) return fail(BORIS_ERR_INVALID_ARG, "FP64 plan");
    if (nsteps < 0 || prm->method != BORIS_RK4 || !(dt > 0))
        return fail(BORIS_ERR_INVALID_ARG, "RK4 with nsteps >= 0 and dt > 0 only");
    const size_t vb = 3 * ncell(p) * sizeof(float);
    int rc;
    if (!p->m_dev_e2e && (rc = dev_alloc(p, &p->m_dev_e2e, vb))) return rc;
    CUDA_TRY(cudaMemcpyAsync(p->m_dev_e2e, m_host, vb, cudaMemcpyHostToDevice, p->stream));
    // the steps replay the plan's CUDA graph captured for the device copy
    if (nsteps > 0 && (rc = boris_llg_run_graph(p, (float*)p->m_dev_e2e, prm, dt, nsteps))) return rc;
    CUDA_TRY(cudaMemcpyAsync(m_host, p->m_dev_e2e, vb, cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    return BORIS_OK;
}

static int energy_impl(boris_plan p, const float* m, const boris_llg_params* prm, double* out, int nout)
{
    if (!p || !m || !prm || !out) return fail(BORIS_ERR_INVALID_ARG, "NULL argument");
    if (p->f64) return fail(BORIS_ERR_INVALID_ARG, "FP64 plan");
    if (p->ml) return fail(BORIS_ERR_INVALID_ARG, "energies of multi-mesh plans are not provided");
    int rc = ensure_llg_workspace<float>(p, false);
    if (rc) return rc;
    LLGArgs<float> a;
    if ((rc = check_params<float>(p, prm, &a, 0.0))) return rc;
    if (!p->energy && (rc = dev_alloc(p, (void**)&p->energy, 8 * sizeof(double)))) return rc;
    if ((rc = demag_apply_t<float>(p, m, (const float*)prm->Ms_map, (float)prm->Ms, (float*)p->Hd))) return rc;
    CUDA_TRY(cudaMemsetAsync(p->energy, 0, 5 * sizeof(double), p->stream));
    CUDA_TRY(timed(p, 4, [&] { return launch_energy<float>(a, m, (const float*)p->Hd, p->energy, p->stream); }));
    double tmp[5];
    CUDA_TRY(cudaMemcpyAsync(tmp, p->energy, 5 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    for (int i = 0; i < nout; i++) out[i] = tmp[i];
    return BORIS_OK;
}

int boris_energy(boris_plan p, const float* m, const boris_llg_params* prm, double out[4])
{
    return energy_impl(p, m, prm, out, 4);
}

int boris_energy_terms(boris_plan p, const float* m, const boris_llg_params* prm, double out[5])
{
    return energy_impl(p, m, prm, out, 5);
}

int boris_thermal_set_step(boris_plan p, unsigned long long step)
{
    if (!p) return fail(BORIS_ERR_INVALID_ARG, "NULL plan");
    if (!p->d_step) {
        int rc = dev_alloc(p, (void**)&p->d_step, sizeof(unsigned long long));
        if (rc) return rc;
    }
    CUDA_TRY(launch_thermal_set(p->d_step, step, p->stream));
    return BORIS_OK;
}

int boris_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n, void* cuda_stream)
{
    if (n < 0 || (n > 0 && (!ctr || !key || !out)))
        return fail(BORIS_ERR_INVALID_ARG, "need n >= 0 and device ctr, key, out");
    CUDA_TRY(launch_philox_words(ctr, key, out, n, (cudaStream_t)cuda_stream));
    return BORIS_OK;
}

int boris_set_field_terms(boris_plan p, const boris_field_terms* t)
{
    if (!p) return fail(BORIS_ERR_INVALID_ARG, "NULL plan");
    p->terms_version++;
    if (!t) {
        p->terms = boris_field_terms{};
        p->has_terms = false;
        return BORIS_OK;
    }
    boris_field_terms v = *t;
    const double vals[] = {v.K2, v.Kc1, v.Kc2, v.D, v.J1, v.J2, v.cubic_e1[0], v.cubic_e1[1], v.cubic_e1[2],
                           v.cubic_e2[0], v.cubic_e2[1], v.cubic_e2[2], v.temperature};
    for (double x : vals)
        if (!std::isfinite(x)) return fail(BORIS_ERR_INVALID_ARG, "field terms must be finite");
    if (v.dmi < BORIS_DMI_NONE || v.dmi > BORIS_DMI_INTERFACIAL) return fail(BORIS_ERR_INVALID_ARG, "unknown DMI kind");
    if (v.dmi == BORIS_DMI_NONE) v.D = 0.0;
    if (v.dmi != BORIS_DMI_NONE && p->ml) return fail(BORIS_ERR_INVALID_ARG, "DMI serves single-mesh plans");
    if (v.temperature < 0) return fail(BORIS_ERR_INVALID_ARG, "temperature must be >= 0");
    if (v.H_add && (p->ml || ((uintptr_t)v.H_add & 15u)))
        return fail(BORIS_ERR_INVALID_ARG, "H_add serves single-mesh plans and must be 16-byte aligned");
    if (v.temperature > 0 && p->ml) return fail(BORIS_ERR_INVALID_ARG, "the thermal field serves single-mesh plans");
    if (v.temperature > 0 && (size_t)ncell(p) >= ((size_t)1 << 32))
        return fail(BORIS_ERR_UNSUPPORTED_SIZE, "thermal field: more than 2^32 cells");
    if (v.temperature > 0 && !p->d_step) {
        int rc = dev_alloc(p, (void**)&p->d_step, sizeof(unsigned long long));
        if (rc) return rc;
        CUDA_TRY(cudaMemsetAsync(p->d_step, 0, sizeof(unsigned long long), p->stream));
    }
    if ((v.J1 != 0.0 || v.J2 != 0.0) && !p->ml)
        return fail(BORIS_ERR_INVALID_ARG, "surface exchange couples the layers of a multi-mesh plan");
    if (v.J1 != 0.0 || v.J2 != 0.0) {
        for (int l = 0; l + 1 < p->mlt.nl; l++)
            if (p->ml_zb[l + 1] < p->ml_zb[l] + p->mlt.nz[l] * (double)p->mlt.hz[l] * (1.0 - 1e-9))
                return fail(BORIS_ERR_INVALID_ARG, "surface exchange needs the layers listed bottom-up");
    }
    if (v.Kc1 != 0.0 || v.Kc2 != 0.0) {
        double n1 = 0, n2 = 0, d = 0;
        for (int c = 0; c < 3; c++) {
            n1 += v.cubic_e1[c] * v.cubic_e1[c];
            n2 += v.cubic_e2[c] * v.cubic_e2[c];
        }
        if (!(n1 > 0) || !(n2 > 0)) return fail(BORIS_ERR_INVALID_ARG, "cubic axes must be nonzero");
        for (int c = 0; c < 3; c++) {
            v.cubic_e1[c] /= std::sqrt(n1);
            v.cubic_e2[c] /= std::sqrt(n2);
            d += v.cubic_e1[c] * v.cubic_e2[c];
        }
        if (std::fabs(d) > 1e-6) return fail(BORIS_ERR_INVALID_ARG, "cubic axes must be orthogonal");
    }
    p->terms = v;
    p->has_terms = v.K2 != 0.0 || v.Kc1 != 0.0 || v.Kc2 != 0.0 || (v.dmi != BORIS_DMI_NONE && v.D != 0.0) ||
                   v.J1 != 0.0 || v.J2 != 0.0 || v.temperature > 0.0 || v.H_add != nullptr;
    if (!p->has_terms) p->terms = boris_field_terms{};
    return BORIS_OK;
}

int boris_sync_status(boris_plan p)
{
    if (!p) return fail(BORIS_ERR_INVALID_ARG, "NULL plan");
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail(BORIS_ERR_CUDA, cudaGetErrorString(e));
    int st = BORIS_OK;
    if (p->d_status) {
        if (cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess)
            return fail(BORIS_ERR_CUDA, "status word");
    }
    if (st == BORIS_ERR_TIMEOUT) return fail(BORIS_ERR_TIMEOUT, "a bounded device-side wait gave up");
    return st;
}

int boris_plan_schedule(boris_plan p, int out[4])
{
    if (!p || !out) return fail(BORIS_ERR_INVALID_ARG, "NULL argument");
    out[0] = p->yz.kind;
    out[1] = p->yz.C;
    out[2] = p->yz.kind == 2 ? (p->tc ? (p->tc6 ? 6 : p->tc5 ? 5 : 4) : p->yz.Qc) : p->yz.threads;
    out[3] = (int)p->yz.smem;
    return BORIS_OK;
}

int boris_plan_padded(boris_plan p, int out[3])
{
    if (!p || !out) return fail(BORIS_ERR_INVALID_ARG, "NULL argument");
    out[0] = p->g.px;
    out[1] = p->g.py;
    out[2] = p->g.pz;
    return BORIS_OK;
}

size_t boris_plan_device_bytes(boris_plan p) { return p ? p->bytes : 0; }

int boris_profile_enable(boris_plan p, int on)
{
    if (!p) return fail(BORIS_ERR_INVALID_ARG, "NULL plan");
    p->prof = on != 0;
    return BORIS_OK;
}

int boris_profile_read(boris_plan p, double ms_out[9], long long launches_out[9], long long* total_launches)
{
    if (!p || !ms_out || !launches_out) return fail(BORIS_ERR_INVALID_ARG, "NULL argument");
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    for (int k = 0; k < NPROF; k++) {
        ms_out[k] = 0.0;
        launches_out[k] = 0;
    }
    for (auto& u : p->ev_used) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, u.second.first, u.second.second) == cudaSuccess && u.first >= 0 &&
            u.first < NPROF) {
            ms_out[u.first] += ms;
            launches_out[u.first]++;
        }
        p->ev_pool.push_back(u.second.first);
        p->ev_pool.push_back(u.second.second);
    }
    p->ev_used.clear();
    if (total_launches) *total_launches = p->launches;
    p->launches = 0;
    return BORIS_OK;
}

void boris_plan_destroy(boris_plan p)
{
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    void* ptrs[] = {p->d_absmax, p->Y16, p->K16, p->Kml, p->d_pairs, p->d_pcode, p->d_invhz, p->Mf, p->Hf, p->K, p->K2, p->d_step, p->X, p->Y, p->Hd, p->msa, p->msb, p->acc, p->kbuf, p->mtrial, p->d_rkf, p->energy,
                    p->m_dev_e2e, p->bw};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (p->tw && p->tw != (void*)p->tw64) cudaFree(p->tw);
    if (p->tw64) cudaFree(p->tw64);
    if (p->h_rkf) cudaFreeHost(p->h_rkf);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->rkf_exec) cudaGraphExecDestroy(p->rkf_exec);
    if (p->gstream) cudaStreamDestroy(p->gstream);
    for (auto& u : p->ev_used) {
        cudaEventDestroy(u.second.first);
        cudaEventDestroy(u.second.second);
    }
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    delete p;
}

}  // extern "C"
