/*
 * boris.h - C ABI of the GB300 finite-difference micromagnetics hot path.
 *
 * Method: "Boris Computational Spintronics" (arXiv 2008.02478).
 *   - Demagnetising field (Table 1, "Demagnetizing Field"; Eq. 4 for one mesh):
 *       H(r0) = -sum_r N(r - r0) M(r),
 *     N the cell-averaged Newell tensor (Ref. [50] of the paper), evaluated by
 *     the convolution theorem on a zero-padded grid (Section 7): forward FFT
 *     of M, point-by-point multiply with the transformed tensor, inverse FFT.
 *   - LLG equation (Eq. 1) with exchange, uniaxial anisotropy (Table 1),
 *     applied and demagnetising fields; RK4 and RKF45 steps (Section 2).
 *
 * Conventions for every call:
 *   - Fields are SoA arrays [3][nz][ny][nx] (x fastest): component c of cell
 *     (i,j,k) at index c*nx*ny*nz + (k*ny + j)*nx + i.  Scalar maps are
 *     [nz][ny][nx].  Units: A/m for M and H, J/m^3 for Ku, J/m for A, m, s.
 *   - Unless a name ends in _host, pointers are DEVICE pointers on the plan's
 *     device; they must be 16-byte aligned.  The caller owns them; the
 *     library never frees or retains them after a call returns.
 *   - All device work is enqueued on the plan's stream (given at plan
 *     creation; NULL = the legacy default stream) without host
 *     synchronisation, except where a call says otherwise.
 *   - Every call returns BORIS_OK (0) or a negative boris_status; the reason
 *     is available from boris_last_error() on the calling thread.  Device-
 *     side errors (a bounded wait that gave up, a step-size controller that
 *     ran out of attempts) are latched in a status word on the device and
 *     returned by boris_sync_status() and by the next synchronising call.
 *   - A plan is reusable for any number of calls but is not thread-safe.
 */
#ifndef BORIS_H
#define BORIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct boris_plan_s* boris_plan;

typedef enum {
    BORIS_OK = 0,
    BORIS_ERR_INVALID_ARG = -1,      /* bad pointer, size, flag or parameter    */
    BORIS_ERR_OOM = -2,              /* device or host allocation failed        */
    BORIS_ERR_CUDA = -3,             /* a CUDA runtime call failed              */
    BORIS_ERR_UNSUPPORTED_SIZE = -4, /* mesh too large for the available kernels */
    BORIS_ERR_TIMEOUT = -5,          /* a bounded device-side wait gave up      */
    BORIS_ERR_STEP_CONTROL = -6      /* RKF45 rejected too many trial steps     */
} boris_status;

/* Plan flags */
#define BORIS_FLAG_F32 0x0u        /* FP32 transforms and LLG (default)                */
#define BORIS_FLAG_F64 0x1u        /* FP64 everywhere: use the *_f64 entry points       */
/* Mixed-precision z stage (FP32 plans, pz = 64, i.e. 17 <= nz <= 32): the
 * zero-padded z transform and its inverse run as dense matrix products on the
 * tensor cores with FP16 (or BF16) operands, one scale per (kx, ky,
 * component) column, FP32 accumulation; everything else stays FP32.  Where
 * py >= 64 the products are tcgen05.mma with accumulators in tensor memory
 * (power-of-two column scales); otherwise, or with BORIS_TC_MMASYNC=1 at plan
 * creation, mma.sync with the exact column maxima as scales.  Where in
 * addition py = 1024 (257 <= ny <= 512), the
 * padded y-z spectrum itself is stored in the 16-bit format between the y and
 * z passes (BF16 as it is; FP16 scaled by the power of two s with
 * s nx ny nz max|Ms M| < 2^14, max|Ms M| found on the device each evaluation)
 * and the tcgen05 z stage takes 128 ky columns as the rows of its products
 * (BORIS_TC_STORE16=0 at plan creation keeps the FP32 spectrum).  The paper
 * has FP32/FP64 only; expected relative L2 error of H_d ~2e-4 (FP16) to
 * ~2e-3 (BF16). */
#define BORIS_FLAG_FP16_TC 0x2u
#define BORIS_FLAG_BF16_TC 0x4u

/* Integration methods (boris_llg_params.method) */
#define BORIS_RK4 0
#define BORIS_RKF45 1

/*
 * boris_demag_plan - prepare H = -N * M for an nx x ny x nz mesh of
 * dx x dy x dz cells (m).
 *   Builds on the device, in FP64, the Newell tensor for every displacement
 *   (exact closed form within 40 cell sizes, the box-averaged dipole expansion
 *   beyond), transforms its zero-padded extension, and stores the real kernel
 *   spectrum (one octant, 6 components, FP32 or FP64 per flags).  Allocates
 *   the transform workspace.  Synchronises the stream before returning.
 *   flags: BORIS_FLAG_F32 or BORIS_FLAG_F64.  cuda_stream: a cudaStream_t or
 *   NULL.  On success *out receives the plan (free with boris_plan_destroy).
 *   Errors: INVALID_ARG (n < 1, cell <= 0, out NULL), UNSUPPORTED_SIZE (a
 *   padded length above 4096 or a y-z plane too large for shared memory),
 *   OOM, CUDA.
 */
int boris_demag_plan(int nx, int ny, int nz, double dx, double dy, double dz, unsigned flags,
                     void* cuda_stream, boris_plan* out);

/*
 * boris_demag_plan_pbc - as boris_demag_plan, with periodic boundary
 *   conditions by the multiple-images method (Section 4, extending Eq. 4):
 *   images[a] > 0 makes axis a (0 x, 1 y, 2 z) periodic with period n_a h_a,
 *   and the field at a mesh cell then includes the sources in the images of
 *   the mesh displaced by up to images[a] periods on each side.  For a
 *   displacement d between two mesh cells the kernel becomes the image sum
 *   sum_k N(d + k L) (|k_a| <= images[a]), built in FP64 on the device with
 *   the same exact / asymptotic forms; the zero-padded transforms are
 *   unchanged (the image sum is a linear convolution over one period).  The
 *   LLG exchange (and DMI) stencil of such a plan wraps around the periodic
 *   axes.  images[a] = 0 leaves axis a open.  The adjoint
 *   (boris_llg_step_backward) serves non-periodic plans only.
 *   Errors: as boris_demag_plan; INVALID_ARG for images NULL or outside 0..1000.
 */
int boris_demag_plan_pbc(int nx, int ny, int nz, double dx, double dy, double dz, const int images[3], unsigned flags,
                         void* cuda_stream, boris_plan* out);

/*
 * boris_oersted_plan - prepare the Oersted field of a current density (Table 1:
 *   H(r0) = sum_r K(r - r0) J(r); the paper takes K from its Ref. [63]).  Here
 *   K is derived: for a uniform current density J in a source cell the
 *   target-cell average of the Biot-Savart field is J x g(D), D = target -
 *   source, with g = -(1/(4 pi V)) grad P, P the two-cell integral of
 *   1/|r - r'|; since Newell's tensor of the same pair is N_ij = d_i g_j, g_k is
 *   built in FP64 on the device as the antiderivative of N_kk along axis k
 *   (Gauss-Legendre over whole cells) closed by the far-field gradient of the
 *   box-averaged potential beyond 40 cell sizes.  Its zero-padded spectrum is
 *   imaginary (g_k odd in axis k only), and the convolution runs as
 *   H^ = i (J^ x G) on the demag transform pipeline (split y-z schedule,
 *   residue-split z stage; a pointwise multiply when nz = 1).  FP32.
 *   Supported: nz = 1, or 3 <= nz <= 32 with ny >= 33.
 *   Errors: INVALID_ARG, UNSUPPORTED_SIZE, OOM, CUDA.  Synchronises the stream.
 */
int boris_oersted_plan(int nx, int ny, int nz, double dx, double dy, double dz, void* cuda_stream, boris_plan* out);

/*
 * boris_oersted_apply - H = Oersted field (A/m) of the current density J
 *   (A/m^2); both device SoA [3][nz][ny][nx] FP32, 16-byte aligned, distinct.
 *   Asynchronous on the plan's stream; a bounded device wait that gives up
 *   latches BORIS_ERR_TIMEOUT (boris_sync_status).
 */
int boris_oersted_apply(boris_plan p, const float* J, float* H);

/*
 * boris_multimesh_plan - prepare the multi-mesh demagnetising field of Eq. 4
 *   for a stack of n_layers (1..16) rectangular meshes:
 *     H(r'_kl) = -sum_i sum_{r_ij in V_i} N(r'_kl - r_ij, h_k, h_i) M(r_ij).
 *   Layer l has nxyz[3l..3l+2] cells of size hxyz[3l..3l+2] (m) with its
 *   lower corner at origin[3l..3l+2] (m).  All layers share the in-plane cell
 *   size, and their in-plane origins differ by whole cells; their z sizes,
 *   z positions and gaps are arbitrary (at most 256 z planes in total).  The
 *   inter-mesh tensor between cells of z size a (target) and b (source) is
 *   Newell's construction with the two-box z stencil, normalised by the
 *   target volume (a far-field dipole expansion beyond 40 cell sizes), built
 *   in FP64 on the device.  The stencil is symmetric in a and b, so
 *   a N_ab = b N_ba: the plan stores the 2D in-plane spectrum of a N_ab once
 *   per distinct (min(a, b), max(a, b), |dz|) and divides by the target's a
 *   in the sum.  The inter-plane sum in transform space is one kernel over
 *   all layer pairs; the plan times its variants (one CTA per tile, staged
 *   rows, or one persistent launch at one or two CTAs per SM) and keeps the
 *   fastest (boris_plan_schedule out[2]; BORIS_ML_MIX=v at plan creation
 *   forces variant v).  flags: BORIS_FLAG_F32 only.  The plan works with
 *   boris_demag_apply on the layers' fields concatenated in layer order, each
 *   SoA [3][nz][ny][nx], and with boris_llg_step (per-cell maps concatenated
 *   the same way).  Synchronises the stream.
 *   Errors: INVALID_ARG, UNSUPPORTED_SIZE (frame transform above 4096 or
 *   more than 256 planes), OOM, CUDA.
 */
int boris_multimesh_plan(int n_layers, const int* nxyz, const double* hxyz, const double* origin, unsigned flags,
                         void* cuda_stream, boris_plan* out);

/* Multi-mesh plan facts: out[0] z planes, out[1] distinct inter-plane spectra,
 * out[2..3] in-plane frame size (cells). */
int boris_plan_multimesh_info(boris_plan p, int out[4]);

/*
 * boris_demag_apply - Hd = -N * M (Table 1), FP32 plan.
 *   M, Hd: device [3][nz][ny][nx] float, A/m; may not alias.
 *   Kernels: zero-padded x real-to-complex transform; the y-z pass (y and z
 *   transforms, kernel multiply, inverse z and y transforms) in the schedule
 *   the plan's autotuner chose (boris_plan_schedule); x complex-to-real
 *   transform.  Asynchronous on the plan's stream.
 */
int boris_demag_apply(boris_plan p, const float* M, float* Hd);
/* FP64 plan variant (same layout, double). */
int boris_demag_apply_f64(boris_plan p, const double* M, double* Hd);

/*
 * boris_demag_apply_noalloc - Hd = -N * M exactly as boris_demag_apply (FP32
 *   plans), for callers that cannot allocate device memory while they run.
 *   The paper has no counterpart: this serves runtimes whose allocator is
 *   locked or forbidden on their hot path.  It allocates nothing: the spectral
 *   workspace is a fixed 32 MiB device array inside the library (held by every
 *   GPU that loads the library until the process exits), so it accepts meshes
 *   whose spectral workspace - (px/2 + 1) * 3 * nz * ny * 8 bytes, plus
 *   (px/2 + 1) * py * 3 * nz * 8 bytes when the plan chose the split y-z
 *   schedule - fits in 32 MiB, and returns BORIS_ERR_UNSUPPORTED_SIZE for
 *   larger ones.  The plan (made at set-up)
 *   still supplies the kernel spectrum.  The plan's device must be current.
 *   The first call on a device looks up the array's device address; make that
 *   first call before any stream capture.  All calls share the one array:
 *   calls that overlap on the GPU race and corrupt each other's output.
 *   Nothing in the array needs clearing: every call overwrites what it reads.
 *   On a plan made with a tensor-core flag it runs an FP32 z stage, so its
 *   result has FP32 accuracy rather than that of the 16-bit stage.
 */
int boris_demag_apply_noalloc(boris_plan p, const float* M, float* Hd);

/*
 * boris_demag_adjoint - gM = (dHd/dM)^T gHd.  The demagnetising operator is
 *   self-adjoint (N_ij = N_ji and N(-r) = N(r)), so this is -N * gHd; the
 *   paper has no adjoint, this call serves gradient computations.
 */
int boris_demag_adjoint(boris_plan p, const float* gHd, float* gM);

/* LLG parameters.  Ms/Ku maps: device [nz][ny][nx] arrays of the plan's
 * precision (float for FP32 plans, double for FP64), or NULL for the uniform
 * value.  gamma in m/(A s) (Eq. 1: gamma = mu0 g_rel |gamma_e|). */
typedef struct {
    const void* Ms_map; /* per-cell saturation magnetisation (A/m) or NULL  */
    double Ms;          /* uniform Ms when Ms_map is NULL                   */
    double A;           /* exchange stiffness (J/m)                         */
    double alpha;       /* Gilbert damping                                  */
    double gamma;       /* gyromagnetic ratio (m/(A s))                     */
    const void* Ku_map; /* per-cell uniaxial anisotropy K1 (J/m^3) or NULL  */
    double Ku;          /* uniform K1 when Ku_map is NULL                   */
    double easy[3];     /* unit easy axis e_A                               */
    double Hext[3];     /* applied field (A/m)                              */
    int method;         /* BORIS_RK4 or BORIS_RKF45                         */
    double tol;         /* RKF45: accept when max |m5 - m4| <= tol          */
    double dt_min;      /* RKF45 step bounds (s)                            */
    double dt_max;
} boris_llg_params;

/*
 * boris_llg_step - advance the unit magnetisation m (device [3][nz][ny][nx],
 *   in place) by one time step of the LLG equation (Eq. 1, Landau-Lifshitz
 *   form), effective field H = Hd(Ms m) + (2A/(mu0 Ms)) lap m (Neumann)
 *   + (2Ku/(mu0 Ms))(m.e)e + Hext.
 *   RK4: four field evaluations (four demag applications), *dt is the step
 *   and is not changed; m is renormalised after the step.
 *   RKF45: trial steps with the embedded error max |m5 - m4| (an FP64 max
 *   over cells) until one is accepted - err <= tol, or dt <= dt_min - at
 *   most 16 trials, else BORIS_ERR_STEP_CONTROL (also latched in the status
 *   word) with m unchanged.  The decision and the step size live on the
 *   device: one step is a CUDA graph whose conditional WHILE node repeats the
 *   trial until a one-thread controller kernel accepts it; no host decision
 *   is taken between trials.  *dt is the step to try on input and, on
 *   return, the controller's next step dt*clip(0.9 (tol/err)^(1/5), 0.2, 2)
 *   within [dt_min, dt_max]; reading it back synchronises the stream once
 *   per accepted step (boris_llg_run_rkf45 takes many steps per
 *   synchronisation).  The graph is captured on the first call and again
 *   when m, *prm or the field terms change (that capture synchronises the
 *   stream once).
 */
int boris_llg_step(boris_plan p, float* m, const boris_llg_params* prm, double* dt);
int boris_llg_step_f64(boris_plan p, double* m, const boris_llg_params* prm, double* dt);

/*
 * boris_llg_step_backward - discrete adjoint of one RK4 step (the paper has
 *   no adjoint; this serves gradient-based fitting of material maps).
 *   Given the step's input state m_in (device [3][nz][ny][nx], unchanged) and
 *   g_m_out = dL/dm_out, writes g_m_in = dL/dm_in (may not alias g_m_out)
 *   and ADDS dL/dMs and dL/dKu into g_Ms and g_Ku (device [nz][ny][nx]; either
 *   may be NULL to skip).  The step is recomputed (four demag applications)
 *   and back-propagated through the renormalisation, the four stages, the
 *   Landau-Lifshitz right-hand side, exchange (the Neumann Laplacian is
 *   symmetric), anisotropy and the demagnetising operator, which is
 *   self-adjoint so each transpose is one more demag application.
 *   prm->method must be BORIS_RK4.  Workspace: 18 fields, allocated once.
 */
int boris_llg_step_backward(boris_plan p, const float* m_in, const boris_llg_params* prm, double dt,
                            const float* g_m_out, float* g_m_in, float* g_Ms, float* g_Ku);
int boris_llg_step_backward_f64(boris_plan p, const double* m_in, const boris_llg_params* prm, double dt,
                                const double* g_m_out, double* g_m_in, double* g_Ms, double* g_Ku);

/*
 * boris_llg_run_graph - nsteps RK4 steps of boris_llg_step (FP32 plans,
 *   single- or multi-mesh), replayed from a CUDA graph: the first call (and
 *   any call whose m, *prm or dt differ from the captured ones) captures one
 *   step - all its kernel launches - on a plan-owned stream and instantiates
 *   it; every step is then one graph launch on the plan's stream.  The device
 *   pointers in *prm and m must stay valid while the plan keeps the graph.
 *   The capture synchronises the plan's stream once.
 */
int boris_llg_run_graph(boris_plan p, float* m, const boris_llg_params* prm, double dt, int nsteps);

/*
 * boris_llg_run_rkf45 - nsteps accepted RKF45 steps of boris_llg_step (FP32
 *   single-mesh plans) with the step control on the device (Section 2:
 *   4th order with an embedded 5th order error estimator): starting from the
 *   step *dt, each step is one launch of the plan's RKF45 step graph (trial
 *   loop as a conditional WHILE node, at most 16 trials), and the step size
 *   carries from step to step in device memory.  The host enqueues the
 *   launches only and synchronises once at the end, to return in *dt the
 *   controller's next step and in *t_elapsed (may be NULL) the simulated
 *   time of the accepted steps.  Returns BORIS_ERR_STEP_CONTROL if any step
 *   exhausted its trials (m then keeps the state before that step).
 */
int boris_llg_run_rkf45(boris_plan p, float* m, const boris_llg_params* prm, double* dt, int nsteps,
                        double* t_elapsed);

/*
 * boris_llg_run_host - end-to-end form for callers holding host memory:
 *   copies m_host (host [3][nz][ny][nx] float; pinned memory is fastest) to
 *   the device, runs nsteps RK4 steps of size dt > 0 (replayed from the
 *   plan's CUDA graph, as boris_llg_run_graph on the device copy), copies the
 *   result back to m_host, and synchronises.  Allocates its device copy once
 *   per plan.  Host-device copies run at about 200 GB/s on GB300 (measured
 *   alike for copy engines and for copy kernels on mapped pinned memory).
 */
int boris_llg_run_host(boris_plan p, float* m_host, const boris_llg_params* prm, double dt,
                       int nsteps);

/*
 * boris_energy - FP64 energies of state m: out = {E_demag, E_exchange,
 *   E_anisotropy, E_Zeeman} in J, with E = sum V [-(mu0 Ms/2) m.(Hd + Hex)
 *   + Ku (1 - (m.e)^2) - mu0 Ms m.Hext].  Synchronises the stream.
 */
int boris_energy(boris_plan p, const float* m, const boris_llg_params* prm, double out[4]);

/* Further effective-field terms (Table 1 of Appendix A; Eq. 5).  All zero
 * (or dmi = BORIS_DMI_NONE) leaves the base field of boris_llg_step. */
#define BORIS_DMI_NONE 0
#define BORIS_DMI_BULK 1        /* H = -(2D/(mu0 Ms)) curl m, dm/dn = (D/2A) n x m       */
#define BORIS_DMI_INTERFACIAL 2 /* H = (2D/(mu0 Ms))((div m) z - grad m_z),
                                   dm/dn = (D/2A)(z x n) x m                          */
typedef struct {
    double K2;          /* uniaxial second order (J/m^3), axis boris_llg_params.easy:
                           eps = K2 (1 - (m.e)^2)^2                                 */
    double Kc1, Kc2;    /* cubic anisotropy (J/m^3): eps = Kc1 (a^2 b^2 + a^2 c^2 + b^2 c^2)
                           + Kc2 a^2 b^2 c^2, a = m.e1, b = m.e2, c = m.e3            */
    double cubic_e1[3]; /* cubic axes e1, e2 (normalised by the call; they must be
                           orthogonal), e3 = e1 x e2                                  */
    double cubic_e2[3];
    int dmi;            /* BORIS_DMI_*; single-mesh plans only, needs A > 0          */
    double D;           /* DMI constant (J/m^2)                                       */
    double J1, J2;      /* surface exchange (J/m^2) of Eq. 5 between consecutive layers of
                           a multi-mesh plan: the top cell plane of layer l and the bottom
                           plane of layer l + 1 where they overlap in-plane, Delta = the
                           receiving cell's z size; layers must be listed bottom-up     */
    double temperature; /* thermal field (K; 0 = off), single-mesh plans, RK4 only:
                           Brown's field in H_eff, each component of cell i at step s
                           sigma g with sigma = sqrt(2 alpha kB T / (gamma mu0 Ms V dt)),
                           g normal from the counter-based generator Philox4x32-10
                           (counter (i, s mod 2^32, s div 2^32, 0), key = seed,
                           Box-Muller), held through the step's four stages          */
    unsigned long long seed;
    const void* H_add;  /* additive field map (A/m), device [3][nz][ny][nx] of the plan's
                           precision, or NULL: added to H_eff like Hext (its energy is
                           counted with the Zeeman term) - e.g. an Oersted field from
                           boris_oersted_apply; single-mesh plans                        */
} boris_field_terms;

/*
 * boris_set_field_terms - set (t != NULL) or clear (t == NULL) the further
 *   field terms of plan p; they enter every later boris_llg_step,
 *   boris_llg_run_graph (a changed set re-captures the graph) and
 *   boris_energy_terms.  DMI changes the exchange boundary to the
 *   non-homogeneous Neumann condition of Table 1: a neighbour outside the
 *   mesh is the ghost m + h dm/dn, which both the exchange Laplacian and the
 *   central DMI differences use.  Stepping with these terms uses the
 *   one-cell-per-thread stage kernel; boris_llg_step_backward covers the base
 *   terms only and fails with BORIS_ERR_INVALID_ARG while terms are set.
 *   Errors: INVALID_ARG (non-finite values, non-orthogonal cubic axes, unknown
 *   dmi kind, DMI on a multi-mesh plan, J1/J2 on a single-mesh plan, layers
 *   not bottom-up).
 */
int boris_set_field_terms(boris_plan p, const boris_field_terms* t);

/*
 * boris_thermal_set_step - set the step counter s of the thermal field (it
 *   starts at 0 and each RK4 step of boris_llg_step / boris_llg_run_graph
 *   advances it by one on the device, so graph replays draw new fields).
 *   Asynchronous on the plan's stream.  Errors: INVALID_ARG, OOM, CUDA.
 */
int boris_thermal_set_step(boris_plan p, unsigned long long step);

/*
 * boris_philox4x32_10 - the thermal field's random-number generator on given
 *   inputs: out[4i..4i+3] = Philox4x32-10(counter ctr[4i..4i+3], key
 *   key[2i..2i+1]) for i < n, the same device function the stage kernels
 *   draw from (Salmon, Moraes, Dror and Shaw, SC'11; the thermal field of
 *   Section 1, Eq. 17).  ctr, key, out: device arrays of 32-bit words.
 *   Asynchronous on cuda_stream (a cudaStream_t or NULL).  It lets a caller
 *   check the generator against its published known-answer vectors.
 *   Errors: INVALID_ARG (n < 0, NULL arrays with n > 0), CUDA.
 */
int boris_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n, void* cuda_stream);

/*
 * boris_energy_terms - as boris_energy, with out = {E_demag, E_exchange,
 *   E_anisotropy (uniaxial K1, K2 and cubic), E_Zeeman, E_DMI} in J; the
 *   exchange and DMI energies are -(mu0 Ms V/2) sum m.H of their fields.
 *   Single-mesh FP32 plans.  Synchronises the stream.
 */
int boris_energy_terms(boris_plan p, const float* m, const boris_llg_params* prm, double out[5]);

/* Device status word: BORIS_OK or the first latched device-side error,
 * which is then cleared.  Synchronises the stream. */
int boris_sync_status(boris_plan p);

/* Human-readable reason for the last failing call on this thread. */
const char* boris_last_error(void);

/* Padded transform lengths chosen by the plan: out[0..2] = px, py, pz. */
int boris_plan_padded(boris_plan p, int out[3]);

/* Schedule of the y-z pass chosen by the plan's autotuner (CUDA-event
 * timing of every candidate that fits the mesh): out[0] kind (0: fused, z
 * stage through shared-memory passes, 1: fused, z stage in registers, 2:
 * split into y-forward / z-convolution / y-inverse kernels; multi-mesh plans
 * report kind 2 with out[2] the inter-plane sum variant: 0 one CTA per tile,
 * 1 staged rows, 2 or 3 one persistent launch with 1 or 2 CTAs per SM).
 * Kinds 0 and 1:
 * out[1] CTAs per cluster, out[2] threads per CTA, out[3] shared memory per
 * CTA.  Kind 2: out[1] CTAs per SM the z convolution's register budget is
 * fitted to, out[2] the z-convolution variant: 1 or 2 for the persistent
 * bulk-copy (TMA) pipeline with one or two tile stages, 3 for the residue-
 * split z convolution, 0 for the shared-memory form; on tensor-core plans 5
 * for the tcgen05 stage, 4 for the mma.sync one and 6 for the plans whose
 * y passes store the spectrum in 16 bits and whose tcgen05 z stage takes the
 * data as the 128-row operand (BORIS_TC_STORE16=0 at plan creation keeps
 * the FP32 spectrum and variant 5).  Variants 1, 2, 3, 5 and 6 bound their
 * mbarrier waits and latch BORIS_ERR_TIMEOUT in the status word read by
 * boris_sync_status.
 * Environment overrides read at plan creation restrict the candidates:
 * BORIS_YZ_KIND, BORIS_YZ_CLUSTER, BORIS_YZ_THREADS, BORIS_YZ_QC (kind 0
 * chunk), BORIS_YZ_TMA (kind 2 variant). */
int boris_plan_schedule(boris_plan p, int out[4]);

/* Bytes of device memory owned by the plan. */
size_t boris_plan_device_bytes(boris_plan p);

/*
 * boris_profile_enable - when on != 0, every kernel the plan launches is
 *   bracketed by two CUDA events recorded on the plan's stream (a few
 *   microseconds of overhead per launch); off by default.
 * boris_profile_read - synchronises, then returns per kernel class the summed
 *   device time in ms and the number of timed launches since the last read:
 *   [0] x real-to-complex, [1] fused y-z pass, [2] x complex-to-real,
 *   [3] LLG stage, [4] other (energies), [5] y forward, [6] z convolution,
 *   [7] y inverse (the last three: split y-z schedule), [8] x complex-to-real
 *   fused with the RK4 stage (FP32 plans with px = 1024 created while the
 *   environment sets BORIS_FUSE_STAGE=1).  *total_launches (may be NULL)
 *   receives every kernel launch counted since the last read, timed or not.
 *   Resets the counters.
 */
int boris_profile_enable(boris_plan p, int on);
int boris_profile_read(boris_plan p, double ms_out[9], long long launches_out[9], long long* total_launches);

/* Free the plan and everything it owns (NULL is ignored).  Synchronises. */
void boris_plan_destroy(boris_plan p);

#ifdef __cplusplus
}
#endif

#endif /* BORIS_H */
