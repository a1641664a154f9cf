// Demag application for callers that cannot allocate device memory while it
// runs: the spectral workspace lives in a fixed, file-scope device array
// instead of plan memory.
//
// Who needs this: code that runs where cudaMalloc is not allowed or not
// wanted - for instance a step that is replayed inside someone else's
// stream-ordered memory budget, a caller whose allocator is locked after
// start-up, or a host runtime that forbids allocation on its hot path.  Such
// callers create the plan once during set-up (the plan still owns the kernel
// spectrum and twiddles) and then call boris_demag_apply_noalloc, which
// allocates nothing.
//
// Costs and limits: the array (NOALLOC_SCRATCH_BYTES, 32 MiB) is held by
// every GPU that loads the library until the process exits; meshes whose
// spectrum needs more are rejected; all calls share one array, so calls that
// overlap on the GPU (different streams, or different host threads on one
// device) race and corrupt each other's results.
#include <mutex>
#include <string>

#include "boris_internal.cuh"

namespace boris {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)32 << 20;

// The workspace.  In host code this name is only a stand-in for the device
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_mu;
void* g_addr[128] = {nullptr};

// Once per device, with that device current: look up the device address of
// the array.  Returns nullptr (and sets the error message) on failure.
void* scratch_address(int dev)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 128) {
        set_error("device ordinal out of range");
        return nullptr;
    }
    if (!g_addr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return nullptr;
        }
        g_addr[dev] = ptr;
    }
    return g_addr[dev];
}
}  // namespace

}  // namespace boris

using namespace boris;

extern "C" int boris_demag_apply_noalloc(boris_plan p, const float* M, float* Hd)
{
    PlanView v;
    if (!plan_view(p, &v) || !M || !Hd) {
        set_error("NULL argument");
        return BORIS_ERR_INVALID_ARG;
    }
    if (v.f64 || v.ml || v.oersted) {
        set_error("boris_demag_apply_noalloc serves FP32 single-mesh demag plans only");
        return BORIS_ERR_INVALID_ARG;
    }
    if (((uintptr_t)M & 15u) || ((uintptr_t)Hd & 15u) || (const void*)M == (const void*)Hd) {
        set_error("M and Hd must be 16-byte aligned and distinct");
        return BORIS_ERR_INVALID_ARG;
    }
    const size_t xbytes = (size_t)v.g.nkx * 3 * v.g.nz * v.g.ny * sizeof(float2);
    // the split y-z schedule also needs the column-major padded spectrum
    const size_t ybytes = v.yz.kind == 2 ? (size_t)v.g.nkx * v.g.py * 3 * v.g.nz * sizeof(float2) : 0;
    const size_t xoff = (xbytes + 255) & ~(size_t)255;
    const size_t need = xoff + ybytes;
    if (need > NOALLOC_SCRATCH_BYTES) {
        set_error("mesh spectrum needs " + std::to_string(need) + " bytes; the allocation-free workspace holds " +
                  std::to_string(NOALLOC_SCRATCH_BYTES) + " bytes (use boris_demag_apply)");
        return BORIS_ERR_UNSUPPORTED_SIZE;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev != v.device) {
        set_error("the plan's device must be current");
        return BORIS_ERR_INVALID_ARG;
    }
    float2* X = (float2*)scratch_address(dev);
    if (!X) return BORIS_ERR_CUDA;
    // every element of the workspace is written before it is read (X by the
    // forward x transform, Y by the y-forward kernel), so nothing needs
    // clearing between calls
    const float2* tw = (const float2*)v.tw;
    float2* Y = (float2*)((unsigned char*)X + xoff);
    if ((e = launch_x_r2c<float>(v.g, M, nullptr, 1.0f, X, tw, v.stream)) == cudaSuccess) {
        if (v.yz.kind == 2) {
            for (int part = 0; part < 3 && e == cudaSuccess; part++)
                e = launch_split<float>(v.g, X, Y, (const float*)v.K, tw, v.stream, part, v.yz.C);
        } else {
            e = launch_yz_conv<float>(v.g, v.yz, X, (const float*)v.K, tw, v.stream);
        }
    }
    if (e == cudaSuccess) e = launch_x_c2r<float>(v.g, X, Hd, tw, v.stream);
    if (e != cudaSuccess) {
        set_error(std::string("demag kernels: ") + cudaGetErrorString(e));
        return BORIS_ERR_CUDA;
    }
    return BORIS_OK;
}
