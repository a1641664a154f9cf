// Instantiations of the register z-stage y-z pass for float.
#include "yz_reg.cuh"

namespace boris {

cudaError_t upload_twiddles_yz_f32() { return upload_small_twiddles_here(); }

template <>
cudaError_t launch_yz_reg<float>(const Geometry& g, const YZSchedule& sc, Cx<float>::t* X, const float* K,
                                const Cx<float>::t* tw, cudaStream_t st)
{
    if (sc.C == 1 && sc.threads == 384) return launch_yz_reg_hz<float, 1, 384>(g, sc.smem, X, K, tw, st);
    if (sc.C == 1 && sc.threads == 768) return launch_yz_reg_hz<float, 1, 768>(g, sc.smem, X, K, tw, st);
    if (sc.C == 8 && sc.threads == 384) return launch_yz_reg_hz<float, 8, 384>(g, sc.smem, X, K, tw, st);
    if (sc.C == 8 && sc.threads == 768) return launch_yz_reg_hz<float, 8, 768>(g, sc.smem, X, K, tw, st);
    if (sc.C == 16 && sc.threads == 384) return launch_yz_reg_hz<float, 16, 384>(g, sc.smem, X, K, tw, st);
    if (sc.C == 16 && sc.threads == 768) return launch_yz_reg_hz<float, 16, 768>(g, sc.smem, X, K, tw, st);
    return cudaErrorInvalidValue;
}

}  // namespace boris
