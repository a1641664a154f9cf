// Instantiations of the register z-stage y-z pass for double.
#include "yz_reg.cuh"

namespace boris {

cudaError_t upload_twiddles_yz_f64() { return upload_small_twiddles_here(); }

template <>
cudaError_t launch_yz_reg<double>(const Geometry& g, const YZSchedule& sc, Cx<double>::t* X, const double* K,
                                const Cx<double>::t* tw, cudaStream_t st)
{
    if (sc.C == 1 && sc.threads == 384) return launch_yz_reg_hz<double, 1, 384>(g, sc.smem, X, K, tw, st);
    if (sc.C == 8 && sc.threads == 384) return launch_yz_reg_hz<double, 8, 384>(g, sc.smem, X, K, tw, st);
    if (sc.C == 16 && sc.threads == 384) return launch_yz_reg_hz<double, 16, 384>(g, sc.smem, X, K, tw, st);
    return cudaErrorInvalidValue;
}

}  // namespace boris
