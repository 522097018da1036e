// Hop kernels and their launcher for the F64 operator.
#include "hop_kernel.cuh"

namespace mdwf {
template int launch_hop_t<MDWF_F64>(mdwf_ctx* c, const HopLaunch& h);
}  // namespace mdwf
