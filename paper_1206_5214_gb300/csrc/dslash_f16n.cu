// Hop kernels and their launcher for the F16N operator.
#include "hop_kernel.cuh"

namespace mdwf {
template int launch_hop_t<MDWF_F16N>(mdwf_ctx* c, const HopLaunch& h);
}  // namespace mdwf
