// Hop launch dispatch over the operator precisions (the kernels are in
// hop_kernel.cuh, instantiated in dslash_f64.cu, dslash_f32.cu and
// dslash_f16n.cu), the block shapes of the hop kernels, and the self-test of
// the bounded device-side wait.
#include "mdwf_internal.cuh"
#include "mbarrier.cuh"

namespace mdwf {

template <int P> int launch_hop_t(mdwf_ctx* c, const HopLaunch& h);

// 4d sites per block: the autotuned value for (precision, nrhs) if there is
// one, else as many whole s-columns as fit 128 threads.
int hop_sites_per_block(const mdwf_ctx* c, int prec, int nrhs) {
    const int t = (nrhs >= 1 && nrhs <= 64) ? c->sb_tune[prec][nrhs] : 0;
    if (t > 0) return t;
    const int sb = 128 / c->g.Ls;
    return sb < 1 ? 1 : sb;
}

// The fused iteration drops its t field when the FUSE_R epilogue can rebuild
// t = I^dag v by shuffles: FP32 or FP16+norm operators at Ls = 16 with the
// closed-form s-operators, whole s-columns in every warp (an even number of
// sites per block) and a load strategy whose kernels fix Ls = 16 at compile
// time (not the two shared-memory staging modes).
bool hop_no_t_ok(const mdwf_ctx* c, int prec, int nrhs) {
    if (prec == MDWF_F64 || c->g.Ls != 16 || c->dense_s || c->sdep) return false;
    if (hop_sites_per_block(c, prec, nrhs) & 1) return false;
    const int mode = c->hop_stage[prec];
    return mode != 1 && mode != 2;
}

int hop_blocks(const mdwf_ctx* c, int prec, int nrhs) {
    const int SB = hop_sites_per_block(c, prec, nrhs);
    return (int)((c->g.Vh + SB - 1) / SB);
}

// One thread waits, bounded, on an mbarrier that expects two arrivals of
// which `arrivals` are made; a wait that gives up sets the error word.
__global__ void k_wait_selftest(int* err, int arrivals) {
    __shared__ unsigned long long bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 2);
    mbar_init_fence();
    for (int k = 0; k < arrivals; ++k) mbar_arrive(&bar);
    if (!mbar_wait(&bar, 0)) atomicOr(err, 1);
}

int launch_hop(mdwf_ctx* c, int prec, const HopLaunch& h) {
    switch (prec) {
        case MDWF_F64: return launch_hop_t<MDWF_F64>(c, h);
        case MDWF_F32: return launch_hop_t<MDWF_F32>(c, h);
        case MDWF_F16N: return launch_hop_t<MDWF_F16N>(c, h);
    }
    return MDWF_EINVAL;
}

}  // namespace mdwf

using namespace mdwf;

extern "C" int mdwf_selftest_wait(mdwf_ctx* c, int arrivals) {
    if (!c || arrivals < 0 || arrivals > 2) return MDWF_EINVAL;
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    k_wait_selftest<<<1, 32, 0, c->stream>>>(c->dev_err, arrivals);
    if ((st = check_launch())) return st;
    return device_wait_status(c);
}
