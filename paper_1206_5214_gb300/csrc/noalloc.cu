// mdwf_apply_noalloc: the operator M (or M^dag) of mdwf_apply without any
// device allocation, for callers that must not allocate while they run:
// code whose device memory is owned by a host framework's pool (a custom
// operator inside another runtime), code on a real-time or latency-critical
// path that must not enter the driver's allocator, or code that has to keep
// a long-lived footprint fixed. Such callers create the context once during
// set-up; after that this entry point touches only the caller's fields, the
// context's read-only data and the fixed scratch below.
//
// The intermediate fields of the operator (z on the even sites, and v = A^dag
// psi for M^dag) and the per-right-hand-side masses live in file-scope device
// arrays that every GPU loading this library holds until the process exits.
// Host code cannot use those array names as device addresses: the device
// address of each is fetched once per device with cudaGetSymbolAddress.
// The masses of a call travel as kernel arguments (by value) to a one-block
// kernel that writes them into their fixed arrays, stream-ordered before the
// operator's kernels: no host buffer has to outlive the call.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "mdwf_internal.cuh"

namespace mdwf {

// Fixed scratch: two intermediate fields of at most kNoAllocFieldBytes each.
constexpr size_t kNoAllocFieldBytes = (size_t)8 << 20;  // 8 MiB per intermediate field
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[2 * kNoAllocFieldBytes];
static __device__ __align__(256) double g_noalloc_mass64[64];
static __device__ __align__(256) float g_noalloc_mass32[64];

struct NoAllocAddrs {
    bool ready = false;
    unsigned char* scratch = nullptr;
    double* mass64 = nullptr;
    float* mass32 = nullptr;
};
static NoAllocAddrs g_noalloc_addrs[kNoAllocMaxDevices];
static std::mutex g_noalloc_mutex;

// Device addresses of the static arrays on the current device (once per device).
static int noalloc_setup(int device, NoAllocAddrs** out) {
    if (device < 0 || device >= kNoAllocMaxDevices) return MDWF_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocAddrs& a = g_noalloc_addrs[device];
    if (!a.ready) {
        void* p = nullptr;
        int st;
        if ((st = cuda_status(cudaGetSymbolAddress(&p, g_noalloc_scratch)))) return st;
        a.scratch = (unsigned char*)p;
        if ((st = cuda_status(cudaGetSymbolAddress(&p, g_noalloc_mass64)))) return st;
        a.mass64 = (double*)p;
        if ((st = cuda_status(cudaGetSymbolAddress(&p, g_noalloc_mass32)))) return st;
        a.mass32 = (float*)p;
        a.ready = true;
    }
    *out = &a;
    return MDWF_OK;
}

// The masses of one call, passed by value.
struct NoAllocMasses {
    double m64[64];
    float m32[64];
    int n;
};

__global__ void k_noalloc_masses(NoAllocMasses m) {
    const int r = threadIdx.x;
    if (r < m.n) {
        g_noalloc_mass64[r] = m.m64[r];
        g_noalloc_mass32[r] = m.m32[r];
    }
}

}  // namespace mdwf

using namespace mdwf;

extern "C" int mdwf_apply_noalloc(mdwf_ctx* c, void* out, const void* in, int prec, int nrhs,
                                  const double* mf_per_rhs, int dagger) {
    NvtxRange nvtx_range("mdwf_apply_noalloc");
    if (!c || !out || !in || out == in || nrhs < 1 || nrhs > 64) return MDWF_EINVAL;
    if (prec != MDWF_F64 && prec != MDWF_F32 && prec != MDWF_F16N) return MDWF_EINVAL;
    if (!c->have_gauge) return MDWF_ENOGAUGE;
    if (c->dense_s) {
        set_error_message("mdwf_apply_noalloc: this context applies dense Ls x Ls tables, which are sized per call; "
                          "only the closed-form path is available without allocation");
        return MDWF_EINVAL;
    }
    const size_t fb = field_bytes(prec, c->g, nrhs);
    if (fb > kNoAllocFieldBytes) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "mdwf_apply_noalloc: an intermediate field of %zu bytes exceeds the fixed scratch of %zu bytes "
                 "per field (8 MiB)", fb, kNoAllocFieldBytes);
        set_error_message(msg);
        return MDWF_EINVAL;
    }
    // the masses: finite, and I = M+ + M- C invertible for each. The closed form
    // (Sec. 3) divides by M+ (1 + m (-r)^Ls), r = M-/M+, the determinant of one
    // chirality's I over M+^Ls; the same test as the dense tables' inversion.
    {
        const double Mp = c->b5 * (4.0 - c->M5) + 1.0, Mm = c->c5 * (4.0 - c->M5) - 1.0;
        const double scale = 1.0 + fabs(4.0 - c->M5) * fmax(fabs(c->b5), fabs(c->c5));
        for (int r = 0; r < nrhs; ++r) {
            const double m = mf_per_rhs ? mf_per_rhs[r] : c->mf;
            if (!isfinite(m)) {
                set_error_message("mdwf_apply_noalloc: a mass is not finite");
                return MDWF_EINVAL;
            }
            const double rr = Mm / Mp;
            double pw = 1.0;
            for (int s = 0; s < c->g.Ls; ++s) pw *= -rr;
            const double den = Mp * (1.0 + m * pw);
            if (!isfinite(den) || fabs(den) <= 1e-12 * scale) {
                set_error_message("the Ls x Ls matrix I = M+ + M- C is singular for these coefficients");
                return MDWF_EINVAL;
            }
        }
    }
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    NoAllocAddrs* a = nullptr;
    if ((st = noalloc_setup(c->device, &a))) return st;
    // masses of this call into the fixed arrays (stream-ordered before the kernels)
    NoAllocMasses ms{};
    ms.n = nrhs;
    for (int r = 0; r < nrhs; ++r) {
        ms.m64[r] = mf_per_rhs ? mf_per_rhs[r] : c->mf;
        ms.m32[r] = (float)ms.m64[r];
    }
    k_noalloc_masses<<<1, 64, 0, c->stream>>>(ms);
    if ((st = check_launch())) return st;
    void* z = a->scratch;
    void* v = a->scratch + kNoAllocFieldBytes;
    const void* mass = prec == MDWF_F64 ? (const void*)a->mass64 : (const void*)a->mass32;
    note_apply(c, prec);
    HopLaunch h{};
    h.nrhs = nrhs;
    h.b5 = c->b5;
    h.c5 = c->c5;
    h.mass = mass;
    if (!dagger) {
        M5Launch m{};  // v = M_phi psi (the first hop then needs no gather along s)
        m.out = v; m.in = in; m.x = nullptr; m.coef = 1.0; m.nrhs = nrhs; m.mass = mass;
        set_sop(c, prec, SOP_MPHI, 0, m);
        if ((st = launch_m5(c, prec, m))) return st;
        h.out = z; h.in = v; h.x = nullptr; h.coef = 1.0; h.out_parity = 0; h.gather = 0; h.dagger = 0;
        set_sop(c, prec, SOP_K, 0, h);
        if ((st = launch_hop(c, prec, h))) return st;
        h.out = out; h.in = z; h.x = in; h.coef = -0.25; h.out_parity = 1; h.gather = 0; h.dagger = 0;
        set_sop(c, prec, SOP_A, 0, h);
        return launch_hop(c, prec, h);
    }
    M5Launch m{};
    m.out = v; m.in = in; m.x = nullptr; m.coef = 1.0; m.nrhs = nrhs; m.mass = mass;
    set_sop(c, prec, SOP_A, 1, m);
    if ((st = launch_m5(c, prec, m))) return st;
    h.out = z; h.in = v; h.x = nullptr; h.coef = 1.0; h.out_parity = 0; h.gather = 0; h.dagger = 1;
    set_sop(c, prec, SOP_K, 1, h);
    if ((st = launch_hop(c, prec, h))) return st;
    h.out = out; h.in = z; h.x = in; h.coef = -0.25; h.out_parity = 1; h.gather = 0; h.dagger = 1;
    set_sop(c, prec, SOP_MPHI, 1, h);
    return launch_hop(c, prec, h);
}
