// Domain decomposition along t: one context per t-slab of the lattice.
//
// The fifth dimension is never split (Sec. 3: the Ls x Ls factors are
// site-local, so only the 4d hopping term couples slabs), and of the four
// directions only t is split, so a slab exchanges two faces per hopping term.
// What crosses a face is a half spinor (12 reals per 5d site and right-hand
// side), spin-projected by the slab that owns the site:
//   face 0 (t' = 0 slice) goes to the slab below, whose forward t-terms take
//          (1 + S g_4) psi there (S = -1 for D_W, +1 for D_W^dag);
//   face 1 (t' = T - 1 slice) goes to the slab above, whose backward t-terms
//          take U_4^dag (1 - S g_4) psi there; the link belongs to the sending
//          slab, so the sender multiplies by it.
// An operator application runs in three stages with two exchanges between
// them (mdwf_slab_stage): the caller moves face buffers from slab to slab
// (device copies for slabs on one GPU, NCCL or another transport across
// processes). The slab's intermediate fields live in its context between the
// stages.
#include "hop_kernel.cuh"

namespace mdwf {

// g[a][i] = sum_j U^dag[i][j] h[a][j] (U row-major complex 3 x 3): the
// backward term's transport, done by the slab that owns the link.
template <typename R>
__device__ __forceinline__ void transport_adj(const R* U, const R* h, R* g) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            R sr = 0, si = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const R ur = U[2 * (3 * j + i)], ui = -U[2 * (3 * j + i) + 1];
                const R hr = h[6 * a + 2 * j], hi = h[6 * a + 2 * j + 1];
                sr = fma(ur, hr, sr);
                sr = fma(-ui, hi, sr);
                si = fma(ur, hi, si);
                si = fma(ui, hr, si);
            }
            g[6 * a + 2 * i] = sr;
            g[6 * a + 2 * i + 1] = si;
        }
}

// send = [face 0 | face 1], each [rhs][face site][chunk of the half spinor][s]
// for the field `in` of parity in_parity (one thread per (face, rhs, site, s),
// s fastest so that the stores of a warp are contiguous).
template <int P, bool DAG>
__global__ void __launch_bounds__(256) k_slab_pack(void* send, Field<P> in, Gauge<P> U, Geom g, int in_parity,
                                                   int nrhs, long long face) {
    typedef typename PrecTraits<P>::real R;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int NCH = P == MDWF_F64 ? 6 : 3;  // chunks of a half spinor
    const long long n = 2LL * nrhs * face * g.Ls;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i % g.Ls);
        long long q = i / g.Ls;
        const long long f = q % face;
        q /= face;
        const int rhs = (int)(q % nrhs);
        const int dir = (int)(q / nrhs);
        const long long j = dir == 0 ? f : (long long)(g.T - 1) * face + f;
        R w[24], h[12];
        in.load((long long)rhs * g.Vh + j, s, w);
        if (dir == 0) {
            project<3, SF>(w, h);
        } else {
            R t[12], u[18];
            project<3, -SF>(w, t);
            U.load(((long long)in_parity * 4 + 3) * g.Vh + j, u);
            transport_adj(u, t, h);
        }
        const long long base = ((long long)dir * nrhs * face + (long long)rhs * face + f) * NCH * g.Ls + s;
        if constexpr (P == MDWF_F64) {
            double2* o = reinterpret_cast<double2*>(send) + base;
#pragma unroll
            for (int k = 0; k < 6; ++k) o[(long long)k * g.Ls] = make_double2(h[2 * k], h[2 * k + 1]);
        } else {
            float4* o = reinterpret_cast<float4*>(send) + base;
#pragma unroll
            for (int k = 0; k < 3; ++k) o[(long long)k * g.Ls] = make_float4(h[4 * k], h[4 * k + 1], h[4 * k + 2], h[4 * k + 3]);
        }
    }
}

static long long slab_face(const mdwf_ctx* c) { return (long long)c->g.X * c->g.Y * c->g.Z / 2; }

static size_t slab_face_bytes(const mdwf_ctx* c, int prec, int nrhs) {
    const size_t real = prec == MDWF_F64 ? sizeof(double) : sizeof(float);
    return 2 * (size_t)nrhs * (size_t)slab_face(c) * c->g.Ls * 12 * real;
}

template <int P>
static int launch_pack(mdwf_ctx* c, void* send, const void* in, int in_parity, int nrhs, int dagger) {
    const long long n = 2LL * nrhs * slab_face(c) * c->g.Ls;
    long long blocks = (n + 255) / 256;
    if (blocks > 152LL * 32) blocks = 152LL * 32;
    Gauge<P> U;
    U.u = reinterpret_cast<decltype(U.u)>(c->gauge[link_copy(P)]);
    U.bnd = make_bounds(8 * c->g.Vh);
    const double real = P == MDWF_F64 ? 8.0 : 4.0;
    LaunchScope scope(c, KB_LAYOUT * 3 + P, (double)n * (site_bytes(P) + 12.0 * real), (double)n * 12.0);
    Field<P> f = make_field<P>(const_cast<void*>(in), c->g, nrhs);
    if (dagger)
        k_slab_pack<P, true><<<(unsigned)blocks, 256, 0, c->stream>>>(send, f, U, c->g, in_parity, nrhs, slab_face(c));
    else
        k_slab_pack<P, false><<<(unsigned)blocks, 256, 0, c->stream>>>(send, f, U, c->g, in_parity, nrhs, slab_face(c));
    return check_launch();
}

static int pack(mdwf_ctx* c, int prec, void* send, const void* in, int in_parity, int nrhs, int dagger) {
    return prec == MDWF_F64 ? launch_pack<MDWF_F64>(c, send, in, in_parity, nrhs, dagger)
                            : launch_pack<MDWF_F32>(c, send, in, in_parity, nrhs, dagger);
}

}  // namespace mdwf

using namespace mdwf;

extern "C" size_t mdwf_slab_face_bytes(const mdwf_ctx* c, int prec, int nrhs) {
    if (!c || !c->slab || nrhs < 1 || (prec != MDWF_F64 && prec != MDWF_F32)) return 0;
    return slab_face_bytes(c, prec, nrhs);
}

extern "C" int mdwf_slab_stage(mdwf_ctx* c, int stage, void* out, const void* in, int prec, int nrhs,
                               const double* mf_per_rhs, int dagger, void* send, const void* recv) {
    NvtxRange nvtx_range("mdwf_slab_stage");
    if (!c || !c->slab) {
        set_error_message("mdwf_slab_stage: the context is not a t-slab (mdwf_create_slab)");
        return MDWF_EINVAL;
    }
    if (prec != MDWF_F64 && prec != MDWF_F32) {
        set_error_message("mdwf_slab_stage: FP64 and FP32 operators only");
        return MDWF_EINVAL;
    }
    if (nrhs < 1 || nrhs > kMaxRhs || stage < 0 || stage > 2) return MDWF_EINVAL;
    if ((stage == 0 && (!in || !send)) || (stage == 1 && (!send || !recv)) || (stage == 2 && (!out || !in || !recv)))
        return MDWF_EINVAL;
    if (!c->have_gauge) return MDWF_ENOGAUGE;
    if (c->sdep) {
        set_error_message("mdwf_slab_stage: per-slice coefficients are not supported on t-slabs");
        return MDWF_EINVAL;
    }
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    if ((st = ensure_tables(c, nrhs, mf_per_rhs))) return st;
    const size_t fb = field_bytes(prec, c->g, nrhs);
    if ((st = ensure_workspace(c->tmp[0], fb))) return st;
    if ((st = ensure_workspace(c->tmp[1], fb))) return st;
    const void* mass = prec == MDWF_F64 ? (const void*)c->mass64 : (const void*)c->mass32;
    if (stage == 0) {
        // the first factor on the odd input: w = M_phi psi (M) or v = A^dag psi (M^dag),
        // then its faces for the neighbours' first hop
        M5Launch m{};
        m.out = c->tmp[1].p; m.in = in; m.x = nullptr; m.coef = 1.0; m.nrhs = nrhs;
        set_sop(c, prec, dagger ? SOP_A : SOP_MPHI, dagger ? 1 : 0, m);
        if ((st = launch_m5(c, prec, m))) return st;
        return pack(c, prec, send, c->tmp[1].p, 1, nrhs, dagger);
    }
    HopLaunch h{};
    h.nrhs = nrhs;
    h.b5 = c->b5;
    h.c5 = c->c5;
    h.mass = mass;
    h.gather = 0;
    h.dagger = dagger ? 1 : 0;
    h.halo = recv;
    if (stage == 1) {
        // z_e = K H_eo w (M) or K^dag H'_eo v (M^dag), then its faces for the second hop
        h.out = c->tmp[0].p; h.in = c->tmp[1].p; h.x = nullptr; h.coef = 1.0; h.out_parity = 0;
        set_sop(c, prec, SOP_K, dagger ? 1 : 0, h);
        if ((st = launch_hop(c, prec, h))) return st;
        return pack(c, prec, send, c->tmp[0].p, 0, nrhs, dagger);
    }
    // out = psi - A H_oe z / 4 (M) or psi - M_phi^dag H'_oe z / 4 (M^dag)
    note_apply(c, prec);
    h.out = out; h.in = c->tmp[0].p; h.x = in; h.coef = -0.25; h.out_parity = 1;
    set_sop(c, prec, dagger ? SOP_MPHI : SOP_A, dagger ? 1 : 0, h);
    return launch_hop(c, prec, h);
}
