// CGNE on M^dag M for the red/black Moebius operator, plain FP64 or mixed
// precision with FP64 reliable updates, for a batch of right-hand sides.
//
// The paper solves with conjugate gradient (Sec. 2.3, Sec. 4) and measures
// cost in Dirac applications; the variant here is CG on the normal
// equations M^dag M x = M^dag b', with b' the red/black-preconditioned source
// of the Schur decomposition (Sec. 3). All CG scalars live on the device
// (alpha, beta, |r|^2 per right-hand side); the host only polls them every
// few iterations. Dot products and norms accumulate in FP64 through a
// two-pass reduction: per-block partials, then one block per right-hand side
// summing the partials in a fixed order, so results do not depend on timing.
//
// Mixed precision: the iteration runs with the operator in FP32 or FP16+norm
// (FP32 arithmetic) on p, M p, M^dag M p, with the iterated residual r_s and
// the correction x_s in FP32. When |r_s| drops below delta * max |r_s| since
// the last update (or below the target), x += x_s and the true residual
// r = M^dag b' - M^dag M x is recomputed with the FP64 operator; r_s = r.
// Each update corrects the search direction for the new residual, and an
// inner breakdown rolls back to the last update (run_mixed).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "mdwf_internal.cuh"

namespace mdwf {

constexpr int kRedThreads = 256;
#define SC(k, r) sc[(k) * kMaxRhs + (r)]

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? ws[lane] : 0.0;
    if (wid == 0) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    }
    return v;
}

#define SITE_LOOP(g)                                                                                 \
    const long long n5 = (g).Vh * (g).Ls;                                                            \
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n5;                     \
         i += (long long)gridDim.x * blockDim.x)

// |a|^2 per right-hand side -> partials
template <int PA>
__global__ void __launch_bounds__(kRedThreads) k_norm(Field<PA> a, double* part, Geom g, const double* sc) {
    typedef typename PrecTraits<PA>::real RA;
    const int rhs = blockIdx.y;
    double acc = 0;
    if (!sc || SC(S_ACTIVE, rhs) != 0.0) {
        SITE_LOOP(g) {
            const int s = (int)(i % g.Ls);
            const long long sr = rhs * g.Vh + i / g.Ls;
            RA v[24];
            a.load(sr, s, v);
#pragma unroll
            for (int k = 0; k < 24; ++k) acc += (double)v[k] * (double)v[k];
        }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[rhs * gridDim.x + blockIdx.x] = acc;
}

// One block of kFinThreads per right-hand side sums the nb partials in a
// fixed order (four independent running sums per thread, so that the loads
// of a thread are in flight together), then updates the CG scalars.
// late = 1: the partials come from the kernel before the previous one, which
// the previous kernel waited for before it let this one start; the block then
// runs beside the previous kernel's end and waits for it only before it exits.
constexpr int kFinThreads = 1024;

__global__ void __launch_bounds__(kFinThreads) k_finalize(const double* part, int nb, double* sc, int mode, int slot,
                                                          int late) {
    if (!late) pdl_wait();  // the partials come from the kernel before
    pdl_release();
    const int rhs = blockIdx.x;
    const double* pp = part + (size_t)rhs * nb;
    const int bd = blockDim.x;
    double v0 = 0, v1 = 0, v2 = 0, v3 = 0;
    int i = threadIdx.x;
    for (; i + 3 * bd < nb; i += 4 * bd) {
        v0 += pp[i];
        v1 += pp[i + bd];
        v2 += pp[i + 2 * bd];
        v3 += pp[i + 3 * bd];
    }
    for (; i < nb; i += bd) v0 += pp[i];
    double v = block_sum((v0 + v1) + (v2 + v3));
    if (threadIdx.x == 0) cg_scalar_update(sc, rhs, mode, slot, v);
    if (late) pdl_wait();  // complete after the previous kernel
}

// Column-blocked update for the fused iteration: block = (Ls, SB) threads
// covering SB whole s-columns. x += alpha p; p = r + beta p; then
// w = M_phi p = b5 p_s + c5 (P+ p_{s-1} + P- p_{s+1}) (mass -m on the
// wrap-around) with the new p of the neighbouring slices taken from shared
// memory, so that the first hop of the next iteration reads w without
// gathering along s. With per-slice coefficients gs holds the gather factors
// of row s, [gown][gfac][gscale] (64 each): b5(s) = gscale gown and
// c5(s) = gscale gfac.
template <int PX, int PR, int PP>
__global__ void __launch_bounds__(128) k_pupd_w(Field<PX> x, Field<PR> r, Field<PP> p, Field<PP> w,
                                               const double* sc, const typename PrecTraits<PP>::real* mass,
                                               const typename PrecTraits<PP>::real* gs, Geom g, double b5,
                                               double c5) {
    typedef typename PrecTraits<PX>::real RX;
    typedef typename PrecTraits<PR>::real RR;
    typedef typename PrecTraits<PP>::real RP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RP* hs = reinterpret_cast<RP*>(smem_raw);
    pdl_wait();  // r and the CG scalars come from the kernels before
    pdl_release();
    const int rhs = blockIdx.y;
    if (SC(S_ACTIVE, rhs) == 0.0) return;  // uniform over the block
    const int Ls = g.Ls, s = threadIdx.x, ly = threadIdx.y;
    const long long site = (long long)blockIdx.x * blockDim.y + ly;
    const bool active = site < g.Vh;
    const long long sr = (long long)rhs * g.Vh + site;
    const double alpha = SC(S_ALPHA, rhs);
    const RP beta = (RP)SC(S_BETA, rhs);
    const int sst = site_stride(Ls);
    RP* row = hs + (size_t)ly * sst;
    RP pv[24];
    if (active) {
        RX xv[24];
        RR rv[24];
        x.load(sr, s, xv);
        r.load(sr, s, rv);
        p.load(sr, s, pv);
#pragma unroll
        for (int k = 0; k < 24; ++k) {
            xv[k] += (RX)alpha * (RX)pv[k];
            pv[k] = (RP)rv[k] + beta * pv[k];
        }
        x.store(sr, s, xv);
        p.store(sr, s, pv);
    } else {
#pragma unroll
        for (int k = 0; k < 24; ++k) pv[k] = 0;
    }
    row_store(row + s * kRowStride, pv);
    __syncthreads();
    if (!active) return;
    const RP m = mass[rhs];
    const int sm = s > 0 ? s - 1 : Ls - 1, sp = s < Ls - 1 ? s + 1 : 0;
    RP bs = (RP)b5, cs = (RP)c5;
    if (gs) {
        bs = gs[128 + s] * gs[s];
        cs = gs[128 + s] * gs[64 + s];
    }
    const RP fm = cs * (s > 0 ? RP(1) : -m), fp = cs * (s < Ls - 1 ? RP(1) : -m);
    RP wv[24];
#pragma unroll
    for (int k = 0; k < 12; ++k) wv[k] = bs * pv[k] + fm * row[sm * kRowStride + k];
#pragma unroll
    for (int k = 12; k < 24; ++k) wv[k] = bs * pv[k] + fp * row[sp * kRowStride + k];
    w.store(sr, s, wv);
}

// dst = src (precision conversion); when sc != null only the right-hand sides
// whose flag in slot `slot` is set
template <int PD, int PS>
__global__ void __launch_bounds__(kRedThreads) k_copy(Field<PD> d, Field<PS> src, const double* sc, int slot,
                                                      Geom g) {
    typedef typename PrecTraits<PD>::real RD;
    typedef typename PrecTraits<PS>::real RS;
    const int rhs = blockIdx.y;
    if (sc && SC(slot, rhs) == 0.0) return;
    SITE_LOOP(g) {
        const int s = (int)(i % g.Ls);
        const long long sr = rhs * g.Vh + i / g.Ls;
        RS v[24];
        RD w[24];
        src.load(sr, s, v);
#pragma unroll
        for (int k = 0; k < 24; ++k) w[k] = (RD)v[k];
        d.store(sr, s, w);
    }
}

// x = 0 for the right-hand sides whose flag in slot `slot` is set
template <int P>
__global__ void __launch_bounds__(kRedThreads) k_zero(Field<P> x, const double* sc, int slot, Geom g) {
    typedef typename PrecTraits<P>::real R;
    const int rhs = blockIdx.y;
    if (SC(slot, rhs) == 0.0) return;
    R z[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) z[k] = R(0);
    SITE_LOOP(g) {
        const int s = (int)(i % g.Ls);
        x.store(rhs * g.Vh + i / g.Ls, s, z);
    }
}

// d = c1 a + c2 b with c1, c2 from slots S_C1, S_C2 (the right-hand sides whose
// flag in slot `slot` is set); d may alias a or b element by element
template <int PD, int PA, int PB>
__global__ void __launch_bounds__(kRedThreads) k_lincomb(Field<PD> d, Field<PA> a, Field<PB> b, const double* sc,
                                                         int slot, Geom g) {
    typedef typename PrecTraits<PD>::real RD;
    typedef typename PrecTraits<PA>::real RA;
    typedef typename PrecTraits<PB>::real RB;
    const int rhs = blockIdx.y;
    if (SC(slot, rhs) == 0.0) return;
    // in the output's arithmetic precision (FP64 arithmetic on FP32 data would run on
    // a pipe at 1/64 of the FP32 rate)
    const RD c1 = (RD)SC(S_C1, rhs), c2 = (RD)SC(S_C2, rhs);
    SITE_LOOP(g) {
        const int s = (int)(i % g.Ls);
        const long long sr = rhs * g.Vh + i / g.Ls;
        RA av[24];
        RB bv[24];
        RD dv[24];
        a.load(sr, s, av);
        b.load(sr, s, bv);
        if (c2 != RD(0)) {
#pragma unroll
            for (int k = 0; k < 24; ++k) dv[k] = fma(c1, (RD)av[k], c2 * (RD)bv[k]);
        } else {  // b not used (it may hold non-finite values)
#pragma unroll
            for (int k = 0; k < 24; ++k) dv[k] = c1 * (RD)av[k];
        }
        d.store(sr, s, dv);
    }
}

// Re <a, b> per right-hand side (flag in slot `slot` set; 0 otherwise) -> partials
template <int PA, int PB>
__global__ void __launch_bounds__(kRedThreads) k_dot2(Field<PA> a, Field<PB> b, double* part, const double* sc,
                                                      int slot, Geom g) {
    typedef typename PrecTraits<PA>::real RA;
    typedef typename PrecTraits<PB>::real RB;
    typedef decltype(RA(0) * RB(0)) RP;  // FP32 products of FP32 / FP16+norm fields
    const int rhs = blockIdx.y;
    double acc = 0;
    if (SC(slot, rhs) != 0.0) {
        SITE_LOOP(g) {
            const int s = (int)(i % g.Ls);
            const long long sr = rhs * g.Vh + i / g.Ls;
            RA av[24];
            RB bv[24];
            a.load(sr, s, av);
            b.load(sr, s, bv);
            RP t = 0;  // a site's 24 products in the fields' precision, the sum over sites in FP64
#pragma unroll
            for (int k = 0; k < 24; ++k) t = fma((RP)av[k], (RP)bv[k], t);
            acc += (double)t;
        }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[rhs * gridDim.x + blockIdx.x] = acc;
}

// y += x; x = 0 (the right-hand sides whose flag in slot `slot` is set)
template <int PY, int PX>
__global__ void __launch_bounds__(kRedThreads) k_accum_zero(Field<PY> y, Field<PX> x, const double* sc, int slot,
                                                            Geom g) {
    typedef typename PrecTraits<PY>::real RY;
    typedef typename PrecTraits<PX>::real RX;
    const int rhs = blockIdx.y;
    if (SC(slot, rhs) == 0.0) return;
    SITE_LOOP(g) {
        const int s = (int)(i % g.Ls);
        const long long sr = rhs * g.Vh + i / g.Ls;
        RY yv[24];
        RX xv[24];
        y.load(sr, s, yv);
        x.load(sr, s, xv);
#pragma unroll
        for (int k = 0; k < 24; ++k) {
            yv[k] += (RY)xv[k];
            xv[k] = 0;
        }
        y.store(sr, s, yv);
        x.store(sr, s, xv);
    }
}

// r = a - b (FP64), optional low-precision copy rs = r; partial |r|^2 (the
// right-hand sides whose flag in slot `slot` is set, or all when sc is null)
template <int PS, bool COPY>
__global__ void __launch_bounds__(kRedThreads) k_residual(Field<MDWF_F64> r, Field<PS> rs, Field<MDWF_F64> a,
                                                         Field<MDWF_F64> b, double* part, const double* sc,
                                                         int slot, Geom g) {
    typedef typename PrecTraits<PS>::real RS;
    const int rhs = blockIdx.y;
    double acc = 0;
    if (!sc || SC(slot, rhs) != 0.0) {
        SITE_LOOP(g) {
            const int s = (int)(i % g.Ls);
            const long long sr = rhs * g.Vh + i / g.Ls;
            double av[24], bv[24];
            a.load(sr, s, av);
            b.load(sr, s, bv);
#pragma unroll
            for (int k = 0; k < 24; ++k) {
                av[k] -= bv[k];
                acc += av[k] * av[k];
            }
            r.store(sr, s, av);
            if (COPY) {
                RS w[24];
#pragma unroll
                for (int k = 0; k < 24; ++k) w[k] = (RS)av[k];
                rs.store(sr, s, w);
            }
        }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[rhs * gridDim.x + blockIdx.x] = acc;
}

// ------------------------------------------------------------------ solver

namespace {

struct Solver {
    mdwf_ctx* c;
    Geom g;
    int nrhs;
    int nb;             // reduction blocks per right-hand side
    double* sc;         // device scalars [S_NUM][kMaxRhs]
    double* part;       // device partials [nrhs][nb]
    double* hpart;      // partials of the fused hop epilogues [nrhs][hop blocks]
    int hb;             // hop blocks per right-hand side
    double* hsc;        // pinned host copy of sc

    dim3 grid() const { return dim3(nb, nrhs); }

    double n5() const { return (double)g.Vh * g.Ls * nrhs; }
    int fin(int mode, int slot = 0) {
        LaunchScope scope(c, KB_BLAS * 3 + MDWF_F64, 8.0 * nrhs * nb, 0.0);
        if (cudaError_t e = launch_pdl(k_finalize, dim3(nrhs), dim3(kFinThreads), 0, c->stream, part, nb, sc, mode,
                                       slot, 0))
            return cuda_status(e);
        return check_launch();
    }
    // late: the partials come from the hop before the previous one (see k_finalize)
    int fin_hop(int mode, int late = 0) {
        LaunchScope scope(c, KB_BLAS * 3 + MDWF_F64, 8.0 * nrhs * hb, 0.0);
        if (cudaError_t e = launch_pdl(k_finalize, dim3(nrhs), dim3(kFinThreads), 0, c->stream, hpart, hb, sc, mode,
                                       0, late))
            return cuda_status(e);
        return check_launch();
    }
    template <int P>
    int norm(const void* a, bool masked, int slot) {
        {
        LaunchScope scope(c, KB_BLAS * 3 + P, n5() * site_bytes(P), n5() * 48.0);
        k_norm<P><<<grid(), kRedThreads, 0, c->stream>>>(make_field<P>(const_cast<void*>(a), g, nrhs), part, g,
                                                         masked ? sc : nullptr);
        }
        int st = check_launch();
        return st ? st : fin(FIN_STORE, slot);
    }
    template <int PD, int PS>
    int copy(void* d, const void* s, bool masked, int slot = S_ACTIVE) {
        LaunchScope scope(c, KB_BLAS * 3 + PD, n5() * (site_bytes(PS) + site_bytes(PD)), 0.0);
        k_copy<PD, PS><<<grid(), kRedThreads, 0, c->stream>>>(make_field<PD>(d, g, nrhs),
                                                               make_field<PS>(const_cast<void*>(s), g, nrhs),
                                                               masked ? sc : nullptr, slot, g);
        return check_launch();
    }
    template <int PD, int PA, int PB>
    int lincomb(void* d, const void* a, const void* b, int slot) {
        LaunchScope scope(c, KB_BLAS * 3 + PD, n5() * (site_bytes(PA) + site_bytes(PB) + site_bytes(PD)),
                          n5() * 72.0);
        k_lincomb<PD, PA, PB><<<grid(), kRedThreads, 0, c->stream>>>(
            make_field<PD>(d, g, nrhs), make_field<PA>(const_cast<void*>(a), g, nrhs),
            make_field<PB>(const_cast<void*>(b), g, nrhs), sc, slot, g);
        return check_launch();
    }
    template <int PA, int PB>
    int dot(const void* a, const void* b, int mask_slot, int out_slot) {
        {
            LaunchScope scope(c, KB_BLAS * 3 + PB, n5() * (site_bytes(PA) + site_bytes(PB)), n5() * 48.0);
            k_dot2<PA, PB><<<grid(), kRedThreads, 0, c->stream>>>(make_field<PA>(const_cast<void*>(a), g, nrhs),
                                                                   make_field<PB>(const_cast<void*>(b), g, nrhs), part,
                                                                   sc, mask_slot, g);
        }
        int st = check_launch();
        return st ? st : fin(FIN_STORE, out_slot);
    }
    int pull() {
        int st = cuda_status(cudaMemcpyAsync(hsc, sc, sizeof(double) * S_NUM * kMaxRhs, cudaMemcpyDeviceToHost,
                                             c->stream));
        return st ? st : cuda_status(cudaStreamSynchronize(c->stream));
    }
    int push() {
        return cuda_status(cudaMemcpyAsync(sc, hsc, sizeof(double) * S_NUM * kMaxRhs, cudaMemcpyHostToDevice,
                                           c->stream));
    }
};

void begin_capture(mdwf_ctx* c) {
    c->capturing = true;
    c->cap_launches = 0;
    for (int p = 0; p < 3; ++p) c->cap_applies[p] = 0;
    for (int k = 0; k < KK_NUM; ++k) c->cap_kstat[k] = KStat{};
}

}  // namespace

struct Fields {
    // FP64: solution, right-hand side of the normal equations, residual, operator temporary
    void *xo, *src, *r, *t64;
    // inner iteration (w = M_phi p, read by the first hop)
    void *xs, *rs, *p, *t, *w;
};

template <int PR, int PP>
static int launch_pupd_w(Solver& S, void* x, void* r, void* p, void* w) {
    mdwf_ctx* c = S.c;
    typedef typename PrecTraits<PP>::real RP;
    const int SB = (128 / S.g.Ls) < 1 ? 1 : 128 / S.g.Ls;
    dim3 block(S.g.Ls, SB), grid((unsigned)((S.g.Vh + SB - 1) / SB), S.nrhs);
    const size_t smem = (size_t)SB * site_stride(S.g.Ls) * sizeof(RP);
    const RP* mass = reinterpret_cast<const RP*>(PP == MDWF_F64 ? (const void*)c->mass64 : (const void*)c->mass32);
    const RP* gs = !c->sdep ? nullptr
                            : reinterpret_cast<const RP*>(PP == MDWF_F64 ? (const void*)c->gs64 : (const void*)c->gs32);
    LaunchScope scope(c, KB_BLAS * 3 + PP, S.n5() * (3.0 * site_bytes(PR) + 3.0 * site_bytes(PP)), S.n5() * 144.0);
    if (cudaError_t e = launch_pdl(k_pupd_w<PR, PR, PP>, grid, block, smem, c->stream, make_field<PR>(x, S.g, S.nrhs),
                                   make_field<PR>(r, S.g, S.nrhs), make_field<PP>(p, S.g, S.nrhs),
                                   make_field<PP>(w, S.g, S.nrhs), (const double*)S.sc, mass, gs, S.g, c->b5, c->c5))
        return cuda_status(e);
    return check_launch();
}

// w = M_phi p (the fused iteration's first hop reads w); with a mask, only the
// right-hand sides whose entry is nonzero
template <int PP>
static int init_w(Solver& S, void* w, const void* p, const double* mask = nullptr) {
    M5Launch m{};
    m.out = w; m.in = p; m.x = nullptr; m.coef = 1.0; m.nrhs = S.nrhs; m.mask = mask;
    set_sop(S.c, PP, SOP_MPHI, 0, m);
    return launch_m5(S.c, PP, m);
}

// One CG iteration on M^dag M with the BLAS folded into the operator kernels
// (structured s-operators or dense tables alike):
//   z = K H_eo M_phi p;  t = p - 1/4 A H_oe z, v = A^dag t, |t|^2 (-> alpha);
//   z = K^dag H'_eo v;   r -= alpha (t - 1/4 M_phi^dag H'_oe z), |r|^2 (-> beta);
//   x += alpha p, p = r + beta p.
//   Where the closed-form s-operators run by shuffles (Ls = 16), t is not
//   stored: K2' forms it again as t = I^dag v from v = A^dag t, a bidiagonal
//   s-operator, which saves one field write per iteration.
template <int PR, int PP>
static int cg_iteration_fused(Solver& S, void* x, void* r, void* p, void* t, void* w) {
    mdwf_ctx* c = S.c;
    int st;
    note_apply(c, PP);
    note_apply(c, PP);
    const bool no_t = hop_no_t_ok(c, PP, S.nrhs);
    HopLaunch h{};
    h.nrhs = S.nrhs;
    h.b5 = c->b5;
    h.c5 = c->c5;
    h.mass = PP == MDWF_F64 ? (const void*)c->mass64 : (const void*)c->mass32;
    // z = K H_eo w, w = M_phi p (formed by the previous update)
    h.out = c->tmp[0].p; h.in = w; h.x = nullptr; h.coef = 1.0; h.out_parity = 0; h.gather = 0; h.dagger = 0;
    set_sop(c, PP, SOP_K, 0, h);
    if ((st = launch_hop(c, PP, h))) return st;
    h.out = t; h.in = c->tmp[0].p; h.x = p; h.coef = -0.25; h.out_parity = 1; h.gather = 0; h.dagger = 0;
    set_sop(c, PP, SOP_A, 0, h);
    h.mat2 = nullptr;
    if (h.sop == SOP_DENSE) {  // the table of A^dag for v
        HopLaunch a{};
        set_sop(c, PP, SOP_A, 1, a);
        h.mat2 = a.mat;
    }
    h.fuse = 1; h.out2 = c->tmp[1].p; h.part = S.hpart; h.sc = S.sc; h.no_t = no_t;
    if ((st = launch_hop(c, PP, h))) return st;
    h.mat2 = nullptr;
    h.no_t = 0;
    // K1' does not need alpha, so alpha is formed after it is launched, beside its end
    h.out = c->tmp[0].p; h.in = c->tmp[1].p; h.x = nullptr; h.coef = 1.0; h.out_parity = 0; h.dagger = 1;
    set_sop(c, PP, SOP_K, 1, h);
    h.fuse = 0;
    if ((st = launch_hop(c, PP, h))) return st;
    if ((st = S.fin_hop(FIN_ALPHA, 1))) return st;
    h.out = c->tmp[1].p; h.in = c->tmp[0].p; h.x = no_t ? c->tmp[1].p : t; h.coef = -0.25; h.out_parity = 1;
    h.dagger = 1;
    set_sop(c, PP, SOP_MPHI, 1, h);
    h.fuse = 2; h.rfield = r; h.part = S.hpart; h.sc = S.sc; h.no_t = no_t;
    if ((st = launch_hop(c, PP, h))) return st;
    if ((st = S.fin_hop(FIN_BETA))) return st;
    return launch_pupd_w<PR, PP>(S, x, r, p, w);
}

template <int PR, int PP>
static int iterate(Solver& S, Fields& F, void* x, void* r) {
    return cg_iteration_fused<PR, PP>(S, x, r, F.p, F.t, F.w);
}

// r = src - M^dag M x in FP64 (active rhs), r_s = r in precision PS; |r|^2 -> S_AUX.
// M^dag M x is formed in r itself (each element is read before it is
// overwritten by the same thread), so no further FP64 field is needed; r of
// an inactive right-hand side is left holding M^dag M x and is not used again.
// only_updating: just the right-hand sides flagged in S_UPD (the operator's
// blocks of the others do nothing, and their r and r_s stay as they are).
template <int PS, bool COPY>
static int true_residual(Solver& S, void* r, void* rs, const void* src, const void* x, void* t64, bool masked,
                         bool only_updating = false) {
    int st;
    const double* mask = only_updating ? S.sc + S_UPD * kMaxRhs : nullptr;
    if ((st = apply_op(S.c, t64, x, MDWF_F64, S.nrhs, 0, 0, mask))) return st;
    if ((st = apply_op(S.c, r, t64, MDWF_F64, S.nrhs, 1, 0, mask))) return st;
    {
    LaunchScope scope(S.c, KB_BLAS * 3 + MDWF_F64, S.n5() * (3.0 * 192.0 + (COPY ? site_bytes(PS) : 0.0)), S.n5() * 48.0);
    k_residual<PS, COPY><<<S.grid(), kRedThreads, 0, S.c->stream>>>(
        make_field<MDWF_F64>(r, S.g, S.nrhs), make_field<PS>(rs ? rs : r, S.g, S.nrhs),
        make_field<MDWF_F64>(const_cast<void*>(src), S.g, S.nrhs), make_field<MDWF_F64>(r, S.g, S.nrhs), S.part,
        (masked || only_updating) ? S.sc : nullptr, only_updating ? S_UPD : S_ACTIVE, S.g);
    }
    if ((st = check_launch())) return st;
    return S.fin(FIN_STORE, S_AUX);
}


// last_true[r] receives |src - M^dag M x|^2 of the FP64 solution x each time
// it is recomputed; x changes only at those points, so the final value
// belongs to the returned x.
template <int PP>
static int run_mixed(Solver& S, Fields& F, const mdwf_solve_params& prm, double tol, int maxiter,
                     std::vector<double>& maxr, std::vector<int>& rupd, std::vector<int>& restarts,
                     std::vector<double>& last_true, cudaGraphExec_t* gexec, bool use_graph) {
    mdwf_ctx* c = S.c;
    const int nrhs = S.nrhs;
    int st;
    // r = src - M^dag M x (x = 0: r = src), r_s = r, x_s = 0, p = r_s
    if ((st = cuda_status(cudaMemsetAsync(F.xs, 0, field_bytes(MDWF_F32, S.g, nrhs), c->stream)))) return st;
    if (prm.guess) {
        if ((st = true_residual<MDWF_F32, true>(S, F.r, F.rs, F.src, F.xo, F.t64, true))) return st;
        if ((st = S.pull())) return st;
        for (int r = 0; r < nrhs; ++r) {
            if (S.hsc[S_ACTIVE * kMaxRhs + r] == 0.0) continue;
            const double rr = S.hsc[S_AUX * kMaxRhs + r];
            S.hsc[S_RR * kMaxRhs + r] = rr;
            if (rr <= tol * tol * S.hsc[S_SRC2 * kMaxRhs + r]) S.hsc[S_ACTIVE * kMaxRhs + r] = 0.0;
        }
        if ((st = S.push())) return st;
        if ((st = S.copy<PP, MDWF_F64>(F.p, F.r, false))) return st;
    } else {
        if ((st = S.copy<MDWF_F64, MDWF_F64>(F.r, F.src, false))) return st;
        if ((st = S.copy<MDWF_F32, MDWF_F64>(F.rs, F.src, false))) return st;
        if ((st = S.copy<PP, MDWF_F64>(F.p, F.src, false))) return st;
        if ((st = S.norm<MDWF_F64>(F.src, false, S_RR))) return st;
    }
    if ((st = init_w<PP>(S, F.w, F.p))) return st;
    if ((st = S.pull())) return st;
    for (int r = 0; r < nrhs; ++r) {
        maxr[r] = sqrt(S.hsc[S_RR * kMaxRhs + r]);
        last_true[r] = S.hsc[S_RR * kMaxRhs + r];
    }
    // FP32 carries ~7 digits, so it can reduce the residual 100x between FP64
    // updates; FP16 storage only ~3, so it updates after every 10x
    const double delta = prm.delta > 0 ? prm.delta : (PP == MDWF_F32 ? 0.005 : 0.1);
    // At a reliable update the search direction is corrected for the new residual.
    // With d = p - r_s = beta p_prev (formed by the last vector update), p_prev
    // loses its component along the true r (in exact CG r is orthogonal to p_prev;
    // after drift it is not), and beta takes the true |r|^2: p = r + gamma (d - c r)
    // with gamma = |r|^2 / |r_s|^2 and c = <r, d> / |r|^2 (real parts: the CG runs
    // on the real vector space of the fields). Where the true |r| exceeds the inner
    // one more than twice (a small delta let the inner recurrence run far below
    // what its precision carries), p restarts from r instead. An update is also
    // forced when the inner |r| climbs 100x above the last true one. An inner
    // breakdown (non-positive or non-finite <p, M^dag M p>) rolls back to the last
    // update: x_s dropped, r_s = r, p = r, and the inner iterations between updates
    // capped at half of the interval that broke down; after kMaxRollbacks of them,
    // or from a non-finite residual, the right-hand side ends with MDWF_EBREAKDOWN.
    constexpr double kDiverge2 = 1e4, kRestartRatio2 = 4.0;
    constexpr int kMaxRollbacks = 8, kMinInterval = 16;
    std::vector<int> since(nrhs, 0), cap(nrhs, maxiter), rollbacks(nrhs, 0);
    const int every = prm.check_every > 0 ? prm.check_every : 8;
    int it = 0;
    bool graph_ready = false;
    while (it < maxiter) {
        const int steps = (maxiter - it) < every ? (maxiter - it) : every;
        if (use_graph) {
            if (!graph_ready) {
                cudaGraph_t graph;
                if ((st = cuda_status(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal)))) return st;
                begin_capture(c);
                int st2 = iterate<MDWF_F32, PP>(S, F, F.xs, F.rs);
                c->capturing = false;
                st = cuda_status(cudaStreamEndCapture(c->stream, &graph));
                if (st2) return st2;
                if (st) return st;
                st = cuda_status(cudaGraphInstantiate(gexec, graph, 0));
                cudaGraphDestroy(graph);
                if (st) return st;
                graph_ready = true;
            }
            for (int k = 0; k < steps; ++k) {
                if ((st = cuda_status(cudaGraphLaunch(*gexec, c->stream)))) return st;
                replay_graph_counts(c, 1);
            }
        } else {
            for (int k = 0; k < steps; ++k)
                if ((st = iterate<MDWF_F32, PP>(S, F, F.xs, F.rs))) return st;
        }
        it += steps;
        if ((st = S.pull())) return st;
        // a right-hand side takes its FP64 reliable update when its inner residual has
        // fallen by delta since its last one (or the inner estimate says it has
        // converged, or the iterations run out, or a safeguard fires); the others go on
        // untouched, so in a batch of masses each pays only for its own updates
        bool any_active = false, need_update = false, any_rollback = false;
        for (int r = 0; r < nrhs; ++r) {
            double* h = S.hsc + r;  // h[slot * kMaxRhs]
            h[S_UPD * kMaxRhs] = 0.0;
            h[S_RESTART * kMaxRhs] = 0.0;
            if (h[S_ACTIVE * kMaxRhs] == 0.0) {
                if (h[S_STATUS * kMaxRhs] == (double)MDWF_EBREAKDOWN && rollbacks[r] < kMaxRollbacks &&
                    std::isfinite(last_true[r]) && it < maxiter) {
                    rollbacks[r] += 1;
                    restarts[r] += 1;
                    cap[r] = std::max(kMinInterval, since[r] / 2);
                    since[r] = 0;
                    h[S_STATUS * kMaxRhs] = (double)MDWF_OK;
                    h[S_ACTIVE * kMaxRhs] = 1.0;
                    h[S_RR * kMaxRhs] = last_true[r];
                    maxr[r] = sqrt(last_true[r]);
                    h[S_RESTART * kMaxRhs] = 1.0;
                    any_rollback = true;
                    any_active = true;
                }
                continue;
            }
            any_active = true;
            since[r] += steps;
            const double rr = h[S_RR * kMaxRhs];
            const double src2 = h[S_SRC2 * kMaxRhs];
            const double rn = sqrt(rr);
            if (rn < delta * maxr[r] || rr <= tol * tol * src2 || it >= maxiter || since[r] >= cap[r] ||
                rr > kDiverge2 * last_true[r]) {
                h[S_UPD * kMaxRhs] = 1.0;
                h[S_C1 * kMaxRhs] = 1.0;
                h[S_C2 * kMaxRhs] = -1.0;
                need_update = true;
            }
            if (rn > maxr[r]) maxr[r] = rn;
        }
        if (!any_active) break;
        if (!need_update && !any_rollback) continue;
        if ((st = S.push())) return st;
        if (need_update) {
            // reliable update of the flagged right-hand sides: d = p - r_s (into w, which
            // is formed again below), x += x_s, x_s = 0, r = src - M^dag M x (FP64),
            // r_s = r, then the corrected p
            NvtxRange nvtx_update("reliable update");
            if ((st = S.lincomb<PP, PP, MDWF_F32>(F.w, F.p, F.rs, S_UPD))) return st;
            {
                LaunchScope scope(c, KB_BLAS * 3 + MDWF_F64, S.n5() * (2.0 * 192.0 + 2.0 * 96.0), S.n5() * 24.0);
                k_accum_zero<MDWF_F64, MDWF_F32><<<S.grid(), kRedThreads, 0, c->stream>>>(
                    make_field<MDWF_F64>(F.xo, S.g, nrhs), make_field<MDWF_F32>(F.xs, S.g, nrhs), S.sc, S_UPD, S.g);
            }
            if ((st = check_launch())) return st;
            if ((st = true_residual<MDWF_F32, true>(S, F.r, F.rs, F.src, F.xo, F.t64, true, true))) return st;
            if ((st = S.dot<MDWF_F32, PP>(F.rs, F.w, S_UPD, S_C1))) return st;
            if ((st = S.pull())) return st;
            for (int r = 0; r < nrhs; ++r) {
                double* h = S.hsc + r;
                if (h[S_ACTIVE * kMaxRhs] == 0.0 || h[S_UPD * kMaxRhs] == 0.0) continue;
                rupd[r] += 1;
                since[r] = 0;
                const double rr = h[S_AUX * kMaxRhs];
                const double rr_inner = h[S_RR * kMaxRhs];
                const double rd = h[S_C1 * kMaxRhs];
                const double src2 = h[S_SRC2 * kMaxRhs];
                last_true[r] = rr;
                h[S_RR * kMaxRhs] = rr;
                maxr[r] = sqrt(rr);
                if (rr <= tol * tol * src2) {
                    h[S_ACTIVE * kMaxRhs] = 0.0;
                    h[S_C1 * kMaxRhs] = 1.0;
                    h[S_C2 * kMaxRhs] = 0.0;
                    continue;
                }
                const double gamma = rr / rr_inner, cr = rd / rr;
                if (rr <= kRestartRatio2 * rr_inner && std::isfinite(gamma) && std::isfinite(cr)) {
                    h[S_C1 * kMaxRhs] = 1.0 - gamma * cr;  // p = (1 - gamma c) r + gamma d
                    h[S_C2 * kMaxRhs] = gamma;
                } else {
                    h[S_C1 * kMaxRhs] = 1.0;  // p = r
                    h[S_C2 * kMaxRhs] = 0.0;
                    restarts[r] += 1;
                }
            }
            if ((st = S.push())) return st;
            if ((st = S.lincomb<PP, MDWF_F32, PP>(F.p, F.rs, F.w, S_UPD))) return st;
            if ((st = init_w<PP>(S, F.w, F.p, S.sc + S_UPD * kMaxRhs))) return st;
        }
        if (any_rollback) {
            // x_s = 0, r_s = r, p = r, w = M_phi p for the right-hand sides rolled back
            {
                LaunchScope scope(c, KB_BLAS * 3 + MDWF_F32, S.n5() * 96.0, 0.0);
                k_zero<MDWF_F32><<<S.grid(), kRedThreads, 0, c->stream>>>(make_field<MDWF_F32>(F.xs, S.g, nrhs), S.sc,
                                                                          S_RESTART, S.g);
            }
            if ((st = check_launch())) return st;
            if ((st = S.copy<MDWF_F32, MDWF_F64>(F.rs, F.r, true, S_RESTART))) return st;
            if ((st = S.copy<PP, MDWF_F64>(F.p, F.r, true, S_RESTART))) return st;
            if ((st = init_w<PP>(S, F.w, F.p, S.sc + S_RESTART * kMaxRhs))) return st;
        }
    }
    return MDWF_OK;
}

static int run_plain(Solver& S, Fields& F, const mdwf_solve_params& prm, double tol, int maxiter,
                     std::vector<double>& last_true, cudaGraphExec_t* gexec, bool use_graph) {
    mdwf_ctx* c = S.c;
    const int nrhs = S.nrhs;
    int st;
    const int every = prm.check_every > 0 ? prm.check_every : 8;
    int it = 0;
    bool graph_ready = false;
    for (;;) {
        // (re)start from the true residual of the current x
        if ((st = true_residual<MDWF_F64, false>(S, F.r, nullptr, F.src, F.xo, F.t64, true))) return st;
        if ((st = S.pull())) return st;
        bool any = false;
        for (int r = 0; r < nrhs; ++r) {
            if (S.hsc[S_ACTIVE * kMaxRhs + r] == 0.0) continue;
            const double rr = S.hsc[S_AUX * kMaxRhs + r];
            last_true[r] = rr;
            S.hsc[S_RR * kMaxRhs + r] = rr;
            if (rr <= tol * tol * S.hsc[S_SRC2 * kMaxRhs + r]) S.hsc[S_ACTIVE * kMaxRhs + r] = 0.0;
            else any = true;
        }
        if ((st = S.push())) return st;
        if (!any || it >= maxiter) break;
        if ((st = S.copy<MDWF_F64, MDWF_F64>(F.p, F.r, true))) return st;
        if ((st = init_w<MDWF_F64>(S, F.w, F.p))) return st;
        while (it < maxiter) {
            const int steps = (maxiter - it) < every ? (maxiter - it) : every;
            if (use_graph) {
                if (!graph_ready) {
                    cudaGraph_t graph;
                    if ((st = cuda_status(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal))))
                        return st;
                    begin_capture(c);
                    int st2 = iterate<MDWF_F64, MDWF_F64>(S, F, F.xo, F.r);
                    c->capturing = false;
                    st = cuda_status(cudaStreamEndCapture(c->stream, &graph));
                    if (st2) return st2;
                    if (st) return st;
                    st = cuda_status(cudaGraphInstantiate(gexec, graph, 0));
                    cudaGraphDestroy(graph);
                    if (st) return st;
                    graph_ready = true;
                }
                for (int k = 0; k < steps; ++k) {
                    if ((st = cuda_status(cudaGraphLaunch(*gexec, c->stream)))) return st;
                    replay_graph_counts(c, 1);
                }
            } else {
                for (int k = 0; k < steps; ++k)
                    if ((st = iterate<MDWF_F64, MDWF_F64>(S, F, F.xo, F.r))) return st;
            }
            it += steps;
            if ((st = S.pull())) return st;
            bool active_left = false, reached = false;
            for (int r = 0; r < nrhs; ++r) {
                if (S.hsc[S_ACTIVE * kMaxRhs + r] == 0.0) continue;
                active_left = true;
                if (S.hsc[S_RR * kMaxRhs + r] <= tol * tol * S.hsc[S_SRC2 * kMaxRhs + r]) reached = true;
            }
            if (!active_left || reached) break;
        }
    }
    return MDWF_OK;
}

// Re <a, b> (or |a|^2 when b == a) per right-hand side of FP64 fields -> partials
__global__ void __launch_bounds__(kRedThreads) k_dot64(Field<MDWF_F64> a, Field<MDWF_F64> b, double* part, Geom g) {
    const int rhs = blockIdx.y;
    double acc = 0;
    SITE_LOOP(g) {
        const int s = (int)(i % g.Ls);
        const long long sr = rhs * g.Vh + i / g.Ls;
        double av[24], bv[24];
        a.load(sr, s, av);
        b.load(sr, s, bv);
#pragma unroll
        for (int k = 0; k < 24; ++k) acc += av[k] * bv[k];
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[rhs * gridDim.x + blockIdx.x] = acc;
}

__global__ void k_sum_partials(const double* part, int nb, double* out) {
    const int rhs = blockIdx.x;
    double v = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) v += part[rhs * nb + i];
    v = block_sum(v);
    if (threadIdx.x == 0) out[rhs] = v;
}

constexpr int kDotBlocks = 2 * 152;

int field_dot64(mdwf_ctx* c, const void* a, const void* b, int nrhs, double* out_host) {
    const size_t need = (size_t)nrhs * kDotBlocks + kMaxRhs;
    if (c->red_partials_len < need) {
        cudaFree(c->red_partials);
        c->red_partials = nullptr;
        c->red_partials_len = 0;
        int st = cuda_status(cudaMalloc(&c->red_partials, need * sizeof(double)));
        if (!st) st = canary_fill(c->red_partials, need * sizeof(double));
        if (st) return st;
        c->red_partials_len = need;
    }
    const Geom& g = c->g;
    const double n5 = (double)g.Vh * g.Ls * nrhs;
    {
        LaunchScope scope(c, KB_BLAS * 3 + MDWF_F64, n5 * 2.0 * 192.0, n5 * 48.0);
        k_dot64<<<dim3(kDotBlocks, nrhs), kRedThreads, 0, c->stream>>>(
            make_field<MDWF_F64>(const_cast<void*>(a), g, nrhs), make_field<MDWF_F64>(const_cast<void*>(b), g, nrhs),
            c->red_partials, g);
    }
    int st = check_launch();
    if (st) return st;
    double* dout = c->red_partials + (size_t)nrhs * kDotBlocks;
    {
        LaunchScope scope(c, KB_BLAS * 3 + MDWF_F64, 8.0 * nrhs * kDotBlocks, 0.0);
        k_sum_partials<<<nrhs, kRedThreads, 0, c->stream>>>(c->red_partials, kDotBlocks, dout);
    }
    if ((st = check_launch())) return st;
    if ((st = cuda_status(cudaMemcpyAsync(out_host, dout, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->stream))))
        return st;
    return cuda_status(cudaStreamSynchronize(c->stream));
}

// Per-slice Re <a, b> of one FP64 field: block (Ls, SB) threads, a fixed grid
// striding over the 4d sites, partials part[block][s]; then one block per
// slice sums them in order (deterministic).
__global__ void __launch_bounds__(128) k_dot_slices(Field<MDWF_F64> a, Field<MDWF_F64> b, double* part, Geom g) {
    extern __shared__ double red_s[];  // [SB][Ls]
    const int s = threadIdx.x, ly = threadIdx.y, Ls = g.Ls;
    double v = 0;
    for (long long site = (long long)blockIdx.x * blockDim.y + ly; site < g.Vh;
         site += (long long)gridDim.x * blockDim.y) {
        double x[24], y[24];
        a.load(site, s, x);
        b.load(site, s, y);
#pragma unroll
        for (int k = 0; k < 24; ++k) v += x[k] * y[k];
    }
    red_s[ly * Ls + s] = v;
    __syncthreads();
    if (ly != 0) return;
    double t = 0;
    for (int l = 0; l < (int)blockDim.y; ++l) t += red_s[l * Ls + s];
    part[(size_t)blockIdx.x * Ls + s] = t;
}

__global__ void __launch_bounds__(kRedThreads) k_sum_slices(const double* part, int nb, int Ls, double* out) {
    const int s = blockIdx.x;
    double v = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) v += part[(size_t)i * Ls + s];
    v = block_sum(v);
    if (threadIdx.x == 0) out[s] = v;
}

int slice_dot64(mdwf_ctx* c, const void* a, const void* b, double* out_host) {
    const Geom& g = c->g;
    const size_t need = (size_t)kDotBlocks * g.Ls + g.Ls;
    if (c->red_partials_len < need) {
        cudaFree(c->red_partials);
        c->red_partials = nullptr;
        c->red_partials_len = 0;
        int st = cuda_status(cudaMalloc(&c->red_partials, need * sizeof(double)));
        if (!st) st = canary_fill(c->red_partials, need * sizeof(double));
        if (st) return st;
        c->red_partials_len = need;
    }
    const int SB = (128 / g.Ls) < 1 ? 1 : 128 / g.Ls;
    const double n5 = (double)g.Vh * g.Ls;
    {
        LaunchScope scope(c, KB_BLAS * 3 + MDWF_F64, n5 * 2.0 * 192.0, n5 * 48.0);
        k_dot_slices<<<kDotBlocks, dim3(g.Ls, SB), sizeof(double) * SB * g.Ls, c->stream>>>(
            make_field<MDWF_F64>(const_cast<void*>(a), g, 1), make_field<MDWF_F64>(const_cast<void*>(b), g, 1),
            c->red_partials, g);
    }
    int st = check_launch();
    if (st) return st;
    double* dout = c->red_partials + (size_t)kDotBlocks * g.Ls;
    {
        LaunchScope scope(c, KB_BLAS * 3 + MDWF_F64, 8.0 * kDotBlocks * g.Ls, 0.0);
        k_sum_slices<<<g.Ls, kRedThreads, 0, c->stream>>>(c->red_partials, kDotBlocks, g.Ls, dout);
    }
    if ((st = check_launch())) return st;
    if ((st = cuda_status(cudaMemcpyAsync(out_host, dout, sizeof(double) * g.Ls, cudaMemcpyDeviceToHost, c->stream))))
        return st;
    return cuda_status(cudaStreamSynchronize(c->stream));
}

static size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Bytes of the solver workspace of solve_normal: FP64 r and t64, the inner
// fields (x_s and r_s in FP32 for a mixed solve; p, t and w), CG scalars and
// reduction partials.
// Blocks per right-hand side of the solver's vector kernels and reductions: a
// few per SM, more when the batch is small, so that one right-hand side fills
// the GPU (two blocks per SM left its HBM bandwidth half used).
static int red_blocks(int nrhs) { return 152 * std::max(2, std::min(8, 16 / nrhs)); }

static size_t solver_bytes(const mdwf_ctx* c, int nrhs, int inner, int nb, int hb) {
    const size_t f64 = field_bytes(MDWF_F64, c->g, nrhs), f32 = field_bytes(MDWF_F32, c->g, nrhs);
    const size_t fpp = field_bytes(inner, c->g, nrhs);
    const int inner_fields = 3;
    return up256(f64) * 2 +
           (inner == MDWF_F64 ? up256(f64) * inner_fields : up256(f32) * 2 + up256(fpp) * inner_fields) +
           up256(sizeof(double) * S_NUM * kMaxRhs) + up256(sizeof(double) * nrhs * nb) +
           up256(sizeof(double) * nrhs * hb);
}

// M x of the returned x, formed by the solve's last FP64 true residual: an FP64
// field of nrhs slots in the solver's workspace (valid until the next solve) and
// the right-hand sides for which it holds (mdwf_cgne reuses it for |b' - M x|)
struct SolvedMx {
    const void* mx = nullptr;
    std::vector<char> ok;
};

static int solve_normal_mx(mdwf_ctx* c, int nrhs, void* xo, const void* src, const mdwf_solve_params& prm,
                           NormalResult& res, SolvedMx* smx);

// Solves M^dag M x = src for nrhs FP64 internal odd fields (x starts at zero).
// Plain FP64 CG or mixed precision with FP64 reliable updates (prm.inner_prec).
int solve_normal(mdwf_ctx* c, int nrhs, void* xo, const void* src, const mdwf_solve_params& prm,
                 NormalResult& res) {
    return solve_normal_mx(c, nrhs, xo, src, prm, res, nullptr);
}

static int solve_normal_mx(mdwf_ctx* c, int nrhs, void* xo, const void* src, const mdwf_solve_params& prm,
                           NormalResult& res, SolvedMx* smx) {
    const double tol = prm.tol > 0 ? prm.tol : 1e-10;
    const int maxiter = prm.maxiter > 0 ? prm.maxiter : 20000;
    const int inner = prm.inner_prec;
    if (inner != MDWF_F64 && inner != MDWF_F32 && inner != MDWF_F16N) return MDWF_EINVAL;
    res.status.assign(nrhs, MDWF_OK);
    res.iters.assign(nrhs, 0);
    res.rupd.assign(nrhs, 0);
    res.restarts.assign(nrhs, 0);
    res.rel.assign(nrhs, 0.0);

    // a captured graph needs a stream other than the legacy default one
    cudaStream_t user_stream = c->stream, own = nullptr;
    const bool use_graph = prm.use_graph != 0 && !c->prof_on;
    int st;
    if (use_graph && user_stream == nullptr) {
        if ((st = cuda_status(cudaStreamCreate(&own)))) return st;
        c->stream = own;
    }
    const Geom g = c->g;
    const size_t f64 = field_bytes(MDWF_F64, g, nrhs), f32 = field_bytes(MDWF_F32, g, nrhs);
    const size_t fpp = field_bytes(inner, g, nrhs);
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    const int nb = red_blocks(nrhs);
    if (c->autotune && c->sb_tune[inner][nrhs] == 0) {
        int sb;
        if ((st = tune_hop(c, inner, nrhs, &sb))) return st;
    }
    if (c->autotune && inner != MDWF_F64 && c->sb_tune[MDWF_F64][nrhs] == 0) {
        int sb;
        if ((st = tune_hop(c, MDWF_F64, nrhs, &sb))) return st;
    }
    const int hb = hop_blocks(c, inner, nrhs);
    const size_t need = solver_bytes(c, nrhs, inner, nb, hb);
    Fields F{};
    Solver S{};
    cudaGraphExec_t gexec = nullptr;
    std::vector<double> maxr(nrhs, 0.0);
    double* hsc = nullptr;
    int ret = MDWF_OK;
    do {
        if ((st = ensure_workspace(c->solver, need))) { ret = st; break; }
        if ((st = ensure_workspace(c->tmp[0], f64)) || (st = ensure_workspace(c->tmp[1], f64))) { ret = st; break; }
        char* w = (char*)c->solver.p;
        auto take = [&](size_t bytes) { void* p = w; w += up(bytes); return p; };
        F.xo = xo;
        F.src = const_cast<void*>(src);
        F.r = take(f64); F.t64 = take(f64);
        const size_t fi = inner == MDWF_F64 ? f64 : fpp;
        if (inner != MDWF_F64) { F.xs = take(f32); F.rs = take(f32); }
        F.p = take(fi); F.t = take(fi);
        F.w = take(fi);  // w = M_phi p
        S.c = c; S.g = g; S.nrhs = nrhs; S.nb = nb;
        S.sc = (double*)take(sizeof(double) * S_NUM * kMaxRhs);
        S.part = (double*)take(sizeof(double) * nrhs * nb);
        S.hpart = (double*)take(sizeof(double) * nrhs * hb);
        S.hb = hb;
        if ((st = cuda_status(cudaMallocHost(&hsc, sizeof(double) * S_NUM * kMaxRhs)))) { ret = st; break; }
        S.hsc = hsc;
        memset(hsc, 0, sizeof(double) * S_NUM * kMaxRhs);
        for (int r = 0; r < nrhs; ++r) hsc[S_ACTIVE * kMaxRhs + r] = 1.0;
        if ((st = S.push())) { ret = st; break; }
        if ((st = S.norm<MDWF_F64>(F.src, false, S_SRC2))) { ret = st; break; }
        if (!prm.guess && (st = cuda_status(cudaMemsetAsync(F.xo, 0, f64, c->stream)))) { ret = st; break; }
        // zero right-hand sides are solved by x = 0
        if ((st = S.pull())) { ret = st; break; }
        for (int r = 0; r < nrhs; ++r)
            if (S.hsc[S_SRC2 * kMaxRhs + r] == 0.0) {
                S.hsc[S_ACTIVE * kMaxRhs + r] = 0.0;
                if (prm.guess) {  // whatever the guess, the solution is zero
                    const size_t f1 = field_bytes(MDWF_F64, g, 1);
                    if ((st = cuda_status(cudaMemsetAsync((char*)F.xo + r * f1, 0, f1, c->stream)))) break;
                }
            }
        if (st) { ret = st; break; }
        if ((st = S.push())) { ret = st; break; }

        std::vector<double> last_true(nrhs, 0.0);
        if (inner == MDWF_F64)
            st = run_plain(S, F, prm, tol, maxiter, last_true, &gexec, use_graph);
        else if (inner == MDWF_F32)
            st = run_mixed<MDWF_F32>(S, F, prm, tol, maxiter, maxr, res.rupd, res.restarts, last_true, &gexec,
                                     use_graph);
        else
            st = run_mixed<MDWF_F16N>(S, F, prm, tol, maxiter, maxr, res.rupd, res.restarts, last_true, &gexec,
                                      use_graph);
        if (st) { ret = st; break; }

        if ((st = S.pull())) { ret = st; break; }
        // x changes only at the FP64 true residuals, which form M x on the way: the plain
        // CG ends on one for every right-hand side, the mixed solve on each one's last
        // update (or the residual of the guess)
        if (smx) {
            smx->mx = F.t64;
            smx->ok.assign(nrhs, 0);
            for (int r = 0; r < nrhs; ++r) smx->ok[r] = inner == MDWF_F64 || prm.guess || res.rupd[r] > 0;
        }
        // the last FP64 true residual |src - M^dag M x| / |src| of every right-hand side
        for (int r = 0; r < nrhs; ++r) {
            res.status[r] = (int)S.hsc[S_STATUS * kMaxRhs + r];
            res.iters[r] = (int)S.hsc[S_ITERS * kMaxRhs + r];
            const double src2 = S.hsc[S_SRC2 * kMaxRhs + r];
            res.rel[r] = src2 > 0 ? sqrt(last_true[r] / src2) : 0.0;
            if (res.status[r] == MDWF_OK && res.rel[r] > tol) res.status[r] = MDWF_ENOCONV;
        }
    } while (0);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (hsc) cudaFreeHost(hsc);
    if (own) {
        cudaStreamSynchronize(own);
        cudaStreamDestroy(own);
        c->stream = user_stream;
    }
    return ret;
}

}  // namespace mdwf

using namespace mdwf;

namespace {

// Single-right-hand-side FP64 scratch of the source preparation and the
// reconstruction; rhs r of the batch (tables and mass of rhs r).
struct RhsScratch {
    void *be, *bp, *xe, *t;
    void* stage;  // one full field when the user buffers are in host memory
};

// b_r -> (b_e, b'_o) with b'_o = A b_o + 1/2 A H_oe M_phi (A b_e), A = I^-1
// (the Schur decomposition, D_br = -1/2 H_oe M_phi); xe and t are scratch.
// M_phi A b_e = K b_e is formed by the site-local pass, so the hop needs no
// gather along s.
int prepare_rhs(mdwf_ctx* c, const RhsScratch& w, const double* b, int where, int r) {
    const Geom& g = c->g;
    const size_t full1 = (size_t)g.Ls * 2 * g.Vh * 24 * sizeof(double);
    int st;
    const double* bdev = b + (size_t)r * full1 / sizeof(double);
    if (where == MDWF_HOST) {
        if ((st = cuda_status(cudaMemcpyAsync(w.stage, bdev, full1, cudaMemcpyHostToDevice, c->stream)))) return st;
        bdev = (const double*)w.stage;
    }
    if ((st = launch_split_full(c, w.be, w.bp, bdev, MDWF_F64, 1))) return st;
    M5Launch m{};
    m.nrhs = 1; m.coef = 1.0; m.x = nullptr;
    set_sop(c, MDWF_F64, SOP_K, 0, m);
    offset_rhs(c, MDWF_F64, r, m);
    m.out = w.xe; m.in = w.be;  // xe = K b_e = M_phi A b_e
    if ((st = launch_m5(c, MDWF_F64, m))) return st;
    m.mat = nullptr; m.mass = nullptr;
    set_sop(c, MDWF_F64, SOP_A, 0, m);
    offset_rhs(c, MDWF_F64, r, m);
    m.out = w.t; m.in = w.bp;   // t = A b_o
    if ((st = launch_m5(c, MDWF_F64, m))) return st;
    HopLaunch h{};
    h.nrhs = 1; h.b5 = c->b5; h.c5 = c->c5; h.mass = c->mass64;
    h.out = w.bp; h.in = w.xe; h.x = w.t; h.coef = 0.5; h.out_parity = 1; h.gather = 0; h.dagger = 0;
    set_sop(c, MDWF_F64, SOP_A, 0, h);
    offset_rhs(c, MDWF_F64, r, h);
    return launch_hop(c, MDWF_F64, h);
}

}  // namespace

extern "C" int mdwf_cgne(mdwf_ctx* c, double* x, const double* b, int nrhs, const double* mf_per_rhs, int where,
                         const mdwf_solve_params* params, mdwf_solve_info* info) {
    NvtxRange nvtx_range("mdwf_cgne");
    auto t0 = std::chrono::steady_clock::now();
    if (!c || !x || !b || nrhs < 1 || nrhs > kMaxRhs || (where != MDWF_HOST && where != MDWF_DEVICE))
        return MDWF_EINVAL;
    if (!c->have_gauge) return MDWF_ENOGAUGE;
    mdwf_solve_params prm{};
    if (params) prm = *params;
    if (prm.inner_prec != MDWF_F64 && prm.inner_prec != MDWF_F32 && prm.inner_prec != MDWF_F16N) return MDWF_EINVAL;
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    if ((st = ensure_tables(c, nrhs, mf_per_rhs))) return st;
    const Geom g = c->g;
    const size_t f64 = field_bytes(MDWF_F64, g, nrhs), f1 = field_bytes(MDWF_F64, g, 1);
    const size_t full1 = (size_t)g.Ls * 2 * g.Vh * 24 * sizeof(double);
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    // batched: x_o and M^dag b'_o; per right-hand side: two temporaries (+ host
    // staging of one full field). b_e and b'_o of every right-hand side are kept
    // from the preparation to the reconstruction when the device has room for
    // them; otherwise they are formed again from b after the solve.
    const size_t lean = up(f64) * 2 + up(f1) * 4 + (where == MDWF_HOST ? up(full1) : 0);
    const size_t keep_need = up(f64) * 4 + up(f1) * 2 + (where == MDWF_HOST ? up(full1) : 0);
    bool keep = true;
    {
        size_t free_b = 0, total_b = 0;
        if ((st = cuda_status(cudaMemGetInfo(&free_b, &total_b)))) return st;
        auto grow = [](size_t need_b, const Workspace& ws) { return need_b > ws.bytes ? need_b - ws.bytes : 0; };
        size_t extra = grow(keep_need, c->io) + grow(f64, c->tmp[0]) + grow(f64, c->tmp[1]);
        // the solver workspace, or the autotuner's two scratch fields before it (freed after tuning)
        size_t later = grow(
            solver_bytes(c, nrhs, prm.inner_prec, red_blocks(nrhs), hop_blocks(c, prm.inner_prec, nrhs)), c->solver);
        if (c->autotune) {
            const size_t tune_f = 2 * up(field_bytes(MDWF_F64, g, nrhs));
            if (tune_f > later) later = tune_f;
        }
        extra += later;
        keep = extra + (size_t(2) << 30) <= free_b;  // 2 GB left for the runtime and the caller
    }
    if ((st = ensure_workspace(c->io, keep ? keep_need : lean))) return st;
    if ((st = ensure_workspace(c->tmp[0], f64)) || (st = ensure_workspace(c->tmp[1], f64))) return st;
    char* w = (char*)c->io.p;
    auto take = [&](size_t bytes) { void* p = w; w += up(bytes); return p; };
    void *xo = take(f64), *src = take(f64);
    void* be_all = keep ? take(f64) : nullptr;
    void* bp_all = keep ? take(f64) : nullptr;
    RhsScratch sw;
    if (!keep) { sw.be = take(f1); sw.bp = take(f1); }
    sw.xe = take(f1); sw.t = take(f1);
    sw.stage = where == MDWF_HOST ? take(full1) : nullptr;
    auto point_at = [&](int r) {
        if (keep) { sw.be = (char*)be_all + (size_t)r * f1; sw.bp = (char*)bp_all + (size_t)r * f1; }
    };

    // src_r = M^dag b'_r, one right-hand side at a time
    for (int r = 0; r < nrhs; ++r) {
        point_at(r);
        if ((st = prepare_rhs(c, sw, b, where, r))) return st;
        if ((st = apply_op(c, (char*)src + (size_t)r * f1, sw.bp, MDWF_F64, 1, 1, r))) return st;
    }
    // an initial guess: the odd part of x
    if (prm.guess)
        for (int r = 0; r < nrhs; ++r) {
            const double* x_r = x + (size_t)r * full1 / sizeof(double);
            if (where == MDWF_HOST) {
                if ((st = cuda_status(cudaMemcpyAsync(sw.stage, x_r, full1, cudaMemcpyHostToDevice, c->stream))))
                    return st;
                x_r = (const double*)sw.stage;
            }
            if ((st = launch_split_full(c, sw.xe, (char*)xo + (size_t)r * f1, x_r, MDWF_F64, 1))) return st;
        }

    NormalResult res;
    SolvedMx smx;
    if ((st = solve_normal_mx(c, nrhs, xo, src, prm, res, &smx))) return st;

    // per right-hand side: |b' - M x| / |b'| and x_e = A b_e + 1/2 A H_eo M_phi x_o
    std::vector<double> bb(nrhs), rr(nrhs);
    for (int r = 0; r < nrhs; ++r) {
        void* xo_r = (char*)xo + (size_t)r * f1;
        point_at(r);
        if (!keep && (st = prepare_rhs(c, sw, b, where, r))) return st;  // b_e, b'_o again
        {
            M5Launch f{};  // xe (scratch until it is formed below) = M_phi x_o
            f.nrhs = 1; f.out = sw.xe; f.in = xo_r; f.x = nullptr; f.coef = 1.0;
            set_sop(c, MDWF_F64, SOP_MPHI, 0, f);
            offset_rhs(c, MDWF_F64, r, f);
            if ((st = launch_m5(c, MDWF_F64, f))) return st;
        }
        HopLaunch h{};  // t = 1/2 A H_eo M_phi x_o
        h.nrhs = 1; h.b5 = c->b5; h.c5 = c->c5; h.mass = c->mass64;
        h.out = sw.t; h.in = sw.xe; h.x = nullptr; h.coef = 0.5; h.out_parity = 0; h.gather = 0; h.dagger = 0;
        set_sop(c, MDWF_F64, SOP_A, 0, h);
        offset_rhs(c, MDWF_F64, r, h);
        if ((st = launch_hop(c, MDWF_F64, h))) return st;
        void* mx = c->tmp[1].p;
        const void* mx_in = mx;
        if (smx.mx && smx.ok[r]) {
            mx_in = (const char*)smx.mx + (size_t)r * f1;  // M x_o from the solve's last true residual
        } else {
            // M x_o = x_o - 1/4 A H_oe z with z = K H_eo M_phi x_o = M_phi (A H_eo M_phi x_o) =
            // 2 M_phi t: the hop of the reconstruction is the first hop of M, so only the second
            // runs here
            void* z = c->tmp[0].p;
            M5Launch f{};
            f.nrhs = 1; f.out = z; f.in = sw.t; f.x = nullptr; f.coef = 2.0;
            set_sop(c, MDWF_F64, SOP_MPHI, 0, f);
            offset_rhs(c, MDWF_F64, r, f);
            if ((st = launch_m5(c, MDWF_F64, f))) return st;
            note_apply(c, MDWF_F64);
            h.out = mx; h.in = z; h.x = xo_r; h.coef = -0.25; h.out_parity = 1; h.gather = 0; h.dagger = 0;
            h.mass = c->mass64;
            set_sop(c, MDWF_F64, SOP_A, 0, h);
            offset_rhs(c, MDWF_F64, r, h);
            if ((st = launch_hop(c, MDWF_F64, h))) return st;
        }
        {
            M5Launch d{};  // mx = b' - M x
            d.nrhs = 1; d.out = mx; d.in = mx_in; d.x = sw.bp; d.coef = -1.0;
            set_sop(c, MDWF_F64, SOP_ID, 0, d);
            offset_rhs(c, MDWF_F64, r, d);
            if ((st = launch_m5(c, MDWF_F64, d))) return st;
        }
        if ((st = field_dot64(c, mx, mx, 1, &rr[r]))) return st;
        if ((st = field_dot64(c, sw.bp, sw.bp, 1, &bb[r]))) return st;
        M5Launch m{};
        m.nrhs = 1; m.out = sw.xe; m.in = sw.be; m.x = sw.t; m.coef = 1.0;
        set_sop(c, MDWF_F64, SOP_A, 0, m);
        offset_rhs(c, MDWF_F64, r, m);
        if ((st = launch_m5(c, MDWF_F64, m))) return st;
        double* x_r = x + (size_t)r * full1 / sizeof(double);
        double* xdev = where == MDWF_HOST ? (double*)sw.stage : x_r;
        if ((st = launch_join_full(c, xdev, sw.xe, xo_r, MDWF_F64, 1))) return st;
        if (where == MDWF_HOST &&
            (st = cuda_status(cudaMemcpyAsync(x_r, sw.stage, full1, cudaMemcpyDeviceToHost, c->stream))))
            return st;
    }
    if ((st = cuda_status(cudaStreamSynchronize(c->stream)))) return st;
    if ((st = device_wait_status(c))) return st;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int ret = MDWF_OK;
    for (int r = 0; r < nrhs; ++r) {
        if (res.status[r] > ret) ret = res.status[r];
        if (info) {
            info[r].status = res.status[r];
            info[r].iters = res.iters[r];
            info[r].reliable_updates = res.rupd[r];
            info[r].restarts = res.restarts[r];
            info[r].true_res = res.rel[r];
            info[r].res_m = bb[r] > 0 ? sqrt(rr[r] / bb[r]) : 0.0;
            info[r].seconds = secs;
        }
    }
    return ret;
}
