// Site-local fifth-dimension operators: out = coef * Op in (+ x), Op one of
// the s-operators of each chirality (I^-1 by the closed-form elimination of
// Sec. 3, M_phi, K = M_phi I^-1, the shift C, or a dense Ls x Ls table), or
// their adjoints (chirality swapped). The Ls spinors of a 4d site are staged
// in shared memory and each (site, component) column is solved by one thread.
#include "mdwf_internal.cuh"

namespace mdwf {

template <int P, bool XPAY>
__global__ void __launch_bounds__(256) m5_kernel(Field<P> out, Field<P> in, Field<P> xf,
                                                 const typename PrecTraits<P>::real* tab,
                                                 const typename PrecTraits<P>::real* mass,
                                                 typename PrecTraits<P>::real coef, Geom g, int sop, int swap,
                                                 SCoef<typename PrecTraits<P>::real> sc, const double* mask) {
    typedef typename PrecTraits<P>::real R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = g.Ls;
    const bool dense = sop == SOP_DENSE;
    R* mat = reinterpret_cast<R*>(smem_raw);
    R* cs = mat + (dense ? 2 * Ls * Ls : 0);
    const int nrhs = (int)(gridDim.x / ((g.Vh + blockDim.y - 1) / blockDim.y));
    const int s = threadIdx.x, ly = threadIdx.y, rhs = blockIdx.x % nrhs;
    if (mask && mask[rhs] == 0.0) return;  // block-uniform, before any barrier
    const long long sblk = blockIdx.x / nrhs;
    const int tid = ly * blockDim.x + s, nthr = blockDim.x * blockDim.y;
    // The bidiagonal operators (M_phi, C, I = M+ + M- C) and the identity need only
    // the s +- 1 neighbours of a column, which share the thread's cache lines: each
    // thread reads its spinor and the two half spinors straight from memory, with no
    // staging and no barrier (the identity also in place; the others out of place,
    // since a neighbour's element may be overwritten). Chirality 0 (reals 0..11)
    // couples to s - 1 and chirality 1 to s + 1; the adjoint (swap) exchanges them;
    // the wrap-around term carries -m. Block-uniform.
    const bool bidiag = sop == SOP_MPHI || sop == SOP_C || sop == SOP_MEE;
    if (!dense && (sop == SOP_ID || (bidiag && (const void*)out.v != (const void*)in.v))) {
        const long long site = sblk * blockDim.y + ly;
        if (site >= g.Vh) return;
        const long long sr = (long long)rhs * g.Vh + site;
        R v[24];
        in.load(sr, s, v);
        if (bidiag) {
            const R w0 = sop == SOP_MPHI ? sc.b5 : sop == SOP_MEE ? sc.Mp : R(0);
            const R w1 = sop == SOP_MPHI ? sc.c5 : sop == SOP_MEE ? sc.Mm : R(1);
            const R m = mass[rhs];
            const bool sw = swap != 0;
            const int up = s + 1 < Ls ? s + 1 : 0, dn = s > 0 ? s - 1 : Ls - 1;
            const R f0 = w1 * ((sw ? s < Ls - 1 : s > 0) ? R(1) : -m);
            const R f1 = w1 * ((sw ? s > 0 : s < Ls - 1) ? R(1) : -m);
            R h0[12], h1[12];
            in.load_half(sr, sw ? up : dn, 0, h0);
            in.load_half(sr, sw ? dn : up, 1, h1);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                v[k] = w0 * v[k] + f0 * h0[k];
                v[12 + k] = w0 * v[12 + k] + f1 * h1[k];
            }
        }
#pragma unroll
        for (int k = 0; k < 24; ++k) v[k] *= coef;
        if (XPAY) {
            R xv[24];
            xf.load(sr, s, xv);
#pragma unroll
            for (int k = 0; k < 24; ++k) v[k] += xv[k];
        }
        out.store(sr, s, v);
        return;
    }
    if (dense) {
        const R* gm = tab + (size_t)rhs * 2 * Ls * Ls;
        for (int i = tid; i < 2 * Ls * Ls; i += nthr) mat[i] = gm[i];
    }
    const long long site = sblk * blockDim.y + ly;
    const bool active = site < g.Vh;
    const long long sr = (long long)rhs * g.Vh + site;
    R v[24];
    if (active) in.load(sr, s, v);
    else {
#pragma unroll
        for (int k = 0; k < 24; ++k) v[k] = 0;
    }
    const int sst = site_stride(Ls);
    R* mine = cs + (size_t)ly * sst + s * kRowStride;
    row_store(mine, v);
    __syncthreads();
    R res[24];
    if (dense) {
        if (!active) return;
#pragma unroll
        for (int k = 0; k < 24; ++k) res[k] = 0;
        const R* col = cs + (size_t)ly * sst;
        for (int sp = 0; sp < Ls; ++sp) {
            const R mp = mat[sp * Ls + s], mm = mat[(Ls + sp) * Ls + s];
            const R* h = col + sp * kRowStride;
#pragma unroll
            for (int k = 0; k < 12; ++k) res[k] += mp * h[k];
#pragma unroll
            for (int k = 12; k < 24; ++k) res[k] += mm * h[k];
        }
    } else {
        // the shared-memory walk: register-held columns measured slower in this 256-thread kernel
        block_columns(cs, blockDim.y, Ls, sop, swap != 0, sc, mass[rhs], tid, nthr, false);
        __syncthreads();
        if (!active) return;
        row_load(mine, res);
    }
#pragma unroll
    for (int k = 0; k < 24; ++k) res[k] *= coef;
    if (XPAY) {
        R xv[24];
        xf.load(sr, s, xv);
#pragma unroll
        for (int k = 0; k < 24; ++k) res[k] += xv[k];
    }
    out.store(sr, s, res);
}

template <int P>
static int launch_m5_t(mdwf_ctx* c, const M5Launch& m) {
    typedef typename PrecTraits<P>::real R;
    const Geom& g = c->g;
    int SB = 128 / g.Ls;
    if (SB < 1) SB = 1;
    dim3 block(g.Ls, SB), grid((unsigned)((g.Vh + SB - 1) / SB * m.nrhs));  // rhs fastest
    size_t smem = (size_t)((m.sop == SOP_DENSE ? 2 * g.Ls * g.Ls : 0) + SB * site_stride(g.Ls)) * sizeof(R);
    Field<P> out = make_field<P>(m.out, g, m.nrhs);
    Field<P> in = make_field<P>(const_cast<void*>(m.in), g, m.nrhs);
    Field<P> xf = m.x ? make_field<P>(const_cast<void*>(m.x), g, m.nrhs) : out;
    const R* tab = reinterpret_cast<const R*>(m.mat);
    const R* mass = m.mass ? reinterpret_cast<const R*>(m.mass)
                           : P == MDWF_F64 ? reinterpret_cast<const R*>(c->mass64)
                                           : reinterpret_cast<const R*>(c->mass32);
    SCoef<R> sc;
    sc.b5 = (R)c->b5;
    sc.c5 = (R)c->c5;
    sc.Mp = (R)(c->b5 * (4.0 - c->M5) + 1.0);
    sc.Mm = (R)(c->c5 * (4.0 - c->M5) - 1.0);
    const double n5 = (double)g.Vh * g.Ls * m.nrhs;
    LaunchScope scope(c, (m.x ? KB_M5_XPAY : KB_M5) * 3 + P, n5 * site_bytes(P) * (m.x ? 3.0 : 2.0),
                      n5 * (144.0 + (m.x ? 24.0 : 0.0)));
    if (m.x) {
        auto k = m5_kernel<P, true>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, block, smem, c->stream>>>(out, in, xf, tab, mass, (R)m.coef, g, m.sop, m.swap, sc, m.mask);
    } else {
        auto k = m5_kernel<P, false>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, block, smem, c->stream>>>(out, in, xf, tab, mass, (R)m.coef, g, m.sop, m.swap, sc, m.mask);
    }
    return check_launch();
}

int launch_m5(mdwf_ctx* c, int prec, const M5Launch& m) {
    switch (prec) {
        case MDWF_F64: return launch_m5_t<MDWF_F64>(c, m);
        case MDWF_F32: return launch_m5_t<MDWF_F32>(c, m);
        case MDWF_F16N: return launch_m5_t<MDWF_F16N>(c, m);
    }
    return MDWF_EINVAL;
}

}  // namespace mdwf
