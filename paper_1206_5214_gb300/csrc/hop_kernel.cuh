// Fused hopping kernel of the red/black Moebius operator (templates; each
// precision is instantiated in its own translation unit, dslash_<prec>.cu).
//
// One launch computes, for every site x of parity `out_parity` and every s,
//   out(x, s) = coef * sum_s' Mat_chi(s, s') [H w](x, s') (+ x_add(x, s))
// where H is the Wilson hopping sum of Eq. (D^Wilson),
//   H w(x) = sum_mu [(1 - g_mu) U_mu(x) w(x+mu) + (1 + g_mu) U_mu(x-mu)^dag w(x-mu)]
// (projector signs flipped for the hopping part of D_W^dag), and w is either
// the input field or the input with the fifth-dimension gather of Sec. 3
// applied first: w_s = b5 psi_s + c5 (P+ psi_{s-1} + P- psi_{s+1}) with the
// mass -m on the wrap-around terms (Eq. DWaction), i.e. w = M_phi psi.
// Mat is an Ls x Ls real matrix per chirality (K = M_phi I^-1, I^-1, ...).
//
// Thread mapping: a block is Ls x SB threads: threadIdx.x = s, threadIdx.y =
// one of SB 4d sites; blockIdx.x = (site block, right-hand side) with the
// right-hand side fastest, so that the blocks running together share sites and
// read their links from L2. The Ls threads of a column load the same link (one
// L1 line, broadcast), so each link is read from HBM once per hop and reused
// across all Ls slices. Spinor chunks of consecutive s are contiguous, so every
// vector load of a warp is coalesced. The neighbour spinors are loaded into
// registers when needed, or one term ahead into a second register buffer
// (prefetch), or staged in shared memory (STAGE below). The s-mixing matrix is
// applied after the hop through shared memory.
#pragma once

#include <atomic>

#include "mdwf_internal.cuh"
#include "mbarrier.cuh"

namespace mdwf {

template <typename R> struct HopParams {
    Geom g;
    int nrhs;        // blocks are (site block, rhs) with rhs fastest: blocks that run
                     // together share sites, so their links come from L2
    int out_parity;
    R coef;
    // input gather w = gscale * (gown psi_s + gfac (P+ psi_{s-1} + P- psi_{s+1})) = M_phi psi;
    // gscale is applied once to the accumulated hop instead of per neighbour
    R gown, gfac, gscale;
    // per-slice gather factors [gown(s)][gfac(s)][gscale(s)] (64 each) for
    // s-dependent b5(s), c5(s), or null; gscale(s) then scales the hop of row s
    // before the s-mixing and gscale above is 1
    const R* gs;
    const R* mass;   // [rhs]
    const R* mat;    // dense tables [rhs][chir][s'][s] (sop == SOP_DENSE)
    const R* mat2;   // dense A^dag tables of the FUSE_T epilogue, same layout
    const int4* nbr; // [parity][site][2] = cb index of x+mu (mu = 0..3), then of x-mu
    int sop, swap;
    SCoef<R> sc;
    // chemical potential (Sec. 6.6): the time-direction terms carry efwd
    // (forward hop) and ebwd (backward hop) when chem is set
    bool chem;
    R efwd, ebwd;
    int* err;        // device error word (bounded waits of the bulk variant)
    // the fused iteration without a t field (Ls = 16, bidiagonal shuffles):
    // FUSE_T does not store t; FUSE_R forms its addend t = I^dag v from x = v
    bool no_t;
    // t-slab (domain decomposition along t): the t-direction neighbours across
    // the slab's faces are read from halo = [dir][rhs][face site][6 / 3 chunks][s]
    // half spinors (dir 0: the forward term's projected neighbour, dir 1: the
    // backward term's neighbour projected and transported by the sending slab);
    // the neighbour table marks them as -1 - face site
    const void* halo;
    long long face;  // 4d sites of one parity in one t-slice
    const double* mask;  // per-rhs flags (null: every right-hand side); 0 skips the blocks
};

// One half spinor (12 reals) of a slab halo: chunk k of (dir, rhs, face site f,
// slice s), in the layout of the precision's field chunks.
template <int P, typename R>
__device__ __forceinline__ void halo_load(const HopParams<R>& hp, int dir, long long rf, int s, R* h) {
    const int Ls = hp.g.Ls;
    const long long base = ((long long)dir * hp.nrhs * hp.face + rf) * (P == MDWF_F64 ? 6 : 3) * Ls + s;
    if constexpr (P == MDWF_F64) {
        const double2* q = reinterpret_cast<const double2*>(hp.halo) + base;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double2 d = __ldg(q + (long long)k * Ls);
            h[2 * k] = d.x; h[2 * k + 1] = d.y;
        }
    } else {
        const float4* q = reinterpret_cast<const float4*>(hp.halo) + base;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 d = __ldg(q + (long long)k * Ls);
            h[4 * k] = d.x; h[4 * k + 1] = d.y; h[4 * k + 2] = d.z; h[4 * k + 3] = d.w;
        }
    }
}

// --------------------------------------------------------- spin structure
//
// Chiral basis g_mu = [[0, A_mu], [A_mu^dag, 0]], A_k = -i sigma_k, A_4 = 1.
// (1 + S g_mu) psi, psi = (u, l) by chirality halves, has upper half
// h = u + S A l and lower half S A^dag h, so only h (2 spins x 3 colours) is
// transported: project -> multiply by the link -> reconstruct.

template <int MU, int S, typename R>
__device__ __forceinline__ void project(const R* w, R* h) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R u0r = w[2 * c], u0i = w[2 * c + 1], u1r = w[6 + 2 * c], u1i = w[7 + 2 * c];
        const R l0r = w[12 + 2 * c], l0i = w[13 + 2 * c], l1r = w[18 + 2 * c], l1i = w[19 + 2 * c];
        R a0r, a0i, a1r, a1i;  // (A l)_0, (A l)_1
        if (MU == 0) {         // A = -i sigma_1: (A l)_0 = -i l1, (A l)_1 = -i l0
            a0r = l1i; a0i = -l1r; a1r = l0i; a1i = -l0r;
        } else if (MU == 1) {  // A = -i sigma_2: (A l)_0 = -l1, (A l)_1 = l0
            a0r = -l1r; a0i = -l1i; a1r = l0r; a1i = l0i;
        } else if (MU == 2) {  // A = -i sigma_3: (A l)_0 = -i l0, (A l)_1 = i l1
            a0r = l0i; a0i = -l0r; a1r = -l1i; a1i = l1r;
        } else {               // A = 1
            a0r = l0r; a0i = l0i; a1r = l1r; a1i = l1i;
        }
        h[2 * c] = u0r + S * a0r;
        h[2 * c + 1] = u0i + S * a0i;
        h[6 + 2 * c] = u1r + S * a1r;
        h[7 + 2 * c] = u1i + S * a1i;
    }
}

// Transport and reconstruction of one hopping term: g[a][i] = sum_j V[i][j] h[a][j]
// with V = U (or U^dag when ADJ; U row-major complex 3x3), then the upper half
// of (1 + S g_mu) gets g and the lower half S A_mu^dag g. It runs one output
// colour i at a time so that only one colour of g is live; `scaled` multiplies
// g by `scale` first (the FP16 norm of the neighbour).
template <bool ADJ, int MU, int S, typename R>
__device__ __forceinline__ void transport_add(R* acc, const R* U, const R* h, R scale, bool scaled) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        R g[4];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            // complex multiply-accumulate as four fused multiply-adds per term
            R sr = 0, si = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const R ur = ADJ ? U[2 * (3 * j + i)] : U[2 * (3 * i + j)];
                const R ui = ADJ ? -U[2 * (3 * j + i) + 1] : U[2 * (3 * i + j) + 1];
                const R hr = h[6 * a + 2 * j], hi = h[6 * a + 2 * j + 1];
                sr = fma(ur, hr, sr);
                sr = fma(-ui, hi, sr);
                si = fma(ur, hi, si);
                si = fma(ui, hr, si);
            }
            g[2 * a] = scaled ? scale * sr : sr;
            g[2 * a + 1] = scaled ? scale * si : si;
        }
        const R g0r = g[0], g0i = g[1], g1r = g[2], g1i = g[3];
        acc[2 * i] += g0r;
        acc[2 * i + 1] += g0i;
        acc[6 + 2 * i] += g1r;
        acc[7 + 2 * i] += g1i;
        R b0r, b0i, b1r, b1i;  // (A^dag g)_0, (A^dag g)_1
        if (MU == 0) {         // A^dag = i sigma_1: (i g1, i g0)
            b0r = -g1i; b0i = g1r; b1r = -g0i; b1i = g0r;
        } else if (MU == 1) {  // A^dag = i sigma_2: (g1, -g0)
            b0r = g1r; b0i = g1i; b1r = -g0r; b1i = -g0i;
        } else if (MU == 2) {  // A^dag = i sigma_3: (i g0, -i g1)
            b0r = -g0i; b0i = g0r; b1r = g1i; b1i = -g1r;
        } else {
            b0r = g0r; b0i = g0i; b1r = g1r; b1i = g1i;
        }
        acc[12 + 2 * i] += S * b0r;
        acc[13 + 2 * i] += S * b0i;
        acc[18 + 2 * i] += S * b1r;
        acc[19 + 2 * i] += S * b1i;
    }
}

// Reconstruction alone, for a half spinor g already transported (the backward
// t-direction term of a slab face, whose link lives on the sending slab):
// upper half += f g, lower half += f S A_mu^dag g.
template <int MU, int S, typename R>
__device__ __forceinline__ void reconstruct_add(R* acc, const R* g, R f) {
    static_assert(MU == 3, "slab faces are t-faces (A_4 = 1)");
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        acc[k] = fma(f, g[k], acc[k]);
        acc[12 + k] = fma(S * f, g[k], acc[12 + k]);
    }
}

// w = psi(s), or M_phi psi at s up to the factor gscale, for the neighbour column sr.
// Returns a factor still to be applied to w (the FP16 norm of an ungathered
// input, which is linear and is applied to the transported half spinor).
template <int P, bool GATHER, typename R>
__device__ __forceinline__ R load_input(const Field<P>& in, long long sr, int s, int Ls, R gown, R gfac,
                                        R mass, R* w) {
    if constexpr (P == MDWF_F16N && !GATHER) {
        return in.load_raw(sr, s, w);
    }
    in.load(sr, s, w);
    if (GATHER) {
        if (gown != R(1)) {
#pragma unroll
            for (int k = 0; k < 24; ++k) w[k] *= gown;
        }
        if (gfac != R(0)) {
            R t[12];
            const int sm = s > 0 ? s - 1 : Ls - 1;
            const R fm = s > 0 ? gfac : -mass * gfac;
            in.load_half(sr, sm, 0, t);  // P+ psi_{s-1}
#pragma unroll
            for (int k = 0; k < 12; ++k) w[k] += fm * t[k];
            const int sp = s < Ls - 1 ? s + 1 : 0;
            const R fp = s < Ls - 1 ? gfac : -mass * gfac;
            in.load_half(sr, sp, 1, t);  // P- psi_{s+1}
#pragma unroll
            for (int k = 0; k < 12; ++k) w[12 + k] += fp * t[k];
        }
    }
    return R(1);
}

// The forward and backward terms of one direction mu together (FP64 operator,
// no gather, no chemical potential on mu): per output colour i,
//   g_f = [U_mu(x) h_f]_i,  s = g_f + [U_mu(x-mu)^dag h_b]_i  (one FMA chain from g_f),
//   upper += s,  lower += SF A_mu^dag (g_f - g_b) with g_f - g_b = 2 g_f - s,
// since the backward term enters the lower half with the opposite sign. This
// takes 12 of the 48 additions of the two reconstructions away (the FP64
// operator is bound by the FP64 pipe). Links are read one row (U) or one
// column (U^dag) at a time.
template <int MU, bool DAG>
__device__ __forceinline__ void hop_pair64(double* acc, const Field<MDWF_F64>& in, const Gauge<MDWF_F64>& U,
                                           const HopParams<double>& hp, const int* nbi, long long site, int s,
                                           long long rbase) {
    constexpr int SF = DAG ? +1 : -1;
    const long long jf = __ldg(nbi + MU), jb = __ldg(nbi + 4 + MU);
    double hf[12], hb[12];
    {
        double w[24];
        in.load(rbase + jf, s, w);
        project<MU, SF>(w, hf);
    }
    {
        double w[24];
        in.load(rbase + jb, s, w);
        project<MU, -SF>(w, hb);
    }
    const double2* uf = U.u + (((long long)hp.out_parity * 4 + MU) * hp.g.Vh + site) * 9;
    const double2* ub = U.u + (((long long)(1 - hp.out_parity) * 4 + MU) * hp.g.Vh + jb) * 9;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double2 rf[3], cb[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            rf[j] = __ldg(uf + 3 * i + j);  // U_f[i][j]
            cb[j] = __ldg(ub + 3 * j + i);  // U_b[j][i]: (U_b^dag)[i][j] = conj
        }
        double sum[4], dif[4];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            double sr = 0, si = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const double ur = rf[j].x, ui = rf[j].y, hr = hf[6 * a + 2 * j], hi = hf[6 * a + 2 * j + 1];
                sr = fma(ur, hr, sr);
                sr = fma(-ui, hi, sr);
                si = fma(ur, hi, si);
                si = fma(ui, hr, si);
            }
            const double fr = sr, fi = si;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const double ur = cb[j].x, ui = -cb[j].y, hr = hb[6 * a + 2 * j], hi = hb[6 * a + 2 * j + 1];
                sr = fma(ur, hr, sr);
                sr = fma(-ui, hi, sr);
                si = fma(ur, hi, si);
                si = fma(ui, hr, si);
            }
            sum[2 * a] = sr;
            sum[2 * a + 1] = si;
            dif[2 * a] = fma(2.0, fr, -sr);
            dif[2 * a + 1] = fma(2.0, fi, -si);
        }
        acc[2 * i] += sum[0];
        acc[2 * i + 1] += sum[1];
        acc[6 + 2 * i] += sum[2];
        acc[7 + 2 * i] += sum[3];
        const double g0r = dif[0], g0i = dif[1], g1r = dif[2], g1i = dif[3];
        double b0r, b0i, b1r, b1i;  // (A^dag d)_0, (A^dag d)_1
        if (MU == 0) {
            b0r = -g1i; b0i = g1r; b1r = -g0i; b1i = g0r;
        } else if (MU == 1) {
            b0r = g1r; b0i = g1i; b1r = -g0r; b1i = -g0i;
        } else if (MU == 2) {
            b0r = -g0i; b0i = g0r; b1r = g1i; b1i = -g1r;
        } else {
            b0r = g0r; b0i = g0i; b1r = g1r; b1i = g1i;
        }
        acc[12 + 2 * i] += SF * b0r;
        acc[13 + 2 * i] += SF * b0i;
        acc[18 + 2 * i] += SF * b1r;
        acc[19 + 2 * i] += SF * b1i;
    }
}

// nbi: the site's eight neighbour indices (x+mu, mu = 0..3, then x-mu), each
// read just before its term so that none is held in a register across terms
template <int P, int MU, bool GATHER, bool DAG, bool DD = false, typename R>
__device__ __forceinline__ void hop_dir(R* acc, const Field<P>& in, const Gauge<P>& U, const HopParams<R>& hp,
                                        const int* nbi, long long site, int s, long long rbase, R mass,
                                        R gown, R gfac, int rhs = 0) {
    if constexpr (P == MDWF_F64 && !GATHER) {
        if (!(MU == 3 && (hp.chem || DD))) {
            hop_pair64<MU, DAG>(acc, in, U, hp, nbi, site, s, rbase);
            return;
        }
    }
    const Geom& g = hp.g;
    constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF g_mu
    constexpr bool SCALED = P == MDWF_F16N && !GATHER;
    if constexpr (DD && MU == 3) {
        // slab faces: the neighbour across a face comes from the halo
        const int jf = __ldg(nbi + 3), jb = __ldg(nbi + 7);
        if (jf < 0) {
            R h[12], u[18];
            halo_load<P>(hp, 0, (long long)rhs * hp.face + (-1 - jf), s, h);
            U.load(((long long)hp.out_parity * 4 + 3) * g.Vh + site, u);
            transport_add<false, 3, SF>(acc, u, h, hp.efwd, hp.chem);
        }
        if (jb < 0) {
            R h[12];
            halo_load<P>(hp, 1, (long long)rhs * hp.face + (-1 - jb), s, h);
            reconstruct_add<3, -SF>(acc, h, hp.chem ? hp.ebwd : R(1));
        }
        if (jf < 0 && jb < 0) return;
        if (jf < 0 || jb < 0) {
            // the other term of this direction lies inside the slab
            const bool fwd = jb < 0;
            const long long j = fwd ? jf : jb;
            R w[24], h[12], u[18];
            const R f = load_input<P, GATHER>(in, rbase + j, s, g.Ls, gown, gfac, mass, w);
            if (fwd) {
                project<3, SF>(w, h);
                U.load(((long long)hp.out_parity * 4 + 3) * g.Vh + site, u);
                transport_add<false, 3, SF>(acc, u, h, hp.chem ? f * hp.efwd : f, SCALED || hp.chem);
            } else {
                project<3, -SF>(w, h);
                U.load(((long long)(1 - hp.out_parity) * 4 + 3) * g.Vh + j, u);
                transport_add<true, 3, -SF>(acc, u, h, hp.chem ? f * hp.ebwd : f, SCALED || hp.chem);
            }
            return;
        }
    }
    {
        const long long jf = __ldg(nbi + MU);
        R w[24], h[12], u[18];
        const R f = load_input<P, GATHER>(in, rbase + jf, s, g.Ls, gown, gfac, mass, w);
        project<MU, SF>(w, h);
        U.load(((long long)hp.out_parity * 4 + MU) * g.Vh + site, u);
        const bool tm = MU == 3 && hp.chem;
        transport_add<false, MU, SF>(acc, u, h, tm ? f * hp.efwd : f, SCALED || tm);
    }
    {
        const long long jb = __ldg(nbi + 4 + MU);
        R w[24], h[12], u[18];
        const R f = load_input<P, GATHER>(in, rbase + jb, s, g.Ls, gown, gfac, mass, w);
        project<MU, -SF>(w, h);
        U.load(((long long)(1 - hp.out_parity) * 4 + MU) * g.Vh + jb, u);
        const bool tm = MU == 3 && hp.chem;
        transport_add<true, MU, -SF>(acc, u, h, tm ? f * hp.ebwd : f, SCALED || tm);
    }
}

// ------------------------------------------------ staged neighbour loads
//
// The staged variant (STAGE) copies each neighbour spinor of a thread into
// shared memory with cp.async (LDGSTS) one neighbour ahead of its use, so two
// neighbour loads per thread are in flight without holding registers; the
// plain variant loads into registers when the spinor is needed. Buffers are
// [2][chunk][thread] so that a warp's 16-byte accesses are contiguous.

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (bytes == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
    else if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// bytes of the staging buffers per thread (two neighbour spinors)
template <int P> struct StageBytes { static constexpr int value = 0; };
template <> struct StageBytes<MDWF_F32> { static constexpr int value = 2 * 6 * 16; };
template <> struct StageBytes<MDWF_F16N> { static constexpr int value = 2 * (6 * 8 + 4); };

template <int P> struct Stager;
template <> struct Stager<MDWF_F32> {
    float4* buf;  // [2][6][nthr]
    int nthr, tid;
    __device__ __forceinline__ void issue(const Field<MDWF_F32>& in, long long sr, int s, int slot) const {
        const float4* src = in.v + sr * 6 * in.Ls + s;
#pragma unroll
        for (int k = 0; k < 6; ++k) cp_async(buf + (slot * 6 + k) * nthr + tid, src + (long long)k * in.Ls, 16);
        cp_async_commit();
    }
    __device__ __forceinline__ float read(int slot, float* w) const {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 d = buf[(slot * 6 + k) * nthr + tid];
            w[4 * k] = d.x; w[4 * k + 1] = d.y; w[4 * k + 2] = d.z; w[4 * k + 3] = d.w;
        }
        return 1.0f;
    }
};
template <> struct Stager<MDWF_F16N> {
    uint2* buf;   // [2][6][nthr]
    float* nrm;   // [2][nthr]
    int nthr, tid;
    __device__ __forceinline__ void issue(const Field<MDWF_F16N>& in, long long sr, int s, int slot) const {
        const uint2* src = in.v + sr * 6 * in.Ls + s;
#pragma unroll
        for (int k = 0; k < 6; ++k) cp_async(buf + (slot * 6 + k) * nthr + tid, src + (long long)k * in.Ls, 8);
        cp_async(nrm + slot * nthr + tid, in.norm + sr * in.Ls + s, 4);
        cp_async_commit();
    }
    // values without the norm (applied to the transported half spinor); returns the norm
    __device__ __forceinline__ float read(int slot, float* w) const {
#pragma unroll
        for (int k = 0; k < 6; ++k) Field<MDWF_F16N>::unpack_raw(buf[(slot * 6 + k) * nthr + tid], w + 4 * k);
        return nrm[slot * nthr + tid];
    }
};

// Hopping term n of the eight (MU, FWD) from staging slot n % 2: wait for its
// copy, project it, refill the slot with neighbour `next` (< 0: none), then
// transport and accumulate.
template <int P, int MU, bool FWD, bool DAG, int WAITN, typename R>
__device__ __forceinline__ void hop_term(R* acc, const Field<P>& in, const Gauge<P>& U, const HopParams<R>& hp,
                                         const Stager<P>& st, long long site, int jb, int next, int s,
                                         long long rbase) {
    constexpr int SF = DAG ? +1 : -1;
    constexpr int S = FWD ? SF : -SF;
    constexpr int SLOT = FWD ? 0 : 1;
    R h[12], u[18];
    cp_async_wait<WAITN>();
    R f;
    {
        R w[24];
        f = st.read(SLOT, w);
        project<MU, S>(w, h);
    }
    if (next >= 0) st.issue(in, rbase + next, s, SLOT);
    if (FWD) U.load(((long long)hp.out_parity * 4 + MU) * hp.g.Vh + site, u);
    else U.load(((long long)(1 - hp.out_parity) * 4 + MU) * hp.g.Vh + jb, u);
    const bool tm = MU == 3 && hp.chem;
    transport_add<!FWD, MU, S>(acc, u, h, tm ? f * (FWD ? hp.efwd : hp.ebwd) : f, P == MDWF_F16N || tm);
}

// The eight terms with the next neighbour in flight while one is computed.
template <int P, bool DAG, typename R>
__device__ __forceinline__ void hop_staged(R* acc, const Field<P>& in, const Gauge<P>& U, const HopParams<R>& hp,
                                           const Stager<P>& st, int4 f, int4 b, long long site, int s,
                                           long long rbase) {
    st.issue(in, rbase + f.x, s, 0);
    st.issue(in, rbase + b.x, s, 1);
    hop_term<P, 0, true, DAG, 1>(acc, in, U, hp, st, site, 0, f.y, s, rbase);
    hop_term<P, 0, false, DAG, 1>(acc, in, U, hp, st, site, b.x, b.y, s, rbase);
    hop_term<P, 1, true, DAG, 1>(acc, in, U, hp, st, site, 0, f.z, s, rbase);
    hop_term<P, 1, false, DAG, 1>(acc, in, U, hp, st, site, b.y, b.z, s, rbase);
    hop_term<P, 2, true, DAG, 1>(acc, in, U, hp, st, site, 0, f.w, s, rbase);
    hop_term<P, 2, false, DAG, 1>(acc, in, U, hp, st, site, b.z, b.w, s, rbase);
    hop_term<P, 3, true, DAG, 1>(acc, in, U, hp, st, site, 0, -1, s, rbase);
    hop_term<P, 3, false, DAG, 0>(acc, in, U, hp, st, site, b.w, -1, s, rbase);
}

// ------------------------------------------ register double buffer
//
// The prefetch variant (STAGE == 3) keeps two neighbour spinors in registers:
// the load of term T + 1 is issued before term T is projected and transported,
// so every thread has the next neighbour in flight while it computes. It
// trades occupancy (72 registers, 7 blocks of 128 threads per SM, against 64
// and 8 for the plain loads) for memory-level parallelism per thread.

constexpr int kPrefetchMinBlocks = 7;

template <int T> struct TermOf {
    static constexpr int MU = T / 2;
    static constexpr bool FWD = T % 2 == 0;
    static constexpr int NB = FWD ? MU : 4 + MU;  // slot in the neighbour table
};

template <int P, int T, bool DAG, typename R>
__device__ __forceinline__ void pf_term(R* acc, const Field<P>& in, const Gauge<P>& U, const HopParams<R>& hp,
                                        const int* nbi, long long site, int s, long long rbase, const R* cur,
                                        R fcur, R* nxt, R& fnxt) {
    constexpr int MU = TermOf<T>::MU;
    constexpr bool FWD = TermOf<T>::FWD;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int S = FWD ? SF : -SF;
    if constexpr (T < 7) {
        const long long jn = __ldg(nbi + TermOf<T + 1>::NB);
        fnxt = load_input<P, false>(in, rbase + jn, s, hp.g.Ls, R(1), R(0), R(0), nxt);
    }
    R h[12], u[18];
    project<MU, S>(cur, h);
    if constexpr (FWD) {
        U.load(((long long)hp.out_parity * 4 + MU) * hp.g.Vh + site, u);
    } else {
        const long long jb = __ldg(nbi + TermOf<T>::NB);
        U.load(((long long)(1 - hp.out_parity) * 4 + MU) * hp.g.Vh + jb, u);
    }
    const bool tm = MU == 3 && hp.chem;
    transport_add<!FWD, MU, S>(acc, u, h, tm ? fcur * (FWD ? hp.efwd : hp.ebwd) : fcur, P == MDWF_F16N || tm);
}

template <int P, bool DAG, typename R>
__device__ __forceinline__ void hop_prefetch(R* acc, const Field<P>& in, const Gauge<P>& U, const HopParams<R>& hp,
                                             const int* nbi, long long site, int s, long long rbase) {
    R wa[24], wb[24];
    R fa, fb = R(1);
    fa = load_input<P, false>(in, rbase + __ldg(nbi + TermOf<0>::NB), s, hp.g.Ls, R(1), R(0), R(0), wa);
    pf_term<P, 0, DAG>(acc, in, U, hp, nbi, site, s, rbase, wa, fa, wb, fb);
    pf_term<P, 1, DAG>(acc, in, U, hp, nbi, site, s, rbase, wb, fb, wa, fa);
    pf_term<P, 2, DAG>(acc, in, U, hp, nbi, site, s, rbase, wa, fa, wb, fb);
    pf_term<P, 3, DAG>(acc, in, U, hp, nbi, site, s, rbase, wb, fb, wa, fa);
    pf_term<P, 4, DAG>(acc, in, U, hp, nbi, site, s, rbase, wa, fa, wb, fb);
    pf_term<P, 5, DAG>(acc, in, U, hp, nbi, site, s, rbase, wb, fb, wa, fa);
    pf_term<P, 6, DAG>(acc, in, U, hp, nbi, site, s, rbase, wa, fa, wb, fb);
    pf_term<P, 7, DAG>(acc, in, U, hp, nbi, site, s, rbase, wb, fb, wa, fa);
}

// ------------------------------------------ bulk copies of neighbour columns
//
// The bulk variant (STAGE == 2) lets the copy engine (TMA, cp.async.bulk)
// fetch whole neighbour columns: in the [site][chunk][s] layout the Ls
// spinors of a 4d site are one contiguous run of 96 Ls bytes (FP32), so one
// instruction of the row's s = 0 thread moves a column into shared memory
// while the threads compute the previous hopping term; the threads spend no
// load instructions on the global copy. Two buffers [2][SB][column] alternate
// over the eight terms, each with an mbarrier that counts the bytes of the
// SB copies of its term. Every wait is bounded: after kWaitLimit polls it sets
// the device error word and gives up (the results are then not valid; the
// host reports MDWF_ETIMEOUT).

template <int P> struct BulkBytes { static constexpr int value = 0; };  // per slice of a column
template <> struct BulkBytes<MDWF_F32> { static constexpr int value = 96; };
template <> struct BulkBytes<MDWF_F16N> { static constexpr int value = 52; };

template <int P> struct Bulk;
template <> struct Bulk<MDWF_F32> {
    float4* buf;  // [2][SB][6 Ls]
    int Ls, SB;
    __device__ __forceinline__ void issue(const Field<MDWF_F32>& in, long long sr, int slot, int ly,
                                          unsigned long long* bar) const {
        const unsigned bytes = 96u * (unsigned)Ls;
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(buf + ((size_t)slot * SB + ly) * 6 * Ls, in.v + sr * 6 * Ls, bytes, bar);
    }
    __device__ __forceinline__ float read(int slot, int ly, int s, float* w) const {
        const float4* p = buf + ((size_t)slot * SB + ly) * 6 * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 d = p[k * Ls];
            w[4 * k] = d.x; w[4 * k + 1] = d.y; w[4 * k + 2] = d.z; w[4 * k + 3] = d.w;
        }
        return 1.0f;
    }
};
template <> struct Bulk<MDWF_F16N> {
    uint2* buf;  // [2][SB][6 Ls]
    float* nrm;  // [2][SB][Ls]
    int Ls, SB;
    __device__ __forceinline__ void issue(const Field<MDWF_F16N>& in, long long sr, int slot, int ly,
                                          unsigned long long* bar) const {
        mbar_arrive_expect_tx(bar, 52u * (unsigned)Ls);
        bulk_g2s(buf + ((size_t)slot * SB + ly) * 6 * Ls, in.v + sr * 6 * Ls, 48u * (unsigned)Ls, bar);
        bulk_g2s(nrm + ((size_t)slot * SB + ly) * Ls, in.norm + sr * Ls, 4u * (unsigned)Ls, bar);
    }
    // values without the norm (applied to the transported half spinor); returns the norm
    __device__ __forceinline__ float read(int slot, int ly, int s, float* w) const {
        const uint2* p = buf + ((size_t)slot * SB + ly) * 6 * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; ++k) Field<MDWF_F16N>::unpack_raw(p[k * Ls], w + 4 * k);
        return nrm[((size_t)slot * SB + ly) * Ls + s];
    }
};

// Hopping term T (0..7 = mu 0 forward, mu 0 backward, mu 1 forward, ...) from
// buffer T % 2: wait for its columns, project, release the buffer to the copy
// of term T + 2 (neighbour `next`), then transport and accumulate. Every
// thread of the block takes part in the waits and barriers.
template <int P, int T, bool DAG, typename R>
__device__ __forceinline__ void bulk_term(R* acc, const Field<P>& in, const Gauge<P>& U, const HopParams<R>& hp,
                                          const Bulk<P>& bk, unsigned long long* bars, bool& ok, bool active,
                                          long long site, int jb, int next, int s, int ly, long long rbase) {
    constexpr int MU = T / 2, SLOT = T % 2;
    constexpr bool FWD = SLOT == 0;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int S = FWD ? SF : -SF;
    if (ok && !mbar_wait(bars + SLOT, (T / 2) & 1)) {
        ok = false;
        atomicOr(hp.err, 1);
    }
    R h[12], f = R(1);
    if (active) {
        R w[24];
        f = bk.read(SLOT, ly, s, w);
        project<MU, S>(w, h);
    }
    if (T + 2 < 8) {
        __syncthreads();  // every thread is done with this buffer
        if (s == 0) {
            if (active && ok) {
                fence_proxy_async();
                bk.issue(in, rbase + next, SLOT, ly, bars + SLOT);
            } else {
                mbar_arrive(bars + SLOT);
            }
        }
    }
    if (active) {
        R u[18];
        if (FWD) U.load(((long long)hp.out_parity * 4 + MU) * hp.g.Vh + site, u);
        else U.load(((long long)(1 - hp.out_parity) * 4 + MU) * hp.g.Vh + jb, u);
        const bool tm = MU == 3 && hp.chem;
        transport_add<!FWD, MU, S>(acc, u, h, tm ? f * (FWD ? hp.efwd : hp.ebwd) : f, P == MDWF_F16N || tm);
    }
}

// The eight terms, two neighbour columns in flight per site row. bars[0..1]
// are initialised here with one arrival per site row of the block.
template <int P, bool DAG, typename R>
__device__ __forceinline__ void hop_bulk(R* acc, const Field<P>& in, const Gauge<P>& U, const HopParams<R>& hp,
                                         const Bulk<P>& bk, unsigned long long* bars, bool active, long long site,
                                         int s, int ly, int tid, long long rbase) {
    int4 f = make_int4(0, 0, 0, 0), b = f;
    if (active) {
        const int4* nb = hp.nbr + ((long long)hp.out_parity * hp.g.Vh + site) * 2;
        f = __ldg(nb);
        b = __ldg(nb + 1);
    }
    if (tid == 0) {
        mbar_init(bars, (unsigned)bk.SB);
        mbar_init(bars + 1, (unsigned)bk.SB);
        mbar_init_fence();
    }
    __syncthreads();
    bool ok = true;
    if (s == 0) {
        if (active) {
            bk.issue(in, rbase + f.x, 0, ly, bars);
            bk.issue(in, rbase + b.x, 1, ly, bars + 1);
        } else {
            mbar_arrive(bars);
            mbar_arrive(bars + 1);
        }
    }
    bulk_term<P, 0, DAG>(acc, in, U, hp, bk, bars, ok, active, site, 0, f.y, s, ly, rbase);
    bulk_term<P, 1, DAG>(acc, in, U, hp, bk, bars, ok, active, site, b.x, b.y, s, ly, rbase);
    bulk_term<P, 2, DAG>(acc, in, U, hp, bk, bars, ok, active, site, 0, f.z, s, ly, rbase);
    bulk_term<P, 3, DAG>(acc, in, U, hp, bk, bars, ok, active, site, b.y, b.z, s, ly, rbase);
    bulk_term<P, 4, DAG>(acc, in, U, hp, bk, bars, ok, active, site, 0, f.w, s, ly, rbase);
    bulk_term<P, 5, DAG>(acc, in, U, hp, bk, bars, ok, active, site, b.z, b.w, s, ly, rbase);
    bulk_term<P, 6, DAG>(acc, in, U, hp, bk, bars, ok, active, site, 0, -1, s, ly, rbase);
    bulk_term<P, 7, DAG>(acc, in, U, hp, bk, bars, ok, active, site, b.w, -1, s, ly, rbase);
}

// Fused CG epilogues (structured s-operators only):
//   FUSE_T : after out = t = M p is formed, also write v = A^dag t (the first
//            factor of M^dag) to out2 and the block's partial |t|^2 to part
//   FUSE_R : out = Ap = M^dag t is not stored; instead r -= alpha Ap in the
//            residual field (precision PR) and the partial |r|^2 goes to part
enum { FUSE_NONE = 0, FUSE_T = 1, FUSE_R = 2 };

// The bidiagonal s-operators (M_phi = b5 + c5 C, C, I = M+ + M- C, and their
// adjoints) for Ls = 16, where the 16 slices of a site fill one half-warp:
// the s +- 1 neighbours of a column are lanes +- 1 of its 16-lane group, so
// the column step needs shuffles and no shared memory. Chirality 0 (reals
// 0..11) couples to s - 1 and chirality 1 to s + 1; the adjoint (swap)
// exchanges them; the wrap-around term carries -m. Every lane of the warp
// must take part.
template <typename R>
__device__ __forceinline__ void bidiag_shuffle16(const R* in, R* out, int s, int op, bool swap, const SCoef<R>& sc,
                                                 R m) {
    const R w0 = op == SOP_MPHI ? sc.b5 : op == SOP_MEE ? sc.Mp : R(0);
    const R w1 = op == SOP_MPHI ? sc.c5 : op == SOP_MEE ? sc.Mm : R(1);
    const int up = (s + 1) & 15, dn = (s + 15) & 15;
    const int src0 = swap ? up : dn, src1 = swap ? dn : up;
    const R f0 = w1 * ((swap ? s < 15 : s > 0) ? R(1) : -m);
    const R f1 = w1 * ((swap ? s > 0 : s < 15) ? R(1) : -m);
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = w0 * in[k] + f0 * __shfl_sync(0xffffffffu, in[k], src0, 16);
#pragma unroll
    for (int k = 12; k < 24; ++k) out[k] = w0 * in[k] + f1 * __shfl_sync(0xffffffffu, in[k], src1, 16);
}

// res = Mat col for the thread's slice s: Mat is the [chir][s'][s] table of one
// right-hand side in shared memory, col the block row of the thread's site.
template <typename R>
__device__ __forceinline__ void dense_columns(const R* mat, const R* col, int s, int Ls, R* res) {
#pragma unroll
    for (int k = 0; k < 24; ++k) res[k] = 0;
    for (int sp = 0; sp < Ls; ++sp) {
        const R mp = mat[sp * Ls + s];         // (s, s') of the P+ matrix
        const R mm = mat[(Ls + sp) * Ls + s];  // (s, s') of the P- matrix
        const R* h = col + sp * kRowStride;
#pragma unroll
        for (int k = 0; k < 12; ++k) res[k] += mp * h[k];
#pragma unroll
        for (int k = 12; k < 24; ++k) res[k] += mm * h[k];
    }
}

template <int P> struct ResPrec { static constexpr int value = P == MDWF_F64 ? MDWF_F64 : MDWF_F32; };

template <int P> struct FuseArgs {
    Field<P> out2;                     // FUSE_T: v = A^dag t
    Field<ResPrec<P>::value> rf;       // FUSE_R: residual r
    double* part;                      // [rhs][blocks per rhs] partial sums
    const double* sc;                  // CG scalars [slot][kMaxRhs]
};

// Block sum of the epilogue's squared norms: the lanes of a warp add in the
// precision A of their partial (a fixed shuffle tree), each warp's sum goes
// to FP64, and thread 0 adds the warps in FP64 in a fixed order. For the FP32
// and FP16+norm operators A is FP32: a lane sums its 24 squares and the warp
// tree 32 lanes, so the rounding is bounded by about 28 ulp of the warp sum
// (2e-6 relative), the FP32 rounding of the vectors themselves; the sums over
// warps and blocks, which the CG scalars take, stay in FP64. Squares and
// conversions in FP64 per element would put 48 FP64 instructions per thread
// on a pipe that runs at 1/64 of the FP32 rate.
template <typename A>
__device__ __forceinline__ double block_sum128(A v, double* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    if ((tid & 31) == 0) red[tid >> 5] = (double)v;
    __syncthreads();
    double tot = 0;
    if (tid == 0)
        for (int w = 0; w < (nthr + 31) / 32; ++w) tot += red[w];
    return tot;
}

// shared memory of a hop block: [4 doubles: block reduction][2 mbarriers] then
// the dense tables and the rows / staging buffers
constexpr int kHopHeader = 4 * sizeof(double) + 2 * sizeof(unsigned long long);

#ifndef MDWF_EPILOGUE_PREFETCH
#define MDWF_EPILOGUE_PREFETCH 1
#endif
constexpr bool kEpiloguePrefetch = MDWF_EPILOGUE_PREFETCH != 0;
#ifndef MDWF_SHUFFLE_BIDIAG
#define MDWF_SHUFFLE_BIDIAG 1
#endif
constexpr bool kShuffleBidiag = MDWF_SHUFFLE_BIDIAG != 0;

#ifndef MDWF_MINB_STAGE
#define MDWF_MINB_STAGE 6
#endif

// STAGE: 0 neighbour spinors loaded into registers, 1 staged per thread with
// cp.async, 2 whole neighbour columns copied by the copy engine (bulk).
// LSR: Ls fixed at compile time for the epilogue's register-held columns (the
// launcher picks it when Ls matches), or -1 for the run-time choice; one
// fixed length leaves the other lengths' code and its register demand out of
// the kernel.
template <int P, bool GATHER, bool DAG, bool XPAY, int FUSE, int STAGE, int LSR, bool DD = false>
__global__ void __launch_bounds__(128, STAGE == 1   ? MDWF_MINB_STAGE
                                      : STAGE == 3 ? kPrefetchMinBlocks
                                                   : PrecTraits<P>::min_blocks - (GATHER ? 1 : 0))
    hop_kernel(Field<P> out, Field<P> in, Field<P> xf, Gauge<P> U, HopParams<typename PrecTraits<P>::real> hp,
               FuseArgs<P> fa) {
    static_assert(!STAGE || (!GATHER && P != MDWF_F64), "staged loads: FP32 / FP16 operators without gather");
    static_assert(!DD || (STAGE == 0 && !GATHER && FUSE == FUSE_NONE), "slab halos: plain loads, unfused");
    typedef typename PrecTraits<P>::real R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = hp.g.Ls;
    const bool dense = hp.sop == SOP_DENSE;
    double* red = reinterpret_cast<double*>(smem_raw);          // [4] block reduction
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem_raw + 4 * sizeof(double));  // [2]
    R* mat = reinterpret_cast<R*>(smem_raw + kHopHeader);       // [chir][s'][s] (dense only)
    R* mat2 = mat + (dense ? 2 * Ls * Ls : 0);                    // A^dag (dense FUSE_T only)
    R* hs = mat2 + (dense && FUSE == FUSE_T ? 2 * Ls * Ls : 0);   // [SB][site_stride], rows of kRowStride
    const int s = threadIdx.x, ly = threadIdx.y;
    const int rhs = blockIdx.x % hp.nrhs;
    const long long sblk = blockIdx.x / hp.nrhs;
    const int tid = ly * blockDim.x + s, nthr = blockDim.x * blockDim.y;
    if (dense) {
        const R* gm = hp.mat + (size_t)rhs * 2 * Ls * Ls;
        for (int i = tid; i < 2 * Ls * Ls; i += nthr) mat[i] = gm[i];
        if (FUSE == FUSE_T) {
            const R* gm2 = hp.mat2 + (size_t)rhs * 2 * Ls * Ls;
            for (int i = tid; i < 2 * Ls * Ls; i += nthr) mat2[i] = gm2[i];
        }
    }
    const long long site = sblk * blockDim.y + ly;
    const bool active = site < hp.g.Vh;
    const long long rbase = (long long)rhs * hp.g.Vh;
    const R mass = hp.mass[rhs];
    R gown = hp.gown, gfac = hp.gfac, gpre = R(1);
    if (GATHER && hp.gs) {
        gown = hp.gs[s];
        gfac = hp.gs[64 + s];
        gpre = hp.gs[128 + s];
    }
    // the site's eight links into L1 before the terms need them (the links come from
    // L2, and a link load that waits for L2 inside a term stalls its chain): thread s
    // of the column asks for the lines of link s / 2 (forward links at the site,
    // backward ones at the neighbour), two lines per 80-byte FP32 link. The links and
    // the neighbour table do not change during a solve, so this runs before the wait
    // for the previous kernel.
    if constexpr (P != MDWF_F64 && STAGE != 2) {
        if (active && s < 16) {
            const int* nbi = reinterpret_cast<const int*>(hp.nbr + ((long long)hp.out_parity * hp.g.Vh + site) * 2);
            const int t = s >> 1, mu = t & 3;
            const bool fwd = t < 4;
            const long long j = fwd ? site : (long long)__ldg(nbi + 4 + mu);
            const long long li = ((long long)(fwd ? hp.out_parity : 1 - hp.out_parity) * 4 + mu) * hp.g.Vh + j;
            if (j >= 0) prefetch_l1(reinterpret_cast<const char*>(U.u + li * 5) + (s & 1) * 64);  // halo: none
        }
    }
    pdl_wait();
    pdl_release();
    // a right-hand side left out of this launch (block-uniform: before any barrier)
    if (hp.mask && hp.mask[rhs] == 0.0) return;
    R acc[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0;
    if constexpr (STAGE == 2) {
        // the buffers alias the rows of the epilogue (used after a barrier)
        Bulk<P> bk;
        bk.Ls = Ls;
        bk.SB = blockDim.y;
        if constexpr (P == MDWF_F32) {
            bk.buf = reinterpret_cast<float4*>(hs);
        } else {
            bk.buf = reinterpret_cast<uint2*>(hs);
            bk.nrm = reinterpret_cast<float*>(bk.buf + (size_t)2 * blockDim.y * 6 * Ls);
        }
        hop_bulk<P, DAG>(acc, in, U, hp, bk, bars, active, site, s, ly, tid, rbase);
    } else if (active) {
        const int4* nb = hp.nbr + ((long long)hp.out_parity * hp.g.Vh + site) * 2;
        if constexpr (STAGE == 3) {
            hop_prefetch<P, DAG>(acc, in, U, hp, reinterpret_cast<const int*>(nb), site, s, rbase);
        } else if constexpr (STAGE == 1) {
            const int4 f = __ldg(nb), b = __ldg(nb + 1);
            // the staging buffers alias the rows of the epilogue (used after a barrier)
            Stager<P> st;
            if constexpr (P == MDWF_F32) {
                st.buf = reinterpret_cast<float4*>(hs);
            } else {
                st.buf = reinterpret_cast<uint2*>(hs);
                st.nrm = reinterpret_cast<float*>(st.buf + 2 * 6 * nthr);
            }
            st.nthr = nthr;
            st.tid = tid;
            hop_staged<P, DAG>(acc, in, U, hp, st, f, b, site, s, rbase);
        } else {
            const int* nbi = reinterpret_cast<const int*>(nb);
            hop_dir<P, 0, GATHER, DAG, DD>(acc, in, U, hp, nbi, site, s, rbase, mass, gown, gfac, rhs);
            hop_dir<P, 1, GATHER, DAG, DD>(acc, in, U, hp, nbi, site, s, rbase, mass, gown, gfac, rhs);
            hop_dir<P, 2, GATHER, DAG, DD>(acc, in, U, hp, nbi, site, s, rbase, mass, gown, gfac, rhs);
            hop_dir<P, 3, GATHER, DAG, DD>(acc, in, U, hp, nbi, site, s, rbase, mass, gown, gfac, rhs);
        }
    }
    if constexpr (STAGE == 1 || STAGE == 2) __syncthreads();
    // the epilogue's own operands (xpay addend, residual) are fetched into L1
    // while the s-operator runs on the shared-memory rows
    if (active && kEpiloguePrefetch) {
        if constexpr (XPAY) xf.prefetch(rbase + site, s);
        if constexpr (FUSE == FUSE_R) fa.rf.prefetch(rbase + site, s);
    }
    if (GATHER && hp.gs) {
#pragma unroll
        for (int k = 0; k < 24; ++k) acc[k] *= gpre;
    }
    if constexpr (FUSE == FUSE_T && XPAY && LSR == 16) {
        // t not stored (closed form, Ls = 16, two columns per warp): the rows go
        // to the column pass as y = cf acc + I p (I = M+ + M- C bidiagonal, by
        // shuffles), so that one pass forms t = A y = cf A acc + p, adds |t|^2
        // and turns t into v = A^dag t: one shared-memory round trip, not two
        if (hp.no_t && !dense && (blockDim.y & 1) == 0) {
            const R cf = hp.coef * hp.gscale;
            R xv[24], y[24];
            if (active) {
                xf.load(rbase + site, s, xv);
            } else {
#pragma unroll
                for (int k = 0; k < 24; ++k) xv[k] = R(0);
            }
            bidiag_shuffle16(xv, y, s, SOP_MEE, false, hp.sc, mass);
#pragma unroll
            for (int k = 0; k < 24; ++k) y[k] = active ? fma(cf, acc[k], y[k]) : R(0);
            R* row = hs + (size_t)ly * site_stride(16) + s * kRowStride;
            row_store(row, y);
            __syncthreads();
            const R sq = block_columns_a_adag<16>(hs, blockDim.y, hp.sc, mass, tid, nthr);
            __syncthreads();
            if (active) {
                row_load(row, y);
                fa.out2.store(rbase + site, s, y);
            }
            const double tot = block_sum128(sq, red);
            if (tid == 0) fa.part[(size_t)rhs * (gridDim.x / hp.nrhs) + sblk] = tot;
            return;
        }
    }
    const int sst = site_stride(Ls);
    R* mine = hs + (size_t)ly * sst + s * kRowStride;
    R res[24];
    // bidiagonal operators at Ls = 16 by shuffles when every warp holds two
    // whole columns (uniform over the block)
    bool shuffled = false;
    if constexpr (LSR == 16) {
        if (kShuffleBidiag && !dense && (blockDim.y & 1) == 0 &&
            (hp.sop == SOP_MPHI || hp.sop == SOP_C || hp.sop == SOP_MEE)) {
            bidiag_shuffle16(acc, res, s, hp.sop, hp.swap != 0, hp.sc, mass);
            shuffled = true;
        }
    }
    if (!shuffled) {
        row_store(mine, acc);
        __syncthreads();
        if (dense) {
            dense_columns(mat, hs + (size_t)ly * sst, s, Ls, res);
        } else {
            block_columns<LSR>(hs, blockDim.y, Ls, hp.sop, hp.swap != 0, hp.sc, mass, tid, nthr);
            __syncthreads();
            row_load(mine, res);
        }
    }
    if (FUSE == FUSE_NONE && !active) return;
    const R cf = hp.coef * hp.gscale;
    bool xdone = false;
    if constexpr (XPAY && FUSE == FUSE_R && LSR == 16) {
        // x holds v = A^dag t: the addend t = I^dag v, I^dag = M+ + M- C^dag
        // bidiagonal, by shuffles (every lane takes part; the launcher admits
        // no_t only where the shuffled s-operators run)
        if (hp.no_t) {
            R xv[24], tv[24];
            if (active) {
                xf.load(rbase + site, s, xv);
            } else {
#pragma unroll
                for (int k = 0; k < 24; ++k) xv[k] = R(0);
            }
            bidiag_shuffle16(xv, tv, s, SOP_MEE, true, hp.sc, mass);
#pragma unroll
            for (int k = 0; k < 24; ++k) res[k] = fma(cf, res[k], tv[k]);
            xdone = true;
        }
    }
    if (xdone) {
    } else if (XPAY && active) {  // res = cf res + x as one fused multiply-add
        R xv[24];
        xf.load(rbase + site, s, xv);
#pragma unroll
        for (int k = 0; k < 24; ++k) res[k] = fma(cf, res[k], xv[k]);
    } else {
#pragma unroll
        for (int k = 0; k < 24; ++k) res[k] *= cf;
    }
    if (FUSE == FUSE_NONE) {
        out.store(rbase + site, s, res);
        return;
    }
    R sq = 0;  // squared norm partial in the operator's arithmetic precision
    if (FUSE == FUSE_T) {
        if (active) {
            if (!hp.no_t) out.store(rbase + site, s, res);
#pragma unroll
            for (int k = 0; k < 24; ++k) sq = fma(res[k], res[k], sq);
        }
        // v = A^dag t through the same column machinery
        __syncthreads();
        if (!active) {
#pragma unroll
            for (int k = 0; k < 24; ++k) res[k] = R(0);
        }
        row_store(mine, res);
        __syncthreads();
        if (dense) {
            dense_columns(mat2, hs + (size_t)ly * sst, s, Ls, res);
            if (active) fa.out2.store(rbase + site, s, res);
        } else {
            block_columns<LSR>(hs, blockDim.y, Ls, SOP_A, true, hp.sc, mass, tid, nthr);
            __syncthreads();
            if (active) {
                row_load(mine, res);
                fa.out2.store(rbase + site, s, res);
            }
        }
    } else {  // FUSE_R
        typedef typename PrecTraits<ResPrec<P>::value>::real RR;
        const bool live = fa.sc[S_ACTIVE * kMaxRhs + rhs] != 0.0;
        if (active && live) {
            const RR alpha = (RR)fa.sc[S_ALPHA * kMaxRhs + rhs];
            RR rv[24];
            fa.rf.load(rbase + site, s, rv);
#pragma unroll
            for (int k = 0; k < 24; ++k) {
                rv[k] -= alpha * (RR)res[k];
                sq = fma((R)rv[k], (R)rv[k], sq);
            }
            fa.rf.store(rbase + site, s, rv);
        }
    }
    const double tot = block_sum128(sq, red);
    if (tid == 0) fa.part[(size_t)rhs * (gridDim.x / hp.nrhs) + sblk] = tot;
}

// ---------------------------------------------------------------- launcher

template <int P, bool G, bool D, bool X, int FU, int ST, int LSR, bool DD = false>
static int launch_hop_variant(mdwf_ctx* c, const HopLaunch& h, const HopParams<typename PrecTraits<P>::real>& hp) {
    typedef typename PrecTraits<P>::real R;
    const Geom& g = c->g;
    const int SB = hop_sites_per_block(c, P, h.nrhs);
    dim3 block(g.Ls, SB), grid((unsigned)((g.Vh + SB - 1) / SB * h.nrhs));
    const size_t rows = (size_t)SB * site_stride(g.Ls) * sizeof(R);
    const size_t stage = ST == 1 ? (size_t)StageBytes<P>::value * g.Ls * SB
                         : ST == 2 ? (size_t)2 * BulkBytes<P>::value * g.Ls * SB : 0;
    const int ntab = hp.sop == SOP_DENSE ? (FU == FUSE_T ? 2 : 1) : 0;
    size_t smem = kHopHeader + (size_t)ntab * 2 * g.Ls * g.Ls * sizeof(R) + (rows > stage ? rows : stage);
    auto kern = hop_kernel<P, G, D, X, FU, ST, LSR, DD>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (ST == 1 || ST == 2) {
        // the staging buffers need shared memory for every resident block (once per device)
        // (contexts on other host threads may launch at the same time: the mask is atomic, and
        // setting the attribute twice is harmless)
        static std::atomic<unsigned long long> carved{0};
        if (c->device < 64 && !(carved.load() >> c->device & 1ull)) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                                 (int)cudaSharedmemCarveoutMaxShared);
            if (e != cudaSuccess) return cuda_status(e);
            carved.fetch_or(1ull << c->device);
        }
    }
    Field<P> out = make_field<P>(h.out, g, h.nrhs);
    Field<P> in = make_field<P>(const_cast<void*>(h.in), g, h.nrhs);
    Field<P> xf = h.x ? make_field<P>(const_cast<void*>(h.x), g, h.nrhs) : out;
    FuseArgs<P> fa;
    fa.out2 = make_field<P>(h.out2 ? h.out2 : h.out, g, h.nrhs);
    fa.rf = make_field<ResPrec<P>::value>(h.rfield ? h.rfield : h.out, g, h.nrhs);
    fa.part = h.part;
    fa.sc = h.sc;
    Gauge<P> U;
    U.u = reinterpret_cast<decltype(U.u)>(c->gauge[link_copy(P)]);
    U.bnd = make_bounds(8 * g.Vh);
    const int base = D ? (X ? KB_HOP_DAG_XPAY : KB_HOP_DAG)
                       : G ? (X ? KB_HOP_GATHER_XPAY : KB_HOP_GATHER) : (X ? KB_HOP_XPAY : KB_HOP);
    const double n5 = (double)g.Vh * g.Ls * h.nrhs;
    // fields moved: in, out (+x), and for the fused epilogues v (FUSE_T) or r read+write instead of out (FUSE_R)
    const double sp = site_bytes(P), sr = site_bytes(ResPrec<P>::value);
    double fields = sp + sp + (X ? sp : 0.0);
    if (FU == FUSE_T && !hp.no_t) fields += sp;  // t (out) and v (out2); no_t stores only v
    if (FU == FUSE_R) fields += 2.0 * sr - sp;
    const double bytes = n5 * fields + 8.0 * g.Vh * link_bytes(P);
    const double flops = n5 * (1320.0 + (G ? 72.0 : 0.0) + 144.0 + (X ? 48.0 : 0.0) + (FU ? 144.0 : 0.0));
    LaunchScope scope(c, base * 3 + P, bytes, flops);
    if (cudaError_t e = launch_pdl(kern, grid, block, smem, c->stream, out, in, xf, U, hp, fa)) return cuda_status(e);
    return check_launch();
}

// Load strategy per launch (mdwf_set_staging). The FP32 and FP16 operators
// without the input gather have the staged variants; by default (mode 0, and
// mode 3) they prefetch the next neighbour into registers. Mode 4 uses the
// plain loads everywhere.
template <int P, bool G, bool D, bool X, int FU>
static int launch_hop_pick(mdwf_ctx* c, const HopLaunch& h, const HopParams<typename PrecTraits<P>::real>& hp) {
    if constexpr (!G && FU == FUSE_NONE && P != MDWF_F16N) {
        if (h.halo) return launch_hop_variant<P, G, D, X, FU, 0, -1, true>(c, h, hp);
    }
    if (h.halo) return MDWF_EINVAL;
    if constexpr (!G && P != MDWF_F64) {
        const int mode = c->hop_stage[P];
        if (mode == 1) return launch_hop_variant<P, G, D, X, FU, 1, -1>(c, h, hp);
        if (mode == 2) return launch_hop_variant<P, G, D, X, FU, 2, -1>(c, h, hp);
        if (mode == 3 || mode == 0) {
            if (c->g.Ls == 16) return launch_hop_variant<P, G, D, X, FU, 3, 16>(c, h, hp);
            return launch_hop_variant<P, G, D, X, FU, 3, -1>(c, h, hp);
        }
    }
    // the FP32 / FP16 operators at Ls = 16 (the common length) with the
    // column length fixed at compile time
    if constexpr (P != MDWF_F64) {
        if (c->g.Ls == 16) return launch_hop_variant<P, G, D, X, FU, 0, 16>(c, h, hp);
    }
    return launch_hop_variant<P, G, D, X, FU, 0, -1>(c, h, hp);
}

template <int P>
int launch_hop_t(mdwf_ctx* c, const HopLaunch& h) {
    typedef typename PrecTraits<P>::real R;
    HopParams<R> hp;
    hp.g = c->g;
    hp.nrhs = h.nrhs;
    hp.out_parity = h.out_parity;
    hp.coef = (R)h.coef;
    // M_phi = b5 + c5 C folded as b5 (1 + (c5/b5) C) when b5 != 0
    if (h.b5 != 0.0) {
        hp.gown = R(1); hp.gfac = (R)(h.c5 / h.b5); hp.gscale = (R)h.b5;
    } else {
        hp.gown = R(0); hp.gfac = (R)h.c5; hp.gscale = R(1);
    }
    if (!h.gather) { hp.gown = R(1); hp.gfac = R(0); hp.gscale = R(1); }
    hp.gs = nullptr;
    if (h.gather && c->sdep) {
        hp.gown = R(1); hp.gfac = R(0); hp.gscale = R(1);
        hp.gs = P == MDWF_F64 ? reinterpret_cast<const R*>(c->gs64) : reinterpret_cast<const R*>(c->gs32);
        if (h.sop != SOP_DENSE || !hp.gs) return MDWF_EINVAL;
    }
    hp.mass = reinterpret_cast<const R*>(h.mass);
    hp.mat = reinterpret_cast<const R*>(h.mat);
    hp.mat2 = reinterpret_cast<const R*>(h.mat2);
    hp.nbr = reinterpret_cast<const int4*>(c->nbr);
    hp.sop = h.sop;
    hp.swap = h.swap;
    hp.sc.b5 = (R)c->b5;
    hp.sc.c5 = (R)c->c5;
    hp.sc.Mp = (R)(c->b5 * (4.0 - c->M5) + 1.0);
    hp.sc.Mm = (R)(c->c5 * (4.0 - c->M5) - 1.0);
    // the adjoint's hopping matrix is transposed: the two factors exchange
    hp.chem = c->chem != 0.0;
    hp.efwd = (R)exp(h.dagger ? -c->chem : c->chem);
    hp.ebwd = (R)exp(h.dagger ? c->chem : -c->chem);
    hp.err = c->dev_err;
    hp.no_t = h.no_t != 0;
    hp.halo = h.halo;
    hp.mask = h.mask;
    if (h.mask && h.fuse != FUSE_NONE) return MDWF_EINVAL;  // the fused reductions cover every block
    hp.face = (long long)c->g.X * c->g.Y * c->g.Z / 2;
    // a t-slab context reads its t-faces from halos: every hop on it needs them
    if (c->slab != (h.halo != nullptr)) {
        set_error_message("a t-slab context applies its hops only through mdwf_slab_stage, with halos");
        return MDWF_EINVAL;
    }
    const bool X = h.x != nullptr;
    if (hp.no_t) {
        if (!hop_no_t_ok(c, P, h.nrhs) || h.fuse == FUSE_NONE || h.sop == SOP_DENSE) return MDWF_EINVAL;
        if (h.fuse == FUSE_R && h.sop != SOP_MPHI) return MDWF_EINVAL;
    }
    if (h.fuse != FUSE_NONE) {
        // fused CG epilogues: t = M p with v = A^dag t, or Ap = M^dag t folded into r
        // (structured s-operators or dense tables)
        if (!X || h.gather || !h.part || !h.sc) return MDWF_EINVAL;
        if (h.sop == SOP_DENSE && (!h.mat || (h.fuse == FUSE_T && !h.mat2))) return MDWF_EINVAL;
        if (h.fuse == FUSE_T && !h.dagger && h.out2) return launch_hop_pick<P, false, false, true, FUSE_T>(c, h, hp);
        if (h.fuse == FUSE_R && h.dagger && h.rfield) return launch_hop_pick<P, false, true, true, FUSE_R>(c, h, hp);
        return MDWF_EINVAL;
    }
    if (h.gather) {
        if (h.dagger) return MDWF_EINVAL;
        return X ? launch_hop_pick<P, true, false, true, FUSE_NONE>(c, h, hp)
                 : launch_hop_pick<P, true, false, false, FUSE_NONE>(c, h, hp);
    }
    if (h.dagger)
        return X ? launch_hop_pick<P, false, true, true, FUSE_NONE>(c, h, hp)
                 : launch_hop_pick<P, false, true, false, FUSE_NONE>(c, h, hp);
    return X ? launch_hop_pick<P, false, false, true, FUSE_NONE>(c, h, hp)
             : launch_hop_pick<P, false, false, false, FUSE_NONE>(c, h, hp);
}

}  // namespace mdwf
