// Fused hopping kernel of the red/black Moebius operator.
//
// One launch computes, for every site x of parity `out_parity` and every s,
//   out(x, s) = coef * sum_s' Mat_chi(s, s') [H w](x, s') (+ x_add(x, s))
// where H is the Wilson hopping sum of Eq. (D^Wilson),
//   H w(x) = sum_mu [(1 - g_mu) U_mu(x) w(x+mu) + (1 + g_mu) U_mu(x-mu)^dag w(x-mu)]
// (projector signs flipped for the hopping part of D_W^dag), and w is either
// the input field or the input with the fifth-dimension gather of Sec. 5
// applied first: w_s = b5 psi_s + c5 (P+ psi_{s-1} + P- psi_{s+1}) with the
// mass -m on the wrap-around terms (Eq. DWaction), i.e. w = M_phi psi.
// Mat is an Ls x Ls real matrix per chirality (K = M_phi I^-1, I^-1, ...).
//
// Thread mapping: a block is Ls x SB threads: threadIdx.x = s, threadIdx.y =
// one of SB 4d sites, blockIdx.y = right-hand side. The Ls threads of a
// column load the same link (one L1 line, broadcast), so each link is read
// from HBM once per hop and reused across all Ls slices. Spinor chunks of
// consecutive s are contiguous, so every vector load of a warp is coalesced.
// The s-mixing matrix is applied after the hop through shared memory.
#include "mdwf_internal.cuh"

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
    const R* mass;   // [rhs]
    const R* mat;    // dense tables [rhs][chir][s'][s] (sop == SOP_DENSE)
    const int4* nbr; // [parity][site][2] = cb index of x+mu (mu = 0..3), then of x-mu
    int sop, swap;
    SCoef<R> sc;
};

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

template <int MU, int S, typename R>
__device__ __forceinline__ void reconstruct_add(R* acc, const R* gin, R scale = R(1), bool scaled = false) {
    R g[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) g[k] = scaled ? scale * gin[k] : gin[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R g0r = g[2 * c], g0i = g[2 * c + 1], g1r = g[6 + 2 * c], g1i = g[7 + 2 * c];
        acc[2 * c] += g0r;
        acc[2 * c + 1] += g0i;
        acc[6 + 2 * c] += g1r;
        acc[7 + 2 * c] += g1i;
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
        acc[12 + 2 * c] += S * b0r;
        acc[13 + 2 * c] += S * b0i;
        acc[18 + 2 * c] += S * b1r;
        acc[19 + 2 * c] += S * b1i;
    }
}

// g[a][i] = sum_j V[i][j] h[a][j], V = U or U^dag; U row-major complex 3x3
template <bool ADJ, typename R>
__device__ __forceinline__ void su3_mul(const R* U, const R* h, R* g) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            R sr = 0, si = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const R ur = ADJ ? U[2 * (3 * j + i)] : U[2 * (3 * i + j)];
                const R ui = ADJ ? -U[2 * (3 * j + i) + 1] : U[2 * (3 * i + j) + 1];
                const R hr = h[6 * a + 2 * j], hi = h[6 * a + 2 * j + 1];
                sr += ur * hr - ui * hi;
                si += ur * hi + ui * hr;
            }
            g[6 * a + 2 * i] = sr;
            g[6 * a + 2 * i + 1] = si;
        }
}

// w = psi(s), or M_phi psi at s up to the factor gscale, for the neighbour column sr.
// Returns a factor still to be applied to w (the FP16 norm of an ungathered
// input, which is linear and is applied to the transported half spinor).
template <int P, bool GATHER, typename R>
__device__ __forceinline__ R load_input(const Field<P>& in, long long sr, int s, int Ls, const HopParams<R>& hp,
                                        R mass, R* w) {
    if constexpr (P == MDWF_F16N && !GATHER) {
        return in.load_raw(sr, s, w);
    }
    in.load(sr, s, w);
    if (GATHER) {
        if (hp.gown != R(1)) {
#pragma unroll
            for (int k = 0; k < 24; ++k) w[k] *= hp.gown;
        }
        if (hp.gfac != R(0)) {
            R t[12];
            const int sm = s > 0 ? s - 1 : Ls - 1;
            const R fm = s > 0 ? hp.gfac : -mass * hp.gfac;
            in.load_half(sr, sm, 0, t);  // P+ psi_{s-1}
#pragma unroll
            for (int k = 0; k < 12; ++k) w[k] += fm * t[k];
            const int sp = s < Ls - 1 ? s + 1 : 0;
            const R fp = s < Ls - 1 ? hp.gfac : -mass * hp.gfac;
            in.load_half(sr, sp, 1, t);  // P- psi_{s+1}
#pragma unroll
            for (int k = 0; k < 12; ++k) w[12 + k] += fp * t[k];
        }
    }
    return R(1);
}

template <int P, int MU, bool GATHER, bool DAG, typename R>
__device__ __forceinline__ void hop_dir(R* acc, const Field<P>& in, const Gauge<P>& U, const HopParams<R>& hp,
                                        long long jf, long long jb, long long site, int s, long long rbase, R mass) {
    const Geom& g = hp.g;
    constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF g_mu
    constexpr bool SCALED = P == MDWF_F16N && !GATHER;
    {
        R w[24], h[12], u[18], gg[12];
        const R f = load_input<P, GATHER>(in, rbase + jf, s, g.Ls, hp, mass, w);
        project<MU, SF>(w, h);
        U.load(((long long)hp.out_parity * 4 + MU) * g.Vh + site, u);
        su3_mul<false>(u, h, gg);
        reconstruct_add<MU, SF>(acc, gg, f, SCALED);
    }
    {
        R w[24], h[12], u[18], gg[12];
        const R f = load_input<P, GATHER>(in, rbase + jb, s, g.Ls, hp, mass, w);
        project<MU, -SF>(w, h);
        U.load(((long long)(1 - hp.out_parity) * 4 + MU) * g.Vh + jb, u);
        su3_mul<true>(u, h, gg);
        reconstruct_add<MU, -SF>(acc, gg, f, SCALED);
    }
}

// Fused CG epilogues (structured s-operators only):
//   FUSE_T : after out = t = M p is formed, also write v = A^dag t (the first
//            factor of M^dag) to out2 and the block's partial |t|^2 to part
//   FUSE_R : out = Ap = M^dag t is not stored; instead r -= alpha Ap in the
//            residual field (precision PR) and the partial |r|^2 goes to part
enum { FUSE_NONE = 0, FUSE_T = 1, FUSE_R = 2 };

template <int P> struct ResPrec { static constexpr int value = P == MDWF_F64 ? MDWF_F64 : MDWF_F32; };

template <int P> struct FuseArgs {
    Field<P> out2;                     // FUSE_T: v = A^dag t
    Field<ResPrec<P>::value> rf;       // FUSE_R: residual r
    double* part;                      // [rhs][blockIdx.x] partial sums
    const double* sc;                  // CG scalars [slot][64]: alpha at slot 2, active flag at slot 5
};

__device__ __forceinline__ double block_sum128(double v, double* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthr = blockDim.x * blockDim.y;
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double tot = 0;
    if (tid == 0)
        for (int w = 0; w < (nthr + 31) / 32; ++w) tot += red[w];
    return tot;
}

template <int P, bool GATHER, bool DAG, bool XPAY, int FUSE>
__global__ void __launch_bounds__(128, PrecTraits<P>::min_blocks - (GATHER ? 1 : 0))
    hop_kernel(Field<P> out, Field<P> in, Field<P> xf, Gauge<P> U, HopParams<typename PrecTraits<P>::real> hp,
               FuseArgs<P> fa) {
    typedef typename PrecTraits<P>::real R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = hp.g.Ls;
    const bool dense = hp.sop == SOP_DENSE;
    double* red = reinterpret_cast<double*>(smem_raw);          // [4] block reduction
    R* mat = reinterpret_cast<R*>(smem_raw + 4 * sizeof(double)); // [chir][s'][s] (dense only)
    R* hs = mat + (dense ? 2 * Ls * Ls : 0);                      // [SB][site_stride], rows of kRowStride
    const int s = threadIdx.x, ly = threadIdx.y;
    const int rhs = blockIdx.x % hp.nrhs;
    const long long sblk = blockIdx.x / hp.nrhs;
    const int tid = ly * blockDim.x + s, nthr = blockDim.x * blockDim.y;
    if (dense) {
        const R* gm = hp.mat + (size_t)rhs * 2 * Ls * Ls;
        for (int i = tid; i < 2 * Ls * Ls; i += nthr) mat[i] = gm[i];
    }
    const long long site = sblk * blockDim.y + ly;
    const bool active = site < hp.g.Vh;
    const long long rbase = (long long)rhs * hp.g.Vh;
    const R mass = hp.mass[rhs];
    R acc[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0;
    if (active) {
        const int4* nb = hp.nbr + ((long long)hp.out_parity * hp.g.Vh + site) * 2;
        const int4 f = __ldg(nb), b = __ldg(nb + 1);
        hop_dir<P, 0, GATHER, DAG>(acc, in, U, hp, f.x, b.x, site, s, rbase, mass);
        hop_dir<P, 1, GATHER, DAG>(acc, in, U, hp, f.y, b.y, site, s, rbase, mass);
        hop_dir<P, 2, GATHER, DAG>(acc, in, U, hp, f.z, b.z, site, s, rbase, mass);
        hop_dir<P, 3, GATHER, DAG>(acc, in, U, hp, f.w, b.w, site, s, rbase, mass);
    }
    const int sst = site_stride(Ls);
    R* mine = hs + (size_t)ly * sst + s * kRowStride;
    row_store(mine, acc);
    __syncthreads();
    R res[24];
    if (dense) {
#pragma unroll
        for (int k = 0; k < 24; ++k) res[k] = 0;
        const R* col = hs + (size_t)ly * sst;
        for (int sp = 0; sp < Ls; ++sp) {
            const R mp = mat[sp * Ls + s];         // (s, s') of the P+ matrix
            const R mm = mat[(Ls + sp) * Ls + s];  // (s, s') of the P- matrix
            const R* h = col + sp * kRowStride;
#pragma unroll
            for (int k = 0; k < 12; ++k) res[k] += mp * h[k];
#pragma unroll
            for (int k = 12; k < 24; ++k) res[k] += mm * h[k];
        }
    } else {
        block_columns(hs, blockDim.y, Ls, hp.sop, hp.swap != 0, hp.sc, mass, tid, nthr);
        __syncthreads();
        row_load(mine, res);
    }
    if (FUSE == FUSE_NONE && !active) return;
    const R cf = hp.coef * hp.gscale;
#pragma unroll
    for (int k = 0; k < 24; ++k) res[k] *= cf;
    if (XPAY && active) {
        R xv[24];
        xf.load(rbase + site, s, xv);
#pragma unroll
        for (int k = 0; k < 24; ++k) res[k] += xv[k];
    }
    if (FUSE == FUSE_NONE) {
        out.store(rbase + site, s, res);
        return;
    }
    double sq = 0;
    if (FUSE == FUSE_T) {
        if (active) {
            out.store(rbase + site, s, res);
#pragma unroll
            for (int k = 0; k < 24; ++k) sq += (double)res[k] * (double)res[k];
        }
        // v = A^dag t through the same column machinery
        __syncthreads();
        if (!active) {
#pragma unroll
            for (int k = 0; k < 24; ++k) res[k] = R(0);
        }
        row_store(mine, res);
        __syncthreads();
        block_columns(hs, blockDim.y, Ls, SOP_A, true, hp.sc, mass, tid, nthr);
        __syncthreads();
        if (active) {
            row_load(mine, res);
            fa.out2.store(rbase + site, s, res);
        }
    } else {  // FUSE_R
        typedef typename PrecTraits<ResPrec<P>::value>::real RR;
        const bool live = fa.sc[5 * 64 + rhs] != 0.0;
        if (active && live) {
            const RR alpha = (RR)fa.sc[2 * 64 + rhs];
            RR rv[24];
            fa.rf.load(rbase + site, s, rv);
#pragma unroll
            for (int k = 0; k < 24; ++k) {
                rv[k] -= alpha * (RR)res[k];
                sq += (double)rv[k] * (double)rv[k];
            }
            fa.rf.store(rbase + site, s, rv);
        }
    }
    const double tot = block_sum128(sq, red);
    if (tid == 0) fa.part[(size_t)rhs * (gridDim.x / hp.nrhs) + sblk] = tot;
}

// ---------------------------------------------------------------- launcher

// 4d sites per block: the autotuned value for (precision, nrhs) if there is
// one, else as many whole s-columns as fit 128 threads.
int hop_sites_per_block(const mdwf_ctx* c, int prec, int nrhs) {
    const int t = (nrhs >= 1 && nrhs <= 64) ? c->sb_tune[prec][nrhs] : 0;
    if (t > 0) return t;
    const int sb = 128 / c->g.Ls;
    return sb < 1 ? 1 : sb;
}

int hop_blocks(const mdwf_ctx* c, int prec, int nrhs) {
    const int SB = hop_sites_per_block(c, prec, nrhs);
    return (int)((c->g.Vh + SB - 1) / SB);
}

template <int P, bool G, bool D, bool X, int FU>
static int launch_hop_variant(mdwf_ctx* c, const HopLaunch& h, const HopParams<typename PrecTraits<P>::real>& hp) {
    typedef typename PrecTraits<P>::real R;
    const Geom& g = c->g;
    const int SB = hop_sites_per_block(c, P, h.nrhs);
    dim3 block(g.Ls, SB), grid((unsigned)((g.Vh + SB - 1) / SB * h.nrhs));
    size_t smem = 4 * sizeof(double) + (size_t)((hp.sop == SOP_DENSE ? 2 * g.Ls * g.Ls : 0) + SB * site_stride(g.Ls)) * sizeof(R);
    auto kern = hop_kernel<P, G, D, X, FU>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_status(e);
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
    const int base = D ? (X ? KB_HOP_DAG_XPAY : KB_HOP_DAG)
                       : G ? (X ? KB_HOP_GATHER_XPAY : KB_HOP_GATHER) : (X ? KB_HOP_XPAY : KB_HOP);
    const double n5 = (double)g.Vh * g.Ls * h.nrhs;
    // fields moved: in, out (+x), and for the fused epilogues v (FUSE_T) or r read+write instead of out (FUSE_R)
    const double sp = site_bytes(P), sr = site_bytes(ResPrec<P>::value);
    double fields = sp + sp + (X ? sp : 0.0);
    if (FU == FUSE_T) fields += sp;
    if (FU == FUSE_R) fields += 2.0 * sr - sp;
    const double bytes = n5 * fields + 8.0 * g.Vh * link_bytes(P);
    const double flops = n5 * (1320.0 + (G ? 72.0 : 0.0) + 144.0 + (X ? 48.0 : 0.0) + (FU ? 144.0 : 0.0));
    LaunchScope scope(c, base * 3 + P, bytes, flops);
    kern<<<grid, block, smem, c->stream>>>(out, in, xf, U, hp, fa);
    return check_launch();
}

template <int P>
static int launch_hop_t(mdwf_ctx* c, const HopLaunch& h) {
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
    hp.mass = reinterpret_cast<const R*>(h.mass);
    hp.mat = reinterpret_cast<const R*>(h.mat);
    hp.nbr = reinterpret_cast<const int4*>(c->nbr);
    hp.sop = h.sop;
    hp.swap = h.swap;
    hp.sc.b5 = (R)c->b5;
    hp.sc.c5 = (R)c->c5;
    hp.sc.Mp = (R)(c->b5 * (4.0 - c->M5) + 1.0);
    hp.sc.Mm = (R)(c->c5 * (4.0 - c->M5) - 1.0);
    const bool X = h.x != nullptr;
    if (h.fuse != FUSE_NONE) {
        // fused CG epilogues: t = M p with v = A^dag t, or Ap = M^dag t folded into r
        if (h.sop == SOP_DENSE || !X || h.gather || !h.part || !h.sc) return MDWF_EINVAL;
        if (h.fuse == FUSE_T && !h.dagger && h.out2) return launch_hop_variant<P, false, false, true, FUSE_T>(c, h, hp);
        if (h.fuse == FUSE_R && h.dagger && h.rfield) return launch_hop_variant<P, false, true, true, FUSE_R>(c, h, hp);
        return MDWF_EINVAL;
    }
    if (h.gather) {
        if (h.dagger) return MDWF_EINVAL;
        return X ? launch_hop_variant<P, true, false, true, FUSE_NONE>(c, h, hp)
                 : launch_hop_variant<P, true, false, false, FUSE_NONE>(c, h, hp);
    }
    if (h.dagger)
        return X ? launch_hop_variant<P, false, true, true, FUSE_NONE>(c, h, hp)
                 : launch_hop_variant<P, false, true, false, FUSE_NONE>(c, h, hp);
    return X ? launch_hop_variant<P, false, false, true, FUSE_NONE>(c, h, hp)
             : launch_hop_variant<P, false, false, false, FUSE_NONE>(c, h, hp);
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
