// Derivatives of S = phi^dag (M^dag M)^-1 phi for the red/black Moebius M.
//
// With X = (M^dag M)^-1 phi (recomputed by CG, never stored between calls)
// and Y = M X, a variation of M gives dS = -2 Re(Y^dag dM X). In the
// factored form M = 1 - 1/4 A H_oe K H_eo M_phi the links enter only through
// the two hopping sums H_eo, H_oe, so
//   dS = 1/2 Re(alpha^dag dH_oe beta) + 1/2 Re(gamma^dag dH_eo delta),
//   alpha = A^dag Y (odd),  beta = K H_eo M_phi X (even),
//   gamma = K^dag H'_eo alpha (even),  delta = M_phi X (odd),
// with H' the hopping part of D_W^dag. For a variation dU of one link,
// Re(a^dag dH b) = Re sum conj(G) dU with G the colour outer products of the
// spin-projected half spinors of the forward and backward terms; the output
// dS/dU = dS/dRe U + i dS/dIm U per link entry (torch's convention).
// The Moebius parameters enter through E = dM_ee (= (4 - M5) 1 for b5,
// (4 - M5) C for c5) and F = dM_phi (= 1 or C):
//   dS/dtheta = 1/2 Re[ -4 alpha^dag E (X - Y) + gamma'^dag (F - K E) A h1 + gamma^dag H_eo F X ],
//   h1 = H_eo M_phi X, gamma' = H'_eo alpha.
#include <math.h>
#include <string.h>

#include <vector>

#include "mdwf_internal.cuh"

namespace mdwf {

// (1 + S g_mu) projection of a spinor: h = u + S A_mu l (2 spins x 3 colours)
template <int S>
__device__ __forceinline__ void proj_mu(int mu, const double* w, double* h) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double u0r = w[2 * c], u0i = w[2 * c + 1], u1r = w[6 + 2 * c], u1i = w[7 + 2 * c];
        const double l0r = w[12 + 2 * c], l0i = w[13 + 2 * c], l1r = w[18 + 2 * c], l1i = w[19 + 2 * c];
        double a0r, a0i, a1r, a1i;
        switch (mu) {
            case 0: a0r = l1i; a0i = -l1r; a1r = l0i; a1i = -l0r; break;     // -i sigma_1
            case 1: a0r = -l1r; a0i = -l1i; a1r = l0r; a1i = l0i; break;     // -i sigma_2
            case 2: a0r = l0i; a0i = -l0r; a1r = -l1i; a1i = l1r; break;     // -i sigma_3
            default: a0r = l0r; a0i = l0i; a1r = l1r; a1i = l1i; break;      // 1
        }
        h[2 * c] = u0r + S * a0r;
        h[2 * c + 1] = u0i + S * a0i;
        h[6 + 2 * c] = u1r + S * a1r;
        h[7 + 2 * c] = u1i + S * a1i;
    }
}

// acc[i][j] += sum_spin p[spin][i] conj(q[spin][j]) (complex 3x3 as 18 reals)
__device__ __forceinline__ void outer_add(double* acc, const double* p, const double* q) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const double pr = p[6 * sp + 2 * i], pi = p[6 * sp + 2 * i + 1];
                const double qr = q[6 * sp + 2 * j], qi = q[6 * sp + 2 * j + 1];
                acc[2 * (3 * i + j)] += pr * qr + pi * qi;
                acc[2 * (3 * i + j) + 1] += pi * qr - pr * qi;
            }
}

// For every link (x, mu) with x of parity `par`: dS/dU_mu(x) into the user
// gauge layout [t][z][y][x][mu][3][3]. fa = field of x's parity used in the
// forward term (gamma on even x, alpha on odd x), fb = its partner at x+mu,
// fc = the out-parity field at x+mu of the backward term, fd = its partner at x.
// With a chemical potential (Sec. 6.6) the time links enter the forward hop
// with e^{+mu} and the backward hop with e^{-mu}: efwd, ebwd scale the two
// outer products of mu = 3 (1 and 1 without).
__global__ void __launch_bounds__(128) force_kernel(double2* dSdU, Field<MDWF_F64> fa, Field<MDWF_F64> fb,
                                                    Field<MDWF_F64> fc, Field<MDWF_F64> fd, const int4* nbr,
                                                    Geom g, int par, double coef, double efwd, double ebwd) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* red = reinterpret_cast<double*>(smem_raw);  // [SB][Ls][18]
    const int Ls = g.Ls;
    const int s = threadIdx.x, ly = threadIdx.y;
    const long long site = (long long)blockIdx.x * blockDim.y + ly;
    const bool active = site < g.Vh;
    int4 f = make_int4(0, 0, 0, 0);
    double a[24], d[24];
    if (active) {
        f = __ldg(nbr + ((long long)par * g.Vh + site) * 2);
        fa.load(site, s, a);
        fd.load(site, s, d);
    }
    long long lex = 0;
    if (active) {
        int c[4];
        cb_coords(g, site, par, c);
        lex = (((long long)c[3] * g.Z + c[2]) * g.Y + c[1]) * g.X + c[0];
    }
    for (int mu = 0; mu < 4; ++mu) {
        double acc[18];
#pragma unroll
        for (int k = 0; k < 18; ++k) acc[k] = 0;
        if (active) {
            const long long j = mu == 0 ? f.x : mu == 1 ? f.y : mu == 2 ? f.z : f.w;
            double b[24], cc[24], h1[12], h2[12];
            fb.load(j, s, b);
            fc.load(j, s, cc);
            const double fw = mu == 3 ? efwd : 1.0, bw = mu == 3 ? ebwd : 1.0;
            // forward: sum (1 - g_mu) a_x (x) conj(b_{x+mu}) via the (1 - g_mu) half spinors
            proj_mu<-1>(mu, a, h1);
            proj_mu<-1>(mu, b, h2);
#pragma unroll
            for (int k = 0; k < 12; ++k) h1[k] *= fw;
            outer_add(acc, h1, h2);
            // backward: [sum (1 + g_mu) c_{x+mu} (x) conj(d_x)]^dag = sum h+(d) (x) conj(h+(c))
            proj_mu<+1>(mu, cc, h1);
            proj_mu<+1>(mu, d, h2);
#pragma unroll
            for (int k = 0; k < 12; ++k) h2[k] *= bw;
            outer_add(acc, h2, h1);
        }
        double* mine = red + ((size_t)ly * Ls + s) * 18;
#pragma unroll
        for (int k = 0; k < 18; ++k) mine[k] = acc[k];
        __syncthreads();
        // sum over s: thread s of a column adds entry k = s, s + Ls, ... of the 18
        if (active) {
            for (int k = s; k < 18; k += Ls) {
                double v = 0;
                for (int t = 0; t < Ls; ++t) v += red[((size_t)ly * Ls + t) * 18 + k];
                double* o = reinterpret_cast<double*>(dSdU + (lex * 4 + mu) * 9);
                o[k] = coef * v;
            }
        }
        __syncthreads();
    }
}

// dSdU = coef [Re(A^dag dH_oe B) + Re(C^dag dH_eo D)] per link, written (not
// accumulated) by one launch per parity of x; both parities cover all links.
int launch_force(mdwf_ctx* c, double* dSdU, const void* A_odd, const void* B_even, const void* C_even,
                 const void* D_odd, double coef) {
    // even x: forward (gamma_x, delta_{x+mu}), backward (alpha_{x+mu}, beta_x)
    // odd x : forward (alpha_x, beta_{x+mu}), backward (gamma_{x+mu}, delta_x)
    const Geom& g = c->g;
    if (c->slab) return MDWF_EINVAL;  // the neighbour table of a t-slab points into halos
    const int SB = (128 / g.Ls) < 1 ? 1 : 128 / g.Ls;
    dim3 block(g.Ls, SB), grid((unsigned)((g.Vh + SB - 1) / SB));
    const size_t smem = (size_t)SB * g.Ls * 18 * sizeof(double);
    const double efwd = exp(c->chem), ebwd = exp(-c->chem);
    auto F = [&](const void* p) { return make_field<MDWF_F64>(const_cast<void*>(p), g, 1); };
    const double n5 = (double)g.Vh * g.Ls;
    int st;
    {
        LaunchScope scope(c, KB_BLAS * 3 + MDWF_F64, n5 * 192.0 * 10.0 + g.Vh * 4 * 144.0, n5 * 4 * 200.0);
        force_kernel<<<grid, block, smem, c->stream>>>((double2*)dSdU, F(C_even), F(D_odd), F(A_odd), F(B_even),
                                                       (const int4*)c->nbr, g, 0, coef, efwd, ebwd);
    }
    if ((st = check_launch())) return st;
    {
        LaunchScope scope(c, KB_BLAS * 3 + MDWF_F64, n5 * 192.0 * 10.0 + g.Vh * 4 * 144.0, n5 * 4 * 200.0);
        force_kernel<<<grid, block, smem, c->stream>>>((double2*)dSdU, F(A_odd), F(B_even), F(C_even), F(D_odd),
                                                       (const int4*)c->nbr, g, 1, coef, efwd, ebwd);
    }
    return check_launch();
}

}  // namespace mdwf

using namespace mdwf;

extern "C" int mdwf_force(mdwf_ctx* c, double* dSdU, double* dSdb5, double* dSdc5, double* S_out,
                          const double* phi, int where, const mdwf_solve_params* params, mdwf_solve_info* info) {
    NvtxRange nvtx_range("mdwf_force");
    if (!c || !phi || (where != MDWF_HOST && where != MDWF_DEVICE)) return MDWF_EINVAL;
    if (!c->have_gauge) return MDWF_ENOGAUGE;
    mdwf_solve_params prm{};
    if (params) prm = *params;
    prm.guess = 0;  // the solves here start from zero
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    if ((st = ensure_tables(c, 1, nullptr))) return st;
    const Geom g = c->g;
    const size_t f64 = field_bytes(MDWF_F64, g, 1);
    const size_t ub = (size_t)g.Ls * g.Vh * 24 * sizeof(double);
    const size_t gb = (size_t)g.Vh * 2 * 4 * 9 * 16;
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t need = up(f64) * 12 + (where == MDWF_HOST ? up(ub) + up(gb) : 0);
    if ((st = ensure_workspace(c->io, need))) return st;
    if ((st = ensure_workspace(c->tmp[0], f64)) || (st = ensure_workspace(c->tmp[1], f64))) return st;
    char* w = (char*)c->io.p;
    auto take = [&](size_t bytes) { void* p = w; w += up(bytes); return p; };
    void *ph = take(f64), *X = take(f64), *Y = take(f64), *al = take(f64), *de = take(f64), *h1 = take(f64);
    void *be = take(f64), *gp = take(f64), *ga = take(f64), *t1 = take(f64), *t2 = take(f64), *t3 = take(f64);
    double* stage_phi = where == MDWF_HOST ? (double*)take(ub) : nullptr;
    double* stage_g = where == MDWF_HOST ? (double*)take(gb) : nullptr;

    const double* pdev = phi;
    if (where == MDWF_HOST) {
        if ((st = cuda_status(cudaMemcpyAsync(stage_phi, phi, ub, cudaMemcpyHostToDevice, c->stream)))) return st;
        pdev = stage_phi;
    }
    if ((st = launch_import_odd(c, ph, pdev, MDWF_F64, 1))) return st;

    NormalResult res;
    if ((st = solve_normal(c, 1, X, ph, prm, res))) return st;
    double S = 0;
    if ((st = field_dot64(c, ph, X, 1, &S))) return st;
    if (info) {
        info->status = res.status[0];
        info->iters = res.iters[0];
        info->reliable_updates = res.rupd[0];
        info->restarts = res.restarts[0];
        info->true_res = res.rel[0];
        info->res_m = 0.0;
        info->seconds = 0.0;
    }
    if (S_out) *S_out = S;
    if (!dSdU && !dSdb5 && !dSdc5) return res.status[0];  // the action alone

    const double wgt = 4.0 - c->M5;
    M5Launch m{};
    m.nrhs = 1; m.x = nullptr; m.coef = 1.0;
    HopLaunch h{};
    h.nrhs = 1; h.b5 = c->b5; h.c5 = c->c5; h.mass = c->mass64; h.x = nullptr; h.coef = 1.0;
    auto m5 = [&](void* out, const void* in, int sop, int swap, double coef, const void* x) {
        m.out = out; m.in = in; m.coef = coef; m.x = x;
        set_sop(c, MDWF_F64, sop, swap, m);
        return launch_m5(c, MDWF_F64, m);
    };
    auto hop = [&](void* out, const void* in, int gather, int dagger) {
        h.out = out; h.in = in; h.gather = gather; h.dagger = dagger; h.out_parity = 0; h.x = nullptr; h.coef = 1.0;
        set_sop(c, MDWF_F64, SOP_ID, 0, h);
        return launch_hop(c, MDWF_F64, h);
    };
    if ((st = apply_op(c, Y, X, MDWF_F64, 1, 0))) return st;        // Y = M X
    if ((st = m5(al, Y, SOP_A, 1, 1.0, nullptr))) return st;         // alpha = A^dag Y
    if ((st = m5(de, X, SOP_MPHI, 0, 1.0, nullptr))) return st;      // delta = M_phi X
    if ((st = hop(h1, X, 1, 0))) return st;                          // h1 = H_eo M_phi X
    if ((st = m5(be, h1, SOP_K, 0, 1.0, nullptr))) return st;        // beta = K h1
    if ((st = hop(gp, al, 0, 1))) return st;                         // gamma' = H'_eo alpha
    if ((st = m5(ga, gp, SOP_K, 1, 1.0, nullptr))) return st;        // gamma = K^dag gamma'

    if (dSdU) {
        double* gdev = where == MDWF_HOST ? stage_g : dSdU;
        if ((st = launch_force(c, gdev, al, be, ga, de, 0.5))) return st;
        if (where == MDWF_HOST &&
            (st = cuda_status(cudaMemcpyAsync(dSdU, stage_g, gb, cudaMemcpyDeviceToHost, c->stream))))
            return st;
    }

    if (!dSdb5 && !dSdc5) {
        if ((st = cuda_status(cudaStreamSynchronize(c->stream)))) return st;
        return res.status[0];
    }
    if (c->sdep) {
        // Per slice s: b5(s) has E = w P_s, F = P_s and c5(s) has E = w P_s C,
        // F = P_s C (P_s the projector on slice s). H_eo is diagonal in s, and
        // gamma'^dag K E v = gamma^dag E v, so every term is a dot product
        // restricted to slice s:
        //   dS/db5(s) = 1/2 [-4 w <alpha, X - Y>_s + <gamma' - w gamma, v>_s + <gamma, H_eo X>_s]
        //   dS/dc5(s) = the same with C (X - Y), C v and H_eo C X, v = A h1.
        const int Ls = g.Ls;
        std::vector<double> r1(Ls), r2(Ls), r3(Ls);
        if ((st = m5(t1, Y, SOP_ID, 0, -1.0, X))) return st;       // t1 = X - Y
        if ((st = m5(t2, h1, SOP_A, 0, 1.0, nullptr))) return st;  // t2 = v = A h1
        if ((st = m5(t3, ga, SOP_ID, 0, -wgt, gp))) return st;     // t3 = gamma' - w gamma
        for (int which = 0; which < 2; ++which) {
            double* dst = which == 0 ? dSdb5 : dSdc5;
            if (!dst) continue;
            const void *a1 = t1, *a2 = t2, *a3 = X;
            if (which == 1) {  // be, de are free after the link force: C (X - Y), C v, C X
                if ((st = m5(de, t1, SOP_C, 0, 1.0, nullptr))) return st;
                if ((st = slice_dot64(c, al, de, r1.data()))) return st;
                if ((st = m5(de, t2, SOP_C, 0, 1.0, nullptr))) return st;
                if ((st = slice_dot64(c, t3, de, r2.data()))) return st;
                if ((st = m5(de, X, SOP_C, 0, 1.0, nullptr))) return st;
                a3 = de;
            } else {
                if ((st = slice_dot64(c, al, a1, r1.data()))) return st;
                if ((st = slice_dot64(c, t3, a2, r2.data()))) return st;
            }
            if ((st = hop(be, a3, 0, 0))) return st;  // H_eo X or H_eo C X
            if ((st = slice_dot64(c, ga, be, r3.data()))) return st;
            for (int k = 0; k < Ls; ++k) dst[k] = 0.5 * (-4.0 * wgt * r1[k] + r2[k] + r3[k]);
        }
        return res.status[0];
    }

    // dS/db5 (E = w 1, F = 1) and dS/dc5 (E = w C, F = C)
    double out[2];
    for (int which = 0; which < 2; ++which) {
        double r1, r2, r3;
        if ((st = m5(t1, Y, SOP_ID, 0, -1.0, X))) return st;            // t1 = X - Y
        if (which == 1 && (st = m5(t1, t1, SOP_C, 0, 1.0, nullptr))) return st;  // C (X - Y)
        if ((st = field_dot64(c, al, t1, 1, &r1))) return st;
        if ((st = m5(t2, h1, SOP_A, 0, 1.0, nullptr))) return st;       // v = A h1
        if (which == 1 && (st = m5(t2, t2, SOP_C, 0, 1.0, nullptr))) return st;  // C v
        if ((st = m5(t3, t2, SOP_K, 0, -wgt, t2))) return st;           // (1 - w K) F v
        if ((st = field_dot64(c, gp, t3, 1, &r2))) return st;
        const void* fx = X;
        if (which == 1) {
            if ((st = m5(t1, X, SOP_C, 0, 1.0, nullptr))) return st;     // C X
            fx = t1;
        }
        if ((st = hop(t2, fx, 0, 0))) return st;                         // H_eo F X
        if ((st = field_dot64(c, ga, t2, 1, &r3))) return st;
        out[which] = 0.5 * (-4.0 * wgt * r1 + r2 + r3);
    }
    if ((st = cuda_status(cudaStreamSynchronize(c->stream)))) return st;
    if (dSdb5) *dSdb5 = out[0];
    if (dSdc5) *dSdc5 = out[1];
    return res.status[0];
}
