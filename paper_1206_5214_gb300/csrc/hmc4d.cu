// The 4d-HMC action with the pseudofermion on the wall (Sec. 2.4) and its
// link force:
//   S = phi^dag P^dag D(m)^-1 D(1) D(1)^dag D(m)^-dag P phi = |D(1)^dag chi|^2,
//   chi = D(m)^-dag P phi,  phi the 4d field on s = 1 (phi_s = phi delta_{s,1}),
// with D = D_DW. Two inversions (Sec. 2.4): chi by the adjoint solve below and
// psi = D(m)^-1 D(1) D(1)^dag chi. With eta = D(1)^dag chi, and since only
// D_W = (4 - M5) - H/2 in D = D_W (x) M_phi + (1 - C) holds links,
//   dS = 2 Re[ chi^dag dD(1) eta - chi^dag dD(m) psi ] = -Re[ chi^dag dH w ],
//   w = M_phi(1) eta - M_phi(m) psi   (M_phi carries the wall mass in its corner),
// split by parity into the outer products of the force kernel.
//
// Adjoint solve D^dag x = b by the red/black decomposition of D^dag: with
// b'_o = b_o - D_eo^dag I^-dag b_e, the odd part solves I^dag M~ x_o = b'_o,
// M~ = I^-dag M^dag I^dag, i.e. M^dag (I^dag x_o) = b'_o; hence
//   x_o = I^-dag M w,  M^dag M w = b'_o   (the solver of mdwf_cgne),
//   x_e = I^-dag (b_e - D_oe^dag x_o),
// with D_eo^dag = -1/2 M_phi^dag H'_oe and D_oe^dag = -1/2 M_phi^dag H'_eo.
#include <vector>

#include "mdwf_internal.cuh"

namespace mdwf {

static void m5_op(mdwf_ctx* c, M5Launch& m, void* out, const void* in, const void* x, double coef, int sop,
                  int swap) {
    m = M5Launch{};
    m.out = out; m.in = in; m.x = x; m.coef = coef; m.nrhs = 1;
    set_sop(c, MDWF_F64, sop, swap, m);
}

// x (full, device) = D(m)^-dag b (full, device); scratch halves in w[0..5]
static int solve_dag_dev(mdwf_ctx* c, double* x, const double* b, void* const* w, const mdwf_solve_params& prm,
                         NormalResult& res) {
    void *be = w[0], *bo = w[1], *t = w[2], *ww = w[3], *y = w[4], *xo = w[5];
    int st;
    if ((st = ensure_tables(c, 1, nullptr))) return st;
    if ((st = launch_split_full(c, be, bo, b, MDWF_F64, 1))) return st;
    M5Launch m;
    m5_op(c, m, t, be, nullptr, 1.0, SOP_A, 1);  // t = I^-dag b_e
    if ((st = launch_m5(c, MDWF_F64, m))) return st;
    HopLaunch h{};
    h.nrhs = 1; h.b5 = c->b5; h.c5 = c->c5; h.mass = c->mass64;
    h.out = bo; h.in = t; h.x = bo; h.coef = 0.5; h.out_parity = 1; h.gather = 0; h.dagger = 1;
    set_sop(c, MDWF_F64, SOP_MPHI, 1, h);  // b'_o = b_o + 1/2 M_phi^dag H'_oe t
    if ((st = launch_hop(c, MDWF_F64, h))) return st;
    if ((st = solve_normal(c, 1, ww, bo, prm, res))) return st;
    if ((st = apply_op(c, y, ww, MDWF_F64, 1, 0))) return st;  // y = M w
    m5_op(c, m, xo, y, nullptr, 1.0, SOP_A, 1);                 // x_o = I^-dag y
    if ((st = launch_m5(c, MDWF_F64, m))) return st;
    h.out = t; h.in = xo; h.x = be; h.coef = 0.5; h.out_parity = 0;
    set_sop(c, MDWF_F64, SOP_MPHI, 1, h);  // t = b_e + 1/2 M_phi^dag H'_eo x_o
    if ((st = launch_hop(c, MDWF_F64, h))) return st;
    m5_op(c, m, be, t, nullptr, 1.0, SOP_A, 1);  // x_e = I^-dag t
    if ((st = launch_m5(c, MDWF_F64, m))) return st;
    return launch_join_full(c, x, be, xo, MDWF_F64, 1);
}

}  // namespace mdwf

using namespace mdwf;

extern "C" int mdwf_force4d(mdwf_ctx* c, double* dSdU, double* S_out, const double* phi, int where,
                            const mdwf_solve_params* params, mdwf_solve_info* info) {
    NvtxRange nvtx_range("mdwf_force4d");
    if (!c || !phi || !S_out || (where != MDWF_HOST && where != MDWF_DEVICE)) return MDWF_EINVAL;
    if (!c->have_gauge) return MDWF_ENOGAUGE;
    if (c->mf == 1.0) return MDWF_EINVAL;
    mdwf_solve_params prm{};
    if (params) prm = *params;
    prm.guess = 0;  // the solves here start from zero
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    const Geom& g = c->g;
    const size_t f1 = field_bytes(MDWF_F64, g, 1);
    const size_t f5 = (size_t)g.Ls * 2 * g.Vh * 24 * sizeof(double);
    const size_t f4 = (size_t)2 * g.Vh * 24 * sizeof(double);
    const size_t gb = (size_t)g.Vh * 2 * 4 * 9 * 16;
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t need = up(f5) * 4 + up(f1) * 6 + up(f4) + (where == MDWF_HOST || !dSdU ? up(gb) : 0);
    if ((st = ensure_workspace(c->h4, need))) return st;
    char* p = (char*)c->h4.p;
    auto take = [&](size_t bytes) { void* q = p; p += up(bytes); return q; };
    double *b5 = (double*)take(f5), *chi = (double*)take(f5), *eta = (double*)take(f5), *e5 = (double*)take(f5);
    void* w[6];
    for (int k = 0; k < 6; ++k) w[k] = take(f1);
    double* phi_dev = (double*)take(f4);
    double* gdev = (where == MDWF_HOST || !dSdU) ? (double*)take(gb) : dSdU;

    if ((st = cuda_status(cudaMemcpyAsync(phi_dev, phi, f4,
                                          where == MDWF_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                          c->stream))))
        return st;
    if ((st = launch_embed_wall(c, b5, phi_dev, 1))) return st;  // P phi
    NormalResult res;
    if ((st = solve_dag_dev(c, chi, b5, w, prm, res))) return st;  // chi = D(m)^-dag P phi
    int worst = res.status.empty() ? MDWF_OK : res.status[0];
    const double one = 1.0;
    if ((st = ensure_tables(c, 1, &one))) return st;
    if ((st = apply_full_dev(c, eta, chi, 1, 1))) return st;  // eta = D(1)^dag chi
    if ((st = apply_full_dev(c, e5, eta, 1, 0))) return st;   // e5 = D(1) eta
    // psi = D(m)^-1 e5 into b5 (mdwf_cgne rebuilds the tables at the context's mass)
    st = mdwf_cgne(c, b5, e5, 1, nullptr, MDWF_DEVICE, &prm, info);
    if (st && st != MDWF_ENOCONV) return st;
    if (st > worst) worst = st;
    // w = M_phi(1) eta - M_phi(m) psi by parity: (eta_e, eta_o) -> w[0], w[1]; psi -> w[2], w[3]
    if ((st = launch_split_full(c, w[0], w[1], eta, MDWF_F64, 1))) return st;
    if ((st = launch_split_full(c, w[2], w[3], b5, MDWF_F64, 1))) return st;
    std::vector<double> sq(2);
    if ((st = field_dot64(c, w[0], w[0], 1, &sq[0]))) return st;
    if ((st = field_dot64(c, w[1], w[1], 1, &sq[1]))) return st;
    *S_out = sq[0] + sq[1];  // |D(1)^dag chi|^2
    if (!dSdU) return worst;
    M5Launch m;
    if ((st = ensure_tables(c, 1, &one))) return st;
    for (int par = 0; par < 2; ++par) {
        m5_op(c, m, w[4 + par], w[par], nullptr, 1.0, SOP_MPHI, 0);
        if ((st = launch_m5(c, MDWF_F64, m))) return st;
    }
    if ((st = ensure_tables(c, 1, nullptr))) return st;
    for (int par = 0; par < 2; ++par) {
        m5_op(c, m, w[4 + par], w[2 + par], w[4 + par], -1.0, SOP_MPHI, 0);
        if ((st = launch_m5(c, MDWF_F64, m))) return st;
    }
    // chi by parity into w[0], w[1]
    if ((st = launch_split_full(c, w[0], w[1], chi, MDWF_F64, 1))) return st;
    // dS = -Re[chi_o^dag dH_oe w_e + chi_e^dag dH_eo w_o]
    if ((st = launch_force(c, gdev, w[1], w[4], w[0], w[5], -1.0))) return st;
    if (where == MDWF_HOST &&
        (st = cuda_status(cudaMemcpyAsync(dSdU, gdev, gb, cudaMemcpyDeviceToHost, c->stream))))
        return st;
    if ((st = cuda_status(cudaStreamSynchronize(c->stream)))) return st;
    return worst;
}
