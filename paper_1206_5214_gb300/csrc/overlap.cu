// The full (unpreconditioned) domain-wall operator D_DW(m) on 5d fields, and
// the two constructions of Sec. 2.2-2.3 built on it with a Pauli-Villars
// (m = 1) solve:
//   effective overlap operator  D_ov(m) psi = [P^dag D_DW(1)^-1 D_DW(m) P psi~]_1
//   bulk reconstruction         Psi_1 = psi,  Psi_s = -Omega_s (s > 1),
//                               Omega = P^dag D_DW(1)^-1 D_DW(m) P psi~,
// with psi~_s = psi delta_{s,1} and the wall permutation
//   (P psi)_s = P- psi_s + P+ psi_{s+1},  (P^dag psi)_s = P- psi_s + P+ psi_{s-1}
// (indices mod Ls). Fields are in the user layout: full 5d
// [rhs][s][t][z][y][x][spin][colour], 4d [rhs][t][z][y][x][spin][colour],
// complex128; P+ is spins 0, 1.
#include <string.h>

#include <vector>

#include "mdwf_internal.cuh"

namespace mdwf {

// out5 = P psi~: P- psi on s = 0, P+ psi on s = Ls - 1, zero elsewhere.
__global__ void k_embed_wall(double2* out5, const double2* in4, long long V, int Ls, int nrhs) {
    const long long per = V * 12;
    const long long n = (long long)nrhs * Ls * per;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long k = i % per;             // site * 12 + spin * 3 + colour
        const int s = (int)((i / per) % Ls);
        const int r = (int)(i / (per * Ls));
        const int spin = (int)((k % 12) / 3);
        const bool lower = spin >= 2;            // P-
        double2 v = make_double2(0.0, 0.0);
        if ((lower && s == 0) || (!lower && s == Ls - 1)) v = in4[(long long)r * per + k];
        out5[i] = v;
    }
}

// MODE 0: out4 = (P^dag x)_0 = P- x_0 + P+ x_{Ls-1}
// MODE 1: out5 = Psi with Psi_0 = psi, Psi_s = -(P- x_s + P+ x_{s-1}) for s > 0
template <int MODE>
__global__ void k_wall_extract(double2* out, const double2* x5, const double2* psi4, long long V, int Ls, int nrhs) {
    const long long per = V * 12;
    const long long n = (long long)nrhs * (MODE == 0 ? 1 : Ls) * per;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long k = i % per;
        const int s = MODE == 0 ? 0 : (int)((i / per) % Ls);
        const int r = (int)(i / (per * (MODE == 0 ? 1 : Ls)));
        const int spin = (int)((k % 12) / 3);
        const int src_s = spin >= 2 ? s : (s == 0 ? Ls - 1 : s - 1);
        const double2 v = x5[((long long)r * Ls + src_s) * per + k];
        if (MODE == 0) {
            out[i] = v;
        } else {
            out[i] = s == 0 ? psi4[(long long)r * per + k] : make_double2(-v.x, -v.y);
        }
    }
}

// out = gamma5 (2 dov - (1 + m) in) / (1 - m) = eps in, from dov = D_ov(m) in
// (Sec. 2.2: D_ov = (1+m)/2 + (1-m)/2 gamma5 eps); per-rhs masses m.
__global__ void k_eps_from_overlap(double2* out, const double2* dov, const double2* in, const double* mass,
                                   long long V, int nrhs) {
    const long long per = V * 12;
    const long long n = (long long)nrhs * per;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / per);
        const int spin = (int)((i % 12) / 3);
        const double m = mass[r];
        const double g = (spin >= 2 ? -1.0 : 1.0) / (1.0 - m);
        const double2 d = dov[i], x = in[i];
        out[i] = make_double2(g * (2.0 * d.x - (1.0 + m) * x.x), g * (2.0 * d.y - (1.0 + m) * x.y));
    }
}

// out = (psi - e2) / 4
__global__ void k_quarter_diff(double2* out, const double2* psi, const double2* e2, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 a = psi[i], b = e2[i];
        out[i] = make_double2(0.25 * (a.x - b.x), 0.25 * (a.y - b.y));
    }
}

static dim3 grid_of(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152LL * 32) b = 152LL * 32;
    return dim3((unsigned)(b < 1 ? 1 : b));
}

// out = D_DW(m) in (dagger: D_DW(m)^dag) on device full fields, FP64:
//   (D in)_e = I in_e - 1/2 H_eo M_phi in_o,   (D in)_o = I in_o - 1/2 H_oe M_phi in_e
//   (D^dag in)_e = I^dag in_e - 1/2 M_phi^dag H'_eo in_o, and likewise for o.
int apply_full_dev(mdwf_ctx* c, double* out, const double* in, int nrhs, int dagger) {
    const Geom& g = c->g;
    const size_t f64 = field_bytes(MDWF_F64, g, nrhs);
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    int st;
    if ((st = ensure_workspace(c->aux, up(f64) * 4))) return st;
    char* w = (char*)c->aux.p;
    void *e = w, *o = w + up(f64), *oe = w + 2 * up(f64), *oo = w + 3 * up(f64);
    if ((st = launch_split_full(c, e, o, in, MDWF_F64, nrhs))) return st;
    for (int par = 0; par < 2; ++par) {
        void* dst = par == 0 ? oe : oo;
        void* same = par == 0 ? e : o;
        void* other = par == 0 ? o : e;
        M5Launch m{};
        m.out = dst; m.in = same; m.x = nullptr; m.coef = 1.0; m.nrhs = nrhs;
        set_sop(c, MDWF_F64, SOP_MEE, dagger, m);
        if ((st = launch_m5(c, MDWF_F64, m))) return st;
        HopLaunch h{};
        h.nrhs = nrhs; h.b5 = c->b5; h.c5 = c->c5; h.mass = c->mass64;
        h.out = dst; h.in = other; h.x = dst; h.coef = -0.5; h.out_parity = par;
        if (!dagger) {
            h.gather = 1; h.dagger = 0;
            set_sop(c, MDWF_F64, SOP_ID, 0, h);
        } else {
            h.gather = 0; h.dagger = 1;
            set_sop(c, MDWF_F64, SOP_MPHI, 1, h);
        }
        if ((st = launch_hop(c, MDWF_F64, h))) return st;
    }
    return launch_join_full(c, out, oe, oo, MDWF_F64, nrhs);
}

int launch_embed_wall(mdwf_ctx* c, double* out5, const double* in4, int nrhs) {
    const long long V = 2 * c->g.Vh;
    k_embed_wall<<<grid_of((long long)nrhs * c->g.Ls * V * 12), 256, 0, c->stream>>>(
        (double2*)out5, (const double2*)in4, V, c->g.Ls, nrhs);
    return check_launch();
}

static size_t full5_bytes(const Geom& g, int nrhs) { return (size_t)nrhs * g.Ls * 2 * g.Vh * 24 * sizeof(double); }
static size_t full4_bytes(const Geom& g, int nrhs) { return (size_t)nrhs * 2 * g.Vh * 24 * sizeof(double); }

// Omega-side work shared by the overlap operator and the reconstruction:
// x = D_DW(1)^-1 D_DW(m) P psi~ into the second half of the workspace.
static int pv_stage(mdwf_ctx* c, const double* psi4_dev, int nrhs, const double* mf_per_rhs,
                    const mdwf_solve_params* prm, mdwf_solve_info* info, double** x_out) {
    const Geom& g = c->g;
    const size_t f5 = full5_bytes(g, nrhs);
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    int st;
    if ((st = ensure_workspace(c->ov, up(f5) * 2 + up(full4_bytes(g, nrhs))))) return st;
    double* a = (double*)c->ov.p;
    double* y = (double*)((char*)c->ov.p + up(f5));
    const long long V = 2 * g.Vh;
    k_embed_wall<<<grid_of((long long)nrhs * g.Ls * V * 12), 256, 0, c->stream>>>(
        (double2*)a, (const double2*)psi4_dev, V, g.Ls, nrhs);
    if ((st = check_launch())) return st;
    if ((st = ensure_tables(c, nrhs, mf_per_rhs))) return st;
    if ((st = apply_full_dev(c, y, a, nrhs, 0))) return st;  // y = D(m) P psi~
    std::vector<double> ones(nrhs, 1.0);
    mdwf_solve_params pv{};
    if (prm) pv = *prm;
    pv.guess = 0;  // a holds P psi~, not a guess
    // x = D(1)^-1 y (the Pauli-Villars solve), into a
    st = mdwf_cgne(c, a, y, nrhs, ones.data(), MDWF_DEVICE, &pv, info);
    *x_out = a;  // also after MDWF_ENOCONV: the last iterate is in a
    return st;
}

}  // namespace mdwf

using namespace mdwf;

extern "C" int mdwf_apply_full(mdwf_ctx* c, double* out, const double* in, int nrhs, const double* mf_per_rhs,
                               int where, int dagger) {
    NvtxRange nvtx_range("mdwf_apply_full");
    if (!c || !out || !in || out == in || nrhs < 1 || nrhs > kMaxRhs || (where != MDWF_HOST && where != MDWF_DEVICE) ||
        (dagger != 0 && dagger != 1))
        return MDWF_EINVAL;
    if (!c->have_gauge) return MDWF_ENOGAUGE;
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    if ((st = ensure_tables(c, nrhs, mf_per_rhs))) return st;
    const size_t f5 = full5_bytes(c->g, nrhs);
    if (where == MDWF_DEVICE) return apply_full_dev(c, out, in, nrhs, dagger);
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    if ((st = ensure_workspace(c->ov, up(f5) * 2))) return st;
    double* a = (double*)c->ov.p;
    double* b = (double*)((char*)c->ov.p + up(f5));
    if ((st = cuda_status(cudaMemcpyAsync(a, in, f5, cudaMemcpyHostToDevice, c->stream)))) return st;
    if ((st = apply_full_dev(c, b, a, nrhs, dagger))) return st;
    if ((st = cuda_status(cudaMemcpyAsync(out, b, f5, cudaMemcpyDeviceToHost, c->stream)))) return st;
    return cuda_status(cudaStreamSynchronize(c->stream));
}

// Shared driver of the two Pauli-Villars constructions.
static int pv_entry(mdwf_ctx* c, double* out, const double* psi4, int nrhs, const double* mf_per_rhs, int where,
                    const mdwf_solve_params* params, mdwf_solve_info* info, int mode) {
    NvtxRange nvtx_range("mdwf_pv");
    if (!c || !out || !psi4 || nrhs < 1 || nrhs > kMaxRhs || (where != MDWF_HOST && where != MDWF_DEVICE))
        return MDWF_EINVAL;
    if (!c->have_gauge) return MDWF_ENOGAUGE;
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    const Geom& g = c->g;
    const size_t f4 = full4_bytes(g, nrhs), f5 = full5_bytes(g, nrhs);
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    // psi on the device: the caller's buffer, or the staging slot after the two 5d fields
    if ((st = ensure_workspace(c->ov, up(f5) * 2 + up(f4)))) return st;
    const double* psi_dev = psi4;
    double* stage4 = (double*)((char*)c->ov.p + 2 * up(f5));
    if (where == MDWF_HOST) {
        if ((st = cuda_status(cudaMemcpyAsync(stage4, psi4, f4, cudaMemcpyHostToDevice, c->stream)))) return st;
        psi_dev = stage4;
    }
    double* x = nullptr;
    if ((st = pv_stage(c, psi_dev, nrhs, mf_per_rhs, params, info, &x)) && st != MDWF_ENOCONV) return st;
    if (!x) return MDWF_EINVAL;
    const int solve_st = st;
    const long long V = 2 * g.Vh;
    // the 5d result goes to the second 5d slot (y is no longer needed), the 4d one to its own slot
    double* res = mode == 0 ? (where == MDWF_HOST ? stage4 : out)
                            : (where == MDWF_HOST ? (double*)((char*)c->ov.p + up(f5)) : out);
    if (mode == 0)
        k_wall_extract<0><<<grid_of((long long)nrhs * V * 12), 256, 0, c->stream>>>(
            (double2*)res, (const double2*)x, nullptr, V, g.Ls, nrhs);
    else
        k_wall_extract<1><<<grid_of((long long)nrhs * g.Ls * V * 12), 256, 0, c->stream>>>(
            (double2*)res, (const double2*)x, (const double2*)psi_dev, V, g.Ls, nrhs);
    if ((st = check_launch())) return st;
    if (where == MDWF_HOST &&
        (st = cuda_status(cudaMemcpyAsync(out, res, mode == 0 ? f4 : f5, cudaMemcpyDeviceToHost, c->stream))))
        return st;
    if ((st = cuda_status(cudaStreamSynchronize(c->stream)))) return st;
    return solve_st;
}

extern "C" int mdwf_overlap_apply(mdwf_ctx* c, double* out4, const double* psi4, int nrhs, const double* mf_per_rhs,
                                  int where, const mdwf_solve_params* params, mdwf_solve_info* info) {
    if (out4 == psi4) return MDWF_EINVAL;
    return pv_entry(c, out4, psi4, nrhs, mf_per_rhs, where, params, info, 0);
}

extern "C" int mdwf_pv_reconstruct(mdwf_ctx* c, double* Psi5, const double* psi4, int nrhs, const double* mf_per_rhs,
                                   int where, const mdwf_solve_params* params, mdwf_solve_info* info) {
    return pv_entry(c, Psi5, psi4, nrhs, mf_per_rhs, where, params, info, 1);
}

// Delta_Ls psi = (1 - eps^2) psi / 4 (Eq. Delta_Ls) with eps from two
// applications of D_ov(m) (m != 1 for every right-hand side).
extern "C" int mdwf_gw_violation(mdwf_ctx* c, double* out4, const double* psi4, int nrhs, const double* mf_per_rhs,
                                 int where, const mdwf_solve_params* params, mdwf_solve_info* info) {
    NvtxRange nvtx_range("mdwf_gw_violation");
    if (!c || !out4 || !psi4 || out4 == psi4 || nrhs < 1 || nrhs > kMaxRhs ||
        (where != MDWF_HOST && where != MDWF_DEVICE))
        return MDWF_EINVAL;
    if (!c->have_gauge) return MDWF_ENOGAUGE;
    std::vector<double> masses(nrhs);
    for (int r = 0; r < nrhs; ++r) {
        masses[r] = mf_per_rhs ? mf_per_rhs[r] : c->mf;
        if (masses[r] == 1.0) return MDWF_EINVAL;
    }
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    const Geom& g = c->g;
    const size_t f4 = full4_bytes(g, nrhs);
    const long long V = 2 * g.Vh, n = (long long)nrhs * V * 12;
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    // psi, D_ov psi (later D_ov eps psi), eps psi, eps^2 psi, per-rhs masses
    if ((st = ensure_workspace(c->gw, up(f4) * 4 + up(sizeof(double) * nrhs)))) return st;
    double2* psi = (double2*)c->gw.p;
    double2* d = (double2*)((char*)c->gw.p + up(f4));
    double2* e1 = (double2*)((char*)c->gw.p + 2 * up(f4));
    double2* e2 = (double2*)((char*)c->gw.p + 3 * up(f4));
    double* md = (double*)((char*)c->gw.p + 4 * up(f4));
    if ((st = cuda_status(cudaMemcpyAsync(psi, psi4, f4, where == MDWF_HOST ? cudaMemcpyHostToDevice
                                                                          : cudaMemcpyDeviceToDevice, c->stream))))
        return st;
    if ((st = cuda_status(cudaMemcpyAsync(md, masses.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice,
                                          c->stream))))
        return st;
    int worst = MDWF_OK;
    for (int pass = 0; pass < 2; ++pass) {
        const double2* src = pass == 0 ? psi : e1;
        st = pv_entry(c, (double*)d, (const double*)src, nrhs, masses.data(), MDWF_DEVICE, params, info, 0);
        if (st && st != MDWF_ENOCONV) return st;
        if (st > worst) worst = st;
        k_eps_from_overlap<<<grid_of(n), 256, 0, c->stream>>>(pass == 0 ? e1 : e2, d, src, md, V, nrhs);
        if ((st = check_launch())) return st;
    }
    double2* res = where == MDWF_HOST ? d : (double2*)out4;
    k_quarter_diff<<<grid_of(n), 256, 0, c->stream>>>(res, psi, e2, n);
    if ((st = check_launch())) return st;
    if (where == MDWF_HOST && (st = cuda_status(cudaMemcpyAsync(out4, res, f4, cudaMemcpyDeviceToHost, c->stream))))
        return st;
    if ((st = cuda_status(cudaStreamSynchronize(c->stream)))) return st;
    return worst;
}
