// C entry points of libmdwf: context, gauge upload, field conversion and the
// red/black preconditioned Moebius operator M and M^dag.
//
// M = 1 - I_bb^-1 D_br I_rr^-1 D_rb (Sec. 3) is applied in the factored form
//   D_rb = -1/2 H_eo M_phi,   I_rr = I_bb = M+ + M- C,   M_phi = b5 + c5 C,
//   M = 1 - 1/4 A H_oe K H_eo M_phi,   A = I^-1,  K = M_phi A,
// with C the fifth-dimension shift (P- psi_{s+1} + P+ psi_{s-1}, mass -m on
// the wrap-around), M+ = b5 (4 - M5) + 1, M- = c5 (4 - M5) - 1. Every s-mixing
// factor is a real Ls x Ls matrix per chirality; A, K and their adjoints are
// built here in FP64 by dense inversion of I. Two launches make one M:
//   z_e  = K H_eo (M_phi psi_o)                  (gather fused into the hop)
//   out  = psi_o - 1/4 A H_oe z_e                (xpay fused)
// and three make M^dag = 1 - 1/4 M_phi^dag H'_oe K^dag H'_eo A^dag (H' the
// hopping part of D_W^dag):
//   v_o  = A^dag psi_o;  z_e = K^dag H'_eo v_o;  out = psi_o - 1/4 M_phi^dag H'_oe z_e.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <mutex>

#include "mdwf_internal.cuh"

namespace {
thread_local char g_last_error[512] = "";
}

namespace mdwf {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return MDWF_OK;
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return MDWF_ENOMEM;
    return MDWF_ECUDA;
}

int check_launch() { return cuda_status(cudaGetLastError()); }

void set_error_message(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

// ----------------------------------------------------------- instrumentation

static cudaEvent_t take_event(mdwf_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

LaunchScope::LaunchScope(mdwf_ctx* c, int kind, double bytes, double flops)
    : c_(c), kind_(kind), bytes_(bytes), flops_(flops) {
    if (c_->prof_on && !c_->capturing) {
        a_ = take_event(c_);
        if (a_) cudaEventRecord(a_, c_->stream);
    }
}

LaunchScope::~LaunchScope() {
    if (c_->capturing) {
        c_->cap_launches += 1;
        c_->cap_kstat[kind_].launches += 1;
        c_->cap_kstat[kind_].bytes += bytes_;
        c_->cap_kstat[kind_].flops += flops_;
        return;
    }
    c_->launches += 1;
    c_->kstat[kind_].launches += 1;
    c_->kstat[kind_].bytes += bytes_;
    c_->kstat[kind_].flops += flops_;
    if (a_) {
        cudaEvent_t b = take_event(c_);
        if (b) {
            cudaEventRecord(b, c_->stream);
            c_->prof_pending.push_back(ProfRec{kind_, a_, b});
        } else {
            c_->ev_pool.push_back(a_);
        }
    }
}

// The bounds word of the debug build, one per device (allocated on first use).
int* bounds_word() {
#if MDWF_BOUNDS_CHECK
    static int* words[64] = {};
    static std::mutex m;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(m);
    if (!words[dev]) {
        if (cudaMalloc(&words[dev], sizeof(int)) != cudaSuccess) return nullptr;
        cudaMemset(words[dev], 0, sizeof(int));
    }
    return words[dev];
#else
    return nullptr;
#endif
}

void note_apply(mdwf_ctx* c, int prec) {
    if (c->capturing) c->cap_applies[prec] += 1;
    else c->applies[prec] += 1;
}

void replay_graph_counts(mdwf_ctx* c, long long replays) {
    c->launches += replays * c->cap_launches;
    for (int p = 0; p < 3; ++p) c->applies[p] += replays * c->cap_applies[p];
    for (int k = 0; k < KK_NUM; ++k) {
        c->kstat[k].launches += replays * c->cap_kstat[k].launches;
        c->kstat[k].bytes += replays * c->cap_kstat[k].bytes;
        c->kstat[k].flops += replays * c->cap_kstat[k].flops;
    }
}

static void kernel_name(int kind, char* out, size_t n) {
    static const char* base[KB_NUM] = {"hop", "hop_gather", "hop_xpay", "hop_gather_xpay", "hop_dag",
                                       "hop_dag_xpay", "m5", "m5_xpay", "blas", "layout"};
    static const char* prec[3] = {"f64", "f32", "f16n"};
    snprintf(out, n, "%s_%s", base[kind / 3], prec[kind % 3]);
}

// With MDWF_CANARY=1 in the environment every allocation of the library is
// filled with 0xFF bytes (a NaN in FP16, FP32 and FP64) before its first use,
// so that a kernel reading memory nothing has written spreads NaN into its
// results, which the parity tests then catch. Off by default.
bool canary_on() {
    static const bool on = [] {
        const char* e = getenv("MDWF_CANARY");
        return e && e[0] == '1';
    }();
    return on;
}

int canary_fill(void* p, size_t bytes) {
    return canary_on() && p ? cuda_status(cudaMemset(p, 0xFF, bytes)) : MDWF_OK;
}

int ensure_workspace(Workspace& w, size_t bytes) {
    if (w.bytes >= bytes) return MDWF_OK;
    if (w.p) {
        cudaError_t e = cudaFree(w.p);
        w.p = nullptr;
        w.bytes = 0;
        if (e != cudaSuccess) return cuda_status(e);
    }
    cudaError_t e = cudaMalloc(&w.p, bytes);
    if (e != cudaSuccess) {
        w.p = nullptr;
        return cuda_status(e);
    }
    w.bytes = bytes;
    return canary_fill(w.p, bytes);
}

// ----------------------------------------------------- Ls x Ls tables (host)

// Gauss-Jordan inverse with partial pivoting, n <= kMaxLs.
// Gauss-Jordan inverse with partial pivoting; false when a pivot is at most
// `tiny` in magnitude (singular to working precision at the entries' scale).
static bool invert(int n, const double* a, double* inv, double tiny) {
    double m[kMaxLs][2 * kMaxLs];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j) m[i][j] = j < n ? a[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(m[r][col]) > fabs(m[piv][col])) piv = r;
        if (!(fabs(m[piv][col]) > tiny)) return false;
        if (piv != col)
            for (int j = 0; j < 2 * n; ++j) { double t = m[col][j]; m[col][j] = m[piv][j]; m[piv][j] = t; }
        double d = 1.0 / m[col][col];
        for (int j = 0; j < 2 * n; ++j) m[col][j] *= d;
        for (int r = 0; r < n; ++r) {
            if (r == col || m[r][col] == 0.0) continue;
            double f = m[r][col];
            for (int j = 0; j < 2 * n; ++j) m[r][j] -= f * m[col][j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) inv[i * n + j] = m[i][n + j];
    return true;
}

static void matmul(int n, const double* a, const double* b, double* c) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0;
            for (int k = 0; k < n; ++k) s += a[i * n + k] * b[k * n + j];
            c[i * n + j] = s;
        }
}

// out[t][chir][s'][s] = Mat_t,chir(s, s') for one mass, t = table_index(sop, swap);
// chir 0 = P+, 1 = P-.
// Ls x Ls factors per chirality (Eq. D_5d_matrix, Sec. 3) with row
// coefficients b5(s), c5(s): C = N' on P- (C_{s,s+1} = 1, C_{Ls,1} = -m) and
// N'^T on P+; M_phi = diag(b5) + diag(c5) C, I = diag(M+) + diag(M-) C,
// A = I^-1, K = M_phi A, and I itself for the full operator. swap = 1 stores
// the transposes of the same chirality, which the adjoint chain applies (for
// constant coefficients these equal the other chirality's matrices).
static bool build_tables(int Ls, double M5, const double* b5s, const double* c5s, double mf, double* out) {
    const int n = Ls, nn = Ls * Ls;
    for (int chir = 0; chir < 2; ++chir) {
        const bool up = chir == 1;  // P-: couples s to s+1
        std::vector<double> C(nn, 0.0), Id(nn, 0.0), Mphi(nn), Mee(nn), A(nn), K(nn);
        for (int s = 0; s < n; ++s) {
            Id[s * n + s] = 1.0;
            if (up) {
                if (s + 1 < n) C[s * n + s + 1] = 1.0;
                else C[s * n + 0] = -mf;
            } else {
                if (s > 0) C[s * n + s - 1] = 1.0;
                else C[0 * n + n - 1] = -mf;
            }
        }
        for (int s = 0; s < n; ++s) {
            const double Mp = b5s[s] * (4.0 - M5) + 1.0, Mm = c5s[s] * (4.0 - M5) - 1.0;
            for (int sp = 0; sp < n; ++sp) {
                const int i = s * n + sp;
                Mphi[i] = b5s[s] * Id[i] + c5s[s] * C[i];
                Mee[i] = Mp * Id[i] + Mm * C[i];
            }
        }
        // the entries of I are differences of terms of size 1 + |4 - M5| max(|b5|, |c5|)
        double scale = 1.0;
        for (int s = 0; s < n; ++s) scale = fmax(scale, 1.0 + fabs(4.0 - M5) * fmax(fabs(b5s[s]), fabs(c5s[s])));
        if (!invert(n, Mee.data(), A.data(), 1e-12 * scale)) return false;
        matmul(n, Mphi.data(), A.data(), K.data());
        const double* mats[6] = {Id.data(), A.data(), Mphi.data(), K.data(), C.data(), Mee.data()};  // SOP_ID .. SOP_MEE
        for (int swap = 0; swap < 2; ++swap)
            for (int op = SOP_ID; op <= SOP_MEE; ++op) {
                double* dst = out + ((size_t)table_index(op, swap) * 2 + chir) * nn;
                const double* M = mats[op - SOP_ID];
                // (s, s') at [s'][s]; the transpose puts (s', s) there
                for (int s = 0; s < n; ++s)
                    for (int sp = 0; sp < n; ++sp) dst[sp * n + s] = swap ? M[sp * n + s] : M[s * n + sp];
            }
    }
    return true;
}

int ensure_tables(mdwf_ctx* c, int nrhs, const double* mf_per_rhs) {
    if (nrhs < 1 || nrhs > 64) return MDWF_EINVAL;
    double masses[64];
    for (int r = 0; r < nrhs; ++r) masses[r] = mf_per_rhs ? mf_per_rhs[r] : c->mf;
    if (c->tab_valid && c->tab_nrhs == nrhs && memcmp(masses, c->tab_masses, sizeof(double) * nrhs) == 0)
        return MDWF_OK;
    const int Ls = c->g.Ls, nn = Ls * Ls;
    const size_t per_rhs = (size_t)kNumTables * 2 * nn;
    const size_t total = per_rhs * nrhs;
    // previous kernels may still read the old tables: let them finish first
    int st = cuda_status(cudaStreamSynchronize(c->stream));
    if (st) return st;
    if (c->tab_cap < nrhs || !c->tab64) {
        cudaFree(c->tab64); cudaFree(c->tab32); cudaFree(c->mass64); cudaFree(c->mass32);
        cudaFreeHost(c->tab_host);
        c->tab64 = nullptr; c->tab32 = nullptr; c->mass64 = nullptr; c->mass32 = nullptr; c->tab_host = nullptr;
        if ((st = cuda_status(cudaMalloc(&c->tab64, total * sizeof(double)))) ||
            (st = canary_fill(c->tab64, total * sizeof(double))))
            return st;
        if ((st = cuda_status(cudaMalloc(&c->tab32, total * sizeof(float)))) ||
            (st = canary_fill(c->tab32, total * sizeof(float))))
            return st;
        if ((st = cuda_status(cudaMalloc(&c->mass64, 64 * sizeof(double))))) return st;
        if ((st = cuda_status(cudaMalloc(&c->mass32, 64 * sizeof(float))))) return st;
        if ((st = cuda_status(cudaMallocHost(&c->tab_host, total * (sizeof(double) + sizeof(float)) + 64 * 12 + 16))))
            return st;
        c->tab_cap = nrhs;
    }
    // host layout: [op][rhs][chir][s'][s]
    double* h64 = c->tab_host;
    float* h32 = reinterpret_cast<float*>(h64 + total);
    double* hm64 = reinterpret_cast<double*>(h32 + total + (total & 1));
    float* hm32 = reinterpret_cast<float*>(hm64 + 64);
    std::vector<double> one(per_rhs), b5s(Ls), c5s(Ls);
    for (int s = 0; s < Ls; ++s) {
        b5s[s] = c->sdep ? c->b5s[s] : c->b5;
        c5s[s] = c->sdep ? c->c5s[s] : c->c5;
    }
    for (int r = 0; r < nrhs; ++r) {
        if (!build_tables(Ls, c->M5, b5s.data(), c5s.data(), masses[r], one.data())) {
            set_error_message("the Ls x Ls matrix I = M+ + M- C is singular for these coefficients");
            return MDWF_EINVAL;
        }
        for (int t = 0; t < kNumTables; ++t)
            memcpy(h64 + ((size_t)t * nrhs + r) * 2 * nn, one.data() + (size_t)t * 2 * nn, sizeof(double) * 2 * nn);
        hm64[r] = masses[r];
        hm32[r] = (float)masses[r];
    }
    for (size_t i = 0; i < total; ++i) h32[i] = (float)h64[i];
    if ((st = cuda_status(cudaMemcpyAsync(c->tab64, h64, total * sizeof(double), cudaMemcpyHostToDevice, c->stream))))
        return st;
    if ((st = cuda_status(cudaMemcpyAsync(c->tab32, h32, total * sizeof(float), cudaMemcpyHostToDevice, c->stream))))
        return st;
    if ((st = cuda_status(cudaMemcpyAsync(c->mass64, hm64, 64 * sizeof(double), cudaMemcpyHostToDevice, c->stream))))
        return st;
    if ((st = cuda_status(cudaMemcpyAsync(c->mass32, hm32, 64 * sizeof(float), cudaMemcpyHostToDevice, c->stream))))
        return st;
    if ((st = cuda_status(cudaStreamSynchronize(c->stream)))) return st;
    memcpy(c->tab_masses, masses, sizeof(double) * nrhs);
    c->tab_nrhs = nrhs;
    c->tab_valid = true;
    return MDWF_OK;
}

// ------------------------------------------------------------ operator chain

int apply_op(mdwf_ctx* c, void* out, const void* in, int prec, int nrhs, int dagger, int rhs0, const double* mask) {
    const size_t fb = field_bytes(prec, c->g, nrhs);
    int st;
    note_apply(c, prec);
    if ((st = ensure_workspace(c->tmp[0], fb))) return st;
    if ((st = ensure_workspace(c->tmp[1], fb))) return st;
    const void* mass = prec == MDWF_F64 ? (const void*)c->mass64 : (const void*)c->mass32;
    HopLaunch h{};
    h.nrhs = nrhs;
    h.b5 = c->b5;
    h.c5 = c->c5;
    h.mass = mass;
    h.mask = mask;
    if (!dagger) {
        // w_o = M_phi psi_o by one site-local pass, so that the first hop loads w
        // without the gather along s (and the FP32 / FP16 hops can prefetch)
        M5Launch m{};
        m.out = c->tmp[1].p; m.in = in; m.x = nullptr; m.coef = 1.0; m.nrhs = nrhs; m.mask = mask;
        set_sop(c, prec, SOP_MPHI, 0, m);
        offset_rhs(c, prec, rhs0, m);
        if ((st = launch_m5(c, prec, m))) return st;
        // z_e = K H_eo w_o
        h.out = c->tmp[0].p; h.in = c->tmp[1].p; h.x = nullptr; h.coef = 1.0; h.out_parity = 0;
        h.gather = 0; h.dagger = 0;
        set_sop(c, prec, SOP_K, 0, h);
        offset_rhs(c, prec, rhs0, h);
        if ((st = launch_hop(c, prec, h))) return st;
        // out = psi_o - 1/4 A H_oe z_e
        h.out = out; h.in = c->tmp[0].p; h.x = in; h.coef = -0.25; h.out_parity = 1;
        h.gather = 0; h.dagger = 0;
        h.mass = mass;
        set_sop(c, prec, SOP_A, 0, h);
        offset_rhs(c, prec, rhs0, h);
        return launch_hop(c, prec, h);
    }
    // v_o = A^dag psi_o
    M5Launch m{};
    m.out = c->tmp[1].p; m.in = in; m.x = nullptr; m.coef = 1.0; m.nrhs = nrhs; m.mask = mask;
    set_sop(c, prec, SOP_A, 1, m);
    offset_rhs(c, prec, rhs0, m);
    if ((st = launch_m5(c, prec, m))) return st;
    // z_e = K^dag H'_eo v_o
    h.out = c->tmp[0].p; h.in = c->tmp[1].p; h.x = nullptr; h.coef = 1.0; h.out_parity = 0;
    h.gather = 0; h.dagger = 1;
    set_sop(c, prec, SOP_K, 1, h);
    offset_rhs(c, prec, rhs0, h);
    if ((st = launch_hop(c, prec, h))) return st;
    // out = psi_o - 1/4 M_phi^dag H'_oe z_e
    h.out = out; h.in = c->tmp[0].p; h.x = in; h.coef = -0.25; h.out_parity = 1;
    h.gather = 0; h.dagger = 1;
    h.mass = mass;
    set_sop(c, prec, SOP_MPHI, 1, h);
    offset_rhs(c, prec, rhs0, h);
    return launch_hop(c, prec, h);
}

// Times M + M^dag for every candidate block shape on scratch fields and keeps
// the fastest for (prec, nrhs). Candidates: whole s-columns per block with
// 32, 64 or 128 threads at most (the hop kernels are built for 128).
int tune_hop(mdwf_ctx* c, int prec, int nrhs, int* chosen) {
    const size_t fb = field_bytes(prec, c->g, nrhs);
    int st;
    // its own scratch: the solver's and the entry points' fields stay untouched
    if ((st = ensure_workspace(c->tune, 2 * ((fb + 255) / 256 * 256)))) return st;
    void* a = c->tune.p;
    void* b = (char*)c->tune.p + (fb + 255) / 256 * 256;
    if ((st = cuda_status(cudaMemsetAsync(a, 0, fb, c->stream)))) return st;
    cudaEvent_t e0, e1;
    if ((st = cuda_status(cudaEventCreate(&e0)))) return st;
    if ((st = cuda_status(cudaEventCreate(&e1)))) { cudaEventDestroy(e0); return st; }
    const int Ls = c->g.Ls;
    int cands[3], nc = 0;
    for (int threads = 128; threads >= 32; threads /= 2) {
        const int sb = threads / Ls;
        if (sb >= 1 && (nc == 0 || cands[nc - 1] != sb)) cands[nc++] = sb;
    }
    if (nc == 0) cands[nc++] = 1;
    const bool prof = c->prof_on;
    c->prof_on = false;
    float best = 1e30f;
    int best_sb = cands[0];
    for (int k = 0; k < nc && !st; ++k) {
        c->sb_tune[prec][nrhs] = cands[k];
        st = apply_op(c, b, a, prec, nrhs, 0);  // warm-up
        if (!st) st = apply_op(c, a, b, prec, nrhs, 1);
        if (!st) st = cuda_status(cudaEventRecord(e0, c->stream));
        for (int rep = 0; rep < 3 && !st; ++rep) {
            st = apply_op(c, b, a, prec, nrhs, 0);
            if (!st) st = apply_op(c, a, b, prec, nrhs, 1);
        }
        if (!st) st = cuda_status(cudaEventRecord(e1, c->stream));
        if (!st) st = cuda_status(cudaEventSynchronize(e1));
        float ms = 0.f;
        if (!st) st = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
        if (!st && ms < best) {
            best = ms;
            best_sb = cands[k];
        }
    }
    c->prof_on = prof;
    c->sb_tune[prec][nrhs] = best_sb;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the scratch fields are needed only while tuning: give the memory back
    const int st2 = cuda_status(cudaStreamSynchronize(c->stream));
    cudaFree(c->tune.p);
    c->tune.p = nullptr;
    c->tune.bytes = 0;
    if (chosen) *chosen = best_sb;
    return st ? st : st2;
}

}  // namespace mdwf

using namespace mdwf;

// ------------------------------------------------------------------- C ABI

namespace mdwf {

int device_wait_status(mdwf_ctx* c) {
    int flag = 0;
    int st;
    if ((st = cuda_status(cudaMemcpyAsync(&flag, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream))) ||
        (st = cuda_status(cudaStreamSynchronize(c->stream))))
        return st;
    if (!flag) return MDWF_OK;
    if ((st = cuda_status(cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream)))) return st;
    set_error_message("a bounded device-side wait gave up");
    return MDWF_ETIMEOUT;
}

}  // namespace mdwf

namespace mdwf {

// Context creation; slab: a t-slab of a lattice split along t (mdwf_create_slab).
static int create_context(mdwf_ctx** out, const int dims[4], int Ls, double M5, double b5, double c5, double mf,
                         const mdwf_opts* opts, bool slab) {
    if (!out || !dims) return MDWF_EINVAL;
    *out = nullptr;
    for (int mu = 0; mu < 4; ++mu)
        if (dims[mu] < 2 || (dims[mu] & 1)) return MDWF_EINVAL;
    if (Ls < 2 || Ls > kMaxLs || (Ls & 1)) return MDWF_EINVAL;
    if (!isfinite(M5) || !isfinite(b5) || !isfinite(c5) || !isfinite(mf)) return MDWF_EINVAL;
    int dev = opts ? opts->device : -1;
    int st;
    if (dev < 0) {
        if ((st = cuda_status(cudaGetDevice(&dev)))) return st;
    } else if ((st = cuda_status(cudaSetDevice(dev)))) {
        return st;
    }
    mdwf_ctx* c = new (std::nothrow) mdwf_ctx();
    if (!c) return MDWF_ENOMEM;
    c->device = dev;
    c->stream = opts ? (cudaStream_t)opts->stream : nullptr;
    c->g.X = dims[0]; c->g.Y = dims[1]; c->g.Z = dims[2]; c->g.T = dims[3];
    c->g.Ls = Ls;
    c->g.Vh = (long long)dims[0] * dims[1] * dims[2] * dims[3] / 2;
    c->M5 = M5; c->b5 = b5; c->c5 = c5; c->mf = mf;
    {
        const double Mp = b5 * (4.0 - M5) + 1.0, Mm = c5 * (4.0 - M5) - 1.0;
        c->dense_s = (opts && opts->dense_s) || Mp == 0.0 || fabs(Mm / Mp) > 0.9;
        c->dense_s_base = c->dense_s;
    }
    c->autotune = opts && opts->autotune;
    c->slab = slab;
    // the default mass tables, so that an apply needs no host round trip
    if ((st = ensure_tables(c, 1, nullptr)) ||
        (st = cuda_status(cudaMalloc(&c->nbr, sizeof(int) * 16 * (size_t)c->g.Vh))) ||
        (st = cuda_status(cudaMalloc(&c->dev_err, sizeof(int)))) ||
        (st = cuda_status(cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream))) ||
        (st = launch_build_neighbours(c)) || (st = cuda_status(cudaStreamSynchronize(c->stream)))) {
        mdwf_destroy(c);
        return st;
    }
    *out = c;
    return MDWF_OK;
}

}  // namespace mdwf

extern "C" {

const char* mdwf_strerror(int status) {
    switch (status) {
        case MDWF_OK: return "MDWF_OK";
        case MDWF_EINVAL: return "MDWF_EINVAL: invalid argument";
        case MDWF_ENOMEM: return "MDWF_ENOMEM: out of memory";
        case MDWF_ECUDA: return "MDWF_ECUDA: CUDA runtime error";
        case MDWF_ENOCONV: return "MDWF_ENOCONV: solver did not converge";
        case MDWF_EBREAKDOWN: return "MDWF_EBREAKDOWN: CG breakdown";
        case MDWF_ETIMEOUT: return "MDWF_ETIMEOUT: device wait limit reached";
        case MDWF_ENOGAUGE: return "MDWF_ENOGAUGE: no gauge field loaded";
    }
    return "unknown mdwf status";
}

const char* mdwf_last_error(void) { return g_last_error; }

int mdwf_create(mdwf_ctx** out, const int dims[4], int Ls, double M5, double b5, double c5, double mf,
                const mdwf_opts* opts) {
    return mdwf::create_context(out, dims, Ls, M5, b5, c5, mf, opts, false);
}

int mdwf_create_slab(mdwf_ctx** out, const int local_dims[4], int Ls, double M5, double b5, double c5, double mf,
                     const mdwf_opts* opts) {
    return mdwf::create_context(out, local_dims, Ls, M5, b5, c5, mf, opts, true);
}

int mdwf_destroy(mdwf_ctx* c) {
    if (!c) return MDWF_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();  // an earlier call's failure was reported by that call
    for (int k = 0; k < 2; ++k) cudaFree(c->gauge[k]);
    cudaFree(c->tab64); cudaFree(c->tab32); cudaFree(c->mass64); cudaFree(c->mass32);
    cudaFreeHost(c->tab_host);
    cudaFree(c->tmp[0].p); cudaFree(c->tmp[1].p);
    cudaFree(c->solver.p);
    cudaFree(c->io.p);
    cudaFree(c->tune.p);
    cudaFree(c->aux.p);
    cudaFree(c->ov.p);
    cudaFree(c->gw.p);
    cudaFree(c->h4.p);
    cudaFree(c->red_partials);
    cudaFree(c->nbr);
    cudaFree(c->dev_err);
    cudaFree(c->gs64); cudaFree(c->gs32);
    for (auto& r : c->prof_pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    delete c;
    return check_launch();
}

int mdwf_set_s_coefficients(mdwf_ctx* c, const double* b5s, const double* c5s) {
    if (!c || (!b5s) != (!c5s)) return MDWF_EINVAL;
    const int Ls = c->g.Ls;
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    // kernels in flight may still read the tables or the gather factors
    if ((st = cuda_status(cudaStreamSynchronize(c->stream)))) return st;
    if (!b5s) {
        c->sdep = false;
        c->dense_s = c->dense_s_base;
        c->tab_valid = false;
        return ensure_tables(c, 1, nullptr);
    }
    for (int s = 0; s < Ls; ++s)
        if (!isfinite(b5s[s]) || !isfinite(c5s[s])) return MDWF_EINVAL;
    if (!c->gs64 && ((st = cuda_status(cudaMalloc(&c->gs64, 3 * 64 * sizeof(double)))) ||
                     (st = canary_fill(c->gs64, 3 * 64 * sizeof(double)))))
        return st;
    if (!c->gs32 && ((st = cuda_status(cudaMalloc(&c->gs32, 3 * 64 * sizeof(float)))) ||
                     (st = canary_fill(c->gs32, 3 * 64 * sizeof(float)))))
        return st;
    // gather factors of row s: M_phi psi at s = gscale (gown psi_s + gfac C psi)
    double h64[3 * 64] = {0};
    float h32[3 * 64] = {0};
    for (int s = 0; s < Ls; ++s) {
        const bool fold = b5s[s] != 0.0;
        h64[s] = fold ? 1.0 : 0.0;
        h64[64 + s] = fold ? c5s[s] / b5s[s] : c5s[s];
        h64[128 + s] = fold ? b5s[s] : 1.0;
    }
    for (int k = 0; k < 3 * 64; ++k) h32[k] = (float)h64[k];
    const bool was_sdep = c->sdep, was_dense = c->dense_s;
    double ob[64], oc[64];
    memcpy(ob, c->b5s, sizeof(ob));
    memcpy(oc, c->c5s, sizeof(oc));
    for (int s = 0; s < Ls; ++s) { c->b5s[s] = b5s[s]; c->c5s[s] = c5s[s]; }
    c->sdep = true;
    c->dense_s = true;
    c->tab_valid = false;
    st = ensure_tables(c, 1, nullptr);
    if (st) {  // singular I: keep the previous coefficients
        memcpy(c->b5s, ob, sizeof(ob));
        memcpy(c->c5s, oc, sizeof(oc));
        c->sdep = was_sdep;
        c->dense_s = was_dense;
        c->tab_valid = false;
        const int s2 = ensure_tables(c, 1, nullptr);
        return s2 ? s2 : st;
    }
    // synchronous copies from pageable host memory: the factors are in place on return
    if ((st = cuda_status(cudaMemcpy(c->gs64, h64, sizeof(h64), cudaMemcpyHostToDevice)))) return st;
    return cuda_status(cudaMemcpy(c->gs32, h32, sizeof(h32), cudaMemcpyHostToDevice));
}

int mdwf_set_chemical_potential(mdwf_ctx* c, double mu) {
    if (!c || !isfinite(mu) || fabs(mu) > 10.0) return MDWF_EINVAL;
    c->chem = mu;
    return MDWF_OK;
}

int mdwf_get_geometry(const mdwf_ctx* c, int dims[4], int* Ls) {
    if (!c || !dims || !Ls) return MDWF_EINVAL;
    dims[0] = c->g.X; dims[1] = c->g.Y; dims[2] = c->g.Z; dims[3] = c->g.T;
    *Ls = c->g.Ls;
    return MDWF_OK;
}

int mdwf_get_s_coefficients(const mdwf_ctx* c, double* b5s, double* c5s, int* per_slice) {
    if (!c || !b5s || !c5s || !per_slice) return MDWF_EINVAL;
    for (int s = 0; s < c->g.Ls; ++s) {
        b5s[s] = c->sdep ? c->b5s[s] : c->b5;
        c5s[s] = c->sdep ? c->c5s[s] : c->c5;
    }
    *per_slice = c->sdep ? 1 : 0;
    return MDWF_OK;
}

int mdwf_set_stream(mdwf_ctx* c, void* stream) {
    if (!c) return MDWF_EINVAL;
    c->stream = (cudaStream_t)stream;
    return MDWF_OK;
}

int mdwf_load_gauge(mdwf_ctx* c, const double* U, int where) {
    NvtxRange nvtx_range("mdwf_load_gauge");
    if (!c || !U || (where != MDWF_HOST && where != MDWF_DEVICE)) return MDWF_EINVAL;
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    const size_t nlink = (size_t)c->g.Vh * 2 * 4;
    const size_t bytes[2] = {nlink * link_store_bytes(MDWF_F64), nlink * link_store_bytes(MDWF_F32)};
    for (int k = 0; k < 2; ++k)
        if (!c->gauge[k] && ((st = cuda_status(cudaMalloc(&c->gauge[k], bytes[k]))) ||
                             (st = canary_fill(c->gauge[k], bytes[k]))))
            return st;
    const double* src = U;
    void* stage = nullptr;
    if (where == MDWF_HOST) {
        if ((st = cuda_status(cudaMalloc(&stage, nlink * 144)))) return st;
        st = cuda_status(cudaMemcpyAsync(stage, U, nlink * 144, cudaMemcpyHostToDevice, c->stream));
        if (st) { cudaFree(stage); return st; }
        src = (const double*)stage;
    }
    st = launch_gauge_pack(c, src);
    if (stage) {
        int s2 = cuda_status(cudaStreamSynchronize(c->stream));
        cudaFree(stage);
        if (!st) st = s2;
    }
    if (!st) c->have_gauge = true;
    return st;
}

size_t mdwf_field_bytes(const mdwf_ctx* c, int prec, int nrhs) {
    if (!c || nrhs < 1) return 0;
    return field_bytes(prec, c->g, nrhs);
}

static bool valid_prec(int p) { return p == MDWF_F64 || p == MDWF_F32 || p == MDWF_F16N; }

int mdwf_field_import(mdwf_ctx* c, void* dst, const double* src, int prec, int nrhs, int where) {
    if (!c || !dst || !src || !valid_prec(prec) || nrhs < 1 || (where != MDWF_HOST && where != MDWF_DEVICE))
        return MDWF_EINVAL;
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    const size_t ub = (size_t)nrhs * c->g.Ls * c->g.Vh * 24 * sizeof(double);
    const double* s = src;
    void* stage = nullptr;
    if (where == MDWF_HOST) {
        if ((st = cuda_status(cudaMalloc(&stage, ub)))) return st;
        st = cuda_status(cudaMemcpyAsync(stage, src, ub, cudaMemcpyHostToDevice, c->stream));
        if (st) { cudaFree(stage); return st; }
        s = (const double*)stage;
    }
    st = launch_import_odd(c, dst, s, prec, nrhs);
    if (stage) {
        int s2 = cuda_status(cudaStreamSynchronize(c->stream));
        cudaFree(stage);
        if (!st) st = s2;
    }
    return st;
}

int mdwf_field_export(mdwf_ctx* c, double* dst, const void* src, int prec, int nrhs, int where) {
    if (!c || !dst || !src || !valid_prec(prec) || nrhs < 1 || (where != MDWF_HOST && where != MDWF_DEVICE))
        return MDWF_EINVAL;
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    const size_t ub = (size_t)nrhs * c->g.Ls * c->g.Vh * 24 * sizeof(double);
    if (where == MDWF_DEVICE) return launch_export_odd(c, dst, src, prec, nrhs);
    void* stage = nullptr;
    if ((st = cuda_status(cudaMalloc(&stage, ub)))) return st;
    st = launch_export_odd(c, (double*)stage, src, prec, nrhs);
    if (!st) st = cuda_status(cudaMemcpyAsync(dst, stage, ub, cudaMemcpyDeviceToHost, c->stream));
    int s2 = cuda_status(cudaStreamSynchronize(c->stream));
    cudaFree(stage);
    return st ? st : s2;
}

static int apply_entry(mdwf_ctx* c, void* out, const void* in, int prec, int nrhs, const double* mf, int dagger) {
    NvtxRange nvtx_range("mdwf_apply");
    if (!c || !out || !in || !valid_prec(prec) || nrhs < 1 || nrhs > 64 || out == in) return MDWF_EINVAL;
    if (!c->have_gauge) return MDWF_ENOGAUGE;
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    if ((st = ensure_tables(c, nrhs, mf))) return st;
    return apply_op(c, out, in, prec, nrhs, dagger);
}

int mdwf_apply(mdwf_ctx* c, void* out, const void* in, int prec, int nrhs, const double* mf_per_rhs) {
    return apply_entry(c, out, in, prec, nrhs, mf_per_rhs, 0);
}

int mdwf_apply_dag(mdwf_ctx* c, void* out, const void* in, int prec, int nrhs, const double* mf_per_rhs) {
    return apply_entry(c, out, in, prec, nrhs, mf_per_rhs, 1);
}

int mdwf_profile_enable(mdwf_ctx* c, int enable) {
    if (!c) return MDWF_EINVAL;
    c->prof_on = enable != 0;
    return MDWF_OK;
}

int mdwf_profile_read(mdwf_ctx* c, mdwf_kernel_stat* out, int max, int* n_out, int reset) {
    if (!c || (max > 0 && !out)) return MDWF_EINVAL;
    int st = cuda_status(cudaStreamSynchronize(c->stream));
    if (st) return st;
    for (auto& r : c->prof_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) c->kstat[r.kind].ms += ms;
        c->ev_pool.push_back(r.a);
        c->ev_pool.push_back(r.b);
    }
    c->prof_pending.clear();
    int n = 0;
    for (int k = 0; k < KK_NUM; ++k) {
        if (c->kstat[k].launches == 0) continue;
        if (n < max) {
            kernel_name(k, out[n].name, sizeof(out[n].name));
            out[n].launches = c->kstat[k].launches;
            out[n].ms = c->kstat[k].ms;
            out[n].bytes = c->kstat[k].bytes;
            out[n].flops = c->kstat[k].flops;
        }
        ++n;
    }
    if (n_out) *n_out = n < max ? n : max;
    if (reset)
        for (int k = 0; k < KK_NUM; ++k) c->kstat[k] = KStat{};
    return MDWF_OK;
}

int mdwf_autotune(mdwf_ctx* c, int prec, int nrhs, int* sites_per_block) {
    NvtxRange nvtx_range("mdwf_autotune");
    if (!c || !valid_prec(prec) || nrhs < 1 || nrhs > 64) return MDWF_EINVAL;
    if (!c->have_gauge) return MDWF_ENOGAUGE;
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    if ((st = ensure_tables(c, nrhs, nullptr))) return st;
    int sb = 0;
    if ((st = tune_hop(c, prec, nrhs, &sb))) return st;
    if (sites_per_block) *sites_per_block = sb;
    return MDWF_OK;
}

int mdwf_set_tuning(mdwf_ctx* c, int prec, int nrhs, int sites_per_block) {
    if (!c || !valid_prec(prec) || nrhs < 1 || nrhs > 64 || sites_per_block < 0) return MDWF_EINVAL;
    if (sites_per_block > 0 && sites_per_block * c->g.Ls > 128) return MDWF_EINVAL;
    c->sb_tune[prec][nrhs] = sites_per_block;
    return MDWF_OK;
}

int mdwf_get_tuning(const mdwf_ctx* c, int prec, int nrhs, int* sites_per_block) {
    if (!c || !valid_prec(prec) || nrhs < 1 || nrhs > 64 || !sites_per_block) return MDWF_EINVAL;
    *sites_per_block = hop_sites_per_block(c, prec, nrhs);
    return MDWF_OK;
}

int mdwf_set_staging(mdwf_ctx* c, int prec, int staged) {
    if (!c || !valid_prec(prec) || staged < 0 || staged > 4) return MDWF_EINVAL;
    if (prec == MDWF_F64 && staged) return MDWF_EINVAL;
    // bulk copies of the FP16 norms need 16-byte columns (4 Ls bytes)
    if (prec == MDWF_F16N && staged == 2 && c->g.Ls % 4 != 0) return MDWF_EINVAL;
    c->hop_stage[prec] = staged;
    return MDWF_OK;
}

int mdwf_get_staging(const mdwf_ctx* c, int prec, int* staged) {
    if (!c || !valid_prec(prec) || !staged) return MDWF_EINVAL;
    *staged = c->hop_stage[prec];
    return MDWF_OK;
}

int mdwf_bounds_status(int* checked, int* violations, int reset) {
    if (!checked || !violations) return MDWF_EINVAL;
    *checked = MDWF_BOUNDS_CHECK ? 1 : 0;
    *violations = 0;
#if MDWF_BOUNDS_CHECK
    int* w = bounds_word();
    if (!w) return MDWF_ECUDA;
    int st;
    if ((st = cuda_status(cudaDeviceSynchronize()))) return st;
    if ((st = cuda_status(cudaMemcpy(violations, w, sizeof(int), cudaMemcpyDeviceToHost)))) return st;
    if (reset && (st = cuda_status(cudaMemset(w, 0, sizeof(int))))) return st;
#else
    (void)reset;
#endif
    return MDWF_OK;
}

int mdwf_device_status(mdwf_ctx* c) {
    if (!c) return MDWF_EINVAL;
    int st;
    if ((st = cuda_status(cudaSetDevice(c->device)))) return st;
    return device_wait_status(c);
}

int mdwf_counters(const mdwf_ctx* c, long long* launches, long long applies[3]) {
    if (!c) return MDWF_EINVAL;
    if (launches) *launches = c->launches;
    if (applies)
        for (int p = 0; p < 3; ++p) applies[p] = c->applies[p];
    return MDWF_OK;
}

}  // extern "C"
