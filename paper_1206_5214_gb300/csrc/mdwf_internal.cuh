// Internal declarations of libmdwf: data layouts in HBM, device-side field
// access and the launchers every translation unit shares.
//
// HBM layout of an internal half (one-parity) field of nrhs right-hand sides:
//   chunk = W consecutive reals of the 24-real spinor [spin][colour][re, im],
//   stored [rhs][site][chunk][s] so that the Ls threads of one 4d site read
//   consecutive chunks (coalesced) and each chunk is one vector load:
//     F64 : W = 2 (double2), 12 chunks  -> 192 B per 5d site
//     F32 : W = 4 (float4),   6 chunks  ->  96 B per 5d site
//     F16N: W = 4 (4 x half), 6 chunks  ->  48 B + a 4-byte FP32 norm per 5d site,
//           norms stored after all values as [rhs][site][s]
//   Chunks 0 .. NC/2-1 hold spins 0, 1 (the P+ half), the rest spins 2, 3 (P-).
//   Sites of a parity are ordered lexicographically (x fastest): the site
//   (x, y, z, t) of that parity has index (((t Z + z) Y + y) X + x) / 2.
// Gauge links: [parity][mu][site of that parity][3][3] complex, in FP64,
//   FP32 and FP16 copies (18 reals per link).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "mdwf.h"

namespace mdwf {

constexpr int kMaxLs = 32;

struct Geom {
    int X, Y, Z, T, Ls;
    long long Vh;  // sites per parity
};

// ---------------------------------------------------------------- precisions

template <int P> struct PrecTraits;
template <> struct PrecTraits<MDWF_F64> {
    typedef double real;
    static constexpr int W = 2, NC = 12;
    static constexpr size_t site_bytes = 192;
};
template <> struct PrecTraits<MDWF_F32> {
    typedef float real;
    static constexpr int W = 4, NC = 6;
    static constexpr size_t site_bytes = 96;
};
template <> struct PrecTraits<MDWF_F16N> {
    typedef float real;
    static constexpr int W = 4, NC = 6;
    static constexpr size_t site_bytes = 52;
};

inline size_t field_bytes(int prec, const Geom& g, int nrhs) {
    size_t n5 = (size_t)g.Vh * g.Ls * (size_t)nrhs;
    switch (prec) {
        case MDWF_F64: return n5 * 192;
        case MDWF_F32: return n5 * 96;
        case MDWF_F16N: return n5 * 52;
    }
    return 0;
}

// Device view of an internal field. `sr` below is rhs * Vh + site.
template <int P> struct Field;

template <> struct Field<MDWF_F64> {
    double2* v;
    int Ls;
    __device__ __forceinline__ void load(long long sr, int s, double* o) const {
        const double2* p = v + sr * 12 * Ls + s;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 d = __ldg(p + (long long)k * Ls);
            o[2 * k] = d.x;
            o[2 * k + 1] = d.y;
        }
    }
    // half = 0: spins 0, 1 (reals 0..11); half = 1: spins 2, 3 (reals 12..23)
    __device__ __forceinline__ void load_half(long long sr, int s, int half, double* o) const {
        const double2* p = v + sr * 12 * Ls + (long long)(6 * half) * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            double2 d = __ldg(p + (long long)k * Ls);
            o[2 * k] = d.x;
            o[2 * k + 1] = d.y;
        }
    }
    __device__ __forceinline__ void store(long long sr, int s, const double* i) const {
        double2* p = v + sr * 12 * Ls + s;
#pragma unroll
        for (int k = 0; k < 12; ++k) p[(long long)k * Ls] = make_double2(i[2 * k], i[2 * k + 1]);
    }
};

template <> struct Field<MDWF_F32> {
    float4* v;
    int Ls;
    __device__ __forceinline__ void load(long long sr, int s, float* o) const {
        const float4* p = v + sr * 6 * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 d = __ldg(p + (long long)k * Ls);
            o[4 * k] = d.x; o[4 * k + 1] = d.y; o[4 * k + 2] = d.z; o[4 * k + 3] = d.w;
        }
    }
    __device__ __forceinline__ void load_half(long long sr, int s, int half, float* o) const {
        const float4* p = v + sr * 6 * Ls + (long long)(3 * half) * Ls + s;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 d = __ldg(p + (long long)k * Ls);
            o[4 * k] = d.x; o[4 * k + 1] = d.y; o[4 * k + 2] = d.z; o[4 * k + 3] = d.w;
        }
    }
    __device__ __forceinline__ void store(long long sr, int s, const float* i) const {
        float4* p = v + sr * 6 * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            p[(long long)k * Ls] = make_float4(i[4 * k], i[4 * k + 1], i[4 * k + 2], i[4 * k + 3]);
    }
};

template <> struct Field<MDWF_F16N> {
    uint2* v;     // 4 halves per chunk
    float* norm;  // [rhs][site][s]
    int Ls;
    __device__ __forceinline__ static void unpack(uint2 d, float nrm, float* o) {
        __half2 a = *reinterpret_cast<__half2*>(&d.x);
        __half2 b = *reinterpret_cast<__half2*>(&d.y);
        float2 fa = __half22float2(a), fb = __half22float2(b);
        o[0] = fa.x * nrm; o[1] = fa.y * nrm; o[2] = fb.x * nrm; o[3] = fb.y * nrm;
    }
    __device__ __forceinline__ void load(long long sr, int s, float* o) const {
        const uint2* p = v + sr * 6 * Ls + s;
        float nrm = __ldg(norm + sr * Ls + s);
#pragma unroll
        for (int k = 0; k < 6; ++k) unpack(__ldg(p + (long long)k * Ls), nrm, o + 4 * k);
    }
    __device__ __forceinline__ void load_half(long long sr, int s, int half, float* o) const {
        const uint2* p = v + sr * 6 * Ls + (long long)(3 * half) * Ls + s;
        float nrm = __ldg(norm + sr * Ls + s);
#pragma unroll
        for (int k = 0; k < 3; ++k) unpack(__ldg(p + (long long)k * Ls), nrm, o + 4 * k);
    }
    __device__ __forceinline__ void store(long long sr, int s, const float* i) const {
        float mx = 0.f;
#pragma unroll
        for (int k = 0; k < 24; ++k) mx = fmaxf(mx, fabsf(i[k]));
        float inv = mx > 0.f ? 1.0f / mx : 0.f;
        uint2* p = v + sr * 6 * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            __half2 a = __floats2half2_rn(i[4 * k] * inv, i[4 * k + 1] * inv);
            __half2 b = __floats2half2_rn(i[4 * k + 2] * inv, i[4 * k + 3] * inv);
            uint2 d;
            d.x = *reinterpret_cast<uint32_t*>(&a);
            d.y = *reinterpret_cast<uint32_t*>(&b);
            p[(long long)k * Ls] = d;
        }
        norm[sr * Ls + s] = mx;
    }
};

// Host-side construction of a field view from a base pointer.
template <int P> inline Field<P> make_field(void* base, const Geom& g, int nrhs);
template <> inline Field<MDWF_F64> make_field<MDWF_F64>(void* base, const Geom& g, int) {
    Field<MDWF_F64> f; f.v = (double2*)base; f.Ls = g.Ls; return f;
}
template <> inline Field<MDWF_F32> make_field<MDWF_F32>(void* base, const Geom& g, int) {
    Field<MDWF_F32> f; f.v = (float4*)base; f.Ls = g.Ls; return f;
}
template <> inline Field<MDWF_F16N> make_field<MDWF_F16N>(void* base, const Geom& g, int nrhs) {
    Field<MDWF_F16N> f;
    f.v = (uint2*)base;
    f.norm = (float*)((char*)base + (size_t)g.Vh * g.Ls * nrhs * 48);
    f.Ls = g.Ls;
    return f;
}

// ------------------------------------------------------------------- gauge

template <int P> struct Gauge;
template <> struct Gauge<MDWF_F64> {
    const double2* u;  // [parity][mu][site][9] complex
    __device__ __forceinline__ void load(long long idx, double* o) const {
        const double2* p = u + idx * 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) { double2 d = __ldg(p + k); o[2 * k] = d.x; o[2 * k + 1] = d.y; }
    }
};
template <> struct Gauge<MDWF_F32> {
    const float2* u;
    __device__ __forceinline__ void load(long long idx, float* o) const {
        const float2* p = u + idx * 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) { float2 d = __ldg(p + k); o[2 * k] = d.x; o[2 * k + 1] = d.y; }
    }
};
template <> struct Gauge<MDWF_F16N> {
    const __half2* u;
    __device__ __forceinline__ void load(long long idx, float* o) const {
        const __half2* p = u + idx * 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) { float2 d = __half22float2(p[k]); o[2 * k] = d.x; o[2 * k + 1] = d.y; }
    }
};

// ----------------------------------------------------------------- geometry

__device__ __forceinline__ void cb_coords(const Geom& g, long long j, int parity, int c[4]) {
    int Xh = g.X >> 1;
    long long r = j;
    int xh = (int)(r % Xh); r /= Xh;
    c[1] = (int)(r % g.Y); r /= g.Y;
    c[2] = (int)(r % g.Z); r /= g.Z;
    c[3] = (int)r;
    c[0] = 2 * xh + ((parity + c[1] + c[2] + c[3]) & 1);
}

__device__ __forceinline__ long long cb_index(const Geom& g, int x, int y, int z, int t) {
    return ((((long long)t * g.Z + z) * g.Y + y) * g.X + x) >> 1;
}

// ------------------------------------------------------------------ tables
//
// Ls x Ls real matrices acting along s, one per chirality, for each operator
// in the chain: table[op][rhs][chir][s'][s] holds element (s, s') (transposed,
// so that the Ls threads of a column read consecutive words). chir 0 is the
// P+ half (spins 0, 1), chir 1 the P- half.
enum TableOp { T_K = 0, T_A = 1, T_ADAG = 2, T_KDAG = 3, T_MPHIDAG = 4, T_ID = 5, T_NUM = 6 };

// ---------------------------------------------------------------- context

struct Workspace {
    void* p = nullptr;
    size_t bytes = 0;
};

// Kernel kinds for profiling and counting: kind = base * 3 + precision.
enum KernelBase {
    KB_HOP = 0, KB_HOP_GATHER, KB_HOP_XPAY, KB_HOP_GATHER_XPAY, KB_HOP_DAG, KB_HOP_DAG_XPAY,
    KB_M5, KB_M5_XPAY, KB_BLAS, KB_LAYOUT, KB_NUM
};
constexpr int KK_NUM = KB_NUM * 3;

struct KStat {
    long long launches = 0;
    double ms = 0, bytes = 0, flops = 0;
};

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};

// algorithmic bytes per 5d site and per link, by precision
inline double site_bytes(int prec) { return prec == MDWF_F64 ? 192.0 : prec == MDWF_F32 ? 96.0 : 52.0; }
inline double link_bytes(int prec) { return prec == MDWF_F64 ? 144.0 : prec == MDWF_F32 ? 72.0 : 36.0; }

}  // namespace mdwf

struct mdwf_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    mdwf::Geom g{};
    double M5 = 0, b5 = 0, c5 = 0, mf = 0;
    bool have_gauge = false;
    void* gauge[3] = {nullptr, nullptr, nullptr};  // F64, F32, F16 copies
    // Ls x Ls tables for the current mass list, FP64 and FP32, plus per-rhs masses
    double* tab64 = nullptr;
    float* tab32 = nullptr;
    double* mass64 = nullptr;
    float* mass32 = nullptr;
    int tab_nrhs = 0;
    double* tab_host = nullptr;     // pinned staging for the tables
    double tab_masses[64] = {0};
    bool tab_valid = false;
    // scratch fields used inside one apply: [0] even-parity z, [1] odd-parity v
    mdwf::Workspace tmp[2];
    // solver workspace
    mdwf::Workspace solver;
    // reduction scratch: per-rhs block partials and scalars
    double* red_partials = nullptr;
    size_t red_partials_len = 0;
    int tab_cap = 0;
    // instrumentation: counters always, CUDA events per launch when prof_on
    bool prof_on = false;
    bool capturing = false;
    std::vector<mdwf::ProfRec> prof_pending;
    std::vector<cudaEvent_t> ev_pool;
    mdwf::KStat kstat[mdwf::KK_NUM];
    long long launches = 0;
    long long applies[3] = {0, 0, 0};
    // content of the CUDA graph being captured (added once per replay)
    long long cap_launches = 0;
    long long cap_applies[3] = {0, 0, 0};
    mdwf::KStat cap_kstat[mdwf::KK_NUM];
};

namespace mdwf {

// Brackets one kernel launch: counts it (or adds it to the graph being
// captured) with its algorithmic bytes and flops, and records CUDA events
// around it on the launch stream while profiling is on.
class LaunchScope {
   public:
    LaunchScope(mdwf_ctx* c, int kind, double bytes, double flops);
    ~LaunchScope();

   private:
    mdwf_ctx* c_;
    int kind_;
    double bytes_, flops_;
    cudaEvent_t a_ = nullptr;
};
void note_apply(mdwf_ctx* c, int prec);
void replay_graph_counts(mdwf_ctx* c, long long replays);

// status helpers (api.cu)
int cuda_status(cudaError_t e);
int check_launch();
int ensure_workspace(Workspace& w, size_t bytes);
int ensure_tables(mdwf_ctx* c, int nrhs, const double* mf_per_rhs);

// table pointers for op, precision
inline const void* table_ptr(const mdwf_ctx* c, int prec, int op) {
    size_t per_op = (size_t)c->tab_nrhs * 2 * c->g.Ls * c->g.Ls;
    if (prec == MDWF_F64) return c->tab64 + op * per_op;
    return c->tab32 + op * per_op;
}

// launchers (dslash.cu, m5.cu)
struct HopLaunch {
    void* out;
    const void* in;
    const void* x;        // xpay addend (same parity as out) or nullptr
    double coef;          // result = coef * Mat (H in) [+ x]
    int out_parity;
    int gather;           // 1: apply M_phi (b5 + c5 C) to the input column before the hop
    int dagger;           // 1: hopping term of D_W^dag (projector signs flipped)
    const void* mat;      // table of the output Ls x Ls matrix (this precision), per rhs
    const void* mass;     // per-rhs masses (double for F64, float otherwise)
    double b5, c5;
    int nrhs;
};
int launch_hop(mdwf_ctx* c, int prec, const HopLaunch& h);

struct M5Launch {
    void* out;
    const void* in;
    const void* x;    // optional addend
    double coef;      // out = coef * Mat in [+ x]
    const void* mat;
    int nrhs;
};
int launch_m5(mdwf_ctx* c, int prec, const M5Launch& m);

// operator chains (api.cu)
int apply_op(mdwf_ctx* c, void* out, const void* in, int prec, int nrhs, int dagger);

// layout kernels (layout.cu)
int launch_import_odd(mdwf_ctx* c, void* dst, const double* src_dev, int prec, int nrhs);
int launch_export_odd(mdwf_ctx* c, double* dst_dev, const void* src, int prec, int nrhs);
int launch_split_full(mdwf_ctx* c, void* dst_even, void* dst_odd, const double* full_dev, int prec, int nrhs);
int launch_join_full(mdwf_ctx* c, double* full_dev, const void* even, const void* odd, int prec, int nrhs);
int launch_gauge_pack(mdwf_ctx* c, const double* U_dev);

}  // namespace mdwf
