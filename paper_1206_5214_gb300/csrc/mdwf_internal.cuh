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
// Gauge links: [parity][mu][site of that parity][3][3] complex, an FP64 copy
//   (144 B per link) and an FP32 copy padded to 80 B (read by the FP32 and
//   FP16+norm operators).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mdwf.h"

// Blocks per SM the hop kernels are compiled for (register budget per thread:
// 65536 / (128 * blocks)); overridable at build time.
#ifndef MDWF_MINB_F64
#define MDWF_MINB_F64 3
#endif
#ifndef MDWF_MINB_F32
#define MDWF_MINB_F32 8
#endif

namespace mdwf {

// An NVTX range around one library call, so that timeline profilers show the
// entry points (header-only NVTX: no cost without an attached tool).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kMaxLs = 32;
constexpr int kMaxRhs = 64;  // right-hand sides per call

// CG scalars per right-hand side, stored [slot][kMaxRhs] in device memory:
// |r|^2, <p, M^dag M p>, alpha, beta, |src|^2, active flag, status, scratch,
// iteration count, the flag of a right-hand side whose FP64 reliable update
// runs now, the flag of one that rolls back to its last update, and two
// coefficients of the search-direction correction of a reliable update.
enum CgSlot {
    S_RR = 0, S_PAP, S_ALPHA, S_BETA, S_SRC2, S_ACTIVE, S_STATUS, S_AUX, S_ITERS, S_UPD, S_RESTART, S_C1, S_C2, S_NUM
};
// What a finished reduction v does: store it in a slot, or form alpha from
// v = <p, M^dag M p>, or beta from v = |r_new|^2 (and count the iteration).
enum FinMode { FIN_STORE = 0, FIN_ALPHA = 1, FIN_BETA = 2 };

__device__ inline void cg_scalar_update(double* sc, int rhs, int mode, int slot, double v) {
    double* S = sc + rhs;  // S[k * kMaxRhs] is slot k of this right-hand side
    const bool active = S[S_ACTIVE * kMaxRhs] != 0.0;
    if (mode == FIN_STORE) {
        S[slot * kMaxRhs] = v;
    } else if (mode == FIN_ALPHA) {
        S[S_PAP * kMaxRhs] = v;
        double a = 0.0;
        if (active) {
            if (!(v > 0.0) || !isfinite(v)) {
                S[S_STATUS * kMaxRhs] = (double)MDWF_EBREAKDOWN;
                S[S_ACTIVE * kMaxRhs] = 0.0;
            } else {
                a = S[S_RR * kMaxRhs] / v;
            }
        }
        S[S_ALPHA * kMaxRhs] = a;
    } else {
        double b = 0.0;
        if (active) {
            if (!isfinite(v)) {
                S[S_STATUS * kMaxRhs] = (double)MDWF_EBREAKDOWN;
                S[S_ACTIVE * kMaxRhs] = 0.0;
            } else {
                b = v / S[S_RR * kMaxRhs];
                S[S_RR * kMaxRhs] = v;
                S[S_ITERS * kMaxRhs] += 1.0;
            }
        }
        S[S_BETA * kMaxRhs] = b;
    }
}

struct Geom {
    int X, Y, Z, T, Ls;
    long long Vh;  // sites per parity
};

// ---------------------------------------------------------------- precisions

template <int P> struct PrecTraits;
template <> struct PrecTraits<MDWF_F64> {
    typedef double real;
    static constexpr int min_blocks = MDWF_MINB_F64;  // 128-thread blocks per SM the hop kernel is compiled for
    static constexpr int W = 2, NC = 12;
    static constexpr size_t site_bytes = 192;
};
template <> struct PrecTraits<MDWF_F32> {
    typedef float real;
    static constexpr int min_blocks = MDWF_MINB_F32;
    static constexpr int W = 4, NC = 6;
    static constexpr size_t site_bytes = 96;
};
template <> struct PrecTraits<MDWF_F16N> {
    typedef float real;
    static constexpr int min_blocks = MDWF_MINB_F32;
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

// Cache hint: fetch the line of p into L1 (no register is written).
__device__ __forceinline__ void prefetch_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];\n" ::"l"(p));
}

// Programmatic dependent launch. A kernel launched by launch_pdl may be
// scheduled while the kernel before it on the stream is still running (its
// blocks then wait on SMs that the earlier kernel has left). Such a kernel
// calls pdl_wait() before it reads anything an earlier kernel wrote, and every
// one of its blocks reaches pdl_wait() before it exits, so that it completes
// after its predecessor. pdl_release() lets the next kernel be scheduled.
// Without a programmatic predecessor both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                              Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Bounds-checked debug build (-DMDWF_BOUNDS_CHECK=1, a separate library): every
// field access checks 0 <= sr < (sites x right-hand sides of the view) and
// 0 <= s < Ls, and every link access 0 <= index < 8 Vh; an access out of range
// is skipped (a load returns zeros), and the device's bounds word records it
// (mdwf_bounds_status). It stands in for a memory checker; the release build
// compiles no checks.
#ifndef MDWF_BOUNDS_CHECK
#define MDWF_BOUNDS_CHECK 0
#endif
int* bounds_word();  // device address of the current device's bounds word (debug build; else null)

struct Bounds {
#if MDWF_BOUNDS_CHECK
    long long n = 0;   // valid indices of the view
    int* err = nullptr;
    __device__ __forceinline__ bool bad(long long i, int s, int Ls) const {
        if (i >= 0 && i < n && s >= 0 && s < Ls) return false;
        atomicOr(err, 1);
        return true;
    }
#else
    __device__ __forceinline__ static constexpr bool bad(long long, int, int) { return false; }
#endif
};

// Device view of an internal field. `sr` below is rhs * Vh + site.
// prefetch(sr, s) asks L1 for the lines that load(sr, s) will read.
template <int P> struct Field;

template <> struct Field<MDWF_F64> {
    double2* v;
    int Ls;
    Bounds bnd;
    __device__ __forceinline__ void load(long long sr, int s, double* o) const {
        if (bnd.bad(sr, s, Ls)) { for (int k = 0; k < 24; ++k) o[k] = 0; return; }
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
        if (bnd.bad(sr, s, Ls)) { for (int k = 0; k < 12; ++k) o[k] = 0; return; }
        const double2* p = v + sr * 12 * Ls + (long long)(6 * half) * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            double2 d = __ldg(p + (long long)k * Ls);
            o[2 * k] = d.x;
            o[2 * k + 1] = d.y;
        }
    }
    __device__ __forceinline__ void prefetch(long long sr, int s) const {
        if (bnd.bad(sr, s, Ls)) return;
        const double2* p = v + sr * 12 * Ls + s;
#pragma unroll
        for (int k = 0; k < 12; ++k) prefetch_l1(p + (long long)k * Ls);
    }
    __device__ __forceinline__ void store(long long sr, int s, const double* i) const {
        if (bnd.bad(sr, s, Ls)) return;
        double2* p = v + sr * 12 * Ls + s;
#pragma unroll
        for (int k = 0; k < 12; ++k) p[(long long)k * Ls] = make_double2(i[2 * k], i[2 * k + 1]);
    }
};

template <> struct Field<MDWF_F32> {
    float4* v;
    int Ls;
    Bounds bnd;
    __device__ __forceinline__ void load(long long sr, int s, float* o) const {
        if (bnd.bad(sr, s, Ls)) { for (int k = 0; k < 24; ++k) o[k] = 0; return; }
        const float4* p = v + sr * 6 * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 d = __ldg(p + (long long)k * Ls);
            o[4 * k] = d.x; o[4 * k + 1] = d.y; o[4 * k + 2] = d.z; o[4 * k + 3] = d.w;
        }
    }
    __device__ __forceinline__ void load_half(long long sr, int s, int half, float* o) const {
        if (bnd.bad(sr, s, Ls)) { for (int k = 0; k < 12; ++k) o[k] = 0; return; }
        const float4* p = v + sr * 6 * Ls + (long long)(3 * half) * Ls + s;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 d = __ldg(p + (long long)k * Ls);
            o[4 * k] = d.x; o[4 * k + 1] = d.y; o[4 * k + 2] = d.z; o[4 * k + 3] = d.w;
        }
    }
    __device__ __forceinline__ void prefetch(long long sr, int s) const {
        if (bnd.bad(sr, s, Ls)) return;
        const float4* p = v + sr * 6 * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; ++k) prefetch_l1(p + (long long)k * Ls);
    }
    __device__ __forceinline__ void store(long long sr, int s, const float* i) const {
        if (bnd.bad(sr, s, Ls)) return;
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
    Bounds bnd;
    __device__ __forceinline__ static void unpack(uint2 d, float nrm, float* o) {
        __half2 a = *reinterpret_cast<__half2*>(&d.x);
        __half2 b = *reinterpret_cast<__half2*>(&d.y);
        float2 fa = __half22float2(a), fb = __half22float2(b);
        o[0] = fa.x * nrm; o[1] = fa.y * nrm; o[2] = fb.x * nrm; o[3] = fb.y * nrm;
    }
    __device__ __forceinline__ static void unpack_raw(uint2 d, float* o) {
        __half2 a = *reinterpret_cast<__half2*>(&d.x);
        __half2 b = *reinterpret_cast<__half2*>(&d.y);
        float2 fa = __half22float2(a), fb = __half22float2(b);
        o[0] = fa.x; o[1] = fa.y; o[2] = fb.x; o[3] = fb.y;
    }
    __device__ __forceinline__ void load(long long sr, int s, float* o) const {
        if (bnd.bad(sr, s, Ls)) { for (int k = 0; k < 24; ++k) o[k] = 0; return; }
        const uint2* p = v + sr * 6 * Ls + s;
        float nrm = __ldg(norm + sr * Ls + s);
#pragma unroll
        for (int k = 0; k < 6; ++k) unpack(__ldg(p + (long long)k * Ls), nrm, o + 4 * k);
    }
    // values without the norm; returns the norm (its factor is applied later)
    __device__ __forceinline__ float load_raw(long long sr, int s, float* o) const {
        if (bnd.bad(sr, s, Ls)) { for (int k = 0; k < 24; ++k) o[k] = 0; return 0.f; }
        const uint2* p = v + sr * 6 * Ls + s;
        const float nrm = __ldg(norm + sr * Ls + s);
#pragma unroll
        for (int k = 0; k < 6; ++k) unpack_raw(__ldg(p + (long long)k * Ls), o + 4 * k);
        return nrm;
    }
    __device__ __forceinline__ void load_half(long long sr, int s, int half, float* o) const {
        if (bnd.bad(sr, s, Ls)) { for (int k = 0; k < 12; ++k) o[k] = 0; return; }
        const uint2* p = v + sr * 6 * Ls + (long long)(3 * half) * Ls + s;
        float nrm = __ldg(norm + sr * Ls + s);
#pragma unroll
        for (int k = 0; k < 3; ++k) unpack(__ldg(p + (long long)k * Ls), nrm, o + 4 * k);
    }
    __device__ __forceinline__ void prefetch(long long sr, int s) const {
        if (bnd.bad(sr, s, Ls)) return;
        const uint2* p = v + sr * 6 * Ls + s;
#pragma unroll
        for (int k = 0; k < 6; ++k) prefetch_l1(p + (long long)k * Ls);
        prefetch_l1(norm + sr * Ls + s);
    }
    __device__ __forceinline__ void store(long long sr, int s, const float* i) const {
        if (bnd.bad(sr, s, Ls)) return;
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
inline Bounds make_bounds(long long n) {
    Bounds b;
#if MDWF_BOUNDS_CHECK
    b.n = n;
    b.err = bounds_word();
#else
    (void)n;
#endif
    return b;
}
template <> inline Field<MDWF_F64> make_field<MDWF_F64>(void* base, const Geom& g, int nrhs) {
    Field<MDWF_F64> f; f.v = (double2*)base; f.Ls = g.Ls; f.bnd = make_bounds(g.Vh * nrhs); return f;
}
template <> inline Field<MDWF_F32> make_field<MDWF_F32>(void* base, const Geom& g, int nrhs) {
    Field<MDWF_F32> f; f.v = (float4*)base; f.Ls = g.Ls; f.bnd = make_bounds(g.Vh * nrhs); return f;
}
template <> inline Field<MDWF_F16N> make_field<MDWF_F16N>(void* base, const Geom& g, int nrhs) {
    Field<MDWF_F16N> f;
    f.v = (uint2*)base;
    f.norm = (float*)((char*)base + (size_t)g.Vh * g.Ls * nrhs * 48);
    f.Ls = g.Ls;
    f.bnd = make_bounds(g.Vh * nrhs);
    return f;
}

// ------------------------------------------------------------------- gauge

template <int P> struct Gauge;
template <> struct Gauge<MDWF_F64> {
    const double2* u;  // [parity][mu][site][9] complex
    Bounds bnd;        // links: 8 Vh
    __device__ __forceinline__ void load(long long idx, double* o) const {
        if (bnd.bad(idx, 0, 1)) { for (int k = 0; k < 18; ++k) o[k] = 0; return; }
        const double2* p = u + idx * 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) { double2 d = __ldg(p + k); o[2 * k] = d.x; o[2 * k + 1] = d.y; }
    }
};
// FP32 links are padded to 20 floats (five 16-byte loads), FP16 links to 24
// halves (three 16-byte loads); the padding is never read into arithmetic.
template <> struct Gauge<MDWF_F32> {
    const float4* u;
    Bounds bnd;        // links: 8 Vh
    __device__ __forceinline__ void load(long long idx, float* o) const {
        if (bnd.bad(idx, 0, 1)) { for (int k = 0; k < 18; ++k) o[k] = 0; return; }
        const float4* p = u + idx * 5;
        float t[20];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            float4 d = __ldg(p + k);
            t[4 * k] = d.x; t[4 * k + 1] = d.y; t[4 * k + 2] = d.z; t[4 * k + 3] = d.w;
        }
#pragma unroll
        for (int k = 0; k < 18; ++k) o[k] = t[k];
    }
};
// The FP16+norm operator reads the FP32 links: FP16 (11 significant bits)
// links would bound its accuracy below what the inner solve needs.
template <> struct Gauge<MDWF_F16N> : Gauge<MDWF_F32> {};
// link storage bytes per precision (with padding); the F16N operator uses the FP32 copy
inline size_t link_store_bytes(int prec) { return prec == MDWF_F64 ? 144 : 80; }
inline int link_copy(int prec) { return prec == MDWF_F64 ? 0 : 1; }

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

// ------------------------------------------------------- s-operators
//
// Every s-mixing factor of M and M^dag is a function of the fifth-dimension
// shift C restricted to one chirality: on P- it is N' (psi_{s+1}, row Ls-1
// takes -m psi_0), on P+ its transpose N'^T (psi_{s-1}, row 0 takes
// -m psi_{Ls-1}); the adjoint of an operator swaps the two. Reflecting
// s -> Ls-1-s turns N'^T into N', so one routine on a reflected index covers
// both. With M+ = b5 (4 - M5) + 1, M- = c5 (4 - M5) - 1:
//   SOP_C    : C psi
//   SOP_MPHI : M_phi psi = b5 psi + c5 C psi
//   SOP_A    : A psi = (M+ + M- C)^-1 psi by the closed-form elimination of
//              Sec. 3: with r = M-/M+, kappa = m r,
//                Psi_{Ls-1} = [b_{Ls-1} + kappa sum_{s<Ls-1} (-r)^s b_s] / (M+ (1 - kappa (-r)^{Ls-1}))
//                Psi_s      = b_s / M+ - r Psi_{s+1}   (s = Ls-2 .. 0)
//   SOP_K    : K psi = M_phi A psi, fused into the back substitution
//   SOP_MEE  : I psi = M+ psi + M- C psi (the site-diagonal block of Eq. D_5d_matrix)
//   SOP_DENSE: a dense Ls x Ls table (any coefficients)
enum SOp { SOP_DENSE = 0, SOP_ID = 1, SOP_A = 2, SOP_MPHI = 3, SOP_K = 4, SOP_C = 5, SOP_MEE = 6 };

template <typename R> struct SCoef {
    R b5, c5, Mp, Mm;
};

// Complex element types for the column tasks (one 8- or 16-byte access each).
template <typename R> struct CPair;
template <> struct CPair<float> { typedef float2 T; };
template <> struct CPair<double> { typedef double2 T; };

// In place on one complex column: element s at base[k(s) * stride] (re, im as
// one vector), k(s) = up ? s : Ls-1-s. m = this rhs's mass.
template <typename R>
__device__ __forceinline__ void column_op(R* base, int stride, int Ls, int op, bool up, const SCoef<R>& sc, R m) {
    typedef typename CPair<R>::T C;
    auto at = [&](int s) -> C* { return reinterpret_cast<C*>(base + (up ? s : Ls - 1 - s) * stride); };
    if (op == SOP_A || op == SOP_K) {
        const R r = sc.Mm / sc.Mp, kappa = m * r, inv = R(1) / sc.Mp;
        C last = *at(Ls - 1);
        R ar = last.x, ai = last.y, pw = kappa;
        for (int s = 0; s < Ls - 1; ++s) {
            const C q = *at(s);
            ar += pw * q.x;
            ai += pw * q.y;
            pw *= -r;
        }
        const R den = sc.Mp * (R(1) - pw);
        R pr = ar / den, pi = ai / den;  // Psi_{Ls-1}
        const R lr = pr, li = pi;
        if (op == SOP_A) {
            C o; o.x = pr; o.y = pi;
            *at(Ls - 1) = o;
            for (int s = Ls - 2; s >= 0; --s) {
                C* t = at(s);
                const C b = *t;
                pr = b.x * inv - r * pr;
                pi = b.y * inv - r * pi;
                o.x = pr; o.y = pi;
                *t = o;
            }
        } else {
            for (int s = Ls - 2; s >= 0; --s) {
                C* t = at(s);
                const C b = *t;
                const R nr = b.x * inv - r * pr, ni = b.y * inv - r * pi;  // Psi_s
                C o;
                o.x = sc.b5 * nr + sc.c5 * pr;                             // (M_phi Psi)_s
                o.y = sc.b5 * ni + sc.c5 * pi;
                *t = o;
                pr = nr;
                pi = ni;
            }
            C o;  // row Ls-1 wraps to Psi_0 (now in pr, pi) with -m
            o.x = sc.b5 * lr - m * sc.c5 * pr;
            o.y = sc.b5 * li - m * sc.c5 * pi;
            *at(Ls - 1) = o;
        }
    } else if (op == SOP_MPHI || op == SOP_C || op == SOP_MEE) {
        const R w0 = op == SOP_MPHI ? sc.b5 : op == SOP_MEE ? sc.Mp : R(0);
        const R w1 = op == SOP_MPHI ? sc.c5 : op == SOP_MEE ? sc.Mm : R(1);
        const C f0 = *at(0);
        C cur = f0;
        for (int s = 0; s < Ls - 1; ++s) {
            const C nxt = *at(s + 1);
            C o;
            o.x = w0 * cur.x + w1 * nxt.x;
            o.y = w0 * cur.y + w1 * nxt.y;
            *at(s) = o;
            cur = nxt;
        }
        C o;
        o.x = w0 * cur.x - m * w1 * f0.x;
        o.y = w0 * cur.y - m * w1 * f0.y;
        *at(Ls - 1) = o;
    }
}

// The closed-form I^-1 (Sec. 3) on a register-held column of LS complex
// values, element s at v[REV ? LS-1-s : s]: first the last element
// Psi_{Ls-1} from the whole column, returned in (pr, pi) ...
template <int LS, bool REV, typename C, typename R>
__device__ __forceinline__ void a_last(const C* v, R r, R kappa, R Mp, R& pr, R& pi) {
    R ar = v[REV ? 0 : LS - 1].x, ai = v[REV ? 0 : LS - 1].y, pw = kappa;
#pragma unroll
    for (int s = 0; s < LS - 1; ++s) {
        ar += pw * v[REV ? LS - 1 - s : s].x;
        ai += pw * v[REV ? LS - 1 - s : s].y;
        pw *= -r;
    }
    const R den = Mp * (R(1) - pw);
    pr = ar / den;
    pi = ai / den;
}

// ... then, with Psi_{Ls-1} in place, Psi_s = v_s / M+ - (M- / M+) Psi_{s+1}
// from s = Ls-2 down, in place: v becomes I^-1 v.
template <int LS, bool REV, typename C, typename R>
__device__ __forceinline__ void a_solve(C* v, R r, R kappa, R inv, R Mp) {
    R pr, pi;
    a_last<LS, REV>(v, r, kappa, Mp, pr, pi);
    v[REV ? 0 : LS - 1].x = pr;
    v[REV ? 0 : LS - 1].y = pi;
#pragma unroll
    for (int s = LS - 2; s >= 0; --s) {
        C& e = v[REV ? LS - 1 - s : s];
        pr = e.x * inv - r * pr;
        pi = e.y * inv - r * pi;
        e.x = pr;
        e.y = pi;
    }
}

// column_op with the column held in registers (Ls known at compile time): all
// Ls elements are loaded at once, the recursion runs on registers, and all are
// stored back; the arithmetic is that of column_op.
template <int LS, typename R>
__device__ __forceinline__ void column_op_reg(R* base, int stride, int op, bool up, const SCoef<R>& sc, R m) {
    typedef typename CPair<R>::T C;
    C v[LS];
#pragma unroll
    for (int s = 0; s < LS; ++s) v[s] = *reinterpret_cast<const C*>(base + (up ? s : LS - 1 - s) * stride);
    if (op == SOP_A || op == SOP_K) {
        const R r = sc.Mm / sc.Mp, kappa = m * r, inv = R(1) / sc.Mp;
        if (op == SOP_A) {
            a_solve<LS, false>(v, r, kappa, inv, sc.Mp);
        } else {
            R pr, pi;
            a_last<LS, false>(v, r, kappa, sc.Mp, pr, pi);  // Psi_{Ls-1}
            const R lr = pr, li = pi;
#pragma unroll
            for (int s = LS - 2; s >= 0; --s) {
                const R nr = v[s].x * inv - r * pr, ni = v[s].y * inv - r * pi;  // Psi_s
                v[s].x = sc.b5 * nr + sc.c5 * pr;                               // (M_phi Psi)_s
                v[s].y = sc.b5 * ni + sc.c5 * pi;
                pr = nr;
                pi = ni;
            }
            v[LS - 1].x = sc.b5 * lr - m * sc.c5 * pr;
            v[LS - 1].y = sc.b5 * li - m * sc.c5 * pi;
        }
    } else if (op == SOP_MPHI || op == SOP_C || op == SOP_MEE) {
        const R w0 = op == SOP_MPHI ? sc.b5 : op == SOP_MEE ? sc.Mp : R(0);
        const R w1 = op == SOP_MPHI ? sc.c5 : op == SOP_MEE ? sc.Mm : R(1);
        const C f0 = v[0];
#pragma unroll
        for (int s = 0; s < LS - 1; ++s) {
            v[s].x = w0 * v[s].x + w1 * v[s + 1].x;
            v[s].y = w0 * v[s].y + w1 * v[s + 1].y;
        }
        v[LS - 1].x = w0 * v[LS - 1].x - m * w1 * f0.x;
        v[LS - 1].y = w0 * v[LS - 1].y - m * w1 * f0.y;
    } else {
        return;
    }
#pragma unroll
    for (int s = 0; s < LS; ++s) *reinterpret_cast<C*>(base + (up ? s : LS - 1 - s) * stride) = v[s];
}

template <typename R>
__device__ __forceinline__ void column_op_any(R* base, int stride, int Ls, int op, bool up, const SCoef<R>& sc, R m) {
    switch (Ls) {
        case 8: column_op_reg<8>(base, stride, op, up, sc, m); return;
        case 12: column_op_reg<12>(base, stride, op, up, sc, m); return;
        case 16: column_op_reg<16>(base, stride, op, up, sc, m); return;
        default: column_op(base, stride, Ls, op, up, sc, m); return;
    }
}

// 24 reals of one (site, s) row in shared memory, as 16-byte vector accesses.
__device__ __forceinline__ void row_store(float* row, const float* v) {
#pragma unroll
    for (int k = 0; k < 6; ++k)
        reinterpret_cast<float4*>(row)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}
__device__ __forceinline__ void row_load(const float* row, float* v) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float4 q = reinterpret_cast<const float4*>(row)[k];
        v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
}
__device__ __forceinline__ void row_store(double* row, const double* v) {
#pragma unroll
    for (int k = 0; k < 12; ++k) reinterpret_cast<double2*>(row)[k] = make_double2(v[2 * k], v[2 * k + 1]);
}
__device__ __forceinline__ void row_load(const double* row, double* v) {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 q = reinterpret_cast<const double2*>(row)[k];
        v[2 * k] = q.x; v[2 * k + 1] = q.y;
    }
}

// Shared-memory staging of a block's columns: spinor (site ly, slice s) at
// hs + ly * site_stride + s * kRowStride. The row stride of 28 words keeps the
// 16-byte row accesses of 8 consecutive threads on distinct banks. The column
// tasks of a warp all belong to one chirality (6 complex components per
// site, consecutive sites), so a site stride = 12 (mod 32) words puts the
// 8-byte accesses of every half-warp on distinct banks.
constexpr int kRowStride = 28;
__host__ __device__ inline int site_stride(int Ls) {
    const int base = Ls * kRowStride;
    return base + ((12 - base % 32) + 32) % 32;
}

// Applies the s-operator to the SB staged columns of a block. Tasks are
// (chirality, site, component): the P+ components (spins 0, 1) fill the first
// half of the task slots and the P- components the second, each half rounded
// up to whole warps so that a warp walks all its columns in one direction.
// Dense tables are applied by the caller instead.
// LSR > 0: the columns are held in registers with Ls = LSR fixed at compile
// time (the caller guarantees Ls == LSR); LSR = -1: held in registers for
// Ls = 8, 12, 16 (chosen at run time) when in_registers, else streamed
// through shared memory.
template <int LSR = -1, typename R>
__device__ __forceinline__ void block_columns(R* hs, int SB, int Ls, int op, bool swap, const SCoef<R>& sc,
                                              R m, int tid, int nthr, bool in_registers = true) {
    const int ss = site_stride(Ls);
    const int per = SB * 6, half = (per + 31) / 32 * 32;
    for (int t = tid; t < 2 * half; t += nthr) {
        const int chir = t >= half ? 1 : 0, r = t - chir * half;
        if (r >= per) continue;
        const int ly = r / 6, j = chir * 6 + (r - 6 * (r / 6));
        const bool up = (chir == 1) != swap;  // P- uses N' unless the adjoint swaps
        if constexpr (LSR > 0) column_op_reg<LSR>(hs + (size_t)ly * ss + 2 * j, kRowStride, op, up, sc, m);
        else if (in_registers) column_op_any(hs + (size_t)ly * ss + 2 * j, kRowStride, Ls, op, up, sc, m);
        else column_op(hs + (size_t)ly * ss + 2 * j, kRowStride, Ls, op, up, sc, m);
    }
}

// The column pass of the fused t, v epilogue (closed form, Ls = LS): with y
// staged in the rows, each column becomes t = A y, its share of |t|^2 goes
// to the returned sum, and then v = A^dag t, which for one chirality is the
// same recursion run from the other end of the column; v replaces y in the
// rows. Tasks as in block_columns.
template <int LS, typename R>
__device__ __forceinline__ R column_a_adag_reg(R* base, int stride, bool up, const SCoef<R>& sc, R m) {
    typedef typename CPair<R>::T C;
    C v[LS];
#pragma unroll
    for (int s = 0; s < LS; ++s) v[s] = *reinterpret_cast<const C*>(base + (up ? s : LS - 1 - s) * stride);
    const R r = sc.Mm / sc.Mp, kappa = m * r, inv = R(1) / sc.Mp;
    a_solve<LS, false>(v, r, kappa, inv, sc.Mp);
    R sq = 0;
#pragma unroll
    for (int s = 0; s < LS; ++s) {
        sq = fma(v[s].x, v[s].x, sq);
        sq = fma(v[s].y, v[s].y, sq);
    }
    a_solve<LS, true>(v, r, kappa, inv, sc.Mp);
#pragma unroll
    for (int s = 0; s < LS; ++s) *reinterpret_cast<C*>(base + (up ? s : LS - 1 - s) * stride) = v[s];
    return sq;
}

template <int LS, typename R>
__device__ __forceinline__ R block_columns_a_adag(R* hs, int SB, const SCoef<R>& sc, R m, int tid, int nthr) {
    const int ss = site_stride(LS);
    const int per = SB * 6, half = (per + 31) / 32 * 32;
    R sq = 0;
    for (int t = tid; t < 2 * half; t += nthr) {
        const int chir = t >= half ? 1 : 0, r = t - chir * half;
        if (r >= per) continue;
        const int ly = r / 6, j = chir * 6 + (r - 6 * (r / 6));
        sq += column_a_adag_reg<LS>(hs + (size_t)ly * ss + 2 * j, kRowStride, chir == 1, sc, m);
    }
    return sq;
}

// ------------------------------------------------------------------ tables
//
// Dense Ls x Ls real matrices of the s-operators, one per chirality:
// table[t][rhs][chir][s'][s] holds element (s, s') (transposed, so that the
// Ls threads of a column read consecutive words); chir 0 is the P+ half
// (spins 0, 1), chir 1 the P- half; t = table_index(sop, swap).
constexpr int kNumTables = 12;
inline int table_index(int sop, int swap) { return (sop - 1) * 2 + (swap ? 1 : 0); }

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
inline double link_bytes(int prec) { return prec == MDWF_F64 ? 144.0 : 72.0; }

}  // namespace mdwf

struct mdwf_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    mdwf::Geom g{};
    double M5 = 0, b5 = 0, c5 = 0, mf = 0;
    bool have_gauge = false;
    void* gauge[2] = {nullptr, nullptr};  // FP64 and FP32 copies
    // Ls x Ls tables for the current mass list, FP64 and FP32, plus per-rhs masses
    double* tab64 = nullptr;
    float* tab32 = nullptr;
    double* mass64 = nullptr;
    float* mass32 = nullptr;
    int tab_nrhs = 0;
    double* tab_host = nullptr;     // pinned staging for the tables
    double tab_masses[64] = {0};
    bool tab_valid = false;
    // neighbour table [parity][site][8]: cb index of x+mu (0..3) and x-mu (4..7)
    int* nbr = nullptr;
    // 1: apply every s-operator as a dense table (any coefficients); 0: the
    // closed-form recursions where they are stable (|M-/M+| <= 0.9)
    bool dense_s = false;
    bool dense_s_base = false;  // the choice for constant coefficients
    // per-slice coefficients b5(s), c5(s) (Sec. 2.1, Sec. 4.3); when set, every s-operator
    // is a dense table and the gather of the hop takes per-slice factors from
    // gs64 / gs32 = [gown(s)][gfac(s)][gscale(s)], 64 entries each
    bool sdep = false;
    // chemical potential on the time links (0: none)
    double chem = 0.0;
    double b5s[64] = {0}, c5s[64] = {0};
    double* gs64 = nullptr;
    float* gs32 = nullptr;
    // scratch fields used inside one apply: [0] even-parity z, [1] odd-parity v
    mdwf::Workspace tmp[2];
    // solver workspace (CG fields) and the fields of the entry points around it
    mdwf::Workspace solver;
    mdwf::Workspace io;
    mdwf::Workspace tune;  // scratch fields of the autotuner
    mdwf::Workspace aux;   // even/odd halves of the full operator
    mdwf::Workspace ov;    // full 5d fields of the Pauli-Villars constructions
    mdwf::Workspace gw;    // 4d fields of the chiral-violation operator
    mdwf::Workspace h4;    // fields of the 4d-HMC force
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
    // autotuned 4d sites per hop block, [precision][nrhs] (0 = default)
    int sb_tune[3][65] = {};
    // load strategy of the FP32 / FP16 hops, [precision]: 0 default (register
    // prefetch), 1 cp.async per thread, 2 bulk copies of whole neighbour columns
    // (TMA), 3 register prefetch (as 0), 4 plain loads
    int hop_stage[3] = {0, 0, 0};
    // device word set by a bounded device-side wait that gave up (0 = none)
    int* dev_err = nullptr;
    bool autotune = false;
    // a t-slab of a lattice split along t (domain decomposition): the t-neighbours
    // across its two faces are remote and come in as halos (mdwf_slab_stage)
    bool slab = false;
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
void set_error_message(const char* msg);
int cuda_status(cudaError_t e);
int check_launch();
// MDWF_ETIMEOUT if a bounded device-side wait gave up since the last call (synchronises)
int device_wait_status(mdwf_ctx* c);
int ensure_workspace(Workspace& w, size_t bytes);
// NaN-canary mode (MDWF_CANARY=1): fill a fresh allocation with 0xFF bytes
bool canary_on();
int canary_fill(void* p, size_t bytes);
int ensure_tables(mdwf_ctx* c, int nrhs, const double* mf_per_rhs);

// table pointers for table t, precision
inline const void* table_ptr(const mdwf_ctx* c, int prec, int t) {
    size_t per_op = (size_t)c->tab_nrhs * 2 * c->g.Ls * c->g.Ls;
    if (prec == MDWF_F64) return c->tab64 + t * per_op;
    return c->tab32 + t * per_op;
}

// Selects the s-operator of a launch: the closed-form recursion, or the dense
// table when the context asks for dense tables (or the recursion is not stable).
template <class L> inline void set_sop(const mdwf_ctx* c, int prec, int sop, int swap, L& l) {
    if (c->dense_s) {
        l.sop = SOP_DENSE;
        l.swap = 0;
        l.mat = table_ptr(c, prec, table_index(sop, swap));
    } else {
        l.sop = sop;
        l.swap = swap;
        l.mat = nullptr;
    }
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
    const void* mat;      // dense table of the output Ls x Ls matrix (sop == SOP_DENSE), per rhs
    const void* mat2;     // dense table of A^dag for the FUSE_T epilogue (sop == SOP_DENSE)
    int sop;              // output s-operator (SOp)
    int swap;             // 1: the adjoint (chirality-swapped) s-operator
    const void* mass;     // per-rhs masses (double for F64, float otherwise)
    double b5, c5;
    int nrhs;
    const double* mask;   // per-rhs flags, or null: the blocks of a right-hand side whose flag is 0 do nothing
    // fused CG epilogues (0: none; 1: also v = A^dag out into out2 and |out|^2
    // partials; 2: r -= alpha out into rfield with |r|^2 partials, out not stored)
    int fuse;
    void* out2;
    void* rfield;         // FP64 field for FP64 operators, FP32 otherwise
    // fused CG iteration without the t field (Ls = 16, structured s-operators):
    // FUSE_T stores only v = A^dag t, not t; FUSE_R takes its xpay addend t as
    // I^dag v, formed from v (its x) by shuffles across the 16 slices
    int no_t;
    // t-slab contexts: the received faces [dir][rhs][face site][half spinor][s]
    // (HopParams::halo); null on ordinary contexts
    const void* halo;
    double* part;         // [rhs][hop_blocks] partial sums
    const double* sc;     // CG scalars
};
int launch_hop(mdwf_ctx* c, int prec, const HopLaunch& h);
// whether the fused CG iteration can run without its t field (HopLaunch::no_t)
bool hop_no_t_ok(const mdwf_ctx* c, int prec, int nrhs);
int hop_sites_per_block(const mdwf_ctx* c, int prec, int nrhs);
int hop_blocks(const mdwf_ctx* c, int prec, int nrhs);

struct M5Launch {
    void* out;
    const void* in;
    const void* x;    // optional addend
    double coef;      // out = coef * Mat in [+ x]
    const void* mat;  // dense table (sop == SOP_DENSE)
    int sop;
    int swap;
    int nrhs;
    const void* mass; // per-rhs masses in this precision; nullptr = the context's
    const double* mask;  // per-rhs flags, or null (as HopLaunch::mask)
};
int launch_m5(mdwf_ctx* c, int prec, const M5Launch& m);

// Points the per-rhs table and mass pointers of a launch (set by set_sop) at
// right-hand side rhs0 of the context's current batch, for launches on a
// slice of nrhs right-hand sides starting at rhs0.
template <class L> inline void offset_rhs(const mdwf_ctx* c, int prec, int rhs0, L& l) {
    if (rhs0 == 0) return;
    const size_t es = prec == MDWF_F64 ? sizeof(double) : sizeof(float);
    if (l.mat) l.mat = (const char*)l.mat + (size_t)rhs0 * 2 * c->g.Ls * c->g.Ls * es;
    const void* m = l.mass ? l.mass : (prec == MDWF_F64 ? (const void*)c->mass64 : (const void*)c->mass32);
    l.mass = (const char*)m + (size_t)rhs0 * es;
}

// full-field operators and the force's outer products (overlap.cu, force.cu)
int apply_full_dev(mdwf_ctx* c, double* out, const double* in, int nrhs, int dagger);
int launch_embed_wall(mdwf_ctx* c, double* out5, const double* in4, int nrhs);
int launch_force(mdwf_ctx* c, double* dSdU, const void* A_odd, const void* B_even, const void* C_even,
                 const void* D_odd, double coef);

// operator chains (api.cu); rhs0: the fields are right-hand sides rhs0 ..
// rhs0 + nrhs - 1 of the batch the tables were built for
int apply_op(mdwf_ctx* c, void* out, const void* in, int prec, int nrhs, int dagger, int rhs0 = 0,
             const double* mask = nullptr);
int tune_hop(mdwf_ctx* c, int prec, int nrhs, int* chosen);

// solver (cg.cu)
struct NormalResult {
    std::vector<int> status, iters, rupd, restarts;
    std::vector<double> rel;  // |src - M^dag M x| / |src| in FP64
};
int solve_normal(mdwf_ctx* c, int nrhs, void* xo, const void* src, const mdwf_solve_params& prm, NormalResult& res);
// Re <a, b> of FP64 internal fields per right-hand side into host memory (synchronises)
int field_dot64(mdwf_ctx* c, const void* a, const void* b, int nrhs, double* out_host);
// out_host[s] = Re <a, b> restricted to slice s (one FP64 field); synchronises
int slice_dot64(mdwf_ctx* c, const void* a, const void* b, double* out_host);

// layout kernels (layout.cu)
int launch_import_odd(mdwf_ctx* c, void* dst, const double* src_dev, int prec, int nrhs);
int launch_export_odd(mdwf_ctx* c, double* dst_dev, const void* src, int prec, int nrhs);
int launch_split_full(mdwf_ctx* c, void* dst_even, void* dst_odd, const double* full_dev, int prec, int nrhs);
int launch_join_full(mdwf_ctx* c, double* full_dev, const void* even, const void* odd, int prec, int nrhs);
int launch_gauge_pack(mdwf_ctx* c, const double* U_dev);
int launch_build_neighbours(mdwf_ctx* c);

}  // namespace mdwf
