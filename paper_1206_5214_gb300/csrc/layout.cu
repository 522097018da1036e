// Conversions between the user formats (complex128, lexicographic) and the
// internal per-parity, s-innermost layouts of every precision.
#include "mdwf_internal.cuh"

namespace mdwf {

template <int P>
__global__ void import_odd_kernel(Field<P> dst, const double* __restrict__ src, Geom g, int nrhs) {
    typedef typename PrecTraits<P>::real R;
    const long long n = (long long)nrhs * g.Vh * g.Ls;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i % g.Ls);
        const long long sr = i / g.Ls;  // rhs * Vh + site
        const long long rhs = sr / g.Vh, site = sr % g.Vh;
        const double* p = src + ((rhs * g.Ls + s) * g.Vh + site) * 24;
        R v[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) v[k] = (R)p[k];
        dst.store(sr, s, v);
    }
}

template <int P>
__global__ void export_odd_kernel(double* __restrict__ dst, Field<P> src, Geom g, int nrhs) {
    typedef typename PrecTraits<P>::real R;
    const long long n = (long long)nrhs * g.Vh * g.Ls;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i % g.Ls);
        const long long sr = i / g.Ls;
        const long long rhs = sr / g.Vh, site = sr % g.Vh;
        R v[24];
        src.load(sr, s, v);
        double* p = dst + ((rhs * g.Ls + s) * g.Vh + site) * 24;
#pragma unroll
        for (int k = 0; k < 24; ++k) p[k] = (double)v[k];
    }
}

// full user field [rhs][s][V][24] <-> internal even / odd fields
template <int P, bool TO_INTERNAL>
__global__ void full_kernel(Field<P> even, Field<P> odd, double* full, Geom g, int nrhs) {
    typedef typename PrecTraits<P>::real R;
    const long long V = 2 * g.Vh;
    const long long n = (long long)nrhs * V * g.Ls;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i % g.Ls);
        const long long r = i / g.Ls;
        const long long rhs = r / V, lex = r % V;
        long long q = lex;
        const int x = (int)(q % g.X); q /= g.X;
        const int y = (int)(q % g.Y); q /= g.Y;
        const int z = (int)(q % g.Z); q /= g.Z;
        const int t = (int)q;
        const int par = (x + y + z + t) & 1;
        const long long sr = rhs * g.Vh + (lex >> 1);
        double* p = full + ((rhs * g.Ls + s) * V + lex) * 24;
        R v[24];
        if (TO_INTERNAL) {
#pragma unroll
            for (int k = 0; k < 24; ++k) v[k] = (R)p[k];
            if (par) odd.store(sr, s, v);
            else even.store(sr, s, v);
        } else {
            if (par) odd.load(sr, s, v);
            else even.load(sr, s, v);
#pragma unroll
            for (int k = 0; k < 24; ++k) p[k] = (double)v[k];
        }
    }
}

__global__ void gauge_pack_kernel(double2* u64, float* u32, const double2* __restrict__ U, Geom g) {
    const long long V = 2 * g.Vh;
    const long long n = V * 4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int mu = (int)(i % 4);
        const long long lex = i / 4;
        long long q = lex;
        const int x = (int)(q % g.X); q /= g.X;
        const int y = (int)(q % g.Y); q /= g.Y;
        const int z = (int)(q % g.Z); q /= g.Z;
        const int t = (int)q;
        const int par = (x + y + z + t) & 1;
        const long long l = ((long long)par * 4 + mu) * g.Vh + (lex >> 1);
        const double2* src = U + i * 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 d = src[k];
            u64[l * 9 + k] = d;
            u32[l * 20 + 2 * k] = (float)d.x;
            u32[l * 20 + 2 * k + 1] = (float)d.y;
        }
        u32[l * 20 + 18] = 0.f;
        u32[l * 20 + 19] = 0.f;
    }
}

// On a t-slab (slab != 0) the t-neighbours across the two faces are marked
// -1 - f, f the site's index within its t-slice (the index of the same
// (x, y, z) in the neighbouring slab's face), so the hops read them from halos.
__global__ void neighbour_kernel(int* nbr, Geom g, int slab) {
    const long long n = 2 * g.Vh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int par = (int)(i / g.Vh);
        const long long j = i % g.Vh;
        int c[4];
        cb_coords(g, j, par, c);
        const int L[4] = {g.X, g.Y, g.Z, g.T};
        int* o = nbr + i * 8;
        for (int mu = 0; mu < 4; ++mu) {
            int f[4] = {c[0], c[1], c[2], c[3]}, b[4] = {c[0], c[1], c[2], c[3]};
            f[mu] = c[mu] + 1 == L[mu] ? 0 : c[mu] + 1;
            b[mu] = c[mu] == 0 ? L[mu] - 1 : c[mu] - 1;
            o[mu] = (int)cb_index(g, f[0], f[1], f[2], f[3]);
            o[4 + mu] = (int)cb_index(g, b[0], b[1], b[2], b[3]);
        }
        if (slab) {
            const long long face = (long long)g.X * g.Y * g.Z / 2;
            if (c[3] == g.T - 1) o[3] = -1 - (int)(j % face);
            if (c[3] == 0) o[7] = -1 - (int)(j % face);
        }
    }
}

static dim3 grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 152LL * 64) b = 152LL * 64;
    if (b < 1) b = 1;
    return dim3((unsigned)b);
}

template <int P>
static int import_t(mdwf_ctx* c, void* dst, const double* src, int nrhs) {
    const long long n = (long long)nrhs * c->g.Vh * c->g.Ls;
    LaunchScope scope(c, KB_LAYOUT * 3 + P, n * (192.0 + site_bytes(P)), 0.0);
    import_odd_kernel<P><<<grid_for(n, 256), 256, 0, c->stream>>>(make_field<P>(dst, c->g, nrhs), src, c->g, nrhs);
    return check_launch();
}

template <int P>
static int export_t(mdwf_ctx* c, double* dst, const void* src, int nrhs) {
    const long long n = (long long)nrhs * c->g.Vh * c->g.Ls;
    LaunchScope scope(c, KB_LAYOUT * 3 + P, n * (192.0 + site_bytes(P)), 0.0);
    export_odd_kernel<P><<<grid_for(n, 256), 256, 0, c->stream>>>(dst, make_field<P>(const_cast<void*>(src), c->g, nrhs),
                                                                   c->g, nrhs);
    return check_launch();
}

template <int P, bool TO>
static int full_t(mdwf_ctx* c, void* even, void* odd, double* full, int nrhs) {
    const long long n = (long long)nrhs * 2 * c->g.Vh * c->g.Ls;
    LaunchScope scope(c, KB_LAYOUT * 3 + P, n * (192.0 + site_bytes(P)), 0.0);
    full_kernel<P, TO><<<grid_for(n, 256), 256, 0, c->stream>>>(make_field<P>(even, c->g, nrhs),
                                                                  make_field<P>(odd, c->g, nrhs), full, c->g, nrhs);
    return check_launch();
}

int launch_import_odd(mdwf_ctx* c, void* dst, const double* src, int prec, int nrhs) {
    switch (prec) {
        case MDWF_F64: return import_t<MDWF_F64>(c, dst, src, nrhs);
        case MDWF_F32: return import_t<MDWF_F32>(c, dst, src, nrhs);
        case MDWF_F16N: return import_t<MDWF_F16N>(c, dst, src, nrhs);
    }
    return MDWF_EINVAL;
}

int launch_export_odd(mdwf_ctx* c, double* dst, const void* src, int prec, int nrhs) {
    switch (prec) {
        case MDWF_F64: return export_t<MDWF_F64>(c, dst, src, nrhs);
        case MDWF_F32: return export_t<MDWF_F32>(c, dst, src, nrhs);
        case MDWF_F16N: return export_t<MDWF_F16N>(c, dst, src, nrhs);
    }
    return MDWF_EINVAL;
}

int launch_split_full(mdwf_ctx* c, void* dst_even, void* dst_odd, const double* full, int prec, int nrhs) {
    double* f = const_cast<double*>(full);
    switch (prec) {
        case MDWF_F64: return full_t<MDWF_F64, true>(c, dst_even, dst_odd, f, nrhs);
        case MDWF_F32: return full_t<MDWF_F32, true>(c, dst_even, dst_odd, f, nrhs);
        case MDWF_F16N: return full_t<MDWF_F16N, true>(c, dst_even, dst_odd, f, nrhs);
    }
    return MDWF_EINVAL;
}

int launch_join_full(mdwf_ctx* c, double* full, const void* even, const void* odd, int prec, int nrhs) {
    void* e = const_cast<void*>(even);
    void* o = const_cast<void*>(odd);
    switch (prec) {
        case MDWF_F64: return full_t<MDWF_F64, false>(c, e, o, full, nrhs);
        case MDWF_F32: return full_t<MDWF_F32, false>(c, e, o, full, nrhs);
        case MDWF_F16N: return full_t<MDWF_F16N, false>(c, e, o, full, nrhs);
    }
    return MDWF_EINVAL;
}

int launch_gauge_pack(mdwf_ctx* c, const double* U) {
    const long long n = 2 * c->g.Vh * 4;
    LaunchScope scope(c, KB_LAYOUT * 3 + MDWF_F64, n * (144.0 * 2 + 80.0), 0.0);
    gauge_pack_kernel<<<grid_for(n, 256), 256, 0, c->stream>>>((double2*)c->gauge[0], (float*)c->gauge[1],
                                                                (const double2*)U, c->g);
    return check_launch();
}

}  // namespace mdwf

namespace mdwf {
int launch_build_neighbours(mdwf_ctx* c) {
    const long long n = 2 * c->g.Vh;
    LaunchScope scope(c, KB_LAYOUT * 3 + MDWF_F64, n * 32.0, 0.0);
    neighbour_kernel<<<grid_for(n, 256), 256, 0, c->stream>>>(c->nbr, c->g, c->slab ? 1 : 0);
    return check_launch();
}
}  // namespace mdwf
