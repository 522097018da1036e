/*
 * mdwf_oracle.c -- plain FP64 CPU oracle for the 4d red/black-preconditioned
 * Moebius domain-wall operator of Brower, Neff and Orginos, "The Moebius
 * Domain Wall Fermion Algorithm" (arXiv:1206.5214).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct
 * statement of what the GPU path computes. Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg load it; the library's product path
 * never calls it and shares no code, header, table or helper with it.
 *
 * Every function follows the paper's own form, not the factored form the GPU
 * kernels use:
 *   - Wilson operator, Eq. (D^Wilson) of Sec. 2 (repeated as Eq. Waction in
 *     App. A): (4 + M5_f) delta - 1/2 sum_mu [(1 - g_mu) U_mu(x) delta_{x+mu,y}
 *     + (1 + g_mu) U_mu(y)^dag delta_{x,y+mu}], with M5_f = -M5 (the numerical
 *     sections quote the wall height M5 = +1.8, so the diagonal is 4 - M5).
 *   - 5d operator, Eq. (MoebiusOp) / Eq. (DWmatrix): block tridiagonal in s with
 *     D+ = b5 D_W + 1 on the diagonal, D- P- above, D- P+ below and
 *     -m D- P+ (row 1, column Ls), -m D- P- (row Ls, column 1) in the corners.
 *   - red/black blocks, Sec. 3: colour x1+x2+x3+x4 even/odd for every s; the
 *     site-diagonal blocks I_rr = I_bb carry M+ = b5(4 - M5) + 1 and
 *     M- = c5(4 - M5) - 1 (Eq. D_5d_matrix, both corners taken as -m M-, the
 *     reading that follows from Eq. MoebiusOp); the off-diagonal blocks keep
 *     the hopping part of every D_W in the tridiagonal.
 *   - I_rr^-1 by the closed-form forward elimination and back substitution of
 *     Sec. 3 on the P- half, the row/column-interchanged recursion on P+.
 *   - Schur complement D_pre = 1 - I_bb^-1 D_br I_rr^-1 D_rb (Sec. 3), solved
 *     on the odd (black) sites by conjugate gradient on D_pre^dag D_pre.
 *
 * Conventions: lattice L = {X, Y, Z, T}, lexicographic site index
 * ((t*Z + z)*Y + y)*X + x; a half (one-parity) field stores the sites of that
 * parity in lexicographic order, so site i sits at half-index i/2 (X even).
 * Fields are [s][site][spin 4][colour 3] complex double, gauge links are
 * [site][mu 4][3][3]. Hermitian Euclidean chiral gamma basis:
 * g_mu = [[0, A_mu], [A_mu^dag, 0]] with A_k = -i sigma_k, A_4 = 1, so that
 * g5 = g1 g2 g3 g4 = diag(1, 1, -1, -1) and P+- = (1 +- g5)/2.
 * Boundary conditions are periodic in all four directions.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int L[4];     /* X, Y, Z, T; every extent even */
    int Ls;       /* fifth-dimension extent */
    double M5;    /* domain-wall height (positive); Wilson diagonal is 4 - M5 */
    double b5;
    double c5;
    double mf;    /* quark mass m of the walls */
    const double *b5s;  /* b5(s), s = 0..Ls-1, or NULL for the constant b5 */
    const double *c5s;  /* c5(s), or NULL for the constant c5 */
    double mu;          /* chemical potential on the time links (Sec. 6.6); 0 for none */
} or_params;

static double b5_of(const or_params *p, int s) { return p->b5s ? p->b5s[s] : p->b5; }
static double c5_of(const or_params *p, int s) { return p->c5s ? p->c5s[s] : p->c5; }

/* ------------------------------------------------------------------ gammas */

static cplx G[4][4][4];   /* g_mu, mu = 0..3 for directions x, y, z, t */
static cplx G5[4][4];
static cplx PP[4][4];     /* P+ = (1 + g5)/2 */
static cplx PM[4][4];     /* P- = (1 - g5)/2 */
static int gammas_ready = 0;

static void matmul4(cplx out[4][4], cplx a[4][4], cplx b[4][4])
{
    cplx t[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += a[i][k] * b[k][j];
            t[i][j] = s;
        }
    memcpy(out, t, sizeof(t));
}

static void init_gammas(void)
{
    if (gammas_ready) return;
    /* Pauli matrices */
    cplx sig[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    cplx A[4][2][2];
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) A[k][i][j] = -I * sig[k][i][j];
    A[3][0][0] = 1; A[3][0][1] = 0; A[3][1][0] = 0; A[3][1][1] = 1;
    memset(G, 0, sizeof(G));
    for (int mu = 0; mu < 4; ++mu)
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                G[mu][i][2 + j] = A[mu][i][j];          /* upper-right block A   */
                G[mu][2 + i][j] = conj(A[mu][j][i]);    /* lower-left block A^dag */
            }
    cplx t[4][4];
    matmul4(t, G[0], G[1]);
    matmul4(t, t, G[2]);
    matmul4(G5, t, G[3]);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx id = (i == j) ? 1.0 : 0.0;
            PP[i][j] = 0.5 * (id + G5[i][j]);
            PM[i][j] = 0.5 * (id - G5[i][j]);
        }
    gammas_ready = 1;
}

/* Copies g_1..g_4 and g5 out (5 x 4 x 4 complex) for the basis tests. */
void or_gammas(cplx *out)
{
    init_gammas();
    memcpy(out, G, sizeof(G));
    memcpy(out + 64, G5, sizeof(G5));
}

/* ------------------------------------------------------------------ lattice */

static long vol4(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords(const int L[4], long i, int x[4])
{
    for (int mu = 0; mu < 4; ++mu) { x[mu] = (int)(i % L[mu]); i /= L[mu]; }
}

static long lex(const int L[4], const int x[4])
{
    return ((long)(x[3] * L[2] + x[2]) * L[1] + x[1]) * L[0] + x[0];
}

static int parity_of(const int x[4]) { return (x[0] + x[1] + x[2] + x[3]) & 1; }

/* site x + dir * mu with periodic wrap */
static long shift(const int L[4], long i, int mu, int dir)
{
    int x[4];
    coords(L, i, x);
    x[mu] = (x[mu] + dir + L[mu]) % L[mu];
    return lex(L, x);
}

/* lexicographic index of half-index j on parity p */
static long half_to_lex(const int L[4], long j, int p)
{
    long i0 = 2 * j;            /* x of i0 is even because X is even */
    int x[4];
    coords(L, i0, x);
    x[0] += (p + x[1] + x[2] + x[3]) & 1;
    return lex(L, x);
}

/* ------------------------------------------------------- spin-colour algebra */

/* out[a][i] += coef * sum_b S[a][b] * (V' in)[b][i], V' = V or V^dag */
static void acc_spin_colour(cplx out[12], cplx coef, cplx S[4][4],
                            const cplx *V, int adj, const cplx *in)
{
    cplx t[4][3];
    for (int b = 0; b < 4; ++b)
        for (int i = 0; i < 3; ++i) {
            cplx s = 0;
            for (int j = 0; j < 3; ++j)
                s += (adj ? conj(V[3 * j + i]) : V[3 * i + j]) * in[3 * b + j];
            t[b][i] = s;
        }
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) {
            cplx s = 0;
            for (int b = 0; b < 4; ++b) s += S[a][b] * t[b][i];
            out[3 * a + i] += coef * s;
        }
}

/* out = S in for a 4-spinor of 3 colours */
static void spin_mat(cplx out[12], cplx S[4][4], const cplx *in)
{
    cplx t[12];
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) {
            cplx s = 0;
            for (int b = 0; b < 4; ++b) s += S[a][b] * in[3 * b + i];
            t[3 * a + i] = s;
        }
    memcpy(out, t, sizeof(t));
}

/* 1 + sgn * g_mu */
static void one_pm_gamma(cplx out[4][4], int mu, double sgn)
{
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) out[a][b] = (a == b ? 1.0 : 0.0) + sgn * G[mu][a][b];
}

/*
 * Hopping sum H at one output site (lexicographic index i):
 *   H f(x) = sum_mu [ (1 - g_mu) U_mu(x) f(x+mu) + (1 + g_mu) U_mu(x-mu)^dag f(x-mu) ]
 * and, for dagger != 0, the adjoint hopping term of D_W^dag, which takes the
 * adjoint of each term of Eq. (D^Wilson): the forward neighbour carries
 * (1 + g_mu) U_mu(x), the backward one (1 - g_mu) U_mu(x-mu)^dag.
 * D_W = (4 - M5) - H/2. The input field f is a full field (half == 0) or
 * the half field of the parity opposite to x (half == 1).
 */
/*
 * The hopping sum at site i with a chemical potential chem on the time links
 * ((1 -+ g_4) U_4 -> e^{+-chem} (1 -+ g_4) U_4 for the forward / backward
 * hop, Sec. 6.6). The adjoint (dagger) has the projectors flipped and, the
 * matrix being transposed, the factor of each direction exchanged.
 */
static void hop_site(cplx out[12], const cplx *f, int half, const cplx *U,
                     const int L[4], long i, int dagger, double chem)
{
    for (int k = 0; k < 12; ++k) out[k] = 0;
    double sf = dagger ? +1.0 : -1.0;
    for (int mu = 0; mu < 4; ++mu) {
        long fw = shift(L, i, mu, +1), bw = shift(L, i, mu, -1);
        cplx Sf[4][4], Sb[4][4];
        one_pm_gamma(Sf, mu, sf);
        one_pm_gamma(Sb, mu, -sf);
        const cplx *ff = f + 12 * (half ? fw / 2 : fw);
        const cplx *fb = f + 12 * (half ? bw / 2 : bw);
        double wf = 1.0, wb = 1.0;
        if (mu == 3 && chem != 0.0) {
            wf = exp(dagger ? -chem : chem);
            wb = exp(dagger ? chem : -chem);
        }
        acc_spin_colour(out, wf, Sf, U + 9 * (4 * i + mu), 0, ff);
        acc_spin_colour(out, wb, Sb, U + 9 * (4 * bw + mu), 1, fb);
    }
}

/* ------------------------------------------------------------- Wilson D_W */

/* out = D_W in (dagger: D_W^dag) on full 4d fields. Eq. (D^Wilson). */
void or_dw(cplx *out, const cplx *in, const cplx *U, const int L[4], double M5, double chem, int dagger)
{
    init_gammas();
    long V = vol4(L);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; ++i) {
        cplx h[12];
        hop_site(h, in, 0, U, L, i, dagger, chem);
        for (int k = 0; k < 12; ++k) out[12 * i + k] = (4.0 - M5) * in[12 * i + k] - 0.5 * h[k];
    }
}

/* ------------------------------------------------ 5d operator (full lattice) */

/* out = c_w D_W in + c_1 in on a full 4d field (D+ : c_w = b5, c_1 = +1; D- : c5, -1) */
static void dw_affine(cplx *out, const cplx *in, const cplx *U, const int L[4], double M5, double chem,
                      int dagger, double c_w, double c_1)
{
    long V = vol4(L);
    or_dw(out, in, U, L, M5, chem, dagger);
    for (long k = 0; k < 12 * V; ++k) out[k] = c_w * out[k] + c_1 * in[k];
}

static void proj_field(cplx *out, cplx S[4][4], const cplx *in, long nsites)
{
    for (long i = 0; i < nsites; ++i) spin_mat(out + 12 * i, S, in + 12 * i);
}

/*
 * out = D_DW(m) in (dagger: D_DW(m)^dag) on full 5d fields [s][site][12],
 * row by row from the tridiagonal of Eq. (MoebiusOp) with the coefficients
 * of row s, D+^(s) = b5(s) D_W + 1 and D-^(s) = c5(s) D_W - 1 (constant
 * b5, c5 unless per-slice arrays are given):
 *   row s:  D+^(s) psi_s + D-^(s) P- psi_{s+1} + D-^(s) P+ psi_{s-1},
 *   row 1:  the P+ term is -m D-^(1) P+ psi_Ls,  row Ls: the P- term is -m D-^(Ls) P- psi_1.
 * The adjoint takes (D^dag)_{s,s'} = (D_{s',s})^dag, so an off-diagonal term
 * of row s carries the coefficient of the row it comes from:
 *   row s:  D+^(s)dag psi_s + P+ D-^(s+1)dag psi_{s+1} + P- D-^(s-1)dag psi_{s-1},
 *   row 1:  -m P- D-^(Ls)dag psi_Ls,   row Ls: -m P+ D-^(1)dag psi_1.
 */
void or_ddw(cplx *out, const cplx *in, const cplx *U, const or_params *p, int dagger)
{
    init_gammas();
    const int Ls = p->Ls;
    long V = vol4(p->L), n = 12 * V;
    cplx *t = malloc(sizeof(cplx) * n), *u = malloc(sizeof(cplx) * n);
    for (int s = 0; s < Ls; ++s) {
        cplx *o = out + s * n;
        dw_affine(o, in + s * n, U, p->L, p->M5, p->mu, dagger, b5_of(p, s), 1.0);   /* D+ psi_s */
        int sp = (s + 1) % Ls, sm = (s - 1 + Ls) % Ls;
        double wp = (s == Ls - 1) ? -p->mf : 1.0;   /* coefficient of the s+1 block */
        double wm = (s == 0) ? -p->mf : 1.0;        /* coefficient of the s-1 block */
        if (!dagger) {
            proj_field(t, PM, in + sp * n, V);
            dw_affine(u, t, U, p->L, p->M5, p->mu, 0, c5_of(p, s), -1.0);
            for (long k = 0; k < n; ++k) o[k] += wp * u[k];
            proj_field(t, PP, in + sm * n, V);
            dw_affine(u, t, U, p->L, p->M5, p->mu, 0, c5_of(p, s), -1.0);
            for (long k = 0; k < n; ++k) o[k] += wm * u[k];
        } else {
            dw_affine(t, in + sp * n, U, p->L, p->M5, p->mu, 1, c5_of(p, sp), -1.0);
            proj_field(u, PP, t, V);
            for (long k = 0; k < n; ++k) o[k] += wp * u[k];
            dw_affine(t, in + sm * n, U, p->L, p->M5, p->mu, 1, c5_of(p, sm), -1.0);
            proj_field(u, PM, t, V);
            for (long k = 0; k < n; ++k) o[k] += wm * u[k];
        }
    }
    free(t);
    free(u);
}

/* ------------------------------------------------------- red/black blocks */

/*
 * Half-field hopping: out (parity po) = coef * W in + (accumulate ? out : 0),
 * W = -H/2 restricted to rows of parity po and columns of parity 1 - po.
 * This is the off-site-diagonal part of D_W (dagger: of D_W^dag).
 */
static void hop_half(cplx *out, const cplx *in, const cplx *U, const int L[4], int po,
                     int dagger, double coef, int accumulate, double chem)
{
    long Vh = vol4(L) / 2;
#pragma omp parallel for schedule(static)
    for (long j = 0; j < Vh; ++j) {
        long i = half_to_lex(L, j, po);
        cplx h[12];
        hop_site(h, in, 1, U, L, i, dagger, chem);
        for (int k = 0; k < 12; ++k) {
            cplx v = -0.5 * coef * h[k];
            out[12 * j + k] = accumulate ? out[12 * j + k] + v : v;
        }
    }
}

/*
 * One red/black block of the 5d operator, built from the tridiagonal of
 * Eq. (MoebiusOp) with every block entry replaced by one of its two parts
 * (cd[s], co[s]: the coefficients of row s):
 *   hop == 0 : the site-diagonal part (Eq. D_5d_matrix); D+^(s) -> cd[s], D-^(s) -> co[s].
 *              With cd = M+(s), co = M-(s) this is I_rr = I_bb.
 *   hop == 1 : the hopping part, D+^(s) -> cd[s] W, D-^(s) -> co[s] W, W = -H/2 from
 *              parity 1 - po to parity po. With cd = b5(s), co = c5(s) this is
 *              D_rb (po even) or D_br (po odd).
 * Rows:    out_s = cd[s] T psi_s + co[s] T P- psi_{s+1} + co[s] T P+ psi_{s-1}
 *          (row Ls: -m co[Ls] T P- psi_1; row 1: -m co[1] T P+ psi_Ls)
 * Adjoint: out_s = cd[s] T^dag psi_s + co[s+1] P+ T^dag psi_{s+1} + co[s-1] P- T^dag psi_{s-1}
 *          (row Ls: -m co[1] P+ T^dag psi_1; row 1: -m co[Ls] P- T^dag psi_Ls)
 * Fields are half fields [s][half site][12].
 */
static void rb_block(cplx *out, const cplx *in, const cplx *U, const or_params *p,
                     int po, int hop, const double *cd, const double *co, int dagger)
{
    init_gammas();
    const int Ls = p->Ls;
    long Vh = vol4(p->L) / 2, n = 12 * Vh;
    cplx *t = malloc(sizeof(cplx) * n), *u = malloc(sizeof(cplx) * n);
    for (int s = 0; s < Ls; ++s) {
        cplx *o = out + s * n;
        int sp = (s + 1) % Ls, sm = (s - 1 + Ls) % Ls;
        /* the coefficient of row s (operator) or of the row the term comes from (adjoint) */
        double wp = (dagger ? co[sp] : co[s]) * ((s == Ls - 1) ? -p->mf : 1.0);
        double wm = (dagger ? co[sm] : co[s]) * ((s == 0) ? -p->mf : 1.0);
        if (hop) {
            hop_half(o, in + s * n, U, p->L, po, dagger, cd[s], 0, p->mu);
            if (!dagger) {
                proj_field(t, PM, in + sp * n, Vh);
                hop_half(o, t, U, p->L, po, 0, wp, 1, p->mu);
                proj_field(t, PP, in + sm * n, Vh);
                hop_half(o, t, U, p->L, po, 0, wm, 1, p->mu);
            } else {
                hop_half(t, in + sp * n, U, p->L, po, 1, wp, 0, p->mu);
                proj_field(u, PP, t, Vh);
                for (long k = 0; k < n; ++k) o[k] += u[k];
                hop_half(t, in + sm * n, U, p->L, po, 1, wm, 0, p->mu);
                proj_field(u, PM, t, Vh);
                for (long k = 0; k < n; ++k) o[k] += u[k];
            }
        } else {
            for (long k = 0; k < n; ++k) o[k] = cd[s] * in[s * n + k];
            if (!dagger) {
                proj_field(t, PM, in + sp * n, Vh);
                for (long k = 0; k < n; ++k) o[k] += wp * t[k];
                proj_field(t, PP, in + sm * n, Vh);
                for (long k = 0; k < n; ++k) o[k] += wm * t[k];
            } else {
                proj_field(t, PP, in + sp * n, Vh);
                for (long k = 0; k < n; ++k) o[k] += wp * t[k];
                proj_field(t, PM, in + sm * n, Vh);
                for (long k = 0; k < n; ++k) o[k] += wm * t[k];
            }
        }
    }
    free(t);
    free(u);
}

/* per-row coefficient arrays (Ls <= 64) */
typedef struct { double v[64]; } coefs;
static coefs fill_const(int Ls, double x)
{
    coefs c = {{0}};
    for (int s = 0; s < Ls; ++s) c.v[s] = x;
    return c;
}
static coefs mplus_s(const or_params *p)
{
    coefs c = {{0}};
    for (int s = 0; s < p->Ls; ++s) c.v[s] = b5_of(p, s) * (4.0 - p->M5) + 1.0;
    return c;
}
static coefs mminus_s(const or_params *p)
{
    coefs c = {{0}};
    for (int s = 0; s < p->Ls; ++s) c.v[s] = c5_of(p, s) * (4.0 - p->M5) - 1.0;
    return c;
}
static coefs b5_s(const or_params *p)
{
    coefs c = {{0}};
    for (int s = 0; s < p->Ls; ++s) c.v[s] = b5_of(p, s);
    return c;
}
static coefs c5_s(const or_params *p)
{
    coefs c = {{0}};
    for (int s = 0; s < p->Ls; ++s) c.v[s] = c5_of(p, s);
    return c;
}

static double mplus(const or_params *p) { return p->b5 * (4.0 - p->M5) + 1.0; }
static double mminus(const or_params *p) { return p->c5 * (4.0 - p->M5) - 1.0; }

/* out = I_rr in (dagger: I_rr^dag); Eq. (D_5d_matrix). */
void or_mee(cplx *out, const cplx *in, const or_params *p, int dagger)
{
    coefs cd = mplus_s(p), co = mminus_s(p);
    rb_block(out, in, NULL, p, 0, 0, cd.v, co.v, dagger);
}

/* Hopping block from parity 1 - po to po (dagger: the block of D_DW^dag). */
void or_dhop(cplx *out, const cplx *in, const cplx *U, const or_params *p, int po, int dagger)
{
    coefs cd = b5_s(p), co = c5_s(p);
    rb_block(out, in, U, p, po, 1, cd.v, co.v, dagger);
}

/*
 * Closed-form solve of A_rr Psi = b along s (Sec. 3), per component; with
 * r = M-/M+ ("alpha" in the paper) and kappa = m r ("M" in the paper), 0-based s:
 *   Psi_{Ls-1} = [b_{Ls-1} + kappa sum_{s=0}^{Ls-2} (-r)^s b_s] / (M+ (1 - kappa (-r)^{Ls-1}))
 *   Psi_s      = -r Psi_{s+1} + b_s / M+,  s = Ls-2 .. 0.
 * transpose != 0 solves A_rr^T Psi = b with rows and columns interchanged:
 *   Psi_0 = [b_0 + kappa sum_{s=1}^{Ls-1} (-r)^{Ls-1-s} b_s] / (M+ (1 - kappa (-r)^{Ls-1}))
 *   Psi_s = -r Psi_{s-1} + b_s / M+,  s = 1 .. Ls-1.
 * b and Psi are strided columns (stride in complex elements).
 */
static void solve_arr(cplx *psi, const cplx *b, long stride, int Ls, double Mp, double Mm,
                      double m, int transpose)
{
    double r = Mm / Mp, kappa = m * r;
    double den = Mp * (1.0 - kappa * pow(-r, Ls - 1));
    if (!transpose) {
        cplx acc = b[(long)(Ls - 1) * stride];
        for (int s = 0; s <= Ls - 2; ++s) acc += kappa * pow(-r, s) * b[(long)s * stride];
        psi[(long)(Ls - 1) * stride] = acc / den;
        for (int s = Ls - 2; s >= 0; --s)
            psi[(long)s * stride] = -r * psi[(long)(s + 1) * stride] + b[(long)s * stride] / Mp;
    } else {
        cplx acc = b[0];
        for (int s = 1; s <= Ls - 1; ++s) acc += kappa * pow(-r, Ls - 1 - s) * b[(long)s * stride];
        psi[0] = acc / den;
        for (int s = 1; s <= Ls - 1; ++s)
            psi[(long)s * stride] = -r * psi[(long)(s - 1) * stride] + b[(long)s * stride] / Mp;
    }
}

/*
 * With per-slice coefficients the two chiral blocks of I_rr (the rows of
 * Eq. D_5d_matrix with M+-(s) = b5(s) (4 - M5) + 1, c5(s) (4 - M5) - 1) are
 *   P- : A_{s,s} = M+(s), A_{s,s+1} = M-(s), A_{Ls,1} = -m M-(Ls)
 *   P+ : B_{s,s} = M+(s), B_{s,s-1} = M-(s), B_{1,Ls} = -m M-(1)
 * and no longer each other's transpose; the closed form of Sec. 3 needs
 * constant coefficients, so these are inverted by plain Gauss-Jordan
 * elimination with partial pivoting.
 */
static void chiral_block(double *a, const or_params *p, int minus, int transpose)
{
    const int Ls = p->Ls;
    coefs mp = mplus_s(p), mm = mminus_s(p);
    for (int i = 0; i < Ls * Ls; ++i) a[i] = 0.0;
    for (int s = 0; s < Ls; ++s) {
        a[s * Ls + s] += mp.v[s];
        if (minus) a[s * Ls + (s + 1) % Ls] += (s == Ls - 1) ? -p->mf * mm.v[s] : mm.v[s];
        else a[s * Ls + (s - 1 + Ls) % Ls] += (s == 0) ? -p->mf * mm.v[s] : mm.v[s];
    }
    if (transpose)
        for (int i = 0; i < Ls; ++i)
            for (int j = i + 1; j < Ls; ++j) {
                double t = a[i * Ls + j];
                a[i * Ls + j] = a[j * Ls + i];
                a[j * Ls + i] = t;
            }
}

static void invert_real(double *inv, const double *a, int n)
{
    const int w = 2 * n;
    double *m = malloc(sizeof(double) * n * w);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < w; ++j) m[i * w + j] = j < n ? a[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(m[r * w + c]) > fabs(m[piv * w + c])) piv = r;
        for (int j = 0; j < w; ++j) {
            double t = m[c * w + j];
            m[c * w + j] = m[piv * w + j];
            m[piv * w + j] = t;
        }
        double d = m[c * w + c];
        for (int j = 0; j < w; ++j) m[c * w + j] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = m[r * w + c];
            for (int j = 0; j < w; ++j) m[r * w + j] -= f * m[c * w + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) inv[i * n + j] = m[i * w + n + j];
    free(m);
}

/*
 * out = I_rr^-1 in = A^-1 P- in + A^{T,-1} P+ in   (Sec. 3)
 * dagger: out = I_rr^{-dag} in = A^{T,-1} P- in + A^-1 P+ in
 * (A_rr is real, so I_rr^dag = A^T P- + A P+). Half fields, nsites sites.
 */
void or_mee_inv(cplx *out, const cplx *in, long nsites, const or_params *p, int dagger)
{
    init_gammas();
    const int Ls = p->Ls;
    long n = 12 * nsites;
    cplx *bm = malloc(sizeof(cplx) * n * Ls), *bp = malloc(sizeof(cplx) * n * Ls);
    cplx *xm = malloc(sizeof(cplx) * n * Ls), *xp = malloc(sizeof(cplx) * n * Ls);
    for (int s = 0; s < Ls; ++s) {
        proj_field(bm + s * n, PM, in + s * n, nsites);
        proj_field(bp + s * n, PP, in + s * n, nsites);
    }
    if (!p->b5s && !p->c5s) {
        double Mp = mplus(p), Mm = mminus(p);
#pragma omp parallel for schedule(static)
        for (long k = 0; k < n; ++k) {
            solve_arr(xm + k, bm + k, n, Ls, Mp, Mm, p->mf, dagger ? 1 : 0);
            solve_arr(xp + k, bp + k, n, Ls, Mp, Mm, p->mf, dagger ? 0 : 1);
        }
    } else {
        double *A = malloc(sizeof(double) * Ls * Ls), *B = malloc(sizeof(double) * Ls * Ls);
        double *Ai = malloc(sizeof(double) * Ls * Ls), *Bi = malloc(sizeof(double) * Ls * Ls);
        chiral_block(A, p, 1, dagger);   /* the P- block (its transpose for the adjoint) */
        chiral_block(B, p, 0, dagger);   /* the P+ block */
        invert_real(Ai, A, Ls);
        invert_real(Bi, B, Ls);
#pragma omp parallel for schedule(static)
        for (long k = 0; k < n; ++k)
            for (int s = 0; s < Ls; ++s) {
                cplx am = 0, ap = 0;
                for (int t = 0; t < Ls; ++t) {
                    am += Ai[s * Ls + t] * bm[(long)t * n + k];
                    ap += Bi[s * Ls + t] * bp[(long)t * n + k];
                }
                xm[(long)s * n + k] = am;
                xp[(long)s * n + k] = ap;
            }
        free(A); free(B); free(Ai); free(Bi);
    }
    for (long k = 0; k < n * Ls; ++k) out[k] = xm[k] + xp[k];
    free(bm); free(bp); free(xm); free(xp);
}

/* --------------------------------------------- preconditioned operator M */

/*
 * out = D_pre in = in - I_bb^-1 D_br I_rr^-1 D_rb in on odd half fields (Sec. 3),
 * red = even, black = odd. dagger: the adjoint
 *   D_pre^dag = 1 - (D_rb)^dag I_rr^{-dag} (D_br)^dag I_bb^{-dag},
 * where (D_br)^dag is the even-row block of D_DW^dag and (D_rb)^dag its odd-row block.
 */
void or_m(cplx *out, const cplx *in, const cplx *U, const or_params *p, int dagger)
{
    long Vh = vol4(p->L) / 2, n = 12 * Vh * p->Ls;
    cplx *a = malloc(sizeof(cplx) * n), *b = malloc(sizeof(cplx) * n);
    if (!dagger) {
        or_dhop(a, in, U, p, 0, 0);        /* D_rb in   (even) */
        or_mee_inv(b, a, Vh, p, 0);        /* I_rr^-1   (even) */
        or_dhop(a, b, U, p, 1, 0);         /* D_br      (odd)  */
        or_mee_inv(b, a, Vh, p, 0);        /* I_bb^-1   (odd)  */
    } else {
        or_mee_inv(a, in, Vh, p, 1);       /* I_bb^-dag (odd)  */
        or_dhop(b, a, U, p, 0, 1);         /* (D_br)^dag: odd -> even */
        or_mee_inv(a, b, Vh, p, 1);        /* I_rr^-dag (even) */
        or_dhop(b, a, U, p, 1, 1);         /* (D_rb)^dag: even -> odd */
    }
    for (long k = 0; k < n; ++k) out[k] = in[k] - b[k];
    free(a);
    free(b);
}

/* --------------------------------------------------------------- algebra */

static cplx dotc(const cplx *a, const cplx *b, long n)
{
    cplx s = 0;
    for (long k = 0; k < n; ++k) s += conj(a[k]) * b[k];
    return s;
}

static double norm2(const cplx *a, long n)
{
    double s = 0;
    for (long k = 0; k < n; ++k) s += creal(a[k]) * creal(a[k]) + cimag(a[k]) * cimag(a[k]);
    return s;
}

/* out = M^dag M in */
void or_mdagm(cplx *out, const cplx *in, const cplx *U, const or_params *p)
{
    long n = 12 * (vol4(p->L) / 2) * p->Ls;
    cplx *t = malloc(sizeof(cplx) * n);
    or_m(t, in, U, p, 0);
    or_m(out, t, U, p, 1);
    free(t);
}

/*
 * Textbook conjugate gradient on M^dag M x = rhs (the paper names CG,
 * Sec. 2.3 and Sec. 4, without fixing its variant). When the iterated residual
 * reaches tol, the true residual |rhs - M^dag M x| / |rhs| is recomputed and
 * CG restarts from x if that is still above tol. x holds the starting guess.
 * Returns 0 on convergence, 1 if maxiter was reached, 2 on breakdown.
 */
static int cg_normal(cplx *x, const cplx *rhs, const cplx *U, const or_params *p, double tol,
                     int maxiter, int *iters, double *true_rel)
{
    long n = 12 * (vol4(p->L) / 2) * p->Ls;
    cplx *r = malloc(sizeof(cplx) * n), *pp = malloc(sizeof(cplx) * n);
    cplx *ap = malloc(sizeof(cplx) * n);
    double src2 = norm2(rhs, n), rel = 0;
    int k = 0, status = 1;
    if (src2 == 0.0) {
        memset(x, 0, sizeof(cplx) * n);
        status = 0;
        goto done;
    }
    for (;;) {
        /* (re)start from the true residual r = rhs - M^dag M x */
        or_mdagm(ap, x, U, p);
        for (long i = 0; i < n; ++i) r[i] = rhs[i] - ap[i];
        double rr = norm2(r, n);
        rel = sqrt(rr / src2);
        if (rel <= tol) { status = 0; break; }
        if (k >= maxiter) break;
        memcpy(pp, r, sizeof(cplx) * n);
        while (k < maxiter) {
            or_mdagm(ap, pp, U, p);
            double pap = creal(dotc(pp, ap, n));
            if (!(pap > 0.0)) { status = 2; goto done; }
            double alpha = rr / pap;
            for (long i = 0; i < n; ++i) { x[i] += alpha * pp[i]; r[i] -= alpha * ap[i]; }
            double rr_new = norm2(r, n);
            ++k;
            if (sqrt(rr_new / src2) <= tol) break;
            double beta = rr_new / rr;
            for (long i = 0; i < n; ++i) pp[i] = r[i] + beta * pp[i];
            rr = rr_new;
        }
    }
done:
    if (iters) *iters = k;
    if (true_rel) *true_rel = rel;
    free(r); free(pp); free(ap);
    return status;
}

/*
 * CGNE: solves M x = b' through M^dag M x = M^dag b'. The reported residual is
 * the true |M^dag b' - M^dag M x| / |M^dag b'|.
 */
int or_cgne(cplx *x, const cplx *bprime, const cplx *U, const or_params *p, double tol,
            int maxiter, int *iters, double *true_rel)
{
    long n = 12 * (vol4(p->L) / 2) * p->Ls;
    cplx *src = malloc(sizeof(cplx) * n);
    or_m(src, bprime, U, p, 1);
    int st = cg_normal(x, src, U, p, tol, maxiter, iters, true_rel);
    free(src);
    return st;
}

/*
 * Solves D_DW(m)^dag x = b on full 5d fields by textbook CG on the Hermitian
 * positive operator D D^dag with right-hand side D b (x = D^-dag b), using only
 * the row-by-row D_DW of Eq. (MoebiusOp) and its adjoint; no red/black split.
 * The reported residual is |D^dag x - b| / |b|.
 */
int or_solve_dag(cplx *x, const cplx *b, const cplx *U, const or_params *p, double tol, int maxiter,
                 int *iters, double *true_rel)
{
    long n = 12 * vol4(p->L) * p->Ls;
    cplx *rhs = malloc(sizeof(cplx) * n), *r = malloc(sizeof(cplx) * n), *pp = malloc(sizeof(cplx) * n);
    cplx *t = malloc(sizeof(cplx) * n), *ap = malloc(sizeof(cplx) * n);
    or_ddw(rhs, b, U, p, 0);
    memset(x, 0, sizeof(cplx) * n);
    double src2 = norm2(rhs, n), b2 = norm2(b, n);
    int k = 0, status = 1;
    if (src2 == 0.0) { status = 0; goto done; }
    memcpy(r, rhs, sizeof(cplx) * n);
    memcpy(pp, r, sizeof(cplx) * n);
    double rr = src2;
    while (k < maxiter) {
        or_ddw(t, pp, U, p, 1);
        or_ddw(ap, t, U, p, 0);      /* D D^dag p */
        double pap = creal(dotc(pp, ap, n));
        if (!(pap > 0.0)) { status = 2; goto done; }
        double alpha = rr / pap;
        for (long i = 0; i < n; ++i) { x[i] += alpha * pp[i]; r[i] -= alpha * ap[i]; }
        double rr_new = norm2(r, n);
        ++k;
        if (sqrt(rr_new / src2) <= tol) { status = 0; break; }
        double beta = rr_new / rr;
        for (long i = 0; i < n; ++i) pp[i] = r[i] + beta * pp[i];
        rr = rr_new;
    }
done:
    or_ddw(t, x, U, p, 1);
    for (long i = 0; i < n; ++i) t[i] -= b[i];
    if (true_rel) *true_rel = b2 > 0 ? sqrt(norm2(t, n) / b2) : 0.0;
    if (iters) *iters = k;
    free(rhs); free(r); free(pp); free(t); free(ap);
    return status;
}

/* ------------------------------------------- source prep and reconstruction */

/* split a full 5d field [s][V][12] into its even and odd half fields */
static void split_parity(cplx *even, cplx *odd, const cplx *full, const or_params *p)
{
    long V = vol4(p->L), Vh = V / 2;
    for (int s = 0; s < p->Ls; ++s)
        for (long i = 0; i < V; ++i) {
            int x[4];
            coords(p->L, i, x);
            cplx *dst = (parity_of(x) ? odd : even) + 12 * (s * Vh + i / 2);
            memcpy(dst, full + 12 * (s * V + i), sizeof(cplx) * 12);
        }
}

static void join_parity(cplx *full, const cplx *even, const cplx *odd, const or_params *p)
{
    long V = vol4(p->L), Vh = V / 2;
    for (int s = 0; s < p->Ls; ++s)
        for (long i = 0; i < V; ++i) {
            int x[4];
            coords(p->L, i, x);
            const cplx *src = (parity_of(x) ? odd : even) + 12 * (s * Vh + i / 2);
            memcpy(full + 12 * (s * V + i), src, sizeof(cplx) * 12);
        }
}

/* b'_o = I_bb^-1 (b_o - D_br I_rr^-1 b_e)   (Schur decomposition, Sec. 3) */
void or_prepare(cplx *bprime, const cplx *b_full, const cplx *U, const or_params *p)
{
    long Vh = vol4(p->L) / 2, n = 12 * Vh * p->Ls;
    cplx *be = malloc(sizeof(cplx) * n), *bo = malloc(sizeof(cplx) * n);
    cplx *t = malloc(sizeof(cplx) * n), *u = malloc(sizeof(cplx) * n);
    split_parity(be, bo, b_full, p);
    or_mee_inv(t, be, Vh, p, 0);
    or_dhop(u, t, U, p, 1, 0);
    for (long k = 0; k < n; ++k) t[k] = bo[k] - u[k];
    or_mee_inv(bprime, t, Vh, p, 0);
    free(be); free(bo); free(t); free(u);
}

/* x_e = I_rr^-1 (b_e - D_rb x_o); x_full = (x_e, x_o) */
void or_reconstruct(cplx *x_full, const cplx *x_odd, const cplx *b_full, const cplx *U,
                    const or_params *p)
{
    long Vh = vol4(p->L) / 2, n = 12 * Vh * p->Ls;
    cplx *be = malloc(sizeof(cplx) * n), *bo = malloc(sizeof(cplx) * n);
    cplx *t = malloc(sizeof(cplx) * n), *xe = malloc(sizeof(cplx) * n);
    split_parity(be, bo, b_full, p);
    or_dhop(t, x_odd, U, p, 0, 0);
    for (long k = 0; k < n; ++k) t[k] = be[k] - t[k];
    or_mee_inv(xe, t, Vh, p, 0);
    join_parity(x_full, xe, x_odd, p);
    free(be); free(bo); free(t); free(xe);
}

/* Full solve of D_DW(m) x = b: prepare, CGNE on the odd sites, reconstruct. */
int or_solve(cplx *x_full, const cplx *b_full, const cplx *U, const or_params *p, double tol,
             int maxiter, int *iters, double *true_rel)
{
    long n = 12 * (vol4(p->L) / 2) * p->Ls;
    cplx *bp = malloc(sizeof(cplx) * n), *xo = calloc((size_t)n, sizeof(cplx));
    or_prepare(bp, b_full, U, p);
    int st = or_cgne(xo, bp, U, p, tol, maxiter, iters, true_rel);
    or_reconstruct(x_full, xo, b_full, U, p);
    free(bp);
    free(xo);
    return st;
}

/* ---------------------------------------------------------------- force */

/*
 * Accumulates into the gauge derivative Gd[site][mu][3][3] the derivative of
 * coef * Re(c^dag W e), W = -H/2 from parity 1 - po to po, with respect to the
 * links: for a variation dU of U_mu(x), Re(c^dag dW e) = Re sum conj(Gd) dU
 * with (outer products over colour, summed over spin and s)
 *   forward  U_mu(x),    x of parity po:  -1/2 sum_s (1 - g_mu) c_x  (x) e_{x+mu}^*
 *   backward U_mu(x-mu), x of parity po:  -1/2 sum_s e_{x-mu} (x) [(1 + g_mu) c_x]^*
 * c lives on parity po, e on 1 - po (half fields [s][site][12]).
 */
static void acc_link_derivative(cplx *Gd, const cplx *c, const cplx *e, const or_params *p,
                                int po, double coef)
{
    long Vh = vol4(p->L) / 2;
    const int Ls = p->Ls;
    for (long j = 0; j < Vh; ++j) {
        long i = half_to_lex(p->L, j, po);
        for (int mu = 0; mu < 4; ++mu) {
            long fw = shift(p->L, i, mu, +1), bw = shift(p->L, i, mu, -1);
            /* the forward time hop of the (undaggered) block carries e^{+mu}, the
               backward one e^{-mu} (Sec. 6.6) */
            const double wf = (mu == 3 && p->mu != 0.0) ? exp(p->mu) : 1.0;
            const double wb = (mu == 3 && p->mu != 0.0) ? exp(-p->mu) : 1.0;
            cplx Sm[4][4], Sp[4][4];
            one_pm_gamma(Sm, mu, -1.0);
            one_pm_gamma(Sp, mu, +1.0);
            cplx *gf = Gd + 9 * (4 * i + mu), *gb = Gd + 9 * (4 * bw + mu);
            for (int s = 0; s < Ls; ++s) {
                cplx pc[12], qc[12];
                spin_mat(pc, Sm, c + 12 * (s * Vh + j));
                spin_mat(qc, Sp, c + 12 * (s * Vh + j));
                const cplx *ef = e + 12 * (s * Vh + fw / 2);
                const cplx *eb = e + 12 * (s * Vh + bw / 2);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        cplx sf = 0, sb = 0;
                        for (int sp = 0; sp < 4; ++sp) {
                            sf += pc[3 * sp + a] * conj(ef[3 * sp + b]);
                            sb += eb[3 * sp + a] * conj(qc[3 * sp + b]);
                        }
                        gf[3 * a + b] += coef * (-0.5) * wf * sf;
                        gb[3 * a + b] += coef * (-0.5) * wb * sb;
                    }
            }
        }
    }
}

/*
 * d/d(theta) of M applied to X, for theta = b5 (which == 0) or c5 (which == 1),
 * constant over the slices (slice < 0) or the coefficient of row `slice` alone:
 *   M = 1 - A D_br A D_rb,  A = I^-1,  dA = -A dI A,
 *   dM X = -[dA D_br A D_rb X + A dD_br A D_rb X + A D_br dA D_rb X + A D_br A dD_rb X]
 * with dI the site-diagonal block whose D+ part is (4 - M5) (b5) or whose D-
 * part is (4 - M5) (c5), and dD the hopping block with D+ -> W (b5) or
 * D- -> W (c5); both follow from D+ = b5 D_W + 1, D- = c5 D_W - 1.
 */
static void dm_dparam_rows(cplx *out, const cplx *X, const cplx *U, const or_params *p, int which, int slice)
{
    long Vh = vol4(p->L) / 2, n = 12 * Vh * p->Ls;
    double w = 4.0 - p->M5;
    double dId = which == 0 ? w : 0.0, dIo = which == 0 ? 0.0 : w;
    double dHd = which == 0 ? 1.0 : 0.0, dHo = which == 0 ? 0.0 : 1.0;
    cplx *e1 = malloc(sizeof(cplx) * n), *e2 = malloc(sizeof(cplx) * n);
    cplx *t = malloc(sizeof(cplx) * n), *u = malloc(sizeof(cplx) * n);
    memset(out, 0, sizeof(cplx) * n);
    /* e1 = D_rb X, e2 = A D_rb X (even) */
    or_dhop(e1, X, U, p, 0, 0);
    or_mee_inv(e2, e1, Vh, p, 0);
    /* term 1: dA D_br A D_rb X = -A dI A D_br e2 */
    or_dhop(t, e2, U, p, 1, 0);
    or_mee_inv(u, t, Vh, p, 0);
    coefs cId = fill_const(p->Ls, dId), cIo = fill_const(p->Ls, dIo);
    coefs cHd = fill_const(p->Ls, dHd), cHo = fill_const(p->Ls, dHo);
    if (slice >= 0)  /* only row `slice` of I and of the hopping block depends on theta */
        for (int k = 0; k < p->Ls; ++k)
            if (k != slice) cId.v[k] = cIo.v[k] = cHd.v[k] = cHo.v[k] = 0.0;
    rb_block(t, u, NULL, p, 1, 0, cId.v, cIo.v, 0);
    or_mee_inv(u, t, Vh, p, 0);
    for (long k = 0; k < n; ++k) out[k] -= -u[k];
    /* term 2: A dD_br e2 */
    rb_block(t, e2, U, p, 1, 1, cHd.v, cHo.v, 0);
    or_mee_inv(u, t, Vh, p, 0);
    for (long k = 0; k < n; ++k) out[k] -= u[k];
    /* term 3: A D_br dA e1 = -A D_br A dI A e1 */
    rb_block(t, e2, NULL, p, 0, 0, cId.v, cIo.v, 0);
    or_mee_inv(u, t, Vh, p, 0);
    or_dhop(t, u, U, p, 1, 0);
    or_mee_inv(u, t, Vh, p, 0);
    for (long k = 0; k < n; ++k) out[k] -= -u[k];
    /* term 4: A D_br A dD_rb X */
    rb_block(t, X, U, p, 0, 1, cHd.v, cHo.v, 0);
    or_mee_inv(u, t, Vh, p, 0);
    or_dhop(t, u, U, p, 1, 0);
    or_mee_inv(u, t, Vh, p, 0);
    for (long k = 0; k < n; ++k) out[k] -= u[k];
    free(e1); free(e2); free(t); free(u);
}

void or_dm_dparam(cplx *out, const cplx *X, const cplx *U, const or_params *p, int which)
{
    dm_dparam_rows(out, X, U, p, which, -1);
}

/*
 * Action S = phi^dag (M^dag M)^-1 phi and its derivatives. With X = (M^dag M)^-1 phi
 * and Y = M X, a variation of M gives dS = -2 Re(Y^dag dM X). M depends on the
 * links only through D_br and D_rb:
 *   dM = -[A dD_br A D_rb + A D_br A dD_rb],
 *   dS = 2 Re(a^dag dD_br b) + 2 Re(c^dag dD_rb X),
 *   a = A^dag Y (odd), b = A D_rb X (even), c = A^dag (D_br)^dag a (even).
 * Each dD is the hopping block, so Re(v^dag dD w) = Re(v^dag dW w~) with w~ the
 * same tridiagonal in s with D+ -> b5, D- -> c5 applied to w.
 * Outputs: dSdU [site][mu][3][3] complex with dS = Re sum conj(dSdU) dU over
 * independent complex link entries (dSdU = dS/dRe U + i dS/dIm U), dS/db5, dS/dc5.
 * Returns the CG status.
 */
int or_force(cplx *dSdU, double *dSdb5, double *dSdc5, double *S, const cplx *phi,
             const cplx *U, const or_params *p, double tol, int maxiter, int *iters)
{
    const int per_slice = p->b5s || p->c5s;
    long V = vol4(p->L), Vh = V / 2, n = 12 * Vh * p->Ls;
    cplx *X = calloc((size_t)n, sizeof(cplx)), *Y = malloc(sizeof(cplx) * n);
    cplx *a = malloc(sizeof(cplx) * n), *b = malloc(sizeof(cplx) * n);
    cplx *c = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
    cplx *w = malloc(sizeof(cplx) * n);
    double rel = 0;
    int st = cg_normal(X, phi, U, p, tol, maxiter, iters, &rel);
    *S = creal(dotc(phi, X, n));
    or_m(Y, X, U, p, 0);
    or_mee_inv(a, Y, Vh, p, 1);             /* a = A^dag Y        (odd)  */
    or_dhop(t, X, U, p, 0, 0);
    or_mee_inv(b, t, Vh, p, 0);             /* b = A D_rb X       (even) */
    or_dhop(t, a, U, p, 0, 1);
    or_mee_inv(c, t, Vh, p, 1);             /* c = A^dag D_br^dag a (even) */
    memset(dSdU, 0, sizeof(cplx) * 9 * 4 * V);
    coefs cb5 = b5_s(p), cc5 = c5_s(p);
    rb_block(w, b, NULL, p, 0, 0, cb5.v, cc5.v, 0);   /* b~ (even) */
    acc_link_derivative(dSdU, a, w, p, 1, 2.0);    /* 2 Re(a^dag dD_br b) */
    rb_block(w, X, NULL, p, 1, 0, cb5.v, cc5.v, 0);   /* X~ (odd) */
    acc_link_derivative(dSdU, c, w, p, 0, 2.0);    /* 2 Re(c^dag dD_rb X) */
    if (per_slice) {  /* dS/db5(s), dS/dc5(s): Ls values each */
        for (int sl = 0; sl < p->Ls; ++sl) {
            dm_dparam_rows(t, X, U, p, 0, sl);
            dSdb5[sl] = -2.0 * creal(dotc(Y, t, n));
            dm_dparam_rows(t, X, U, p, 1, sl);
            dSdc5[sl] = -2.0 * creal(dotc(Y, t, n));
        }
    } else {
        or_dm_dparam(t, X, U, p, 0);
        *dSdb5 = -2.0 * creal(dotc(Y, t, n));
        or_dm_dparam(t, X, U, p, 1);
        *dSdc5 = -2.0 * creal(dotc(Y, t, n));
    }
    free(X); free(Y); free(a); free(b); free(c); free(t); free(w);
    return st;
}

/* ---------------------------------------------------------------- threads */

void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
