/*
 * mdwf.h -- C ABI of libmdwf: the 4d red/black-preconditioned Moebius
 * domain-wall operator and its CG solve on one GB300 GPU (sm_103a).
 *
 * Method: R. C. Brower, H. Neff, K. Orginos, "The Moebius Domain Wall Fermion
 * Algorithm", arXiv:1206.5214.
 *
 * Operator conventions (shared with every caller):
 *   D_W   = (4 - M5) - H/2,  H = sum_mu [(1 - g_mu) U_mu(x) d_{x+mu,y}
 *                                       + (1 + g_mu) U_mu(y)^dag d_{x,y+mu}]
 *           (Eq. D^Wilson with the Wilson mass -M5; M5 > 0 is the wall height).
 *   D_DW  = the tridiagonal of Eq. MoebiusOp with D+ = b5 D_W + 1,
 *           D- = c5 D_W - 1 and the mass-mf corners.
 *   red/black = checkerboard on x+y+z+t, the same for every s (Sec. 3).
 *   M     = 1 - I_bb^-1 D_br I_rr^-1 D_rb on the odd (black) sites (Sec. 3),
 *           the operator every mdwf_apply computes and mdwf_cgne inverts.
 *   Chiral gamma basis g_mu = [[0, A_mu], [A_mu^dag, 0]], A_k = -i sigma_k,
 *   A_4 = 1, g5 = diag(1, 1, -1, -1); P+ is spins 0, 1 and P- spins 2, 3.
 *   Periodic boundary conditions in all four directions.
 *
 * User data formats (complex128 = two doubles, C order):
 *   gauge      U[t][z][y][x][mu][3][3], mu = 0..3 for x, y, z, t; U_mu(x) links
 *              x to x+mu.
 *   full field [rhs][s][t][z][y][x][spin 4][colour 3]
 *   odd field  [rhs][s][t][z][y][x/2][spin 4][colour 3]: the odd sites
 *              (x+y+z+t odd) of every (y, z, t) row in increasing x.
 *   dims = {X, Y, Z, T}, every extent even and >= 2, Ls even and >= 2.
 *
 * Internal fields are opaque device buffers of mdwf_field_bytes() bytes
 * (256-byte aligned pointers), one per precision: the caller allocates them
 * (cudaMalloc, torch.empty, ...) and owns them; the library never frees
 * caller memory. The context owns its own workspace (gauge copies, Ls x Ls
 * tables, temporaries) and frees it in mdwf_destroy.
 *
 * Streams and synchronisation: every call enqueues its GPU work on the
 * context's stream (mdwf_opts.stream, or mdwf_set_stream) and returns after
 * the enqueue, except where a function says it synchronises. Calls on one
 * context must not run concurrently from several host threads.
 *
 * Errors: every function returns an mdwf_status; nothing is thrown across the
 * ABI. MDWF_ECUDA reports a failed CUDA call (the CUDA error string is kept
 * for mdwf_last_error()).
 */
#ifndef MDWF_H
#define MDWF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MDWF_OK = 0,
    MDWF_EINVAL = 1,      /* bad argument: odd/zero extent, Ls < 2 or odd, NULL pointer, bad enum */
    MDWF_ENOMEM = 2,      /* device or host allocation failed */
    MDWF_ECUDA = 3,       /* a CUDA runtime call failed */
    MDWF_ENOCONV = 4,     /* the solve reached maxiter; x holds the last iterate */
    MDWF_EBREAKDOWN = 5,  /* CG breakdown: <p, M^dag M p> <= 0 or a non-finite scalar */
    MDWF_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
    MDWF_ENOGAUGE = 7     /* no gauge field loaded yet */
} mdwf_status;

typedef enum {
    MDWF_F64 = 0,         /* FP64 values, FP64 arithmetic */
    MDWF_F32 = 1,         /* FP32 values, FP32 arithmetic */
    MDWF_F16N = 2         /* FP16 values with one FP32 norm per (site, s); FP32 arithmetic */
} mdwf_precision;

typedef enum {
    MDWF_HOST = 0,        /* pointer is host memory (pageable or pinned) */
    MDWF_DEVICE = 1       /* pointer is device memory of the context's device */
} mdwf_where;

typedef struct mdwf_ctx mdwf_ctx;

typedef struct {
    void *stream;         /* cudaStream_t to enqueue on; NULL = the legacy default stream */
    int device;           /* CUDA device ordinal; -1 = the device current at mdwf_create */
    int dense_s;          /* 1: apply the Ls x Ls factors (I^-1, K, M_phi) as dense matrices built on
                             the host; 0: by the closed-form elimination of Sec. 3 wherever
                             |M-/M+| <= 0.9 (dense otherwise) */
    int autotune;         /* 1: the first solve of each (precision, nrhs) tunes the hop kernels'
                             block shape (see mdwf_autotune) */
} mdwf_opts;

/*
 * Creates a context for one lattice and one set of Moebius parameters
 * (Eq. MoebiusOp with constant b5(s) = b5, c5(s) = c5, Sec. 2.1).
 * dims: {X, Y, Z, T}, each even and >= 2. Ls: even, 2 <= Ls <= 32.
 * M5: wall height (D_W diagonal 4 - M5). mf: wall mass m (Eq. DWaction).
 * opts may be NULL. On success *out owns device workspace until mdwf_destroy.
 */
int mdwf_create(mdwf_ctx **out, const int dims[4], int Ls, double M5, double b5, double c5,
                double mf, const mdwf_opts *opts);

/*
 * Domain decomposition along t (Sec. 3: the Ls x Ls factors are site-local,
 * so only the 4d hopping term couples sub-lattices; the fifth dimension is
 * never split). The lattice {X, Y, Z, T} is cut into n slabs of T/n
 * t-slices each, slab r holding global t = r T/n .. (r+1) T/n - 1; T/n must be
 * even (so that every slab keeps the global even/odd parity) and >= 2.
 *
 * mdwf_create_slab creates the context of one slab: local_dims = {X, Y, Z, T/n},
 * other arguments as for mdwf_create. Load the slab's own links with
 * mdwf_load_gauge (the gauge field restricted to its t-slices, user layout)
 * and import its fields with mdwf_field_import (its odd sites in user order:
 * the contiguous block of the global odd sites that lie in the slab). A slab
 * context applies its operator only through mdwf_slab_stage; every other
 * operator, solve or force call on it returns MDWF_EINVAL.
 */
int mdwf_create_slab(mdwf_ctx **out, const int local_dims[4], int Ls, double M5, double b5, double c5,
                     double mf, const mdwf_opts *opts);

/*
 * Bytes of one face buffer of a slab: both faces, [face 0 | face 1], each
 * [rhs][site of one parity in a t-slice][half spinor, 12 reals][s] in the
 * precision's reals (FP64 or FP32). 0 for a context that is not a slab or
 * for MDWF_F16N.
 */
size_t mdwf_slab_face_bytes(const mdwf_ctx *ctx, int prec, int nrhs);

/*
 * One stage of out = M in (dagger = 0) or M^dag in (dagger = 1) on a slab,
 * for nrhs internal odd fields of precision MDWF_F64 or MDWF_F32 (device).
 * The three stages run in order with the same prec, nrhs, mf_per_rhs and
 * dagger; between them the caller delivers the faces:
 *   stage 0: reads in; writes the faces of the first factor's output into send;
 *   stage 1: reads recv (the neighbours' stage-0 faces); first hop; writes the
 *            faces of its output into send;
 *   stage 2: reads recv (the neighbours' stage-1 faces) and in; writes out.
 * send and recv are caller-owned device buffers of mdwf_slab_face_bytes bytes.
 * Delivery: face 0 of slab r's send goes to face 0 of slab r-1's recv, face 1
 * of slab r's send to face 1 of slab r+1's recv (periodic in r); face 0 holds
 * the t' = 0 slice projected with the forward t-projector of the receiving
 * hop, face 1 the t' = T/n - 1 slice projected with the backward one and
 * multiplied by the sender's U_t^dag. The slab keeps its intermediate fields
 * between the stages (do not interleave other operator calls on it).
 * Errors: MDWF_EINVAL (not a slab, F16N, bad stage or pointer, per-slice
 * coefficients), MDWF_ENOGAUGE, MDWF_ENOMEM, MDWF_ECUDA.
 */
int mdwf_slab_stage(mdwf_ctx *ctx, int stage, void *out, const void *in, int prec, int nrhs,
                    const double *mf_per_rhs, int dagger, void *send, const void *recv);

/*
 * Bounds checks of the debug build. A library compiled with
 * -DMDWF_BOUNDS_CHECK=1 (build(debug_bounds=True): _build_bounds/libmdwf.so)
 * checks every field and link index its kernels compute against the extent
 * of the buffer view, skips an access out of range and records it in a
 * device word of the current device. No paper counterpart: it stands in for
 * a device memory checker. *checked = 1 for that build, 0 for the release
 * build (no checks; *violations = 0). *violations = 1 if an access was out
 * of range since the last reset (synchronises the device). reset != 0 clears
 * the word. Errors: MDWF_EINVAL (NULL pointer), MDWF_ECUDA.
 */
int mdwf_bounds_status(int *checked, int *violations, int reset);

/* Frees the context and its workspace (synchronises the context's stream). NULL is accepted. */
int mdwf_destroy(mdwf_ctx *ctx);

/* Changes the stream later calls enqueue on. */
int mdwf_set_stream(mdwf_ctx *ctx, void *stream);

/*
 * Per-slice Moebius coefficients (Sec. 2.1, Eq. DWaction with D+^(s) =
 * b5(s) D_W + 1, D-^(s) = c5(s) D_W - 1; the Zolotarev form of Sec. 4.3 takes
 * b5(s) - c5(s) fixed and b5(s) + c5(s) from the Zolotarev coefficients).
 * b5s, c5s: Ls values each in host memory, index s = 0..Ls-1 for slices
 * 1..Ls of the paper; copied, so the caller may free them on return. Both
 * NULL: back to the constant b5, c5 of mdwf_create.
 * While per-slice coefficients are set, every Ls x Ls factor is a dense
 * matrix (the closed form of Sec. 3 needs constant coefficients) applied in
 * the hop epilogues, mdwf_force returns dS/db5(s) and dS/dc5(s) per slice,
 * and mdwf_apply_noalloc returns MDWF_EINVAL (its fixed scratch holds no
 * dense tables). Waits for the context's stream. Errors: MDWF_EINVAL for
 * one array NULL and not the other, a non-finite value, or a singular
 * I = diag(M+(s)) + diag(M-(s)) C (the previous coefficients stay in force).
 */
int mdwf_set_s_coefficients(mdwf_ctx *ctx, const double *b5s, const double *c5s);

/*
 * Chemical potential mu on the time links (Sec. 6.6): the forward time hop of
 * D_W carries e^{+mu} and the backward one e^{-mu} ((1 -+ g_4) U_{+-4} ->
 * e^{+-mu} (1 -+ g_4) U_{+-4}); D_W is then no longer gamma5-Hermitian and
 * every operator, solve and construction of this library uses D_W(mu) (the
 * adjoints D_W(mu)^dag). 0 turns it off. The operators, solves and both
 * forces (mdwf_force, mdwf_force4d) include it. Errors: MDWF_EINVAL for a
 * non-finite or |mu| > 10 value.
 */
int mdwf_set_chemical_potential(mdwf_ctx *ctx, double mu);

/* The lattice of the context: dims[4] = x, y, z, t extents (host) and *Ls. */
int mdwf_get_geometry(const mdwf_ctx *ctx, int dims[4], int *Ls);

/* Writes the Ls coefficients in force to b5s, c5s (host, Ls values each) and
 * sets *per_slice to 1 when they are per-slice, 0 when constant. */
int mdwf_get_s_coefficients(const mdwf_ctx *ctx, double *b5s, double *c5s, int *per_slice);

/*
 * Loads the SU(3) links U_mu(x) (Eq. D^Wilson) from complex128
 * U[t][z][y][x][mu][3][3] in host (where = MDWF_HOST) or device memory.
 * The data is copied into per-parity, per-direction link arrays in FP64 and
 * FP32 (the FP32 copy also serves the FP16+norm operator); the caller's buffer
 * may be reused once the call returns (host) or once the stream has passed
 * this point (device).
 */
int mdwf_load_gauge(mdwf_ctx *ctx, const double *U, int where);

/* Bytes of one internal odd- (or even-) parity field of nrhs right-hand sides. */
size_t mdwf_field_bytes(const mdwf_ctx *ctx, int prec, int nrhs);

/*
 * Converts nrhs odd-site fields from the user odd format (complex128) in
 * host or device memory into the internal layout of precision prec (dst:
 * device, mdwf_field_bytes(ctx, prec, nrhs) bytes). F16N stores each (site, s)
 * spinor as FP16 values scaled by their max-abs component, kept as an FP32 norm.
 */
int mdwf_field_import(mdwf_ctx *ctx, void *dst, const double *src, int prec, int nrhs, int where);

/* Inverse of mdwf_field_import: internal field (device) -> user odd format (host or device). */
int mdwf_field_export(mdwf_ctx *ctx, double *dst, const void *src, int prec, int nrhs, int where);

/*
 * out = M in on the odd sites, M = 1 - I_bb^-1 D_br I_rr^-1 D_rb (Sec. 3),
 * for nrhs internal fields of precision prec (device buffers, in != out).
 * mf_per_rhs: NULL (every right-hand side uses the context's mf) or nrhs
 * masses (host memory), one per right-hand side.
 */
int mdwf_apply(mdwf_ctx *ctx, void *out, const void *in, int prec, int nrhs, const double *mf_per_rhs);

/* out = M^dag in, the adjoint of mdwf_apply's operator (same arguments). */
int mdwf_apply_dag(mdwf_ctx *ctx, void *out, const void *in, int prec, int nrhs, const double *mf_per_rhs);

/*
 * Allocation-free variant of mdwf_apply / mdwf_apply_dag (dagger != 0); the
 * paper has no counterpart: it exists for callers that must not allocate
 * device memory while they run, such as a custom operator inside a framework
 * whose pool owns all device memory, a latency-critical path that must stay
 * out of the driver's allocator, or a service whose footprint must stay fixed.
 * Create the context (which allocates) during set-up; this call then
 * allocates nothing and frees nothing.
 * Arguments as for mdwf_apply. The operator's intermediate fields live in a
 * fixed scratch area that every GPU loading the library holds until the
 * process exits: at most 8 MiB per intermediate field, i.e.
 * mdwf_field_bytes(ctx, prec, nrhs) <= 8 MiB (MDWF_EINVAL with a message in
 * mdwf_last_error() otherwise; also MDWF_EINVAL for a context created with
 * dense_s = 1, for a mass that is not finite, and for a mass at which
 * I = M+ + M- C is singular, as mdwf_apply reports it). The per-rhs masses
 * are passed by value to a kernel that writes them into a fixed device array;
 * the caller's mf_per_rhs buffer is not read after the call returns.
 * The first call on a device looks up the scratch's device address (once
 * per device); make that first call before any stream capture.
 * All calls share the scratch and keep the last call's contents (every call
 * overwrites what it reads, so nothing needs clearing): calls whose GPU work
 * overlaps (different streams or contexts at the same time) race.
 */
int mdwf_apply_noalloc(mdwf_ctx *ctx, void *out, const void *in, int prec, int nrhs, const double *mf_per_rhs,
                       int dagger);

typedef struct {
    double tol;           /* target |M^dag b' - M^dag M x| / |M^dag b'| (FP64, recomputed); 0 = 1e-10 */
    int maxiter;          /* CG iteration cap; 0 = 20000 */
    int inner_prec;       /* MDWF_F64: plain FP64 CG; MDWF_F32 / MDWF_F16N: mixed precision
                             with FP64 reliable updates of x and the true residual */
    double delta;         /* reliable-update threshold on |r| / max |r|; 0 = 0.005 (FP32 inner), 0.1 (FP16N) */
    int check_every;      /* iterations between host convergence polls; 0 = 8 */
    int use_graph;        /* 1: replay the CG iteration as a captured CUDA graph */
    int guess;            /* 1: x holds an initial guess on entry and the CG starts from its odd
                             part (a restart or warm start); 0: the CG starts from zero */
} mdwf_solve_params;

typedef struct {
    int status;           /* MDWF_OK, MDWF_ENOCONV or MDWF_EBREAKDOWN for this right-hand side */
    int iters;            /* CG iterations */
    int reliable_updates; /* FP64 true-residual recomputations (mixed solves) */
    double true_res;      /* final FP64 |M^dag b' - M^dag M x| / |M^dag b'| */
    double res_m;         /* final FP64 |b' - M x| / |b'| */
    double seconds;       /* wall time of the whole call (same for every right-hand side) */
    int restarts;         /* mixed solves: reliable updates after which p restarted from the
                             true residual (it exceeded the inner estimate more than twice),
                             and roll-backs to the last update after an inner breakdown
                             (non-positive or non-finite <p, M^dag M p>) */
} mdwf_solve_info;

/*
 * Solves D_DW(m) x = b for nrhs full 5d right-hand sides (user full format,
 * complex128, host or device as where says): b'_o = I_bb^-1 (b_o - D_br
 * I_rr^-1 b_e), CG on M^dag M x_o = M^dag b'_o (Sec. 3; the solver of Sec. 4), then
 * x_e = I_rr^-1 (b_e - D_rb x_o). x has b's format and location.
 * mf_per_rhs: NULL or nrhs masses (host). params may be NULL (defaults).
 * info: NULL or an array of nrhs entries. Synchronises the stream.
 * Mixed precision: each right-hand side takes its own FP64 reliable update
 * when its inner |r| has fallen by delta (or the inner estimate reaches tol,
 * or maxiter is reached, or the inner |r| climbs 100x above the last true
 * one); the update corrects the search direction for the true residual, or
 * restarts it when the true |r| exceeds the inner one more than twice; an
 * inner breakdown rolls back to the last update (at most 8 times, then
 * MDWF_EBREAKDOWN). The reported true_res and the tol test are always the
 * FP64 residual of the returned x.
 * Returns the worst per-rhs status.
 */
int mdwf_cgne(mdwf_ctx *ctx, double *x, const double *b, int nrhs, const double *mf_per_rhs,
              int where, const mdwf_solve_params *params, mdwf_solve_info *info);

/*
 * out = D_DW(m) in (dagger = 1: D_DW(m)^dag), the full unpreconditioned
 * operator of Eq. MoebiusOp on nrhs full 5d fields (user full format,
 * complex128, host or device as where says; in != out). FP64. mf_per_rhs:
 * NULL or nrhs masses (host). Synchronises the stream for host buffers.
 */
int mdwf_apply_full(mdwf_ctx *ctx, double *out, const double *in, int nrhs, const double *mf_per_rhs,
                    int where, int dagger);

/*
 * The effective 4d overlap operator of Sec. 2.2 on nrhs 4d fields psi (user
 * 4d format [rhs][t][z][y][x][spin][colour], complex128, host or device):
 *   out = D_ov(m) psi = [P^dag D_DW(1)^-1 D_DW(m) P psi~]_{s=1},  psi~_s = psi delta_{s,1},
 * P the wall permutation of Sec. 2.2 ((P x)_s = P- x_s + P+ x_{s+1}). The
 * inverse is a Pauli-Villars solve (mdwf_cgne at mass 1 for every right-hand
 * side, params and info as there). out != psi. Synchronises the stream.
 * Returns the solve's status (MDWF_ENOCONV still writes out).
 */
int mdwf_overlap_apply(mdwf_ctx *ctx, double *out, const double *psi, int nrhs, const double *mf_per_rhs,
                       int where, const mdwf_solve_params *params, mdwf_solve_info *info);

/*
 * Bulk domain-wall solution from a 4d overlap solution (Sec. 2.3): given
 * psi = D_ov(m)^-1 b, writes the 5d Psi = P^dag D_DW(m)^-1 D_DW(1) P B of the
 * wall source B_s = b delta_{s,1} as Psi_1 = psi, Psi_s = -Omega_s (s > 1),
 * Omega = P^dag D_DW(1)^-1 D_DW(m) P psi~ (one Pauli-Villars solve).
 * Psi: full 5d user format; psi: 4d user format; both host or both device.
 * Synchronises the stream; returns the solve's status.
 */
int mdwf_pv_reconstruct(mdwf_ctx *ctx, double *Psi, const double *psi, int nrhs, const double *mf_per_rhs,
                        int where, const mdwf_solve_params *params, mdwf_solve_info *info);

/*
 * The chiral-symmetry violation of the effective overlap operator,
 * out = Delta_Ls psi = (1 - eps_Ls^2) psi / 4 (Eq. Delta_Ls), with
 * eps_Ls psi = gamma5 (2 D_ov(m) psi - (1 + m) psi) / (1 - m) from two
 * applications of mdwf_overlap_apply (two Pauli-Villars solves). 4d user
 * format, host or device; out != psi; every mass must differ from 1.
 * info receives the second solve's statistics. Synchronises the stream.
 */
int mdwf_gw_violation(mdwf_ctx *ctx, double *out, const double *psi, int nrhs, const double *mf_per_rhs,
                      int where, const mdwf_solve_params *params, mdwf_solve_info *info);

/*
 * Derivatives of the action S = phi^dag (M^dag M)^-1 phi with M the operator
 * of mdwf_apply (the Schur complement of Sec. 3) at the context's mass:
 *   dSdU  : complex128 in the gauge layout U[t][z][y][x][mu][3][3]: for every
 *           link entry dS/dRe U + i dS/dIm U, so that a variation dU changes S
 *           by Re sum conj(dSdU) dU (the entries are treated as independent
 *           complex numbers, not restricted to SU(3));
 *   dSdb5, dSdc5: dS/db5 and dS/dc5 of the same S (M's dependence on b5, c5
 *           through M_phi = b5 + c5 C and I = (b5 (4 - M5) + 1) + (c5 (4 - M5) - 1) C);
 *           with per-slice coefficients (mdwf_set_s_coefficients) each receives
 *           Ls values, dS/db5(s) and dS/dc5(s), s = 0..Ls-1 (host memory);
 *   S     : the action.
 * phi: one odd field in the user odd format; phi and dSdU are both host or
 * both device memory (where). X = (M^dag M)^-1 phi is recomputed by the CG
 * of mdwf_cgne (params as there; the force arithmetic is FP64 throughout).
 * info (may be NULL) reports that solve. dSdU, dSdb5, dSdc5, S may each be NULL;
 * with the three derivatives NULL only the action is computed.
 * Synchronises the stream. Returns the solve's status.
 */
int mdwf_force(mdwf_ctx *ctx, double *dSdU, double *dSdb5, double *dSdc5, double *S, const double *phi,
               int where, const mdwf_solve_params *params, mdwf_solve_info *info);

/*
 * The action with the pseudofermion on the wall (Sec. 2.4) and its link force:
 *   S = phi^dag P^dag D_DW(m)^-1 D_DW(1) D_DW(1)^dag D_DW(m)^-dag P phi,
 * phi a 4d field on s = 1 (user 4d format, host or device), P the wall
 * permutation of Sec. 2.2. Two inversions: an adjoint solve
 * chi = D_DW(m)^-dag P phi (red/black, CG on M^dag M) and a solve
 * psi = D_DW(m)^-1 D_DW(1) D_DW(1)^dag chi (mdwf_cgne); S = |D_DW(1)^dag chi|^2.
 * dSdU (NULL: action only) has the gauge layout and the convention of
 * mdwf_force (dS/dRe U + i dS/dIm U). One right-hand side; mf != 1; per-slice
 * coefficients are allowed. info receives the second solve's statistics.
 * Synchronises the stream; returns the worst solve status.
 */
int mdwf_force4d(mdwf_ctx *ctx, double *dSdU, double *S, const double *phi, int where,
                 const mdwf_solve_params *params, mdwf_solve_info *info);

/*
 * Per-kernel timing. While enabled, every kernel the context launches outside
 * a CUDA-graph capture is bracketed by two CUDA events on the launch stream
 * (solves then run without graphs). mdwf_profile_read synchronises the
 * stream, adds up the event pairs and fills up to max entries (kernels with
 * at least one launch): launches, total milliseconds and the algorithmic
 * bytes and flops of those launches (the model the roofline uses: every
 * input and output field read or written once, every link read once per
 * hop; 1320 flops per 5d site for the hopping term). reset != 0 clears the
 * accumulators afterwards.
 */
typedef struct {
    char name[40];        /* e.g. "hop_gather_f32", "hop_dag_xpay_f16n", "m5_f64", "blas_f32" */
    long long launches;
    double ms;
    double bytes;
    double flops;
} mdwf_kernel_stat;

int mdwf_profile_enable(mdwf_ctx *ctx, int enable);
int mdwf_profile_read(mdwf_ctx *ctx, mdwf_kernel_stat *out, int max, int *n_out, int reset);

/*
 * Cumulative counters since mdwf_create: kernel launches of this library
 * (a replayed CUDA graph counts every kernel it holds) and operator
 * applications M or M^dag per precision (applies[MDWF_F64 .. MDWF_F16N], one
 * count per right-hand side batch). Either pointer may be NULL.
 */
int mdwf_counters(const mdwf_ctx *ctx, long long *launches, long long applies[3]);

/*
 * Tunes the block shape of the hopping kernels (4d sites per thread block,
 * each site a whole s-column) for fields of precision prec and nrhs
 * right-hand sides: every candidate is timed with CUDA events on an M and an
 * M^dag application of the context's own scratch fields, and the fastest is
 * kept for later launches of that (prec, nrhs). Allocates scratch fields and
 * synchronises the stream. *sites_per_block receives the choice (may be NULL).
 * mdwf_set_tuning / mdwf_get_tuning store and read a choice directly, so a
 * caller can keep tuned values across runs (0 = the default shape).
 */
int mdwf_autotune(mdwf_ctx *ctx, int prec, int nrhs, int *sites_per_block);
int mdwf_set_tuning(mdwf_ctx *ctx, int prec, int nrhs, int sites_per_block);
int mdwf_get_tuning(const mdwf_ctx *ctx, int prec, int nrhs, int *sites_per_block);

/*
 * Load strategy of the FP32 and FP16+norm hopping kernels (no counterpart in
 * the paper; a GPU implementation choice), for the kernels without the input
 * gather. staged = 0 (default) prefetches the next neighbour spinor into a
 * second register buffer while the current one is transported, in every such
 * kernel. 1 copies each neighbour spinor into shared memory with
 * per-thread asynchronous copies one neighbour ahead of its use; 2 has the copy
 * engine (bulk copies, TMA) move whole neighbour s-columns of the block's sites
 * into shared memory, two hopping terms ahead, behind mbarriers; 3 is the
 * same as 0; 4 loads into registers when needed in every kernel. Results are identical (the same arithmetic in the same order).
 * prec MDWF_F64 accepts 0 only; staged = 2 with MDWF_F16N needs Ls % 4 == 0
 * (MDWF_EINVAL otherwise). The waits of mode 2 are bounded: one that gives up
 * marks the context, and the next mdwf_cgne or mdwf_device_status returns
 * MDWF_ETIMEOUT. mdwf_get_staging reads the setting.
 */
int mdwf_set_staging(mdwf_ctx *ctx, int prec, int staged);
int mdwf_get_staging(const mdwf_ctx *ctx, int prec, int *staged);

/*
 * Waits for the work enqueued on the context's stream and reports whether a
 * bounded device-side wait gave up since the last report: MDWF_ETIMEOUT if
 * one did (the mark is cleared), MDWF_ECUDA on a CUDA error, else MDWF_OK.
 */
int mdwf_device_status(mdwf_ctx *ctx);

/*
 * Self-test of the bounded device-side wait: one thread waits on an mbarrier
 * that expects two arrivals, of which `arrivals` (0, 1 or 2) are made. With
 * fewer than two the wait gives up after its limit (well under a second)
 * and the call returns MDWF_ETIMEOUT; with two it returns MDWF_OK. The
 * context stays usable either way.
 */
int mdwf_selftest_wait(mdwf_ctx *ctx, int arrivals);

/* Human-readable name of a status code (static string). */
const char *mdwf_strerror(int status);

/* Text of the last CUDA error seen by this thread, or "" (static/thread-local string). */
const char *mdwf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MDWF_H */
