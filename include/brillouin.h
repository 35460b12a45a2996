/*
 * brillouin.h -- C ABI of the GB300 (sm_103a) Brillouin Dirac operator library.
 *
 * The operator (Duerr & Koutsou, "Brillouin improvement for Wilson fermions",
 * Eq. def_pref with c_SW = 0, a = 1):
 *
 *   D = sum_mu gamma_mu nabla^iso_mu - (1/2) Laplacian^bri + m0
 *
 * written in the rho/lambda class form of Sec. 8 with the der_iso / lap_bri
 * weights of Tab. rholambda:
 *
 *   (D psi)(x) = (m0 + lambda_0) psi(x)
 *              + sum_{d in {-1,0,1}^4, d != 0} s_d(x) [lambda_n 1 + rho_n sum_mu d_mu gamma_mu]
 *                                                      (x) W_d(x) psi(x+d),     n = |d|_1
 *
 *   lambda = (240, -8, -4, -2, -1)/128,  rho_1..4 = (64, 16, 4, 1)/432.
 *
 * W_{+-mu}(x) are the links U_mu(x), U_mu(x-mu)^dagger; every off-axis hop is
 * the sum over all shortest lattice paths x -> x+d, back-projected to SU(3) in
 * a single step (Sec. 5.1), with the projection of Eq. proj_SU (Sec. 5.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Lattice: extents L[0..3] (x, y, z, t), each >= 3; site index
 *    x + L0*(y + L1*(z + L2*t)).  Links are periodic.  The fermion field gets
 *    the boundary phase bc_sign[mu] (+1 or -1) on every hop that wraps around
 *    direction mu; the default is antiperiodic in t, {1, 1, 1, -1}.
 *  - Gauge field U: device memory, [V][4][3][3] complex128 (interleaved
 *    re/im, row-major 3x3), U[x][mu] connecting x to x+mu.
 *  - Spinors: device memory, [nrhs][V][4][3] complex (spin, colour) with
 *    interleaved re/im, element type complex128 for BRI_F64 and complex64 for
 *    BRI_F32 and BRI_F16 (BRI_F16 means half-precision hopping fields with
 *    FP32 spinors and FP32 arithmetic).  BRI_F16H (apply, overlap kernel and
 *    bri_convert_spinor only) means half-precision hopping fields with FP16
 *    spinors: each right-hand side is bri_h16_field_bytes(V) bytes, [V][4][3]
 *    half2 (re, im) followed by [V] float scales (one per site; entry = half
 *    value x scale, the scale a power of two with the site's largest
 *    component in [scale/2, scale)) and unused padding to a multiple of 16
 *    bytes; arithmetic in FP32.
 *  - Gamma matrices: the hermitian chiral (DeGrand-Rossi) basis,
 *    gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1).
 *  - Ownership: the caller owns every buffer passed in; the library owns the
 *    hopping fields, its work spaces and its tuning cache, all released by
 *    bri_destroy.  Nothing is retained from caller buffers beyond the call,
 *    except that bri_build_hops keeps a device copy of U (used by the force).
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  All
 *    work is enqueued on it; calls return once the work is enqueued, except
 *    where stated (solvers synchronise the stream to read convergence data).
 *  - Errors: every call returns a bri_status; no exception crosses the ABI.
 *    bri_last_error(ctx) returns a human-readable description of the last
 *    failure on that context.  A CUDA launch or runtime failure is returned as
 *    BRI_ECUDA.  Arguments are validated before any work is enqueued.
 *  - Thread safety: one context must not be used from two host threads at
 *    once.
 */
#ifndef BRILLOUIN_H
#define BRILLOUIN_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BRI_OK = 0,
    BRI_EINVAL = -1,      /* invalid argument (null pointer, bad size, misaligned buffer) */
    BRI_ENOMEM = -2,      /* device allocation failed */
    BRI_ECUDA = -3,       /* CUDA runtime / launch error */
    BRI_ENOTCONV = -4,    /* solver reached maxit without meeting tol */
    BRI_EBREAKDOWN = -5,  /* BiCGstab breakdown (rho or omega vanished) */
    BRI_ENAN = -6,        /* NaN / Inf met in a solve */
    BRI_ETIMEOUT = -7,    /* a bounded device-side wait gave up */
    BRI_ESTATE = -8       /* call out of order (e.g. apply before build_hops) */
} bri_status;

typedef enum { BRI_F64 = 0, BRI_F32 = 1, BRI_F16 = 2, BRI_F16H = 3 } bri_prec;

/* storage of the hopping fields (each W_d(x) is in SU(3), Sec. 5.2) */
typedef enum {
    BRI_LINK_FULL = 0,   /* 18 reals */
    BRI_LINK_2ROW = 1,   /* 12 reals, third row = conj(row0 x row1) */
    BRI_LINK_8PARAM = 2  /* 8 reals: U01, U02, U10, arg U00, arg U20 */
} bri_comp;

typedef struct {
    int L[4];       /* extents, each >= 3 */
    int bc_sign[4]; /* fermion boundary phase per direction, +1 or -1 */
} bri_lattice;

typedef struct bri_ctx bri_ctx; /* opaque */

/* Create a context for one lattice on the current CUDA device.
 * Errors: BRI_EINVAL (null pointers, extent < 3, |bc_sign| != 1, volume
 * beyond 2^31 sites), BRI_ENOMEM. */
bri_status bri_create(const bri_lattice *lat, bri_ctx **out);

/* Release the context and every device buffer it owns.  Null is allowed. */
bri_status bri_destroy(bri_ctx *ctx);

/* Build the 80 path-averaged hopping fields from the links U (Sec. 5.1,
 * Sec. 5.2): path sums over all shortest paths for the 2-, 3- and 4-hop
 * offsets (2, 6 and 24 paths), one SU(3) back-projection each (Eq. proj_SU),
 * computed in FP64.  The 40 fields W_d with the last non-zero component of d
 * positive are stored; W_{-d}(x) = W_d(x-d)^dagger supplies the rest.
 * The FP64 fields are always kept; if prec != BRI_F64 a copy in (prec, comp)
 * is stored as well.  U: device, [V][4][3][3] complex128, 16-byte aligned;
 * the library keeps its own copy.  Errors: BRI_EINVAL, BRI_ENOMEM, BRI_ECUDA. */
bri_status bri_build_hops(bri_ctx *ctx, const double *U, bri_prec prec, bri_comp comp, void *stream);

/* Store an additional (prec, comp) copy of the FP64 hopping fields built by
 * the last bri_build_hops (no recomputation).  Errors: BRI_ESTATE if no
 * fields were built, BRI_EINVAL, BRI_ENOMEM. */
bri_status bri_store_hops(bri_ctx *ctx, bri_prec prec, bri_comp comp, void *stream);

/* Copy the 40 stored FP64 hopping fields to out: device, [V][40][3][3]
 * complex128; field j has offset d = digits of (j + 41) in base 3 minus 1,
 * x fastest (d_mu = ((j+41) / 3^mu) % 3 - 1).  Errors: BRI_ESTATE, BRI_EINVAL. */
bri_status bri_get_hops(bri_ctx *ctx, double *out, void *stream);

/* out = D psi (dagger = 0) or D^dagger psi = gamma_5 D gamma_5 psi (dagger = 1,
 * Sec. 1), for nrhs right-hand sides, with the hopping fields stored in prec
 * (for BRI_F32 / BRI_F16 the compression of the last build/store in that
 * precision).  in/out: device, [nrhs][V][4][3] complex (see conventions),
 * 16-byte aligned, must not overlap.  Errors: BRI_EINVAL, BRI_ESTATE
 * (fields of that precision not built), BRI_ECUDA. */
bri_status bri_apply(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int dagger,
                     bri_prec prec, void *stream);

/* bri_apply with in and out in HOST memory: the library copies the input to
 * its own device buffers in slabs of time slices, computes each slab of the
 * output once the slab and its neighbours in t have arrived, and copies it
 * back, so host-to-device copies, the stencil and device-to-host copies of
 * different slabs overlap.  Page-locked host buffers (cudaHostAlloc or
 * cudaHostRegister) are needed for the copies to run asynchronously; pageable
 * buffers work but serialise.  Asynchronous on `stream`: the host buffers must
 * stay valid, and out unread, until the stream has been synchronised.  The
 * device staging buffers (2 x nrhs spinor fields) are owned by the context.
 * Errors: as bri_apply. */
bri_status bri_apply_host(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int dagger,
                          bri_prec prec, void *stream);

/* Hermitian overlap kernel H = gamma_5 (D_B - rho), D_B at m0 = 0 (the shifted
 * kernel of Sec. 7.4 entering Eq. def_over; rho = 1 there).  Same buffers and
 * errors as bri_apply. */
bri_status bri_apply_overlap_kernel(bri_ctx *ctx, void *out, const void *in, int nrhs, double rho,
                                    bri_prec prec, void *stream);

typedef struct {
    int iters;          /* inner (or only) BiCGstab iterations */
    int outer_iters;    /* defect-correction cycles (0 for mode 0) */
    double true_resid;  /* ||b - D x|| / ||b||, recomputed in FP64 */
    double seconds;     /* wall time of this right-hand side's solve */
    bri_status status;  /* BRI_OK, BRI_ENOTCONV, BRI_EBREAKDOWN or BRI_ENAN */
} bri_solve_info;

/* Solve D x = b (BiCGstab, Sec. 6.4) for nrhs right-hand sides to the true
 * relative residual tol.
 *   mode 0: FP64 BiCGstab, one right-hand side after the other.
 *   mode 1: FP64 defect correction around an FP32 BiCGstab (FP32 hops as
 *           last stored, FP32 spinors, FP64 dot products).
 *   mode 2: as mode 1 with the FP16 hopping fields.
 *   Modes 1 and 2 solve the right-hand sides one after the other.
 *   mode 3: batched: all nrhs right-hand sides advance together through one
 *           multi-RHS apply per step (mode-2 inner precision), each with its
 *           own BiCGstab scalars, inside one CUDA graph per block of steps.
 *   mode 4: as mode 3 with the FP32 hopping fields (mode-1 inner precision).
 * x: device, [nrhs][V][4][3] complex128, used as the initial guess and
 * overwritten with the solution; b: device, same layout.  info: host array of
 * nrhs entries (may be null).  Synchronises the stream.  Returns BRI_OK when
 * every right-hand side converged, otherwise the first failing status (a
 * right-hand side that fails to converge does not stop the others; BRI_EINVAL
 * for a mode outside 0..4). */
bri_status bri_solve(bri_ctx *ctx, double *x, const double *b, int nrhs, double m0, double tol,
                     int maxit, int mode, bri_solve_info *info, void *stream);

/* Fermion force dU += d Re(chi^dagger D[U] psi) / dU for the U of the last
 * bri_build_hops, with the convention dU = df/dRe U + i df/dIm U per link
 * entry, U treated as an unconstrained complex matrix (the hops of Sec. 5.1
 * and the projection of Sec. 5.2 differentiated exactly).
 * recompute_hops = 1 recomputes the projected fields instead of reading the
 * stored FP64 ones.  dU: device [V][4][3][3] complex128 (accumulated);
 * chi, psi: device [V][4][3] complex128.  Errors: BRI_ESTATE, BRI_EINVAL,
 * BRI_ENOMEM, BRI_ECUDA. */
bri_status bri_force(bri_ctx *ctx, double *dU, const double *chi, const double *psi, double m0,
                     int recompute_hops, void *stream);

/* dU += d( phi^dagger (D^dagger D)^{-1} phi ) / dU = -2 d Re(Y^dagger D X)/dU
 * with X = (D^dagger D)^{-1} phi, Y = D X, both solved to the true FP64
 * relative residual tol: by FP64 defect correction around FP32 BiCGstab when
 * FP32 hopping fields are stored (bri_solve mode 1), else by FP64 BiCGstab.
 * phi: device [V][4][3] complex128.  info (host, may be null) receives the
 * second solve's data.  Synchronises the stream. */
bri_status bri_force_inverse(bri_ctx *ctx, double *dU, const double *phi, double m0, double tol,
                             int maxit, bri_solve_info *info, void *stream);

/* The quantity whose link derivative bri_force_inverse gives, with its
 * derivatives (the pseudofermion action of the second adjoint quantity):
 *   S = phi^dagger (D^dagger D)^{-1} phi = |Y|^2,  X = (D^dagger D)^{-1} phi,
 *   Y = D X,  dS/dU = -2 d Re(Y^dagger D X)/dU  (convention of bri_force),
 *   dS/dRe phi + i dS/dIm phi = 2 X.
 * The two solves run as in bri_force_inverse (FP64 defect correction when
 * FP32 fields are stored, else FP64 BiCGstab) to the true relative residual
 * tol.  S: host, 1 double (may be null);  X: device [V][4][3] complex128
 * output (may be null);  dU: device [V][4][3][3] complex128, accumulated
 * (+=; may be null);  phi: device [V][4][3] complex128.  info (host, may be
 * null) receives the second solve's data.  Synchronises the stream.
 * Errors: BRI_EINVAL (misaligned pointers, tol <= 0, maxit < 1), BRI_ESTATE
 * (no fields built; dU with the clover term on), the solver's status. */
bri_status bri_inverse_action(bri_ctx *ctx, double *S, double *X, double *dU, const double *phi, double m0,
                              double tol, int maxit, bri_solve_info *info, void *stream);

/* Batched SU(3) projection Y_i = P_SU(3)(A_i) (Eq. proj_SU), FP64.
 * A, Y: device, [n][3][3] complex128 (may alias).  Errors: BRI_EINVAL. */
bri_status bri_project_su3(bri_ctx *ctx, double *Y, const double *A, long n, void *stream);

/* Hop precompute that allocates nothing: the stateless, allocation-free form
 * of bri_build_hops + bri_get_hops, for callers that cannot allocate device
 * memory (an application whose own pool owns all device memory, an embedding
 * that must not grow its device footprint while running).  The paper has no
 * counterpart to this entry point.
 *   lat: the lattice, at most 4096 sites;  U: device, [V][4][3][3] complex128;
 *   W:   device output, [V][40][3][3] complex128, the layout of bri_get_hops.
 * The path sums live in a fixed scratch array inside the library (81 x 144
 * bytes per site for 4096 sites, about 45.6 MiB, held on every GPU that loads
 * the library until the process exits).  All calls share it and it keeps the
 * last call's contents (nothing needs to start at zero); calls that overlap
 * on the GPU race, so the caller serialises them.  The first call on a device
 * looks up the array's device address with that device current: make it
 * before any stream capture.  The address is looked up again after the
 * device's context was destroyed and re-created (cudaDeviceReset).  Errors
 * (message via bri_last_error(NULL)): BRI_EINVAL (null or misaligned
 * pointers, extents < 3, bad bc_sign, more than 4096 sites), BRI_ECUDA. */
bri_status bri_build_hops_noalloc(const bri_lattice *lat, const double *U, double *W, void *stream);

/* Measured arithmetic peak of the current GPU in TFLOP/s (FMA = 2 flops):
 * independent FMA chains on every SM timed with CUDA events, the fastest of
 * five launches.  prec = BRI_F32: packed FP32 FMAs (fma.rn.f32x2, the form
 * of the FP32 stencil); BRI_F64: FP64 FMAs.  These are the ALU rooflines the
 * stencil's flop rate is compared with.  The paper has no counterpart.
 * Synchronises the device's default stream.  Errors: BRI_EINVAL, BRI_ECUDA
 * (message via bri_last_error(NULL)). */
bri_status bri_alu_peak(int prec, double *tflops);

/* Bytes of one right-hand side in the BRI_F16H spinor storage (see the
 * conventions): 48 V + 4 V rounded up to a multiple of 16.  No device work. */
size_t bri_h16_field_bytes(int V);

/* Convert nrhs spinor fields between storages: BRI_F64 (complex128), BRI_F32
 * (complex64) and BRI_F16H (FP16 + per-site scale, rounded to nearest).
 * dst, src: device buffers of the sizes the storages imply; must not
 * overlap.  Asynchronous on stream.  Errors: BRI_EINVAL (null or misaligned
 * pointers, nrhs < 1, another storage, overlap), BRI_ECUDA. */
bri_status bri_convert_spinor(bri_ctx *ctx, void *dst, bri_prec dst_prec, const void *src, bri_prec src_prec,
                              int nrhs, void *stream);

/* result[0] + i result[1] = <a, b> = sum conj(a) b over nrhs spinor fields
 * (the dot product of the Krylov solvers, FP64 accumulation: per-block partial
 * sums added in block order, deterministic).  a, b: device, [nrhs][V][4][3]
 * complex in the storage of prec; result: host, 2 doubles.  Synchronises the
 * stream.  Errors: BRI_EINVAL. */
bri_status bri_cdot(bri_ctx *ctx, double *result, const void *a, const void *b, int nrhs, bri_prec prec,
                    void *stream);

/* Class weights of the operator (Sec. 8): D(x, x+d) = s_d(x) [lambda_n +
 * rho_n sum_mu d_mu gamma_mu] (x) W_d(x) for n = |d|_1 = 1..4 and
 * D(x, x) = m0 + lambda_0.  The default is the der_iso / lap_bri column of
 * Tab. rholambda (the Brillouin operator); the other columns (Wilson:
 * lambda = (4, -1/2, 0, 0, 0), rho_1 = 1/2; the hypercube operator) or any
 * other member of the class can be set.  Classes with lambda_n = rho_n = 0
 * are skipped by the apply.  lambda, rho: host arrays of 5 doubles (rho[0]
 * ignored).  Applies to every later apply, solve and force on ctx.
 * Errors: BRI_EINVAL (null or non-finite weights). */
bri_status bri_set_weights(bri_ctx *ctx, const double *lambda, const double *rho);
bri_status bri_get_weights(bri_ctx *ctx, double *lambda, double *rho);

/* ---- link smearing and the clover term (Eq. def_ape, Eq. def_pref) --------- */

/* nsteps steps of APE smearing (Eq. def_ape):
 *   V_mu(x) = P_SU(3){ (1 - alpha) 1 + alpha/6 sum_{+-nu != mu}
 *             U_nu(x) U_mu(x+nu) U_nu(x+mu)^dagger U_mu(x)^dagger } U_mu(x)
 * (the paper uses alpha = 0.72 and 1 or 5 steps), P the projection of
 * Eq. proj_SU, FP64.  Feeding V to bri_build_hops gives the fat-link operator
 * of Sec. 5 (every thin link replaced, the clover term included).  U, V:
 * device [V][4][3][3] complex128, distinct buffers; nsteps = 0 copies.
 * Steps beyond the first use a temporary of the size of U (allocated and freed
 * inside the call, which then synchronises the stream).  alpha in [0, 1],
 * nsteps in [0, 1000].  Errors: BRI_EINVAL, BRI_ENOMEM. */
bri_status bri_ape_smear(bri_ctx *ctx, double *V, const double *U, double alpha, int nsteps, void *stream);

/* Switch on (csw != 0) or off (csw = 0) the clover term of Eq. def_pref,
 *   -(c_SW/2) sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x) delta_{x,y},
 * sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], F_{mu nu} = (Q - Q^dagger)/(8 i)
 * the hermitian clover-leaf field strength (Q: the four plaquettes of the
 * (mu, nu) plane around x, all oriented mu -> nu), from the links of the last
 * bri_build_hops (rebuilt by every later bri_build_hops).  The paper takes the
 * tree-level value c_SW = 1 (Sec. 5.3).  Every later apply (D, D^dagger, the
 * overlap kernel, all precisions), solve and overlap setup includes the term;
 * the force calls return BRI_ESTATE while it is on.  Stored per site as two
 * hermitian 6x6 chiral blocks (576 B FP64 + 288 B FP32).  Errors: BRI_EINVAL,
 * BRI_ESTATE (no links), BRI_ENOMEM. */
bri_status bri_set_clover(bri_ctx *ctx, double csw, void *stream);

/* ---- spectra and the overlap operator (Sec. 7) ------------------------------ */

typedef struct {
    int nconv;        /* wanted Ritz pairs whose residual estimate met tol */
    int krylov_dim;   /* Lanczos vectors built */
    int applies;      /* stencil applications */
    double max_resid; /* largest relative residual estimate |A y - theta y| / theta */
    double seconds;
    bri_status status;
} bri_eig_info;

/* Extremal eigenvalues of A = D(m0)^dagger D(m0) = (gamma5 D(m0))^2 -- the
 * Ritz values of the Lanczos process on A that Sec. 7.4 compares between
 * kernels (at m0 = -rho, A is the square of the shifted hermitian kernel).
 * Lanczos with full reorthogonalisation; the basis (max_krylov + 1 FP64
 * vectors of 12 V complex numbers) is allocated for the call and freed.
 * evals: host, nev doubles, the nev smallest eigenvalues ascending; lmax: host
 * double or NULL, the largest; evecs: device [nev][V][4][3] complex128 or NULL,
 * the Ritz vectors (unit norm).  Converged when every residual estimate is
 * below tol x its Ritz value.  prec: BRI_F64 (FP64 fields, vectors and
 * arithmetic), or BRI_F32 / BRI_F16 (the Lanczos vectors and applies in FP32
 * with the FP32 / FP16 fields, FP64 sums: about 100x faster on this GPU, Ritz
 * values good to about 1e-7 relative, so tol below ~1e-6 cannot be met).
 * Uses the class weights set on ctx.  Synchronises the stream.  nev in
 * [1, 64], max_krylov in [nev + 1, 12 V].  Errors: BRI_EINVAL, BRI_ESTATE (no
 * fields of that precision), BRI_ENOTCONV (max_krylov reached; evals hold the
 * last Ritz values), BRI_ENOMEM. */
bri_status bri_eigs_ddag_d(bri_ctx *ctx, double *evals, double *lmax, double *evecs, int nev, double m0,
                           int max_krylov, double tol, bri_prec prec, bri_eig_info *info, void *stream);

typedef struct {
    int nlow;          /* deflated eigenpairs of H */
    int degree;        /* degree of the Chebyshev polynomial p, p(x) ~ 1/sqrt(x) */
    double lo, hi;     /* interval of H^2 (deflated) on which p is built */
    double err_bound;  /* max over [lo, hi] of |1 - sqrt(x) p(x)| (dense grid) */
    double defl_resid; /* largest ||H z - lambda z|| of the deflated pairs */
    int krylov_dim;    /* Lanczos vectors built, both runs */
    int applies;       /* stencil applications of the setup */
    double seconds;
    bri_status status;
} bri_overlap_info;

/* Prepare the overlap operator of Eq. def_over on the current operator D
 * (links and class weights of ctx): H = gamma5 (D - rho),
 *   sign(H) psi = sum_i sign(lambda_i) z_i <z_i, psi> + H p(P H^2 P) P psi,
 * with (lambda_i, z_i) the nlow eigenpairs of H of smallest |lambda| (Lanczos
 * on H^2 to relative residual tol, then Rayleigh-Ritz with H), P the projector
 * orthogonal to them, and p the Chebyshev interpolant of 1/sqrt(x) on
 * [lo, hi] (the rest of the spectrum of H^2: the extreme Ritz values, minus /
 * plus their residuals, of a second Lanczos run on the deflated operator to
 * relative residual max(tol, 1e-4), widened by 2%) of the smallest degree
 * whose sign error
 * max |1 - sqrt(x) p(x)| is <= eps.  prec: arithmetic of the polynomial
 * (BRI_F64, or BRI_F32 / BRI_F16 with the FP32 / FP16 hopping fields of that
 * precision).  With BRI_F32 / BRI_F16 the Lanczos runs, the Rayleigh-Ritz step
 * and the deflation vectors use that precision too (tol is raised to at least
 * 1e-6; the deflated eigenvalues are then good to about 1e-7), while the
 * projection of the input and the final sum stay FP64.  State is kept in ctx
 * until the next setup; changing the links or weights invalidates it.
 * Synchronises the stream.  rho in (0, 2), nlow in [0, 64], eps in
 * [1e-14, 0.1].  Errors: BRI_EINVAL (also when the degree would exceed
 * 60000), BRI_ESTATE, BRI_ENOTCONV, BRI_ENOMEM. */
bri_status bri_overlap_setup(bri_ctx *ctx, double rho, int nlow, double eps, int max_krylov, double tol,
                             bri_prec prec, bri_overlap_info *info, void *stream);

/* The deflated eigenpairs of the last setup: lambda (host, nlow doubles,
 * ascending |lambda|) and/or vecs (device [nlow][V][4][3] complex128); either
 * may be NULL.  Errors: BRI_ESTATE (no valid setup). */
bri_status bri_overlap_modes(bri_ctx *ctx, double *lambda, double *vecs, void *stream);

/* out = sign(H) in (bri_apply_sign) or out = D_ov,m in with
 * D_ov,m = (1 - m / (2 rho)) rho [1 + gamma5 sign(H)] + m (bri_apply_overlap,
 * Eq. def_over and Eq. def_mass, lattice spacing 1).  in, out: device
 * [nrhs][V][4][3] complex128, distinct.  Errors: BRI_EINVAL, BRI_ESTATE. */
bri_status bri_apply_sign(bri_ctx *ctx, double *out, const double *in, int nrhs, void *stream);
bri_status bri_apply_overlap(bri_ctx *ctx, double *out, const double *in, int nrhs, double m, void *stream);

/* Tune the launch shape of the apply kernels for (prec, nrhs) on this
 * lattice (timed with CUDA events, result cached in the context and, when the
 * environment variable BRI_TUNE_CACHE names a file, in that file).
 * Requires the fields of that precision.  Synchronises the stream. */
bri_status bri_tune(bri_ctx *ctx, bri_prec prec, int nrhs, void *stream);

/* Set / read the launch shape of the apply kernels for (prec, nrhs) (what
 * bri_tune chooses): threads per block of the plain kernel (32..1024, rounded
 * down to a multiple of 32, clamped to the kernel's limit at launch), or 0 for
 * the shared-memory tiled kernel (FP32 spinors; extents multiples of
 * 8, 4, 2, 2; otherwise 0 falls back to 128 threads).  Adding 2048 selects
 * the L2 link-prefetch variant of the plain FP32 kernel, adding 4096
 * the cp.async shared-memory link-prefetch variant (at most 256 threads),
 * adding 6144 the site-pair kernel (two sites per thread, full and 2-row
 * storage with an even t extent, its interleaved copy of the fields built on
 * first use; otherwise the plain kernel), adding 8192 the
 * plain kernel without the separate accumulator for the +-i gamma entries,
 * adding 10240 the L2 link-prefetch kernel that combines the hops d and -d
 * before their gamma terms, adding 12288 that kernel held to 128 registers,
 * adding 14336 the same pair loop with the gamma terms after the spin loop,
 * 18432 the loop of 10240 with the per-site part of the link addresses
 * computed once and the next pair's neighbours carried over, 20480 the loop
 * of 10240 with the links staged in shared memory by 1-D bulk copies
 * (cp.async.bulk into a ring of stages per warp, completion counted on an
 * mbarrier; at most 256 threads; with 32 threads and an x extent of 32 one
 * warp per x line), 22528 the one-warp-per-x-line loop with the neighbour
 * spinor lines staged by bulk copies as well (x extent 32 only, otherwise as
 * 20480; one warp per block whatever the low bits, which select one buffer per
 * spinor line when 64 and a two-deep ring of them otherwise).  A bulk-copy wait that has not completed after
 * one second gives up, and the next apply call on the context then returns
 * BRI_ETIMEOUT,
 * 16384 the tensor-core multi-RHS kernel (Sec. 8 class form as one complex
 * (15 x 240) x (240 x 4 nrhs) product per site on mma.sync with FP16
 * operands and FP32 accumulation; full link storage only, otherwise the
 * untuned shape; accuracy that of FP16 operands, about 1e-4 of max |out|;
 * the tuner considers it for BRI_F16 fields and nrhs >= 2 only, the accuracy
 * class it shares).  For 16384 the low bits give the right-hand sides one
 * warp takes per pass (an even number 2..12; 0 or anything else: 12).
 * bri_get_threads returns the current choice or a negative bri_status;
 * untuned: the unrolled kernel at 128 threads (BRI_F64); on an x extent of
 * 32, 22528 + 64 (FP32 and FP16 fields); otherwise 128 threads with variant 10240 (FP32 full fields), 18432
 * (FP32 2-row, FP16 full and 2-row fields) or 12288 (8-parameter fields).  bri_set_threads returns BRI_EINVAL for nrhs < 1, a
 * negative value, 1..31 or more than 1024 threads (other than with 16384), or
 * a variant above 22528. */
bri_status bri_set_threads(bri_ctx *ctx, bri_prec prec, int nrhs, int threads);
int bri_get_threads(bri_ctx *ctx, bri_prec prec, int nrhs);

/* Number of kernels this context launched so far (diagnostics). */
long bri_kernel_launches(bri_ctx *ctx);

/* Diagnostics of the bounded waits: with on != 0 the bulk-copy applies (launch
 * variants 20480 and 22528) announce 16 bytes more to their first link
 * stage's barrier than its copies deliver, so every warp's wait runs out after
 * one second, the kernel drains its other copies and returns, and the next
 * apply call returns BRI_ETIMEOUT (and clears the flag).  No memory is accessed out of bounds
 * and nothing is left in flight.  on = 0 restores normal operation.
 * Errors: BRI_EINVAL (null ctx). */
bri_status bri_debug_stall(bri_ctx *ctx, int on);

/* Description of the last error on ctx (or of the last bri_create failure
 * when ctx is null).  The string stays valid until the next call on ctx. */
const char *bri_last_error(bri_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* BRILLOUIN_H */
