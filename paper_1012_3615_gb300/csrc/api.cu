// C ABI entry points (include/brillouin.h): argument validation, context
// management, the launch-shape tuner and dispatch to the kernels.
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "ctx.h"
#include "tile.cuh"

using namespace bri;

static std::string g_create_error;

// out = gamma_5 in (spins 2, 3 negated) or out = a * in, over n sites
__global__ void k_gamma5_scale(double2 *out, const double2 *in, size_t n, int g5, double a) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * 12; i += (size_t)gridDim.x * blockDim.x) {
        double f = g5 ? ((i % 12) >= 6 ? -1.0 : 1.0) : a;
        out[i] = make_double2(f * in[i].x, f * in[i].y);
    }
}
static bri_status gamma5_scale(bri_ctx *ctx, double2 *out, const double2 *in, int g5, double a, cudaStream_t s) {
    k_gamma5_scale<<<608, 256, 0, s>>>(out, in, (size_t)ctx->g.V, g5, a);
    BRI_LAUNCHED(ctx);
    return BRI_OK;
}

bri_status bri_fail(bri_ctx *ctx, bri_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    else g_create_error = msg;
    return st;
}

static cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

static bri_status check_prec(bri_ctx *ctx, bri_prec p) {
    if (p != BRI_F64 && p != BRI_F32 && p != BRI_F16) return bri_fail(ctx, BRI_EINVAL, "invalid precision");
    return BRI_OK;
}

// ---- tuning cache file: one "key threads" line per entry ----------------------
// a launch shape bri_set_threads accepts: threads per block in the low 11 bits
// (0 or 32..1024; for the tensor-core variant 8 the RHS per warp pass), kernel
// variant above them (0..11)
static bool valid_shape(int threads) {
    const int thr = threads & 2047, variant = threads >> 11;
    return threads >= 0 && variant <= 11 && (variant == 8 || !((thr > 0 && thr < 32) || thr > 1024));
}
static void tune_load(bri_ctx *ctx) {
    const char *f = getenv("BRI_TUNE_CACHE");
    if (!f || !*f) return;
    std::ifstream in(f);
    std::string key;
    int thr;
    while (in >> key >> thr)
        if (valid_shape(thr)) ctx->tune[key] = thr;
}
static void tune_save_entry(const std::string &key, int thr) {
    const char *f = getenv("BRI_TUNE_CACHE");
    if (!f || !*f) return;
    std::ofstream out(f, std::ios::app);
    out << key << " " << thr << "\n";
}

extern "C" {

bri_status bri_create(const bri_lattice *lat, bri_ctx **out) {
    if (!lat || !out) return bri_fail(nullptr, BRI_EINVAL, "null argument");
    long long V = 1;
    for (int mu = 0; mu < 4; mu++) {
        if (lat->L[mu] < 3) return bri_fail(nullptr, BRI_EINVAL, "lattice extents must be >= 3");
        if (lat->bc_sign[mu] != 1 && lat->bc_sign[mu] != -1)
            return bri_fail(nullptr, BRI_EINVAL, "bc_sign must be +1 or -1");
        V *= lat->L[mu];
    }
    if (V * 12 >= (1LL << 31)) return bri_fail(nullptr, BRI_EINVAL, "lattice volume too large");
    bri_ctx *ctx = new bri_ctx();
    for (int mu = 0; mu < 4; mu++) {
        ctx->g.L[mu] = lat->L[mu];
        ctx->g.bc[mu] = lat->bc_sign[mu];
    }
    ctx->g.V = (int)V;
    ctx->g.s0 = 0;
    ctx->g.s1 = (int)V;
    {
        double lam[5], rho[5];
        for (int n = 0; n < 5; n++) {
            lam[n] = lambda_w(n);
            rho[n] = rho_w(n);
        }
        geom_set_weights(ctx->g, lam, rho);
    }
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        delete ctx;
        return bri_fail(nullptr, BRI_ECUDA, "no CUDA device");
    }
    if (cudaHostAlloc((void **)&ctx->werr_h, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&ctx->g.werr, ctx->werr_h, 0) != cudaSuccess) {
        cudaFreeHost(ctx->werr_h);
        delete ctx;
        return bri_fail(nullptr, BRI_ENOMEM, "host-mapped status word");
    }
    *ctx->werr_h = 0;
    tune_load(ctx);
    *out = ctx;
    return BRI_OK;
}

bri_status bri_destroy(bri_ctx *ctx) {
    if (!ctx) return BRI_OK;
    bri_solver_free(ctx);
    bri_overlap_free(ctx);
    bri_host_apply_free(ctx);
    cudaFree(ctx->clov64);
    cudaFree(ctx->clov32);
    cudaFree(ctx->tc_amax);
    cudaFree(ctx->tc_f);
    cudaFree(ctx->U);
    cudaFree(ctx->hops64);
    cudaFreeHost(ctx->werr_h);
    for (LinkStore *st : {&ctx->f32, &ctx->f16, &ctx->p32, &ctx->p16}) {
        cudaFree(st->a);
        cudaFree(st->b);
    }
    delete ctx;
    return BRI_OK;
}

bri_status bri_build_hops(bri_ctx *ctx, const double *U, bri_prec prec, bri_comp comp, void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (!U || !bri_aligned16(U)) return bri_fail(ctx, BRI_EINVAL, "U must be a 16-byte aligned device pointer");
    BRI_RETURN_IF(check_prec(ctx, prec));
    if (comp != BRI_LINK_FULL && comp != BRI_LINK_2ROW && comp != BRI_LINK_8PARAM)
        return bri_fail(ctx, BRI_EINVAL, "invalid compression");
    cudaStream_t s = as_stream(stream);
    const size_t bytes = sizeof(double2) * 36 * (size_t)ctx->g.V;
    if (!ctx->U) BRI_TRY_CUDA(ctx, cudaMalloc(&ctx->U, bytes));
    BRI_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->U, U, bytes, cudaMemcpyDeviceToDevice, s));
    ctx->gen++;
    BRI_RETURN_IF(bri_hops_build_impl(ctx, s));
    if (ctx->csw != 0.0) BRI_RETURN_IF(bri_clover_build_impl(ctx, s));  // F from the new links
    return bri_hops_store_impl(ctx, prec, comp, s);
}

bri_status bri_store_hops(bri_ctx *ctx, bri_prec prec, bri_comp comp, void *stream) {
    if (!ctx) return BRI_EINVAL;
    BRI_RETURN_IF(check_prec(ctx, prec));
    if (comp != BRI_LINK_FULL && comp != BRI_LINK_2ROW && comp != BRI_LINK_8PARAM)
        return bri_fail(ctx, BRI_EINVAL, "invalid compression");
    if (!ctx->have64) return bri_fail(ctx, BRI_ESTATE, "no hopping fields built");
    ctx->gen++;
    return bri_hops_store_impl(ctx, prec, comp, as_stream(stream));
}

bri_status bri_get_hops(bri_ctx *ctx, double *out, void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (!out || !bri_aligned16(out)) return bri_fail(ctx, BRI_EINVAL, "out must be a 16-byte aligned device pointer");
    if (!ctx->have64) return bri_fail(ctx, BRI_ESTATE, "no hopping fields built");
    return bri_export_hops_impl(ctx, (double2 *)out, as_stream(stream));
}

static size_t spinor_bytes(bri_ctx *ctx, bri_prec prec, int nrhs) {
    if (prec == BRI_F16H) return bri_h16_bytes(ctx->g.V) * nrhs;
    return (prec == BRI_F64 ? 16 : 8) * 12 * (size_t)ctx->g.V * nrhs;
}

static bri_status check_apply(bri_ctx *ctx, void *out, const void *in, int nrhs, bri_prec prec) {
    if (!out || !in) return bri_fail(ctx, BRI_EINVAL, "null spinor pointer");
    if (!bri_aligned16(out) || !bri_aligned16(in)) return bri_fail(ctx, BRI_EINVAL, "spinors must be 16-byte aligned");
    if (nrhs < 1 || nrhs > 65535) return bri_fail(ctx, BRI_EINVAL, "nrhs must be in [1, 65535]");
    if (prec != BRI_F16H) BRI_RETURN_IF(check_prec(ctx, prec));
    const size_t bytes = spinor_bytes(ctx, prec, nrhs);
    const char *o = (const char *)out, *i = (const char *)in;
    if (o < i + bytes && i < o + bytes) return bri_fail(ctx, BRI_EINVAL, "in and out overlap");
    return BRI_OK;
}

bri_status bri_apply(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int dagger, bri_prec prec,
                     void *stream) {
    if (!ctx) return BRI_EINVAL;
    BRI_RETURN_IF(check_apply(ctx, out, in, nrhs, prec));
    if (prec == BRI_F16H) {
        if (!ctx->f16.valid) return bri_fail(ctx, BRI_ESTATE, "FP16 hopping fields not built");
        if (ctx->csw != 0.0) return bri_fail(ctx, BRI_ESTATE, "FP16 spinors with the clover term are not built");
        return bri_dslash_h16(ctx, out, in, nrhs, m0, dagger ? 1 : 0, nullptr, as_stream(stream));
    }
    return bri_dslash_impl(ctx, out, in, nrhs, m0, dagger ? 1 : 0, prec, as_stream(stream));
}

bri_status bri_apply_host(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int dagger, bri_prec prec,
                          void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (!out || !in) return bri_fail(ctx, BRI_EINVAL, "null spinor pointer");
    if (nrhs < 1 || nrhs > 65535) return bri_fail(ctx, BRI_EINVAL, "nrhs must be in [1, 65535]");
    BRI_RETURN_IF(check_prec(ctx, prec));
    const size_t bytes = (prec == BRI_F64 ? 16 : 8) * 12 * (size_t)ctx->g.V * nrhs;
    const char *o = (const char *)out, *i = (const char *)in;
    if (o < i + bytes && i < o + bytes) return bri_fail(ctx, BRI_EINVAL, "in and out overlap");
    if (prec == BRI_F64 && !ctx->have64) return bri_fail(ctx, BRI_ESTATE, "FP64 hopping fields not built");
    if (prec != BRI_F64 && !(prec == BRI_F32 ? ctx->f32 : ctx->f16).valid)
        return bri_fail(ctx, BRI_ESTATE, "hopping fields of this precision not built");
    return bri_apply_host_impl(ctx, out, in, nrhs, m0, dagger ? 1 : 0, prec, as_stream(stream));
}

bri_status bri_apply_overlap_kernel(bri_ctx *ctx, void *out, const void *in, int nrhs, double rho, bri_prec prec,
                                    void *stream) {
    if (!ctx) return BRI_EINVAL;
    BRI_RETURN_IF(check_apply(ctx, out, in, nrhs, prec));
    if (prec == BRI_F16H) {
        if (!ctx->f16.valid) return bri_fail(ctx, BRI_ESTATE, "FP16 hopping fields not built");
        if (ctx->csw != 0.0) return bri_fail(ctx, BRI_ESTATE, "FP16 spinors with the clover term are not built");
        return bri_dslash_h16(ctx, out, in, nrhs, -rho, 2, nullptr, as_stream(stream));
    }
    return bri_dslash_impl(ctx, out, in, nrhs, -rho, 2, prec, as_stream(stream));
}

size_t bri_h16_field_bytes(int V) { return V > 0 ? bri_h16_bytes(V) : 0; }

bri_status bri_convert_spinor(bri_ctx *ctx, void *dst, bri_prec dst_prec, const void *src, bri_prec src_prec,
                              int nrhs, void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (!dst || !src || !bri_aligned16(dst) || !bri_aligned16(src))
        return bri_fail(ctx, BRI_EINVAL, "dst and src must be 16-byte aligned device pointers");
    if (nrhs < 1 || nrhs > 65535) return bri_fail(ctx, BRI_EINVAL, "nrhs must be in [1, 65535]");
    auto fmt = [](bri_prec p) { return p == BRI_F64 ? 0 : p == BRI_F32 ? 1 : p == BRI_F16H ? 3 : -1; };
    if (fmt(dst_prec) < 0 || fmt(src_prec) < 0)
        return bri_fail(ctx, BRI_EINVAL, "spinor storages are BRI_F64, BRI_F32 and BRI_F16H");
    const size_t db = spinor_bytes(ctx, dst_prec, nrhs), sb = spinor_bytes(ctx, src_prec, nrhs);
    const char *d = (const char *)dst, *c = (const char *)src;
    if (d < c + sb && c < d + db) return bri_fail(ctx, BRI_EINVAL, "dst and src overlap");
    return bri_convert_spinor_impl(ctx, dst, fmt(dst_prec), src, fmt(src_prec), nrhs, as_stream(stream));
}

bri_status bri_solve(bri_ctx *ctx, double *x, const double *b, int nrhs, double m0, double tol, int maxit, int mode,
                     bri_solve_info *info, void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (!x || !b || !bri_aligned16(x) || !bri_aligned16(b))
        return bri_fail(ctx, BRI_EINVAL, "x and b must be 16-byte aligned device pointers");
    if (nrhs < 1 || nrhs > 65535) return bri_fail(ctx, BRI_EINVAL, "nrhs must be in [1, 65535]");
    if (!(tol > 0) || maxit < 1) return bri_fail(ctx, BRI_EINVAL, "tol must be > 0 and maxit >= 1");
    if (mode < 0 || mode > 4) return bri_fail(ctx, BRI_EINVAL, "mode must be 0..4");
    if (!ctx->have64) return bri_fail(ctx, BRI_ESTATE, "no hopping fields built");
    const size_t bytes = 16 * 12 * (size_t)ctx->g.V * nrhs;
    if ((const char *)x < (const char *)b + bytes && (const char *)b < (const char *)x + bytes)
        return bri_fail(ctx, BRI_EINVAL, "x and b overlap");
    return bri_solve_impl(ctx, x, b, nrhs, m0, tol, maxit, mode, info, as_stream(stream));
}

bri_status bri_force(bri_ctx *ctx, double *dU, const double *chi, const double *psi, double m0, int recompute_hops,
                     void *stream) {
    (void)m0;              // the mass term does not depend on U
    (void)recompute_hops;  // the force always recomputes the path sums; the projections are redone from them
    if (!ctx) return BRI_EINVAL;
    if (!dU || !chi || !psi || !bri_aligned16(dU) || !bri_aligned16(chi) || !bri_aligned16(psi))
        return bri_fail(ctx, BRI_EINVAL, "dU, chi, psi must be 16-byte aligned device pointers");
    if (!ctx->U) return bri_fail(ctx, BRI_ESTATE, "no links: call bri_build_hops first");
    if (ctx->csw != 0.0) return bri_fail(ctx, BRI_ESTATE, "the force of the clover term is not built (csw must be 0)");
    return bri_force_impl(ctx, (double2 *)dU, (const double2 *)chi, (const double2 *)psi, as_stream(stream));
}

// S = phi^dagger (D^dagger D)^{-1} phi = |Y|^2 with X = (D^dagger D)^{-1} phi,
// Y = D X; optionally X itself and dU += dS/dU = -2 d Re(Y^dagger D X)/dU.
static bri_status inverse_action(bri_ctx *ctx, double *S, double *Xout, double *dU, const double *phi, double m0,
                                 double tol, int maxit, bri_solve_info *info, cudaStream_t s) {
    const size_t n = (size_t)ctx->g.V * 12, bytes = n * sizeof(double2);
    DevBuf work;
    BRI_TRY_CUDA(ctx, cudaMalloc(&work.p, 4 * bytes));
    double2 *Z = work.as<double2>(), *X = Z + n, *Y = X + n, *t = Y + n;
    bri_status st = BRI_OK;
    bri_solve_info i1{}, i2{};
    // FP64 defect correction around FP32 BiCGstab when FP32 fields are stored
    // (same FP64 true residual, far fewer FP64 applies), else FP64 BiCGstab
    const int mode = ctx->f32.valid ? 1 : 0;
    do {
        // D^dagger Z = phi  <=>  D (g5 Z) = g5 phi
        if ((st = gamma5_scale(ctx, t, (const double2 *)phi, 1, 0.0, s)) != BRI_OK) break;
        BRI_TRY_CUDA(ctx, cudaMemsetAsync(Z, 0, bytes, s));
        if ((st = bri_solve_impl(ctx, (double *)Z, (const double *)t, 1, m0, tol, maxit, mode, &i1, s)) != BRI_OK) break;
        if ((st = gamma5_scale(ctx, t, Z, 1, 0.0, s)) != BRI_OK) break;  // Z = g5 w
        BRI_TRY_CUDA(ctx, cudaMemsetAsync(X, 0, bytes, s));
        if ((st = bri_solve_impl(ctx, (double *)X, (const double *)t, 1, m0, tol, maxit, mode, &i2, s)) != BRI_OK) break;
        if ((st = bri_dslash_impl(ctx, Y, X, 1, m0, 0, BRI_F64, s)) != BRI_OK) break;
        if (S) {
            double r[2];
            if ((st = bri_cdot_impl(ctx, r, Y, Y, n, BRI_F64, s)) != BRI_OK) break;
            *S = r[0];
        }
        if (Xout) BRI_TRY_CUDA(ctx, cudaMemcpyAsync(Xout, X, bytes, cudaMemcpyDeviceToDevice, s));
        if (dU) {
            // -2 d Re(Y^dagger D X)/dU: scale Y by -2
            if ((st = gamma5_scale(ctx, t, Y, 0, -2.0, s)) != BRI_OK) break;
            st = bri_force_impl(ctx, (double2 *)dU, t, X, s);
        }
    } while (0);
    cudaStreamSynchronize(s);
    if (info) *info = i2;
    if (st == BRI_OK && (i1.status != BRI_OK || i2.status != BRI_OK)) st = i1.status != BRI_OK ? i1.status : i2.status;
    return st;
}

bri_status bri_force_inverse(bri_ctx *ctx, double *dU, const double *phi, double m0, double tol, int maxit,
                             bri_solve_info *info, void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (!dU || !phi || !bri_aligned16(dU) || !bri_aligned16(phi))
        return bri_fail(ctx, BRI_EINVAL, "dU and phi must be 16-byte aligned device pointers");
    if (!ctx->have64) return bri_fail(ctx, BRI_ESTATE, "no hopping fields built");
    if (ctx->csw != 0.0) return bri_fail(ctx, BRI_ESTATE, "the force of the clover term is not built (csw must be 0)");
    return inverse_action(ctx, nullptr, nullptr, dU, phi, m0, tol, maxit, info, as_stream(stream));
}

bri_status bri_inverse_action(bri_ctx *ctx, double *S, double *X, double *dU, const double *phi, double m0,
                              double tol, int maxit, bri_solve_info *info, void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (!phi || !bri_aligned16(phi) || (X && !bri_aligned16(X)) || (dU && !bri_aligned16(dU)))
        return bri_fail(ctx, BRI_EINVAL, "phi, X and dU must be 16-byte aligned device pointers");
    if (!(tol > 0) || maxit < 1) return bri_fail(ctx, BRI_EINVAL, "tol must be > 0 and maxit >= 1");
    if (!ctx->have64) return bri_fail(ctx, BRI_ESTATE, "no hopping fields built");
    if (dU && ctx->csw != 0.0)
        return bri_fail(ctx, BRI_ESTATE, "the force of the clover term is not built (csw must be 0)");
    return inverse_action(ctx, S, X, dU, phi, m0, tol, maxit, info, as_stream(stream));
}

bri_status bri_project_su3(bri_ctx *ctx, double *Y, const double *A, long n, void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (n < 0 || (n > 0 && (!Y || !A || !bri_aligned16(Y) || !bri_aligned16(A))))
        return bri_fail(ctx, BRI_EINVAL, "A and Y must be 16-byte aligned device pointers, n >= 0");
    return bri_project_impl(ctx, (double2 *)Y, (const double2 *)A, n, as_stream(stream));
}

bri_status bri_cdot(bri_ctx *ctx, double *result, const void *a, const void *b, int nrhs, bri_prec prec,
                    void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (!result || !a || !b || !bri_aligned16(a) || !bri_aligned16(b))
        return bri_fail(ctx, BRI_EINVAL, "result must be a host pointer, a and b 16-byte aligned device pointers");
    if (nrhs < 1) return bri_fail(ctx, BRI_EINVAL, "nrhs must be >= 1");
    BRI_RETURN_IF(check_prec(ctx, prec));
    return bri_cdot_impl(ctx, result, a, b, (size_t)ctx->g.V * 12 * nrhs, prec, as_stream(stream));
}

bri_status bri_set_weights(bri_ctx *ctx, const double *lambda, const double *rho) {
    if (!ctx) return BRI_EINVAL;
    if (!lambda || !rho) return bri_fail(ctx, BRI_EINVAL, "null weights");
    for (int n = 0; n < 5; n++)
        if (!std::isfinite(lambda[n]) || (n > 0 && !std::isfinite(rho[n])))
            return bri_fail(ctx, BRI_EINVAL, "weights must be finite");
    geom_set_weights(ctx->g, lambda, rho);
    ctx->gen++;
    return BRI_OK;
}

// ---- APE smearing and the clover term -------------------------------------------------
bri_status bri_ape_smear(bri_ctx *ctx, double *V, const double *U, double alpha, int nsteps, void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (!V || !U || !bri_aligned16(V) || !bri_aligned16(U))
        return bri_fail(ctx, BRI_EINVAL, "V and U must be 16-byte aligned device pointers");
    const size_t bytes = sizeof(double2) * 36 * (size_t)ctx->g.V;
    if ((const char *)V < (const char *)U + bytes && (const char *)U < (const char *)V + bytes)
        return bri_fail(ctx, BRI_EINVAL, "V and U overlap");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return bri_fail(ctx, BRI_EINVAL, "alpha must be in [0, 1]");
    if (nsteps < 0 || nsteps > 1000) return bri_fail(ctx, BRI_EINVAL, "nsteps must be in [0, 1000]");
    return bri_ape_impl(ctx, (double2 *)V, (const double2 *)U, alpha, nsteps, as_stream(stream));
}

bri_status bri_set_clover(bri_ctx *ctx, double csw, void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (!std::isfinite(csw)) return bri_fail(ctx, BRI_EINVAL, "csw must be finite");
    ctx->gen++;
    ctx->csw = csw;
    if (csw == 0.0) {
        ctx->g.clov64 = nullptr;
        ctx->g.clov32 = nullptr;
        return BRI_OK;
    }
    if (!ctx->U) return bri_fail(ctx, BRI_ESTATE, "no links: call bri_build_hops first");
    return bri_clover_build_impl(ctx, as_stream(stream));
}

// ---- spectra and the overlap operator ------------------------------------------------
bri_status bri_eigs_ddag_d(bri_ctx *ctx, double *evals, double *lmax, double *evecs, int nev, double m0,
                           int max_krylov, double tol, bri_prec prec, bri_eig_info *info, void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (!evals) return bri_fail(ctx, BRI_EINVAL, "evals must be a host array of nev doubles");
    if (evecs && !bri_aligned16(evecs)) return bri_fail(ctx, BRI_EINVAL, "evecs must be 16-byte aligned");
    if (nev < 1 || nev > 64) return bri_fail(ctx, BRI_EINVAL, "nev must be in [1, 64]");
    if (max_krylov <= nev || (size_t)max_krylov > 12 * (size_t)ctx->g.V)
        return bri_fail(ctx, BRI_EINVAL, "max_krylov must be in [nev + 1, 12 V]");
    if (!(tol > 0) || !std::isfinite(m0)) return bri_fail(ctx, BRI_EINVAL, "tol must be > 0 and m0 finite");
    BRI_RETURN_IF(check_prec(ctx, prec));
    if (!ctx->have64) return bri_fail(ctx, BRI_ESTATE, "no hopping fields built");
    if ((prec == BRI_F32 && !ctx->f32.valid) || (prec == BRI_F16 && !ctx->f16.valid))
        return bri_fail(ctx, BRI_ESTATE, "hopping fields of this precision not built");
    return bri_eigs_impl(ctx, evals, lmax, evecs, nev, m0, max_krylov, tol, prec, info, as_stream(stream));
}

bri_status bri_overlap_setup(bri_ctx *ctx, double rho, int nlow, double eps, int max_krylov, double tol,
                             bri_prec prec, bri_overlap_info *info, void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (!(rho > 0 && rho < 2)) return bri_fail(ctx, BRI_EINVAL, "rho must be in (0, 2)");
    if (nlow < 0 || nlow > 64) return bri_fail(ctx, BRI_EINVAL, "nlow must be in [0, 64]");
    if (!(eps >= 1e-14 && eps <= 0.1)) return bri_fail(ctx, BRI_EINVAL, "eps must be in [1e-14, 0.1]");
    if (max_krylov <= nlow + 1 || (size_t)max_krylov > 12 * (size_t)ctx->g.V)
        return bri_fail(ctx, BRI_EINVAL, "max_krylov must be in [nlow + 2, 12 V]");
    if (!(tol > 0)) return bri_fail(ctx, BRI_EINVAL, "tol must be > 0");
    BRI_RETURN_IF(check_prec(ctx, prec));
    if (!ctx->have64) return bri_fail(ctx, BRI_ESTATE, "no hopping fields built");
    if ((prec == BRI_F32 && !ctx->f32.valid) || (prec == BRI_F16 && !ctx->f16.valid))
        return bri_fail(ctx, BRI_ESTATE, "hopping fields of this precision not built");
    return bri_overlap_setup_impl(ctx, rho, nlow, eps, max_krylov, tol, prec, info, as_stream(stream));
}

bri_status bri_overlap_modes(bri_ctx *ctx, double *lambda, double *vecs, void *stream) {
    if (!ctx) return BRI_EINVAL;
    if (vecs && !bri_aligned16(vecs)) return bri_fail(ctx, BRI_EINVAL, "vecs must be 16-byte aligned");
    return bri_overlap_modes_impl(ctx, lambda, vecs, as_stream(stream));
}

bri_status bri_apply_sign(bri_ctx *ctx, double *out, const double *in, int nrhs, void *stream) {
    if (!ctx) return BRI_EINVAL;
    BRI_RETURN_IF(check_apply(ctx, out, in, nrhs, BRI_F64));
    return bri_overlap_apply_impl(ctx, out, in, nrhs, 0, 0.0, as_stream(stream));
}

bri_status bri_apply_overlap(bri_ctx *ctx, double *out, const double *in, int nrhs, double m, void *stream) {
    if (!ctx) return BRI_EINVAL;
    BRI_RETURN_IF(check_apply(ctx, out, in, nrhs, BRI_F64));
    if (!std::isfinite(m)) return bri_fail(ctx, BRI_EINVAL, "m must be finite");
    return bri_overlap_apply_impl(ctx, out, in, nrhs, 1, m, as_stream(stream));
}

bri_status bri_get_weights(bri_ctx *ctx, double *lambda, double *rho) {
    if (!ctx) return BRI_EINVAL;
    if (!lambda || !rho) return bri_fail(ctx, BRI_EINVAL, "null weights");
    for (int n = 0; n < 5; n++) {
        lambda[n] = ctx->g.lamd[n];
        rho[n] = ctx->g.rhod[n];
    }
    return BRI_OK;
}

bri_status bri_tune(bri_ctx *ctx, bri_prec prec, int nrhs, void *stream) {
    if (!ctx) return BRI_EINVAL;
    BRI_RETURN_IF(check_prec(ctx, prec));
    if (nrhs < 1 || nrhs > 65535) return bri_fail(ctx, BRI_EINVAL, "nrhs must be in [1, 65535]");
    return bri_tune_impl(ctx, prec, nrhs, as_stream(stream));
}

bri_status bri_set_threads(bri_ctx *ctx, bri_prec prec, int nrhs, int threads) {
    if (!ctx) return BRI_EINVAL;
    BRI_RETURN_IF(check_prec(ctx, prec));
    const int thr = threads & 2047, variant = threads >> 11;
    if (nrhs < 1 || !valid_shape(threads)) return bri_fail(ctx, BRI_EINVAL, "bad nrhs or threads");
    // variant 8 (tensor cores): the low bits are the right-hand sides per warp pass
    ctx->tune[bri_tune_key(ctx, prec, nrhs)] = variant == 8 ? threads : (thr & ~31) | (variant << 11);
    return BRI_OK;
}

int bri_get_threads(bri_ctx *ctx, bri_prec prec, int nrhs) {
    if (!ctx) return BRI_EINVAL;
    if (check_prec(ctx, prec) != BRI_OK || nrhs < 1) return BRI_EINVAL;
    return bri_dslash_threads(ctx, prec, nrhs);
}

bri_status bri_debug_stall(bri_ctx *ctx, int on) {
    if (!ctx) return BRI_EINVAL;
    ctx->g.stall = on ? 1 : 0;
    return BRI_OK;
}

long bri_kernel_launches(bri_ctx *ctx) { return ctx ? ctx->launches : 0; }

const char *bri_last_error(bri_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

// ---- launch-shape tuner ---------------------------------------------------------
bri_status bri_tune_impl(bri_ctx *ctx, bri_prec prec, int nrhs, cudaStream_t s) {
    const size_t elt = prec == BRI_F64 ? 16 : 8;
    const size_t bytes = elt * 12 * (size_t)ctx->g.V * nrhs;
    DevBuf inb, outb;
    BRI_TRY_CUDA(ctx, cudaMalloc(&inb.p, bytes));
    BRI_TRY_CUDA(ctx, cudaMalloc(&outb.p, bytes));
    void *in = inb.p, *out = outb.p;
    BRI_TRY_CUDA(ctx, cudaMemsetAsync(in, 0, bytes, s));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 128;
    float best_ms = 1e30f;
    bri_status st = BRI_OK;
    // candidates: tiled kernel (0), plain kernel at 64..512 threads, and the
    // variants of the FP32 plain kernel (launch shape above bit 11)
    for (int thr : {0, 64, 128, 256, 512, 128 | 2048, 128 | 4096, 256 | 4096, 64 | 6144, 128 | 6144, 128 | 8192,
                    256 | 8192, 512 | 8192, 64 | 10240, 128 | 10240, 256 | 10240, 128 | 12288, 128 | 14336,
                    16384 | 4, 16384 | 6, 16384 | 8, 16384 | 12, 128 | 18432, 256 | 18432, 32 | 20480,
                    128 | 20480, 32 | 22528, 64 | 22528}) {
        if (thr == 0 && (prec == BRI_F64 || !tiled_ok(ctx->g))) continue;
        // the tensor-core kernel has FP16-operand accuracy: a candidate for FP16
        // fields (same accuracy class) with full storage only
        if ((thr >> 11) == 8 && (prec != BRI_F16 || ctx->f16.comp != BRI_LINK_FULL || nrhs < 2)) continue;
        if ((thr >> 11) && prec == BRI_F64) continue;
        if ((st = bri_dslash_raw(ctx, out, in, nrhs, 0.0, 0, prec, nullptr, thr, s)) != BRI_OK) break;  // warm-up
        cudaEventRecord(e0, s);
        const int reps = 3;
        for (int r = 0; r < reps && st == BRI_OK; r++) st = bri_dslash_raw(ctx, out, in, nrhs, 0.0, 0, prec, nullptr, thr, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st != BRI_OK) break;
        if (ms < best_ms) { best_ms = ms; best = thr; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != BRI_OK) return st;
    const std::string key = bri_tune_key(ctx, prec, nrhs);
    ctx->tune[key] = best;
    tune_save_entry(key, best);
    return BRI_OK;
}
