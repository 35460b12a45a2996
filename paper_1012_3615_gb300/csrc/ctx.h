// Internal state of a bri_ctx and helpers shared by the library's .cu files.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>

#include "brillouin.h"
#include "common.cuh"

// One stored copy of the 40 hopping fields in a reduced precision.
struct LinkStore {
    bool valid = false;
    bri_comp comp = BRI_LINK_FULL;
    void *a = nullptr;  // main array (16-byte chunks, [40][chunks][V])
    void *b = nullptr;  // tail array (8/4-byte chunk, [40][V]) or null
};

struct SolverWork;   // solver work spaces (solve.cu)
struct OverlapWork;  // Lanczos / overlap state (overlap.cu)
struct HostApplyWork;  // staging buffers and streams of bri_apply_host (hostapply.cu)

struct bri_ctx {
    bri::Geom g;
    int device = 0;
    double2 *U = nullptr;       // copy of the links, [V][4][9]
    double2 *hops64 = nullptr;  // FP64 hops, [40][9][V]
    bool have64 = false;
    LinkStore f32, f16;
    LinkStore p32, p16;  // site-pair interleaved copies (full / 2-row, even t extent)
    SolverWork *work = nullptr;
    OverlapWork *ov = nullptr;
    HostApplyWork *hw = nullptr;
    double csw = 0.0;              // clover coefficient (0: no clover term)
    double2 *clov64 = nullptr;     // clover blocks, see Geom
    float4 *clov32 = nullptr;
    unsigned *tc_amax = nullptr;   // per-RHS max |psi| of the tensor-core apply (65536 entries)
    void *tc_f = nullptr;          // FP16 copy of the spinors for the tensor-core apply
    size_t tc_fbytes = 0;
    int *werr_h = nullptr;         // host-mapped wait-timeout flag (g.werr is its device address)
    long gen = 0;  // bumped whenever the operator changes (links, weights)
    std::map<std::string, int> tune;  // launch-shape cache: key -> threads per block
    std::string err;
    long launches = 0;
};

bri_status bri_fail(bri_ctx *ctx, bri_status st, const std::string &msg);

#define BRI_TRY_CUDA(ctx, call)                                                            \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return bri_fail((ctx), e_ == cudaErrorMemoryAllocation ? BRI_ENOMEM : BRI_ECUDA, \
                            std::string(#call) + ": " + cudaGetErrorString(e_));           \
    } while (0)

// check the launch that was just enqueued
#define BRI_LAUNCHED(ctx)                                                                  \
    do {                                                                                   \
        (ctx)->launches++;                                                                 \
        cudaError_t e_ = cudaGetLastError();                                               \
        if (e_ != cudaSuccess)                                                             \
            return bri_fail((ctx), BRI_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

#define BRI_RETURN_IF(st)              \
    do {                               \
        bri_status s_ = (st);          \
        if (s_ != BRI_OK) return s_;   \
    } while (0)

inline bool bri_aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// device buffer released when it goes out of scope (cudaFree waits for the
// work that may still use it)
struct DevBuf {
    void *p = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    template <typename T> T *as() const { return (T *)p; }
};

// entry points implemented in the individual translation units
bri_status bri_hops_build_impl(bri_ctx *ctx, cudaStream_t s);
bri_status bri_hops_store_impl(bri_ctx *ctx, bri_prec prec, bri_comp comp, cudaStream_t s);
bri_status bri_pair_store_impl(bri_ctx *ctx, bri_prec prec, cudaStream_t s);
bri_status bri_project_impl(bri_ctx *ctx, double2 *Y, const double2 *A, long n, cudaStream_t s);
// dslash: out = D in (mode 0), D^dagger in (mode 1), gamma5 (D - rho) in (mode 2, m0 = -rho)
bri_status bri_dslash_impl(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int mode,
                           bri_prec prec, cudaStream_t s);
bri_status bri_tune_impl(bri_ctx *ctx, bri_prec prec, int nrhs, cudaStream_t s);
// FP16-spinor apply (BRI_F16H) and spinor storage conversions (dslash_h16.cu)
size_t bri_h16_bytes(int V);
bri_status bri_dslash_h16(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int mode, const int *skip,
                          cudaStream_t s);
bri_status bri_convert_spinor_impl(bri_ctx *ctx, void *dst, int dfmt, const void *src, int sfmt, int nrhs,
                                   cudaStream_t s);
// multi-RHS apply on the tensor cores (launch variant 8; FP32/FP16 full fields)
// (cap: right-hand sides per warp pass, an even number 2..12; anything else: 12)
bri_status bri_dslash_tc(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int mode, bri_prec prec,
                         const int *skip, int cap, cudaStream_t s);
bri_status bri_tc_reserve(bri_ctx *ctx, int nrhs, int cap);
// dslash with an explicit launch shape; skip[r] != 0 skips right-hand side r
bri_status bri_dslash_raw(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int mode, bri_prec prec,
                          const int *skip, int threads, cudaStream_t s);
int bri_dslash_threads(bri_ctx *ctx, bri_prec prec, int nrhs);
std::string bri_tune_key(bri_ctx *ctx, bri_prec prec, int nrhs);
bri_status bri_export_hops_impl(bri_ctx *ctx, double2 *out, cudaStream_t s);
void bri_solver_free(bri_ctx *ctx);
bri_status bri_cdot_impl(bri_ctx *ctx, double *res, const void *a, const void *b, size_t n, bri_prec prec,
                         cudaStream_t user);
bri_status bri_dp_levels(bri_ctx *ctx, void *A, const int *klist, const int start[6], cudaStream_t s);
bri_status bri_force_impl(bri_ctx *ctx, double2 *dU, const double2 *chi, const double2 *psi, cudaStream_t s);
void bri_overlap_free(bri_ctx *ctx);
void bri_host_apply_free(bri_ctx *ctx);
bri_status bri_apply_host_impl(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int mode,
                               bri_prec prec, cudaStream_t user);
bri_status bri_ape_impl(bri_ctx *ctx, double2 *V, const double2 *U, double alpha, int nsteps, cudaStream_t s);
// (re)build the clover blocks from ctx->U with ctx->csw and switch the term on
bri_status bri_clover_build_impl(bri_ctx *ctx, cudaStream_t s);
bri_status bri_eigs_impl(bri_ctx *ctx, double *evals, double *lmax, double *evecs, int nev, double m0, int max_krylov,
                         double tol, bri_prec prec, bri_eig_info *info, cudaStream_t s);
bri_status bri_overlap_setup_impl(bri_ctx *ctx, double rho, int nlow, double eps, int max_krylov, double tol,
                                  bri_prec prec, bri_overlap_info *info, cudaStream_t s);
bri_status bri_overlap_modes_impl(bri_ctx *ctx, double *lambda, double *vecs, cudaStream_t s);
// mode 0: out = sign(H) in; mode 1: out = D_ov,m in
bri_status bri_overlap_apply_impl(bri_ctx *ctx, double *out, const double *in, int nrhs, int mode, double m,
                                  cudaStream_t s);
bri_status bri_solve_impl(bri_ctx *ctx, double *x, const double *b, int nrhs, double m0, double tol, int maxit,
                          int mode, bri_solve_info *info, cudaStream_t user);
