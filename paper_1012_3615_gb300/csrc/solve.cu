// Krylov solves with the Brillouin operator: BiCGstab (van der Vorst), the
// solver the paper uses for its propagators (Sec. 6.4), on the device.
//
// All BiCGstab scalars live in device memory, one set per right-hand side, so
// an iteration needs no host round trip: seven launches (p update, apply,
// <rhat,v> + alpha, s update, apply, <t,s>,<t,t> + omega, x/r update +
// <rhat,r>,<r,r> + rho).  Each reduction kernel writes per-block FP64 partial
// sums (a thread's own few elements are summed in the vectors' precision); the
// last block to finish (atomic ticket) adds them in a fixed order, so the sums
// are deterministic, and updates the scalars.  Blocks of iterations
// are captured once into a CUDA graph and replayed; the host reads the
// convergence flags between replays only.  Converged right-hand sides are
// skipped by every kernel (flag array), including the stencil apply.
//
// Modes: 0 = FP64 BiCGstab; 1/2 = FP64 defect correction (true residual,
// solution update and norms in FP64) around an FP32 BiCGstab with the FP32 /
// FP16 hopping fields; 3 = mode 2 for all right-hand sides at once.
#include <chrono>
#include <cmath>
#include <map>
#include <vector>

#include "ctx.h"

using namespace bri;

namespace {

constexpr int RT = 256;     // threads of the vector / reduction kernels
constexpr int RBLK = 304;   // blocks per right-hand side of the reduction kernels (2 x 152 SMs)
constexpr int NPART = 4;    // doubles per partial sum

struct BiState {
    double2 rho, rho_old, alpha, omega;
    double rr, tol2, bb;
    int iters, maxit;
};

template <typename T> struct Real;
template <> struct Real<float2> { using R = float; };
template <> struct Real<double2> { using R = double; };

BRI_D double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum of NV doubles; the result is valid in thread 0
template <int NV> BRI_D void block_sum(double v[NV]) {
    __shared__ double sm[NV][RT / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        v[k] = warp_sum(v[k]);
        if (l == 0) sm[k][w] = v[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double t = l < RT / 32 ? sm[k][l] : 0.0;
            v[k] = warp_sum(t);
        }
    }
    __syncthreads();
}

// stores this block's partials; returns true (in every thread) for the last block
template <int NV>
BRI_D bool partial_and_ticket(double v[NV], double *part, unsigned *ticket) {
    __shared__ bool last;
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) part[(size_t)blockIdx.x * NPART + k] = v[k];
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// in the last block, all threads: sum the partials of every block (thread t
// takes blocks t, t + RT, ... in order, then a fixed tree); result in thread 0
template <int NV> BRI_D void gather_partials(const double *part, double out[NV]) {
    for (int k = 0; k < NV; k++) out[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += RT)
        for (int k = 0; k < NV; k++) out[k] += ((volatile const double *)part)[(size_t)b * NPART + k];
    block_sum<NV>(out);
}

// per-thread accumulator of the BiCGstab reductions: FP32 vectors sum their few
// elements per thread in FP32 (FP64 is 1/64 of the FP32 rate on this GPU),
// FP64 vectors in FP64; partials across threads and blocks are always FP64
template <typename T> struct AccT { using A = double; };
template <> struct AccT<float2> { using A = float; };

BRI_D double2 dcdiv(double2 a, double2 b) {
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
BRI_D bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

template <typename T> BRI_D T tc(double2 z) { return mk<T>(z.x, z.y); }

// ---- BiCGstab step kernels (grid: RBLK x nrhs) ------------------------------
template <typename T>
__global__ void k_bi_p(T *p, const T *r, const T *v, const BiState *st, const int *flag, size_t n) {
    const int rh = blockIdx.y;
    if (flag[rh]) return;
    const BiState s = st[rh];
    const double2 beta = cmul(dcdiv(s.rho, s.rho_old), dcdiv(s.alpha, s.omega));
    const T b = tc<T>(beta), om = tc<T>(s.omega);
    p += rh * n; r += rh * n; v += rh * n;
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT)
        p[i] = cadd(r[i], cmul(b, csub(p[i], cmul(om, v[i]))));
}

template <typename T>
__global__ void k_bi_alpha(const T *rhat, const T *v, BiState *st, int *flag, double *part, unsigned *tick,
                           size_t n) {
    const int rh = blockIdx.y;
    if (flag[rh]) return;
    rhat += rh * n; v += rh * n;
    using A = typename AccT<T>::A;
    A ac[2] = {0, 0};
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
        T a = rhat[i], b = v[i];
        ac[0] += (A)a.x * b.x + (A)a.y * b.y;
        ac[1] += (A)a.x * b.y - (A)a.y * b.x;
    }
    double acc[2] = {ac[0], ac[1]};
    if (partial_and_ticket<2>(acc, part + (size_t)rh * RBLK * NPART, tick + rh)) {
        double s[2];
        gather_partials<2>(part + (size_t)rh * RBLK * NPART, s);
        if (threadIdx.x != 0) return;
        double2 rv = make_double2(s[0], s[1]);
        if (!finite2(rv)) flag[rh] = 3;
        else if (rv.x == 0.0 && rv.y == 0.0) flag[rh] = 2;
        else st[rh].alpha = dcdiv(st[rh].rho, rv);
        tick[rh] = 0;
    }
}

template <typename T>
__global__ void k_bi_s(T *s, const T *r, const T *v, const BiState *st, const int *flag, size_t n) {
    const int rh = blockIdx.y;
    if (flag[rh]) return;
    const T a = tc<T>(st[rh].alpha);
    s += rh * n; r += rh * n; v += rh * n;
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT)
        s[i] = csub(r[i], cmul(a, v[i]));
}

template <typename T>
__global__ void k_bi_omega(const T *t, const T *s, BiState *st, int *flag, double *part, unsigned *tick, size_t n) {
    const int rh = blockIdx.y;
    if (flag[rh]) return;
    t += rh * n; s += rh * n;
    using A = typename AccT<T>::A;
    A ac[3] = {0, 0, 0};
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
        T a = t[i], b = s[i];
        ac[0] += (A)a.x * b.x + (A)a.y * b.y;
        ac[1] += (A)a.x * b.y - (A)a.y * b.x;
        ac[2] += (A)a.x * a.x + (A)a.y * a.y;
    }
    double acc[3] = {ac[0], ac[1], ac[2]};
    if (partial_and_ticket<3>(acc, part + (size_t)rh * RBLK * NPART, tick + rh)) {
        double q[3];
        gather_partials<3>(part + (size_t)rh * RBLK * NPART, q);
        if (threadIdx.x != 0) return;
        if (!isfinite(q[0]) || !isfinite(q[1]) || !isfinite(q[2])) flag[rh] = 3;
        else if (q[2] == 0.0) flag[rh] = 2;
        else st[rh].omega = make_double2(q[0] / q[2], q[1] / q[2]);
        tick[rh] = 0;
    }
}

template <typename T>
__global__ void k_bi_xr(T *x, T *r, const T *p, const T *s, const T *t, const T *rhat, BiState *st, int *flag,
                        double *part, unsigned *tick, size_t n) {
    const int rh = blockIdx.y;
    if (flag[rh]) return;
    const T a = tc<T>(st[rh].alpha), om = tc<T>(st[rh].omega);
    const size_t o = rh * n;
    using A = typename AccT<T>::A;
    A ac[3] = {0, 0, 0};
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
        T si = s[o + i];
        x[o + i] = cadd(x[o + i], cadd(cmul(a, p[o + i]), cmul(om, si)));
        T ri = csub(si, cmul(om, t[o + i]));
        r[o + i] = ri;
        T h = rhat[o + i];
        ac[0] += (A)h.x * ri.x + (A)h.y * ri.y;
        ac[1] += (A)h.x * ri.y - (A)h.y * ri.x;
        ac[2] += (A)ri.x * ri.x + (A)ri.y * ri.y;
    }
    double acc[3] = {ac[0], ac[1], ac[2]};
    if (partial_and_ticket<3>(acc, part + (size_t)rh * RBLK * NPART, tick + rh)) {
        double q[3];
        gather_partials<3>(part + (size_t)rh * RBLK * NPART, q);
        if (threadIdx.x != 0) return;
        BiState &S = st[rh];
        S.iters++;
        S.rho_old = S.rho;
        S.rho = make_double2(q[0], q[1]);
        S.rr = q[2];
        if (!isfinite(q[0]) || !isfinite(q[1]) || !isfinite(q[2])) flag[rh] = 3;
        else if (q[2] <= S.tol2) flag[rh] = 1;
        else if ((q[0] == 0.0 && q[1] == 0.0) || (S.omega.x == 0.0 && S.omega.y == 0.0)) flag[rh] = 2;
        else if (S.iters >= S.maxit) flag[rh] = 4;
        tick[rh] = 0;
    }
}

// r = b - Ax (Ax in r on entry when have_ax), rhat = r, p = v = 0, scalars reset
template <typename T>
__global__ void k_bi_init(T *r, T *rhat, T *p, T *v, const T *b, int have_ax, BiState *st, int *flag, double tol,
                          int maxit, double *part, unsigned *tick, size_t n) {
    const int rh = blockIdx.y;
    const size_t o = rh * n;
    using A = typename AccT<T>::A;
    A ac[2] = {0, 0};
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
        T bi = b[o + i];
        T ri = have_ax ? csub(bi, r[o + i]) : bi;
        r[o + i] = ri;
        rhat[o + i] = ri;
        p[o + i] = mk<T>(0, 0);
        v[o + i] = mk<T>(0, 0);
        ac[0] += (A)ri.x * ri.x + (A)ri.y * ri.y;
        ac[1] += (A)bi.x * bi.x + (A)bi.y * bi.y;
    }
    double acc[2] = {ac[0], ac[1]};
    if (partial_and_ticket<2>(acc, part + (size_t)rh * RBLK * NPART, tick + rh)) {
        double q[2];
        gather_partials<2>(part + (size_t)rh * RBLK * NPART, q);
        if (threadIdx.x != 0) return;
        BiState S;
        S.rho = make_double2(q[0], 0.0);
        S.rho_old = S.alpha = S.omega = make_double2(1.0, 0.0);
        S.rr = q[0];
        S.bb = q[1];
        S.tol2 = tol * tol * q[1];
        S.iters = 0;
        S.maxit = maxit;
        st[rh] = S;
        if (!isfinite(q[0]) || !isfinite(q[1])) flag[rh] = 3;
        else flag[rh] = (q[0] <= S.tol2) ? 1 : 0;
        tick[rh] = 0;
    }
}

// ---- FP64 outer-loop helpers --------------------------------------------------
// r = b - Ax (in place in ax); norms ||r||^2, ||b||^2 per right-hand side into nrm[2*rh]
__global__ void k_residual64(double2 *ax, const double2 *b, double *nrm, double *part, unsigned *tick, size_t n) {
    const int rh = blockIdx.y;
    const size_t o = rh * n;
    double acc[2] = {0, 0};
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
        double2 bi = b[o + i], ri = csub(bi, ax[o + i]);
        ax[o + i] = ri;
        acc[0] += ri.x * ri.x + ri.y * ri.y;
        acc[1] += bi.x * bi.x + bi.y * bi.y;
    }
    if (partial_and_ticket<2>(acc, part + (size_t)rh * RBLK * NPART, tick + rh)) {
        double q[2];
        gather_partials<2>(part + (size_t)rh * RBLK * NPART, q);
        if (threadIdx.x != 0) return;
        nrm[2 * rh] = q[0];
        nrm[2 * rh + 1] = q[1];
        tick[rh] = 0;
    }
}
// ||x||^2 per right-hand side into nrm[2*rh] (is the initial guess zero?)
__global__ void k_norm64(const double2 *x, double *nrm, double *part, unsigned *tick, size_t n) {
    const int rh = blockIdx.y;
    const size_t o = rh * n;
    double acc[2] = {0, 0};
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
        double2 v = x[o + i];
        acc[0] += v.x * v.x + v.y * v.y;
    }
    if (partial_and_ticket<2>(acc, part + (size_t)rh * RBLK * NPART, tick + rh)) {
        double q[2];
        gather_partials<2>(part + (size_t)rh * RBLK * NPART, q);
        if (threadIdx.x != 0) return;
        nrm[2 * rh] = q[0];
        tick[rh] = 0;
    }
}
// out32 = r64 / ||r64||
// (finished right-hand sides get a zero source, which BiCGstab flags as converged at once)
__global__ void k_to32(float2 *out, const double2 *in, const double *nrm, const int *done, size_t n) {
    const int rh = blockIdx.y;
    const double inv = (done[rh] || !(nrm[2 * rh] > 0)) ? 0.0 : 1.0 / sqrt(nrm[2 * rh]);
    const size_t o = rh * n;
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
        double2 v = in[o + i];
        out[o + i] = make_float2((float)(v.x * inv), (float)(v.y * inv));
    }
}
// x64 += ||r64|| e32
__global__ void k_accum64(double2 *x, const float2 *e, const double *nrm, const int *done, size_t n) {
    const int rh = blockIdx.y;
    if (done[rh]) return;
    const double sc = sqrt(nrm[2 * rh]);
    const size_t o = rh * n;
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
        float2 v = e[o + i];
        x[o + i] = make_double2(x[o + i].x + sc * v.x, x[o + i].y + sc * v.y);
    }
}
// <a, b> = sum conj(a) b over n complex elements, FP64 accumulation; the last
// block writes the result to out[0..1]
template <typename T>
__global__ void k_cdot(const T *a, const T *b, size_t n, double *out, double *part, unsigned *tick) {
    double acc[2] = {0, 0};
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
        T x = a[i], y = b[i];
        acc[0] += (double)x.x * y.x + (double)x.y * y.y;
        acc[1] += (double)x.x * y.y - (double)x.y * y.x;
    }
    if (partial_and_ticket<2>(acc, part, tick)) {
        double q[2];
        gather_partials<2>(part, q);
        if (threadIdx.x != 0) return;
        out[0] = q[0];
        out[1] = q[1];
        tick[0] = 0;
    }
}

template <typename T> __global__ void k_zero(T *x, size_t n) {
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) x[i] = mk<T>(0, 0);
}

}  // namespace

// ---- work spaces ---------------------------------------------------------------
struct VecSet {
    void *x = nullptr, *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr;
};

struct SolverWork {
    size_t n = 0;
    int nrhs = 0;
    VecSet v64, v32;
    double2 *r64 = nullptr;
    BiState *st = nullptr;
    int *flag = nullptr;
    int *done = nullptr;
    double *part = nullptr;
    unsigned *tick = nullptr;
    double *nrm = nullptr;
    cudaStream_t own = nullptr;
    std::map<std::string, cudaGraphExec_t> graphs;
};

static void free_vecs(VecSet &v) {
    void **a[] = {&v.x, &v.r, &v.rhat, &v.p, &v.v, &v.s, &v.t};
    for (void **p : a) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
}

void bri_solver_free(bri_ctx *ctx) {
    SolverWork *w = ctx->work;
    if (!w) return;
    for (auto &kv : w->graphs) cudaGraphExecDestroy(kv.second);
    free_vecs(w->v64);
    free_vecs(w->v32);
    cudaFree(w->r64);
    cudaFree(w->st);
    cudaFree(w->flag);
    cudaFree(w->done);
    cudaFree(w->part);
    cudaFree(w->tick);
    cudaFree(w->nrm);
    if (w->own) cudaStreamDestroy(w->own);
    delete w;
    ctx->work = nullptr;
}

static bri_status alloc_vecs(bri_ctx *ctx, VecSet &v, size_t bytes) {
    void **a[] = {&v.x, &v.r, &v.rhat, &v.p, &v.v, &v.s, &v.t};
    for (void **p : a) BRI_TRY_CUDA(ctx, cudaMalloc(p, bytes));
    return BRI_OK;
}

// work spaces for nrhs right-hand sides; need32 / need64 select the vector sets
static bri_status ensure_work(bri_ctx *ctx, int nrhs, bool need64, bool need32) {
    const size_t n = (size_t)ctx->g.V * 12;
    SolverWork *w = ctx->work;
    if (w && w->nrhs >= nrhs && (!need64 || w->v64.x) && (!need32 || w->v32.x)) return BRI_OK;
    const int have_nrhs = w ? w->nrhs : 0;
    const bool had64 = w && w->v64.x, had32 = w && w->v32.x;
    bri_solver_free(ctx);
    w = new SolverWork();
    ctx->work = w;
    w->n = n;
    w->nrhs = nrhs > have_nrhs ? nrhs : have_nrhs;
    const size_t R = w->nrhs;
    if (need64 || had64) BRI_RETURN_IF(alloc_vecs(ctx, w->v64, sizeof(double2) * n * R));
    if (need32 || had32) {
        BRI_RETURN_IF(alloc_vecs(ctx, w->v32, sizeof(float2) * n * R));
        BRI_TRY_CUDA(ctx, cudaMalloc(&w->r64, sizeof(double2) * n * R));
    }
    BRI_TRY_CUDA(ctx, cudaMalloc(&w->st, sizeof(BiState) * R));
    BRI_TRY_CUDA(ctx, cudaMalloc(&w->flag, sizeof(int) * R));
    BRI_TRY_CUDA(ctx, cudaMalloc(&w->done, sizeof(int) * R));
    BRI_TRY_CUDA(ctx, cudaMalloc(&w->part, sizeof(double) * NPART * RBLK * R));
    BRI_TRY_CUDA(ctx, cudaMalloc(&w->tick, sizeof(unsigned) * R));
    BRI_TRY_CUDA(ctx, cudaMemset(w->tick, 0, sizeof(unsigned) * R));
    BRI_TRY_CUDA(ctx, cudaMalloc(&w->nrm, sizeof(double) * 2 * R));
    BRI_TRY_CUDA(ctx, cudaStreamCreateWithFlags(&w->own, cudaStreamNonBlocking));
    return BRI_OK;
}

namespace {

// enqueue `iters` BiCGstab iterations on vectors vs (element T) for nrhs right-hand sides
template <typename T>
bri_status enqueue_iters(bri_ctx *ctx, const VecSet &vs, int nrhs, double m0, bri_prec prec, int iters,
                         cudaStream_t s) {
    SolverWork *w = ctx->work;
    const size_t n = w->n;
    dim3 grid(RBLK, nrhs);
    T *x = (T *)vs.x, *r = (T *)vs.r, *rh = (T *)vs.rhat, *p = (T *)vs.p, *v = (T *)vs.v, *sv = (T *)vs.s,
      *t = (T *)vs.t;
    const int thr = bri_dslash_threads(ctx, prec, nrhs);
    for (int it = 0; it < iters; it++) {
        k_bi_p<T><<<grid, RT, 0, s>>>(p, r, v, w->st, w->flag, n);
        BRI_LAUNCHED(ctx);
        BRI_RETURN_IF(bri_dslash_raw(ctx, v, p, nrhs, m0, 0, prec, w->flag, thr, s));
        k_bi_alpha<T><<<grid, RT, 0, s>>>(rh, v, w->st, w->flag, w->part, w->tick, n);
        BRI_LAUNCHED(ctx);
        k_bi_s<T><<<grid, RT, 0, s>>>(sv, r, v, w->st, w->flag, n);
        BRI_LAUNCHED(ctx);
        BRI_RETURN_IF(bri_dslash_raw(ctx, t, sv, nrhs, m0, 0, prec, w->flag, thr, s));
        k_bi_omega<T><<<grid, RT, 0, s>>>(t, sv, w->st, w->flag, w->part, w->tick, n);
        BRI_LAUNCHED(ctx);
        k_bi_xr<T><<<grid, RT, 0, s>>>(x, r, p, sv, t, rh, w->st, w->flag, w->part, w->tick, n);
        BRI_LAUNCHED(ctx);
    }
    return BRI_OK;
}

// Run BiCGstab on (vs.x, b) in element type T until every right-hand side has a
// flag (converged / breakdown / nan) or maxit iterations were done.  x is the
// initial guess when have_x0.  Returns the iterations performed.
template <typename T>
bri_status bicgstab(bri_ctx *ctx, const VecSet &vs, const T *b, bool have_x0, int nrhs, double m0, bri_prec prec,
                    double tol, int maxit, cudaStream_t s, std::vector<int> &flags, std::vector<int> &iters) {
    SolverWork *w = ctx->work;
    const size_t n = w->n;
    dim3 grid(RBLK, nrhs);
    if (have_x0) {
        BRI_RETURN_IF(bri_dslash_raw(ctx, vs.r, vs.x, nrhs, m0, 0, prec, nullptr, bri_dslash_threads(ctx, prec, nrhs), s));
    } else {
        k_zero<T><<<RBLK, RT, 0, s>>>((T *)vs.x, n * nrhs);
        BRI_LAUNCHED(ctx);
    }
    k_bi_init<T><<<grid, RT, 0, s>>>((T *)vs.r, (T *)vs.rhat, (T *)vs.p, (T *)vs.v, b, have_x0 ? 1 : 0, w->st,
                                      w->flag, tol, maxit, w->part, w->tick, n);
    BRI_LAUNCHED(ctx);
    // block of iterations per graph replay: short for expensive FP64 applies
    const int K = sizeof(T) == 16 ? 4 : 16;
    char key[192];
    snprintf(key, sizeof key, "bi:%d:%d:%d:%.17g:%p:%p:%p:%d", (int)sizeof(T), (int)prec, nrhs, m0, vs.x, vs.s,
             vs.t, bri_dslash_threads(ctx, prec, nrhs));
    cudaGraphExec_t exec = nullptr;
    auto it = w->graphs.find(key);
    if (it != w->graphs.end()) {
        exec = it->second;
    } else {
        // the tensor-core apply and the site-pair kernel allocate on first use:
        // not inside the capture
        const int thr = bri_dslash_threads(ctx, prec, nrhs);
        if ((thr >> 11) == 8) BRI_RETURN_IF(bri_tc_reserve(ctx, nrhs, thr & 2047));
        if ((thr >> 11) == 3 && prec != BRI_F64 && !(prec == BRI_F32 ? ctx->p32 : ctx->p16).valid &&
            !ctx->g.clov64)
            BRI_RETURN_IF(bri_pair_store_impl(ctx, prec, s));
        cudaGraph_t graph;
        BRI_TRY_CUDA(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        bri_status st = enqueue_iters<T>(ctx, vs, nrhs, m0, prec, K, s);
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (st != BRI_OK) return st;
        if (e != cudaSuccess) return bri_fail(ctx, BRI_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        BRI_TRY_CUDA(ctx, cudaGraphInstantiate(&exec, graph, 0));
        cudaGraphDestroy(graph);
        w->graphs[key] = exec;
        ctx->launches -= 7 * K;  // captured, not launched
    }
    flags.assign(nrhs, 0);
    iters.assign(nrhs, 0);
    std::vector<BiState> hs(nrhs);
    for (int done = 0; done < maxit + K; done += K) {
        BRI_TRY_CUDA(ctx, cudaMemcpyAsync(flags.data(), w->flag, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
        BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        bool all = true;
        for (int r = 0; r < nrhs; r++) all = all && flags[r] != 0;
        if (all) break;
        BRI_TRY_CUDA(ctx, cudaGraphLaunch(exec, s));
        ctx->launches += 7 * K;
    }
    BRI_TRY_CUDA(ctx, cudaMemcpyAsync(flags.data(), w->flag, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
    BRI_TRY_CUDA(ctx, cudaMemcpyAsync(hs.data(), w->st, sizeof(BiState) * nrhs, cudaMemcpyDeviceToHost, s));
    BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    for (int r = 0; r < nrhs; r++) iters[r] = hs[r].iters;
    return BRI_OK;
}

// FP64 true residual of (x, b): nrm[2r] = ||b - Dx||^2, nrm[2r+1] = ||b||^2, r64 holds b - Dx
// r64 = b - D x and the norms ||r||^2, ||b||^2 (host nrm).  x_zero: the guess is
// zero for every RHS, so D x = 0 needs no apply; skip (device, optional): RHS
// whose residual is not needed
bri_status true_residual(bri_ctx *ctx, const double2 *x, const double2 *b, double2 *r64, int nrhs, double m0,
                         cudaStream_t s, std::vector<double> &nrm, bool x_zero = false, const int *skip = nullptr) {
    SolverWork *w = ctx->work;
    if (x_zero)
        BRI_TRY_CUDA(ctx, cudaMemsetAsync(r64, 0, sizeof(double2) * w->n * nrhs, s));
    else
        BRI_RETURN_IF(
            bri_dslash_raw(ctx, r64, x, nrhs, m0, 0, BRI_F64, skip, bri_dslash_threads(ctx, BRI_F64, nrhs), s));
    k_residual64<<<dim3(RBLK, nrhs), RT, 0, s>>>(r64, b, w->nrm, w->part, w->tick, w->n);
    BRI_LAUNCHED(ctx);
    nrm.resize(2 * nrhs);
    BRI_TRY_CUDA(ctx, cudaMemcpyAsync(nrm.data(), w->nrm, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, s));
    BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    return BRI_OK;
}


double now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// mode 0: one right-hand side, FP64 BiCGstab with restarts from the true residual
bri_status solve_fp64(bri_ctx *ctx, double2 *x, const double2 *b, double m0, double tol, int maxit,
                      bri_solve_info *info, cudaStream_t s) {
    SolverWork *w = ctx->work;
    const size_t bytes = sizeof(double2) * w->n;
    BRI_TRY_CUDA(ctx, cudaMemcpyAsync(w->v64.x, x, bytes, cudaMemcpyDeviceToDevice, s));
    std::vector<int> flags, iters;
    std::vector<double> nrm;
    int total = 0;
    bri_status st = BRI_ENOTCONV;
    double rel = 0;
    for (int restart = 0; restart < 6 && total < maxit; restart++) {
        // target slightly below tol so the recomputed true residual meets it
        BRI_RETURN_IF(bicgstab<double2>(ctx, w->v64, b, true, 1, m0, BRI_F64, 0.5 * tol, maxit - total, s, flags, iters));
        total += iters[0];
        BRI_RETURN_IF(true_residual(ctx, (double2 *)w->v64.x, b, w->r64 ? w->r64 : (double2 *)w->v64.t, 1, m0, s, nrm));
        if (!std::isfinite(nrm[0]) || !std::isfinite(nrm[1])) { st = BRI_ENAN; rel = NAN; break; }
        rel = nrm[1] > 0 ? sqrt(nrm[0] / nrm[1]) : 0.0;
        if (rel <= tol) { st = BRI_OK; break; }
        if (flags[0] == 3) { st = BRI_ENAN; break; }
        st = flags[0] == 2 ? BRI_EBREAKDOWN : BRI_ENOTCONV;
        if (flags[0] == 0) break;  // out of iterations
    }
    BRI_TRY_CUDA(ctx, cudaMemcpyAsync(x, w->v64.x, bytes, cudaMemcpyDeviceToDevice, s));
    if (info) {
        info->iters = total;
        info->outer_iters = 0;
        info->true_resid = rel;
        info->status = st;
    }
    return BRI_OK;
}

// modes 1..3: FP64 defect correction around FP32 BiCGstab (links in prec)
bri_status solve_mixed(bri_ctx *ctx, double2 *x, const double2 *b, int nrhs, double m0, double tol, int maxit,
                       bri_prec prec, bri_solve_info *info, cudaStream_t s) {
    SolverWork *w = ctx->work;
    const size_t n = w->n;
    const double inner_tol = prec == BRI_F32 ? 1e-5 : 2e-3;
    std::vector<int> done(nrhs, 0), flags, iters, tot(nrhs, 0), outer(nrhs, 0);
    std::vector<double> nrm, rel(nrhs, 0.0);
    std::vector<bri_status> sts(nrhs, BRI_ENOTCONV);
    // a zero initial guess (the usual case) needs no FP64 apply for r = b
    bool x_zero = true;
    {
        k_norm64<<<dim3(RBLK, nrhs), RT, 0, s>>>(x, w->nrm, w->part, w->tick, n);
        BRI_LAUNCHED(ctx);
        std::vector<double> xn(2 * nrhs);
        BRI_TRY_CUDA(ctx, cudaMemcpyAsync(xn.data(), w->nrm, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, s));
        BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        for (int r = 0; r < nrhs; r++)
            if (xn[2 * r] != 0.0) x_zero = false;
    }
    BRI_TRY_CUDA(ctx, cudaMemcpyAsync(w->done, done.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
    for (int cyc = 0; cyc < 200; cyc++) {
        // converged right-hand sides (device flags of the previous cycle) are skipped
        BRI_RETURN_IF(true_residual(ctx, x, b, w->r64, nrhs, m0, s, nrm, cyc == 0 && x_zero, w->done));
        bool all = true;
        for (int r = 0; r < nrhs; r++) {
            if (done[r]) continue;
            if (!std::isfinite(nrm[2 * r]) || !std::isfinite(nrm[2 * r + 1])) {
                rel[r] = NAN;
                done[r] = 1;
                sts[r] = BRI_ENAN;
                continue;
            }
            rel[r] = nrm[2 * r + 1] > 0 ? sqrt(nrm[2 * r] / nrm[2 * r + 1]) : 0.0;
            if (rel[r] <= tol) { done[r] = 1; sts[r] = BRI_OK; continue; }
            if (tot[r] >= maxit) { done[r] = 1; sts[r] = BRI_ENOTCONV; continue; }
            all = false;
        }
        if (all) break;
        BRI_TRY_CUDA(ctx, cudaMemcpyAsync(w->done, done.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
        dim3 grid(RBLK, nrhs);
        // inner source r / ||r|| in the b slot (v32.s); BiCGstab's own s and t
        // vectors use v32.t and the FP64 residual buffer, free until the next cycle
        k_to32<<<grid, RT, 0, s>>>((float2 *)w->v32.s, w->r64, w->nrm, w->done, n);
        BRI_LAUNCHED(ctx);
        int budget = 1;
        for (int r = 0; r < nrhs; r++)
            if (!done[r]) budget = std::max(budget, maxit - tot[r]);
        VecSet inner = w->v32;
        inner.s = w->v32.t;
        inner.t = (void *)w->r64;
        BRI_RETURN_IF(bicgstab<float2>(ctx, inner, (const float2 *)w->v32.s, false, nrhs, m0, prec, inner_tol, budget,
                                       s, flags, iters));
        k_accum64<<<grid, RT, 0, s>>>(x, (const float2 *)w->v32.x, w->nrm, w->done, n);
        BRI_LAUNCHED(ctx);
        for (int r = 0; r < nrhs; r++)
            if (!done[r]) {
                tot[r] += iters[r];
                outer[r]++;
                if (flags[r] == 3) { done[r] = 1; sts[r] = BRI_ENAN; }
            }
    }
    if (info)
        for (int r = 0; r < nrhs; r++) {
            info[r].iters = tot[r];
            info[r].outer_iters = outer[r];
            info[r].true_resid = rel[r];
            info[r].status = sts[r];
        }
    return BRI_OK;
}

}  // namespace

bri_status bri_solve_impl(bri_ctx *ctx, double *x, const double *b, int nrhs, double m0, double tol, int maxit,
                          int mode, bri_solve_info *info, cudaStream_t user) {
    const size_t n = (size_t)ctx->g.V * 12;
    if (mode == 0) {
        BRI_RETURN_IF(ensure_work(ctx, 1, true, false));
        if (!ctx->work->r64) BRI_TRY_CUDA(ctx, cudaMalloc(&ctx->work->r64, sizeof(double2) * n * ctx->work->nrhs));
    } else {
        if (mode <= 2 && nrhs > 1) {
            // sequential right-hand sides in modes 1, 2; a right-hand side that
            // does not converge does not stop the others (its status is returned)
            bri_status worst = BRI_OK;
            for (int r = 0; r < nrhs; r++) {
                const bri_status st = bri_solve_impl(ctx, x + 2 * r * n, b + 2 * r * n, 1, m0, tol, maxit, mode,
                                                     info ? info + r : nullptr, user);
                if (st != BRI_OK && st != BRI_ENOTCONV && st != BRI_EBREAKDOWN && st != BRI_ENAN) return st;
                if (st != BRI_OK && worst == BRI_OK) worst = st;
            }
            return worst;
        }
        BRI_RETURN_IF(ensure_work(ctx, nrhs, false, true));
    }
    cudaStream_t s = user ? user : ctx->work->own;
    if (!user) BRI_TRY_CUDA(ctx, cudaDeviceSynchronize());
    const bri_prec prec = mode == 1 || mode == 4 ? BRI_F32 : BRI_F16;
    if (mode != 0) {
        const LinkStore &st = prec == BRI_F32 ? ctx->f32 : ctx->f16;
        if (!st.valid) return bri_fail(ctx, BRI_ESTATE, "inner-precision hopping fields not built");
    }
    bri_status worst = BRI_OK;
    if (mode == 0) {
        for (int r = 0; r < nrhs; r++) {
            double t0 = now();
            bri_solve_info inf{};
            BRI_RETURN_IF(solve_fp64(ctx, (double2 *)x + r * n, (const double2 *)b + r * n, m0, tol, maxit, &inf, s));
            inf.seconds = now() - t0;
            if (info) info[r] = inf;
            if (inf.status != BRI_OK && worst == BRI_OK) worst = inf.status;
        }
    } else {
        double t0 = now();
        std::vector<bri_solve_info> inf(nrhs);
        BRI_RETURN_IF(solve_mixed(ctx, (double2 *)x, (const double2 *)b, nrhs, m0, tol, maxit, prec, inf.data(), s));
        double dt = now() - t0;
        for (int r = 0; r < nrhs; r++) {
            inf[r].seconds = dt;
            if (info) info[r] = inf[r];
            if (inf[r].status != BRI_OK && worst == BRI_OK) worst = inf[r].status;
        }
    }
    if (!user) BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    return worst;
}

// complex dot product of two device vectors of n complex elements (FP64 or FP32
// storage), FP64 accumulation; result to the host (synchronises the stream)
bri_status bri_cdot_impl(bri_ctx *ctx, double *res, const void *a, const void *b, size_t n, bri_prec prec,
                         cudaStream_t user) {
    BRI_RETURN_IF(ensure_work(ctx, 1, false, false));
    SolverWork *w = ctx->work;
    cudaStream_t s = user ? user : w->own;
    if (!user) BRI_TRY_CUDA(ctx, cudaDeviceSynchronize());
    if (prec == BRI_F64) k_cdot<double2><<<RBLK, RT, 0, s>>>((const double2 *)a, (const double2 *)b, n, w->nrm, w->part, w->tick);
    else k_cdot<float2><<<RBLK, RT, 0, s>>>((const float2 *)a, (const float2 *)b, n, w->nrm, w->part, w->tick);
    BRI_LAUNCHED(ctx);
    BRI_TRY_CUDA(ctx, cudaMemcpyAsync(res, w->nrm, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    return BRI_OK;
}
