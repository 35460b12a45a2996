// Spectra of the hermitian kernel and the overlap operator built on the
// class-weight operator D (Sec. 7).
//
//  * Lanczos on A = (gamma5 D(m0))^2 = D(m0)^dagger D(m0) with full
//    reorthogonalisation (a classical Gram-Schmidt pass after every
//    three-term step) against a basis
//    held in device memory: the extremal Ritz values compared in Sec. 7.4 and,
//    for the overlap, the low eigenpairs of H^2 at m0 = -rho.
//  * Eq. def_over: D_ov = rho [1 + gamma5 sign(H)], H = gamma5 (D - rho).
//    sign(H) psi = sum_i sign(lambda_i) z_i <z_i, psi>  (the nlow smallest
//    |lambda| eigenpairs of H, exact) + H p(P H^2 P) P psi with P the
//    projector orthogonal to the z_i and p a Chebyshev approximation of
//    1/sqrt(x) on the interval [lo, hi] that holds the rest of the spectrum of
//    H^2 (evaluated by Clenshaw's recurrence).  Eq. def_mass gives the
//    massive operator (1 - m / (2 rho)) D_ov + m.
//
// Every step runs on the device: stencil applications, dot products (FP64
// accumulation, fixed summation order), vector updates, the tridiagonal and
// small hermitian eigenproblems (single-thread kernels, eig_small.cuh) and the
// Chebyshev coefficients.  The host only reads Ritz values and residual
// estimates between blocks of Lanczos steps and picks the polynomial degree.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"
#include "eig_small.cuh"

using namespace bri;

namespace {

constexpr int VT = 256;         // threads of the vector kernels
constexpr int DB = 152;         // blocks per vector of the dot-product kernels
constexpr int MAX_WANT = 64;    // largest number of wanted low eigenpairs
constexpr int MAX_DEGREE = 60000;

BRI_D double2 d2(double2 v) { return v; }
BRI_D double2 d2(float2 v) { return make_double2(v.x, v.y); }
template <typename T> BRI_D T from_d2(double2 v);
template <> BRI_D double2 from_d2<double2>(double2 v) { return v; }
template <> BRI_D float2 from_d2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }

// block-wide sum of a complex value; valid in thread 0
BRI_D double2 block_sum2(double2 v) {
    __shared__ double2 sm[VT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sm[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < VT / 32 ? sm[l] : make_double2(0.0, 0.0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        }
    }
    __syncthreads();
    return v;
}

// per-block partial sums of <V_j, w> = sum conj(V_j) w, j = blockIdx.y
template <typename T>
__global__ void k_mdot_part(const T *__restrict__ Vb, size_t ldv, const T *__restrict__ w, size_t n, double2 *part) {
    const T *v = Vb + (size_t)blockIdx.y * ldv;
    double2 acc = make_double2(0.0, 0.0);
    if constexpr (sizeof(T) == 8) {
        // FP32 vectors: FP32 products per thread (FP64 is 1/64 of the FP32 rate),
        // FP64 across threads and blocks
        float2 f = make_float2(0.f, 0.f);
        for (size_t i = (size_t)blockIdx.x * VT + threadIdx.x; i < n; i += (size_t)gridDim.x * VT) {
            const T a = v[i], b = w[i];
            f.x = fmaf(a.x, b.x, fmaf(a.y, b.y, f.x));
            f.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, f.y));
        }
        acc = make_double2(f.x, f.y);
    } else {
        for (size_t i = (size_t)blockIdx.x * VT + threadIdx.x; i < n; i += (size_t)gridDim.x * VT) {
            const double2 a = d2(v[i]), b = d2(w[i]);
            acc.x += a.x * b.x + a.y * b.y;
            acc.y += a.x * b.y - a.y * b.x;
        }
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

// h[j] = sum of the partials of vector j in block order; the real part of
// h[m - 1] is also added to *racc when racc is given (Lanczos alpha)
__global__ void k_mdot_final(const double2 *__restrict__ part, int nb, int m, double2 *h, double *racc) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < nb; b++) s = cadd(s, part[(size_t)j * nb + b]);
    h[j] = s;
    if (racc && j == m - 1) *racc += s.x;
}

// w -= sum_j h_j V_j
template <typename T>
__global__ void k_maxpy(T *__restrict__ w, const T *__restrict__ Vb, size_t ldv, const double2 *__restrict__ h, int m,
                        size_t n) {
    for (size_t i = (size_t)blockIdx.x * VT + threadIdx.x; i < n; i += (size_t)gridDim.x * VT) {
        if constexpr (sizeof(T) == 8) {  // FP32 vectors: FP32 arithmetic
            float2 acc = w[i];
            for (int j = 0; j < m; j++) {
                const float2 c = make_float2((float)h[j].x, (float)h[j].y), v = Vb[(size_t)j * ldv + i];
                acc = csub(acc, cmul(c, v));
            }
            w[i] = acc;
        } else {
            double2 acc = d2(w[i]);
            int j = 0;
            for (; j + 4 <= m; j += 4) {
                double2 v[4];
#pragma unroll
                for (int q = 0; q < 4; q++) v[q] = d2(Vb[(size_t)(j + q) * ldv + i]);
#pragma unroll
                for (int q = 0; q < 4; q++) acc = csub(acc, cmul(h[j + q], v[q]));
            }
            for (; j < m; j++) acc = csub(acc, cmul(h[j], d2(Vb[(size_t)j * ldv + i])));
            w[i] = from_d2<T>(acc);
        }
    }
}

// out_k = sum_j C[k][j] V_j, k < nk (four outputs per grid row)
template <typename T>
__global__ void k_combine(T *__restrict__ out, size_t ldo, const T *__restrict__ Vb, size_t ldv,
                          const double2 *__restrict__ C, int ldc, int m, int nk, size_t n) {
    const int k0 = blockIdx.y * 4;
    for (size_t i = (size_t)blockIdx.x * VT + threadIdx.x; i < n; i += (size_t)gridDim.x * VT) {
        double2 acc[4];
#pragma unroll
        for (int q = 0; q < 4; q++) acc[q] = make_double2(0.0, 0.0);
        for (int j = 0; j < m; j++) {
            const double2 v = d2(Vb[(size_t)j * ldv + i]);
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (k0 + q < nk) acc[q] = cadd(acc[q], cmul(C[(size_t)(k0 + q) * ldc + j], v));
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (k0 + q < nk) out[(size_t)(k0 + q) * ldo + i] = from_d2<T>(acc[q]);
    }
}

// per-block partial sums of |w|^2 (in .x)
template <typename T>
__global__ void k_norm_part(const T *__restrict__ w, size_t n, double2 *part) {
    double2 acc = make_double2(0.0, 0.0);
    for (size_t i = (size_t)blockIdx.x * VT + threadIdx.x; i < n; i += (size_t)gridDim.x * VT) {
        const double2 a = d2(w[i]);
        acc.x += a.x * a.x + a.y * a.y;
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// v = w / ||w|| (norm from the partials, fixed order); block 0 stores ||w||
template <typename T>
__global__ void k_normalize(T *__restrict__ v, const T *__restrict__ w, const double2 *__restrict__ part, int nb,
                            double *nrm_out, size_t n) {
    __shared__ double nrm;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; b++) s += part[b].x;
        nrm = sqrt(s);
        if (blockIdx.x == 0 && nrm_out) *nrm_out = nrm;
    }
    __syncthreads();
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (size_t i = (size_t)blockIdx.x * VT + threadIdx.x; i < n; i += (size_t)gridDim.x * VT)
        v[i] = from_d2<T>(cscale(d2(w[i]), inv));
}

// start vector: uniform entries in [-1/2, 1/2) from a counter-based hash (splitmix64)
BRI_D unsigned long long splitmix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
template <typename T>
__global__ void k_rand_vec(T *v, size_t n, unsigned long long seed) {
    for (size_t i = (size_t)blockIdx.x * VT + threadIdx.x; i < n; i += (size_t)gridDim.x * VT) {
        const unsigned long long a = splitmix64(seed ^ (2 * i)), b = splitmix64(seed ^ (2 * i + 1));
        v[i] = from_d2<T>(make_double2((double)(a >> 11) * 0x1.0p-53 - 0.5, (double)(b >> 11) * 0x1.0p-53 - 0.5));
    }
}

// Ritz values of the Lanczos matrix T_m (alpha[0..m), beta[1..m)): out[0..nlow)
// the nlow smallest, out[nlow] the largest, out[nlow + 1 + k] their residual
// estimates beta[m] |s_k[m-1]|.  final: eigenvectors of the nlow smallest
// (sequential, clusters orthogonalised) into S[k][0..m) as complex numbers.
// Work: (nlow + 1) x 5m doubles and (nlow + 1) x m bytes.
__global__ void k_tri_ritz(const double *__restrict__ alpha, const double *__restrict__ beta, int m, int nlow, int final,
                           double *out, double2 *S, double *work, unsigned char *pw) {
    __shared__ double th[MAX_WANT + 1];
    const int t = threadIdx.x, nw = nlow + 1;
    if (t < nw) th[t] = tri_eigenvalue(alpha, beta, m, t < nlow ? t : m - 1);
    __syncthreads();
    const size_t W = 5 * (size_t)m;
    double scale = 0.0;
    for (int k = 0; k < nw; k++) scale = fmax(scale, fabs(th[k]));
    if (!final) {
        if (t < nw) {
            double *u = work + t * W;
            tri_eigenvector(alpha, beta, m, th[t], u, u + m, u + 2 * m, u + 3 * m, pw + (size_t)t * m, u + 4 * m,
                            nullptr, 0, 0);
            out[t] = th[t];
            out[nw + t] = beta[m] * fabs(u[4 * m + m - 1]);
        }
        return;
    }
    if (t != 0) return;
    // eigenvectors in ascending order; a vector whose eigenvalue lies within
    // 1e-3 ||T|| of the previous ones is kept orthogonal to them (the x rows are
    // contiguous: row k at work + k * W + 4m, stride W)
    for (int k = 0; k < nw; k++) {
        int c0 = k;
        if (k < nlow)
            while (c0 > 0 && th[k] - th[c0 - 1] <= 1e-3 * scale) c0--;
        else
            c0 = k;
        double *u = work + k * W;
        tri_eigenvector(alpha, beta, m, th[k], u, u + m, u + 2 * m, u + 3 * m, pw + (size_t)k * m, u + 4 * m,
                        work + c0 * W + 4 * m, k - c0, W);
        out[k] = th[k];
        out[nw + k] = beta[m] * fabs(u[4 * m + m - 1]);
        if (k < nlow && S)
            for (int i = 0; i < m; i++) S[(size_t)k * m + i] = make_double2(u[4 * m + i], 0.0);
    }
}

// Rayleigh-Ritz of H on the Ritz vectors: M = Y^dagger H Y (k x k, column b =
// h[b * k ..]); eigenpairs by Jacobi, sorted by |lambda|; C[q][j] = Q[j][q]
// so that z_q = sum_j C[q][j] y_j; lam[q] the eigenvalues.
__global__ void k_small_herm(const double2 *__restrict__ YHY, int k, double2 *M, double2 *Q, double2 *C, double *lam) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int a = 0; a < k; a++)
        for (int b = 0; b < k; b++) {
            // hermitian part of <y_a, H y_b> (rounding makes it slightly non-hermitian)
            const double2 x = YHY[(size_t)b * k + a], y = YHY[(size_t)a * k + b];
            M[a * k + b] = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
        }
    herm_jacobi(M, Q, k);
    int order[MAX_WANT];
    for (int q = 0; q < k; q++) order[q] = q;
    for (int a = 1; a < k; a++) {  // insertion sort by |lambda|
        const int o = order[a];
        int b = a;
        while (b > 0 && fabs(M[order[b - 1] * k + order[b - 1]].x) > fabs(M[o * k + o].x)) {
            order[b] = order[b - 1];
            b--;
        }
        order[b] = o;
    }
    for (int q = 0; q < k; q++) {
        const int c = order[q];
        lam[q] = M[c * k + c].x;
        for (int j = 0; j < k; j++) C[(size_t)q * k + j] = Q[j * k + c];
    }
}

// Chebyshev coefficients of f(x) = 1/sqrt(x) on [lo, hi] from its values at
// the N Chebyshev nodes: c_k = (2/N) sum_j f(x_j) cos(pi k (j + 1/2) / N)
__global__ void k_cheb_coef(double *c, int N, double lo, double hi) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double s = 0.0;
    for (int j = 0; j < N; j++) {
        const double x = 0.5 * (hi + lo) + 0.5 * (hi - lo) * cospi((j + 0.5) / N);
        s += cospi((double)k * (j + 0.5) / N) / sqrt(x);
    }
    c[k] = 2.0 * s / N;
}

// max over G points of [lo, hi] (denser towards the ends) of |1 - sqrt(x) p(x)|,
// p = c_0/2 + sum_k c_k T_k(t) by Clenshaw; *err (non-negative double bits)
// must start at zero
__global__ void k_cheb_err(const double *__restrict__ c, int N, double lo, double hi, int G,
                           unsigned long long *err) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const double x = lo + (hi - lo) * 0.5 * (1.0 - cospi((double)g / (G - 1)));
    const double t = (2.0 * x - hi - lo) / (hi - lo);
    double b1 = 0.0, b2 = 0.0;
    for (int k = N - 1; k >= 1; k--) {
        const double b0 = c[k] + 2.0 * t * b1 - b2;
        b2 = b1;
        b1 = b0;
    }
    const double p = 0.5 * c[0] + t * b1 - b2;
    double e = fabs(1.0 - sqrt(x) * p);
    if (!(e == e)) e = 1e300;
    atomicMax(err, (unsigned long long)__double_as_longlong(e));
}

// one Clenshaw step on vectors: out = ck v + s2 Bb - t2 b1 - b2 (out may alias b2)
template <typename T>
__global__ void k_cheb_step(T *out, const T *__restrict__ v, const T *__restrict__ Bb, const T *__restrict__ b1,
                            const T *b2, double ck, double s2, double t2, int have_b1, int have_b2, size_t n) {
    using R = decltype(T().x);  // arithmetic in the vectors' precision
    const R c = (R)ck, s = (R)s2, t = (R)t2;
    for (size_t i = (size_t)blockIdx.x * VT + threadIdx.x; i < n; i += (size_t)gridDim.x * VT) {
        T r = cscale(v[i], c);
        if (have_b1) {
            r = cadd(r, cscale(Bb[i], s));
            r = csub(r, cscale(b1[i], t));
        }
        if (have_b2) r = csub(r, b2[i]);
        out[i] = r;
    }
}

__global__ void k_f64_to_f32(float2 *out, const double2 *__restrict__ in, size_t n) {
    for (size_t i = (size_t)blockIdx.x * VT + threadIdx.x; i < n; i += (size_t)gridDim.x * VT)
        out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
__global__ void k_f32_to_f64(double2 *out, const float2 *__restrict__ in, size_t n) {
    for (size_t i = (size_t)blockIdx.x * VT + threadIdx.x; i < n; i += (size_t)gridDim.x * VT)
        out[i] = make_double2(in[i].x, in[i].y);
}

// deflation coefficients d_i = -sign(lambda_i) c_i (k_maxpy subtracts)
__global__ void k_defl_coef(double2 *d, const double2 *__restrict__ c, const double *__restrict__ lam, int k) {
    const int i = threadIdx.x;
    if (i < k) d[i] = cscale(c[i], lam[i] > 0 ? -1.0 : 1.0);
}

// out = (rho' + m) psi + rho' gamma5 s, rho' = rho - m/2 (Eq. def_over, def_mass)
__global__ void k_overlap_final(double2 *out, const double2 *__restrict__ psi, const double2 *__restrict__ s, double rp,
                                double m, size_t n) {
    for (size_t i = (size_t)blockIdx.x * VT + threadIdx.x; i < n; i += (size_t)gridDim.x * VT) {
        const double g5 = (i % 12) < 6 ? 1.0 : -1.0;
        out[i] = cadd(cscale(psi[i], rp + m), cscale(s[i], rp * g5));
    }
}

unsigned vec_blocks(size_t n) {
    const size_t b = (n + VT - 1) / VT;
    return (unsigned)std::min<size_t>(b, 152 * 16);
}

}  // namespace

// ---- work spaces -----------------------------------------------------------------
struct OverlapWork {
    size_t n = 0;
    // state of the last bri_overlap_setup
    bool ready = false;
    long gen = -1;
    double rho = 1.0;
    bri_prec prec = BRI_F64;
    int nlow = 0;
    int degree = 0;
    double lo = 0.0, hi = 0.0;
    std::vector<double> coef;
    double2 *Z = nullptr;   // [nlow][n] eigenvectors of H
    float2 *Z32 = nullptr;  // FP32 copy for the FP32 / FP16 polynomial
    double *lam = nullptr;  // [nlow] eigenvalues of H
    // vectors of the sign application: FP64 v, q, b1, b2, Bb, tmp, sign;
    // FP32 v, q, b1, b2, Bb, tmp
    double2 *v64[7] = {};
    float2 *v32[6] = {};
    double2 *cdef = nullptr;  // [2 MAX_WANT]: <z_i, psi> and the deflation coefficients
    // reductions
    double2 *part = nullptr;  // [MAX_WANT... ] partial sums
    size_t part_cap = 0;
    double2 *h = nullptr;     // coefficients
    size_t h_cap = 0;
};

static void free_ptr(void *p) {
    if (p) cudaFree(p);
}

void bri_overlap_free(bri_ctx *ctx) {
    OverlapWork *w = ctx->ov;
    if (!w) return;
    free_ptr(w->Z);
    free_ptr(w->Z32);
    free_ptr(w->lam);
    for (auto &p : w->v64) free_ptr(p);
    for (auto &p : w->v32) free_ptr(p);
    free_ptr(w->part);
    free_ptr(w->h);
    free_ptr(w->cdef);
    delete w;
    ctx->ov = nullptr;
}

namespace {

bri_status ensure_ov(bri_ctx *ctx) {
    if (ctx->ov) return BRI_OK;
    OverlapWork *w = new OverlapWork();
    ctx->ov = w;
    w->n = (size_t)ctx->g.V * 12;
    BRI_TRY_CUDA(ctx, cudaMalloc(&w->cdef, 2 * MAX_WANT * sizeof(double2)));
    return BRI_OK;
}

bri_status ensure_red(bri_ctx *ctx, int m) {
    OverlapWork *w = ctx->ov;
    const size_t need_part = (size_t)std::max(m, 1) * DB, need_h = (size_t)std::max(m, MAX_WANT * MAX_WANT);
    if (w->part_cap < need_part) {
        free_ptr(w->part);
        w->part = nullptr;
        BRI_TRY_CUDA(ctx, cudaMalloc(&w->part, need_part * sizeof(double2)));
        w->part_cap = need_part;
    }
    if (w->h_cap < need_h) {
        free_ptr(w->h);
        w->h = nullptr;
        BRI_TRY_CUDA(ctx, cudaMalloc(&w->h, need_h * sizeof(double2)));
        w->h_cap = need_h;
    }
    return BRI_OK;
}

// h[0..m) = V[0..m)^dagger w (FP64 sums); racc += Re h[m-1] when given
template <typename T>
bri_status mdot(bri_ctx *ctx, double2 *h, const T *V, size_t ldv, int m, const T *w, double *racc, cudaStream_t s) {
    OverlapWork *o = ctx->ov;
    if (m <= 0) return BRI_OK;
    BRI_RETURN_IF(ensure_red(ctx, m));
    k_mdot_part<T><<<dim3(DB, m), VT, 0, s>>>(V, ldv, w, o->n, o->part);
    BRI_LAUNCHED(ctx);
    k_mdot_final<<<(m + 127) / 128, 128, 0, s>>>(o->part, DB, m, h, racc);
    BRI_LAUNCHED(ctx);
    return BRI_OK;
}

template <typename T>
bri_status maxpy(bri_ctx *ctx, T *w, const T *V, size_t ldv, const double2 *h, int m, cudaStream_t s) {
    if (m <= 0) return BRI_OK;
    k_maxpy<T><<<vec_blocks(ctx->ov->n), VT, 0, s>>>(w, V, ldv, h, m, ctx->ov->n);
    BRI_LAUNCHED(ctx);
    return BRI_OK;
}

// w <- w - Z (Z^dagger w): one classical Gram-Schmidt pass against k vectors
template <typename T>
bri_status project_out(bri_ctx *ctx, T *w, const T *Z, int k, double2 *h, cudaStream_t s) {
    if (k <= 0) return BRI_OK;
    BRI_RETURN_IF(mdot<T>(ctx, h, Z, ctx->ov->n, k, w, nullptr, s));
    return maxpy<T>(ctx, w, Z, ctx->ov->n, h, k, s);
}

// v = w / ||w||; *nrm (device) receives ||w||
template <typename T>
bri_status normalize(bri_ctx *ctx, T *v, const T *w, double *nrm, cudaStream_t s) {
    OverlapWork *o = ctx->ov;
    BRI_RETURN_IF(ensure_red(ctx, 1));
    k_norm_part<T><<<DB, VT, 0, s>>>(w, o->n, o->part);
    BRI_LAUNCHED(ctx);
    k_normalize<T><<<vec_blocks(o->n), VT, 0, s>>>(v, w, o->part, DB, nrm, o->n);
    BRI_LAUNCHED(ctx);
    return BRI_OK;
}

struct LanczosResult {
    std::vector<double> theta;  // nlow smallest, then the largest
    std::vector<double> resid;  // residual estimates (absolute)
    int m = 0;
    int applies = 0;
    int nconv = 0;
    bool converged = false;
};

// Lanczos for A = (gamma5 D(m0))^2 restricted to the complement of Z[0..nz):
// the nlow smallest and the largest Ritz value, converged when every residual
// estimate is below tol x its Ritz value (tol x the largest for the top).
// Y (when given) receives the Ritz vectors of the nlow smallest.
template <typename T>
bri_status lanczos(bri_ctx *ctx, bri_prec aprec, double m0, int nlow, int mmax, double tol, const T *Z, int nz, T *Y,
                   unsigned long long seed, LanczosResult &res, cudaStream_t s) {
    OverlapWork *o = ctx->ov;
    const size_t n = o->n;
    mmax = (int)std::min<size_t>((size_t)mmax, n);
    if (nlow + 1 > mmax) return bri_fail(ctx, BRI_EINVAL, "max_krylov must exceed the number of wanted eigenpairs");
    const int nw = nlow + 1;
    DevBuf Vb, wb, tmpb, abb, outb, workb, pwb, Sb;
    BRI_TRY_CUDA(ctx, cudaMalloc(&Vb.p, sizeof(T) * n * (size_t)(mmax + 1)));
    BRI_TRY_CUDA(ctx, cudaMalloc(&wb.p, sizeof(T) * n));
    BRI_TRY_CUDA(ctx, cudaMalloc(&tmpb.p, sizeof(T) * n));
    BRI_TRY_CUDA(ctx, cudaMalloc(&abb.p, sizeof(double) * 2 * (size_t)(mmax + 2)));
    BRI_TRY_CUDA(ctx, cudaMalloc(&outb.p, sizeof(double) * 2 * nw));
    BRI_TRY_CUDA(ctx, cudaMalloc(&workb.p, sizeof(double) * 5 * (size_t)mmax * nw));
    BRI_TRY_CUDA(ctx, cudaMalloc(&pwb.p, (size_t)mmax * nw));
    if (nlow > 0 && Y) BRI_TRY_CUDA(ctx, cudaMalloc(&Sb.p, sizeof(double2) * (size_t)mmax * nlow));
    T *V = Vb.as<T>(), *w = wb.as<T>(), *tmp = tmpb.as<T>();
    double2 *S = Sb.as<double2>();
    double *ab = abb.as<double>(), *tri_out = outb.as<double>(), *tri_work = workb.as<double>();
    unsigned char *tri_pw = pwb.as<unsigned char>();
    double *alpha = ab, *beta = ab + (mmax + 2);
    BRI_RETURN_IF(ensure_red(ctx, mmax + 1));
    double2 *h = o->h;
    BRI_TRY_CUDA(ctx, cudaMemsetAsync(ab, 0, sizeof(double) * 2 * (size_t)(mmax + 2), s));
    k_rand_vec<T><<<vec_blocks(n), VT, 0, s>>>(w, n, seed);
    BRI_LAUNCHED(ctx);
    BRI_RETURN_IF(project_out<T>(ctx, w, Z, nz, h, s));
    BRI_RETURN_IF(project_out<T>(ctx, w, Z, nz, h, s));
    BRI_RETURN_IF(normalize(ctx, V, w, beta, s));
    std::vector<double> hout(2 * nw), hab(2 * (size_t)(mmax + 2));
    int m = 0, next_check = std::min(mmax, std::max(nw + 10, 20));
    res = LanczosResult();
    while (m < mmax) {
        T *vj = V + (size_t)m * n;
        BRI_RETURN_IF(bri_dslash_impl(ctx, tmp, vj, 1, m0, 2, aprec, s));
        BRI_RETURN_IF(bri_dslash_impl(ctx, w, tmp, 1, m0, 2, aprec, s));
        res.applies += 2;
        // three-term step against v_{j-1}, v_j, then one Gram-Schmidt pass
        // against the whole basis (its coefficients are at rounding level)
        const int j0 = m > 0 ? m - 1 : 0;
        BRI_RETURN_IF(mdot<T>(ctx, h, V + (size_t)j0 * n, n, m + 1 - j0, w, alpha + m, s));
        BRI_RETURN_IF(maxpy<T>(ctx, w, V + (size_t)j0 * n, n, h, m + 1 - j0, s));
        BRI_RETURN_IF(mdot<T>(ctx, h, V, n, m + 1, w, alpha + m, s));
        BRI_RETURN_IF(maxpy<T>(ctx, w, V, n, h, m + 1, s));
        // deflation last: a component along Z left in the new basis vector would
        // grow from step to step (Z is an eigenspace of value 0 of P A P)
        BRI_RETURN_IF(project_out<T>(ctx, w, Z, nz, h, s));
        BRI_RETURN_IF(normalize(ctx, V + (size_t)(m + 1) * n, w, beta + m + 1, s));
        m++;
        if (m < next_check && m < mmax) continue;
        next_check = std::min(mmax, m + std::max(10, m / 8));
        k_tri_ritz<<<1, 96, 0, s>>>(alpha, beta, m, nlow, 0, tri_out, nullptr, tri_work, tri_pw);
        BRI_LAUNCHED(ctx);
        BRI_TRY_CUDA(ctx, cudaMemcpyAsync(hout.data(), tri_out, sizeof(double) * 2 * nw, cudaMemcpyDeviceToHost, s));
        BRI_TRY_CUDA(ctx, cudaMemcpyAsync(hab.data(), ab, sizeof(double) * hab.size(), cudaMemcpyDeviceToHost, s));
        BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        for (double v : hout)
            if (!std::isfinite(v)) return bri_fail(ctx, BRI_ENAN, "lanczos: non-finite Ritz value");
        const double theta_max = hout[nlow];
        int nconv = 0;
        for (int k = 0; k < nlow; k++)
            if (hout[nw + k] <= tol * fabs(hout[k])) nconv++;
        const bool top = hout[nw + nlow] <= tol * fabs(theta_max);
        // invariant subspace: the residual of the basis vanishes, every Ritz value is exact
        const bool exhausted = hab[(mmax + 2) + m] <= 1e-13 * fabs(theta_max);
        res.nconv = exhausted ? nw : nconv + (top ? 1 : 0);
        if ((nconv == nlow && top) || exhausted) {
            res.converged = true;
            break;
        }
    }
    res.m = m;
    const bool vectors = nlow > 0 && Y;
    k_tri_ritz<<<1, 96, 0, s>>>(alpha, beta, m, nlow, vectors ? 1 : 0, tri_out, vectors ? S : nullptr, tri_work,
                                tri_pw);
    BRI_LAUNCHED(ctx);
    if (vectors) {
        k_combine<T><<<dim3(vec_blocks(n), (nlow + 3) / 4), VT, 0, s>>>(Y, n, V, n, S, m, m, nlow, n);
        BRI_LAUNCHED(ctx);
    }
    BRI_TRY_CUDA(ctx, cudaMemcpyAsync(hout.data(), tri_out, sizeof(double) * 2 * nw, cudaMemcpyDeviceToHost, s));
    BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    res.theta.assign(hout.begin(), hout.begin() + nw);
    res.resid.assign(hout.begin() + nw, hout.end());
    return BRI_OK;
}

// Chebyshev coefficients of 1/sqrt(x) on [lo, hi] with the smallest tried degree
// whose sign error max |1 - sqrt(x) p(x)| is at most eps; returns the error
bri_status build_poly(bri_ctx *ctx, double lo, double hi, double eps, std::vector<double> &coef, double &err,
                      cudaStream_t s) {
    const double kappa = hi / lo;
    // the error falls like ((sqrt(kappa) - 1) / (sqrt(kappa) + 1))^N: start a
    // little below that estimate and grow by 10% until the bound holds
    const double rate = std::log((std::sqrt(kappa) + 1.0) / (std::sqrt(kappa) - 1.0));
    int N = std::max(8, (int)std::floor(0.9 * std::log(1.0 / eps) / rate));
    DevBuf eb_, cb;
    BRI_TRY_CUDA(ctx, cudaMalloc(&eb_.p, sizeof(unsigned long long)));
    BRI_TRY_CUDA(ctx, cudaMalloc(&cb.p, sizeof(double) * MAX_DEGREE));
    double *c = cb.as<double>();
    unsigned long long *e = eb_.as<unsigned long long>();
    for (;;) {
        if (N > MAX_DEGREE)
            return bri_fail(ctx, BRI_EINVAL,
                            "overlap setup: the polynomial would need degree > 60000; deflate more low modes or "
                            "relax eps");
        k_cheb_coef<<<(N + 127) / 128, 128, 0, s>>>(c, N, lo, hi);
        BRI_LAUNCHED(ctx);
        BRI_TRY_CUDA(ctx, cudaMemsetAsync(e, 0, sizeof(unsigned long long), s));
        const int G = std::max(4096, 8 * N);
        k_cheb_err<<<(G + 127) / 128, 128, 0, s>>>(c, N, lo, hi, G, e);
        BRI_LAUNCHED(ctx);
        unsigned long long bits = 0;
        BRI_TRY_CUDA(ctx, cudaMemcpyAsync(&bits, e, sizeof(bits), cudaMemcpyDeviceToHost, s));
        BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        double ev;
        memcpy(&ev, &bits, sizeof(ev));
        if (ev <= eps) {
            coef.resize(N);
            BRI_TRY_CUDA(ctx, cudaMemcpyAsync(coef.data(), c, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
            BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
            err = ev;
            return BRI_OK;
        }
        N = std::max(N + 2, (int)std::ceil(N * 1.1));
    }
}

// q = p(P H^2 P) v (Clenshaw), with T-precision vectors and stencil
template <typename T>
bri_status poly_apply(bri_ctx *ctx, T *q, const T *v, T *b1, T *b2, T *Bb, T *tmp, const T *Z, bri_prec prec,
                      cudaStream_t s) {
    OverlapWork *o = ctx->ov;
    const size_t n = o->n;
    const int N = (int)o->coef.size();
    const double lo = o->lo, hi = o->hi;
    const double sg = 2.0 / (hi - lo), tg = (hi + lo) / (hi - lo);
    const double m0 = -o->rho;
    const unsigned nb = vec_blocks(n);
    // The projector P is applied to every new b_k instead of to H^2 b: the
    // vectors stay orthogonal to Z, so P H^2 P b = P H^2 b, and no component
    // along Z can build up through the recurrence (there the polynomial is
    // evaluated at x = 0, far outside [lo, hi]).
    auto B = [&](T *out, const T *in) -> bri_status {  // out = H^2 in
        BRI_RETURN_IF(bri_dslash_impl(ctx, tmp, in, 1, m0, 2, prec, s));
        return bri_dslash_impl(ctx, out, tmp, 1, m0, 2, prec, s);
    };
    // b_{N-1} = c_{N-1} v, then b_k = c_k v + 2 t(B) b_{k+1} - b_{k+2} down to k = 1
    k_cheb_step<T><<<nb, VT, 0, s>>>(b1, v, nullptr, nullptr, nullptr, o->coef[N - 1], 0.0, 0.0, 0, 0, n);
    BRI_LAUNCHED(ctx);
    bool have_b2 = false;
    for (int k = N - 2; k >= 1; k--) {
        BRI_RETURN_IF(B(Bb, b1));
        k_cheb_step<T><<<nb, VT, 0, s>>>(b2, v, Bb, b1, b2, o->coef[k], 2.0 * sg, 2.0 * tg, 1, have_b2 ? 1 : 0, n);
        BRI_LAUNCHED(ctx);
        BRI_RETURN_IF(project_out<T>(ctx, b2, Z, o->nlow, o->h, s));
        std::swap(b1, b2);
        have_b2 = true;
    }
    // p(B) v = c_0/2 v + t(B) b_1 - b_2
    BRI_RETURN_IF(B(Bb, b1));
    k_cheb_step<T><<<nb, VT, 0, s>>>(q, v, Bb, b1, b2, 0.5 * o->coef[0], sg, tg, 1, have_b2 ? 1 : 0, n);
    BRI_LAUNCHED(ctx);
    return project_out<T>(ctx, q, Z, o->nlow, o->h, s);
}

bri_status alloc_vecs(bri_ctx *ctx, bri_prec prec) {
    OverlapWork *o = ctx->ov;
    for (auto &p : o->v64)
        if (!p) BRI_TRY_CUDA(ctx, cudaMalloc(&p, sizeof(double2) * o->n));
    if (prec != BRI_F64)
        for (auto &p : o->v32)
            if (!p) BRI_TRY_CUDA(ctx, cudaMalloc(&p, sizeof(float2) * o->n));
    return BRI_OK;
}

// out = sign(H) in for one vector (FP64 in and out; out must not alias the work vectors)
bri_status sign_one(bri_ctx *ctx, double2 *out, const double2 *in, cudaStream_t s) {
    OverlapWork *o = ctx->ov;
    const size_t n = o->n;
    const int k = o->nlow;
    double2 *c = o->cdef, *d = o->cdef + MAX_WANT;
    double2 *vp = o->v64[0];
    BRI_TRY_CUDA(ctx, cudaMemcpyAsync(vp, in, sizeof(double2) * n, cudaMemcpyDeviceToDevice, s));
    if (k > 0) {  // vp = P in, c_i = <z_i, in>
        BRI_RETURN_IF(mdot<double2>(ctx, c, o->Z, n, k, in, nullptr, s));
        BRI_RETURN_IF(maxpy<double2>(ctx, vp, o->Z, n, c, k, s));
        BRI_RETURN_IF(project_out<double2>(ctx, vp, o->Z, k, o->h, s));
    }
    const double m0 = -o->rho;
    if (o->prec == BRI_F64) {
        double2 *q = o->v64[1];
        BRI_RETURN_IF(poly_apply<double2>(ctx, q, vp, o->v64[2], o->v64[3], o->v64[4], o->v64[5], o->Z, BRI_F64, s));
        BRI_RETURN_IF(bri_dslash_impl(ctx, out, q, 1, m0, 2, BRI_F64, s));
    } else {
        float2 **f = o->v32;
        k_f64_to_f32<<<vec_blocks(n), VT, 0, s>>>(f[0], vp, n);
        BRI_LAUNCHED(ctx);
        BRI_RETURN_IF(poly_apply<float2>(ctx, f[1], f[0], f[2], f[3], f[4], f[5], o->Z32, o->prec, s));
        BRI_RETURN_IF(bri_dslash_impl(ctx, f[2], f[1], 1, m0, 2, o->prec, s));
        k_f32_to_f64<<<vec_blocks(n), VT, 0, s>>>(out, f[2], n);
        BRI_LAUNCHED(ctx);
    }
    if (k > 0) {  // + sum_i sign(lambda_i) c_i z_i
        k_defl_coef<<<1, MAX_WANT, 0, s>>>(d, c, o->lam, k);
        BRI_LAUNCHED(ctx);
        BRI_RETURN_IF(maxpy<double2>(ctx, out, o->Z, n, d, k, s));
    }
    return BRI_OK;
}

struct SetupStats {
    double lo = 0.0, hi = 0.0, defl_resid = 0.0;
    int applies = 0, kdim = 0;
};

// The nlow eigenpairs of H of smallest |lambda| into Z (vectors of type T) and
// o->lam, and the interval [lo, hi] of the rest of the spectrum of H^2:
// Lanczos on H^2 for the low modes, Rayleigh-Ritz with H on their Ritz vectors,
// a second Lanczos on the deflated operator for the interval.  Stencil applies
// in aprec.
template <typename T>
bri_status setup_modes(bri_ctx *ctx, bri_prec aprec, double m0, int nlow, int max_krylov, double tol, T *Z,
                       SetupStats &st, cudaStream_t s) {
    OverlapWork *o = ctx->ov;
    const size_t n = o->n;
    LanczosResult r1;
    if (nlow == 0) {
        BRI_RETURN_IF(lanczos<T>(ctx, aprec, m0, 1, max_krylov, std::max(tol, 1e-4), nullptr, 0, nullptr, 0x3615ull, r1,
                                 s));
        st.applies += r1.applies;
        st.kdim += r1.m;
        if (!r1.converged) return bri_fail(ctx, BRI_ENOTCONV, "overlap setup: spectral interval of H^2 did not converge");
        st.lo = (r1.theta[0] - r1.resid[0]) * 0.98;
        st.hi = (r1.theta[1] + r1.resid[1]) * 1.02;
        return BRI_OK;
    }
    DevBuf Yb, HYb, Mb;
    BRI_TRY_CUDA(ctx, cudaMalloc(&Yb.p, sizeof(T) * n * nlow));
    BRI_TRY_CUDA(ctx, cudaMalloc(&HYb.p, sizeof(T) * n * nlow));
    BRI_TRY_CUDA(ctx, cudaMalloc(&Mb.p, sizeof(double2) * nlow * nlow * 4));
    T *Y = Yb.as<T>(), *HY = HYb.as<T>();
    double2 *M = Mb.as<double2>();
    double2 *Q = M + nlow * nlow, *C = Q + nlow * nlow, *YHY = C + nlow * nlow;
    BRI_RETURN_IF(lanczos<T>(ctx, aprec, m0, nlow, max_krylov, tol, nullptr, 0, Y, 0x1012ull, r1, s));
    st.applies += r1.applies;
    st.kdim += r1.m;
    if (!r1.converged)
        return bri_fail(ctx, BRI_ENOTCONV, "overlap setup: low modes of H^2 did not converge; raise max_krylov");
    // Rayleigh-Ritz of H on the Ritz vectors of H^2
    for (int b = 0; b < nlow; b++) {
        BRI_RETURN_IF(bri_dslash_impl(ctx, HY + (size_t)b * n, Y + (size_t)b * n, 1, m0, 2, aprec, s));
        st.applies++;
        BRI_RETURN_IF(mdot<T>(ctx, YHY + (size_t)b * nlow, Y, n, nlow, HY + (size_t)b * n, nullptr, s));
    }
    k_small_herm<<<1, 32, 0, s>>>(YHY, nlow, M, Q, C, o->lam);
    BRI_LAUNCHED(ctx);
    k_combine<T><<<dim3(vec_blocks(n), (nlow + 3) / 4), VT, 0, s>>>(Z, n, Y, n, C, nlow, nlow, nlow, n);
    BRI_LAUNCHED(ctx);
    // residuals ||H z - lambda z|| of the deflated pairs
    std::vector<double> lam(nlow);
    BRI_TRY_CUDA(ctx, cudaMemcpyAsync(lam.data(), o->lam, sizeof(double) * nlow, cudaMemcpyDeviceToHost, s));
    BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    std::vector<double2> coefs(nlow), parts(DB);
    for (int b = 0; b < nlow; b++) coefs[b] = make_double2(lam[b], 0.0);
    BRI_TRY_CUDA(ctx, cudaMemcpyAsync(o->cdef, coefs.data(), sizeof(double2) * nlow, cudaMemcpyHostToDevice, s));
    for (int b = 0; b < nlow; b++) {
        BRI_RETURN_IF(bri_dslash_impl(ctx, HY, Z + (size_t)b * n, 1, m0, 2, aprec, s));
        st.applies++;
        BRI_RETURN_IF(maxpy<T>(ctx, HY, Z + (size_t)b * n, n, o->cdef + b, 1, s));
        k_norm_part<T><<<DB, VT, 0, s>>>(HY, n, o->part);
        BRI_LAUNCHED(ctx);
        BRI_TRY_CUDA(ctx, cudaMemcpyAsync(parts.data(), o->part, sizeof(double2) * DB, cudaMemcpyDeviceToHost, s));
        BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        double sum = 0.0;
        for (auto &v : parts) sum += v.x;
        st.defl_resid = std::max(st.defl_resid, std::sqrt(sum));
    }
    o->nlow = nlow;
    // the rest of the spectrum of H^2: Lanczos on the deflated operator
    LanczosResult r2;
    BRI_RETURN_IF(lanczos<T>(ctx, aprec, m0, 1, max_krylov, std::max(tol, 1e-4), Z, nlow, nullptr, 0x3615ull, r2, s));
    st.applies += r2.applies;
    st.kdim += r2.m;
    if (!r2.converged)
        return bri_fail(ctx, BRI_ENOTCONV, "overlap setup: spectral interval of the deflated H^2 did not converge");
    st.lo = (r2.theta[0] - r2.resid[0]) * 0.98;
    st.hi = (r2.theta[1] + r2.resid[1]) * 1.02;
    return BRI_OK;
}

}  // namespace

// ---- entry points (argument checks in api.cu) ---------------------------------------
bri_status bri_eigs_impl(bri_ctx *ctx, double *evals, double *lmax, double *evecs, int nev, double m0, int max_krylov,
                         double tol, bri_prec prec, bri_eig_info *info, cudaStream_t s) {
    auto t0 = std::chrono::steady_clock::now();
    BRI_RETURN_IF(ensure_ov(ctx));
    LanczosResult r;
    if (prec == BRI_F64) {
        BRI_RETURN_IF(lanczos<double2>(ctx, BRI_F64, m0, nev, max_krylov, tol, nullptr, 0, (double2 *)evecs, 0x1012ull,
                                       r, s));
    } else {
        // FP32 Lanczos (FP32 or FP16 hopping fields): Ritz vectors converted to FP64
        DevBuf y32;
        if (evecs) BRI_TRY_CUDA(ctx, cudaMalloc(&y32.p, sizeof(float2) * ctx->ov->n * nev));
        BRI_RETURN_IF(lanczos<float2>(ctx, prec, m0, nev, max_krylov, tol, nullptr, 0, y32.as<float2>(), 0x1012ull, r,
                                      s));
        if (evecs) {
            k_f32_to_f64<<<vec_blocks(ctx->ov->n * nev), VT, 0, s>>>((double2 *)evecs, y32.as<float2>(),
                                                                      ctx->ov->n * nev);
            BRI_LAUNCHED(ctx);
            BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        }
    }
    for (int k = 0; k < nev; k++) evals[k] = r.theta[k];
    if (lmax) *lmax = r.theta[nev];
    double mr = 0.0;
    for (int k = 0; k <= nev; k++) mr = std::max(mr, r.resid[k] / std::max(fabs(r.theta[k]), 1e-300));
    if (info) {
        info->nconv = r.nconv;
        info->krylov_dim = r.m;
        info->applies = r.applies;
        info->max_resid = mr;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->status = r.converged ? BRI_OK : BRI_ENOTCONV;
    }
    return r.converged ? BRI_OK : BRI_ENOTCONV;
}

bri_status bri_overlap_setup_impl(bri_ctx *ctx, double rho, int nlow, double eps, int max_krylov, double tol,
                                  bri_prec prec, bri_overlap_info *info, cudaStream_t s) {
    auto t0 = std::chrono::steady_clock::now();
    BRI_RETURN_IF(ensure_ov(ctx));
    OverlapWork *o = ctx->ov;
    o->ready = false;
    const size_t n = o->n;
    free_ptr(o->Z);
    free_ptr(o->Z32);
    free_ptr(o->lam);
    o->Z = nullptr;
    o->Z32 = nullptr;
    o->lam = nullptr;
    o->nlow = 0;
    o->rho = rho;
    o->prec = prec;
    BRI_RETURN_IF(alloc_vecs(ctx, prec));
    BRI_RETURN_IF(ensure_red(ctx, MAX_WANT));
    const double m0 = -rho;
    SetupStats st;
    if (nlow > 0) BRI_TRY_CUDA(ctx, cudaMalloc(&o->lam, sizeof(double) * nlow));
    if (prec == BRI_F64) {
        if (nlow > 0) BRI_TRY_CUDA(ctx, cudaMalloc(&o->Z, sizeof(double2) * n * nlow));
        BRI_RETURN_IF(setup_modes<double2>(ctx, BRI_F64, m0, nlow, max_krylov, tol, o->Z, st, s));
    } else {
        // FP32 / FP16 polynomial: the Lanczos runs, the Rayleigh-Ritz step and the
        // deflation vectors in FP32 too (their accuracy matches the polynomial's);
        // an FP64 copy of the vectors serves the FP64 deflation of the input
        if (nlow > 0) {
            BRI_TRY_CUDA(ctx, cudaMalloc(&o->Z32, sizeof(float2) * n * nlow));
            BRI_TRY_CUDA(ctx, cudaMalloc(&o->Z, sizeof(double2) * n * nlow));
        }
        BRI_RETURN_IF(setup_modes<float2>(ctx, prec, m0, nlow, max_krylov, std::max(tol, 1e-6), o->Z32, st, s));
        if (nlow > 0) {
            k_f32_to_f64<<<vec_blocks(n * nlow), VT, 0, s>>>(o->Z, o->Z32, n * nlow);
            BRI_LAUNCHED(ctx);
        }
    }
    const double lo = st.lo, hi = st.hi, defl_resid = st.defl_resid;
    const int applies = st.applies, kdim = st.kdim;
    if (!(lo > 0.0) || !(hi > lo)) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "overlap setup: H^2 has a (near) zero mode outside the deflated space (interval [%.3e, %.3e])", lo, hi);
        return bri_fail(ctx, BRI_EINVAL, msg);
    }
    double err = 0.0;
    BRI_RETURN_IF(build_poly(ctx, lo, hi, eps, o->coef, err, s));
    o->lo = lo;
    o->hi = hi;
    o->degree = (int)o->coef.size() - 1;
    o->gen = ctx->gen;
    o->ready = true;
    if (info) {
        info->nlow = nlow;
        info->degree = o->degree;
        info->lo = lo;
        info->hi = hi;
        info->err_bound = err;
        info->defl_resid = defl_resid;
        info->krylov_dim = kdim;
        info->applies = applies;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->status = BRI_OK;
    }
    return BRI_OK;
}

bri_status bri_overlap_check(bri_ctx *ctx) {
    OverlapWork *o = ctx->ov;
    if (!o || !o->ready) return bri_fail(ctx, BRI_ESTATE, "call bri_overlap_setup first");
    if (o->gen != ctx->gen) return bri_fail(ctx, BRI_ESTATE, "operator changed since bri_overlap_setup; call it again");
    return BRI_OK;
}

bri_status bri_overlap_modes_impl(bri_ctx *ctx, double *lambda, double *vecs, cudaStream_t s) {
    BRI_RETURN_IF(bri_overlap_check(ctx));
    OverlapWork *o = ctx->ov;
    if (o->nlow == 0) return BRI_OK;
    if (lambda) {
        BRI_TRY_CUDA(ctx, cudaMemcpyAsync(lambda, o->lam, sizeof(double) * o->nlow, cudaMemcpyDeviceToHost, s));
        BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    }
    if (vecs)
        BRI_TRY_CUDA(ctx, cudaMemcpyAsync(vecs, o->Z, sizeof(double2) * o->n * o->nlow, cudaMemcpyDeviceToDevice, s));
    return BRI_OK;
}

// mode 0: out = sign(H) in; mode 1: out = D_ov,m in
bri_status bri_overlap_apply_impl(bri_ctx *ctx, double *out, const double *in, int nrhs, int mode, double m,
                                  cudaStream_t s) {
    BRI_RETURN_IF(bri_overlap_check(ctx));
    OverlapWork *o = ctx->ov;
    const size_t n = o->n;
    for (int r = 0; r < nrhs; r++) {
        const double2 *x = (const double2 *)in + (size_t)r * n;
        double2 *y = (double2 *)out + (size_t)r * n;
        if (mode == 0) {
            BRI_RETURN_IF(sign_one(ctx, y, x, s));
        } else {
            double2 *sg = o->v64[6];
            BRI_RETURN_IF(sign_one(ctx, sg, x, s));
            k_overlap_final<<<vec_blocks(n), VT, 0, s>>>(y, x, sg, o->rho - 0.5 * m, m, n);
            BRI_LAUNCHED(ctx);
        }
    }
    return BRI_OK;
}
