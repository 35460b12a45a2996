// Link precompute: path-averaged hops (Sec. 5.1), SU(3) back-projection
// (Sec. 5.2) and storage in reduced precision / compressed SU(3) forms.
//
// Path sums by dynamic programming over the first step of every path:
//   A_d(x) = (1/n) sum_{mu in supp d} F_{mu, d_mu}(x) A_{d - d_mu mu}(x + d_mu mu),
//   F_{mu,+}(x) = U_mu(x),  F_{mu,-}(x) = U_mu(x - mu)^dagger,  A_0 = 1,
// which is the average over all n! shortest paths (every path starts with one
// of the n unit steps of d).  The factor 1/n per level only rescales A and the
// projection is invariant under positive rescaling.  Level n reads level n-1
// at neighbouring sites, so each level is one launch over (site, offset).
#include <cuda_fp16.h>

#include "ctx.h"
#include "links.cuh"
#include "project.cuh"

using namespace bri;

namespace {

// A: [81][V] of M3<double2> (offset-major), U: [V][4][9]
__global__ void k_dp_level(int n, const int *__restrict__ klist, int nk, const double2 *__restrict__ U,
                           M3<double2> *__restrict__ A, Geom g) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= g.V || blockIdx.y >= (unsigned)nk) return;
    const int k = klist[blockIdx.y];
    int x[4];
    SiteNb nb = site_nb(g, site, x);
    M3<double2> acc = m3_zero<double2>();
    int p3 = 1;
    for (int mu = 0; mu < 4; mu++, p3 *= 3) {
        const int c = (k / p3) % 3 - 1;
        if (c == 0) continue;
        M3<double2> F;
        if (c > 0) {
            const double2 *u = U + ((size_t)site * 4 + mu) * 9;
#pragma unroll
            for (int i = 0; i < 9; i++) F.e[i] = u[i];
        } else {
            const double2 *u = U + ((size_t)(site + nb.bw[mu]) * 4 + mu) * 9;
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) F.e[3 * i + j] = cconj(u[3 * j + i]);
        }
        if (n == 1) {
            acc = F;
        } else {
            const int y = site + (c > 0 ? nb.fw[mu] : nb.bw[mu]);
            const int kk = k - c * p3;
            acc = m3_mad(acc, F, A[(size_t)kk * g.V + y]);
        }
    }
    const double inv = 1.0 / n;
#pragma unroll
    for (int i = 0; i < 9; i++) acc.e[i] = cscale(acc.e[i], inv);
    A[(size_t)k * g.V + site] = acc;
}

// canonical fields: W_j(x) = A (1-hop) or P_SU(3)(A) (2..4 hops); hops64: [40][9][V]
__global__ void k_project_hops(const M3<double2> *__restrict__ A, double2 *__restrict__ hops64, Geom g) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (site >= g.V) return;
    const int k = canon_k(j);
    M3<double2> a = A[(size_t)k * g.V + site];
    M3<double2> w = off_class(k) == 1 ? a : project_su3(a);
#pragma unroll
    for (int e = 0; e < 9; e++) hops64[((size_t)j * 9 + e) * g.V + site] = w.e[e];
}

__global__ void k_project_batch(const M3<double2> *__restrict__ A, M3<double2> *__restrict__ Y, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    M3<double2> a = A[i];
    Y[i] = project_su3(a);
}

// ---- reduced-precision stores -------------------------------------------------
// chunk q (of nq) of field j at site s in the 32-site blocked layout of the
// FP32/FP16 stores (links.cuh): [40][Vp/32][nq][32], Vp = V rounded up to 32
BRI_D size_t blk_idx(int j, int q, int s, int nq, size_t VP) {
    return ((size_t)j * VP + (s & ~31)) * nq + (size_t)q * 32 + (s & 31);
}
BRI_HD size_t pad32(size_t V) { return (V + 31) & ~(size_t)31; }

template <bri_comp C> __global__ void k_store_f32(const double2 *__restrict__ h, LinkStore st, Geom g) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (site >= g.V) return;
    double2 w[9];
#pragma unroll
    for (int e = 0; e < 9; e++) w[e] = h[((size_t)j * 9 + e) * g.V + site];
    float4 *a = (float4 *)st.a;
    const size_t VP = pad32(g.V);
    if (C == BRI_LINK_FULL) {
#pragma unroll
        for (int q = 0; q < 4; q++)
            a[blk_idx(j, q, site, 4, VP)] =
                make_float4((float)w[2 * q].x, (float)w[2 * q].y, (float)w[2 * q + 1].x, (float)w[2 * q + 1].y);
        ((float2 *)st.b)[(size_t)j * VP + site] = make_float2((float)w[8].x, (float)w[8].y);
    } else if (C == BRI_LINK_2ROW) {
#pragma unroll
        for (int q = 0; q < 3; q++)
            a[blk_idx(j, q, site, 3, VP)] =
                make_float4((float)w[2 * q].x, (float)w[2 * q].y, (float)w[2 * q + 1].x, (float)w[2 * q + 1].y);
    } else {
        float p[8];
        eight_params(w, p);
        a[blk_idx(j, 0, site, 2, VP)] = make_float4(p[0], p[1], p[2], p[3]);
        a[blk_idx(j, 1, site, 2, VP)] = make_float4(p[4], p[5], p[6], p[7]);
    }
}

BRI_D uint32_t pack_h2(double a, double b) {
    __half2 h = __floats2half2_rn((float)a, (float)b);
    return *reinterpret_cast<uint32_t *>(&h);
}

template <bri_comp C> __global__ void k_store_f16(const double2 *__restrict__ h, LinkStore st, Geom g) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (site >= g.V) return;
    double2 w[9];
#pragma unroll
    for (int e = 0; e < 9; e++) w[e] = h[((size_t)j * 9 + e) * g.V + site];
    uint4 *a = (uint4 *)st.a;
    const size_t VP = pad32(g.V);
    if (C == BRI_LINK_FULL) {
#pragma unroll
        for (int q = 0; q < 2; q++)
            a[blk_idx(j, q, site, 2, VP)] =
                make_uint4(pack_h2(w[4 * q].x, w[4 * q].y), pack_h2(w[4 * q + 1].x, w[4 * q + 1].y),
                           pack_h2(w[4 * q + 2].x, w[4 * q + 2].y), pack_h2(w[4 * q + 3].x, w[4 * q + 3].y));
        ((uint32_t *)st.b)[(size_t)j * VP + site] = pack_h2(w[8].x, w[8].y);
    } else if (C == BRI_LINK_2ROW) {
        a[blk_idx(j, 0, site, 1, VP)] = make_uint4(pack_h2(w[0].x, w[0].y), pack_h2(w[1].x, w[1].y),
                                                   pack_h2(w[2].x, w[2].y), pack_h2(w[3].x, w[3].y));
        ((uint2 *)st.b)[(size_t)j * VP + site] = make_uint2(pack_h2(w[4].x, w[4].y), pack_h2(w[5].x, w[5].y));
    } else {
        float p[8];
        eight_params(w, p);
        a[blk_idx(j, 0, site, 1, VP)] =
            make_uint4(pack_h2(p[0], p[1]), pack_h2(p[2], p[3]), pack_h2(p[4], p[5]), pack_h2(p[6], p[7]));
    }
}

// site-pair interleaved copies: entry e of field j for sites (i, i + V/2) as
// (Re_i, Re_{i+V/2}, Im_i, Im_{i+V/2}); E = 9 (full) or 6 (2-row)
template <int E> __global__ void k_store_pair_f32(const double2 *__restrict__ h, float4 *__restrict__ out, Geom g) {
    const int H = g.V / 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= H) return;
#pragma unroll
    for (int e = 0; e < E; e++) {
        const double2 wa = h[((size_t)j * 9 + e) * g.V + i], wb = h[((size_t)j * 9 + e) * g.V + i + H];
        out[((size_t)j * E + e) * H + i] = make_float4((float)wa.x, (float)wb.x, (float)wa.y, (float)wb.y);
    }
}
template <int E> __global__ void k_store_pair_f16(const double2 *__restrict__ h, uint2 *__restrict__ out, Geom g) {
    const int H = g.V / 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= H) return;
#pragma unroll
    for (int e = 0; e < E; e++) {
        const double2 wa = h[((size_t)j * 9 + e) * g.V + i], wb = h[((size_t)j * 9 + e) * g.V + i + H];
        out[((size_t)j * E + e) * H + i] = make_uint2(pack_h2(wa.x, wb.x), pack_h2(wa.y, wb.y));
    }
}

// [40][9][V] -> [V][40][9]
__global__ void k_export_hops(const double2 *__restrict__ h, double2 *__restrict__ out, Geom g) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (site >= g.V) return;
#pragma unroll
    for (int e = 0; e < 9; e++) out[((size_t)site * NCANON + j) * 9 + e] = h[((size_t)j * 9 + e) * g.V + site];
}

size_t store_bytes_a(bri_prec p, bri_comp c) {
    if (p == BRI_F32) return c == BRI_LINK_FULL ? 64 : c == BRI_LINK_2ROW ? 48 : 32;
    return c == BRI_LINK_FULL ? 32 : 16;
}
size_t store_bytes_b(bri_prec p, bri_comp c) {
    if (p == BRI_F32) return c == BRI_LINK_FULL ? 8 : 0;
    return c == BRI_LINK_FULL ? 4 : c == BRI_LINK_2ROW ? 8 : 0;
}

}  // namespace

// path sums of every offset into A ([81][V]); klist/start: offsets packed by class
bri_status bri_dp_levels(bri_ctx *ctx, void *Av, const int *klist, const int start[6], cudaStream_t s) {
    const Geom g = ctx->g;
    const size_t V = g.V;
    M3<double2> *A = (M3<double2> *)Av;
    const int T = 128;
    for (int n = 1; n <= 4; n++) {
        dim3 grid((unsigned)((V + T - 1) / T), (unsigned)(start[n + 1] - start[n]));
        k_dp_level<<<grid, T, 0, s>>>(n, klist + start[n], start[n + 1] - start[n], ctx->U, A, g);
        BRI_LAUNCHED(ctx);
    }
    return BRI_OK;
}

bri_status bri_hops_build_impl(bri_ctx *ctx, cudaStream_t s) {
    const Geom g = ctx->g;
    const size_t V = g.V;
    if (!ctx->hops64) BRI_TRY_CUDA(ctx, cudaMalloc(&ctx->hops64, sizeof(double2) * 9 * NCANON * V));
    M3<double2> *A = nullptr;
    int *klist = nullptr;
    BRI_TRY_CUDA(ctx, cudaMallocAsync((void **)&A, sizeof(M3<double2>) * NOFF * V, s));
    BRI_TRY_CUDA(ctx, cudaMallocAsync((void **)&klist, sizeof(int) * NOFF, s));
    int hk[NOFF], start[6] = {0}, cnt = 0;
    for (int n = 1; n <= 4; n++) {
        start[n] = cnt;
        for (int k = 0; k < NOFF; k++)
            if (off_class(k) == n) hk[cnt++] = k;
    }
    start[5] = cnt;
    BRI_TRY_CUDA(ctx, cudaMemcpyAsync(klist, hk, sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
    BRI_RETURN_IF(bri_dp_levels(ctx, A, klist, start, s));
    const int T = 128;
    {
        dim3 grid((unsigned)((V + T - 1) / T), NCANON);
        k_project_hops<<<grid, T, 0, s>>>(A, ctx->hops64, g);
        BRI_LAUNCHED(ctx);
    }
    BRI_TRY_CUDA(ctx, cudaFreeAsync(A, s));
    BRI_TRY_CUDA(ctx, cudaFreeAsync(klist, s));
    ctx->have64 = true;
    ctx->f32.valid = false;
    ctx->f16.valid = false;
    ctx->p32.valid = false;
    ctx->p16.valid = false;
    return BRI_OK;
}

bri_status bri_hops_store_impl(bri_ctx *ctx, bri_prec prec, bri_comp comp, cudaStream_t s) {
    if (prec == BRI_F64) return BRI_OK;
    LinkStore &st = prec == BRI_F32 ? ctx->f32 : ctx->f16;
    const size_t V = ctx->g.V;
    // (re)allocate for this compression
    if (st.a && st.comp != comp) {
        cudaFree(st.a);
        if (st.b) cudaFree(st.b);
        st.a = st.b = nullptr;
    }
    st.valid = false;
    if (!st.a) {
        BRI_TRY_CUDA(ctx, cudaMalloc(&st.a, store_bytes_a(prec, comp) * NCANON * pad32(V)));
        size_t nb = store_bytes_b(prec, comp);
        if (nb) BRI_TRY_CUDA(ctx, cudaMalloc(&st.b, nb * NCANON * pad32(V)));
    }
    st.comp = comp;
    const int T = 128;
    dim3 grid((unsigned)((V + T - 1) / T), NCANON);
    if (prec == BRI_F32) {
        if (comp == BRI_LINK_FULL) k_store_f32<BRI_LINK_FULL><<<grid, T, 0, s>>>(ctx->hops64, st, ctx->g);
        else if (comp == BRI_LINK_2ROW) k_store_f32<BRI_LINK_2ROW><<<grid, T, 0, s>>>(ctx->hops64, st, ctx->g);
        else k_store_f32<BRI_LINK_8PARAM><<<grid, T, 0, s>>>(ctx->hops64, st, ctx->g);
    } else {
        if (comp == BRI_LINK_FULL) k_store_f16<BRI_LINK_FULL><<<grid, T, 0, s>>>(ctx->hops64, st, ctx->g);
        else if (comp == BRI_LINK_2ROW) k_store_f16<BRI_LINK_2ROW><<<grid, T, 0, s>>>(ctx->hops64, st, ctx->g);
        else k_store_f16<BRI_LINK_8PARAM><<<grid, T, 0, s>>>(ctx->hops64, st, ctx->g);
    }
    BRI_LAUNCHED(ctx);
    st.valid = true;
    // the site-pair copy follows on first use of its launch variant
    (prec == BRI_F32 ? ctx->p32 : ctx->p16).valid = false;
    return BRI_OK;
}

// site-pair interleaved copy of the stored fields for the pair kernel (full
// and 2-row storage, even t extent), built from the FP64 fields when the pair
// launch variant is first asked for
bri_status bri_pair_store_impl(bri_ctx *ctx, bri_prec prec, cudaStream_t s) {
    const LinkStore &st = prec == BRI_F32 ? ctx->f32 : ctx->f16;
    LinkStore &ps = prec == BRI_F32 ? ctx->p32 : ctx->p16;
    const bri_comp comp = st.comp;
    const size_t V = ctx->g.V;
    const int T = 128;
    ps.valid = false;
    if (!ctx->have64 || comp == BRI_LINK_8PARAM || ctx->g.L[3] % 2 != 0) return BRI_OK;
    const int E = comp == BRI_LINK_FULL ? 9 : 6;
    if (ps.a && ps.comp != comp) {
        cudaFree(ps.a);
        ps.a = nullptr;
    }
    if (!ps.a) BRI_TRY_CUDA(ctx, cudaMalloc(&ps.a, (prec == BRI_F32 ? 16 : 8) * (size_t)E * NCANON * (V / 2)));
    ps.comp = comp;
    dim3 pg((unsigned)((V / 2 + T - 1) / T), NCANON);
    if (prec == BRI_F32) {
        if (E == 9) k_store_pair_f32<9><<<pg, T, 0, s>>>(ctx->hops64, (float4 *)ps.a, ctx->g);
        else k_store_pair_f32<6><<<pg, T, 0, s>>>(ctx->hops64, (float4 *)ps.a, ctx->g);
    } else {
        if (E == 9) k_store_pair_f16<9><<<pg, T, 0, s>>>(ctx->hops64, (uint2 *)ps.a, ctx->g);
        else k_store_pair_f16<6><<<pg, T, 0, s>>>(ctx->hops64, (uint2 *)ps.a, ctx->g);
    }
    BRI_LAUNCHED(ctx);
    ps.valid = true;
    return BRI_OK;
}

bri_status bri_project_impl(bri_ctx *ctx, double2 *Y, const double2 *A, long n, cudaStream_t s) {
    if (n == 0) return BRI_OK;
    const int T = 128;
    k_project_batch<<<(unsigned)((n + T - 1) / T), T, 0, s>>>((const M3<double2> *)A, (M3<double2> *)Y, n);
    BRI_LAUNCHED(ctx);
    return BRI_OK;
}

bri_status bri_export_hops_impl(bri_ctx *ctx, double2 *out, cudaStream_t s) {
    const int T = 128;
    dim3 grid((unsigned)((ctx->g.V + T - 1) / T), NCANON);
    k_export_hops<<<grid, T, 0, s>>>(ctx->hops64, out, ctx->g);
    BRI_LAUNCHED(ctx);
    return BRI_OK;
}
