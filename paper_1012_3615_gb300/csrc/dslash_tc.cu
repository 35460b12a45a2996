// Multi-RHS stencil apply on the tensor cores (mma.sync m16n8k16, FP16
// operands, FP32 accumulation): launch variant 8 for FP32 and FP16 fields in
// full storage.
//
// Per site x the class form of Sec. 8 is one small dense contraction.  With
// K = (hop h, colour c') over the 80 hops (240 complex), the five
// accumulators k = 0 (lambda) and k = 1..4 (rho gamma_mu) and the colour c:
//
//   T_k[c][(s', r)] = sum_{h, c'} B_k(h) W_h(x)[c][c'] psi_r(x + d_h)[s'][c']
//   B_0(h) = s_h lambda_n,  B_mu(h) = s_h rho_n d_mu       (n = |d_h|_1)
//   out_r(x)[s][c]  = (m0 + lambda_0) psi_r(x)[s][c] + T_0[c][(s, r)]
//                   + sum_mu (gamma_mu)_{s, s'} T_mu[c][(s', r)]
//
// i.e. a (15 x 240) x (240 x 4N) complex product per site: the links, scaled
// by the class weights (A operand), times the gathered neighbour spinors of
// all right-hand sides (B operand).  Complex arithmetic as real: the A operand
// is the 32 x 480 real embedding [[Re, -Im], [Im, Re]] (rows: real parts of the
// 15 (k, c) columns then their imaginary parts, padded to 16 each), the B
// operand holds (Re, Im) of each spinor entry in consecutive K rows, so every
// B register is one complex number as an f16 pair.  One warp owns one site and
// up to 12 right-hand sides (6 n-tiles of 8 (s', r) columns); a k-step of 16
// covers 8 complex K slots, and three k-steps cover 8 hops: in the first two,
// lane group t takes hop t (resp. 4 + t) with colours 0 and 1, in the third
// hops 2t and 2t + 1 with colour 2.
//
// Precision: the A operand is f16(64 B_k W) and the B operand f16(psi / sigma_r)
// with sigma_r a power of two per right-hand side (max |psi_r| / sigma_r in
// [512, 1024)), so no operand over- or underflows; products are summed in
// FP32.  Relative accuracy is that of 11-bit operands (~1e-4 of max |out|),
// the diagonal term is added in FP32.  The clover term and site ranges are not
// taken by this kernel (the dispatcher uses the FP32-arithmetic stencil there).
#include <algorithm>

#include "ctx.h"
#include "links.cuh"

namespace bri {

constexpr int TC_WARPS = 4;            // warps per block
constexpr int TC_SITES = 16;           // sites per block: a 2x2x2x2 tile when every extent is even
constexpr int TC_MAXNT = 6;            // n-tiles of 8 columns per warp (12 RHS)
constexpr float TC_ASCALE = 64.f;      // A operand scale (keeps the small weights normal in f16)
constexpr int TC_MAXH = 2 * NCANON;    // hops

// per-warp shared memory: the site's 80 link matrices (backward hops already
// daggered), later reused for the epilogue; neighbour sites; weights.  The
// arrays are entry-major with a padded hop stride (81), so lanes that touch
// consecutive hops, or the same hop at different entries, hit distinct banks.
constexpr int TC_HS = TC_MAXH + 1;
struct TcShared {
    union {
        float2 W[9][TC_HS];                // W_h[c][c'] as the hop uses it, at W[3 c + c'][h]
        float2 T[2 * TC_MAXNT][4][17];     // epilogue: T[r][s'][k c] (padded)
    } u;
    int y[TC_MAXH];        // neighbour site of hop h
    float cf[5][TC_HS];    // accumulator weights x boundary phase x TC_ASCALE, cf[k][h]
    float sc[2 * TC_MAXNT];  // output scale sigma_r / TC_ASCALE of the chunk's right-hand sides
};

BRI_D uint32_t pack_h2(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

BRI_D void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// power-of-two scale of a right-hand side from its max |component| m:
// psi / sigma has max in [512, 1024)
BRI_D float tc_inv_sigma(unsigned mbits) {
    const float m = __uint_as_float(mbits);
    int e2;
    frexpf(m, &e2);
    return m > 0.f ? ldexpf(1.f, 10 - e2) : 1.f;
}

// FP16 copy of the spinors for the B operand: [V][Rp][4 spins][4 colours]
// half2 (colour 3 zero, right-hand sides >= nrhs zero), each entry psi / sigma_r
__global__ void k_tc_pack(const float2 *__restrict__ in, uint4 *__restrict__ f, int V, int nrhs, int Rp,
                          const unsigned *__restrict__ amax) {
    const size_t n = (size_t)V * Rp * 4;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int sp = (int)(i & 3);
        const size_t q = i >> 2;
        const int r = (int)(q % Rp);
        const size_t site = q / Rp;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r < nrhs) {
            const float is = tc_inv_sigma(amax[r]);
            const float2 *p = in + ((size_t)r * V + site) * 12 + 3 * sp;
            const float2 a = p[0], b = p[1], c = p[2];
            v = make_uint4(pack_h2(a.x * is, a.y * is), pack_h2(b.x * is, b.y * is), pack_h2(c.x * is, c.y * is), 0u);
        }
        f[i] = v;
    }
}

// the apply at one site for right-hand sides r0 .. r0 + nr - 1 (one warp)
template <class LL, int NT>
__device__ __forceinline__ void tc_site(int mode, const LL &ll, const float2 *__restrict__ in,
                                        const uint32_t *__restrict__ f, float2 *__restrict__ out, int site, int r0,
                                        int nr, int Rp, const Geom &g, const HopArg *hops, float diag,
                                        const unsigned *__restrict__ amax, const int *__restrict__ skip,
                                        TcShared &S, int lane) {
    const float rsign = mode == 1 ? -1.f : 1.f;
    if (lane < nr) S.sc[lane] = 1.f / (tc_inv_sigma(amax[r0 + lane]) * TC_ASCALE);

    // hop table of this site and its link matrices
    int x[4];
    const SiteNb nb = site_nb(g, site, x);
    const int nh = 2 * g.nhop;
    for (int h = lane; h < nh; h += 32) {
        const HopArg &hp = hops[h >> 1];
        int yf, yb;
        float phf, phb;
        hop_nb(hp.dm, site, nb, yf, phf, yb, phb);
        const int dir = h & 1;
        const float ph = (dir ? phb : phf) * TC_ASCALE;
        S.y[h] = dir ? yb : yf;
        S.cf[0][h] = hp.lam * ph;
#pragma unroll
        for (int mu = 0; mu < 4; mu++) S.cf[1 + mu][h] = hp.rho * hp.fd[mu] * rsign * (dir ? -ph : ph);
        const M3<float2> m = ll.load(hp.j, dir ? yb : site);
#pragma unroll
        for (int c = 0; c < 3; c++)
#pragma unroll
            for (int cp = 0; cp < 3; cp++)
                S.u.W[3 * c + cp][h] = dir ? cconj(m.e[3 * cp + c]) : m.e[3 * c + cp];
    }
    __syncwarp();

    const int gid = lane >> 2, tig = lane & 3;
    // A rows of this lane: nc = gid and gid + 8 (k = nc / 3, colour nc % 3); nc = 15 is padding
    const int k1 = gid / 3, cc1 = gid - 3 * k1;
    const int n2 = gid + 8;
    const float pad2 = n2 == 15 ? 0.f : 1.f;
    // the padding row reads accumulator 4's weight (times 0): k stays in 0..4
    const int k2 = n2 == 15 ? 4 : n2 / 3, cc2 = n2 == 15 ? 0 : n2 - 3 * k2;
    // B column of this lane in n-tile t: (r, s') = (r0 + 2 t + gid / 4, gid % 4); its FP16
    // row of site y starts at ((y Rp + r0 + gid / 4) 4 + gid % 4) 4, n-tiles 32 apart
    const uint32_t lrow = (uint32_t)(((r0 + (gid >> 2)) * 4 + (gid & 3)) * 4);
    const size_t ystride = (size_t)Rp * 16;

    float acc[2][NT][4];
#pragma unroll
    for (int p = 0; p < 2; p++)
#pragma unroll
        for (int t = 0; t < NT; t++)
#pragma unroll
            for (int i = 0; i < 4; i++) acc[p][t][i] = 0.f;

    const int ng = (nh + 7) / 8;
#pragma unroll 1
    for (int G = 0; G < ng; G++) {
        // lane group tig owns hops hA = 8G + tig and hB = 8G + 4 + tig; the three
        // k-steps take (hA c'0, hA c'1), (hB c'0, hB c'1), (hA c'2, hB c'2) as its
        // two K slots, so each lane loads every spinor row it needs once
        const int hA = 8 * G + tig, hB = hA + 4;
        const bool vA = hA < nh, vB = hB < nh;
        const uint32_t *fA = f + (vA ? (size_t)S.y[hA] * ystride + lrow : 0);
        const uint32_t *fB = f + (vB ? (size_t)S.y[hB] * ystride + lrow : 0);
        // B operands of the group, all n-tiles: one 16-byte row (c'0, c'1, c'2, 0) per hop
        uint4 rA[NT], rB[NT];
#pragma unroll
        for (int t = 0; t < NT; t++) {
            rA[t] = vA ? *reinterpret_cast<const uint4 *>(fA + 32 * t) : make_uint4(0u, 0u, 0u, 0u);
            rB[t] = vB ? *reinterpret_cast<const uint4 *>(fB + 32 * t) : make_uint4(0u, 0u, 0u, 0u);
        }
        // A operand weights and link entries of the two hops
        const int hA0 = vA ? hA : 0, hB0 = vB ? hB : 0;
        const float fA1 = vA ? S.cf[k1][hA0] : 0.f, fA2 = vA ? S.cf[k2][hA0] * pad2 : 0.f;
        const float fB1 = vB ? S.cf[k1][hB0] : 0.f, fB2 = vB ? S.cf[k2][hB0] * pad2 : 0.f;
#pragma unroll
        for (int st = 0; st < 3; st++) {
            // slots: (h1, c1) and (h2, c2) of this k-step
            const int h1 = st == 1 ? hB0 : hA0, h2 = st == 0 ? hA0 : hB0;
            const int c1 = st < 2 ? 0 : 2, c2 = st < 2 ? 1 : 2;
            const float g11 = st == 1 ? fB1 : fA1, g12 = st == 1 ? fB2 : fA2;
            const float g21 = st == 0 ? fA1 : fB1, g22 = st == 0 ? fA2 : fB2;
            const float2 w1 = S.u.W[3 * cc1 + c1][h1], w2 = S.u.W[3 * cc2 + c1][h1];
            const float2 w3 = S.u.W[3 * cc1 + c2][h2], w4 = S.u.W[3 * cc2 + c2][h2];
            const float2 z[4] = {make_float2(g11 * w1.x, g11 * w1.y), make_float2(g12 * w2.x, g12 * w2.y),
                                 make_float2(g21 * w3.x, g21 * w3.y), make_float2(g22 * w4.x, g22 * w4.y)};
            // m-tile 0 (real parts of the outputs): (Re z, -Im z); m-tile 1: (Im z, Re z);
            // register order of the A fragment: (g, s1) (g+8, s1) (g, s2) (g+8, s2)
            uint32_t are[4], aim[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                are[q] = pack_h2(z[q].x, -z[q].y);
                aim[q] = pack_h2(z[q].y, z[q].x);
            }
#pragma unroll
            for (int t = 0; t < NT; t++) {
                const uint32_t b0 = st == 0 ? rA[t].x : st == 1 ? rB[t].x : rA[t].z;
                const uint32_t b1 = st == 0 ? rA[t].y : st == 1 ? rB[t].y : rB[t].z;
                mma16816(acc[0][t], are, b0, b1);
                mma16816(acc[1][t], aim, b0, b1);
            }
        }
    }

    // epilogue: accumulators to shared memory as T[r][s'][nc] (complex), then
    // the gamma structure, the scales and the diagonal per output entry
    __syncwarp();
#pragma unroll
    for (int t = 0; t < NT; t++) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int col = 2 * tig + (i & 1);
            const int rl = 2 * t + (col >> 2), s = col & 3;
            const int nc = gid + ((i >> 1) << 3);
            S.u.T[rl][s][nc] = make_float2(acc[0][t][i], acc[1][t][i]);
        }
    }
    __syncwarp();
    for (int o = lane; o < nr * 12; o += 32) {
        const int rl = o / 12, s = (o - 12 * rl) / 3, c = o - 12 * rl - 3 * s;
        const int r = r0 + rl;
        if (skip && skip[r]) continue;
        float2 vv = S.u.T[rl][s][c];
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            const float2 tv = S.u.T[rl][gcol(mu, s)][3 * (mu + 1) + c];
            const float gr = (float)gre(mu, s), gi = (float)gim(mu, s);
            vv.x += gr * tv.x - gi * tv.y;
            vv.y += gr * tv.y + gi * tv.x;
        }
        const float sc = S.sc[rl];
        const size_t idx = ((size_t)r * g.V + site) * 12 + 3 * s + c;
        const float2 p = in[idx];
        float2 res = make_float2(diag * p.x + sc * vv.x, diag * p.y + sc * vv.y);
        if (mode == 2 && s >= 2) res = make_float2(-res.x, -res.y);
        out[idx] = res;
    }
    __syncwarp();  // the next site of this warp reuses S
}

// One block per tile of TC_SITES sites and chunk of right-hand sides (chunk
// fastest); each warp takes TC_SITES / TC_WARPS sites of the tile one after the
// other.  A 2x2x2x2 tile keeps the union of its sites' neighbourhoods (4^4
// sites) small, so neighbour rows fetched for one site are found in L1 by the
// next.  The hop table moves from the kernel parameters to shared memory once
// per block (the per-site set-up indexes it per lane).
template <class LL, int NT>
__global__ void __launch_bounds__(32 * TC_WARPS) k_dslash_tc(int mode, LL ll, const float2 *__restrict__ in,
                                                            const uint32_t *__restrict__ f, float2 *__restrict__ out,
                                                            int nrhs, int rchunk, int Rp, Geom g, float diag,
                                                            const unsigned *__restrict__ amax,
                                                            const int *__restrict__ skip) {
    __shared__ TcShared shm[TC_WARPS];
    __shared__ HopArg hops[NCANON];
    constexpr int HW = (int)(sizeof(HopArg) / sizeof(int));
    for (int i = threadIdx.x; i < g.nhop * HW; i += blockDim.x)
        reinterpret_cast<int *>(hops)[i] = reinterpret_cast<const int *>(g.hop)[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nchunks = (nrhs + rchunk - 1) / rchunk;
    const int chunk = (int)blockIdx.x % nchunks;
    const int tile = (int)blockIdx.x / nchunks;
    const int r0 = chunk * rchunk;
    const int nr = min(rchunk, nrhs - r0);
    const bool t4 = !((g.L[0] | g.L[1] | g.L[2] | g.L[3]) & 1);
#pragma unroll 1
    for (int it = 0; it < TC_SITES / TC_WARPS; it++) {
        const int l = w + TC_WARPS * it;
        int site;
        if (t4) {
            int q = tile;
            const int tx = q % (g.L[0] >> 1);
            q /= g.L[0] >> 1;
            const int ty = q % (g.L[1] >> 1);
            q /= g.L[1] >> 1;
            const int tz = q % (g.L[2] >> 1);
            const int tt = q / (g.L[2] >> 1);
            site = (2 * tx + (l & 1)) +
                   g.L[0] * ((2 * ty + ((l >> 1) & 1)) + g.L[1] * ((2 * tz + ((l >> 2) & 1)) + g.L[2] * (2 * tt + (l >> 3))));
        } else {
            site = tile * TC_SITES + l;
        }
        if (site < g.V)  // uniform across the warp
            tc_site<LL, NT>(mode, ll, in, f, out, site, r0, nr, Rp, g, hops, diag, amax, skip, shm[w], lane);
    }
}

// max |component| of each right-hand side, as float bits (non-negative floats
// order like their bit patterns); amax must be zero on entry
__global__ void k_absmax(const float *__restrict__ in, size_t per_rhs, unsigned *__restrict__ amax) {
    const int r = blockIdx.y;
    const float *p = in + (size_t)r * per_rhs;
    float m = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_rhs; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(p[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(amax + r, __float_as_uint(m));
}

template <class LL, int NT>
static void launch_tc(int mode, const LL &ll, const float2 *in, const uint32_t *f, float2 *out, int nrhs, int rchunk,
                      int Rp, const Geom &g, float diag, const unsigned *amax, const int *skip, cudaStream_t s) {
    const int nchunks = (nrhs + rchunk - 1) / rchunk;
    const unsigned blocks = (unsigned)((g.V + TC_SITES - 1) / TC_SITES) * (unsigned)nchunks;
    k_dslash_tc<LL, NT><<<blocks, 32 * TC_WARPS, 0, s>>>(mode, ll, in, f, out, nrhs, rchunk, Rp, g, diag, amax, skip);
}

// right-hand sides per warp: at most cap (an even number 2..12, else 12),
// chunks of equal size; the FP16 copy holds Rp = chunks x 2 NT of them
BRI_HD void tc_chunks(int nrhs, int cap, int &rchunk, int &nt, int &Rp) {
    cap = cap >= 2 && cap <= 2 * TC_MAXNT ? cap & ~1 : 2 * TC_MAXNT;
    const int nchunks = (nrhs + cap - 1) / cap;
    rchunk = (nrhs + nchunks - 1) / nchunks;
    nt = (rchunk + 1) / 2;
    Rp = nchunks * 2 * nt;
}

template <class LL>
static void dslash_tc_launch(int mode, const LL &ll, const void *in, void *out, int nrhs, int cap, const Geom &g,
                             double diag, unsigned *amax, uint4 *f, const int *skip, cudaStream_t s) {
    int rchunk, nt, Rp;
    tc_chunks(nrhs, cap, rchunk, nt, Rp);
    cudaMemsetAsync(amax, 0, sizeof(unsigned) * nrhs, s);
    {
        const size_t per = (size_t)g.V * 24;
        const unsigned bx = (unsigned)std::min<size_t>((per + 255) / 256, 152 * 4);
        k_absmax<<<dim3(bx, (unsigned)nrhs), 256, 0, s>>>((const float *)in, per, amax);
    }
    {
        const size_t n = (size_t)g.V * Rp * 4;
        const unsigned bx = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
        k_tc_pack<<<bx, 256, 0, s>>>((const float2 *)in, f, g.V, nrhs, Rp, amax);
    }
    const float2 *ip = (const float2 *)in;
    const uint32_t *fp = (const uint32_t *)f;
    float2 *op = (float2 *)out;
    const float dg = (float)diag;
    switch (nt) {
        case 1: launch_tc<LL, 1>(mode, ll, ip, fp, op, nrhs, rchunk, Rp, g, dg, amax, skip, s); break;
        case 2: launch_tc<LL, 2>(mode, ll, ip, fp, op, nrhs, rchunk, Rp, g, dg, amax, skip, s); break;
        case 3: launch_tc<LL, 3>(mode, ll, ip, fp, op, nrhs, rchunk, Rp, g, dg, amax, skip, s); break;
        case 4: launch_tc<LL, 4>(mode, ll, ip, fp, op, nrhs, rchunk, Rp, g, dg, amax, skip, s); break;
        case 5: launch_tc<LL, 5>(mode, ll, ip, fp, op, nrhs, rchunk, Rp, g, dg, amax, skip, s); break;
        default: launch_tc<LL, 6>(mode, ll, ip, fp, op, nrhs, rchunk, Rp, g, dg, amax, skip, s); break;
    }
}

}  // namespace bri

using namespace bri;

// work buffers of the tensor-core apply for nrhs right-hand sides (cap: as in
// bri_dslash_tc); the apply allocates them on first use, which a stream
// capture does not allow, so callers that capture reserve them first
bri_status bri_tc_reserve(bri_ctx *ctx, int nrhs, int cap) {
    if (!ctx->tc_amax) BRI_TRY_CUDA(ctx, cudaMalloc(&ctx->tc_amax, sizeof(unsigned) * 65536));
    int rchunk, nt, Rp;
    tc_chunks(nrhs, cap & 511, rchunk, nt, Rp);
    const size_t fbytes = (size_t)ctx->g.V * Rp * 4 * sizeof(uint4);
    if (ctx->tc_fbytes < fbytes) {
        cudaFree(ctx->tc_f);
        ctx->tc_f = nullptr;
        ctx->tc_fbytes = 0;
        BRI_TRY_CUDA(ctx, cudaMalloc(&ctx->tc_f, fbytes));
        ctx->tc_fbytes = fbytes;
    }
    return BRI_OK;
}

// the tensor-core apply for the stored FP32 or FP16 fields of prec (full
// storage); the caller has checked that they exist
bri_status bri_dslash_tc(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int mode, bri_prec prec,
                         const int *skip, int cap, cudaStream_t s) {
    const Geom &g = ctx->g;
    const LinkStore &st = prec == BRI_F32 ? ctx->f32 : ctx->f16;
    if (st.comp != BRI_LINK_FULL) return bri_fail(ctx, BRI_EINVAL, "tensor-core apply needs full link storage");
    BRI_RETURN_IF(bri_tc_reserve(ctx, nrhs, cap));
    const int VP = (g.V + 31) & ~31;
    const double diag = m0 + g.lamd[0];
    if (prec == BRI_F32)
        dslash_tc_launch(mode, LinkF32<BRI_LINK_FULL>{(const float4 *)st.a, (const float2 *)st.b, VP}, in, out, nrhs,
                         cap, g, diag, ctx->tc_amax, (uint4 *)ctx->tc_f, skip, s);
    else
        dslash_tc_launch(mode, LinkF16<BRI_LINK_FULL>{(const uint4 *)st.a, st.b, VP}, in, out, nrhs, cap, g, diag,
                         ctx->tc_amax, (uint4 *)ctx->tc_f, skip, s);
    ctx->launches += 2;  // k_absmax, k_tc_pack; BRI_LAUNCHED counts the stencil
    BRI_LAUNCHED(ctx);
    return BRI_OK;
}
