// Stencil apply on FP16 spinors with one FP32 scale per site (prec BRI_F16H):
// FP16 hopping fields, neighbour spinors read as half2 and rescaled, FP32
// arithmetic (the (d, -d) pair loop of the FP32 stencil), result rounded to
// FP16 with a new per-site scale.
//
// Storage of one right-hand side (bri_h16_field_bytes(V) bytes): [V][12] half2
// (spin-major, 48 bytes per site) followed by [V] float scales and unused
// padding to a multiple of 16 bytes; entry = half value x scale.  The writer picks the
// scale as the power of two 2^e with max |component| of the site in
// [2^(e-1), 2^e), so the halves lie in (-1, 1) and carry 11 significant bits
// relative to the site's largest component (reading A14 of the spinor
// precision: FP16 = IEEE binary16, round to nearest).
#include "dslash_kernel.cuh"

namespace bri {

BRI_HD size_t h16_field_bytes(int V) { return (size_t)48 * V + (((size_t)4 * V + 15) & ~(size_t)15); }

struct SpinH16 {
    const uint4 *__restrict__ d;  // 3 x 16 bytes per site
    const float *__restrict__ s;
    BRI_D void load(int y, float2 o[12]) const {
        const uint4 *p = d + (size_t)y * 3;
        const float sc = s[y];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const uint4 v = p[i];
            const float2 a = h2f(v.x), b = h2f(v.y), c = h2f(v.z), e = h2f(v.w);
            o[4 * i] = make_float2(a.x * sc, a.y * sc);
            o[4 * i + 1] = make_float2(b.x * sc, b.y * sc);
            o[4 * i + 2] = make_float2(c.x * sc, c.y * sc);
            o[4 * i + 3] = make_float2(e.x * sc, e.y * sc);
        }
    }
};

BRI_D uint32_t h2pack(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// o[12] of one site to the FP16 field (d, s) with its power-of-two scale
BRI_D void h16_store(uint4 *__restrict__ d, float *__restrict__ s, int site, const float2 o[12]) {
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 12; i++) m = fmaxf(m, fmaxf(fabsf(o[i].x), fabsf(o[i].y)));
    int e = 0;
    frexpf(m, &e);
    const float sc = m > 0.f ? ldexpf(1.f, e) : 1.f, is = m > 0.f ? ldexpf(1.f, -e) : 1.f;
    uint4 *p = d + (size_t)site * 3;
#pragma unroll
    for (int i = 0; i < 3; i++)
        p[i] = make_uint4(h2pack(o[4 * i].x * is, o[4 * i].y * is), h2pack(o[4 * i + 1].x * is, o[4 * i + 1].y * is),
                          h2pack(o[4 * i + 2].x * is, o[4 * i + 2].y * is),
                          h2pack(o[4 * i + 3].x * is, o[4 * i + 3].y * is));
    s[site] = sc;
}

// The FP16-spinor storage for the bulk-copy line kernel (x extent 32): a staged
// x line is the 32 sites' halves (1,536 bytes) followed by their 32 scales
// (128 bytes), each copied as one run.  Halves at a 48-byte pitch, 3 x 16
// bytes per site, fall on distinct bank groups for any 8 consecutive slots.
struct LineSpinH16 {
    static constexpr uint32_t LINE = 32u * 48u + 128u;
    static constexpr bool SCALED = true;
    const uint4 *__restrict__ d;
    const float *__restrict__ s;
    uint4 *__restrict__ od;
    float *__restrict__ os;
    BRI_D LineSpinH16(const void *i, void *o, int rhs, int V) {
        const size_t fb = h16_field_bytes(V);
        const unsigned char *ib = (const unsigned char *)i + rhs * fb;
        unsigned char *ob = (unsigned char *)o + rhs * fb;
        d = (const uint4 *)ib;
        s = (const float *)(ib + (size_t)48 * V);
        od = (uint4 *)ob;
        os = (float *)(ob + (size_t)48 * V);
    }
    BRI_D void issue1(int ln, uint32_t dst, uint32_t bar) const {
        bulk_elect2(bar, LINE, dst, d + (size_t)ln * 96, 1536u, dst + 1536u, s + (size_t)ln * 32, 128u);
    }
    BRI_D void issue2(int l0, int l1, uint32_t dst, uint32_t bar) const {
        bulk_elect4(bar, 2 * LINE, dst, d + (size_t)l0 * 96, 1536u, dst + 1536u, s + (size_t)l0 * 32, 128u,
                    dst + LINE, d + (size_t)l1 * 96, 1536u, dst + LINE + 1536u, s + (size_t)l1 * 32, 128u);
    }
    // the halves at a slot (unscaled) and the site's scale: the loop folds the
    // scale (a power of two) into the pair's coefficients
    BRI_D float load(uint32_t ln, uint32_t slot, float2 o[12]) const {
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const uint4 v = lds4u(ln + 48u * slot + 16u * i);
            o[4 * i] = h2f(v.x);
            o[4 * i + 1] = h2f(v.y);
            o[4 * i + 2] = h2f(v.z);
            o[4 * i + 3] = h2f(v.w);
        }
        return __uint_as_float(lds1u(ln + 1536u + 4u * slot));
    }
    BRI_D void finish(int mode, int site, const Geom &g, double diag, const AccF &acc) const {
        float2 p[12];
        SpinH16{d, s}.load(site, p);
        const float dg = (float)diag;
        float2 o[12];
#pragma unroll
        for (int i = 0; i < 12; i++) {
            o[i].x = dg * p[i].x + acc.a[i].x - acc.ai[i].y;
            o[i].y = dg * p[i].y + acc.a[i].y + acc.ai[i].x;
            if (mode == 2 && i >= 6) { o[i].x = -o[i].x; o[i].y = -o[i].y; }
        }
        h16_store(od, os, site, o);
    }
};

// BODY 2: the gamma terms inside the spin loop (pair_body_s); 3: after it (pair_body)
template <class LL, int BODY>
__global__ void k_dslash_h16(int mode, LL ll, const unsigned char *__restrict__ in, unsigned char *__restrict__ out,
                             Geom g, double diag, const int *__restrict__ skip) {
    const int nblk = (g.s1 - g.s0 + (int)blockDim.x - 1) / (int)blockDim.x;
    const int nr = (int)gridDim.x / nblk;
    const int rhs = (int)blockIdx.x % nr;
    const int site = g.s0 + ((int)blockIdx.x / nr) * (int)blockDim.x + (int)threadIdx.x;
    if (site >= g.s1) return;
    if (skip && skip[rhs]) return;
    const size_t fb = h16_field_bytes(g.V);
    const SpinH16 sp{reinterpret_cast<const uint4 *>(in + rhs * fb),
                     reinterpret_cast<const float *>(in + rhs * fb + (size_t)48 * g.V)};
    int x[4];
    const SiteNb nb = site_nb(g, site, x);
    AccF acc;
#pragma unroll
    for (int i = 0; i < 12; i++) {
        acc.a[i] = make_float2(0.f, 0.f);
        acc.ai[i] = make_float2(0.f, 0.f);
    }
    const float rsign = mode == 1 ? -1.f : 1.f;
#pragma unroll 1
    for (int t = 0; t < g.nhop; t++) {
        if (t + 1 < g.nhop) {  // links of the next pair into L2
            const HopArg hp = g.hop[t + 1];
            int pyf, pyb;
            float pphf, pphb;
            hop_nb(hp.dm, site, nb, pyf, pphf, pyb, pphb);
            ll.prefetch_field_l2(hp.j, site);
            ll.prefetch_field_l2(hp.j, pyb);
        }
        const HopArg hc = g.hop[t];
        int yf, yb;
        float phf, phb;
        hop_nb(hc.dm, site, nb, yf, phf, yb, phb);
        float2 cf[12];
        {
            const M3<float2> W = ll.load(hc.j, site);
            float2 q[12];
            sp.load(yf, q);
            colour_mv<1>(W, q, cf);
        }
        const M3<float2> W = ll.load(hc.j, yb);
        float2 q[12];
        sp.load(yb, q);
        if constexpr (BODY == 3) pair_body(cf, W, q, hc.lam * phf, phf * phb, hc.rho * rsign * phf, hc, acc);
        else pair_body_s<false>(cf, W, q, hc.lam * phf, phf * phb, hc.rho * rsign * phf, hc, acc);
    }
    float2 p[12];
    sp.load(site, p);
    const float dg = (float)diag;
    float2 o[12];
#pragma unroll
    for (int i = 0; i < 12; i++) {
        o[i].x = dg * p[i].x + acc.a[i].x - acc.ai[i].y;
        o[i].y = dg * p[i].y + acc.a[i].y + acc.ai[i].x;
        if (mode == 2 && i >= 6) { o[i].x = -o[i].x; o[i].y = -o[i].y; }
    }
    h16_store(reinterpret_cast<uint4 *>(out + rhs * fb), reinterpret_cast<float *>(out + rhs * fb + (size_t)48 * g.V),
              site, o);
}

template <class LL, int BODY>
static void launch_h16(int mode, const LL &ll, const void *in, void *out, int nrhs, const Geom &g, double diag,
                       const int *skip, cudaStream_t s) {
    if (g.L[0] == 32 && g.s0 % 32 == 0 && g.s1 % 32 == 0) {
        // the bulk-copy line kernel: links and FP16 spinor lines staged, one
        // buffer per spinor line, 128 registers
        constexpr unsigned smem = line2_smem<LL, true, LineSpinH16>();
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_dslash_bulk_line2_r128<LL, true, LineSpinH16>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(k_dslash_bulk_line2_r128<LL, true, LineSpinH16>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
            attr = true;
        }
        const int nl = (g.s1 - g.s0) / 32;
        const int rmax = (int)(0x7fffffffULL / (unsigned long long)nl < 65535ULL ? 0x7fffffffULL / nl : 65535ULL);
        const size_t fb = h16_field_bytes(g.V);
        for (int r0 = 0; r0 < nrhs; r0 += rmax) {
            const int nr = nrhs - r0 < rmax ? nrhs - r0 : rmax;
            k_dslash_bulk_line2_r128<LL, true, LineSpinH16><<<dim3((unsigned)nl * (unsigned)nr), 32, smem, s>>>(
                mode, ll, (const unsigned char *)in + r0 * fb, (unsigned char *)out + r0 * fb, g, diag,
                skip ? skip + r0 : nullptr);
        }
        return;
    }
    const int threads = 128;
    const size_t fb = h16_field_bytes(g.V);
    // grid.x holds site blocks x RHS: split the RHS so that it stays below 2^31
    const size_t nbmax = (size_t)(g.s1 - g.s0 + threads - 1) / threads;
    const int rmax = (int)(0x7fffffffULL / nbmax < 65535ULL ? 0x7fffffffULL / nbmax : 65535ULL);
    for (int r0 = 0; r0 < nrhs; r0 += rmax) {
        const int nr = nrhs - r0 < rmax ? nrhs - r0 : rmax;
        const dim3 grid((unsigned)nbmax * (unsigned)nr);
        k_dslash_h16<LL, BODY><<<grid, threads, 0, s>>>(mode, ll, (const unsigned char *)in + r0 * fb,
                                                        (unsigned char *)out + r0 * fb, g, diag,
                                                        skip ? skip + r0 : nullptr);
    }
}

// conversion between spinor storages: fmt 0 = complex128, 1 = complex64, 3 = FP16 + scale
__global__ void k_convert_spinor(unsigned char *__restrict__ dst, int dfmt, const unsigned char *__restrict__ src,
                                 int sfmt, int V, int nrhs) {
    const size_t n = (size_t)V * nrhs;
    const size_t fb = h16_field_bytes(V);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / V), site = (int)(i - (size_t)r * V);
        double2 v[12];
        if (sfmt == 0) {
            const double2 *p = reinterpret_cast<const double2 *>(src) + i * 12;
#pragma unroll
            for (int k = 0; k < 12; k++) v[k] = p[k];
        } else if (sfmt == 1) {
            const float2 *p = reinterpret_cast<const float2 *>(src) + i * 12;
#pragma unroll
            for (int k = 0; k < 12; k++) v[k] = make_double2(p[k].x, p[k].y);
        } else {
            const SpinH16 sp{reinterpret_cast<const uint4 *>(src + r * fb),
                             reinterpret_cast<const float *>(src + r * fb + (size_t)48 * V)};
            float2 q[12];
            sp.load(site, q);
#pragma unroll
            for (int k = 0; k < 12; k++) v[k] = make_double2(q[k].x, q[k].y);
        }
        if (dfmt == 0) {
            double2 *p = reinterpret_cast<double2 *>(dst) + i * 12;
#pragma unroll
            for (int k = 0; k < 12; k++) p[k] = v[k];
        } else if (dfmt == 1) {
            float2 *p = reinterpret_cast<float2 *>(dst) + i * 12;
#pragma unroll
            for (int k = 0; k < 12; k++) p[k] = make_float2((float)v[k].x, (float)v[k].y);
        } else {
            float2 q[12];
#pragma unroll
            for (int k = 0; k < 12; k++) q[k] = make_float2((float)v[k].x, (float)v[k].y);
            h16_store(reinterpret_cast<uint4 *>(dst + r * fb), reinterpret_cast<float *>(dst + r * fb + (size_t)48 * V),
                      site, q);
        }
    }
}

}  // namespace bri

using namespace bri;

size_t bri_h16_bytes(int V) { return h16_field_bytes(V); }

// FP16-spinor apply on the stored FP16 fields (any compression); the caller
// has checked that they exist
bri_status bri_dslash_h16(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int mode, const int *skip,
                          cudaStream_t s) {
    if (ctx->werr_h && *(volatile int *)ctx->werr_h) {
        *(volatile int *)ctx->werr_h = 0;
        return bri_fail(ctx, BRI_ETIMEOUT, "a bounded wait of an earlier apply gave up; its output is invalid");
    }
    const Geom &g = ctx->g;
    const LinkStore &st = ctx->f16;
    const int VP = (g.V + 31) & ~31;
    const double diag = m0 + g.lamd[0];
    if (st.comp == BRI_LINK_FULL)
        launch_h16<LinkF16<BRI_LINK_FULL>, 3>(mode, LinkF16<BRI_LINK_FULL>{(const uint4 *)st.a, st.b, VP}, in, out,
                                                nrhs, g, diag, skip, s);
    else if (st.comp == BRI_LINK_2ROW)
        launch_h16<LinkF16<BRI_LINK_2ROW>, 2>(mode, LinkF16<BRI_LINK_2ROW>{(const uint4 *)st.a, st.b, VP}, in, out,
                                                nrhs, g, diag, skip, s);
    else
        launch_h16<LinkF16<BRI_LINK_8PARAM>, 2>(mode, LinkF16<BRI_LINK_8PARAM>{(const uint4 *)st.a, nullptr, VP}, in,
                                                  out, nrhs, g, diag, skip, s);
    BRI_LAUNCHED(ctx);
    return BRI_OK;
}

bri_status bri_convert_spinor_impl(bri_ctx *ctx, void *dst, int dfmt, const void *src, int sfmt, int nrhs,
                                   cudaStream_t s) {
    const size_t n = (size_t)ctx->g.V * nrhs;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 8);
    k_convert_spinor<<<blocks, 256, 0, s>>>((unsigned char *)dst, dfmt, (const unsigned char *)src, sfmt, ctx->g.V,
                                            nrhs);
    BRI_LAUNCHED(ctx);
    return BRI_OK;
}
