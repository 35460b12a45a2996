// Dispatch of the stencil apply over the stored link formats.
#include <string>

#include "ctx.h"
#include "links.cuh"
#include "tile.cuh"

namespace bri {
// defined in dslash_kernel.cuh, instantiated once per format in dslash_*.cu
template <class LL>
void dslash_launch(int mode, const LL &ll, const void *in, void *out, int nrhs, const Geom &g, double diag,
                   const int *skip, int threads, cudaStream_t s);
// defined in dslash_pair.cuh, instantiated in dslash_pair_*.cu
template <class PL>
void dslash_pair_launch(int mode, const PL &pl, const void *in, void *out, int nrhs, const Geom &g, double diag,
                        const int *skip, int threads, cudaStream_t s);
}  // namespace bri

using namespace bri;

std::string bri_tune_key(bri_ctx *ctx, bri_prec prec, int nrhs) {
    const LinkStore &st = prec == BRI_F32 ? ctx->f32 : ctx->f16;
    char buf[160];
    snprintf(buf, sizeof buf, "dslash:%dx%dx%dx%d:p%d:c%d:n%d", ctx->g.L[0], ctx->g.L[1], ctx->g.L[2], ctx->g.L[3],
             (int)prec, prec == BRI_F64 ? 0 : (int)st.comp, nrhs);
    return buf;
}

// Untuned launch shape per storage format: FP64 -> unrolled kernel (128
// threads).  FP32 and FP16 fields on an x extent of 32: the line kernel with
// the links and neighbour spinors staged by bulk copies (variant 11, one warp
// per x line) in its form with one buffer per spinor line (low bits 64), whose
// smaller stages leave room for more warps per SM: 10-20% faster than the
// L2-prefetch loops on 32^3x64 and 0.2-10% faster than with the two-deep
// ring.  Other extents, 128 threads: the pair loop with
// L2 link prefetch, (d, -d) combined before the gamma terms (variant 5) for
// FP32 full fields, the same loop with the per-site part of the link addresses
// computed once and the next pair's neighbours carried over (variant 9) for
// FP32 2-row, FP16 full and FP16 2-row fields, variant 5 held to 128 registers
// (variant 6) for 8-parameter fields.  The register allocation, and with it the
// fastest form, differs between the link decoders.
static int default_shape(bri_ctx *ctx, bri_prec prec) {
    if (prec == BRI_F64) return 128;
    const bri_comp c = (prec == BRI_F32 ? ctx->f32 : ctx->f16).comp;
    if (ctx->g.L[0] == 32) return 64 | (11 << 11);
    if (prec == BRI_F32 && c == BRI_LINK_FULL) return 128 | (5 << 11);
    if (c == BRI_LINK_8PARAM) return 128 | (6 << 11);
    return 128 | (9 << 11);
}

// launch shape (threads per block, kernel variant in bits 11+; see
// bri_set_threads): the tuned one for (lattice, prec, storage, nrhs) if any
int bri_dslash_threads(bri_ctx *ctx, bri_prec prec, int nrhs) {
    auto it = ctx->tune.find(bri_tune_key(ctx, prec, nrhs));
    if (it != ctx->tune.end()) return it->second;
    return default_shape(ctx, prec);
}

static bri_status dslash_geom(bri_ctx *ctx, const Geom &g, void *out, const void *in, int nrhs, double m0, int mode,
                              bri_prec prec, const int *skip, int threads, cudaStream_t s);

bri_status bri_dslash_raw(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int mode, bri_prec prec,
                          const int *skip, int threads, cudaStream_t s) {
    return dslash_geom(ctx, ctx->g, out, in, nrhs, m0, mode, prec, skip, threads, s);
}

// only sites [s0, s1) of out are written (the plain kernels; the tiled and
// site-pair kernels cover the whole lattice)
bri_status bri_dslash_range(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int mode, bri_prec prec,
                            int s0, int s1, cudaStream_t s) {
    Geom g = ctx->g;
    g.s0 = s0;
    g.s1 = s1;
    int threads = bri_dslash_threads(ctx, prec, nrhs);
    if ((threads & 2047) == 0 || (threads >> 11) == 3) threads = default_shape(ctx, prec);
    return dslash_geom(ctx, g, out, in, nrhs, m0, mode, prec, nullptr, threads, s);
}

static bri_status dslash_geom(bri_ctx *ctx, const Geom &g, void *out, const void *in, int nrhs, double m0, int mode,
                              bri_prec prec, const int *skip, int threads, cudaStream_t s) {
    if (ctx->werr_h && *(volatile int *)ctx->werr_h) {
        *(volatile int *)ctx->werr_h = 0;
        return bri_fail(ctx, BRI_ETIMEOUT, "a bounded wait of an earlier apply gave up; its output is invalid");
    }
    const double diag = m0 + g.lamd[0];
    if (prec == BRI_F64) {
        if (!ctx->have64) return bri_fail(ctx, BRI_ESTATE, "FP64 hopping fields not built");
        LinkF64 ll{ctx->hops64, g.V};
        dslash_launch(mode, ll, in, out, nrhs, g, diag, skip, threads, s);
    } else {
        const LinkStore &st = prec == BRI_F32 ? ctx->f32 : ctx->f16;
        if (!st.valid) return bri_fail(ctx, BRI_ESTATE, "hopping fields of this precision not built");
        if ((threads >> 11) == 8) {
            // tensor-core apply: full link storage, whole lattice, no clover term
            if (st.comp == BRI_LINK_FULL && !g.clov64 && g.s0 == 0 && g.s1 == g.V)
                return bri_dslash_tc(ctx, out, in, nrhs, m0, mode, prec, skip, threads & 2047, s);
            threads = default_shape(ctx, prec);
        }
        const LinkStore &ps = prec == BRI_F32 ? ctx->p32 : ctx->p16;
        if ((threads >> 11) == 3 && !ps.valid && !g.clov64 && g.s0 == 0 && g.s1 == g.V)
            BRI_RETURN_IF(bri_pair_store_impl(ctx, prec, s));  // first use of the site-pair kernel
        if ((threads >> 11) == 3 && ps.valid && !g.clov64 && g.s0 == 0 && g.s1 == g.V) {
            // site-pair kernel on the interleaved copy
            const int thr = (threads & 2047) ? (threads & 2047) : 64;
            const int H = g.V / 2;
            if (prec == BRI_F32) {
                if (ps.comp == BRI_LINK_FULL)
                    dslash_pair_launch(mode, PairF32<9>{(const float4 *)ps.a, H}, in, out, nrhs, g, diag, skip, thr, s);
                else
                    dslash_pair_launch(mode, PairF32<6>{(const float4 *)ps.a, H}, in, out, nrhs, g, diag, skip, thr, s);
            } else {
                if (ps.comp == BRI_LINK_FULL)
                    dslash_pair_launch(mode, PairF16<9>{(const uint2 *)ps.a, H}, in, out, nrhs, g, diag, skip, thr, s);
                else
                    dslash_pair_launch(mode, PairF16<6>{(const uint2 *)ps.a, H}, in, out, nrhs, g, diag, skip, thr, s);
            }
            BRI_LAUNCHED(ctx);
            return BRI_OK;
        }
        if ((threads >> 11) == 3) threads = 128;  // no pair copy for this storage: plain kernel
        const int VP = (g.V + 31) & ~31;          // sites per field of the blocked FP32/FP16 layout
        if (prec == BRI_F32) {
            if (st.comp == BRI_LINK_FULL)
                dslash_launch(mode, LinkF32<BRI_LINK_FULL>{(const float4 *)st.a, (const float2 *)st.b, VP}, in, out, nrhs,
                       g, diag, skip, threads, s);
            else if (st.comp == BRI_LINK_2ROW)
                dslash_launch(mode, LinkF32<BRI_LINK_2ROW>{(const float4 *)st.a, nullptr, VP}, in, out, nrhs, g, diag, skip,
                       threads, s);
            else
                dslash_launch(mode, LinkF32<BRI_LINK_8PARAM>{(const float4 *)st.a, nullptr, VP}, in, out, nrhs, g, diag,
                       skip, threads, s);
        } else {
            if (st.comp == BRI_LINK_FULL)
                dslash_launch(mode, LinkF16<BRI_LINK_FULL>{(const uint4 *)st.a, st.b, VP}, in, out, nrhs, g, diag, skip,
                       threads, s);
            else if (st.comp == BRI_LINK_2ROW)
                dslash_launch(mode, LinkF16<BRI_LINK_2ROW>{(const uint4 *)st.a, st.b, VP}, in, out, nrhs, g, diag, skip,
                       threads, s);
            else
                dslash_launch(mode, LinkF16<BRI_LINK_8PARAM>{(const uint4 *)st.a, nullptr, VP}, in, out, nrhs, g, diag,
                       skip, threads, s);
        }
    }
    BRI_LAUNCHED(ctx);
    return BRI_OK;
}

bri_status bri_dslash_impl(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int mode, bri_prec prec,
                           cudaStream_t s) {
    return bri_dslash_raw(ctx, out, in, nrhs, m0, mode, prec, nullptr, bri_dslash_threads(ctx, prec, nrhs), s);
}
