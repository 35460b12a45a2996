// Storage formats of the 40 hopping fields and their device-side loaders.
//
// FP64 fields are stored structure-of-arrays over sites ([40][9][V]).  The FP32
// and FP16 fields are cut into 16-byte chunks stored in blocks of 32 sites,
// [40][Vp/32][chunks][32] with Vp = V rounded up to 32: a warp reading one
// chunk of 32 consecutive sites issues fully coalesced 128-bit loads, and the
// chunks of one site lie at compile-time offsets (q x 512 bytes) from its first
// one, so a field costs one address computation, not one per chunk.  The last
// 8 or 4 bytes of a full or 2-row field go to a second array [40][Vp]:
//   FP64 full    9 x double2                      144 B
//   FP32 full    4 x float4 + 1 x float2           72 B
//   FP32 2-row   3 x float4                        48 B
//   FP32 8-param 2 x float4                        32 B
//   FP16 full    2 x uint4 (8 half2) + 1 half2     36 B
//   FP16 2-row   1 x uint4 + 1 x uint2             24 B
//   FP16 8-param 1 x uint4                         16 B
// The reduced forms use that every W_d(x) is in SU(3) (Sec. 5.2): the third row
// is conj(row0 x row1), and (8-param) U01, U02, U10 with the phases of U00 and
// U20 fix the rest through unitarity and det = 1:
//   |U00|^2 = 1 - |U01|^2 - |U02|^2, |U20|^2 = 1 - |U00|^2 - |U10|^2, and with
//   N = |U01|^2 + |U02|^2, rows 1 and 2 follow from orthogonality to row 0 and
//   the cofactor identity U^* = cof(U):
//   (U11, U12) = (U01 a - U02^* b, U02 a + U01^* b) / N, a = -U10 U00^*, b = U20^*
//   (U21, U22) = (U01 a' - U02^* b', U02 a' + U01^* b') / N, a' = -U20 U00^*, b' = -U10^*
#pragma once
#include <cuda_fp16.h>

#include "brillouin.h"
#include "common.cuh"

namespace bri {

BRI_D float2 h2f(uint32_t u) {
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    return __half22float2(h);
}

template <typename T> BRI_D void third_row(M3<T> &m) {
    m.e[6] = cconj(csub(cmul(m.e[1], m.e[5]), cmul(m.e[2], m.e[4])));
    m.e[7] = cconj(csub(cmul(m.e[2], m.e[3]), cmul(m.e[0], m.e[5])));
    m.e[8] = cconj(csub(cmul(m.e[0], m.e[4]), cmul(m.e[1], m.e[3])));
}

// p = (U01.re, U01.im, U02.re, U02.im, U10.re, U10.im, arg U00, arg U20)
BRI_D void eight_params(const double2 w[9], float p[8]) {
    p[0] = (float)w[1].x; p[1] = (float)w[1].y;
    p[2] = (float)w[2].x; p[3] = (float)w[2].y;
    p[4] = (float)w[3].x; p[5] = (float)w[3].y;
    p[6] = (float)atan2(w[0].y, w[0].x);
    p[7] = (float)atan2(w[6].y, w[6].x);
}

BRI_D M3<float2> from_eight(const float p[8]) {
    M3<float2> m;
    const float2 a1 = make_float2(p[0], p[1]), a2 = make_float2(p[2], p[3]), b0 = make_float2(p[4], p[5]);
    const float N = a1.x * a1.x + a1.y * a1.y + a2.x * a2.x + a2.y * a2.y;
    const float r00 = sqrtf(fmaxf(0.f, 1.f - N));
    float s0, c0, s2, c2;
    __sincosf(p[6], &s0, &c0);
    __sincosf(p[7], &s2, &c2);
    const float2 u00 = make_float2(r00 * c0, r00 * s0);
    const float r20 = sqrtf(fmaxf(0.f, N - (b0.x * b0.x + b0.y * b0.y)));
    const float2 u20 = make_float2(r20 * c2, r20 * s2);
    const float inv = 1.f / N;
    float2 al = cscale(cmulc(u00, b0), -1.f);  // -U10 U00^*
    float2 be = cconj(u20);
    m.e[4] = cscale(csub(cmul(a1, al), cmul(cconj(a2), be)), inv);
    m.e[5] = cscale(cadd(cmul(a2, al), cmul(cconj(a1), be)), inv);
    float2 al2 = cscale(cmulc(u00, u20), -1.f);  // -U20 U00^*
    float2 be2 = cscale(cconj(b0), -1.f);
    m.e[7] = cscale(csub(cmul(a1, al2), cmul(cconj(a2), be2)), inv);
    m.e[8] = cscale(cadd(cmul(a2, al2), cmul(cconj(a1), be2)), inv);
    m.e[0] = u00; m.e[1] = a1; m.e[2] = a2;
    m.e[3] = b0;  m.e[6] = u20;
    return m;
}

// asynchronous global -> shared copies of 16, 8 or 4 bytes (sm_80+ cp.async)
BRI_D void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
BRI_D void cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
BRI_D void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
BRI_D float4 lds4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
BRI_D uint4 lds4u(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}

BRI_D float2 lds2(uint32_t a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
BRI_D uint2 lds2u(uint32_t a) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}
BRI_D uint32_t lds1u(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// ---- 1-D bulk copies into shared memory, completion counted on an mbarrier ----
// (cp.async.bulk: source and destination 16-byte aligned, size a multiple of
// 16 bytes; the mbarrier's phase completes when its expected arrivals have
// arrived and the announced bytes have landed)
BRI_D void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// makes the initialised barriers visible to the copy engine
BRI_D void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// one arrival that also announces the bytes the stage's copies deliver
BRI_D void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
BRI_D bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
BRI_D unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait for the phase of the given parity; false if it has not completed after
// limit_ns nanoseconds (the caller reports BRI_ETIMEOUT)
BRI_D bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
// orders this thread's earlier shared-memory accesses (and those of the lanes
// it synchronised with) before its later bulk copies into the same bytes
BRI_D void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
BRI_D void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// The same from a converged warp without a branch: elect.sync picks one lane,
// which announces tx bytes on bar and issues the copies (sizes a multiple of
// 16 bytes).  (A form that also took a warp-uniform condition as a predicate,
// instead of the caller's branch, measured 3% slower in the stencil loop.)
BRI_D void bulk_elect1(uint32_t bar, uint32_t tx, uint32_t d0, const void *s0, uint32_t n0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\telect.sync _|p, 0xffffffff;\n\t"
        "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%2], [%3], %4, [%0];\n\t}" ::"r"(bar), "r"(tx), "r"(d0), "l"(s0), "r"(n0)
        : "memory");
}
BRI_D void bulk_elect2(uint32_t bar, uint32_t tx, uint32_t d0, const void *s0, uint32_t n0, uint32_t d1,
                       const void *s1, uint32_t n1) {
    asm volatile(
        "{\n\t.reg .pred p;\n\telect.sync _|p, 0xffffffff;\n\t"
        "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%2], [%3], %4, [%0];\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%5], [%6], %7, [%0];\n\t}" ::"r"(bar), "r"(tx), "r"(d0), "l"(s0), "r"(n0), "r"(d1), "l"(s1), "r"(n1)
        : "memory");
}
BRI_D void bulk_elect4(uint32_t bar, uint32_t tx, uint32_t d0, const void *s0, uint32_t n0, uint32_t d1,
                       const void *s1, uint32_t n1, uint32_t d2, const void *s2, uint32_t n2, uint32_t d3,
                       const void *s3, uint32_t n3) {
    asm volatile(
        "{\n\t.reg .pred p;\n\telect.sync _|p, 0xffffffff;\n\t"
        "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%2], [%3], %4, [%0];\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%5], [%6], %7, [%0];\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%8], [%9], %10, [%0];\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%11], [%12], %13, [%0];\n\t}" ::"r"(bar), "r"(tx), "r"(d0), "l"(s0), "r"(n0), "r"(d1), "l"(s1), "r"(n1), "r"(d2), "l"(s2), "r"(n2), "r"(d3),
        "l"(s3), "r"(n3)
        : "memory");
}

// L2 prefetch of one 16-byte chunk (brings the line to L2, no register cost)
BRI_D void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

struct LinkF64 {
    using T = double2;
    const double2 *__restrict__ h;
    int V;
    BRI_D M3<double2> load(int j, int site) const {
        M3<double2> m;
#pragma unroll
        for (int e = 0; e < 9; e++) m.e[e] = h[((size_t)j * 9 + e) * V + site];
        return m;
    }
};

template <bri_comp C> struct LinkF32 {
    using T = float2;
    static constexpr bri_comp COMP = C;
    // 16-byte shared-memory slots one field occupies when prefetched
    static constexpr int SLOTS = C == BRI_LINK_FULL ? 5 : C == BRI_LINK_2ROW ? 3 : 2;
    static constexpr int NQ = C == BRI_LINK_FULL ? 4 : C == BRI_LINK_2ROW ? 3 : 2;  // float4 chunks
    const float4 *__restrict__ a;
    const float2 *__restrict__ b;
    int VP;  // sites per field, V rounded up to a multiple of 32
    // first chunk of field j at site s (chunk q follows at + 32 q)
    BRI_D const float4 *chunk0(int j, int s) const {
        return a + ((size_t)j * VP + (s & ~31)) * NQ + (s & 31);
    }
    // shared-memory slots are chunk-major across the block: chunk q of this
    // thread's field at dst + q * stride (stride = 16 bytes x threads), so a
    // warp's 16-byte accesses are consecutive and free of bank conflicts
    BRI_D void prefetch(int j, int site, uint32_t dst, uint32_t stride) const {
        const float4 *p = chunk0(j, site);
#pragma unroll
        for (int q = 0; q < NQ; q++) cp_async16(dst + stride * q, p + 32 * q);
        if (C == BRI_LINK_FULL) cp_async8(dst + stride * 4, b + (size_t)j * VP + site);
    }
    BRI_D void prefetch_field_l2(int j, int site) const {
        const float4 *p = chunk0(j, site);
#pragma unroll
        for (int q = 0; q < NQ; q++) prefetch_l2(p + 32 * q);
        if (C == BRI_LINK_FULL) prefetch_l2(b + (size_t)j * VP + site);
    }
    // chunk offset of site s within any field (field j adds j VP NQ): lets a
    // loop over fields reuse the per-site part of the address
    BRI_D long long cidx(int s) const { return (long long)(s & ~31) * NQ + (s & 31); }
    BRI_D void prefetch_ci(int j, long long ci, int s) const {
        const float4 *p = a + (long long)j * VP * NQ + ci;
#pragma unroll
        for (int q = 0; q < NQ; q++) prefetch_l2(p + 32 * q);
        if (C == BRI_LINK_FULL) prefetch_l2(b + (long long)j * VP + s);
    }
    BRI_D M3<float2> load_ci(int j, long long ci, int s) const {
        const float4 *p = a + (long long)j * VP * NQ + ci;
        if (C == BRI_LINK_8PARAM) {
            float4 v0 = p[0], v1 = p[32];
            float pr[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            return from_eight(pr);
        }
        M3<float2> m;
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            float4 v = p[32 * q];
            m.e[2 * q] = make_float2(v.x, v.y);
            m.e[2 * q + 1] = make_float2(v.z, v.w);
        }
        if (C == BRI_LINK_FULL) m.e[8] = b[(long long)j * VP + s];
        else third_row(m);
        return m;
    }
    // One 32-site block of field j as the bulk-copy kernel stages it: the NQ
    // chunk rows (RUN_A bytes; chunk q of slot l at 512 q + 16 l), then for
    // full storage the block's 32 third-row entries (8 bytes each).  Both parts
    // are contiguous in global memory and start on 256-byte boundaries.
    static constexpr uint32_t RUN_A = 512u * NQ;
    static constexpr uint32_t RUN_B = C == BRI_LINK_FULL ? 256u : 0u;
    BRI_D void bulk_run(int j, int blk, uint32_t dst, uint32_t bar) const {
        bulk_g2s(dst, a + ((size_t)j * VP + 32 * (size_t)blk) * NQ, RUN_A, bar);
        if (RUN_B) bulk_g2s(dst + RUN_A, b + (size_t)j * VP + 32 * (size_t)blk, RUN_B, bar);
    }
    // from a converged warp: the runs of field j at blocks bf and bb into dst and
    // dst + RUN_A + RUN_B, announced together with extra bytes on bar
    BRI_D void bulk_pair(int j, int bf, int bb, uint32_t dst, uint32_t bar, uint32_t extra) const {
        constexpr uint32_t RUN = RUN_A + RUN_B;
        const float4 *aj = a + (size_t)j * VP * NQ;
        if (RUN_B) {
            const float2 *bj = b + (size_t)j * VP;
            bulk_elect4(bar, 2 * RUN + extra, dst, aj + (size_t)bf * 32 * NQ, RUN_A, dst + RUN_A, bj + (size_t)bf * 32,
                        RUN_B, dst + RUN, aj + (size_t)bb * 32 * NQ, RUN_A, dst + RUN + RUN_A, bj + (size_t)bb * 32,
                        RUN_B);
        } else {
            bulk_elect2(bar, 2 * RUN + extra, dst, aj + (size_t)bf * 32 * NQ, RUN_A, dst + RUN,
                        aj + (size_t)bb * 32 * NQ, RUN_A);
        }
    }
    BRI_D M3<float2> load_run(uint32_t run, int l) const {
        const uint32_t p = run + 16u * (uint32_t)l;
        if (C == BRI_LINK_8PARAM) {
            float4 v0 = lds4(p), v1 = lds4(p + 512);
            float pr[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            return from_eight(pr);
        }
        M3<float2> m;
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            float4 v = lds4(p + 512 * q);
            m.e[2 * q] = make_float2(v.x, v.y);
            m.e[2 * q + 1] = make_float2(v.z, v.w);
        }
        if (C == BRI_LINK_FULL) m.e[8] = lds2(run + RUN_A + 8u * (uint32_t)l);
        else third_row(m);
        return m;
    }
    BRI_D M3<float2> load_smem(uint32_t src, uint32_t stride) const {
        M3<float2> m;
        if (C == BRI_LINK_8PARAM) {
            float4 v0 = lds4(src), v1 = lds4(src + stride);
            float p[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            return from_eight(p);
        }
#pragma unroll
        for (int q = 0; q < (C == BRI_LINK_FULL ? 4 : 3); q++) {
            float4 v = lds4(src + stride * q);
            m.e[2 * q] = make_float2(v.x, v.y);
            m.e[2 * q + 1] = make_float2(v.z, v.w);
        }
        if (C == BRI_LINK_FULL) {
            float4 v = lds4(src + stride * 4);
            m.e[8] = make_float2(v.x, v.y);
        } else {
            third_row(m);
        }
        return m;
    }
    BRI_D M3<float2> load(int j, int site) const {
        M3<float2> m;
        const float4 *p = chunk0(j, site);
        if (C == BRI_LINK_8PARAM) {
            float4 v0 = p[0], v1 = p[32];
            float pr[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            return from_eight(pr);
        }
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            float4 v = p[32 * q];
            m.e[2 * q] = make_float2(v.x, v.y);
            m.e[2 * q + 1] = make_float2(v.z, v.w);
        }
        if (C == BRI_LINK_FULL) m.e[8] = b[(size_t)j * VP + site];
        else third_row(m);
        return m;
    }
};

template <bri_comp C> struct LinkF16 {
    using T = float2;
    static constexpr bri_comp COMP = C;
    static constexpr int SLOTS = C == BRI_LINK_FULL ? 3 : C == BRI_LINK_2ROW ? 2 : 1;
    static constexpr int NQ = C == BRI_LINK_FULL ? 2 : 1;  // uint4 chunks
    const uint4 *__restrict__ a;
    const void *__restrict__ b;
    int VP;  // sites per field, V rounded up to a multiple of 32
    BRI_D const uint4 *chunk0(int j, int s) const {
        if (NQ == 1) return a + (size_t)j * VP + s;  // one chunk: plain [40][Vp]
        return a + ((size_t)j * VP + (s & ~31)) * NQ + (s & 31);
    }
    BRI_D void prefetch(int j, int site, uint32_t dst, uint32_t stride) const {
        const uint4 *p = chunk0(j, site);
        if (C == BRI_LINK_FULL) {
            cp_async16(dst, p);
            cp_async16(dst + stride, p + 32);
            cp_async4(dst + 2 * stride, (const uint32_t *)b + (size_t)j * VP + site);
        } else if (C == BRI_LINK_2ROW) {
            cp_async16(dst, p);
            cp_async8(dst + stride, (const uint2 *)b + (size_t)j * VP + site);
        } else {
            cp_async16(dst, p);
        }
    }
    BRI_D void prefetch_field_l2(int j, int site) const {
        const uint4 *p = chunk0(j, site);
        prefetch_l2(p);
        if (C == BRI_LINK_FULL) {
            prefetch_l2(p + 32);
            prefetch_l2((const uint32_t *)b + (size_t)j * VP + site);
        } else if (C == BRI_LINK_2ROW) {
            prefetch_l2((const uint2 *)b + (size_t)j * VP + site);
        }
    }
    BRI_D long long cidx(int s) const { return NQ == 1 ? (long long)s : (long long)(s & ~31) * NQ + (s & 31); }
    BRI_D void prefetch_ci(int j, long long ci, int s) const {
        const uint4 *p = a + (long long)j * VP * NQ + ci;
        prefetch_l2(p);
        if (C == BRI_LINK_FULL) {
            prefetch_l2(p + 32);
            prefetch_l2((const uint32_t *)b + (long long)j * VP + s);
        } else if (C == BRI_LINK_2ROW) {
            prefetch_l2((const uint2 *)b + (long long)j * VP + s);
        }
    }
    BRI_D M3<float2> load_ci(int j, long long ci, int s) const {
        const uint4 *p = a + (long long)j * VP * NQ + ci;
        M3<float2> m;
        if (C == BRI_LINK_FULL) {
#pragma unroll
            for (int q = 0; q < 2; q++) {
                uint4 v = p[32 * q];
                m.e[4 * q] = h2f(v.x);
                m.e[4 * q + 1] = h2f(v.y);
                m.e[4 * q + 2] = h2f(v.z);
                m.e[4 * q + 3] = h2f(v.w);
            }
            m.e[8] = h2f(((const uint32_t *)b)[(long long)j * VP + s]);
        } else if (C == BRI_LINK_2ROW) {
            uint4 v = p[0];
            uint2 t = ((const uint2 *)b)[(long long)j * VP + s];
            m.e[0] = h2f(v.x); m.e[1] = h2f(v.y); m.e[2] = h2f(v.z); m.e[3] = h2f(v.w);
            m.e[4] = h2f(t.x); m.e[5] = h2f(t.y);
            third_row(m);
        } else {
            uint4 v = p[0];
            float2 q0 = h2f(v.x), q1 = h2f(v.y), q2 = h2f(v.z), q3 = h2f(v.w);
            float pr[8] = {q0.x, q0.y, q1.x, q1.y, q2.x, q2.y, q3.x, q3.y};
            m = from_eight(pr);
        }
        return m;
    }
    // one 32-site block of field j as the bulk-copy kernel stages it (see
    // LinkF32): NQ chunk rows of 512 bytes, then the tail entries (4 bytes per
    // site for full, 8 for 2-row storage)
    static constexpr uint32_t RUN_A = 512u * NQ;
    static constexpr uint32_t RUN_B = C == BRI_LINK_FULL ? 128u : C == BRI_LINK_2ROW ? 256u : 0u;
    BRI_D void bulk_run(int j, int blk, uint32_t dst, uint32_t bar) const {
        bulk_g2s(dst, a + ((size_t)j * VP + 32 * (size_t)blk) * NQ, RUN_A, bar);
        if (C == BRI_LINK_FULL) bulk_g2s(dst + RUN_A, (const uint32_t *)b + (size_t)j * VP + 32 * (size_t)blk, RUN_B, bar);
        if (C == BRI_LINK_2ROW) bulk_g2s(dst + RUN_A, (const uint2 *)b + (size_t)j * VP + 32 * (size_t)blk, RUN_B, bar);
    }
    BRI_D void bulk_pair(int j, int bf, int bb, uint32_t dst, uint32_t bar, uint32_t extra) const {
        constexpr uint32_t RUN = RUN_A + RUN_B;
        const uint4 *aj = a + (size_t)j * VP * NQ;
        if (RUN_B) {
            const char *bj = (const char *)b + (size_t)j * VP * (RUN_B / 32);
            bulk_elect4(bar, 2 * RUN + extra, dst, aj + (size_t)bf * 32 * NQ, RUN_A, dst + RUN_A,
                        bj + (size_t)bf * RUN_B, RUN_B, dst + RUN, aj + (size_t)bb * 32 * NQ, RUN_A,
                        dst + RUN + RUN_A, bj + (size_t)bb * RUN_B, RUN_B);
        } else {
            bulk_elect2(bar, 2 * RUN + extra, dst, aj + (size_t)bf * 32 * NQ, RUN_A, dst + RUN,
                        aj + (size_t)bb * 32 * NQ, RUN_A);
        }
    }
    BRI_D M3<float2> load_run(uint32_t run, int l) const {
        const uint32_t p = run + 16u * (uint32_t)l;
        M3<float2> m;
        if (C == BRI_LINK_FULL) {
            uint4 v = lds4u(p), w = lds4u(p + 512);
            m.e[0] = h2f(v.x); m.e[1] = h2f(v.y); m.e[2] = h2f(v.z); m.e[3] = h2f(v.w);
            m.e[4] = h2f(w.x); m.e[5] = h2f(w.y); m.e[6] = h2f(w.z); m.e[7] = h2f(w.w);
            m.e[8] = h2f(lds1u(run + RUN_A + 4u * (uint32_t)l));
        } else if (C == BRI_LINK_2ROW) {
            uint4 v = lds4u(p);
            uint2 t = lds2u(run + RUN_A + 8u * (uint32_t)l);
            m.e[0] = h2f(v.x); m.e[1] = h2f(v.y); m.e[2] = h2f(v.z); m.e[3] = h2f(v.w);
            m.e[4] = h2f(t.x); m.e[5] = h2f(t.y);
            third_row(m);
        } else {
            uint4 v = lds4u(p);
            float2 q0 = h2f(v.x), q1 = h2f(v.y), q2 = h2f(v.z), q3 = h2f(v.w);
            float pr[8] = {q0.x, q0.y, q1.x, q1.y, q2.x, q2.y, q3.x, q3.y};
            m = from_eight(pr);
        }
        return m;
    }
    BRI_D M3<float2> load_smem(uint32_t src, uint32_t stride) const {
        M3<float2> m;
        if (C == BRI_LINK_FULL) {
            uint4 v = lds4u(src), w = lds4u(src + stride), t = lds4u(src + 2 * stride);
            m.e[0] = h2f(v.x); m.e[1] = h2f(v.y); m.e[2] = h2f(v.z); m.e[3] = h2f(v.w);
            m.e[4] = h2f(w.x); m.e[5] = h2f(w.y); m.e[6] = h2f(w.z); m.e[7] = h2f(w.w);
            m.e[8] = h2f(t.x);
        } else if (C == BRI_LINK_2ROW) {
            uint4 v = lds4u(src), t = lds4u(src + stride);
            m.e[0] = h2f(v.x); m.e[1] = h2f(v.y); m.e[2] = h2f(v.z); m.e[3] = h2f(v.w);
            m.e[4] = h2f(t.x); m.e[5] = h2f(t.y);
            third_row(m);
        } else {
            uint4 v = lds4u(src);
            float2 q0 = h2f(v.x), q1 = h2f(v.y), q2 = h2f(v.z), q3 = h2f(v.w);
            float p[8] = {q0.x, q0.y, q1.x, q1.y, q2.x, q2.y, q3.x, q3.y};
            m = from_eight(p);
        }
        return m;
    }
    BRI_D M3<float2> load(int j, int site) const {
        M3<float2> m;
        const uint4 *p = chunk0(j, site);
        if (C == BRI_LINK_FULL) {
#pragma unroll
            for (int q = 0; q < 2; q++) {
                uint4 v = p[32 * q];
                m.e[4 * q] = h2f(v.x);
                m.e[4 * q + 1] = h2f(v.y);
                m.e[4 * q + 2] = h2f(v.z);
                m.e[4 * q + 3] = h2f(v.w);
            }
            m.e[8] = h2f(((const uint32_t *)b)[(size_t)j * VP + site]);
        } else if (C == BRI_LINK_2ROW) {
            uint4 v = p[0];
            uint2 t = ((const uint2 *)b)[(size_t)j * VP + site];
            m.e[0] = h2f(v.x); m.e[1] = h2f(v.y); m.e[2] = h2f(v.z); m.e[3] = h2f(v.w);
            m.e[4] = h2f(t.x); m.e[5] = h2f(t.y);
            third_row(m);
        } else {
            uint4 v = p[0];
            float2 q0 = h2f(v.x), q1 = h2f(v.y), q2 = h2f(v.z), q3 = h2f(v.w);
            float pr[8] = {q0.x, q0.y, q1.x, q1.y, q2.x, q2.y, q3.x, q3.y};
            m = from_eight(pr);
        }
        return m;
    }
};

}  // namespace bri

namespace bri {

// ---- site-pair interleaved storage -------------------------------------------
// For the pair kernel a thread owns sites i and i + V/2 (a translation by half
// the t extent), and every packed register holds one quantity of both sites.
// Field j, complex entry e of sites (i, i + V/2) is stored as
// (Re_i, Re_{i+V/2}, Im_i, Im_{i+V/2}) at [j][e][V/2]: FP32 as one float4, FP16
// as four halves (uint2).  Full storage keeps e = 0..8, 2-row e = 0..5.
template <int E> struct PairF32 {
    static constexpr int NE = E;
    const float4 *__restrict__ a;
    int H;  // V / 2
    BRI_D void load(int j, int i, float2 R[E], float2 I[E]) const {
#pragma unroll
        for (int e = 0; e < E; e++) {
            const float4 v = a[((size_t)j * E + e) * H + i];
            R[e] = make_float2(v.x, v.y);
            I[e] = make_float2(v.z, v.w);
        }
    }
};
template <int E> struct PairF16 {
    static constexpr int NE = E;
    const uint2 *__restrict__ a;
    int H;
    BRI_D void load(int j, int i, float2 R[E], float2 I[E]) const {
#pragma unroll
        for (int e = 0; e < E; e++) {
            const uint2 v = a[((size_t)j * E + e) * H + i];
            R[e] = h2f(v.x);
            I[e] = h2f(v.y);
        }
    }
};

}  // namespace bri
