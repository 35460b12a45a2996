// Site-pair stencil kernel (FP32 arithmetic): one thread applies D to the two
// sites i and i + V/2, which differ by a translation of half the t extent.
// Both sites see the same hop structure, so every packed FP32 register (f32x2)
// holds the same quantity of the two sites and the complex arithmetic is plain
// packed FMAs: Re/Im parts are kept in separate registers, products need no
// operand broadcasts or swaps, and the +-i entries of the gamma matrices only
// change which register is accumulated into.  Links come from the
// pair-interleaved storage; the reversed hop of site i reads the field at
// z = i - d, whose partner is z + V/2 (or z - V/2 when z wrapped into the
// upper half, in which case the two halves are exchanged).
#pragma once
#include "dslash_kernel.cuh"

namespace bri {

BRI_D float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }
BRI_D float2 pswap(float2 a) { return make_float2(a.y, a.x); }

// third row of a 2-row SU(3) field, for both sites: conj(row0 x row1)
BRI_D void pair_third_row(float2 R[9], float2 I[9]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int p = (c + 1) % 3, q = (c + 2) % 3;
        // z = r0[p] r1[q] - r0[q] r1[p]; row2[c] = conj(z)
        float2 zr = __fmul2_rn(R[p], R[3 + q]);
        zr = __ffma2_rn(pneg(I[p]), I[3 + q], zr);
        zr = __ffma2_rn(pneg(R[q]), R[3 + p], zr);
        zr = __ffma2_rn(I[q], I[3 + p], zr);
        float2 zi = __fmul2_rn(R[p], I[3 + q]);
        zi = __ffma2_rn(I[p], R[3 + q], zi);
        zi = __ffma2_rn(pneg(R[q]), I[3 + p], zi);
        zi = __ffma2_rn(pneg(I[q]), R[3 + p], zi);
        R[6 + c] = zr;
        I[6 + c] = pneg(zi);
    }
}

// acc[k] for both sites: accR = (Re_a, Re_b), accI = (Im_a, Im_b)
struct PairAcc {
    float2 r[12], i[12];
};

// one hop for both sites; SGN = -1: the matrix is W^dagger.  pR/pI: the
// neighbour spinors of the two sites, re-paired.  l, r: class weights times
// the boundary phase of each site (r with the dagger sign).
template <int SGN>
BRI_D void pair_hop(const float2 R[9], const float2 I[9], const float2 *__restrict__ psa,
                    const float2 *__restrict__ psb, float2 l, float2 r, const int dm[4], PairAcc &acc) {
    float2 NI[9];
#pragma unroll
    for (int e = 0; e < 9; e++) NI[e] = pneg(I[e]);
    const float2 nr = pneg(r);
    // coefficient of direction mu for a +1 gamma entry (and its negative)
    float2 cpos[4], cneg[4];
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        cpos[mu] = SGN * dm[mu] > 0 ? r : nr;
        cneg[mu] = SGN * dm[mu] > 0 ? nr : r;
    }
#pragma unroll
    for (int half = 0; half < 2; half++) {
        // spins 2 half, 2 half + 1 of the two neighbour spinors (48 bytes each)
        float2 pR[6], pI[6];
        {
            const float4 *qa = reinterpret_cast<const float4 *>(psa) + 3 * half;
            const float4 *qb = reinterpret_cast<const float4 *>(psb) + 3 * half;
#pragma unroll
            for (int t = 0; t < 3; t++) {
                const float4 va = qa[t], vb = qb[t];
                pR[2 * t] = make_float2(va.x, vb.x);
                pI[2 * t] = make_float2(va.y, vb.y);
                pR[2 * t + 1] = make_float2(va.z, vb.z);
                pI[2 * t + 1] = make_float2(va.w, vb.w);
            }
        }
#pragma unroll
    for (int sl = 0; sl < 2; sl++) {
        const int sp = 2 * half + sl;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float2 cr = make_float2(0.f, 0.f), ci = make_float2(0.f, 0.f);
#pragma unroll
            for (int cp = 0; cp < 3; cp++) {
                const int e = SGN > 0 ? 3 * c + cp : 3 * cp + c;
                const float2 mi = SGN > 0 ? I[e] : NI[e];   // Im of the matrix entry
                const float2 nmi = SGN > 0 ? NI[e] : I[e];  // -Im
                cr = __ffma2_rn(R[e], pR[3 * sl + cp], cr);
                cr = __ffma2_rn(nmi, pI[3 * sl + cp], cr);
                ci = __ffma2_rn(R[e], pI[3 * sl + cp], ci);
                ci = __ffma2_rn(mi, pR[3 * sl + cp], ci);
            }
            acc.r[3 * sp + c] = __ffma2_rn(l, cr, acc.r[3 * sp + c]);
            acc.i[3 * sp + c] = __ffma2_rn(l, ci, acc.i[3 * sp + c]);
#pragma unroll
            for (int mu = 0; mu < 4; mu++) {
                if (dm[mu] == 0) continue;  // uniform across the warp
                const int s = gcol(mu, sp);
                const int gr = gre(mu, s), gi = gim(mu, s);
                const int g = gr != 0 ? gr : gi;  // compile-time sign
                const float2 cf = g > 0 ? cpos[mu] : cneg[mu];
                const float2 ncf = g > 0 ? cneg[mu] : cpos[mu];
                if (gr != 0) {
                    acc.r[3 * s + c] = __ffma2_rn(cf, cr, acc.r[3 * s + c]);
                    acc.i[3 * s + c] = __ffma2_rn(cf, ci, acc.i[3 * s + c]);
                } else {  // coefficient * i * chi
                    acc.r[3 * s + c] = __ffma2_rn(ncf, ci, acc.r[3 * s + c]);
                    acc.i[3 * s + c] = __ffma2_rn(cf, cr, acc.i[3 * s + c]);
                }
            }
        }
    }
    }
}

template <class PL>
BRI_D void pair_load(const PL &pl, int j, int i, float2 R[9], float2 I[9]) {
    pl.load(j, i, R, I);
    if constexpr (PL::NE == 6) pair_third_row(R, I);
}

template <class PL>
__global__ void k_dslash_pair(int mode, PL pl, const float2 *__restrict__ in, float2 *__restrict__ out, Geom g,
                              double diag, const int *__restrict__ skip) {
    const int H = g.V / 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H) return;
    if (skip && skip[blockIdx.y]) return;
    const size_t off = (size_t)blockIdx.y * g.V * 12;
    in += off;
    out += off;
    const int sa = i, sb = i + H;
    // the two sites differ only in t: x, y, z neighbour data are shared
    int xa[4], xb[4];
    const SiteNb na = site_nb(g, sa, xa);
    SiteNb nb = na;
    {
        const int Lt = g.L[3], st = H / (Lt / 2);  // t stride = L0 L1 L2
        const int tb = xa[3] + Lt / 2;
        xb[3] = tb;
        const bool top = tb == Lt - 1;
        nb.fw[3] = top ? -(Lt - 1) * st : st;
        nb.bw[3] = -st;  // tb >= Lt/2 >= 1: never wraps backwards
        nb.sfw[3] = top ? (float)g.bc[3] : 1.f;
        nb.sbw[3] = 1.f;
    }
    PairAcc acc;
#pragma unroll
    for (int k = 0; k < 12; k++) acc.r[k] = acc.i[k] = make_float2(0.f, 0.f);
    const float rsign = mode == 1 ? -1.f : 1.f;
#pragma unroll 1
    for (int t = 0; t < g.nhop; t++) {
        const HopArg hc = g.hop[t];
        const int j = hc.j;
        int yfa, yba, yfb, ybb;
        float pfa, pba, pfb, pbb;
        hop_nb(hc.dm, sa, na, yfa, pfa, yba, pba);
        hop_nb(hc.dm, sb, nb, yfb, pfb, ybb, pbb);
        float2 R[9], I[9];
        // forward hop: fields of the pair itself
        pair_load(pl, j, i, R, I);
        pair_hop<1>(R, I, in + (size_t)yfa * 12, in + (size_t)yfb * 12, make_float2(hc.lam * pfa, hc.lam * pfb),
                    make_float2(hc.rho * rsign * pfa, hc.rho * rsign * pfb), hc.dm, acc);
        // reversed hop: fields at z = site - d for both sites
        const bool upper = yba >= H;
        pair_load(pl, j, upper ? ybb : yba, R, I);
        if (upper) {
#pragma unroll
            for (int e = 0; e < 9; e++) { R[e] = pswap(R[e]); I[e] = pswap(I[e]); }
        }
        pair_hop<-1>(R, I, in + (size_t)yba * 12, in + (size_t)ybb * 12, make_float2(hc.lam * pba, hc.lam * pbb),
                     make_float2(hc.rho * rsign * pba, hc.rho * rsign * pbb), hc.dm, acc);
    }
    const float dg = (float)diag;
    float2 pa[12], pb[12], oa[12], ob[12];
    load_spinor(in + (size_t)sa * 12, pa);
    load_spinor(in + (size_t)sb * 12, pb);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        float2 va = make_float2(dg * pa[k].x + acc.r[k].x, dg * pa[k].y + acc.i[k].x);
        float2 vb = make_float2(dg * pb[k].x + acc.r[k].y, dg * pb[k].y + acc.i[k].y);
        if (mode == 2 && k >= 6) { va = pneg(va); vb = pneg(vb); }
        oa[k] = va;
        ob[k] = vb;
    }
    store_spinor(out + (size_t)sa * 12, oa);
    store_spinor(out + (size_t)sb * 12, ob);
}

template <class PL>
void dslash_pair_launch(int mode, const PL &pl, const void *in, void *out, int nrhs, const Geom &g, double diag,
                        const int *skip, int threads, cudaStream_t s) {
    const int H = g.V / 2;
    dim3 grid((unsigned)((H + threads - 1) / threads), (unsigned)nrhs);
    k_dslash_pair<<<grid, threads, 0, s>>>(mode, pl, (const float2 *)in, (float2 *)out, g, diag, skip);
}

}  // namespace bri

#define BRI_INSTANTIATE_DSLASH_PAIR(PL) \
    template void bri::dslash_pair_launch<PL>(int, const PL &, const void *, void *, int, const bri::Geom &, double, const int *, int, cudaStream_t);
