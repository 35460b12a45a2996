// The stencil apply (Eq. def_pref, c_SW = 0, in the class form of Sec. 8):
//
//   out(x) = (m0 + lambda_0) psi(x)
//          + sum_{d != 0} s_d(x) [lambda_n + rho_n sum_mu d_mu gamma_mu] (x) W_d(x) psi(x + d)
//
// One thread per (site, right-hand side).  The 80 hops are walked as 40 pairs
// (d, -d) over the stored canonical fields: W_d(x) for the forward hop and
// W_d(x - d)^dagger for the reversed one.  Each hop is: load W (coalesced
// 128-bit SoA chunks), load the neighbour spinor, four colour mat-vecs; the spin
// structure is taken as real-coefficient accumulations (gamma entries are +-1,
// +-i), in most variants once per pair on the difference of the two colour
// products.  FP64: the pair loop is a compile-time fold (offsets and gamma signs
// constant); FP32 arithmetic: a loop over the hop table in the kernel
// parameters (the unrolled form does not fit the instruction cache).
//   mode 0: D;  mode 1: D^dagger = gamma_5 D gamma_5 (rho -> -rho, Sec. 1);
//   mode 2: gamma_5 (D - rho): diagonal -rho + lambda_0, gamma_5 applied to the
//           result (overlap kernel, Sec. 7.4).
// Each link format is instantiated in its own translation unit (dslash_*.cu)
// so the kernels compile in parallel.
#pragma once
#include <utility>

#include "ctx.h"
#include "links.cuh"
#include "tile.cuh"

namespace bri {


BRI_D void load_spinor(const float2 *__restrict__ p, float2 o[12]) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < 6; i++) {
        float4 v = q[i];
        o[2 * i] = make_float2(v.x, v.y);
        o[2 * i + 1] = make_float2(v.z, v.w);
    }
}
BRI_D void load_spinor(const double2 *__restrict__ p, double2 o[12]) {
#pragma unroll
    for (int i = 0; i < 12; i++) o[i] = p[i];
}
BRI_D void store_spinor(float2 *__restrict__ p, const float2 o[12]) {
    float4 *q = reinterpret_cast<float4 *>(p);
#pragma unroll
    for (int i = 0; i < 6; i++) q[i] = make_float4(o[2 * i].x, o[2 * i].y, o[2 * i + 1].x, o[2 * i + 1].y);
}
BRI_D void store_spinor(double2 *__restrict__ p, const double2 o[12]) {
#pragma unroll
    for (int i = 0; i < 12; i++) p[i] = o[i];
}

template <typename T> struct RealOf;
template <> struct RealOf<float2> { using R = float; };
template <> struct RealOf<double2> { using R = double; };

// acc += s * z  and  acc += s * (i z)
template <typename T, typename R> BRI_D void acc_re(T &acc, R s, T z) {
    acc.x += s * z.x;
    acc.y += s * z.y;
}
template <typename T, typename R> BRI_D void acc_im(T &acc, R s, T z) {
    acc.x -= s * z.y;
    acc.y += s * z.x;
}

// Accumulators.  FP32: the terms with a real gamma entry go to a, those with
// an imaginary entry (+-i) to ai, and out = a + i ai at the end, so every
// accumulation is a real-coefficient packed FMA (fma.rn.f32x2 on sm_103a: two
// FP32 FMAs per instruction, halving the issue slots of the arithmetic).
struct AccF {
    float2 a[12], ai[12];
};
struct AccD {
    double2 a[12];
};
template <typename T> struct AccOf;
template <> struct AccOf<float2> { using A = AccF; };
template <> struct AccOf<double2> { using A = AccD; };

BRI_D float2 f2(float v) { return make_float2(v, v); }

// FP32 hop with packed FMAs, chi = W psi as sum_c' (psi.re * w + psi.im * (i w)),
// with the offset d a runtime value: the FP32 kernels loop over the 40 (d, -d)
// pairs instead of unrolling them, which keeps the kernel small enough for the
// instruction cache (the unrolled form stalls on instruction fetch).  The gamma
// terms are taken under warp-uniform branches on d_mu, so no arithmetic is
// wasted; the spin permutations stay compile-time.
template <int SGN>
BRI_D void hop_body(const M3<float2> &W, const float2 p[12], float l, float r, const int dm[4], AccF &acc) {
    float2 A[9], B[9];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int cp = 0; cp < 3; cp++) {
            const float2 w = SGN > 0 ? W.e[3 * c + cp] : make_float2(W.e[3 * cp + c].x, -W.e[3 * cp + c].y);
            A[3 * c + cp] = w;
            B[3 * c + cp] = make_float2(-w.y, w.x);
        }
#pragma unroll
    for (int sp = 0; sp < 4; sp++) {
        float2 chi[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float2 t = __fmul2_rn(A[3 * c], f2(p[3 * sp].x));
            t = __ffma2_rn(B[3 * c], f2(p[3 * sp].y), t);
            t = __ffma2_rn(A[3 * c + 1], f2(p[3 * sp + 1].x), t);
            t = __ffma2_rn(B[3 * c + 1], f2(p[3 * sp + 1].y), t);
            t = __ffma2_rn(A[3 * c + 2], f2(p[3 * sp + 2].x), t);
            t = __ffma2_rn(B[3 * c + 2], f2(p[3 * sp + 2].y), t);
            chi[c] = t;
        }
#pragma unroll
        for (int c = 0; c < 3; c++) acc.a[3 * sp + c] = __ffma2_rn(f2(l), chi[c], acc.a[3 * sp + c]);
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            if (dm[mu] == 0) continue;  // uniform across the warp
            const int s = gcol(mu, sp);
            const int gr = gre(mu, s), gi = gim(mu, s);
            const float cf = r * (float)(SGN * dm[mu] * (gr != 0 ? gr : gi));
#pragma unroll
            for (int c = 0; c < 3; c++) {
                if (gr != 0) acc.a[3 * s + c] = __ffma2_rn(f2(cf), chi[c], acc.a[3 * s + c]);
                else acc.ai[3 * s + c] = __ffma2_rn(f2(cf), chi[c], acc.ai[3 * s + c]);
            }
        }
    }
}


// Variant of hop_body without the separate accumulator for the +-i gamma
// entries: i chi is formed where it is needed (fewer registers, more moves).
template <int SGN>
BRI_D void hop_body_w(const M3<float2> &W, const float2 p[12], float l, float r, const int dm[4], AccF &acc) {
    float2 A[9], B[9];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int cp = 0; cp < 3; cp++) {
            const float2 w = SGN > 0 ? W.e[3 * c + cp] : make_float2(W.e[3 * cp + c].x, -W.e[3 * cp + c].y);
            A[3 * c + cp] = w;
            B[3 * c + cp] = make_float2(-w.y, w.x);
        }
#pragma unroll
    for (int sp = 0; sp < 4; sp++) {
        float2 chi[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float2 t = __fmul2_rn(A[3 * c], f2(p[3 * sp].x));
            t = __ffma2_rn(B[3 * c], f2(p[3 * sp].y), t);
            t = __ffma2_rn(A[3 * c + 1], f2(p[3 * sp + 1].x), t);
            t = __ffma2_rn(B[3 * c + 1], f2(p[3 * sp + 1].y), t);
            t = __ffma2_rn(A[3 * c + 2], f2(p[3 * sp + 2].x), t);
            t = __ffma2_rn(B[3 * c + 2], f2(p[3 * sp + 2].y), t);
            chi[c] = t;
        }
#pragma unroll
        for (int c = 0; c < 3; c++) acc.a[3 * sp + c] = __ffma2_rn(f2(l), chi[c], acc.a[3 * sp + c]);
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            if (dm[mu] == 0) continue;  // uniform across the warp
            const int s = gcol(mu, sp);
            const int gr = gre(mu, s), gi = gim(mu, s);
            const float cf = r * (float)(SGN * dm[mu] * (gr != 0 ? gr : gi));
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float2 z = gr != 0 ? chi[c] : make_float2(-chi[c].y, chi[c].x);
                acc.a[3 * s + c] = __ffma2_rn(f2(cf), z, acc.a[3 * s + c]);
            }
        }
    }
}

// chi = W psi (SGN = 1) or W^dagger psi (SGN = -1) for the four spins, with
// packed FMAs as in hop_body
template <int SGN>
BRI_D void colour_mv(const M3<float2> &W, const float2 p[12], float2 chi[12]) {
    float2 A[9], B[9];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int cp = 0; cp < 3; cp++) {
            const float2 w = SGN > 0 ? W.e[3 * c + cp] : make_float2(W.e[3 * cp + c].x, -W.e[3 * cp + c].y);
            A[3 * c + cp] = w;
            B[3 * c + cp] = make_float2(-w.y, w.x);
        }
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float2 t = __fmul2_rn(A[3 * c], f2(p[3 * sp].x));
            t = __ffma2_rn(B[3 * c], f2(p[3 * sp].y), t);
            t = __ffma2_rn(A[3 * c + 1], f2(p[3 * sp + 1].x), t);
            t = __ffma2_rn(B[3 * c + 1], f2(p[3 * sp + 1].y), t);
            t = __ffma2_rn(A[3 * c + 2], f2(p[3 * sp + 2].x), t);
            t = __ffma2_rn(B[3 * c + 2], f2(p[3 * sp + 2].y), t);
            chi[3 * sp + c] = t;
        }
}

// One (d, -d) pair at once.  With q = phf phb (boundary phases, +-1) the two
// hops add up to
//   phf [ lam (chi_f + q chi_b) + rsign rho sum_mu d_mu gamma_mu (chi_f - q chi_b) ],
// chi_f = W_d(x) psi(x + d), chi_b = W_d(x - d)^dagger psi(x - d): the gamma
// terms are taken once per pair on the difference instead of once per hop, which
// saves 12 (n - 1) packed FMAs per pair of class n.  cf holds chi_f on entry and
// is overwritten with the difference, so the gamma terms run after the spin
// loop with one warp-uniform branch per direction.  W and p are the reversed
// hop's field and spinor; L = lam phf, R = rsign rho phf.
BRI_D void pair_body(float2 cf[12], const M3<float2> &W, const float2 p[12], float L, float q, float R,
                     const HopArg &h, AccF &acc) {
    float2 A[9], B[9];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int cp = 0; cp < 3; cp++) {
            const float2 w = make_float2(W.e[3 * cp + c].x, -W.e[3 * cp + c].y);
            A[3 * c + cp] = w;
            B[3 * c + cp] = make_float2(-w.y, w.x);
        }
#pragma unroll
    for (int sp = 0; sp < 4; sp++) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float2 t = __fmul2_rn(A[3 * c], f2(p[3 * sp].x));
            t = __ffma2_rn(B[3 * c], f2(p[3 * sp].y), t);
            t = __ffma2_rn(A[3 * c + 1], f2(p[3 * sp + 1].x), t);
            t = __ffma2_rn(B[3 * c + 1], f2(p[3 * sp + 1].y), t);
            t = __ffma2_rn(A[3 * c + 2], f2(p[3 * sp + 2].x), t);
            t = __ffma2_rn(B[3 * c + 2], f2(p[3 * sp + 2].y), t);
            const float2 sm = __ffma2_rn(f2(q), t, cf[3 * sp + c]);
            cf[3 * sp + c] = __ffma2_rn(f2(-q), t, cf[3 * sp + c]);
            acc.a[3 * sp + c] = __ffma2_rn(f2(L), sm, acc.a[3 * sp + c]);
        }
    }
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        if (h.dm[mu] == 0) continue;  // uniform across the warp
        const float rd = R * h.fd[mu];
#pragma unroll
        for (int sp = 0; sp < 4; sp++) {
            const int s = gcol(mu, sp);
            const int gr = gre(mu, s), gi = gim(mu, s);
            const float cfm = gr != 0 ? (gr > 0 ? rd : -rd) : (gi > 0 ? rd : -rd);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                if (gr != 0) acc.a[3 * s + c] = __ffma2_rn(f2(cfm), cf[3 * sp + c], acc.a[3 * s + c]);
                else acc.ai[3 * s + c] = __ffma2_rn(f2(cfm), cf[3 * sp + c], acc.ai[3 * s + c]);
            }
        }
    }
}

// One (d, -d) pair at once with the gamma terms inside the spin loop (launch
// variants 5 and 6; pair_body below is the same arithmetic with the gamma
// terms after the spin loop, variant 7).  With q = phf phb (boundary phases, +-1) the two
// hops add up to
//   phf [ lam (chi_f + q chi_b) + rsign rho sum_mu d_mu gamma_mu (chi_f - q chi_b) ],
// chi_f = W_d(x) psi(x + d), chi_b = W_d(x - d)^dagger psi(x - d): the gamma
// terms are taken once per pair on the difference instead of once per hop, which
// saves 12 (n - 1) packed FMAs per pair of class n.  cf holds chi_f; W and p are
// the reversed hop's field and spinor; L = lam phf, R = rsign rho phf.
// ALLMU = false takes the gamma terms of the directions with d_mu != 0 under
// warp-uniform branches; ALLMU = true takes all four with zero coefficients
// where d_mu = 0 (12 (4 - n) more packed FMAs, no branch inside the pair),
// which leaves the compiler one block to schedule and fewer live registers
// (the line kernel with FP32 full fields: 126 instead of 144).
template <bool ALLMU>
BRI_D void pair_body_s(const float2 cf[12], const M3<float2> &W, const float2 p[12], float L, float q, float R,
                       const HopArg &h, AccF &acc) {
    float2 A[9], B[9];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int cp = 0; cp < 3; cp++) {
            const float2 w = make_float2(W.e[3 * cp + c].x, -W.e[3 * cp + c].y);
            A[3 * c + cp] = w;
            B[3 * c + cp] = make_float2(-w.y, w.x);
        }
    float rd[4];
#pragma unroll
    for (int mu = 0; mu < 4; mu++) rd[mu] = R * h.fd[mu];
#pragma unroll
    for (int sp = 0; sp < 4; sp++) {
        float2 sm[3], df[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float2 t = __fmul2_rn(A[3 * c], f2(p[3 * sp].x));
            t = __ffma2_rn(B[3 * c], f2(p[3 * sp].y), t);
            t = __ffma2_rn(A[3 * c + 1], f2(p[3 * sp + 1].x), t);
            t = __ffma2_rn(B[3 * c + 1], f2(p[3 * sp + 1].y), t);
            t = __ffma2_rn(A[3 * c + 2], f2(p[3 * sp + 2].x), t);
            t = __ffma2_rn(B[3 * c + 2], f2(p[3 * sp + 2].y), t);
            sm[c] = __ffma2_rn(f2(q), t, cf[3 * sp + c]);
            df[c] = __ffma2_rn(f2(-q), t, cf[3 * sp + c]);
        }
#pragma unroll
        for (int c = 0; c < 3; c++) acc.a[3 * sp + c] = __ffma2_rn(f2(L), sm[c], acc.a[3 * sp + c]);
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            if (!ALLMU && h.dm[mu] == 0) continue;  // uniform across the warp
            const int s = gcol(mu, sp);
            const int gr = gre(mu, s), gi = gim(mu, s);
            const float cfm = gr != 0 ? (gr > 0 ? rd[mu] : -rd[mu]) : (gi > 0 ? rd[mu] : -rd[mu]);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                if (gr != 0) acc.a[3 * s + c] = __ffma2_rn(f2(cfm), df[c], acc.a[3 * s + c]);
                else acc.ai[3 * s + c] = __ffma2_rn(f2(cfm), df[c], acc.ai[3 * s + c]);
            }
        }
    }
}

// FP32 stencil over the 40 (d, -d) pairs as a compact loop.  PF = true also
// prefetches the two links of the next pair into L2 (the links stream from DRAM;
// the neighbour spinors mostly hit L1/L2).
template <bool PF, int BODY, class LL>
BRI_D void f32_hops(const LL &ll, const float2 *__restrict__ in, int site, const SiteNb &nb, float rsign,
                    const Geom &g, AccF &acc) {
    if constexpr (BODY == 2 || BODY == 3) {
        // pair-combined body (pair_body), links of the next pair prefetched into L2
#pragma unroll 1
        for (int t = 0; t < g.nhop; t++) {
            if (PF && t + 1 < g.nhop) {
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
                M3<float2> W = ll.load(hc.j, site);
                float2 q[12];
                load_spinor(in + (size_t)yf * 12, q);
                colour_mv<1>(W, q, cf);
            }
            M3<float2> W = ll.load(hc.j, yb);
            float2 q[12];
            load_spinor(in + (size_t)yb * 12, q);
            if constexpr (BODY == 3) pair_body(cf, W, q, hc.lam * phf, phf * phb, hc.rho * rsign * phf, hc, acc);
            else
                pair_body_s<LL::COMP != BRI_LINK_8PARAM>(cf, W, q, hc.lam * phf, phf * phb, hc.rho * rsign * phf, hc,
                                                         acc);
        }
    } else if constexpr (!PF && BODY == 1) {
#pragma unroll 1
        for (int t = 0; t < g.nhop; t++) {
            const HopArg hc = g.hop[t];
            const int j = hc.j;
            int yf, yb;
            float phf, phb;
            hop_nb(hc.dm, site, nb, yf, phf, yb, phb);
            {
                M3<float2> W = ll.load(j, site);
                float2 q[12];
                load_spinor(in + (size_t)yf * 12, q);
                hop_body_w<1>(W, q, hc.lam * phf, hc.rho * rsign * phf, hc.dm, acc);
            }
            {
                M3<float2> W = ll.load(j, yb);
                float2 q[12];
                load_spinor(in + (size_t)yb * 12, q);
                hop_body_w<-1>(W, q, hc.lam * phb, hc.rho * rsign * phb, hc.dm, acc);
            }
        }
    } else if constexpr (!PF) {
#pragma unroll 1
        for (int t = 0; t < g.nhop; t++) {
            const HopArg hc = g.hop[t];
            const int j = hc.j;
            int yf, yb;
            float phf, phb;
            hop_nb(hc.dm, site, nb, yf, phf, yb, phb);
            {
                M3<float2> W = ll.load(j, site);
                float2 q[12];
                load_spinor(in + (size_t)yf * 12, q);
                hop_body<1>(W, q, hc.lam * phf, hc.rho * rsign * phf, hc.dm, acc);
            }
            {
                M3<float2> W = ll.load(j, yb);
                float2 q[12];
                load_spinor(in + (size_t)yb * 12, q);
                hop_body<-1>(W, q, hc.lam * phb, hc.rho * rsign * phb, hc.dm, acc);
            }
        }
    } else {
        // the links of pair t + 1 are prefetched into L2 while pair t is computed
        // (measured: distance 1 > 2 > 3; prefetch into L1 instead makes no difference)
#pragma unroll 1
        for (int t = 0; t < g.nhop; t++) {
            if (t + 1 < g.nhop) {
                const HopArg hp = g.hop[t + 1];
                int pyf, pyb;
                float pphf, pphb;
                hop_nb(hp.dm, site, nb, pyf, pphf, pyb, pphb);
                ll.prefetch_field_l2(hp.j, site);
                ll.prefetch_field_l2(hp.j, pyb);
            }
            const HopArg hc = g.hop[t];
            const int j = hc.j;
            int yf, yb;
            float phf, phb;
            hop_nb(hc.dm, site, nb, yf, phf, yb, phb);
            {
                M3<float2> W = ll.load(j, site);
                float2 q[12];
                load_spinor(in + (size_t)yf * 12, q);
                hop_body<1>(W, q, hc.lam * phf, hc.rho * rsign * phf, hc.dm, acc);
            }
            {
                M3<float2> W = ll.load(j, yb);
                float2 q[12];
                load_spinor(in + (size_t)yb * 12, q);
                hop_body<-1>(W, q, hc.lam * phb, hc.rho * rsign * phb, hc.dm, acc);
            }
        }
    }
}


// The pair loop of variant 5 with cheaper addressing (launch variant 9): the
// per-site part of every link address is computed once, each field adds
// j VP NQ, and the neighbours of the next pair (found for its L2 prefetch)
// are carried into the next iteration instead of being recomputed.
template <class LL>
BRI_D void f32_hops_lean(const LL &ll, const float2 *__restrict__ in, int site, const SiteNb &nb, float rsign,
                         const Geom &g, AccF &acc) {
    if (g.nhop == 0) return;
    const long long sc = ll.cidx(site);
    int yf, yb;
    float phf, phb;
    hop_nb(g.hop[0].dm, site, nb, yf, phf, yb, phb);
    long long bc = ll.cidx(yb);
#pragma unroll 1
    for (int t = 0; t < g.nhop; t++) {
        const int cyf = yf, cyb = yb;
        const float cphf = phf, cphb = phb;
        const long long cbc = bc;
        if (t + 1 < g.nhop) {
            const int jn = g.hop[t + 1].j;
            hop_nb(g.hop[t + 1].dm, site, nb, yf, phf, yb, phb);
            bc = ll.cidx(yb);
            ll.prefetch_ci(jn, sc, site);
            ll.prefetch_ci(jn, bc, yb);
        }
        const HopArg hc = g.hop[t];
        float2 cf[12];
        {
            const M3<float2> W = ll.load_ci(hc.j, sc, site);
            float2 q[12];
            load_spinor(in + (size_t)cyf * 12, q);
            colour_mv<1>(W, q, cf);
        }
        const M3<float2> W = ll.load_ci(hc.j, cbc, cyb);
        float2 q[12];
        load_spinor(in + (size_t)cyb * 12, q);
        pair_body_s<LL::COMP == BRI_LINK_2ROW>(cf, W, q, hc.lam * cphf, cphf * cphb, hc.rho * rsign * cphf, hc, acc);
    }
}

// FP32 stencil loop with the links of pair j + 1 copied asynchronously
// (cp.async) into this thread's double-buffered shared-memory slots while pair
// j is computed: the DRAM latency of the links overlaps the arithmetic and
// costs no registers.  lbase: this thread's slots (2 stages x 2 links).
template <class LL>
BRI_D void f32_hops_cpasync(const LL &ll, const float2 *__restrict__ in, int site, const SiteNb &nb, float rsign,
                            const Geom &g, uint32_t lbase, AccF &acc) {
    // layout [stage][field][chunk][thread] of 16-byte slots; lbase = this thread's
    // slot of stage 0, field 0, chunk 0
    const uint32_t stride = 16u * blockDim.x;      // between chunks
    const uint32_t LB = stride * LL::SLOTS;        // between the two fields of a stage
    if (g.nhop == 0) return;
    HopArg hc = g.hop[0];
    int yf, yb;
    float phf, phb;
    hop_nb(hc.dm, site, nb, yf, phf, yb, phb);
    ll.prefetch(hc.j, site, lbase, stride);
    ll.prefetch(hc.j, yb, lbase + LB, stride);
    asm volatile("cp.async.commit_group;" ::: "memory");
#pragma unroll 1
    for (int t = 0; t < g.nhop; t++) {
        const HopArg h = hc;
        const int cyf = yf, cyb = yb;
        const float cphf = phf, cphb = phb;
        const uint32_t cur = lbase + (uint32_t)(t & 1) * 2 * LB;
        if (t + 1 < g.nhop) {
            hc = g.hop[t + 1];
            hop_nb(hc.dm, site, nb, yf, phf, yb, phb);
            const uint32_t nxt = lbase + (uint32_t)((t + 1) & 1) * 2 * LB;
            ll.prefetch(hc.j, site, nxt, stride);
            ll.prefetch(hc.j, yb, nxt + LB, stride);
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 1;" ::: "memory");
        {
            const M3<float2> W = ll.load_smem(cur, stride);
            float2 q[12];
            load_spinor(in + (size_t)cyf * 12, q);
            hop_body<1>(W, q, h.lam * cphf, h.rho * rsign * cphf, h.dm, acc);
        }
        {
            const M3<float2> W = ll.load_smem(cur + LB, stride);
            float2 q[12];
            load_spinor(in + (size_t)cyb * 12, q);
            hop_body<-1>(W, q, h.lam * cphb, h.rho * rsign * cphb, h.dm, acc);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---- bulk-copy link pipeline (launch variant 10) ---------------------------
// Every warp stages the links of its coming pairs in a ring of ST shared-memory
// stages.  A stage holds 32-site blocks ("runs", LL::RUN_A + LL::RUN_B bytes)
// of the pair's field j: the block of the warp's own 32 sites (forward hop,
// W_d(x)) and the blocks that hold lane 0's and lane 31's x - d (reversed hop,
// W_d(x - d)).  NB = 1 stages lane 0's block only, which holds every lane's
// x - d when the x extent is 32 (a warp is one x line, and x - d is one x line
// again).  Lane 0 issues the runs as 1-D bulk copies, counted in bytes on the
// stage's mbarrier, ST - 1 pairs ahead of the pair being computed, so the
// links cost each lane neither address arithmetic nor prefetch instructions; a
// lane whose x - d lies in no staged block loads that link from global memory.
// A wait that has not completed after BULK_WAIT_NS gives up: the loop drains
// the stages still in flight (with the same limit) and returns false.
constexpr unsigned long long BULK_WAIT_NS = 1000000000ull;

template <class LL, int NB>
BRI_D void bulk_issue(const LL &ll, const Geom &g, int t, int site, const SiteNb &nb, int wblk, uint32_t dst,
                      uint32_t bar, uint32_t extra) {
    constexpr uint32_t RUN = LL::RUN_A + LL::RUN_B;
    int yf, yb;
    float pf, pb;
    hop_nb(g.hop[t].dm, site, nb, yf, pf, yb, pb);
    const int c0 = __shfl_sync(0xffffffffu, yb >> 5, 0);
    const int c1 = NB == 2 ? __shfl_sync(0xffffffffu, yb >> 5, 31) : c0;
    if ((threadIdx.x & 31) == 0) {
        const int j = g.hop[t].j;
        fence_async_smem();
        mbar_arrive_tx(bar, (c1 != c0 ? 3u : 2u) * RUN + extra);
        ll.bulk_run(j, wblk, dst, bar);
        ll.bulk_run(j, c0, dst + RUN, bar);
        if (c1 != c0) ll.bulk_run(j, c1, dst + 2 * RUN, bar);
    }
}

template <class LL, int ST, int NB>
BRI_D bool f32_hops_bulk(const LL &ll, const float2 *__restrict__ in, int site, int wblk, const SiteNb &nb,
                         float rsign, const Geom &g, uint32_t ring, uint32_t bars, AccF &acc) {
    constexpr uint32_t RUN = LL::RUN_A + LL::RUN_B;
    constexpr uint32_t STAGE = RUN * (1 + NB);
    const int lane = (int)threadIdx.x & 31;
    const int nh = g.nhop;
    const uint32_t extra0 = g.stall ? 16u : 0u;
#pragma unroll
    for (int t = 0; t < ST - 1; t++)
        if (t < nh) bulk_issue<LL, NB>(ll, g, t, site, nb, wblk, ring + STAGE * t, bars + 8u * t, t == 0 ? extra0 : 0u);
    int s = 0;          // stage of pair t
    uint32_t par = 0;   // parity of its current phase
#pragma unroll 1
    for (int t = 0; t < nh; t++) {
        if (t + ST - 1 < nh) {
            // the stage pair t - 1 used: every lane has read it
            __syncwarp();
            const int sn = s == 0 ? ST - 1 : s - 1;
            bulk_issue<LL, NB>(ll, g, t + ST - 1, site, nb, wblk, ring + STAGE * sn, bars + 8u * sn, 0u);
        }
        const HopArg hc = g.hop[t];
        int yf, yb;
        float phf, phb;
        hop_nb(hc.dm, site, nb, yf, phf, yb, phb);
        const int c0 = __shfl_sync(0xffffffffu, yb >> 5, 0);
        const int c1 = NB == 2 ? __shfl_sync(0xffffffffu, yb >> 5, 31) : c0;
        const uint32_t cur = ring + STAGE * s;
        if (!mbar_wait(bars + 8u * s, par, BULK_WAIT_NS)) {
            // drain the later stages this warp has issued, then give up
            int sd = s;
            uint32_t pd = par;
            for (int u = t + 1; u < nh && u < t + ST; u++) {
                if (++sd == ST) { sd = 0; pd ^= 1u; }
                mbar_wait(bars + 8u * sd, pd, BULK_WAIT_NS);
            }
            return false;
        }
        float2 cf[12];
        {
            const M3<float2> W = ll.load_run(cur, lane);
            float2 q[12];
            load_spinor(in + (size_t)yf * 12, q);
            colour_mv<1>(W, q, cf);
        }
        const int cb = yb >> 5;
        M3<float2> W;
        if (cb == c0) W = ll.load_run(cur + RUN, yb & 31);
        else if (NB == 2 && cb == c1) W = ll.load_run(cur + 2 * RUN, yb & 31);
        else W = ll.load(hc.j, yb);
        float2 q[12];
        load_spinor(in + (size_t)yb * 12, q);
        pair_body_s<false>(cf, W, q, hc.lam * phf, phf * phb, hc.rho * rsign * phf, hc, acc);
        if (++s == ST) { s = 0; par ^= 1u; }
    }
    return true;
}

// FP64 row products chi[c] = sum_c' w_cc' p_c' of spin sp as explicit FMA
// chains (one multiply and five FMAs per real component): w = W (SGN = 1) or
// W^dagger (SGN = -1).  Complex products followed by complex adds would cost
// 16 FP64 operations per row instead of 12, and GB300's FP64 pipe is the limit.
template <int SGN>
BRI_D void mv64(const M3<double2> &W, const double2 p[12], int sp, double2 chi[3]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        double re = 0, im = 0;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const double2 e = SGN > 0 ? W.e[3 * c + k] : W.e[3 * k + c];
            const double wx = e.x, wy = SGN > 0 ? e.y : -e.y;
            const double2 v = p[3 * sp + k];
            if (k == 0) {
                re = wx * v.x;
                im = wx * v.y;
            } else {
                re = fma(wx, v.x, re);
                im = fma(wx, v.y, im);
            }
            re = fma(-wy, v.y, re);
            im = fma(wy, v.x, im);
        }
        chi[c] = make_double2(re, im);
    }
}

// FP64 (d, -d) pair with offsets, weights and gamma signs fixed at compile time:
// with q = phf phb the two hops add up to
//   phf [ lam (chi_f + q chi_b) + rsign rho sum_mu d_mu gamma_mu (chi_f - q chi_b) ]
// (the gamma terms once per pair, on the difference; cf is overwritten with it).
template <int J, class LL>
BRI_D void hop_pair(const LL &ll, const typename LL::T *__restrict__ in, int site, const SiteNb &nb,
                    float rsign, const Geom &g, typename AccOf<typename LL::T>::A &acc) {
    constexpr int K = canon_k(J);
    constexpr int n = off_class(K);
    if (g.lamd[n] == 0.0 && g.rhod[n] == 0.0) return;  // class not in the operator
    float phf, phb;
    const int yf = nb_index<K, 1>(nb, site, phf);
    const int yb = nb_index<K, -1>(nb, site, phb);
    double2 cf[12];
    {
        const M3<double2> W = ll.load(J, site);
        double2 p[12];
        load_spinor(in + (size_t)yf * 12, p);
#pragma unroll
        for (int sp = 0; sp < 4; sp++) mv64<1>(W, p, sp, cf + 3 * sp);
    }
    const double q = (double)(phf * phb);
    const double L = g.lamd[n] * (double)phf, R = g.rhod[n] * (double)(phf * rsign);
    {
        const M3<double2> W = ll.load(J, yb);
        double2 p[12];
        load_spinor(in + (size_t)yb * 12, p);
#pragma unroll
        for (int sp = 0; sp < 4; sp++) {
            double2 cb[3];
            mv64<-1>(W, p, sp, cb);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                double2 &f = cf[3 * sp + c];
                const double sx = fma(q, cb[c].x, f.x), sy = fma(q, cb[c].y, f.y);
                f.x = fma(-q, cb[c].x, f.x);
                f.y = fma(-q, cb[c].y, f.y);
                acc.a[3 * sp + c].x = fma(L, sx, acc.a[3 * sp + c].x);
                acc.a[3 * sp + c].y = fma(L, sy, acc.a[3 * sp + c].y);
            }
        }
    }
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int dm = off_comp(K, mu);
        if (dm == 0) continue;
#pragma unroll
        for (int sp = 0; sp < 4; sp++) {
            // row s of gamma_mu has its entry in column sp
            const int s = gcol(mu, sp);
            const int gr = gre(mu, s), gi = gim(mu, s);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                if (gr != 0) acc_re(acc.a[3 * s + c], R * (double)(dm * gr), cf[3 * sp + c]);
                else acc_im(acc.a[3 * s + c], R * (double)(dm * gi), cf[3 * sp + c]);
            }
        }
    }
}

template <class LL, int... Js>
BRI_D void all_hops(std::integer_sequence<int, Js...>, const LL &ll, const typename LL::T *__restrict__ in,
                    int site, const SiteNb &nb, float rsign, const Geom &g,
                    typename AccOf<typename LL::T>::A &acc) {
    (hop_pair<Js>(ll, in, site, nb, rsign, g, acc), ...);
}

// o += C(x) p with the packed clover blocks of Geom (hermitian 6x6 per chirality)
template <typename T>
BRI_D void clover_block(const T c[18], const T *p, T *o) {
    using R = decltype(c[0].x);
    R d[6] = {c[0].x, c[0].y, c[1].x, c[1].y, c[2].x, c[2].y};
    T r[6];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        r[i].x = d[i] * p[i].x;
        r[i].y = d[i] * p[i].y;
    }
    int k = 3;
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int j = i + 1; j < 6; j++, k++) {
            const T e = c[k];  // C_ij; C_ji = conj(C_ij)
            r[i].x += e.x * p[j].x - e.y * p[j].y;
            r[i].y += e.x * p[j].y + e.y * p[j].x;
            r[j].x += e.x * p[i].x + e.y * p[i].y;
            r[j].y += e.x * p[i].y - e.y * p[i].x;
        }
#pragma unroll
    for (int i = 0; i < 6; i++) {
        o[i].x += r[i].x;
        o[i].y += r[i].y;
    }
}
template <typename T>
BRI_D void clover_add(const Geom &g, int site, const T p[12], T o[12]) {
#pragma unroll
    for (int b = 0; b < 2; b++) {
        T c[18];
        if constexpr (sizeof(T) == 16) {
#pragma unroll
            for (int e = 0; e < 18; e++) c[e] = g.clov64[(size_t)(18 * b + e) * g.V + site];
        } else {
#pragma unroll
            for (int e = 0; e < 9; e++) {
                const float4 q = g.clov32[(size_t)(9 * b + e) * g.V + site];
                c[2 * e] = make_float2(q.x, q.y);
                c[2 * e + 1] = make_float2(q.z, q.w);
            }
        }
        clover_block(c, p + 6 * b, o + 6 * b);
    }
}

// out(x) = diag psi(x) + the hop sum (+ the clover term), times gamma_5 for mode 2
template <typename T, bool CLOV>
BRI_D void dslash_finish(int mode, const T *__restrict__ in, T *__restrict__ out, int site, const Geom &g, double diag,
                         const typename AccOf<T>::A &acc) {
    using R = typename RealOf<T>::R;
    T p[12];
    load_spinor(in + (size_t)site * 12, p);
    const R dg = (R)diag;
    T o[12];
#pragma unroll
    for (int i = 0; i < 12; i++) {
        T v;
        v.x = dg * p[i].x + acc.a[i].x;
        v.y = dg * p[i].y + acc.a[i].y;
        if constexpr (sizeof(T) == 8) {
            v.x -= acc.ai[i].y;
            v.y += acc.ai[i].x;
        }
        o[i] = v;
    }
    if constexpr (CLOV) clover_add(g, site, p, o);
    if (mode == 2) {
#pragma unroll
        for (int i = 6; i < 12; i++) { o[i].x = -o[i].x; o[i].y = -o[i].y; }
    }
    store_spinor(out + (size_t)site * 12, o);
}

// CLOV: add the clover term of Geom in the epilogue (a separate instantiation,
// so that the kernels without it keep their register budget)
template <class LL, int VAR, bool CLOV>
BRI_D void dslash_body(int mode, const LL &ll, const typename LL::T *__restrict__ in, typename LL::T *__restrict__ out,
                       const Geom &g, double diag, const int *__restrict__ skip) {
    using T = typename LL::T;
    // grid.x = site blocks x right-hand sides with the RHS fastest, so the blocks
    // of all RHS over the same sites run together and read each link from DRAM
    // once (the others hit L2)
    const int nblk = (g.s1 - g.s0 + (int)blockDim.x - 1) / (int)blockDim.x;
    const int nr = (int)gridDim.x / nblk;
    const int rhs = (int)blockIdx.x % nr;
    const int site = g.s0 + ((int)blockIdx.x / nr) * (int)blockDim.x + (int)threadIdx.x;
    if (site >= g.s1) return;
    if (skip && skip[rhs]) return;
    const size_t off = (size_t)rhs * g.V * 12;
    in += off;
    out += off;
    int x[4];
    const SiteNb nb = site_nb(g, site, x);
    typename AccOf<T>::A acc;
#pragma unroll
    for (int i = 0; i < 12; i++) acc.a[i] = mk<T>(0, 0);
    if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int i = 0; i < 12; i++) acc.ai[i] = mk<T>(0, 0);
    }
    const float rsign = mode == 1 ? -1.f : 1.f;
    if constexpr (sizeof(T) == 8) {
        if constexpr (VAR == 2) {
            extern __shared__ float4 lslots[];
            const uint32_t lbase = (uint32_t)__cvta_generic_to_shared(lslots) + threadIdx.x * 16u;
            f32_hops_cpasync(ll, in, site, nb, rsign, g, lbase, acc);
        } else if constexpr (VAR == 9) {
            f32_hops_lean(ll, in, site, nb, rsign, g, acc);
        } else {
            // VAR 5 (and 6, through k_dslash_r128): pair_body_s; VAR 7: pair_body.
            // The branch-free gamma terms (pair_body_s<true>) measured 1-2% faster
            // in variants 5 and 9 for full and 2-row fields, and 1-3% slower for
            // 8-parameter fields and, in variant 9, FP16 full ones
            f32_hops<VAR == 1 || VAR >= 5, VAR == 4 ? 1 : VAR == 5 ? 2 : VAR == 7 ? 3 : 0>(ll, in, site, nb, rsign, g,
                                                                                          acc);
        }
    } else {
        all_hops(std::make_integer_sequence<int, NCANON>{}, ll, in, site, nb, rsign, g, acc);
    }
    dslash_finish<T, CLOV>(mode, in, out, site, g, diag, acc);
}

template <class LL, int VAR, bool CLOV = false>
__global__ void k_dslash(int mode, LL ll, const typename LL::T *__restrict__ in, typename LL::T *__restrict__ out,
                         Geom g, double diag, const int *__restrict__ skip) {
    dslash_body<LL, VAR, CLOV>(mode, ll, in, out, g, diag, skip);
}
// launch variant 6: variant 5 held to 128 registers (16 warps per SM)
template <class LL>
__global__ void __maxnreg__(128) k_dslash_r128(int mode, LL ll, const typename LL::T *__restrict__ in,
                                               typename LL::T *__restrict__ out, Geom g, double diag,
                                               const int *__restrict__ skip) {
    dslash_body<LL, 5, false>(mode, ll, in, out, g, diag, skip);
}

// launch variant 10: the bulk-copy link pipeline.  Needs s0 a multiple of 32
// (every warp covers one 32-site block); lanes past s1 compute on the range's
// last site and store nothing.  Dynamic shared memory: bulk_smem<LL, ST, NB>.
template <class LL, int ST, int NB> BRI_HD constexpr uint32_t bulk_bar_bytes(int warps) {
    return (uint32_t)((8 * ST * warps + 127) & ~127);
}
template <class LL, int ST, int NB> BRI_HD constexpr uint32_t bulk_smem(int warps) {
    return bulk_bar_bytes<LL, ST, NB>(warps) + (uint32_t)warps * ST * (1 + NB) * (LL::RUN_A + LL::RUN_B);
}
template <class LL, int ST, int NB>
__global__ void k_dslash_bulk(int mode, LL ll, const float2 *__restrict__ in, float2 *__restrict__ out, Geom g,
                              double diag, const int *__restrict__ skip) {
    extern __shared__ __align__(128) unsigned char bulk_sm[];
    const int nblk = (g.s1 - g.s0 + (int)blockDim.x - 1) / (int)blockDim.x;
    const int nr = (int)gridDim.x / nblk;
    const int rhs = (int)blockIdx.x % nr;
    const int lane = (int)threadIdx.x & 31, warp = (int)threadIdx.x >> 5;
    const int wsite = g.s0 + ((int)blockIdx.x / nr) * (int)blockDim.x + warp * 32;  // lane 0's site
    if (wsite >= g.s1) return;  // the whole warp is past the range
    if (skip && skip[rhs]) return;
    const bool active = wsite + lane < g.s1;
    const int site = active ? wsite + lane : g.s1 - 1;
    const size_t off = (size_t)rhs * g.V * 12;
    in += off;
    out += off;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(bulk_sm);
    const uint32_t bars = base + 8u * ST * warp;
    const uint32_t ring = base + bulk_bar_bytes<LL, ST, NB>((int)blockDim.x >> 5) +
                          (uint32_t)warp * ST * (1 + NB) * (LL::RUN_A + LL::RUN_B);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < ST; i++) mbar_init(bars + 8u * i, 1);
        mbar_init_fence();
    }
    __syncwarp();
    int x[4];
    const SiteNb nb = site_nb(g, site, x);
    AccF acc;
#pragma unroll
    for (int i = 0; i < 12; i++) acc.a[i] = acc.ai[i] = make_float2(0.f, 0.f);
    const float rsign = mode == 1 ? -1.f : 1.f;
    if (!f32_hops_bulk<LL, ST, NB>(ll, in, site, wsite >> 5, nb, rsign, g, ring, bars, acc)) {
        if (lane == 0 && g.werr) *(volatile int *)g.werr = 1;
        return;
    }
    if (active) dslash_finish<float2, false>(mode, in, out, site, g, diag, acc);
}

// Launch variant 10 at 32 threads per block with an x extent of 32: one warp
// per block and one x line per warp.  The operands of every copy (the block's
// line, the line holding x - d, the field) then follow from blockIdx and the
// pair index alone, the same in every lane, and every lane's x - d lies in the
// one staged backward run: no shuffles, no fallback loads.  Needs s0 and s1
// multiples of 32.  Dynamic shared memory: 128 + ST x 2 runs.
template <class LL, int ST>
__global__ void __launch_bounds__(32) k_dslash_bulk_line(int mode, LL ll, const float2 *__restrict__ in,
                                                         float2 *__restrict__ out, Geom g, double diag,
                                                         const int *__restrict__ skip) {
    extern __shared__ __align__(128) unsigned char bulk_sm[];
    constexpr uint32_t RUN = LL::RUN_A + LL::RUN_B;
    constexpr uint32_t STAGE = 2 * RUN;
    const int nl = (g.s1 - g.s0) >> 5;
    const int nr = (int)gridDim.x / nl;
    const int rhs = (int)blockIdx.x % nr;
    const int line = (g.s0 >> 5) + (int)blockIdx.x / nr;
    if (skip && skip[rhs]) return;
    const int lane = (int)threadIdx.x;
    const int site = line * 32 + lane;
    const size_t off = (size_t)rhs * g.V * 12;
    in += off;
    out += off;
    const uint32_t bars = (uint32_t)__cvta_generic_to_shared(bulk_sm);
    const uint32_t ring = bars + 128u;
    const int L1 = g.L[1], L2 = g.L[2], L3 = g.L[3];
    const int ly = line % L1, lz = (line / L1) % L2, lt = line / (L1 * L2);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < ST; i++) mbar_init(bars + 8u * i, 1);
        mbar_init_fence();
    }
    __syncwarp();
    int x[4];
    const SiteNb nb = site_nb(g, site, x);
    AccF acc;
#pragma unroll
    for (int i = 0; i < 12; i++) acc.a[i] = acc.ai[i] = make_float2(0.f, 0.f);
    const float rsign = mode == 1 ? -1.f : 1.f;
    const int nh = g.nhop;
    // the runs of pair t into stage sn: field j at this line and at the line of x - d
    auto issue = [&](int t, int sn, uint32_t extra) {
        const HopArg &h = g.hop[t];
        int y = ly - h.dm[1], z = lz - h.dm[2], w = lt - h.dm[3];
        y += y < 0 ? L1 : y >= L1 ? -L1 : 0;
        z += z < 0 ? L2 : z >= L2 ? -L2 : 0;
        w += w < 0 ? L3 : w >= L3 ? -L3 : 0;
        const int bl = y + L1 * (z + L2 * w);
        if (lane == 0) {
            const uint32_t bar = bars + 8u * sn, dst = ring + STAGE * sn;
            mbar_arrive_tx(bar, 2 * RUN + extra);
            ll.bulk_run(h.j, line, dst, bar);
            ll.bulk_run(h.j, bl, dst + RUN, bar);
        }
    };
#pragma unroll
    for (int t = 0; t < ST - 1; t++)
        if (t < nh) issue(t, t, t == 0 && g.stall ? 16u : 0u);
    int s = 0;
    uint32_t par = 0;
    bool ok = true;
#pragma unroll 1
    for (int t = 0; t < nh; t++) {
        if (t + ST - 1 < nh) {
            __syncwarp();  // every lane has read the stage pair t - 1 used
            issue(t + ST - 1, s == 0 ? ST - 1 : s - 1, 0u);
        }
        const HopArg hc = g.hop[t];
        int yf, yb;
        float phf, phb;
        hop_nb(hc.dm, site, nb, yf, phf, yb, phb);
        const uint32_t cur = ring + STAGE * s;
        if (!mbar_wait(bars + 8u * s, par, BULK_WAIT_NS)) {
            int sd = s;
            uint32_t pd = par;
            for (int u = t + 1; u < nh && u < t + ST; u++) {
                if (++sd == ST) { sd = 0; pd ^= 1u; }
                mbar_wait(bars + 8u * sd, pd, BULK_WAIT_NS);
            }
            ok = false;
            break;
        }
        float2 cf[12];
        {
            const M3<float2> W = ll.load_run(cur, lane);
            float2 q[12];
            load_spinor(in + (size_t)yf * 12, q);
            colour_mv<1>(W, q, cf);
        }
        const M3<float2> W = ll.load_run(cur + RUN, yb & 31);
        float2 q[12];
        load_spinor(in + (size_t)yb * 12, q);
        pair_body_s<false>(cf, W, q, hc.lam * phf, phf * phb, hc.rho * rsign * phf, hc, acc);
        if (++s == ST) { s = 0; par ^= 1u; }
    }
    if (!ok) {
        if (lane == 0 && g.werr) *(volatile int *)g.werr = 1;
        return;
    }
    dslash_finish<float2, false>(mode, in, out, site, g, diag, acc);
}

// Launch variant 11: the line kernel with the neighbour spinors staged too.
// The hops of one group, the (up to three) pairs that differ only in d_x, read
// their spinors from the same two x lines, the line shifted by
// +(d_y, d_z, d_t) and the one shifted by -(d_y, d_z, d_t); a ring of two
// spinor stages holds both lines (3,072 bytes each) of the current group while
// the next group's are copied, beside a ring of two link stages.  A lane then
// finds psi(x + d) at slot (x + d_x) mod 32 of the forward line and
// psi(x - d) at slot (x - d_x) mod 32 of the backward one, and its boundary
// phase is the group's (uniform) y, z, t part times its own x part; the lines
// and phases are worked out once per group.  The loop has no global loads and
// no per-lane neighbour arithmetic left.  All copies are issued by one lane
// that elect.sync picks from the converged warp.  Needs an x extent of 32 and
// s0, s1 multiples of 32.  Dynamic shared memory: line2_smem<LL, SB, SP>().
//
// SB = true keeps one buffer per spinor line instead of a two-deep ring: both
// lines of the next group are copied once the group's last pair has consumed
// its spinors.  That gives up about a pair of lead for 6 KB less shared memory
// per warp (14 instead of 10 warps per SM for FP32 full fields).

// Spinor storage of the line kernel, FP32: 12 complex per site, one x line
// (3,072 bytes) copied as one run.  (The FP16-spinor storage is LineSpinH16,
// next to its apply.)  A policy holds the right-hand side's input and output
// and provides the line copies, the per-slot load from a staged line and the
// epilogue.
struct LineSpinF32 {
    static constexpr uint32_t LINE = 32u * 96u;
    static constexpr bool SCALED = false;  // load returns 1
    const float2 *__restrict__ in;
    float2 *__restrict__ out;
    BRI_D LineSpinF32(const void *i, void *o, int rhs, int V)
        : in((const float2 *)i + (size_t)rhs * V * 12), out((float2 *)o + (size_t)rhs * V * 12) {}
    BRI_D void issue1(int ln, uint32_t dst, uint32_t bar) const {
        bulk_elect1(bar, LINE, dst, in + (size_t)ln * 384, LINE);
    }
    BRI_D void issue2(int l0, int l1, uint32_t dst, uint32_t bar) const {
        bulk_elect2(bar, 2 * LINE, dst, in + (size_t)l0 * 384, LINE, dst + LINE, in + (size_t)l1 * 384, LINE);
    }
    // the spinor at a slot of a staged line, as q x (returned scale)
    BRI_D float load(uint32_t ln, uint32_t slot, float2 q[12]) const {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const float4 v = lds4(ln + 96u * slot + 16u * k);
            q[2 * k] = make_float2(v.x, v.y);
            q[2 * k + 1] = make_float2(v.z, v.w);
        }
        return 1.f;
    }
    BRI_D void finish(int mode, int site, const Geom &g, double diag, const AccF &acc) const {
        dslash_finish<float2, false>(mode, in, out, site, g, diag, acc);
    }
};

template <class LL, bool SB, class SP = LineSpinF32> BRI_HD constexpr unsigned line2_smem() {
    return 128u + 4u * (LL::RUN_A + LL::RUN_B) + (SB ? 2u : 4u) * SP::LINE;
}

struct LineShift {
    int fl, bl;    // the lines shifted by +(d_y, d_z, d_t) and by -(d_y, d_z, d_t)
    float uf, ub;  // boundary phases of their y, z, t wraps
};

template <class LL, bool SB, class SP>
BRI_D void dslash_bulk_line2(int mode, const LL &ll, const void *__restrict__ in, void *__restrict__ out,
                             const Geom &g, double diag, const int *__restrict__ skip) {
    extern __shared__ __align__(128) unsigned char bulk_sm[];
    constexpr uint32_t RUN = LL::RUN_A + LL::RUN_B;
    constexpr uint32_t LSTAGE = 2 * RUN;
    constexpr uint32_t SLINE = SP::LINE;  // one staged x line of spinors
    constexpr uint32_t SSTAGE = 2 * SLINE;
    const int nl = (g.s1 - g.s0) >> 5;
    const int nr = (int)gridDim.x / nl;
    const int rhs = (int)blockIdx.x % nr;
    const int line = (g.s0 >> 5) + (int)blockIdx.x / nr;
    if (skip && skip[rhs]) return;
    const int lane = (int)threadIdx.x;
    const int site = line * 32 + lane;
    const SP io(in, out, rhs, g.V);
    // barriers: link stages 0, 1, spinor stages 0, 1 (SB: forward line, backward line)
    const uint32_t lbars = (uint32_t)__cvta_generic_to_shared(bulk_sm);
    const uint32_t sbars = lbars + 16u;
    const uint32_t lring = lbars + 128u;
    const uint32_t sring = lring + 2 * LSTAGE;
    const int L1 = g.L[1], L2 = g.L[2], L3 = g.L[3];
    const int ly = line % L1, lz = (line / L1) % L2, lt = line / (L1 * L2);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 4; i++) mbar_init(lbars + 8u * i, 1);
        mbar_init_fence();
    }
    __syncwarp();
    AccF acc;
#pragma unroll
    for (int i = 0; i < 12; i++) acc.a[i] = acc.ai[i] = make_float2(0.f, 0.f);
    const float rsign = mode == 1 ? -1.f : 1.f;
    const float e31 = lane == 31 ? (float)g.bc[0] : 1.f, e0 = lane == 0 ? (float)g.bc[0] : 1.f;
    const int nh = g.nhop;
    auto wrap = [](int c, int n, float &ph, float b) {
        if (c < 0) { ph *= b; return c + n; }
        if (c >= n) { ph *= b; return c - n; }
        return c;
    };
    auto shifts = [&](int t) {
        const HopArg &h = g.hop[t];
        LineShift r;
        r.uf = r.ub = 1.f;
        const float b1 = (float)g.bc[1], b2 = (float)g.bc[2], b3 = (float)g.bc[3];
        r.fl = wrap(ly + h.dm[1], L1, r.uf, b1) +
               L1 * (wrap(lz + h.dm[2], L2, r.uf, b2) + L2 * wrap(lt + h.dm[3], L3, r.uf, b3));
        r.bl = wrap(ly - h.dm[1], L1, r.ub, b1) +
               L1 * (wrap(lz - h.dm[2], L2, r.ub, b2) + L2 * wrap(lt - h.dm[3], L3, r.ub, b3));
        return r;
    };
    // the copies are issued by one elected lane of the converged warp
    auto issue_links = [&](int t, int bl, int sn, uint32_t extra) {
        ll.bulk_pair(g.hop[t].j, line, bl, lring + LSTAGE * sn, lbars + 8u * sn, extra);
    };
    auto issue_spinors = [&](const LineShift &ls, int sn) {
        io.issue2(ls.fl, ls.bl, sring + SSTAGE * sn, sbars + 8u * sn);
    };
    // SB: one line into buffer k (0 forward, 1 backward)
    auto issue_line = [&](int ln, int k) { io.issue1(ln, sring + SLINE * k, sbars + 8u * k); };
    if (nh > 0) {
        LineShift cur = shifts(0), nxt = cur;
        int gend = g.hop[0].ge;  // first pair of the next group
        if constexpr (SB) {
            issue_line(cur.fl, 0);
            issue_line(cur.bl, 1);
            if (gend < nh) nxt = shifts(gend);
        } else {
            issue_spinors(cur, 0);
            if (gend < nh) {
                nxt = shifts(gend);
                issue_spinors(nxt, 1);
            }
        }
        issue_links(0, cur.bl, 0, g.stall ? 16u : 0u);
        int gi = 0;  // group of pair t
        int t = 0;
        bool ok = true;
        // pair t in link stage S (= t mod 2)
        auto step = [&](int t, auto S) -> bool {
            constexpr int s = decltype(S)::value;
            if (t == gend) {
                gi++;
                cur = nxt;
                gend = g.hop[t].ge;
                if (gend < nh) {
                    nxt = shifts(gend);
                    if constexpr (!SB) {
                        // the stage of group gi + 1 is the one group gi - 1 used: the
                        // proxy fence orders the lanes' reads of it (generic proxy)
                        // before the bulk copy into it (async proxy)
                        fence_async_smem();
                        __syncwarp();
                        issue_spinors(nxt, (gi + 1) & 1);
                    }
                }
            }
            if (t + 1 < nh) {
                // every lane has read the link stage pair t - 1 used; those reads
                // precede the group-boundary branch above, so they are complete
                // here without a proxy fence (one measured 1.2% slower)
                __syncwarp();
                issue_links(t + 1, t + 1 < gend ? cur.bl : nxt.bl, s ^ 1, 0u);
            }
            if (!mbar_wait(lbars + 8u * s, (uint32_t)(t >> 1) & 1u, BULK_WAIT_NS)) return false;
            // (waiting on the spinor stage at every pair, not just the group's
            // first, measured faster: the conditional form takes 13 more registers;
            // SB: both lines are waited for here, before any load of the pair, so
            // that the pair's loads and arithmetic form one block without a wait
            // or branch in between: 0.3% faster alone, 5% with pair_body_s<true>)
            uint32_t sp;  // the group's forward line; its backward line follows at + SLINE
            if constexpr (SB) {
                if (!mbar_wait(sbars, (uint32_t)gi & 1u, BULK_WAIT_NS)) return false;
                if (!mbar_wait(sbars + 8u, (uint32_t)gi & 1u, BULK_WAIT_NS)) return false;
                sp = sring;
            } else {
                if (!mbar_wait(sbars + 8u * (uint32_t)(gi & 1), (uint32_t)(gi >> 1) & 1u, BULK_WAIT_NS))
                    return false;
                sp = sring + SSTAGE * (uint32_t)(gi & 1);
            }
            const HopArg hc = g.hop[t];
            const int dx = hc.dm[0];
            const float phf = cur.uf * (dx > 0 ? e31 : dx < 0 ? e0 : 1.f);
            const float phb = cur.ub * (dx > 0 ? e0 : dx < 0 ? e31 : 1.f);
            const uint32_t lk = lring + LSTAGE * (uint32_t)s;
            const uint32_t sf = (uint32_t)((lane + dx) & 31), sb = (uint32_t)((lane - dx) & 31);
            // SB: the group's last pair releases both line buffers to the next group
            const bool last = SB && t + 1 == gend && gend < nh;
            float2 cf[12];
            {
                const M3<float2> W = ll.load_run(lk, lane);
                float2 q[12];
                const float scf = io.load(sp, sf, q);
                colour_mv<1>(W, q, cf);
                if constexpr (SP::SCALED) {
#pragma unroll
                    for (int i = 0; i < 12; i++) cf[i] = __fmul2_rn(cf[i], f2(scf));
                }
            }
            const M3<float2> W = ll.load_run(lk + RUN, (int)sb);
            float2 q[12];
            // a scaled storage's backward scale goes into the phase factor
            const float scb = io.load(sp + SLINE, sb, q);
            pair_body_s<true>(cf, W, q, hc.lam * phf, SP::SCALED ? phf * phb * scb : phf * phb, hc.rho * rsign * phf,
                              hc, acc);
            if (last) {
                // every lane has read its spinors: the proxy fence orders those
                // reads (generic proxy) before the copies into the same buffers
                // (async proxy); without it a copy issued right after the reads
                // can overwrite a line before it is read
                fence_async_smem();
                __syncwarp();
                issue_line(nxt.fl, 0);
                issue_line(nxt.bl, 1);
            }
            return true;
        };
        // two pairs per trip, so that the link stage of each is a constant
#pragma unroll 1
        for (; t < nh; t += 2) {
            if (!step(t, std::integral_constant<int, 0>{})) { ok = false; break; }
            if (t + 1 < nh && !step(t + 1, std::integral_constant<int, 1>{})) { ok = false; t++; break; }
        }
        if (!ok) {
            // wait (bounded) for the stages still in flight: the links of pairs
            // t and t + 1 and the spinors of groups gi and gi + 1
            for (int u = t; u < nh && u < t + 2; u++)
                mbar_wait(lbars + 8u * (uint32_t)(u & 1), (uint32_t)(u >> 1) & 1u, BULK_WAIT_NS);
            if constexpr (SB) {
                // group gi's lines, then group gi + 1's if they were issued (if not,
                // the wait on that unarmed phase runs out after its limit)
                for (uint32_t k = 0; k < 2; k++) {
                    mbar_wait(sbars + 8u * k, (uint32_t)gi & 1u, BULK_WAIT_NS);
                    if (gend < nh) mbar_wait(sbars + 8u * k, (uint32_t)(gi + 1) & 1u, BULK_WAIT_NS);
                }
            } else {
                mbar_wait(sbars + 8u * (uint32_t)(gi & 1), (uint32_t)(gi >> 1) & 1u, BULK_WAIT_NS);
                if (gend < nh)
                    mbar_wait(sbars + 8u * (uint32_t)((gi + 1) & 1), (uint32_t)((gi + 1) >> 1) & 1u, BULK_WAIT_NS);
            }
            if (lane == 0 && g.werr) *(volatile int *)g.werr = 1;
            return;
        }
    }
    io.finish(mode, site, g, diag, acc);
}
// FP32 full fields: the stages allow at most 14 blocks per SM (126 registers
// without a cap; the two-deep spinor ring: 150, 3 warps per scheduler)
template <class LL, bool SB, class SP = LineSpinF32>
__global__ void __launch_bounds__(32) k_dslash_bulk_line2(int mode, LL ll, const void *__restrict__ in,
                                                          void *__restrict__ out, Geom g, double diag,
                                                          const int *__restrict__ skip) {
    dslash_bulk_line2<LL, SB, SP>(mode, ll, in, out, g, diag, skip);
}
// the other formats: held to 128 registers (no spills), 4 warps per scheduler
// (16 per SM) where their smaller stages fit; 2-8% faster than uncapped
template <class LL, bool SB, class SP = LineSpinF32>
__global__ void __maxnreg__(128) k_dslash_bulk_line2_r128(int mode, LL ll, const void *__restrict__ in,
                                                          void *__restrict__ out, Geom g, double diag,
                                                          const int *__restrict__ skip) {
    dslash_bulk_line2<LL, SB, SP>(mode, ll, in, out, g, diag, skip);
}

// ---- shared-memory tiled variant (FP32 spinors) ------------------------------
// A CTA owns a TX x TY x TZ x TT tile of sites (one thread per site).  The
// tile's spinors plus a one-site halo in every direction are copied to shared
// memory with coalesced 16-byte asynchronous copies (periodic wrap handled on
// the way in), so each of the 81 neighbour reads is a shared-memory load whose
// address offset is a compile-time constant.  Sites are padded to 112 bytes (7
// float4) so a quarter-warp of LDS.128 hits eight distinct bank groups.  The
// result goes back through shared memory for coalesced stores.
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2, HT = TT + 2;
constexpr int HSITES = HX * HY * HZ * HT;
constexpr int SSTR = 7;  // float4 slots per site in shared memory
constexpr int TILE_THREADS = TX * TY * TZ * TT;
constexpr int TILE_SMEM = HSITES * SSTR * 16;

BRI_D void lds_spinor(uint32_t addr, float2 o[12]) {
#pragma unroll
    for (int i = 0; i < 6; i++) {
        float4 v;
        asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
            : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
            : "r"(addr + 16 * i));
        o[2 * i] = make_float2(v.x, v.y);
        o[2 * i + 1] = make_float2(v.z, v.w);
    }
}

BRI_HD constexpr int halo_delta(int K) {
    return off_comp(K, 0) + HX * (off_comp(K, 1) + HY * (off_comp(K, 2) + HZ * off_comp(K, 3)));
}

template <class LL>
__global__ void __launch_bounds__(TILE_THREADS) k_dslash_tiled(int mode, LL ll, const float2 *__restrict__ in,
                                                               float2 *__restrict__ out, Geom g, double diag,
                                                               const int *__restrict__ skip) {
    extern __shared__ float4 smem[];
    if (skip && skip[blockIdx.y]) return;
    const size_t off = (size_t)blockIdx.y * g.V * 12;
    in += off;
    out += off;
    // tile origin
    const int ntx = g.L[0] / TX, nty = g.L[1] / TY, ntz = g.L[2] / TZ;
    int b = blockIdx.x;
    const int x0 = (b % ntx) * TX; b /= ntx;
    const int y0 = (b % nty) * TY; b /= nty;
    const int z0 = (b % ntz) * TZ; b /= ntz;
    const int t0 = b * TT;
    // stage the halo tile: HSITES sites x 6 chunks of 16 bytes
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    for (int c = threadIdx.x; c < HSITES * 6; c += TILE_THREADS) {
        const int h = c / 6, q = c - 6 * h;
        int r = h;
        int gx = x0 - 1 + r % HX; r /= HX;
        int gy = y0 - 1 + r % HY; r /= HY;
        int gz = z0 - 1 + r % HZ;
        int gt = t0 - 1 + r / HZ;
        gx += gx < 0 ? g.L[0] : (gx >= g.L[0] ? -g.L[0] : 0);
        gy += gy < 0 ? g.L[1] : (gy >= g.L[1] ? -g.L[1] : 0);
        gz += gz < 0 ? g.L[2] : (gz >= g.L[2] ? -g.L[2] : 0);
        gt += gt < 0 ? g.L[3] : (gt >= g.L[3] ? -g.L[3] : 0);
        const size_t gs = (size_t)gx + (size_t)g.L[0] * (gy + (size_t)g.L[1] * (gz + (size_t)g.L[2] * gt));
        const float4 *src = reinterpret_cast<const float4 *>(in + gs * 12) + q;
        const uint32_t dst = sbase + (uint32_t)((h * SSTR + q) * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = (tid / TX) % TY, lz = (tid / (TX * TY)) % TZ, lt = tid / (TX * TY * TZ);
    const int site = (x0 + lx) + g.L[0] * ((y0 + ly) + g.L[1] * ((z0 + lz) + g.L[2] * (t0 + lt)));
    const int hc = (lx + 1) + HX * ((ly + 1) + HY * ((lz + 1) + HZ * (lt + 1)));
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
        const HopArg h = g.hop[t];
        const int j = h.j;
        int yf, yb;
        float phf, phb;
        hop_nb(h.dm, site, nb, yf, phf, yb, phb);
        {
            M3<float2> W = ll.load(j, site);
            float2 q[12];
            lds_spinor(sbase + (uint32_t)((hc + h.hd) * SSTR * 16), q);
            hop_body<1>(W, q, h.lam * phf, h.rho * rsign * phf, h.dm, acc);
        }
        {
            M3<float2> W = ll.load(j, yb);
            float2 q[12];
            lds_spinor(sbase + (uint32_t)((hc - h.hd) * SSTR * 16), q);
            hop_body<-1>(W, q, h.lam * phb, h.rho * rsign * phb, h.dm, acc);
        }
    }
    float2 p[12];
    lds_spinor(sbase + (uint32_t)(hc * SSTR * 16), p);
    const float dg = (float)diag;
    float2 o[12];
#pragma unroll
    for (int i = 0; i < 12; i++) {
        float2 v;
        v.x = dg * p[i].x + acc.a[i].x - acc.ai[i].y;
        v.y = dg * p[i].y + acc.a[i].y + acc.ai[i].x;
        if (mode == 2 && i >= 6) { v.x = -v.x; v.y = -v.y; }
        o[i] = v;
    }
    // write the tile through shared memory (tile-local order, 7 slots per site)
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 6; i++)
        smem[tid * SSTR + i] = make_float4(o[2 * i].x, o[2 * i].y, o[2 * i + 1].x, o[2 * i + 1].y);
    __syncthreads();
    for (int c = threadIdx.x; c < TILE_THREADS * 6; c += TILE_THREADS) {
        const int h = c / 6, q = c - 6 * h;
        const int hx = h % TX, hy = (h / TX) % TY, hz = (h / (TX * TY)) % TZ, ht = h / (TX * TY * TZ);
        const size_t gs = (size_t)(x0 + hx) + (size_t)g.L[0] * ((y0 + hy) + (size_t)g.L[1] * ((z0 + hz) + (size_t)g.L[2] * (t0 + ht)));
        reinterpret_cast<float4 *>(out + gs * 12)[q] = smem[h * SSTR + q];
    }
}

template <class LL>
void dslash_launch(int mode, const LL &ll, const void *in, void *out, int nrhs, const Geom &g, double diag,
                   const int *skip, int threads, cudaStream_t s) {
    using T = typename LL::T;
    {
        // grid.x holds site blocks x RHS: split the RHS so that it stays below 2^31
        const size_t nbmax = (size_t)(g.s1 - g.s0 + 31) / 32;  // blocks at the smallest shape
        const int rmax = (int)(0x7fffffffULL / nbmax < 65535ULL ? 0x7fffffffULL / nbmax : 65535ULL);
        if (nrhs > rmax) {
            const size_t field = sizeof(T) * 12 * (size_t)g.V;
            for (int r0 = 0; r0 < nrhs; r0 += rmax) {
                const int nr = nrhs - r0 < rmax ? nrhs - r0 : rmax;
                dslash_launch(mode, ll, (const char *)in + r0 * field, (char *)out + r0 * field, nr, g, diag,
                              skip ? skip + r0 : nullptr, threads, s);
            }
            return;
        }
    }
    if (g.clov64) {  // clover term on: the plain kernel (link prefetch variant for FP32) with the term
        constexpr int VC = sizeof(T) == 8 ? 5 : 0;
        static int max_c = 0;
        if (max_c == 0) {
            cudaFuncAttributes attr;
            max_c = cudaFuncGetAttributes(&attr, k_dslash<LL, VC, true>) == cudaSuccess ? attr.maxThreadsPerBlock : 128;
        }
        int t = threads & 2047;
        if (t == 0) t = 128;
        if (t > max_c) t = max_c & ~31;
        const dim3 grid((unsigned)((g.s1 - g.s0 + t - 1) / t) * (unsigned)nrhs);
        k_dslash<LL, VC, true><<<grid, t, 0, s>>>(mode, ll, (const T *)in, (T *)out, g, diag, skip);
        return;
    }
    if constexpr (sizeof(T) == 8) {
        if ((threads & 2047) == 0 && (threads >> 11) == 0 && tiled_ok(g) && g.s0 == 0 && g.s1 == g.V) {
            static bool attr_set = false;
            if (!attr_set) {
                cudaFuncSetAttribute(k_dslash_tiled<LL>, cudaFuncAttributeMaxDynamicSharedMemorySize, TILE_SMEM);
                attr_set = true;
            }
            dim3 grid((unsigned)(g.V / TILE_THREADS), (unsigned)nrhs);
            k_dslash_tiled<<<grid, TILE_THREADS, TILE_SMEM, s>>>(mode, ll, (const float2 *)in, (float2 *)out, g,
                                                                   diag, skip);
            return;
        }
    }
    // launch shape: threads per block in the low 11 bits, kernel variant above
    const int variant = threads >> 11;
    threads &= 2047;
    if (threads == 0) threads = 128;
    static int max_threads[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // per-kernel limit from its register use
    dim3 grid;
    if constexpr (sizeof(T) == 8) {
        if (variant == 11 && g.L[0] == 32 && g.s0 % 32 == 0 && g.s1 % 32 == 0) {
            // line kernel with staged links and spinors, one warp per block; low
            // bits 64: one buffer per spinor line
            grid = dim3((unsigned)((g.s1 - g.s0) / 32) * (unsigned)nrhs);
            constexpr bool big = LL::RUN_A + LL::RUN_B > 2048;  // FP32 full fields
            static bool l2_attr = false;
            if (!l2_attr) {
                // dynamic shared memory above 48 KB is not needed, but the carveout is:
                // all of the unified L1 / shared memory as shared memory holds the
                // stages of 12-16 blocks per SM, and the loop reads nothing through L1
                if constexpr (big) {
                    cudaFuncSetAttribute(k_dslash_bulk_line2<LL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)line2_smem<LL, false>());
                    cudaFuncSetAttribute(k_dslash_bulk_line2<LL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)line2_smem<LL, true>());
                    cudaFuncSetAttribute(k_dslash_bulk_line2<LL, false>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
                    cudaFuncSetAttribute(k_dslash_bulk_line2<LL, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
                } else {
                    cudaFuncSetAttribute(k_dslash_bulk_line2_r128<LL, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)line2_smem<LL, false>());
                    cudaFuncSetAttribute(k_dslash_bulk_line2_r128<LL, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)line2_smem<LL, true>());
                    cudaFuncSetAttribute(k_dslash_bulk_line2_r128<LL, false>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
                    cudaFuncSetAttribute(k_dslash_bulk_line2_r128<LL, true>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
                }
                l2_attr = true;
            }
            const bool sb = threads == 64;
            if constexpr (big) {
                if (sb)
                    k_dslash_bulk_line2<LL, true><<<grid, 32, line2_smem<LL, true>(), s>>>(mode, ll, in, out, g, diag,
                                                                                          skip);
                else
                    k_dslash_bulk_line2<LL, false><<<grid, 32, line2_smem<LL, false>(), s>>>(mode, ll, in, out, g,
                                                                                            diag, skip);
            } else {
                if (sb)
                    k_dslash_bulk_line2_r128<LL, true><<<grid, 32, line2_smem<LL, true>(), s>>>(mode, ll, in, out, g,
                                                                                               diag, skip);
                else
                    k_dslash_bulk_line2_r128<LL, false><<<grid, 32, line2_smem<LL, false>(), s>>>(mode, ll, in, out,
                                                                                                 g, diag, skip);
            }
            return;
        }
        if (variant >= 10 && g.s0 % 32 == 0) {
            // bulk-copy link pipeline: 3 stages of 2 runs when a warp is one x
            // line (x extent 32), else 2 stages of 3 runs
            const bool line = g.L[0] == 32;
            static bool attr_set = false;
            if (max_threads[10] == 0) {
                cudaFuncAttributes a1, a2;
                const bool ok = cudaFuncGetAttributes(&a1, k_dslash_bulk<LL, 3, 1>) == cudaSuccess &&
                                cudaFuncGetAttributes(&a2, k_dslash_bulk<LL, 2, 2>) == cudaSuccess;
                max_threads[10] = ok ? (a1.maxThreadsPerBlock < a2.maxThreadsPerBlock ? a1.maxThreadsPerBlock
                                                                                      : a2.maxThreadsPerBlock)
                                     : 128;
                if (max_threads[10] > 256) max_threads[10] = 256;
            }
            if (!attr_set) {
                cudaFuncSetAttribute(k_dslash_bulk<LL, 3, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bulk_smem<LL, 3, 1>(8));
                cudaFuncSetAttribute(k_dslash_bulk<LL, 2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bulk_smem<LL, 2, 2>(8));
                attr_set = true;
            }
            if (line && threads == 32 && g.s1 % 32 == 0) {
                // one warp per block, one x line per warp
                static bool line_attr = false;
                if (!line_attr) {
                    cudaFuncSetAttribute(k_dslash_bulk_line<LL, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         128 + 3 * 2 * (int)(LL::RUN_A + LL::RUN_B));
                    line_attr = true;
                }
                grid = dim3((unsigned)((g.s1 - g.s0) / 32) * (unsigned)nrhs);
                k_dslash_bulk_line<LL, 3><<<grid, 32, 128 + 3 * 2 * (LL::RUN_A + LL::RUN_B), s>>>(
                    mode, ll, (const T *)in, (T *)out, g, diag, skip);
                return;
            }
            if (threads > max_threads[10]) threads = max_threads[10] & ~31;
            grid = dim3((unsigned)((g.s1 - g.s0 + threads - 1) / threads) * (unsigned)nrhs);
            const int w = threads >> 5;
            if (line)
                k_dslash_bulk<LL, 3, 1><<<grid, threads, bulk_smem<LL, 3, 1>(w), s>>>(mode, ll, (const T *)in, (T *)out,
                                                                                     g, diag, skip);
            else
                k_dslash_bulk<LL, 2, 2><<<grid, threads, bulk_smem<LL, 2, 2>(w), s>>>(mode, ll, (const T *)in, (T *)out,
                                                                                     g, diag, skip);
            return;
        }
        const int v = (variant == 1 || variant == 2 || (variant >= 4 && variant <= 9)) ? variant : variant >= 10 ? 5 : 0;
        if (max_threads[v] == 0) {
            cudaFuncAttributes attr;
            cudaError_t e = v == 1 ? cudaFuncGetAttributes(&attr, k_dslash<LL, 1>)
                          : v == 2 ? cudaFuncGetAttributes(&attr, k_dslash<LL, 2>)
                          : v == 4 ? cudaFuncGetAttributes(&attr, k_dslash<LL, 4>)
                          : v == 5 ? cudaFuncGetAttributes(&attr, k_dslash<LL, 5>)
                          : v == 6 ? cudaFuncGetAttributes(&attr, k_dslash_r128<LL>)
                          : v == 7 ? cudaFuncGetAttributes(&attr, k_dslash<LL, 7>)
                          : v == 9 ? cudaFuncGetAttributes(&attr, k_dslash<LL, 9>)
                                   : cudaFuncGetAttributes(&attr, k_dslash<LL, 0>);
            max_threads[v] = e == cudaSuccess ? attr.maxThreadsPerBlock : 128;
            if (v == 2) {
                // per-thread link slots: 2 stages x 2 fields; allow up to 256 threads
                cudaFuncSetAttribute(k_dslash<LL, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     256 * 4 * LL::SLOTS * 16);
                if (max_threads[v] > 256) max_threads[v] = 256;
            }
        }
        if (threads > max_threads[v]) threads = max_threads[v] & ~31;
        grid = dim3((unsigned)((g.s1 - g.s0 + threads - 1) / threads) * (unsigned)nrhs);
        if (v == 1) k_dslash<LL, 1><<<grid, threads, 0, s>>>(mode, ll, (const T *)in, (T *)out, g, diag, skip);
        else if (v == 4) k_dslash<LL, 4><<<grid, threads, 0, s>>>(mode, ll, (const T *)in, (T *)out, g, diag, skip);
        else if (v == 5) k_dslash<LL, 5><<<grid, threads, 0, s>>>(mode, ll, (const T *)in, (T *)out, g, diag, skip);
        else if (v == 6) k_dslash_r128<LL><<<grid, threads, 0, s>>>(mode, ll, (const T *)in, (T *)out, g, diag, skip);
        else if (v == 7) k_dslash<LL, 7><<<grid, threads, 0, s>>>(mode, ll, (const T *)in, (T *)out, g, diag, skip);
        else if (v == 9) k_dslash<LL, 9><<<grid, threads, 0, s>>>(mode, ll, (const T *)in, (T *)out, g, diag, skip);
        else if (v == 2)
            k_dslash<LL, 2><<<grid, threads, threads * 4 * LL::SLOTS * 16, s>>>(mode, ll, (const T *)in, (T *)out, g,
                                                                                 diag, skip);
        else k_dslash<LL, 0><<<grid, threads, 0, s>>>(mode, ll, (const T *)in, (T *)out, g, diag, skip);
    } else {
        (void)variant;
        if (max_threads[0] == 0) {
            cudaFuncAttributes attr;
            max_threads[0] =
                cudaFuncGetAttributes(&attr, k_dslash<LL, 0>) == cudaSuccess ? attr.maxThreadsPerBlock : 128;
        }
        if (threads > max_threads[0]) threads = max_threads[0] & ~31;
        grid = dim3((unsigned)((g.s1 - g.s0 + threads - 1) / threads) * (unsigned)nrhs);
        k_dslash<LL, 0><<<grid, threads, 0, s>>>(mode, ll, (const T *)in, (T *)out, g, diag, skip);
    }
}

}  // namespace bri

#define BRI_INSTANTIATE_DSLASH(LL) \
    template void bri::dslash_launch<LL>(int, const LL &, const void *, void *, int, const bri::Geom &, double, const int *, int, cudaStream_t);
