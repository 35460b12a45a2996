// Shared device-side definitions of the Brillouin operator library (sm_103a).
//
// The operator is the rho/lambda class form of Sec. 8 with the der_iso /
// lap_bri weights of Tab. rholambda; hops are indexed by their offset
// d in {-1,0,1}^4.  The 40 "canonical" offsets are those whose last non-zero
// component is +1; with k(d) = 40 + sum_mu d_mu 3^mu they are exactly
// k = 41..80, so canonical field j has d = base-3 digits of (j + 41) minus 1.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define BRI_HD __host__ __device__ __forceinline__
#define BRI_D __device__ __forceinline__

namespace bri {

constexpr int NCANON = 40;  // stored hopping fields per site
constexpr int NOFF = 81;    // offsets in the 3^4 hypercube, centre = 40

// ---- offsets --------------------------------------------------------------
BRI_HD constexpr int pow3(int m) { return m == 0 ? 1 : 3 * pow3(m - 1); }
// component mu of the offset with hypercube index k (0..80)
BRI_HD constexpr int off_comp(int k, int mu) { return (k / pow3(mu)) % 3 - 1; }
BRI_HD constexpr int off_class(int k) {
    return (off_comp(k, 0) != 0) + (off_comp(k, 1) != 0) + (off_comp(k, 2) != 0) + (off_comp(k, 3) != 0);
}
BRI_HD constexpr int canon_k(int j) { return j + 41; }

// ---- weights (Sec. 8 / Tab. rholambda), written as closed forms -------------
// lambda_0 = 240/128 and lambda_n = -2^(4-n)/128: the lap_bri stencil of App. C
// is 2^(4-n)/64 off-centre and -240/64 at the centre, and D carries -1/2 of it.
// rho_n = 4^(4-n)/432: the der_iso stencil of App. C.
BRI_HD constexpr double lambda_w(int n) {
    return n == 0 ? 240.0 / 128.0 : -double(1 << (4 - n)) / 128.0;
}
BRI_HD constexpr double rho_w(int n) { return n == 0 ? 0.0 : double(1 << (2 * (4 - n))) / 432.0; }

// ---- gamma matrices: hermitian chiral (DeGrand-Rossi) basis -----------------
// Every row of gamma_mu holds one non-zero entry: (gamma_mu)_{s, gcol(mu,s)} =
// phase, phase in {+1, -1, +i, -i}.  gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4
// = diag(1, 1, -1, -1).
BRI_HD constexpr int gcol(int mu, int s) {
    return mu == 0 ? 3 - s : mu == 1 ? 3 - s : mu == 2 ? (s + 2) % 4 : (s + 2) % 4;
}
// real and imaginary part of the entry
BRI_HD constexpr int gre(int mu, int s) {
    return mu == 1 ? (s == 0 || s == 3 ? -1 : 1) : mu == 3 ? 1 : 0;
}
BRI_HD constexpr int gim(int mu, int s) {
    return mu == 0 ? (s < 2 ? 1 : -1) : mu == 2 ? ((s == 0 || s == 3) ? 1 : -1) : 0;
}

// ---- complex helpers --------------------------------------------------------
template <typename R> struct C2;
template <> struct C2<double> { using T = double2; };
template <> struct C2<float> { using T = float2; };

template <typename T> BRI_HD T mk(double re, double im);
template <> BRI_HD double2 mk<double2>(double re, double im) { return make_double2(re, im); }
template <> BRI_HD float2 mk<float2>(double re, double im) { return make_float2((float)re, (float)im); }

template <typename T> BRI_HD T cadd(T a, T b) { T r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename T> BRI_HD T csub(T a, T b) { T r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename T> BRI_HD T cmul(T a, T b) {
    T r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename T> BRI_HD T cconj(T a) { T r; r.x = a.x; r.y = -a.y; return r; }
// conj(a) * b
template <typename T> BRI_HD T cmulc(T a, T b) {
    T r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.x * b.y - a.y * b.x;
    return r;
}
template <typename T, typename S> BRI_HD T cscale(T a, S s) { T r; r.x = a.x * s; r.y = a.y * s; return r; }
template <typename T> BRI_HD double cnorm2(T a) { return (double)a.x * a.x + (double)a.y * a.y; }

// 3x3 complex matrix, row-major
template <typename T> struct M3 {
    T e[9];
};
// c = acc + a b (ACC) or a b, each entry one multiply and five (or six) FMAs
// per real component: complex products followed by complex adds cost a third
// more on the FP64 pipe
template <bool ACC, typename T>
BRI_HD M3<T> m3_mul_acc(const M3<T> &acc, const M3<T> &a, const M3<T> &b) {
    M3<T> c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const T a0 = a.e[3 * i], a1 = a.e[3 * i + 1], a2 = a.e[3 * i + 2];
            const T b0 = b.e[j], b1 = b.e[3 + j], b2 = b.e[6 + j];
            auto re = ACC ? fma(a0.x, b0.x, acc.e[3 * i + j].x) : a0.x * b0.x;
            auto im = ACC ? fma(a0.x, b0.y, acc.e[3 * i + j].y) : a0.x * b0.y;
            re = fma(-a0.y, b0.y, re);
            im = fma(a0.y, b0.x, im);
            re = fma(a1.x, b1.x, re);
            im = fma(a1.x, b1.y, im);
            re = fma(-a1.y, b1.y, re);
            im = fma(a1.y, b1.x, im);
            re = fma(a2.x, b2.x, re);
            im = fma(a2.x, b2.y, im);
            re = fma(-a2.y, b2.y, re);
            im = fma(a2.y, b2.x, im);
            c.e[3 * i + j].x = re;
            c.e[3 * i + j].y = im;
        }
    return c;
}
template <typename T> BRI_HD M3<T> m3_mul(const M3<T> &a, const M3<T> &b) { return m3_mul_acc<false>(a, a, b); }
// acc + a b
template <typename T> BRI_HD M3<T> m3_mad(const M3<T> &acc, const M3<T> &a, const M3<T> &b) {
    return m3_mul_acc<true>(acc, a, b);
}
template <typename T> BRI_HD M3<T> m3_dag(const M3<T> &a) {
    M3<T> c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) c.e[3 * i + j] = cconj(a.e[3 * j + i]);
    return c;
}
template <typename T> BRI_HD M3<T> m3_add(const M3<T> &a, const M3<T> &b) {
    M3<T> c;
#pragma unroll
    for (int i = 0; i < 9; i++) c.e[i] = cadd(a.e[i], b.e[i]);
    return c;
}
template <typename T> BRI_HD M3<T> m3_zero() {
    M3<T> c;
#pragma unroll
    for (int i = 0; i < 9; i++) c.e[i] = mk<T>(0, 0);
    return c;
}
template <typename T> BRI_HD M3<T> m3_eye() {
    M3<T> c = m3_zero<T>();
    c.e[0] = c.e[4] = c.e[8] = mk<T>(1, 0);
    return c;
}

// ---- geometry ---------------------------------------------------------------
// Tile shape of the shared-memory stencil kernel (sites per CTA along x, y, z, t).
constexpr int TX = 8, TY = 4, TZ = 2, TT = 2;

// One (d, -d) hop pair of the stencil: offset d, stored field index j, the
// class weights of |d|_1 and the offset of d within the shared-memory halo tile.
struct HopArg {
    int dm[4];
    // j and ge as 16-bit values keep the struct at 48 bytes, a multiple of 16:
    // the kernels index g.hop[] by a run-time hop number, and at 52 bytes the
    // FP32 stencil loop took two more registers and ran 17% slower
    short j;
    short ge;  // first hop index after this hop's run of equal (d_y, d_z, d_t)
    int hd;
    float lam, rho;
    float fd[4];  // d_mu as floats (no conversions in the hop loop)
};
static_assert(sizeof(HopArg) == 48, "HopArg: keep a multiple of 16 bytes");

// Lattice geometry and the class weights of the operator (lambda_0..4,
// rho_0..4 with rho_0 unused; by default the der_iso / lap_bri weights above).
// hop[0..nhop) lists the hop pairs whose class has a nonzero weight, in
// canonical order; the FP32/FP16 stencils loop over it (kernel parameter
// space, read with a warp-uniform index).
struct Geom {
    int L[4];
    int bc[4];
    int V;
    float lam[5], rho[5];
    double lamd[5], rhod[5];
    int nhop;
    HopArg hop[NCANON];
    // clover term -(c_SW/2) sum_{mu<nu} sigma_{mu nu} F_{mu nu} (Eq. def_pref) as two
    // hermitian 6x6 chiral blocks per site (spins 0-1 and 2-3 x colour), each
    // packed as 18 complex slots: the 6 real diagonal entries in slots 0-2, then
    // the 15 upper entries row by row; FP64 [36][V], FP32 [18][V] float4
    // (two slots each).  Null when the term is off.
    const double2 *clov64;
    const float4 *clov32;
    // sites an apply covers, [s0, s1) (the whole lattice: 0, V); a t-slab of
    // the lattice is a contiguous range
    int s0, s1;
    // set to 1 by a kernel whose bounded wait gave up (host-mapped, read by
    // the next apply call); stall != 0 makes the bulk-copy kernel announce 16
    // bytes more than its first stage delivers, so that its waits run out
    int *werr;
    int stall;
};
inline void geom_set_weights(Geom &g, const double lam[5], const double rho[5]) {
    for (int n = 0; n < 5; n++) {
        g.lamd[n] = lam[n];
        g.rhod[n] = n == 0 ? 0.0 : rho[n];
        g.lam[n] = (float)g.lamd[n];
        g.rho[n] = (float)g.rhod[n];
    }
    g.nhop = 0;
    for (int j = 0; j < NCANON; j++) {
        const int k = canon_k(j), n = off_class(k);
        if (g.lamd[n] == 0.0 && g.rhod[n] == 0.0) continue;
        HopArg &h = g.hop[g.nhop++];
        for (int mu = 0; mu < 4; mu++) {
            h.dm[mu] = off_comp(k, mu);
            h.fd[mu] = (float)h.dm[mu];
        }
        h.j = (short)j;
        h.hd = h.dm[0] + (TX + 2) * (h.dm[1] + (TY + 2) * (h.dm[2] + (TZ + 2) * h.dm[3]));
        h.lam = g.lam[n];
        h.rho = g.rho[n];
    }
    // the hops of one run of equal (d_y, d_z, d_t) (d_x = -1, 0, 1: consecutive
    // canonical indices) read their neighbour spinors from the same two x lines
    for (int t = g.nhop - 1; t >= 0; t--) {
        const HopArg &h = g.hop[t];
        const bool same = t + 1 < g.nhop && g.hop[t + 1].dm[1] == h.dm[1] && g.hop[t + 1].dm[2] == h.dm[2] &&
                          g.hop[t + 1].dm[3] == h.dm[3];
        g.hop[t].ge = (short)(same ? g.hop[t + 1].ge : t + 1);
    }
}

// Per-site neighbour deltas (with periodic wrap) and boundary phases.
struct SiteNb {
    int fw[4], bw[4];       // index delta of x+mu, x-mu
    float sfw[4], sbw[4];   // fermion phase picked up by x -> x+mu, x -> x-mu
};
BRI_D SiteNb site_nb(const Geom &g, int site, int x[4]) {
    SiteNb n;
    int s = site;
    int stride = 1;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        x[mu] = s % g.L[mu];
        s /= g.L[mu];
        bool top = x[mu] == g.L[mu] - 1, bot = x[mu] == 0;
        n.fw[mu] = top ? -(g.L[mu] - 1) * stride : stride;
        n.bw[mu] = bot ? (g.L[mu] - 1) * stride : -stride;
        n.sfw[mu] = top ? (float)g.bc[mu] : 1.f;
        n.sbw[mu] = bot ? (float)g.bc[mu] : 1.f;
        stride *= g.L[mu];
    }
    return n;
}
// neighbour index and phase of offset k (0..80), sign = +1 forward, -1 reversed
template <int K, int SGN> BRI_D int nb_index(const SiteNb &n, int site, float &ph) {
    int y = site;
    float p = 1.f;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int c = SGN * off_comp(K, mu);
        if (c > 0) { y += n.fw[mu]; p *= n.sfw[mu]; }
        if (c < 0) { y += n.bw[mu]; p *= n.sbw[mu]; }
    }
    ph = p;
    return y;
}

// neighbour index and boundary phase of the forward (d) and reversed (-d) hop
BRI_D void hop_nb(const int dm[4], int site, const SiteNb &nb, int &yf, float &phf, int &yb, float &phb) {
    yf = yb = site;
    phf = phb = 1.f;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        if (dm[mu] > 0) { yf += nb.fw[mu]; phf *= nb.sfw[mu]; yb += nb.bw[mu]; phb *= nb.sbw[mu]; }
        else if (dm[mu] < 0) { yf += nb.bw[mu]; phf *= nb.sbw[mu]; yb += nb.fw[mu]; phb *= nb.sfw[mu]; }
    }
}

}  // namespace bri
