// Link smearing and the clover term of the operator (Eq. def_ape, Eq. def_pref).
//
//  * APE smearing: V_mu(x) = P_SU(3){(1 - alpha) U_mu(x) + alpha/6 S_mu(x)},
//    S the sum of the six staples U_{s nu}(x) U_mu(x + s nu) U_{s nu}(x + mu)^dagger.
//    Eq. def_ape projects the bracket (1 - alpha) 1 + alpha/6 S U_mu^dagger and
//    multiplies by U_mu(x) afterwards; the projection commutes with right
//    multiplication by a unitary matrix (P(X U) = P(X) U), so projecting
//    (1 - alpha) U + alpha/6 S once is the same map.  One thread per link, FP64,
//    the projection of Sec. 5.2 (project.cuh).
//  * Clover term: F_{mu nu}(x) = (Q - Q^dagger) / (8 i) with Q the four
//    plaquette leaves of the (mu, nu) plane at x, all oriented mu -> nu; the
//    site term C(x) = -(c_SW/2) sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x),
//    sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], is block diagonal in the chiral
//    basis and stored as two packed hermitian 6x6 blocks per site (common.cuh).
//    The stencil kernels add C(x) psi(x) in their epilogue.
#include <cstring>
#include <string>

#include "ctx.h"
#include "project.cuh"

using namespace bri;

namespace {

// the 2x2 chiral blocks of sigma_{mu nu} for the six planes (01, 02, 03, 12, 13, 23)
struct SigmaBlocks {
    double2 s[6][2][4];
};

BRI_D int wrap_index(const Geom &g, const int x[4]) {
    int s = 0;
    for (int mu = 3; mu >= 0; mu--) {
        int c = x[mu] % g.L[mu];
        if (c < 0) c += g.L[mu];
        s = s * g.L[mu] + c;
    }
    return s;
}

// link leaving site x in direction sgn * mu
BRI_D M3<double2> link_dir(const double2 *__restrict__ U, const Geom &g, const int x[4], int mu, int sgn) {
    M3<double2> m;
    if (sgn > 0) {
        const double2 *u = U + ((size_t)wrap_index(g, x) * 4 + mu) * 9;
        for (int i = 0; i < 9; i++) m.e[i] = u[i];
    } else {
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[mu] -= 1;
        const double2 *u = U + ((size_t)wrap_index(g, y) * 4 + mu) * 9;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) m.e[3 * i + j] = cconj(u[3 * j + i]);
    }
    return m;
}

__global__ void k_ape(const double2 *__restrict__ U, double2 *__restrict__ Vout, Geom g, double alpha) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    const int mu = blockIdx.y;
    if (site >= g.V) return;
    int x[4];
    {
        int s = site;
        for (int m = 0; m < 4; m++) {
            x[m] = s % g.L[m];
            s /= g.L[m];
        }
    }
    M3<double2> S = m3_zero<double2>();
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        for (int sg = -1; sg <= 1; sg += 2) {
            int xn[4] = {x[0], x[1], x[2], x[3]}, xm[4] = {x[0], x[1], x[2], x[3]};
            xn[nu] += sg;
            xm[mu] += 1;
            const M3<double2> a = link_dir(U, g, x, nu, sg);
            const M3<double2> b = link_dir(U, g, xn, mu, 1);
            const M3<double2> c = m3_dag(link_dir(U, g, xm, nu, sg));
            S = m3_mad(S, m3_mul(a, b), c);
        }
    }
    const M3<double2> u = link_dir(U, g, x, mu, 1);
    M3<double2> X;
    for (int i = 0; i < 9; i++) X.e[i] = cadd(cscale(u.e[i], 1.0 - alpha), cscale(S.e[i], alpha / 6.0));
    const M3<double2> Y = project_su3(X);
    double2 *v = Vout + ((size_t)site * 4 + mu) * 9;
    for (int i = 0; i < 9; i++) v[i] = Y.e[i];
}

// leaf U_{s mu}(x) U_{t nu}(x + s mu) U_{s mu}(x + t nu)^dagger U_{t nu}(x)^dagger
BRI_D M3<double2> leaf(const double2 *__restrict__ U, const Geom &g, const int x[4], int mu, int s, int nu, int t) {
    int xm[4] = {x[0], x[1], x[2], x[3]}, xn[4] = {x[0], x[1], x[2], x[3]};
    xm[mu] += s;
    xn[nu] += t;
    const M3<double2> a = link_dir(U, g, x, mu, s);
    const M3<double2> b = link_dir(U, g, xm, nu, t);
    const M3<double2> c = m3_dag(link_dir(U, g, xn, mu, s));
    const M3<double2> d = m3_dag(link_dir(U, g, x, nu, t));
    return m3_mul(m3_mul(a, b), m3_mul(c, d));
}

__global__ void k_clover_build(const double2 *__restrict__ U, Geom g, SigmaBlocks sb, double csw,
                               double2 *__restrict__ out64, float4 *__restrict__ out32) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= g.V) return;
    int x[4];
    {
        int s = site;
        for (int m = 0; m < 4; m++) {
            x[m] = s % g.L[m];
            s /= g.L[m];
        }
    }
    double2 C[2][36];  // two 6x6 blocks, row-major
    for (int b = 0; b < 2; b++)
        for (int i = 0; i < 36; i++) C[b][i] = make_double2(0.0, 0.0);
    int p = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++, p++) {
            M3<double2> Q = leaf(U, g, x, mu, 1, nu, 1);
            Q = m3_add(Q, leaf(U, g, x, nu, 1, mu, -1));
            Q = m3_add(Q, leaf(U, g, x, mu, -1, nu, -1));
            Q = m3_add(Q, leaf(U, g, x, nu, -1, mu, 1));
            M3<double2> F;  // (Q - Q^dagger) / (8 i)
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) {
                    const double2 d = csub(Q.e[3 * i + j], cconj(Q.e[3 * j + i]));
                    F.e[3 * i + j] = make_double2(d.y / 8.0, -d.x / 8.0);
                }
            for (int b = 0; b < 2; b++)
                for (int s1 = 0; s1 < 2; s1++)
                    for (int s2 = 0; s2 < 2; s2++) {
                        const double2 sg = cscale(sb.s[p][b][2 * s1 + s2], -0.5 * csw);
                        for (int c1 = 0; c1 < 3; c1++)
                            for (int c2 = 0; c2 < 3; c2++) {
                                double2 &e = C[b][6 * (3 * s1 + c1) + 3 * s2 + c2];
                                e = cadd(e, cmul(sg, F.e[3 * c1 + c2]));
                            }
                    }
        }
    for (int b = 0; b < 2; b++) {
        double2 slot[18];
        for (int k = 0; k < 3; k++) slot[k] = make_double2(C[b][7 * (2 * k)].x, C[b][7 * (2 * k + 1)].x);
        int k = 3;
        for (int i = 0; i < 6; i++)
            for (int j = i + 1; j < 6; j++) slot[k++] = C[b][6 * i + j];
        for (int e = 0; e < 18; e++) out64[(size_t)(18 * b + e) * g.V + site] = slot[e];
        for (int e = 0; e < 9; e++)
            out32[(size_t)(9 * b + e) * g.V + site] =
                make_float4((float)slot[2 * e].x, (float)slot[2 * e].y, (float)slot[2 * e + 1].x,
                            (float)slot[2 * e + 1].y);
    }
}

// dense gamma_mu from the library's table (one non-zero entry per row)
void gamma_dense(int mu, double2 G[16]) {
    for (int i = 0; i < 16; i++) G[i] = make_double2(0.0, 0.0);
    for (int s = 0; s < 4; s++) G[4 * s + gcol(mu, s)] = make_double2(gre(mu, s), gim(mu, s));
}

bool sigma_blocks(SigmaBlocks &sb) {
    double2 G[4][16];
    for (int mu = 0; mu < 4; mu++) gamma_dense(mu, G[mu]);
    int p = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++, p++) {
            double2 S[16];
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++) {
                    double2 c = make_double2(0.0, 0.0);
                    for (int k = 0; k < 4; k++)
                        c = cadd(c, csub(cmul(G[mu][4 * a + k], G[nu][4 * k + b]), cmul(G[nu][4 * a + k], G[mu][4 * k + b])));
                    S[4 * a + b] = make_double2(-0.5 * c.y, 0.5 * c.x);  // (i/2) c
                }
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++)
                    if ((a < 2) != (b < 2) && (S[4 * a + b].x != 0.0 || S[4 * a + b].y != 0.0)) return false;
            for (int blk = 0; blk < 2; blk++)
                for (int a = 0; a < 2; a++)
                    for (int b = 0; b < 2; b++) sb.s[p][blk][2 * a + b] = S[4 * (2 * blk + a) + 2 * blk + b];
        }
    return true;
}

}  // namespace

bri_status bri_ape_impl(bri_ctx *ctx, double2 *V, const double2 *U, double alpha, int nsteps, cudaStream_t s) {
    const size_t bytes = sizeof(double2) * 36 * (size_t)ctx->g.V;
    if (nsteps == 0) {
        BRI_TRY_CUDA(ctx, cudaMemcpyAsync(V, U, bytes, cudaMemcpyDeviceToDevice, s));
        return BRI_OK;
    }
    DevBuf tmpb;
    if (nsteps > 1) BRI_TRY_CUDA(ctx, cudaMalloc(&tmpb.p, bytes));
    double2 *tmp = tmpb.as<double2>();
    const unsigned nb = (unsigned)((ctx->g.V + 127) / 128);
    const double2 *src = U;
    for (int k = 0; k < nsteps; k++) {
        // the last step lands in V: alternate so that it does
        double2 *dst = ((nsteps - 1 - k) % 2 == 0) ? V : tmp;
        k_ape<<<dim3(nb, 4), 128, 0, s>>>(src, dst, ctx->g, alpha);
        BRI_LAUNCHED(ctx);
        src = dst;
    }
    if (tmp) BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));  // the temporary is freed on return
    return BRI_OK;
}

bri_status bri_clover_build_impl(bri_ctx *ctx, cudaStream_t s) {
    if (!ctx->clov64) {
        BRI_TRY_CUDA(ctx, cudaMalloc(&ctx->clov64, sizeof(double2) * 36 * (size_t)ctx->g.V));
        BRI_TRY_CUDA(ctx, cudaMalloc(&ctx->clov32, sizeof(float4) * 18 * (size_t)ctx->g.V));
    }
    SigmaBlocks sb;
    if (!sigma_blocks(sb)) return bri_fail(ctx, BRI_ESTATE, "sigma_{mu nu} is not block diagonal in this basis");
    k_clover_build<<<(ctx->g.V + 127) / 128, 128, 0, s>>>(ctx->U, ctx->g, sb, ctx->csw, ctx->clov64, ctx->clov32);
    BRI_LAUNCHED(ctx);
    ctx->g.clov64 = ctx->clov64;
    ctx->g.clov32 = ctx->clov32;
    return BRI_OK;
}
