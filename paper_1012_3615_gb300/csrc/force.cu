// Fermion force: dU += d Re(chi^dagger D[U] psi) / dU, with the hops of
// Sec. 5.1 and the projection of Sec. 5.2 differentiated exactly (U treated as
// an unconstrained complex matrix, gradient = df/dRe U + i df/dIm U).
//
// 1. hop gradients: the hop (x, d) contributes Re tr(W_d(x) Z_d(x)) with
//    Z_d(x)[c'][c] = s_d(x) sum_{a,b} chi(x)[a][c]^* M_d[a][b] psi(x+d)[b][c'],
//    M_d = lambda_n + rho_n sum_mu d_mu gamma_mu, so dW_d(x) gets Z_d(x)^dagger.
//    With W_{-d}(x+d) = W_d(x)^dagger the canonical field j collects
//    G_j(x) = Z_d(x)^dagger + Z_{-d}(x+d).
// 2. projection: Y = P(A) maximises Re tr(A^dagger Y) on SU(3), so the traceless
//    anti-hermitian part of A^dagger Y vanishes.  Writing dY = Y dOmega,
//    dOmega in su(3), the derivative of that condition is
//    L(dOmega) = -TA(dA^dagger Y), L(O) = {H, O}/2 - tr(H O)/3, with H the
//    hermitian part of A^dagger Y = V diag(s_i e^{i theta_i}) V^dagger.  In the
//    basis V, L scales the off-diagonal entries by (h_i + h_j)/2
//    (h_i = s_i cos theta_i) and is a rank-one update of diag(h) on the
//    diagonal, so it is inverted in closed form.  L is self-adjoint for
//    <X, Z> = -Re tr(X Z), which gives the vector-Jacobian product
//    G_A = -Y L^{-1}(TA(G^dagger Y)).
// 3. path sums: the averaging recursion A_d(x) = (1/n) sum F(x) A_{d'}(x') is
//    run backwards level by level (gather form, no atomics), and every
//    occurrence of a link collects its share.
#include "ctx.h"
#include "project.cuh"

using namespace bri;

namespace {

// step 1 (thread per site, canonical field j = blockIdx.y)
__global__ void k_hop_grad(const double2 *__restrict__ chi, const double2 *__restrict__ psi, M3<double2> *GA,
                           Geom g) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (site >= g.V) return;
    const int k = canon_k(j);
    const int n = off_class(k);
    const double lam = g.lamd[n], rho = g.rhod[n];
    int x[4];
    SiteNb nb = site_nb(g, site, x);
    int d[4];
    float ph = 1.f;
    int y = site;
    for (int mu = 0; mu < 4; mu++) {
        d[mu] = off_comp(k, mu);
        if (d[mu] > 0) { y += nb.fw[mu]; ph *= nb.sfw[mu]; }
        if (d[mu] < 0) { y += nb.bw[mu]; ph *= nb.sbw[mu]; }
    }
    // forward hop (x, d):   zf[cp][c] = sum_a chi(x)[a][c]^* (M_d psi(y))[a][cp]
    // reversed hop (y, -d): zb[cp][c] = sum_a chi(y)[a][c]^* (M_{-d} psi(x))[a][cp]
    // (the boundary phase of y -> x equals that of x -> y);  G = ph (zf^dagger + zb)
    M3<double2> Zf, Zb;  // [cp][c]
    for (int cp = 0; cp < 3; cp++)
        for (int c = 0; c < 3; c++) {
            double2 zf = make_double2(0, 0), zb = make_double2(0, 0);
            for (int a = 0; a < 4; a++) {
                double2 mf = cscale(psi[(size_t)y * 12 + 3 * a + cp], lam);
                double2 mb = cscale(psi[(size_t)site * 12 + 3 * a + cp], lam);
                for (int mu = 0; mu < 4; mu++) {
                    if (!d[mu]) continue;
                    const int col = gcol(mu, a);
                    const double2 e = make_double2(gre(mu, a), gim(mu, a));
                    mf = cadd(mf, cscale(cmul(e, psi[(size_t)y * 12 + 3 * col + cp]), rho * d[mu]));
                    mb = cadd(mb, cscale(cmul(e, psi[(size_t)site * 12 + 3 * col + cp]), -rho * d[mu]));
                }
                zf = cadd(zf, cmulc(chi[(size_t)site * 12 + 3 * a + c], mf));
                zb = cadd(zb, cmulc(chi[(size_t)y * 12 + 3 * a + c], mb));
            }
            Zf.e[3 * cp + c] = zf;
            Zb.e[3 * cp + c] = zb;
        }
    M3<double2> G = m3_add(m3_dag(Zf), Zb);
    for (int i = 0; i < 9; i++) G.e[i] = cscale(G.e[i], (double)ph);
    GA[(size_t)k * g.V + site] = G;
}

// step 2: G_A = VJP of the projection (off-axis canonical fields, in place)
__global__ void k_project_vjp(const M3<double2> *__restrict__ A, M3<double2> *GA, Geom g) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (site >= g.V) return;
    const int k = canon_k(j);
    if (off_class(k) < 2) return;
    const M3<double2> a = A[(size_t)k * g.V + site];
    const M3<double2> G = GA[(size_t)k * g.V + site];
    ProjectionParts pp;
    M3<double2> Y = project_su3(a, &pp);
    // P = TA(G^dagger Y) in the basis V: P' = V^dagger TA(G^dagger Y) V
    M3<double2> B = m3_mul(m3_dag(G), Y);
    M3<double2> Vm, Vd;
    for (int i = 0; i < 9; i++) Vm.e[i] = pp.V[i];
    Vd = m3_dag(Vm);
    M3<double2> Bp = m3_mul(Vd, m3_mul(B, Vm));
    double h[3];
    for (int i = 0; i < 3; i++) h[i] = pp.s[i] * cos(pp.th[i]);
    // anti-hermitian part of Bp (the trace part is removed through the diagonal solve)
    M3<double2> Q;
    for (int i = 0; i < 3; i++)
        for (int jj = 0; jj < 3; jj++) {
            double2 pij = cscale(csub(Bp.e[3 * i + jj], cconj(Bp.e[3 * jj + i])), 0.5);
            if (i != jj) Q.e[3 * i + jj] = cscale(pij, 2.0 / (h[i] + h[jj]));
            else Q.e[3 * i + jj] = pij;
        }
    // diagonal: p_i imaginary, made traceless; q_i = (p_i + m)/h_i, sum q_i = 0
    double p[3], tr = 0;
    for (int i = 0; i < 3; i++) { p[i] = Q.e[4 * i].y; tr += p[i]; }
    for (int i = 0; i < 3; i++) p[i] -= tr / 3.0;
    double sp = 0, sh = 0;
    for (int i = 0; i < 3; i++) { sp += p[i] / h[i]; sh += 1.0 / h[i]; }
    const double m = -sp / sh;
    for (int i = 0; i < 3; i++) Q.e[4 * i] = make_double2(0.0, (p[i] + m) / h[i]);
    M3<double2> Qv = m3_mul(Vm, m3_mul(Q, Vd));
    M3<double2> out = m3_mul(Y, Qv);
    for (int i = 0; i < 9; i++) out.e[i] = cscale(out.e[i], -1.0);
    GA[(size_t)k * g.V + site] = out;
}

// step 3a: G_{A_{d'}}(y) += sum_{mu notin supp d', s} (1/n) F_{mu,s}(y - s mu)^dagger G_{A_{d'+s mu}}(y - s mu)
__global__ void k_dp_back(int nlow, const int *__restrict__ klist, int nk, const double2 *__restrict__ U,
                          M3<double2> *GA, Geom g) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= g.V || blockIdx.y >= (unsigned)nk) return;
    const int kp = klist[blockIdx.y];
    int x[4];
    SiteNb nb = site_nb(g, site, x);
    M3<double2> acc = GA[(size_t)kp * g.V + site];
    const double inv = 1.0 / (nlow + 1);
    int p3 = 1;
    for (int mu = 0; mu < 4; mu++, p3 *= 3) {
        if (off_comp(kp, mu) != 0) continue;
        for (int sg = -1; sg <= 1; sg += 2) {
            const int k = kp + sg * p3;                  // d = d' + s mu
            const int z = site + (sg > 0 ? nb.bw[mu] : nb.fw[mu]);  // z = y - s mu
            // F_{mu,+}(z) = U_mu(z); F_{mu,-}(z) = U_mu(z - mu)^dagger = U_mu(y)^dagger
            M3<double2> Fd;  // F^dagger
            const double2 *u = U + ((size_t)(sg > 0 ? z : site) * 4 + mu) * 9;
            M3<double2> Um;
            for (int i = 0; i < 9; i++) Um.e[i] = u[i];
            Fd = sg > 0 ? m3_dag(Um) : Um;
            M3<double2> t = m3_mul(Fd, GA[(size_t)k * g.V + z]);
            for (int i = 0; i < 9; i++) acc.e[i] = cadd(acc.e[i], cscale(t.e[i], inv));
        }
    }
    GA[(size_t)kp * g.V + site] = acc;
}

// step 3b: link gradients (thread per site, mu = blockIdx.y), accumulated into dU [V][4][9]
__global__ void k_link_grad(const M3<double2> *__restrict__ A, const M3<double2> *__restrict__ GA,
                            double2 *__restrict__ dU, Geom g) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    const int mu = blockIdx.y;
    if (site >= g.V) return;
    int x[4];
    SiteNb nb = site_nb(g, site, x);
    const int xp = site + nb.fw[mu];
    const int p3 = pow3(mu);
    M3<double2> acc = m3_zero<double2>();
    for (int k = 0; k < NOFF; k++) {
        const int c = off_comp(k, mu);
        if (c == 0) continue;
        const int n = off_class(k);
        if (c > 0) {
            // A_d(x) with d_mu = +1: first step U_mu(x)
            const M3<double2> G = GA[(size_t)k * g.V + site];
            if (n == 1) acc = m3_add(acc, G);
            else {
                M3<double2> t = m3_mul(G, m3_dag(A[(size_t)(k - p3) * g.V + xp]));
                for (int i = 0; i < 9; i++) acc.e[i] = cadd(acc.e[i], cscale(t.e[i], 1.0 / n));
            }
        } else {
            // A_d(x+mu) with d_mu = -1: first step U_mu(x)^dagger
            const M3<double2> G = GA[(size_t)k * g.V + xp];
            if (n == 1) acc = m3_add(acc, m3_dag(G));
            else {
                M3<double2> t = m3_mul(A[(size_t)(k + p3) * g.V + site], m3_dag(G));
                for (int i = 0; i < 9; i++) acc.e[i] = cadd(acc.e[i], cscale(t.e[i], 1.0 / n));
            }
        }
    }
    double2 *o = dU + ((size_t)site * 4 + mu) * 9;
    for (int i = 0; i < 9; i++) o[i] = cadd(o[i], acc.e[i]);
}

}  // namespace

bri_status bri_force_impl(bri_ctx *ctx, double2 *dU, const double2 *chi, const double2 *psi, cudaStream_t s) {
    const Geom g = ctx->g;
    const size_t V = g.V;
    M3<double2> *A = nullptr, *GA = nullptr;
    int *klist = nullptr;
    BRI_TRY_CUDA(ctx, cudaMallocAsync((void **)&A, sizeof(M3<double2>) * NOFF * V, s));
    BRI_TRY_CUDA(ctx, cudaMallocAsync((void **)&GA, sizeof(M3<double2>) * NOFF * V, s));
    BRI_TRY_CUDA(ctx, cudaMallocAsync((void **)&klist, sizeof(int) * NOFF, s));
    BRI_TRY_CUDA(ctx, cudaMemsetAsync(GA, 0, sizeof(M3<double2>) * NOFF * V, s));
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
    const unsigned nb = (unsigned)((V + T - 1) / T);
    k_hop_grad<<<dim3(nb, NCANON), T, 0, s>>>(chi, psi, GA, g);
    BRI_LAUNCHED(ctx);
    k_project_vjp<<<dim3(nb, NCANON), T, 0, s>>>(A, GA, g);
    BRI_LAUNCHED(ctx);
    for (int nlow = 3; nlow >= 1; nlow--) {
        k_dp_back<<<dim3(nb, start[nlow + 1] - start[nlow]), T, 0, s>>>(nlow, klist + start[nlow],
                                                                        start[nlow + 1] - start[nlow], ctx->U, GA, g);
        BRI_LAUNCHED(ctx);
    }
    k_link_grad<<<dim3(nb, 4), T, 0, s>>>(A, GA, dU, g);
    BRI_LAUNCHED(ctx);
    BRI_TRY_CUDA(ctx, cudaFreeAsync(A, s));
    BRI_TRY_CUDA(ctx, cudaFreeAsync(GA, s));
    BRI_TRY_CUDA(ctx, cudaFreeAsync(klist, s));
    return BRI_OK;
}
