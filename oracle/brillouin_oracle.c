/*
 * Brillouin Dirac operator -- plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  It
 * shares no code, header, table or helper with the CUDA library in
 * paper_1012_3615_gb300/, and neither side imports the other.
 *
 * What it computes (Duerr & Koutsou, "Brillouin improvement for Wilson
 * fermions"):
 *   D(x,y) = sum_mu gamma_mu rho_mu(x-y) + lambda(x-y)                (Sec. 8)
 *   with the der_iso / lap_bri weights of Tab. "rholambda", i.e.
 *   D = sum_mu gamma_mu nabla^iso_mu - (1/2) Laplacian^bri + m0        (Eq. def_pref, c_SW = 0)
 *   Off-axis hops carry the sum over all shortest lattice paths, followed by
 *   a single back-projection to SU(3) (Sec. 5.1); the projection is the
 *   variational one of Eq. proj_SU, solved by SVD + phase maximisation
 *   (Sec. 5.2).  The maximisation uses a dense grid scan followed by Newton
 *   polishing, i.e. the scan-then-local-maximisation strategy described in the
 *   footnote of Sec. 5.2, with a much finer grid than pi/3.
 *
 * Everything is written for clarity, not speed: every hop is stored
 * independently (80 per site), paths are enumerated explicitly, the SVD is a
 * textbook one-sided (Hestenes) Jacobi iteration, the adjoint of D is the
 * literal transpose-conjugate of the stencil.
 *
 * Conventions (stated here, independently of the CUDA library):
 *   site index   x0 + L0*(x1 + L1*(x2 + L2*x3)), mu = 0..3 <-> paper's 1..4
 *   links U      [V][4][3][3]  complex double, U_mu(x) connects x to x+mu
 *   hops  W      [V][81][3][3] complex double, offset index
 *                k(d) = sum_mu (d_mu+1)*3^mu, k = 40 is d = 0 (unused)
 *   spinors      [V][4][3] complex double (spin, colour)
 *   fermion boundary phase bc[mu] = +1 / -1, applied to every hop that
 *   wraps around direction mu (not folded into W).
 *   gamma basis  hermitian chiral (DeGrand-Rossi) basis, gamma_5 =
 *                gamma_1 gamma_2 gamma_3 gamma_4 = diag(1,1,-1,-1).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define PI 3.14159265358979323846

#define NDIR 4
#define NHOP 81
#define CENTRE 40

/* ------------------------------------------------------------------ */
/* small dense 3x3 helpers (row-major)                                 */
/* ------------------------------------------------------------------ */
static void m3_eye(cplx *a) {
    for (int i = 0; i < 9; i++) a[i] = 0;
    a[0] = a[4] = a[8] = 1;
}
static void m3_mul(const cplx *a, const cplx *b, cplx *c) { /* c = a b */
    cplx t[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx s = 0;
            for (int k = 0; k < 3; k++) s += a[3 * i + k] * b[3 * k + j];
            t[3 * i + j] = s;
        }
    memcpy(c, t, sizeof t);
}
static void m3_dag(const cplx *a, cplx *c) { /* c = a^dagger */
    cplx t[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) t[3 * i + j] = conj(a[3 * j + i]);
    memcpy(c, t, sizeof t);
}
static cplx m3_det(const cplx *a) {
    return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
           a[2] * (a[3] * a[7] - a[4] * a[6]);
}
static cplx m3_trace(const cplx *a) { return a[0] + a[4] + a[8]; }

/* ------------------------------------------------------------------ */
/* lattice geometry                                                    */
/* ------------------------------------------------------------------ */
static long volume(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }
static void coords(const int L[4], long s, int x[4]) {
    for (int mu = 0; mu < 4; mu++) { x[mu] = (int)(s % L[mu]); s /= L[mu]; }
}
static long index_of(const int L[4], const int x[4]) {
    return x[0] + (long)L[0] * (x[1] + (long)L[1] * (x[2] + (long)L[2] * x[3]));
}
/* site x+d with periodic wrap; *phase = product of bc[mu] over wrapped mu */
static long shifted(const int L[4], const int bc[4], const int x[4], const int d[4], double *phase) {
    int y[4];
    double ph = 1.0;
    for (int mu = 0; mu < 4; mu++) {
        y[mu] = x[mu] + d[mu];
        if (y[mu] < 0) { y[mu] += L[mu]; if (bc) ph *= bc[mu]; }
        if (y[mu] >= L[mu]) { y[mu] -= L[mu]; if (bc) ph *= bc[mu]; }
    }
    if (phase) *phase = ph;
    return index_of(L, y);
}
static void offset_of(int k, int d[4]) {
    for (int mu = 0; mu < 4; mu++) { d[mu] = k % 3 - 1; k /= 3; }
}
static int hop_class(const int d[4]) {
    return abs(d[0]) + abs(d[1]) + abs(d[2]) + abs(d[3]);
}

/* ------------------------------------------------------------------ */
/* weights: Tab. "rholambda" (default: columns der_iso and lap_bri)     */
/* ------------------------------------------------------------------ */
/* The operator's class weights; bo_set_weights replaces them (other columns of
 * Tab. rholambda, e.g. Wilson's), bo_reset_weights restores the table's
 * der_iso / lap_bri column. */
static double g_lam[5], g_rho[5];
static int g_weights_set = 0;
int bo_reset_weights(void) {
    static const double lam_num[5] = {240, -8, -4, -2, -1}; /* / 128 */
    static const double rho_num[5] = {0, 64, 16, 4, 1};     /* / 432 */
    for (int n = 0; n < 5; n++) {
        g_lam[n] = lam_num[n] / 128.0;
        g_rho[n] = rho_num[n] / 432.0;
    }
    g_weights_set = 1;
    return 0;
}
int bo_set_weights(const double lam[5], const double rho[5]) {
    for (int n = 0; n < 5; n++) {
        g_lam[n] = lam[n];
        g_rho[n] = n == 0 ? 0.0 : rho[n];
    }
    g_weights_set = 1;
    return 0;
}
int bo_weights(double lam[5], double rho[5]) {
    if (!g_weights_set) bo_reset_weights();
    for (int n = 0; n < 5; n++) {
        lam[n] = g_lam[n];
        rho[n] = g_rho[n];
    }
    return 0;
}

/* gamma_mu, mu = 0..3, and gamma_5 for mu = 4; out is 4x4 row-major */
int bo_gamma(int mu, cplx *out) {
    const cplx J = _Complex_I;
    static cplx g[5][16];
    static int init = 0;
    if (!init) {
        memset(g, 0, sizeof g);
        /* gamma_1 */
        g[0][0 * 4 + 3] = J;  g[0][1 * 4 + 2] = J;  g[0][2 * 4 + 1] = -J; g[0][3 * 4 + 0] = -J;
        /* gamma_2 */
        g[1][0 * 4 + 3] = -1; g[1][1 * 4 + 2] = 1;  g[1][2 * 4 + 1] = 1;  g[1][3 * 4 + 0] = -1;
        /* gamma_3 */
        g[2][0 * 4 + 2] = J;  g[2][1 * 4 + 3] = -J; g[2][2 * 4 + 0] = -J; g[2][3 * 4 + 1] = J;
        /* gamma_4 */
        g[3][0 * 4 + 2] = 1;  g[3][1 * 4 + 3] = 1;  g[3][2 * 4 + 0] = 1;  g[3][3 * 4 + 1] = 1;
        /* gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 (computed, not typed in) */
        cplx t[16], u[16];
        memcpy(t, g[0], sizeof t);
        for (int m = 1; m < 4; m++) {
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++) {
                    cplx s = 0;
                    for (int k = 0; k < 4; k++) s += t[4 * i + k] * g[m][4 * k + j];
                    u[4 * i + j] = s;
                }
            memcpy(t, u, sizeof t);
        }
        memcpy(g[4], t, sizeof t);
        init = 1;
    }
    if (mu < 0 || mu > 4) return -1;
    memcpy(out, g[mu], 16 * sizeof(cplx));
    return 0;
}

/* spin matrix of hop d: lambda_n 1 + rho_n sum_mu d_mu gamma_mu (Sec. 8) */
static void hop_spin_matrix(const int d[4], double sgn_rho, cplx M[16]) {
    double lam[5], rho[5];
    cplx g[16];
    bo_weights(lam, rho);
    int n = hop_class(d);
    for (int i = 0; i < 16; i++) M[i] = 0;
    for (int i = 0; i < 4; i++) M[5 * i] = lam[n];
    for (int mu = 0; mu < 4; mu++) {
        if (!d[mu]) continue;
        bo_gamma(mu, g);
        for (int i = 0; i < 16; i++) M[i] += sgn_rho * rho[n] * d[mu] * g[i];
    }
}

/* ------------------------------------------------------------------ */
/* SVD of a complex 3x3 matrix by one-sided (Hestenes) Jacobi rotations */
/* A = U diag(s) V^dagger                                               */
/* ------------------------------------------------------------------ */
int bo_svd3(const cplx *A, cplx *U, double *s, cplx *V) {
    cplx W[9];
    memcpy(W, A, sizeof W);
    m3_eye(V);
    for (int sweep = 0; sweep < 60; sweep++) {
        int rotated = 0;
        for (int p = 0; p < 2; p++)
            for (int q = p + 1; q < 3; q++) {
                double alpha = 0, beta = 0;
                cplx gamma = 0;
                for (int i = 0; i < 3; i++) {
                    alpha += creal(W[3 * i + p] * conj(W[3 * i + p]));
                    beta += creal(W[3 * i + q] * conj(W[3 * i + q]));
                    gamma += conj(W[3 * i + p]) * W[3 * i + q];
                }
                double g = cabs(gamma);
                if (g <= 1e-17 * sqrt(alpha * beta) || g == 0.0) continue;
                rotated = 1;
                cplx eph = conj(gamma) / g; /* e^{-i phase(gamma)} */
                double zeta = (beta - alpha) / (2.0 * g);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                for (int i = 0; i < 3; i++) {
                    cplx wp = W[3 * i + p], wq = eph * W[3 * i + q];
                    W[3 * i + p] = c * wp - sn * wq;
                    W[3 * i + q] = sn * wp + c * wq;
                    cplx vp = V[3 * i + p], vq = eph * V[3 * i + q];
                    V[3 * i + p] = c * vp - sn * vq;
                    V[3 * i + q] = sn * vp + c * vq;
                }
            }
        if (!rotated) break;
    }
    for (int k = 0; k < 3; k++) {
        double nrm = 0;
        for (int i = 0; i < 3; i++) nrm += creal(W[3 * i + k] * conj(W[3 * i + k]));
        nrm = sqrt(nrm);
        s[k] = nrm;
        for (int i = 0; i < 3; i++) U[3 * i + k] = nrm > 0 ? W[3 * i + k] / nrm : (i == k);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* phase problem of Sec. 5.2: maximise s1 cos t1 + s2 cos t2 + s3 cos t3 */
/* subject to t1 + t2 + t3 + phi = 0 (mod 2 pi)                          */
/* ------------------------------------------------------------------ */
#define GRID 128
static double phase_f(const double s[3], double phi, double t1, double t2) {
    return s[0] * cos(t1) + s[1] * cos(t2) + s[2] * cos(-phi - t1 - t2);
}
static double newton_polish(const double s[3], double phi, double *t1, double *t2) {
    double a = *t1, b = *t2;
    double f = phase_f(s, phi, a, b);
    double scale = s[0] + s[1] + s[2];
    for (int it = 0; it < 200; it++) {
        double t3 = -phi - a - b;
        double g1 = -s[0] * sin(a) + s[2] * sin(t3);
        double g2 = -s[1] * sin(b) + s[2] * sin(t3);
        if (sqrt(g1 * g1 + g2 * g2) < 1e-15 * scale) break;
        double h11 = -s[0] * cos(a) - s[2] * cos(t3);
        double h22 = -s[1] * cos(b) - s[2] * cos(t3);
        double h12 = -s[2] * cos(t3);
        double det = h11 * h22 - h12 * h12;
        double da, db;
        if (h11 < 0 && det > 0) { /* Newton step on a concave patch */
            da = -(h22 * g1 - h12 * g2) / det;
            db = -(-h12 * g1 + h11 * g2) / det;
        } else { /* plain gradient ascent */
            da = g1 / scale;
            db = g2 / scale;
        }
        double step = 1.0, fn = f;
        int accepted = 0;
        int newton = (h11 < 0 && det > 0);
        if (newton && fabs(da) + fabs(db) < 1e-3) {
            /* inside the quadratic basin: take the full Newton step (comparing
             * f values cannot resolve steps below ~sqrt(machine epsilon)) */
            fn = phase_f(s, phi, a + da, b + db);
            accepted = 1;
        } else {
            for (int ls = 0; ls < 60; ls++) {
                fn = phase_f(s, phi, a + step * da, b + step * db);
                if (fn >= f) { accepted = 1; break; }
                step *= 0.5;
            }
        }
        if (!accepted) break;
        a += step * da;
        b += step * db;
        if (fabs(step * da) + fabs(step * db) < 1e-16) { f = fn; break; }
        f = fn;
    }
    *t1 = a;
    *t2 = b;
    return f;
}
int bo_phase_max(const double s[3], double phi, double theta[3]) {
    double c1[GRID], c2[GRID], c3[2 * GRID];
    const double h = 2.0 * PI / GRID;
    for (int i = 0; i < GRID; i++) {
        c1[i] = s[0] * cos(-PI + h * i);
        c2[i] = s[1] * cos(-PI + h * i);
    }
    for (int m = 0; m < 2 * GRID; m++) c3[m] = s[2] * cos(-phi + 2.0 * PI - h * m);
    static double F[GRID][GRID];
#pragma omp threadprivate(F)
    for (int i = 0; i < GRID; i++)
        for (int j = 0; j < GRID; j++) F[i][j] = c1[i] + c2[j] + c3[i + j];
    /* candidate starts: the four best grid-local maxima */
    int ci[4] = {-1, -1, -1, -1}, cj[4] = {0};
    double cf[4] = {-1e300, -1e300, -1e300, -1e300};
    for (int i = 0; i < GRID; i++)
        for (int j = 0; j < GRID; j++) {
            double v = F[i][j];
            int is_max = 1;
            for (int di = -1; di <= 1 && is_max; di++)
                for (int dj = -1; dj <= 1; dj++) {
                    if (!di && !dj) continue;
                    if (F[(i + di + GRID) % GRID][(j + dj + GRID) % GRID] > v) { is_max = 0; break; }
                }
            if (!is_max) continue;
            for (int k = 0; k < 4; k++)
                if (v > cf[k]) {
                    for (int m = 3; m > k; m--) { cf[m] = cf[m - 1]; ci[m] = ci[m - 1]; cj[m] = cj[m - 1]; }
                    cf[k] = v; ci[k] = i; cj[k] = j;
                    break;
                }
        }
    double best = -1e300, bt1 = 0, bt2 = 0;
    for (int k = 0; k < 4; k++) {
        if (ci[k] < 0) continue;
        double t1 = -PI + h * ci[k], t2 = -PI + h * cj[k];
        double f = newton_polish(s, phi, &t1, &t2);
        if (f > best) { best = f; bt1 = t1; bt2 = t2; }
    }
    theta[0] = bt1;
    theta[1] = bt2;
    theta[2] = -phi - bt1 - bt2;
    return 0;
}

/* P_SU(3){A} = argmin_{Y in SU(3)} tr (A-Y)^dagger (A-Y)   (Eq. proj_SU) */
int bo_project_su3(const cplx *A, cplx *Y) {
    cplx U[9], V[9], D[9], T[9], Vd[9];
    double s[3], theta[3];
    bo_svd3(A, U, s, V);
    /* det(A) = rho e^{i phi}, e^{i phi} = det(U) det(V)^*  (step 2) */
    double phi = carg(m3_det(U) * conj(m3_det(V)));
    bo_phase_max(s, phi, theta); /* step 3 */
    for (int i = 0; i < 9; i++) D[i] = 0;
    for (int k = 0; k < 3; k++) D[4 * k] = cexp(_Complex_I * theta[k]);
    m3_mul(U, D, T);
    m3_dag(V, Vd);
    m3_mul(T, Vd, Y); /* Y = U D V^dagger */
    return 0;
}

/* ------------------------------------------------------------------ */
/* path sums (Sec. 5.1): sum over all shortest lattice paths x -> x+d   */
/* ------------------------------------------------------------------ */
static const cplx *link_at(const int L[4], const cplx *U, long site, int mu) {
    (void)L;
    return U + (site * 4 + mu) * 9;
}
/* product of links along the path whose k-th step is direction mu[order[k]] */
static void path_product(const int L[4], const cplx *U, const int x[4], int n, const int *mus,
                         const int *sgn, const int *order, cplx *P) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    m3_eye(P);
    for (int k = 0; k < n; k++) {
        int mu = mus[order[k]], s = sgn[order[k]];
        cplx l[9];
        if (s > 0) {
            memcpy(l, link_at(L, U, index_of(L, y), mu), sizeof l);
            y[mu] = (y[mu] + 1) % L[mu];
        } else {
            y[mu] = (y[mu] - 1 + L[mu]) % L[mu];
            m3_dag(link_at(L, U, index_of(L, y), mu), l);
        }
        m3_mul(P, l, P);
    }
}
static int next_permutation(int *a, int n) {
    int i = n - 2;
    while (i >= 0 && a[i] >= a[i + 1]) i--;
    if (i < 0) return 0;
    int j = n - 1;
    while (a[j] <= a[i]) j--;
    int t = a[i]; a[i] = a[j]; a[j] = t;
    for (int l = i + 1, r = n - 1; l < r; l++, r--) { t = a[l]; a[l] = a[r]; a[r] = t; }
    return 1;
}
/* A = sum over all n! orderings of the unit steps of d (unnormalised) */
int bo_path_sum(const int L[4], const cplx *U, long site, const int d[4], cplx *A, int *npaths) {
    int x[4], mus[4], sgn[4], order[4], n = 0;
    coords(L, site, x);
    for (int mu = 0; mu < 4; mu++)
        if (d[mu]) { mus[n] = mu; sgn[n] = d[mu]; n++; }
    for (int i = 0; i < 9; i++) A[i] = 0;
    if (n == 0) { m3_eye(A); if (npaths) *npaths = 1; return 0; }
    for (int k = 0; k < n; k++) order[k] = k;
    int count = 0;
    do {
        cplx P[9];
        path_product(L, U, x, n, mus, sgn, order, P);
        for (int i = 0; i < 9; i++) A[i] += P[i];
        count++;
    } while (next_permutation(order, n));
    if (npaths) *npaths = count;
    return 0;
}

/* W_d(x) for all 80 offsets: the link itself for 1-hop offsets, the projected
 * path sum otherwise.  W[x][40] is set to the identity. */
int bo_build_hops(const int L[4], const cplx *U, cplx *W) {
    long V = volume(L);
    for (int mu = 0; mu < 4; mu++)
        if (L[mu] < 3) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (long s = 0; s < V; s++) {
        for (int k = 0; k < NHOP; k++) {
            int d[4];
            offset_of(k, d);
            cplx *out = W + (s * NHOP + k) * 9;
            cplx A[9];
            bo_path_sum(L, U, s, d, A, NULL);
            if (hop_class(d) >= 2)
                bo_project_su3(A, out);
            else
                memcpy(out, A, sizeof A);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* the operator                                                         */
/* ------------------------------------------------------------------ */
/* out = D psi, D(x,x+d) = phase * M_d (x) W_d(x), D(x,x) = m0 + lambda_0.
 * dagger != 0: out = D^dagger psi computed as the literal adjoint
 * (D^dagger psi)(x) = sum_d D(x-d, x)^dagger psi(x-d). */
int bo_apply(const int L[4], const int bc[4], const cplx *W, double m0, int dagger,
             const cplx *in, cplx *out) {
    long V = volume(L);
    double lam[5], rho[5];
    bo_weights(lam, rho);
    cplx M[NHOP][16];
    for (int k = 0; k < NHOP; k++) {
        int d[4];
        offset_of(k, d);
        hop_spin_matrix(d, 1.0, M[k]);
    }
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        int x[4];
        coords(L, s, x);
        cplx acc[12];
        for (int i = 0; i < 12; i++) acc[i] = (m0 + lam[0]) * in[s * 12 + i];
        for (int k = 0; k < NHOP; k++) {
            if (k == CENTRE) continue;
            int d[4], md[4];
            offset_of(k, d);
            double ph;
            if (!dagger) {
                long y = shifted(L, bc, x, d, &ph);
                const cplx *w = W + (s * NHOP + k) * 9;
                for (int a = 0; a < 4; a++)
                    for (int c = 0; c < 3; c++) {
                        cplx sum = 0;
                        for (int b = 0; b < 4; b++)
                            for (int cc = 0; cc < 3; cc++)
                                sum += M[k][4 * a + b] * w[3 * c + cc] * in[y * 12 + 3 * b + cc];
                        acc[3 * a + c] += ph * sum;
                    }
            } else {
                /* y = x - d, entry D(y, y+d)^dagger */
                for (int mu = 0; mu < 4; mu++) md[mu] = -d[mu];
                long y = shifted(L, bc, x, md, &ph);
                const cplx *w = W + (y * NHOP + k) * 9;
                for (int a = 0; a < 4; a++)
                    for (int c = 0; c < 3; c++) {
                        cplx sum = 0;
                        for (int b = 0; b < 4; b++)
                            for (int cc = 0; cc < 3; cc++)
                                sum += conj(M[k][4 * b + a]) * conj(w[3 * cc + c]) * in[y * 12 + 3 * b + cc];
                        acc[3 * a + c] += ph * sum;
                    }
            }
        }
        for (int i = 0; i < 12; i++) out[s * 12 + i] = acc[i];
    }
    return 0;
}

/* hermitian overlap kernel H = gamma_5 (D_{m0} - rho)   (Sec. 7.1, 7.4) */
int bo_overlap_kernel(const int L[4], const int bc[4], const cplx *W, double m0, double rho,
                      const cplx *in, cplx *out) {
    long V = volume(L);
    cplx g5[16];
    bo_gamma(4, g5);
    bo_apply(L, bc, W, m0 - rho, 0, in, out);
    for (long s = 0; s < V; s++) {
        cplx t[12];
        for (int a = 0; a < 4; a++)
            for (int c = 0; c < 3; c++) {
                cplx sum = 0;
                for (int b = 0; b < 4; b++) sum += g5[4 * a + b] * out[s * 12 + 3 * b + c];
                t[3 * a + c] = sum;
            }
        memcpy(out + s * 12, t, sizeof t);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* BiCGstab (van der Vorst 1992) for D x = b, the solver of Sec. 6.4      */
/* ------------------------------------------------------------------ */
static cplx vdot(long n, const cplx *a, const cplx *b) {
    cplx s = 0;
    for (long i = 0; i < n; i++) s += conj(a[i]) * b[i];
    return s;
}
int bo_bicgstab(const int L[4], const int bc[4], const cplx *W, double m0, const cplx *b, cplx *x,
                double tol, int maxit, int *iters, double *true_resid) {
    long n = volume(L) * 12;
    cplx *r = calloc(n, sizeof(cplx)), *rh = calloc(n, sizeof(cplx)), *p = calloc(n, sizeof(cplx));
    cplx *v = calloc(n, sizeof(cplx)), *s = calloc(n, sizeof(cplx)), *t = calloc(n, sizeof(cplx));
    double bnorm = sqrt(creal(vdot(n, b, b)));
    int status = -4, it = 0;
    bo_apply(L, bc, W, m0, 0, x, r);
    for (long i = 0; i < n; i++) { r[i] = b[i] - r[i]; rh[i] = r[i]; }
    cplx rho_old = 1, alpha = 1, omega = 1;
    if (bnorm == 0.0) { status = 0; goto done; }
    if (sqrt(creal(vdot(n, r, r))) <= tol * bnorm) { status = 0; goto done; }
    for (it = 1; it <= maxit; it++) {
        cplx rho = vdot(n, rh, r);
        if (cabs(rho) == 0.0) { status = -5; break; }
        cplx beta = (rho / rho_old) * (alpha / omega);
        for (long i = 0; i < n; i++) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        bo_apply(L, bc, W, m0, 0, p, v);
        cplx rv = vdot(n, rh, v);
        if (cabs(rv) == 0.0) { status = -5; break; }
        alpha = rho / rv;
        for (long i = 0; i < n; i++) s[i] = r[i] - alpha * v[i];
        bo_apply(L, bc, W, m0, 0, s, t);
        double tt = creal(vdot(n, t, t));
        omega = tt > 0 ? vdot(n, t, s) / tt : 0;
        for (long i = 0; i < n; i++) {
            x[i] += alpha * p[i] + omega * s[i];
            r[i] = s[i] - omega * t[i];
        }
        rho_old = rho;
        if (sqrt(creal(vdot(n, r, r))) <= tol * bnorm) { status = 0; break; }
        if (omega == 0.0) { status = -5; break; }
    }
    if (it > maxit) it = maxit;
done:
    bo_apply(L, bc, W, m0, 0, x, t);
    {
        double rr = 0;
        for (long i = 0; i < n; i++) rr += creal((b[i] - t[i]) * conj(b[i] - t[i]));
        if (true_resid) *true_resid = bnorm > 0 ? sqrt(rr) / bnorm : sqrt(rr);
        if (status == 0 && true_resid && *true_resid > tol) status = -4;
    }
    if (iters) *iters = it;
    free(r); free(rh); free(p); free(v); free(s); free(t);
    return status;
}

/* ------------------------------------------------------------------ */
/* derivative of the projection (vector-Jacobian product)              */
/* ------------------------------------------------------------------ */
/* Basis of su(3): T_a = i lambda_a / 2 (Gell-Mann), tr T_a T_b = -delta_ab/2 */
static void su3_basis(cplx T[8][9]) {
    const cplx J = _Complex_I;
    memset(T, 0, 8 * 9 * sizeof(cplx));
    cplx l[8][9];
    memset(l, 0, sizeof l);
    l[0][1] = 1; l[0][3] = 1;
    l[1][1] = -J; l[1][3] = J;
    l[2][0] = 1; l[2][4] = -1;
    l[3][2] = 1; l[3][6] = 1;
    l[4][2] = -J; l[4][6] = J;
    l[5][5] = 1; l[5][7] = 1;
    l[6][5] = -J; l[6][7] = J;
    l[7][0] = 1.0 / sqrt(3.0); l[7][4] = 1.0 / sqrt(3.0); l[7][8] = -2.0 / sqrt(3.0);
    for (int a = 0; a < 8; a++)
        for (int i = 0; i < 9; i++) T[a][i] = 0.5 * J * l[a][i];
}
static int solve8(double A[8][8], double b[8]) { /* Gaussian elimination, partial pivoting */
    for (int c = 0; c < 8; c++) {
        int p = c;
        for (int r = c + 1; r < 8; r++)
            if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
        if (A[p][c] == 0.0) return -1;
        if (p != c) {
            for (int k = 0; k < 8; k++) { double t = A[c][k]; A[c][k] = A[p][k]; A[p][k] = t; }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < 8; r++) {
            double f = A[r][c] / A[c][c];
            for (int k = c; k < 8; k++) A[r][k] -= f * A[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int c = 7; c >= 0; c--) {
        double s = b[c];
        for (int k = c + 1; k < 8; k++) s -= A[c][k] * b[k];
        b[c] = s / A[c][c];
    }
    return 0;
}
/* Given Y = P(A) and G = df/dRe(Y) + i df/dIm(Y), return GA = df/dRe(A) + i df/dIm(A).
 * Y maximises Re tr(A^dagger Y) on SU(3) (Eq. proj_SU), so the traceless
 * anti-hermitian part of A^dagger Y vanishes; differentiating that condition
 * with dY = Y dOmega, dOmega in su(3), gives an 8x8 real linear system. */
int bo_project_vjp(const cplx *A, const cplx *G, cplx *GA) {
    cplx T[8][9], Y[9], Ad[9], M[9], Gd[9], GdY[9];
    bo_project_su3(A, Y);
    su3_basis(T);
    m3_dag(A, Ad);
    m3_mul(Ad, Y, M); /* M = A^dagger Y */
    m3_dag(G, Gd);
    m3_mul(Gd, Y, GdY);
    double Lt[8][8], g[8];
    for (int a = 0; a < 8; a++) {
        cplx t[9];
        m3_mul(GdY, T[a], t);
        g[a] = creal(m3_trace(t));
        for (int b = 0; b < 8; b++) {
            cplx u[9];
            m3_mul(M, T[b], u);
            m3_mul(u, T[a], u);
            Lt[b][a] = -2.0 * creal(m3_trace(u)); /* transpose of L_ab */
        }
    }
    if (solve8(Lt, g)) return -1;
    cplx Um[9];
    for (int i = 0; i < 9; i++) {
        Um[i] = 0;
        for (int a = 0; a < 8; a++) Um[i] += g[a] * T[a][i];
    }
    m3_mul(Y, Um, GA);
    for (int i = 0; i < 9; i++) GA[i] *= 2.0;
    return 0;
}

/* ------------------------------------------------------------------ */
/* fermion force: dU += d Re(chi^dagger D[U] psi) / dU                  */
/* (gradient convention df/dRe U + i df/dIm U, U unconstrained)         */
/* ------------------------------------------------------------------ */
int bo_force(const int L[4], const int bc[4], const cplx *U, double m0, const cplx *chi,
             const cplx *psi, cplx *dU) {
    (void)m0; /* the mass term does not depend on U */
    long V = volume(L);
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    cplx *buf = calloc((size_t)nthr * V * 36, sizeof(cplx));
    if (!buf) return -2;
    cplx Mk[NHOP][16];
    for (int k = 0; k < NHOP; k++) {
        int d[4];
        offset_of(k, d);
        hop_spin_matrix(d, 1.0, Mk[k]);
    }
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        cplx *acc = buf + (size_t)tid * V * 36;
#pragma omp for schedule(dynamic, 4)
        for (long s = 0; s < V; s++) {
            int x[4];
            coords(L, s, x);
            for (int k = 0; k < NHOP; k++) {
                if (k == CENTRE) continue;
                int d[4];
                offset_of(k, d);
                double ph;
                long y = shifted(L, bc, x, d, &ph);
                /* this hop contributes Re tr(W_d(x) Z) to f, with
                 * Z[c'][c] = ph * sum_{a,b} chi(x)[a][c]^* M[a][b] psi(y)[b][c'] */
                cplx Z[9];
                for (int cp = 0; cp < 3; cp++)
                    for (int c = 0; c < 3; c++) {
                        cplx sum = 0;
                        for (int a = 0; a < 4; a++)
                            for (int b = 0; b < 4; b++)
                                sum += conj(chi[s * 12 + 3 * a + c]) * Mk[k][4 * a + b] * psi[y * 12 + 3 * b + cp];
                        Z[3 * cp + c] = ph * sum;
                    }
                cplx GW[9];
                m3_dag(Z, GW); /* G_W = Z^dagger */
                int n = hop_class(d);
                if (n == 1) {
                    int mu = 0;
                    while (!d[mu]) mu++;
                    if (d[mu] > 0) {
                        cplx *t = acc + (s * 4 + mu) * 9;
                        for (int i = 0; i < 9; i++) t[i] += GW[i];
                    } else {
                        int m1[4] = {0, 0, 0, 0};
                        m1[mu] = -1;
                        long z = shifted(L, NULL, x, m1, NULL);
                        cplx GWd[9];
                        m3_dag(GW, GWd);
                        cplx *t = acc + (z * 4 + mu) * 9;
                        for (int i = 0; i < 9; i++) t[i] += GWd[i];
                    }
                    continue;
                }
                cplx A[9], GA[9], GAd[9];
                bo_path_sum(L, U, s, d, A, NULL);
                bo_project_vjp(A, GW, GA);
                m3_dag(GA, GAd);
                /* product rule along every path */
                int mus[4], sg[4], order[4], nn = 0;
                for (int mu = 0; mu < 4; mu++)
                    if (d[mu]) { mus[nn] = mu; sg[nn] = d[mu]; nn++; }
                for (int i = 0; i < nn; i++) order[i] = i;
                do {
                    cplx Lk[4][9];
                    long zk[4];
                    int y2[4] = {x[0], x[1], x[2], x[3]};
                    for (int st = 0; st < nn; st++) {
                        int mu = mus[order[st]];
                        if (sg[order[st]] > 0) {
                            zk[st] = index_of(L, y2);
                            memcpy(Lk[st], link_at(L, U, zk[st], mu), 9 * sizeof(cplx));
                            y2[mu] = (y2[mu] + 1) % L[mu];
                        } else {
                            y2[mu] = (y2[mu] - 1 + L[mu]) % L[mu];
                            zk[st] = index_of(L, y2);
                            m3_dag(link_at(L, U, zk[st], mu), Lk[st]);
                        }
                    }
                    for (int st = 0; st < nn; st++) {
                        cplx P[9], S[9];
                        m3_eye(P);
                        for (int q = 0; q < st; q++) m3_mul(P, Lk[q], P);
                        m3_eye(S);
                        for (int q = st + 1; q < nn; q++) m3_mul(S, Lk[q], S);
                        int mu = mus[order[st]];
                        cplx R[9], t1[9], t2[9];
                        if (sg[order[st]] > 0) { /* A contains P U S: grad += P^dag GA S^dag */
                            cplx Pd[9], Sd[9];
                            m3_dag(P, Pd);
                            m3_dag(S, Sd);
                            m3_mul(Pd, GA, t1);
                            m3_mul(t1, Sd, R);
                        } else { /* A contains P U^dag S: grad += S GA^dag P */
                            m3_mul(S, GAd, t2);
                            m3_mul(t2, P, R);
                        }
                        cplx *t = acc + (zk[st] * 4 + mu) * 9;
                        for (int i = 0; i < 9; i++) t[i] += R[i];
                    }
                } while (next_permutation(order, nn));
            }
        }
    }
    for (int t = 0; t < nthr; t++)
        for (long i = 0; i < V * 36; i++) dU[i] += buf[(size_t)t * V * 36 + i];
    free(buf);
    return 0;
}

int bo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
void bo_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* batched helpers for the tests: n independent 3x3 matrices */
int bo_project_batch(long n, const cplx *A, cplx *Y) {
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < n; i++) bo_project_su3(A + 9 * i, Y + 9 * i);
    return 0;
}
int bo_project_vjp_batch(long n, const cplx *A, const cplx *G, cplx *GA) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
    for (long i = 0; i < n; i++) bad |= bo_project_vjp(A + 9 * i, G + 9 * i, GA + 9 * i) != 0;
    return bad ? -1 : 0;
}

/* (D psi)(x) at one site, with the 80 hops of that site built from U on the
 * spot (path sums + projection): lets tests sample large lattices one output
 * site at a time without building every hop. out: 12 complex. */
int bo_apply_site(const int L[4], const int bc[4], const cplx *U, double m0, long s, const cplx *in, cplx *out) {
    double lam[5], rho[5];
    bo_weights(lam, rho);
    int x[4];
    coords(L, s, x);
    for (int i = 0; i < 12; i++) out[i] = (m0 + lam[0]) * in[s * 12 + i];
    for (int k = 0; k < NHOP; k++) {
        if (k == CENTRE) continue;
        int d[4];
        offset_of(k, d);
        cplx A[9], w[9], M[16];
        bo_path_sum(L, U, s, d, A, NULL);
        if (hop_class(d) >= 2) bo_project_su3(A, w);
        else memcpy(w, A, sizeof A);
        hop_spin_matrix(d, 1.0, M);
        double ph;
        long y = shifted(L, bc, x, d, &ph);
        for (int a = 0; a < 4; a++)
            for (int c = 0; c < 3; c++) {
                cplx sum = 0;
                for (int b = 0; b < 4; b++)
                    for (int cc = 0; cc < 3; cc++) sum += M[4 * a + b] * w[3 * c + cc] * in[y * 12 + 3 * b + cc];
                out[3 * a + c] += ph * sum;
            }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* APE smearing (Eq. def_ape) and the clover term of Eq. def_pref       */
/* ------------------------------------------------------------------ */
/* U_{s mu}(x): the link leaving x in direction s*mu (s = +1 or -1),
 * U_{-mu}(x) = U_mu(x - mu)^dagger */
static void dir_link(const int L[4], const cplx *U, const int x[4], int mu, int s, cplx out[9]) {
    if (s > 0) {
        memcpy(out, U + (index_of(L, x) * 4 + mu) * 9, 9 * sizeof(cplx));
    } else {
        int d[4] = {0, 0, 0, 0};
        d[mu] = -1;
        long y = shifted(L, NULL, x, d, NULL);
        m3_dag(U + (y * 4 + mu) * 9, out);
    }
}

/* one APE step, written as printed: for every link
 *   V_mu(x) = P_SU(3){ (1 - alpha) 1 + alpha/6 sum_{+-nu != mu}
 *             U_nu(x) U_mu(x+nu) U_nu(x+mu)^dagger U_mu(x)^dagger } U_mu(x)
 * where for nu negative every U_nu is the link in direction -nu. */
int bo_ape_step(const int L[4], const cplx *U, double alpha, cplx *Vout) {
    long V = volume(L);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        int x[4];
        coords(L, s, x);
        for (int mu = 0; mu < 4; mu++) {
            const cplx *Umu = U + (s * 4 + mu) * 9;
            cplx Umu_dag[9], S[9];
            m3_dag(Umu, Umu_dag);
            for (int i = 0; i < 9; i++) S[i] = 0;
            for (int nu = 0; nu < 4; nu++) {
                if (nu == mu) continue;
                for (int sg = -1; sg <= 1; sg += 2) {
                    int dn[4] = {0, 0, 0, 0}, dm[4] = {0, 0, 0, 0};
                    dn[nu] = sg;
                    dm[mu] = 1;
                    int xn[4], xm[4];
                    coords(L, shifted(L, NULL, x, dn, NULL), xn);
                    coords(L, shifted(L, NULL, x, dm, NULL), xm);
                    cplx a[9], b[9], c[9], t[9];
                    dir_link(L, U, x, nu, sg, a);                           /* U_nu(x) */
                    memcpy(b, U + (index_of(L, xn) * 4 + mu) * 9, sizeof b); /* U_mu(x + nu) */
                    dir_link(L, U, xm, nu, sg, c);                          /* U_nu(x + mu) */
                    m3_dag(c, c);
                    m3_mul(a, b, t);
                    m3_mul(t, c, t);
                    m3_mul(t, Umu_dag, t);
                    for (int i = 0; i < 9; i++) S[i] += t[i];
                }
            }
            cplx X[9], Y[9];
            m3_eye(X);
            for (int i = 0; i < 9; i++) X[i] = (1.0 - alpha) * X[i] + alpha / 6.0 * S[i];
            bo_project_su3(X, Y);
            m3_mul(Y, Umu, Vout + (s * 4 + mu) * 9);
        }
    }
    return 0;
}

int bo_ape_smear(const int L[4], const cplx *U, double alpha, int nsteps, cplx *Vout) {
    long n = volume(L) * 36;
    cplx *a = malloc(n * sizeof(cplx));
    if (!a) return -1;
    memcpy(Vout, U, n * sizeof(cplx));
    for (int k = 0; k < nsteps; k++) {
        bo_ape_step(L, Vout, alpha, a);
        memcpy(Vout, a, n * sizeof(cplx));
    }
    free(a);
    return 0;
}

/* plaquette leaf U_{s mu}(x) U_{t nu}(x + s mu) U_{s mu}(x + t nu)^dagger U_{t nu}(x)^dagger */
static void leaf(const int L[4], const cplx *U, const int x[4], int mu, int s, int nu, int t, cplx out[9]) {
    int dmu[4] = {0, 0, 0, 0}, dnu[4] = {0, 0, 0, 0};
    dmu[mu] = s;
    dnu[nu] = t;
    int xm[4], xn[4];
    coords(L, shifted(L, NULL, x, dmu, NULL), xm);
    coords(L, shifted(L, NULL, x, dnu, NULL), xn);
    cplx a[9], b[9], c[9], d[9];
    dir_link(L, U, x, mu, s, a);
    dir_link(L, U, xm, nu, t, b);
    dir_link(L, U, xn, mu, s, c);
    dir_link(L, U, x, nu, t, d);
    m3_dag(c, c);
    m3_dag(d, d);
    m3_mul(a, b, out);
    m3_mul(out, c, out);
    m3_mul(out, d, out);
}

/* hermitian clover-leaf field strength F_{mu nu}(x) = (Q - Q^dagger) / (8 i),
 * Q = sum of the four leaves of the (mu, nu) plane at x, all with the same
 * orientation (mu then nu; nu then -mu; -mu then -nu; -nu then mu).
 * F: [V][6][3][3] for the planes (01, 02, 03, 12, 13, 23). */
int bo_clover_field(const int L[4], const cplx *U, cplx *F) {
    long V = volume(L);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        int x[4];
        coords(L, s, x);
        int p = 0;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++, p++) {
                cplx Q[9], t[9];
                for (int i = 0; i < 9; i++) Q[i] = 0;
                leaf(L, U, x, mu, +1, nu, +1, t);
                for (int i = 0; i < 9; i++) Q[i] += t[i];
                leaf(L, U, x, nu, +1, mu, -1, t);
                for (int i = 0; i < 9; i++) Q[i] += t[i];
                leaf(L, U, x, mu, -1, nu, -1, t);
                for (int i = 0; i < 9; i++) Q[i] += t[i];
                leaf(L, U, x, nu, -1, mu, +1, t);
                for (int i = 0; i < 9; i++) Q[i] += t[i];
                cplx *f = F + (s * 6 + p) * 9;
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) f[3 * i + j] = (Q[3 * i + j] - conj(Q[3 * j + i])) / (8.0 * _Complex_I);
            }
    }
    return 0;
}

/* out += -(c_SW / 2) sum_{mu < nu} sigma_{mu nu} (x) F_{mu nu}(x) in(x),
 * sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu]; F from the links U */
int bo_clover_add(const int L[4], const cplx *U, double csw, const cplx *in, cplx *out) {
    long V = volume(L);
    cplx *F = malloc(V * 54 * sizeof(cplx));
    if (!F) return -1;
    bo_clover_field(L, U, F);
    cplx g[4][16], sig[6][16];
    for (int mu = 0; mu < 4; mu++) bo_gamma(mu, g[mu]);
    int p = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++, p++)
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++) {
                    cplx c = 0;
                    for (int k = 0; k < 4; k++) c += g[mu][4 * a + k] * g[nu][4 * k + b] - g[nu][4 * a + k] * g[mu][4 * k + b];
                    sig[p][4 * a + b] = 0.5 * _Complex_I * c;
                }
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++)
        for (int a = 0; a < 4; a++)
            for (int c = 0; c < 3; c++) {
                cplx sum = 0;
                for (int q = 0; q < 6; q++)
                    for (int b = 0; b < 4; b++)
                        for (int cc = 0; cc < 3; cc++)
                            sum += sig[q][4 * a + b] * F[(s * 6 + q) * 9 + 3 * c + cc] * in[s * 12 + 3 * b + cc];
                out[s * 12 + 3 * a + c] += -0.5 * csw * sum;
            }
    free(F);
    return 0;
}
