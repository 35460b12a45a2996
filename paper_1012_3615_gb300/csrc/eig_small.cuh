// Small dense eigenproblems solved inside single-thread device code: the
// Lanczos tridiagonal matrix (eigenvalues by Sturm-count bisection,
// eigenvectors by inverse iteration with a partially pivoted tridiagonal LU)
// and a complex hermitian k x k matrix (cyclic Jacobi rotations).  Textbook
// methods (Wilkinson, "The Algebraic Eigenvalue Problem"; Golub & Van Loan,
// Sec. 8.4-8.5); host-callable as well.
#pragma once
#include <math.h>

#include "common.cuh"

namespace bri {

#define BRI_EIG __host__ __device__ inline

// Symmetric tridiagonal T of order m: diagonal a[0..m), off-diagonal b[1..m)
// with b[i] = T[i-1][i] = T[i][i-1].

// number of eigenvalues of T below x (signs of the LDL^T pivots of T - x)
BRI_EIG int tri_count_below(const double *a, const double *b, int m, double x, double pivmin) {
    int cnt = 0;
    double d = a[0] - x;
    if (fabs(d) < pivmin) d = -pivmin;
    if (d < 0) cnt++;
    for (int i = 1; i < m; i++) {
        d = (a[i] - x) - b[i] * b[i] / d;
        if (fabs(d) < pivmin) d = -pivmin;
        if (d < 0) cnt++;
    }
    return cnt;
}

// Gershgorin interval of T
BRI_EIG void tri_bounds(const double *a, const double *b, int m, double &lo, double &hi) {
    lo = 1e300;
    hi = -1e300;
    for (int i = 0; i < m; i++) {
        const double r = (i > 0 ? fabs(b[i]) : 0.0) + (i + 1 < m ? fabs(b[i + 1]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
    }
}

// k-th smallest eigenvalue (k = 0 .. m-1) by bisection to rounding level
BRI_EIG double tri_eigenvalue(const double *a, const double *b, int m, int k) {
    double lo, hi;
    tri_bounds(a, b, m, lo, hi);
    const double scale = fmax(fabs(lo), fabs(hi));
    const double pivmin = 1e-300 + 1e-30 * scale * scale;
    lo -= 1e-14 * scale + 1e-300;
    hi += 1e-14 * scale + 1e-300;
    for (int it = 0; it < 200; it++) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (tri_count_below(a, b, m, mid, pivmin) > k) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Inverse iteration for the eigenvector of T at eigenvalue th.  Work arrays of
// length m: u0, u1, u2 (rows of U), l (multipliers), p (1 = rows swapped); x
// returns the unit eigenvector.  Vectors prev[0..nprev) (each of length m,
// stride ldp) are projected out at every step (eigenvalues in a cluster).
BRI_EIG void tri_eigenvector(const double *a, const double *b, int m, double th, double *u0, double *u1,
                                   double *u2, double *l, unsigned char *p, double *x, const double *prev, int nprev,
                                   size_t ldp) {
    if (m == 1) {
        x[0] = 1.0;
        return;
    }
    double scale = 0.0;
    for (int i = 0; i < m; i++) scale = fmax(scale, fabs(a[i]) + (i > 0 ? fabs(b[i]) : 0.0));
    const double tiny = 1e-15 * scale + 1e-300;
    // factor P (T - th) = L U with U upper triangular of bandwidth 2
    double d = a[0] - th, e = b[1], f = 0.0;
    for (int i = 0; i + 1 < m; i++) {
        const double lo = b[i + 1], dn = a[i + 1] - th, en = i + 2 < m ? b[i + 2] : 0.0;
        if (fabs(d) >= fabs(lo)) {
            const double mu = d != 0.0 ? lo / d : 0.0;
            u0[i] = d; u1[i] = e; u2[i] = f; l[i] = mu; p[i] = 0;
            d = dn - mu * e;
            e = en - mu * f;
        } else {
            const double mu = d / lo;
            u0[i] = lo; u1[i] = dn; u2[i] = en; l[i] = mu; p[i] = 1;
            d = e - mu * dn;
            e = f - mu * en;
        }
        f = 0.0;
    }
    u0[m - 1] = d; u1[m - 1] = 0.0; u2[m - 1] = 0.0;
    for (int i = 0; i < m; i++)
        if (fabs(u0[i]) < tiny) u0[i] = u0[i] < 0 ? -tiny : tiny;
    // start: a fixed vector with no special structure
    for (int i = 0; i < m; i++) x[i] = 1.0 + 0.1 * sin(1.0 + 7.0 * i);
    for (int it = 0; it < 4; it++) {
        for (int v = 0; v < nprev; v++) {
            const double *q = prev + (size_t)v * ldp;
            double s = 0.0;
            for (int i = 0; i < m; i++) s += q[i] * x[i];
            for (int i = 0; i < m; i++) x[i] -= s * q[i];
        }
        // solve (T - th) y = x in place: forward with L and the swaps, back with U
        for (int i = 0; i + 1 < m; i++) {
            if (p[i]) {
                const double t = x[i];
                x[i] = x[i + 1];
                x[i + 1] = t;
            }
            x[i + 1] -= l[i] * x[i];
        }
        x[m - 1] /= u0[m - 1];
        x[m - 2] = (x[m - 2] - u1[m - 2] * x[m - 1]) / u0[m - 2];
        for (int i = m - 3; i >= 0; i--) x[i] = (x[i] - u1[i] * x[i + 1] - u2[i] * x[i + 2]) / u0[i];
        double mx = 0.0;
        for (int i = 0; i < m; i++) mx = fmax(mx, fabs(x[i]));
        if (!(mx > 0.0) || !isfinite(mx)) break;
        double nn = 0.0;
        for (int i = 0; i < m; i++) {
            x[i] /= mx;
            nn += x[i] * x[i];
        }
        nn = 1.0 / sqrt(nn);
        for (int i = 0; i < m; i++) x[i] *= nn;
    }
    for (int v = 0; v < nprev; v++) {
        const double *q = prev + (size_t)v * ldp;
        double s = 0.0;
        for (int i = 0; i < m; i++) s += q[i] * x[i];
        for (int i = 0; i < m; i++) x[i] -= s * q[i];
    }
    double nn = 0.0;
    for (int i = 0; i < m; i++) nn += x[i] * x[i];
    nn = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (int i = 0; i < m; i++) x[i] *= nn;
}

// Eigen-decomposition of the complex hermitian k x k matrix M (row-major,
// overwritten; its diagonal returns the eigenvalues) by cyclic Jacobi
// rotations; Q (row-major) returns the eigenvectors as columns.
BRI_EIG void herm_jacobi(double2 *M, double2 *Q, int k) {
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++) Q[i * k + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < k; i++)
            for (int j = 0; j < k; j++) {
                const double v = M[i * k + j].x * M[i * k + j].x + M[i * k + j].y * M[i * k + j].y;
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < k; p++)
            for (int q = p + 1; q < k; q++) {
                const double2 z = M[p * k + q];
                const double r = sqrt(z.x * z.x + z.y * z.y);
                if (r == 0.0) continue;
                // phase e^{-i phi} of z = r e^{i phi} moves into column q; then a real rotation
                const double2 ph = make_double2(z.x / r, -z.y / r);
                const double app = M[p * k + p].x, aqq = M[q * k + q].x;
                const double tau = (aqq - app) / (2.0 * r);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                // G: G_pp = c, G_pq = s, G_qp = -s ph, G_qq = c ph
                const double2 gpp = make_double2(c, 0.0), gpq = make_double2(s, 0.0);
                const double2 gqp = make_double2(-s * ph.x, -s * ph.y), gqq = make_double2(c * ph.x, c * ph.y);
                for (int i = 0; i < k; i++) {  // M <- M G, Q <- Q G (columns p, q)
                    const double2 mp = M[i * k + p], mq = M[i * k + q];
                    M[i * k + p] = cadd(cmul(mp, gpp), cmul(mq, gqp));
                    M[i * k + q] = cadd(cmul(mp, gpq), cmul(mq, gqq));
                    const double2 qp = Q[i * k + p], qq = Q[i * k + q];
                    Q[i * k + p] = cadd(cmul(qp, gpp), cmul(qq, gqp));
                    Q[i * k + q] = cadd(cmul(qp, gpq), cmul(qq, gqq));
                }
                for (int j = 0; j < k; j++) {  // M <- G^dagger M (rows p, q)
                    const double2 mp = M[p * k + j], mq = M[q * k + j];
                    M[p * k + j] = cadd(cmul(cconj(gpp), mp), cmul(cconj(gqp), mq));
                    M[q * k + j] = cadd(cmul(cconj(gpq), mp), cmul(cconj(gqq), mq));
                }
                M[p * k + q] = make_double2(0.0, 0.0);
                M[q * k + p] = make_double2(0.0, 0.0);
                M[p * k + p].y = 0.0;
                M[q * k + q].y = 0.0;
            }
    }
}

}  // namespace bri
