// FP64 back-projection to SU(3) (Sec. 5.2, Eq. proj_SU) on the device.
//
//   P_SU(3){A} = argmax_{Y in SU(3)} Re tr(A^dagger Y)
//
// With A = U S V^dagger, Y = U diag(e^{i theta}) V^dagger and the constraint
// sum theta_i + phi = 0 (mod 2 pi), e^{i phi} = det A / |det A|, the problem is
// to maximise sum_i s_i cos(theta_i).  The paper suggests a grid scan and a local
// maximisation.  Here the stationary points are used directly instead: a
// Lagrange multiplier kappa gives s_i sin(theta_i) = kappa for every i.  At a
// maximum only the smallest singular value may have cos(theta) < 0 (swapping
// phase between two indices would otherwise increase the sum), so the maximum is
//   branch A: theta_i = asin(kappa / s_i) for all i, when sum_i asin(kappa/s_i)
//             can reach the target -phi (mod 2 pi) for kappa in [-s_3, s_3];
//   branch B: theta_3 = pi - asin(kappa / s_3) otherwise.
// Branch A's sum is strictly increasing in kappa, so its root is unique; the
// rarely needed branch B is bracketed by a scan.  A (A^dagger A) eigen-
// decomposition by cyclic complex Jacobi rotations supplies S and V, and
// Y = U diag(e^{i theta_i}) V^dagger with U = A V S^{-1}.
#pragma once
#include "common.cuh"

namespace bri {

// Hermitian 3x3 eigen-decomposition H = V diag(e) V^dagger by Jacobi rotations.
BRI_D void herm_eig3(double2 H[9], double2 V[9], double e[3]) {
#pragma unroll
    for (int i = 0; i < 9; i++) V[i] = make_double2(i % 4 == 0 ? 1.0 : 0.0, 0.0);
    for (int sweep = 0; sweep < 20; sweep++) {
        double off = cnorm2(H[1]) + cnorm2(H[2]) + cnorm2(H[5]);
        double dg = H[0].x * H[0].x + H[4].x * H[4].x + H[8].x * H[8].x;
        if (off <= 1e-34 * dg || off == 0.0) break;
#pragma unroll
        for (int pq = 0; pq < 3; pq++) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            double2 h = H[3 * p + q];
            const double n2 = cnorm2(h);
            if (n2 == 0.0) continue;
            // FP64 divisions and square roots are long sequences on the FP64
            // pipe: one reciprocal square root serves |h|^-1, one the cosine
            const double ig = rsqrt(n2);
            double a = H[4 * p].x, b = H[4 * q].x;
            double tau = 0.5 * (b - a) * ig;
            double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(fma(tau, tau, 1.0)));
            double c = rsqrt(fma(t, t, 1.0)), s = t * c;
            double2 ep = make_double2(h.x * ig, -h.y * ig);  // e^{-i arg h}
            double2 se = cscale(ep, s), ce = cscale(ep, c);
            // H <- H J, V <- V J   (columns p, q), as FMA chains:
            //   new p = c x_p - x_q se,  new q = s x_p + x_q ce
#pragma unroll
            for (int i = 0; i < 3; i++) {
                double2 hp = H[3 * i + p], hq = H[3 * i + q];
                H[3 * i + p] = make_double2(fma(-hq.x, se.x, fma(hq.y, se.y, c * hp.x)),
                                            fma(-hq.x, se.y, fma(-hq.y, se.x, c * hp.y)));
                H[3 * i + q] = make_double2(fma(hq.x, ce.x, fma(-hq.y, ce.y, s * hp.x)),
                                            fma(hq.x, ce.y, fma(hq.y, ce.x, s * hp.y)));
                double2 vp = V[3 * i + p], vq = V[3 * i + q];
                V[3 * i + p] = make_double2(fma(-vq.x, se.x, fma(vq.y, se.y, c * vp.x)),
                                            fma(-vq.x, se.y, fma(-vq.y, se.x, c * vp.y)));
                V[3 * i + q] = make_double2(fma(vq.x, ce.x, fma(-vq.y, ce.y, s * vp.x)),
                                            fma(vq.x, ce.y, fma(vq.y, ce.x, s * vp.y)));
            }
            // H <- J^dagger H   (rows p, q):
            //   new p = c y_p - conj(se) y_q,  new q = s y_p + conj(ce) y_q
#pragma unroll
            for (int j = 0; j < 3; j++) {
                double2 hp = H[3 * p + j], hq = H[3 * q + j];
                H[3 * p + j] = make_double2(fma(-se.x, hq.x, fma(-se.y, hq.y, c * hp.x)),
                                            fma(-se.x, hq.y, fma(se.y, hq.x, c * hp.y)));
                H[3 * q + j] = make_double2(fma(ce.x, hq.x, fma(ce.y, hq.y, s * hp.x)),
                                            fma(ce.x, hq.y, fma(-ce.y, hq.x, s * hp.y)));
            }
            H[3 * p + q] = make_double2(0, 0);
            H[3 * q + p] = make_double2(0, 0);
            H[4 * p].y = 0;
            H[4 * q].y = 0;
        }
    }
    e[0] = H[0].x;
    e[1] = H[4].x;
    e[2] = H[8].x;
}

// sum_i asin(kappa/s_i) - t and its derivative (is: the reciprocals 1/s_i)
BRI_D double branch_a(const double s[3], const double is[3], double kappa, double t, double &deriv) {
    double f = -t, d = 0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        double r = kappa * is[i];
        r = fmin(1.0, fmax(-1.0, r));
        f += asin(r);
        d += rsqrt(fmax(fma(s[i], s[i], -kappa * kappa), 1e-300));
    }
    deriv = d;
    return f;
}

// root of branch A for target t, |t| <= M guaranteed by the caller
BRI_D double solve_branch_a(const double s[3], double t) {
    double lo = -s[2], hi = s[2];
    const double is[3] = {1.0 / s[0], 1.0 / s[1], 1.0 / s[2]};
    double kappa = t / (is[0] + is[1] + is[2]);
    kappa = fmin(hi, fmax(lo, kappa));
    for (int it = 0; it < 200; it++) {
        double d;
        double f = branch_a(s, is, kappa, t, d);
        if (f == 0.0) break;
        if (f > 0) hi = kappa; else lo = kappa;
        double kn = kappa - f / d;
        if (!(kn > lo && kn < hi)) kn = 0.5 * (lo + hi);
        if (fabs(kn - kappa) <= 2e-16 * s[2] || hi - lo <= 2e-16 * s[2]) { kappa = kn; break; }
        kappa = kn;
    }
    return kappa;
}

BRI_D double branch_b(const double s[3], double kappa, double t) {
    double r0 = fmin(1.0, fmax(-1.0, kappa / s[0]));
    double r1 = fmin(1.0, fmax(-1.0, kappa / s[1]));
    double r2 = fmin(1.0, fmax(-1.0, kappa / s[2]));
    return asin(r0) + asin(r1) + 3.14159265358979323846 - asin(r2) - t;
}

// maximiser of s1 cos t1 + s2 cos t2 + s3 cos t3 with t1+t2+t3 = -phi (mod 2 pi);
// s must be sorted descending and positive.
BRI_D void phase_solve(const double s[3], double phi, double th[3]) {
    const double PI = 3.14159265358979323846;
    const double c = -phi;
    const double M = asin(fmin(1.0, s[2] / s[0])) + asin(fmin(1.0, s[2] / s[1])) + 0.5 * PI;
    double best = -1e300;
    // Branch A: of the targets t = -phi + 2 pi k only the one of smallest |t|
    // (k = 0, phi in (-pi, pi]) can be the maximum -- the root kappa(t) grows in
    // |kappa| with |t| and the objective sum_i sqrt(s_i^2 - kappa^2) falls with
    // |kappa| -- and if it is out of reach (|t| > M) so are the others.
    if (fabs(c) <= M) {
        const double kappa = solve_branch_a(s, c);
#pragma unroll
        for (int i = 0; i < 3; i++) th[i] = asin(fmin(1.0, fmax(-1.0, kappa / s[i])));
        // place the rounding residue of the constraint on theta_3
        th[2] = c - th[0] - th[1];
        return;
    }
    // branch B: theta_3 = pi - asin(kappa/s_3); the target lies in (M, 2 pi - M)
    double t = c < 0 ? c + 2.0 * PI : c;
    const int NS = 64;
    double prevk = -s[2], prevg = branch_b(s, prevk, t);
    for (int i = 1; i <= NS; i++) {
        double k = -s[2] + 2.0 * s[2] * i / NS;
        double g = branch_b(s, k, t);
        if (prevg == 0.0 || (prevg < 0) != (g < 0)) {
            double lo = prevk, hi = k, glo = prevg;
            for (int it = 0; it < 80; it++) {
                double mid = 0.5 * (lo + hi);
                double gm = branch_b(s, mid, t);
                if ((gm < 0) == (glo < 0)) { lo = mid; glo = gm; } else hi = mid;
            }
            double kappa = 0.5 * (lo + hi);
            double t0 = asin(fmin(1.0, fmax(-1.0, kappa / s[0])));
            double t1 = asin(fmin(1.0, fmax(-1.0, kappa / s[1])));
            double t2 = t - t0 - t1;
            double f = s[0] * cos(t0) + s[1] * cos(t1) + s[2] * cos(t2);
            if (f > best) { best = f; th[0] = t0; th[1] = t1; th[2] = t2; }
        }
        prevk = k;
        prevg = g;
    }
}

BRI_D void swap_cols(double2 U[9], double2 V[9], int a, int b) {
#pragma unroll
    for (int i = 0; i < 3; i++) {
        double2 t = U[3 * i + a]; U[3 * i + a] = U[3 * i + b]; U[3 * i + b] = t;
        t = V[3 * i + a]; V[3 * i + a] = V[3 * i + b]; V[3 * i + b] = t;
    }
}

BRI_D double2 det3(const double2 A[9]) {
    double2 m0 = csub(cmul(A[4], A[8]), cmul(A[5], A[7]));
    double2 m1 = csub(cmul(A[3], A[8]), cmul(A[5], A[6]));
    double2 m2 = csub(cmul(A[3], A[7]), cmul(A[4], A[6]));
    return cadd(csub(cmul(A[0], m0), cmul(A[1], m1)), cmul(A[2], m2));
}

// singular basis and phases of a projection (for its derivative)
struct ProjectionParts {
    double2 V[9];
    double s[3], th[3];
};

BRI_D M3<double2> project_su3(const M3<double2> &A, ProjectionParts *parts = nullptr) {
    double2 H[9], V[9];
    double e[3];
    // H = A^dagger A
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            double2 sum = make_double2(0, 0);
#pragma unroll
            for (int k = 0; k < 3; k++) sum = cadd(sum, cmulc(A.e[3 * k + i], A.e[3 * k + j]));
            H[3 * i + j] = sum;
        }
    herm_eig3(H, V, e);
    // sort eigenpairs descending
    int o[3] = {0, 1, 2};
    if (e[o[0]] < e[o[1]]) { int t = o[0]; o[0] = o[1]; o[1] = t; }
    if (e[o[1]] < e[o[2]]) { int t = o[1]; o[1] = o[2]; o[2] = t; }
    if (e[o[0]] < e[o[1]]) { int t = o[0]; o[0] = o[1]; o[1] = t; }
    double2 Vs[9];
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int i = 0; i < 3; i++) Vs[3 * i + k] = V[3 * i + o[k]];
    // U = A V S^{-1}: the columns of A V are orthogonal with norms s_k.  Taking s_k
    // as those column norms (not as square roots of the eigenvalues of A^dagger A)
    // keeps small singular values accurate; one Gram-Schmidt pass removes the
    // residual non-orthogonality.
    double2 Um[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            double2 sum = make_double2(0, 0);
#pragma unroll
            for (int l = 0; l < 3; l++) sum = cadd(sum, cmul(A.e[3 * i + l], Vs[3 * l + k]));
            Um[3 * i + k] = sum;
        }
    double s[3];
    const double tiny = 1e-300;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        // remove the components along the previous (orthonormal) columns
#pragma unroll
        for (int q = 0; q < k; q++) {
            double2 dot = make_double2(0, 0);
#pragma unroll
            for (int i = 0; i < 3; i++) dot = cadd(dot, cmulc(Um[3 * i + q], Um[3 * i + k]));
#pragma unroll
            for (int i = 0; i < 3; i++) Um[3 * i + k] = csub(Um[3 * i + k], cmul(Um[3 * i + q], dot));
        }
        double nrm = 0;
#pragma unroll
        for (int i = 0; i < 3; i++) nrm += cnorm2(Um[3 * i + k]);
        nrm = sqrt(nrm);
        s[k] = fmax(nrm, tiny);
#pragma unroll
        for (int i = 0; i < 3; i++) Um[3 * i + k] = cscale(Um[3 * i + k], 1.0 / s[k]);
    }
    // the ordering s_0 >= s_1 >= s_2 of the eigenvalues survives up to rounding;
    // restore it exactly for the phase solve
    if (s[0] < s[1]) { double t = s[0]; s[0] = s[1]; s[1] = t; swap_cols(Um, Vs, 0, 1); }
    if (s[1] < s[2]) { double t = s[1]; s[1] = s[2]; s[2] = t; swap_cols(Um, Vs, 1, 2); }
    if (s[0] < s[1]) { double t = s[0]; s[0] = s[1]; s[1] = t; swap_cols(Um, Vs, 0, 1); }
    // e^{i phi} = det(U V^dagger)
    double2 dU = det3(Um), dV = det3(Vs);
    double2 dd = cmulc(dV, dU);
    double phi = atan2(dd.y, dd.x);
    double th[3];
    phase_solve(s, phi, th);
    if (parts) {
#pragma unroll
        for (int i = 0; i < 9; i++) parts->V[i] = Vs[i];
#pragma unroll
        for (int k = 0; k < 3; k++) { parts->s[k] = s[k]; parts->th[k] = th[k]; }
    }
    // Y = U diag(e^{i th}) V^dagger
    double2 ph[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        double sn, cs;
        sincos(th[k], &sn, &cs);
        ph[k] = make_double2(cs, sn);
    }
    M3<double2> Y;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            double2 sum = make_double2(0, 0);
#pragma unroll
            for (int k = 0; k < 3; k++) sum = cadd(sum, cmul(cmul(Um[3 * i + k], ph[k]), cconj(Vs[3 * j + k])));
            Y.e[3 * i + j] = sum;
        }
    return Y;
}

}  // namespace bri
