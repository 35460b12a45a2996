"""Pins of the oracle's SU(3) back-projection (Sec. 5.2, Eqs. def_projection,
proj_UN, proj_SU) and of its derivative."""
import numpy as np
import pytest

import oracle
from paper_1012_3615_gb300 import synth


def _dist2(A, Y):
    D = A - Y
    return float(np.real(np.trace(D.conj().T @ D)))


def _random_A(rng, n, noise=0.7):
    """Sums of random SU(3) matrices plus noise: generic complex 3x3 matrices."""
    base = synth.random_su3(n, int(rng.integers(1 << 30)))
    Z = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    return base + noise * Z


def _brute_max(A, grid=2048):
    """Max of Re tr(A^dagger Y) over Y = U diag(e^{i t}) V^dagger in SU(3), on a
    grid of (t1, t2), with numpy's SVD (a library routine, not the oracle's)."""
    U, s, Vh = np.linalg.svd(A)
    phi = np.angle(np.linalg.det(U) * np.linalg.det(Vh))
    t = np.linspace(-np.pi, np.pi, grid, endpoint=False)
    f = (s[0] * np.cos(t)[:, None] + s[1] * np.cos(t)[None, :]
         + s[2] * np.cos(-phi - t[:, None] - t[None, :]))
    return float(f.max())


def test_svd_matches_numpy():
    rng = np.random.default_rng(1)
    for A in _random_A(rng, 50):
        U, s, V = oracle.svd3(A)
        assert np.allclose(U @ np.diag(s) @ V.conj().T, A, atol=1e-13)
        assert np.allclose(U.conj().T @ U, np.eye(3), atol=1e-13)
        assert np.allclose(V.conj().T @ V, np.eye(3), atol=1e-13)
        assert np.allclose(np.sort(s), np.sort(np.linalg.svd(A, compute_uv=False)), atol=1e-13)


def test_projection_is_special_unitary():
    rng = np.random.default_rng(2)
    Y = oracle.project_su3(_random_A(rng, 200))
    for y in Y:
        assert np.allclose(y.conj().T @ y, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(y) - 1) < 1e-14


def test_projection_fixed_point_and_scale_invariance():
    rng = np.random.default_rng(3)
    G = synth.random_su3(50, 7)
    assert np.allclose(oracle.project_su3(G), G, atol=1e-14)
    A = _random_A(rng, 50)
    assert np.allclose(oracle.project_su3(3.7 * A), oracle.project_su3(A), atol=1e-13)


def test_projection_covariance():
    """P(g1 A g2^dagger) = g1 P(A) g2^dagger (end of Sec. 5.2)."""
    rng = np.random.default_rng(4)
    A = _random_A(rng, 100)
    g1 = synth.random_su3(100, 11)
    g2 = synth.random_su3(100, 12)
    lhs = oracle.project_su3(g1 @ A @ g2.conj().transpose(0, 2, 1))
    rhs = g1 @ oracle.project_su3(A) @ g2.conj().transpose(0, 2, 1)
    assert np.allclose(lhs, rhs, atol=1e-12)


def test_positive_determinant_reduces_to_polar_factor():
    """If det A > 0 the phase problem is solved by theta = 0 and P_SU(3)(A) is the
    U(3) projection A (A^dagger A)^{-1/2} of Eq. def_projection (textbook polar
    factor, computed here with numpy's eigh)."""
    rng = np.random.default_rng(5)
    for A in _random_A(rng, 40, noise=0.3):
        A = A / np.linalg.det(A) ** (1 / 3)  # det A = 1 > 0
        A = A * 1.3
        w, Q = np.linalg.eigh(A.conj().T @ A)
        polar = A @ Q @ np.diag(w ** -0.5) @ Q.conj().T
        assert np.allclose(oracle.project_su3(A), polar, atol=1e-13)


def test_global_optimality_against_dense_grid():
    rng = np.random.default_rng(6)
    A = _random_A(rng, 60, noise=1.5)
    Y = oracle.project_su3(A)
    for a, y in zip(A, Y):
        got = float(np.real(np.trace(a.conj().T @ y)))
        assert got >= _brute_max(a) - 1e-9


def test_local_optimality_against_perturbations():
    rng = np.random.default_rng(7)
    A = _random_A(rng, 30, noise=1.0)
    Y = oracle.project_su3(A)
    lam = synth._gell_mann()
    for a, y in zip(A, Y):
        d0 = _dist2(a, y)
        for _ in range(20):
            h = rng.standard_normal(8) * 1e-3
            H = np.einsum("a,aij->ij", h, lam)
            w, Q = np.linalg.eigh(H)
            y2 = y @ (Q @ np.diag(np.exp(1j * w)) @ Q.conj().T)
            assert _dist2(a, y2) >= d0 - 1e-14


def test_footnote_case_two_su3_sum_with_negative_determinant():
    """Footnote of Sec. 5.2: det(U+V) is real for U, V in SU(3) and can be
    negative; dividing the U(3) projection by a cube root of its determinant is
    then not the closest SU(3) matrix."""
    rng = np.random.default_rng(8)
    found = 0
    for trial in range(4000):
        U, V = synth.random_su3(2, 1000 + trial)
        A = U + V
        dA = np.linalg.det(A)
        assert abs(dA.imag) < 1e-12 * max(1.0, abs(dA))
        if dA.real >= -1e-3:
            continue
        found += 1
        Uu, s, Vh = np.linalg.svd(A)
        B = Uu @ Vh                              # P_U(3)(A), det B = -1
        naive = B / np.linalg.det(B) ** (1 / 3)  # principal cube root
        Y = oracle.project_su3(A)
        assert abs(np.linalg.det(Y) - 1) < 1e-13
        assert _dist2(A, Y) < _dist2(A, naive) - 1e-9
        assert float(np.real(np.trace(A.conj().T @ Y))) >= _brute_max(A) - 1e-9
        if found >= 5:
            break
    assert found >= 5


def test_phase_max_degenerate_unitary_input():
    """A unitary with det = -1 (s = 1,1,1, phi = pi): the maximum distributes the
    phase evenly, value 3 cos(pi/3) = 3/2."""
    th = oracle.phase_max(np.ones(3), np.pi)
    f = np.sum(np.cos(th))
    assert abs(f - 1.5) < 1e-13
    assert abs((np.sum(th) + np.pi) / (2 * np.pi) - round((np.sum(th) + np.pi) / (2 * np.pi))) < 1e-13


def test_projection_vjp_against_central_differences():
    rng = np.random.default_rng(9)
    A = _random_A(rng, 40, noise=0.5)
    G = rng.standard_normal((40, 3, 3)) + 1j * rng.standard_normal((40, 3, 3))
    E = rng.standard_normal((40, 3, 3)) + 1j * rng.standard_normal((40, 3, 3))
    GA = oracle.project_vjp(A, G)
    eps = 1e-5
    Yp = oracle.project_su3(A + eps * E)
    Ym = oracle.project_su3(A - eps * E)
    for i in range(40):
        fd = np.real(np.vdot(G[i], (Yp[i] - Ym[i]) / (2 * eps)))
        an = np.real(np.vdot(GA[i], E[i]))
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))
