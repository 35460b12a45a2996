"""Pins of the oracle's BiCGstab (Sec. 6.4) against a dense LU solve, and of
its fermion force against central finite differences."""
import numpy as np

import oracle
from paper_1012_3615_gb300 import synth

AP = (1, 1, 1, -1)


def _dense(L, bc, W, m0):
    V = synth.volume(L)
    n = V * 12
    M = np.zeros((n, n), complex)
    e = np.zeros((V, 4, 3), complex)
    for j in range(n):
        e.reshape(-1)[j] = 1
        M[:, j] = oracle.apply(L, bc, W, m0, e).reshape(-1)
        e.reshape(-1)[j] = 0
    return M


def test_bicgstab_matches_dense_lu():
    L = (3, 3, 3, 4)
    U = synth.random_su3_links(L, 0.4, 1)
    W = oracle.build_hops(L, U)
    b = synth.z2_spinor(L, 1, 2)[0]
    x, st, it, tr = oracle.bicgstab(L, AP, W, -0.05, b, tol=1e-12)
    assert st == 0 and tr <= 1e-12
    xd = np.linalg.solve(_dense(L, AP, W, -0.05), b.reshape(-1)).reshape(b.shape)
    assert np.abs(x - xd).max() <= 1e-10 * np.abs(xd).max()


def test_bicgstab_singular_operator_reports_nonconvergence():
    """Free field, fully periodic, m0 = 0 has an exact zero mode at k = 0: the
    solve must stop at maxit with a non-convergence status instead of hanging."""
    L = (3, 3, 3, 3)
    W = oracle.build_hops(L, synth.unit_links(L))
    b = np.ones((synth.volume(L), 4, 3), complex)  # k = 0 mode only
    x, st, it, tr = oracle.bicgstab(L, (1, 1, 1, 1), W, 0.0, b, tol=1e-10, maxit=50)
    assert st != 0
    assert it <= 50


def test_zero_source():
    L = (3, 3, 3, 3)
    W = oracle.build_hops(L, synth.random_su3_links(L, 0.3, 3))
    b = np.zeros((synth.volume(L), 4, 3), complex)
    x, st, it, tr = oracle.bicgstab(L, AP, W, 0.0, b)
    assert st == 0 and np.all(x == 0)


def _f(L, U, chi, psi, m0):
    W = oracle.build_hops(L, U)
    return float(np.real(np.vdot(chi, oracle.apply(L, AP, W, m0, psi))))


def test_force_against_central_differences():
    """d Re(chi^dagger D[U] psi)/dU, U unconstrained, eps = 1e-5 (config of the
    adjoint workload), on random (site, mu, entry, Re/Im) coordinates."""
    L = (3, 3, 3, 3)
    U = synth.random_su3_links(L, 0.3, 4)
    chi, psi = synth.gaussian_spinor(L, 2, 5)
    m0 = 0.0
    G = oracle.force(L, AP, U, m0, chi, psi)
    rng = np.random.default_rng(6)
    eps = 1e-5
    for _ in range(16):
        s = int(rng.integers(0, synth.volume(L)))
        mu = int(rng.integers(0, 4))
        i, j = (int(t) for t in rng.integers(0, 3, size=2))
        for part, unit in (("re", 1.0), ("im", 1j)):
            Up = U.copy()
            Um = U.copy()
            Up[s, mu, i, j] += eps * unit
            Um[s, mu, i, j] -= eps * unit
            fd = (_f(L, Up, chi, psi, m0) - _f(L, Um, chi, psi, m0)) / (2 * eps)
            an = G[s, mu, i, j].real if part == "re" else G[s, mu, i, j].imag
            assert abs(fd - an) <= 1e-8 * max(1.0, np.abs(G).max()), (s, mu, i, j, part, fd, an)


def test_force_is_linear_in_chi_and_psi():
    L = (3, 3, 3, 3)
    U = synth.random_su3_links(L, 0.3, 7)
    chi, psi, eta = synth.gaussian_spinor(L, 3, 8)
    G1 = oracle.force(L, AP, U, 0.0, chi, psi)
    G2 = oracle.force(L, AP, U, 0.0, chi, eta)
    G3 = oracle.force(L, AP, U, 0.0, chi, psi + 2 * eta)
    assert np.abs(G3 - (G1 + 2 * G2)).max() < 1e-12
