"""Pins of the oracle's APE smearing (Eq. def_ape) and clover term (Eq.
def_pref, Sec. 1: sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], F the hermitian
clover-leaf field strength).

APE: alpha = 0 is the identity, the result is special unitary, gauge
covariant, and to first order in the algebra (U = exp(i eps H), eps -> 0) it
is the linear smoothing (1 - alpha) H_mu(x) + alpha/6 sum over the six
staples of their three link generators.  Clover: a constant abelian flux
through the (0, 1) planes gives F_01 = diag(sin(Phi q)) exactly and every
other F zero; F is hermitian and gauge covariant; D with the clover term
stays gamma5-hermitian."""
import numpy as np
import pytest

import oracle
from paper_1012_3615_gb300 import synth

AP = (1, 1, 1, -1)


def _sites(L):
    V = int(np.prod(L))
    s = np.arange(V)
    x = np.stack([(s // int(np.prod(L[:m]))) % L[m] for m in range(4)], 1)
    return x


def _index(L, x):
    x = np.mod(x, L)
    return x[:, 0] + L[0] * (x[:, 1] + L[1] * (x[:, 2] + L[2] * x[:, 3]))


def _shift(L, mu, s):
    x = _sites(L)
    x[:, mu] += s
    return _index(L, x)


def _gauge_rotate(L, U, g):
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[:, mu] = g @ U[:, mu] @ g[_shift(L, mu, 1)].conj().transpose(0, 2, 1)
    return Ug


def test_ape_identity_and_unitarity():
    L = (3, 3, 3, 4)
    U = synth.random_su3_links(L, 0.5, 31)
    assert np.abs(oracle.ape_smear(L, U, 0.0) - U).max() == 0.0
    V = oracle.ape_smear(L, U, 0.72, 3)
    assert np.abs(V @ V.conj().transpose(0, 1, 3, 2) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(V) - 1).max() < 1e-13
    assert np.abs(V - U).max() > 0.05  # it does smooth


def test_ape_gauge_covariance():
    L = (3, 4, 3, 3)
    U = synth.random_su3_links(L, 0.6, 32)
    g = synth.gauge_transform(L, 33)
    lhs = oracle.ape_smear(L, _gauge_rotate(L, U, g), 0.72, 2)
    rhs = _gauge_rotate(L, oracle.ape_smear(L, U, 0.72, 2), g)
    assert np.abs(lhs - rhs).max() < 1e-12


def _log_unitary(U):
    w, Q = np.linalg.eig(U)
    return (Q * np.angle(w)[..., None, :]) @ np.linalg.inv(Q)


def test_ape_first_order_smoothing():
    L = (3, 3, 4, 3)
    eps, alpha = 1e-6, 0.72
    U = synth.random_su3_links(L, eps, 34)
    H = _log_unitary(U) / eps  # U = exp(i eps H)
    V = oracle.ape_smear(L, U, alpha)
    for mu in range(4):
        h = (1 - alpha) * H[:, mu]
        for nu in range(4):
            if nu == mu:
                continue
            up = H[:, nu] + H[_shift(L, nu, 1), mu] - H[_shift(L, mu, 1), nu]
            xm = _shift(L, nu, -1)
            x = _sites(L)
            x[:, nu] -= 1
            x[:, mu] += 1
            dn = -H[xm, nu] + H[xm, mu] + H[_index(L, x), nu]
            h = h + alpha / 6 * (up + dn)
        got = (V[:, mu] - np.eye(3)) / (1j * eps)
        assert np.abs(got - h).max() < 1e-4 * np.abs(h).max()


def _flux_links(L, k=1):
    """U_1(x) = diag(e^{i Phi q x_0}), U_0(x) = diag(e^{-i Phi q L_0 x_1}) on
    x_0 = L_0 - 1 (1 elsewhere), U_2 = U_3 = 1, q = (1, 1, -2),
    Phi = 2 pi k / (L_0 L_1): every (0, 1) plaquette equals diag(e^{i Phi q})."""
    q = np.array([1.0, 1.0, -2.0])
    phi = 2 * np.pi * k / (L[0] * L[1])
    x = _sites(L)
    U = synth.unit_links(L).copy()
    U[:, 1] = np.einsum("xc,cd->xcd", np.exp(1j * phi * np.outer(x[:, 0], q)), np.eye(3))
    edge = x[:, 0] == L[0] - 1
    U0 = np.einsum("xc,cd->xcd", np.exp(-1j * phi * L[0] * np.outer(x[:, 1], q)), np.eye(3))
    U[edge, 0] = U0[edge]
    return U, phi, q


@pytest.mark.parametrize("k", [1, 2])
def test_clover_constant_flux(k):
    L = (4, 3, 3, 3)
    U, phi, q = _flux_links(L, k)
    F = oracle.clover_field(L, U)
    want = np.diag(np.sin(phi * q))
    assert np.abs(F[:, 0] - want).max() < 1e-14
    assert np.abs(F[:, 1:]).max() < 1e-14
    # the clover term on a spinor: -(c_SW/2) sigma_01 (x) F_01
    g0, g1 = oracle.gamma(0), oracle.gamma(1)
    sig01 = 0.5j * (g0 @ g1 - g1 @ g0)
    W = oracle.build_hops(L, U)
    psi = synth.gaussian_spinor(L, 1, 35)[0]
    diff = oracle.apply_clover(L, AP, W, U, 0.1, 1.0, psi) - oracle.apply(L, AP, W, 0.1, psi)
    expect = -0.5 * np.einsum("ab,cd,xbd->xac", sig01, want, psi)
    assert np.abs(diff - expect).max() < 1e-14


def test_clover_hermitian_covariant_and_gamma5_hermitian():
    L = (3, 3, 4, 3)
    U = synth.random_su3_links(L, 0.5, 36)
    F = oracle.clover_field(L, U)
    assert np.abs(F - F.conj().transpose(0, 1, 3, 2)).max() < 1e-15
    g = synth.gauge_transform(L, 37)
    Fg = oracle.clover_field(L, _gauge_rotate(L, U, g))
    assert np.abs(Fg - g[:, None] @ F @ g[:, None].conj().transpose(0, 1, 3, 2)).max() < 1e-13
    W = oracle.build_hops(L, U)
    psi, phi = synth.gaussian_spinor(L, 2, 38)
    g5 = oracle.gamma(4)
    Dpsi = oracle.apply_clover(L, AP, W, U, -0.1, 1.0, psi)
    Dphi = oracle.apply_clover(L, AP, W, U, -0.1, 1.0, phi)
    lhs = np.vdot(phi, np.einsum("ab,xbc->xac", g5, oracle.apply_clover(
        L, AP, W, U, -0.1, 1.0, np.einsum("ab,xbc->xac", g5, psi))))
    rhs = np.vdot(Dphi, psi)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    # dagger path: D^dagger = adjoint stencil + the same hermitian clover term
    Dd = oracle.apply_clover(L, AP, W, U, -0.1, 1.0, phi, dagger=True)
    assert abs(np.vdot(Dd, psi) - np.vdot(phi, Dpsi)) < 1e-12 * abs(np.vdot(phi, Dpsi))
