"""Pins of the dense overlap oracle (Sec. 7.1, Eq. def_over, Eq. def_mass;
spectra of Sec. 7.4).

The free field is fixed in closed form: with unit links every plane wave
e^{ik.x} u is an eigenvector of D with the 4x4 spin symbol D(k) of the printed
momentum-space forms, so D_ov(k) = rho [1 + X(k) (X(k)^dagger X(k))^(-1/2)]
with X(k) = D(k) - rho, and the eigenvalues of D^dagger D are those of
X(k)^dagger X(k) over the lattice momenta.  On random links the overlap
operator must satisfy the Ginsparg-Wilson relation (Eq. def_ginswils), be
normal, have its massive spectrum on the circle stated with Eq. def_mass, and
the two forms of Eq. def_over must agree."""
import numpy as np
import pytest

import oracle
from oracle import overlap as ov
from paper_1012_3615_gb300 import synth

AP = (1, 1, 1, -1)
L3 = (3, 3, 3, 3)
WILSON = ((4.0, -0.5, 0.0, 0.0, 0.0), (0.0, 0.5, 0.0, 0.0, 0.0))


@pytest.fixture
def wilson_weights():
    oracle.set_weights(*WILSON)
    yield
    oracle.reset_weights()


def _brillouin_symbol(k, m0):
    """Spin symbol of the Brillouin operator from the closed forms
    -(1/2) Lap^bri = 2 - 2 prod cos^2(k/2), nabla^iso_mu = i sin k_mu
    prod_{nu != mu} (cos k_nu + 2) / 27."""
    k = np.asarray(k, float)
    M = (m0 + 2 - 2 * np.prod(np.cos(k / 2) ** 2)) * np.eye(4, dtype=complex)
    for mu in range(4):
        other = np.prod([np.cos(k[nu]) + 2 for nu in range(4) if nu != mu])
        M = M + 1j * np.sin(k[mu]) * other / 27 * oracle.gamma(mu)
    return M


def _wilson_symbol(k, m0):
    """Textbook Wilson symbol m0 + sum (1 - cos k) + i sum gamma_mu sin k_mu."""
    k = np.asarray(k, float)
    M = (m0 + np.sum(1 - np.cos(k))) * np.eye(4, dtype=complex)
    for mu in range(4):
        M = M + 1j * np.sin(k[mu]) * oracle.gamma(mu)
    return M


def _momenta(L, bc):
    axes = [[(2 * j + (1 if bc[mu] < 0 else 0)) * np.pi / L[mu] for j in range(L[mu])] for mu in range(4)]
    return [np.array(k) for k in np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 4)]


def _inv_sqrt_psd(M):
    w, Q = np.linalg.eigh(M)
    return (Q / np.sqrt(w)) @ Q.conj().T


def _plane_wave_check(Dov, L, bc, symbol, rho, rng):
    for k in _momenta(L, bc)[::7]:
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        X = symbol(k, -rho)
        Sym = rho * (np.eye(4) + X @ _inv_sqrt_psd(X.conj().T @ X))
        got = (Dov @ synth.plane_wave(L, k, u).reshape(-1)).reshape(-1, 4, 3)
        want = synth.plane_wave(L, k, Sym @ u)
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("rho", [1.0, 1.3])
def test_free_field_overlap_brillouin(rho):
    W = oracle.build_hops(L3, synth.unit_links(L3))
    Dov = ov.overlap_matrix(L3, AP, W, rho)
    _plane_wave_check(Dov, L3, AP, _brillouin_symbol, rho, np.random.default_rng(3))


def test_free_field_overlap_wilson(wilson_weights):
    W = oracle.build_hops(L3, synth.unit_links(L3))
    Dov = ov.overlap_matrix(L3, AP, W, 1.0)
    _plane_wave_check(Dov, L3, AP, _wilson_symbol, 1.0, np.random.default_rng(4))


@pytest.mark.parametrize("symbol,weights", [(_brillouin_symbol, None), (_wilson_symbol, WILSON)])
def test_free_field_ddag_d_spectrum(symbol, weights):
    """Eigenvalues of A = D^dagger D at m0 = -1 = the multiset of the spin
    symbol's |X(k)|^2 eigenvalues over all lattice momenta, three colours each."""
    if weights:
        oracle.set_weights(*weights)
    try:
        W = oracle.build_hops(L3, synth.unit_links(L3))
        got = ov.ddag_d_eigenvalues(L3, AP, W, -1.0)
    finally:
        oracle.reset_weights()
    want = []
    for k in _momenta(L3, AP):
        X = symbol(k, -1.0)
        want.extend(list(np.linalg.eigvalsh(X.conj().T @ X)) * 3)
    assert np.allclose(got, np.sort(want), rtol=1e-11, atol=1e-12)


@pytest.fixture(scope="module")
def random_case():
    L = (3, 3, 3, 4)
    W = oracle.build_hops(L, synth.random_su3_links(L, 0.5, 71))
    return L, W


@pytest.mark.parametrize("rho", [1.0, 1.4])
def test_ginsparg_wilson_and_normality(random_case, rho):
    L, W = random_case
    D = ov.overlap_matrix(L, AP, W, rho)
    G5 = ov.gamma5_matrix(L)
    gw = G5 @ D + D @ G5 - D @ G5 @ D / rho
    assert np.abs(gw).max() < 1e-11 * rho
    assert np.abs(D @ D.conj().T - D.conj().T @ D).max() < 1e-11 * rho ** 2
    assert np.abs(D - ov.overlap_matrix_invsqrt(L, AP, W, rho)).max() < 1e-11 * rho


def test_massive_spectrum_on_circle(random_case):
    L, W = random_case
    rho, m = 1.0, 0.12
    lam = np.linalg.eigvals(ov.overlap_matrix(L, AP, W, rho, m))
    assert np.abs(np.abs(lam - (rho + m / 2)) - (rho - m / 2)).max() < 1e-11


def test_kernel_spectra_consistent(random_case):
    """A = H^2 (gamma5^2 = 1): eigenvalues of D(-rho)^dagger D(-rho) are the
    squares of those of H; eigenpairs of H satisfy H v = lambda v."""
    L, W = random_case
    lamA = ov.ddag_d_eigenvalues(L, AP, W, -1.0)
    lamH, Q = ov.kernel_eigenpairs(L, AP, W, 1.0)
    assert np.allclose(np.sort(lamH ** 2), lamA, rtol=1e-11, atol=1e-13)
    H = ov.hermitian_kernel(L, AP, W, 1.0)
    assert np.abs(H @ Q[:, :5] - Q[:, :5] * lamH[:5]).max() < 1e-12
    assert np.all(np.diff(np.abs(lamH)) >= 0)
