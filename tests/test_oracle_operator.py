"""Pins of the oracle's hop construction and of the operator itself:
free-field momentum-space forms (Eq. def_4Dbri, App. C), the doubler lift of
Sec. 8, path counts and a dynamic-programming path sum (Sec. 5.1), constant
abelian and pure-gauge backgrounds, gauge covariance, gamma5-hermiticity
(Sec. 1) and the overlap kernel of Sec. 7.4."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1012_3615_gb300 import synth

AP = (1, 1, 1, -1)  # antiperiodic in t for the fermion field
PER = (1, 1, 1, 1)


def _free_symbol(k, m0):
    """4x4 spin matrix of D in momentum space, from the printed closed forms:
    -(1/2) Lap^bri = 2 - 2 prod cos^2(k/2)  and
    nabla^iso_mu = i sin k_mu prod_{nu != mu} (cos k_nu + 2) / 27."""
    k = np.asarray(k, dtype=float)
    lap = 4 * np.prod(np.cos(k / 2) ** 2) - 4
    M = (m0 - 0.5 * lap) * np.eye(4, dtype=complex)
    for mu in range(4):
        other = np.prod([np.cos(k[nu]) + 2 for nu in range(4) if nu != mu])
        M = M + 1j * np.sin(k[mu]) * other / 27 * oracle.gamma(mu)
    return M


def _momenta(L, bc, rng, n):
    out = []
    for _ in range(n):
        k = []
        for mu in range(4):
            j = int(rng.integers(0, L[mu]))
            k.append((2 * j + (1 if bc[mu] < 0 else 0)) * np.pi / L[mu])
        out.append(k)
    return out


@pytest.mark.parametrize("L,bc", [((4, 4, 4, 4), AP), ((3, 5, 4, 6), AP), ((4, 3, 3, 4), PER)])
def test_free_field_plane_waves(L, bc):
    U = synth.unit_links(L)
    W = oracle.build_hops(L, U)
    rng = np.random.default_rng(sum(L))
    for k in _momenta(L, bc, rng, 6):
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = synth.plane_wave(L, k, u)
        m0 = float(rng.uniform(-0.3, 0.3))
        out = oracle.apply(L, bc, W, m0, psi)
        expect = synth.plane_wave(L, k, _free_symbol(k, m0) @ u)
        assert np.abs(out - expect).max() < 1e-13 * np.abs(expect).max()


def test_free_field_worked_value():
    """8^4, antiperiodic t, k = (2pi/8, 0, 6pi/8, pi/8): scalar part of the symbol
    -(1/2)a^2 Lap^bri and the four derivative components evaluated from the
    closed forms (values recorded with the inputs in this test)."""
    k = np.array([2 * np.pi / 8, 0, 6 * np.pi / 8, np.pi / 8])
    lap_part = 2 - 2 * np.prod(np.cos(k / 2) ** 2)
    assert abs(lap_part - 1.759515058436089) < 1e-14
    L = (8, 8, 8, 8)
    W = oracle.build_hops(L, synth.unit_links(L))
    u = np.zeros((4, 3), complex)
    u[0, 0] = 1
    psi = synth.plane_wave(L, k, u)
    out = oracle.apply(L, AP, W, 0.0, psi)
    M = out[0] / psi[0, 0, 0]
    assert abs(M[0, 0] - lap_part) < 1e-13
    # derivative part on spin component 0 -> rows of gamma_mu acting on e_0
    nab = [np.sin(k[mu]) * np.prod([np.cos(k[nu]) + 2 for nu in range(4) if nu != mu]) / 27
           for mu in range(4)]
    assert np.allclose(nab, [0.297005591485214, 0, 0.621881095097579, 0.148821334808646], atol=1e-14)
    expect_col = 1j * sum(nab[mu] * oracle.gamma(mu)[:, 0] for mu in range(4))
    assert np.allclose(M[1:, 0], expect_col[1:], atol=1e-13)


def test_doublers_lifted_to_two():
    """Sec. 8: at k in {0, pi}^4 \\ {0} the free operator equals m0 + 2."""
    L = (4, 4, 4, 4)
    W = oracle.build_hops(L, synth.unit_links(L))
    rng = np.random.default_rng(5)
    for corner in itertools.product([0, 1], repeat=4):
        if not any(corner):
            continue
        k = np.pi * np.array(corner, float)
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = synth.plane_wave(L, k, u)
        out = oracle.apply(L, PER, W, 0.1, psi)
        assert np.abs(out - 2.1 * psi).max() < 1e-13


def test_path_counts():
    """1, 2, 6, 24 shortest paths for 1-, 2-, 3-, 4-hop offsets (Sec. 5.1)."""
    L = (3, 3, 3, 3)
    U = synth.random_su3_links(L, 0.3, 1)
    for d, n in [((1, 0, 0, 0), 1), ((1, -1, 0, 0), 2), ((0, 1, 1, -1), 6), ((1, 1, -1, 1), 24)]:
        _, cnt = oracle.path_sum(L, U, 5, d)
        assert cnt == n


def _dp_path_sums(L, U):
    """Path sums for every offset by the recursion over the first step,
    A_d(x) = sum_{mu in supp d} U_{s mu}(x) A_{d - s mu}(x + s mu)  (numpy)."""
    V = synth.volume(L)
    x = synth.coordinates(L)

    def nb(mu, s):
        y = x.copy()
        y[:, mu] = (y[:, mu] + s) % L[mu]
        return y[:, 0] + L[0] * (y[:, 1] + L[1] * (y[:, 2] + L[2] * y[:, 3]))

    A = {}
    for d in itertools.product([-1, 0, 1], repeat=4):
        n = sum(abs(t) for t in d)
        if n == 0:
            A[d] = np.broadcast_to(np.eye(3, dtype=complex), (V, 3, 3)).copy()
    for n in range(1, 5):
        for d in itertools.product([-1, 0, 1], repeat=4):
            if sum(abs(t) for t in d) != n:
                continue
            acc = np.zeros((V, 3, 3), complex)
            for mu in range(4):
                if d[mu] == 0:
                    continue
                s = d[mu]
                rest = list(d)
                rest[mu] = 0
                first = U[:, mu] if s > 0 else U[nb(mu, -1), mu].conj().transpose(0, 2, 1)
                acc += first @ A[tuple(rest)][nb(mu, s)]
            A[d] = acc
    return A


def test_path_enumeration_equals_recursion():
    for L in [(3, 3, 3, 3), (4, 3, 4, 3)]:
        U = synth.random_su3_links(L, 0.5, 2)
        A = _dp_path_sums(L, U)
        for site in [0, 7, synth.volume(L) - 1]:
            for d in [(1, 1, 0, 0), (-1, 0, 1, 1), (1, -1, -1, 1), (0, -1, 0, -1)]:
                got, _ = oracle.path_sum(L, U, site, d)
                assert np.abs(got - A[d][site]).max() < 1e-13


def test_hops_are_projected_path_sums_and_reverse_relation():
    L = (3, 4, 3, 3)
    U = synth.random_su3_links(L, 0.4, 3)
    W = oracle.build_hops(L, U)
    A = _dp_path_sums(L, U)
    x = synth.coordinates(L)
    for d, Ad in A.items():
        n = sum(abs(t) for t in d)
        k = oracle.offset_index(d)
        if n == 0:
            continue
        if n == 1:
            assert np.abs(W[:, k] - Ad).max() < 1e-15
            continue
        idx = [0, 5, 17, synth.volume(L) - 1]
        assert np.abs(W[idx, k] - oracle.project_su3(Ad[idx])).max() < 1e-13
        # W_{-d}(x) = W_d(x-d)^dagger
        y = (x - np.array(d)) % np.array(L)
        yi = y[:, 0] + L[0] * (y[:, 1] + L[1] * (y[:, 2] + L[2] * y[:, 3]))
        kk = oracle.offset_index([-t for t in d])
        assert np.abs(W[:, kk] - W[yi, k].conj().transpose(0, 2, 1)).max() < 1e-13


def test_constant_abelian_background():
    """Constant diagonal links U_mu = diag(exp(i a_mu^c)), sum_c a_mu^c = 0: all
    paths commute, W_d = prod_mu U_mu^{d_mu}, and D acts on colour c like the
    free operator at momentum k + a^c."""
    L = (4, 4, 4, 4)
    rng = np.random.default_rng(11)
    a = rng.uniform(-0.6, 0.6, size=(4, 3))
    a[:, 2] = -a[:, 0] - a[:, 1]
    U = np.zeros((synth.volume(L), 4, 3, 3), complex)
    for mu in range(4):
        U[:, mu] = np.diag(np.exp(1j * a[mu]))
    W = oracle.build_hops(L, U)
    for k in _momenta(L, AP, rng, 4):
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = synth.plane_wave(L, k, u)
        out = oracle.apply(L, AP, W, 0.05, psi)
        expect = np.zeros((4, 3), complex)
        for c in range(3):
            expect[:, c] = _free_symbol(np.array(k) + a[:, c], 0.05) @ u[:, c]
        assert np.abs(out - synth.plane_wave(L, k, expect)).max() < 1e-13


def _gauge_rotate(L, U, g):
    x = synth.coordinates(L)
    Ug = np.empty_like(U)
    for mu in range(4):
        y = x.copy()
        y[:, mu] = (y[:, mu] + 1) % L[mu]
        yi = y[:, 0] + L[0] * (y[:, 1] + L[1] * (y[:, 2] + L[2] * y[:, 3]))
        Ug[:, mu] = g @ U[:, mu] @ g[yi].conj().transpose(0, 2, 1)
    return Ug


def test_pure_gauge_equals_rotated_free_operator():
    L = (4, 3, 3, 4)
    g = synth.gauge_transform(L, 21)
    U = _gauge_rotate(L, synth.unit_links(L), g)  # U_mu(x) = g(x) g(x+mu)^dagger
    W = oracle.build_hops(L, U)
    Wf = oracle.build_hops(L, synth.unit_links(L))
    psi = synth.gaussian_spinor(L, 1, 4)[0]
    gd = g.conj().transpose(0, 2, 1)
    lhs = oracle.apply(L, AP, W, 0.2, psi)
    rhs = np.einsum("xab,xsb->xsa", g, oracle.apply(L, AP, Wf, 0.2, np.einsum("xab,xsb->xsa", gd, psi)))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_gauge_covariance_random_links():
    L = (3, 4, 3, 4)
    U = synth.random_su3_links(L, 0.4, 5)
    g = synth.gauge_transform(L, 6)
    psi = synth.gaussian_spinor(L, 1, 7)[0]
    W = oracle.build_hops(L, U)
    Wg = oracle.build_hops(L, _gauge_rotate(L, U, g))
    gpsi = np.einsum("xab,xsb->xsa", g, psi)
    lhs = oracle.apply(L, AP, Wg, -0.1, gpsi)
    rhs = np.einsum("xab,xsb->xsa", g, oracle.apply(L, AP, W, -0.1, psi))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_gamma5_hermiticity_and_adjoint():
    """gamma5 D gamma5 = D^dagger (Sec. 1); the oracle's D^dagger is the literal
    adjoint, so both the identity and <phi, D psi> = <D^dagger phi, psi> are checked."""
    L = (3, 3, 4, 4)
    U = synth.random_su3_links(L, 0.5, 8)
    W = oracle.build_hops(L, U)
    psi, phi = synth.gaussian_spinor(L, 2, 9)
    g5 = oracle.gamma(4)
    D = lambda v: oracle.apply(L, AP, W, 0.03, v)
    Dd = lambda v: oracle.apply(L, AP, W, 0.03, v, dagger=True)
    G5 = lambda v: np.einsum("ab,xbc->xac", g5, v)
    assert np.abs(G5(D(G5(psi))) - Dd(psi)).max() < 1e-13
    assert abs(np.vdot(phi, D(psi)) - np.vdot(Dd(phi), psi)) < 1e-11


def test_overlap_kernel_hermitian_and_square():
    L = (3, 3, 3, 4)
    U = synth.random_su3_links(L, 0.5, 10)
    W = oracle.build_hops(L, U)
    psi, phi = synth.gaussian_spinor(L, 2, 11)
    H = lambda v: oracle.overlap_kernel(L, AP, W, 0.0, 1.0, v)
    assert abs(np.vdot(phi, H(psi)) - np.vdot(H(phi), psi)) < 1e-11
    # H^2 = (D - rho)^dagger (D - rho)
    Dm = lambda v: oracle.apply(L, AP, W, -1.0, v)
    Dmd = lambda v: oracle.apply(L, AP, W, -1.0, v, dagger=True)
    assert np.abs(H(H(psi)) - Dmd(Dm(psi))).max() < 1e-12
