"""The oracle with other members of the rho/lambda class of Sec. 8: Wilson's
column of Tab. rholambda must give the Wilson operator of Eq. def_wils
(free-field symbol m0 + sum_mu (1 - cos k_mu) + i sum_mu gamma_mu sin k_mu),
and the hypercube column must satisfy the two normalisation conditions of
Sec. 8 that all three columns obey."""
import os

import numpy as np
import pytest

import oracle
from paper_1012_3615_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _column(col):
    rows = {}
    for line in open(os.path.join(GOLD, "rholambda.txt")):
        line = line.split("#")[0].strip()
        if line:
            p = line.split()
            rows[p[0]] = p[1:]
    def val(t):
        if "/" in t:
            a, b = t.split("/")
            return float(a) / float(b)
        return float(t)
    lam = [val(rows["lambda%d" % n][col]) for n in range(5)]
    rho = [0.0] + [val(rows["rho%d" % n][col]) for n in range(1, 5)]
    return lam, rho


@pytest.fixture
def weights():
    yield
    oracle.reset_weights()


def test_wilson_column_is_the_wilson_operator(weights):
    lam, rho = _column(0)
    oracle.set_weights(lam, rho)
    L, bc = (4, 3, 5, 6), (1, 1, 1, -1)
    W = oracle.build_hops(L, synth.unit_links(L))
    rng = np.random.default_rng(3)
    for _ in range(5):
        k = np.array([2 * np.pi * rng.integers(0, L[m]) / L[m] for m in range(3)]
                     + [(2 * rng.integers(0, L[3]) + 1) * np.pi / L[3]])
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        m0 = 0.17
        M = (m0 + np.sum(1 - np.cos(k))) * np.eye(4, dtype=complex)
        for mu in range(4):
            M = M + 1j * np.sin(k[mu]) * oracle.gamma(mu)
        out = oracle.apply(L, bc, W, m0, synth.plane_wave(L, k, u))
        assert np.abs(out - synth.plane_wave(L, k, M @ u)).max() < 1e-13


def test_wilson_column_has_only_nearest_neighbour_hops(weights):
    """With Wilson's weights, D(x, y) vanishes unless |x - y|_1 <= 1 (random links)."""
    lam, rho = _column(0)
    oracle.set_weights(lam, rho)
    L, bc = (3, 3, 3, 4), (1, 1, 1, -1)
    W = oracle.build_hops(L, synth.random_su3_links(L, 0.5, 4))
    V = synth.volume(L)
    e = np.zeros((V, 4, 3), complex)
    src = 40
    e[src, 1, 2] = 1.0
    out = oracle.apply(L, bc, W, 0.0, e)
    x = synth.coordinates(L)
    d = (x - x[src] + np.array(L) // 2) % np.array(L) - np.array(L) // 2
    far = np.abs(d).sum(1) > 1
    assert np.abs(out[far]).max() == 0.0
    assert np.abs(out[~far]).max() > 0.1


def test_hypercube_column_normalisation():
    lam, rho = _column(1)
    assert abs(2 * rho[1] + 12 * rho[2] + 24 * rho[3] + 16 * rho[4] - 1) < 1e-7
    assert abs(lam[0] + 8 * lam[1] + 24 * lam[2] + 32 * lam[3] + 16 * lam[4]) < 1e-7


def test_reset_restores_brillouin(weights):
    oracle.set_weights([1, 2, 3, 4, 5], [0, 1, 1, 1, 1])
    oracle.reset_weights()
    lam, rho = oracle.weights()
    assert lam[0] == 240 / 128 and rho[1] == 64 / 432
