"""Pins of the oracle's stencil weights and gamma basis.

The weights must reproduce Tab. rholambda, the App. C stencil tables and the
linear constraints of Sec. 8; the gamma matrices must satisfy the Euclidean
Clifford algebra with hermitian gamma_mu.
"""
import os
from fractions import Fraction

import numpy as np

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_table(name):
    rows = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            parts = line.split()
            rows[parts[0]] = parts[1:]
    return rows


def _frac(s):
    return Fraction(s) if "." not in s else float(s)


def test_weights_equal_table_rholambda():
    tab = _read_table("rholambda.txt")
    lam, rho = oracle.weights()
    for n in range(1, 5):
        assert rho[n] == float(_frac(tab["rho%d" % n][2]))
    for n in range(5):
        assert lam[n] == float(_frac(tab["lambda%d" % n][2]))


def test_weights_equal_appendix_c_stencils():
    tab = _read_table("stencils_appC.txt")
    lam, rho = oracle.weights()
    lap = [Fraction(int(v), int(tab["lap_bri"][0])) for v in tab["lap_bri"][1:]]
    der = [Fraction(int(v), int(tab["der_iso"][0])) for v in tab["der_iso"][1:]]
    # D = sum gamma nabla^iso - (1/2) Laplacian^bri + m0  (Eq. def_pref)
    for n in range(5):
        assert abs(lam[n] - float(-lap[n] / 2)) < 1e-17
    for n in range(1, 5):
        assert abs(rho[n] - float(der[n])) < 1e-17


def test_weight_constraints_sec8():
    """All seven linear relations of Sec. 8, in exact rational arithmetic."""
    tab = _read_table("rholambda.txt")
    r = [None] + [_frac(tab["rho%d" % n][2]) for n in range(1, 5)]
    l = [_frac(tab["lambda%d" % n][2]) for n in range(5)]
    assert 2 * r[1] + 12 * r[2] + 24 * r[3] + 16 * r[4] == 1
    assert l[0] + 8 * l[1] + 24 * l[2] + 32 * l[3] + 16 * l[4] == 0
    assert l[0] + 4 * l[1] - 16 * l[3] - 16 * l[4] == 2
    assert l[0] - 8 * l[2] + 16 * l[4] == 2
    assert l[0] - 4 * l[1] + 16 * l[3] - 16 * l[4] == 2
    assert l[0] - 8 * l[1] + 24 * l[2] - 32 * l[3] + 16 * l[4] == 2
    assert 12 * r[2] + 48 * r[3] + 48 * r[4] - 1 == 0
    # the other two columns obey the first two relations as well
    for col in (0, 1):
        rr = [None] + [_frac(tab["rho%d" % n][col]) for n in range(1, 5)]
        ll = [_frac(tab["lambda%d" % n][col]) for n in range(5)]
        assert abs(float(2 * rr[1] + 12 * rr[2] + 24 * rr[3] + 16 * rr[4]) - 1) < 1e-7
        assert abs(float(ll[0] + 8 * ll[1] + 24 * ll[2] + 32 * ll[3] + 16 * ll[4])) < 1e-7  # nine printed decimals


def test_class_sizes():
    """8 / 24 / 32 / 16 offsets per hop class (the coefficients of Sec. 8)."""
    counts = [0] * 5
    for k in range(81):
        d = [(k // 3 ** m) % 3 - 1 for m in range(4)]
        counts[sum(abs(t) for t in d)] += 1
    assert counts == [1, 8, 24, 32, 16]


def test_gamma_algebra():
    g = [oracle.gamma(mu) for mu in range(4)]
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T, atol=0)
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2 * (a == b) * np.eye(4), atol=0)
    g5 = oracle.gamma(4)
    assert np.allclose(g5, g[0] @ g[1] @ g[2] @ g[3], atol=0)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=0)
    for a in range(4):
        assert np.allclose(g5 @ g[a] + g[a] @ g5, 0, atol=0)
