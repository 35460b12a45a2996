"""Other members of the rho/lambda class of Sec. 8 on the GPU (Wilson and
hypercube columns of Tab. rholambda) against the oracle with the same
weights, the library dot product, and the largest eigenvalue of D^dagger D in
the free field (the bound behind the footnote of Sec. 6.4: the Brillouin
operator's spectrum is far narrower than Wilson's)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1012_3615_gb300 import Brillouin, synth
from paper_1012_3615_gb300.core import WEIGHTS

pytestmark = pytest.mark.gpu
AP = (1, 1, 1, -1)


@pytest.mark.parametrize("name", ["wilson", "hypercube", "brillouin"])
def test_weight_columns_match_oracle(gpu, oracle_weights, name):
    lam, rho = WEIGHTS[name]
    oracle_weights(lam, rho)
    L = (4, 3, 5, 6)
    U = synth.random_su3_links(L, 0.4, 61)
    psi = synth.gaussian_spinor(L, 2, 62)
    W = oracle.build_hops(L, U)
    op = Brillouin(L, AP)
    op.set_weights(lam, rho)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f32", comp="full")
    x64 = torch.as_tensor(psi, device=gpu)
    x32 = torch.as_tensor(psi.astype(np.complex64), device=gpu)
    for dag in (False, True):
        o64 = op.apply(x64, 0.03, dagger=dag).cpu().numpy()
        o32 = op.apply(x32, 0.03, dagger=dag, prec="f32").cpu().numpy()
        for r in range(2):
            ref = oracle.apply(L, AP, W, 0.03, psi[r], dagger=dag)
            assert np.abs(o64[r] - ref).max() <= 1e-13 * np.abs(ref).max()
            assert np.abs(o32[r] - ref).max() <= 1e-6 * np.abs(ref).max()
    got = op.weights()
    assert np.allclose(got[0], lam) and np.allclose(got[1][1:], rho[1:])


def test_wilson_solve_and_force(gpu, oracle_weights):
    lam, rho = WEIGHTS["wilson"]
    oracle_weights(lam, rho)
    L = (4, 4, 4, 4)
    U = synth.random_su3_links(L, 0.3, 63)
    b = synth.z2_spinor(L, 1, 64)
    op = Brillouin(L, AP)
    op.set_weights(lam, rho)
    op.build_hops(torch.as_tensor(U, device=gpu))
    x, info = op.solve(torch.as_tensor(b, device=gpu), m0=0.2, tol=1e-10, mode=0)
    assert info[0]["status"] == "BRI_OK"
    W = oracle.build_hops(L, U)
    r = b[0] - oracle.apply(L, AP, W, 0.2, x.cpu().numpy()[0])
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b[0])
    chi, psi = synth.gaussian_spinor((3, 3, 3, 3), 2, 65)
    U3 = synth.random_su3_links((3, 3, 3, 3), 0.3, 66)
    op3 = Brillouin((3, 3, 3, 3), AP)
    op3.set_weights(lam, rho)
    op3.build_hops(torch.as_tensor(U3, device=gpu))
    dU = op3.force(torch.as_tensor(chi, device=gpu), torch.as_tensor(psi, device=gpu)).cpu().numpy()
    ref = oracle.force((3, 3, 3, 3), AP, U3, 0.0, chi, psi)
    assert np.abs(dU - ref).max() <= 1e-10 * np.abs(ref).max()


def test_cdot(gpu):
    L = (4, 3, 3, 4)
    a, b = synth.gaussian_spinor(L, 2, 67)
    op = Brillouin(L, AP)
    ref = np.vdot(a, b)
    assert abs(op.cdot(torch.as_tensor(a, device=gpu), torch.as_tensor(b, device=gpu)) - ref) < 1e-10 * abs(ref)
    a32 = torch.as_tensor(a.astype(np.complex64), device=gpu)
    b32 = torch.as_tensor(b.astype(np.complex64), device=gpu)
    ref32 = np.vdot(a.astype(np.complex64).astype(np.complex128), b.astype(np.complex64).astype(np.complex128))
    assert abs(op.cdot(a32, b32, prec="f32") - ref32) < 1e-10 * abs(ref32)


def _free_max_symbol2(L, lam, rho):
    """max over the lattice momenta of |D(k)|^2 at m0 = 0 from the class form
    D(k) = lambda(k) + i sum_mu gamma_mu rho_mu(k) (periodic lattice)."""
    ks = np.stack(np.meshgrid(*[2 * np.pi * np.arange(n) / n for n in L], indexing="ij"), -1).reshape(-1, 4)
    best = 0.0
    offs = np.array([[(k // 3 ** m) % 3 - 1 for m in range(4)] for k in range(81)])
    cls = np.abs(offs).sum(1)
    ph = np.exp(1j * ks @ offs.T)  # (nk, 81)
    lk = (ph * np.array([lam[c] for c in cls])).sum(1).real
    rk = [(ph * np.array([rho[c] if c else 0 for c in cls]) * offs[:, mu]).sum(1) for mu in range(4)]
    s2 = sum(np.abs(r) ** 2 for r in rk)  # (i rho_mu(k) is real times i)
    return float(np.max(lk ** 2 + s2))


def _power_iteration(op, iters, m0, prec, seed=0):
    """largest eigenvalue of D^dagger D: applies and dot products in the
    library, the normalisation and the Rayleigh quotient here"""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    x = torch.complex(torch.randn((1, op.V, 4, 3), generator=g, device="cuda"),
                      torch.randn((1, op.V, 4, 3), generator=g, device="cuda"))
    y = torch.empty_like(x)
    lam = 0.0
    for _ in range(iters):
        x = x / op.cdot(x, x, prec).real ** 0.5
        op.apply(x, m0, prec=prec, out=y)
        z = op.apply(y, m0, dagger=True, prec=prec)
        lam = op.cdot(x, z, prec).real
        x = z
    return lam


@pytest.mark.parametrize("name,expect", [("brillouin", 4.12), ("wilson", 64.0)])
def test_free_field_largest_eigenvalue(gpu, name, expect):
    L = (8, 8, 8, 8)
    lam, rho = WEIGHTS[name]
    op = Brillouin(L, (1, 1, 1, 1))
    op.set_weights(lam, rho)
    op.build_hops(torch.as_tensor(synth.unit_links(L), device=gpu), prec="f32", comp="full")
    got = _power_iteration(op, 400, 0.0, "f32")
    exact = _free_max_symbol2(L, lam, rho)
    assert abs(exact - expect) < 0.01 * expect
    # the Rayleigh quotient approaches the top from below; the Brillouin
    # spectrum is flat near its top (next values 4.1139, 4.1111), so 400 steps
    # leave it within about 3e-4 of the maximum
    assert exact * (1 - 2e-3) <= got <= exact * (1 + 1e-5)
