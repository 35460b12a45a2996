"""APE smearing (Eq. def_ape) and the clover term of Eq. def_pref on the GPU
against the oracle: smeared links, the operator with the clover term in every
precision and mode, solves with it, the constant-flux closed form at a size
beyond the oracle's reach, switching the term off, and the force refusing it."""
import numpy as np
import pytest
import torch

import oracle
from paper_1012_3615_gb300 import Brillouin, synth
from paper_1012_3615_gb300.core import BriError

pytestmark = pytest.mark.gpu
AP = (1, 1, 1, -1)


@pytest.mark.parametrize("nsteps", [1, 2, 3])
def test_ape_matches_oracle(gpu, nsteps):
    L = (3, 3, 4, 3)
    U = synth.random_su3_links(L, 0.6, 41)
    ref = oracle.ape_smear(L, U, 0.72, nsteps)
    op = Brillouin(L, AP)
    got = op.ape_smear(torch.as_tensor(U, device=gpu), 0.72, nsteps).cpu().numpy()
    assert np.abs(got - ref).max() < 1e-12


@pytest.fixture(scope="module")
def clover_case():
    L = (4, 3, 3, 4)
    U0 = synth.random_su3_links(L, 0.5, 42)
    V = oracle.ape_smear(L, U0, 0.72, 1)
    psi = synth.gaussian_spinor(L, 2, 43)
    return L, V, oracle.build_hops(L, V), psi


def test_clover_apply_matches_oracle(gpu, clover_case):
    L, V, W, psi = clover_case
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(V, device=gpu), prec="f32", comp="full")
    op.store_hops("f32", "2row")
    op.set_clover(1.0)
    x64 = torch.as_tensor(psi, device=gpu)
    x32 = torch.as_tensor(psi.astype(np.complex64), device=gpu)
    g5 = oracle.gamma(4)
    for dag in (False, True):
        ref = [oracle.apply_clover(L, AP, W, V, 0.05, 1.0, psi[r], dagger=dag) for r in range(2)]
        o64 = op.apply(x64, 0.05, dagger=dag).cpu().numpy()
        o32 = op.apply(x32, 0.05, dagger=dag, prec="f32").cpu().numpy()
        for r in range(2):
            assert np.abs(o64[r] - ref[r]).max() <= 1e-13 * np.abs(ref[r]).max()
            assert np.abs(o32[r] - ref[r]).max() <= 1e-6 * np.abs(ref[r]).max()
    # the shifted hermitian kernel gamma5 (D - rho) includes the term too
    h = op.overlap_kernel(x64, 1.0).cpu().numpy()
    for r in range(2):
        ref = np.einsum("ab,xbc->xac", g5, oracle.apply_clover(L, AP, W, V, -1.0, 1.0, psi[r]))
        assert np.abs(h[r] - ref).max() <= 1e-13 * np.abs(ref).max()


def test_clover_off_restores_operator(gpu, clover_case):
    L, V, W, psi = clover_case
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(V, device=gpu))
    x = torch.as_tensor(psi, device=gpu)
    plain = op.apply(x, 0.1)
    op.set_clover(1.0)
    with_c = op.apply(x, 0.1)
    op.set_clover(0.0)
    assert torch.equal(op.apply(x, 0.1), plain)
    assert (with_c - plain).abs().max().item() > 1e-3


@pytest.mark.parametrize("mode", [0, 1])
def test_solve_with_clover(gpu, clover_case, mode):
    L, V, W, _ = clover_case
    b = synth.z2_spinor(L, 1, 44)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(V, device=gpu), prec="f32", comp="2row")
    op.set_clover(1.0)
    x, info = op.solve(torch.as_tensor(b, device=gpu), m0=0.05, tol=1e-10, mode=mode)
    assert info[0]["status"] == "BRI_OK", info
    r = b[0] - oracle.apply_clover(L, AP, W, V, 0.05, 1.0, x.cpu().numpy()[0])
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b[0])


def test_constant_flux_closed_form_8x8x8x8(gpu):
    """Abelian flux Phi q through every (0,1) plaquette: the clover term is
    -(c_SW/2) sigma_01 (x) diag(sin(Phi q)) at every site (free hops unchanged
    in the other planes), checked as D(c_SW) psi - D(0) psi at a size the
    oracle does not reach."""
    L = (8, 8, 8, 8)
    q = np.array([1.0, 1.0, -2.0])
    phi = 2 * np.pi / 64
    V = int(np.prod(L))
    s = np.arange(V)
    x0, x1 = s % 8, (s // 8) % 8
    U = synth.unit_links(L).copy()
    U[:, 1] = np.einsum("xc,cd->xcd", np.exp(1j * phi * np.outer(x0, q)), np.eye(3))
    edge = x0 == 7
    U[edge, 0] = np.einsum("xc,cd->xcd", np.exp(-1j * phi * 8 * np.outer(x1[edge], q)), np.eye(3))
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu))
    psi = torch.as_tensor(synth.gaussian_spinor(L, 1, 45), device=gpu)
    d0 = op.apply(psi, 0.0)
    op.set_clover(1.3)
    diff = (op.apply(psi, 0.0) - d0).cpu().numpy()[0]
    g0, g1 = oracle.gamma(0), oracle.gamma(1)
    sig01 = 0.5j * (g0 @ g1 - g1 @ g0)
    want = -0.65 * np.einsum("ab,cd,xbd->xac", sig01, np.diag(np.sin(phi * q)), psi.cpu().numpy()[0])
    assert np.abs(diff - want).max() < 1e-13


def test_force_refuses_clover(gpu, clover_case):
    L, V, W, psi = clover_case
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(V, device=gpu))
    op.set_clover(1.0)
    x = torch.as_tensor(psi[0], device=gpu)
    with pytest.raises(BriError):
        op.force(x, x)


def test_overlap_with_clover_kernel_ginsparg_wilson(gpu, clover_case):
    L, V, W, psi = clover_case
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(V, device=gpu))
    op.set_clover(1.0)
    info = op.overlap_setup(rho=1.0, nlow=4, eps=1e-10, max_krylov=1000, tol=1e-10)
    assert info["status"] == "BRI_OK", info
    x = torch.as_tensor(psi[:1], device=gpu)
    g5 = torch.tensor([1, 1, -1, -1], dtype=torch.complex128, device=gpu).view(1, 1, 4, 1)
    Dx = op.overlap(x)
    viol = (g5 * Dx + op.overlap(g5 * x) - op.overlap(g5 * Dx)).norm().item() / x.norm().item()
    assert viol < 1e-8
