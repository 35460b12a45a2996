"""GPU fermion force (adjoint through the path sums of Sec. 5.1 and the
projection of Sec. 5.2) against the CPU oracle, and the autograd Function."""
import numpy as np
import pytest
import torch

import oracle
from paper_1012_3615_gb300 import Brillouin, DiracFunction, synth

pytestmark = pytest.mark.gpu
AP = (1, 1, 1, -1)


@pytest.mark.parametrize("L", [(3, 3, 3, 3), (4, 3, 3, 4)])
def test_force_matches_oracle(gpu, L):
    U = synth.random_su3_links(L, 0.3, 1)
    chi, psi = synth.gaussian_spinor(L, 2, 2)
    ref = oracle.force(L, AP, U, 0.0, chi, psi)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu))
    dU = op.force(torch.as_tensor(chi, device=gpu), torch.as_tensor(psi, device=gpu)).cpu().numpy()
    assert np.abs(dU - ref).max() <= 1e-10 * np.abs(ref).max()


def test_force_accumulates(gpu):
    L = (3, 3, 3, 3)
    U = synth.random_su3_links(L, 0.3, 3)
    chi, psi = synth.gaussian_spinor(L, 2, 4)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu))
    c, p = torch.as_tensor(chi, device=gpu), torch.as_tensor(psi, device=gpu)
    a = op.force(c, p)
    b = op.force(c, p, dU=a.clone())
    assert torch.allclose(b, 2 * a, rtol=0, atol=1e-13 * a.abs().max().item())


@pytest.mark.parametrize("f32", [False, True])
def test_force_inverse_matches_oracle(gpu, f32):
    """d(phi^dagger (D^dagger D)^{-1} phi)/dU = -2 d Re(Y^dagger D X)/dU; with FP32
    fields stored the two solves run as FP64 defect correction."""
    L = (3, 3, 3, 4)
    m0 = 0.1
    U = synth.random_su3_links(L, 0.3, 5)
    phi = synth.gaussian_spinor(L, 1, 6)[0]
    W = oracle.build_hops(L, U)
    g5 = np.diag([1, 1, -1, -1]).astype(complex)
    w, st, _, _ = oracle.bicgstab(L, AP, W, m0, np.einsum("ab,xbc->xac", g5, phi), tol=1e-13)
    Z = np.einsum("ab,xbc->xac", g5, w)  # D^dagger Z = phi
    X, st2, _, _ = oracle.bicgstab(L, AP, W, m0, Z, tol=1e-13)
    Y = oracle.apply(L, AP, W, m0, X)
    ref = oracle.force(L, AP, U, m0, -2 * Y, X)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f32" if f32 else "f64")
    dU, info = op.force_inverse(torch.as_tensor(phi, device=gpu), m0=m0, tol=1e-13)
    assert info["status"] == "BRI_OK" and (info["outer_iters"] > 0) == f32, info
    assert np.abs(dU.cpu().numpy() - ref).max() <= 1e-8 * np.abs(ref).max()


def test_autograd_function(gpu):
    L = (3, 3, 3, 3)
    U = torch.as_tensor(synth.random_su3_links(L, 0.3, 7), device=gpu).requires_grad_(True)
    psi = torch.as_tensor(synth.gaussian_spinor(L, 1, 8)[0], device=gpu).requires_grad_(True)
    chi = torch.as_tensor(synth.gaussian_spinor(L, 1, 9)[0], device=gpu)
    op = Brillouin(L, AP)
    out = DiracFunction.apply(U, psi, op, 0.05)
    loss = torch.real(torch.vdot(chi.reshape(-1), out.reshape(-1)))
    loss.backward()
    Un = U.detach().cpu().numpy()
    ref_U = oracle.force(L, AP, Un, 0.05, chi.cpu().numpy(), psi.detach().cpu().numpy())
    assert np.abs(U.grad.cpu().numpy() - ref_U).max() <= 1e-10 * np.abs(ref_U).max()
    W = oracle.build_hops(L, Un)
    ref_psi = oracle.apply(L, AP, W, 0.05, chi.cpu().numpy(), dagger=True)
    assert np.abs(psi.grad.cpu().numpy() - ref_psi).max() <= 1e-12 * np.abs(ref_psi).max()


def test_inverse_action_function(gpu):
    """S = phi^dagger (D^dagger D)^{-1} phi through InverseActionFunction: S,
    dS/dU and dS/dphi against the oracle's solves and force (1e-8 relative),
    and dS/dU against central finite differences of S (eps = 1e-5) in single
    link entries, real and imaginary parts."""
    from paper_1012_3615_gb300 import InverseActionFunction

    L, m0 = (4, 3, 3, 4), 0.1
    Un = synth.random_su3_links(L, 0.3, 21)
    phin = synth.gaussian_spinor(L, 1, 22)[0]
    U = torch.as_tensor(Un, device=gpu).requires_grad_(True)
    phi = torch.as_tensor(phin, device=gpu).requires_grad_(True)
    op = Brillouin(L, AP)
    S = InverseActionFunction.apply(U, phi, op, m0, 1e-13)
    S.backward()
    # oracle: D^dagger Z = phi (via gamma5), D X = Z, Y = D X
    W = oracle.build_hops(L, Un)
    g5 = np.diag([1, 1, -1, -1]).astype(complex)
    w, _, _, _ = oracle.bicgstab(L, AP, W, m0, np.einsum("ab,xbc->xac", g5, phin), tol=1e-14)
    X, _, _, _ = oracle.bicgstab(L, AP, W, m0, np.einsum("ab,xbc->xac", g5, w), tol=1e-14)
    Y = oracle.apply(L, AP, W, m0, X)
    S_ref = np.vdot(Y, Y).real
    assert abs(S.item() - S_ref) <= 1e-10 * S_ref
    ref_U = oracle.force(L, AP, Un, m0, -2 * Y, X)
    assert np.abs(U.grad.cpu().numpy() - ref_U).max() <= 1e-8 * np.abs(ref_U).max()
    assert np.abs(phi.grad.cpu().numpy() - 2 * X).max() <= 1e-8 * np.abs(2 * X).max()
    # central differences of S in single entries of single links
    rng = np.random.default_rng(23)
    eps = 1e-5
    G = U.grad.cpu().numpy()
    V = synth.volume(L)
    for _ in range(6):
        x, mu, a, b = rng.integers(0, V), rng.integers(0, 4), rng.integers(0, 3), rng.integers(0, 3)
        for part, unit in ((0, 1.0), (1, 1j)):
            Sp = []
            for sgn in (1, -1):
                Up = Un.copy()
                Up[x, mu, a, b] += sgn * eps * unit
                Sp.append(InverseActionFunction.apply(torch.as_tensor(Up, device=gpu), phi.detach(), op, m0,
                                                      1e-13).item())
            fd = (Sp[0] - Sp[1]) / (2 * eps)
            an = G[x, mu, a, b].real if part == 0 else G[x, mu, a, b].imag
            assert abs(fd - an) <= 1e-6 * np.abs(G).max() + 1e-6 * abs(an), (x, mu, a, b, part, fd, an)
