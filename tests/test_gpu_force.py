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
