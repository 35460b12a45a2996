"""GPU link precompute (path sums, Sec. 5.1; SU(3) projection, Sec. 5.2)
against the CPU oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1012_3615_gb300 import Brillouin, synth

pytestmark = pytest.mark.gpu
AP = (1, 1, 1, -1)


@pytest.mark.parametrize("L,eps,seed", [((4, 4, 4, 4), 0.4, 1), ((3, 5, 4, 6), 0.3, 2), ((3, 3, 3, 3), 0.8, 3)])
def test_hops_match_oracle(gpu, L, eps, seed):
    U = synth.random_su3_links(L, eps, seed)
    W = oracle.build_hops(L, U)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu))
    Wg = op.hops().cpu().numpy()
    for j in range(40):
        assert np.abs(Wg[:, j] - W[:, j + 41]).max() < 1e-12, j


def _su3_check(Y, tol=1e-13):
    eye = np.eye(3)
    assert np.abs(np.einsum("nji,njk->nik", Y.conj(), Y) - eye).max() < tol
    assert np.abs(np.linalg.det(Y) - 1).max() < tol


def test_projection_generic_matrices(gpu):
    rng = np.random.default_rng(4)
    n = 3000
    A = (synth.random_su3(n, 5) + 1.5 * (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))))
    A[:500] *= 1e-3  # scale invariance over magnitudes
    A[500:1000] = synth.random_su3(500, 6) * (1 + 1e-7 * rng.standard_normal((500, 1, 1)))  # near-degenerate s
    op = Brillouin((3, 3, 3, 3), AP)
    Y = op.project_su3(torch.as_tensor(A, device=gpu)).cpu().numpy()
    _su3_check(Y)
    ref = oracle.project_su3(A)
    assert np.abs(Y - ref).max() < 1e-11


def test_projection_negative_determinant_sums(gpu):
    """Footnote of Sec. 5.2: det(U+V) can be negative real; then two phase
    choices tie, so compare the maximised objective and check Y in SU(3)."""
    As = []
    for t in range(6000):
        U, V = synth.random_su3(2, 5000 + t)
        A = U + V
        if np.linalg.det(A).real < -1e-3:
            As.append(A)
        if len(As) >= 40:
            break
    A = np.array(As)
    op = Brillouin((3, 3, 3, 3), AP)
    Y = op.project_su3(torch.as_tensor(A, device=gpu)).cpu().numpy()
    _su3_check(Y)
    ref = oracle.project_su3(A)
    fg = np.real(np.einsum("nij,nij->n", A.conj(), Y))
    fo = np.real(np.einsum("nij,nij->n", A.conj(), ref))
    assert np.abs(fg - fo).max() < 1e-12


def test_projection_branch_b_inputs(gpu):
    """det A with phase near pi and well separated singular values: the
    maximum needs the smallest singular value's phase beyond pi/2."""
    rng = np.random.default_rng(7)
    A = []
    for _ in range(200):
        s = np.sort(rng.uniform(0.05, 2.0, 3))[::-1]
        Uq = synth.random_su3(1, int(rng.integers(1 << 30)))[0]
        Vq = synth.random_su3(1, int(rng.integers(1 << 30)))[0]
        ph = np.exp(1j * rng.uniform(2.6, 3.1) / 3)
        A.append(Uq @ np.diag(s * ph) @ Vq.conj().T)
    A = np.array(A)
    op = Brillouin((3, 3, 3, 3), AP)
    Y = op.project_su3(torch.as_tensor(A, device=gpu)).cpu().numpy()
    _su3_check(Y)
    ref = oracle.project_su3(A)
    fg = np.real(np.einsum("nij,nij->n", A.conj(), Y))
    fo = np.real(np.einsum("nij,nij->n", A.conj(), ref))
    assert np.abs(fg - fo).max() < 1e-12
    assert np.abs(Y - ref).max() < 1e-9


def test_empty_projection_batch(gpu):
    op = Brillouin((3, 3, 3, 3), AP)
    A = torch.zeros((0, 3, 3), dtype=torch.complex128, device=gpu)
    assert op.project_su3(A).shape == (0, 3, 3)
