"""The seeded synthetic inputs (links exp(i eps H), Gaussian and Z2 spinors,
point sources): the device-side link generator used for the large lattices
draws the same distribution as the host one and returns SU(3) matrices; run on
the CPU here."""
import numpy as np
import torch

from paper_1012_3615_gb300 import synth


def test_torch_matrix_exponential_matches_eigendecomposition():
    rng = np.random.default_rng(3)
    h = rng.standard_normal((64, 8))
    H = np.einsum("na,aij->nij", h, synth._gell_mann()) / 2.0
    for eps in (0.3, 0.4):
        w, Q = np.linalg.eigh(H)
        ref = np.einsum("nij,nj,nkj->nik", Q, np.exp(1j * eps * w), Q.conj())
        got = synth._expm_i_torch(torch.as_tensor(1j * eps * H)).numpy()
        assert np.abs(got - ref).max() < 1e-13


def test_device_link_generator_is_su3_with_the_host_distribution():
    L = (8, 8, 4, 4)
    for eps in (0.3, 0.4):
        Ut = synth.random_su3_links_torch(L, eps, 11, device="cpu").numpy().reshape(-1, 3, 3)
        Un = synth.random_su3_links(L, eps, 11).reshape(-1, 3, 3)
        eye = np.eye(3)
        assert np.abs(np.einsum("nji,njk->nik", Ut.conj(), Ut) - eye).max() < 1e-13
        assert np.abs(np.linalg.det(Ut) - 1).max() < 1e-13
        # same distribution: mean and spread of Re tr U / 3 agree within sampling error
        a, b = np.real(np.trace(Ut, axis1=1, axis2=2)) / 3, np.real(np.trace(Un, axis1=1, axis2=2)) / 3
        se = np.hypot(a.std(), b.std()) / np.sqrt(a.size)
        assert abs(a.mean() - b.mean()) < 5 * se
        assert abs(a.std() - b.std()) < 0.1 * b.std()


def test_spinor_and_source_generators():
    L = (4, 4, 4, 4)
    g = synth.gaussian_spinor(L, 3, 5)
    assert g.shape == (3, 256, 4, 3) and abs(np.mean(np.abs(g) ** 2) - 1) < 0.1
    z = synth.z2_spinor(L, 2, 6)
    assert set(np.unique(z.real)) == {-1.0, 1.0} and np.all(z.imag == 0)
    b, x0 = synth.point_sources(L, 7)
    assert b.shape == (12, 256, 4, 3) and np.count_nonzero(b) == 12
    for r in range(12):
        assert b[r, x0, r // 3, r % 3] == 1
    gt = synth.gaussian_spinor_torch(L, 2, 8, device="cpu", dtype=torch.complex64)
    assert gt.dtype == torch.complex64 and gt.shape == (2, 256, 4, 3)
    assert abs(gt.abs().pow(2).mean().item() - 1) < 0.1
