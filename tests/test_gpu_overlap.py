"""Lanczos spectra of D^dagger D and the overlap operator (Sec. 7) on the GPU
against the dense oracle (oracle/overlap.py), plus properties that hold at
sizes the dense oracle cannot reach: the Ginsparg-Wilson relation
(Eq. def_ginswils) and the free-field momentum-space form."""
import numpy as np
import pytest
import torch

import oracle
from oracle import overlap as ov
from paper_1012_3615_gb300 import Brillouin, synth
from paper_1012_3615_gb300.core import WEIGHTS

pytestmark = pytest.mark.gpu
AP = (1, 1, 1, -1)
LS = (3, 3, 3, 4)  # 1296 unknowns: dense eigendecompositions take a second


@pytest.fixture(scope="module")
def small_case():
    U = synth.random_su3_links(LS, 0.5, 81)
    psi = synth.gaussian_spinor(LS, 2, 82)
    return U, psi


def _op(gpu, L, U, name="brillouin", f32=False):
    op = Brillouin(L, AP)
    lam, rho = WEIGHTS[name]
    op.set_weights(lam, rho)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f32" if f32 else "f64", comp="full")
    return op


@pytest.mark.parametrize("name,m0", [("brillouin", -1.0), ("brillouin", 0.1), ("wilson", -1.0)])
def test_lanczos_matches_dense_spectrum(gpu, small_case, name, m0):
    U, _ = small_case
    lam, rho = WEIGHTS[name]
    oracle.set_weights(lam, rho)
    try:
        ref = ov.ddag_d_eigenvalues(LS, AP, oracle.build_hops(LS, U), m0)
    finally:
        oracle.reset_weights()
    op = _op(gpu, LS, U, name)
    ev, lmax, vecs, info = op.eigs_ddag_d(8, m0=m0, max_krylov=1200, tol=1e-11, vectors=True)
    assert info["status"] == "BRI_OK", info
    assert np.allclose(ev, ref[:8], rtol=1e-8, atol=0)
    assert abs(lmax - ref[-1]) <= 1e-10 * ref[-1]
    # Ritz vectors: unit norm, A y = theta y
    for k in (0, 7):
        y = vecs[k:k + 1]
        Ay = op.apply(op.apply(y, m0), m0, dagger=True)
        assert abs(op.cdot(y, y) - 1) < 1e-10
        r = Ay - ev[k] * y
        assert op.cdot(r, r).real ** 0.5 <= 1e-8 * ref[-1]


@pytest.mark.parametrize("nlow,prec,tol", [(6, "f64", 1e-9), (0, "f64", 1e-9), (6, "f32", 2e-5)])
def test_overlap_matches_dense_oracle(gpu, small_case, nlow, prec, tol):
    U, psi = small_case
    W = oracle.build_hops(LS, U)
    rho, m = 1.0, 0.07
    S = ov.sign_hermitian(ov.hermitian_kernel(LS, AP, W, rho))
    Dm = ov.overlap_matrix(LS, AP, W, rho, m)
    op = _op(gpu, LS, U, f32=(prec == "f32"))
    info = op.overlap_setup(rho=rho, nlow=nlow, eps=1e-10, max_krylov=1200, tol=1e-11, prec=prec)
    assert info["status"] == "BRI_OK" and info["err_bound"] <= 1e-10, info
    x = torch.as_tensor(psi, device=gpu)
    sg = op.sign(x).cpu().numpy().reshape(2, -1)
    dov = op.overlap(x, m).cpu().numpy().reshape(2, -1)
    for r in range(2):
        v = psi[r].reshape(-1)
        nv = np.linalg.norm(v)
        assert np.linalg.norm(sg[r] - S @ v) <= tol * nv
        assert np.linalg.norm(dov[r] - Dm @ v) <= 2 * tol * nv
    if nlow:
        lam_ref, _ = ov.kernel_eigenpairs(LS, AP, W, rho)
        lam, _ = op.overlap_modes(nlow)
        # FP32 setups find the modes with FP32 applies: eigenvalues to ~1e-7
        ltol, rtol = (1e-8, 1e-8) if prec == "f64" else (1e-6, 1e-5)
        assert np.allclose(lam, lam_ref[:nlow], rtol=ltol, atol=1e-12)
        assert info["defl_resid"] < rtol


def test_ginsparg_wilson_relation_6x6x6x6(gpu):
    """gamma5 D + D gamma5 = D gamma5 D / rho, on random links at a size the
    dense oracle cannot reach; the violation is bounded by the sign error."""
    L = (6, 6, 6, 6)
    op = _op(gpu, L, synth.random_su3_links(L, 0.3, 83))
    rho = 1.0
    info = op.overlap_setup(rho=rho, nlow=4, eps=1e-10, max_krylov=800, tol=1e-10)
    assert info["status"] == "BRI_OK", info
    psi = torch.as_tensor(synth.gaussian_spinor(L, 1, 84), device=gpu)
    g5 = torch.tensor([1, 1, -1, -1], dtype=torch.complex128, device=gpu).view(1, 1, 4, 1)
    Dp = op.overlap(psi)
    lhs = g5 * Dp + op.overlap(g5 * psi)
    rhs = op.overlap(g5 * Dp) / rho
    viol = (lhs - rhs).norm().item() / psi.norm().item()
    assert viol < 1e-8, (viol, info)


def test_free_field_plane_waves_8x8x8x8(gpu):
    """Unit links: D_ov e^{ik.x} u = rho [1 + X(k) (X(k)^dagger X(k))^(-1/2)] e^{ik.x} u
    with X(k) the spin symbol of D at m0 = -rho (closed forms of Sec. 3)."""
    L = (8, 8, 8, 8)
    op = _op(gpu, L, synth.unit_links(L))
    info = op.overlap_setup(rho=1.0, nlow=0, eps=1e-11, max_krylov=400, tol=1e-10)
    assert info["status"] == "BRI_OK", info
    rng = np.random.default_rng(85)
    for _ in range(3):
        k = np.array([(2 * rng.integers(0, 8) + (1 if AP[mu] < 0 else 0)) * np.pi / 8 for mu in range(4)])
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        X = (-1.0 + 2 - 2 * np.prod(np.cos(k / 2) ** 2)) * np.eye(4, dtype=complex)
        for mu in range(4):
            other = np.prod([np.cos(k[nu]) + 2 for nu in range(4) if nu != mu])
            X = X + 1j * np.sin(k[mu]) * other / 27 * oracle.gamma(mu)
        w, Q = np.linalg.eigh(X.conj().T @ X)
        Sym = np.eye(4) + X @ ((Q / np.sqrt(w)) @ Q.conj().T)
        psi = synth.plane_wave(L, k, u)
        got = op.overlap(torch.as_tensor(psi[None], device=gpu)).cpu().numpy()[0]
        want = synth.plane_wave(L, k, Sym @ u)
        assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()


def test_fp32_lanczos_spectrum(gpu, small_case):
    """FP32 Lanczos (FP32 fields and vectors, FP64 sums): Ritz values to 1e-5."""
    U, _ = small_case
    ref = ov.ddag_d_eigenvalues(LS, AP, oracle.build_hops(LS, U), -1.0)
    op = _op(gpu, LS, U, f32=True)
    ev, lmax, vecs, info = op.eigs_ddag_d(6, m0=-1.0, max_krylov=1200, tol=1e-6, vectors=True, prec="f32")
    assert info["status"] == "BRI_OK", info
    assert np.allclose(ev, ref[:6], rtol=1e-5, atol=0)
    assert abs(lmax - ref[-1]) <= 1e-5 * ref[-1]
    y = vecs[0:1]
    r = op.apply(op.apply(y, -1.0), -1.0, dagger=True) - ev[0] * y
    assert op.cdot(r, r).real ** 0.5 <= 1e-4 * ref[-1]
