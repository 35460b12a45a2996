"""Seeded synthetic inputs shaped like the quenched lattices of the paper.

This module only draws random numbers and builds input fields; it holds none
of the operator's arithmetic, so both the CUDA path and the CPU oracle take
their inputs from here.

* links: ``U = exp(i eps H)`` per link, ``H = sum_a h_a lambda_a / 2`` with
  ``h_a ~ N(0, 1)`` (Gell-Mann matrices, ``tr T_a T_b = delta_ab / 2``),
  exponentiated through a Hermitian eigendecomposition and rescaled to unit
  determinant.
* spinors: complex Gaussian (Re, Im ~ N(0, 1/2)), Z2 noise (+-1 real) or
  spin-colour point sources.
* gauge transforms: Haar-random SU(3) per site (QR of a complex Gaussian).

All arrays are numpy complex128 in the library's layouts:
``U[V, 4, 3, 3]`` and ``psi[nrhs, V, 4, 3]`` (site index
``x0 + L0*(x1 + L1*(x2 + L2*x3))``).
"""
import numpy as np

_GELL_MANN = None


def _gell_mann():
    global _GELL_MANN
    if _GELL_MANN is None:
        l = np.zeros((8, 3, 3), np.complex128)
        l[0][0, 1] = l[0][1, 0] = 1
        l[1][0, 1], l[1][1, 0] = -1j, 1j
        l[2][0, 0], l[2][1, 1] = 1, -1
        l[3][0, 2] = l[3][2, 0] = 1
        l[4][0, 2], l[4][2, 0] = -1j, 1j
        l[5][1, 2] = l[5][2, 1] = 1
        l[6][1, 2], l[6][2, 1] = -1j, 1j
        l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
        _GELL_MANN = l
    return _GELL_MANN


def volume(L):
    return int(np.prod(L))


def random_su3_links(L, eps, seed):
    """Links ``exp(i eps H)``, one Gaussian traceless Hermitian H per link."""
    rng = np.random.default_rng(seed)
    V = volume(L)
    h = rng.standard_normal((V, 4, 8))
    H = np.einsum("xma,aij->xmij", h, _gell_mann()) / 2.0
    w, Q = np.linalg.eigh(H)
    U = np.einsum("xmij,xmj,xmkj->xmik", Q, np.exp(1j * eps * w), Q.conj())
    det = np.linalg.det(U)
    U = U / (det ** (1.0 / 3.0))[..., None, None]
    return np.ascontiguousarray(U)


def unit_links(L):
    V = volume(L)
    U = np.zeros((V, 4, 3, 3), np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def random_su3(n, seed):
    """n Haar-random SU(3) matrices."""
    rng = np.random.default_rng(seed)
    Z = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(Q)
    Q = Q / (det ** (1.0 / 3.0))[:, None, None]
    return np.ascontiguousarray(Q)


def gauge_transform(L, seed):
    return random_su3(volume(L), seed)


def gaussian_spinor(L, nrhs, seed):
    rng = np.random.default_rng(seed)
    V = volume(L)
    re = rng.standard_normal((nrhs, V, 4, 3))
    im = rng.standard_normal((nrhs, V, 4, 3))
    return np.ascontiguousarray((re + 1j * im) / np.sqrt(2.0))


def z2_spinor(L, nrhs, seed):
    rng = np.random.default_rng(seed)
    V = volume(L)
    s = rng.integers(0, 2, size=(nrhs, V, 4, 3)) * 2 - 1
    return np.ascontiguousarray(s.astype(np.complex128))


def point_sources(L, seed):
    """The 12 spin-colour point sources at one random site; returns (psi[12, V, 4, 3], site)."""
    rng = np.random.default_rng(seed)
    V = volume(L)
    x0 = int(rng.integers(0, V))
    psi = np.zeros((12, V, 4, 3), np.complex128)
    for s in range(4):
        for c in range(3):
            psi[3 * s + c, x0, s, c] = 1.0
    return psi, x0


def coordinates(L):
    """(V, 4) integer coordinates of every site."""
    V = volume(L)
    idx = np.arange(V)
    out = np.zeros((V, 4), np.int64)
    for mu in range(4):
        out[:, mu] = idx % L[mu]
        idx = idx // L[mu]
    return out


def plane_wave(L, k, u):
    """psi(x) = exp(i k.x) u for a constant (4,3) spinor u."""
    x = coordinates(L)
    ph = np.exp(1j * (x @ np.asarray(k, dtype=np.float64)))
    return np.ascontiguousarray(ph[:, None, None] * np.asarray(u, np.complex128)[None])


def _det3_torch(M):
    return (M[:, 0, 0] * (M[:, 1, 1] * M[:, 2, 2] - M[:, 1, 2] * M[:, 2, 1])
            - M[:, 0, 1] * (M[:, 1, 0] * M[:, 2, 2] - M[:, 1, 2] * M[:, 2, 0])
            + M[:, 0, 2] * (M[:, 1, 0] * M[:, 2, 1] - M[:, 1, 1] * M[:, 2, 0]))


def _mm3(A, B):
    """Batched 3x3 product as three broadcast multiply-adds (elementwise kernels)."""
    return A[:, :, 0, None] * B[:, None, 0, :] + A[:, :, 1, None] * B[:, None, 1, :] + A[:, :, 2, None] * B[:, None, 2, :]


def _expm_i_torch(X):
    """exp(X) for a batch of small anti-hermitian 3x3 matrices by Taylor series
    with scaling and squaring (elementwise products only)."""
    import torch

    k = 6  # ||X|| / 64 is far below 1 for these inputs
    Y = X / (2 ** k)
    eye = torch.eye(3, dtype=X.dtype, device=X.device).expand_as(Y)
    E = eye.clone()
    term = eye.clone()
    for n in range(1, 13):
        term = _mm3(term, Y) / n
        E = E + term
    for _ in range(k):
        E = _mm3(E, E)
    return E


def random_su3_links_torch(L, eps, seed, device="cuda", chunk=1 << 20):
    """Same distribution as random_su3_links, drawn with torch on the device
    (for lattices too large to generate on the host in reasonable time; the
    random stream differs from the numpy one).  Uses matmuls only."""
    import torch

    V = volume(L)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    lam = torch.as_tensor(_gell_mann(), device=device)
    U = torch.empty((V * 4, 3, 3), dtype=torch.complex128, device=device)
    for s in range(0, V * 4, chunk):
        e = min(V * 4, s + chunk)
        h = torch.randn((e - s, 8), generator=g, dtype=torch.float64, device=device)
        H = torch.einsum("na,aij->nij", h.to(torch.complex128), lam) / 2.0
        M = _expm_i_torch(1j * eps * H)
        M = _mm3(M, 1.5 * torch.eye(3, dtype=M.dtype, device=device) - 0.5 * _mm3(M.conj().transpose(1, 2), M))
        det = _det3_torch(M)
        U[s:e] = M / (det ** (1.0 / 3.0))[:, None, None]
    return U.reshape(V, 4, 3, 3)


def gaussian_spinor_torch(L, nrhs, seed, device="cuda", dtype=None):
    import torch

    dtype = dtype or torch.complex128
    V = volume(L)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    rdt = torch.float64 if dtype == torch.complex128 else torch.float32
    re = torch.randn((nrhs, V, 4, 3), generator=g, dtype=rdt, device=device)
    im = torch.randn((nrhs, V, 4, 3), generator=g, dtype=rdt, device=device)
    return torch.complex(re, im) / 2 ** 0.5
