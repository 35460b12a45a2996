"""Plain FP64 CPU oracle for the Brillouin Dirac operator.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``; the
product package never imports it.  The arithmetic lives in
``brillouin_oracle.c`` (compiled with gcc on first use); this module only
marshals numpy arrays.

Array conventions (the oracle's own):
  U   (V, 4, 3, 3) complex128   links, U[x, mu] connects x to x + mu
  W   (V, 81, 3, 3) complex128  hops, offset index k(d) = sum_mu (d_mu+1) 3^mu
  psi (V, 4, 3)     complex128  spinor (spin, colour)
  L   (L0, L1, L2, L3), x0 fastest; bc = fermion boundary phases (+1/-1).

Parity unpinned: nothing -- every function is pinned by tests/test_oracle_*.py.
"""
import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brillouin_oracle.c")
_BUILD = os.path.join(_HERE, "_build", platform.machine())
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None

c_dp = ctypes.POINTER(ctypes.c_double)
c_ip = ctypes.POINTER(ctypes.c_int)


def build(force=False):
    """Compile the oracle shared library with gcc (OpenMP, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.bo_num_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(c_dp)


def _iv(v):
    return (ctypes.c_int * 4)(*[int(t) for t in v])


def _c(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if shape is not None:
        a = a.reshape(shape)
    return a


def num_threads():
    return lib().bo_num_threads()


def set_num_threads(n):
    lib().bo_set_num_threads(int(n))


def weights():
    """(lambda_0..4, rho_0..4) of Tab. rholambda (rho_0 = 0)."""
    lam = np.zeros(5)
    rho = np.zeros(5)
    lib().bo_weights(_p(lam), _p(rho))
    return lam, rho


def set_weights(lam, rho):
    """Replace the class weights (lambda_0..4, rho_0..4; rho_0 ignored)."""
    la = np.ascontiguousarray(lam, dtype=np.float64)
    ra = np.ascontiguousarray(rho, dtype=np.float64)
    lib().bo_set_weights(_p(la), _p(ra))


def reset_weights():
    """Restore the der_iso / lap_bri column of Tab. rholambda."""
    lib().bo_reset_weights()


def gamma(mu):
    """Dense 4x4 gamma_mu (mu=0..3) or gamma_5 (mu=4)."""
    g = np.zeros((4, 4), np.complex128)
    if lib().bo_gamma(int(mu), _p(g)) != 0:
        raise ValueError(mu)
    return g


def svd3(A):
    A = _c(A, (3, 3))
    U = np.zeros((3, 3), np.complex128)
    V = np.zeros((3, 3), np.complex128)
    s = np.zeros(3)
    lib().bo_svd3(_p(A), _p(U), _p(s), _p(V))
    return U, s, V


def phase_max(s, phi):
    s = np.ascontiguousarray(s, dtype=np.float64)
    th = np.zeros(3)
    lib().bo_phase_max(_p(s), ctypes.c_double(phi), _p(th))
    return th


def project_su3(A):
    """P_SU(3) of one (3,3) or a batch (..., 3, 3) of matrices."""
    A = _c(A)
    shp = A.shape
    A2 = A.reshape(-1, 9)
    Y = np.zeros_like(A2)
    lib().bo_project_batch(ctypes.c_long(A2.shape[0]), _p(A2), _p(Y))
    return Y.reshape(shp)


def project_vjp(A, G):
    A = _c(A)
    G = _c(G)
    shp = A.shape
    A2 = A.reshape(-1, 9)
    G2 = G.reshape(-1, 9)
    GA = np.zeros_like(A2)
    rc = lib().bo_project_vjp_batch(ctypes.c_long(A2.shape[0]), _p(A2), _p(G2), _p(GA))
    if rc != 0:
        raise RuntimeError("singular projection derivative")
    return GA.reshape(shp)


def path_sum(L, U, site, d):
    """Unnormalised sum over all shortest paths from site to site+d; returns (A, npaths)."""
    U = _c(U)
    A = np.zeros((3, 3), np.complex128)
    n = ctypes.c_int(0)
    lib().bo_path_sum(_iv(L), _p(U), ctypes.c_long(site), _iv(d), _p(A), ctypes.byref(n))
    return A, n.value


def offset_index(d):
    return sum((int(d[m]) + 1) * 3 ** m for m in range(4))


def build_hops(L, U):
    V = int(np.prod(L))
    U = _c(U, (V, 4, 3, 3))
    W = np.zeros((V, 81, 3, 3), np.complex128)
    if lib().bo_build_hops(_iv(L), _p(U), _p(W)) != 0:
        raise ValueError("lattice extents must be >= 3")
    return W


def apply(L, bc, W, m0, psi, dagger=False):
    V = int(np.prod(L))
    W = _c(W, (V, 81, 3, 3))
    psi = _c(psi, (V, 4, 3))
    out = np.zeros_like(psi)
    lib().bo_apply(_iv(L), _iv(bc), _p(W), ctypes.c_double(m0), int(bool(dagger)), _p(psi), _p(out))
    return out


def overlap_kernel(L, bc, W, m0, rho, psi):
    V = int(np.prod(L))
    W = _c(W, (V, 81, 3, 3))
    psi = _c(psi, (V, 4, 3))
    out = np.zeros_like(psi)
    lib().bo_overlap_kernel(_iv(L), _iv(bc), _p(W), ctypes.c_double(m0), ctypes.c_double(rho),
                            _p(psi), _p(out))
    return out


def bicgstab(L, bc, W, m0, b, tol=1e-10, maxit=10000, x0=None):
    """Returns (x, status, iterations, true relative residual)."""
    V = int(np.prod(L))
    W = _c(W, (V, 81, 3, 3))
    b = _c(b, (V, 4, 3))
    x = np.zeros_like(b) if x0 is None else _c(x0, (V, 4, 3)).copy()
    it = ctypes.c_int(0)
    tr = ctypes.c_double(0)
    st = lib().bo_bicgstab(_iv(L), _iv(bc), _p(W), ctypes.c_double(m0), _p(b), _p(x),
                           ctypes.c_double(tol), int(maxit), ctypes.byref(it), ctypes.byref(tr))
    return x, st, it.value, tr.value


def force(L, bc, U, m0, chi, psi):
    """d Re(chi^dagger D[U] psi)/dU as (V,4,3,3), convention d/dReU + i d/dImU."""
    V = int(np.prod(L))
    U = _c(U, (V, 4, 3, 3))
    chi = _c(chi, (V, 4, 3))
    psi = _c(psi, (V, 4, 3))
    dU = np.zeros((V, 4, 3, 3), np.complex128)
    rc = lib().bo_force(_iv(L), _iv(bc), _p(U), ctypes.c_double(m0), _p(chi), _p(psi), _p(dU))
    if rc != 0:
        raise RuntimeError("oracle force failed (%d)" % rc)
    return dU


def apply_sites(L, bc, U, m0, psi, sites):
    """(D psi)(x) for the listed sites only, hops built from U per site."""
    V = int(np.prod(L))
    U = _c(U, (V, 4, 3, 3))
    psi = _c(psi, (V, 4, 3))
    out = np.zeros((len(sites), 4, 3), np.complex128)
    for i, s in enumerate(sites):
        o = np.zeros((4, 3), np.complex128)
        lib().bo_apply_site(_iv(L), _iv(bc), _p(U), ctypes.c_double(m0), ctypes.c_long(int(s)), _p(psi), _p(o))
        out[i] = o
    return out


def ape_smear(L, U, alpha, nsteps=1):
    """nsteps APE steps (Eq. def_ape, projection of Eq. proj_SU) of the links U."""
    V = int(np.prod(L))
    U = _c(U, (V, 4, 3, 3))
    out = np.zeros_like(U)
    if lib().bo_ape_smear(_iv(L), _p(U), ctypes.c_double(alpha), int(nsteps), _p(out)) != 0:
        raise MemoryError("ape_smear")
    return out


def clover_field(L, U):
    """Hermitian clover-leaf F_{mu nu}(x), (V, 6, 3, 3), planes 01, 02, 03, 12, 13, 23."""
    V = int(np.prod(L))
    U = _c(U, (V, 4, 3, 3))
    F = np.zeros((V, 6, 3, 3), np.complex128)
    lib().bo_clover_field(_iv(L), _p(U), _p(F))
    return F


def apply_clover(L, bc, W, U, m0, csw, psi, dagger=False):
    """D psi with the clover term -(c_SW/2) sum sigma F of Eq. def_pref, F built
    from the links U (the same links the hops W were built from)."""
    out = apply(L, bc, W, m0, psi, dagger=dagger)
    V = int(np.prod(L))
    psi = _c(psi, (V, 4, 3))
    U = _c(U, (V, 4, 3, 3))
    if lib().bo_clover_add(_iv(L), _p(U), ctypes.c_double(csw), _p(psi), _p(out)) != 0:
        raise MemoryError("apply_clover")
    return out
