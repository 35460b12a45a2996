"""Torch-facing wrapper of the C ABI: tensors in, tensors out.

PyTorch provides device memory and the current stream only; every operation
is one call into libbrillouin.so.
"""
import ctypes

import torch

from . import abi

_PREC = {"f64": abi.BRI_F64, "f32": abi.BRI_F32, "f16": abi.BRI_F16, "f16h": abi.BRI_F16H}
_COMP = {"full": abi.BRI_LINK_FULL, "2row": abi.BRI_LINK_2ROW, "8param": abi.BRI_LINK_8PARAM}


# Columns of Tab. rholambda: (lambda_0..4, rho_0..4)
WEIGHTS = {
    "brillouin": ([240 / 128, -8 / 128, -4 / 128, -2 / 128, -1 / 128], [0, 64 / 432, 16 / 432, 4 / 432, 1 / 432]),
    "wilson": ([4.0, -0.5, 0, 0, 0], [0, 0.5, 0, 0, 0]),
    "hypercube": ([1.852720547, -0.060757866, -0.030036032, -0.015967620, -0.008426812],
                  [0, 0.136846794, 0.032077284, 0.011058131, 0.004748991]),
}


class BriError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (abi.STATUS_NAMES.get(status, status), msg))
        self.status = status


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def spinor_dtype(prec):
    return torch.complex128 if prec == "f64" else torch.complex64


class Brillouin:
    """One lattice (extents L, fermion boundary phases bc) on the current GPU."""

    def __init__(self, L, bc=(1, 1, 1, -1)):
        self.lib = abi.load()
        self.L = tuple(int(v) for v in L)
        self.bc = tuple(int(v) for v in bc)
        self.V = self.L[0] * self.L[1] * self.L[2] * self.L[3]
        lat = abi.bri_lattice((ctypes.c_int * 4)(*self.L), (ctypes.c_int * 4)(*self.bc))
        h = ctypes.c_void_p()
        st = self.lib.bri_create(ctypes.byref(lat), ctypes.byref(h))
        if st != 0:
            raise BriError(st, self.lib.bri_last_error(None).decode())
        self.ctx = h

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and ctx.value:
            self.lib.bri_destroy(ctx)
            self.ctx = None

    def _check(self, st):
        if st != 0:
            raise BriError(st, self.lib.bri_last_error(self.ctx).decode())

    def h16_field_bytes(self):
        """bytes of one right-hand side in the FP16-spinor storage (prec "f16h")"""
        return int(self.lib.bri_h16_field_bytes(self.V))

    def to_h16(self, psi):
        """spinors (complex64 or complex128, (n, V, 4, 3)) to the FP16 storage
        with per-site scales: a uint8 tensor (n, h16_field_bytes())"""
        n = self._spinor(psi, "f64" if psi.dtype == torch.complex128 else "f32")
        out = torch.empty((n, self.h16_field_bytes()), dtype=torch.uint8, device="cuda")
        self._check(self.lib.bri_convert_spinor(self.ctx, _ptr(out), abi.BRI_F16H, _ptr(psi),
                                                abi.BRI_F64 if psi.dtype == torch.complex128 else abi.BRI_F32, n,
                                                _stream()))
        return out

    def from_h16(self, buf, dtype=torch.complex64):
        """FP16-storage spinors back to complex64 / complex128 (n, V, 4, 3)"""
        n = self._spinor(buf, "f16h")
        out = torch.empty((n, self.V, 4, 3), dtype=dtype, device="cuda")
        self._check(self.lib.bri_convert_spinor(self.ctx, _ptr(out),
                                                abi.BRI_F64 if dtype == torch.complex128 else abi.BRI_F32, _ptr(buf),
                                                abi.BRI_F16H, n, _stream()))
        return out

    def _spinor(self, t, prec):
        if prec == "f16h":
            fb = self.h16_field_bytes()
            if not (t.is_cuda and t.dtype == torch.uint8 and t.is_contiguous() and t.numel() % fb == 0):
                raise ValueError("FP16 spinors must be a contiguous cuda uint8 tensor of n x %d bytes" % fb)
            return t.numel() // fb
        dt = spinor_dtype(prec)
        if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise ValueError("spinor must be a contiguous cuda %s tensor" % dt)
        if t.numel() % (self.V * 12) != 0:
            raise ValueError("spinor size is not a multiple of V*12")
        return t.numel() // (self.V * 12)

    # ---- link precompute (Sec. 5.1, 5.2) -------------------------------------
    def build_hops(self, U, prec="f64", comp="full"):
        if not (U.is_cuda and U.dtype == torch.complex128 and U.is_contiguous() and U.numel() == self.V * 36):
            raise ValueError("U must be a contiguous cuda complex128 (V, 4, 3, 3) tensor")
        self._U = U
        self._check(self.lib.bri_build_hops(self.ctx, _ptr(U), _PREC[prec], _COMP[comp], _stream()))

    def store_hops(self, prec, comp="full"):
        self._check(self.lib.bri_store_hops(self.ctx, _PREC[prec], _COMP[comp], _stream()))

    def hops(self):
        out = torch.empty((self.V, 40, 3, 3), dtype=torch.complex128, device="cuda")
        self._check(self.lib.bri_get_hops(self.ctx, _ptr(out), _stream()))
        return out

    def project_su3(self, A):
        A = A.contiguous()
        Y = torch.empty_like(A)
        self._check(self.lib.bri_project_su3(self.ctx, _ptr(Y), _ptr(A), A.numel() // 9, _stream()))
        return Y

    # ---- stencil (Eq. def_pref) ------------------------------------------------
    def apply(self, psi, m0=0.0, dagger=False, prec="f64", out=None):
        n = self._spinor(psi, prec)
        out = torch.empty_like(psi) if out is None else out
        self._check(self.lib.bri_apply(self.ctx, _ptr(out), _ptr(psi), n, float(m0), int(bool(dagger)),
                                       _PREC[prec], _stream()))
        return out

    def apply_host(self, psi, m0=0.0, dagger=False, prec="f64", out=None):
        """D psi for a spinor in (pinned) host memory; the copies overlap the
        stencil inside the library.  Returns after enqueueing on the current
        stream: synchronise before reading out."""
        dt = spinor_dtype(prec)
        if psi.is_cuda or psi.dtype != dt or not psi.is_contiguous() or psi.numel() % (self.V * 12):
            raise ValueError("psi must be a contiguous host %s tensor of nrhs*V*12 elements" % dt)
        out = torch.empty_like(psi, pin_memory=psi.is_pinned()) if out is None else out
        n = psi.numel() // (self.V * 12)
        self._check(self.lib.bri_apply_host(self.ctx, out.data_ptr(), psi.data_ptr(), n, float(m0),
                                            int(bool(dagger)), _PREC[prec], _stream()))
        return out

    def overlap_kernel(self, psi, rho=1.0, prec="f64", out=None):
        n = self._spinor(psi, prec)
        out = torch.empty_like(psi) if out is None else out
        self._check(self.lib.bri_apply_overlap_kernel(self.ctx, _ptr(out), _ptr(psi), n, float(rho), _PREC[prec],
                                                      _stream()))
        return out

    # ---- solver (Sec. 6.4) -------------------------------------------------------
    def solve(self, b, m0=0.0, tol=1e-10, maxit=10000, mode=0, x0=None):
        n = self._spinor(b, "f64")
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        info = (abi.bri_solve_info * n)()
        st = self.lib.bri_solve(self.ctx, _ptr(x), _ptr(b), n, float(m0), float(tol), int(maxit), int(mode),
                                info, _stream())
        infos = [info[i].as_dict() for i in range(n)]
        if st not in (0, abi.BRI_ENOTCONV, abi.BRI_EBREAKDOWN, abi.BRI_ENAN):
            self._check(st)
        return x, infos

    # ---- force ---------------------------------------------------------------------
    def force(self, chi, psi, m0=0.0, dU=None, recompute_hops=True):
        self._spinor(chi, "f64")
        self._spinor(psi, "f64")
        dU = torch.zeros((self.V, 4, 3, 3), dtype=torch.complex128, device="cuda") if dU is None else dU
        self._check(self.lib.bri_force(self.ctx, _ptr(dU), _ptr(chi), _ptr(psi), float(m0), int(bool(recompute_hops)),
                                       _stream()))
        return dU

    def force_inverse(self, phi, m0=0.0, tol=1e-12, maxit=20000, dU=None):
        self._spinor(phi, "f64")
        dU = torch.zeros((self.V, 4, 3, 3), dtype=torch.complex128, device="cuda") if dU is None else dU
        info = abi.bri_solve_info()
        self._check(self.lib.bri_force_inverse(self.ctx, _ptr(dU), _ptr(phi), float(m0), float(tol), int(maxit),
                                               ctypes.byref(info), _stream()))
        return dU, info.as_dict()

    def inverse_action(self, phi, m0=0.0, tol=1e-12, maxit=20000, want_x=False, dU=None):
        """S = phi^dagger (D^dagger D)^{-1} phi; returns (S, X or None, dU or
        None, info) with X = (D^dagger D)^{-1} phi and dU += dS/dU when dU is
        given (a zero tensor to obtain the force alone)."""
        self._spinor(phi, "f64")
        S = ctypes.c_double()
        X = torch.empty_like(phi) if want_x else None
        info = abi.bri_solve_info()
        self._check(self.lib.bri_inverse_action(self.ctx, ctypes.byref(S), _ptr(X) if want_x else None,
                                                _ptr(dU) if dU is not None else None, _ptr(phi), float(m0),
                                                float(tol), int(maxit), ctypes.byref(info), _stream()))
        return S.value, X, dU, info.as_dict()

    def cdot(self, a, b, prec="f64"):
        """<a, b> = sum conj(a) b (FP64 accumulation in the library)."""
        n = self._spinor(a, prec)
        self._spinor(b, prec)
        r = (ctypes.c_double * 2)()
        self._check(self.lib.bri_cdot(self.ctx, r, _ptr(a), _ptr(b), n, _PREC[prec], _stream()))
        return complex(r[0], r[1])

    # ---- link smearing and the clover term (Eq. def_ape, Eq. def_pref) ---------------
    def ape_smear(self, U, alpha=0.72, nsteps=1, out=None):
        """nsteps APE steps of the links U (cuda complex128 (V, 4, 3, 3))."""
        if not (U.is_cuda and U.dtype == torch.complex128 and U.is_contiguous() and U.numel() == self.V * 36):
            raise ValueError("U must be a contiguous cuda complex128 tensor of V*36 elements")
        out = torch.empty_like(U) if out is None else out
        self._check(self.lib.bri_ape_smear(self.ctx, _ptr(out), _ptr(U), float(alpha), int(nsteps), _stream()))
        return out

    def set_clover(self, csw):
        """Clover coefficient c_SW of Eq. def_pref (0 switches the term off)."""
        self._check(self.lib.bri_set_clover(self.ctx, float(csw), _stream()))

    # ---- spectra and the overlap operator (Sec. 7) -----------------------------------
    def eigs_ddag_d(self, nev, m0=0.0, max_krylov=500, tol=1e-10, vectors=False, prec="f64"):
        """nev smallest and the largest eigenvalue of D(m0)^dagger D(m0) (Lanczos
        in the library).  Returns (evals, lmax, info) or (evals, lmax, vecs, info)."""
        ev = (ctypes.c_double * nev)()
        lmax = ctypes.c_double()
        info = abi.bri_eig_info()
        vecs = torch.empty((nev, self.V, 4, 3), dtype=torch.complex128, device="cuda") if vectors else None
        st = self.lib.bri_eigs_ddag_d(self.ctx, ev, ctypes.byref(lmax), _ptr(vecs) if vectors else None, int(nev),
                                      float(m0), int(max_krylov), float(tol), _PREC[prec], ctypes.byref(info),
                                      _stream())
        if st not in (0, abi.BRI_ENOTCONV):
            self._check(st)
        out = (list(ev), lmax.value) + ((vecs,) if vectors else ()) + (info.as_dict(),)
        return out

    def overlap_setup(self, rho=1.0, nlow=0, eps=1e-10, max_krylov=500, tol=1e-10, prec="f64"):
        """Prepare sign(H), H = gamma5 (D - rho) (Eq. def_over); returns the setup info."""
        info = abi.bri_overlap_info()
        self._check(self.lib.bri_overlap_setup(self.ctx, float(rho), int(nlow), float(eps), int(max_krylov),
                                               float(tol), _PREC[prec], ctypes.byref(info), _stream()))
        return info.as_dict()

    def overlap_modes(self, nlow):
        lam = (ctypes.c_double * max(nlow, 1))()
        vecs = torch.empty((max(nlow, 1), self.V, 4, 3), dtype=torch.complex128, device="cuda")
        self._check(self.lib.bri_overlap_modes(self.ctx, lam, _ptr(vecs), _stream()))
        return list(lam)[:nlow], vecs[:nlow]

    def sign(self, psi, out=None):
        n = self._spinor(psi, "f64")
        out = torch.empty_like(psi) if out is None else out
        self._check(self.lib.bri_apply_sign(self.ctx, _ptr(out), _ptr(psi), n, _stream()))
        return out

    def overlap(self, psi, m=0.0, out=None):
        """D_ov,m psi (Eq. def_over, Eq. def_mass) after overlap_setup."""
        n = self._spinor(psi, "f64")
        out = torch.empty_like(psi) if out is None else out
        self._check(self.lib.bri_apply_overlap(self.ctx, _ptr(out), _ptr(psi), n, float(m), _stream()))
        return out

    # ---- weights of the rho/lambda class (Sec. 8, Tab. rholambda) -------------
    def set_weights(self, lam, rho):
        """lam: lambda_0..4, rho: rho_0..4 (rho_0 ignored)."""
        la = (ctypes.c_double * 5)(*[float(v) for v in lam])
        ra = (ctypes.c_double * 5)(*[float(v) for v in rho])
        self._check(self.lib.bri_set_weights(self.ctx, la, ra))

    def weights(self):
        la = (ctypes.c_double * 5)()
        ra = (ctypes.c_double * 5)()
        self._check(self.lib.bri_get_weights(self.ctx, la, ra))
        return list(la), list(ra)

    def tune(self, prec="f32", nrhs=1):
        self._check(self.lib.bri_tune(self.ctx, _PREC[prec], int(nrhs), _stream()))

    def set_threads(self, prec, nrhs, threads):
        self._check(self.lib.bri_set_threads(self.ctx, _PREC[prec], int(nrhs), int(threads)))

    def threads(self, prec, nrhs=1):
        t = self.lib.bri_get_threads(self.ctx, _PREC[prec], int(nrhs))
        if t < 0:
            self._check(t)
        return t

    def kernel_launches(self):
        return int(self.lib.bri_kernel_launches(self.ctx))


def alu_peak(prec="f32"):
    """measured FMA peak of the current GPU in TFLOP/s (FP32 packed or FP64)"""
    lib = abi.load()
    v = ctypes.c_double()
    st = lib.bri_alu_peak(_PREC[prec], ctypes.byref(v))
    if st != 0:
        raise BriError(st, lib.bri_last_error(None).decode())
    return v.value


def build_hops_noalloc(L, bc, U, out=None):
    """The 40 canonical hopping fields of links U (cuda complex128 (V, 4, 3, 3))
    computed without any device allocation by the library (at most 4096
    sites); returns (V, 40, 3, 3) complex128 in out (allocated here if None)."""
    lib = abi.load()
    L = tuple(int(v) for v in L)
    V = L[0] * L[1] * L[2] * L[3]
    if not (U.is_cuda and U.dtype == torch.complex128 and U.is_contiguous() and U.numel() == V * 36):
        raise ValueError("U must be a contiguous cuda complex128 (V, 4, 3, 3) tensor")
    out = torch.empty((V, 40, 3, 3), dtype=torch.complex128, device=U.device) if out is None else out
    lat = abi.bri_lattice((ctypes.c_int * 4)(*L), (ctypes.c_int * 4)(*[int(v) for v in bc]))
    st = lib.bri_build_hops_noalloc(ctypes.byref(lat), _ptr(U), _ptr(out), _stream())
    if st != 0:
        raise BriError(st, lib.bri_last_error(None).decode())
    return out
