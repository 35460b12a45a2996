"""ctypes declarations of the C ABI in include/brillouin.h (same names).

Argument marshalling only: every step of the computation runs in
libbrillouin.so.  Loading fails loudly when the library has not been built;
there is no fallback.
"""
import ctypes
import os

from . import build as _build

c_int, c_long, c_double, c_void_p = ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_void_p

BRI_OK, BRI_EINVAL, BRI_ENOMEM, BRI_ECUDA, BRI_ENOTCONV, BRI_EBREAKDOWN, BRI_ENAN, BRI_ETIMEOUT, BRI_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
STATUS_NAMES = {0: "BRI_OK", -1: "BRI_EINVAL", -2: "BRI_ENOMEM", -3: "BRI_ECUDA", -4: "BRI_ENOTCONV",
                -5: "BRI_EBREAKDOWN", -6: "BRI_ENAN", -7: "BRI_ETIMEOUT", -8: "BRI_ESTATE"}
BRI_F64, BRI_F32, BRI_F16, BRI_F16H = 0, 1, 2, 3
BRI_LINK_FULL, BRI_LINK_2ROW, BRI_LINK_8PARAM = 0, 1, 2


class bri_lattice(ctypes.Structure):
    _fields_ = [("L", c_int * 4), ("bc_sign", c_int * 4)]


class bri_solve_info(ctypes.Structure):
    _fields_ = [("iters", c_int), ("outer_iters", c_int), ("true_resid", c_double), ("seconds", c_double),
                ("status", c_int)]

    def as_dict(self):
        return {"iters": self.iters, "outer_iters": self.outer_iters, "true_resid": self.true_resid,
                "seconds": self.seconds, "status": STATUS_NAMES.get(self.status, self.status)}


class bri_eig_info(ctypes.Structure):
    _fields_ = [("nconv", c_int), ("krylov_dim", c_int), ("applies", c_int), ("max_resid", c_double),
                ("seconds", c_double), ("status", c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status"] = STATUS_NAMES.get(self.status, self.status)
        return d


class bri_overlap_info(ctypes.Structure):
    _fields_ = [("nlow", c_int), ("degree", c_int), ("lo", c_double), ("hi", c_double), ("err_bound", c_double),
                ("defl_resid", c_double), ("krylov_dim", c_int), ("applies", c_int), ("seconds", c_double),
                ("status", c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status"] = STATUS_NAMES.get(self.status, self.status)
        return d


# name -> (restype, argtypes), mirroring include/brillouin.h
SIGNATURES = {
    "bri_create": (c_int, [ctypes.POINTER(bri_lattice), ctypes.POINTER(c_void_p)]),
    "bri_destroy": (c_int, [c_void_p]),
    "bri_build_hops": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "bri_store_hops": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "bri_get_hops": (c_int, [c_void_p, c_void_p, c_void_p]),
    "bri_apply": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_int, c_int, c_void_p]),
    "bri_apply_host": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_int, c_int, c_void_p]),
    "bri_apply_overlap_kernel": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_int, c_void_p]),
    "bri_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_double, c_int, c_int,
                          ctypes.POINTER(bri_solve_info), c_void_p]),
    "bri_force": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_int, c_void_p]),
    "bri_force_inverse": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_double, c_int,
                                  ctypes.POINTER(bri_solve_info), c_void_p]),
    "bri_inverse_action": (c_int, [c_void_p, ctypes.POINTER(c_double), c_void_p, c_void_p, c_void_p, c_double,
                                   c_double, c_int, ctypes.POINTER(bri_solve_info), c_void_p]),
    "bri_project_su3": (c_int, [c_void_p, c_void_p, c_void_p, c_long, c_void_p]),
    "bri_build_hops_noalloc": (c_int, [ctypes.POINTER(bri_lattice), c_void_p, c_void_p, c_void_p]),
    "bri_cdot": (c_int, [c_void_p, ctypes.POINTER(c_double), c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "bri_set_weights": (c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "bri_get_weights": (c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "bri_ape_smear": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, c_void_p]),
    "bri_set_clover": (c_int, [c_void_p, c_double, c_void_p]),
    "bri_eigs_ddag_d": (c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_double), c_void_p, c_int,
                                c_double, c_int, c_double, c_int, ctypes.POINTER(bri_eig_info), c_void_p]),
    "bri_overlap_setup": (c_int, [c_void_p, c_double, c_int, c_double, c_int, c_double, c_int,
                                  ctypes.POINTER(bri_overlap_info), c_void_p]),
    "bri_overlap_modes": (c_int, [c_void_p, ctypes.POINTER(c_double), c_void_p, c_void_p]),
    "bri_apply_sign": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "bri_apply_overlap": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_void_p]),
    "bri_tune": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "bri_set_threads": (c_int, [c_void_p, c_int, c_int, c_int]),
    "bri_get_threads": (c_int, [c_void_p, c_int, c_int]),
    "bri_kernel_launches": (c_long, [c_void_p]),
    "bri_debug_stall": (c_int, [c_void_p, c_int]),
    "bri_last_error": (ctypes.c_char_p, [c_void_p]),
    "bri_alu_peak": (c_int, [c_int, ctypes.POINTER(c_double)]),
    "bri_h16_field_bytes": (ctypes.c_size_t, [c_int]),
    "bri_convert_spinor": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int, c_int, c_void_p]),
}

_lib = None


def library_path():
    return _build.LIB


def load():
    """Load libbrillouin.so (built by __graft_entry__.build() / build.build())."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libbrillouin.so is not built (%s); run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
