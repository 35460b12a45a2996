"""GB300 (sm_103a) implementation of the Brillouin Dirac operator.

``D = sum_mu gamma_mu nabla^iso_mu - (1/2) Laplacian^bri + m0`` (Eq. def_pref of
Duerr & Koutsou, c_SW = 0): an 81-point stencil whose off-axis hops carry the
path-averaged, SU(3)-projected transports of Sec. 5.  The computation lives in
the CUDA library libbrillouin.so (C ABI in include/brillouin.h); this package
only marshals torch tensors into it.

    from paper_1012_3615_gb300 import Brillouin
    op = Brillouin((8, 8, 8, 8))
    op.build_hops(U)             # U: cuda complex128 (V, 4, 3, 3)
    out = op.apply(psi, m0=0.0)  # psi: cuda complex128 (V, 4, 3) or (n, V, 4, 3)
"""

__all__ = ["Brillouin", "BriError", "DiracFunction", "InverseActionFunction"]


def __getattr__(name):
    if name in ("Brillouin", "BriError"):
        from . import core
        return getattr(core, name)
    if name in ("DiracFunction", "InverseActionFunction"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
