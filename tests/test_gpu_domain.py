"""The domain-decomposed apply driven through the library on one GPU: the
block of a single rank plus its halo (all regions from itself, with the
boundary phases) as an extended lattice; hops built and the operator applied
there by the library; interior outputs equal the apply on the lattice itself."""
import numpy as np
import pytest
import torch

from paper_1012_3615_gb300 import Brillouin, synth
from paper_1012_3615_gb300.domain import Decomposition, exchange

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,bc", [((4, 4, 4, 6), (1, 1, 1, -1)), ((3, 5, 4, 4), (-1, 1, 1, -1))])
def test_extended_lattice_apply_on_gpu(gpu, L, bc):
    dec = Decomposition(L, (1, 1, 1, 1), bc)
    U = torch.as_tensor(synth.random_su3_links(L, 0.4, 12), device=gpu)
    psi = torch.as_tensor(synth.gaussian_spinor(L, 1, 13)[0], device=gpu)
    Ue = exchange(dec, 0, U, None, spinor=False).contiguous()
    pe = exchange(dec, 0, psi, None, spinor=True).contiguous()
    ext = Brillouin(dec.E, (1, 1, 1, 1))
    ext.build_hops(Ue, prec="f32")
    op = Brillouin(L, bc)
    op.build_hops(U, prec="f32")
    idx = torch.as_tensor(dec.interior(), device=gpu)
    got64 = ext.apply(pe.unsqueeze(0), 0.05)[0][idx]
    ref64 = op.apply(psi.unsqueeze(0), 0.05)[0]
    assert (torch.abs(got64 - ref64).max() / torch.abs(ref64).max()).item() < 1e-13
    got32 = ext.apply(pe.unsqueeze(0).to(torch.complex64), 0.05, prec="f32")[0][idx]
    ref32 = op.apply(psi.unsqueeze(0).to(torch.complex64), 0.05, prec="f32")[0]
    assert (torch.abs(got32 - ref32).max() / torch.abs(ref32).max()).item() < 1e-6
