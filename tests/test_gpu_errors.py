"""Argument and state checks of the newer entry points: every misuse returns
a status (no fault, nothing enqueued) and the context stays usable."""
import numpy as np
import pytest
import torch

from paper_1012_3615_gb300 import Brillouin, BriError, synth

pytestmark = pytest.mark.gpu
AP = (1, 1, 1, -1)
L = (4, 3, 3, 4)


@pytest.fixture
def op(gpu):
    o = Brillouin(L, AP)
    return o


def _status(exc):
    return exc.value.args[0] if exc.value.args else None


def test_state_errors_before_build(op, gpu):
    x = torch.zeros((1, op.V, 4, 3), dtype=torch.complex128, device=gpu)
    for call in (lambda: op.set_clover(1.0), lambda: op.eigs_ddag_d(2, max_krylov=50),
                 lambda: op.overlap_setup(nlow=0, max_krylov=50), lambda: op.overlap(x), lambda: op.sign(x)):
        with pytest.raises(BriError):
            call()


def test_argument_errors(op, gpu):
    U = torch.as_tensor(synth.random_su3_links(L, 0.3, 61), device=gpu)
    op.build_hops(U)
    x = torch.as_tensor(synth.gaussian_spinor(L, 1, 62), device=gpu)
    bad = [
        lambda: op.eigs_ddag_d(0, max_krylov=50),            # nev < 1
        lambda: op.eigs_ddag_d(65, max_krylov=500),          # nev > 64
        lambda: op.eigs_ddag_d(4, max_krylov=4),             # max_krylov <= nev
        lambda: op.eigs_ddag_d(4, max_krylov=12 * op.V + 1),  # beyond the space
        lambda: op.overlap_setup(rho=0.0, max_krylov=50),
        lambda: op.overlap_setup(rho=2.0, max_krylov=50),
        lambda: op.overlap_setup(nlow=65, max_krylov=500),
        lambda: op.overlap_setup(eps=0.5, max_krylov=50),
        lambda: op.overlap_setup(prec="f32", max_krylov=50),  # no FP32 fields stored
        lambda: op.ape_smear(U, alpha=1.5),
        lambda: op.ape_smear(U, nsteps=-1),
        lambda: op.ape_smear(U, out=U),                       # in place
        lambda: op.set_clover(float("nan")),
        lambda: op.apply_host(x.cpu().to(torch.complex64), prec="f32"),  # FP32 fields not stored
    ]
    for call in bad:
        with pytest.raises(BriError):
            call()
    # the context is still usable
    y = op.apply(x, 0.1)
    assert torch.isfinite(y.abs()).all()


def test_apply_host_rejects_overlapping_buffers(op, gpu):
    op.build_hops(torch.as_tensor(synth.unit_links(L), device=gpu))
    xh = torch.zeros((2, op.V, 4, 3), dtype=torch.complex128).pin_memory()
    with pytest.raises(BriError):
        op.apply_host(xh[0:1], out=xh[0:1])
    with pytest.raises(ValueError):
        op.apply_host(xh.to(gpu))  # device tensor given to the host-buffer call


def test_overlap_state_invalidated_by_new_links(op, gpu):
    op.build_hops(torch.as_tensor(synth.random_su3_links(L, 0.3, 63), device=gpu))
    op.overlap_setup(nlow=2, max_krylov=400)
    x = torch.as_tensor(synth.gaussian_spinor(L, 1, 64), device=gpu)
    op.overlap(x)
    op.build_hops(torch.as_tensor(synth.random_su3_links(L, 0.3, 65), device=gpu))
    with pytest.raises(BriError):
        op.overlap(x)
    op.set_weights(*[(4.0, -0.5, 0, 0, 0), (0, 0.5, 0, 0, 0)])
    with pytest.raises(BriError):
        op.sign(x)
