"""Bounded waits of the bulk-copy applies (launch variants 10 and 11).

With the stall switch (bri_debug_stall) on, every warp announces 16 bytes
more to its first stage's barrier than its copies deliver, so each wait on
that stage runs out after its one-second limit.  The kernel then waits for
its other stages (whose copies do complete), flags the timeout in the
context's host-mapped status word and returns: no copy is left in flight and
nothing is accessed out of bounds.  The next apply call reports BRI_ETIMEOUT
and clears the flag, and the context stays usable: the apply after it matches
the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1012_3615_gb300 import Brillouin, BriError, abi, synth

pytestmark = pytest.mark.gpu
AP = (1, 1, 1, -1)


@pytest.mark.parametrize("L,shape", [((32, 3, 4, 4), 10 * 2048 + 128), ((32, 3, 4, 4), 10 * 2048 + 32),
                                     ((16, 4, 3, 4), 10 * 2048 + 128), ((32, 3, 4, 4), 11 * 2048 + 32),
                                     ((32, 3, 4, 4), 11 * 2048 + 64)])
def test_bulk_wait_runs_out_and_is_reported(gpu, L, shape):
    U = synth.random_su3_links(L, 0.4, 7 + L[0])
    psi = synth.gaussian_spinor(L, 1, 8 + L[0])
    ref = oracle.apply(L, AP, oracle.build_hops(L, U), 0.05, psi[0])
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f32", comp="full")
    op.set_threads("f32", 1, shape)
    x = torch.as_tensor(psi.astype(np.complex64), device=gpu)
    assert op.lib.bri_debug_stall(op.ctx, 1) == abi.BRI_OK
    op.apply(x, m0=0.05, prec="f32")  # enqueued; its waits give up on the device
    torch.cuda.synchronize()
    assert op.lib.bri_debug_stall(op.ctx, 0) == abi.BRI_OK
    with pytest.raises(BriError) as e:
        op.apply(x, m0=0.05, prec="f32")
    assert e.value.status == abi.BRI_ETIMEOUT
    out = op.apply(x, m0=0.05, prec="f32").cpu().numpy()[0]
    assert np.abs(out - ref).max() / np.abs(ref).max() < 1e-6
