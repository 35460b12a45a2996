"""The allocation-free hop precompute (bri_build_hops_noalloc) gives the same
fields as bri_build_hops + bri_get_hops.

It exists for callers that cannot allocate device memory themselves; its
work space is a fixed array inside the library, shared by every call, so the
test makes two calls in a row (the second must not see stale state) and
checks the size limit.  Collected last so that a run stopping at the first
failure has run everything else already."""
import numpy as np
import pytest
import torch

from paper_1012_3615_gb300 import Brillouin, BriError, synth
from paper_1012_3615_gb300.core import build_hops_noalloc

pytestmark = pytest.mark.gpu
AP = (1, 1, 1, -1)


@pytest.mark.parametrize("L", [(8, 8, 8, 8), (3, 5, 4, 6)])
def test_noalloc_matches_build_hops_on_two_calls(gpu, L):
    op = Brillouin(L, AP)
    for call, seed in enumerate((101, 202)):
        U = torch.as_tensor(synth.random_su3_links(L, 0.3 + 0.1 * call, seed), device=gpu)
        W = build_hops_noalloc(L, AP, U)
        op.build_hops(U)
        ref = op.hops()
        torch.cuda.synchronize()
        assert torch.abs(W - ref).max().item() < 1e-12, call


def test_noalloc_rejects_lattices_beyond_its_scratch(gpu):
    L = (8, 8, 8, 16)  # 8192 sites > 4096
    U = torch.zeros((8192, 4, 3, 3), dtype=torch.complex128, device=gpu)
    with pytest.raises(BriError, match="4096-site"):
        build_hops_noalloc(L, AP, U)
