"""The allocation-free hop precompute (bri_build_hops_noalloc).

It exists for callers that cannot allocate device memory themselves (an
application whose pool owns all device memory, an embedding that must not
grow its footprint while running); its work space is a fixed array inside the
library, shared by every call.  The fields are checked element by element
against the oracle's path enumeration and projection, on two calls in a row
(the second must not see the first call's state), and against the
allocating entry point.  Collected last so that a run stopping at the first
failure has run everything else already."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1012_3615_gb300 import Brillouin, BriError, abi, synth
from paper_1012_3615_gb300.core import build_hops_noalloc

pytestmark = pytest.mark.gpu
AP = (1, 1, 1, -1)


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (3, 5, 4, 6), (8, 8, 8, 8)])
def test_noalloc_matches_oracle_on_two_calls(gpu, L):
    op = Brillouin(L, AP)
    for call, seed in enumerate((101, 202)):
        Uh = synth.random_su3_links(L, 0.3 + 0.1 * call, seed + sum(L))
        U = torch.as_tensor(Uh, device=gpu)
        W = build_hops_noalloc(L, AP, U).cpu().numpy()
        Wo = oracle.build_hops(L, Uh)
        for j in range(40):
            assert np.abs(W[:, j] - Wo[:, j + 41]).max() < 1e-12, (call, j)
        op.build_hops(U)
        assert np.abs(W - op.hops().cpu().numpy()).max() < 1e-12, call


def test_noalloc_rejects_lattices_beyond_its_scratch(gpu):
    L = (8, 8, 8, 16)  # 8192 sites > 4096
    U = torch.zeros((8192, 4, 3, 3), dtype=torch.complex128, device=gpu)
    with pytest.raises(BriError, match="4096-site"):
        build_hops_noalloc(L, AP, U)


def test_noalloc_rejects_null_and_misaligned_pointers(gpu):
    lib = abi.load()
    L = (4, 4, 4, 4)
    lat = abi.bri_lattice((ctypes.c_int * 4)(*L), (ctypes.c_int * 4)(*AP))
    U = torch.zeros((256, 4, 3, 3), dtype=torch.complex128, device=gpu)
    W = torch.zeros((256 * 40 * 9 + 1,), dtype=torch.complex128, device=gpu)
    u, w = U.data_ptr(), W.data_ptr()
    assert lib.bri_build_hops_noalloc(ctypes.byref(lat), None, w, None) == abi.BRI_EINVAL
    assert lib.bri_build_hops_noalloc(ctypes.byref(lat), u, None, None) == abi.BRI_EINVAL
    assert lib.bri_build_hops_noalloc(None, u, w, None) == abi.BRI_EINVAL
    assert lib.bri_build_hops_noalloc(ctypes.byref(lat), u, w + 8, None) == abi.BRI_EINVAL
    assert lib.bri_build_hops_noalloc(ctypes.byref(lat), u + 8, w, None) == abi.BRI_EINVAL
    assert b"aligned" in lib.bri_last_error(None)
    torch.cuda.synchronize()
