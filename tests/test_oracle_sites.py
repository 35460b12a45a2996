"""The single-site oracle entry agrees with the whole-lattice oracle apply."""
import numpy as np

import oracle
from paper_1012_3615_gb300 import synth


def test_apply_sites_matches_full_apply():
    L = (3, 4, 3, 4)
    U = synth.random_su3_links(L, 0.4, 1)
    psi = synth.gaussian_spinor(L, 1, 2)[0]
    W = oracle.build_hops(L, U)
    full = oracle.apply(L, (1, 1, 1, -1), W, 0.07, psi)
    sites = [0, 13, 77, synth.volume(L) - 1]
    part = oracle.apply_sites(L, (1, 1, 1, -1), U, 0.07, psi, sites)
    assert np.abs(part - full[sites]).max() < 1e-14
