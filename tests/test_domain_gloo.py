"""Domain-decomposed apply with depth-1 halos (the multi-GPU form of the
operator): every rank builds the hops and applies the operator on its block
plus the halo it received, and the interior outputs gathered from all ranks
equal the single-domain apply.  Ranks are gloo processes on the CPU and the
local compute is the oracle; the same host logic drives the library on a GPU
per rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp
from mp_util import collect


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, L, grid, bc, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1012_3615_gb300 import synth
    from paper_1012_3615_gb300.domain import Decomposition, exchange

    dist.init_process_group("gloo", rank=rank, world_size=world)
    dec = Decomposition(L, grid, bc)
    U = synth.random_su3_links(L, 0.4, 7)
    psi = synth.gaussian_spinor(L, 1, 8)[0]
    mine = dec.global_sites(rank)
    Ue = exchange(dec, rank, torch.as_tensor(U[mine]), dist, spinor=False).numpy()
    pe = exchange(dec, rank, torch.as_tensor(psi[mine]), dist, spinor=True).numpy()
    We = oracle.build_hops(dec.E, Ue)
    out = oracle.apply(dec.E, (1, 1, 1, 1), We, 0.07, pe)[dec.interior()]
    q.put((rank, mine, out))
    dist.destroy_process_group()


@pytest.mark.parametrize("L,grid,bc", [((3, 4, 3, 6), (1, 1, 1, 2), (1, 1, 1, -1)),
                                       ((4, 3, 4, 3), (2, 1, 1, 1), (-1, 1, 1, -1)),
                                       ((4, 4, 3, 3), (1, 2, 1, 1), (1, 1, 1, -1))])
def test_two_rank_halo_apply_equals_single_domain(L, grid, bc):
    import oracle
    from paper_1012_3615_gb300 import synth

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, L, grid, bc, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = collect(q, procs, 2, 300)
    U = synth.random_su3_links(L, 0.4, 7)
    psi = synth.gaussian_spinor(L, 1, 8)[0]
    ref = oracle.apply(L, bc, oracle.build_hops(L, U), 0.07, psi)
    covered = np.zeros(len(ref), bool)
    for rank, sites, out in got:
        assert np.abs(out - ref[sites]).max() <= 1e-13 * np.abs(ref).max(), rank
        covered[sites] = True
    assert covered.all()


def test_single_rank_halo_is_the_periodic_wrap():
    """One rank: every halo region comes from the rank itself, with the
    boundary phase; the extended apply reproduces the periodic one."""
    import torch

    import oracle
    from paper_1012_3615_gb300 import synth
    from paper_1012_3615_gb300.domain import OFFSETS, Decomposition, exchange

    L, bc = (3, 3, 4, 3), (1, -1, 1, -1)
    dec = Decomposition(L, (1, 1, 1, 1), bc)
    assert len(OFFSETS) == 80 and dec.E == (5, 5, 6, 5)
    U = synth.random_su3_links(L, 0.4, 9)
    psi = synth.gaussian_spinor(L, 1, 10)[0]
    Ue = exchange(dec, 0, torch.as_tensor(U), None, spinor=False).numpy()
    pe = exchange(dec, 0, torch.as_tensor(psi), None, spinor=True).numpy()
    out = oracle.apply(dec.E, (1, 1, 1, 1), oracle.build_hops(dec.E, Ue), -0.1, pe)[dec.interior()]
    ref = oracle.apply(L, bc, oracle.build_hops(L, U), -0.1, psi)
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max()
    # the halo regions tile the shell of the extended lattice exactly once
    shell = np.concatenate([dec.region(d)[0] for d in OFFSETS])
    assert len(set(shell.tolist())) == len(shell) == dec.Ve - dec.Vl
