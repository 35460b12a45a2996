"""The domain-decomposed apply with two ranks, each a separate process that
drives the library on the GPU: the halos of links and spinors move between the
ranks through torch.distributed point-to-point calls (gloo, host memory), each
rank builds the hops and applies the operator on its extended block on the
device, and the interior outputs of both ranks equal the single-domain apply
of the same fields (FP64 to 1e-13, FP32 to 1e-6 of max |out|).

Both ranks share the one GPU; their kernels never wait on each other (every
exchange happens on the host between launches)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp
from mp_util import collect

from paper_1012_3615_gb300 import Brillouin, synth

pytestmark = pytest.mark.gpu


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

    from paper_1012_3615_gb300 import Brillouin, synth
    from paper_1012_3615_gb300.domain import Decomposition, exchange

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dev = torch.device("cuda", 0)
        dec = Decomposition(L, grid, bc)
        U = synth.random_su3_links(L, 0.4, 31)
        psi = synth.gaussian_spinor(L, 1, 32)[0]
        mine = dec.global_sites(rank)
        Ue = exchange(dec, rank, torch.as_tensor(U[mine]), dist, spinor=False)
        pe = exchange(dec, rank, torch.as_tensor(psi[mine]), dist, spinor=True)
        ext = Brillouin(dec.E, (1, 1, 1, 1))
        ext.build_hops(Ue.to(dev).contiguous(), prec="f32")
        x = pe.to(dev).unsqueeze(0).contiguous()
        idx = torch.as_tensor(dec.interior(), device=dev)
        out64 = ext.apply(x, 0.07)[0][idx].cpu().numpy()
        out32 = ext.apply(x.to(torch.complex64), 0.07, prec="f32")[0][idx].cpu().numpy()
        q.put((rank, mine, out64, out32))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("L,grid,bc", [((4, 4, 4, 6), (1, 1, 1, 2), (1, 1, 1, -1)),
                                       ((6, 4, 3, 4), (2, 1, 1, 1), (-1, 1, 1, -1))])
def test_two_ranks_on_the_gpu_equal_the_single_domain_apply(gpu, L, grid, bc):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, L, grid, bc, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = collect(q, procs, 2, 600)
    op = Brillouin(L, bc)
    op.build_hops(torch.as_tensor(synth.random_su3_links(L, 0.4, 31), device=gpu), prec="f32")
    x = torch.as_tensor(synth.gaussian_spinor(L, 1, 32), device=gpu)
    ref64 = op.apply(x, 0.07)[0].cpu().numpy()
    ref32 = op.apply(x.to(torch.complex64), 0.07, prec="f32")[0].cpu().numpy()
    covered = np.zeros(len(ref64), bool)
    for rank, sites, out64, out32 in got:
        assert np.abs(out64 - ref64[sites]).max() <= 1e-13 * np.abs(ref64).max(), rank
        assert np.abs(out32 - ref32[sites]).max() <= 1e-6 * np.abs(ref32).max(), rank
        covered[sites] = True
    assert covered.all()
