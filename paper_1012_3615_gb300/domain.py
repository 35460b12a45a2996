"""4D block domain decomposition of the lattice with depth-1 halos (the
multi-GPU form of the apply).

The lattice is cut into P0 x P1 x P2 x P3 blocks, one per rank.  A rank holds
its block of links and spinors plus a halo one site deep in all 80
directions (faces, edges, corners), i.e. an extended lattice of extents
l_mu + 2.  Every hop of an interior site x stays inside it, and both fields a
hop of x reads, W_d(x) and W_d(x - d)^dagger, are path sums over links of the
hypercube between x and x +- d (Sec. 5.1), also inside it.  So the
single-GPU library builds the hops and applies the operator on the extended
lattice unchanged (periodic in its own extents, which no interior hop uses)
and the outputs of the interior sites are those of the global operator.  The
fermion boundary phase of the global lattice is put on the halo spinors that
crossed a global boundary; links carry none.

Per apply only the spinor halo moves (the link halo once per gauge field):
for each offset d the source rank sends its slab of sites one layer deep
(a 3D face, 2D edge, 1D line or single corner site) to the rank at -d.  The
exchange is written against torch.distributed point-to-point calls (NCCL on
GPUs, gloo on CPUs); a rank that is its own neighbour copies locally.  The
Krylov dot products of a distributed solve add an all-reduce of the per-rank
FP64 partial sums.
"""
import itertools

import numpy as np

OFFSETS = [d for d in itertools.product((-1, 0, 1), repeat=4) if any(d)]


class Decomposition:
    """Blocks of extents L / P over a process grid P (rank = c0 + P0 (c1 + ...))."""

    def __init__(self, L, grid, bc=(1, 1, 1, -1)):
        self.L = tuple(int(v) for v in L)
        self.P = tuple(int(v) for v in grid)
        self.bc = tuple(int(v) for v in bc)
        for mu in range(4):
            if self.P[mu] < 1 or self.L[mu] % self.P[mu]:
                raise ValueError("grid must divide the lattice extents")
        self.l = tuple(self.L[mu] // self.P[mu] for mu in range(4))
        self.E = tuple(v + 2 for v in self.l)
        self.size = int(np.prod(self.P))
        self.Vl = int(np.prod(self.l))
        self.Ve = int(np.prod(self.E))
        self._regions = {}

    def coords(self, rank):
        c = []
        for mu in range(4):
            c.append(rank % self.P[mu])
            rank //= self.P[mu]
        return tuple(c)

    def rank_of(self, c):
        r, s = 0, 1
        for mu in range(4):
            r += (c[mu] % self.P[mu]) * s
            s *= self.P[mu]
        return r

    def _ext(self, x):
        """extended index of local coordinates x (each in [-1, l_mu])"""
        E = self.E
        return (x[0] + 1) + E[0] * ((x[1] + 1) + E[1] * ((x[2] + 1) + E[2] * (x[3] + 1)))

    def _grid(self, ranges):
        g = np.stack(np.meshgrid(*ranges, indexing="ij"), -1).reshape(-1, 4)
        # order: x0 fastest, like the site index
        return g[np.lexsort((g[:, 0], g[:, 1], g[:, 2], g[:, 3]))]

    def interior(self):
        """extended indices of the block's sites, in local site order"""
        x = self._grid([np.arange(self.l[mu]) for mu in range(4)])
        return self._ext(x.T)

    def global_sites(self, rank):
        """global site indices of the block's sites, in local site order"""
        c = self.coords(rank)
        x = self._grid([np.arange(self.l[mu]) for mu in range(4)])
        g = x + np.array([c[mu] * self.l[mu] for mu in range(4)])
        L = self.L
        return g[:, 0] + L[0] * (g[:, 1] + L[1] * (g[:, 2] + L[2] * g[:, 3]))

    def region(self, d):
        """(extended indices of the halo region in direction d, local site
        indices of the source rank's slab that fills it), in the same order"""
        if d not in self._regions:
            rr, sr = [], []
            for mu in range(4):
                if d[mu] > 0:
                    rr.append(np.array([self.l[mu]]))
                    sr.append(np.array([0]))
                elif d[mu] < 0:
                    rr.append(np.array([-1]))
                    sr.append(np.array([self.l[mu] - 1]))
                else:
                    rr.append(np.arange(self.l[mu]))
                    sr.append(np.arange(self.l[mu]))
            xr = self._grid(rr)
            xs = self._grid(sr)
            l = self.l
            src = xs[:, 0] + l[0] * (xs[:, 1] + l[1] * (xs[:, 2] + l[2] * xs[:, 3]))
            self._regions[d] = (self._ext(xr.T), src)
        return self._regions[d]

    def phase(self, rank, d):
        """fermion phase of the halo region d of rank: bc_mu for every direction
        in which the source block lies across a global boundary"""
        c = self.coords(rank)
        p = 1
        for mu in range(4):
            if d[mu] and not 0 <= c[mu] + d[mu] < self.P[mu]:
                p *= self.bc[mu]
        return p


def exchange(dec, rank, local, comm=None, spinor=True):
    """The extended array of rank from its local array (leading dimension the
    local sites, any trailing shape): interior copied, the 80 halo regions
    received from the neighbouring ranks (fermion phases applied when spinor).
    comm: torch.distributed (point-to-point) or None for a single rank."""
    import torch

    local = torch.as_tensor(local)
    ext = torch.zeros((dec.Ve,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    ext[torch.as_tensor(dec.interior(), device=local.device)] = local
    c = dec.coords(rank)
    pending = []
    for k, d in enumerate(OFFSETS):
        reg, src_slab = dec.region(d)
        src = dec.rank_of(tuple(c[mu] + d[mu] for mu in range(4)))
        dst = dec.rank_of(tuple(c[mu] - d[mu] for mu in range(4)))
        send = local[torch.as_tensor(src_slab, device=local.device)].contiguous()
        if src == rank and dst == rank:
            recv = send
        else:
            recv = torch.empty_like(send)
            sv = torch.view_as_real(send) if send.is_complex() else send
            rv = torch.view_as_real(recv) if recv.is_complex() else recv
            pending.append(comm.isend(sv, dst, tag=k))
            pending.append(comm.irecv(rv, src, tag=k))
        pending_fill = (reg, recv, dec.phase(rank, d) if spinor else 1)
        pending.append(pending_fill)
    for item in pending:
        if isinstance(item, tuple):
            continue
        item.wait()
    for item in pending:
        if isinstance(item, tuple):
            reg, recv, ph = item
            ext[torch.as_tensor(reg, device=local.device)] = recv if ph == 1 else -recv
    return ext
