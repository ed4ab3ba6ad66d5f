"""Transport between the parts of a 4D domain decomposition held by different processes:
one part per process over torch.distributed (any backend that moves CPU tensors, e.g. gloo).
A part's rank is its grid position in lexicographic order, x fastest.  The library packs the
spin-projected faces and takes the block sums; this module only moves them: each face with
a point-to-point message tagged by its face index k = 2 mu + side, each sum with all_reduce
(the same result on every rank)."""
import datetime

import torch
import torch.distributed as dist

from . import dwf


def grid_rank(coord, grid) -> int:
    """Rank of the part at grid position coord (x fastest)."""
    return coord[0] + grid[0] * (coord[1] + grid[1] * (coord[2] + grid[2] * coord[3]))


def grid_coord(rank, grid) -> list:
    """Grid position of the part of the given rank."""
    c = []
    for g in grid:
        c.append(rank % g)
        rank //= g
    return c


class TorchPartComm:
    """The dwf_part_comm of the part at `coord` of `grid` (pass .comm to dwf_part_*_comm).
    timeout (seconds): how long a face message may take before the exchange fails (the
    library call then returns DWF_ECOMM), so that a part whose peer has failed does not wait
    for ever; None leaves it to the process group."""

    def __init__(self, grid, coord, group=None, timeout=None):
        self.grid, self.coord, self.group = list(grid), list(coord), group
        self.timeout = None if timeout is None else datetime.timedelta(seconds=timeout)
        self.comm = dwf.part_comm(self.exchange, self.allreduce)

    def neighbour(self, mu, side) -> int:
        """Rank of the part below (side 0) or above (side 1) along mu, periodic."""
        c = list(self.coord)
        c[mu] = (c[mu] + (1 if side else -1)) % self.grid[mu]
        return grid_rank(c, self.grid)

    def exchange(self, send, recv):
        """Face k goes to the neighbour on side k & 1 as message k; recv[k] is that neighbour's
        message k ^ 1 (its face towards this part)."""
        reqs = []
        for k in range(8):
            if send[k] is None:
                continue
            peer = self.neighbour(k >> 1, k & 1)
            reqs.append(dist.isend(torch.from_numpy(send[k]), peer, group=self.group, tag=k))
            reqs.append(dist.irecv(torch.from_numpy(recv[k]), peer, group=self.group, tag=k ^ 1))
        for r in reqs:
            if self.timeout is None:
                r.wait()
            elif not r.wait(self.timeout):
                raise TimeoutError("face message timed out")

    def allreduce(self, v):
        dist.all_reduce(torch.from_numpy(v), group=self.group)
