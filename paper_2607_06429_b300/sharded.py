"""Row-sharded operator apply over several GPUs, one process per GPU.

Every collocation row of Eq. (vsie) sums over all far-field source points, so the rows are
independent and carry equal far-field work: rank r of G computes the contiguous rows
``row_partition(n, G)[r]`` of y = A x with ``vsie_apply_rows`` on its own device (each rank
holds the whole operator and all of x), and one all-gather assembles y on every rank.  The
all-gather is the only exchange of an apply.  Its payload is 16 bytes per unknown; the
charges q, u of the source points would be 20 to 48 bytes per point, with more points than
unknowns.  Peer memory is never an operand of a kernel: the collective lands every slice
in local buffers.

This module is argument plumbing around the library call and one torch.distributed
collective; the arithmetic of the apply runs in the library's kernels.
"""
from __future__ import annotations

from typing import Callable, List, Tuple


def row_partition(n: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous row ranges [r0, r1) of 0..n for ``world`` ranks, sizes differing by at most
    one (rows carry equal far-field work), earlier ranks taking the extra rows."""
    if world < 1 or n < 0:
        raise ValueError("world must be >= 1 and n >= 0")
    base, extra = divmod(n, world)
    out = []
    r0 = 0
    for r in range(world):
        r1 = r0 + base + (1 if r < extra else 0)
        out.append((r0, r1))
        r0 = r1
    return out


def gather_rows(local, n: int, world: int, group=None):
    """All-gather the row slices of ``world`` ranks (each rank's slice of ``row_partition``)
    into the full length-n complex vector on every rank.  Slices are padded to the largest
    slice so that one equal-size all-gather (NCCL or gloo) carries them; complex values
    travel as pairs of float64."""
    import torch
    import torch.distributed as dist
    parts = row_partition(n, world)
    width = max(r1 - r0 for r0, r1 in parts) if parts else 0
    send = torch.zeros((width, 2), dtype=torch.float64, device=local.device)
    if local.shape[0]:
        send[:local.shape[0]] = torch.view_as_real(local.contiguous())
    recv = torch.empty((world * width, 2), dtype=torch.float64, device=local.device)
    dist.all_gather_into_tensor(recv, send, group=group)
    full = torch.empty(n, dtype=torch.complex128, device=local.device)
    fr = torch.view_as_real(full)
    for r, (r0, r1) in enumerate(parts):
        fr[r0:r1] = recv[r * width:r * width + (r1 - r0)]
    return full


class RowShardedApply:
    """y = A x over the ranks of a process group, each rank computing its row slice.

    ``rows_fn(x, r0, r1)`` returns rows r0..r1-1 of A x on this rank (by default the
    library's ``Operator.apply_rows``); it is a parameter so that the partition and gather
    logic runs with any row source, e.g. on CPU ranks in tests."""

    def __init__(self, n: int, rows_fn: Callable, group=None):
        import torch.distributed as dist
        self.n = int(n)
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.rows = row_partition(self.n, self.world)[self.rank]
        self.rows_fn = rows_fn

    @classmethod
    def from_operator(cls, op, precision: int = 32, group=None):
        return cls(op.n, lambda x, r0, r1: op.apply_rows(x, r0, r1, precision=precision), group)

    def __call__(self, x):
        r0, r1 = self.rows
        local = self.rows_fn(x, r0, r1)
        return gather_rows(local, self.n, self.world, self.group)
