"""The row-sharded apply's partition and gather on world-size-2 and world-size-3 gloo process
groups on the CPU: every rank fills its row slice from the oracle's rows (the stand-in for
``vsie_apply_rows`` on its GPU) and the gathered vector equals the oracle's full apply on
every rank, for ragged splits too."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from oracle import vsie_oracle as O
    from paper_2607_06429_b300 import sharded as SH
    from paper_2607_06429_b300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.smooth_density_ball(6, 1, 1, 3.0)
    D = O.Discretisation.from_workload(w)
    x = W.random_vector(D.n, 5)

    calls = []

    def rows_fn(xt, r0, r1):
        calls.append((r0, r1))
        return torch.from_numpy(D.apply_rows(xt.numpy(), np.arange(r0, r1)))

    ap = SH.RowShardedApply(D.n, rows_fn)
    y = ap(torch.from_numpy(x)).numpy()
    q.put((rank, y, calls))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gathered_rows_equal_the_full_apply(world):
    sys.path.insert(0, ROOT)
    from oracle import vsie_oracle as O
    from paper_2607_06429_b300 import sharded as SH
    from paper_2607_06429_b300 import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = W.smooth_density_ball(6, 1, 1, 3.0)
    D = O.Discretisation.from_workload(w)
    ref = D.apply(W.random_vector(D.n, 5))
    parts = SH.row_partition(D.n, world)
    assert D.n % world != 0 or world == 2      # world 3 gives a ragged split here
    for rank, y, calls in out:
        assert calls == [parts[rank]]           # each rank computes only its own rows
        assert np.allclose(y, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_row_partition_is_contiguous_and_balanced():
    sys.path.insert(0, ROOT)
    from paper_2607_06429_b300 import sharded as SH
    for n in (0, 1, 7, 1772416):
        for world in (1, 2, 3, 8):
            parts = SH.row_partition(n, world)
            assert len(parts) == world and parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        SH.row_partition(5, 0)
