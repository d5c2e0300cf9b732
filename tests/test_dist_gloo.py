"""The multi-rank logic of the benchmark on CPU: two gloo ranks, weak scaling,
barrier and max-over-ranks timing (no GPU, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2006_12838_gb300 import dist as D
    assert D.init("gloo")
    r, w, lr = D.rank_info()
    D.barrier()
    fake_seconds = 1.0 + 0.5 * r            # rank 1 is the slower one
    m = D.max_over_ranks(fake_seconds)
    lo, hi = D.shard(1000, r, w)
    # batched curvature: whole fields per rank, balanced by interface cells;
    # each rank sums its own fields' work, the sum over ranks covers all
    import torch
    work = [5538, 120000, 300, 56478, 2691, 0, 77777, 1024]
    mine = [i for i, o in enumerate(D.assign_fields(work, w)) if o == r]
    t = torch.tensor([sum(work[i] for i in mine)], dtype=torch.float64)
    import torch.distributed as dist
    dist.all_reduce(t)
    D.barrier()
    q.put((r, m, lo, hi, D.weak_scaling_value(1 << 28, w, 10, m), float(t.item()), mine))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert out[0][1] == out[1][1] == 1.5                      # max over ranks
    assert (out[0][2], out[0][3], out[1][2], out[1][3]) == (0, 500, 500, 1000)
    assert out[0][4] == pytest.approx((1 << 28) * 2 * 10 / 1.5)
    work = [5538, 120000, 300, 56478, 2691, 0, 77777, 1024]
    assert out[0][5] == out[1][5] == sum(work)                 # every field on one rank
    assert sorted(out[0][6] + out[1][6]) == list(range(len(work)))


def test_assign_fields_balances_whole_fields():
    from paper_2006_12838_gb300 import dist as D
    import random
    rnd = random.Random(5)
    for world in (1, 2, 3, 8):
        for _ in range(20):
            work = [rnd.randint(0, 200000) for _ in range(rnd.randint(0, 70))]
            owner = D.assign_fields(work, world)
            assert len(owner) == len(work) and all(0 <= o < world for o in owner)
            loads = [sum(w for w, o in zip(work, owner) if o == r) for r in range(world)]
            # the greedy bound: no rank exceeds the mean by more than one field
            if work:
                assert max(loads) <= sum(work) / world + max(work)
            assert owner == D.assign_fields(list(work), world)     # deterministic


def test_shard_covers_everything():
    from paper_2006_12838_gb300 import dist as D
    for n in (0, 1, 7, 1000, 12345):
        for w in (1, 2, 3, 8):
            ranges = [D.shard(n, r, w) for r in range(w)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            assert max(b - a for a, b in ranges) - min(b - a for a, b in ranges) <= 1
