"""One cluster over several ranks (sections 3.2-3.5): the Eq. 17 partition
and the redistribution plan pinned by the paper's worked example, and the
sharded sort and duplicated-array potential on two and three gloo ranks on
the host, which must give the single-process sorted order and potential bit
for bit.  The per-rank compute is the oracle's here (test infrastructure);
on GPUs it is the library's kernels."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1206_5878_gb300 import shard  # noqa: E402


def test_partition_is_eq17_and_the_papers_example():
    # section 3.5's example: 450 stars on 4 processors are 120, 120, 100, 110
    s = shard.partition_starts(450, 4)
    assert s == [0, 120, 240, 340, 450]
    for rank in range(4):
        for i in (0, 7, s[rank + 1] - s[rank] - 1):
            assert shard.global_index(i, rank, 450, 4) == s[rank] + i
    # the processors received 100, 130, 140 and 80 stars after the sort; the
    # third holds global positions 230..369 and sends 230..239 to the second
    # processor and 340..369 to the fourth (the paper counts from 1)
    plan = shard.redistribution_counts([100, 130, 140, 80], 450, 4)
    assert plan[2] == [0, 10, 100, 30]
    assert plan[0] == [100, 0, 0, 0] and plan[1] == [20, 110, 0, 0]
    assert plan[3] == [0, 0, 0, 80]
    assert [sum(col) for col in zip(*plan)] == [120, 120, 100, 110]


@pytest.mark.parametrize("n,p", [(0, 3), (19, 2), (20, 2), (1013, 3), (10_000, 7), (123_457, 64)])
def test_partition_multiples_of_20(n, p):
    s = shard.partition_starts(n, p)
    sizes = [s[k + 1] - s[k] for k in range(p)]
    assert sum(sizes) == n and s[0] == 0
    assert all(x % 20 == 0 for x in sizes[:-1])
    # blocks of 20 differ by at most one between ranks; the last rank also
    # takes the n mod 20 leftover stars
    chunks = [x // 20 for x in sizes]
    assert max(chunks) - min(chunks) <= 1
    assert sizes[-1] % 20 == n % 20
    assert all(shard.global_index(0, k, n, p) == s[k] for k in range(p))


def test_sample_and_splitter_positions():
    assert shard.sample_positions(100, 4) == [12, 37, 62, 87]
    assert shard.sample_positions(3, 8) == [0, 1, 2]
    assert shard.sample_positions(0, 8) == []
    assert shard.splitter_positions(4 * 16, 16, 4) == [16, 32, 48]
    r = torch.tensor([1.0, 2.0, 2.0, 2.0, 5.0], dtype=torch.float64)
    i = torch.tensor([4, 1, 3, 9, 0], dtype=torch.int32)
    cuts = shard.cut_points(r, i, torch.tensor([2.0, 2.0], dtype=torch.float64),
                            torch.tensor([3, 10], dtype=torch.int32))
    assert cuts == [0, 2, 4, 5]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_sort(r, ids):
    import oracle
    return torch.from_numpy(oracle.sort_perm(r.numpy(), ids.numpy().view(np.uint32)))


def _oracle_potential(r, m):
    import oracle
    return torch.from_numpy(oracle.potential(r.numpy(), m.numpy(), "dd"))


def _state(n, seed):
    import initial_conditions as ic
    d = ic.plummer(n, seed=seed)
    g = np.random.default_rng(seed)
    d["r"] = d["r"] * g.uniform(0.5, 1.5, n)  # moved stars: any order
    d["r"][g.choice(n, n // 50, replace=False)] = np.inf  # escapers
    d["r"][:4] = d["r"][4]  # a tie in r, broken by id
    return d


def _rank(rank, world, port, n, seed, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d = _state(n, seed)
        # stars dealt to the ranks in an arbitrary, uneven way
        owner = np.random.default_rng(seed + 1).integers(0, world, n)
        mine = np.flatnonzero(owner == rank)
        rec = {k: torch.from_numpy(np.ascontiguousarray(d[k][mine])) for k in ("r", "vr", "vt", "m")}
        rec["id"] = torch.from_numpy(d["id"][mine].view(np.int32).copy())
        sc = shard.ShardedCluster(n, samples_per_rank=16, local_sort=_oracle_sort,
                                  potential=_oracle_potential)
        block = sc.sort(rec)
        phi_local, phi_all = sc.local_potential(block)
        q.put((rank, {k: v.numpy() for k, v in block.items()}, phi_local.numpy(),
               phi_all.numpy()))
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, 4_099), (3, 10_013)])
def test_sharded_sort_and_potential_equal_single_process(orc, world, n):
    seed = 5
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, world, port, n, seed, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(world)), key=lambda x: x[0])
    for p in ps:
        p.join(60)
    assert all(p.exitcode == 0 for p in ps)
    # the single-process reference: the whole cluster sorted by (r, id)
    d = _state(n, seed)
    perm = orc.sort_perm(d["r"], d["id"])
    starts = shard.partition_starts(n, world)
    for rank, blk, phi_local, phi_all in res:
        sl = slice(starts[rank], starts[rank + 1])
        for k in ("r", "vr", "vt", "m"):
            np.testing.assert_array_equal(blk[k], d[k][perm][sl], err_msg=k)
        np.testing.assert_array_equal(blk["id"].view(np.uint32), d["id"][perm][sl])
        nb = int(np.isfinite(d["r"]).sum())
        phi = np.zeros(n)
        phi[:nb] = orc.potential(d["r"][perm][:nb], d["m"][perm][:nb], "dd")
        np.testing.assert_array_equal(phi_all, phi)
        np.testing.assert_array_equal(phi_local, phi[sl])
    assert len(res[-1][1]["r"]) == starts[-1] - starts[-2]
    assert np.isinf(res[-1][1]["r"][-1])  # escapers on the last rank
