"""The multi-GPU path of the benchmark is replicas (each rank steps its own
workers' data; no data-path collective): timing is the maximum over ranks and
the value the units of all ranks over that time.  Exercised with two gloo
ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    ms = bench.max_over_ranks(local_ms, world, "cpu")
    value = bench.weak_scaling_value(1.0, world, ms * 1e-3)
    out.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 150.0
        assert value == pytest.approx(2 / 0.150)


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.weak_scaling_value(512.0, 1, 2.0) == 256.0


# ---------------------------------------------------------------- worker sharding


def test_partition_balances_data_ciphertexts():
    from paper_2006_10091_gb300.sharding import partition_shards
    sizes = [5, 1, 9, 3, 3, 8, 2]
    parts = partition_shards(sizes, 3)
    assert sorted(k for p in parts for k in p) == list(range(len(sizes)))
    loads = [sum(sizes[k] for k in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)
    assert parts == partition_shards(sizes, 3)  # every rank computes the same partition
    assert partition_shards(sizes, 1) == [list(range(len(sizes)))]
    assert partition_shards([4], 2) == [[0], []]


def _oracle_and_cts(rank_seed_base=40):
    import oracle
    from paper_2006_10091_gb300 import workloads
    o = oracle.Oracle(8, 3, 40, 1, 60, 2.0 ** 40, seed=9)
    cts = [o.encrypt(workloads.int_poly(rank_seed_base + r, o.n, 1 << 30), 3, cid=r) for r in range(2)]
    return o, cts


def _oracle_add(o):
    import oracle
    import numpy as np

    def add(ctx, cts, out):
        acc = oracle.Ciphertext(cts[0].tensor.numpy().view(np.uint64).copy(), cts[0].level, cts[0].scale)
        for c in cts[1:]:
            acc = o.add(acc, oracle.Ciphertext(c.tensor.numpy().view(np.uint64).copy(), c.level, c.scale))
        out.tensor[:, : acc.level].copy_(torch.from_numpy(acc.data.view(np.int64)))
        out.level, out.scale = acc.level, acc.scale
        return out
    return add


def _shard_rank(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    import paper_2006_10091_gb300 as he
    from paper_2006_10091_gb300 import sharding
    o, cts = _oracle_and_cts()
    mine = cts[rank]
    ct = he.Ciphertext(torch.from_numpy(mine.data.view(np.int64).copy()), 3, 3, mine.scale)
    res = he.Ciphertext(torch.zeros((2, 3, o.n), dtype=torch.int64), 3)
    sharding.allreduce_ciphertext(None, ct, res, add=_oracle_add(o))
    got_sum = res.tensor.numpy().view(np.uint64).copy()
    # the key holder's residues reach every rank
    b = he.Ciphertext(torch.from_numpy(cts[0].data.view(np.int64).copy()) if rank == 0
                      else torch.zeros((2, 3, o.n), dtype=torch.int64), 3, 3 if rank == 0 else 0,
                      cts[0].scale if rank == 0 else 0.0)
    sharding.broadcast_ciphertext(b, 0)
    out.put((rank, got_sum, b.tensor.numpy().view(np.uint64).copy(), b.level, b.scale))
    dist.destroy_process_group()


def test_two_ranks_sum_weights_modulo_each_prime():
    """Two gloo ranks, each holding one worker's encrypted weights: the
    all-gathered residues summed modulo each prime equal the oracle's
    homomorphic addition of the two ciphertexts (Eq. 1), on both ranks; the
    key holder's broadcast reaches rank 1 with its level and scale."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import numpy as np
    o, cts = _oracle_and_cts()
    want = o.add(cts[0], cts[1]).data
    assert int(np.count_nonzero(want >= np.array(o.primes[:3], dtype=np.uint64)[None, :, None])) == 0
    plain = cts[0].data + cts[1].data  # the integer sum a plain all-reduce would give
    assert not np.array_equal(plain, want)
    for rank, got, bcast, level, scale in res:
        assert np.array_equal(got, want), rank
        assert np.array_equal(bcast, cts[0].data) and level == 3 and scale == cts[0].scale


# ---------------------------------------------------------------- refresh failures (host side)


def _check_in_rank(rank: int, port: int, scenario: str, out):
    import datetime
    import time
    from paper_2006_10091_gb300 import sharding
    store = dist.TCPStore("127.0.0.1", port, 2, rank == 0, timeout=datetime.timedelta(seconds=30))
    level, scale = 4, 2.0 ** 40
    try:
        if rank == 1 and scenario == "drop":  # the worker's refresh never arrives
            out.put((rank, "skipped", None))
            time.sleep(3.0)  # keep the connection while rank 0 waits
            return
        if rank == 1 and scenario == "stale":  # weights from an older step: one level more
            level = 5
        if rank == 1 and scenario == "delay":
            time.sleep(0.5)
        sharding.refresh_check_in(store, 7, rank, 2, level, scale, timeout_s=1.5 if scenario == "drop" else 10.0)
        out.put((rank, "ok", None))
    except sharding.RefreshError as e:
        out.put((rank, "error", e.code))
    if rank == 0:
        time.sleep(1.0)  # the store lives in rank 0: let rank 1 finish reading it


@pytest.mark.parametrize("scenario", ["ok", "delay", "drop", "stale"])
def test_refresh_check_in_detects_failed_ranks(scenario):
    """Two CPU ranks check in before the key holder's aggregation: on time or
    late but within the limit, both proceed; if rank 1's refresh never
    arrives, rank 0 gets HE_ETIMEOUT after the limit instead of blocking in a
    collective; if rank 1 brings weights at another level, both get HE_ESCALE."""
    import paper_2006_10091_gb300 as he
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_check_in_rank, args=(r, port, scenario, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (s, c)) for r, s, c in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    if scenario in ("ok", "delay"):
        assert res == {0: ("ok", None), 1: ("ok", None)}
    elif scenario == "drop":
        assert res[0] == ("error", he.HE_ETIMEOUT)
    else:
        assert res == {0: ("error", he.HE_ESCALE), 1: ("error", he.HE_ESCALE)}
