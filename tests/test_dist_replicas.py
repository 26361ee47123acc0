"""The multi-rank (torchrun) form of the benchmark: independent grids per rank, no collective on the
data path, job time = max over ranks.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    import gridgen
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def max_over(v):
        t = torch.tensor([v], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    local_ms = 10.0 * (rank + 1)          # rank 1 is the slow one
    t_max, value = bench.replica_throughput(local_ms, 1000, 4, world, max_over)
    # each rank's grid is its own and the oracle runs on it without any exchange
    x = gridgen.random_grid(64, bench.rank_seed(rank))
    y = oracle.forward(x)
    q.put((rank, t_max, value, float(x[0, 0]), float(y[33, 0])))
    dist.destroy_process_group()


def test_two_rank_replicas_weak_scaling():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, x0, y0), (r1, t1, v1, x1, y1) = res
    assert t0 == t1 == 20.0                          # max over ranks
    assert v0 == v1 == 2 * 1000 * 4 / 20e-3          # all ranks' points over the slowest time
    assert x0 != x1 and y0 != y1                     # independent grids


def test_single_rank_is_plain_throughput():
    import bench
    t, v = bench.replica_throughput(8.0, 2 ** 24, 10, 1)
    assert t == 8.0 and v == 2 ** 24 * 10 / 8e-3


def test_bench_gpus_flag_runs_that_many_replicas():
    """`bench.py --gpus 2` without a launcher re-runs itself as two ranks (torch.distributed.run, gloo on
    the CPU in launcher-check mode): rank 0 reports n_gpus = 2 and two different grids."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--launcher-check"],
                       capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(s) for s in r.stdout.splitlines() if s.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = lines[0]
    assert line["n_gpus"] == 2 and line["gpus_arg"] == 2
    ranks = sorted(line["ranks"], key=lambda v: v["rank"])
    assert [v["rank"] for v in ranks] == [0, 1]
    assert ranks[0]["seed"] != ranks[1]["seed"] and ranks[0]["grid_sha"] != ranks[1]["grid_sha"]


def test_bench_refuses_world_size_that_contradicts_gpus():
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "4", "--launcher-check"],
                       capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode == 2 and "WORLD_SIZE=1" in r.stderr


def test_lpt_partition_covers_and_balances():
    """The longest-processing-time split of a multi-domain batch: every subgrid on exactly one part,
    deterministic, and the largest share within the largest subgrid of the average share."""
    import random
    from paper_1804_10120_gb300.shard import lpt_partition
    import gridgen
    sizes = [s ** 3 for s in gridgen.subgrid_sides(600, 2)]
    for parts in (1, 2, 3, 8):
        split = lpt_partition(sizes, parts)
        assert len(split) == parts
        flat = sorted(i for p in split for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in split]
        assert max(loads) <= sum(sizes) / parts + max(sizes)
        assert split == lpt_partition(sizes, parts)
    assert lpt_partition([5, 5, 5], 2) == [[0, 2], [1]]          # ties: lower index first, lower part first
    assert lpt_partition([3, 1], 4) == [[0], [1], [], []]
    assert lpt_partition([], 3) == [[], [], []]
    rng = random.Random(4)
    for _ in range(50):
        sz = [rng.randint(0, 1000) for _ in range(rng.randint(1, 40))]
        m = rng.randint(1, 6)
        loads = [sum(sz[i] for i in p) for p in lpt_partition(sz, m)]
        assert sum(loads) == sum(sz) and max(loads) <= sum(sz) / m + max(sz)
    with pytest.raises(ValueError):
        lpt_partition([1], 0)
    with pytest.raises(ValueError):
        lpt_partition([-1], 2)


def test_bench_batched_form_shards_the_subgrids_across_ranks():
    """`bench.py --gpus 2 --only batched --launcher-check`: the two ranks (gloo on the CPU) hold disjoint
    LPT shares of the 600 subgrids whose point counts add up to the whole batch."""
    import json
    import subprocess
    import sys
    import gridgen
    from paper_1804_10120_gb300.shard import lpt_partition
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--only", "batched",
                        "--launcher-check"], capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [json.loads(s) for s in r.stdout.splitlines() if s.startswith("{")][0]
    ranks = sorted(line["ranks"], key=lambda v: v["rank"])
    sizes = [s ** 3 for s in gridgen.subgrid_sides(600, 2)]
    assert sum(v["grids"] for v in ranks) == 600 and sum(v["points"] for v in ranks) == sum(sizes)
    split = lpt_partition(sizes, 2)
    assert [v["points"] for v in ranks] == [sum(sizes[i] for i in p) for p in split]
    assert ranks[0]["indices_sha"] != ranks[1]["indices_sha"]
