"""Multi-GPU sharding host logic, run as world-size-2 gloo process groups on
the CPU: the LPT partition and the gather of per-event results (per-event
work done by the oracle on small events)."""
import os
import socket

import numpy as np
import pytest

from paper_1309_6275_gb300 import shard


def test_partition_covers_every_event_once_and_balances():
    rng = np.random.default_rng(0)
    costs = np.exp(rng.uniform(np.log(2000), np.log(60000), 257)).astype(np.int64)
    for world in (1, 2, 3, 8):
        parts = shard.partition(costs, world)
        allv = np.sort(np.concatenate(parts))
        assert np.array_equal(allv, np.arange(costs.shape[0]))
        ld = shard.loads(costs, parts)
        # LPT: no rank exceeds another by more than the largest event
        assert max(ld) - min(ld) <= costs.max()
        # and LPT is within 4/3 of the lower bound on the makespan
        assert max(ld) <= 4 / 3 * max(costs.sum() / world, costs.max()) + 1
    # deterministic, and equal costs split evenly
    assert all(np.array_equal(a, b) for a, b in zip(shard.partition(costs, 4),
                                                   shard.partition(costs, 4)))
    eq = shard.partition(np.full(10, 7), 2)
    assert [len(p) for p in eq] == [5, 5]
    assert shard.partition([], 3)[0].shape == (0,)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_events, outdir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import oracle
    import synth
    from paper_1309_6275_gb300 import shard as sh
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    name = "single_64"
    g = synth.geometry_of(name)
    gen = synth.CONFIGS[name]["gen"]
    events = [synth.make_event(gen, 100 + e) for e in range(n_events)]
    parts = sh.partition([ev.n_hits for ev in events], world)
    local = {}
    for e in parts[rank]:
        ev = events[e]
        r = oracle.run_event(g, ev.x, ev.y, ev.z, threads=1)
        local[int(e)] = (int(r["count"]), r["peaks"].tobytes(), r["assign"].tobytes())
    merged = sh.gather_results(local)
    if rank == 0:
        import pickle
        with open(os.path.join(outdir, "merged.pkl"), "wb") as f:
            pickle.dump(merged, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_what_a_serial_run_computes(tmp_path):
    import pickle
    import torch.multiprocessing as tmp
    import oracle
    import synth
    n = 6
    tmp.spawn(_worker, args=(2, _free_port(), n, str(tmp_path)), nprocs=2, join=True)
    with open(tmp_path / "merged.pkl", "rb") as f:
        merged = pickle.load(f)
    assert sorted(merged) == list(range(n))
    g = synth.geometry_of("single_64")
    gen = synth.CONFIGS["single_64"]["gen"]
    for e in range(n):
        ev = synth.make_event(gen, 100 + e)
        r = oracle.run_event(g, ev.x, ev.y, ev.z, threads=1)
        assert merged[e] == (int(r["count"]), r["peaks"].tobytes(), r["assign"].tobytes())


def test_gather_without_a_process_group_is_local():
    assert shard.gather_results({3: "x"}) == {3: "x"}


def test_gather_rejects_an_event_done_twice(tmp_path):
    import torch.multiprocessing as tmp
    with pytest.raises(Exception):
        tmp.spawn(_dup_worker, args=(2, _free_port()), nprocs=2, join=True)


def _dup_worker(rank, world, port):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    from paper_1309_6275_gb300 import shard as sh
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sh.gather_results({0: rank})     # both ranks claim event 0: rank 0 raises
    finally:
        dist.destroy_process_group()


def _dead_rank_worker(rank, world, port, outdir):
    import sys
    from datetime import timedelta
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    from paper_1309_6275_gb300 import shard as sh
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=10))
    if rank == 1:
        os._exit(3)                      # dies between steps, before the gather
    try:
        sh.gather_results({0: "done"})
        msg = "gathered"
    except Exception as e:               # the peer is gone: an error, not a hang
        msg = f"failed: {type(e).__name__}"
    with open(os.path.join(outdir, "rank0.txt"), "w") as f:
        f.write(msg)
    os._exit(0)


def test_a_rank_that_dies_before_the_gather_is_reported_not_waited_for(tmp_path):
    """Failure detection on the host: rank 1 exits without joining the
    result gather; rank 0's gather ends with an error within the process
    group's timeout instead of hanging."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    ps = [ctx.Process(target=_dead_rank_worker, args=(r, 2, port, str(tmp_path)))
          for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(90)
    alive = [p for p in ps if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung"
    assert ps[1].exitcode == 3
    assert ps[0].exitcode == 0
    assert (tmp_path / "rank0.txt").read_text().startswith("failed")
