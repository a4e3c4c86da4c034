"""The multi-GPU exchange step on CPU ranks (gloo, world size 2).

Paths shard across ranks with no exchange; the one exchange is the merge of
per-station statistics.  Each rank takes its own path ranges (rank-interleaved
blocks, as bench.py does), reduces them to station states (n, mean, M2 of u and
d, steps), all-gathers the states and merges them with mcg_states_merge in
rank order.  The merged statistics must equal the single-process statistics
of all paths, and every rank must get the identical answer.  Per-path values
come from the oracle (the GPU is not needed for the host-side logic).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1709_07469_gb300 import build as B
from paper_1709_07469_gb300 import mcgrav as M

N_PATHS, BLOCK, S = 1200, 100, 5


def per_path_values():
    import oracle
    from paper_1709_07469_gb300 import workloads as W
    from tests.helpers import oracle_spec
    w = W.sphere_line(paths=N_PATHS, dt=4e-3).with_(stations=W.sphere_line().stations[:S])
    r = oracle.solve(oracle_spec(w), w.stations, N_PATHS, per_path=True, threads=2)
    return r.pp_u, r.pp_d, r.pp_steps


def state_of(u, d, steps):
    """Two-pass statistics of one rank's paths, per station -> [S, 8]."""
    out = np.zeros((u.shape[0], 8))
    for s in range(u.shape[0]):
        out[s, 0] = u.shape[1]
        out[s, 1] = u[s].mean()
        out[s, 2] = np.sum((u[s] - out[s, 1]) ** 2)
        out[s, 3] = d[s].mean()
        out[s, 4] = np.sum((d[s] - out[s, 3]) ** 2)
        out[s, 5] = steps[s].sum()
    return out


def worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        M.load()
        u, d, steps = per_path_values()
        blocks = [b for b in range(N_PATHS // BLOCK) if b % world == rank]
        cols = np.concatenate([np.arange(b * BLOCK, (b + 1) * BLOCK) for b in blocks])
        mine = torch.from_numpy(state_of(u[:, cols], d[:, cols], steps[:, cols]))
        gathered = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(gathered, mine)
        merged = M.mcg_states_merge(torch.stack(gathered).numpy())
        q.put((rank, merged))
    finally:
        dist.destroy_process_group()


def bench_worker(rank, world, port, q):
    """The benchmark's own exchange step (bench.merge_rank_states), on gloo."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        M.load()
        u, d, steps = per_path_values()
        blocks = [b for b in range(N_PATHS // BLOCK) if b % world == rank]
        cols = np.concatenate([np.arange(b * BLOCK, (b + 1) * BLOCK) for b in blocks])
        mine = torch.from_numpy(state_of(u[:, cols], d[:, cols], steps[:, cols]).reshape(-1).copy())
        merged = bench.merge_rank_states(M, mine, S, world)
        q.put((rank, merged.numpy().reshape(S, 8)))
    finally:
        dist.destroy_process_group()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2])
def test_sharded_states_merge_to_single_process(world):
    B.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    u, d, steps = per_path_values()
    ref = state_of(u, d, steps)
    for r in range(world):
        got = results[r]
        assert np.array_equal(got, results[0])          # every rank, same answer
        assert np.array_equal(got[:, 0], ref[:, 0])
        np.testing.assert_allclose(got[:, [1, 3]], ref[:, [1, 3]], rtol=1e-13)
        np.testing.assert_allclose(got[:, [2, 4]], ref[:, [2, 4]], rtol=1e-11)
        assert np.array_equal(got[:, 5], ref[:, 5])


def test_merge_rank_order_and_empty_parts():
    M.load()
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 900))
    parts = np.stack([state_of(x[:, :300], x[:, :300], np.ones((3, 300))),
                      np.zeros((3, 8)),                                  # an idle rank
                      state_of(x[:, 300:], x[:, 300:], np.ones((3, 600)))])
    got = M.mcg_states_merge(parts)
    ref = state_of(x, x, np.ones((3, 900)))
    np.testing.assert_allclose(got[:, :6], ref[:, :6], rtol=1e-12)


def test_bench_exchange_step_on_gloo():
    """bench.py's N > 1 branch merges the ranks' station states with this
    function; on two gloo ranks it gives every rank the single-process
    statistics of all paths."""
    B.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=bench_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    u, d, steps = per_path_values()
    ref = state_of(u, d, steps)
    assert np.array_equal(results[0], results[1])
    assert np.array_equal(results[0][:, 0], ref[:, 0])
    np.testing.assert_allclose(results[0][:, [1, 3]], ref[:, [1, 3]], rtol=1e-13)
    np.testing.assert_allclose(results[0][:, [2, 4]], ref[:, [2, 4]], rtol=1e-11)
