"""The multi-GPU form is replicas only: every rank runs the whole workload
with disjoint env keys, and only the timing and the whole-job frame count
cross ranks.  This runs bench.py's replica helpers as two gloo ranks on the
CPU: value = frames of all ranks / slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import sys
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK="0")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    w, r, local = bench.dist_setup(backend="gloo")
    seconds = [0.50, 0.80][r]             # this rank's timed region
    frames = [4096 * 4 * 10, 4096 * 4 * 10][r]
    t_max = bench.allreduce_max(seconds, w)
    f_all = bench.allreduce_sum(frames, w)
    keys = bench.replica_env_keys(4096, r)
    bench.barrier(w)
    out.put((r, w, t_max, f_all, int(keys[0]), int(keys[-1])))
    dist.destroy_process_group()


def test_two_gloo_replicas_report_whole_job_throughput():
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
    (r0, w0, t0, f0, a0, b0), (r1, w1, t1, f1, a1, b1) = res
    assert w0 == w1 == 2
    assert t0 == t1 == 0.80                         # the slowest rank's time
    assert f0 == f1 == 2 * 4096 * 4 * 10            # units of all ranks
    assert (a0, b0) == (0, 4095) and (a1, b1) == (4096, 8191)   # disjoint env keys


def _replica_rank(rank, ws, port, out):
    import sys
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK="0")
    sys.path.insert(0, ROOT)
    import time

    import numpy as np
    import torch.distributed as dist

    import bench
    from oracle import OracleEnvs
    from paper_1907_08467_gb300 import synth
    w, r, _ = bench.dist_setup(backend="gloo")
    wl = synth.workload(2, n_envs=24)
    keys = bench.replica_env_keys(wl.n_envs, r)
    o = OracleEnvs([x.data for x in wl.roms], [x.score_addr for x in wl.roms], [x.gameover_addr for x in wl.roms],
                   wl.env_rom, luma=synth.luma_table(), env_key=keys, seed=wl.seed)
    acts = synth.actions(5, 6, wl.n_envs)
    bench.barrier(w)
    t0 = time.perf_counter()
    rews = []
    for s in range(6):
        _, rew, _ = o.step(acts[s])
        rews.append(rew)
    dt = time.perf_counter() - t0
    t_max = bench.allreduce_max(dt, w)
    frames = bench.allreduce_sum(wl.n_envs * 4 * 6, w)
    out.put((r, keys.tolist(), np.stack(rews).tolist(), o.state().tolist(), t_max, frames, dt))
    dist.destroy_process_group()


def test_two_gloo_replicas_run_disjoint_envs_of_one_batch():
    """Each of two gloo ranks runs the workload's replica (the oracle here, on
    the CPU) with its own env keys; the ranks together equal one batch of
    twice the envs keyed 0..2n-1, element by element; the reported time is
    the slowest rank's and the frame count is the sum over ranks."""
    import numpy as np

    from oracle import OracleEnvs
    from paper_1907_08467_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = synth.workload(2, n_envs=24)
    both = OracleEnvs([x.data for x in wl.roms], [x.score_addr for x in wl.roms], [x.gameover_addr for x in wl.roms],
                      wl.env_rom + wl.env_rom, luma=synth.luma_table(), env_key=np.arange(48), seed=wl.seed)
    acts = synth.actions(5, 6, wl.n_envs)
    rews = [both.step(np.concatenate([acts[s], acts[s]]))[1] for s in range(6)]
    st = both.state()
    for r, keys, rew, state, t_max, frames, dt in res:
        assert keys == list(range(24 * r, 24 * r + 24))
        assert np.array_equal(np.asarray(rew), np.stack(rews)[:, 24 * r:24 * r + 24])
        assert np.array_equal(np.asarray(state, np.uint8), st[24 * r:24 * r + 24])
        assert frames == 2 * 24 * 4 * 6 and t_max >= dt
    assert res[0][4] == res[1][4]
