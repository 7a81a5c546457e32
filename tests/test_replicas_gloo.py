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
