"""GPU tests of the serving loop: a session's results are bit-identical alone,
in a mix of concurrent sessions, and through a plain batched env (and the
oracle) with the same keys; admission by budget; busy and idle rules; the
native load generator."""
import threading
import time

import numpy as np
import pytest
import torch

from oracle import OracleEnvs
from paper_1907_08467_gb300 import synth
from paper_1907_08467_gb300.env import FORM_BATCHED, AtariEnv
from paper_1907_08467_gb300.server import EAGAIN, EBUSY, ESESSION, AtariServer, ServerError, footprint

pytestmark = pytest.mark.gpu

# cartridges of the banked workload: 4 KB, F8 and F6 bank switching
ROM_IDX = [0, 1, 12, 13, 22, 23]
STEPS = 6


@pytest.fixture(scope="module")
def roms():
    w = synth.workload(3, n_envs=32)
    return [w.roms[i] for i in ROM_IDX]


def _server(roms, **kw):
    kw.setdefault("sticky", True)
    kw.setdefault("seed", 3)
    return AtariServer.from_roms(roms, **kw)


def _run_session(srv, rom, n, key, acts, pinned=False):
    s = srv.open(rom, n, key)
    out = []
    for t in range(acts.shape[0]):
        if pinned:
            obs = torch.empty((n, 4, 84, 84), dtype=torch.uint8).pin_memory()
            o, r, d = s.step(acts[t], obs=obs)
            o = o.numpy()
        else:
            o, r, d = s.step(acts[t])
        out.append((o.copy(), r.copy(), d.copy()))
    s.close()
    return out


SESSIONS = [(0, 37, 1 << 11), (4, 5, 2 << 11), (2, 64, 3 << 11), (5, 130, 4 << 11), (0, 1, 5 << 11)]


def test_mix_equals_alone_equals_env(roms):
    rng = np.random.default_rng(11)
    acts = {i: rng.integers(0, 18, (STEPS, n), dtype=np.uint8) for i, (_, n, _) in enumerate(SESSIONS)}
    srv = _server(roms, budget_bytes=4 << 30, max_slots=1024)
    mix = {}

    def client(i):
        rom, n, key = SESSIONS[i]
        mix[i] = _run_session(srv, rom, n, key, acts[i], pinned=(i % 2 == 1))

    th = [threading.Thread(target=client, args=(i,)) for i in range(len(SESSIONS))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    st = srv.stats()
    assert st["requests"] == STEPS * len(SESSIONS)
    assert st["free_slots"] == st["capacity"]
    # alone, one session at a time on the same server
    for i, (rom, n, key) in enumerate(SESSIONS):
        alone = _run_session(srv, rom, n, key, acts[i])
        for t in range(STEPS):
            for a, b in zip(mix[i][t], alone[t]):
                assert np.array_equal(a, b), (i, t)
    srv.close()
    # a plain batched env with the same cartridge list and keys
    for i, (rom, n, key) in enumerate(SESSIONS):
        env = AtariEnv([r.data for r in roms], [(r.score_addr, r.gameover_addr) for r in roms], [rom] * n,
                       luma=synth.luma_table(), env_key=np.arange(n, dtype=np.uint32) + np.uint32(key),
                       form=FORM_BATCHED, sticky=True, seed=3, envs_per_warp=32, envs_per_block=128)
        for t in range(STEPS):
            o, r, d = env.step(torch.from_numpy(acts[i][t]).cuda())
            torch.cuda.synchronize()
            assert np.array_equal(o.cpu().numpy(), mix[i][t][0]), (i, t)
            assert np.array_equal(r.cpu().numpy(), mix[i][t][1]), (i, t)
            assert np.array_equal(d.cpu().numpy(), mix[i][t][2]), (i, t)
        env.close()


def test_session_matches_oracle(roms):
    rom, n, key = 4, 9, 77 << 11
    acts = synth.actions(5, STEPS, n)
    srv = _server(roms, budget_bytes=1 << 30, max_slots=64)
    got = _run_session(srv, rom, n, key, acts)
    srv.close()
    o = OracleEnvs([r.data for r in roms], [r.score_addr for r in roms], [r.gameover_addr for r in roms],
                   [rom] * n, sticky=True, seed=3, luma=synth.luma_table(),
                   env_key=np.arange(n, dtype=np.uint32) + np.uint32(key))
    for t in range(STEPS):
        oo, orw, od = o.step(acts[t], n_threads=4)
        assert np.array_equal(got[t][0], oo), t
        assert np.array_equal(got[t][1], orw), t
        assert np.array_equal(got[t][2], od), t


def test_admission_by_budget(roms):
    cfg = dict(sticky=True, seed=3)
    budget = footprint(100, 100, len(roms), **cfg)
    srv = _server(roms, budget_bytes=budget)
    st = srv.stats()
    assert st["capacity"] == 100 and st["bytes_in_use"] <= budget
    a = srv.open(0, 60, 0)
    with pytest.raises(ServerError) as e:
        srv.open(1, 50, 4096, timeout_ms=100)        # 40 free: not admitted in time
    assert e.value.rc == EAGAIN
    got = {}

    def late():
        got["s"] = srv.open(1, 50, 4096)             # waits until `a` closes
    t = threading.Thread(target=late)
    t.start()
    time.sleep(0.2)
    assert t.is_alive() and srv.stats()["queued_sessions"] == 1
    a.step(np.zeros(60, np.uint8), want_obs=False)
    a.close()
    t.join(timeout=10)
    assert not t.is_alive() and got["s"].n == 50
    st = srv.stats()
    assert st["free_slots"] == 50 and st["bytes_in_use"] <= budget
    with pytest.raises(ServerError) as e:
        srv.open(0, 101, 0)
    assert e.value.rc in (-22, -12)
    got["s"].close()
    srv.close()


def test_busy_and_idle_reclaim(roms):
    srv = _server(roms, budget_bytes=1 << 30, max_slots=64, idle_timeout_ms=150)
    s = srv.open(3, 8, 123)
    s.step(np.ones(8, np.uint8))
    time.sleep(0.5)                                   # idle past the timeout: reclaimed
    assert srv.stats()["free_slots"] == 64
    with pytest.raises(ServerError) as e:
        s.step(np.ones(8, np.uint8))
    assert e.value.rc == ESESSION
    # two steps of one session at once: the second is refused, never mixed in
    s2 = srv.open(3, 8, 456)
    errs = []

    def stepper():
        for _ in range(20):
            try:
                s2.step(np.ones(8, np.uint8), want_obs=False)
            except ServerError as ex:
                errs.append(ex.rc)
    th = [threading.Thread(target=stepper) for _ in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert set(errs) <= {EBUSY}
    s2.close()
    srv.close()


def test_loadgen_smoke(roms):
    srv = _server(roms, budget_bytes=2 << 30, max_slots=2048)
    r = srv.loadgen(n_clients=8, seconds=2.0, think_mean_ms=2.0, min_envs=1, max_envs=128, session_steps_mean=10,
                    seed=1, want_obs=True)
    assert r["requests"] > 20 and r["frames"] == 4 * r["env_steps"] > 0
    assert 0 < r["p50_ms"] <= r["p99_ms"] <= r["max_ms"]
    assert r["ticks"] > 0 and r["mean_tick_envs"] >= 1
    st = srv.stats()
    assert st["free_slots"] == st["capacity"] and st["pending_requests"] == 0
    srv.close()


@pytest.mark.parametrize("inflight", [1, 2])
def test_ticks_overlap_on_the_device(roms, inflight):
    """Continuous batching overlaps ticks on the GPU, not only on the host:
    with two tick contexts in flight and enough clients to keep both busy,
    ticks begin on the device (CUDA events on their streams) before the
    previous tick has ended; with one context they never do."""
    srv = _server(roms, budget_bytes=4 << 30, max_slots=4096, inflight=inflight)
    r = srv.loadgen(n_clients=32, seconds=3.0, think_mean_ms=0.5, min_envs=64, max_envs=256,
                    session_steps_mean=20, seed=7, want_obs=True)
    st = srv.stats()
    srv.close()
    assert r["ticks"] >= 10
    if inflight == 1:
        assert st["overlapped_ticks"] == 0
    else:
        assert st["overlapped_ticks"] > 0, (st["overlapped_ticks"], r["ticks"])
