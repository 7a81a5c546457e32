"""Full-size GPU parity in the benchmark's launch configuration (batched form,
autotuned shape and grouping, the workloads' own env keys), against the
oracle, bit for bit:

- every env for the first 50 steps: observations (84x84x4 stacks), rewards,
  dones and the whole 256-byte canonical state after every step;
- then a seeded sample of 256 envs for several hundred more steps, long
  enough that episodes end and envs restart from the start-state cache on the
  device many times: the same outputs and the sample's full state after every
  step (the oracle runs just those envs, with their own keys, from step 0).

Workloads: 4096 envs over 8 sprite cartridges; 32768 envs over 32 banked
4 KB / F8 / F6 cartridges with sticky actions; the 16384-env inference loop
(policy kernel picking every action, rollout ring).
"""
import os

import numpy as np
import pytest
import torch

from oracle import OracleEnvs
from paper_1907_08467_gb300 import synth
from paper_1907_08467_gb300.env import FORM_BATCHED, AtariEnv

pytestmark = pytest.mark.gpu

THREADS = max(8, 2 * (os.cpu_count() or 4))   # oracle threads (contiguous env ranges; more than cores balances them)
ALL_STEPS = 50


def _oracle(w, idx):
    return OracleEnvs([r.data for r in w.roms], [r.score_addr for r in w.roms], [r.gameover_addr for r in w.roms],
                      [w.env_rom[i] for i in idx], luma=synth.luma_table(), env_key=np.asarray(idx),
                      seed=w.seed, sticky=w.sticky, output_mode=w.output_mode, frameskip=w.frameskip)


def _same(tag, got, exp):
    if not np.array_equal(got, exp):
        bad = np.argwhere(got != exp)
        raise AssertionError(f"{tag}: {len(bad)} mismatches, first at {tuple(bad[0])}")


def _sample(w, seed, k=256):
    """k envs spread over every cartridge (seeded)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(w.n_envs, k, replace=False))


@pytest.mark.parametrize("config,sample_steps", [(2, 600), (3, 1000)])
def test_full_size_every_env_then_long_sample(config, sample_steps):
    w = synth.workload(config)
    n = w.n_envs
    g = AtariEnv.from_workload(w, form=FORM_BATCHED)
    idx = _sample(w, 100 + config)
    o_all = _oracle(w, np.arange(n))
    o_s = _oracle(w, idx)
    acts = synth.actions(500 + config, ALL_STEPS + sample_steps, n)
    obs, rew, done = g.alloc_outputs()
    resets = 0
    for s in range(ALL_STEPS + sample_steps):
        g.step(torch.from_numpy(acts[s]).cuda(), obs, rew, done)
        so, sr, sd = o_s.step(acts[s][idx], n_threads=THREADS)
        if o_all is not None:
            ao, ar, ad = o_all.step(acts[s], n_threads=THREADS)
            torch.cuda.synchronize()
            _same(f"step {s} rewards", rew.cpu().numpy(), ar)
            _same(f"step {s} dones", done.cpu().numpy(), ad)
            _same(f"step {s} obs", obs.cpu().numpy(), ao)
            _same(f"step {s} state", g.state().cpu().numpy(), o_all.state())
            if s == ALL_STEPS - 1:
                o_all = None
        it = torch.from_numpy(idx).cuda()
        _same(f"step {s} sample rewards", rew[it].cpu().numpy(), sr)
        _same(f"step {s} sample dones", done[it].cpu().numpy(), sd)
        _same(f"step {s} sample obs", obs[it].cpu().numpy(), so)
        _same(f"step {s} sample state", g.state()[it].cpu().numpy(), o_s.state())
        resets += int(sd.sum())
    assert resets >= 100, resets            # many on-device resets inside the compared run
    assert int(g.status().abs().sum().item()) == 0


def test_full_size_inference_loop_every_env_then_long_sample():
    """The 16384-env inference loop as the benchmark runs it (one rollout
    iteration per step: policy, step, ring append): every env's action,
    stack, reward, done, ring plane and reward and state for 50 steps, then
    a 256-env sample for 600 more."""
    w = synth.workload(5)
    n, R, sample_steps = w.n_envs, 5, 600
    g = AtariEnv.from_workload(w, form=FORM_BATCHED)
    idx = _sample(w, 105)
    it = torch.from_numpy(idx).cuda()
    o_all = _oracle(w, np.arange(n))
    o_s = _oracle(w, idx)
    W = synth.policy_weights(w.seed)
    Wd = torch.from_numpy(W.view(np.int16)).cuda()
    obs = torch.zeros((n, 4, 84, 84), dtype=torch.uint8, device="cuda")
    act = torch.empty(n, dtype=torch.uint8, device="cuda")
    rew = torch.empty(n, dtype=torch.int32, device="cuda")
    done = torch.empty(n, dtype=torch.uint8, device="cuda")
    ring = torch.zeros((R, n, 84 * 84), dtype=torch.uint8, device="cuda")
    ring_r = torch.zeros((R, n), dtype=torch.float32, device="cuda")
    obs_a = np.zeros((n, 4, 84, 84), np.uint8)
    obs_s = np.zeros((len(idx), 4, 84, 84), np.uint8)
    resets = 0
    for t in range(ALL_STEPS + sample_steps):
        g.rollout(Wd, 1, obs, act, rew, done, ring, ring_r, ring_start=t)
        a_s, _ = o_s.policy(obs_s, W, n_threads=THREADS)
        obs_s, r_s, d_s = o_s.step(a_s, n_threads=THREADS)
        if o_all is not None:
            a_a, _ = o_all.policy(obs_a, W, n_threads=THREADS)
            obs_a, r_a, d_a = o_all.step(a_a, n_threads=THREADS)
            torch.cuda.synchronize()
            _same(f"step {t} actions", act.cpu().numpy(), a_a)
            _same(f"step {t} obs", obs.cpu().numpy(), obs_a)
            _same(f"step {t} rewards", rew.cpu().numpy(), r_a)
            _same(f"step {t} dones", done.cpu().numpy(), d_a)
            _same(f"step {t} ring plane", ring[t % R].cpu().numpy(), obs_a[:, 3].reshape(n, -1))
            _same(f"step {t} ring reward", ring_r[t % R].cpu().numpy(), r_a.astype(np.float32))
            _same(f"step {t} state", g.state().cpu().numpy(), o_all.state())
            if t == ALL_STEPS - 1:
                o_all = obs_a = None
        _same(f"step {t} sample actions", act[it].cpu().numpy(), a_s)
        _same(f"step {t} sample obs", obs[it].cpu().numpy(), obs_s)
        _same(f"step {t} sample rewards", rew[it].cpu().numpy(), r_s)
        _same(f"step {t} sample dones", done[it].cpu().numpy(), d_s)
        _same(f"step {t} sample state", g.state()[it].cpu().numpy(), o_s.state())
        resets += int(d_s.sum())
    assert resets >= 100, resets
    assert int(g.status().abs().sum().item()) == 0
