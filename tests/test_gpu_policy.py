"""GPU parity of the inference-path loop (policy kernel, env step, rollout
ring) against the oracle: logits bit-exact in fp32, actions, observations,
rewards, dones and ring contents identical."""
import numpy as np
import pytest
import torch

from oracle import OracleEnvs
from paper_1907_08467_gb300 import synth
from paper_1907_08467_gb300.env import FORM_BATCHED, FORM_PLAIN, AtariEnv

pytestmark = pytest.mark.gpu


def _pair(w, form, n):
    luma = synth.luma_table()
    g = AtariEnv.from_workload(w, form=form)
    o = OracleEnvs([r.data for r in w.roms], [r.score_addr for r in w.roms], [r.gameover_addr for r in w.roms],
                   w.env_rom, luma=luma, seed=w.seed)
    return g, o


@pytest.mark.parametrize("form", [FORM_PLAIN, FORM_BATCHED])
def test_policy_logits_and_actions_bit_exact(form):
    w = synth.workload(5, n_envs=48)
    g, o = _pair(w, form, 48)
    W = synth.policy_weights(5)
    Wd = torch.from_numpy(W.view(np.int16)).cuda()
    obs_d = torch.zeros((48, 4, 84, 84), dtype=torch.uint8, device="cuda")
    obs_h = np.zeros((48, 4, 84, 84), np.uint8)
    logits = torch.empty((48, 18), dtype=torch.float32, device="cuda")
    for s in range(12):
        act_d = g.policy(obs_d, Wd, logits=logits)
        act_h, logit_h = o.policy(obs_h, W, n_threads=8)
        torch.cuda.synchronize()
        assert np.array_equal(logits.cpu().numpy().view(np.uint32), logit_h.view(np.uint32)), s
        assert np.array_equal(act_d.cpu().numpy(), act_h), s
        obs_d, rew_d, done_d = g.step(act_d)
        obs_h, rew_h, done_h = o.step(act_h, n_threads=8)
        assert np.array_equal(obs_d.cpu().numpy(), obs_h)
        assert np.array_equal(rew_d.cpu().numpy(), rew_h)
        assert np.array_equal(done_d.cpu().numpy(), done_h)


def test_rollout_ring_matches_oracle_loop():
    """Seven device iterations of policy -> step -> ring append (ring depth 5,
    wrapping) equal the oracle run of the same loop."""
    n, T, R = 32, 7, 5
    w = synth.workload(5, n_envs=n)
    g, o = _pair(w, FORM_BATCHED, n)
    W = synth.policy_weights(5)
    Wd = torch.from_numpy(W.view(np.int16)).cuda()
    obs = torch.zeros((n, 4, 84, 84), dtype=torch.uint8, device="cuda")
    act = torch.empty(n, dtype=torch.uint8, device="cuda")
    rew = torch.empty(n, dtype=torch.int32, device="cuda")
    done = torch.empty(n, dtype=torch.uint8, device="cuda")
    ring = torch.zeros((R, n, 84 * 84), dtype=torch.uint8, device="cuda")
    ring_r = torch.zeros((R, n), dtype=torch.float32, device="cuda")
    g.rollout(Wd, T, obs, act, rew, done, ring, ring_r, ring_start=0)
    torch.cuda.synchronize()
    obs_h = np.zeros((n, 4, 84, 84), np.uint8)
    ring_h = np.zeros((R, n, 84 * 84), np.uint8)
    ring_rh = np.zeros((R, n), np.float32)
    for t in range(T):
        a, _ = o.policy(obs_h, W, n_threads=8)
        obs_h, r, d = o.step(a, n_threads=8)
        ring_h[t % R] = obs_h[:, 3].reshape(n, -1)
        ring_rh[t % R] = r.astype(np.float32)
    assert np.array_equal(obs.cpu().numpy(), obs_h)
    assert np.array_equal(ring.cpu().numpy(), ring_h)
    assert np.array_equal(ring_r.cpu().numpy(), ring_rh)
    assert np.array_equal(g.state().cpu().numpy(), o.state())
