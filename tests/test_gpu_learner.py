"""GPU parity of the learner-side targets (N-step returns, V-trace targets and
advantages over a device rollout ring) against the double-precision oracle,
and of the training buffer the rollout loop fills (dones and behaviour
probabilities of the sampled actions) against the oracle loop, bit for bit.

Tolerance of the fp32 kernels, derived from their arithmetic (u = 2^-24, one
rounding per operation, each step reusing the next step's rounded result):
a step adds at most a few roundings of the magnitudes it combines, and the
error carried from step t+1 is scaled by gamma_t (N-step) or gamma_t c_t
(V-trace) <= 1.  So with M_t the sum of the magnitudes step t combines,
|err_t| <= 6 u M_t + gamma_t c_t |err_{t+1}|, summed from the end of the
rollout; the advantage adds 6 u rho_t (|r_t| + |v_{t+1}| + |V_t|) and
rho_t gamma_t |err_{t+1}|.  The tests compute that bound from the oracle's
values element by element.
"""
import numpy as np
import pytest
import torch

from oracle import OracleEnvs, nstep_returns, policy_mu, vtrace
from paper_1907_08467_gb300 import synth
from paper_1907_08467_gb300.env import FORM_BATCHED, AtariEnv, AtariError
from paper_1907_08467_gb300.env import nstep_returns as g_nstep
from paper_1907_08467_gb300.env import vtrace as g_vtrace

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _ordered(ring, depth, start, T):
    return np.stack([ring[(start + t) % depth] for t in range(T)])


def _nstep_tol(r, d, R, V_T, g):
    T = r.shape[0]
    tol = np.zeros_like(R)
    carry = np.zeros(R.shape[1])
    for t in range(T - 1, -1, -1):
        gt = np.where(d[t] != 0, 0.0, g)
        nxt = R[t + 1] if t + 1 < T else V_T
        carry = 6 * U * (np.abs(r[t]) + np.abs(R[t]) + gt * np.abs(nxt)) + gt * carry
        tol[t] = carry
    return tol + 1e-30


def _vtrace_tol(r, d, V, pi, mu, vs, g, rho_bar, c_bar):
    T = r.shape[0]
    ratio = pi.astype(np.float64) / mu.astype(np.float64)
    rho = np.minimum(rho_bar, ratio)
    c = np.minimum(c_bar, ratio)
    tv, ta = np.zeros_like(vs), np.zeros_like(vs)
    carry = np.zeros(vs.shape[1])
    for t in range(T - 1, -1, -1):
        gt = np.where(d[t] != 0, 0.0, g)
        vn = vs[t + 1] if t + 1 < T else V[T]
        m = (np.abs(V[t]) + rho[t] * (np.abs(r[t]) + np.abs(V[t + 1]) + np.abs(V[t])) + np.abs(vs[t])
             + c[t] * (np.abs(vn) + np.abs(V[t + 1])))
        ta[t] = 6 * U * rho[t] * (np.abs(r[t]) + np.abs(vn) + np.abs(V[t])) + rho[t] * gt * carry
        carry = 6 * U * m + gt * c[t] * carry
        tv[t] = carry
    return tv + 1e-30, ta + 1e-30


def _inputs(seed, depth, n, T):
    rng = np.random.default_rng(seed)
    rew = rng.integers(-4, 9, size=(depth, n)).astype(np.float32)
    done = (rng.random((depth, n)) < 0.2).astype(np.uint8)
    mu = rng.uniform(0.02, 1.0, size=(depth, n)).astype(np.float32)
    vals = rng.normal(0, 3, size=(T + 1, n)).astype(np.float32)
    pi = rng.uniform(0.0, 1.0, size=(T, n)).astype(np.float32)
    return rew, done, mu, vals, pi


@pytest.mark.parametrize("depth,start,T,n", [(5, 0, 5, 1), (7, 5, 5, 1000), (16, 13, 9, 4097), (5, 9, 3, 33)])
@pytest.mark.parametrize("g,rho_bar,c_bar", [(0.99, 1.0, 1.0), (0.9, 2.0, 0.5)])
def test_targets_match_oracle_within_fp32_bound(depth, start, T, n, g, rho_bar, c_bar):
    """Seeded rollouts with ragged env counts and ring offsets that wrap."""
    rew, done, mu, vals, pi = _inputs(depth * 1000 + n, depth, n, T)
    d = lambda a: torch.from_numpy(a).cuda()
    R_g = g_nstep(d(rew), d(done), d(vals), T, g, ring_start=start).cpu().numpy()
    vs_g, adv_g = g_vtrace(d(rew), d(done), d(mu), d(vals), d(pi), T, g, rho_bar, c_bar, ring_start=start)
    r_o, d_o, m_o = (_ordered(x, depth, start, T) for x in (rew, done, mu))
    R_o = nstep_returns(r_o, d_o, vals, g)
    vs_o, adv_o = vtrace(r_o, d_o, vals, pi, m_o, g, rho_bar, c_bar)
    assert (np.abs(R_g - R_o) <= _nstep_tol(r_o, d_o, R_o, vals[T].astype(np.float64), g)).all()
    tv, ta = _vtrace_tol(r_o, d_o, vals.astype(np.float64), pi, m_o, vs_o, g, rho_bar, c_bar)
    assert (np.abs(vs_g.cpu().numpy() - vs_o) <= tv).all()
    assert (np.abs(adv_g.cpu().numpy() - adv_o) <= ta).all()


def test_special_cases_and_argument_errors():
    """Every step done: returns are the rewards and the targets V + rho (r - V);
    pi = mu with unit truncation: targets are the N-step returns (to the fp32
    bound); n = 0 is a no-op; T > ring_depth, rho_bar < c_bar and gamma > 1
    are rejected."""
    T, n = 4, 300
    rew, done, mu, vals, pi = _inputs(3, T, n, T)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ones = np.ones_like(done)
    R = g_nstep(d(rew), d(ones), d(vals), T, 0.9).cpu().numpy()
    assert np.array_equal(R, rew)
    vs, _ = g_vtrace(d(rew), d(done), d(mu), d(vals), d(mu[:T]), T, 0.95, 1.0, 1.0)
    R2 = nstep_returns(rew, done, vals, 0.95)
    assert (np.abs(vs.cpu().numpy() - R2) <= 1e-4 * (1 + np.abs(R2))).all()
    z = torch.zeros((T, 0), dtype=torch.float32, device="cuda")
    g_nstep(z, z.to(torch.uint8), torch.zeros((T + 1, 0), device="cuda"), T, 0.9)
    with pytest.raises(AtariError):
        g_nstep(d(rew[:3]), d(done[:3]), d(vals), T, 0.9)
    with pytest.raises(AtariError):
        g_vtrace(d(rew), d(done), d(mu), d(vals), d(pi), T, 0.9, 0.5, 1.0)
    with pytest.raises(AtariError):
        g_nstep(d(rew), d(done), d(vals), T, 1.5)


def test_rollout_buffer_and_vtrace_against_the_oracle_loop():
    """Seven device iterations of policy -> step -> ring append into a 5-deep
    ring that also keeps dones and behaviour probabilities: the ring equals
    the oracle loop's (mu bit-exact: the same fp32 weights, total and
    division); then V-trace over the ring's five steps in order (start slot
    2) with seeded values and target probabilities matches the oracle."""
    n, T, R = 64, 7, 5
    w = synth.workload(5, n_envs=n)
    g = AtariEnv.from_workload(w, form=FORM_BATCHED)
    o = OracleEnvs([r.data for r in w.roms], [r.score_addr for r in w.roms], [r.gameover_addr for r in w.roms],
                   w.env_rom, luma=synth.luma_table(), seed=w.seed)
    W = synth.policy_weights(w.seed)
    Wd = torch.from_numpy(W.view(np.int16)).cuda()
    obs = torch.zeros((n, 4, 84, 84), dtype=torch.uint8, device="cuda")
    act = torch.empty(n, dtype=torch.uint8, device="cuda")
    rew = torch.empty(n, dtype=torch.int32, device="cuda")
    done = torch.empty(n, dtype=torch.uint8, device="cuda")
    ring = torch.zeros((R, n, 84 * 84), dtype=torch.uint8, device="cuda")
    ring_r = torch.zeros((R, n), dtype=torch.float32, device="cuda")
    ring_d = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    ring_mu = torch.zeros((R, n), dtype=torch.float32, device="cuda")
    g.rollout_ex(Wd, T, obs, act, rew, done, ring, ring_r, ring_d, ring_mu, ring_start=0)
    torch.cuda.synchronize()
    obs_h = np.zeros((n, 4, 84, 84), np.uint8)
    rd_h = np.zeros((R, n), np.uint8)
    rr_h = np.zeros((R, n), np.float32)
    mu_h = np.zeros((R, n), np.float32)
    for t in range(T):
        a, logits = o.policy(obs_h, W, n_threads=8)
        mu_h[t % R] = policy_mu(logits, a)
        obs_h, r, dn = o.step(a, n_threads=8)
        rr_h[t % R] = r
        rd_h[t % R] = dn
    assert np.array_equal(ring_r.cpu().numpy(), rr_h)
    assert np.array_equal(ring_d.cpu().numpy(), rd_h)
    assert np.array_equal(ring_mu.cpu().numpy().view(np.uint32), mu_h.view(np.uint32))
    # the ring's oldest step is t = 2 (slot 2): steps 2..6 in order
    rng = np.random.default_rng(77)
    vals = rng.normal(0, 2, size=(R + 1, n)).astype(np.float32)
    pi = np.clip(mu_h * rng.uniform(0.5, 1.5, size=(R, n)), 0, 1).astype(np.float32)
    pi_ord = _ordered(pi, R, 2, R)
    vs, adv = g_vtrace(ring_r, ring_d, ring_mu, torch.from_numpy(vals).cuda(), torch.from_numpy(pi_ord).cuda(), R,
                       0.99, 1.0, 1.0, ring_start=2)
    r_o, d_o, m_o = (_ordered(x, R, 2, R) for x in (rr_h, rd_h, mu_h))
    vs_o, adv_o = vtrace(r_o, d_o, vals, pi_ord, m_o, 0.99, 1.0, 1.0)
    tv, ta = _vtrace_tol(r_o, d_o, vals.astype(np.float64), pi_ord, m_o, vs_o, 0.99, 1.0, 1.0)
    assert (np.abs(vs.cpu().numpy() - vs_o) <= tv).all()
    assert (np.abs(adv.cpu().numpy() - adv_o) <= ta).all()
    # the plain rollout entry point fills the same planes and rewards
    g2 = AtariEnv.from_workload(w, form=FORM_BATCHED)
    obs2 = torch.zeros_like(obs)
    ring2 = torch.zeros_like(ring)
    ring_r2 = torch.zeros_like(ring_r)
    g2.rollout(Wd, T, obs2, act, rew, done, ring2, ring_r2, ring_start=0)
    assert torch.equal(ring2, ring) and torch.equal(ring_r2, ring_r)
