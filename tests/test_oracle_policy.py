"""Oracle pins for the inference-path policy: exp, the fp32 logits in their
canonical order, and the inverse-CDF sampling."""
import math

import numpy as np
import pytest

from oracle import OracleEnvs, exp_own, philox4x32_10, policy_logits, policy_sample
from paper_1907_08467_gb300 import synth

K, A = 28224, 18


def ulp32(v: float) -> float:
    if v == 0.0:
        return 2.0 ** -149
    e = math.frexp(abs(v))[1]
    return 2.0 ** max(e - 24, -149)


def test_exp_own_within_two_ulp():
    """Cody-Waite + degree-7 polynomial against the double-precision exp
    (itself within a double ulp), over [-87, 1] on a dense grid and random
    points; exact at 0."""
    assert exp_own(0.0) == 1.0
    xs = np.concatenate([np.arange(-87.0, 1.0, 0.0013), np.random.default_rng(1).uniform(-87, 1, 20000)])
    worst = 0.0
    for x in xs:
        xf = float(np.float32(x))
        ref = math.exp(xf)
        got = exp_own(xf)
        worst = max(worst, abs(got - ref) / ulp32(ref))
    assert worst <= 2.0, worst
    assert exp_own(-88.0) == 0.0 and exp_own(-200.0) == 0.0


def _bf16_to_f32(b):
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


def test_logits_within_fp32_bound_of_exact_dot_product():
    """|fp32 logits - exact| <= 73 u sum|x w| (64 sequential fmaf per chunk
    plus 9 levels of the pairwise tree; u = 2^-24): a dropped term, a wrong
    index or a transposed weight matrix breaks the bound by orders of
    magnitude."""
    rng = np.random.default_rng(2)
    w = synth.policy_weights(3)
    wf = _bf16_to_f32(w).astype(np.float64).reshape(K, A)
    for trial in range(3):
        x = rng.integers(0, 256, K, dtype=np.uint8)
        got = policy_logits(x, w).astype(np.float64)
        exact = x.astype(np.float64) @ wf
        bound = 73 * 2.0 ** -24 * (np.abs(x.astype(np.float64))[:, None] * np.abs(wf)).sum(0)
        assert (np.abs(got - exact) <= bound + 1e-30).all(), np.max(np.abs(got - exact) / bound)
        # and it is not trivially exact: the bound is tight enough to matter
        assert np.abs(got - exact).max() < 1e-3


def test_single_row_is_exact_and_pins_the_flattening():
    """With only row k of W nonzero, logit j is exactly stack[k] * W[k][j]
    for the stack flattened as plane * 7056 + row * 84 + column."""
    rng = np.random.default_rng(3)
    stack = rng.integers(1, 256, (4, 84, 84), dtype=np.uint8)
    for (c, h, wcol) in [(0, 0, 0), (1, 17, 40), (3, 83, 83), (2, 50, 3)]:
        k = c * 7056 + h * 84 + wcol
        w = np.zeros((K, A), np.uint16)
        w[k] = synth.policy_weights(4)[k]
        got = policy_logits(stack, w.reshape(-1))
        exact = np.float32(stack[c, h, wcol]) * _bf16_to_f32(w[k])
        assert np.array_equal(got, exact.astype(np.float32))


def test_sampling_special_cases():
    l = np.zeros(A, np.float32)
    # equal logits: action = the bin of u = (x >> 8) 2^-24 in 18 equal parts
    for x in [0, 1 << 20, (1 << 32) - 1, 0x80000000, 0x38E38E00]:
        j = policy_sample(l, x)
        assert j == min(17, int((x >> 8) / 2 ** 24 * 18)), (x, j)
    # one dominant logit wins whatever the draw
    l2 = np.full(A, -50.0, np.float32)
    l2[7] = 50.0
    assert all(policy_sample(l2, u) == 7 for u in [0, 12345, (1 << 32) - 1])


def test_sampling_matches_softmax_distribution():
    rng = np.random.default_rng(5)
    logits = rng.normal(0, 1.5, A).astype(np.float32)
    p = np.exp(logits - logits.max())
    p /= p.sum()
    n = 60000
    us = rng.integers(0, 1 << 32, n, dtype=np.uint64)
    counts = np.bincount([policy_sample(logits, int(u)) for u in us], minlength=A)
    chi2 = ((counts - n * p) ** 2 / (n * p)).sum()
    assert chi2 < 45.0, chi2     # 17 dof: p ~ 3e-4 at 45


def test_env_policy_uses_the_env_stream():
    """orc_envs_policy = sample(logits(obs_i), philox(seed; env_key, step, 4 << 8, episode))."""
    w_ = synth.workload(2, n_envs=12)
    e = OracleEnvs([r.data for r in w_.roms], [r.score_addr for r in w_.roms], [r.gameover_addr for r in w_.roms],
                   w_.env_rom, luma=synth.luma_table(), seed=w_.seed)
    W = synth.policy_weights(5)
    obs = np.zeros((12, 4, 84, 84), np.uint8)
    for s in range(3):
        act, logits = e.policy(obs, W, n_threads=4)
        st = e.state()
        for i in range(12):
            ep, step, key = (int(st[i, 0x60:0x64].view(np.uint32)[0]), int(st[i, 0x64:0x68].view(np.uint32)[0]),
                             int(st[i, 0x68:0x6C].view(np.uint32)[0]))
            u = philox4x32_10([key, step, 4 << 8, ep], [w_.seed, 0])[0]
            assert np.array_equal(logits[i], policy_logits(obs[i], W))
            assert act[i] == policy_sample(logits[i], u)
        obs, _, _ = e.step(act)
