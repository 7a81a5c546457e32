"""Oracle pins for the learner-side targets over a rollout (paper Appendix,
"A2C": the bootstrapped N-step return; "V-trace": the off-policy target with
truncated importance weights, its recursive form and the actor's advantage).

The oracle writes each target as its sum definition.  These tests pin it to
what the definitions fix independently of that code:

- closed forms (a geometric series) and a hand-worked two-step example;
- the paper's second, recursive formulation of the V-trace target, evaluated
  here step by step from the end of the rollout;
- the reduction of V-trace to the N-step return when the behaviour and
  target policies agree and the truncation levels are 1 (the on-policy case
  of the V-trace construction), which ties two separately written sums;
- zero importance weights (the target is the value itself);
- episode ends inside the rollout: nothing after a done changes the earlier
  targets.

Planted one-line mistakes in the oracle (the weight of step u included in its
own product, rho in place of c in the product, dones ignored, the bootstrap
kept after a done, V(s_{t+1}) in place of v_{t+1} in the advantage, one
power of gamma too many on the bootstrap) each fail at least one test here.
"""
import numpy as np
import pytest

from oracle import nstep_returns, policy_mu, policy_prob, vtrace


def _rollout(seed, T=6, n=40, p_done=0.15):
    rng = np.random.default_rng(seed)
    r = rng.integers(-3, 8, size=(T, n)).astype(np.float32)
    d = (rng.random((T, n)) < p_done).astype(np.uint8)
    v = rng.normal(0, 2, size=(T + 1, n)).astype(np.float32)
    mu = rng.uniform(0.05, 1.0, size=(T, n)).astype(np.float32)
    pi = np.clip(mu * rng.uniform(0.0, 3.0, size=(T, n)), 0, 1).astype(np.float32)
    return r, d, v, pi, mu


def test_nstep_geometric_closed_form():
    """Constant reward 1, no episode end, bootstrap value b: R_t =
    (1 - g^k) / (1 - g) + g^k b with k = T - t."""
    T, n, g, b = 7, 3, 0.9, 2.0
    r = np.ones((T, n), np.float32)
    d = np.zeros((T, n), np.uint8)
    v = np.zeros((T + 1, n), np.float32)
    v[T] = b
    R = nstep_returns(r, d, v, g)
    for t in range(T):
        k = T - t
        assert np.allclose(R[t], (1 - g ** k) / (1 - g) + g ** k * b, rtol=1e-13, atol=0)


def test_nstep_hand_example_with_episode_end():
    """g = 0.5, r = 1, 2, 3, 4, done after step 1, bootstrap 8:
    R0 = 1 + 0.5 * 2 = 2 (ends at step 1), R1 = 2, R2 = 3 + 0.5 * 4 + 0.25 * 8
    = 7, R3 = 4 + 0.5 * 8 = 8.  Later rewards and the bootstrap do not reach
    R0 and R1."""
    r = np.array([[1], [2], [3], [4]], np.float32)
    d = np.array([[0], [1], [0], [0]], np.uint8)
    v = np.array([[5], [6], [7], [9], [8]], np.float32)
    assert nstep_returns(r, d, v, 0.5)[:, 0].tolist() == [2.0, 2.0, 7.0, 8.0]
    r2, v2 = r.copy(), v.copy()
    r2[2:] = 100
    v2[4] = -50
    assert nstep_returns(r2, d, v2, 0.5)[:2, 0].tolist() == [2.0, 2.0]


def test_vtrace_hand_example():
    """Two steps, g = 0.5, rho_bar = 2, c_bar = 1, V = 1, 2, bootstrap 4,
    r = 1, 1, pi/mu = 0.5/0.25 = 2 then 0.2/0.4 = 0.5 (exact in fp32):
    rho0 = 2, c0 = 1, rho1 = c1 = 0.5.
    delta0 = 2 (1 + 0.5*2 - 1) = 2;  delta1 = 0.5 (1 + 0.5*4 - 2) = 0.5.
    v1 = 2 + 0.5 = 2.5;  v0 = 1 + 2 + 0.5*1*0.5 = 3.25.
    A0 = 2 (1 + 0.5*2.5 - 1) = 2.5;  A1 = 0.5 (1 + 0.5*4 - 2) = 0.5."""
    r = np.array([[1], [1]], np.float32)
    d = np.zeros((2, 1), np.uint8)
    v = np.array([[1], [2], [4]], np.float32)
    pi = np.array([[0.5], [0.2]], np.float32)
    mu = np.array([[0.25], [0.4]], np.float32)
    vs, adv = vtrace(r, d, v, pi, mu, 0.5, 2.0, 1.0)
    assert vs[:, 0].tolist() == [3.25, 2.5]
    assert adv[:, 0].tolist() == [2.5, 0.5]


@pytest.mark.parametrize("seed,rho_bar,c_bar", [(1, 1.0, 1.0), (2, 1.0, 0.9), (3, 2.0, 0.5), (4, 1e9, 1e9)])
def test_vtrace_equals_the_papers_recursive_form(seed, rho_bar, c_bar):
    """v_t = V(s_t) + delta_t + gamma_t c_t (v_{t+1} - V(s_{t+1})), v_T =
    V(s_T), evaluated here backwards in double precision, equals the sum
    definition; the advantage follows from the same v."""
    g = 0.97
    r, d, v, pi, mu = _rollout(seed)
    vs, adv = vtrace(r, d, v, pi, mu, g, rho_bar, c_bar)
    T, n = r.shape
    R = r.astype(np.float64)
    V = v.astype(np.float64)
    ratio = pi.astype(np.float64) / mu.astype(np.float64)
    rho = np.minimum(rho_bar, ratio)
    c = np.minimum(c_bar, ratio)
    gt = np.where(d != 0, 0.0, g)
    rec = np.zeros((T + 1, n))
    rec[T] = V[T]
    for t in range(T - 1, -1, -1):
        delta = rho[t] * (R[t] + gt[t] * V[t + 1] - V[t])
        rec[t] = V[t] + delta + gt[t] * c[t] * (rec[t + 1] - V[t + 1])
    assert np.allclose(vs, rec[:T], rtol=1e-12, atol=1e-12)
    a = rho * (R + gt * rec[1:] - V[:T])
    assert np.allclose(adv, a, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_vtrace_on_policy_is_the_nstep_return(seed):
    """pi = mu with rho_bar = c_bar = 1 makes every weight 1: the V-trace
    target is the bootstrapped N-step return and the advantage is R_t - V(s_t)."""
    g = 0.9
    r, d, v, _, mu = _rollout(seed)
    vs, adv = vtrace(r, d, v, mu, mu, g, 1.0, 1.0)
    R = nstep_returns(r, d, v, g)
    assert np.allclose(vs, R, rtol=1e-12, atol=1e-12)
    assert np.allclose(adv, R - v[:-1].astype(np.float64), rtol=1e-12, atol=1e-12)


def test_vtrace_zero_target_probability_gives_the_value():
    r, d, v, _, mu = _rollout(8)
    vs, adv = vtrace(r, d, v, np.zeros_like(mu), mu, 0.99, 1.0, 1.0)
    assert np.array_equal(vs, v[:-1].astype(np.float64))
    assert not adv.any()


def test_vtrace_episode_end_cuts_the_target():
    """Rewards, values and weights after the first done of a column do not
    change that column's targets up to the done."""
    r, d, v, pi, mu = _rollout(9, T=8, n=1, p_done=0.0)
    d[3, 0] = 1
    vs, adv = vtrace(r, d, v, pi, mu, 0.95, 1.0, 1.0)
    r2, v2, pi2 = r.copy(), v.copy(), pi.copy()
    r2[4:] += 7
    v2[5:] -= 3          # V(s_4) is the value after the done: it enters nothing up to step 3
    pi2[4:] = 0.01
    vs2, adv2 = vtrace(r2, d, v2, pi2, mu, 0.95, 1.0, 1.0)
    assert np.array_equal(vs[:4], vs2[:4]) and np.array_equal(adv[:4], adv2[:4])


def test_behaviour_probability_is_the_softmax_weight():
    """mu(a|s) = exp(l_a - max) / sum_j exp(l_j - max): equal logits give
    1/18 for every action, a logit 40 above the rest gives its action
    probability 1 (the others underflow below fp32's ulp of 1), and the
    values sum to 1 within fp32 rounding."""
    eq = np.zeros(18, np.float32)
    assert all(abs(policy_prob(eq, a) - 1 / 18) < 1e-7 for a in range(18))
    dom = np.zeros(18, np.float32)
    dom[5] = 40.0
    assert policy_prob(dom, 5) == 1.0
    rng = np.random.default_rng(3)
    l = rng.normal(0, 3, size=(50, 18)).astype(np.float32)
    tot = np.zeros(50)
    for a in range(18):
        tot += policy_mu(l, np.full(50, a, np.uint8))
    assert np.allclose(tot, 1.0, atol=1e-5)
    ref = np.exp(l - l.max(1, keepdims=True))
    ref /= ref.sum(1, keepdims=True)
    got = np.stack([policy_mu(l, np.full(50, a, np.uint8)) for a in range(18)], 1)
    assert np.allclose(got, ref, rtol=2e-6, atol=1e-9)
