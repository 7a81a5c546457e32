"""Oracle pins for the environment layer: Philox, preprocessing, start-state
cache, rewards, dones, sticky actions and resets."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import OracleEnvs, OracleMachine, philox4x32_10, preprocess
from paper_1907_08467_gb300 import synth
from paper_1907_08467_gb300.synth.roms import FC, VALID_NIBBLES


def test_philox_known_answers():
    """Known-answer vectors published with Random123 (Salmon et al., SC'11)."""
    assert philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]) == \
        [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def _area_reference(m):
    """Exact area average of a 210x160 image over the 84x84 output grid in
    real source-pixel units (output pixel (i, j) spans rows [2.5 i, 2.5 i + 2.5)
    and columns [160 j / 84, 160 (j + 1) / 84)), rounded half up."""
    out = np.zeros((84, 84), np.uint8)
    h0, w0 = Fraction(210, 84), Fraction(160, 84)

    def overlaps(lo, hi, n):
        res = []
        for p in range(int(lo), min(n, int(hi) + 1)):
            a, b = max(lo, p), min(hi, p + 1)
            if b > a:
                res.append((p, b - a))
        return res
    for i in range(84):
        ys = overlaps(h0 * i, h0 * (i + 1), 210)
        for j in range(84):
            xs = overlaps(w0 * j, w0 * (j + 1), 160)
            s = sum(wy * wx * int(m[y, x]) for y, wy in ys for x, wx in xs)
            avg = s / (h0 * w0)
            out[i, j] = int(avg + Fraction(1, 2))
    return out


def test_preprocess_exact_area_and_max():
    rng = np.random.default_rng(7)
    luma = bytes(rng.integers(0, 256, 128, dtype=np.uint8))
    lt = np.frombuffer(luma, np.uint8)
    for trial in range(2):
        f3 = rng.integers(0, 256, (210, 160), dtype=np.uint8)
        f4 = rng.integers(0, 256, (210, 160), dtype=np.uint8)
        got = preprocess(f3, f4, luma)
        m = np.maximum(lt[f3 >> 1], lt[f4 >> 1])
        assert (got == _area_reference(m)).all()


def test_preprocess_constant_and_max_special_cases():
    luma = synth.luma_table()
    lt = np.frombuffer(luma, np.uint8)
    for v in (0, 0x0E, 0x44, 0xFE):
        f = np.full((210, 160), v, np.uint8)
        assert (preprocess(f, f, luma) == lt[v >> 1]).all()
    a = np.full((210, 160), 0x0E, np.uint8)
    b = np.zeros((210, 160), np.uint8)
    hi = max(lt[7], lt[0])
    assert (preprocess(a, b, luma) == hi).all() and (preprocess(b, a, luma) == hi).all()


def _envs(w, **kw):
    args = dict(output_mode=w.output_mode, seed=w.seed, luma=synth.luma_table(), sticky=w.sticky)
    args.update(kw)
    return OracleEnvs([r.data for r in w.roms], [r.score_addr for r in w.roms],
                      [r.gameover_addr for r in w.roms], w.env_rom, **args)


def test_cache_is_startup_plus_random_noops():
    """Section 3 reset strategy: start state k of ROM r is the machine after
    64 + n_k no-op frames from power-on, n_k = mulhi32(philox(seed, (r, k,
    3 << 8, 0)), 31)."""
    w = synth.workload(2, n_envs=8)
    e = _envs(w)
    cache = e.cache()
    key = [w.seed & 0xFFFFFFFF, w.seed >> 32]
    for r in (0, 5):
        m = OracleMachine(w.roms[r].data)
        snaps = {}
        for f in range(64 + 31):
            if f >= 64:
                snaps[f - 64] = m.state()
            m.set_action(0)
            m.run_frame()
        snaps[31] = m.state()
        for k in range(30):
            n = (philox4x32_10([r, k, 3 << 8, 0], key)[0] * 31) >> 32
            assert (cache[r, k] == snaps[n]).all(), (r, k, n)


def test_done_at_generator_gameover_frame():
    """R18: the playfield generator sets game-over once its frame counter
    reaches L; every frame adds one, so from a start state with counter c0
    the env is done exactly at step ceil((L - c0) / 4)."""
    w = synth.workload(1, n_envs=16)
    L = w.roms[0].info["gameover_frame_counter"]
    e = _envs(w)
    st = e.state()
    c0 = st[:, 0x80 + (FC & 0x7F)].astype(int) | st[:, 0x80 + (FC & 0x7F) + 1].astype(int) << 8
    first_done = np.full(16, -1)
    for s in range(1, 120):
        _, _, done = e.step(np.zeros(16, np.uint8))
        for i in np.nonzero(done)[0]:
            if first_done[i] < 0:
                first_done[i] = s
    exp = -(-(L - c0) // 4)
    assert (first_done == exp).all(), (first_done, exp)


def test_reward_closed_form_playfield():
    """R17: the playfield program adds one to its score byte in every frame
    whose joystick nibble equals its seeded condition, so a step's reward is
    4 when the action's nibble matches and 0 otherwise."""
    w = synth.workload(1, n_envs=18)
    cond = w.roms[0].info["score_nibble"]
    e = _envs(w)
    acts = np.arange(18, dtype=np.uint8)
    dirs = {0: 0xF0, 1: 0xF0, 2: 0xE0, 3: 0x70, 4: 0xB0, 5: 0xD0, 6: 0x60, 7: 0xA0, 8: 0x50, 9: 0x90}
    nib = [dirs[a] if a < 10 else dirs[[2, 3, 4, 5, 6, 7, 8, 9][a - 10]] for a in range(18)]
    assert cond in VALID_NIBBLES
    for _ in range(30):
        _, rew, _ = e.step(acts)
        assert (rew == np.array([4 if n == cond else 0 for n in nib])).all()


def test_sticky_repeat_rate():
    """R20 (sticky actions, p = 1/4 per frame): alternating a matching and a
    non-matching action each step, the expected reward of a matching step is
    4 - (1/4 + 1/16 + 1/64 + 1/256) and of the other step the complement."""
    w = synth.workload(1, n_envs=32)
    cond = w.roms[0].info["score_nibble"]
    dirs = {0xF0: 0, 0xE0: 2, 0x70: 3, 0xB0: 4, 0xD0: 5, 0x60: 6, 0xA0: 7, 0x50: 8, 0x90: 9}
    match = dirs[cond]
    other = next(a for n, a in dirs.items() if n != cond)
    e = _envs(w, sticky=True)
    rm, ro = [], []
    for s in range(300):
        a = match if s % 2 == 0 else other
        _, rew, _ = e.step(np.full(32, a, np.uint8), n_threads=8)
        (rm if a == match else ro).append(rew.astype(float))
    rm, ro = np.concatenate(rm[1:]), np.concatenate(ro)
    q = 0.25 + 0.25 ** 2 + 0.25 ** 3 + 0.25 ** 4
    se = 0.75 / np.sqrt(len(rm))
    assert abs(rm.mean() - (4 - q)) < 4 * se, rm.mean()
    assert abs(ro.mean() - q) < 4 * se, ro.mean()


def test_reset_semantics_and_stack():
    """R19/R21: after a done step the env restarts from a cached state,
    episode + 1, the frame stack is zeroed (the next observation holds only
    the newest plane) and the score baseline is the new state's score."""
    w = synth.workload(2, n_envs=64)
    e = _envs(w)
    cache = e.cache()
    prev_obs = None
    seen = 0
    acts = synth.actions(5, 200, 64)
    for s in range(200):
        obs, rew, done = e.step(acts[s], n_threads=8)
        if prev_obs is not None:
            # push order: slot 3 newest, older planes shift down
            keep = ~prev_done
            assert (obs[keep, :3] == prev_obs[keep, 1:]).all()
            if prev_done.any():
                assert not obs[prev_done, :3].any()
        st = e.state()
        for i in np.nonzero(done)[0]:
            seen += 1
            ep = int(st[i, 0x60])
            assert ep >= 1
            rom = int(st[i, 0x72])
            assert any((st[i, :0x60] == cache[rom, k, :0x60]).all() and
                       (st[i, 0x80:] == cache[rom, k, 0x80:]).all() for k in range(30))
            sa = w.roms[rom].score_addr
            assert st[i, 0x71] == st[i, 0x80 + (sa & 0x7F)]
        prev_obs, prev_done = obs, done.astype(bool)
    assert seen > 10


def test_deterministic_rerun_and_state_roundtrip():
    w = synth.workload(3, n_envs=32)
    a = _envs(w)
    b = _envs(w)
    acts = synth.actions(3, 12, 32)
    for s in range(12):
        oa = a.step(acts[s], n_threads=4)
        ob = b.step(acts[s], n_threads=1)
        assert all((x == y).all() for x, y in zip(oa, ob))
    assert (a.state() == b.state()).all()


def test_subset_env_keys_match_full_batch():
    """Envs are independent: a subset run with the same env keys reproduces
    the full batch's outputs for those envs (used for sampled parity)."""
    w = synth.workload(2, n_envs=64)
    full = _envs(w)
    idx = np.array([3, 17, 40, 63])
    sub = OracleEnvs([r.data for r in w.roms], [r.score_addr for r in w.roms],
                     [r.gameover_addr for r in w.roms], [w.env_rom[i] for i in idx],
                     output_mode=1, seed=w.seed, luma=synth.luma_table(), env_key=idx)
    acts = synth.actions(9, 30, 64)
    for s in range(30):
        of = full.step(acts[s], n_threads=8)
        os_ = sub.step(acts[s][idx])
        for x, y in zip(of, os_):
            assert (x[idx] == y).all()
    assert (full.state()[idx] == sub.state()).all()


def test_reset_mask_api():
    w = synth.workload(1, n_envs=4)
    e = _envs(w)
    e.reset(np.array([1, 0, 1, 0], np.uint8))
    st = e.state()
    assert list(st[:, 0x60]) == [1, 0, 1, 0]


def test_bad_rom_size_rejected():
    w = synth.workload(1, n_envs=2)
    with pytest.raises(ValueError):
        OracleEnvs([w.roms[0].data[:3000]], [0x80], [0x81], [0, 0])
