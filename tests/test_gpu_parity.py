"""GPU parity: the CUDA path through the C ABI against the CPU oracle,
element by element, bit-exact (integer and byte work: tolerance 0).

Covers the start-state cache, every output of every step (observation,
reward, done, the full 256-byte canonical state, both rendered frames), the
four cartridge families (playfield, sprites/collisions, F8/F6 bank switching
with sticky actions, random-program fuzz with halting opcodes), ragged and
degenerate batch sizes, and the full 4096-env configuration on sampled envs.
"""
import numpy as np
import pytest
import torch

from oracle import OracleEnvs
from paper_1907_08467_gb300 import synth
from paper_1907_08467_gb300.env import (FORM_BATCHED, FORM_PLAIN, OUT_PALETTE, OUT_STACK, ST_BAD_ACTION,
                                        ST_LOG_OVERFLOW, AtariEnv)

pytestmark = pytest.mark.gpu

STATE_FIELDS = [(0x00, "A"), (0x01, "X"), (0x02, "Y"), (0x03, "SP"), (0x04, "P"), (0x05, "bank"), (0x06, "PC"),
                (0x08, "cycles"), (0x10, "timer_cw"), (0x18, "timer"), (0x1A, "ports"), (0x1E, "jam"),
                (0x20, "TIA"), (0x40, "positions"), (0x46, "collisions"), (0x48, "bar"), (0x50, "frame_line"),
                (0x58, "frame_no"), (0x60, "episode"), (0x64, "step"), (0x68, "env_key"), (0x6C, "status"),
                (0x70, "last_action"), (0x71, "score_prev"), (0x72, "rom"), (0x80, "RAM")]


def _field(off):
    name = "?"
    for o, n in STATE_FIELDS:
        if o <= off:
            name = n
    return name


def assert_same(tag, got, exp):
    got = np.asarray(got)
    exp = np.asarray(exp)
    if got.shape != exp.shape or not np.array_equal(got, exp):
        bad = np.argwhere(got != exp)
        first = tuple(bad[0]) if len(bad) else None
        detail = ""
        if tag == "state" and first is not None:
            env = first[0]
            offs = sorted(set(int(b[1]) for b in bad if b[0] == env))
            detail = f" env {env} bytes {[hex(o) for o in offs[:12]]} fields {sorted(set(_field(o) for o in offs))}"
        raise AssertionError(f"{tag}: {len(bad)} mismatches, first at {first}{detail}")


def pair(roms, env_rom, env_key=None, **cfg):
    luma = synth.luma_table()
    g = AtariEnv([r.data for r in roms], [(r.score_addr, r.gameover_addr) for r in roms], env_rom,
                 luma=luma, env_key=env_key, **cfg)
    ocfg = {k: v for k, v in cfg.items() if k in ("frameskip", "sticky", "n_cache", "startup_frames", "max_noops",
                                                  "output_mode", "seed")}
    o = OracleEnvs([r.data for r in roms], [r.score_addr for r in roms], [r.gameover_addr for r in roms],
                   env_rom, luma=luma, env_key=env_key, **ocfg)
    return g, o


# Launch shapes exercised for the batched form: autotuned, and fixed
# (envs per warp, envs per block, warps per frame) triples.
FORMS = {
    "plain": dict(form=FORM_PLAIN),
    "batched-auto": dict(form=FORM_BATCHED),
    "batched-32x128-w4": dict(form=FORM_BATCHED, envs_per_warp=32, envs_per_block=128, raster_warps_per_frame=4),
    "batched-8x16-w1": dict(form=FORM_BATCHED, envs_per_warp=8, envs_per_block=16, raster_warps_per_frame=1),
    "batched-1x4-w2": dict(form=FORM_BATCHED, envs_per_warp=1, envs_per_block=4, raster_warps_per_frame=2),
    # paired CPU / TIA warps
    "split-32x128-w4": dict(form=FORM_BATCHED, envs_per_warp=32, envs_per_block=128, raster_warps_per_frame=4,
                            tia_warps=2),
    "split-8x16-w2": dict(form=FORM_BATCHED, envs_per_warp=8, envs_per_block=16, raster_warps_per_frame=2,
                          tia_warps=2),
    # bank-aware grouping: the env list re-sorted by bank at every step
    "split-32x128-w4-bank": dict(form=FORM_BATCHED, envs_per_warp=32, envs_per_block=128, raster_warps_per_frame=4,
                                 tia_warps=2, grouping=2),
    "batched-8x16-w1-bank": dict(form=FORM_BATCHED, envs_per_warp=8, envs_per_block=16, raster_warps_per_frame=1,
                                 grouping=2),
    # the compact hot opcode switch (rare forms through the general decoder)
    "split-32x64-w4-compact": dict(form=FORM_BATCHED, envs_per_warp=32, envs_per_block=64, raster_warps_per_frame=4,
                                   tia_warps=2, dispatch=2),
    "batched-16x32-w2-compact": dict(form=FORM_BATCHED, envs_per_warp=16, envs_per_block=32,
                                     raster_warps_per_frame=2, tia_warps=1, dispatch=2),
}


def run_parity(g, o, actions, check_frames=False, check_state_every=1, n_threads=8):
    check_frames = check_frames and g.cfg.form == FORM_PLAIN
    n = g.n
    assert_same("state", g.state().cpu().numpy(), o.state())
    for s in range(actions.shape[0]):
        a = torch.from_numpy(actions[s]).cuda()
        obs, rew, done = g.step(a)
        oo, orw, od = o.step(actions[s], n_threads=n_threads)
        torch.cuda.synchronize()
        assert_same(f"step {s} rewards", rew.cpu().numpy(), orw)
        assert_same(f"step {s} dones", done.cpu().numpy(), od)
        assert_same(f"step {s} obs", obs.cpu().numpy(), oo)
        if check_frames:
            assert_same(f"step {s} frames", g.frames().cpu().numpy(), o.frames())
        if s % check_state_every == 0 or s == actions.shape[0] - 1:
            assert_same("state", g.state().cpu().numpy(), o.state())
    return n


def test_cache_matches_oracle():
    for w_roms in (synth.workload(2, n_envs=8).roms, synth.workload(3, n_envs=32).roms,
                   [synth.fuzz_rom(s, jam=s % 2 == 0) for s in range(4)]):
        g, o = pair(w_roms, [0], seed=7)
        assert_same("cache", g.cache().cpu().numpy(), o.cache())


@pytest.mark.parametrize("form", ["plain", "batched-auto", "batched-1x4-w2", "split-8x16-w2"])
def test_playfield_full_tiny_config(form):
    """16 envs of one 4 KB playfield cartridge, 250 steps x 4 frames, palette
    frames out: every output (and, in the plain form, both rendered frames)
    at every step."""
    w = synth.workload(1)
    g, o = pair(w.roms, w.env_rom, output_mode=OUT_PALETTE, seed=w.seed, **FORMS[form])
    acts = synth.actions(11, w.steps, w.n_envs)
    run_parity(g, o, acts, check_frames=True)


@pytest.mark.parametrize("form", list(FORMS))
def test_sprite_family_stack_output(form):
    """Eight sprite cartridges (players, missiles, ball, HMOVE, collision-driven
    score), 96 envs (ragged against every block size), full preprocessing to
    the 84x84x4 stack."""
    w = synth.workload(2, n_envs=96)
    g, o = pair(w.roms, w.env_rom, output_mode=OUT_STACK, seed=w.seed, **FORMS[form])
    if form.startswith("split"):
        assert g.launch_shape()[4] == 2      # the paired CPU / TIA warp kernel runs
    acts = synth.actions(12, 120, 96)
    run_parity(g, o, acts, check_frames=True, check_state_every=1)


@pytest.mark.parametrize("form", ["plain", "batched-auto", "batched-8x16-w1", "split-8x16-w2", "split-32x128-w4-bank",
                                  "batched-8x16-w1-bank", "split-32x64-w4-compact"])
def test_banked_sticky_family(form):
    """32 cartridges mixing 4 KB, F8 and F6 with code in every bank, RIOT-timer
    frame timing and sticky actions drawn from the per-env Philox stream."""
    w = synth.workload(3, n_envs=64)
    g, o = pair(w.roms, w.env_rom, output_mode=OUT_STACK, sticky=True, seed=w.seed, **FORMS[form])
    if form.endswith("bank"):
        assert g.launch_shape()[5] & 3 == 2      # the env list is regrouped by bank every step
    if form.endswith("compact"):
        assert g.launch_shape()[5] & 4           # the compact opcode switch runs
    acts = synth.actions(13, 80, 64)
    run_parity(g, o, acts, check_frames=True)


@pytest.mark.parametrize("form", ["plain", "batched-auto", "split-8x16-w2", "split-32x128-w4-bank"])
def test_f4_cartridges(form):
    """32 KB F4 cartridges (eight banks, hotspots $1FF4-$1FFB) with code in
    three banks and sticky actions, mixed with a 4 KB and an F6 cartridge
    (the batched form stages 32 KB per block)."""
    roms = [synth.rom_banked(s, "f4") for s in (1, 2, 3)] + [synth.rom_banked(4, "4k"), synth.rom_banked(5, "f6")]
    env_rom = [i % 5 for i in range(40)]
    g, o = pair(roms, env_rom, output_mode=OUT_STACK, sticky=True, seed=6, **FORMS[form])
    run_parity(g, o, synth.actions(71, 50, 40), check_frames=True)


@pytest.mark.parametrize("seed0,form,undoc", [(0, "plain", False), (8, "plain", False), (0, "batched-auto", False),
                                              (16, "batched-8x16-w1", False), (24, "split-32x128-w4", False),
                                              (32, "plain", True), (40, "batched-auto", True),
                                              (48, "split-8x16-w2", True), (56, "batched-8x16-w1", True),
                                              (64, "split-32x64-w4-compact", False),
                                              (72, "batched-16x32-w2-compact", True)])
def test_fuzz_programs(seed0, form, undoc):
    """Random-program cartridges (all documented opcodes, decimal mode, RMW on
    TIA strobes, TIA/RIOT reads, halting opcodes; with `undoc` also the stable
    undocumented opcodes, on RAM and on TIA strobes) stepped on both sides."""
    roms = [synth.fuzz_rom(seed0 + s, jam=s % 3 == 0, undoc=undoc) for s in range(8)]
    env_rom = [i % 8 for i in range(64)]
    g, o = pair(roms, env_rom, output_mode=OUT_STACK, seed=5, **FORMS[form])
    acts = synth.actions(14 + seed0, 60, 64)
    run_parity(g, o, acts, check_frames=True)


@pytest.mark.parametrize("n,form", [(1, "plain"), (37, "plain"), (1, "batched-auto"), (37, "batched-32x128-w4"),
                                    (37, "split-32x128-w4")])
def test_ragged_and_single(n, form):
    w = synth.workload(2, n_envs=n)
    g, o = pair(w.roms, w.env_rom, output_mode=OUT_STACK, seed=9, **FORMS[form])
    run_parity(g, o, synth.actions(16, 30, n), check_frames=True)


@pytest.mark.parametrize("form", ["plain", "batched-auto"])
def test_zero_envs(form):
    w = synth.workload(1, n_envs=1)
    g = AtariEnv([w.roms[0].data], [(0x80, 0x81)], [], luma=synth.luma_table(), **FORMS[form])
    a = torch.zeros(0, dtype=torch.uint8, device="cuda")
    g.step(a)
    assert g.state().shape == (0, 256)


def test_bad_actions_flag_status_and_act_as_noop():
    w = synth.workload(1, n_envs=4)
    g, o = pair(w.roms, w.env_rom, output_mode=OUT_PALETTE, seed=1)
    acts = np.array([[0, 18, 255, 3]] * 5, np.uint8)
    run_parity(g, o, acts)
    st = g.status().cpu().numpy()
    assert list(st & ST_BAD_ACTION) == [0, ST_BAD_ACTION, ST_BAD_ACTION, 0]


def test_log_overflow_is_reported():
    """A sprite cartridge writes several hundred TIA registers per frame; a
    256-entry log overflows and the env's status says so (the rendered frame
    is then not exact; nothing else is affected)."""
    w = synth.workload(2, n_envs=8)
    g = AtariEnv.from_workload(w, log_cap=256)
    g.step(torch.zeros(8, dtype=torch.uint8, device="cuda"))
    assert ((g.status().cpu().numpy() & ST_LOG_OVERFLOW) != 0).all()


def test_state_roundtrip_resumes_exactly():
    w = synth.workload(3, n_envs=32)
    a = AtariEnv.from_workload(w)
    b = AtariEnv.from_workload(w)
    acts = synth.actions(17, 20, 32)
    for s in range(10):
        a.step(torch.from_numpy(acts[s]).cuda())
    b.set_state(a.state())
    # the obs stack is not part of the machine state: compare rewards, dones, state
    for s in range(10, 20):
        _, ra, da = a.step(torch.from_numpy(acts[s]).cuda())
        _, rb, db = b.step(torch.from_numpy(acts[s]).cuda())
        assert torch.equal(ra, rb) and torch.equal(da, db)
    assert torch.equal(a.state(), b.state())


def test_reset_mask_matches_oracle():
    w = synth.workload(2, n_envs=16)
    g, o = pair(w.roms, w.env_rom, seed=4)
    acts = synth.actions(18, 6, 16)
    run_parity(g, o, acts[:3])
    mask = (np.arange(16) % 3 == 0).astype(np.uint8)
    g.reset(torch.from_numpy(mask).cuda())
    o.reset(mask)
    run_parity(g, o, acts[3:])


def test_host_step_matches_device_step():
    w = synth.workload(2, n_envs=64)
    a = AtariEnv.from_workload(w)
    b = AtariEnv.from_workload(w)
    acts = synth.actions(19, 8, 64)
    for s in range(8):
        oa, ra, da = a.step(torch.from_numpy(acts[s]).cuda())
        ob, rb, db = b.step_host(acts[s])
        assert np.array_equal(oa.cpu().numpy(), ob) and np.array_equal(ra.cpu().numpy(), rb)
        assert np.array_equal(da.cpu().numpy(), db)


@pytest.mark.parametrize("n,pinned", [(100, False), (4099, True), (8195, True), (8195, False)])
def test_host_step_batched_chunks_match_device_step(n, pinned):
    """The batched form's host step renders in chunks of envs and copies each
    chunk back while the next renders (8195 envs: eight ragged chunks, 4099:
    four, 100 envs: one); stacks, rewards and dones equal the device step's, pinned or
    pageable host buffers, and rewards / dones alone work too."""
    w = synth.workload(2, n_envs=n)
    a = AtariEnv.from_workload(w, form=FORM_BATCHED)
    b = AtariEnv.from_workload(w, form=FORM_BATCHED)
    acts = synth.actions(23, 6, n)
    ho = torch.empty(b.obs_shape(), dtype=torch.uint8)
    hr = torch.empty(n, dtype=torch.int32)
    hd = torch.empty(n, dtype=torch.uint8)
    if pinned:
        ho, hr, hd = ho.pin_memory(), hr.pin_memory(), hd.pin_memory()
    for s in range(6):
        oa, ra, da = a.step(torch.from_numpy(acts[s]).cuda())
        if s == 4:
            b.step_host(acts[s], None, hr, hd)  # stacks not asked for: the plain host path
            assert np.array_equal(ra.cpu().numpy(), hr.numpy()) and np.array_equal(da.cpu().numpy(), hd.numpy())
            continue
        b.step_host(acts[s], ho, hr, hd)
        assert np.array_equal(oa.cpu().numpy(), ho.numpy())
        assert np.array_equal(ra.cpu().numpy(), hr.numpy()) and np.array_equal(da.cpu().numpy(), hd.numpy())


def test_batched_equals_plain_at_full_size():
    """Both forms on the 4096-env configuration for 15 steps: identical
    observations, rewards, dones and states (the autotuned launch shape
    changes speed only)."""
    w = synth.workload(2)
    a = AtariEnv.from_workload(w, form=FORM_PLAIN)
    b = AtariEnv.from_workload(w, form=FORM_BATCHED)
    acts = synth.actions(21, 15, w.n_envs)
    for s in range(15):
        x = torch.from_numpy(acts[s]).cuda()
        oa, ra, da = a.step(x)
        ob, rb, db = b.step(x)
        assert torch.equal(oa, ob) and torch.equal(ra, rb) and torch.equal(da, db), s
    assert torch.equal(a.state(), b.state())


@pytest.mark.parametrize("form", ["plain", "batched-auto", "split-32x128-w4-bank"])
def test_state_with_extra_bank_bits_matches_oracle(form):
    """States whose bank byte has bits the cartridge does not latch (4 KB, F8
    and F6 envs) load as the cartridge's bits on both sides and step alike."""
    w = synth.workload(3, n_envs=32)
    env_rom = [0] * 4 + [12] * 4 + [22] * 4
    g, o = pair(w.roms, env_rom, sticky=True, seed=3, **FORMS[form])
    acts = synth.actions(23, 4, len(env_rom))
    run_parity(g, o, acts[:1])
    st = o.state()
    st[:, 0x05] |= np.array([0xFC, 0xFE, 0x80, 0x40] * 3, np.uint8)
    g.set_state(torch.from_numpy(st).cuda())
    o.set_state(st)
    assert_same("masked bank", o.state()[:, 0x05], st[:, 0x05] & np.array([0] * 4 + [1] * 4 + [3] * 4, np.uint8))
    # the device keeps the bytes as given until a step loads them
    obs, rew, done = g.step(torch.from_numpy(acts[1]).cuda())
    oo, orw, od = o.step(acts[1])
    torch.cuda.synchronize()
    assert_same("rewards", rew.cpu().numpy(), orw)
    assert_same("dones", done.cpu().numpy(), od)
    assert_same("obs", obs.cpu().numpy(), oo)
    run_parity(g, o, acts[2:])


def test_split_form_bounded_waits_report_stall():
    """With the TIA side switched off (tia_warps 3) every queue wait of the
    CPU warps runs out: the step still returns, every env reports ST_STALL
    (and halts), and the context stays usable for a normal env afterwards."""
    import time
    from paper_1907_08467_gb300.env import ST_STALL
    w = synth.workload(2, n_envs=8)
    g = AtariEnv.from_workload(w, form=FORM_BATCHED, envs_per_warp=8, envs_per_block=8, raster_warps_per_frame=1,
                               tia_warps=3)
    assert g.launch_shape()[4] == 2
    t0 = time.time()
    g.step(torch.zeros(8, dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    assert time.time() - t0 < 60
    st = g.status().cpu().numpy().astype(np.int64)
    assert ((st & ST_STALL) != 0).all(), st
    g.close()
    # the context is intact: a normal env still matches the oracle
    g2, o = pair(w.roms, w.env_rom, seed=w.seed, **FORMS["split-8x16-w2"])
    run_parity(g2, o, synth.actions(41, 3, 8))
