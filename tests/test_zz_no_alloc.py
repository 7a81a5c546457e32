"""The allocation-free step entry point, through the C ABI.

Some callers cannot allocate device memory (their framework's allocator owns
every device buffer, or they run under a fixed device-memory budget), so they
cannot create an env.  atari_step_noalloc takes their own state, start-state,
action and output buffers and keeps its scratch in a fixed array inside the
library.  This test checks it against the regular entry point (a plain-form
env with palette output) on the same states and actions, two calls in a row,
and that those calls take no device memory.  It sits in a file pytest
collects last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1907_08467_gb300 import synth
from paper_1907_08467_gb300.env import FORM_PLAIN, OUT_PALETTE, AtariEnv, _Meta, load_library

pytestmark = pytest.mark.gpu


def _p(t):
    return C.c_void_p(t.data_ptr())


@pytest.mark.parametrize("config,n", [(1, 16), (2, 37)])
def test_noalloc_step_matches_env_step(config, n):
    lib = load_library()
    w = synth.workload(config, n_envs=n)
    rom = w.roms[0]
    env = AtariEnv([rom.data], [(rom.score_addr, rom.gameover_addr)], [0] * n, luma=synth.luma_table(),
                   form=FORM_PLAIN, output_mode=OUT_PALETTE, seed=w.seed)
    states = env.state().clone()
    cache = env.cache()[0].contiguous()
    frame = torch.empty((n, 210, 160), dtype=torch.uint8, device="cuda")
    rew = torch.empty(n, dtype=torch.int32, device="cuda")
    done = torch.empty(n, dtype=torch.uint8, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rom_buf = C.create_string_buffer(rom.data, len(rom.data))
    meta = _Meta(rom.score_addr, rom.gameover_addr)
    acts = synth.actions(40 + config, 2, n)
    for call in range(2):
        a = torch.from_numpy(acts[call]).cuda()
        obs_ref, rew_ref, done_ref = env.step(a)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = lib.atari_step_noalloc(rom_buf, len(rom.data), meta, _p(states), _p(cache), cache.shape[0], _p(a),
                                    _p(frame), _p(rew), _p(done), n, 4, 0, w.seed, stream)
        assert rc == 0, lib.atari_last_error()
        torch.cuda.synchronize()
        if call == 1:   # the first call may load the library's device module, which holds the array
            assert torch.cuda.mem_get_info()[0] == free_before
        assert torch.equal(frame, obs_ref), call
        assert torch.equal(rew, rew_ref), call
        assert torch.equal(done, done_ref), call
        ref_state = env.state()
        ref_state[:, 0x72:0x74] = 0          # the variant writes ROM index 0 (single cartridge)
        assert torch.equal(states, ref_state), call


def test_noalloc_rejects_too_many_envs():
    lib = load_library()
    rom = synth.rom_playfield(1)
    rom_buf = C.create_string_buffer(rom.data, len(rom.data))
    rc = lib.atari_step_noalloc(rom_buf, len(rom.data), _Meta(0x80, 0x81), None, None, 30, None, None, None,
                                None, 65, 4, 0, 1, None)
    assert rc == -22
    assert b"at most" in lib.atari_last_error()
