"""The allocation-free step entry point, through the C ABI.

Some callers cannot allocate device memory (their framework's allocator owns
every device buffer, or they run under a fixed device-memory budget), so they
cannot create an env.  atari_step_noalloc takes their own state, start-state,
action and output buffers and keeps its scratch in a fixed array inside the
library.  This test checks it against the regular entry point (a plain-form
env with palette output) on the same states and actions, two calls in a row,
and that those calls take no device memory, for every cartridge size it
accepts (2 KB, 4 KB, F8, F6) with and without sticky actions.  It sits in a file pytest
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


ROM_2K = """
        .org $F800
Start:  LDX #$FF
        TXS
        LDA #0
        STA $80
        STA $81
Frame:  LDA #2
        STA WSYNC
        STA VSYNC
        STA WSYNC
        STA WSYNC
        STA WSYNC
        LDA #0
        STA VSYNC
        STA VBLANK
        LDA SWCHA
        AND #$80
        BNE NoR
        INC $80
NoR:    INC $82
        LDX #250
Lines:  STA WSYNC
        STX COLUBK
        TXA
        ADC $82
        STA PF1
        DEX
        BNE Lines
        JMP Frame
        .org $FFFA
        .word Start, Start, Start
"""


def _cartridge(config, which):
    """(image, score address, game-over address, seed): a workload's cartridge,
    or a 2 KB image (mirrored into both halves of the 4 KB window)."""
    if config == 0:
        return synth.Assembler().assemble(ROM_2K, org=0xF800, size=2048), 0x80, 0x81, 7
    w = synth.workload(config, n_envs=32)
    r = w.roms[which]
    return r.data, r.score_addr, r.gameover_addr, w.seed


# (workload config, cartridge, envs, sticky): 4 KB playfield and sprite
# cartridges, an 8 KB F8 and a 16 KB F6 banked cartridge with sticky actions,
# and a 2 KB image
@pytest.mark.parametrize("config,which,n,sticky", [(1, 0, 16, 0), (2, 0, 37, 0), (3, 12, 24, 1), (3, 22, 24, 1),
                                                   (0, 0, 8, 1)])
def test_noalloc_step_matches_env_step(config, which, n, sticky):
    lib = load_library()
    data, score_addr, gameover_addr, seed = _cartridge(config, which)
    assert len(data) == {0: 2048, 1: 4096, 2: 4096, 3: 8192 if which < 22 else 16384}[config]
    env = AtariEnv([data], [(score_addr, gameover_addr)], [0] * n, luma=synth.luma_table(),
                   form=FORM_PLAIN, output_mode=OUT_PALETTE, seed=seed, sticky=bool(sticky))
    states = env.state().clone()
    cache = env.cache()[0].contiguous()
    frame = torch.empty((n, 210, 160), dtype=torch.uint8, device="cuda")
    rew = torch.empty(n, dtype=torch.int32, device="cuda")
    done = torch.empty(n, dtype=torch.uint8, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rom_buf = C.create_string_buffer(data, len(data))
    meta = _Meta(score_addr, gameover_addr)
    acts = synth.actions(40 + config + which, 2, n)
    for call in range(2):
        a = torch.from_numpy(acts[call]).cuda()
        obs_ref, rew_ref, done_ref = env.step(a)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = lib.atari_step_noalloc(rom_buf, len(data), meta, _p(states), _p(cache), cache.shape[0], _p(a),
                                    _p(frame), _p(rew), _p(done), n, 4, sticky, seed, stream)
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
