"""GPU parity of RIOT-timer wait loops (LDA INTIM / BNE back), which the
batched form retires at once when the timer counts in intervals of 8 cycles
or more: every timer rate (TIM1T runs every iteration, TIM8T, TIM64T,
T1024T), a loop whose branch crosses a page (period 8 cycles), a loop
entered after the timer passed zero (it runs until the free-running count
wraps to zero), and exit cycles made visible by position strobes and timer
reads right after each loop.  The batched and split forms must equal the
oracle (cycle counter, timer state, RAM, TIA registers, stacks) with the
skipping on and off, and the skipping must leave the TIA-write count
unchanged while executing fewer instructions in fewer issue rounds.
"""
import numpy as np
import pytest
import torch

from paper_1907_08467_gb300 import synth
from paper_1907_08467_gb300.env import FORM_BATCHED, AtariEnv
from paper_1907_08467_gb300.synth.asm6502 import assemble
from paper_1907_08467_gb300.synth.roms import Rom

from tests.test_gpu_parity import pair, run_parity

pytestmark = pytest.mark.gpu

SRC = """
Reset:  SEI
        CLD
        LDX #$FF
        TXS
Frame:  LDA #2
        STA VSYNC
        STA WSYNC
        STA WSYNC
        STA WSYNC
        LDA #0
        STA VSYNC
        LDA #20             ; TIM64T: skipped in 64-cycle steps
        STA TIM64T
W1:     LDA INTIM
        BNE W1
        STA RESP0
        LDA INTIM
        STA $80
        LDA $81             ; TIM8T from a per-frame count: the timer phase varies by env and frame
        AND #$1F
        ORA #$04
        STA TIM8T
W2:     LDA INTIM
        BNE W2
        STA RESP1
        LDA TIMINT
        STA $82
        INC $81
        LDA #2              ; T1024T
        STA T1024T
W3:     LDA INTIM
        BNE W3
        STA RESM0
        LDA #60             ; TIM1T: one-cycle intervals, never skipped
        STA TIM1T
W4:     LDA INTIM
        BNE W4
        STA RESBL
        LDA #1              ; TIM8T #1, then a delay: the loop starts after zero
        STA TIM8T
        NOP
        NOP
        NOP
        NOP
        NOP
        NOP
        NOP
W5:     LDA INTIM
        BNE W5
        STA RESM1
        LDA INTIM
        STA $83
        JMP Page
Back:   STA WSYNC
        LDA #$42
        STA COLUP0
        LDA #$FF
        STA GRP0
        STA GRP1
        STA ENAM0
        STA ENABL
        LDX #150
Lines:  STA WSYNC
        STX COLUBK
        DEX
        BNE Lines
        JMP Frame

        .org $F2F5
Page:   LDA #9              ; the loop's branch crosses from page $F2 to $F3
        STA TIM64T
        NOP
        NOP
W6:     LDA INTIM
        BNE W6
        STA RESP0
        LDA INTIM
        STA $84
        JMP Back
"""


def _rom():
    img, labels = assemble(SRC + """
        .org $FFFA
        .word Reset, Reset, Reset
""")
    assert labels["W6"] == 0xF2FC  # LDA INTIM at $F2FC, BNE at $F2FF: target page differs from $F301
    return Rom("timer-waits", bytes(img), 0x85, 0x86)


@pytest.mark.parametrize("shape", [
    dict(envs_per_warp=32, envs_per_block=64, raster_warps_per_frame=4, tia_warps=2),
    dict(envs_per_warp=8, envs_per_block=16, raster_warps_per_frame=2),
    dict(envs_per_warp=1, envs_per_block=4, raster_warps_per_frame=1),
])
@pytest.mark.parametrize("idle_skip", [1, 0])
def test_timer_wait_loops_match_oracle(shape, idle_skip):
    rom = _rom()
    n = 96
    g, o = pair([rom], [0] * n, form=FORM_BATCHED, idle_skip=idle_skip, **shape)
    run_parity(g, o, synth.actions(31, 6, n))


def test_skipping_keeps_instruction_counts_and_saves_rounds():
    """Same workload with skipping on and off: identical states, stacks,
    rewards and TIA-write counts; fewer instructions executed and fewer
    lockstep rounds with it on.  Also on a banked cartridge family whose
    frame loop waits on TIM64T."""
    banked = [r for i, r in enumerate(synth.workload(3, n_envs=256).roms) if i in (0, 12, 22)]  # 4K, F8, F6
    for roms, n in (([_rom()], 64), (banked, 256)):
        env_rom = [i * len(roms) // n for i in range(n)]
        envs = [AtariEnv([r.data for r in roms], [(r.score_addr, r.gameover_addr) for r in roms], env_rom,
                         luma=synth.luma_table(), form=FORM_BATCHED, idle_skip=s, envs_per_warp=32,
                         envs_per_block=64, raster_warps_per_frame=4, tia_warps=2) for s in (1, 0)]
        acts = synth.actions(37, 4, n)
        counts = []
        for e in envs:
            c = []
            for s in range(4):
                obs, rew, done = e.step(torch.from_numpy(acts[s]).cuda())
                c.append(e.counters())
            counts.append((c, e.state().cpu().numpy(), obs.cpu().numpy(), rew.cpu().numpy()))
        (c1, st1, ob1, rw1), (c0, st0, ob0, rw0) = counts
        assert np.array_equal(st1, st0) and np.array_equal(ob1, ob0) and np.array_equal(rw1, rw0)
        assert [x[1] for x in c1] == [x[1] for x in c0]      # TIA writes logged
        assert sum(x[0] for x in c1) < sum(x[0] for x in c0)  # instructions executed
        assert sum(x[2] for x in c1) < sum(x[2] for x in c0)  # issue rounds
