"""Oracle pins for the TIA registers whose effect is a copy or a clear
(vertical delay, missile-to-player reset, CXCLR, HMCLR) and for the BRK / RTI
pair, each by real register writes in hand-assembled programs.

Every expected value below is worked out by hand from the machine definition
and the readings of the oracle's header (not by calling the oracle):

- VDELP0 / VDELP1 / VDELBL select the "old" copy of GRP0 / GRP1 / ENABL.  A
  GRP0 write copies GRP1's new value into GRP1's old one; a GRP1 write copies
  GRP0 new -> old and ENABL new -> old.
- RESMPx: while D1 is set the missile is hidden; on D1 going 1 -> 0 it is
  placed at the player's position + 4 x the player's scale (1, 2, 4).
- CXCLR clears all fifteen collision latches; HMCLR zeroes the five motion
  registers.
- BRK pushes PC + 2 (high byte first), then P with B and bit 5 set, sets I and
  jumps through the vector at $1FFE; RTI pulls P (B dropped, bit 5 set) and
  then the return address, which it uses as is.

Each test names the one-line oracle mistakes it catches; every one of them was
planted in the oracle and seen to fail the test.
"""
import numpy as np
import pytest

from oracle import OracleMachine
from paper_1907_08467_gb300.synth.asm6502 import Assembler
from tests.helpers import JAM, rom, run_to_jam

# Frame loop with VBLANK off on every line; per-line code runs after each
# WSYNC with X counting the lines down from 250 (line X = 250 first).
FRAME = """
Frame:  LDA #2
        STA WSYNC
        STA VSYNC
        STA WSYNC
        STA WSYNC
        STA WSYNC
        LDA #0
        STA VSYNC
        STA VBLANK
        LDX #250
Lines:  STA WSYNC
{PERLINE}
        DEX
        BNE Lines
        JMP Frame
"""

BG, C0, C1, CF = 0x02, 0x1E, 0x3E, 0x5E     # COLUBK, COLUP0, COLUP1, COLUPF (even: stored as is)
INIT_COLORS = f"""
        LDA #${BG:02X}
        STA COLUBK
        LDA #${C0:02X}
        STA COLUP0
        LDA #${C1:02X}
        STA COLUP1
        LDA #${CF:02X}
        STA COLUPF
        LDA #0
        STA CTRLPF
"""


def frame_rom(init: str, perline: str) -> bytes:
    return rom("Start:\n" + INIT_COLORS + init + FRAME.replace("{PERLINE}", perline))


def at_line(x: int, body: str, label: str) -> str:
    """Per-line code that runs `body` only on the line where X == x."""
    return f"        CPX #{x}\n        BNE {label}\n{body}{label}:\n"


def set_pos(m, **pos):
    off = {"p0": 0x40, "p1": 0x41, "m0": 0x42, "m1": 0x43, "bl": 0x44}
    st = m.state()
    for k, v in pos.items():
        st[off[k]] = v
    m.set_state(st)


def line(p0=0, p1=0, ball=False, missile=None):
    """One window row: background, P0 pattern at 20..27, P1 at 60..67, the
    ball (1 pixel, COLUPF) at 100, a missile pixel (COLUP0) at `missile`."""
    r = np.full(160, BG, np.uint8)
    if ball:
        r[100] = CF
    if missile is not None:
        r[missile] = C0
    for i in range(8):
        if (p1 >> (7 - i)) & 1:
            r[60 + i] = C1
    for i in range(8):
        if (p0 >> (7 - i)) & 1:
            r[20 + i] = C0
    return r


def runs(fb):
    """Distinct consecutive row contents of a frame: [(first row, row), ...]."""
    out = []
    for r in range(fb.shape[0]):
        if not out or not np.array_equal(fb[r], out[-1][1]):
            out.append((r, fb[r].copy()))
    return out


VDEL_LINES = (at_line(200, "        LDA #2\n        STA ENABL\n", "A1") +
              at_line(180, "        LDA #$F0\n        STA GRP0\n", "A2") +
              at_line(150, "        LDA #$0F\n        STA GRP1\n", "A3") +
              at_line(120, "        LDA #$AA\n        STA GRP0\n", "A4") +
              at_line(2, "        LDA #0\n        STA ENABL\n        STA GRP0\n        STA GRP1\n"
                         "        STA GRP0\n", "A5"))


@pytest.mark.parametrize("vdel", [0, 1])
def test_vertical_delay_old_registers(vdel):
    """Writes in one frame: ENABL = 2 (line X=200), GRP0 = $F0 (X=180),
    GRP1 = $0F (X=150), GRP0 = $AA (X=120); all six registers are zero
    before.  Worked by hand:

      after write      GRP0 new/old   GRP1 new/old   ENABL new/old
      ENABL = 2          00 / 00        00 / 00         2 / 0
      GRP0 = F0          F0 / 00        00 / 00         2 / 0   (GRP1 old <- 00)
      GRP1 = 0F          F0 / F0        0F / 00         2 / 2   (GRP0 old <- F0, ENABL old <- 2)
      GRP0 = AA          AA / F0        0F / 0F         2 / 2   (GRP1 old <- 0F)

    Without delay the rows show the new values: ball from X=200, P0 $F0 from
    X=180, P1 $0F from X=150, P0 $AA from X=120.  With VDELP0/VDELP1/VDELBL
    set they show the old ones: nothing until X=150, then P0 $F0 and the
    ball, then from X=120 P1 $0F too.

    Catches: a GRP0 write copying GRP0 (not GRP1) new -> old; the GRP1 write
    copying GRP1 (not GRP0); the ENABL copy on a GRP0 write; a delay bit
    selecting the new register."""
    init = f"        LDA #{vdel}\n        STA VDELP0\n        STA VDELP1\n        STA VDELBL\n"
    m = OracleMachine(frame_rom(init, VDEL_LINES))
    m.run_frame()
    set_pos(m, p0=20, p1=60, bl=100)
    m.run_frame()
    fb = m.run_frame(render=True)[1]
    got = runs(fb)
    if vdel:
        exp = [line(), line(p0=0xF0, ball=True), line(p0=0xF0, p1=0x0F, ball=True)]
        gaps = [30]                                   # X = 150 -> 120
    else:
        exp = [line(), line(ball=True), line(p0=0xF0, ball=True), line(p0=0xF0, p1=0x0F, ball=True),
               line(p0=0xAA, p1=0x0F, ball=True)]
        gaps = [20, 30, 30]                           # X = 200 -> 180 -> 150 -> 120
    assert len(got) == len(exp), [r for r, _ in got]
    for (r, row), e in zip(got, exp):
        assert np.array_equal(row, e), (r, np.nonzero(row != e)[0])
    assert got[0][0] == 0
    assert [b[0] - a[0] for a, b in zip(got[1:], got[2:])] == gaps
    # the frame ended with the registers cleared: old and new copies all zero
    st = m.state()
    assert list(st[0x30:0x36]) == [0] * 6 and list(st[0x36:0x39]) == [vdel] * 3


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("nusiz,scale", [(0, 1), (5, 2), (7, 4)])
def test_resmp_hides_and_places_missile(nusiz, scale, which):
    """ENAM0 = 2 and RESMP0 = 2 from the start; the missile sits at column 100
    and P0 (no graphics) at 40.  On line X=150 RESMP0 is written 0: the
    missile is placed at 40 + 4 x scale (player scale 1, 2, 4 for NUSIZ0 0,
    5, 7; the missile stays 1 pixel wide).  Rows before show only the
    background (the missile is hidden, not drawn at 100); rows after show
    one missile pixel.

    Catches: the missile drawn while RESMP D1 is set; a fixed offset of 4
    (no scale); the placement taken on the 0 -> 1 edge instead of 1 -> 0.
    The same for player 1 / missile 1 (COLUP1), which catches a swapped
    player or missile index."""
    w = which
    init = (f"        LDA #2\n        STA ENAM{w}\n        STA RESMP{w}\n        LDA #{nusiz}\n"
            f"        STA NUSIZ{w}\n")
    lines = (at_line(150, f"        LDA #0\n        STA RESMP{w}\n", "B1") +
             at_line(2, f"        LDA #2\n        STA RESMP{w}\n", "B2"))
    m = OracleMachine(frame_rom(init, lines))
    m.run_frame()
    set_pos(m, **{f"p{w}": 40, f"p{1 - w}": 10, f"m{w}": 100})
    fb = m.run_frame(render=True)[1]
    got = runs(fb)
    assert len(got) == 2, [r for r, _ in got]
    assert np.array_equal(got[0][1], line())
    exp = line()
    exp[40 + 4 * scale] = C1 if w else C0
    assert np.array_equal(got[1][1], exp), np.nonzero(got[1][1] != exp)[0]
    assert m.state()[0x42 + w] == 40 + 4 * scale and m.state()[0x39 + w] & 2


def test_cxclr_clears_every_latch():
    """P0 (40..47) and P1 (44..51) overlap, and M0 (50) lies inside P1, on
    every line until X=150, where GRP0, GRP1 and ENAM0 are cleared.  On line
    X=120 the program reads CXPPMM (P0-P1 is D7: $80) and CXM0P (M0-P1 is D7,
    M0-P0 D6: $80) into RAM $80/$81; on X=100 it strobes CXCLR; on X=90 it
    reads both again ($00, $00) into $82/$83.  Line X=2 restores the
    objects, so at the end of the frame exactly the two pairs of lines X=2
    and X=1 are latched again (P0-P1 and M0-P1, nothing else).

    Catches: CXCLR ignored, or clearing only the low or the high byte of the
    latch word."""
    init = "        LDA #$FF\n        STA GRP0\n        STA GRP1\n        LDA #2\n        STA ENAM0\n"
    lines = (at_line(150, "        LDA #0\n        STA GRP0\n        STA GRP1\n        STA ENAM0\n", "C1") +
             at_line(120, "        LDA CXPPMM\n        STA $80\n        LDA CXM0P\n        STA $81\n", "C2") +
             at_line(100, "        STA CXCLR\n", "C3") +
             at_line(90, "        LDA CXPPMM\n        STA $82\n        LDA CXM0P\n        STA $83\n", "C4") +
             at_line(2, "        LDA #$FF\n        STA GRP0\n        STA GRP1\n        LDA #2\n        STA ENAM0\n",
                     "C5"))
    m = OracleMachine(frame_rom(init, lines))
    m.run_frame()
    set_pos(m, p0=40, p1=44, m0=50)
    st = m.state()
    st[0x46] = st[0x47] = 0
    m.set_state(st)
    m.run_frame()
    ram = m.ram()
    assert ram[0] == 0x80 and ram[1] == 0x80
    assert ram[2] == 0x00 and ram[3] == 0x00
    cx = int(m.state()[0x46]) | int(m.state()[0x47]) << 8
    assert cx == (1 << 15) | (1 << 1)


def test_hmclr_zeroes_all_motion_registers():
    """HMP0, HMP1, HMM0, HMM1 and HMBL are written $30 (3 pixels left), then
    HMCLR is strobed, then HMOVE: no object moves and the five registers read
    zero in the state.  Without the HMCLR the same program moves every object
    3 pixels left.

    Catches: HMCLR ignored, or leaving any one of the five registers set."""
    for clear in (True, False):
        src = ("Start:  LDA #$30\n        STA HMP0\n        STA HMP1\n        STA HMM0\n        STA HMM1\n"
               "        STA HMBL\n" + ("        STA HMCLR\n" if clear else "") +
               "        STA WSYNC\n        STA HMOVE\n" + JAM)
        m = OracleMachine(rom(src))
        m.step()
        set_pos(m, p0=50, p1=60, m0=70, m1=80, bl=90)
        run_to_jam(m)
        st = m.state()
        want = [50, 60, 70, 80, 90] if clear else [47, 57, 67, 77, 87]
        assert list(st[0x40:0x45]) == want
        assert list(st[0x3B:0x40]) == ([0] * 5 if clear else [0x30] * 5)


BRK_PROGRAM = """
        .org $F000
Start:  LDX #$FF
        TXS
        SEC
        CLI
Brk:    BRK
        .byte $EA
After:  STX $86
        .byte $02
Handler:
        TSX
        STX $80
        PHP
        PLA
        STA $81
        LDA $01FD
        STA $82
        LDA $01FE
        STA $84
        LDA $01FF
        STA $85
        RTI
        .org $FFFA
        .word Start, Start, Handler
"""


def test_brk_rti_stack_flags_and_vector():
    """BRK at $F005 with P = N | bit 5 | C ($A1; LDX #$FF set N, CLI cleared
    the power-on I).  By hand: BRK pushes $F0 (PCH of $F007) to $01FF, $07 to
    $01FE, then P | B | bit 5 = $B1 to $01FD; SP ends at $FC; I is set and
    the handler (vector at $FFFE, not the reset vector at $FFFC) runs with
    P = $A5, so its PHP pushes $B5.  RTI restores P = $A1 (B dropped) and
    returns to $F007 itself (no +1 as RTS has), where STX $86 stores the
    handler's X ($FC, from its TSX) without touching the flags.  The stack page mirrors RAM, so $01FD..$01FF are RAM $7D..$7F.

    Catches: the return bytes pushed low first; B or bit 5 missing from the
    pushed P; I not set; the reset vector used; RTI keeping B; RTI adding 1
    to the return address."""
    m = OracleMachine(Assembler().assemble(BRK_PROGRAM, org=0xF000, size=4096))
    run_to_jam(m)
    ram = m.ram()
    assert ram[0] == 0xFC                       # SP inside the handler
    assert ram[1] == 0xB5                       # handler's P (I set) as pushed by PHP
    assert ram[2] == 0xB1                       # P pushed by BRK
    assert ram[4] == 0x07 and ram[5] == 0xF0    # return address $F007, high byte pushed first
    assert list(ram[0x7D:0x80]) == [0xB1, 0x07, 0xF0]
    assert ram[6] == 0xFC                       # RTI returned to $F007 itself
    st = m.state()
    assert st[0x04] == 0xA1                     # P after RTI: B clear, bit 5 set, I clear again
    assert st[0x03] == 0xFF                     # stack balanced


def test_undriven_reads_and_ignored_writes():
    """R9: INPT0..INPT3 read $00, INPT5 $80, INPT4 $80 with fire released;
    TIA read addresses decode A3..A0 only ($3C reads INPT4, $3D INPT5); the
    unused read registers $0E/$0F read $00.  Writes to the audio registers,
    RSYNC and the unused addresses $2D..$3F change no state byte.

    Catches: a paddle input reading $80, INPT5 reading $00, a read decoded on
    more than four address bits, an audio write landing in the TIA file."""
    src = """
Start:  LDA INPT0
        STA $80
        LDA INPT1
        STA $81
        LDA INPT2
        STA $82
        LDA INPT3
        STA $83
        LDA INPT4
        STA $84
        LDA INPT5
        STA $85
        LDA $3C
        STA $86
        LDA $3D
        STA $87
        LDA $0E
        STA $88
        LDA $0F
        STA $89
""" + JAM
    m = OracleMachine(rom(src))
    run_to_jam(m)
    assert list(m.ram()[:10]) == [0, 0, 0, 0, 0x80, 0x80, 0x80, 0x80, 0, 0]
    writes = "".join(f"        STA ${a:02X}\n" for a in [0x03, 0x15, 0x16, 0x17, 0x18, 0x19, 0x1A] + list(range(0x2D, 0x40)))
    m = OracleMachine(rom("Start:  LDA #$FF\n" + writes + JAM))
    m.step()
    before = m.state()
    run_to_jam(m)
    after = m.state()
    # only PC, the cycle counter and the halt byte of the closing JAM may change
    changed = sorted(set(np.nonzero(before != after)[0].tolist()) - set(range(0x06, 0x10)) - {0x1E})
    assert changed == [], [hex(c) for c in changed]
