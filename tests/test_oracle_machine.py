"""Oracle pins for the TIA, RIOT, cartridge and frame model: closed-form
images, documented register layouts and hand-assembled programs."""
import numpy as np
import pytest

from oracle import OracleMachine
from paper_1907_08467_gb300 import synth
from paper_1907_08467_gb300.synth.asm6502 import Assembler
from tests.helpers import JAM, rom, run_to_jam

# A frame loop that keeps VBLANK off on every line: 254-line frames, all 210
# window rows visible.  Registers are set by INIT, which runs once.
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


def frame_rom(init: str, perline: str = "") -> bytes:
    return rom("Start:\n" + init + FRAME.replace("{PERLINE}", perline))


def render(m, frames_before=2):
    for _ in range(frames_before):
        m.run_frame()
    return m.run_frame(render=True)[1]


def set_regs(m, **kw):
    """Write TIA fields of the canonical state (offsets of the state layout)."""
    off = {"nusiz0": 0x22, "nusiz1": 0x23, "colup0": 0x24, "colup1": 0x25, "colupf": 0x26,
           "colubk": 0x27, "ctrlpf": 0x28, "refp0": 0x29, "refp1": 0x2A, "pf0": 0x2B, "pf1": 0x2C,
           "pf2": 0x2D, "enam0": 0x2E, "enam1": 0x2F, "enabl": 0x30, "grp0": 0x32, "grp1": 0x34,
           "p0": 0x40, "p1": 0x41, "m0": 0x42, "m1": 0x43, "bl": 0x44}
    st = m.state()
    for k, v in kw.items():
        st[off[k]] = v
    m.set_state(st)


def test_window_solid_background():
    """R2: COLUBK solid, VBLANK off from line L0+40 to L0+231: rows 9..200 carry
    the color (value & 0xFE), every other row is 0."""
    src = """
Start:  LDA #$5B
        STA COLUBK
        STA WSYNC
Frame:  LDA #2
        STA VSYNC
        STA VBLANK
        STA WSYNC
        STA WSYNC
        STA WSYNC
        LDA #0
        STA VSYNC
        LDX #36
V1:     STA WSYNC
        DEX
        BNE V1
        STA WSYNC
        LDA #0
        STA VBLANK
        LDX #192
V2:     STA WSYNC
        DEX
        BNE V2
        LDA #2
        STA VBLANK
        LDX #29
V3:     STA WSYNC
        DEX
        BNE V3
        STA WSYNC
        JMP Frame
"""
    m = OracleMachine(rom(src))
    fb = render(m)
    exp = np.zeros((210, 160), np.uint8)
    exp[9:201] = 0x5A
    assert (fb == exp).all()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_generated_frames_262_lines(seed):
    """R1: the generators' frame loops rise VSYNC exactly 262 * 76 = 19,912
    CPU cycles apart (NTSC: 262 lines of 228 color clocks = 76 CPU cycles)."""
    for r in (synth.rom_playfield(seed), synth.rom_sprite(seed)):
        m = OracleMachine(r.data)
        m.run_frame()
        m.run_frame()     # the first loop entry comes from reset, not from JMP Main
        prev = m.last_vsync()
        for _ in range(5):
            assert m.run_frame() == 262
            v = m.last_vsync()
            assert v - prev == 262 * 76
            prev = v


def test_wsync_aligns_to_76():
    m = OracleMachine(rom("""
Start:  LDX #20
Loop:   NOP
        STA WSYNC
        LDA $80
        STA WSYNC
        DEX
        BNE Loop
""" + JAM))
    marks = []
    for _ in range(200):
        n = m.step()
        if n < 0:
            break
        if m.cycles % 76 == 0:
            marks.append(m.cycles)
    d = np.diff(marks)
    assert len(marks) >= 40 and (d == 76).all()


def test_frame_cap_and_jam_frame():
    m = OracleMachine(rom("Start:  STA WSYNC\n        JMP Start\n"))
    assert m.run_frame() == 400
    m = OracleMachine(rom("Start:  LDX #10\nL: STA WSYNC\n DEX\n BNE L\n" + JAM))
    assert m.run_frame() == 10


def _pf_expected(pf0, pf1, pf2, reflect):
    """Playfield definition: 20 bits per half, PF0 D4..D7, PF1 D7..D0, PF2 D0..D7,
    4 pixels per bit; right half repeats, or mirrors when reflected."""
    bits = [(pf0 >> b) & 1 for b in (4, 5, 6, 7)] + [(pf1 >> b) & 1 for b in range(7, -1, -1)] + \
           [(pf2 >> b) & 1 for b in range(8)]
    right = bits[::-1] if reflect else bits
    return np.repeat(np.array(bits + right, np.uint8), 4)


@pytest.mark.parametrize("pf0,pf1,pf2,ctrl", [(0x10, 0, 0, 0), (0xA0, 0x81, 0x3C, 0), (0x50, 0x0F, 0xF0, 1),
                                              (0xF0, 0xFF, 0xFF, 1), (0x00, 0x01, 0x80, 0)])
def test_playfield_bits(pf0, pf1, pf2, ctrl):
    m = OracleMachine(frame_rom(f"""
        LDA #$02
        STA COLUBK
        LDA #$45
        STA COLUPF
        LDA #${pf0:02X}
        STA PF0
        LDA #${pf1:02X}
        STA PF1
        LDA #${pf2:02X}
        STA PF2
        LDA #${ctrl:02X}
        STA CTRLPF
"""))
    fb = render(m)
    exp = np.where(_pf_expected(pf0, pf1, pf2, ctrl & 1) == 1, 0x44, 0x02)
    assert (fb[100] == exp).all()
    assert (fb[20] == exp).all()


# NUSIZ: (copy offsets in pixels, player scale) from the documented table.
NUSIZ = {0: ([0], 1), 1: ([0, 16], 1), 2: ([0, 32], 1), 3: ([0, 16, 32], 1), 4: ([0, 64], 1),
         5: ([0], 2), 6: ([0, 32, 64], 1), 7: ([0], 4)}


@pytest.mark.parametrize("mode", range(8))
@pytest.mark.parametrize("pos,grp,refl", [(30, 0x80, 0), (150, 0xC1, 0), (10, 0x81, 8)])
def test_player_copies_and_scale(mode, pos, grp, refl):
    m = OracleMachine(frame_rom(""))
    m.run_frame()
    set_regs(m, colubk=0, colup0=0x2E, grp0=grp, nusiz0=mode, p0=pos, refp0=refl)
    fb = m.run_frame(render=True)[1]
    offs, scale = NUSIZ[mode]
    exp = np.zeros(160, np.uint8)
    pattern = [(grp >> (7 - i)) & 1 for i in range(8)]
    if refl:
        pattern = pattern[::-1]
    for o in offs:
        for i, bit in enumerate(pattern):
            if bit:
                for s in range(scale):
                    exp[(pos + o + i * scale + s) % 160] = 0x2E
    assert (fb[50] == exp).all(), (mode, np.nonzero(fb[50])[0], np.nonzero(exp)[0])


@pytest.mark.parametrize("mode,width", [(0x00, 1), (0x10, 2), (0x20, 4), (0x31, 8), (0x03, 1), (0x26, 4)])
def test_missile_and_ball_width(mode, width):
    m = OracleMachine(frame_rom(""))
    m.run_frame()
    set_regs(m, colubk=0, colup0=0x1C, colupf=0x66, nusiz0=mode, m0=20, enam0=2, enabl=2, bl=120,
             ctrlpf=(mode & 0x30))
    fb = m.run_frame(render=True)[1]
    offs, _ = NUSIZ[mode & 7] if (mode & 7) not in (5, 7) else ([0], 1)
    exp = np.zeros(160, np.uint8)
    for o in offs:
        for s in range(width):
            exp[(20 + o + s) % 160] = 0x1C
    for s in range(width):
        exp[(120 + s) % 160] = 0x66
    assert (fb[80] == exp).all()


def test_priorities_and_score_mode():
    base = dict(colubk=0x02, colup0=0x1E, colup1=0x3E, colupf=0x5E, pf0=0xF0, pf1=0xFF, pf2=0xFF,
                grp0=0xFF, p0=20, grp1=0xFF, p1=24)
    m = OracleMachine(frame_rom(""))
    m.run_frame()
    set_regs(m, ctrlpf=0, **base)
    fb = m.run_frame(render=True)[1]
    assert fb[60, 20] == 0x1E and fb[60, 26] == 0x1E and fb[60, 30] == 0x3E and fb[60, 100] == 0x5E
    set_regs(m, ctrlpf=4, **base)              # playfield priority
    fb = m.run_frame(render=True)[1]
    assert fb[60, 20] == 0x5E and fb[60, 30] == 0x5E
    set_regs(m, ctrlpf=2, **base)              # score mode
    fb = m.run_frame(render=True)[1]
    assert fb[60, 20] == 0x1E and fb[60, 40] == 0x1E and fb[60, 100] == 0x3E
    set_regs(m, ctrlpf=6, **base)              # PFP wins over score mode (R8)
    fb = m.run_frame(render=True)[1]
    assert fb[60, 40] == 0x5E and fb[60, 100] == 0x5E


def test_collisions_latch_and_blank_rules():
    m = OracleMachine(frame_rom(""))
    m.run_frame()
    set_regs(m, grp0=0xFF, grp1=0xFF, p0=40, p1=44)
    m.run_frame()
    cx = int(m.state()[0x46]) | int(m.state()[0x47]) << 8
    assert cx == 1 << 15                        # only CXPPMM D7 (P0-P1)
    # missile 0 over player 1 and the ball over the playfield
    set_regs(m, grp0=0, grp1=0xFF, p1=44, enam0=2, m0=46, enabl=2, bl=100, pf1=0x40)
    st = m.state(); st[0x46] = st[0x47] = 0; m.set_state(st)
    m.run_frame()
    cx = int(m.state()[0x46]) | int(m.state()[0x47]) << 8
    # PF1 D6 lights columns 20..23 and 100..103: the ball (col 100) hits it,
    # P1 (cols 44..51) does not; M0 (col 46) is inside P1.
    # CXM0P D7 = M0-P1 is bit 1, CXBLPF D7 = BL-PF is bit 13.
    assert cx == (1 << 1) | (1 << 13)
    # R6: overlap only under VBLANK latches nothing
    src = """
Start:  LDA #$FF
        STA GRP0
        STA GRP1
        STA WSYNC
Frame:  LDA #2
        STA VSYNC
        STA VBLANK
        STA WSYNC
        STA WSYNC
        STA WSYNC
        LDA #0
        STA VSYNC
        LDX #250
L1:     STA WSYNC
        DEX
        BNE L1
        STA WSYNC
        JMP Frame
"""
    m = OracleMachine(rom(src))
    m.run_frame()              # lines before the first VBLANK write are unblanked
    set_regs(m, p0=40, p1=44)
    st = m.state(); st[0x46] = st[0x47] = 0; m.set_state(st)
    m.run_frame(); m.run_frame()
    assert int(m.state()[0x46]) | int(m.state()[0x47]) == 0


def test_hmove_bar_blanks_and_blocks_collisions():
    """R5/R6: HMOVE strobed right after WSYNC (effect in HBLANK) blanks columns
    0..7 of that line; overlaps there latch nothing.  Every line of this
    program strobes HMOVE at its start."""
    src = """
Start:  LDA #$4A
        STA COLUBK
Frame:  STA WSYNC
        STA HMOVE
        LDA #2
        STA VSYNC
        STA VBLANK
        STA WSYNC
        STA HMOVE
        STA WSYNC
        STA HMOVE
        STA WSYNC
        STA HMOVE
        LDA #0
        STA VSYNC
        STA VBLANK
        LDX #250
Lines:  STA WSYNC
        STA HMOVE
        DEX
        BNE Lines
        JMP Frame
"""
    m = OracleMachine(rom(src))
    m.run_frame()
    set_regs(m, grp0=0xFF, grp1=0xFF, p0=0, p1=0)
    st = m.state(); st[0x46] = st[0x47] = 0; m.set_state(st)
    fb = m.run_frame(render=True)[1]
    assert (fb[50, :8] == 0).all() and (fb[50, 8:] == 0x4A).all()
    assert int(m.state()[0x46]) | int(m.state()[0x47]) == 0
    # the same overlap one pixel further right (cols 8..15) does latch
    set_regs(m, p0=8, p1=8)
    m.run_frame()
    assert (int(m.state()[0x46]) | int(m.state()[0x47]) << 8) == 1 << 15


def test_resp_position_closed_form():
    """R3/R4: RESP0 executed after n NOPs from a WSYNC: the store's access
    cycle is 2n + 2 within the line, the effect clock 3 (2n + 3); player at
    (clock - 68 + 5) mod 160, or 3 when the clock is in HBLANK."""
    for n in range(0, 34):
        src = "Start:  STA WSYNC\n" + "        NOP\n" * n + "        STA RESP0\n" + JAM
        m = OracleMachine(rom(src))
        run_to_jam(m)
        clk = 3 * (2 * n + 3)
        exp = 3 if clk < 68 else (clk - 68 + 5) % 160
        assert m.state()[0x40] == exp, n


def test_hmove_shifts():
    for hm, delta in [(0x30, -3), (0xD0, 3), (0x70, -7), (0x80, 8), (0x00, 0)]:
        m = OracleMachine(rom(f"""
Start:  LDA #${hm:02X}
        STA HMP0
        STA HMBL
        STA WSYNC
        STA HMOVE
""" + JAM))
        m.step()
        set_regs(m, p0=50, bl=1)
        run_to_jam(m)
        assert m.state()[0x40] == 50 + delta and m.state()[0x44] == (1 + delta) % 160


def test_rmw_strobe_writes_twice():
    """R14: INC on a strobe register writes twice (old value, then new)."""
    m = OracleMachine(rom("""
Start:  LDA #$10
        STA HMP0
        INC HMOVE
""" + JAM))
    m.step(); m.step()
    set_regs(m, p0=50)
    w0 = m.tia_writes
    run_to_jam(m)
    assert m.tia_writes - w0 == 2 and m.state()[0x40] == 48


def test_riot_timer_ticks():
    """R10: after writing v to a timer with interval I, INTIM holds v through
    the first I cycles, then decrements once per I cycles; after it passes
    zero it counts down once per cycle from $FF and TIMINT bit 7 is set."""
    for reg, interval, v in [("TIM1T", 1, 5), ("TIM8T", 8, 3), ("TIM64T", 64, 1)]:
        m = OracleMachine(rom(f"""
Start:  LDA #{v}
        STA {reg}
        LDX #0
Loop:   LDA INTIM
        STA $80,X
        INX
        CPX #48
        BNE Loop
        LDA TIMINT
        STA $F0
""" + JAM))
        run_to_jam(m)
        # write access: LDA #v (2) then STA abs (4): cycle 5.  Sample i is the
        # LDA INTIM access of iteration i: 6 + 2 (LDX) + 15 i + 3.
        w = 5

        def intim_at(c):
            count, pre, fast = v, 0, False
            for _ in range(w + 1, c):
                if fast:
                    count = (count - 1) & 0xFF
                    continue
                pre += 1
                if pre == interval:
                    pre = 0
                    if count == 0:
                        count, fast = 0xFF, True
                    else:
                        count -= 1
            return count
        ram = m.ram()
        for i in range(48):
            c = w + 1 + 2 + 15 * i + 3
            assert ram[i] == intim_at(c), (reg, i)
        assert ram[0x70] == 0x80


def test_bank_switch_f8_reads_new_bank():
    """R16: an F8 hotspot read switches first and returns the new bank's byte."""
    b0 = Assembler().assemble("""
        .org $F000
Start:  LDA $1FF9
        .org $F00A
        STA $81
        .byte $02
        .org $FFF8
        .byte $A0, $A0
        .word Start, Start, Start
""", org=0xF000, size=4096)
    b1 = Assembler().assemble("""
        .org $F003
        LDA #$B1
        STA $80
        LDA $1FF8
        .org $FFF8
        .byte $A1, $A1
        .word $F000, $F000, $F000
""", org=0xF000, size=4096)
    m = OracleMachine(b0 + b1)
    run_to_jam(m)
    assert m.ram()[0] == 0xB1 and m.ram()[1] == 0xA0 and m.state()[0x05] == 0


def test_bank_switch_f6_all_banks():
    banks = []
    for b in range(4):
        nxt = (b + 1) % 4
        banks.append(Assembler().assemble(f"""
        .org $F000
Start:  LDA #{b}
        STA $80+{b}
        LDA ${0x1FF6 + nxt:04X}
        .org $F007
        .byte $02
        .org $FFFA
        .word Start, Start, Start
""", org=0xF000, size=4096))
    # bank 0 runs, switches to 1, whose code at $F007 is a JAM; so only bank 0 stored
    m = OracleMachine(b"".join(banks))
    run_to_jam(m)
    assert m.ram()[0] == 0 and m.state()[0x05] == 1


def test_bank_switch_f4_all_banks():
    """F4 (32 KB, 8 banks): reading $1FF4 + j selects bank j.  Bank b stores b
    at $80 + b, then reads the hotspot of bank b + 1; the next instruction
    ($F007) comes from that bank, which jumps to its own Start.  Bank 7
    selects bank 0, whose $F007 halts.  Every hotspot is visited once."""
    banks = []
    for b in range(8):
        nxt = (b + 1) % 8
        tail = "        .byte $02\n" if b == 0 else "        JMP Start\n"
        banks.append(Assembler().assemble(f"""
        .org $F000
Start:  LDA #{b}
        STA $80+{b}
        LDA ${0x1FF4 + nxt:04X}
        .org $F007
""" + tail + """
        .org $FFFA
        .word Start, Start, Start
""", org=0xF000, size=4096))
    m = OracleMachine(b"".join(banks))
    run_to_jam(m)
    assert list(m.ram()[:8]) == list(range(8)) and m.state()[0x05] == 0


ALE = ["NOOP", "FIRE", "UP", "RIGHT", "LEFT", "DOWN", "UPRIGHT", "UPLEFT", "DOWNRIGHT", "DOWNLEFT",
       "UPFIRE", "RIGHTFIRE", "LEFTFIRE", "DOWNFIRE", "UPRIGHTFIRE", "UPLEFTFIRE", "DOWNRIGHTFIRE",
       "DOWNLEFTFIRE"]


@pytest.mark.parametrize("a", range(18))
def test_action_to_ports(a):
    """The 18 ALE actions on the P0 joystick (SWCHA D7 right, D6 left, D5 down,
    D4 up, active low; P1 nibble idle) and fire (INPT4 D7 low when pressed)."""
    m = OracleMachine(rom("""
Start:  LDA SWCHA
        STA $80
        LDA INPT4
        STA $81
        LDA SWCHB
        STA $82
""" + JAM))
    m.set_action(a)
    run_to_jam(m)
    name = ALE[a]
    exp = 0xFF
    for word, bit in (("RIGHT", 0x80), ("LEFT", 0x40), ("DOWN", 0x20), ("UP", 0x10)):
        if word in name:
            exp &= ~bit
    assert m.ram()[0] == exp
    assert m.ram()[1] == (0x00 if "FIRE" in name else 0x80)
    assert m.ram()[2] == 0x0B


def test_inpt4_latch():
    m = OracleMachine(rom("""
Start:  LDA #$40
        STA VBLANK
        LDA INPT4
        STA $80
        NOP
        LDA INPT4
        STA $81
        LDA #0
        STA VBLANK
        LDA INPT4
        STA $82
""" + JAM))
    m.set_action(1)
    for _ in range(4):
        m.step()
    m.set_action(0)
    run_to_jam(m)
    assert list(m.ram()[:3]) == [0x00, 0x00, 0x80]


def test_port_ddr_mixes_output():
    m = OracleMachine(rom("""
Start:  LDA #$F0
        STA SWACNT
        LDA #$50
        STA SWCHA
        LDA SWCHA
        STA $80
""" + JAM))
    m.set_action(3)   # RIGHT: input pins 0x7F; output bits 7..4 come from the latch
    run_to_jam(m)
    assert m.ram()[0] == 0x5F


def test_state_bank_byte_keeps_only_the_cartridges_bank_bits():
    """A 2K/4K cartridge has no bank latch, F8 one bank bit, F6 two and F4
    three: a state whose bank byte has more bits set loads as those bits
    only."""
    for size, mask in [(2048, 0), (4096, 0), (8192, 1), (16384, 3), (32768, 7)]:
        m = OracleMachine(bytes(size))
        for b in (0xFF, 0xFE, 0x05, 0x02):
            s = m.state()
            s[0x05] = b
            m.set_state(s)
            assert m.state()[0x05] == b & mask, (size, b)
