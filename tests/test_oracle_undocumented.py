"""Oracle pins for the stable undocumented NMOS opcodes (real cartridges use
them; the paper's ALE games run on that part).

The opcode matrix and timing rules below are typed from the published
descriptions of the part's undocumented instructions, not from the oracle:

- SLO, RLA, SRE, RRA, DCP, ISC: a read-modify-write of memory (always the
  long cycle count: zp 5, zp,X 6, abs 6, abs,X / abs,Y 7, (zp,X) / (zp),Y 8)
  followed by ORA, AND, EOR, ADC, CMP, SBC with the new memory value;
- SAX stores A AND X (store timing); LAX loads A and X (read timing, with the
  page-cross cycle); ANC, ALR, SBX and SBC $EB take an immediate (2 cycles);
- NOPs of one, two and three bytes; those with a memory operand read it
  (zp 3, zp,X 4, abs 4, abs,X 4 + page cross);
- the other 21 opcodes (the 12 that halt the part and ANE, LXA, SHA, SHX, SHY,
  TAS, LAS, ARR, whose results depend on the chip or are not described
  consistently) halt the CPU here.

Results of each class are worked by hand in the test docstrings.  Planted
one-line mistakes in the oracle (SLO's ORA with the old value, RRA adding
without the rotated carry, ISC using the old value, DCP's compare on X, SAX
storing A, ANC leaving the carry, SBX honouring decimal mode or the carry, a
NOP abs skipping its read, LAX's page-cross cycle dropped) each fail a test.
"""
import pytest

from oracle import OracleMachine, base_cycles
from paper_1907_08467_gb300.synth.asm6502 import OPCODES, Assembler
from tests.helpers import JAM, rom, run_to_jam

RMWU = {"zp": 5, "zpx": 6, "abs": 6, "abx": 7, "aby": 7, "izx": 8, "izy": 8}
UNDOC = {
    "SLO": ({"zp": 0x07, "zpx": 0x17, "abs": 0x0F, "abx": 0x1F, "aby": 0x1B, "izx": 0x03, "izy": 0x13}, RMWU),
    "RLA": ({"zp": 0x27, "zpx": 0x37, "abs": 0x2F, "abx": 0x3F, "aby": 0x3B, "izx": 0x23, "izy": 0x33}, RMWU),
    "SRE": ({"zp": 0x47, "zpx": 0x57, "abs": 0x4F, "abx": 0x5F, "aby": 0x5B, "izx": 0x43, "izy": 0x53}, RMWU),
    "RRA": ({"zp": 0x67, "zpx": 0x77, "abs": 0x6F, "abx": 0x7F, "aby": 0x7B, "izx": 0x63, "izy": 0x73}, RMWU),
    "DCP": ({"zp": 0xC7, "zpx": 0xD7, "abs": 0xCF, "abx": 0xDF, "aby": 0xDB, "izx": 0xC3, "izy": 0xD3}, RMWU),
    "ISC": ({"zp": 0xE7, "zpx": 0xF7, "abs": 0xEF, "abx": 0xFF, "aby": 0xFB, "izx": 0xE3, "izy": 0xF3}, RMWU),
    "SAX": ({"zp": 0x87, "zpy": 0x97, "abs": 0x8F, "izx": 0x83}, {"zp": 3, "zpy": 4, "abs": 4, "izx": 6}),
    "LAX": ({"zp": 0xA7, "zpy": 0xB7, "abs": 0xAF, "aby": 0xBF, "izx": 0xA3, "izy": 0xB3},
            {"zp": 3, "zpy": 4, "abs": 4, "aby": 4, "izx": 6, "izy": 5}),
    "ANC": ({"imm": 0x0B, "imm2": 0x2B}, {"imm": 2, "imm2": 2}),
    "ALR": ({"imm": 0x4B}, {"imm": 2}),
    "SBX": ({"imm": 0xCB}, {"imm": 2}),
    "SBC": ({"imm": 0xEB}, {"imm": 2}),
}
NOPS = {0x1A: 2, 0x3A: 2, 0x5A: 2, 0x7A: 2, 0xDA: 2, 0xFA: 2, 0x80: 2, 0x82: 2, 0x89: 2, 0xC2: 2, 0xE2: 2,
        0x04: 3, 0x44: 3, 0x64: 3, 0x14: 4, 0x34: 4, 0x54: 4, 0x74: 4, 0xD4: 4, 0xF4: 4, 0x0C: 4,
        0x1C: 4, 0x3C: 4, 0x5C: 4, 0x7C: 4, 0xDC: 4, 0xFC: 4}
HALTING = [0x02, 0x12, 0x22, 0x32, 0x42, 0x52, 0x62, 0x72, 0x92, 0xB2, 0xD2, 0xF2,
           0x8B, 0xAB, 0x93, 0x9F, 0x9E, 0x9C, 0x9B, 0xBB, 0x6B]


def undoc_cycles():
    out = dict(NOPS)
    for ops, cyc in UNDOC.values():
        for mode, opc in ops.items():
            out[opc] = cyc[mode]
    return out


def test_opcode_matrix_and_base_cycles():
    """151 documented + 84 stable undocumented opcodes have their published
    base cycle counts; the other 21 have none (they halt)."""
    doc = {op for modes in OPCODES.values() for op in modes.values()}
    und = undoc_cycles()
    assert len(doc) == 151 and len(und) == 84 and not (doc & set(und))
    assert set(range(256)) - doc - set(und) == set(HALTING)
    for op, c in und.items():
        assert base_cycles(op) == c, hex(op)
    for op in HALTING:
        assert base_cycles(op) == 0, hex(op)


@pytest.mark.parametrize("op", HALTING)
def test_unmodelled_opcodes_halt(op):
    m = OracleMachine(rom(f"Start: LDA #1\n STA $80\n .byte ${op:02X}, $00, $00\n LDA #2\n STA $80\n"))
    assert m.step() == 2 and m.step() == 3
    assert m.step() == -1 and m.state()[0x1E] == 1 and m.ram()[0] == 1


def _run(src):
    m = OracleMachine(rom("Start:  LDX #$FF\n        TXS\n" + src + JAM))
    run_to_jam(m)
    return m


def _p(m):
    return int(m.state()[0x04])


def test_rmw_accumulator_classes():
    """Hand-worked (C = carry, binary mode):
    SLO $90: M $81 -> $02, C 1; A $04 | $02 = $06.
    RLA $91: M $40, C 1 -> $81, C 0; A $FF & $81 = $81 (N).
    SRE $92: M $03 -> $01, C 1; A $01 ^ $01 = $00 (Z).
    RRA $93: M $02, C 1 -> $81, C 0; A $10 + $81 + 0 = $91 (N, no C).
    DCP $94: M $10 -> $0F; CMP A $0F: Z and C set.
    ISC $95: M $FF -> $00; A $05 - $00 - (1 - C=1) = $05, C 1."""
    m = _run("""
        LDA #$81
        STA $90
        LDA #$04
        SLO $90
        STA $A0
        PHP
        PLA
        STA $A1
        LDA #$40
        STA $91
        SEC
        LDA #$FF
        RLA $91
        STA $A2
        PHP
        PLA
        STA $A3
        LDA #$03
        STA $92
        LDA #$01
        SRE $92
        STA $A4
        PHP
        PLA
        STA $A5
        LDA #$02
        STA $93
        SEC
        LDA #$10
        RRA $93
        STA $A6
        PHP
        PLA
        STA $A7
        LDA #$10
        STA $94
        LDA #$0F
        DCP $94
        PHP
        PLA
        STA $A8
        LDA #$FF
        STA $95
        SEC
        LDA #$05
        ISC $95
        STA $A9
        PHP
        PLA
        STA $AA
""")
    r = m.ram()
    N, Z, C, V = 0x80, 0x02, 0x01, 0x40
    assert (r[0x10], r[0x20], r[0x21] & (N | Z | C)) == (0x02, 0x06, C)
    assert (r[0x11], r[0x22], r[0x23] & (N | Z | C)) == (0x81, 0x81, N)
    assert (r[0x12], r[0x24], r[0x25] & (N | Z | C)) == (0x01, 0x00, Z | C)
    assert (r[0x13], r[0x26], r[0x27] & (N | Z | C | V)) == (0x81, 0x91, N)
    assert (r[0x14], r[0x28] & (N | Z | C)) == (0x0F, Z | C)
    assert (r[0x15], r[0x29], r[0x2A] & (N | Z | C)) == (0x00, 0x05, C)


def test_rra_and_isc_follow_decimal_mode():
    """With D set the add and subtract are decimal: RRA $96 with M $50, C 0
    rotates to $28 (C 0); A $19 + $28 = $47.  ISC $97 with M $08 -> $09 (the
    increment itself is binary); A $25 - $09 (C set: no borrow) = $16."""
    m = _run("""
        SED
        LDA #$50
        STA $96
        CLC
        LDA #$19
        RRA $96
        STA $B0
        LDA #$08
        STA $97
        SEC
        LDA #$25
        ISC $97
        STA $B1
        CLD
""")
    r = m.ram()
    assert (r[0x16], r[0x30]) == (0x28, 0x47)
    assert (r[0x17], r[0x31]) == (0x09, 0x16)


def test_sax_lax_and_immediates():
    """SAX $98 with A $F0, X $3C stores $30 and leaves P alone; LAX $98 loads
    $30 into A and X; LAX ($99),Y reads through a pointer; ANC #$80 with A $FF
    gives $80 with C = N = 1; ALR #$03 with A $07 gives $01 with C 1; SBX #$05
    with A $0F, X $FC and C clear gives X = ($0F & $FC) - 5 = $07 with C 1
    (the old carry is not a borrow); with D and C set, A $1F, X $12 it gives
    $12 - $05 = $0D (binary, decimal mode ignored); SBC #$01 ($EB) with A $10,
    C 1 gives $0F."""
    m = _run("""
        LDA #$F0
        LDX #$3C
        CLC
        SAX $98
        PHP
        PLA
        STA $B2
        LDA #0
        LDX #0
        LAX $98
        STA $B3
        STX $B4
        LDA #$C0
        STA $99
        LDA #$00
        STA $9A
        LDY #$01
        LDA #$77
        STA $C1
        LAX ($99),Y
        STX $B5
        LDA #$FF
        ANC #$80
        PHP
        STA $B6
        PLA
        STA $B7
        LDA #$07
        ALR #$03
        STA $B8
        PHP
        PLA
        STA $B9
        SED
        SEC
        LDA #$1F
        LDX #$12
        SBX #$05
        STX $BD
        CLD
        CLC
        LDA #$0F
        LDX #$FC
        SBX #$05
        STX $BA
        PHP
        PLA
        STA $BB
        SEC
        LDA #$10
        .byte $EB, $01
        STA $BC
""")
    r = m.ram()
    assert r[0x18] == 0x30 and r[0x32] & 0x01 == 0
    assert r[0x33] == 0x30 and r[0x34] == 0x30 and r[0x35] == 0x77
    assert r[0x36] == 0x80 and r[0x37] & 0x81 == 0x81
    assert r[0x38] == 0x01 and r[0x39] & 0x01 == 1
    assert r[0x3A] == 0x07 and r[0x3B] & 0x83 == 0x01
    assert r[0x3D] == 0x0D          # $12 - $05 in binary although D is set
    assert r[0x3C] == 0x0F


def test_nops_take_their_cycles_and_change_no_register():
    """Each NOP form takes its published cycles (+1 for abs,X across a page)
    and leaves A, X, Y, SP and P unchanged."""
    for op, c in NOPS.items():
        size = 1 if c == 2 and op in (0x1A, 0x3A, 0x5A, 0x7A, 0xDA, 0xFA) else (3 if op in (0x0C, 0x1C, 0x3C, 0x5C, 0x7C, 0xDC, 0xFC) else 2)
        operand = {1: "", 2: ", $80", 3: ", $80, $00"}[size]
        m = OracleMachine(rom(f"Start: LDX #$05\n .byte ${op:02X}{operand}\n" + JAM))
        m.step()
        before = m.state()
        assert m.step() == c, hex(op)
        after = m.state()
        assert list(after[0:5]) == list(before[0:5]), hex(op)
    m = OracleMachine(rom("Start: LDX #$FF\n .byte $1C, $01, $80\n" + JAM))   # $8001 + $FF crosses a page
    m.step()
    assert m.step() == 5


def test_nop_absolute_reads_a_bank_hotspot():
    """NOP $1FF9 ($0C $F9 $1F) in bank 0 of an F8 cartridge reads the hotspot:
    the next instruction comes from bank 1, which stores $B1 (bank 0 would
    store $B0 there)."""
    def bank(tag):
        return Assembler().assemble(f"""
        .org $F000
Start:  .byte $0C, $F9, $FF
        LDA #${tag:02X}
        STA $80
        .byte $02
        .org $FFFA
        .word Start, Start, Start
""", org=0xF000, size=4096)
    m = OracleMachine(bank(0xB0) + bank(0xB1))
    run_to_jam(m)
    assert m.ram()[0] == 0xB1 and m.state()[0x05] == 1


def test_lax_page_cross_cycle():
    m = OracleMachine(rom("Start: LDY #$FF\n LAX $8001,Y\n" + JAM))
    m.step()
    assert m.step() == 5
    m = OracleMachine(rom("Start: LDY #$00\n LAX $8001,Y\n" + JAM))
    m.step()
    assert m.step() == 4


def test_undocumented_rmw_on_a_strobe_writes_twice():
    """Like the documented read-modify-write instructions, ISC HMOVE writes the
    old value, then the new one: two HMOVE strobes, so P0 (HMP0 = $10, one
    pixel left per strobe) moves from 50 to 48."""
    m = OracleMachine(rom("""
Start:  LDA #$10
        STA HMP0
        ISC HMOVE
""" + JAM))
    m.step()
    m.step()
    st = m.state()
    st[0x40] = 50
    m.set_state(st)
    w0 = m.tia_writes
    run_to_jam(m)
    assert m.tia_writes - w0 == 2 and m.state()[0x40] == 48
